// Launch helpers shared between translation units.
#pragma once

#include "pn_internal.cuh"

// Y (=|+=) X W + b on value rows; float32 layers of group `grp` (a
// PN_TC_* bit) go to the tensor cores when the system enables that group
// (s may be null: CUDA cores).
enum { PN_TC_LAYERS = 1, PN_TC_HEADS = 2, PN_TC_VALUE = 4 };
template <typename R>
int pn_linear(const DevSys* s, int grp, const R* X, int ldx, const R* W, int ldw, const R* b, R* Y, int ldy, int rows,
              int Kd, int Nout, int T, int acc, cudaStream_t st);

// Float32 Y (=|+=) X W^T, W stored [Nout][Kd] with row stride ldw, on the
// pipelined GEMM tiles; PN_ENOTREADY when X is not float4-aligned.
int pn_linear_bt_f32(const float* X, int ldx, const float* W, int ldw, float* Y, int ldy, int rows, int Kd, int Nout,
                     int acc, cudaStream_t st);

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the multiply-xor
// bijection with the key bumped by the Weyl constants between rounds.
__device__ inline void pn_philox(unsigned c[4], unsigned k0, unsigned k1) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const unsigned hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const unsigned hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__device__ inline double pn_u01(unsigned x) { return ((double)x + 0.5) * 2.3283064365386962890625e-10; }

// Normal number m (0-based) of stream (seed, walker, step): block m/4,
// Box-Muller pair (m%4)/2, cosine for even m, sine for odd m.
__device__ inline void pn_normals4(unsigned long long seed, unsigned walker, unsigned long long step, unsigned j,
                                   double out[4]) {
  unsigned c[4] = {j, walker, (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
  pn_philox(c, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
  for (int pr = 0; pr < 2; ++pr) {
    const double u0 = pn_u01(c[2 * pr]), u1 = pn_u01(c[2 * pr + 1]);
    const double rad = sqrt(-2.0 * log(u0));
    const double ang = 2.0 * 3.141592653589793 * u1;
    out[2 * pr] = rad * cos(ang);
    out[2 * pr + 1] = rad * sin(ang);
  }
}

// Algorithmic float32/float64 network work of one value pass of one walker
// (multiply-add = 2): the filter networks of every pair and layer, the maps
// h (none in the first layer, whose input is the one shared embedding) and
// the stacked receiving maps, the messages, and both heads.
inline double pn_value_pass_flops(const DevSys& s) {
  const double N = s.N, M = s.M, D = s.D, Zd = s.Zd, K = s.K, Hw = s.Hw, L = s.L, P = s.Ppair;
  const double filt = L * P * 2.0 * (K * Hw + Hw * Zd);
  const double lin = N * 2.0 * ((L - 1) * D * Zd + L * 3.0 * Zd * D + 2.0 * D * D + D * s.n_orb) + 2.0 * (2.0 * D * D + D);
  const double msg = L * N * Zd * (N - 1 + M) * 2.0;
  return filt + lin + msg;
}

int pn_launch_geometry_orbitals(const DevSys& s, const double* r, int Wn, double* geo, double* phi, cudaStream_t st);
// deriv = 1 also writes the first and second distance derivatives of the features
template <typename R>
int pn_launch_features_init(const DevSys& s, const R* x0, const double* geo, int Wn, int deriv, R* ef, R* X,
                            cudaStream_t st);
template <typename R>
int pn_launch_sum_electrons(const R* X, R* Xs, int Wn, int N, int D, cudaStream_t st);

// Filter networks of layer n on tiles of 64 pair rows of one channel
// (filter_tiles.cu, float32): value pass with the tape (Ah, w), jet pass
// (w and its two distance derivatives, [row][3][Zd]), backward for the
// weight gradients (dAh, ssp(Ah)) and backward to the pair distances
// (dd += ...).  PN_ENOTREADY when a tile does not fit in shared memory.
int pn_filter_tile_value(const DevSys& s, const DevNet<float>& net, int n, const float* ef, int Wn, float* Ah,
                         float* wv, cudaStream_t st);
// the forward value pass: w into the jet layout's value rows ([P][3][Zd]), no Ah
int pn_filter_tile_value_fwd(const DevSys& s, const DevNet<float>& net, int n, const float* ef, int Wn, float* wj,
                             cudaStream_t st);
int pn_filter_tile_jet(const DevSys& s, const DevNet<float>& net, int n, const float* ef, int Wn, float* wj,
                       cudaStream_t st);
int pn_filter_tile_bwd(const DevSys& s, const DevNet<float>& net, int n, const float* Ah, const float* dw, int Wn,
                       float* dAh, float* Sh, cudaStream_t st);
int pn_filter_tile_dist(const DevSys& s, const DevNet<float>& net, int n, const float* Ah, const float* ef,
                        const float* dw, int Wn, double* dd, cudaStream_t st);

// One Box-Muller pair (normals 4j + 2*pair and 4j + 2*pair + 1) of the same
// stream as pn_normals4, so that the pairs of one block can go to different
// lanes.
__device__ inline void pn_normal_pair(unsigned long long seed, unsigned walker, unsigned long long step, unsigned j,
                                      int pair, double out[2]) {
  unsigned c[4] = {j, walker, (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
  pn_philox(c, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
  const double u0 = pn_u01(c[2 * pair]), u1 = pn_u01(c[2 * pair + 1]);
  const double rad = sqrt(-2.0 * log(u0));
  const double ang = 2.0 * 3.141592653589793 * u1;
  out[0] = rad * cos(ang);
  out[1] = rad * sin(ang);
}

// Orbital tables in the sampler's orbital precision C.
template <typename C>
struct OrbTab {
  const C *R, *pexp, *pcoef, *mo, *rc, *cC, *cs, *ca;
};
template <typename C>
__device__ inline OrbTab<C> orb_tab(const DevSys& s);
template <>
__device__ inline OrbTab<double> orb_tab<double>(const DevSys& s) {
  return {s.R, s.pexp, s.pcoef, s.mo, s.cusp_rc, s.cusp_C, s.cusp_s, s.cusp_a};
}
template <>
__device__ inline OrbTab<float> orb_tab<float>(const DevSys& s) {
  return {s.R32, s.pexp32, s.pcoef32, s.mo32, s.cusp_rc32, s.cusp_C32, s.cusp_s32, s.cusp_a32};
}


// One Box-Muller pair in C precision from the shared Philox stream.
template <typename C>
__device__ inline void normal_pair(unsigned long long seed, unsigned walker, unsigned long long step, unsigned j,
                                   int pair, C out[2]) {
  if constexpr (sizeof(C) == 8) {
    pn_normal_pair(seed, walker, step, j, pair, out);
  } else {
    unsigned c[4] = {j, walker, (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
    pn_philox(c, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
    const float u0 = ((float)c[2 * pair] + 0.5f) * 2.3283064365386963e-10f;
    const float u1 = ((float)c[2 * pair + 1] + 0.5f) * 2.3283064365386963e-10f;
    const float rad = sqrtf(-2.0f * logf(u0));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    out[0] = rad * cs;
    out[1] = rad * sn;
  }
}

