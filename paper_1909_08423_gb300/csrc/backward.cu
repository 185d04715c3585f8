// Parameter gradient of ln|psi| (reverse mode, hand written): the backward
// pass needed by the VMC loss gradient, Eq. (trainig) of the paper:
//   grad_theta L = 2 E[(E_loc - L) grad_theta ln|psi|]
// = sum_w u_w grad_theta ln|psi_w| with per-walker weights u_w (cotangent).
//
// For each chunk of walkers the value pass is recomputed with every
// activation kept on a tape; then the chain runs back through the
// determinants, the backflow and Jastrow heads, the interaction layers
// (receiving maps g, messages, filters w, input maps h) to x0 and Y.
// Weight gradients are sums over rows (walkers x electrons or pairs): each
// is formed as per-block partial tiles in float64 and reduced in a fixed
// order, so the result is deterministic.
//
// The same tape and chain with weight 1 per walker and no weight gradients
// give grad_r ln|psi|, the drift of the Langevin proposal (Methods, ansatz
// optimisation, sampling): the chain then ends at the pair distances
// (through each layer's filter features and the cusp factor gamma) and at
// the orbitals (through the backflowed determinant entries).
#include <math.h>

#include <algorithm>

#include "kernels.cuh"
#include "pn_internal.cuh"

namespace pnb {

inline unsigned nblk(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename R>
__device__ inline R sigm_(R x) { return R(1) / (R(1) + exp(-x)); }
template <typename R>
__device__ inline R ssp_(R x) {
  return (x > R(0) ? x : R(0)) + log1p(exp(-fabs(x))) - R(0.69314718055994530942);
}

__device__ inline int pair_channel(const DevSys& s, int p) {
  if (p >= s.Pee) return 2;
  int a = 0, rem = p;
  while (rem >= s.N - 1 - a) { rem -= s.N - 1 - a; ++a; }
  int b = a + 1 + rem;
  return ((a < s.n_up) == (b < s.n_up)) ? 0 : 1;
}

// ------------------------------------------------------------ forward tape
// Value-only filter nets keeping the hidden pre-activation:
// Ah[row][h] = b1 + e W1, w[row][z] = b2 + ssp(Ah) W2.
template <typename R>
__global__ void k_filter_tape(DevSys s, DevNet<R> net, int n, const R* __restrict__ ef, int Wn, R* __restrict__ Ah,
                              R* __restrict__ wout) {
  __shared__ R sh_e[8][64];
  __shared__ R sh_h[8][128];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t row = (size_t)blockIdx.x * 8 + wid;
  if (row >= (size_t)Wn * s.Ppair) return;
  const int ch = pair_channel(s, row % s.Ppair);
  const int K = s.K, Hw = s.Hw, Zd = s.Zd;
  for (int k = lane; k < K; k += 32) sh_e[wid][k] = ef[row * 3 * K + k];
  __syncwarp();
  const R* W1 = net.p + net.off.W1[n][ch];
  const R* b1 = net.p + net.off.b1[n][ch];
  const R* W2 = net.p + net.off.W2[n][ch];
  const R* b2 = net.p + net.off.b2[n][ch];
  for (int h = lane; h < Hw; h += 32) {
    R a = b1[h];
    for (int k = 0; k < K; ++k) a += sh_e[wid][k] * W1[k * Hw + h];
    Ah[row * Hw + h] = a;
    sh_h[wid][h] = ssp_(a);
  }
  __syncwarp();
  for (int z = lane; z < Zd; z += 32) {
    R o = b2[z];
    for (int h = 0; h < Hw; ++h) o += sh_h[wid][h] * W2[h * Zd + z];
    wout[row * Zd + z] = o;
  }
}

// Value-only messages: Z[w][i][c*Zd + z] from filter outputs w[w][p][z].
template <typename R>
__global__ void k_message_value(DevSys s, const R* __restrict__ Y, const R* __restrict__ wv, const R* __restrict__ H,
                                int Wn, R* __restrict__ Z) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int Zd = s.Zd, N = s.N;
  if (idx >= (size_t)Wn * N * Zd) return;
  const int z = idx % Zd;
  const int i = (idx / Zd) % N;
  const int w = idx / ((size_t)Zd * N);
  const R* ww = wv + (size_t)w * s.Ppair * Zd;
  const R* hw = H + (size_t)w * N * Zd;
  R zs = 0, za = 0, zn = 0;
  const bool si = i < s.n_up;
  for (int j = 0; j < N; ++j) {
    if (j == i) continue;
    const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
    const R v = ww[(size_t)p * Zd + z] * hw[(size_t)j * Zd + z];
    if ((j < s.n_up) == si) zs += v; else za += v;
  }
  for (int I = 0; I < s.M; ++I) zn += ww[(size_t)(s.Pee + i * s.M + I) * Zd + z] * Y[I * Zd + z];
  R* o = Z + ((size_t)w * N + i) * 3 * Zd;
  o[z] = zs;
  o[Zd + z] = za;
  o[2 * Zd + z] = zn;
}

template <typename R>
__global__ void k_ssp_copy(const R* __restrict__ A, R* __restrict__ S, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) S[i] = ssp_(A[i]);
}

// ---------------------------------------------------------- backward kernels
// Determinant part: d ln|psi| / d F[w][i][mu] (f = 1 + F) for weight u_w,
// with omega_p = c_p s_p e^{ld_p} / S and d ln|det A| / dA = A^{-T}, in three
// passes so that every (walker, determinant, spin) block gets a thread:
// k_slater_lu forms ln|det| and the sign of each block, k_slater_inv the
// weighted inverse omega_p A^{-T} of each block, k_slater_gather sums the
// blocks for each electron row in determinant order (a fixed order, so the
// result is deterministic).

// LU factorisation with partial pivoting of spin block sp of determinant p:
// A[a][b] = phi_{occ_b}(r_{e0+a}) (1 + F_{e0+a, occ_b}).  Returns false for
// a singular block; perm (optional) receives the row permutation.
template <typename R>
__device__ inline bool slater_block_lu(const DevSys& s, const double* phw, const R* Fw, int p, int sp, double* LU,
                                       int* perm, double& ld, double& sgn) {
  const int no = s.n_orb, ns = sp ? s.n_dn : s.n_up, e0 = sp ? s.n_up : 0;
  const int* occ = s.occ + p * s.N + e0;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b)
      LU[a * ns + b] = phw[((e0 + a) * no + occ[b]) * 5] * (1.0 + (double)Fw[(e0 + a) * no + occ[b]]);
  if (perm)
    for (int c = 0; c < ns; ++c) perm[c] = c;
  ld = 0;
  sgn = 1;
  for (int c = 0; c < ns; ++c) {
    int best = c;
    double bv = fabs(LU[c * ns + c]);
    for (int rr = c + 1; rr < ns; ++rr)
      if (fabs(LU[rr * ns + c]) > bv) { bv = fabs(LU[rr * ns + c]); best = rr; }
    if (!(bv > 0.0)) { sgn = 0; return false; }
    if (best != c) {
      for (int k = 0; k < ns; ++k) { double t = LU[c * ns + k]; LU[c * ns + k] = LU[best * ns + k]; LU[best * ns + k] = t; }
      if (perm) { int t = perm[c]; perm[c] = perm[best]; perm[best] = t; }
      sgn = -sgn;
    }
    const double piv = LU[c * ns + c];
    if (piv < 0) sgn = -sgn;
    ld += log(fabs(piv));
    for (int rr = c + 1; rr < ns; ++rr) {
      const double f = LU[rr * ns + c] / piv;
      LU[rr * ns + c] = f;
      for (int k = c + 1; k < ns; ++k) LU[rr * ns + k] -= f * LU[c * ns + k];
    }
  }
  return true;
}

// lds[w][p][sp] = (ln|det|, sign); one thread per (walker, determinant, spin).
template <typename R>
__global__ void k_slater_lu(DevSys s, const double* __restrict__ phi, const R* __restrict__ F, int Wn,
                            double* __restrict__ lds) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Wn * s.n_det * 2) return;
  const int sp = idx & 1, p = (idx >> 1) % s.n_det;
  const size_t w = (idx >> 1) / s.n_det;
  double* o = lds + idx * 2;
  if ((sp ? s.n_dn : s.n_up) == 0) { o[0] = 0; o[1] = 1; return; }
  double LU[PN_MAX_SPIN * PN_MAX_SPIN];
  double ld, sg;
  slater_block_lu<R>(s, phi + w * s.N * s.n_orb * 5, F + w * s.N * s.n_orb, p, sp, LU, nullptr, ld, sg);
  o[0] = ld;
  o[1] = sg;
}

// Walker-level log-sum of the determinants from the block table:
// m = max ln|det_p| over live determinants, S = sum_p c_p s_p e^{ld_p - m}.
__device__ inline void slater_logsum(const DevSys& s, const double* lw, double& m, double& S) {
  m = -INFINITY;
  for (int p = 0; p < s.n_det; ++p) {
    const double* q = lw + p * 4;
    if (s.ci[p] != 0.0 && q[1] != 0.0 && q[3] != 0.0) m = fmax(m, q[0] + q[2]);
  }
  S = 0;
  for (int p = 0; p < s.n_det; ++p) {
    const double* q = lw + p * 4;
    const double sg = q[1] * q[3];
    if (sg != 0.0) S += s.ci[p] * sg * exp(q[0] + q[2] - m);
  }
}

// inv[w][p][sp][a][b] = u_w omega_p (A^{-1})[b][a] = d ln|psi| / dA[a][b]
// contributed by block (p, sp); zero where the block or the walker is
// singular.  One thread per (walker, determinant, spin).
template <typename R>
__global__ void k_slater_inv(DevSys s, const double* __restrict__ phi, const R* __restrict__ F,
                             const double* __restrict__ u, const double* __restrict__ lds, int Wn, int inv_stride,
                             double* __restrict__ inv) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Wn * s.n_det * 2) return;
  const int sp = idx & 1, p = (idx >> 1) % s.n_det;
  const size_t w = (idx >> 1) / s.n_det;
  const int ns = sp ? s.n_dn : s.n_up;
  if (ns == 0) return;
  double* o = inv + w * inv_stride + (size_t)p * (s.n_up * s.n_up + s.n_dn * s.n_dn) + (sp ? s.n_up * s.n_up : 0);
  const double* lw = lds + w * s.n_det * 4;
  double m, S;
  slater_logsum(s, lw, m, S);
  const double sg = lw[p * 4 + 1] * lw[p * 4 + 3];
  if (!(S != 0.0) || !(m > -INFINITY) || sg == 0.0) {
    for (int k = 0; k < ns * ns; ++k) o[k] = 0;
    return;
  }
  const double om = (u ? u[w] : 1.0) * s.ci[p] * sg * exp(lw[p * 4] + lw[p * 4 + 2] - m) / S;
  double LU[PN_MAX_SPIN * PN_MAX_SPIN];
  int perm[PN_MAX_SPIN];
  double ld, sgb;
  slater_block_lu<R>(s, phi + w * s.N * s.n_orb * 5, F + w * s.N * s.n_orb, p, sp, LU, perm, ld, sgb);
  // column `col` of A^{-1}: entry (b, col) pairs with A[col][b]
  for (int col = 0; col < ns; ++col) {
    double y[PN_MAX_SPIN];
    for (int rr = 0; rr < ns; ++rr) {
      double v = (perm[rr] == col) ? 1.0 : 0.0;
      for (int k = 0; k < rr; ++k) v -= LU[rr * ns + k] * y[k];
      y[rr] = v;
    }
    for (int rr = ns - 1; rr >= 0; --rr) {
      double v = y[rr];
      for (int k = rr + 1; k < ns; ++k) v -= LU[rr * ns + k] * y[k];
      y[rr] = v / LU[rr * ns + rr];
    }
    for (int b = 0; b < ns; ++b) o[col * ns + b] = om * y[b];
  }
}

// Per electron row i: dphit[mu] = sum_p sum_{b: occ_b = mu} inv[p][i][b]
// (determinant order), then dF = dphit phi and, with gr, the orbital part
// of grad_r ln|psi|, sum_mu dphit (1 + F) grad phi_mu(r_i).  Row 0 also
// writes the walker's J cotangent u_w and, with lse, ln|sum_p c_p det_p|.
// One thread per (walker, electron).
template <typename R>
__global__ void k_slater_gather(DevSys s, const double* __restrict__ phi, const R* __restrict__ F,
                                const double* __restrict__ u, const double* __restrict__ lds,
                                const double* __restrict__ inv, int Wn, int inv_stride, R* __restrict__ dF,
                                R* __restrict__ dJ, double* __restrict__ gr, double* __restrict__ lse) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Wn * s.N) return;
  const int N = s.N, no = s.n_orb, i = idx % N;
  const size_t w = idx / N;
  const int sp = i < s.n_up ? 0 : 1, ns = sp ? s.n_dn : s.n_up, e0 = sp ? s.n_up : 0, a = i - e0;
  const int blk = s.n_up * s.n_up + s.n_dn * s.n_dn, off = sp ? s.n_up * s.n_up : 0;
  double dphit[PN_MAX_ORBITALS];
  for (int mu = 0; mu < no; ++mu) dphit[mu] = 0;
  const double* iw = inv + w * inv_stride;
  for (int p = 0; p < s.n_det; ++p) {
    const int* occ = s.occ + p * N + e0;
    const double* q = iw + (size_t)p * blk + off + a * ns;
    for (int b = 0; b < ns; ++b) dphit[occ[b]] += q[b];
  }
  const double* ph = phi + idx * no * 5;
  const R* Fi = F + idx * no;
  for (int mu = 0; mu < no; ++mu) dF[idx * no + mu] = (R)(dphit[mu] * ph[mu * 5]);
  if (gr) {
    double g[3] = {0, 0, 0};
    for (int mu = 0; mu < no; ++mu) {
      const double c = dphit[mu] * (1.0 + (double)Fi[mu]);
      for (int x = 0; x < 3; ++x) g[x] += c * ph[mu * 5 + 1 + x];
    }
    for (int x = 0; x < 3; ++x) gr[idx * 3 + x] = g[x];
  }
  if (i == 0) {
    dJ[w] = (R)(u ? u[w] : 1.0);
    if (lse) {
      double m, S;
      slater_logsum(s, lds + w * s.n_det * 4, m, S);
      lse[w] = (S != 0.0 && m > -INFINITY) ? m + log(fabs(S)) : -INFINITY;
    }
  }
}

// d *= sigmoid(a), in place
template <typename R>
__global__ void k_mul_sigmoid(R* __restrict__ d, const R* __restrict__ a, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] *= sigm_(a[i]);
}

// dJ [Wn] times eta.W3^T -> dS2s [Wn][D]
template <typename R>
__global__ void k_outer_row(const R* __restrict__ dj, const R* __restrict__ w3, R* __restrict__ out, int Wn, int D) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (size_t)Wn * D) out[i] = dj[i / D] * w3[i % D];
}

// dX[w][i][d] += dXs[w][d]
template <typename R>
__global__ void k_bcast_add(R* __restrict__ dX, const R* __restrict__ dXs, int Wn, int N, int D) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)Wn * N * D) return;
  const int d = i % D;
  const int w = i / ((size_t)N * D);
  dX[i] += dXs[(size_t)w * D + d];
}

// Message backward, filter side: dw[w][p][z].
template <typename R>
__global__ void k_msg_bwd_w(DevSys s, const R* __restrict__ Y, const R* __restrict__ H, const R* __restrict__ dZ, int Wn,
                            R* __restrict__ dw) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int Zd = s.Zd, N = s.N;
  if (idx >= (size_t)Wn * s.Ppair * Zd) return;
  const int z = idx % Zd;
  const int p = (idx / Zd) % s.Ppair;
  const int w = idx / ((size_t)Zd * s.Ppair);
  const R* dZw = dZ + (size_t)w * N * 3 * Zd;
  R v;
  if (p < s.Pee) {
    int a = 0, rem = p;
    while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
    const int b = a + 1 + rem;
    const int c = ((a < s.n_up) == (b < s.n_up)) ? 0 : 1;
    const R* Hw_ = H + (size_t)w * N * Zd;
    v = dZw[(size_t)a * 3 * Zd + c * Zd + z] * Hw_[(size_t)b * Zd + z] +
        dZw[(size_t)b * 3 * Zd + c * Zd + z] * Hw_[(size_t)a * Zd + z];
  } else {
    const int q = p - s.Pee, i = q / s.M, I = q % s.M;
    v = dZw[(size_t)i * 3 * Zd + 2 * Zd + z] * Y[I * Zd + z];
  }
  dw[idx] = v;
}

// Message backward, sender side: dH[w][j][z] = sum_i w_ij dZ_{c(i,j)}[i][z];
// nuclear embedding rows: dYr[w][i][I*Zd + z] = w_iI dZ_nuc[i][z].
template <typename R>
__global__ void k_msg_bwd_h(DevSys s, const R* __restrict__ wv, const R* __restrict__ dZ, int Wn, R* __restrict__ dH,
                            R* __restrict__ dYr) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int Zd = s.Zd, N = s.N;
  if (idx >= (size_t)Wn * N * Zd) return;
  const int z = idx % Zd;
  const int j = (idx / Zd) % N;
  const int w = idx / ((size_t)Zd * N);
  const R* ww = wv + (size_t)w * s.Ppair * Zd;
  const R* dZw = dZ + (size_t)w * N * 3 * Zd;
  R acc = 0;
  for (int i = 0; i < N; ++i) {
    if (i == j) continue;
    const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
    const int c = ((i < s.n_up) == (j < s.n_up)) ? 0 : 1;
    acc += ww[(size_t)p * Zd + z] * dZw[(size_t)i * 3 * Zd + c * Zd + z];
  }
  dH[idx] = acc;
  if (dYr)
    for (int I = 0; I < s.M; ++I)
    dYr[(((size_t)w * N + j) * s.M + I) * Zd + z] =
          ww[(size_t)(s.Pee + j * s.M + I) * Zd + z] * dZw[(size_t)j * 3 * Zd + 2 * Zd + z];
}

// Filter backward through the hidden layer: dAh = (dw W2^T) * sigmoid(Ah),
// Sh = ssp(Ah) kept for the W2 gradient.  One warp per pair row.
constexpr int FB_ROWS = 8;  // pair rows per warp in k_filter_bwd
template <typename R>
__global__ void __launch_bounds__(256) k_filter_bwd(DevSys s, DevNet<R> net, int n, const R* __restrict__ Ah,
                                                    const R* __restrict__ dw, int Wn, R* __restrict__ dAh,
                                                    R* __restrict__ Sh) {
  // the three channels' W2 [Hw][Zd] in shared memory, rows padded by one so
  // that lanes running over h hit distinct banks; one warp per pair row,
  // FB_ROWS rows per warp
  extern __shared__ __align__(16) unsigned char fb_smem[];
  const int Hw = s.Hw, Zd = s.Zd, LZ = Zd + 1;
  R* W2s = (R*)fb_smem;                 // [3][Hw][LZ]
  R* dsh = W2s + (size_t)3 * Hw * LZ;   // [8][Zd]
  for (int q = threadIdx.x; q < 3 * Hw * Zd; q += blockDim.x) {
    const int c = q / (Hw * Zd), h = (q / Zd) % Hw, z = q % Zd;
    W2s[((size_t)c * Hw + h) * LZ + z] = net.p[net.off.W2[n][c] + (size_t)h * Zd + z];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  R* dv = dsh + wid * Zd;
  const size_t rows = (size_t)Wn * s.Ppair;
  for (int k = 0; k < FB_ROWS; ++k) {
    const size_t row = ((size_t)blockIdx.x * 8 + wid) * FB_ROWS + k;
    if (row >= rows) break;
    const int ch = pair_channel(s, row % s.Ppair);
    const R* W2 = W2s + (size_t)ch * Hw * LZ;
    for (int z = lane; z < Zd; z += 32) dv[z] = dw[row * Zd + z];
    __syncwarp();
    for (int h = lane; h < Hw; h += 32) {
      R acc = 0;
      for (int z = 0; z < Zd; ++z) acc += dv[z] * W2[h * LZ + z];
      const R a = Ah[row * Hw + h];
      dAh[row * Hw + h] = acc * sigm_(a);
      Sh[row * Hw + h] = ssp_(a);
    }
    __syncwarp();
  }
}

// Same, reading W2 from global memory: for filter widths whose weights do not
// fit in shared memory.
template <typename R>
__global__ void k_filter_bwd_global(DevSys s, DevNet<R> net, int n, const R* __restrict__ Ah, const R* __restrict__ dw, int Wn,
                             R* __restrict__ dAh, R* __restrict__ Sh) {
  __shared__ R sh_d[8][128];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t row = (size_t)blockIdx.x * 8 + wid;
  if (row >= (size_t)Wn * s.Ppair) return;
  const int ch = pair_channel(s, row % s.Ppair);
  const int Hw = s.Hw, Zd = s.Zd;
  for (int z = lane; z < Zd; z += 32) sh_d[wid][z] = dw[row * Zd + z];
  __syncwarp();
  const R* W2 = net.p + net.off.W2[n][ch];
  for (int h = lane; h < Hw; h += 32) {
    R acc = 0;
    for (int z = 0; z < Zd; ++z) acc += sh_d[wid][z] * W2[h * Zd + z];
    const R a = Ah[row * Hw + h];
    dAh[row * Hw + h] = acc * sigm_(a);
    Sh[row * Hw + h] = ssp_(a);
  }
}

// Filter backward towards the pair distance, for grad_r ln|psi|: the hidden
// cotangent dAh = (dw W2^T) * sigmoid(Ah) of pair row p meets the distance
// derivative of the hidden pre-activation, q = e'(d_p) W1, and
// dd[p] += sum_h dAh q.  One warp per pair row, FB_ROWS rows per warp; with
// SW the three channels' W2 sit in shared memory (rows padded by one).
template <typename R, bool SW>
__global__ void __launch_bounds__(256) k_filter_bwd_dist(DevSys s, DevNet<R> net, int n, const R* __restrict__ Ah,
                                                         const R* __restrict__ ef, const R* __restrict__ dw, int Wn,
                                                         double* __restrict__ dd) {
  extern __shared__ __align__(16) unsigned char fd_smem[];
  const int Hw = s.Hw, Zd = s.Zd, K = s.K, LZ = SW ? Zd + 1 : Zd;
  R* W2s = (R*)fd_smem;                               // [3][Hw][LZ] (SW only)
  R* dsh = W2s + (SW ? (size_t)3 * Hw * LZ : 0);      // [8][Zd]
  R* esh = dsh + 8 * Zd;                              // [8][K]
  if (SW) {
    for (int q = threadIdx.x; q < 3 * Hw * Zd; q += blockDim.x) {
      const int c = q / (Hw * Zd), h = (q / Zd) % Hw, z = q % Zd;
      W2s[((size_t)c * Hw + h) * LZ + z] = net.p[net.off.W2[n][c] + (size_t)h * Zd + z];
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  R* dv = dsh + wid * Zd;
  R* ev = esh + wid * K;
  const size_t rows = (size_t)Wn * s.Ppair;
  for (int k = 0; k < FB_ROWS; ++k) {
    const size_t row = ((size_t)blockIdx.x * 8 + wid) * FB_ROWS + k;
    if (row >= rows) break;
    const int ch = pair_channel(s, row % s.Ppair);
    const R* W2 = SW ? W2s + (size_t)ch * Hw * LZ : net.p + net.off.W2[n][ch];
    const R* W1 = net.p + net.off.W1[n][ch];
    for (int z = lane; z < Zd; z += 32) dv[z] = dw[row * Zd + z];
    for (int q = lane; q < K; q += 32) ev[q] = ef[row * 3 * K + K + q];
    __syncwarp();
    double part = 0;
    for (int h = lane; h < Hw; h += 32) {
      R acc = 0;
      for (int z = 0; z < Zd; ++z) acc += dv[z] * W2[h * LZ + z];
      R q = 0;
      for (int kk = 0; kk < K; ++kk) q += ev[kk] * W1[kk * Hw + h];
      part += (double)(acc * sigm_(Ah[row * Hw + h])) * (double)q;
    }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) dd[row] += part;
    __syncwarp();
  }
}

// ln|psi| = gamma + J + ln|sum_p c_p det_p| and
// grad_r ln|psi| = orbital part + sum over pairs of (d ln|psi| / d d_p) grad_r d_p,
// the distance cotangent collecting the filters of every layer and the
// electronic cusp factor gamma.  One thread per walker.
template <typename R>
__global__ void k_drift_combine(DevSys s, const double* __restrict__ geo, const double* __restrict__ lse,
                                const R* __restrict__ J, const double* __restrict__ gr, const double* __restrict__ dd,
                                int Wn, double* __restrict__ logabs, double* __restrict__ grad) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int N = s.N, n3 = 3 * N, P = s.Ppair;
  double g[3 * PN_MAX_ELECTRONS];
  for (int t = 0; t < n3; ++t) g[t] = gr[(size_t)w * n3 + t];
  const double* gw = geo + (size_t)w * P * 4;
  const double* dw = dd + (size_t)w * P;
  double gam = 0;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      const int p = pn_pair_index(a, b, N);
      const double* u = gw + p * 4;
      double c = dw[p];
      if (s.use_gamma) {
        const double cc = ((a < s.n_up) == (b < s.n_up)) ? 0.25 : 0.5;
        const double e = 1.0 / (1.0 + u[0]);
        gam -= cc * e;
        c += cc * e * e;
      }
      for (int x = 0; x < 3; ++x) {
        g[3 * a + x] += c * u[1 + x];
        g[3 * b + x] -= c * u[1 + x];
      }
    }
  for (int q = 0; q < s.Pen; ++q) {
    const int i = q / s.M;
    const double* u = gw + (s.Pee + q) * 4;
    const double c = dw[s.Pee + q];
    for (int x = 0; x < 3; ++x) g[3 * i + x] += c * u[1 + x];
  }
  logabs[w] = gam + (double)J[w] + lse[w];
  for (int t = 0; t < n3; ++t) grad[(size_t)w * n3 + t] = g[t];
}

// ------------------------------------------------------------ weight grads
// part[split][ka][nb] = sum over this split's rows r of A[r][ka] * B[r][nb];
// Weight gradients grad[block] += sum_rows A^T B, many parameter blocks per
// launch.  A == nullptr means a column of ones (bias gradient, Ka = 1).
// With a pair map, logical row r is walker r / cnt, pair map[r % cnt] (the
// pairs of one filter channel), i.e. storage row (r / cnt) * P + map[r % cnt].
// Rows per block are at most about 256; each block sums its rows of one
// 32 x 32 tile in R and writes a float64 partial; the last block of a tile
// to finish (counted with an atomic) adds the partials of all blocks in
// split order and updates the gradient, so the result does not depend on
// block scheduling.  rows_per_c > 0 splits the K rows over three parameter
// blocks stride_c apart (stacked receiving maps).
constexpr int kWgMaxJobs = 24;
constexpr int kWgMaxCtr = 4096;  // 32 x 32 tiles in one group
template <typename R>
struct WgJob {
  const R* A;
  const R* B;
  const int* map;
  int64_t part0, base, stride_c, dst_stride;
  int lda, ldb, rows, Ka, Nb, cnt, rps, nsplit, tn, tk, blk0, ctr0, rows_per_c, ndst;
};
template <typename R>
struct WgGroup {
  int n, P;
  WgJob<R> j[kWgMaxJobs];
};

template <typename R>
__device__ inline void wg_load4(const R* p, R v[4]) {
  if constexpr (sizeof(R) == 4) {
    const float4 q = *(const float4*)p;
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 q0 = *(const double2*)p, q1 = *(const double2*)(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
}

// One block = one (job, split, 32 x 32 tile); 128 threads, each 2 rows (k)
// x 4 columns (n) of the tile.  The storage rows of each 32-row chunk are
// resolved once into shared memory.
template <typename R>
__global__ void __launch_bounds__(128) k_wgrad(const __grid_constant__ WgGroup<R> G, double* __restrict__ part,
                                               unsigned* __restrict__ ctr, double* __restrict__ grad) {
  __shared__ __align__(16) R As[32][32 + 4];
  __shared__ __align__(16) R Bs[32][32 + 4];
  __shared__ long long srow[256];
  __shared__ bool last;
  int ji = 0;
  while (ji + 1 < G.n && (int)blockIdx.x >= G.j[ji + 1].blk0) ++ji;
  const WgJob<R>& J = G.j[ji];
  const int local = (int)blockIdx.x - J.blk0;
  const int ntile = J.tn * J.tk, split = local / ntile, tile = local % ntile;
  const int k0 = (tile / J.tn) * 32, n0 = (tile % J.tn) * 32;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;  // 4 columns x 2 rows each
  const int r_begin = split * J.rps;
  const int r_end = min(J.rows, r_begin + J.rps);
  R acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  if (!J.A) {
    // bias gradient (Ka = 1): column sums of B; thread = (column, row group)
    const int c = tid & 31, grp = tid >> 5;
    R cs = 0;
    if (n0 + c < J.Nb)
      for (int r = r_begin + grp; r < r_end; r += 4) {
        const long long row = J.map ? (long long)(r / J.cnt) * G.P + J.map[r % J.cnt] : (long long)r;
        cs += J.B[row * J.ldb + n0 + c];
      }
    As[grp][c] = cs;
    __syncthreads();
    // thread (tx, ty = 0) holds columns 4 tx .. 4 tx + 3 of row k = 0
    if (ty == 0)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        acc[0][j] = ((As[0][4 * tx + j] + As[1][4 * tx + j]) + As[2][4 * tx + j]) + As[3][4 * tx + j];
  }
  // matrix jobs: rows in segments of 256 (their storage rows resolved once),
  // each segment in 32-row chunks with the next chunk's loads in flight
  // while the current one is summed
  for (int s0 = r_begin; J.A && s0 < r_end; s0 += 256) {
    const int s1 = min(r_end, s0 + 256);
    __syncthreads();  // srow of the previous segment no longer read
    for (int q = tid; q < 256; q += 128) {
      const int r = s0 + q;
      srow[q] = r < s1 ? (J.map ? (long long)(r / J.cnt) * G.P + J.map[r % J.cnt] : (long long)r) : -1;
    }
    __syncthreads();
    R va[8], vb[8];
    auto fetch = [&](int c0) {
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const int e = tid + 128 * l, q = e >> 5, c = e & 31;
        const long long row = c0 + q < 256 ? srow[c0 + q] : -1;
        va[l] = (row >= 0 && k0 + c < J.Ka) ? J.A[row * J.lda + k0 + c] : R(0);
        vb[l] = (row >= 0 && n0 + c < J.Nb) ? J.B[row * J.ldb + n0 + c] : R(0);
      }
    };
    fetch(0);
    for (int c0 = 0; c0 < s1 - s0; c0 += 32) {
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const int e = tid + 128 * l, q = e >> 5, c = e & 31;
        As[q][c] = va[l];
        Bs[q][c] = vb[l];
      }
      __syncthreads();
      if (c0 + 32 < s1 - s0) fetch(c0 + 32);
#pragma unroll 8
      for (int q = 0; q < 32; ++q) {
        const R a0 = As[q][2 * ty], a1 = As[q][2 * ty + 1];
        R b[4];
        wg_load4(&Bs[q][4 * tx], b);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[0][j] += a0 * b[j];
          acc[1][j] += a1 * b[j];
        }
      }
      __syncthreads();
    }
  }
  double* pj = part + J.part0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + 2 * ty + i, nn = n0 + 4 * tx + j;
      if (k < J.Ka && nn < J.Nb) pj[((size_t)split * J.Ka + k) * J.Nb + nn] = (double)acc[i][j];
    }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&ctr[J.ctr0 + tile], 1u) == (unsigned)(J.nsplit - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // each element summed over the splits in split order; a thread's eight
  // elements are interleaved so that their loads overlap
  double sum[2][4];
  bool ok[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ok[i][j] = k0 + 2 * ty + i < J.Ka && n0 + 4 * tx + j < J.Nb;
      sum[i][j] = 0;
    }
#pragma unroll 2
  for (int sp = 0; sp < J.nsplit; ++sp)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (ok[i][j]) sum[i][j] += __ldcg(pj + ((size_t)sp * J.Ka + (k0 + 2 * ty + i)) * J.Nb + n0 + 4 * tx + j);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!ok[i][j]) continue;
      const int k = k0 + 2 * ty + i, nn = n0 + 4 * tx + j;
      int64_t dst;
      if (J.rows_per_c > 0)
        dst = J.base + (int64_t)(k / J.rows_per_c) * J.stride_c + (int64_t)(k % J.rows_per_c) * J.Nb + nn;
      else
        dst = J.base + (int64_t)k * J.Nb + nn;
      for (int d = 0; d < J.ndst; ++d) grad[dst + d * J.dst_stride] += sum[i][j];
    }
  if (tid == 0) ctr[J.ctr0 + tile] = 0u;  // ready for the next launch
}

__global__ void k_add_to(double* __restrict__ grad, int64_t off, const double* __restrict__ v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) grad[off + i] += v[i];
}

}  // namespace pnb

using namespace pnb;


// Y (+)= X W^T for W stored [Nout][Kd] (the backward of y = x W).
template <typename R>
__global__ void __launch_bounds__(256) k_linear_bt(const R* __restrict__ X, int ldx, const R* __restrict__ W, int ldw,
                                                   R* __restrict__ Y, int ldy, int rows, int Kd, int Nout, int accumulate) {
  __shared__ R As[16][64 + 1];
  __shared__ R Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;  // row tiles in x: no 65535 limit
  R acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    for (int l = 0; l < 4; ++l) {
      const int e = threadIdx.x + l * 256;
      const int rr = e >> 4, kk = e & 15;
      As[kk][rr] = (row0 + rr < rows && k0 + kk < Kd) ? X[(size_t)(row0 + rr) * ldx + k0 + kk] : R(0);
      // B(k, n) = W[n][k]
      const int cb = e >> 4, kb = e & 15;
      Bs[kb][cb] = (k0 + kb < Kd && col0 + cb < Nout) ? W[(size_t)(col0 + cb) * ldw + k0 + kb] : R(0);
    }
    __syncthreads();
    for (int kk = 0; kk < 16; ++kk) {
      R a[4], b[4];
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + ty * 4 + i;
    if (gr >= rows) continue;
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc >= Nout) continue;
      R* y = Y + (size_t)gr * ldy + gc;
      *y = accumulate ? *y + acc[i][j] : acc[i][j];
    }
  }
}

namespace {

template <typename R>
struct Tape {
  int Wb;
  double* geo;
  double* phi;
  double* u;
  R *ef, *X, *H, *Z, *Ah, *wv;            // per layer stacks
  R *kA1, *kS1, *kA2, *kS2, *F;           // kappa
  R *Xs, *eA1, *eS1, *eA2, *eS2, *J;      // eta
  R *dX, *dX2, *dH, *dZ, *dw, *dAh, *Sh, *dYr, *dF, *dJ, *dA, *dB, *dXs, *dAs, *dBs;
  double *lds, *inv;      // determinant blocks: (ln|det|, sign) per spin, weighted inverses
  double *dd, *gr, *lse;  // position gradient: distance cotangents, orbital part, determinant log-sum
  double* part;
  size_t part_elems;
  unsigned* ctr;  // per-tile completion counters of k_wgrad (kept at zero between launches)
  double* bias_tmp;
  char* end;  // one past the last carved byte
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename R>
size_t tape_bytes_per_walker(const DevSys& s) {
  const size_t N = s.N, D = s.D, Zd = s.Zd, L = s.L, P = s.Ppair, Hw = s.Hw, no = s.n_orb;
  size_t e = 0;
  e += P * 3 * s.K + (L + 1) * N * D + L * N * Zd + L * N * 3 * Zd + L * P * Hw + L * P * Zd;
  e += 4 * N * D + N * no + 5 * D + 1;
  e += 2 * N * D + N * Zd + N * 3 * Zd + P * Zd + 2 * P * Hw + N * s.M * Zd + N * no + 1 + 2 * N * D + 3 * D;
  const size_t blocks = (size_t)s.n_det * (4 + s.n_up * s.n_up + s.n_dn * s.n_dn);
  return e * sizeof(R) + (P * 4 + N * no * 5 + 1 + P + 3 * N + 1 + blocks) * 8 + 64 * 29;
}

template <typename R>
Tape<R> carve_tape(const DevSys& s, int Wb, void* base, size_t part_elems) {
  Tape<R> t;
  char* p = (char*)base;
  const size_t W = Wb, N = s.N, D = s.D, Zd = s.Zd, L = s.L, P = s.Ppair, Hw = s.Hw, no = s.n_orb;
  auto take = [&](size_t bytes) { char* q = p; p += al(bytes); return (void*)q; };
  const size_t r = sizeof(R);
  t.Wb = Wb;
  t.geo = (double*)take(W * P * 4 * 8);
  t.phi = (double*)take(W * N * no * 5 * 8);
  t.u = (double*)take(W * 8);
  t.ef = (R*)take(W * P * 3 * s.K * r);
  t.X = (R*)take((L + 1) * W * N * D * r);
  t.H = (R*)take(L * W * N * Zd * r + r);
  t.Z = (R*)take(L * W * N * 3 * Zd * r + r);
  t.Ah = (R*)take(L * W * P * Hw * r + r);
  t.wv = (R*)take(L * W * P * Zd * r + r);
  t.kA1 = (R*)take(W * N * D * r);
  t.kS1 = (R*)take(W * N * D * r);
  t.kA2 = (R*)take(W * N * D * r);
  t.kS2 = (R*)take(W * N * D * r);
  t.F = (R*)take(W * N * no * r);
  t.Xs = (R*)take(W * D * r);
  t.eA1 = (R*)take(W * D * r);
  t.eS1 = (R*)take(W * D * r);
  t.eA2 = (R*)take(W * D * r);
  t.eS2 = (R*)take(W * D * r);
  t.J = (R*)take(W * r);
  t.dX = (R*)take(W * N * D * r);
  t.dX2 = (R*)take(W * N * D * r);
  t.dH = (R*)take(W * N * Zd * r);
  t.dZ = (R*)take(W * N * 3 * Zd * r);
  t.dw = (R*)take(W * P * Zd * r);
  t.dAh = (R*)take(W * P * Hw * r);
  t.Sh = (R*)take(W * P * Hw * r);
  t.dYr = (R*)take(W * N * s.M * Zd * r);
  t.dF = (R*)take(W * N * no * r);
  t.dJ = (R*)take(W * r);
  t.dA = (R*)take(W * N * D * r);
  t.dB = (R*)take(W * N * D * r);
  t.dXs = (R*)take(W * D * r);
  t.dAs = (R*)take(W * D * r);
  t.dBs = (R*)take(W * D * r);
  t.lds = (double*)take(W * s.n_det * 4 * 8);
  t.inv = (double*)take(W * s.n_det * (s.n_up * s.n_up + s.n_dn * s.n_dn) * 8);
  t.dd = (double*)take(W * P * 8);
  t.gr = (double*)take(W * N * 3 * 8);
  t.lse = (double*)take(W * 8);
  t.part = (double*)take(part_elems * 8);
  t.part_elems = part_elems;
  t.ctr = (unsigned*)take(kWgMaxCtr * 4);
  t.bias_tmp = nullptr;
  t.end = p;
  return t;
}

// Collects the weight-gradient blocks of one dependency group (their A and
// B stay valid until flush) and runs them as one k_wgrad launch.
template <typename R>
struct WgBatch {
  const DevSys* s;
  Tape<R>* t;
  double* grad;
  WgGroup<R> G;
  int64_t rows_total[kWgMaxJobs];
  void reset() { G.n = 0; G.P = s->Ppair; }
  // grad += sum_rows A^T B (or column sums of B when A is null) into the
  // parameter block at `base`; ch >= 0 restricts the rows to the pairs of
  // filter channel ch (rows then count walkers x pairs)
  int add(const R* A, int lda, const R* B, int ldb, int rows, int Ka, int Nb, int ch, int64_t base,
          int64_t stride_c, int rows_per_c, int ndst = 1, int64_t dst_stride = 0) {
    const int* map = nullptr;
    int cnt = 0;
    if (ch >= 0) {
      cnt = s->ch_off[ch + 1] - s->ch_off[ch];
      map = s->ch_pairs + s->ch_off[ch];
      rows = (rows / s->Ppair) * cnt;
    }
    if (rows <= 0) return PN_OK;
    if (G.n == kWgMaxJobs) {
      pn_set_error("internal: weight-gradient group full");
      return PN_EINVAL;
    }
    WgJob<R>& J = G.j[G.n++];
    J.A = A; J.B = B; J.map = map; J.cnt = cnt;
    J.lda = lda; J.ldb = ldb; J.rows = rows; J.Ka = Ka; J.Nb = Nb;
    J.base = base; J.stride_c = stride_c; J.rows_per_c = rows_per_c;
    J.ndst = ndst; J.dst_stride = dst_stride;
    J.tn = (Nb + 31) / 32;
    J.tk = (Ka + 31) / 32;
    return PN_OK;
  }
  int flush(cudaStream_t st) {
    if (G.n == 0) return PN_OK;
    constexpr int kRowsPerBlock = 256;
    // splits of about 256 rows, fewer if the partial buffer would overflow
    size_t need = 0;
    for (int i = 0; i < G.n; ++i)
      need += (size_t)G.j[i].Ka * G.j[i].Nb * ((G.j[i].rows + kRowsPerBlock - 1) / kRowsPerBlock);
    const double scale = need > t->part_elems ? (double)t->part_elems / (double)need : 1.0;
    int64_t part0 = 0;
    int blk = 0, ctr0 = 0;
    for (int i = 0; i < G.n; ++i) {
      WgJob<R>& J = G.j[i];
      const int want = (J.rows + kRowsPerBlock - 1) / kRowsPerBlock;
      J.nsplit = std::max(1, std::min(want, (int)(want * scale)));
      J.rps = (J.rows + J.nsplit - 1) / J.nsplit;
      J.nsplit = (J.rows + J.rps - 1) / J.rps;
      J.part0 = part0;
      J.blk0 = blk;
      J.ctr0 = ctr0;
      part0 += (int64_t)J.nsplit * J.Ka * J.Nb;
      blk += J.nsplit * J.tn * J.tk;
      ctr0 += J.tn * J.tk;
    }
    if ((size_t)part0 > t->part_elems || ctr0 > kWgMaxCtr) {
      pn_set_error("internal: weight-gradient partials exceed their buffer");
      return PN_EINVAL;
    }
    PN_LAUNCH("k_wgrad", st, k_wgrad<R><<<blk, 128, 0, st>>>(G, t->part, t->ctr, grad));
    reset();
    return PN_OK;
  }
};

// The three determinant passes (one profiling class, "k_slater_bwd"); gr
// and lse may be null.
template <typename R>
int slater_bwd(const DevSys& s, Tape<R>& t, const double* u, int Wn, double* gr, double* lse, cudaStream_t st) {
  const size_t nb = (size_t)Wn * s.n_det * 2;
  const int inv_stride = s.n_det * (s.n_up * s.n_up + s.n_dn * s.n_dn);
  PN_LAUNCH("k_slater_bwd", st, k_slater_lu<R><<<nblk(nb, 64), 64, 0, st>>>(s, t.phi, t.F, Wn, t.lds));
  PN_LAUNCH("k_slater_bwd", st,
            k_slater_inv<R><<<nblk(nb, 64), 64, 0, st>>>(s, t.phi, t.F, u, t.lds, Wn, inv_stride, t.inv));
  PN_LAUNCH("k_slater_bwd", st,
            k_slater_gather<R><<<nblk((size_t)Wn * s.N, 64), 64, 0, st>>>(s, t.phi, t.F, u, t.lds, t.inv, Wn,
                                                                          inv_stride, t.dF, t.dJ, gr, lse));
  return PN_OK;
}

template <typename R>
int linear_bt(const R* X, int ldx, const R* W, int ldw, R* Y, int ldy, int rows, int Kd, int Nout, int acc,
              cudaStream_t st) {
  if (rows <= 0) return PN_OK;
  if constexpr (sizeof(R) == 4) {
    const int e = pn_linear_bt_f32((const float*)X, ldx, (const float*)W, ldw, (float*)Y, ldy, rows, Kd, Nout, acc, st);
    if (e != PN_ENOTREADY) return e;
  }
  dim3 grid((rows + 63) / 64, (Nout + 63) / 64);
  PN_LAUNCH("k_linear_bt", st, k_linear_bt<R><<<grid, 256, 0, st>>>(X, ldx, W, ldw, Y, ldy, rows, Kd, Nout, acc));
  return PN_OK;
}

}  // namespace



// Value pass keeping every activation on the tape.  With `drift` the
// features also carry their distance derivatives and the Jastrow factor J
// itself is formed (the parameter gradient needs neither).
template <typename R>
static int tape_value_pass(const DevSys& s, const DevNet<R>& net, Tape<R>& t, const double* r, int Wn, bool drift,
                           cudaStream_t st) {
  const int N = s.N, D = s.D, Zd = s.Zd, L = s.L, P = s.Ppair, Hw = s.Hw, no = s.n_orb;
  const NetOff& o = net.off;
  const int rows = Wn * N;
  const size_t WND = (size_t)Wn * N * D;
  if (int e = pn_launch_geometry_orbitals(s, r, Wn, t.geo, t.phi, st)) return e;
  if (int e = pn_launch_features_init<R>(s, net.p + o.x0, t.geo, Wn, drift ? 1 : 0, t.ef, t.X, st)) return e;
  for (int n = 0; n < L; ++n) {
    R* Xn = t.X + (size_t)n * WND;
    R* Xn1 = t.X + (size_t)(n + 1) * WND;
    R* Hn = t.H + (size_t)n * rows * Zd;
    R* Zn = t.Z + (size_t)n * rows * 3 * Zd;
    R* Ahn = t.Ah + (size_t)n * Wn * P * Hw;
    R* wn = t.wv + (size_t)n * Wn * P * Zd;
    if (int e = pn_linear<R>(&s, PN_TC_VALUE, Xn, D, net.p + o.hW[n], Zd, net.p + o.hb[n], Hn, Zd, rows, D, Zd, 1, 0, st)) return e;
    int fe = PN_ENOTREADY;
    if constexpr (sizeof(R) == 4)
      fe = pn_filter_tile_value(s, net, n, (const float*)t.ef, Wn, (float*)Ahn, (float*)wn, st);
    if (fe != PN_OK && fe != PN_ENOTREADY) return fe;
    if (fe == PN_ENOTREADY)
      PN_LAUNCH("k_filter_tape", st, k_filter_tape<R><<<nblk((size_t)Wn * P, 8), 256, 0, st>>>(s, net, n, t.ef, Wn, Ahn, wn));
    PN_LAUNCH("k_message_value", st, k_message_value<R><<<nblk((size_t)rows * Zd, 256), 256, 0, st>>>(s, net.p + o.Y, wn, Hn, Wn, Zn));
    PN_CUDA(cudaMemcpyAsync(Xn1, Xn, WND * sizeof(R), cudaMemcpyDeviceToDevice, st));
    if (int e = pn_linear<R>(&s, PN_TC_VALUE, Zn, 3 * Zd, net.Gcat + (size_t)n * 3 * Zd * D, D, net.Gb + (size_t)n * D, Xn1, D, rows,
                             3 * Zd, D, 1, 1, st))
      return e;
  }
  R* XL = t.X + (size_t)L * WND;
  // kappa
  if (int e = pn_linear<R>(&s, PN_TC_VALUE, XL, D, net.p + o.kW[0], D, net.p + o.kb[0], t.kA1, D, rows, D, D, 1, 0, st)) return e;
  PN_LAUNCH("k_ssp_copy", st, k_ssp_copy<R><<<nblk(WND, 256), 256, 0, st>>>(t.kA1, t.kS1, WND));
  if (int e = pn_linear<R>(&s, PN_TC_VALUE, t.kS1, D, net.p + o.kW[1], D, net.p + o.kb[1], t.kA2, D, rows, D, D, 1, 0, st)) return e;
  PN_LAUNCH("k_ssp_copy", st, k_ssp_copy<R><<<nblk(WND, 256), 256, 0, st>>>(t.kA2, t.kS2, WND));
  if (int e = pn_linear<R>(&s, PN_TC_VALUE, t.kS2, D, net.p + o.kW[2], no, net.p + o.kb[2], t.F, no, rows, D, no, 1, 0, st)) return e;
  // eta
  if (int e = pn_launch_sum_electrons<R>(XL, t.Xs, Wn, N, D, st)) return e;
  if (int e = pn_linear<R>(&s, PN_TC_VALUE, t.Xs, D, net.p + o.eW[0], D, net.p + o.eb[0], t.eA1, D, Wn, D, D, 1, 0, st)) return e;
  PN_LAUNCH("k_ssp_copy", st, k_ssp_copy<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.eA1, t.eS1, (size_t)Wn * D));
  if (int e = pn_linear<R>(&s, PN_TC_VALUE, t.eS1, D, net.p + o.eW[1], D, net.p + o.eb[1], t.eA2, D, Wn, D, D, 1, 0, st)) return e;
  PN_LAUNCH("k_ssp_copy", st, k_ssp_copy<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.eA2, t.eS2, (size_t)Wn * D));
  if (drift)
    if (int e = pn_linear<R>(&s, PN_TC_VALUE, t.eS2, D, net.p + o.eW[2], 1, net.p + o.eb[2], t.J, 1, Wn, D, 1, 1, 0, st))
      return e;
  return PN_OK;
}

// Filter backward towards the distances for layer n (shared-memory W2 when it fits).
template <typename R>
static int filter_bwd_dist(const DevSys& s, const DevNet<R>& net, int n, const R* Ah, const R* ef, const R* dw, int Wn,
                           double* dd, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    const int fe = pn_filter_tile_dist(s, net, n, (const float*)Ah, (const float*)ef, (const float*)dw, Wn, dd, st);
    if (fe != PN_ENOTREADY) return fe;
  }
  const size_t tail = (size_t)8 * (s.Zd + s.K) * sizeof(R);
  const size_t fb = (size_t)3 * s.Hw * (s.Zd + 1) * sizeof(R) + tail;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const unsigned grid = nblk((size_t)Wn * s.Ppair, 8 * FB_ROWS);
  if (fb <= (size_t)maxsm) {
    if (fb > 48 * 1024)
      PN_CUDA(pn_allow_max_smem(k_filter_bwd_dist<R, true>));
    PN_LAUNCH("k_filter_bwd_dist", st,
              (k_filter_bwd_dist<R, true><<<grid, 256, fb, st>>>(s, net, n, Ah, ef, dw, Wn, dd)));
  } else {
    PN_LAUNCH("k_filter_bwd_dist", st,
              (k_filter_bwd_dist<R, false><<<grid, 256, tail, st>>>(s, net, n, Ah, ef, dw, Wn, dd)));
  }
  return PN_OK;
}

// ln|psi| and grad_r ln|psi| of Wn walkers by reverse mode: the value pass
// on the tape, then the chain back from ln|psi| (weight 1 per walker)
// through the determinants, both heads and the interaction layers to the
// pair distances and the orbitals, with no weight gradients formed.
template <typename R>
static int drift_chunk(const DevSys& s, const DevNet<R>& net, Tape<R>& t, const double* r, int Wn, double* logabs,
                       double* grad, cudaStream_t st) {
  const int N = s.N, D = s.D, Zd = s.Zd, L = s.L, P = s.Ppair, Hw = s.Hw, no = s.n_orb;
  const NetOff& o = net.off;
  const int rows = Wn * N;
  const size_t WND = (size_t)Wn * N * D;
  if (int e = tape_value_pass<R>(s, net, t, r, Wn, true, st)) return e;
  PN_CUDA(cudaMemsetAsync(t.dd, 0, (size_t)Wn * P * 8, st));
  if (int e = slater_bwd<R>(s, t, nullptr, Wn, t.gr, t.lse, st)) return e;
  // kappa head
  if (int e = linear_bt<R>(t.dF, no, net.p + o.kW[2], no, t.dA, D, rows, no, D, 0, st)) return e;
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk(WND, 256), 256, 0, st>>>(t.dA, t.kA2, WND));
  if (int e = linear_bt<R>(t.dA, D, net.p + o.kW[1], D, t.dB, D, rows, D, D, 0, st)) return e;
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk(WND, 256), 256, 0, st>>>(t.dB, t.kA1, WND));
  if (int e = linear_bt<R>(t.dB, D, net.p + o.kW[0], D, t.dX, D, rows, D, D, 0, st)) return e;
  // eta head
  PN_LAUNCH("k_outer_row", st, k_outer_row<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.dJ, net.p + o.eW[2], t.dAs, Wn, D));
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.dAs, t.eA2, (size_t)Wn * D));
  if (int e = linear_bt<R>(t.dAs, D, net.p + o.eW[1], D, t.dBs, D, Wn, D, D, 0, st)) return e;
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.dBs, t.eA1, (size_t)Wn * D));
  if (int e = linear_bt<R>(t.dBs, D, net.p + o.eW[0], D, t.dXs, D, Wn, D, D, 0, st)) return e;
  PN_LAUNCH("k_bcast_add", st, k_bcast_add<R><<<nblk(WND, 256), 256, 0, st>>>(t.dX, t.dXs, Wn, N, D));
  // interaction layers, last to first; t.dX holds d/dX^(n+1)
  for (int n = L - 1; n >= 0; --n) {
    R* Hn = t.H + (size_t)n * rows * Zd;
    R* Ahn = t.Ah + (size_t)n * Wn * P * Hw;
    R* wn = t.wv + (size_t)n * Wn * P * Zd;
    if (int e = linear_bt<R>(t.dX, D, net.Gcat + (size_t)n * 3 * Zd * D, D, t.dZ, 3 * Zd, rows, D, 3 * Zd, 0, st))
      return e;
    PN_LAUNCH("k_msg_bwd_w", st, k_msg_bwd_w<R><<<nblk((size_t)Wn * P * Zd, 256), 256, 0, st>>>(s, net.p + o.Y, Hn, t.dZ, Wn, t.dw));
    PN_LAUNCH("k_msg_bwd_h", st,
              k_msg_bwd_h<R><<<nblk((size_t)rows * Zd, 256), 256, 0, st>>>(s, wn, t.dZ, Wn, t.dH, (R*)nullptr));
    if (int e = filter_bwd_dist<R>(s, net, n, Ahn, t.ef, t.dw, Wn, t.dd, st)) return e;
    if (n > 0)  // x^(0) is the constant embedding
      if (int e = linear_bt<R>(t.dH, Zd, net.p + o.hW[n], Zd, t.dX, D, rows, Zd, D, 1, st)) return e;
  }
  PN_LAUNCH("k_drift_combine", st,
            k_drift_combine<R><<<nblk(Wn, 64), 64, 0, st>>>(s, t.geo, t.lse, t.J, t.gr, t.dd, Wn, logabs, grad));
  return PN_OK;
}

template <typename R>
static int grad_chunk(const DevSys& s, const DevNet<R>& net, Tape<R>& t, const double* r, const double* u, int Wn,
                      double* grad, cudaStream_t st) {
  const int N = s.N, D = s.D, Zd = s.Zd, L = s.L, P = s.Ppair, Hw = s.Hw, no = s.n_orb, K = s.K;
  const NetOff& o = net.off;
  const int rows = Wn * N;
  const size_t WND = (size_t)Wn * N * D;
  R* XL = t.X + (size_t)L * WND;
  if (int e = tape_value_pass<R>(s, net, t, r, Wn, false, st)) return e;

  // ---------------- backward
  WgBatch<R> wg;
  wg.s = &s;
  wg.t = &t;
  wg.grad = grad;
  wg.reset();
  if (int e = slater_bwd<R>(s, t, u, Wn, nullptr, nullptr, st)) return e;
  // kappa head
  if (int e = wg.add(t.kS2, D, t.dF, no, rows, D, no, -1, o.kW[2], 0, 0)) return e;
  if (int e = wg.add(nullptr, 0, t.dF, no, rows, 1, no, -1, o.kb[2], 0, 0)) return e;
  if (int e = linear_bt<R>(t.dF, no, net.p + o.kW[2], no, t.dA, D, rows, no, D, 0, st)) return e;
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk(WND, 256), 256, 0, st>>>(t.dA, t.kA2, WND));
  if (int e = wg.add(t.kS1, D, t.dA, D, rows, D, D, -1, o.kW[1], 0, 0)) return e;
  if (int e = wg.add(nullptr, 0, t.dA, D, rows, 1, D, -1, o.kb[1], 0, 0)) return e;
  if (int e = linear_bt<R>(t.dA, D, net.p + o.kW[1], D, t.dB, D, rows, D, D, 0, st)) return e;
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk(WND, 256), 256, 0, st>>>(t.dB, t.kA1, WND));
  if (int e = wg.add(XL, D, t.dB, D, rows, D, D, -1, o.kW[0], 0, 0)) return e;
  if (int e = wg.add(nullptr, 0, t.dB, D, rows, 1, D, -1, o.kb[0], 0, 0)) return e;
  if (int e = linear_bt<R>(t.dB, D, net.p + o.kW[0], D, t.dX, D, rows, D, D, 0, st)) return e;
  // eta head (J = eta(sum_i x_i); dJ/d out = u)
  if (int e = wg.add(t.eS2, D, t.dJ, 1, Wn, D, 1, -1, o.eW[2], 0, 0)) return e;
  if (int e = wg.add(nullptr, 0, t.dJ, 1, Wn, 1, 1, -1, o.eb[2], 0, 0)) return e;
  PN_LAUNCH("k_outer_row", st, k_outer_row<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.dJ, net.p + o.eW[2], t.dAs, Wn, D));
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.dAs, t.eA2, (size_t)Wn * D));
  if (int e = wg.add(t.eS1, D, t.dAs, D, Wn, D, D, -1, o.eW[1], 0, 0)) return e;
  if (int e = wg.add(nullptr, 0, t.dAs, D, Wn, 1, D, -1, o.eb[1], 0, 0)) return e;
  if (int e = linear_bt<R>(t.dAs, D, net.p + o.eW[1], D, t.dBs, D, Wn, D, D, 0, st)) return e;
  PN_LAUNCH("k_mul_sigmoid", st, k_mul_sigmoid<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(t.dBs, t.eA1, (size_t)Wn * D));
  if (int e = wg.add(t.Xs, D, t.dBs, D, Wn, D, D, -1, o.eW[0], 0, 0)) return e;
  if (int e = wg.add(nullptr, 0, t.dBs, D, Wn, 1, D, -1, o.eb[0], 0, 0)) return e;
  if (int e = linear_bt<R>(t.dBs, D, net.p + o.eW[0], D, t.dXs, D, Wn, D, D, 0, st)) return e;
  if (int e = wg.flush(st)) return e;  // both heads' weight gradients
  PN_LAUNCH("k_bcast_add", st, k_bcast_add<R><<<nblk(WND, 256), 256, 0, st>>>(t.dX, t.dXs, Wn, N, D));
  // interaction layers, last to first; t.dX holds d/dX^(n+1)
  for (int n = L - 1; n >= 0; --n) {
    R* Xn = t.X + (size_t)n * WND;
    R* Hn = t.H + (size_t)n * rows * Zd;
    R* Zn = t.Z + (size_t)n * rows * 3 * Zd;
    R* Ahn = t.Ah + (size_t)n * Wn * P * Hw;
    R* wn = t.wv + (size_t)n * Wn * P * Zd;
    // receiving maps: X^(n+1) = X^(n) + [z_same z_anti z_nuc] Gcat + sum of biases
    if (int e = wg.add(Zn, 3 * Zd, t.dX, D, rows, 3 * Zd, D, -1, o.GW[n][0], o.GW[n][1] - o.GW[n][0], Zd))
      return e;
    // the three receiving-map biases share one gradient, the column sums of dX
    if (int e = wg.add(nullptr, 0, t.dX, D, rows, 1, D, -1, o.Gb[n][0], 0, 0, 3, o.Gb[n][1] - o.Gb[n][0])) return e;
    if (int e = linear_bt<R>(t.dX, D, net.Gcat + (size_t)n * 3 * Zd * D, D, t.dZ, 3 * Zd, rows, D, 3 * Zd, 0, st))
      return e;
    // messages
    PN_LAUNCH("k_msg_bwd_w", st, k_msg_bwd_w<R><<<nblk((size_t)Wn * P * Zd, 256), 256, 0, st>>>(s, net.p + o.Y, Hn, t.dZ, Wn, t.dw));
    PN_LAUNCH("k_msg_bwd_h", st, k_msg_bwd_h<R><<<nblk((size_t)rows * Zd, 256), 256, 0, st>>>(s, wn, t.dZ, Wn, t.dH, t.dYr));
    if (int e = wg.add(nullptr, 0, t.dYr, s.M * Zd, rows, 1, s.M * Zd, -1, o.Y, 0, 0)) return e;
    // filters, per channel
    int fe = PN_ENOTREADY;
    if constexpr (sizeof(R) == 4)
      fe = pn_filter_tile_bwd(s, net, n, (const float*)Ahn, (const float*)t.dw, Wn, (float*)t.dAh, (float*)t.Sh, st);
    if (fe != PN_OK && fe != PN_ENOTREADY) return fe;
    if (fe == PN_ENOTREADY) {
      const size_t fb = ((size_t)3 * Hw * (Zd + 1) + 8 * Zd) * sizeof(R);
      int dev = 0, maxsm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (fb <= (size_t)maxsm) {
        if (fb > 48 * 1024)
          PN_CUDA(pn_allow_max_smem(k_filter_bwd<R>));
        PN_LAUNCH("k_filter_bwd", st,
                  k_filter_bwd<R><<<nblk((size_t)Wn * P, 8 * FB_ROWS), 256, fb, st>>>(s, net, n, Ahn, t.dw, Wn,
                                                                                     t.dAh, t.Sh));
      } else {
        PN_LAUNCH("k_filter_bwd", st,
                  k_filter_bwd_global<R><<<nblk((size_t)Wn * P, 8), 256, 0, st>>>(s, net, n, Ahn, t.dw, Wn, t.dAh,
                                                                                  t.Sh));
      }
    }
    for (int c = 0; c < 3; ++c) {
      if (int e = wg.add(t.Sh, Hw, t.dw, Zd, Wn * P, Hw, Zd, c, o.W2[n][c], 0, 0)) return e;
      if (int e = wg.add(nullptr, 0, t.dw, Zd, Wn * P, 1, Zd, c, o.b2[n][c], 0, 0)) return e;
      if (int e = wg.add(t.ef, 3 * K, t.dAh, Hw, Wn * P, K, Hw, c, o.W1[n][c], 0, 0)) return e;
      if (int e = wg.add(nullptr, 0, t.dAh, Hw, Wn * P, 1, Hw, c, o.b1[n][c], 0, 0)) return e;
    }
    // input map h
    if (int e = wg.add(Xn, D, t.dH, Zd, rows, D, Zd, -1, o.hW[n], 0, 0)) return e;
    if (int e = wg.add(nullptr, 0, t.dH, Zd, rows, 1, Zd, -1, o.hb[n], 0, 0)) return e;
    if (int e = wg.flush(st)) return e;  // this layer's weight gradients, before dX changes
    // d/dX^(n) = d/dX^(n+1) + dH Wh^T
    if (int e = linear_bt<R>(t.dH, Zd, net.p + o.hW[n], Zd, t.dX, D, rows, Zd, D, 1, st)) return e;
  }
  // shared electron embedding
  if (int e = wg.add(nullptr, 0, t.dX, D, rows, 1, D, -1, o.x0, 0, 0)) return e;
  return wg.flush(st);
}

// Grows the system's tape allocation to at least `bytes` (never shrinks it).
static int ensure_tape(pn_system_s* sys, size_t bytes) {
  if (bytes <= sys->tape_bytes) return PN_OK;
  if (sys->tape_mem) cudaFree(sys->tape_mem);
  sys->tape_mem = nullptr;
  sys->tape_bytes = 0;
  if (cudaMalloc(&sys->tape_mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    pn_set_error("cannot allocate %zu bytes of tape", bytes);
    return PN_ENOMEM;
  }
  sys->tape_bytes = bytes;
  return PN_OK;
}

template <typename R>
static int grad_impl(pn_system_s* sys, const double* r, int W, const double* cot, double* grad, size_t budget,
                     cudaStream_t st) {
  const DevSys& s = sys->ds;
  const DevNet<R> net = pn_devnet<R>(sys);
  const int N = s.N;
  const size_t per = tape_bytes_per_walker<R>(s);
  // partial tiles: enough for the largest weight block times 256 splits
  size_t maxKN = std::max<size_t>({(size_t)s.D * s.D, (size_t)3 * s.Zd * s.D, (size_t)s.K * s.Hw,
                                   (size_t)s.Hw * s.Zd, (size_t)s.D * s.n_orb, (size_t)s.M * s.Zd, 1});
  const size_t part_elems = maxKN * 256;
  const size_t fixed = part_elems * 8 + kWgMaxCtr * 4 + 4096 * 64;
  // default: room for one workspace chunk (at least 256 walkers)
  if (budget == 0) budget = fixed + per * (size_t)std::min(W, std::max(sys->Wc, 256)) + 65536;
  if (budget <= fixed + per) {
    pn_set_error("grad: memory budget %zu below one walker's tape (%zu bytes)", budget, fixed + per);
    return PN_EINVAL;
  }
  int Wb = (int)std::min<size_t>((size_t)W, (budget - fixed) / per);
  Wb = std::max(1, Wb);
  const size_t bytes = fixed + per * Wb + 65536;
  if (int e = ensure_tape(sys, bytes)) return e;
  Tape<R> t = carve_tape<R>(s, Wb, sys->tape_mem, part_elems);
  if (t.end > (char*)sys->tape_mem + sys->tape_bytes) {
    pn_set_error("grad: tape layout (%zu bytes) exceeds its allocation (%zu)", (size_t)(t.end - (char*)sys->tape_mem),
                 sys->tape_bytes);
    return PN_EINVAL;
  }
  PN_CUDA(cudaMemsetAsync(t.ctr, 0, kWgMaxCtr * 4, st));
  const bool rdev = pn_is_device_ptr(r), udev = pn_is_device_ptr(cot), gdev = pn_is_device_ptr(grad);
  double* gd = grad;
  if (!gdev) {
    PN_CUDA(cudaMallocAsync((void**)&gd, (size_t)sys->off.total * 8, st));
  }
  PN_CUDA(cudaMemsetAsync(gd, 0, (size_t)sys->off.total * 8, st));
  // r staging reuses the system workspace's position buffer when needed
  double* rstage = nullptr;
  if (!rdev) PN_CUDA(cudaMallocAsync((void**)&rstage, (size_t)Wb * N * 3 * 8, st));
  for (int c0 = 0; c0 < W; c0 += Wb) {
    const int Wn = std::min(Wb, W - c0);
    const double* rc = r + (size_t)c0 * N * 3;
    if (!rdev) {
      PN_CUDA(cudaMemcpyAsync(rstage, rc, (size_t)Wn * N * 3 * 8, cudaMemcpyHostToDevice, st));
      rc = rstage;
    }
    PN_CUDA(cudaMemcpyAsync(t.u, cot + c0, (size_t)Wn * 8, udev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (int e = grad_chunk<R>(s, net, t, rc, t.u, Wn, gd, st)) return e;
  }
  // ablation variants: a removed head is not part of the model
  const NetOff& o = sys->off;
  if (sys->no_jastrow) PN_CUDA(cudaMemsetAsync(gd + o.eW[0], 0, (size_t)(o.eb[2] + 1 - o.eW[0]) * 8, st));
  if (sys->no_backflow)
    PN_CUDA(cudaMemsetAsync(gd + o.kW[0], 0, (size_t)(o.kb[2] + s.n_orb - o.kW[0]) * 8, st));
  if (!gdev) {
    PN_CUDA(cudaMemcpyAsync(grad, gd, (size_t)sys->off.total * 8, cudaMemcpyDeviceToHost, st));
    PN_CUDA(cudaFreeAsync(gd, st));
  }
  if (rstage) PN_CUDA(cudaFreeAsync(rstage, st));
  if (!rdev || !udev || !gdev) PN_CUDA(cudaStreamSynchronize(st));
  return PN_OK;
}

template <typename R>
int pn_drift_reverse(pn_system_s* sys, const double* r, int Wn, double* logabs, double* grad, cudaStream_t st) {
  if (Wn <= 0) return PN_OK;
  const DevSys& s = sys->ds;
  // the tape is sized for a whole workspace chunk so that it is carved once
  const int Wb = std::max(Wn, sys->Wc);
  const size_t bytes = tape_bytes_per_walker<R>(s) * (size_t)Wb + 4096 * 64 + 65536;
  if (int e = ensure_tape(sys, bytes)) return e;
  Tape<R> t = carve_tape<R>(s, Wb, sys->tape_mem, 0);
  if (t.end > (char*)sys->tape_mem + sys->tape_bytes) {
    pn_set_error("drift: tape layout (%zu bytes) exceeds its allocation (%zu)", (size_t)(t.end - (char*)sys->tape_mem),
                 sys->tape_bytes);
    return PN_EINVAL;
  }
  return drift_chunk<R>(s, pn_devnet<R>(sys), t, r, Wn, logabs, grad, st);
}
template int pn_drift_reverse<double>(pn_system_s*, const double*, int, double*, double*, cudaStream_t);
template int pn_drift_reverse<float>(pn_system_s*, const double*, int, double*, double*, cudaStream_t);

extern "C" int pn_grad_logpsi(pn_system_t s, const double* r, int W, const double* cot, double* grad, size_t budget,
                              void* stream) {
  if (!s || W < 0 || !grad || (W > 0 && (!r || !cot))) { pn_set_error("bad arguments"); return PN_EINVAL; }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != s->device) PN_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (W == 0) {
    PN_CUDA(cudaMemsetAsync(grad, 0, (size_t)s->off.total * 8, st));
    return PN_OK;
  }
  return s->precision == PN_FP64 ? grad_impl<double>(s, r, W, cot, grad, budget, st)
                                 : grad_impl<float>(s, r, W, cot, grad, budget, st);
}
