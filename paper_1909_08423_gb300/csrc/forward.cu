// Forward pass of the ansatz over a chunk of walkers, in value mode (T = 1)
// or jet mode (T = 3N + 2 rows: value, d/dr_{k,a} for every coordinate,
// Laplacian).  The network runs in R (double or float); orbitals,
// geometry, determinants and the final combination run in double.
//
// Jet row index t: 0 value, 1 + 3k + a derivative along coordinate a of
// electron k, 3N + 1 Laplacian (sum over all 3N second derivatives).
#include <math.h>

#include <algorithm>

#include "ansatz_dev.cuh"
#include "slater_dev.cuh"
#include "kernels.cuh"
#include "pn_internal.cuh"

namespace pnk {

// ------------------------------------------------------------ geometry
// geo[w][p] = (d, unit vector).  Electron pairs a<b store (r_a - r_b)/d,
// electron-nucleus pairs (i, I) store (r_i - R_I)/d.
__global__ void k_geometry(DevSys s, const double* __restrict__ r, int Wn, double* __restrict__ geo) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Wn * s.Ppair) return;
  int w = idx / s.Ppair, p = idx - w * s.Ppair;
  const double* rw = r + (size_t)w * s.N * 3;
  double v[3];
  if (p < s.Pee) {
    int a = 0, rem = p;
    while (rem >= s.N - 1 - a) { rem -= s.N - 1 - a; ++a; }
    int b = a + 1 + rem;
    for (int x = 0; x < 3; ++x) v[x] = rw[3 * a + x] - rw[3 * b + x];
  } else {
    int q = p - s.Pee, i = q / s.M, I = q - i * s.M;
    for (int x = 0; x < 3; ++x) v[x] = rw[3 * i + x] - s.R[3 * I + x];
  }
  double d = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double inv = 1.0 / d;
  double* g = geo + (size_t)idx * 4;
  g[0] = d;
  g[1] = v[0] * inv;
  g[2] = v[1] * inv;
  g[3] = v[2] * inv;
}

// ------------------------------------------------------------- orbitals
// phi[w][i][mu][0..4] = value, gradient (3), Laplacian of the cusp-spliced
// molecular orbital mu at electron i (one thread per electron).
// JET = false: the values only (component 0 of each 5-slot record), for
// value passes that need no derivatives.
template <bool JET>
__global__ void k_orbitals(DevSys s, const double* __restrict__ r, int Wn, double* __restrict__ phi) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Wn * s.N) return;
  constexpr int Q = JET ? 5 : 1;
  double acc[PN_MAX_ORBITALS * Q];
  pn_orbitals_at<JET>(s, r + (size_t)idx * 3, acc);
  const int no = s.n_orb;
  double* o = phi + (size_t)idx * no * 5;
  if (JET)
    for (int k = 0; k < no * 5; ++k) o[k] = acc[k];
  else
    for (int k = 0; k < no; ++k) o[5 * k] = acc[k];
}

// ------------------------------------------------------------- features
// e_k(d) = d^2 exp(-d - (d - mu_k)^2 / sigma_k^2) and its first two
// derivatives in d, for every pair: efeat[w][p][c][k], c = value, d/dd, d2/dd2.
// Evaluated in the network's precision R: a float32 network consumes float32
// features, and float64 exponentials run at a small fraction of the float32
// rate on this GPU.
template <typename R>
__global__ void k_features(DevSys s, const double* __restrict__ geo, int Wn, int jet, R* __restrict__ ef) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)Wn * s.Ppair * s.K;
  if (idx >= total) return;
  const int k = idx % s.K;
  const size_t wp = idx / s.K;
  const R d = (R)geo[wp * 4];
  const R mu = sizeof(R) == 4 ? (R)s.feat_mu32[k] : (R)s.feat_mu[k];
  const R is2 = sizeof(R) == 4 ? (R)s.feat_isig2_32[k] : (R)s.feat_isig2[k];
  const R E = exp(-d - (d - mu) * (d - mu) * is2);
  R* o = ef + wp * 3 * s.K;
  o[k] = d * d * E;
  if (jet) {
    const R q = R(-1) - R(2) * (d - mu) * is2;  // derivative of the exponent
    o[s.K + k] = E * (R(2) * d + d * d * q);
    o[2 * s.K + k] = E * (R(2) + R(4) * d * q + d * d * (q * q - R(2) * is2));
  }
}

template <typename R>
__device__ inline R ssp_(R x) {
  return (x > R(0) ? x : R(0)) + log1p(exp(-fabs(x))) - R(0.69314718055994530942);
}
template <typename R>
__device__ inline R sigm_(R x) { return R(1) / (R(1) + exp(-x)); }

// ------------------------------------------------------------- filters
// (sh, sl) += (ah + al)(bh + bl) in float32-pair arithmetic: the product's
// rounding error by an FMA, the sum's by an error-free two-sum (explicit
// roundings, so that no contraction merges the steps).
__device__ inline void f32x2_mac(float& sh, float& sl, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float pe = fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p)));
  const float t = __fadd_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sl = __fadd_rn(sl, __fadd_rn(er, pe));
  sh = t;
}
// x = hi + lo to about 48 bits.  For the usual magnitudes by integer work
// on the bits alone (hi: the sign, exponent and leading 23 stored mantissa
// bits; lo: the remaining 29 bits, rounded to a float and scaled), since
// float64 arithmetic issues at 1/64 of the float32 rate on this part; zero,
// tiny, huge and non-finite values take the float64 route.
__device__ inline float2 f32x2_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hiw = (unsigned)(u >> 32), sign = hiw & 0x80000000u;
  if ((u << 1) == 0ull) return make_float2(__uint_as_float(sign), 0.f);
  const int e = (int)((hiw >> 20) & 0x7FFu);
  if (e < 949 || e > 1150) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
  }
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
  const float lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull)) * __uint_as_float((unsigned)(e - 948) << 23);
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) ^ sign));
}

// One pair row of the float64 filter net (the guard's re-evaluation) with
// its dot products in float32-pair arithmetic on the (hi, lo) weight copy;
// biases, activations and outputs in float64.  e2 and h2 are the warp's
// shared rows (3 K and 3 Hw pairs).
__device__ inline void pn_filter_row_f32x2(const DevSys& s, const DevNet<double>& net, int n, int ch,
                                           const double* __restrict__ e, int nc, int lane, float2* e2, float2* h2,
                                           double* __restrict__ o) {
  const int K = s.K, Hw = s.Hw, Zd = s.Zd;
  for (int k = lane; k < K; k += 32)
    for (int c = 0; c < nc; ++c) e2[c * K + k] = f32x2_split(e[c * K + k]);
  __syncwarp();
  const float2* W1 = (const float2*)net.p2 + net.off.W1[n][ch];
  const float2* W2 = (const float2*)net.p2 + net.off.W2[n][ch];
  const double* b1 = net.p + net.off.b1[n][ch];
  const double* b2 = net.p + net.off.b2[n][ch];
  for (int h = lane; h < Hw; h += 32) {
    const float2 bb = f32x2_split(b1[h]);
    float a0h = bb.x, a0l = bb.y, a1h = 0.f, a1l = 0.f, a2h = 0.f, a2l = 0.f;
    for (int k = 0; k < K; ++k) {
      const float2 wv = W1[k * Hw + h];
      f32x2_mac(a0h, a0l, e2[k], wv);
      if (nc == 3) {
        f32x2_mac(a1h, a1l, e2[K + k], wv);
        f32x2_mac(a2h, a2l, e2[2 * K + k], wv);
      }
    }
    const double a0 = (double)a0h + (double)a0l;
    const double sg = sigm_(a0);
    h2[h] = f32x2_split(ssp_(a0));
    if (nc == 3) {
      const double a1 = (double)a1h + (double)a1l, a2 = (double)a2h + (double)a2l;
      h2[Hw + h] = f32x2_split(sg * a1);
      h2[2 * Hw + h] = f32x2_split(sg * a2 + sg * (1.0 - sg) * a1 * a1);
    }
  }
  __syncwarp();
  for (int z = lane; z < Zd; z += 32) {
    const float2 bb = f32x2_split(b2[z]);
    float o0h = bb.x, o0l = bb.y, o1h = 0.f, o1l = 0.f, o2h = 0.f, o2l = 0.f;
    for (int h = 0; h < Hw; ++h) {
      const float2 wv = W2[h * Zd + z];
      f32x2_mac(o0h, o0l, h2[h], wv);
      if (nc == 3) {
        f32x2_mac(o1h, o1l, h2[Hw + h], wv);
        f32x2_mac(o2h, o2l, h2[2 * Hw + h], wv);
      }
    }
    o[z] = (double)o0h + (double)o0l;
    if (nc == 3) {
      o[Zd + z] = (double)o1h + (double)o1l;
      o[2 * Zd + z] = (double)o2h + (double)o2l;
    }
  }
}

// w^{(n,c)}(e) = W2 ssp(W1 e + b1) + b2 for every pair, carrying the jet in
// the scalar distance (value, d/dd, d2/dd2).  One warp per pair row.
// Channel: same-spin electron pair 0, opposite spin 1, electron-nucleus 2.
constexpr int FW = 8;  // warps per block

template <typename R>
__global__ void __launch_bounds__(FW * 32) k_filter(DevSys s, DevNet<R> net, int n, const R* __restrict__ ef,
                                                    int Wn, int jet, R* __restrict__ wj) {
  __shared__ R sh_e[FW][3 * 64];
  __shared__ R sh_h[FW][3 * 128];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t row = (size_t)blockIdx.x * FW + wid;
  if (row >= (size_t)Wn * s.Ppair) return;
  const int p = row % s.Ppair;
  int ch;
  if (p >= s.Pee) ch = 2;
  else {
    int a = 0, rem = p;
    while (rem >= s.N - 1 - a) { rem -= s.N - 1 - a; ++a; }
    int b = a + 1 + rem;
    ch = ((a < s.n_up) == (b < s.n_up)) ? 0 : 1;
  }
  const int K = s.K, Hw = s.Hw, Zd = s.Zd;
  const int nc = jet ? 3 : 1;
  const R* e = ef + row * 3 * K;
  if constexpr (sizeof(R) == 8) {
    if (s.lin_f32x2 && net.p2) {
      pn_filter_row_f32x2(s, net, n, ch, (const double*)e, nc, lane, (float2*)sh_e[wid], (float2*)sh_h[wid],
                          (double*)(wj + row * 3 * Zd));
      return;
    }
  }
  for (int k = lane; k < K; k += 32)
    for (int c = 0; c < nc; ++c) sh_e[wid][c * K + k] = e[c * K + k];
  __syncwarp();
  const R* W1 = net.p + net.off.W1[n][ch];
  const R* b1 = net.p + net.off.b1[n][ch];
  const R* W2 = net.p + net.off.W2[n][ch];
  const R* b2 = net.p + net.off.b2[n][ch];
  for (int h = lane; h < Hw; h += 32) {
    R a0 = b1[h], a1 = 0, a2 = 0;
    for (int k = 0; k < K; ++k) {
      const R wv = W1[k * Hw + h];
      a0 += sh_e[wid][k] * wv;
      if (jet) {
        a1 += sh_e[wid][K + k] * wv;
        a2 += sh_e[wid][2 * K + k] * wv;
      }
    }
    const R sg = sigm_(a0);
    sh_h[wid][h] = ssp_(a0);
    if (jet) {
      sh_h[wid][Hw + h] = sg * a1;
      sh_h[wid][2 * Hw + h] = sg * a2 + sg * (R(1) - sg) * a1 * a1;
    }
  }
  __syncwarp();
  R* o = wj + row * 3 * Zd;
  for (int z = lane; z < Zd; z += 32) {
    R o0 = b2[z], o1 = 0, o2 = 0;
    for (int h = 0; h < Hw; ++h) {
      const R wv = W2[h * Zd + z];
      o0 += sh_h[wid][h] * wv;
      if (jet) {
        o1 += sh_h[wid][Hw + h] * wv;
        o2 += sh_h[wid][2 * Hw + h] * wv;
      }
    }
    o[z] = o0;
    if (jet) {
      o[Zd + z] = o1;
      o[2 * Zd + z] = o2;
    }
  }
}

// --------------------------------------------------------------- linear
// Y[rows][Nout] (+)= X[rows][Kd] W[Kd][Nout] + b on value rows (row % T == 0).
// 64x64 output tile, 16-deep k tiles, 4x4 outputs per thread.
template <typename R>
__global__ void __launch_bounds__(256) k_linear(const R* __restrict__ X, int ldx, const R* __restrict__ Wt, int ldw,
                                                const R* __restrict__ bias, R* __restrict__ Y, int ldy, int rows,
                                                int Kd, int Nout, int T, int accumulate) {
  __shared__ R As[16][64 + 1];
  __shared__ R Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;  // row tiles in x: no 65535 limit
  R acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < Kd; k0 += 16) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = threadIdx.x + l * 256;
      const int rr = e >> 4, kk = e & 15;
      const int gr = row0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < rows && gk < Kd) ? X[(size_t)gr * ldx + gk] : R(0);
      const int kb = e >> 6, cb = e & 63;
      const int gkb = k0 + kb, gc = col0 + cb;
      Bs[kb][cb] = (gkb < Kd && gc < Nout) ? Wt[(size_t)gkb * ldw + gc] : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      R a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + ty * 4 + i;
    if (gr >= rows) continue;
    const bool val = (gr % T) == 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc >= Nout) continue;
      R v = acc[i][j] + ((bias && val) ? bias[gc] : R(0));
      R* y = Y + (size_t)gr * ldy + gc;
      *y = accumulate ? *y + v : v;
    }
  }
}

// Float64 Y (+)= X W + b with float32-pair arithmetic: every operand split
// into hi + lo floats (f32x2_split), each product formed as ah bh exactly (its rounding error by an
// FMA) plus ah bl + al bh, and the products summed in a (sum, correction)
// pair with an error-free two-sum.  That keeps about 44 bits of the
// float64 result (about 1e-13 of sum |x w|) at float32 issue rates, which
// on this part run 64 times the float64 rate.  Same tiling as k_linear.
__global__ void __launch_bounds__(256) k_linear_f32x2(const double* __restrict__ X, int ldx,
                                                      const double* __restrict__ Wt, int ldw,
                                                      const double* __restrict__ bias, double* __restrict__ Y,
                                                      int ldy, int rows, int Kd, int Nout, int T, int accumulate) {
  __shared__ float Ah[16][64 + 1], Al[16][64 + 1];
  __shared__ float Bh[16][64], Bl[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
  for (int k0 = 0; k0 < Kd; k0 += 16) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = threadIdx.x + l * 256;
      const int rr = e >> 4, kk = e & 15;
      const int gr = row0 + rr, gk = k0 + kk;
      const float2 a = f32x2_split((gr < rows && gk < Kd) ? X[(size_t)gr * ldx + gk] : 0.0);
      Ah[kk][rr] = a.x;
      Al[kk][rr] = a.y;
      const int kb = e >> 6, cb = e & 63;
      const int gkb = k0 + kb, gc = col0 + cb;
      const float2 b = f32x2_split((gkb < Kd && gc < Nout) ? Wt[(size_t)gkb * ldw + gc] : 0.0);
      Bh[kb][cb] = b.x;
      Bl[kb][cb] = b.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Ah[kk][ty * 4 + i];
        al[i] = Al[kk][ty * 4 + i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bh[j] = Bh[kk][tx * 4 + j];
        bl[j] = Bl[kk][tx * 4 + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // explicit roundings: no contraction may merge the product
          // into the two-sum
          const float p = __fmul_rn(ah[i], bh[j]);
          const float pe = fmaf(ah[i], bl[j], fmaf(al[i], bh[j], fmaf(ah[i], bh[j], -p)));
          const float t = __fadd_rn(sh[i][j], p);
          const float z = __fsub_rn(t, sh[i][j]);
          const float e = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));
          sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(e, pe));
          sh[i][j] = t;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + ty * 4 + i;
    if (gr >= rows) continue;
    const bool val = (gr % T) == 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc >= Nout) continue;
      const double v = ((double)sh[i][j] + (double)sl[i][j]) + ((bias && val) ? bias[gc] : 0.0);
      double* y = Y + (size_t)gr * ldy + gc;
      *y = accumulate ? *y + v : v;
    }
  }
}

// Float32 Y (+)= X W + b (bias on value rows only): BM x BN output tiles,
// 8 x TN outputs per thread -- 256 x 32 (TN 4) for maps at most 32 wide so
// that no half-empty tiles are computed, 128 x 64 (TN 4) up to 64, 128 x 128
// (TN 8, the thread's columns in two float4 groups 64 apart) beyond.  16-deep
// k slices are double-buffered in shared memory: the next slice's global
// loads are issued before the current slice's multiply-adds and stored
// after them, one barrier per slice.  Requires ldx and Kd multiples of 4 and
// a 16-byte aligned X (the caller checks).  VEC_W: float4 loads of W (ldw,
// Nout multiples of 4, W aligned), else element loads; VEC_Y: float4 stores
// of Y (ldy, Nout multiples of 4, Y aligned), else element stores.  TB:
// the weight is stored transposed, W[n][k] with row stride ldw (Y = X W^T,
// the backward's maps); its float4 loads then run along k.
template <int BM, int BN, int TN, bool VEC_W, bool VEC_Y, bool TB = false>
__global__ void __launch_bounds__(256, TN == 8 ? 2 : 3)
    k_linear_v4(const float* __restrict__ X, int ldx, const float* __restrict__ W, int ldw,
                const float* __restrict__ bias, float* __restrict__ Y, int ldy, int rows, int Kd, int Nout, int T,
                int accumulate) {
  static_assert((BM / 8) * (BN / TN) == 256 && (TN == 4 || TN == 8), "256 threads x 8 x TN outputs");
  constexpr int TX = BN / TN;            // threads across the columns
  constexpr int CG = TN / 4;             // float4 column groups per thread
  constexpr int CS = BN / CG;            // distance between a thread's column groups
  constexpr int AL = BM / 64;            // float4 loads of an A slice per thread
  constexpr int BL = (4 * BN + 255) / 256;  // float4 loads of a B slice per thread
  constexpr int BS = 16 * BN / 256;      // element loads of a B slice per thread
  __shared__ __align__(16) float As[2][16][BM + 4];
  __shared__ __align__(16) float Bs[2][16][BN];
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;  // row tiles in x: no 65535 limit
  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  float4 ra[AL];
  float4 rb4[BL];
  float rbs[BS > 0 ? BS : 1];
  auto load = [&](int k0) {
#pragma unroll
    for (int l = 0; l < AL; ++l) {
      const int e = tid + l * 256;
      const int gr = row0 + (e >> 2), gk = k0 + (e & 3) * 4;
      ra[l] = (gr < rows && gk < Kd) ? *(const float4*)(X + (size_t)gr * ldx + gk) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (TB && VEC_W) {  // float4 along k of row n of W
#pragma unroll
      for (int l = 0; l < BL; ++l) {
        const int e = tid + l * 256;
        if (e < 4 * BN) {
          const int gc = col0 + (e >> 2), gk = k0 + (e & 3) * 4;
          rb4[l] = (gk < Kd && gc < Nout) ? *(const float4*)(W + (size_t)gc * ldw + gk)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else if constexpr (TB) {
#pragma unroll
      for (int l = 0; l < BS; ++l) {
        const int e = tid + l * 256;
        const int gk = k0 + (e & 15), gc = col0 + (e >> 4);
        rbs[l] = (gk < Kd && gc < Nout) ? W[(size_t)gc * ldw + gk] : 0.f;
      }
    } else if constexpr (VEC_W) {
#pragma unroll
      for (int l = 0; l < BL; ++l) {
        const int e = tid + l * 256;
        if (e < 4 * BN) {
          const int gk = k0 + e / (BN / 4), gc = col0 + (e % (BN / 4)) * 4;
          rb4[l] = (gk < Kd && gc < Nout) ? *(const float4*)(W + (size_t)gk * ldw + gc)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else {
#pragma unroll
      for (int l = 0; l < BS; ++l) {
        const int e = tid + l * 256;
        const int gk = k0 + e / BN, gc = col0 + e % BN;
        rbs[l] = (gk < Kd && gc < Nout) ? W[(size_t)gk * ldw + gc] : 0.f;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int l = 0; l < AL; ++l) {
      const int e = tid + l * 256;
      const int rr = e >> 2, k4 = (e & 3) * 4;
      As[buf][k4][rr] = ra[l].x;
      As[buf][k4 + 1][rr] = ra[l].y;
      As[buf][k4 + 2][rr] = ra[l].z;
      As[buf][k4 + 3][rr] = ra[l].w;
    }
    if constexpr (TB && VEC_W) {
#pragma unroll
      for (int l = 0; l < BL; ++l) {
        const int e = tid + l * 256;
        if (e < 4 * BN) {
          const int n = e >> 2, k4 = (e & 3) * 4;
          Bs[buf][k4][n] = rb4[l].x;
          Bs[buf][k4 + 1][n] = rb4[l].y;
          Bs[buf][k4 + 2][n] = rb4[l].z;
          Bs[buf][k4 + 3][n] = rb4[l].w;
        }
      }
    } else if constexpr (TB) {
#pragma unroll
      for (int l = 0; l < BS; ++l) {
        const int e = tid + l * 256;
        Bs[buf][e & 15][e >> 4] = rbs[l];
      }
    } else if constexpr (VEC_W) {
#pragma unroll
      for (int l = 0; l < BL; ++l) {
        const int e = tid + l * 256;
        if (e < 4 * BN) *(float4*)&Bs[buf][e / (BN / 4)][(e % (BN / 4)) * 4] = rb4[l];
      }
    } else {
#pragma unroll
      for (int l = 0; l < BS; ++l) {
        const int e = tid + l * 256;
        Bs[buf][e / BN][e % BN] = rbs[l];
      }
    }
  };
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    const bool more = k0 + 16 < Kd;
    if (more) load(k0 + 16);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a0 = *(const float4*)&As[buf][kk][ty * 8], a1 = *(const float4*)&As[buf][kk][ty * 8 + 4];
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bb[TN];
#pragma unroll
      for (int g = 0; g < CG; ++g) {
        const float4 b = *(const float4*)&Bs[buf][kk][g * CS + tx * 4];
        bb[4 * g] = b.x;
        bb[4 * g + 1] = b.y;
        bb[4 * g + 2] = b.z;
        bb[4 * g + 3] = b.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int g = 0; g < CG; ++g) {
    const int gc = col0 + g * CS + tx * 4;
    if (gc >= Nout) continue;
    float bv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = (bias && gc + j < Nout) ? bias[gc + j] : 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gr = row0 + ty * 8 + i;
      if (gr >= rows) break;
      const bool val = (gr % T) == 0;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = acc[i][4 * g + j] + (val ? bv[j] : 0.f);
      float* y = Y + (size_t)gr * ldy + gc;
      if constexpr (VEC_Y) {
        if (accumulate) {
          const float4 o = *(const float4*)y;
          v[0] += o.x;
          v[1] += o.y;
          v[2] += o.z;
          v[3] += o.w;
        }
        *(float4*)y = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (gc + j < Nout) y[j] = accumulate ? y[j] + v[j] : v[j];
      }
    }
  }
}

// h0 = x^(0) W_h + b_h of the first layer: one row, the same for every
// electron of every walker.
template <typename R>
__global__ void k_h0_row(const R* __restrict__ x0, const R* __restrict__ W, const R* __restrict__ b, int D, int Zd,
                         R* __restrict__ h0) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= Zd) return;
  R acc = b[z];
  for (int d = 0; d < D; ++d) acc += x0[d] * W[(size_t)d * Zd + z];
  h0[z] = acc;
}

// x^(0): the shared electron embedding on value rows, zero derivatives.
template <typename R>
__global__ void k_init_x(const R* __restrict__ x0, R* __restrict__ X, size_t groups, int T, int D) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= groups * T * D) return;
  const int d = idx % D;
  const int t = (idx / D) % T;
  X[idx] = t == 0 ? x0[d] : R(0);
}

// ------------------------------------------------------------- messages
// z_i^{same|anti} = sum_j w_ij * h_j, z_i^nuc = sum_I w_iI * Y_I with the
// product rule through the jet.  Zb[w][i][t][c*Zd + z].
template <typename R>
__global__ void __launch_bounds__(256) k_message(DevSys s, const R* __restrict__ Y, const double* __restrict__ geo,
                                                 const R* __restrict__ wj, const R* __restrict__ H, int ldH, int Wn,
                                                 int T, R* __restrict__ Zb, int ldZ) {
  // one block per (walker, electron i); the geometry of i's partners
  // (electrons j != i, then nuclei) is read once and kept in R as
  // (d, 1/d, unit vector from the partner to i)
  extern __shared__ __align__(16) unsigned char msg_smem[];
  R* gsh = (R*)msg_smem;
  const int Zd = s.Zd, N = s.N, M = s.M;
  const int w = blockIdx.x / N, i = blockIdx.x % N;
  const int npart = N - 1 + M;
  for (int k = threadIdx.x; k < npart; k += blockDim.x) {
    int p;
    double sgn = 1.0;
    if (k < N - 1) {
      const int j = k < i ? k : k + 1;
      if (i < j) p = pn_pair_index(i, j, N);
      else { p = pn_pair_index(j, i, N); sgn = -1.0; }
    } else {
      p = s.Pee + i * M + (k - (N - 1));
    }
    const double* g = geo + ((size_t)w * s.Ppair + p) * 4;
    R* o = gsh + k * 5;
    o[0] = (R)g[0];
    o[1] = (R)(1.0 / g[0]);
    o[2] = (R)(sgn * g[1]);
    o[3] = (R)(sgn * g[2]);
    o[4] = (R)(sgn * g[3]);
  }
  __syncthreads();
  const int lap = T - 1;
  const bool si = i < s.n_up;
  const R* Hw_ = H + (size_t)w * N * T * ldH;
  const R* ww = wj + (size_t)w * s.Ppair * 3 * Zd;
  R* ob = Zb + (size_t)(w * N + i) * T * ldZ;
  for (int q = threadIdx.x; q < T * Zd; q += blockDim.x) {
    const int t = q / Zd, z = q % Zd;
    int tk = -1, ta = 0;
    if (t > 0 && t < lap) { tk = (t - 1) / 3; ta = (t - 1) % 3; }
    R zs = 0, za = 0, zn = 0;
    for (int k = 0; k < N - 1; ++k) {
      const int j = k < i ? k : k + 1;
      const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
      const R* gk = gsh + k * 5;
      const R w0 = ww[(size_t)p * 3 * Zd + z];
      const R* hj = Hw_ + (size_t)j * T * ldH;
      const R h0 = hj[z];
      R v;
      if (t == 0) {
        v = w0 * h0;
      } else if (t < lap) {
        const R w1 = ww[(size_t)p * 3 * Zd + Zd + z];
        const R u = gk[2 + ta];
        const R dd = (tk == i) ? u : ((tk == j) ? -u : R(0));
        v = w1 * dd * h0 + w0 * hj[(size_t)t * ldH + z];
      } else {
        const R w1 = ww[(size_t)p * 3 * Zd + Zd + z];
        const R w2 = ww[(size_t)p * 3 * Zd + 2 * Zd + z];
        R cross = 0;
        for (int a = 0; a < 3; ++a)
          cross += gk[2 + a] * (hj[(size_t)(1 + 3 * i + a) * ldH + z] - hj[(size_t)(1 + 3 * j + a) * ldH + z]);
        v = (R(2) * w2 + R(4) * w1 * gk[1]) * h0 + w0 * hj[(size_t)lap * ldH + z] + R(2) * w1 * cross;
      }
      if ((j < s.n_up) == si) zs += v; else za += v;
    }
    for (int I = 0; I < M; ++I) {
      const int p = s.Pee + i * M + I;
      const R* gk = gsh + (N - 1 + I) * 5;
      const R y = Y[I * Zd + z];
      const R* wp = ww + (size_t)p * 3 * Zd;
      if (t == 0) zn += wp[z] * y;
      else if (t < lap) {
        if (tk == i) zn += wp[Zd + z] * gk[2 + ta] * y;
      } else {
        zn += (wp[2 * Zd + z] + R(2) * wp[Zd + z] * gk[1]) * y;
      }
    }
    R* o = ob + (size_t)t * ldZ;
    o[z] = zs;
    o[Zd + z] = za;
    o[2 * Zd + z] = zn;
  }
}

// Same messages, one thread per (walker, row chunk, electron i, column z):
// chunk c < ceil(N/KC) holds the tangent rows of electrons KC c .. KC c +
// KC - 1 (t = 1 + 3k + a), the last chunk the value row and the Laplacian
// row.
// Each partner's filter jet, geometry and value row are read once per
// chunk, and the product-rule factor d d_ij / d r_{k,a} is resolved per
// electron k, so a row costs one h load and two multiply-adds per partner.
// Arithmetic per row is that of k_message.
// HC: the first layer, whose h is one row h0 = H[0 .. Zd) shared by every
// electron with no tangent or Laplacian (x^(0) is the same constant for all
// electrons), so that its h GEMM and the x^(0) jet need not exist.
constexpr int MSG_KC = 2;  // electrons per tangent-row chunk of k_message_c
template <typename R, bool HC>
__global__ void __launch_bounds__(256) k_message_c(DevSys s, const R* __restrict__ Y, const double* __restrict__ geo,
                                                   const R* __restrict__ wj, const R* __restrict__ H, int ldH, int Wn,
                                                   int T, R* __restrict__ Zb, int ldZ) {
  constexpr int KC = MSG_KC;
  const int Zd = s.Zd, N = s.N, M = s.M;
  const int nTan = (N + KC - 1) / KC, nC = nTan + 1;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Wn * nC * N * Zd) return;
  const int z = idx % Zd;
  const int i = (idx / Zd) % N;
  const int c = (idx / ((size_t)Zd * N)) % nC;
  const int w = idx / ((size_t)Zd * N * nC);
  const int lap = T - 1;
  const bool si = i < s.n_up;
  const R* Hw_ = HC ? H + z : H + (size_t)w * N * T * ldH + z;
  const R* ww = wj + (size_t)w * s.Ppair * 3 * Zd + z;
  const double* gw = geo + (size_t)w * s.Ppair * 4;
  R* ob = Zb + (size_t)(w * N + i) * T * ldZ + z;
  if (c < nTan) {
    const int k0 = KC * c, nk = min(KC, N - k0);
    R zs[3 * KC], za[3 * KC], zq[3 * KC];
#pragma unroll
    for (int q = 0; q < 3 * KC; ++q) zs[q] = za[q] = zq[q] = 0;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
      const double* g = gw + p * 4;
      const R sg = i < j ? R(1) : R(-1);  // unit vector from j to i
      const R u[3] = {sg * (R)g[1], sg * (R)g[2], sg * (R)g[3]};
      const R w0 = ww[(size_t)p * 3 * Zd], w1 = ww[(size_t)p * 3 * Zd + Zd];
      const R* hj = HC ? Hw_ : Hw_ + (size_t)j * T * ldH;
      const R h0 = hj[0];
      const bool same = (j < s.n_up) == si;
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        if (kk >= nk) break;
        const int k = k0 + kk;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const R dd = (k == i) ? u[a] : ((k == j) ? -u[a] : R(0));
          const R v = HC ? w1 * dd * h0 : w1 * dd * h0 + w0 * hj[(size_t)(1 + 3 * k + a) * ldH];
          if (same) zs[3 * kk + a] += v; else za[3 * kk + a] += v;
        }
      }
    }
    // nuclei move no electron but i: their terms sit in i's rows only
    if (i >= k0 && i < k0 + nk)
      for (int I = 0; I < M; ++I) {
        const int p = s.Pee + i * M + I;
        const double* g = gw + p * 4;
        const R y = Y[I * Zd + z];
        const R w1 = ww[(size_t)p * 3 * Zd + Zd];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
          if (kk >= nk) break;
          if (k0 + kk == i)
#pragma unroll
            for (int a = 0; a < 3; ++a) zq[3 * kk + a] += w1 * (R)g[1 + a] * y;
        }
      }
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      if (kk >= nk) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R* o = ob + (size_t)(1 + 3 * (k0 + kk) + a) * ldZ;
        o[0] = zs[3 * kk + a];
        o[Zd] = za[3 * kk + a];
        o[2 * Zd] = zq[3 * kk + a];
      }
    }
    return;
  }
  // value row and Laplacian row
  R vs = 0, va = 0, vq = 0, ls = 0, la = 0, lq = 0;
  for (int j = 0; j < N; ++j) {
    if (j == i) continue;
    const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
    const double* g = gw + p * 4;
    const R sg = i < j ? R(1) : R(-1);
    const R id = R(1) / (R)g[0];
    const R w0 = ww[(size_t)p * 3 * Zd], w1 = ww[(size_t)p * 3 * Zd + Zd], w2 = ww[(size_t)p * 3 * Zd + 2 * Zd];
    const R* hj = HC ? Hw_ : Hw_ + (size_t)j * T * ldH;
    const R h0 = hj[0];
    R cross = 0;
    if (!HC)
      for (int a = 0; a < 3; ++a)
        cross += sg * (R)g[1 + a] * (hj[(size_t)(1 + 3 * i + a) * ldH] - hj[(size_t)(1 + 3 * j + a) * ldH]);
    const R v0 = w0 * h0;
    const R vl = HC ? (R(2) * w2 + R(4) * w1 * id) * h0
                    : (R(2) * w2 + R(4) * w1 * id) * h0 + w0 * hj[(size_t)lap * ldH] + R(2) * w1 * cross;
    if ((j < s.n_up) == si) { vs += v0; ls += vl; } else { va += v0; la += vl; }
  }
  for (int I = 0; I < M; ++I) {
    const int p = s.Pee + i * M + I;
    const double* g = gw + p * 4;
    const R y = Y[I * Zd + z];
    const R* wp = ww + (size_t)p * 3 * Zd;
    vq += wp[0] * y;
    lq += (wp[2 * Zd] + R(2) * wp[Zd] * (R(1) / (R)g[0])) * y;
  }
  ob[0] = vs;
  ob[Zd] = va;
  ob[2 * Zd] = vq;
  R* ol = ob + (size_t)lap * ldZ;
  ol[0] = ls;
  ol[Zd] = la;
  ol[2 * Zd] = lq;
}

// Same messages with the walker's operands staged in shared memory: a block
// per (walker, tile of 16 columns z), one half-warp per electron i, its
// lanes over z (16 columns keep a block near 64 KB for the N2 shape, so
// that three blocks share an SM and one block's staging overlaps another's
// arithmetic).  The block first copies the walker's h-jet rows [N][T][16],
// its pair filter jets [P][3][16] and pair geometry (d, 1/d, unit vector);
// each thread then forms all T rows of z_i^same, z_i^anti and z_i^nuc for
// its column from shared memory:
//   value      z_i = sum_j w_ij h_j
//   tangent    z_i[k,a] = sum_j w_ij h_j[k,a] + w'_ij (d d_ij / d r_ka) h_j
//   Laplacian  z_i[lap] = sum_j (2 w''_ij + 4 w'_ij / d_ij) h_j + w_ij h_j[lap]
//                         + 2 w'_ij u_ij . (grad_i h_j - grad_j h_j)
// (electron pairs move with both electrons, so their Laplacian over all
// coordinates is twice the one-electron one; nuclear pairs move with i only).
// Requires Zd a multiple of 16; HC as in k_message_c.
constexpr int MSGW_ZT = 16;
constexpr int MSGW_NMAX = 16;  // electrons of the staged kernel (partner values in registers)
// Double-float numbers (hi + lo floats, about 44 bits) for the float64
// messages of the guard's re-evaluation: float32 issue rates are 64 times
// the float64 rate on this part.  Products by an FMA-exact hi product plus
// the cross terms, sums by a two-sum of the high parts; every result
// renormalised.  Explicit roundings keep contraction out of the steps.
struct FF {
  float hi, lo;
  __device__ FF() {}
  __device__ FF(int x) : hi((float)x), lo(0.f) {}
  __device__ FF(float h, float l) : hi(h), lo(l) {}
};
__device__ inline FF ff_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return FF(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ inline FF operator+(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi), z = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
  return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ inline FF operator-(FF a) { return FF(-a.hi, -a.lo); }
__device__ inline FF operator-(FF a, FF b) { return a + (-b); }
__device__ inline FF operator*(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return ff_norm(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p))));
}
__device__ inline FF& operator+=(FF& a, FF b) { return a = a + b; }

// Conversions between a buffer type R and a compute type C.
template <typename C>
__device__ inline C to_c(double x) { return (C)x; }
template <>
__device__ inline FF to_c<FF>(double x) {
  const float2 p = f32x2_split(x);
  return FF(p.x, p.y);
}
template <typename C>
__device__ inline C to_c(float x) { return (C)x; }
template <typename R>
__device__ inline R from_c(R x) { return x; }
template <typename R>
__device__ inline R from_c(FF x) { return (R)((double)x.hi + (double)x.lo); }

// C: the arithmetic type (R, or FF for float64 buffers in float32-pair
// arithmetic); shared-memory rows hold C.
template <typename R, bool HC, typename C = R>
__global__ void k_message_w(DevSys s, const R* __restrict__ Y, const double* __restrict__ geo,
                            const R* __restrict__ wj, const R* __restrict__ H, int ldH, int Wn, int T,
                            R* __restrict__ Zb, int ldZ) {
  static_assert(sizeof(C) == sizeof(R), "shared rows are sized for R");
  extern __shared__ __align__(16) unsigned char mw_smem[];
  const int N = s.N, M = s.M, Zd = s.Zd, P = s.Ppair, lap = T - 1;
  const int ntile = Zd / MSGW_ZT;
  const int w = blockIdx.x / ntile, z0 = (blockIdx.x % ntile) * MSGW_ZT;
  const int lane = threadIdx.x & 31, i = ((threadIdx.x >> 5) << 1) | (lane >> 4);
  const int HT = HC ? 1 : T;  // rows of h staged per electron (one shared row for HC)
  const int HN = HC ? 1 : N;
  C* hs = (C*)mw_smem;                       // [HN][HT][16]
  C* ws = hs + (size_t)HN * HT * MSGW_ZT;    // [P][3][16]
  C* gs = ws + (size_t)P * 3 * MSGW_ZT;      // [P][5]: d, 1/d, unit vector
  const int nth = blockDim.x;
  // rows of 16 columns from global memory (row stride ld) into shared
  // memory, eight loads of a thread in flight before its stores
  auto stage = [&](C* dst, const R* src, int n, int ld) {
    for (int q0 = threadIdx.x; q0 < n; q0 += 8 * nth) {
      R v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * nth, row = q / MSGW_ZT, c = q - row * MSGW_ZT;
        v[u] = q < n ? src[(size_t)row * ld + c] : R(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + u * nth < n) dst[q0 + u * nth] = to_c<C>(v[u]);
    }
  };
  if (HC) {
    for (int q = threadIdx.x; q < MSGW_ZT; q += nth) hs[q] = to_c<C>(H[z0 + q]);
  } else {
    stage(hs, H + (size_t)w * N * T * ldH + z0, N * T * MSGW_ZT, ldH);
  }
  stage(ws, wj + (size_t)w * P * 3 * Zd + z0, P * 3 * MSGW_ZT, Zd);
  const double* gw = geo + (size_t)w * P * 4;
  for (int p = threadIdx.x; p < P; p += nth) {
    const double d = gw[4 * p];
    gs[5 * p] = to_c<C>(d);
    gs[5 * p + 1] = to_c<C>(1.0 / d);
    gs[5 * p + 2] = to_c<C>(gw[4 * p + 1]);
    gs[5 * p + 3] = to_c<C>(gw[4 * p + 2]);
    gs[5 * p + 4] = to_c<C>(gw[4 * p + 3]);
  }
  __syncthreads();
  if (i >= N) return;
  const int z = lane & (MSGW_ZT - 1);
  const bool si = i < s.n_up;
  auto hrow = [&](int j, int t) -> C { return HC ? (t == 0 ? hs[z] : C(0)) : hs[((size_t)j * T + t) * MSGW_ZT + z]; };
  auto pidx = [&](int j) { return i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N); };
  R* ob = Zb + (size_t)(w * N + i) * T * ldZ + z0 + z;
  // per-thread sums that the tangent rows of electron i itself reuse
  C s1s[3] = {C(0), C(0), C(0)}, s1a[3] = {C(0), C(0), C(0)}, n1[3] = {C(0), C(0), C(0)};
  C vs = C(0), va = C(0), vn = C(0), ls = C(0), la = C(0), ln = C(0);
  for (int j = 0; j < N; ++j) {
    if (j == i) continue;
    const int p = pidx(j);
    const C sg = i < j ? C(1) : C(-1);  // unit vector from j to i
    const C* g = gs + 5 * p;
    const C w0 = ws[(3 * p) * MSGW_ZT + z], w1 = ws[(3 * p + 1) * MSGW_ZT + z], w2 = ws[(3 * p + 2) * MSGW_ZT + z];
    const C h0 = hrow(j, 0);
    const bool same = (j < s.n_up) == si;
    C cross = C(0);
    if (!HC)
#pragma unroll
      for (int a = 0; a < 3; ++a) cross += sg * g[2 + a] * (hrow(j, 1 + 3 * i + a) - hrow(j, 1 + 3 * j + a));
    const C v0 = w0 * h0;
    const C vl = HC ? (C(2) * w2 + C(4) * w1 * g[1]) * h0
                    : (C(2) * w2 + C(4) * w1 * g[1]) * h0 + w0 * hrow(j, lap) + C(2) * w1 * cross;
    if (same) {
      vs += v0;
      ls += vl;
#pragma unroll
      for (int a = 0; a < 3; ++a) s1s[a] += w1 * sg * g[2 + a] * h0;
    } else {
      va += v0;
      la += vl;
#pragma unroll
      for (int a = 0; a < 3; ++a) s1a[a] += w1 * sg * g[2 + a] * h0;
    }
  }
  for (int I = 0; I < M; ++I) {
    const int p = s.Pee + i * M + I;
    const C* g = gs + 5 * p;
    const C y = to_c<C>(Y[I * Zd + z0 + z]);
    const C w0 = ws[(3 * p) * MSGW_ZT + z], w1 = ws[(3 * p + 1) * MSGW_ZT + z], w2 = ws[(3 * p + 2) * MSGW_ZT + z];
    vn += w0 * y;
    ln += (w2 + C(2) * w1 * g[1]) * y;
#pragma unroll
    for (int a = 0; a < 3; ++a) n1[a] += w1 * g[2 + a] * y;
  }
  ob[0] = from_c<R>(vs);
  ob[Zd] = from_c<R>(va);
  ob[2 * Zd] = from_c<R>(vn);
  R* ol = ob + (size_t)lap * ldZ;
  ol[0] = from_c<R>(ls);
  ol[Zd] = from_c<R>(la);
  ol[2 * Zd] = from_c<R>(ln);
  // tangent rows t = 1 + 3k + a.  The partners' filter values, split by
  // channel (zero for the other channel and for j = i), sit in registers,
  // so a row costs one shared-memory load and two multiply-adds per partner.
  C w0s[MSGW_NMAX], w0a[MSGW_NMAX];
#pragma unroll
  for (int j = 0; j < MSGW_NMAX; ++j) {
    w0s[j] = w0a[j] = C(0);
    if (!HC && j < N && j != i) {
      const C w0 = ws[(3 * pidx(j)) * MSGW_ZT + z];
      if ((j < s.n_up) == si) w0s[j] = w0; else w0a[j] = w0;
    }
  }
  for (int k = 0; k < N; ++k) {
    // the partner k's own move: d d_ik / d r_ka = -u_ik[a]
    C pk[3] = {C(0), C(0), C(0)};
    bool ksame = true;
    if (k != i) {
      const int p = pidx(k);
      const C sg = i < k ? C(1) : C(-1);
      const C f = -ws[(3 * p + 1) * MSGW_ZT + z] * sg * hrow(k, 0);
#pragma unroll
      for (int a = 0; a < 3; ++a) pk[a] = f * gs[5 * p + 2 + a];
      ksame = (k < s.n_up) == si;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int t = 1 + 3 * k + a;
      C zs = C(0), za = C(0);
      if (!HC) {
        const C* hcol = hs + (size_t)t * MSGW_ZT + z;
#pragma unroll
        for (int j = 0; j < MSGW_NMAX; ++j) {
          if (j < N) {
            const C h = hcol[(size_t)j * T * MSGW_ZT];
            zs += w0s[j] * h;
            za += w0a[j] * h;
          }
        }
      }
      C zq = C(0);
      if (k == i) {
        zs += s1s[a];
        za += s1a[a];
        zq = n1[a];
      } else if (ksame) {
        zs += pk[a];
      } else {
        za += pk[a];
      }
      R* o = ob + (size_t)t * ldZ;
      o[0] = from_c<R>(zs);
      o[Zd] = from_c<R>(za);
      o[2 * Zd] = from_c<R>(zq);
    }
  }
}

// ---------------------------------------------------- activation on a jet
// s = ssp(a): s_t = sigma(a) a_t, lap s = sigma(a) lap a + sigma'(a) sum_t a_t^2.
template <typename R>
__global__ void k_ssp_jet(R* __restrict__ A, int ld, size_t groups, int T, int dim) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= groups * dim) return;
  const int d = idx % dim;
  const size_t g = idx / dim;
  R* a = A + g * T * ld + d;
  const R a0 = a[0];
  const R sg = sigm_(a0);
  a[0] = ssp_(a0);
  if (T == 1) return;
  R sq = 0;
  for (int t = 1; t < T - 1; ++t) {
    const R v = a[(size_t)t * ld];
    sq += v * v;
    a[(size_t)t * ld] = sg * v;
  }
  a[(size_t)(T - 1) * ld] = sg * a[(size_t)(T - 1) * ld] + sg * (R(1) - sg) * sq;
}

// Xs[w][t][d] = sum_i X[w][i][t][d]
template <typename R>
__global__ void k_sum_electrons(const R* __restrict__ X, R* __restrict__ Xs, int Wn, int N, int T, int D) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Wn * T * D) return;
  const int d = idx % D;
  const int t = (idx / D) % T;
  const int w = idx / ((size_t)D * T);
  R acc = 0;
  for (int i = 0; i < N; ++i) acc += X[(((size_t)w * N + i) * T + t) * D + d];
  Xs[idx] = acc;
}

// ----------------------------------------------------------- determinants
// One thread per (walker, determinant, spin): the block computed directly
// (pn_slater_block).  det[w][p][s] = {ln|det|, sign, lap, grad[3N]}.
template <typename R>
__global__ void k_slater(DevSys s, const double* __restrict__ phi, const R* __restrict__ F, int Wn, int T, int jet,
                         double* __restrict__ det) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Wn * s.n_det * 2) return;
  const int sg = idx & 1;
  const int p = (idx >> 1) % s.n_det;
  const int w = (idx >> 1) / s.n_det;
  const int N = s.N, no = s.n_orb;
  pn_slater_block<R, PN_MAX_SPIN>(s, phi + (size_t)w * N * no * 5, F + (size_t)w * N * T * no, p, sg, T, jet,
                                  det + (size_t)idx * (3 + 3 * N));
}

// ------------------------------------------------------------ combination
// ln|psi| = gamma + J + ln|sum_p c_p s_p e^{ld_p}| (signed log-sum-exp over
// determinants) and, in jet mode, E_loc = -1/2 (lap ln|psi| + |grad|^2) + V.
template <typename R>
__global__ void k_combine(DevSys s, const double* __restrict__ geo, const double* __restrict__ det,
                          const R* __restrict__ Jj, int Wn, int T, int jet, double* __restrict__ logabs,
                          double* __restrict__ sign, double* __restrict__ eloc, int* __restrict__ status,
                          double* __restrict__ grad_out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Wn) return;
  const int N = s.N, nd = s.n_det, stride = 3 + 3 * N;
  const double* dw = det + (size_t)w * nd * 2 * stride;
  double m = -INFINITY;
  for (int p = 0; p < nd; ++p) {
    const double* u = dw + (size_t)(2 * p) * stride;
    const double* d = u + stride;
    if (s.ci[p] != 0.0 && u[1] != 0.0 && d[1] != 0.0) m = fmax(m, u[0] + d[0]);
  }
  double S = 0;
  if (m > -INFINITY)
    for (int p = 0; p < nd; ++p) {
      const double* u = dw + (size_t)(2 * p) * stride;
      const double* d = u + stride;
      if (u[1] != 0.0 && d[1] != 0.0) S += s.ci[p] * u[1] * d[1] * exp(u[0] + d[0] - m);
    }
  const double* gw = geo + (size_t)w * s.Ppair * 4;
  // electronic cusp factor gamma and the Coulomb potential
  double gam = 0, V = s.Vnn;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      const double d = gw[pn_pair_index(a, b, N) * 4];
      V += 1.0 / d;
      if (s.use_gamma) {
        const double c = ((a < s.n_up) == (b < s.n_up)) ? 0.25 : 0.5;
        gam -= c / (1.0 + d);
      }
    }
  for (int q = 0; q < s.Pen; ++q) V -= s.Z[q % s.M] / gw[(s.Pee + q) * 4];
  const R* J = Jj + (size_t)w * T;
  int st = PN_WALKER_OK;
  if (!(S != 0.0) || !(m > -INFINITY)) st = PN_WALKER_SINGULAR;
  const double la = gam + (double)J[0] + m + log(fabs(S));
  logabs[w] = la;
  sign[w] = S > 0 ? 1.0 : (S < 0 ? -1.0 : 0.0);
  if (!jet) {
    if (st == PN_WALKER_OK && !isfinite(la)) st = PN_WALKER_NONFINITE;
    if (status) status[w] = st;
    return;
  }
  double g[3 * PN_MAX_ELECTRONS];
  const int n3 = 3 * N;
  for (int t = 0; t < n3; ++t) g[t] = 0;
  double lapS = 0;
  if (st == PN_WALKER_OK) {
    for (int p = 0; p < nd; ++p) {
      const double* u = dw + (size_t)(2 * p) * stride;
      const double* d = u + stride;
      if (u[1] == 0.0 || d[1] == 0.0) continue;
      const double om = s.ci[p] * u[1] * d[1] * exp(u[0] + d[0] - m) / S;
      double sq = 0;
      for (int t = 0; t < n3; ++t) {
        const double gt = u[3 + t] + d[3 + t];
        g[t] += om * gt;
        sq += gt * gt;
      }
      lapS += om * (u[2] + d[2] + sq);
    }
  }
  double g2 = 0;
  for (int t = 0; t < n3; ++t) g2 += g[t] * g[t];
  double lap = lapS - g2 + (double)J[T - 1];
  for (int t = 0; t < n3; ++t) g[t] += (double)J[1 + t];
  if (s.use_gamma) {
    for (int a = 0; a < N; ++a)
      for (int b = a + 1; b < N; ++b) {
        const double* gg = gw + pn_pair_index(a, b, N) * 4;
        const double d = gg[0];
        const double c = ((a < s.n_up) == (b < s.n_up)) ? 0.25 : 0.5;
        const double e = 1.0 / (1.0 + d);
        const double g1 = c * e * e;          // d gamma_ab / d d
        const double g2_ = -2.0 * c * e * e * e;
        for (int x = 0; x < 3; ++x) {
          g[3 * a + x] += g1 * gg[1 + x];
          g[3 * b + x] -= g1 * gg[1 + x];
        }
        lap += 2.0 * (g2_ + 2.0 * g1 / d);
      }
  }
  double gn = 0;
  for (int t = 0; t < n3; ++t) gn += g[t] * g[t];
  if (grad_out)
    for (int t = 0; t < n3; ++t) grad_out[(size_t)w * n3 + t] = g[t];
  const double E = -0.5 * (lap + gn) + V;
  eloc[w] = E;
  if (st == PN_WALKER_OK && !(isfinite(E) && isfinite(la))) st = PN_WALKER_NONFINITE;
  if (status) status[w] = st;
}

// The same combination with a warp per walker: lanes over determinants for
// the signed log-sum, over electron pairs for gamma and V, and over the 3N
// coordinates for the gradient (three per lane at most).
__device__ inline double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename R>
__global__ void k_combine_w(DevSys s, const double* __restrict__ geo, const double* __restrict__ det,
                            const R* __restrict__ Jj, int Wn, int T, int jet, double* __restrict__ logabs,
                            double* __restrict__ sign, double* __restrict__ eloc, int* __restrict__ status,
                            double* __restrict__ grad_out) {
  const int lane = threadIdx.x & 31;
  const int w = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= Wn) return;
  const int N = s.N, nd = s.n_det, stride = 3 + 3 * N, n3 = 3 * N;
  const double* dw = det + (size_t)w * nd * 2 * stride;
  double m = -INFINITY;
  for (int p = lane; p < nd; p += 32) {
    const double* u = dw + (size_t)(2 * p) * stride;
    const double* d = u + stride;
    if (s.ci[p] != 0.0 && u[1] != 0.0 && d[1] != 0.0) m = fmax(m, u[0] + d[0]);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  double S = 0;
  if (m > -INFINITY)
    for (int p = lane; p < nd; p += 32) {
      const double* u = dw + (size_t)(2 * p) * stride;
      const double* d = u + stride;
      if (u[1] != 0.0 && d[1] != 0.0) S += s.ci[p] * u[1] * d[1] * exp(u[0] + d[0] - m);
    }
  S = wsum(S);
  const double* gw = geo + (size_t)w * s.Ppair * 4;
  double gam = 0, V = 0, lapg = 0;
  for (int q = lane; q < s.Pee; q += 32) {
    int a = 0, rem = q;
    while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
    const int b = a + 1 + rem;
    const double d = gw[q * 4];
    V += 1.0 / d;
    if (s.use_gamma) {
      const double c = ((a < s.n_up) == (b < s.n_up)) ? 0.25 : 0.5;
      gam -= c / (1.0 + d);
      const double e = 1.0 / (1.0 + d);
      const double g1 = c * e * e, g2 = -2.0 * c * e * e * e;
      lapg += 2.0 * (g2 + 2.0 * g1 / d);
    }
  }
  for (int q = lane; q < s.Pen; q += 32) V -= s.Z[q % s.M] / gw[(s.Pee + q) * 4];
  gam = wsum(gam);
  V = wsum(V) + s.Vnn;
  const R* J = Jj + (size_t)w * T;
  int st = PN_WALKER_OK;
  if (!(S != 0.0) || !(m > -INFINITY)) st = PN_WALKER_SINGULAR;
  const double la = gam + (double)J[0] + m + log(fabs(S));
  if (lane == 0) {
    logabs[w] = la;
    sign[w] = S > 0 ? 1.0 : (S < 0 ? -1.0 : 0.0);
  }
  if (!jet) {
    if (st == PN_WALKER_OK && !isfinite(la)) st = PN_WALKER_NONFINITE;
    if (status && lane == 0) status[w] = st;
    return;
  }
  lapg = wsum(lapg);
  double g[3] = {0, 0, 0}, sq = 0, lap0 = 0;
  if (st == PN_WALKER_OK)
    for (int p = 0; p < nd; ++p) {
      const double* u = dw + (size_t)(2 * p) * stride;
      const double* d = u + stride;
      if (u[1] == 0.0 || d[1] == 0.0) continue;
      const double om = s.ci[p] * u[1] * d[1] * exp(u[0] + d[0] - m) / S;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int t = lane + 32 * k;
        if (t < n3) {
          const double gt = u[3 + t] + d[3 + t];
          g[k] += om * gt;
          sq += om * gt * gt;
        }
      }
      lap0 += om * (u[2] + d[2]);
    }
  double g2 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) g2 += g[k] * g[k];
  g2 = wsum(g2);
  double lap = lap0 + wsum(sq) - g2 + (double)J[T - 1];
  if (s.use_gamma) lap += lapg;
  double gn = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int t = lane + 32 * k;
    if (t >= n3) continue;
    g[k] += (double)J[1 + t];
    if (s.use_gamma) {
      const int a = t / 3, x = t - 3 * a;
      for (int b = 0; b < N; ++b) {
        if (b == a) continue;
        const int p = a < b ? pn_pair_index(a, b, N) : pn_pair_index(b, a, N);
        const double* gg = gw + p * 4;
        const double c = ((a < s.n_up) == (b < s.n_up)) ? 0.25 : 0.5;
        const double e = 1.0 / (1.0 + gg[0]);
        // gg holds (r_lo - r_hi)/d for the pair (lo, hi)
        g[k] += (a < b ? 1.0 : -1.0) * c * e * e * gg[1 + x];
      }
    }
    gn += g[k] * g[k];
    if (grad_out) grad_out[(size_t)w * n3 + t] = g[k];
  }
  gn = wsum(gn);
  const double E = -0.5 * (lap + gn) + V;
  if (lane == 0) {
    eloc[w] = E;
    if (st == PN_WALKER_OK && !(isfinite(E) && isfinite(la))) st = PN_WALKER_NONFINITE;
    if (status) status[w] = st;
  }
}

}  // namespace pnk

// ------------------------------------------------------------------ driver
using namespace pnk;

static inline unsigned nblk(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Tile shape by output width, then the load/store widths.
template <bool TB>
static int linear_v4_launch(const float* xf, int ldx, const float* wf, int ldw, const float* bf, float* yf, int ldy,
                            int rows, int Kd, int Nout, int T, int acc, bool vw, bool vy, cudaStream_t st) {
  const char* kname = TB ? "k_linear_bt" : "k_linear";
#define PN_LIN(BM, BN, TN)                                                                                    \
  do {                                                                                                        \
    dim3 grid((rows + BM - 1) / BM, (Nout + BN - 1) / BN);                                                    \
    if (vw && vy)                                                                                             \
      PN_LAUNCH_WB(kname, st, 2.0 * rows * Kd * Nout, 4.0 * rows * (Kd + Nout * (acc ? 2 : 1)), (k_linear_v4<BM, BN, TN, true, true, TB><<<grid, 256, 0, st>>>(xf, ldx, wf, ldw, bf, yf, ldy, rows, Kd, Nout, T, acc)));   \
    else if (vy)                                                                                              \
      PN_LAUNCH_WB(kname, st, 2.0 * rows * Kd * Nout, 4.0 * rows * (Kd + Nout * (acc ? 2 : 1)), (k_linear_v4<BM, BN, TN, false, true, TB><<<grid, 256, 0, st>>>(xf, ldx, wf, ldw, bf, yf, ldy, rows, Kd, Nout, T, acc)));  \
    else                                                                                                      \
      PN_LAUNCH_WB(kname, st, 2.0 * rows * Kd * Nout, 4.0 * rows * (Kd + Nout * (acc ? 2 : 1)), (k_linear_v4<BM, BN, TN, false, false, TB><<<grid, 256, 0, st>>>(xf, ldx, wf, ldw, bf, yf, ldy, rows, Kd, Nout, T, acc))); \
  } while (0)
  if (Nout <= 32) PN_LIN(256, 32, 4);  // narrow maps
  else if (Nout <= 64) PN_LIN(128, 64, 4);
  else PN_LIN(128, 128, 8);
#undef PN_LIN
  return PN_OK;
}

// Float32 Y (=|+=) X W^T with W stored [Nout][Kd] (row stride ldw): the
// backward's products through transposed weights on the pipelined tiles.
// PN_ENOTREADY when X is not float4-aligned (the caller's scalar kernel).
int pn_linear_bt_f32(const float* X, int ldx, const float* W, int ldw, float* Y, int ldy, int rows, int Kd, int Nout,
                     int acc, cudaStream_t st) {
  if (ldx % 4 || Kd % 4 || ((uintptr_t)X & 15)) return PN_ENOTREADY;
  if (rows <= 0) return PN_OK;
  const bool vw = ldw % 4 == 0 && ((uintptr_t)W & 15) == 0;
  const bool vy = ldy % 4 == 0 && Nout % 4 == 0 && ((uintptr_t)Y & 15) == 0;
  return linear_v4_launch<true>(X, ldx, W, ldw, nullptr, Y, ldy, rows, Kd, Nout, 1, acc, vw, vy, st);
}

template <typename R>
int pn_linear(const DevSys* s, int grp, const R* X, int ldx, const R* W, int ldw, const R* b, R* Y, int ldy, int rows,
              int Kd, int Nout, int T, int acc, cudaStream_t st) {
  if (rows <= 0) return PN_OK;
  if constexpr (sizeof(R) == 4) {
    // value passes (T == 1) use the PN_TC_VALUE bit, jet passes the group bit
    const int bit = T == 1 ? PN_TC_VALUE : grp;
    // the persistent tensor-core kernel splits the weight into shared
    // memory once per CTA: below a few thousand rows the CUDA-core tiles win
    if (s && (s->tensor_cores & bit) && pn_tc_supported(Nout) && rows >= 8192) {
      const int e = pn_linear_tc((const float*)X, ldx, (const float*)W, ldw, (const float*)b, (float*)Y, ldy, rows, Kd,
                                 Nout, T, acc, s->dev_err, st);
      if (e != PN_ENOTREADY) return e;  // else: the weight does not fit in shared memory, CUDA cores below
    }
  }
  if constexpr (sizeof(R) == 4) {
    if (ldx % 4 == 0 && Kd % 4 == 0 && ((uintptr_t)X & 15) == 0) {
      const bool vw = ldw % 4 == 0 && Nout % 4 == 0 && ((uintptr_t)W & 15) == 0;
      const bool vy = ldy % 4 == 0 && Nout % 4 == 0 && ((uintptr_t)Y & 15) == 0;
      const float *xf = (const float*)X, *wf = (const float*)W, *bf = (const float*)b;
      float* yf = (float*)Y;
      return linear_v4_launch<false>(xf, ldx, wf, ldw, bf, yf, ldy, rows, Kd, Nout, T, acc, vw, vy, st);
    }
  }
  dim3 grid((rows + 63) / 64, (Nout + 63) / 64);
  if constexpr (sizeof(R) == 8) {
    if (s && s->lin_f32x2) {
      PN_LAUNCH_WB("k_linear_f32x2", st, 2.0 * rows * Kd * Nout, 8.0 * rows * (Kd + Nout * (acc ? 2 : 1)),
                   k_linear_f32x2<<<grid, 256, 0, st>>>((const double*)X, ldx, (const double*)W, ldw,
                                                        (const double*)b, (double*)Y, ldy, rows, Kd, Nout, T, acc));
      return PN_OK;
    }
  }
  // float64 maps form a class of their own (bound by the float64 pipe)
  PN_LAUNCH_WB(sizeof(R) == 8 ? "k_linear_f64" : "k_linear", st, 2.0 * rows * Kd * Nout,
               (double)sizeof(R) * rows * (Kd + Nout * (acc ? 2 : 1)),
               k_linear<R><<<grid, 256, 0, st>>>(X, ldx, W, ldw, b, Y, ldy, rows, Kd, Nout, T, acc));
  return PN_OK;
}
template int pn_linear<double>(const DevSys*, int, const double*, int, const double*, int, const double*, double*, int,
                               int, int, int, int, int, cudaStream_t);
template int pn_linear<float>(const DevSys*, int, const float*, int, const float*, int, const float*, float*, int, int,
                              int, int, int, int, cudaStream_t);

template <typename R>
int pn_ssp_jet(R* A, int ld, size_t groups, int T, int dim, cudaStream_t st) {
  PN_LAUNCH("k_ssp_jet", st, k_ssp_jet<R><<<nblk(groups * dim, 256), 256, 0, st>>>(A, ld, groups, T, dim));
  return PN_OK;
}

template <typename R>
int pn_network_layers(const DevSys& s, const DevNet<R>& net, Work<R>& w, int Wn, int T, int jet, cudaStream_t st) {
  const size_t groups = (size_t)Wn * s.N;
  const int rows = (int)(groups * T);
  PN_LAUNCH("k_features", st, k_features<R><<<nblk((size_t)Wn * s.Ppair * s.K, 256), 256, 0, st>>>(s, w.geo, Wn, jet, w.efeat));
  // jet passes: the first layer's input is the constant x^(0), so its h is
  // one row (k_h0_row, into the Xs scratch that the heads use later) and its
  // receiving map writes X with x^(0) folded into the value rows' bias
  const bool first_const = jet;
  if (first_const)
    PN_LAUNCH("k_h0_row", st, k_h0_row<R><<<nblk(s.Zd, 64), 64, 0, st>>>(net.p + net.off.x0, net.p + net.off.hW[0],
                                                                        net.p + net.off.hb[0], s.D, s.Zd, w.Xs));
  else
    PN_LAUNCH("k_init_x", st, k_init_x<R><<<nblk(groups * T * s.D, 256), 256, 0, st>>>(net.p + net.off.x0, w.X, groups, T, s.D));
  for (int n = 0; n < s.L; ++n) {
    const bool hc = first_const && n == 0;
    if (!hc)
      if (int e = pn_linear<R>(&s, PN_TC_LAYERS, w.X, s.D, net.p + net.off.hW[n], s.Zd, net.p + net.off.hb[n], w.H, w.ldH,
                               rows, s.D, s.Zd, T, 0, st))
        return e;
    // jet filters on pair-row tiles for large batches; below about 128 k pair
    // rows the per-row kernel's many small blocks hide latency better (Be,
    // 4096 walkers x 10 pairs: 0.154 ms per pass per-row, 0.174 ms tiled)
    int fe = PN_ENOTREADY;
    if constexpr (sizeof(R) == 4)
      if ((size_t)Wn * s.Ppair >= ((size_t)1 << 17))
        fe = jet ? pn_filter_tile_jet(s, net, n, (const float*)w.efeat, Wn, (float*)w.wjet, st)
                 : pn_filter_tile_value_fwd(s, net, n, (const float*)w.efeat, Wn, (float*)w.wjet, st);
    if (fe != PN_OK && fe != PN_ENOTREADY) return fe;
    // kernel classes: float64 launches (the float64 path, the guard's
    // re-evaluation) and value passes apart from the float32 jet passes
    const char* fname = sizeof(R) == 8 ? "k_filter_f64" : (jet ? "k_filter" : "k_filter_value");
    const char* mname = sizeof(R) == 8 ? "k_message_f64" : (jet ? "k_message" : "k_message_value");
    if (fe == PN_ENOTREADY)
      PN_LAUNCH_W(fname, st, 2.0 * (jet ? 3 : 1) * Wn * s.Ppair * (double)(s.K * s.Hw + s.Hw * s.Zd),
                  k_filter<R><<<nblk((size_t)Wn * s.Ppair, FW), FW * 32, 0, st>>>(s, net, n, w.efeat, Wn, jet, w.wjet));
    if (jet) {
      const size_t nthr = (size_t)Wn * ((s.N + MSG_KC - 1) / MSG_KC + 1) * s.N * s.Zd;
      // bytes that must cross HBM: the h rows and filter jets read once,
      // the message rows written once
      const double bytes = (double)sizeof(R) * Wn * ((double)s.N * T * s.Zd + 3.0 * s.Ppair * s.Zd + 3.0 * s.N * T * s.Zd);
      // staged per-walker kernel where Zd tiles by 16 and the walker's rows fit
      const size_t mw_bytes = sizeof(R) * ((size_t)(hc ? 1 : s.N * T) * MSGW_ZT + (size_t)s.Ppair * 3 * MSGW_ZT +
                                           (size_t)s.Ppair * 5);
      const bool staged = s.Zd % MSGW_ZT == 0 && s.N <= MSGW_NMAX && mw_bytes <= 160 * 1024 && !s.msg_per_row;
      if (staged) {
        const unsigned grid = (unsigned)((size_t)Wn * (s.Zd / MSGW_ZT));
        const unsigned blk = (unsigned)((s.N + 1) / 2 * 32);
        const R* hsrc = hc ? w.Xs : w.H;
        const int ldh = hc ? 0 : w.ldH;
        // float64 buffers of the guard's re-evaluation: float32-pair arithmetic
        bool pair = false;
        if constexpr (sizeof(R) == 8) pair = s.lin_f32x2 != 0;
        if (pair) {
          if constexpr (sizeof(R) == 8) {
            if (hc) {
              PN_CUDA(pn_allow_max_smem(k_message_w<double, true, FF>));
              PN_LAUNCH_W(mname, st, bytes, (k_message_w<double, true, FF><<<grid, blk, mw_bytes, st>>>(
                                                s, net.p + net.off.Y, w.geo, w.wjet, hsrc, ldh, Wn, T, w.Zb, w.ldZ)));
            } else {
              PN_CUDA(pn_allow_max_smem(k_message_w<double, false, FF>));
              PN_LAUNCH_W(mname, st, bytes, (k_message_w<double, false, FF><<<grid, blk, mw_bytes, st>>>(
                                                s, net.p + net.off.Y, w.geo, w.wjet, hsrc, ldh, Wn, T, w.Zb, w.ldZ)));
            }
          }
        } else if (hc) {
          PN_CUDA(pn_allow_max_smem(k_message_w<R, true>));
          PN_LAUNCH_W(mname, st, bytes, (k_message_w<R, true><<<grid, blk, mw_bytes, st>>>(
                                            s, net.p + net.off.Y, w.geo, w.wjet, hsrc, ldh, Wn, T, w.Zb, w.ldZ)));
        } else {
          PN_CUDA(pn_allow_max_smem(k_message_w<R, false>));
          PN_LAUNCH_W(mname, st, bytes, (k_message_w<R, false><<<grid, blk, mw_bytes, st>>>(
                                            s, net.p + net.off.Y, w.geo, w.wjet, hsrc, ldh, Wn, T, w.Zb, w.ldZ)));
        }
      } else if (hc) {
        PN_LAUNCH_W(mname, st, bytes,
                    (k_message_c<R, true><<<nblk(nthr, 256), 256, 0, st>>>(s, net.p + net.off.Y, w.geo, w.wjet, w.Xs, 0,
                                                                           Wn, T, w.Zb, w.ldZ)));
      } else {
        PN_LAUNCH_W(mname, st, bytes,
                    (k_message_c<R, false><<<nblk(nthr, 256), 256, 0, st>>>(s, net.p + net.off.Y, w.geo, w.wjet, w.H,
                                                                            w.ldH, Wn, T, w.Zb, w.ldZ)));
      }
    } else {
      PN_LAUNCH(mname, st,
                k_message<R><<<(unsigned)((size_t)Wn * s.N), std::min(256, (T * s.Zd + 31) / 32 * 32),
                               (size_t)(s.N - 1 + s.M) * 5 * sizeof(R), st>>>(
                    s, net.p + net.off.Y, w.geo, w.wjet, w.H, w.ldH, Wn, T, w.Zb, w.ldZ));
    }
    if (int e = pn_linear<R>(&s, PN_TC_LAYERS, w.Zb, w.ldZ, net.Gcat + (size_t)n * 3 * s.Zd * s.D, s.D,
                             hc ? net.Gbx0 : net.Gb + (size_t)n * s.D, w.X, s.D, rows, 3 * s.Zd, s.D, T, hc ? 0 : 1, st))
      return e;
  }
  return PN_OK;
}

template <typename R>
int pn_heads(const DevSys& s, const DevNet<R>& net, Work<R>& w, int Wn, int T, cudaStream_t st) {
  const size_t groups = (size_t)Wn * s.N;
  const int rows = (int)(groups * T);
  const NetOff& o = net.off;
  const int D = s.D;
  // backflow head kappa on every electron
  if (int e = pn_linear<R>(&s, PN_TC_HEADS, w.X, D, net.p + o.kW[0], D, net.p + o.kb[0], w.Zb, w.ldZ, rows, D, D, T, 0, st)) return e;
  if (int e = pn_ssp_jet<R>(w.Zb, w.ldZ, groups, T, D, st)) return e;
  if (int e = pn_linear<R>(&s, PN_TC_HEADS, w.Zb, w.ldZ, net.p + o.kW[1], D, net.p + o.kb[1], w.H, w.ldH, rows, D, D, T, 0, st)) return e;
  if (int e = pn_ssp_jet<R>(w.H, w.ldH, groups, T, D, st)) return e;
  if (int e = pn_linear<R>(&s, PN_TC_HEADS, w.H, w.ldH, net.p + o.kW[2], s.n_orb, net.p + o.kb[2], w.F, s.n_orb, rows, D, s.n_orb, T, 0, st))
    return e;
  // Jastrow head eta on the electron sum
  PN_LAUNCH("k_sum_electrons", st, k_sum_electrons<R><<<nblk((size_t)Wn * T * D, 256), 256, 0, st>>>(w.X, w.Xs, Wn, s.N, T, D));
  const int rs = Wn * T;
  if (int e = pn_linear<R>(&s, PN_TC_HEADS, w.Xs, D, net.p + o.eW[0], D, net.p + o.eb[0], w.As, D, rs, D, D, T, 0, st)) return e;
  if (int e = pn_ssp_jet<R>(w.As, D, (size_t)Wn, T, D, st)) return e;
  if (int e = pn_linear<R>(&s, PN_TC_HEADS, w.As, D, net.p + o.eW[1], D, net.p + o.eb[1], w.Bs, D, rs, D, D, T, 0, st)) return e;
  if (int e = pn_ssp_jet<R>(w.Bs, D, (size_t)Wn, T, D, st)) return e;
  if (int e = pn_linear<R>(&s, PN_TC_HEADS, w.Bs, D, net.p + o.eW[2], 1, net.p + o.eb[2], w.Jj, 1, rs, D, 1, T, 0, st)) return e;
  return PN_OK;
}

// Algorithmic float64 work of the determinants of one walker: per
// (determinant, spin) block of size n the LU (2/3 n^3 multiply-adds); in jet
// mode also the inverse (n^3), tr(A^-1 lap A) (n^2) and, per coordinate t,
// A^-1 dA_t (n^3) and tr((A^-1 dA_t)^2) (n^2).
static double pn_slater_flops(const DevSys& s, int jet) {
  double f = 0;
  for (int sg = 0; sg < 2; ++sg) {
    const double n = sg ? s.n_dn : s.n_up;
    if (n == 0) continue;
    f += 2.0 * (2.0 / 3.0) * n * n * n;
    if (jet) f += 2.0 * (n * n * n + n * n + 3.0 * s.N * (n * n * n + n * n));
  }
  return f * s.n_det;
}

// Determinant blocks: the table kernel for jet passes where the system has
// a table, else one thread per block.
template <typename R>
static int pn_slater(const DevSys& s, const double* phi, const R* F, int Wn, int T, int jet, double* det,
                     cudaStream_t st) {
  if (!s.no_table) {
    const int e = pn_slater_table_launch<R>(s, phi, F, Wn, T, jet, det, st);
    if (e != PN_ENOTREADY) return e;
  }
  PN_LAUNCH_W("k_slater", st, Wn * pn_slater_flops(s, jet),
              k_slater<R><<<nblk((size_t)Wn * s.n_det * 2, 64), 64, 0, st>>>(s, phi, F, Wn, T, jet, det));
  return PN_OK;
}

template <typename R>
int pn_forward_chunk(const DevSys& s, const DevNet<R>& net, Work<R>& w, const double* r, int Wn, int jet,
                     cudaStream_t st) {
  if (Wn <= 0) return PN_OK;
  const int T = jet ? 3 * s.N + 2 : 1;
  PN_LAUNCH("k_geometry", st, k_geometry<<<nblk((size_t)Wn * s.Ppair, 128), 128, 0, st>>>(s, r, Wn, w.geo));
  if (jet)
    PN_LAUNCH("k_orbitals", st, k_orbitals<true><<<nblk((size_t)Wn * s.N, 64), 64, 0, st>>>(s, r, Wn, w.phi));
  else
    PN_LAUNCH("k_orbitals", st, k_orbitals<false><<<nblk((size_t)Wn * s.N, 64), 64, 0, st>>>(s, r, Wn, w.phi));
  if (int e = pn_network_layers<R>(s, net, w, Wn, T, jet, st)) return e;
  if (int e = pn_heads<R>(s, net, w, Wn, T, st)) return e;
  if (int e = pn_slater<R>(s, w.phi, w.F, Wn, T, jet, w.det, st)) return e;
  PN_LAUNCH("k_combine", st, k_combine_w<R><<<nblk((size_t)Wn * 32, 128), 128, 0, st>>>(s, w.geo, w.det, w.Jj, Wn, T, jet,
                                                                                     w.out_logabs, w.out_sign,
                                                                                     w.out_eloc, w.out_status,
                                                                                     w.out_grad));
  return PN_OK;
}

// Second evaluation of a guarded mixed chunk.  Probe 0: the heads again
// with the other unit for their linear maps (their rounding differs), the
// determinants of the new backflow, and E_loc with the new Jastrow factor.
// Probe 1: the first pass's backflow and Jastrow jets perturbed by
// +-2^-19 relative, then the determinants and E_loc again.  Probe 2: as 1
// with a third of 2^-19 at the heads' term scale added (k_perturb_abs).  ln|psi| and
// sign of this pass go to scratch (the proposal buffers), E_loc to e_probe;
// the first pass's outputs stay in w.
int pn_probe_heads_chunk(const DevSys& s, const DevNet<float>& net, Work<float>& w, int Wn, double* e_probe,
                         cudaStream_t st) {
  if (Wn <= 0) return PN_OK;
  const int T = 3 * s.N + 2;
  if (s.guard_probe == 1) {
    const size_t nf = (size_t)Wn * s.N * T * s.n_orb, nj = (size_t)Wn * T;
    if (int e = pn_perturb_rel(w.F, nf, 1.9073486e-6f, st)) return e;
    if (int e = pn_perturb_rel(w.Jj, nj, 1.9073486e-6f, st)) return e;
  } else if (s.guard_probe == 2) {
    // the last maps of both heads: backflow f = H W_k2 (+ b), Jastrow
    // jets J = B W_e2 (+ b); their inputs H and B are still in place.
    // +-2^-19 relative, plus a third of that at the scale of the terms
    // The terms' scale |x| |W| comes from the tensor-core map in
    // absolute-value mode into the first head's hidden buffer Zb (free by
    // now), else from the CUDA-core kernel.
    const NetOff& o = net.off;
    const float er = 1.9073486e-6f, ea = 1.9073486e-6f / 3.f;
    const size_t zb = (size_t)Wn * s.N * T * w.ldZ;
    const size_t rf = (size_t)Wn * s.N * T, rj = (size_t)Wn * T;
    int e = (s.tensor_cores & PN_TC_HEADS)
                ? pn_perturb_abs_tc(w.H, w.ldH, net.p + o.kW[2], s.n_orb, w.F, s.n_orb, rf, s.D, s.n_orb, er, ea, w.Zb,
                                    zb, s.dev_err, st)
                : PN_ENOTREADY;
    if (e == PN_ENOTREADY)
      e = pn_perturb_abs(w.H, w.ldH, net.p + o.kW[2], s.n_orb, w.F, s.n_orb, rf, s.D, s.n_orb, er, ea, st);
    if (e) return e;
    e = (s.tensor_cores & PN_TC_HEADS)
            ? pn_perturb_abs_tc(w.Bs, s.D, net.p + o.eW[2], 1, w.Jj, 1, rj, s.D, 1, er, ea, w.Zb, zb, s.dev_err, st)
            : PN_ENOTREADY;
    if (e == PN_ENOTREADY) e = pn_perturb_abs(w.Bs, s.D, net.p + o.eW[2], 1, w.Jj, 1, rj, s.D, 1, er, ea, st);
    if (e) return e;
  } else {
    DevSys s2 = s;
    s2.tensor_cores ^= PN_TC_HEADS;
    if (int e = pn_heads<float>(s2, net, w, Wn, T, st)) return e;
  }
  if (int e = pn_slater<float>(s, w.phi, w.F, Wn, T, 1, w.det, st)) return e;
  PN_LAUNCH("k_combine", st, k_combine_w<float><<<nblk((size_t)Wn * 32, 128), 128, 0, st>>>(
                                 s, w.geo, w.det, w.Jj, Wn, T, 1, w.lp_prop, w.r_prop, e_probe, nullptr, nullptr));
  return PN_OK;
}

template int pn_forward_chunk<double>(const DevSys&, const DevNet<double>&, Work<double>&, const double*, int, int,
                                      cudaStream_t);
template int pn_forward_chunk<float>(const DevSys&, const DevNet<float>&, Work<float>&, const double*, int, int,
                                     cudaStream_t);

// Launchers used by the backward pass (value mode).
int pn_launch_geometry_orbitals(const DevSys& s, const double* r, int Wn, double* geo, double* phi, cudaStream_t st) {
  PN_LAUNCH("k_geometry", st, k_geometry<<<nblk((size_t)Wn * s.Ppair, 128), 128, 0, st>>>(s, r, Wn, geo));
  PN_LAUNCH("k_orbitals", st, k_orbitals<true><<<nblk((size_t)Wn * s.N, 64), 64, 0, st>>>(s, r, Wn, phi));
  return PN_OK;
}

template <typename R>
int pn_launch_features_init(const DevSys& s, const R* x0, const double* geo, int Wn, int deriv, R* ef, R* X,
                            cudaStream_t st) {
  PN_LAUNCH("k_features", st, k_features<R><<<nblk((size_t)Wn * s.Ppair * s.K, 256), 256, 0, st>>>(s, geo, Wn, deriv, ef));
  PN_LAUNCH("k_init_x", st, k_init_x<R><<<nblk((size_t)Wn * s.N * s.D, 256), 256, 0, st>>>(x0, X, (size_t)Wn * s.N, 1, s.D));
  return PN_OK;
}
template int pn_launch_features_init<double>(const DevSys&, const double*, const double*, int, int, double*, double*,
                                             cudaStream_t);
template int pn_launch_features_init<float>(const DevSys&, const float*, const double*, int, int, float*, float*,
                                            cudaStream_t);

template <typename R>
int pn_launch_sum_electrons(const R* X, R* Xs, int Wn, int N, int D, cudaStream_t st) {
  PN_LAUNCH("k_sum_electrons", st, k_sum_electrons<R><<<nblk((size_t)Wn * D, 256), 256, 0, st>>>(X, Xs, Wn, N, 1, D));
  return PN_OK;
}
template int pn_launch_sum_electrons<double>(const double*, double*, int, int, int, cudaStream_t);
template int pn_launch_sum_electrons<float>(const float*, float*, int, int, int, cudaStream_t);
