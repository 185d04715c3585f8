// Filter networks w^(n,c)(e) = W2 ssp(W1 e + b1) + b2 of the interaction
// layers (Methods, the PauliNet extension of SchNet: filters of the
// electron-electron and electron-nucleus distance features), evaluated on
// tiles of pair rows for the float32 path: a block takes 64 pair rows of one
// filter channel (same-spin pairs, opposite-spin pairs, electron-nucleus
// pairs; the channel's pair list gives the rows), keeps both weight matrices
// in shared memory and forms each product as a register-tiled matrix
// product (4 rows x NJ columns per thread, columns tx + 16 j).  Four forms:
//   value  -- hidden pre-activation Ah (kept for the backward) and w;
//   jet    -- value, first and second distance derivative rows (chain rule
//             through ssp: h' = s a', h'' = s a'' + s (1 - s) a'^2, s = sigmoid(a));
//   bwd    -- dAh = (dw W2^T) sigmoid(Ah) and ssp(Ah) for the weight gradients;
//   dist   -- the distance cotangent dd += sum_h dAh (e'(d) W1)_h.
// Launchers return PN_ENOTREADY when a tile does not fit in shared memory;
// the caller then runs the per-row kernels.
#include <math.h>

#include <algorithm>

#include "kernels.cuh"
#include "pn_internal.cuh"

namespace {

constexpr int RB = 64;       // pair rows per block
constexpr int LA = RB + 4;   // row stride of transposed operand tiles (16-byte aligned float4 reads)

struct FTiles {
  int t0[4];  // first block of each channel; t0[3] = grid size
};

__device__ inline float sigmf_(float x) { return 1.f / (1.f + expf(-x)); }
__device__ inline float sspf_(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))) - 0.69314718055994530942f; }

// This block's channel and its rows' global pair-row indices (w * P + p;
// -1 past the channel's last row).
__device__ inline int tile_setup(const DevSys& s, const FTiles& ft, int Wn, int* sgr) {
  const int b = blockIdx.x;
  const int c = b < ft.t0[1] ? 0 : (b < ft.t0[2] ? 1 : 2);
  const int cnt = s.ch_off[c + 1] - s.ch_off[c];
  const int r0 = (b - ft.t0[c]) * RB;
  const int nr = min(RB, Wn * cnt - r0);
  for (int q = threadIdx.x; q < RB; q += blockDim.x) {
    int g = -1;
    if (q < nr) {
      const int r = r0 + q;
      g = (r / cnt) * s.Ppair + s.ch_pairs[s.ch_off[c] + r % cnt];
    }
    sgr[q] = g;
  }
  return c;
}

// Ws[r][cc] = W[r][cc] for cc < cols, zero up to ldw.
__device__ inline void stage_w(const float* __restrict__ W, int rows, int cols, float* Ws, int ldw) {
  for (int q = threadIdx.x; q < rows * ldw; q += blockDim.x) {
    const int r = q / ldw, cc = q % ldw;
    Ws[q] = cc < cols ? W[(size_t)r * cols + cc] : 0.f;
  }
}

// Ws[cc][r] = W[r][cc] (the transpose, cols x ldw), zero for r >= rows.
__device__ inline void stage_wt(const float* __restrict__ W, int rows, int cols, float* Ws, int ldw) {
  for (int q = threadIdx.x; q < cols * ldw; q += blockDim.x) {
    const int cc = q / ldw, r = q % ldw;
    Ws[q] = r < rows ? W[(size_t)r * cols + cc] : 0.f;
  }
}

// At[k][q] = src[sgr[q] * ld + off + k] for k < Kin (zero rows past the tile).
__device__ inline void stage_rows_t(const float* __restrict__ src, size_t ld, int off, int Kin, const int* sgr,
                                   float* At) {
  for (int q = threadIdx.x; q < Kin * RB; q += blockDim.x) {
    const int row = q / Kin, k = q % Kin;
    const int g = sgr[row];
    At[k * LA + row] = g >= 0 ? src[(size_t)g * ld + off + k] : 0.f;
  }
}

// acc[i][j] += sum_k At[k][4 ty + i] Bs[k][tx + 16 j].
template <int NJ>
__device__ inline void tile_mm(const float* At, const float* Bs, int ldb, int Kc, int ty, int tx, float acc[4][NJ]) {
#pragma unroll 4
  for (int k = 0; k < Kc; ++k) {
    const float4 a = *(const float4*)(At + k * LA + ty * 4);
    const float* b = Bs + k * ldb + tx;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float bj = b[16 * j];
      acc[0][j] = fmaf(a.x, bj, acc[0][j]);
      acc[1][j] = fmaf(a.y, bj, acc[1][j]);
      acc[2][j] = fmaf(a.z, bj, acc[2][j]);
      acc[3][j] = fmaf(a.w, bj, acc[3][j]);
    }
  }
}

// acc[i][j] = bias[tx + 16 j] (zero past n): products start from the bias,
// as the per-row kernels' sums do, so both give the same float32 rounding.
template <int NJ>
__device__ inline void bias_acc(float acc[4][NJ], const float* __restrict__ bias, int n, int tx) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const float b = tx + 16 * j < n ? bias[tx + 16 * j] : 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][j] = b;
  }
}

template <int NJ>
__device__ inline void zero_acc(float acc[4][NJ]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.f;
}

// ---------------------------------------------------------------- value
template <int NJ>
__global__ void __launch_bounds__(256) k_filter_tile_value(DevSys s, DevNet<float> net, int n,
                                                           const float* __restrict__ ef, int Wn, FTiles ft,
                                                           float* __restrict__ Ah, float* __restrict__ wv,
                                                           int ldw) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int sgr[RB];
  const int K = s.K, Hw = s.Hw, Zd = s.Zd, LW = 16 * NJ;
  float* W1s = fsm;             // [K][LW]
  float* W2s = W1s + K * LW;    // [Hw][LW]
  float* At = W2s + Hw * LW;    // [K][LA]
  float* Ht = At + K * LA;      // [LW][LA]
  const int c = tile_setup(s, ft, Wn, sgr);
  stage_w(net.p + net.off.W1[n][c], K, Hw, W1s, LW);
  stage_w(net.p + net.off.W2[n][c], Hw, Zd, W2s, LW);
  __syncthreads();
  stage_rows_t(ef, (size_t)3 * K, 0, K, sgr, At);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][NJ];
  bias_acc<NJ>(acc, net.p + net.off.b1[n][c], Hw, tx);
  tile_mm<NJ>(At, W1s, LW, K, ty, tx, acc);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int h = tx + 16 * j;
    if (h >= Hw) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = ty * 4 + i, g = sgr[row];
      const float a = acc[i][j];
      if (Ah && g >= 0) Ah[(size_t)g * Hw + h] = a;
      Ht[h * LA + row] = sspf_(a);
    }
  }
  __syncthreads();
  bias_acc<NJ>(acc, net.p + net.off.b2[n][c], Zd, tx);
  tile_mm<NJ>(Ht, W2s, LW, Hw, ty, tx, acc);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int z = tx + 16 * j;
    if (z >= Zd) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = sgr[ty * 4 + i];
      if (g >= 0) wv[(size_t)g * ldw + z] = acc[i][j];
    }
  }
}

// ------------------------------------------------------------------ jet
template <int NJ>
__global__ void __launch_bounds__(256) k_filter_tile_jet(DevSys s, DevNet<float> net, int n,
                                                         const float* __restrict__ ef, int Wn, FTiles ft,
                                                         float* __restrict__ wj) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int sgr[RB];
  const int K = s.K, Hw = s.Hw, Zd = s.Zd, LW = 16 * NJ;
  float* W1s = fsm;                  // [K][LW]
  float* W2s = W1s + K * LW;         // [Hw][LW]
  float* At = W2s + Hw * LW;         // [3][K][LA]: e, e', e''
  float* Ht = At + 3 * K * LA;       // [3][LW][LA]: h, h', h''
  const int c = tile_setup(s, ft, Wn, sgr);
  stage_w(net.p + net.off.W1[n][c], K, Hw, W1s, LW);
  stage_w(net.p + net.off.W2[n][c], Hw, Zd, W2s, LW);
  __syncthreads();
  for (int d = 0; d < 3; ++d) stage_rows_t(ef, (size_t)3 * K, d * K, K, sgr, At + d * K * LA);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float sg[4][NJ];
  {
    float acc[4][NJ];
    bias_acc<NJ>(acc, net.p + net.off.b1[n][c], Hw, tx);
    tile_mm<NJ>(At, W1s, LW, K, ty, tx, acc);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int h = tx + 16 * j;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float a = acc[i][j];
        sg[i][j] = sigmf_(a);
        if (h < Hw) Ht[h * LA + ty * 4 + i] = sspf_(a);
      }
    }
  }
  {
    float a1[4][NJ], a2[4][NJ];
    zero_acc<NJ>(a1);
    zero_acc<NJ>(a2);
    tile_mm<NJ>(At + K * LA, W1s, LW, K, ty, tx, a1);
    tile_mm<NJ>(At + 2 * K * LA, W1s, LW, K, ty, tx, a2);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int h = tx + 16 * j;
      if (h >= Hw) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float q = sg[i][j];
        Ht[(LW + h) * LA + ty * 4 + i] = q * a1[i][j];
        Ht[(2 * LW + h) * LA + ty * 4 + i] = q * a2[i][j] + q * (1.f - q) * a1[i][j] * a1[i][j];
      }
    }
  }
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    float acc[4][NJ];
    if (d == 0)
      bias_acc<NJ>(acc, net.p + net.off.b2[n][c], Zd, tx);
    else
      zero_acc<NJ>(acc);
    tile_mm<NJ>(Ht + d * LW * LA, W2s, LW, Hw, ty, tx, acc);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int z = tx + 16 * j;
      if (z >= Zd) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int g = sgr[ty * 4 + i];
        if (g >= 0) wj[(size_t)g * 3 * Zd + d * Zd + z] = acc[i][j];
      }
    }
  }
}

// --------------------------------------------------------------- bwd
template <int NJ>
__global__ void __launch_bounds__(256) k_filter_tile_bwd(DevSys s, DevNet<float> net, int n,
                                                         const float* __restrict__ Ah, const float* __restrict__ dw,
                                                         int Wn, FTiles ft, float* __restrict__ dAh,
                                                         float* __restrict__ Sh) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int sgr[RB];
  const int Hw = s.Hw, Zd = s.Zd, LW = 16 * NJ;
  float* W2t = fsm;             // [Zd][LW]: W2 transposed
  float* At = W2t + Zd * LW;    // [Zd][LA]: dw rows
  const int c = tile_setup(s, ft, Wn, sgr);
  stage_wt(net.p + net.off.W2[n][c], Hw, Zd, W2t, LW);
  __syncthreads();
  stage_rows_t(dw, (size_t)Zd, 0, Zd, sgr, At);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][NJ];
  zero_acc<NJ>(acc);
  tile_mm<NJ>(At, W2t, LW, Zd, ty, tx, acc);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int h = tx + 16 * j;
    if (h >= Hw) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = sgr[ty * 4 + i];
      if (g < 0) continue;
      const float a = Ah[(size_t)g * Hw + h];
      dAh[(size_t)g * Hw + h] = acc[i][j] * sigmf_(a);
      Sh[(size_t)g * Hw + h] = sspf_(a);
    }
  }
}

// -------------------------------------------------------------- dist
template <int NJ>
__global__ void __launch_bounds__(256) k_filter_tile_dist(DevSys s, DevNet<float> net, int n,
                                                          const float* __restrict__ Ah, const float* __restrict__ ef,
                                                          const float* __restrict__ dw, int Wn, FTiles ft,
                                                          double* __restrict__ dd) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int sgr[RB];
  const int K = s.K, Hw = s.Hw, Zd = s.Zd, LW = 16 * NJ;
  float* W2t = fsm;             // [Zd][LW]
  float* W1s = W2t + Zd * LW;   // [K][LW]
  float* Ad = W1s + K * LW;     // [Zd][LA]: dw rows
  float* Ae = Ad + Zd * LA;     // [K][LA]: e' rows
  const int c = tile_setup(s, ft, Wn, sgr);
  stage_wt(net.p + net.off.W2[n][c], Hw, Zd, W2t, LW);
  stage_w(net.p + net.off.W1[n][c], K, Hw, W1s, LW);
  __syncthreads();
  stage_rows_t(dw, (size_t)Zd, 0, Zd, sgr, Ad);
  stage_rows_t(ef, (size_t)3 * K, K, K, sgr, Ae);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float gacc[4][NJ], qacc[4][NJ];
  zero_acc<NJ>(gacc);
  zero_acc<NJ>(qacc);
  tile_mm<NJ>(Ad, W2t, LW, Zd, ty, tx, gacc);
  tile_mm<NJ>(Ae, W1s, LW, K, ty, tx, qacc);
  double part[4] = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int h = tx + 16 * j;
    if (h >= Hw) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = sgr[ty * 4 + i];
      if (g < 0) continue;
      part[i] += (double)(gacc[i][j] * sigmf_(Ah[(size_t)g * Hw + h])) * (double)qacc[i][j];
    }
  }
  // the 16 threads of a row group are lanes 16 (ty & 1) + tx of one warp
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double v = part[i];
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int g = sgr[ty * 4 + i];
    if (tx == 0 && g >= 0) dd[g] += v;
  }
}

// ---------------------------------------------------------------- host
FTiles tiles_of(const DevSys& s, int Wn) {
  FTiles ft;
  int b = 0;
  for (int c = 0; c < 3; ++c) {
    ft.t0[c] = b;
    const int cnt = s.ch_off[c + 1] - s.ch_off[c];
    b += (int)(((size_t)Wn * cnt + RB - 1) / RB);
  }
  ft.t0[3] = b;
  return ft;
}

int nj_of(const DevSys& s) {
  const int w = std::max(s.Hw, s.Zd);
  return w <= 32 ? 2 : (w <= 64 ? 4 : (w <= 128 ? 8 : 0));
}

int max_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Launch kern<NJ> for the system's NJ with `bytes` of dynamic shared memory.
// ft_work (algorithmic FLOPs of the launch) must be in scope.
#define PN_FT_LAUNCH(NAME, KERN, BYTES_OF, ...)                                                       \
  do {                                                                                               \
    const int nj = nj_of(s);                                                                         \
    if (nj == 0) return PN_ENOTREADY;                                                                \
    const size_t bytes = (BYTES_OF(16 * nj)) * sizeof(float);                                        \
    if (bytes + RB * sizeof(int) + 1024 > (size_t)max_smem()) return PN_ENOTREADY;                   \
    const FTiles ft = tiles_of(s, Wn);                                                               \
    if (ft.t0[3] == 0) return PN_OK;                                                                 \
    switch (nj) {                                                                                    \
      case 2:                                                                                        \
        if (bytes > 48 * 1024)                                                                       \
          PN_CUDA(pn_allow_max_smem(KERN<2>)); \
        PN_LAUNCH_W(NAME, st, ft_work, (KERN<2><<<ft.t0[3], 256, bytes, st>>>(__VA_ARGS__)));                  \
        break;                                                                                       \
      case 4:                                                                                        \
        if (bytes > 48 * 1024)                                                                       \
          PN_CUDA(pn_allow_max_smem(KERN<4>)); \
        PN_LAUNCH_W(NAME, st, ft_work, (KERN<4><<<ft.t0[3], 256, bytes, st>>>(__VA_ARGS__)));                  \
        break;                                                                                       \
      default:                                                                                       \
        if (bytes > 48 * 1024)                                                                       \
          PN_CUDA(pn_allow_max_smem(KERN<8>)); \
        PN_LAUNCH_W(NAME, st, ft_work, (KERN<8><<<ft.t0[3], 256, bytes, st>>>(__VA_ARGS__)));                  \
        break;                                                                                       \
    }                                                                                                \
    return PN_OK;                                                                                    \
  } while (0)

}  // namespace

int pn_filter_tile_value(const DevSys& s, const DevNet<float>& net, int n, const float* ef, int Wn, float* Ah,
                         float* wv, cudaStream_t st) {
#define BYTES(LW) ((size_t)s.K * (LW) + (size_t)s.Hw * (LW) + (size_t)s.K * LA + (size_t)(LW) * LA)
  const double ft_work = 2.0 * Wn * s.Ppair * ((double)s.K * s.Hw + (double)s.Hw * s.Zd);
  PN_FT_LAUNCH("k_filter_tape", k_filter_tile_value, BYTES, s, net, n, ef, Wn, ft, Ah, wv, s.Zd);
#undef BYTES
}

int pn_filter_tile_value_fwd(const DevSys& s, const DevNet<float>& net, int n, const float* ef, int Wn, float* wj,
                             cudaStream_t st) {
#define BYTES(LW) ((size_t)s.K * (LW) + (size_t)s.Hw * (LW) + (size_t)s.K * LA + (size_t)(LW) * LA)
  const double ft_work = 2.0 * Wn * s.Ppair * ((double)s.K * s.Hw + (double)s.Hw * s.Zd);
  // the forward workspace's layout: value rows of [P][3][Zd] filter jets
  PN_FT_LAUNCH("k_filter_value", k_filter_tile_value, BYTES, s, net, n, ef, Wn, ft, (float*)nullptr, wj, 3 * s.Zd);
#undef BYTES
}

int pn_filter_tile_jet(const DevSys& s, const DevNet<float>& net, int n, const float* ef, int Wn, float* wj,
                       cudaStream_t st) {
#define BYTES(LW) ((size_t)s.K * (LW) + (size_t)s.Hw * (LW) + (size_t)3 * s.K * LA + (size_t)3 * (LW) * LA)
  const double ft_work = 6.0 * Wn * s.Ppair * ((double)s.K * s.Hw + (double)s.Hw * s.Zd);
  PN_FT_LAUNCH("k_filter", k_filter_tile_jet, BYTES, s, net, n, ef, Wn, ft, wj);
#undef BYTES
}

int pn_filter_tile_bwd(const DevSys& s, const DevNet<float>& net, int n, const float* Ah, const float* dw, int Wn,
                       float* dAh, float* Sh, cudaStream_t st) {
#define BYTES(LW) ((size_t)s.Zd * (LW) + (size_t)s.Zd * LA)
  const double ft_work = 0;  // not reported
  PN_FT_LAUNCH("k_filter_bwd", k_filter_tile_bwd, BYTES, s, net, n, Ah, dw, Wn, ft, dAh, Sh);
#undef BYTES
}

int pn_filter_tile_dist(const DevSys& s, const DevNet<float>& net, int n, const float* Ah, const float* ef,
                        const float* dw, int Wn, double* dd, cudaStream_t st) {
#define BYTES(LW) ((size_t)s.Zd * (LW) + (size_t)s.K * (LW) + (size_t)s.Zd * LA + (size_t)s.K * LA)
  const double ft_work = 0;  // not reported
  PN_FT_LAUNCH("k_filter_bwd_dist", k_filter_tile_dist, BYTES, s, net, n, Ah, ef, dw, Wn, ft, dd);
#undef BYTES
}
