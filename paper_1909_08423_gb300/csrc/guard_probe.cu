// Perturbations of the guard's second evaluation (the local-energy guard of
// the mixed path): deterministic +-1 signs from a hash of each element's
// index stand in for rounding noise, at the element's own scale (relative)
// or at the scale of the terms that formed it (a linear map's
// sum_k |x_k| |W_kn|).
#include <stdint.h>

#include "pn_internal.cuh"

namespace {

inline unsigned nblk(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Relative perturbation of every element by +-eta, the sign a hash of the
// element's index (a deterministic stand-in for rounding noise).
__global__ void k_perturb(float* __restrict__ A, size_t n, float eta) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = (uint32_t)i * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  A[i] *= (h & 1u) ? 1.0f + eta : 1.0f - eta;
}

// Perturbation of a linear map's output at the scale of its terms: for
// every element y[row][n] of Y = X W, y += (+-1) * (eta_rel |y| + eta_abs
// sum_k |x[row][k]| |W[k][n]|) (sign a hash of the element's index, the same
// as k_perturb's).  Rounding in the map, and rounding carried in from its
// input, enters y at the second scale and not at |y|, which cancellation can
// make far smaller.  A block takes 128 rows, a thread one row: |W| in shared
// memory (every thread reads the same weight: broadcast), the rows' |x| staged
// 32 columns at a time by coalesced loads (row stride 33: conflict-free),
// outputs in chunks of 16 registers.
constexpr int PB_ROWS = 128, PB_KC = 32;
__global__ void __launch_bounds__(PB_ROWS) k_perturb_abs(const float* __restrict__ X, int ldx,
                                                         const float* __restrict__ W, int ldw, float* __restrict__ Y,
                                                         int ldy, int rows, int Kd, int Nout, float eta_rel,
                                                         float eta_abs) {
  extern __shared__ __align__(16) float pb_sm[];
  const int NP = (Nout + 15) & ~15;    // |W| rows padded with zeros to whole chunks
  float* wabs = pb_sm;                 // [Kd][NP]
  float* xs = pb_sm + Kd * NP;         // [PB_ROWS][PB_KC + 1]
  for (int q = threadIdx.x; q < Kd * NP; q += PB_ROWS) {
    const int k = q / NP, n = q - k * NP;
    wabs[q] = n < Nout ? fabsf(W[(size_t)k * ldw + n]) : 0.f;
  }
  const int row0 = blockIdx.x * PB_ROWS, row = row0 + threadIdx.x;
  for (int n0 = 0; n0 < Nout; n0 += 16) {
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.f;
    for (int k0 = 0; k0 < Kd; k0 += PB_KC) {
      __syncthreads();  // the previous slice (and, first, |W|) complete
      // all of a thread's loads in flight before its stores
      float v[PB_KC];
#pragma unroll
      for (int u = 0; u < PB_KC; ++u) {
        const int q = threadIdx.x + u * PB_ROWS, r = q / PB_KC, c = q - r * PB_KC;
        v[u] = (row0 + r < rows && k0 + c < Kd) ? fabsf(X[(size_t)(row0 + r) * ldx + k0 + c]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < PB_KC; ++u) {
        const int q = threadIdx.x + u * PB_ROWS, r = q / PB_KC, c = q - r * PB_KC;
        xs[r * (PB_KC + 1) + c] = v[u];
      }
      __syncthreads();
      const int kn = min(PB_KC, Kd - k0);
      for (int c = 0; c < kn; ++c) {
        const float ax = xs[threadIdx.x * (PB_KC + 1) + c];
        const float4* wk = (const float4*)(wabs + (k0 + c) * NP + n0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 w4 = wk[q];
          acc[4 * q] = fmaf(ax, w4.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(ax, w4.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(ax, w4.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(ax, w4.w, acc[4 * q + 3]);
        }
      }
    }
    if (row < rows) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + j;
        if (n >= Nout) break;
        uint32_t h = (uint32_t)((size_t)row * Nout + n) * 0x9E3779B1u;
        h ^= h >> 15;
        h *= 0x85EBCA77u;
        h ^= h >> 13;
        float* y = Y + (size_t)row * ldy + n;
        const float d = fmaf(eta_rel, fabsf(*y), eta_abs * acc[j]);
        *y += (h & 1u) ? d : -d;
      }
    }
  }
}

}  // namespace

int pn_perturb_abs(const float* X, int ldx, const float* W, int ldw, float* Y, int ldy, size_t rows, int Kd,
                          int Nout, float eta_rel, float eta_abs, cudaStream_t st) {
  if (rows == 0) return PN_OK;
  if (rows > (size_t)INT32_MAX - PB_ROWS) {
    pn_set_error("guard probe: %zu rows exceed the kernel's index range", rows);
    return PN_EINVAL;
  }
  const size_t smem = ((size_t)Kd * ((Nout + 15) & ~15) + (size_t)PB_ROWS * (PB_KC + 1)) * sizeof(float);
  if (smem > 48 * 1024) PN_CUDA(pn_allow_max_smem(k_perturb_abs));
  PN_LAUNCH("k_perturb", st, k_perturb_abs<<<(unsigned)((rows + PB_ROWS - 1) / PB_ROWS), PB_ROWS, smem, st>>>(
                                 X, ldx, W, ldw, Y, ldy, (int)rows, Kd, Nout, eta_rel, eta_abs));
  return PN_OK;
}


// y += (+-1) (eta_rel |y| + eta_abs S) with S the term scale already formed
// (by the tensor-core map in absolute-value mode), S rows of stride lds.
static __global__ void k_perturb_apply(float* __restrict__ Y, int ldy, const float* __restrict__ S, int lds, size_t rows,
                                int Nout, float eta_rel, float eta_abs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * Nout) return;
  const size_t row = idx / Nout;
  const int n = (int)(idx - row * Nout);
  uint32_t h = (uint32_t)idx * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA77u;
  h ^= h >> 13;
  float* y = Y + row * ldy + n;
  const float d = fmaf(eta_rel, fabsf(*y), eta_abs * S[row * lds + n]);
  *y += (h & 1u) ? d : -d;
}

int pn_perturb_abs_tc(const float* X, int ldx, const float* W, int ldw, float* Y, int ldy, size_t rows, int Kd,
                      int Nout, float eta_rel, float eta_abs, float* scratch, size_t scratch_floats, int* err,
                      cudaStream_t st) {
  if (rows == 0) return PN_OK;
  if (rows * (size_t)Nout > scratch_floats || rows > (size_t)INT32_MAX) return PN_ENOTREADY;
  const int e = pn_linear_tc(X, ldx, W, ldw, nullptr, scratch, Nout, (int)rows, Kd, Nout, 1, 0, err, st, 1);
  if (e) return e;
  PN_LAUNCH("k_perturb", st, k_perturb_apply<<<nblk(rows * Nout, 256), 256, 0, st>>>(Y, ldy, scratch, Nout, rows, Nout,
                                                                                     eta_rel, eta_abs));
  return PN_OK;
}

int pn_perturb_rel(float* A, size_t n, float eta, cudaStream_t st) {
  if (n == 0) return PN_OK;
  PN_LAUNCH("k_perturb", st, k_perturb<<<nblk(n, 256), 256, 0, st>>>(A, n, eta));
  return PN_OK;
}
