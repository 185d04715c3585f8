// Dense network layers on the 5th-generation tensor cores (tcgen05).
//
// Y (=|+=) X W + b, with b added on value rows (row % T == 0) of a jet,
// for float32 X [rows][K] and W [K][Nout].  Each CTA owns 128 rows and all
// output columns: operands are staged in shared memory in the canonical
// K-major layout without swizzle (8 x 16-byte core matrices), one thread
// issues tcgen05.mma for the CTA, the accumulator lives in tensor memory
// (TMEM) and comes back through tcgen05.ld for the epilogue.
//
// Precision: each float32 operand is split into three bfloat16 pieces
// a = a0 + a1 + a2 (each the nearest bf16 of what is left), which together
// carry 24 mantissa bits, and the product is formed from the six pieces
// whose weight reaches 2^-16: a0b0, a0b1, a1b0, a0b2, a2b0, a1b1, with
// float32 accumulation in tensor memory.  That keeps the float32 accuracy
// the local-energy bound needs; plain bf16 or tf32 loses 16 or 13 bits, and
// a two-piece tf32 split still loses about 3.
//
// Every wait on the MMA completion barrier is bounded; on expiry the kernel
// records a flag, waits (bounded) once more, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "pn_internal.cuh"

namespace {

constexpr int TC_M = 128;    // rows per CTA (UMMA M)
constexpr int TC_KC = 32;    // K elements staged per round
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_LBO = 128;              // bytes between core matrices along K
constexpr uint32_t TC_SBO = TC_KC / 8 * 128;  // bytes between 8-row groups (8 bf16 per core row)
constexpr int TC_PIECES = 3;

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (sm_100 family): start address, leading
// and stride byte offsets (all >> 4), version 1, no swizzle.
__device__ inline uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor (kind::f16): f32 accumulator, bf16 A and B, both
// K-major.
__host__ __device__ inline uint32_t bf16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of bf16 element (row, k) inside a staged tile
__device__ inline uint32_t tile_off(int row, int k) {
  return (uint32_t)(row >> 3) * TC_SBO + (uint32_t)(k >> 3) * TC_LBO + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// a -> three bf16 pieces, nearest rounding at each stage
__device__ inline void split3(float a, unsigned short p[3]) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r2);
  p[0] = __bfloat16_as_ushort(h0);
  p[1] = __bfloat16_as_ushort(h1);
  p[2] = __bfloat16_as_ushort(h2);
}

__device__ inline bool mbar_try(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ inline bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try(bar, phase)) return true;
  return false;
}

__global__ void __launch_bounds__(TC_THREADS) k_linear_tc(const float* __restrict__ X, int ldx,
                                                          const float* __restrict__ Wt, int ldw,
                                                          const float* __restrict__ bias, float* __restrict__ Y,
                                                          int ldy, int rows, int K, int Nout, int Npad, int T,
                                                          int accumulate, uint32_t tmem_cols,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  // pieces 0..2 of the A tile (128 x KC bf16), then of the B tile (Npad x KC)
  const uint32_t a_bytes = TC_M * TC_KC * 2, b_bytes = (uint32_t)Npad * TC_KC * 2;
  unsigned char* sA = smem;
  unsigned char* sB = smem + TC_PIECES * a_bytes;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t bar = smem_u32(&mbar);
  const uint32_t idesc = bf16_idesc(TC_M, Npad);
  uint32_t phase = 0;
  bool ok = true;

  for (int k0 = 0; k0 < K && ok; k0 += TC_KC) {
    // stage A (128 x KC) and B (Npad x KC, from W[k][n]) as three bf16 pieces
    for (int idx = tid; idx < TC_M * TC_KC; idx += TC_THREADS) {
      const int row = idx / TC_KC, k = idx % TC_KC;
      const int gr = m0 + row, gk = k0 + k;
      const float a = (gr < rows && gk < K) ? X[(size_t)gr * ldx + gk] : 0.0f;
      unsigned short p[3];
      split3(a, p);
      const uint32_t off = tile_off(row, k);
      for (int q = 0; q < TC_PIECES; ++q) *(unsigned short*)(sA + q * a_bytes + off) = p[q];
    }
    for (int idx = tid; idx < Npad * TC_KC; idx += TC_THREADS) {
      const int n = idx % Npad, k = idx / Npad;
      const int gk = k0 + k;
      const float b = (n < Nout && gk < K) ? Wt[(size_t)gk * ldw + n] : 0.0f;
      unsigned short p[3];
      split3(b, p);
      const uint32_t off = tile_off(n, k);
      for (int q = 0; q < TC_PIECES; ++q) *(unsigned short*)(sB + q * b_bytes + off) = p[q];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      // (A piece, B piece) pairs whose weight reaches 2^-16, smallest first
      const int pa[6] = {1, 2, 0, 1, 0, 0};
      const int pb[6] = {1, 0, 2, 0, 1, 0};
      for (int s = 0; s < TC_KC / 16; ++s) {
        const uint32_t step = (uint32_t)s * 2u * TC_LBO;  // 16 bf16 = two core matrices along K
        for (int t = 0; t < 6; ++t) {
          const uint64_t da = smem_desc(a0 + pa[t] * a_bytes + step);
          const uint64_t db = smem_desc(b0 + pb[t] * b_bytes + step);
          const uint32_t acc_in = (k0 == 0 && s == 0 && t == 0) ? 0u : 1u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc_in));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    mbar_wait_bounded(bar, phase ^ 1u);  // give in-flight MMAs a last bounded chance
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w reads TMEM lanes 32w..32w+31 = rows m0 + 32w + lane,
    // 16 columns at a time, and writes them out through a shared-memory
    // transpose so that each store instruction covers whole row segments
    float* tr = (float*)smem + warp * 32 * 17;  // staging area is free now
    for (int c0 = 0; c0 < Npad; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) tr[lane * 17 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int jj = lane & 15;
      const int col = c0 + jj;
      for (int rr = lane >> 4; rr < 32; rr += 2) {
        const int row = m0 + warp * 32 + rr;
        if (row < rows && col < Nout) {
          const float y = tr[rr * 17 + jj] + ((bias && (row % T) == 0) ? bias[col] : 0.0f);
          float* dst = Y + (size_t)row * ldy + col;
          *dst = accumulate ? *dst + y : y;
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

int* g_tc_err = nullptr;  // device flag per process (allocated on first use)

}  // namespace

size_t pn_tc_smem_bytes(int Nout) {
  const int Npad = ((Nout + 15) / 16) * 16;
  return (size_t)TC_PIECES * (TC_M + Npad) * TC_KC * 2;
}

bool pn_tc_supported(int Nout) { return Nout >= 1 && Nout <= 256; }

int pn_linear_tc(const float* X, int ldx, const float* W, int ldw, const float* b, float* Y, int ldy, int rows, int K,
                 int Nout, int T, int acc, int* err, cudaStream_t st) {
  if (rows <= 0) return PN_OK;
  if (!pn_tc_supported(Nout)) { pn_set_error("tensor-core linear: Nout %d outside 1..256", Nout); return PN_EINVAL; }
  const int Npad = ((Nout + 15) / 16) * 16;
  uint32_t cols = 32;
  while ((int)cols < Npad) cols <<= 1;
  const size_t smem = pn_tc_smem_bytes(Nout);
  PN_CUDA(cudaFuncSetAttribute(k_linear_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int blocks = (rows + TC_M - 1) / TC_M;
  PN_LAUNCH_W("k_linear_tc", st, 2.0 * rows * K * Nout,
            k_linear_tc<<<blocks, TC_THREADS, smem, st>>>(X, ldx, W, ldw, b, Y, ldy, rows, K, Nout, Npad, T, acc, cols,
                                                          err));
  return PN_OK;
}

// Self-test entry: one GEMM on caller buffers, synchronised, with the
// completion-wait flag checked.
extern "C" int pn_test_linear_tc(const float* X, int ldx, const float* W, int ldw, const float* b, float* Y, int ldy,
                                 int rows, int K, int Nout, int T, int accumulate, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!g_tc_err) {
    PN_CUDA(cudaMalloc((void**)&g_tc_err, sizeof(int)));
  }
  PN_CUDA(cudaMemsetAsync(g_tc_err, 0, sizeof(int), st));
  if (int e = pn_linear_tc(X, ldx, W, ldw, b, Y, ldy, rows, K, Nout, T, accumulate, g_tc_err, st)) return e;
  int h = 0;
  PN_CUDA(cudaMemcpyAsync(&h, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PN_CUDA(cudaStreamSynchronize(st));
  if (h) {
    pn_set_error("tensor-core linear: MMA completion wait expired");
    return PN_ETIMEOUT;
  }
  return PN_OK;
}
