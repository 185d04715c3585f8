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
// float32 accumulation in tensor memory -- the leading a0b0 terms in an
// accumulator of their own, the five smaller ones in a second, added in the
// epilogue.  That keeps the float32 accuracy
// the local-energy bound needs; plain bf16 or tf32 loses 16 or 13 bits, and
// a two-piece tf32 split still loses about 3.
//
// Every wait on the MMA completion barrier is bounded; on expiry the kernel
// records a flag, waits (bounded) once more, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "pn_internal.cuh"

namespace {

constexpr int TC_M = 128;       // rows per tile (UMMA M)
constexpr int TC_KC = 32;       // k-slice per pipeline stage
constexpr int TC_NPROD = 16;    // producer warps
constexpr int TC_NEPI = 4;      // epilogue warps
constexpr int TC_WMMA = TC_NPROD;                      // the warp after the producers issues the MMAs
constexpr int TC_CELLS = TC_M * TC_KC / 8 / (32 * TC_NPROD);  // (row, 8-wide k group) cells per producer thread
static_assert(TC_CELLS >= 1 && TC_CELLS * 8 * 32 * TC_NPROD == TC_M * TC_KC, "producers must tile a stage");
constexpr int TC_THREADS = 32 * (TC_NPROD + 1 + TC_NEPI);
constexpr uint32_t TC_LBO = 128;                       // bytes between core matrices along K
constexpr uint32_t TC_SBO_A = TC_KC / 8 * 128;         // bytes between 8-row groups of an A stage
constexpr uint32_t TC_STAGE = 3u * TC_M * TC_KC * 2;   // three bf16 pieces of a 128 x 32 slice
constexpr int TC_SPIN = 1 << 22;                       // polls per bounded wait

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (sm_100 family): start address, leading
// and stride byte offsets (all >> 4), version 1, no swizzle.
__device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor (kind::f16): f32 accumulator, bf16 A and B, both
// K-major.
__host__ __device__ inline uint32_t bf16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of bf16 element (row, k) in a K-major tile whose 8-row groups
// are sbo bytes apart
__device__ inline uint32_t tile_off(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * TC_LBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// a -> three bf16 pieces, nearest rounding at each stage
__device__ inline void split3(float a, unsigned short& p0, unsigned short& p1, unsigned short& p2) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r2);
  p0 = __bfloat16_as_ushort(h0);
  p1 = __bfloat16_as_ushort(h1);
  p2 = __bfloat16_as_ushort(h2);
}

// Two floats -> their three pieces as packed bf16x2 words (the lower half
// from a, the upper from b): one conversion instruction per piece and pair;
// the same pieces as split3.
__device__ inline void split3x2(float a, float b, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w0) : "f"(b), "f"(a));
  const float ra = a - __uint_as_float(w0 << 16), rb = b - __uint_as_float(w0 & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w1) : "f"(rb), "f"(ra));
  const float sa = ra - __uint_as_float(w1 << 16), sb = rb - __uint_as_float(w1 & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w2) : "f"(sb), "f"(sa));
}

__device__ inline bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait that also gives up once another role of the CTA has given
// up (*abort set); returns false then.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  for (int it = 0; it < TC_SPIN; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  *abort = 1;
  return false;
}

// Y (=|+=) X W + b on value rows; see the file comment.  VX: X rows are
// 16-byte aligned (float4 loads).  absval: |X| |W| instead (the scale of the
// product's terms, for the local-energy guard's probe).
template <bool VX>
__global__ void __launch_bounds__(TC_THREADS, 1) k_linear_tc(const float* __restrict__ X, int ldx,
                                                              const float* __restrict__ Wt, int ldw,
                                                              const float* __restrict__ bias, float* __restrict__ Y,
                                                              int ldy, int rows, int K, int Kp, int Nout, int Npad,
                                                              int T, int accumulate, int nstage, uint32_t tmem_cols,
                                                              int vy, int nbuf, int* __restrict__ err, int absval) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2 * 8 + 4 + 1];  // full[8], empty[8], acc_full[2], acc_empty[2], drain
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_piece = (uint32_t)Npad * Kp * 2;         // bytes of one weight piece
  const uint32_t sbo_b = (uint32_t)(Kp / 8) * 128u;
  unsigned char* sB = smem;                                  // 3 weight pieces [Npad][Kp]
  unsigned char* sA = smem + 3 * b_piece;                    // nstage x 3 pieces [128][KC]
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[8]);
  const uint32_t accf0 = smem_u32(&bars[16]), acce0 = smem_u32(&bars[18]), drain = smem_u32(&bars[20]);
  const int ntiles = (rows + TC_M - 1) / TC_M;
  const int nk = Kp / TC_KC;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstage; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * s), "r"(TC_NPROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf0 + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acce0 + 8 * b), "r"(TC_NEPI));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(drain));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == TC_WMMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the weight's three pieces, once per CTA: B is [Npad][Kp] K-major
  for (int idx = tid; idx < Npad * Kp; idx += TC_THREADS) {
    const int n = idx / Kp, k = idx - n * Kp;
    float b = (n < Nout && k < K) ? Wt[(size_t)k * ldw + n] : 0.0f;
    if (absval) b = fabsf(b);
    unsigned short p0, p1, p2;
    split3(b, p0, p1, p2);
    const uint32_t off = tile_off(n, k, sbo_b);
    *(unsigned short*)(sB + off) = p0;
    *(unsigned short*)(sB + b_piece + off) = p1;
    *(unsigned short*)(sB + 2 * b_piece + off) = p2;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  volatile int* abort = &abort_flag;

  if (warp < TC_NPROD) {
    // ---------------------------------------------------------- producers
    // thread p owns TC_CELLS (row, 8-wide k group) cells of every stage; its
    // global loads run two stages ahead of the splitting and storing, so
    // that enough bytes are in flight to cover the memory latency.  A warp
    // takes one 8-row group: its lanes 8q..8q+7 store rows 0..7 of k group
    // q, one 128-byte core matrix per quarter-warp (16-byte stores without
    // bank conflicts)
    const int p = tid;  // 0 .. 32 TC_NPROD - 1
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nstages_total = my_tiles * nk;
    auto load = [&](int gg, float* dst) {
      const int tile = blockIdx.x + (gg / nk) * gridDim.x;
      const int k0 = (gg % nk) * TC_KC;
      const int r0 = tile * TC_M;
#pragma unroll
      for (int j = 0; j < TC_CELLS; ++j) {
        const int idx = p + 32 * TC_NPROD * j;
        const int row = ((idx >> 5) << 3) | (idx & 7), gk = ((idx >> 3) & 3) * 8;
        const int gr = r0 + row;
        if (VX && gr < rows && k0 + gk + 8 <= K) {
          const float4* src = (const float4*)(X + (size_t)gr * ldx + k0 + gk);
          const float4 a = src[0], b = src[1];
          dst[8 * j + 0] = a.x; dst[8 * j + 1] = a.y; dst[8 * j + 2] = a.z; dst[8 * j + 3] = a.w;
          dst[8 * j + 4] = b.x; dst[8 * j + 5] = b.y; dst[8 * j + 6] = b.z; dst[8 * j + 7] = b.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = k0 + gk + e;
            dst[8 * j + e] = (gr < rows && k < K) ? X[(size_t)gr * ldx + k] : 0.0f;
          }
        }
      }
    };
    bool alive = true;
    // stage g from cur while stage g + 2 loads into pf
    auto step = [&](int g, const float* cur, float* pf) {
      if (!alive || g >= nstages_total) return;
      if (g + 2 < nstages_total) load(g + 2, pf);
      const int s = g % nstage;
      if (!mbar_wait(empty0 + 8 * s, ((g / nstage) & 1) ^ 1, abort)) { alive = false; return; }
      unsigned char* st = sA + (size_t)s * TC_STAGE;
#pragma unroll
      for (int j = 0; j < TC_CELLS; ++j) {
        const int idx = p + 32 * TC_NPROD * j;
        const int row = ((idx >> 5) << 3) | (idx & 7), gk = ((idx >> 3) & 3) * 8;
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float x0 = cur[8 * j + 2 * e], x1 = cur[8 * j + 2 * e + 1];
          split3x2(absval ? fabsf(x0) : x0, absval ? fabsf(x1) : x1, w0[e], w1[e], w2[e]);
        }
        const uint32_t off = tile_off(row, gk, TC_SBO_A);
        *(uint4*)(st + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *(uint4*)(st + TC_M * TC_KC * 2 + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *(uint4*)(st + 2 * TC_M * TC_KC * 2 + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(full0 + 8 * s);
    };
    float va[8 * TC_CELLS], vb[8 * TC_CELLS], vc[8 * TC_CELLS];
    if (nstages_total > 0) load(0, va);
    if (nstages_total > 1) load(1, vb);
    for (int g = 0; g < nstages_total && alive; g += 3) {
      step(g, va, vc);
      step(g + 1, vb, va);
      step(g + 2, vc, vb);
    }
  } else if (warp == TC_WMMA) {
    // --------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = bf16_idesc(TC_M, Npad);
      const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
      // (A piece, B piece) pairs whose weight reaches 2^-16, smallest first
      constexpr int pa[6] = {1, 2, 0, 1, 0, 0};
      constexpr int pb[6] = {1, 0, 2, 0, 1, 0};
      // Descriptors: the start-address field holds the byte address >> 4 in
      // its low 14 bits and shared memory ends below 2^18 bytes, so the
      // descriptor of base + offset is the base's plus offset >> 4 (no
      // carry).  Base descriptors once, the per-MMA offsets from constants.
      const uint64_t da0 = smem_desc(a_base, TC_SBO_A), db0 = smem_desc(b_base, sbo_b);
      uint32_t ob[TC_KC / 16][6];
#pragma unroll
      for (int ks = 0; ks < TC_KC / 16; ++ks)
#pragma unroll
        for (int q = 0; q < 6; ++q) ob[ks][q] = (uint32_t)(pb[q] * b_piece + ks * 2u * TC_LBO) >> 4;
      int g = 0, it = 0;
      bool issued = false;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int buf = it % nbuf;
        if (!mbar_wait(acce0 + 8 * buf, ((it / nbuf) & 1) ^ 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // the five smaller piece products accumulate at dt, the leading
        // a0 b0 products at dt + Npad: the long accumulation of the large
        // terms then takes one rounding per k-step instead of six
        const uint32_t dt = tmem + (uint32_t)(buf * 2 * Npad);
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int s = g % nstage;
          if (!mbar_wait(full0 + 8 * s, (g / nstage) & 1, abort)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t da_s = da0 + (((uint32_t)s * TC_STAGE) >> 4);
          const uint64_t db_k = db0 + (((uint32_t)kc * (TC_KC / 16) * 2u * TC_LBO) >> 4);
#pragma unroll
          for (int ks = 0; ks < TC_KC / 16; ++ks) {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const uint64_t da = da_s + ((uint32_t)(pa[q] * (TC_M * TC_KC * 2) + ks * 2 * TC_LBO) >> 4);
              const uint64_t db = db_k + ob[ks][q];
              const bool big = q == 5;  // (a0, b0)
              const uint32_t acc_in = (kc == 0 && ks == 0 && (q == 0 || big)) ? 0u : 1u;
              const uint32_t d = big ? dt + (uint32_t)Npad : dt;
              asm volatile(
                  "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                  "l"(da), "l"(db), "r"(idesc), "r"(acc_in));
            }
          }
          issued = true;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           empty0 + 8 * s)
                       : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(accf0 + 8 * buf)
                     : "memory");
      }
      // every MMA issued has completed before the TMEM is freed
      if (issued) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain)
                     : "memory");
        for (int k = 0; k < TC_SPIN && !mbar_try(drain, 0); ++k) {
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    const int quarter = warp & 3;  // TMEM lanes 32 quarter .. 32 quarter + 31
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int buf = it % nbuf;
      if (!mbar_wait(accf0 + 8 * buf, (it / nbuf) & 1, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int row = tile * TC_M + quarter * 32 + lane;
      const bool val = (row % T) == 0;
      for (int c0 = 0; c0 < Npad; c0 += 16) {
        uint32_t v[16], u[16];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 2 * Npad + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
              "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
            : "r"(taddr + (uint32_t)Npad));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(u[j]));
        if (row < rows) {
          float* yr = Y + (size_t)row * ldy;
          if (vy && c0 + 16 <= Nout) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              float4 y = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                                     __uint_as_float(v[j + 3]));
              if (bias && val) {
                y.x += bias[c0 + j]; y.y += bias[c0 + j + 1]; y.z += bias[c0 + j + 2]; y.w += bias[c0 + j + 3];
              }
              if (accumulate) {
                const float4 o = *(const float4*)(yr + c0 + j);
                y.x += o.x; y.y += o.y; y.z += o.z; y.w += o.w;
              }
              *(float4*)(yr + c0 + j) = y;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = c0 + j;
              if (col < Nout) {
                float y = __uint_as_float(v[j]) + ((bias && val) ? bias[col] : 0.0f);
                if (accumulate) y += yr[col];
                yr[col] = y;
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * buf);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (abort_flag && tid == 0) atomicExch(err, 1);
  if (warp == TC_WMMA) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  }
}

int* g_tc_err = nullptr;  // device flag per process (allocated on first use)

// Shared memory of a launch: the weight's pieces plus as many pipeline
// stages (2..8) as fit; 0 if fewer than two fit.
size_t tc_plan(int K, int Nout, int* Kp_out, int* nstage_out) {
  const int Kp = ((K + TC_KC - 1) / TC_KC) * TC_KC;
  const int Npad = ((Nout + 15) / 16) * 16;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t wbytes = (size_t)3 * Npad * Kp * 2;
  const size_t room = (size_t)maxsm - 1024;  // static shared memory and slack
  if (wbytes + 2 * TC_STAGE > room) return 0;
  const int ns = (int)std::min<size_t>(8, (room - wbytes) / TC_STAGE);
  *Kp_out = Kp;
  *nstage_out = ns;
  return wbytes + (size_t)ns * TC_STAGE;
}

}  // namespace

bool pn_tc_supported(int Nout) { return Nout >= 1 && Nout <= 256; }

int pn_linear_tc(const float* X, int ldx, const float* W, int ldw, const float* b, float* Y, int ldy, int rows, int K,
                 int Nout, int T, int acc, int* err, cudaStream_t st, int absval) {
  if (rows <= 0) return PN_OK;
  if (!pn_tc_supported(Nout)) { pn_set_error("tensor-core linear: Nout %d outside 1..256", Nout); return PN_EINVAL; }
  int Kp = 0, ns = 0;
  const size_t smem = tc_plan(K, Nout, &Kp, &ns);
  if (!smem) return PN_ENOTREADY;  // weight too large to stay resident: the caller uses CUDA cores
  const int Npad = ((Nout + 15) / 16) * 16;
  // two accumulators per tile; two tiles in flight where TMEM holds them
  const int nbuf = 4 * Npad <= 512 ? 2 : 1;
  uint32_t cols = 32;
  while ((int)cols < 2 * nbuf * Npad) cols <<= 1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (rows + TC_M - 1) / TC_M;
  const int grid = std::min(tiles, sms);
  const bool vx = ldx % 4 == 0 && ((uintptr_t)X & 15) == 0;
  const int vy = ldy % 4 == 0 && ((uintptr_t)Y & 15) == 0;
  if (vx) {
    PN_CUDA(pn_allow_max_smem(k_linear_tc<true>));
    PN_LAUNCH_WB("k_linear_tc", st, 2.0 * rows * K * Nout, 4.0 * rows * (K + Nout * (acc ? 2 : 1)),
                (k_linear_tc<true><<<grid, TC_THREADS, smem, st>>>(X, ldx, W, ldw, b, Y, ldy, rows, K, Kp, Nout, Npad, T,
                                                                   acc, ns, cols, vy, nbuf, err, absval)));
  } else {
    PN_CUDA(pn_allow_max_smem(k_linear_tc<false>));
    PN_LAUNCH_WB("k_linear_tc", st, 2.0 * rows * K * Nout, 4.0 * rows * (K + Nout * (acc ? 2 : 1)),
                (k_linear_tc<false><<<grid, TC_THREADS, smem, st>>>(X, ldx, W, ldw, b, Y, ldy, rows, K, Kp, Nout, Npad,
                                                                    T, acc, ns, cols, vy, nbuf, err, absval)));
  }
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
