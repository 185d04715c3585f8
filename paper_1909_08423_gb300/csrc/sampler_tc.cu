// Metropolis sampler with the network on the 5th-generation tensor cores.
//
// One CTA (sixteen warps) owns a tile of WT walkers, so that its electrons
// (WT * N <= 128) and the pairs of each filter channel (WT * count <= 128)
// each fill one 128-row tcgen05 tile.  Every linear map of every step is
// one or a few tcgen05.mma groups over the whole tile:
//  - activations are written by the CUDA cores into shared memory as three
//    bf16 pieces in the canonical K-major layout (8 x 16-byte core
//    matrices), weights arrive the same way by a TMA bulk copy of a block
//    prepared at parameter upload, triple-buffered two stages ahead;
//  - the weight pieces of a block lie one after another, which is itself a
//    canonical tile of 3 Np rows, so one thread issues per 16-wide k-step
//    three MMAs, a0 [b0; b1; b2], a1 [b0; b1] and a2 b0, accumulating the
//    products with b0, b1, b2 in three float32 column blocks of tensor
//    memory (the six products of the split, three instructions), and
//    commits to an mbarrier (an MMA costs about the same whatever its N);
//  - warps w, w + 4, w + 8, w + 12 read TMEM lanes 32(w % 4)..+31 (their
//    32 rows), taking every fourth 8-column chunk, sum the three column
//    blocks (smallest first) and apply bias and activation, writing the
//    next operand or float state.
// h of the first layer is one row for every electron (x^(0) is shared), so
// it is formed once per launch and its GEMM is not in the stage list.
// Geometry, orbitals (float32), features, messages, determinants (float64
// LU; each determinant kept as mantissa x 2^exponent so that the signed sum
// over determinants needs one logarithm per walker) and the accept test run
// on the CUDA cores between the MMA stages.  Every wait is bounded: on expiry the CTA raises the device error
// word, drains what it started (bounded) and frees its TMEM.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "ansatz_dev.cuh"
#include "kernels.cuh"
#include "pn_internal.cuh"

namespace {

constexpr int TM = 128;  // tile rows
constexpr int NT = 512;        // threads
constexpr int WPQ = NT / 128;  // warps per TMEM lane quadrant

__device__ inline uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major canonical layout: 8-row groups SBO = K/8 * 128 bytes apart, core
// matrices along K 128 bytes apart.
__device__ inline uint32_t t_off(int row, int k, int K) {
  return (uint32_t)(row >> 3) * (uint32_t)(K >> 3) * 128u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

__device__ inline uint64_t sdesc(uint32_t addr, int K) {
  const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ inline uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// Eight consecutive k of one row -> one 16-byte store per bf16 piece (one
// row of a core matrix).  k8 is a multiple of 8.  The split truncates: the
// high 16 bits of a float are a bf16 (8 significant bits), the remainder
// a - hi is exact and has at most 16 significant bits, and so on, so that
// a = a0 + a1 + a2 exactly for every normal float.  Pairs are packed with
// the even k in the low half.
__device__ inline void put3x8(unsigned char* A, int piece_bytes, int row, int k8, int K, const float v[8]) {
  uint32_t w0[4], w1[4], w2[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t ua = __float_as_uint(v[2 * j]), ub = __float_as_uint(v[2 * j + 1]);
    const float ra = v[2 * j] - __uint_as_float(ua & 0xFFFF0000u), rb = v[2 * j + 1] - __uint_as_float(ub & 0xFFFF0000u);
    const uint32_t ura = __float_as_uint(ra), urb = __float_as_uint(rb);
    const float qa = ra - __uint_as_float(ura & 0xFFFF0000u), qb = rb - __uint_as_float(urb & 0xFFFF0000u);
    w0[j] = __byte_perm(ua, ub, 0x7632);
    w1[j] = __byte_perm(ura, urb, 0x7632);
    w2[j] = __byte_perm(__float_as_uint(qa), __float_as_uint(qb), 0x7632);
  }
  const uint32_t off = t_off(row, k8, K);
  *(uint4*)(A + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  *(uint4*)(A + piece_bytes + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  *(uint4*)(A + 2 * piece_bytes + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

__device__ inline bool try_bar(uint32_t bar, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(par)
      : "memory");
  return ok != 0;
}
__device__ inline bool wait_bar(uint32_t bar, uint32_t par) {
  for (int it = 0; it < (1 << 22); ++it)
    if (try_bar(bar, par)) return true;
  return false;
}

// Shifted softplus ln(1 + e^x) - ln 2 = max(x, 0) + log1p(e^-|x|) - ln 2, with
// log1p(t) = 2 artanh(t / (2 + t)) summed as the Taylor series of artanh:
// s = t / (2 + t) <= 1/3 on t in (0, 1], and the terms up to s^13 / 13 leave
// a relative remainder below 2e-8.
__device__ inline float sspf(float x) {
  const float t = __expf(-fabsf(x));
  const float s = __fdividef(t, 2.f + t);
  const float s2 = s * s;
  float q = 1.f / 13.f;
  q = fmaf(q, s2, 1.f / 11.f);
  q = fmaf(q, s2, 1.f / 9.f);
  q = fmaf(q, s2, 1.f / 7.f);
  q = fmaf(q, s2, 1.f / 5.f);
  q = fmaf(q, s2, 1.f / 3.f);
  q = fmaf(q, s2, 1.f);
  return fmaxf(x, 0.f) + 2.f * s * q - 0.69314718055994530942f;
}

// Eight consecutive fp32 columns of this thread's TMEM lane, summed over the
// three product blocks at taddr, taddr + np, taddr + 2 np (b2 + b1 + b0).
__device__ inline void tmem_ld8x3(uint32_t taddr, uint32_t np, float v[8]) {
  uint32_t u0[8], u1[8], u2[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(u0[0]), "=r"(u0[1]), "=r"(u0[2]), "=r"(u0[3]), "=r"(u0[4]), "=r"(u0[5]), "=r"(u0[6]), "=r"(u0[7])
               : "r"(taddr));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(u1[0]), "=r"(u1[1]), "=r"(u1[2]), "=r"(u1[3]), "=r"(u1[4]), "=r"(u1[5]), "=r"(u1[6]), "=r"(u1[7])
               : "r"(taddr + np));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(u2[0]), "=r"(u2[1]), "=r"(u2[2]), "=r"(u2[3]), "=r"(u2[4]), "=r"(u2[5]), "=r"(u2[6]), "=r"(u2[7])
               : "r"(taddr + 2u * np));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j)
    v[j] = (__uint_as_float(u2[j]) + __uint_as_float(u1[j])) + __uint_as_float(u0[j]);
}

// LU with partial pivoting in float64 of an ns x ns matrix (row-major,
// overwritten); det(A) = mant * 2^ex with the sign in mant, rescaled after
// every pivot so that products of small orbital values do not underflow.
// mant = 0 for a singular matrix.
__device__ inline void det_scaled(double* A, int ns, double* mant, int* ex) {
  double m = 1.0;
  int e = 0;
  for (int c = 0; c < ns; ++c) {
    int best = c;
    double bv = fabs(A[c * ns + c]);
    for (int rr = c + 1; rr < ns; ++rr) {
      const double v = fabs(A[rr * ns + c]);
      if (v > bv) { bv = v; best = rr; }
    }
    if (!(bv > 0.0)) { *mant = 0.0; *ex = 0; return; }
    if (best != c) {
      for (int k = 0; k < ns; ++k) {
        const double t0 = A[c * ns + k];
        A[c * ns + k] = A[best * ns + k];
        A[best * ns + k] = t0;
      }
      m = -m;
    }
    const double piv = A[c * ns + c];
    int pe;
    m = frexp(m * piv, &pe);
    e += pe;
    const double ip = 1.0 / piv;
    for (int rr = c + 1; rr < ns; ++rr) {
      const double f = A[rr * ns + c] * ip;
      for (int k = c + 1; k < ns; ++k) A[rr * ns + k] -= f * A[c * ns + k];
    }
  }
  *mant = m;
  *ex = e;
}

struct TcLayout {
  int WT;
  int a_bytes;  // one piece of the A tile region (128 rows x Kmax bf16)
  int b_bytes;  // one weight buffer
  size_t A, B[3], x, h, wv, h0, Y, msg, r, rp, rpf, d, phi, rad, ic, det, dex, F, J, lp, bytes;
  int E;  // partner slots per (channel, electron): N - 1 + M
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 127) & ~(size_t)127; }

inline TcLayout tc_layout(const DevSys& s, int max_bytes, int WT) {
  TcLayout L;
  L.WT = WT;
  const int Kmax = std::max(std::max(s.D, s.K), std::max(s.Hw, s.Zd));
  L.a_bytes = TM * Kmax * 2;
  L.b_bytes = (int)a16(max_bytes);
  size_t o = 0;
  auto put = [&](size_t b) { size_t q = o; o += a16(b); return q; };
  const size_t N = s.N, P = s.Ppair, no = s.n_orb;
  L.A = put(3 * (size_t)L.a_bytes);
  for (int b = 0; b < 3; ++b) L.B[b] = put(L.b_bytes);
  // float state rows padded by 4 floats: lanes run over rows, so an unpadded
  // power-of-two stride would put every lane in the same bank
  L.x = put((size_t)TM * (s.D + 4) * 4);
  L.h = put((size_t)TM * (s.Zd + 4) * 4);
  L.wv = put((size_t)TM * (s.Zd + 4) * 4);
  L.h0 = put((size_t)s.Zd * 4);
  L.Y = put((size_t)s.M * s.Zd * 4);
  L.E = s.N - 1 + s.M;
  L.msg = put((size_t)3 * s.N * (L.E + 1) * 4);
  L.r = put(WT * N * 3 * 8);
  L.rp = put(WT * N * 3 * 8);
  L.rpf = put(WT * N * 3 * 4);
  L.d = put(WT * P * 4);
  L.phi = put(WT * N * no * 4);
  L.rad = put(WT * N * (size_t)s.n_shells * 4);
  L.ic = put(WT * N * 4);
  L.det = put((size_t)WT * s.n_det * 2 * 8);
  L.dex = put((size_t)WT * s.n_det * 2 * 4);
  L.F = put(WT * N * no * 4);
  L.J = put(WT * 4);
  L.lp = put(WT * 8);
  L.bytes = o;
  return L;
}

__global__ void __launch_bounds__(NT, 1) k_metropolis_tc(DevSys s, DevNet<float> net,
                                                         const TcStages* __restrict__ tsp,
                                                         const unsigned short* __restrict__ tcpack, TcLayout L,
                                                         double* __restrict__ r, double* __restrict__ lp, int W,
                                                         unsigned walker0, int n_steps, double sigma,
                                                         unsigned long long seed, unsigned long long step0,
                                                         unsigned long long* __restrict__ n_acc, uint32_t tmem_cols) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_w[3];
  __shared__ long issued;  // weight copies issued (thread 0 writes)
  __shared__ __align__(8) uint64_t bar_m;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ unsigned acc_count;
  __shared__ int st_K[PN_MAX_TC_STAGES], st_Np[PN_MAX_TC_STAGES], st_bytes[PN_MAX_TC_STAGES];
  __shared__ long long st_off[PN_MAX_TC_STAGES];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = s.N, P = s.Ppair, D = s.D, Zd = s.Zd, K = s.K, Hw = s.Hw, no = s.n_orb, nd = s.n_det;
  const int n3 = 3 * N, nblk4 = (n3 + 3) / 4;
  const NetOff& o = net.off;
  const int nst = tsp->n;
  for (int i = tid; i < nst; i += NT) {
    st_K[i] = tsp->K[i];
    st_Np[i] = tsp->Np[i];
    st_bytes[i] = tsp->bytes[i];
    st_off[i] = tsp->off[i];
  }
  const int w0 = blockIdx.x * L.WT;
  const int WTt = min(L.WT, W - w0);
  const int rowsN = WTt * N;
  const int LX = D + 4, LH = Zd + 4;  // padded row strides of x and of h / w
  unsigned char* sA = smem + L.A;
  unsigned char* sB[3] = {smem + L.B[0], smem + L.B[1], smem + L.B[2]};
  float* sh0 = (float*)(smem + L.h0);
  float* sY = (float*)(smem + L.Y);
  int* smsg = (int*)(smem + L.msg);  // [3][N][1 + E]: count, then (pos << 16 | partner)
  float* sx = (float*)(smem + L.x);
  float* sh = (float*)(smem + L.h);
  float* swv = (float*)(smem + L.wv);
  double* sr = (double*)(smem + L.r);
  double* srp = (double*)(smem + L.rp);
  float* srpf = (float*)(smem + L.rpf);
  float* sd = (float*)(smem + L.d);
  float* sphi = (float*)(smem + L.phi);
  float* srad = (float*)(smem + L.rad);
  int* sic = (int*)(smem + L.ic);
  double* sdet = (double*)(smem + L.det);
  int* sdex = (int*)(smem + L.dex);
  float* sF = (float*)(smem + L.F);
  float* sJ = (float*)(smem + L.J);
  double* slp = (double*)(smem + L.lp);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar_w[b])));
    issued = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar_m)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    acc_count = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t col_g = (uint32_t)(tmem_cols / 2);  // receiving-map accumulator (3 blocks of D columns)

  // ---- weight stages (TMA, two ahead) and MMA completion phases
  const long total = (long)n_steps * nst;
  uint32_t mma_phase = 0;
  bool mma_pending = false;  // thread 0: a committed MMA group not yet waited for
  uint32_t pend_phase = 0;
  // ring positions: producer (thread 0) and consumer stage / buffer / phase
  long n_issued = 0;
  int pj = 0, pb = 0;
  int cj = 0, cb = 0;
  uint32_t cpar = 0;
  auto issue = [&]() {
    if (n_issued >= total) return;
    const uint32_t bar = saddr(&bar_w[pb]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(st_bytes[pj]) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(sB[pb])),
                 "l"(tcpack + st_off[pj]), "r"(st_bytes[pj]), "r"(bar)
                 : "memory");
    issued = ++n_issued;
    pj = pj + 1 == nst ? 0 : pj + 1;
    pb = pb == 2 ? 0 : pb + 1;
  };
  if (tid == 0) {
    issue();
    issue();
    issue();
  }
  // One GEMM stage: the A tile (K columns) is in sA, written and fenced by
  // every thread before the barrier that precedes this call.  Accumulates
  // the b0, b1, b2 products into TMEM column blocks [col + q Np, +Np),
  // q = 0, 1, 2; acc_first says whether the first product adds to what the
  // columns hold.  Returns Np, the block width the epilogue reads.
  auto gemm = [&](uint32_t col, bool acc_first) -> uint32_t {
    const int b = cb;
    const int Kg = st_K[cj], Np = st_Np[cj];
    if (!abort_flag && !wait_bar(saddr(&bar_w[b]), cpar)) abort_flag = 1;
    if (tid == 0 && !abort_flag) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = saddr(sA), b0 = saddr(sB[b]);
      const uint32_t i3 = idesc_bf16(3 * Np), i2 = idesc_bf16(2 * Np), i1 = idesc_bf16(Np);
      // descriptors built once; a k-step of 16 bf16 (256 bytes) advances
      // only the start-address field (addr >> 4)
      const uint64_t dA0 = sdesc(a0, Kg), dA1 = sdesc(a0 + (uint32_t)L.a_bytes, Kg),
                     dA2 = sdesc(a0 + 2u * (uint32_t)L.a_bytes, Kg), dB = sdesc(b0, Kg);
      const uint32_t dcol = tmem + col;
      for (int st = 0; st < Kg / 16; ++st) {
        const uint64_t adv = (uint64_t)(st * 16);
        const uint32_t first = (st == 0) ? (acc_first ? 1u : 0u) : 1u;
        asm volatile(
            "{\n\t.reg .pred pf, pt;\n\t"
            "setp.ne.b32 pf, %8, 0;\n\t"
            "setp.eq.b32 pt, %8, %8;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %5, pf;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %4, %6, pt;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %4, %7, pt;\n\t}" ::"r"(dcol),
            "l"(dA0 + adv), "l"(dA1 + adv), "l"(dA2 + adv), "l"(dB + adv), "r"(i3), "r"(i2), "r"(i1), "r"(first));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&bar_m))
                   : "memory");
      mma_pending = true;
      pend_phase = mma_phase;
    }
    if (!abort_flag) {
      if (wait_bar(saddr(&bar_m), mma_phase))
        mma_pending = false;
      else
        abort_flag = 1;
    }
    mma_phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // the weight buffer is free once the MMAs completed
    if (tid == 0 && !abort_flag) issue();
    cj = cj + 1 == nst ? 0 : cj + 1;
    if (++cb == 3) {
      cb = 0;
      cpar ^= 1u;
    }
    return (uint32_t)Np;
  };
  // A stage this thread does not take part in: advance the ring as gemm()
  // does, without waiting.
  auto skip_stage = [&]() {
    mma_phase ^= 1u;
    cj = cj + 1 == nst ? 0 : cj + 1;
    if (++cb == 3) {
      cb = 0;
      cpar ^= 1u;
    }
  };
  // End of an epilogue that wrote the next A tile: make the generic-proxy
  // stores visible to the tensor core, then meet at the barrier.
  auto fence_sync = [&]() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  };
  // warp w reads TMEM lane quadrant w % 4 (tile rows 32 (w % 4) + lane);
  // the WPQ warps of a quadrant take every WPQ-th 8-column chunk
  const int quad = warp & 3, sub = warp >> 2;
  const int arow = quad * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);

  // ---- walker state
  for (int i = tid; i < WTt * n3; i += NT) sr[i] = r[(size_t)w0 * n3 + i];
  for (int i = tid; i < WTt; i += NT) slp[i] = lp[w0 + i];
  for (int q = tid; q < s.M * Zd; q += NT) sY[q] = net.p[o.Y + q];
  // message partners: for channel c and electron i, the positions k of the
  // channel's pairs that contain i and the other particle (electron or
  // nucleus) of each
  for (int q = tid; q < 3 * N; q += NT) {
    const int c = q / N, i = q % N;
    int* ent = smsg + q * (L.E + 1);
    int cntp = 0;
    const int* pl = s.ch_pairs + s.ch_off[c];
    for (int k = 0; k < s.ch_off[c + 1] - s.ch_off[c]; ++k) {
      const int p = pl[k];
      int other = -1;
      if (p < s.Pee) {
        int a = 0, rem = p;
        while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
        const int bb = a + 1 + rem;
        other = a == i ? bb : (bb == i ? a : -1);
      } else if ((p - s.Pee) / s.M == i) {
        other = (p - s.Pee) % s.M;
      }
      if (other >= 0) ent[1 + cntp++] = (k << 16) | other;
    }
    ent[0] = cntp;
  }
  for (int z = tid; z < Zd; z += NT) {  // h^(0) row (float32, in input order)
    float acc = net.p[o.hb[0] + z];
    for (int d = 0; d < D; ++d) acc = fmaf(net.p[o.x0 + d], net.p[o.hW[0] + (size_t)d * Zd + z], acc);
    sh0[z] = acc;
  }
  unsigned nacc = 0;
  __syncthreads();
  const OrbTab<float> tab = orb_tab<float>(s);

  // abort decisions are taken at barriers (__syncthreads_or) so that every
  // thread leaves the loops at the same point
  for (int kstep = 0; kstep < n_steps; ++kstep) {
    bool stop = false;
    const unsigned long long step = step0 + (unsigned long long)kstep;
    // proposals (float32 normals, float64 positions)
    for (int q = tid; q < WTt * 2 * nblk4; q += NT) {
      const int w = q / (2 * nblk4), jj = (q % (2 * nblk4)) >> 1, pr = q & 1;
      if (4 * jj + 2 * pr >= n3) continue;
      float zz[2];
      normal_pair<float>(seed, walker0 + (unsigned)(w0 + w), step, jj, pr, zz);
      for (int t = 0; t < 2; ++t) {
        const int m = 4 * jj + 2 * pr + t;
        if (m < n3) {
          srp[w * n3 + m] = sr[w * n3 + m] + sigma * (double)zz[t];
          srpf[w * n3 + m] = (float)srp[w * n3 + m];
        }
      }
    }
    __syncthreads();
    // pair distances
    for (int q = tid; q < WTt * P; q += NT) {
      const int w = q / P, p = q % P;
      const float* rw = srpf + w * n3;
      float v[3];
      if (p < s.Pee) {
        int a = 0, rem = p;
        while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
        const int bb = a + 1 + rem;
        for (int x = 0; x < 3; ++x) v[x] = rw[3 * a + x] - rw[3 * bb + x];
      } else {
        const int qq = p - s.Pee, i = qq / s.M, I = qq % s.M;
        for (int x = 0; x < 3; ++x) v[x] = rw[3 * i + x] - tab.R[3 * I + x];
      }
      sd[q] = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
    // orbitals: cusp sphere, radial parts, contractions (float32)
    for (int e = tid; e < rowsN; e += NT) {
      int Ic = -1;
      if (s.use_cusp)
        for (int I = 0; I < s.M; ++I) {
          const float v0 = srpf[3 * e] - tab.R[3 * I], v1 = srpf[3 * e + 1] - tab.R[3 * I + 1],
                      v2 = srpf[3 * e + 2] - tab.R[3 * I + 2];
          if (v0 * v0 + v1 * v1 + v2 * v2 < tab.rc[I] * tab.rc[I]) Ic = I;
        }
      sic[e] = Ic;
    }
    for (int q = tid; q < rowsN * s.n_shells; q += NT) {
      const int e = q / s.n_shells, sh_ = q % s.n_shells;
      const int c = s.sh_center[sh_], np_ = s.sh_nprim[sh_], po = s.sh_poff[sh_];
      const float v0 = srpf[3 * e] - tab.R[3 * c], v1 = srpf[3 * e + 1] - tab.R[3 * c + 1],
                  v2 = srpf[3 * e + 2] - tab.R[3 * c + 2];
      const float r2 = v0 * v0 + v1 * v1 + v2 * v2;
      float ev = 0;
      if (s.sh_l[sh_] == -1)
        ev = tab.pcoef[po] * expf(-tab.pexp[po] * sqrtf(r2));
      else
        for (int k = 0; k < np_; ++k) ev += tab.pcoef[po + k] * expf(-tab.pexp[po + k] * r2);
      srad[q] = ev;
    }
    // x^(0) on real rows, zero elsewhere
    for (int q = tid; q < TM * D; q += NT) sx[(q / D) * LX + q % D] = (q / D) < rowsN ? net.p[o.x0 + q % D] : 0.f;
    __syncthreads();
    for (int q = tid; q < rowsN * no; q += NT) {
      const int e = q / no, mu = q % no;
      const int Ic = sic[e];
      float acc = 0;
      for (int sh_ = 0; sh_ < s.n_shells; ++sh_) {
        const int c = s.sh_center[sh_], l = s.sh_l[sh_], bo = s.sh_boff[sh_];
        const float ev = srad[e * s.n_shells + sh_];
        if (l <= 0) {
          if (l == 0 && c == Ic && s.cusp_on[Ic * no + mu]) continue;
          acc += tab.mo[(size_t)bo * no + mu] * ev;
          continue;
        }
        const float v0 = srpf[3 * e] - tab.R[3 * c], v1 = srpf[3 * e + 1] - tab.R[3 * c + 1],
                    v2 = srpf[3 * e + 2] - tab.R[3 * c + 2];
        const float* m = tab.mo + (size_t)bo * no + mu;
        if (l == 1)
          acc += ev * (m[0] * v0 + m[no] * v1 + m[2 * no] * v2);
        else
          acc += ev * (m[0] * v0 * v0 + m[no] * v0 * v1 + m[2 * no] * v0 * v2 + m[3 * no] * v1 * v1 +
                       m[4 * no] * v1 * v2 + m[5 * no] * v2 * v2);
      }
      if (Ic >= 0 && s.cusp_on[Ic * no + mu]) {
        const float v0 = srpf[3 * e] - tab.R[3 * Ic], v1 = srpf[3 * e + 1] - tab.R[3 * Ic + 1],
                    v2 = srpf[3 * e + 2] - tab.R[3 * Ic + 2];
        const float dd = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        const int k = Ic * no + mu;
        const float* a = tab.ca + (size_t)k * 5;
        acc += tab.cC[k] + tab.cs[k] * expf(a[0] + dd * (a[1] + dd * (a[2] + dd * (a[3] + dd * a[4]))));
      }
      sphi[q] = acc;
    }
    // ---- interaction layers
    for (int n = 0; n < s.L; ++n) {
      if (n == 0) {  // h^(0) = x^(0) Wh + bh, the same row for every electron
        for (int q = tid; q < TM * (Zd / 4); q += NT) {
          const int row = q / (Zd / 4), z4 = (q % (Zd / 4)) * 4;
          *(float4*)(sh + row * LH + z4) = *(const float4*)(sh0 + z4);
        }
      } else {
      // A <- x (K = D); h = x Wh + bh
      for (int q = tid; q < rowsN * (D / 8); q += NT) {
        const int row = q % rowsN, k8 = (q / rowsN) * 8;
        float v[8];
        const float4 p0 = *(const float4*)(sx + row * LX + k8), p1 = *(const float4*)(sx + row * LX + k8 + 4);
        v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w; v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
        put3x8(sA, L.a_bytes, row, k8, D, v);
      }
      fence_sync();
      const uint32_t np = gemm(0, false);
      if (quad * 32 < rowsN)
      for (int c0 = sub * 8; c0 < Zd; c0 += WPQ * 8) {
        float v[8];
        tmem_ld8x3(trow + (uint32_t)c0, np, v);
        const float* hb = net.p + o.hb[n] + c0;
        for (int jj = 0; jj < 8; jj += 4)
          *(float4*)(sh + arow * LH + c0 + jj) =
              make_float4(v[jj] + hb[jj], v[jj + 1] + hb[jj + 1], v[jj + 2] + hb[jj + 2], v[jj + 3] + hb[jj + 3]);
      }
      }
      bool g_started = false;
      for (int c = 0; c < 3; ++c) {
        const int cnt = s.ch_off[c + 1] - s.ch_off[c];
        if (cnt == 0) continue;
        const int* pl = s.ch_pairs + s.ch_off[c];
        const int rowsP = WTt * cnt;
        // A <- distance features of this channel's pairs (K = s.K)
        __syncthreads();  // A is free (the previous MMA completed) and sh is written
        const float* fm = s.feat_mu32;
        const float* fi = s.feat_isig2_32;
        // (rows of the tile past the real ones are left as they are: a row
        // of the product depends only on the same row of A, and those rows
        // are never read back)
        for (int q = tid; q < rowsP * (K / 8); q += NT) {
          const int row = q % rowsP, k8 = (q / rowsP) * 8;
          float v[8];
          const float dd = sd[(row / cnt) * P + pl[row % cnt]];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const float dm = dd - fm[k8 + t];
            v[t] = dd * dd * __expf(-dd - dm * dm * fi[k8 + t]);
          }
          put3x8(sA, L.a_bytes, row, k8, K, v);
        }
        fence_sync();
        uint32_t np = gemm(0, false);  // hidden = e W1
        if (quad * 32 < rowsP)
          for (int c0 = sub * 8; c0 < Hw; c0 += WPQ * 8) {
            float v[8];
            tmem_ld8x3(trow + (uint32_t)c0, np, v);
            const float* b1 = net.p + o.b1[n][c] + c0;
            for (int jj = 0; jj < 8; ++jj) v[jj] = sspf(v[jj] + b1[jj]);
            put3x8(sA, L.a_bytes, arow, c0, Hw, v);
          }
        fence_sync();
        np = gemm(0, false);  // w = hidden W2
        if (quad * 32 < rowsP)
        for (int c0 = sub * 8; c0 < Zd; c0 += WPQ * 8) {
          float v[8];
          tmem_ld8x3(trow + (uint32_t)c0, np, v);
          const float* b2 = net.p + o.b2[n][c] + c0;
          for (int jj = 0; jj < 8; jj += 4)
            *(float4*)(swv + arow * LH + c0 + jj) =
                make_float4(v[jj] + b2[jj], v[jj + 1] + b2[jj + 1], v[jj + 2] + b2[jj + 2], v[jj + 3] + b2[jj + 3]);
        }
        __syncthreads();
        // A <- z_c: messages of this channel for every electron (K = Zd)
        for (int q = tid; q < rowsN * (Zd / 8); q += NT) {
          const int e = q % rowsN, z8 = (q / rowsN) * 8;
          const int w = e / N, i = e % N;
          const int* ent = smsg + (c * N + i) * (L.E + 1);
          float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
          for (int u = 1; u <= ent[0]; ++u) {
            const int k = ent[u] >> 16, src = ent[u] & 0xFFFF;
            const float* wr = swv + (w * cnt + k) * LH + z8;
            const float* hr = c < 2 ? sh + (w * N + src) * LH + z8 : sY + src * Zd + z8;
            const float4 w0 = *(const float4*)wr, w1 = *(const float4*)(wr + 4);
            const float4 h0 = *(const float4*)hr, h1 = *(const float4*)(hr + 4);
            acc[0] += w0.x * h0.x; acc[1] += w0.y * h0.y; acc[2] += w0.z * h0.z; acc[3] += w0.w * h0.w;
            acc[4] += w1.x * h1.x; acc[5] += w1.y * h1.y; acc[6] += w1.z * h1.z; acc[7] += w1.w * h1.w;
          }
          put3x8(sA, L.a_bytes, e, z8, Zd, acc);
        }
        fence_sync();
        gemm(col_g, g_started);  // x update += z_c G_c (blocks of D columns)
        g_started = true;
      }
      // x += accumulated update + receiving biases
      if (quad * 32 < rowsN)
      for (int c0 = sub * 8; c0 < D; c0 += WPQ * 8) {
        float v[8];
        tmem_ld8x3(trow + col_g + (uint32_t)c0, (uint32_t)D, v);
        if (arow < rowsN) {
          const float* gb = net.Gb + (size_t)n * D + c0;
          for (int jj = 0; jj < 8; jj += 4) {
            float4 xv = *(float4*)(sx + arow * LX + c0 + jj);
            xv.x += v[jj] + gb[jj];
            xv.y += v[jj + 1] + gb[jj + 1];
            xv.z += v[jj + 2] + gb[jj + 2];
            xv.w += v[jj + 3] + gb[jj + 3];
            *(float4*)(sx + arow * LX + c0 + jj) = xv;
          }
        }
      }
      if (__syncthreads_or(abort_flag)) {
        stop = true;
        break;
      }
    }
    if (stop) break;
    // ---- backflow head kappa: three maps on every electron row
    for (int q = tid; q < rowsN * (D / 8); q += NT) {
      const int row = q % rowsN, k8 = (q / rowsN) * 8;
      float v[8];
      const float4 p0 = *(const float4*)(sx + row * LX + k8), p1 = *(const float4*)(sx + row * LX + k8 + 4);
      v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w; v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
      put3x8(sA, L.a_bytes, row, k8, D, v);
    }
    fence_sync();
    for (int layer = 0; layer < 2; ++layer) {
      const uint32_t np = gemm(0, false);
      if (quad * 32 < rowsN)
      for (int c0 = sub * 8; c0 < D; c0 += WPQ * 8) {
        float v[8];
        tmem_ld8x3(trow + (uint32_t)c0, np, v);
        const float* kb = net.p + o.kb[layer] + c0;
        for (int jj = 0; jj < 8; ++jj) v[jj] = sspf(v[jj] + kb[jj]);
        put3x8(sA, L.a_bytes, arow, c0, D, v);
      }
      fence_sync();
    }
    uint32_t np = gemm(0, false);
    if (quad * 32 < rowsN)
    for (int c0 = sub * 8; c0 < no; c0 += WPQ * 8) {
      float v[8];
      tmem_ld8x3(trow + (uint32_t)c0, np, v);
      if (arow < rowsN)
        for (int jj = 0; jj < 8 && c0 + jj < no; ++jj) sF[arow * no + c0 + jj] = v[jj] + net.p[o.kb[2] + c0 + jj];
    }
    __syncthreads();
    // ---- Jastrow head eta on the electron sums (rows = walkers), and the
    // determinants.  When the walkers fit one TMEM lane quadrant (WTt <= 32)
    // the four warps of quadrant 0 run the eta maps while the other twelve
    // warps form the determinants (float64 LU), meeting at the next barrier.
    const bool split = WTt <= 32;
    const bool in_e = !split || quad == 0;
    if (in_e) {
      const int ge = split ? sub * 32 + lane : tid, ne = split ? 128 : NT;
      auto esync = [&]() {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (split)
          asm volatile("bar.sync 1, 128;" ::: "memory");
        else
          __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
      };
      for (int q = ge; q < WTt * (D / 8); q += ne) {
        const int w = q % WTt, d8 = (q / WTt) * 8;
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < N; ++i) {
          const float4 p0 = *(const float4*)(sx + (w * N + i) * LX + d8), p1 = *(const float4*)(sx + (w * N + i) * LX + d8 + 4);
          acc[0] += p0.x; acc[1] += p0.y; acc[2] += p0.z; acc[3] += p0.w;
          acc[4] += p1.x; acc[5] += p1.y; acc[6] += p1.z; acc[7] += p1.w;
        }
        put3x8(sA, L.a_bytes, w, d8, D, acc);
      }
      esync();
      for (int layer = 0; layer < 2; ++layer) {
        const uint32_t npl = gemm(0, false);
        if (quad * 32 < WTt)
          for (int c0 = sub * 8; c0 < D; c0 += WPQ * 8) {
            float v[8];
            tmem_ld8x3(trow + (uint32_t)c0, npl, v);
            const float* eb = net.p + o.eb[layer] + c0;
            for (int jj = 0; jj < 8; ++jj) v[jj] = sspf(v[jj] + eb[jj]);
            put3x8(sA, L.a_bytes, arow, c0, D, v);
          }
        esync();
      }
      np = gemm(0, false);
      if (sub == 0 && quad * 32 < WTt) {
        float v[8];
        tmem_ld8x3(trow, np, v);
        if (arow < WTt) sJ[arow] = v[0] + net.p[o.eb[2]];
      }
    } else {
      for (int k = 0; k < 3; ++k) skip_stage();  // keep the stage ring in step with quadrant 0
    }
    if (!split || !in_e) {
      // one thread per (walker, det, spin)
      const int gd = split ? ((sub * 3 + quad - 1) * 32 + lane) : tid, nthr = split ? NT - 128 : NT;
      for (int q = gd; q < WTt * nd * 2; q += nthr) {
        const int sp = q & 1, p = (q >> 1) % nd, w = (q >> 1) / nd;
        const int ns = sp ? s.n_dn : s.n_up, e0 = sp ? s.n_up : 0;
        double mant = 1.0;
        int ex = 0;
        if (ns > 0) {
          double A[PN_MAX_SPIN * PN_MAX_SPIN];
          const int* occ = s.occ + p * N + e0;
          for (int a = 0; a < ns; ++a)
            for (int bb = 0; bb < ns; ++bb) {
              const int e = w * N + e0 + a, mu = occ[bb];
              A[a * ns + bb] = (double)sphi[e * no + mu] * (1.0 + (double)sF[e * no + mu]);
            }
          det_scaled(A, ns, &mant, &ex);
        }
        sdet[q] = mant;
        sdex[q] = ex;
      }
    }
    if (__syncthreads_or(abort_flag)) break;
    // ---- ln|psi'| = gamma + J + ln|sum_p c_p det_up,p det_dn,p| (float64
    // sum of the determinant products scaled by the largest power of two)
    // and the accept test
    for (int w = tid; w < WTt; w += NT) {
      const double* dm = sdet + (size_t)w * nd * 2;
      const int* de = sdex + (size_t)w * nd * 2;
      int emax = INT_MIN;
      for (int p = 0; p < nd; ++p)
        if (s.ci[p] != 0.0 && dm[2 * p] != 0.0 && dm[2 * p + 1] != 0.0) emax = max(emax, de[2 * p] + de[2 * p + 1]);
      double S = 0;
      if (emax != INT_MIN)
        for (int p = 0; p < nd; ++p) {
          const int sh = de[2 * p] + de[2 * p + 1] - emax;  // <= 0
          if (sh > -1022 && dm[2 * p] != 0.0 && dm[2 * p + 1] != 0.0)
            S += s.ci[p] * (dm[2 * p] * dm[2 * p + 1]) * __longlong_as_double((long long)(1023 + sh) << 52);
        }
      const double m = emax == INT_MIN ? -INFINITY : (double)emax * 0.69314718055994530942;
      float gam = 0.f;
      if (s.use_gamma)
        for (int a = 0; a < N; ++a)
          for (int bb = a + 1; bb < N; ++bb) {
            const float c = ((a < s.n_up) == (bb < s.n_up)) ? 0.25f : 0.5f;
            gam -= c / (1.f + sd[w * P + pn_pair_index(a, bb, N)]);
          }
      const double lpn = (double)gam + (double)sJ[w] + m + log(fabs(S));
      unsigned c4[4] = {(unsigned)nblk4, walker0 + (unsigned)(w0 + w), (unsigned)(step & 0xffffffffull),
                        (unsigned)(step >> 32)};
      pn_philox(c4, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
      const float u = ((float)c4[0] + 0.5f) * 2.3283064365386963e-10f;
      if (u < expf((float)(2.0 * (lpn - slp[w])))) {
        for (int q = 0; q < n3; ++q) sr[w * n3 + q] = srp[w * n3 + q];
        slp[w] = lpn;
        ++nacc;
      }
    }
    if (__syncthreads_or(abort_flag)) break;
  }
  if (abort_flag && tid == 0) {
    atomicExch(s.dev_err, 3);
    // drain what this CTA may have in flight: the weight copies (at most
    // three outstanding; thread 0 issued them) and the last MMA group
    for (long q = issued - 3 < 0 ? 0 : issued - 3; q < issued; ++q)
      wait_bar(saddr(&bar_w[q % 3]), (uint32_t)((q / 3) & 1));
    if (mma_pending) wait_bar(saddr(&bar_m), pend_phase);
  }
  for (int i = tid; i < WTt * n3; i += NT) r[(size_t)w0 * n3 + i] = sr[i];
  for (int i = tid; i < WTt; i += NT) lp[w0 + i] = slp[i];
  if (nacc) atomicAdd(&acc_count, nacc);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && n_acc && acc_count) atomicAdd(n_acc, (unsigned long long)acc_count);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

}  // namespace

// Launch the tensor-core sampler; PN_ENOTREADY if the system's tiles do not fit.
int pn_run_metropolis_tc(const DevSys& s, const DevNet<float>& net, double* r, double* lp, int W, unsigned walker0,
                         int n_steps, double sigma, unsigned long long seed, unsigned long long step0,
                         unsigned long long* n_acc, cudaStream_t st) {
  if (net.tc_n == 0 || !net.tcpack || !net.tcst || W <= 0) return PN_ENOTREADY;
  int maxcnt = 1;
  for (int c = 0; c < 3; ++c) maxcnt = std::max(maxcnt, s.ch_off[c + 1] - s.ch_off[c]);
  int dev = 0, sms = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int WT = std::min(TM / s.N, TM / maxcnt);
  WT = std::min(WT, std::max(1, (W + sms - 1) / sms));
  if (WT < 1) return PN_ENOTREADY;
  const TcLayout L = tc_layout(s, net.tc_max_bytes, WT);
  if (L.bytes + 4096 > (size_t)maxsm) return PN_ENOTREADY;  // + static shared memory
  // TMEM: three column blocks of the widest map at 0, three blocks of D for
  // the receiving-map accumulator at 256
  const int widest = std::max(std::max(s.D, s.Hw), std::max(s.Zd, (s.n_orb + 15) / 16 * 16));
  if (3 * widest > 256) return PN_ENOTREADY;
  const uint32_t cols = 512u;
  PN_CUDA(pn_allow_max_smem(k_metropolis_tc));
  const int blocks = (W + WT - 1) / WT;
  PN_LAUNCH_W("k_metropolis_tc", st, (double)W * n_steps * pn_value_pass_flops(s),
            k_metropolis_tc<<<blocks, NT, L.bytes, st>>>(s, net, net.tcst, net.tcpack, L, r, lp, W, walker0, n_steps,
                                                         sigma, seed, step0, n_acc, cols));
  return PN_OK;
}
