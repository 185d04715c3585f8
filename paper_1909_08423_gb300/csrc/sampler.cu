// Fused Metropolis sampler: one launch runs every step for a tile of walkers.
//
// The value pass of psi is small per walker (positions, one feature vector
// per electron, one filter output per pair), so a CTA keeps a whole tile of
// walkers in shared memory for all n_steps steps: propose (Philox),
// geometry, orbitals, distance features, the L interaction layers, the two
// heads, the determinants and the accept test, with no trip through global
// memory except the weights (read through L1/L2, shared by every CTA) and
// the tile's final positions.  The staged path (one kernel per stage over
// the whole batch) remains for systems whose tile does not fit.
//
// Proposals and acceptance uniforms use the same Philox stream as the staged
// path, so both sample the same chain up to floating-point rounding of
// ln|psi| in the network.
#include <math.h>

#include <algorithm>

#include "ansatz_dev.cuh"
#include "kernels.cuh"
#include "pn_internal.cuh"

namespace {

template <typename R>
__device__ inline const R* feat_mu_of(const DevSys& s);
template <>
__device__ inline const double* feat_mu_of<double>(const DevSys& s) { return s.feat_mu; }
template <>
__device__ inline const float* feat_mu_of<float>(const DevSys& s) { return s.feat_mu32; }
template <typename R>
__device__ inline const R* feat_is_of(const DevSys& s);
template <>
__device__ inline const double* feat_is_of<double>(const DevSys& s) { return s.feat_isig2; }
template <>
__device__ inline const float* feat_is_of<float>(const DevSys& s) { return s.feat_isig2_32; }

template <typename R>
__device__ inline R ssp_(R x) {
  return (x > R(0) ? x : R(0)) + log1p(exp(-fabs(x))) - R(0.69314718055994530942);
}

// Shared-memory layout of one tile (offsets in bytes).
struct Layout {
  int WT;
  size_t r, rp, geo, phi, lp, lpp, det, x, h, e, bufA, wv, bufB, F, xs, a1s, a2s, J, bytes;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename R>
__host__ __device__ inline Layout make_layout(const DevSys& s, int WT) {
  Layout L;
  L.WT = WT;
  const size_t W = WT, N = s.N, P = s.Ppair, D = s.D, Zd = s.Zd, K = s.K, Hw = s.Hw, no = s.n_orb;
  size_t o = 0;
  auto put = [&](size_t bytes) { size_t q = o; o += al16(bytes); return q; };
  L.r = put(W * N * 3 * 8);
  L.rp = put(W * N * 3 * 8);
  L.geo = put(W * P * 4 * 8);
  L.phi = put(W * N * no * 8);
  L.lp = put(W * 8);
  L.lpp = put(W * 8);
  L.det = put(W * s.n_det * 2 * 8);
  const size_t r = sizeof(R);
  L.x = put(W * N * D * r);
  L.h = put(W * N * Zd * r);
  L.e = put(W * P * K * r);
  L.bufA = put(W * (P * Hw > N * D ? P * Hw : N * D) * r);
  L.wv = put(W * P * Zd * r);
  L.bufB = put(W * (N * 3 * Zd > N * D ? N * 3 * Zd : N * D) * r);
  L.F = put(W * N * no * r);
  L.xs = put(W * D * r);
  L.a1s = put(W * D * r);
  L.a2s = put(W * D * r);
  L.J = put(W * r);
  L.bytes = o;
  return L;
}

// Y[row] (=|+=) act(X[row] W + b) for rows given by pointer maps; each
// thread computes four rows of one output column, reading W[k][col] once
// per k for all four.
template <typename R, bool SSP, bool ACC, class RX, class RY>
__device__ inline void cta_gemm(int rows, int K, const R* __restrict__ W, int Nout, const R* __restrict__ b, RX rx,
                                RY ry) {
  const int rb = (rows + 3) >> 2;
  for (int idx = threadIdx.x; idx < rb * Nout; idx += blockDim.x) {
    const int col = idx % Nout;
    const int r0 = (idx / Nout) << 2;
    const R* x0 = rx(r0);
    const R* x1 = rx(min(r0 + 1, rows - 1));
    const R* x2 = rx(min(r0 + 2, rows - 1));
    const R* x3 = rx(min(r0 + 3, rows - 1));
    const R bias = b ? b[col] : R(0);
    R a0 = bias, a1 = bias, a2 = bias, a3 = bias;
    const R* wc = W + col;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const R w = __ldg(wc + (size_t)k * Nout);
      a0 += x0[k] * w;
      a1 += x1[k] * w;
      a2 += x2[k] * w;
      a3 += x3[k] * w;
    }
    R v[4] = {a0, a1, a2, a3};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (r0 + q >= rows) break;
      R val = SSP ? ssp_(v[q]) : v[q];
      R* y = ry(r0 + q) + col;
      *y = ACC ? *y + val : val;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_metropolis_fused(DevSys s, DevNet<R> net, Layout L, double* __restrict__ r,
                                                          double* __restrict__ lp, int W, unsigned walker0,
                                                          int n_steps, double sigma,
                                                          unsigned long long seed, unsigned long long step0,
                                                          unsigned long long* __restrict__ n_acc) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* sr = (double*)(smem + L.r);
  double* srp = (double*)(smem + L.rp);
  double* sgeo = (double*)(smem + L.geo);
  double* sphi = (double*)(smem + L.phi);
  double* slp = (double*)(smem + L.lp);
  double* sdet = (double*)(smem + L.det);
  R* sx = (R*)(smem + L.x);
  R* sh = (R*)(smem + L.h);
  R* se = (R*)(smem + L.e);
  R* sA = (R*)(smem + L.bufA);
  R* swv = (R*)(smem + L.wv);
  R* sB = (R*)(smem + L.bufB);
  R* sF = (R*)(smem + L.F);
  R* sxs = (R*)(smem + L.xs);
  R* sa1 = (R*)(smem + L.a1s);
  R* sa2 = (R*)(smem + L.a2s);
  R* sJ = (R*)(smem + L.J);
  __shared__ unsigned long long acc_count;

  const int N = s.N, P = s.Ppair, D = s.D, Zd = s.Zd, K = s.K, Hw = s.Hw, no = s.n_orb, nd = s.n_det;
  const int n3 = 3 * N;
  const int nblk4 = (n3 + 3) / 4;
  const NetOff& o = net.off;
  const int tiles = (W + L.WT - 1) / L.WT;
  if (threadIdx.x == 0) acc_count = 0;

  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int w0 = tile * L.WT;
    const int Wt = min(L.WT, W - w0);
    for (int i = threadIdx.x; i < Wt * n3; i += blockDim.x) sr[i] = r[(size_t)w0 * n3 + i];
    for (int i = threadIdx.x; i < Wt; i += blockDim.x) slp[i] = lp[w0 + i];
    __syncthreads();
    for (int k = 0; k < n_steps; ++k) {
      const unsigned long long step = step0 + (unsigned long long)k;
      // -- proposal r' = r + sigma xi
      for (int idx = threadIdx.x; idx < Wt * nblk4; idx += blockDim.x) {
        const int w = idx / nblk4, j = idx % nblk4;
        double z[4];
        pn_normals4(seed, walker0 + (unsigned)(w0 + w), step, j, z);
        for (int q = 0; q < 4; ++q) {
          const int m = 4 * j + q;
          if (m < n3) srp[w * n3 + m] = sr[w * n3 + m] + sigma * z[q];
        }
      }
      __syncthreads();
      // -- geometry, orbitals, distance features, x^(0)
      for (int idx = threadIdx.x; idx < Wt * P; idx += blockDim.x) {
        const int w = idx / P, p = idx % P;
        const double* rw = srp + w * n3;
        double v[3];
        if (p < s.Pee) {
          int a = 0, rem = p;
          while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
          const int bb = a + 1 + rem;
          for (int x = 0; x < 3; ++x) v[x] = rw[3 * a + x] - rw[3 * bb + x];
        } else {
          const int q = p - s.Pee, i = q / s.M, I = q % s.M;
          for (int x = 0; x < 3; ++x) v[x] = rw[3 * i + x] - s.R[3 * I + x];
        }
        const double d = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        sgeo[idx * 4] = d;
        // distance features e_k(d) = d^2 exp(-d - (d - mu_k)^2 / sigma_k^2)
        const R dr = (R)d;
        const R* fm = feat_mu_of<R>(s);
        const R* fi = feat_is_of<R>(s);
        for (int kk = 0; kk < K; ++kk) {
          const R dm = dr - fm[kk];
          se[(size_t)idx * K + kk] = dr * dr * exp(-dr - dm * dm * fi[kk]);
        }
      }
      for (int idx = threadIdx.x; idx < Wt * N; idx += blockDim.x)
        pn_orbitals_at<false>(s, srp + idx * 3, sphi + (size_t)idx * no);
      for (int idx = threadIdx.x; idx < Wt * N * D; idx += blockDim.x) sx[idx] = net.p[o.x0 + idx % D];
      __syncthreads();
      // -- interaction layers
      const int rowsN = Wt * N;
      for (int n = 0; n < s.L; ++n) {
        cta_gemm<R, false, false>(
            rowsN, D, net.p + o.hW[n], Zd, net.p + o.hb[n], [&](int q) { return (const R*)(sx + (size_t)q * D); },
            [&](int q) { return sh + (size_t)q * Zd; });
        for (int c = 0; c < 3; ++c) {
          const int cnt = s.ch_off[c + 1] - s.ch_off[c];
          if (cnt == 0) continue;
          const int* pl = s.ch_pairs + s.ch_off[c];
          auto prow = [&](int q) { return (size_t)(q / cnt) * P + pl[q % cnt]; };
          cta_gemm<R, true, false>(
              Wt * cnt, K, net.p + o.W1[n][c], Hw, net.p + o.b1[n][c],
              [&](int q) { return (const R*)(se + prow(q) * K); }, [&](int q) { return sA + prow(q) * Hw; });
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c) {
          const int cnt = s.ch_off[c + 1] - s.ch_off[c];
          if (cnt == 0) continue;
          const int* pl = s.ch_pairs + s.ch_off[c];
          auto prow = [&](int q) { return (size_t)(q / cnt) * P + pl[q % cnt]; };
          cta_gemm<R, false, false>(
              Wt * cnt, Hw, net.p + o.W2[n][c], Zd, net.p + o.b2[n][c],
              [&](int q) { return (const R*)(sA + prow(q) * Hw); }, [&](int q) { return swv + prow(q) * Zd; });
        }
        __syncthreads();
        // messages z_i = sum_j w_ij h_j (same / opposite spin), sum_I w_iI Y_I
        for (int idx = threadIdx.x; idx < rowsN * Zd; idx += blockDim.x) {
          const int z = idx % Zd;
          const int wi = idx / Zd;
          const int w = wi / N, i = wi % N;
          const R* ww = swv + (size_t)w * P * Zd;
          const R* hw = sh + (size_t)w * N * Zd;
          R zs = 0, za = 0, zn = 0;
          const bool si = i < s.n_up;
          for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
            const R v = ww[(size_t)p * Zd + z] * hw[(size_t)j * Zd + z];
            if ((j < s.n_up) == si) zs += v; else za += v;
          }
          for (int I = 0; I < s.M; ++I) zn += ww[(size_t)(s.Pee + i * s.M + I) * Zd + z] * net.p[o.Y + I * Zd + z];
          R* zo = sB + (size_t)wi * 3 * Zd;
          zo[z] = zs;
          zo[Zd + z] = za;
          zo[2 * Zd + z] = zn;
        }
        __syncthreads();
        cta_gemm<R, false, true>(
            rowsN, 3 * Zd, net.Gcat + (size_t)n * 3 * Zd * D, D, net.Gb + (size_t)n * D,
            [&](int q) { return (const R*)(sB + (size_t)q * 3 * Zd); }, [&](int q) { return sx + (size_t)q * D; });
        __syncthreads();
      }
      // -- heads: kappa on every electron, eta on the electron sum
      cta_gemm<R, true, false>(
          rowsN, D, net.p + o.kW[0], D, net.p + o.kb[0], [&](int q) { return (const R*)(sx + (size_t)q * D); },
          [&](int q) { return sA + (size_t)q * D; });
      for (int idx = threadIdx.x; idx < Wt * D; idx += blockDim.x) {
        const int w = idx / D, d = idx % D;
        R acc = 0;
        for (int i = 0; i < N; ++i) acc += sx[((size_t)w * N + i) * D + d];
        sxs[idx] = acc;
      }
      __syncthreads();
      cta_gemm<R, true, false>(
          rowsN, D, net.p + o.kW[1], D, net.p + o.kb[1], [&](int q) { return (const R*)(sA + (size_t)q * D); },
          [&](int q) { return sB + (size_t)q * D; });
      cta_gemm<R, true, false>(
          Wt, D, net.p + o.eW[0], D, net.p + o.eb[0], [&](int q) { return (const R*)(sxs + (size_t)q * D); },
          [&](int q) { return sa1 + (size_t)q * D; });
      __syncthreads();
      cta_gemm<R, false, false>(
          rowsN, D, net.p + o.kW[2], no, net.p + o.kb[2], [&](int q) { return (const R*)(sB + (size_t)q * D); },
          [&](int q) { return sF + (size_t)q * no; });
      cta_gemm<R, true, false>(
          Wt, D, net.p + o.eW[1], D, net.p + o.eb[1], [&](int q) { return (const R*)(sa1 + (size_t)q * D); },
          [&](int q) { return sa2 + (size_t)q * D; });
      __syncthreads();
      cta_gemm<R, false, false>(
          Wt, D, net.p + o.eW[2], 1, net.p + o.eb[2], [&](int q) { return (const R*)(sa2 + (size_t)q * D); },
          [&](int q) { return sJ + q; });
      // -- determinants, one thread per (walker, determinant, spin)
      for (int idx = threadIdx.x; idx < Wt * nd * 2; idx += blockDim.x) {
        const int sp = idx & 1, p = (idx >> 1) % nd, w = (idx >> 1) / nd;
        const int ns = sp ? s.n_dn : s.n_up, e0 = sp ? s.n_up : 0;
        double ld = 0, sg = 1;
        if (ns > 0) {
          double A[PN_MAX_SPIN * PN_MAX_SPIN];
          const int* occ = s.occ + p * N + e0;
          for (int a = 0; a < ns; ++a)
            for (int bb = 0; bb < ns; ++bb) {
              const int i = e0 + a, mu = occ[bb];
              A[a * ns + bb] = sphi[((size_t)w * N + i) * no + mu] * (1.0 + (double)sF[((size_t)w * N + i) * no + mu]);
            }
          pn_slogdet(A, ns, &ld, &sg);
        }
        sdet[(size_t)idx * 2] = ld;
        sdet[(size_t)idx * 2 + 1] = sg;
      }
      __syncthreads();
      // -- ln|psi'| and the accept test, one thread per walker
      for (int w = threadIdx.x; w < Wt; w += blockDim.x) {
        const double* dw = sdet + (size_t)w * nd * 4;
        double m = -INFINITY;
        for (int p = 0; p < nd; ++p) {
          const double sg = dw[4 * p + 1] * dw[4 * p + 3];
          if (s.ci[p] != 0.0 && sg != 0.0) m = fmax(m, dw[4 * p] + dw[4 * p + 2]);
        }
        double S = 0;
        if (m > -INFINITY)
          for (int p = 0; p < nd; ++p) {
            const double sg = dw[4 * p + 1] * dw[4 * p + 3];
            if (sg != 0.0) S += s.ci[p] * sg * exp(dw[4 * p] + dw[4 * p + 2] - m);
          }
        double gam = 0;
        if (s.use_gamma)
          for (int a = 0; a < N; ++a)
            for (int bb = a + 1; bb < N; ++bb) {
              const double c = ((a < s.n_up) == (bb < s.n_up)) ? 0.25 : 0.5;
              gam -= c / (1.0 + sgeo[((size_t)w * P + pn_pair_index(a, bb, N)) * 4]);
            }
        const double lpn = gam + (double)sJ[w] + m + log(fabs(S));
        unsigned c4[4] = {(unsigned)nblk4, walker0 + (unsigned)(w0 + w), (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
        pn_philox(c4, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
        const double u = pn_u01(c4[0]);
        if (u < exp(2.0 * (lpn - slp[w]))) {
          for (int q = 0; q < n3; ++q) sr[w * n3 + q] = srp[w * n3 + q];
          slp[w] = lpn;
          atomicAdd(&acc_count, 1ull);
        }
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < Wt * n3; i += blockDim.x) r[(size_t)w0 * n3 + i] = sr[i];
    for (int i = threadIdx.x; i < Wt; i += blockDim.x) lp[w0 + i] = slp[i];
    __syncthreads();
  }
  if (threadIdx.x == 0 && n_acc) atomicAdd(n_acc, acc_count);
}


// ---------------------------------------------------------------------------
// Warp-per-walker sampler for small systems: each warp owns one walker for
// all steps, so no stage waits on a block barrier, and a CTA holds many
// walkers' state in shared memory.  Lanes run over output columns; each
// lane keeps up to four rows (electrons or pairs) in registers so that one
// weight load serves four multiply-adds.

// Per-warp shared-memory layout (bytes).
struct WLayout {
  size_t r, rp, rpf, dr, phi, rad, ic, det, x, h, z, wv, hid, e, F, xs, a1s, a2s, J, bytes;
  int G;  // largest pair group of one filter channel
};

template <typename R>
__host__ __device__ inline WLayout make_wlayout(const DevSys& s) {
  WLayout L;
  const size_t N = s.N, P = s.Ppair, D = s.D, Zd = s.Zd, K = s.K, Hw = s.Hw, no = s.n_orb;
  int G = 1;
  for (int c = 0; c < 3; ++c) G = (s.ch_off[c + 1] - s.ch_off[c]) > G ? (s.ch_off[c + 1] - s.ch_off[c]) : G;
  L.G = G;
  size_t o = 0;
  auto put = [&](size_t bytes) { size_t q = o; o += al16(bytes); return q; };
  const size_t r = sizeof(R);
  L.r = put(N * 3 * 8);
  L.rp = put(N * 3 * 8);
  L.rpf = put(N * 3 * r);
  L.dr = put(P * r);
  L.phi = put(N * no * r);
  L.rad = put(N * (size_t)s.n_shells * r);
  L.ic = put(N * 4);
  L.det = put((size_t)s.n_det * 4 * 8);
  L.x = put(N * D * r);
  L.h = put(N * Zd * r);
  L.z = put(N * (3 * Zd > D ? 3 * Zd : D) * r);       // messages; kappa hidden 1
  L.wv = put((P * Zd > N * D ? P * Zd : N * D) * r);  // filter outputs; kappa hidden 2
  L.hid = put((size_t)G * Hw * r);
  L.e = put((size_t)G * K * r);
  L.F = put(N * no * r);
  L.xs = put(D * r);
  L.a1s = put(D * r);
  L.a2s = put(D * r);
  L.J = put(16);
  L.bytes = o;
  return L;
}

// Y[q] (=|+=) act(X[q] W + b), q < rows; lanes over output columns.
template <typename R, bool SSP, bool ACC, bool LDG = true, class RX, class RY>
__device__ inline void warp_gemm(int lane, int rows, int K, const R* __restrict__ W, int Nout, const R* __restrict__ b,
                                 RX rx, RY ry) {
  auto ldw = [&](const R* p) { return LDG ? __ldg(p) : *p; };
  for (int col = lane; col < Nout; col += 32) {
    const R bias = b ? __ldg(b + col) : R(0);
    const R* wc = W + col;
    for (int r0 = 0; r0 < rows; r0 += 4) {
      const R* x0 = rx(r0);
      const R* x1 = rx(min(r0 + 1, rows - 1));
      const R* x2 = rx(min(r0 + 2, rows - 1));
      const R* x3 = rx(min(r0 + 3, rows - 1));
      R a0 = bias, a1 = bias, a2 = bias, a3 = bias;
      int k = 0;
      if constexpr (sizeof(R) == 4) {
        // rows are 16-byte aligned with K a multiple of 4: one 128-bit
        // shared load brings four k values of a row
        if ((K & 3) == 0) {
#pragma unroll 2
          for (; k < K; k += 4) {
            const float4 p0 = *(const float4*)(x0 + k), p1 = *(const float4*)(x1 + k);
            const float4 p2 = *(const float4*)(x2 + k), p3 = *(const float4*)(x3 + k);
            const R w0 = ldw(wc + (size_t)k * Nout), w1 = ldw(wc + (size_t)(k + 1) * Nout);
            const R w2 = ldw(wc + (size_t)(k + 2) * Nout), w3 = ldw(wc + (size_t)(k + 3) * Nout);
            a0 += p0.x * w0 + p0.y * w1 + p0.z * w2 + p0.w * w3;
            a1 += p1.x * w0 + p1.y * w1 + p1.z * w2 + p1.w * w3;
            a2 += p2.x * w0 + p2.y * w1 + p2.z * w2 + p2.w * w3;
            a3 += p3.x * w0 + p3.y * w1 + p3.z * w2 + p3.w * w3;
          }
        }
      }
#pragma unroll 4
      for (; k < K; ++k) {
        const R w = ldw(wc + (size_t)k * Nout);
        a0 += x0[k] * w;
        a1 += x1[k] * w;
        a2 += x2[k] * w;
        a3 += x3[k] * w;
      }
      const R v[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (r0 + q >= rows) break;
        const R val = SSP ? ssp_(v[q]) : v[q];
        R* y = ry(r0 + q) + col;
        *y = ACC ? *y + val : val;
      }
    }
  }
}


// Value of every cusp-spliced orbital at every electron, spread over the
// warp: lanes first take (electron, shell) radial parts, then (electron,
// orbital) contractions, so that each instruction does up to 32 lanes of
// work (this matters most in float64, whose warp instructions cost the same
// on GB300 whatever the active lane count).  Arithmetic in C (double in
// PN_FP64, float in PN_MIXED, where only the acceptance ratio needs it).
// rp: [N][3] positions in C; rad: [N][n_shells] scratch; ic: [N].
template <typename C>
__device__ inline void warp_orbitals(const DevSys& s, int lane, const C* __restrict__ rp, C* __restrict__ phi,
                                     C* __restrict__ rad, int* __restrict__ ic) {
  const OrbTab<C> t = orb_tab<C>(s);
  const int N = s.N, ns = s.n_shells, no = s.n_orb;
  for (int i = lane; i < N; i += 32) {
    int Ic = -1;
    if (s.use_cusp)
      for (int I = 0; I < s.M; ++I) {
        const C v0 = rp[3 * i] - t.R[3 * I], v1 = rp[3 * i + 1] - t.R[3 * I + 1], v2 = rp[3 * i + 2] - t.R[3 * I + 2];
        if (v0 * v0 + v1 * v1 + v2 * v2 < t.rc[I] * t.rc[I]) Ic = I;
      }
    ic[i] = Ic;
  }
  for (int q = lane; q < N * ns; q += 32) {
    const int i = q / ns, sh = q % ns;
    const int c = s.sh_center[sh], np = s.sh_nprim[sh], po = s.sh_poff[sh];
    const C v0 = rp[3 * i] - t.R[3 * c], v1 = rp[3 * i + 1] - t.R[3 * c + 1], v2 = rp[3 * i + 2] - t.R[3 * c + 2];
    const C r2 = v0 * v0 + v1 * v1 + v2 * v2;
    C e = 0;
    if (s.sh_l[sh] == -1) {
      e = t.pcoef[po] * exp(-t.pexp[po] * sqrt(r2));
    } else {
      for (int k = 0; k < np; ++k) e += t.pcoef[po + k] * exp(-t.pexp[po + k] * r2);
    }
    rad[q] = e;
  }
  __syncwarp();
  for (int q = lane; q < N * no; q += 32) {
    const int i = q / no, mu = q % no;
    const int Ic = ic[i];
    C acc = 0;
    for (int sh = 0; sh < ns; ++sh) {
      const int c = s.sh_center[sh], l = s.sh_l[sh], bo = s.sh_boff[sh];
      const C e = rad[i * ns + sh];
      if (l <= 0) {
        if (l == 0 && c == Ic && s.cusp_on[Ic * no + mu]) continue;  // replaced inside the cusp sphere
        acc += t.mo[(size_t)bo * no + mu] * e;
        continue;
      }
      const C v0 = rp[3 * i] - t.R[3 * c], v1 = rp[3 * i + 1] - t.R[3 * c + 1], v2 = rp[3 * i + 2] - t.R[3 * c + 2];
      const C* m = t.mo + (size_t)bo * no + mu;
      if (l == 1) {
        acc += e * (m[0] * v0 + m[no] * v1 + m[2 * no] * v2);
      } else {
        acc += e * (m[0] * v0 * v0 + m[no] * v0 * v1 + m[2 * no] * v0 * v2 + m[3 * no] * v1 * v1 +
                    m[4 * no] * v1 * v2 + m[5 * no] * v2 * v2);
      }
    }
    if (Ic >= 0 && s.cusp_on[Ic * no + mu]) {
      const C v0 = rp[3 * i] - t.R[3 * Ic], v1 = rp[3 * i + 1] - t.R[3 * Ic + 1], v2 = rp[3 * i + 2] - t.R[3 * Ic + 2];
      const C d = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      const int k = Ic * no + mu;
      const C* a = t.ca + (size_t)k * 5;
      const C p = a[0] + d * (a[1] + d * (a[2] + d * (a[3] + d * a[4])));
      acc += t.cC[k] + t.cs[k] * exp(p);
    }
    phi[q] = acc;
  }
  __syncwarp();
}

__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (bar_try(bar, parity)) return true;
  return false;
}

// STAGED: the warps of a block walk the network in lockstep and each
// weight block is bulk-copied (cp.async.bulk, completion on an mbarrier)
// from the packed weights into one of two shared buffers, one stage ahead
// of its use.  Otherwise each warp reads the packed weights through L1.
template <typename R, bool STAGED>
__global__ void __launch_bounds__(256) k_metropolis_warp(DevSys s, DevNet<R> net, WLayout L, StageTab st,
                                                         const R* __restrict__ wpack, int wbuf_off, int wbuf_bytes,
                                                         double* __restrict__ r, double* __restrict__ lp, int W,
                                                         unsigned walker0, int n_steps, double sigma,
                                                         unsigned long long seed, unsigned long long step0,
                                                         unsigned long long* __restrict__ n_acc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t wbar[2];
  __shared__ int abort_flag;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, tid = threadIdx.x;
  const int w = blockIdx.x * (blockDim.x >> 5) + wid;
  const bool active = w < W;
  if (!STAGED && !active) return;  // without block barriers idle warps can leave
  unsigned char* base = smem + (size_t)wid * L.bytes;
  double* sr = (double*)(base + L.r);
  double* srp = (double*)(base + L.rp);
  R* srpf = (R*)(base + L.rpf);
  R* sdr = (R*)(base + L.dr);
  R* sphi = (R*)(base + L.phi);
  R* srad = (R*)(base + L.rad);
  int* sic = (int*)(base + L.ic);
  double* sdet = (double*)(base + L.det);
  R* sx = (R*)(base + L.x);
  R* sh = (R*)(base + L.h);
  R* sz = (R*)(base + L.z);
  R* swv = (R*)(base + L.wv);
  R* shid = (R*)(base + L.hid);
  R* se = (R*)(base + L.e);
  R* sF = (R*)(base + L.F);
  R* sxs = (R*)(base + L.xs);
  R* sa1 = (R*)(base + L.a1s);
  R* sa2 = (R*)(base + L.a2s);
  R* sJ = (R*)(base + L.J);
  R* wbuf[2] = {(R*)(smem + wbuf_off), (R*)(smem + wbuf_off + wbuf_bytes)};
  const int N = s.N, P = s.Ppair, D = s.D, Zd = s.Zd, K = s.K, Hw = s.Hw, no = s.n_orb, nd = s.n_det;
  const int n3 = 3 * N, nblk4 = (n3 + 3) / 4;
  const NetOff& o = net.off;
  const unsigned wid_g = walker0 + (unsigned)w;

  // -- weight stages
  const long total = (long)n_steps * st.n;
  long g = 0;  // stage counter over all steps
  auto issue = [&](long q) {
    if (q >= total) return;
    const int j = (int)(q % st.n), b = (int)(q & 1);
    const uint32_t bar = smem_addr(&wbar[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(st.bytes[j]) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(wbuf[b])),
                 "l"(wpack + st.off[j]), "r"(st.bytes[j]), "r"(bar)
                 : "memory");
  };
  auto acquire = [&]() -> const R* {
    const int j = (int)(g % st.n);
    if (!STAGED) return wpack + st.off[j];
    const int b = (int)(g & 1);
    if (!bar_wait(smem_addr(&wbar[b]), (uint32_t)((g >> 1) & 1))) abort_flag = 1;
    return wbuf[b];
  };
  auto release = [&]() {
    if (STAGED) {
      __syncthreads();  // every warp is done with this buffer
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(g + 2);
      }
    }
    ++g;
  };
  if (STAGED) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&wbar[0])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&wbar[1])));
      asm volatile("fence.mbarrier_init.release.cluster;");
      abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0) {
      issue(0);
      issue(1);
    }
  }

  double lpw = 0;
  unsigned naccw = 0;
  if (active) {
    for (int i = lane; i < n3; i += 32) sr[i] = r[(size_t)w * n3 + i];
    lpw = lp[w];
  }
  __syncwarp();
  for (int k = 0; k < n_steps; ++k) {
    const unsigned long long step = step0 + (unsigned long long)k;
    if (active) {
      // proposal; positions stay float64, the value pass reads an R copy
      for (int q = lane; q < 2 * nblk4; q += 32) {
        const int j = q >> 1, pr = q & 1;
        if (4 * j + 2 * pr >= n3) continue;
        R zz[2];
        normal_pair<R>(seed, wid_g, step, j, pr, zz);
        for (int t = 0; t < 2; ++t) {
          const int m = 4 * j + 2 * pr + t;
          if (m < n3) {
            srp[m] = sr[m] + sigma * (double)zz[t];
            srpf[m] = (R)srp[m];
          }
        }
      }
      __syncwarp();
      const OrbTab<R> tab = orb_tab<R>(s);
      for (int p = lane; p < P; p += 32) {
        R v[3];
        if (p < s.Pee) {
          int a = 0, rem = p;
          while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
          const int bb = a + 1 + rem;
          for (int x = 0; x < 3; ++x) v[x] = srpf[3 * a + x] - srpf[3 * bb + x];
        } else {
          const int q = p - s.Pee, i = q / s.M, I = q % s.M;
          for (int x = 0; x < 3; ++x) v[x] = srpf[3 * i + x] - tab.R[3 * I + x];
        }
        sdr[p] = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      }
      warp_orbitals<R>(s, lane, srpf, sphi, srad, sic);
      for (int q = lane; q < N * D; q += 32) sx[q] = net.p[o.x0 + q % D];
      __syncwarp();
    }
    for (int n = 0; n < s.L; ++n) {
      {
        const R* Wt = acquire();
        if (active)
          warp_gemm<R, false, false, !STAGED>(
              lane, N, D, Wt, Zd, net.p + o.hb[n], [&](int q) { return (const R*)(sx + (size_t)q * D); },
              [&](int q) { return sh + (size_t)q * Zd; });
        release();
      }
      for (int c = 0; c < 3; ++c) {
        const int cnt = s.ch_off[c + 1] - s.ch_off[c];
        const int* pl = s.ch_pairs + s.ch_off[c];
        {
          const R* Wt = acquire();
          if (active && cnt > 0) {
            // distance features of this channel's pairs
            const R* fm = feat_mu_of<R>(s);
            const R* fi = feat_is_of<R>(s);
            for (int q = lane; q < cnt * K; q += 32) {
              const int gg = q / K, kk = q % K;
              const R d = sdr[pl[gg]];
              const R dm = d - fm[kk];
              se[q] = d * d * exp(-d - dm * dm * fi[kk]);
            }
            __syncwarp();
            warp_gemm<R, true, false, !STAGED>(
                lane, cnt, K, Wt, Hw, net.p + o.b1[n][c], [&](int q) { return (const R*)(se + (size_t)q * K); },
                [&](int q) { return shid + (size_t)q * Hw; });
            __syncwarp();
          }
          release();
        }
        {
          const R* Wt = acquire();
          if (active && cnt > 0) {
            warp_gemm<R, false, false, !STAGED>(
                lane, cnt, Hw, Wt, Zd, net.p + o.b2[n][c], [&](int q) { return (const R*)(shid + (size_t)q * Hw); },
                [&](int q) { return swv + (size_t)pl[q] * Zd; });
            __syncwarp();
          }
          release();
        }
      }
      {
        const R* Wt = acquire();
        if (active) {
          for (int q = lane; q < N * Zd; q += 32) {
            const int z = q % Zd, i = q / Zd;
            R zs = 0, za = 0, zn = 0;
            const bool si = i < s.n_up;
            for (int j = 0; j < N; ++j) {
              if (j == i) continue;
              const int p = i < j ? pn_pair_index(i, j, N) : pn_pair_index(j, i, N);
              const R v = swv[(size_t)p * Zd + z] * sh[(size_t)j * Zd + z];
              if ((j < s.n_up) == si) zs += v; else za += v;
            }
            for (int I = 0; I < s.M; ++I) zn += swv[(size_t)(s.Pee + i * s.M + I) * Zd + z] * net.p[o.Y + I * Zd + z];
            R* zo = sz + (size_t)i * 3 * Zd;
            zo[z] = zs;
            zo[Zd + z] = za;
            zo[2 * Zd + z] = zn;
          }
          __syncwarp();
          warp_gemm<R, false, true, !STAGED>(
              lane, N, 3 * Zd, Wt, D, net.Gb + (size_t)n * D,
              [&](int q) { return (const R*)(sz + (size_t)q * 3 * Zd); }, [&](int q) { return sx + (size_t)q * D; });
          __syncwarp();
        }
        release();
      }
    }
    // heads: kappa on every electron, eta on the electron sum
    {
      const R* Wt = acquire();
      if (active) {
        for (int dd = lane; dd < D; dd += 32) {
          R acc = 0;
          for (int i = 0; i < N; ++i) acc += sx[(size_t)i * D + dd];
          sxs[dd] = acc;
        }
        warp_gemm<R, true, false, !STAGED>(
            lane, N, D, Wt, D, net.p + o.kb[0], [&](int q) { return (const R*)(sx + (size_t)q * D); },
            [&](int q) { return sz + (size_t)q * D; });
        __syncwarp();
      }
      release();
    }
    {
      const R* Wt = acquire();
      if (active) {
        warp_gemm<R, true, false, !STAGED>(
            lane, N, D, Wt, D, net.p + o.kb[1], [&](int q) { return (const R*)(sz + (size_t)q * D); },
            [&](int q) { return swv + (size_t)q * D; });
        __syncwarp();
      }
      release();
    }
    {
      const R* Wt = acquire();
      if (active) {
        warp_gemm<R, false, false, !STAGED>(
            lane, N, D, Wt, no, net.p + o.kb[2], [&](int q) { return (const R*)(swv + (size_t)q * D); },
            [&](int q) { return sF + (size_t)q * no; });
        __syncwarp();
      }
      release();
    }
    {
      const R* Wt = acquire();
      if (active) {
        warp_gemm<R, true, false, !STAGED>(
            lane, 1, D, Wt, D, net.p + o.eb[0], [&](int q) { return (const R*)sxs; }, [&](int q) { return sa1; });
        __syncwarp();
      }
      release();
    }
    {
      const R* Wt = acquire();
      if (active) {
        warp_gemm<R, true, false, !STAGED>(
            lane, 1, D, Wt, D, net.p + o.eb[1], [&](int q) { return (const R*)sa1; }, [&](int q) { return sa2; });
        __syncwarp();
      }
      release();
    }
    {
      const R* Wt = acquire();
      if (active) {
        warp_gemm<R, false, false, !STAGED>(
            lane, 1, D, Wt, 1, net.p + o.eb[2], [&](int q) { return (const R*)sa2; }, [&](int q) { return sJ; });
        __syncwarp();
      }
      release();
    }
    if (active) {
      // determinants: one lane per (determinant, spin)
      for (int q = lane; q < nd * 2; q += 32) {
        const int sp = q & 1, p = q >> 1;
        const int ns = sp ? s.n_dn : s.n_up, e0 = sp ? s.n_up : 0;
        double ld = 0, sg = 1;
        if (ns > 0) {
          double A[PN_MAX_SPIN * PN_MAX_SPIN];
          const int* occ = s.occ + p * N + e0;
          for (int a = 0; a < ns; ++a)
            for (int bb = 0; bb < ns; ++bb) {
              const int i = e0 + a, mu = occ[bb];
              A[a * ns + bb] = (double)sphi[(size_t)i * no + mu] * (1.0 + (double)sF[(size_t)i * no + mu]);
            }
          pn_slogdet(A, ns, &ld, &sg);
        }
        sdet[2 * q] = ld;
        sdet[2 * q + 1] = sg;
      }
      __syncwarp();
      // signed log-sum over determinants and gamma, reduced across lanes
      double m = -INFINITY;
      for (int p = lane; p < nd; p += 32) {
        const double sg = sdet[4 * p + 1] * sdet[4 * p + 3];
        if (s.ci[p] != 0.0 && sg != 0.0) m = fmax(m, sdet[4 * p] + sdet[4 * p + 2]);
      }
      for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
      double S = 0;
      R gam = 0;
      if (m > -INFINITY)
        for (int p = lane; p < nd; p += 32) {
          const double sg = sdet[4 * p + 1] * sdet[4 * p + 3];
          if (sg != 0.0) S += s.ci[p] * sg * exp(sdet[4 * p] + sdet[4 * p + 2] - m);
        }
      if (s.use_gamma)
        for (int p = lane; p < s.Pee; p += 32) {
          int a = 0, rem = p;
          while (rem >= N - 1 - a) { rem -= N - 1 - a; ++a; }
          const int bb = a + 1 + rem;
          const R c = ((a < s.n_up) == (bb < s.n_up)) ? R(0.25) : R(0.5);
          gam -= c / (R(1) + sdr[p]);
        }
      for (int off = 16; off > 0; off >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, off);
        gam += __shfl_xor_sync(0xffffffffu, gam, off);
      }
      const double lpn = (double)gam + (double)sJ[0] + m + log(fabs(S));
      unsigned c4[4] = {(unsigned)nblk4, wid_g, (unsigned)(step & 0xffffffffull), (unsigned)(step >> 32)};
      pn_philox(c4, (unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
      bool accept;
      if constexpr (sizeof(R) == 8) {
        accept = pn_u01(c4[0]) < exp(2.0 * (lpn - lpw));
      } else {
        accept = ((float)c4[0] + 0.5f) * 2.3283064365386963e-10f < expf((float)(2.0 * (lpn - lpw)));
      }
      if (accept) {
        for (int q = lane; q < n3; q += 32) sr[q] = srp[q];
        lpw = lpn;
        ++naccw;
      }
      __syncwarp();
    }
    if (STAGED && abort_flag) break;  // uniform: read after the last release's barrier
  }
  if (STAGED && abort_flag) {
    // a weight copy did not arrive in time: flag it, give the copies in
    // flight a last bounded wait and leave the walkers at their last state
    if (tid == 0) atomicExch(s.dev_err, 2);
    bar_wait(smem_addr(&wbar[g & 1]), (uint32_t)((g >> 1) & 1));
    bar_wait(smem_addr(&wbar[(g + 1) & 1]), (uint32_t)(((g + 1) >> 1) & 1));
  }
  if (active) {
    for (int i = lane; i < n3; i += 32) r[(size_t)w * n3 + i] = sr[i];
    if (lane == 0) {
      lp[w] = lpw;
      if (n_acc && naccw) atomicAdd(n_acc, (unsigned long long)naccw);
    }
  }
}

}  // namespace

// Tile size for the fused sampler, 0 when even one walker does not fit.
template <typename R>
int pn_fused_tile(const DevSys& s, int W, int* smem_bytes) {
  int dev = 0, sms = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t cap = (size_t)maxsm - 1024;
  if (make_layout<R>(s, 1).bytes > cap) return 0;
  // aim for every SM busy with a couple of resident tiles
  int want = std::max(1, (W + 2 * sms - 1) / (2 * sms));
  int WT = std::min(want, 64);
  while (WT > 1 && make_layout<R>(s, WT).bytes > cap / 2) --WT;
  *smem_bytes = (int)make_layout<R>(s, WT).bytes;
  return WT;
}

template <typename R>
int pn_run_metropolis_fused(const DevSys& s, const DevNet<R>& net, double* r, double* lp, int W, unsigned walker0,
                            int n_steps, double sigma, unsigned long long seed, unsigned long long step0,
                            unsigned long long* n_acc, cudaStream_t st) {
  // small systems: one warp per walker when a walker's state is small
  const WLayout WL = make_wlayout<R>(s);
  if (s.fused_sampler != 2 && WL.bytes <= 24 * 1024) {  // 1, 3 (and 4 when the tensor-core tiles do not fit)
    const StageTab& stt = net.stab;
    const R* wp = net.wpack;
    int warps = (int)std::min<size_t>(8, (200 * 1024) / WL.bytes);
    // lockstep with shared weight buffers when two of the largest block fit beside the warps' state
    int wbuf_bytes = (stt.max_bytes + 127) / 128 * 128;
    const size_t cap = 220 * 1024;
    // TMA-fed lockstep only on request: measured slower on the Be workload
    // (its 128 registers per thread halve the resident warps)
    bool staged = s.fused_sampler == 3;
    while (staged && warps > 1 && WL.bytes * warps + 2 * (size_t)wbuf_bytes > cap) --warps;
    if (WL.bytes * warps + 2 * (size_t)wbuf_bytes > cap) staged = false;
    const int wbuf_off = (int)((WL.bytes * warps + 127) / 128 * 128);
    const int smem = staged ? wbuf_off + 2 * wbuf_bytes : (int)(WL.bytes * warps);
    const int blocks = (W + warps - 1) / warps;
    if (staged) {
      PN_CUDA(pn_allow_max_smem(k_metropolis_warp<R, true>));
      PN_LAUNCH_W("k_metropolis_warp", st, (double)W * n_steps * pn_value_pass_flops(s),
                k_metropolis_warp<R, true><<<blocks, warps * 32, smem, st>>>(
                    s, net, WL, stt, wp, wbuf_off, wbuf_bytes, r, lp, W, walker0, n_steps, sigma, seed, step0, n_acc));
    } else {
      PN_CUDA(pn_allow_max_smem(k_metropolis_warp<R, false>));
      PN_LAUNCH_W("k_metropolis_warp", st, (double)W * n_steps * pn_value_pass_flops(s),
                k_metropolis_warp<R, false><<<blocks, warps * 32, smem, st>>>(
                    s, net, WL, stt, wp, 0, 0, r, lp, W, walker0, n_steps, sigma, seed, step0, n_acc));
    }
    return PN_OK;
  }
  int smem = 0;
  const int WT = pn_fused_tile<R>(s, W, &smem);
  if (WT == 0) return PN_ENOTREADY;  // caller takes the staged path
  const Layout L = make_layout<R>(s, WT);
  PN_CUDA(pn_allow_max_smem(k_metropolis_fused<R>));
  const int tiles = (W + WT - 1) / WT;
  PN_LAUNCH_W("k_metropolis_fused", st, (double)W * n_steps * pn_value_pass_flops(s),
            k_metropolis_fused<R><<<tiles, 256, smem, st>>>(s, net, L, r, lp, W, walker0, n_steps, sigma, seed, step0,
                                                           n_acc));
  return PN_OK;
}
template int pn_run_metropolis_fused<double>(const DevSys&, const DevNet<double>&, double*, double*, int, unsigned,
                                             int, double, unsigned long long, unsigned long long, unsigned long long*,
                                             cudaStream_t);
template int pn_run_metropolis_fused<float>(const DevSys&, const DevNet<float>&, double*, double*, int, unsigned, int,
                                            double, unsigned long long, unsigned long long, unsigned long long*,
                                            cudaStream_t);
