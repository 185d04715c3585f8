// Multi-determinant jet by the table method.
//
// The determinants of one spin share their rows (the electrons) and differ
// in a few columns (orbitals): determinant p takes the reference
// determinant 0's occupation with k_p orbitals replaced.  With A the n x
// (n + n_virt) matrix of the backflowed orbitals phi~ over the reference and
// the virtual orbitals, A_0 its reference block and T = A_0^-1 A,
//   det A_p = s_p det A_0 det R_p,   R_p = T[holes_p, particles_p] (k_p x k_p),
// (Jacobi's formula and the determinant of a matrix that differs from the
// identity in k columns), so that
//   d_t ln|det A_p| = tr(A_0^-1 d_t A_0) + tr(R_p^-1 d_t R_p),
//   lap ln|det A_p| = [tr(A_0^-1 lap A_0) - sum_t tr((A_0^-1 d_t A_0)^2)]
//                   + [tr(R_p^-1 lap R_p) - sum_t tr((R_p^-1 d_t R_p)^2)],
// with d_t T = A_0^-1 (d_t A - d_t A_0 T) and
//   lap T = A_0^-1 (lap A - lap A_0 T - 2 sum_t d_t A_0 d_t T).
// The same quantities as the direct per-block kernel, exactly in exact
// arithmetic, for about an eighth of the float64 work of the N2-shaped
// system (32 determinants of 7 x 7 blocks).  T carries rounding amplified by
// the condition of A_0 (the derivatives about its square, through the
// cancellation of the reference and minor terms), so a walker whose
// reference block has a 1-norm condition number beyond kCondMax is computed
// directly, block by block.
//
// One warp per (walker, spin); the warp's matrices live in shared memory.
#include <math.h>

#include "kernels.cuh"
#include "pn_internal.cuh"
#include "slater_dev.cuh"

namespace {

// warps per block: two, so that a warp that takes long (the block-by-block
// path of an ill-conditioned walker) holds only one other warp's shared
// memory until it ends
constexpr int TW = 2;
constexpr int TW_BLOCKS = 10;  // blocks per SM the registers must allow (at most 102 a thread: 20 warps)
constexpr double kCondMax = 1e3;    // largest 1-norm condition number of A_0 for the table method (jet)
constexpr double kCondMaxValue = 1e5;  // the same for ln|det| alone

inline unsigned nblk(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// k x k LU with partial pivoting and inverse (k <= PN_TAB_KMAX); false if
// exactly singular.
__device__ inline bool small_inverse(const double* Rm, int k, double* Ri, double* ld, double* sg) {
  double L[PN_TAB_KMAX * PN_TAB_KMAX];
  int pm[PN_TAB_KMAX];
  for (int q = 0; q < k * k; ++q) L[q] = Rm[q];
  for (int c = 0; c < k; ++c) pm[c] = c;
  double l = 0, s = 1;
  for (int c = 0; c < k; ++c) {
    int b = c;
    double bv = fabs(L[c * k + c]);
    for (int r = c + 1; r < k; ++r)
      if (fabs(L[r * k + c]) > bv) { bv = fabs(L[r * k + c]); b = r; }
    if (!(bv > 0.0)) return false;
    if (b != c) {
      for (int q = 0; q < k; ++q) { const double t = L[c * k + q]; L[c * k + q] = L[b * k + q]; L[b * k + q] = t; }
      const int t = pm[c]; pm[c] = pm[b]; pm[b] = t;
      s = -s;
    }
    const double piv = L[c * k + c];
    if (piv < 0) s = -s;
    l += log(fabs(piv));
    for (int r = c + 1; r < k; ++r) {
      const double f = L[r * k + c] / piv;
      L[r * k + c] = f;
      for (int q = c + 1; q < k; ++q) L[r * k + q] -= f * L[c * k + q];
    }
  }
  for (int col = 0; col < k; ++col) {
    double y[PN_TAB_KMAX];
    for (int r = 0; r < k; ++r) {
      double v = pm[r] == col ? 1.0 : 0.0;
      for (int q = 0; q < r; ++q) v -= L[r * k + q] * y[q];
      y[r] = v;
    }
    for (int r = k - 1; r >= 0; --r) {
      double v = y[r];
      for (int q = r + 1; q < k; ++q) v -= L[r * k + q] * y[q];
      y[r] = v / L[r * k + r];
    }
    for (int r = 0; r < k; ++r) Ri[r * k + col] = y[r];
  }
  *ld = l;
  *sg = s;
  return true;
}

// Packed minor records of one spin: determinant p's starts after those of
// determinants 0..p-1, each k^2 + 3 doubles.
__device__ inline int pn_table_minor_offset(const int* recs, int p, int sg) {
  int off = 0;
  for (int q = 0; q < p; ++q) {
    const int k = recs[(size_t)(2 * q + sg) * PN_TAB_REC];
    off += k * k + 3;
  }
  return off;
}
__device__ inline int pn_table_minor_doubles(const int* recs, int nd, int sg) {
  return pn_table_minor_offset(recs, nd, sg);
}

template <typename R>
__global__ void __launch_bounds__(TW * 32, TW_BLOCKS) k_slater_table(DevSys s, const double* __restrict__ phi,
                                                          const R* __restrict__ F, int Wn, int T, int jet,
                                                          double* __restrict__ det) {
  extern __shared__ __align__(16) double tsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = blockIdx.x * TW + wid;
  if (gw >= 2 * Wn) return;  // the whole warp leaves together
  const int w = gw >> 1, sg = gw & 1;
  const int N = s.N, no = s.n_orb, n3 = 3 * N, lap = T - 1, stride = 3 + n3, nd = s.n_det;
  const int n = sg ? s.n_dn : s.n_up, e0 = sg ? s.n_up : 0;
  double* outw = det + (size_t)w * nd * 2 * stride;
  const double* phw = phi + (size_t)w * N * no * 5;
  const R* Fw = F + (size_t)w * N * T * no;
  if (n == 0) {
    for (int p = 0; p < nd; ++p) {
      double* o = outw + (size_t)(2 * p + sg) * stride;
      for (int q = lane; q < stride; q += 32) o[q] = q == 1 ? 1.0 : 0.0;
    }
    return;
  }
  const int* hdr = s.xtab + sg * (1 + PN_MAX_ORBITALS);
  const int nv = hdr[0];
  const int* V = hdr + 1;
  const int* occ0 = s.occ + e0;
  const int ncol = n + nv;
  double* Af = tsm + (size_t)wid * s.tab_wstride;  // [n][ncol] values
  double* LA = Af + n * ncol;                      // [n][ncol] Laplacians
  double* dA = LA + n * ncol;                      // [n][ncol] current tangent
  double* LU = dA + n * ncol;                      // [n][n]
  double* M = LU + n * n;                          // [n][n] A_0^-1
  double* B = M + n * n;                           // [n][n] A_0^-1 d_t A_0
  double* Tv = B + n * n;                          // [n][nv]
  double* Dt = Tv + n * nv;                        // [n][nv]
  double* S = Dt + n * nv;                         // [n][nv] sum_t d_t A_0 d_t T
  double* LTv = S + n * nv;                        // [n][nv] lap T
  double* g0 = LTv + n * nv;                       // [3N] reference gradient
  double* dT = g0 + n3;                            // [3N][n][nv]
  int* perm = (int*)(dT + (size_t)n3 * n * nv);    // [n]
  // the determinants' minors, packed (per determinant R_p^-1 then ln|det
  // R_p|, its sign -- 0 if singular -- and tr(R_p^-1 lap R_p)): over the
  // region Af..B, dead by then, where it fits (pn_table_minor_doubles),
  // else after perm
  const int* recs = s.xtab + 2 * (1 + PN_MAX_ORBITALS);
  const int rd_need = pn_table_minor_doubles(recs, nd, sg);
  double* RD = rd_need <= 3 * n * ncol + 3 * n * n ? Af : dT + (size_t)n3 * n * nv + n + 2;
  auto mu_of = [&](int c) { return c < n ? occ0[c] : V[c - n]; };

  for (int q = lane; q < n * ncol; q += 32) {
    const int a = q / ncol, c = q - a * ncol, i = e0 + a, mu = mu_of(c);
    const double* ph = phw + (i * no + mu) * 5;
    const R* f = Fw + (size_t)i * T * no + mu;
    Af[q] = ph[0] * (1.0 + (double)f[0]);
    if (jet) LA[q] = pn_aelem_lap(ph, f, no, i, lap);
  }
  for (int q = lane; q < n * nv; q += 32) S[q] = 0.0;
  if (lane < n) perm[lane] = lane;
  __syncwarp();
  for (int q = lane; q < n * n; q += 32) LU[q] = Af[(q / n) * ncol + q % n];
  __syncwarp();
  // LU of the reference block, rows spread over the lanes
  double ld = 0, sgn = 1;
  bool sing = false;
  for (int c = 0; c < n; ++c) {
    double v = (lane >= c && lane < n) ? fabs(LU[lane * n + c]) : -1.0;
    int bi = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int b2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (v2 > v || (v2 == v && b2 < bi)) { v = v2; bi = b2; }
    }
    if (!(v > 0.0)) { sing = true; break; }
    if (bi != c) {
      for (int k = lane; k < n; k += 32) {
        const double t0 = LU[c * n + k];
        LU[c * n + k] = LU[bi * n + k];
        LU[bi * n + k] = t0;
      }
      if (lane == 0) { const int tp = perm[c]; perm[c] = perm[bi]; perm[bi] = tp; }
      sgn = -sgn;
    }
    __syncwarp();
    const double piv = LU[c * n + c];
    if (piv < 0) sgn = -sgn;
    ld += log(fabs(piv));
    if (lane > c && lane < n) {
      const double f = LU[lane * n + c] / piv;
      LU[lane * n + c] = f;
      for (int k = c + 1; k < n; ++k) LU[lane * n + k] -= f * LU[c * n + k];
    }
    __syncwarp();
  }
  // M = A_0^-1, one column per lane
  if (!sing && lane < n) {
    double y[PN_TAB_NMAX];
    for (int r = 0; r < n; ++r) {
      double v = perm[r] == lane ? 1.0 : 0.0;
      for (int k = 0; k < r; ++k) v -= LU[r * n + k] * y[k];
      y[r] = v;
    }
    for (int r = n - 1; r >= 0; --r) {
      double v = y[r];
      for (int k = r + 1; k < n; ++k) v -= LU[r * n + k] * y[k];
      y[r] = v / LU[r * n + r];
    }
    for (int r = 0; r < n; ++r) M[r * n + lane] = y[r];
  }
  __syncwarp();
  // 1-norm condition number of A_0: max column sums of |A_0| and |M|
  double ca = 0, cm = 0;
  if (!sing && lane < n)
    for (int r = 0; r < n; ++r) {
      ca += fabs(Af[r * ncol + lane]);
      cm += fabs(M[r * n + lane]);
    }
  for (int o = 16; o > 0; o >>= 1) {
    ca = fmax(ca, __shfl_xor_sync(0xffffffffu, ca, o));
    cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
  }
  // value mode needs no derivative, so its rounding grows only with the
  // condition number itself
  if (sing || !(ca * cm <= (jet ? kCondMax : kCondMaxValue)) || s.no_table == 2) {
    // ill-conditioned reference block: every determinant directly
    for (int p = lane; p < nd; p += 32)
      pn_slater_block<R, PN_TAB_NMAX>(s, phw, Fw, p, sg, T, jet, outw + (size_t)(2 * p + sg) * stride);
    return;
  }
  for (int q = lane; q < n * nv; q += 32) {
    const int a = q / nv, v = q - a * nv;
    double x = 0;
    for (int c = 0; c < n; ++c) x += M[a * n + c] * Af[c * ncol + n + v];
    Tv[q] = x;
  }
  __syncwarp();
  if (!jet) {
    // ln|det| and sign of every determinant from its minor of T
    for (int p = lane; p < nd; p += 32) {
      const int* rec = recs + (size_t)(2 * p + sg) * PN_TAB_REC;
      const int k = rec[0];
      double Rm[PN_TAB_KMAX * PN_TAB_KMAX], Ri[PN_TAB_KMAX * PN_TAB_KMAX];
      double ldR = 0, sR = 1;
      for (int r = 0; r < k; ++r)
        for (int q = 0; q < k; ++q) Rm[r * k + q] = Tv[rec[2 + r] * nv + rec[2 + PN_TAB_KMAX + q]];
      double* o = outw + (size_t)(2 * p + sg) * stride;
      if (k > 0 && !small_inverse(Rm, k, Ri, &ldR, &sR)) {
        o[0] = -INFINITY;
        o[1] = 0.0;
        continue;
      }
      o[0] = ld + ldR;
      o[1] = sgn * rec[1] * sR;
    }
    return;
  }
  // tangents, one after another, the warp's lanes over matrix entries
  double l2 = 0;
  for (int t = 1; t < lap; ++t) {
    for (int q = lane; q < n * ncol; q += 32) {
      const int a = q / ncol, c = q - a * ncol, i = e0 + a, mu = mu_of(c);
      dA[q] = pn_aelem_tangent(phw + (i * no + mu) * 5, Fw + (size_t)i * T * no + mu, no, i, t);
    }
    __syncwarp();
    double tr1 = 0, tr2 = 0;
    for (int q = lane; q < n * n; q += 32) {
      const int a = q / n, b = q - a * n;
      double x = 0;
      for (int c = 0; c < n; ++c) x += M[a * n + c] * dA[c * ncol + b];
      B[q] = x;
    }
    for (int q = lane; q < n * nv; q += 32) {
      const int a = q / nv, v = q - a * nv;
      double x = dA[a * ncol + n + v];
      for (int j = 0; j < n; ++j) x -= dA[a * ncol + j] * Tv[j * nv + v];
      Dt[q] = x;
    }
    __syncwarp();
    for (int q = lane; q < n * n; q += 32) {
      const int a = q / n, b = q - a * n;
      if (a == b) tr1 += B[q];
      tr2 += B[q] * B[b * n + a];
    }
    tr1 = warp_sum(tr1);
    tr2 = warp_sum(tr2);
    if (lane == 0) g0[t - 1] = tr1;
    l2 += tr2;
    double* dTt = dT + (size_t)(t - 1) * n * nv;
    for (int q = lane; q < n * nv; q += 32) {
      const int a = q / nv, v = q - a * nv;
      double x = 0;
      for (int c = 0; c < n; ++c) x += M[a * n + c] * Dt[c * nv + v];
      dTt[q] = x;
    }
    __syncwarp();
    for (int q = lane; q < n * nv; q += 32) {
      const int a = q / nv, v = q - a * nv;
      double x = 0;
      for (int j = 0; j < n; ++j) x += dA[a * ncol + j] * dTt[j * nv + v];
      S[q] += x;
    }
    __syncwarp();
  }
  // reference Laplacian and lap T
  double trl = 0;
  for (int q = lane; q < n * n; q += 32) {
    const int a = q / n, b = q - a * n;
    trl += M[a * n + b] * LA[b * ncol + a];
  }
  trl = warp_sum(trl);
  const double lap0 = trl - l2;
  for (int q = lane; q < n * nv; q += 32) {
    const int a = q / nv, v = q - a * nv;
    double x = LA[a * ncol + n + v] - 2.0 * S[q];
    for (int j = 0; j < n; ++j) x -= LA[a * ncol + j] * Tv[j * nv + v];
    Dt[q] = x;
  }
  __syncwarp();
  for (int q = lane; q < n * nv; q += 32) {
    const int a = q / nv, v = q - a * nv;
    double x = 0;
    for (int c = 0; c < n; ++c) x += M[a * n + c] * Dt[c * nv + v];
    LTv[q] = x;
  }
  __syncwarp();
  // every determinant's minor R_p of T: inverse, ln|det|, sign and
  // tr(R_p^-1 lap R_p), one determinant per lane (the float64 pipe runs a
  // warp instruction at the same cost whatever its active lanes, so the
  // small LUs run side by side rather than one after another)
  for (int p = lane; p < nd; p += 32) {
    const int* rec = recs + (size_t)(2 * p + sg) * PN_TAB_REC;
    const int k = rec[0];
    const int* H = rec + 2;
    const int* P = rec + 2 + PN_TAB_KMAX;
    double* rd = RD + pn_table_minor_offset(recs, p, sg);
    double Rm[PN_TAB_KMAX * PN_TAB_KMAX];
    double ldR = 0, sR = 1;
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) Rm[r * k + q] = Tv[H[r] * nv + P[q]];
    if (k > 0 && !small_inverse(Rm, k, rd, &ldR, &sR)) {
      rd[k * k + 1] = 0.0;
      continue;
    }
    double trlR = 0;
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) trlR += rd[q * k + r] * LTv[H[r] * nv + P[q]];
    rd[k * k] = ldR;
    rd[k * k + 1] = sR;
    rd[k * k + 2] = trlR;
  }
  __syncwarp();
  // then per determinant its tangents, the lanes over the coordinates
  for (int p = 0, off = 0; p < nd; ++p) {
    const int* rec = recs + (size_t)(2 * p + sg) * PN_TAB_REC;
    const int k = rec[0];
    const int* H = rec + 2;
    const int* P = rec + 2 + PN_TAB_KMAX;
    double* o = outw + (size_t)(2 * p + sg) * stride;
    const double* Ri = RD + off;
    off += k * k + 3;
    const double ldR = Ri[k * k], sR = Ri[k * k + 1], trlR = Ri[k * k + 2];
    if (sR == 0.0) {
      for (int q = lane; q < stride; q += 32) o[q] = q == 0 ? -INFINITY : 0.0;
      continue;
    }
    double l2p = 0;
    for (int t0 = lane; t0 < n3; t0 += 32) {
      const double* dTt = dT + (size_t)t0 * n * nv;
      double X[PN_TAB_KMAX * PN_TAB_KMAX];
      double t1 = 0;
      for (int r = 0; r < k; ++r)
        for (int q = 0; q < k; ++q) {
          double x = 0;
          for (int m = 0; m < k; ++m) x += Ri[r * k + m] * dTt[H[m] * nv + P[q]];
          X[r * k + q] = x;
          if (r == q) t1 += x;
        }
      double t2 = 0;
      for (int r = 0; r < k; ++r)
        for (int q = 0; q < k; ++q) t2 += X[r * k + q] * X[q * k + r];
      o[3 + t0] = g0[t0] + t1;
      l2p += t2;
    }
    l2p = warp_sum(l2p);
    if (lane == 0) {
      o[0] = ld + ldR;
      o[1] = sgn * rec[1] * sR;
      o[2] = lap0 + trlR - l2p;
    }
  }
}

}  // namespace

// Float64 work of the table kernel for one walker (multiply-add = 2).
double pn_slater_table_flops(const DevSys& s, int jet) {
  double f = 0;
  for (int sg = 0; sg < 2; ++sg) {
    const double n = sg ? s.n_dn : s.n_up, nv = s.tab_nv[sg], t = 3.0 * s.N;
    if (n == 0) continue;
    f += 2.0 * (2.0 / 3.0 * n * n * n + n * n * n + n * n * nv);   // LU, inverse, T
    if (!jet) {
      f += 2.0 * s.tab_k3[sg] / 3.0;                                 // LU of the minors
      continue;
    }
    f += t * 2.0 * (n * n * n + 3.0 * n * n * nv + n * n);          // per tangent
    f += 2.0 * (n * n + 3.0 * n * n * nv);                           // lap T
    f += t * 2.0 * s.tab_k3[sg];                                     // per determinant and tangent: R^-1 d_t R
  }
  return f;
}

// Jet determinants by the table method when the system has a table and
// the warp's matrices fit in shared memory; PN_ENOTREADY otherwise.
template <typename R>
int pn_slater_table_launch(const DevSys& s, const double* phi, const R* F, int Wn, int T, int jet, double* det,
                           cudaStream_t st) {
  if (!s.xtab || s.tab_wstride <= 0 || Wn <= 0) return PN_ENOTREADY;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem = (size_t)TW * s.tab_wstride * sizeof(double);
  if (smem > (size_t)maxsm) return PN_ENOTREADY;
  PN_CUDA(pn_allow_max_smem(k_slater_table<R>));
  PN_LAUNCH_W("k_slater", st, Wn * pn_slater_table_flops(s, jet),
              k_slater_table<R><<<nblk((size_t)2 * Wn, TW), TW * 32, smem, st>>>(s, phi, F, Wn, T, jet, det));
  return PN_OK;
}
template int pn_slater_table_launch<double>(const DevSys&, const double*, const double*, int, int, int, double*,
                                            cudaStream_t);
template int pn_slater_table_launch<float>(const DevSys&, const double*, const float*, int, int, int, double*,
                                           cudaStream_t);
