// Determinant blocks of the backflowed orbitals, computed one block at a
// time (Eq. ansatz; the derivatives follow Jacobi's formula):
//   A[a][b] = phi_{occ_b}(r_{e0+a}) f_{occ_b, e0+a},  ln|det A| by LU with
//   partial pivoting;  in jet mode also
//   d_t ln|det A| = tr(A^-1 d_t A),
//   lap ln|det A| = tr(A^-1 lap A) - sum_t tr((A^-1 d_t A)^2).
// out = {ln|det|, sign, lap, grad[3N]}.  Shared by the per-block kernel and
// the fallback of the table kernel.
#pragma once

#include <math.h>

#include "pn_internal.cuh"

// Jet of one element of A: value, tangent t, Laplacian (phi depends on r_i
// only; f on every coordinate).  ph = phi jet [5] of (i, mu), f = backflow
// jet column (stride no between rows t).
template <typename R>
__device__ inline double pn_aelem_tangent(const double* ph, const R* f, int no, int i, int t) {
  const int tk = (t - 1) / 3, ta = (t - 1) % 3;
  double v = ph[0] * (double)f[(size_t)t * no];
  if (tk == i) v += ph[1 + ta] * (1.0 + (double)f[0]);
  return v;
}
template <typename R>
__device__ inline double pn_aelem_lap(const double* ph, const R* f, int no, int i, int lap) {
  const double f0 = 1.0 + (double)f[0];
  double l = ph[4] * f0 + ph[0] * (double)f[(size_t)lap * no];
  for (int x = 0; x < 3; ++x) l += 2.0 * ph[1 + x] * (double)f[(size_t)(1 + 3 * i + x) * no];
  return l;
}

// Block (determinant p, spin sg) of one walker directly: phw = phi [N][no][5]
// of the walker, Fw = backflow jet [N][T][no].
template <typename R, int NS>
__device__ inline void pn_slater_block(const DevSys& s, const double* __restrict__ phw, const R* __restrict__ Fw, int p,
                                       int sg, int T, int jet, double* __restrict__ out) {
  const int N = s.N, no = s.n_orb;
  const int ns = sg ? s.n_dn : s.n_up;
  const int e0 = sg ? s.n_up : 0;
  if (ns == 0) {
    out[0] = 0; out[1] = 1; out[2] = 0;
    if (jet) for (int t = 0; t < 3 * N; ++t) out[3 + t] = 0;
    return;
  }
  const int* occ = s.occ + p * N + e0;
  double LU[NS * NS];
  int perm[NS];
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      const int i = e0 + a, mu = occ[b];
      LU[a * ns + b] = phw[(i * no + mu) * 5] * (1.0 + (double)Fw[(size_t)i * T * no + mu]);
    }
  double ld = 0, sign = 1;
  bool sing = false;
  for (int c = 0; c < ns; ++c) perm[c] = c;
  for (int c = 0; c < ns; ++c) {
    int best = c;
    double bv = fabs(LU[c * ns + c]);
    for (int rr = c + 1; rr < ns; ++rr) {
      const double v = fabs(LU[rr * ns + c]);
      if (v > bv) { bv = v; best = rr; }
    }
    if (!(bv > 0.0)) { sing = true; break; }
    if (best != c) {
      for (int k = 0; k < ns; ++k) {
        const double t0 = LU[c * ns + k];
        LU[c * ns + k] = LU[best * ns + k];
        LU[best * ns + k] = t0;
      }
      const int tp = perm[c]; perm[c] = perm[best]; perm[best] = tp;
      sign = -sign;
    }
    const double piv = LU[c * ns + c];
    if (piv < 0) sign = -sign;
    ld += log(fabs(piv));
    for (int rr = c + 1; rr < ns; ++rr) {
      const double f = LU[rr * ns + c] / piv;
      LU[rr * ns + c] = f;
      for (int k = c + 1; k < ns; ++k) LU[rr * ns + k] -= f * LU[c * ns + k];
    }
  }
  if (sing) {
    out[0] = -INFINITY; out[1] = 0; out[2] = 0;
    if (jet) for (int t = 0; t < 3 * N; ++t) out[3 + t] = 0;
    return;
  }
  out[0] = ld;
  out[1] = sign;
  if (!jet) return;
  // inverse: solve A X = I with the factors (P A = L U)
  double Ai[NS * NS];
  for (int col = 0; col < ns; ++col) {
    double y[NS];
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
    for (int rr = 0; rr < ns; ++rr) Ai[rr * ns + col] = y[rr];
  }
  const int lap = T - 1;
  double trl = 0;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      const int i = e0 + a, mu = occ[b];
      trl += Ai[b * ns + a] * pn_aelem_lap(phw + (i * no + mu) * 5, Fw + (size_t)i * T * no + mu, no, i, lap);
    }
  double lsum = trl;
  for (int t = 1; t < lap; ++t) {
    double dA[NS * NS];
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) {
        const int i = e0 + a, mu = occ[b];
        dA[a * ns + b] = pn_aelem_tangent(phw + (i * no + mu) * 5, Fw + (size_t)i * T * no + mu, no, i, t);
      }
    double B[NS * NS];
    double tr = 0;
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) {
        double v = 0;
        for (int c = 0; c < ns; ++c) v += Ai[a * ns + c] * dA[c * ns + b];
        B[a * ns + b] = v;
        if (a == b) tr += v;
      }
    double tr2 = 0;
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) tr2 += B[a * ns + b] * B[b * ns + a];
    out[3 + t - 1] = tr;
    lsum -= tr2;
  }
  out[2] = lsum;
}
