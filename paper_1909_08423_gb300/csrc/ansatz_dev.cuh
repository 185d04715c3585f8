// Device functions shared by the staged and the fused paths.
#pragma once

#include <math.h>

#include "pn_internal.cuh"

// Cusp-spliced molecular orbitals at one electron position `re`.
// JET: acc[mu*5 + q] = value, d/dx, d/dy, d/dz, Laplacian; else acc[mu] = value.
__device__ inline double pn_pw(double x, int n) { return n == 0 ? 1.0 : (n == 1 ? x : x * x); }

template <bool JET>
__device__ inline void pn_orbitals_at(const DevSys& s, const double* __restrict__ re, double* __restrict__ acc) {
  constexpr int Q = JET ? 5 : 1;
  const int no = s.n_orb;
  for (int k = 0; k < no * Q; ++k) acc[k] = 0.0;
  int Ic = -1;
  double vc[3] = {0, 0, 0}, dcn = 0;
  if (s.use_cusp) {
    for (int I = 0; I < s.M; ++I) {
      double v0 = re[0] - s.R[3 * I], v1 = re[1] - s.R[3 * I + 1], v2 = re[2] - s.R[3 * I + 2];
      double d = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      if (d < s.cusp_rc[I]) { Ic = I; vc[0] = v0; vc[1] = v1; vc[2] = v2; dcn = d; }
    }
  }
  for (int sh = 0; sh < s.n_shells; ++sh) {
    const int c = s.sh_center[sh], l = s.sh_l[sh], np = s.sh_nprim[sh], po = s.sh_poff[sh], bo = s.sh_boff[sh];
    const double v[3] = {re[0] - s.R[3 * c], re[1] - s.R[3 * c + 1], re[2] - s.R[3 * c + 2]};
    const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (l == -1) {
      const double zeta = s.pexp[po], d = sqrt(r2);
      const double e = s.pcoef[po] * exp(-zeta * d);
      const double* mrow = s.mo + (size_t)bo * no;
      if (JET) {
        const double gfac = -zeta * e / d;
        const double jet[5] = {e, gfac * v[0], gfac * v[1], gfac * v[2], zeta * zeta * e - 2.0 * zeta * e / d};
        for (int mu = 0; mu < no; ++mu)
          for (int q = 0; q < Q; ++q) acc[mu * Q + q] += mrow[mu] * jet[q];
      } else {
        for (int mu = 0; mu < no; ++mu) acc[mu] += mrow[mu] * e;
      }
      continue;
    }
    double E0 = 0, E1 = 0, E2 = 0;
    for (int k = 0; k < np; ++k) {
      const double a = s.pexp[po + k];
      const double e = s.pcoef[po + k] * exp(-a * r2);
      E0 += e;
      if (JET) {
        E1 += a * e;
        E2 += a * a * e;
      }
    }
    const bool skip_s = (l == 0 && c == Ic);  // replaced inside the cusp sphere
    const int nc = l == 0 ? 1 : (l == 1 ? 3 : 6);
    for (int cc = 0; cc < nc; ++cc) {
      int ex, ey, ez;
      if (l == 0) { ex = ey = ez = 0; }
      else if (l == 1) { ex = cc == 0; ey = cc == 1; ez = cc == 2; }
      else {
        const int t2[6][3] = {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
        ex = t2[cc][0]; ey = t2[cc][1]; ez = t2[cc][2];
      }
      const double px = pn_pw(v[0], ex), py = pn_pw(v[1], ey), pz = pn_pw(v[2], ez);
      const double P = px * py * pz;
      const double* mrow = s.mo + (size_t)(bo + cc) * no;
      if (JET) {
        const double dPx = ex ? ex * pn_pw(v[0], ex - 1) * py * pz : 0.0;
        const double dPy = ey ? ey * px * pn_pw(v[1], ey - 1) * pz : 0.0;
        const double dPz = ez ? ez * px * py * pn_pw(v[2], ez - 1) : 0.0;
        const double lapP =
            (ex == 2 ? 2.0 * py * pz : 0.0) + (ey == 2 ? 2.0 * px * pz : 0.0) + (ez == 2 ? 2.0 * px * py : 0.0);
        // chi = P E(r^2): grad = grad P E0 - 2 v P E1,
        // lap = lap P E0 - 4 l P E1 + P (4 r^2 E2 - 6 E1)
        const double jet[5] = {P * E0, dPx * E0 - 2.0 * v[0] * P * E1, dPy * E0 - 2.0 * v[1] * P * E1,
                               dPz * E0 - 2.0 * v[2] * P * E1,
                               lapP * E0 - 4.0 * l * P * E1 + P * (4.0 * r2 * E2 - 6.0 * E1)};
        for (int mu = 0; mu < no; ++mu) {
          if (skip_s && s.cusp_on[Ic * no + mu]) continue;
          for (int q = 0; q < Q; ++q) acc[mu * Q + q] += mrow[mu] * jet[q];
        }
      } else {
        const double val = P * E0;
        for (int mu = 0; mu < no; ++mu) {
          if (skip_s && s.cusp_on[Ic * no + mu]) continue;
          acc[mu] += mrow[mu] * val;
        }
      }
    }
  }
  if (Ic >= 0) {
    const double d = dcn, inv = 1.0 / d;
    for (int mu = 0; mu < no; ++mu) {
      const int k = Ic * no + mu;
      if (!s.cusp_on[k]) continue;
      const double* a = s.cusp_a + (size_t)k * 5;
      const double p = a[0] + d * (a[1] + d * (a[2] + d * (a[3] + d * a[4])));
      const double f = s.cusp_s[k] * exp(p);
      acc[mu * Q + 0] += s.cusp_C[k] + f;
      if (JET) {
        const double p1 = a[1] + d * (2.0 * a[2] + d * (3.0 * a[3] + d * 4.0 * a[4]));
        const double p2 = 2.0 * a[2] + d * (6.0 * a[3] + d * 12.0 * a[4]);
        const double f1 = f * p1, f2 = f * (p2 + p1 * p1);
        acc[mu * Q + 1] += f1 * vc[0] * inv;
        acc[mu * Q + 2] += f1 * vc[1] * inv;
        acc[mu * Q + 3] += f1 * vc[2] * inv;
        acc[mu * Q + 4] += f2 + 2.0 * f1 * inv;
      }
    }
  }
}

// ln|det A| and its sign by LU with partial pivoting (A is overwritten).
// Returns false (sign 0) for an exactly singular or non-finite matrix.
__device__ inline bool pn_slogdet(double* A, int ns, double* ld, double* sign) {
  double l = 0, sg = 1;
  for (int c = 0; c < ns; ++c) {
    int best = c;
    double bv = fabs(A[c * ns + c]);
    for (int rr = c + 1; rr < ns; ++rr) {
      const double v = fabs(A[rr * ns + c]);
      if (v > bv) { bv = v; best = rr; }
    }
    if (!(bv > 0.0)) { *ld = -INFINITY; *sign = 0; return false; }
    if (best != c) {
      for (int k = 0; k < ns; ++k) {
        const double t0 = A[c * ns + k];
        A[c * ns + k] = A[best * ns + k];
        A[best * ns + k] = t0;
      }
      sg = -sg;
    }
    const double piv = A[c * ns + c];
    if (piv < 0) sg = -sg;
    l += log(fabs(piv));
    for (int rr = c + 1; rr < ns; ++rr) {
      const double f = A[rr * ns + c] / piv;
      for (int k = c + 1; k < ns; ++k) A[rr * ns + k] -= f * A[c * ns + k];
    }
  }
  *ld = l;
  *sign = sg;
  return true;
}
