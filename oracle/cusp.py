"""Nuclear cusp correction coefficients (Methods, "Cusp conditions"; the
technique of Ma, Towler, Drummond & Needs, J. Chem. Phys. 122, 224322 (2005),
with the value at the nucleus as a free parameter).

For molecular orbital mu and nucleus I, phi_s(r) is the part of phi_mu built
from the l=0 Gaussian shells centred on I (a radial function of
r = |r_e - R_I|) and eta the rest of the orbital.  Inside r < r_c the s part is
replaced by

    phi_s(r)  ->  C + s * exp(p(r)),   p(r) = a0 + a1 r + a2 r^2 + a3 r^3 + a4 r^4

with five conditions:
  p(r_c), p'(r_c), p''(r_c) continue ln|phi_s - C| smoothly at r_c,
  p(0) = ln|phi0 - C| (phi0: the s part's value at the nucleus, a parameter
         that defaults to phi_s(0)),
  a1 = -Z (phi0 + eta(0)) / (phi0 - C)   (Kato cusp of the whole orbital: the
         spherical average of eta has zero slope at the nucleus).
r_c = 0.5 / Z_I.  C = 0 unless phi_s changes sign on [0, r_c] (checked on a
64-point grid); then C shifts phi_s - C to one sign with a 10 % margin.

Parity: pinned by tests of value/slope/curvature continuity at r_c and of the
cusp slope at the nucleus.
"""

from __future__ import annotations

import numpy as np


def s_part_radial(sys, I, mu, r):
    """phi_s(r) and its first two radial derivatives, for l=0 Gaussian shells
    on nucleus I only."""
    r = np.asarray(r, dtype=np.float64)
    v = np.zeros_like(r)
    d1 = np.zeros_like(r)
    d2 = np.zeros_like(r)
    b = 0
    o = 0
    C = sys["mo_coeffs"]
    for s in range(len(sys["shell_l"])):
        l = int(sys["shell_l"][s])
        npr = int(sys["shell_nprim"][s])
        ncart = 1 if l <= 0 else (3 if l == 1 else 6)
        if l == 0 and int(sys["shell_center"][s]) == I:
            for k in range(npr):
                a = sys["prim_exp"][o + k]
                dk = sys["prim_coef"][o + k] * C[b, mu]
                e = np.exp(-a * r * r)
                v += dk * e
                d1 += dk * (-2.0 * a * r) * e
                d2 += dk * (4.0 * a * a * r * r - 2.0 * a) * e
        o += npr
        b += ncart
    return v, d1, d2


def has_s_part(sys, I):
    return any(int(l) == 0 and int(c) == I for l, c in zip(sys["shell_l"], sys["shell_center"]))


def cusp_tables(sys, orbital_at):
    """Per nucleus I: dict(rc, active[n_orb], C[n_orb], sgn[n_orb], a[n_orb,5]).

    ``orbital_at(point) -> phi[n_orb]`` evaluates the uncorrected orbitals at one
    point (used for eta(0) = phi(R_I) - phi_s(0))."""
    Z = sys["Z"]
    R = sys["R"]
    n_orb = sys["mo_coeffs"].shape[1]
    phi0_in = sys.get("cusp_phi0")
    tabs = []
    for I in range(len(Z)):
        rc = 0.5 / Z[I]
        active = np.zeros(n_orb, dtype=bool)
        Cs = np.zeros(n_orb)
        sg = np.ones(n_orb)
        al = np.zeros((n_orb, 5))
        if sys["use_cusp"] and has_s_part(sys, I):
            phi_full0 = orbital_at(R[I])
            grid = np.linspace(0.0, rc, 64)
            for mu in range(n_orb):
                vs, _, _ = s_part_radial(sys, I, mu, grid)
                scale = np.max(np.abs(vs))
                if scale < 1e-14:
                    continue
                s0 = vs[0]
                eta0 = phi_full0[mu] - s0
                c0 = 0.0
                if vs.min() < 0.0 < vs.max():
                    vrc = vs[-1]
                    c0 = vs.min() - 0.1 * scale if vrc > 0 else vs.max() + 0.1 * scale
                vr, d1, d2 = s_part_radial(sys, I, mu, np.array([rc]))
                vr, d1, d2 = vr[0], d1[0], d2[0]
                s = 1.0 if vr - c0 > 0 else -1.0
                phi0 = s0 if phi0_in is None else float(np.asarray(phi0_in).reshape(n_orb, len(Z))[mu, I])
                if (phi0 - c0) * s <= 0:
                    raise ValueError("cusp: phi0 - C has the wrong sign")
                a0 = np.log(abs(phi0 - c0))
                a1 = -Z[I] * (phi0 + eta0) / (phi0 - c0)
                X1 = np.log(abs(vr - c0))
                X2 = d1 / (vr - c0)
                X3 = d2 / (vr - c0) - X2 * X2
                A = np.array([[rc**2, rc**3, rc**4],
                              [2 * rc, 3 * rc**2, 4 * rc**3],
                              [2.0, 6 * rc, 12 * rc**2]])
                rhs = np.array([X1 - a0 - a1 * rc, X2 - a1, X3])
                a234 = np.linalg.solve(A, rhs)
                active[mu] = True
                Cs[mu] = c0
                sg[mu] = s
                al[mu] = [a0, a1, *a234]
        tabs.append(dict(rc=rc, active=active, C=Cs, sgn=sg, a=al))
    return tabs
