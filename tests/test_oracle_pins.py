"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Each test names what it pins.  None of them retypes an oracle formula: they
use closed forms, brute force, finite differences, symmetries and limits.
"""

import itertools
import math

import numpy as np
import pytest
import torch

from oracle import clip as oclip
from oracle import philox, sampling
from oracle.ansatz import DT, Oracle, features, network, params_to_torch
from paper_1909_08423_gb300 import synth

RNG = np.random.default_rng(1234)


def _pts(W, N, scale=1.5, seed=0):
    return np.random.default_rng(seed).normal(scale=scale, size=(W, N, 3))


# ---------------------------------------------------------------- closed forms

def test_hydrogen_atom_local_energy_is_minus_half():
    """psi = exp(-r) for the hydrogen atom gives E_loc = -1/2 Ha everywhere."""
    o = Oracle(synth.hydrogen_like_sto(1.0, 1.0))
    E, _, _ = o.local_energy(_pts(64, 1))
    assert np.max(np.abs(E + 0.5)) < 1e-12


@pytest.mark.parametrize("Z,zeta", [(1.0, 1.3), (3.0, 2.2), (2.0, 0.6)])
def test_hydrogen_like_sto_closed_form(Z, zeta):
    """exp(-zeta r) in a nucleus of charge Z: E_loc = -zeta^2/2 + (zeta - Z)/r."""
    o = Oracle(synth.hydrogen_like_sto(Z, zeta))
    r = _pts(64, 1, seed=2)
    E, _, _ = o.local_energy(r)
    d = np.linalg.norm(r[:, 0], axis=-1)
    assert np.max(np.abs(E - (-zeta ** 2 / 2 + (zeta - Z) / d))) < 1e-11


@pytest.mark.parametrize("Z,alpha", [(1.0, 0.7), (4.0, 2.5)])
def test_single_gaussian_closed_form(Z, alpha):
    """exp(-alpha r^2): lap psi / psi = 4 alpha^2 r^2 - 6 alpha."""
    o = Oracle(synth.single_gto(Z, alpha))
    r = _pts(64, 1, seed=3)
    E, _, _ = o.local_energy(r)
    d = np.linalg.norm(r[:, 0], axis=-1)
    assert np.max(np.abs(E - (-0.5 * (4 * alpha ** 2 * d ** 2 - 6 * alpha) - Z / d))) < 1e-10


@pytest.mark.parametrize("l,component", [(1, k) for k in range(3)] + [(2, k) for k in range(6)])
def test_cartesian_gaussian_closed_form(l, component):
    """x^a y^b z^c exp(-alpha r^2): lap psi / psi = 4 alpha^2 r^2
    - (6 + 4(a + b + c)) alpha + a(a-1)/x^2 + b(b-1)/y^2 + c(c-1)/z^2
    (product rule), and ln|psi| = a ln|x| + b ln|y| + c ln|z| - alpha r^2:
    pins each Cartesian component's powers."""
    Z, alpha = 2.0, 0.8
    a, b, c = synth.CART[l][component]
    o = Oracle(synth.single_cartesian_gto(Z, alpha, l, component))
    r = _pts(64, 1, seed=13)
    E, _, _ = o.local_energy(r)
    x, y, z = r[:, 0, 0], r[:, 0, 1], r[:, 0, 2]
    d2 = x * x + y * y + z * z
    ratio = (4 * alpha ** 2 * d2 - (6 + 4 * (a + b + c)) * alpha
             + a * (a - 1) / x ** 2 + b * (b - 1) / y ** 2 + c * (c - 1) / z ** 2)
    exact = -0.5 * ratio - Z / np.sqrt(d2)
    assert np.max(np.abs(E - exact) / (1 + np.abs(exact))) < 1e-10
    # the value fixes which axis each power belongs to (the p components
    # share one E_loc formula)
    lp, _ = o.eval_logpsi(r)
    ln_chi = a * np.log(np.abs(x)) + b * np.log(np.abs(y)) + c * np.log(np.abs(z)) - alpha * d2
    assert np.max(np.abs(lp - ln_chi)) < 1e-12


@pytest.mark.parametrize("l,component", [(0, 0), (1, 2), (2, 1)])
def test_contracted_gaussian_closed_form(l, component):
    """A contraction of three primitives, x^a y^b z^c sum_k d_k g_k with
    g_k = exp(-alpha_k r^2): lap psi / psi = sum_k d_k [4 alpha_k^2 r^2
    - (6 + 4(a + b + c)) alpha_k] g_k / sum_k d_k g_k + a(a-1)/x^2 + ...;
    a primitive dropped, or one exponent paired with another's
    coefficient, fails it."""
    Z, alphas, coefs = 2.0, np.array([3.1, 0.9, 0.25]), np.array([0.3, 0.8, 0.45])
    a, b, c = synth.CART[l][component]
    o = Oracle(synth.single_cartesian_gto(Z, alphas, l, component, coefs=tuple(coefs)))
    r = _pts(64, 1, seed=14)
    E, _, _ = o.local_energy(r)
    x, y, z = r[:, 0, 0], r[:, 0, 1], r[:, 0, 2]
    d2 = x * x + y * y + z * z
    g = coefs[None, :] * np.exp(-alphas[None, :] * d2[:, None])
    rad = (g * (4 * alphas[None, :] ** 2 * d2[:, None] - (6 + 4 * (a + b + c)) * alphas[None, :])).sum(1) / g.sum(1)
    ratio = rad + a * (a - 1) / x ** 2 + b * (b - 1) / y ** 2 + c * (c - 1) / z ** 2
    exact = -0.5 * ratio - Z / np.sqrt(d2)
    assert np.max(np.abs(E - exact) / (1 + np.abs(exact))) < 1e-10


def test_helium_like_product_closed_form():
    """exp(-zeta (r1 + r2)), 1 up 1 down, gamma off:
    E_loc = -zeta^2 + (zeta - Z)(1/r1 + 1/r2) + 1/r12."""
    Z, zeta = 2.0, 1.6875
    o = Oracle(synth.helium_like_product(Z, zeta))
    r = _pts(64, 2, seed=4)
    E, _, _ = o.local_energy(r)
    r1 = np.linalg.norm(r[:, 0], axis=-1)
    r2 = np.linalg.norm(r[:, 1], axis=-1)
    r12 = np.linalg.norm(r[:, 0] - r[:, 1], axis=-1)
    assert np.max(np.abs(E - (-zeta ** 2 + (zeta - Z) * (1 / r1 + 1 / r2) + 1 / r12))) < 1e-11


@pytest.mark.parametrize("Z,zeta", [(2.0, 1.6875), (3.0, 2.4)])
def test_helium_like_product_with_electronic_cusp_factor_closed_form(Z, zeta):
    """exp(-zeta (r1 + r2) + u(r12)), 1 up 1 down, with the paper's
    electronic cusp factor u(r) = -c/(1 + r), c = 1/2 for opposite spins
    (cusp conditions, Methods).  By hand, with u' = c/(1+r)^2 and
    u'' = -2c/(1+r)^3 and unit vectors e1, e2, e12 = (r1 - r2)/r12:
      lap ln psi = -2 zeta/r1 - 2 zeta/r2 + 2 u'' + 4 u'/r12,
      |grad ln psi|^2 = 2 zeta^2 + 2 u'^2 - 2 zeta u' (e1 - e2) . e12,
    and E_loc = -(lap + |grad|^2)/2 - Z/r1 - Z/r2 + 1/r12.  A wrong form
    with the right slope at contact (-c e^-r), a wrong sign of the factor,
    the same-spin c for this pair or a dropped cross term fails it (forms
    that differ by a constant, such as c r/(1 + r), give the same E_loc)."""
    c = 0.5
    o = Oracle(synth.helium_like_product(Z, zeta, use_gamma=1))
    r = _pts(64, 2, seed=11)
    E, _, _ = o.local_energy(r)
    r1v, r2v = r[:, 0], r[:, 1]
    r1 = np.linalg.norm(r1v, axis=-1)
    r2 = np.linalg.norm(r2v, axis=-1)
    r12 = np.linalg.norm(r1v - r2v, axis=-1)
    e1, e2, e12 = r1v / r1[:, None], r2v / r2[:, None], (r1v - r2v) / r12[:, None]
    up = c / (1 + r12) ** 2
    upp = -2 * c / (1 + r12) ** 3
    lap = -2 * zeta / r1 - 2 * zeta / r2 + 2 * upp + 4 * up / r12
    g2 = 2 * zeta ** 2 + 2 * up ** 2 - 2 * zeta * up * ((e1 - e2) * e12).sum(-1)
    exact = -0.5 * (lap + g2) - Z / r1 - Z / r2 + 1 / r12
    assert np.max(np.abs(E - exact)) < 1e-11


def test_two_orbital_product_closed_form():
    """Up electron in phi_0, down electron in phi_1, phi_mu = sum_b
    C[b][mu] d_b exp(-zeta_b r) (the molecular orbitals of the ansatz, Eq.
    (ansatz), with the network off): each electron's kinetic part is
    sum_b C[b][mu] d_b (-zeta_b^2/2 + zeta_b/r) exp(-zeta_b r) / phi_mu(r), so
    E_loc = that for electron 1 in phi_0 and electron 2 in phi_1
            - Z/r1 - Z/r2 + 1/r12.
    A transposed coefficient matrix or the spins' orbitals swapped fails it."""
    Z, zetas, coefs = 3.0, (2.7, 0.9), (1.3, 0.6)
    C = np.array([[0.8, 0.3], [0.5, 1.1]])
    o = Oracle(synth.two_orbital_product(Z, zetas, coefs, C))
    r = _pts(64, 2, seed=12)
    E, _, _ = o.local_energy(r)

    def kinetic_over_phi(d, mu):
        num = sum(C[b, mu] * coefs[b] * (-zetas[b] ** 2 / 2 + zetas[b] / d) * np.exp(-zetas[b] * d) for b in range(2))
        den = sum(C[b, mu] * coefs[b] * np.exp(-zetas[b] * d) for b in range(2))
        return num / den

    r1 = np.linalg.norm(r[:, 0], axis=-1)
    r2 = np.linalg.norm(r[:, 1], axis=-1)
    r12 = np.linalg.norm(r[:, 0] - r[:, 1], axis=-1)
    exact = kinetic_over_phi(r1, 0) + kinetic_over_phi(r2, 1) - Z / r1 - Z / r2 + 1 / r12
    assert np.max(np.abs(E - exact)) < 1e-10


@pytest.mark.parametrize("zeta", [1.0, 1.3])
def test_nucleus_nucleus_repulsion_closed_form(zeta):
    """exp(-zeta r_A) on nucleus A (Z_A = 1) beside bare nuclei B, C (no
    basis functions): the kinetic part is that of the hydrogen-like atom and
    V adds every electron-nucleus attraction and every nucleus pair's
    repulsion (the Hamiltonian of the variational principle, Methods):
    E_loc = -zeta^2/2 + (zeta - 1)/r_A - Z_B/r_B - Z_C/r_C
            + Z_A Z_B/R_AB + Z_A Z_C/R_AC + Z_B Z_C/R_BC.
    A dropped, doubled or once-counted nucleus pair fails it."""
    bare = ((2.0, (0.0, 0.0, 1.7)), (3.0, (1.1, -0.4, -1.2)))
    o = Oracle(synth.sto_beside_bare_nuclei(1.0, zeta, bare))
    r = _pts(64, 1, seed=9)
    E, _, _ = o.local_energy(r)
    RA, (ZB, RB), (ZC, RC) = np.zeros(3), (bare[0][0], np.array(bare[0][1])), (bare[1][0], np.array(bare[1][1]))
    dist = lambda a, b: np.linalg.norm(a - b, axis=-1)
    exact = (-zeta ** 2 / 2 + (zeta - 1.0) / dist(r[:, 0], RA) - ZB / dist(r[:, 0], RB) - ZC / dist(r[:, 0], RC)
             + ZB / dist(RA, RB) + ZC / dist(RA, RC) + ZB * ZC / dist(RB, RC))
    assert np.max(np.abs(E - exact)) < 1e-11


# ------------------------------------------------------------- determinants

def _leibniz(A):
    n = A.shape[-1]
    tot = np.zeros(A.shape[0])
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for a in range(n) for b in range(a + 1, n) if perm[a] > perm[b])
        term = np.ones(A.shape[0])
        for row, col in enumerate(perm):
            term = term * A[:, row, col]
        tot += (-1) ** inv * term
    return tot


@pytest.mark.parametrize("make", [synth.be, synth.h10])
def test_determinants_match_permutation_sums(make):
    """Eq. (ansatz) assembled by Leibniz permutation sums (n_sigma <= 5)."""
    S = make()
    o = Oracle(S)
    r = synth.random_walkers(S, 6, 7)
    c = o.components(r)
    phit = c["phi"] * c["f"]
    nu = S["n_up"]
    tot = np.zeros(len(r))
    for p in range(len(S["ci"])):
        du = _leibniz(phit[:, :nu][:, :, S["occ_up"][p]])
        dd = _leibniz(phit[:, nu:][:, :, S["occ_dn"][p]])
        tot += S["ci"][p] * du * dd
    from oracle.ansatz import gamma
    g = gamma(S, torch.as_tensor(r, dtype=DT)).numpy()
    psi = np.exp(g + c["J"]) * tot
    lp, sg = o.eval_logpsi(r)
    np.testing.assert_allclose(lp, np.log(np.abs(psi)), rtol=0, atol=1e-11)
    np.testing.assert_array_equal(sg, np.sign(psi))


# ---------------------------------------------------- finite differences

@pytest.mark.parametrize("make", [synth.h2, synth.be, synth.h10])
def test_derivatives_match_central_differences(make):
    """grad ln|psi| and lap ln|psi| against 4th-order central differences of
    ln|psi| itself."""
    S = make()
    o = Oracle(S)
    r = synth.random_walkers(S, 3, 11)
    lp, _, g, lap = o.derivatives(r)
    h = 1e-3
    N = r.shape[1]
    gfd = np.zeros_like(g)
    lfd = np.zeros(len(r))
    f0 = o.eval_logpsi(r)[0]
    for i in range(N):
        for a in range(3):
            vals = {}
            for k in (-2, -1, 1, 2):
                rr = r.copy()
                rr[:, i, a] += k * h
                vals[k] = o.eval_logpsi(rr)[0]
            gfd[:, i, a] = (vals[-2] - 8 * vals[-1] + 8 * vals[1] - vals[2]) / (12 * h)
            lfd += (-vals[-2] + 16 * vals[-1] - 30 * f0 + 16 * vals[1] - vals[2]) / (12 * h * h)
    np.testing.assert_allclose(g, gfd, atol=2e-7 * max(1, np.abs(g).max()))
    np.testing.assert_allclose(lap, lfd, atol=2e-5 * max(1, np.abs(lap).max()))


# ------------------------------------------------------------ symmetries

@pytest.mark.parametrize("make", [synth.be, synth.h10, synth.n2])
def test_antisymmetry_same_spin_exchange(make):
    """Eq. (antisymmetry): exchanging two same-spin electrons flips the sign
    and leaves ln|psi| unchanged."""
    S = make()
    o = Oracle(S)
    r = synth.random_walkers(S, 4, 5)
    lp, sg = o.eval_logpsi(r)
    nu = S["n_up"]
    for (i, j) in ((0, 1), (nu, nu + 1)):
        rs = r.copy()
        rs[:, [i, j]] = rs[:, [j, i]]
        lp2, sg2 = o.eval_logpsi(rs)
        np.testing.assert_allclose(lp2, lp, atol=1e-11)
        np.testing.assert_array_equal(sg2, -sg)


@pytest.mark.parametrize("make", [synth.be, synth.h10])
def test_jastrow_invariant_backflow_equivariant(make):
    """J(P r) = J(r) and f_{mu i}(P r) = f_{mu P(i)}(r) for same-spin
    permutations; with n_up = n_dn, J is also invariant under exchanging the
    whole up and down blocks (the channels are relative, not absolute)."""
    S = make()
    P = params_to_torch(S)
    r = torch.as_tensor(synth.random_walkers(S, 4, 9), dtype=DT)
    J, f = network(S, P, r)
    nu, N = S["n_up"], S["n_up"] + S["n_dn"]
    perm = list(range(N))
    perm[0], perm[nu - 1] = perm[nu - 1], perm[0]
    perm[nu], perm[N - 1] = perm[N - 1], perm[nu]
    J2, f2 = network(S, P, r[:, perm])
    torch.testing.assert_close(J2, J, atol=1e-12, rtol=0)
    torch.testing.assert_close(f2, f[:, perm], atol=1e-12, rtol=0)
    flip = list(range(nu, N)) + list(range(nu))
    J3, f3 = network(S, P, r[:, flip])
    torch.testing.assert_close(J3, J, atol=1e-12, rtol=0)
    torch.testing.assert_close(f3, f[:, flip], atol=1e-12, rtol=0)


def test_network_rotation_invariant_for_an_atom():
    """For one nucleus at the origin the network sees distances only, so J
    and f do not change when all electrons rotate about the nucleus."""
    S = synth.be()
    P = params_to_torch(S)
    r = torch.as_tensor(synth.random_walkers(S, 4, 2), dtype=DT)
    q, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
    Q = torch.as_tensor(q, dtype=DT)
    J, f = network(S, P, r)
    J2, f2 = network(S, P, r @ Q.T)
    torch.testing.assert_close(J2, J, atol=1e-12, rtol=0)
    torch.testing.assert_close(f2, f, atol=1e-12, rtol=0)


# ------------------------------------------------------------------- cusps

def _unit_dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("make,I", [(synth.h2, 0), (synth.be, 0), (synth.n2, 1)])
def test_electron_nucleus_cusp(make, I):
    """Methods (cusp conditions, Kato): the spherical average of psi around a
    nucleus has slope -Z_I psi at the nucleus."""
    S = make()
    o = Oracle(S)
    base = synth.random_walkers(S, 1, 3)[0]
    base[0] = S["R"][I]
    dirs = _unit_dirs(24, 1)
    psi0 = np.exp(o.eval_logpsi(base[None])[0][0])

    def avg(h):
        rs = np.repeat(base[None], 2 * len(dirs), 0)
        rs[:len(dirs), 0] += h * dirs
        rs[len(dirs):, 0] -= h * dirs
        lp, sg = o.eval_logpsi(rs)
        return np.mean(sg * np.exp(lp)) * np.sign(o.eval_logpsi(base[None])[1][0])

    h = 1e-5
    slope = (avg(h) / psi0 - 1) / h
    slope2 = (avg(2 * h) / psi0 - 1) / (2 * h)
    est = 2 * slope - slope2
    assert abs(est + S["Z"][I]) < 2e-3 * S["Z"][I]


@pytest.mark.parametrize("make", [synth.h2, synth.be])
def test_electron_electron_cusps(make):
    """Methods (gamma): opposite spins give a kink of slope 1/2, same spins a
    relative factor (1 + r/4) on the odd part."""
    S = make()
    o = Oracle(S)
    base = synth.random_walkers(S, 1, 8)[0]
    nu = S["n_up"]
    n = _unit_dirs(1, 4)[0]

    def at(i, j, u):
        r = base.copy()
        c = 0.5 * (base[i] + base[j])
        r[i] = c + u / 2
        r[j] = c - u / 2
        lp, sg = o.eval_logpsi(r[None])
        return sg[0] * np.exp(lp[0])

    # opposite spin
    i, j = 0, nu
    p0 = at(i, j, np.zeros(3))
    ests = []
    for h in (1e-5, 2e-5):
        ests.append(((at(i, j, h * n) + at(i, j, -h * n)) / 2 / p0 - 1) / h)
    est = 2 * ests[0] - ests[1]
    assert abs(est - 0.5) < 1e-3
    # same spin (needs two up electrons)
    if nu >= 2:
        h = 1e-4
        c1 = (at(0, 1, 2 * h * n) / (2 * at(0, 1, h * n)) - 1) / h
        c2 = (at(0, 1, 4 * h * n) / (2 * at(0, 1, 2 * h * n)) - 1) / (2 * h)
        assert abs((2 * c1 - c2) - 0.25) < 1e-3


def test_features_vanish_quadratically_at_zero():
    """e_k(0) = e_k'(0) = 0: e_k(h)/h^2 tends to a finite limit."""
    S = synth.be()
    d = torch.tensor([0.0, 1e-4, 2e-4], dtype=DT)
    e = features(S, d).numpy()
    assert np.all(e[0] == 0.0)
    ratio = e[1] / 1e-8, e[2] / 4e-8
    np.testing.assert_allclose(ratio[0], ratio[1], rtol=1e-3)


@pytest.mark.parametrize("kind", ["ee", "en"])
def test_network_is_cuspless(kind):
    """Eq. (cuspless): J and f have no kink where an electron meets another
    electron or a nucleus (antipodal slope -> 0)."""
    S = synth.be()
    P = params_to_torch(S)
    base = torch.as_tensor(synth.random_walkers(S, 1, 6), dtype=DT)
    n = torch.as_tensor(_unit_dirs(1, 9)[0], dtype=DT)

    def at(u):
        r = base.clone()
        if kind == "ee":
            c = 0.5 * (base[0, 0] + base[0, 2])
            r[0, 0] = c + u / 2
            r[0, 2] = c - u / 2
        else:
            r[0, 0] = u
        with torch.no_grad():
            J, f = network(S, P, r)
        return J[0].item(), f[0].numpy()

    J0, f0 = at(torch.zeros(3, dtype=DT))
    h = 1e-4
    Jp, fp = at(h * n)
    Jm, fm = at(-h * n)
    assert abs(((Jp + Jm) / 2 - J0) / h) < 1e-3
    assert np.max(np.abs(((fp + fm) / 2 - f0) / h)) < 1e-3


@pytest.mark.parametrize("make", [synth.h2, synth.be, synth.n2])
def test_cusp_splice_is_smooth_at_rc(make):
    """The spliced orbital continues value, slope and curvature across r_c
    (the three matching conditions of the Ma et al. correction)."""
    S = make()
    o = Oracle(S)
    I = 0
    rc = o.cusp[I]["rc"]
    n = _unit_dirs(1, 3)[0]
    eps = 1e-6

    def phi(rad):
        p = torch.as_tensor(S["R"][I] + rad * n, dtype=DT).reshape(1, 1, 3)
        with torch.no_grad():
            return o.orbitals(p).numpy()[0, 0]

    hs = 1e-3
    inside = [phi(rc - eps - k * hs) for k in range(3)]
    outside = [phi(rc + eps + k * hs) for k in range(3)]
    scale = np.abs(outside[0]).max()
    np.testing.assert_allclose(inside[0], outside[0], atol=1e-5 * scale)
    d_in = (inside[0] - inside[1]) / hs
    d_out = (outside[1] - outside[0]) / hs
    np.testing.assert_allclose(d_in, d_out, atol=2e-2 * max(1, np.abs(d_out).max()))
    # curvature at r_c from either side: the one-sided second derivative of
    # second order, (2 f0 - 5 f1 + 4 f2 - f3) / h^2 with f_k at r_c -+ k h
    # (a plain second difference is off by h times the third derivative,
    # larger than a kink would be)
    hc = 1e-4
    fin = [phi(rc - 1e-9 - k * hc) for k in range(4)]
    fout = [phi(rc + 1e-9 + k * hc) for k in range(4)]
    c_in = (2 * fin[0] - 5 * fin[1] + 4 * fin[2] - fin[3]) / hc ** 2
    c_out = (2 * fout[0] - 5 * fout[1] + 4 * fout[2] - fout[3]) / hc ** 2
    np.testing.assert_allclose(c_in, c_out, atol=1e-3 * max(1, np.abs(c_out).max()))


@pytest.mark.parametrize("make", [synth.h2, synth.be, synth.n2])
def test_cusp_splice_keeps_the_value_at_the_nucleus(make):
    """With the nucleus value phi0 at its default (the l = 0 part's own value
    there), the spliced orbitals equal the unspliced ones at the nucleus:
    p(0) = ln|phi0 - C| puts C + s exp(p(0)) = phi0 in place of that part."""
    from oracle.ansatz import basis_values
    S = make()
    o = Oracle(S)
    for I in range(len(S["Z"])):
        at = torch.as_tensor(S["R"][I], dtype=DT).reshape(1, 1, 3)
        with torch.no_grad():
            spliced = o.orbitals(at).numpy()[0, 0]
            plain = (basis_values(S, at) @ o.C).numpy()[0, 0]
        active = np.asarray(o.cusp[I]["active"], dtype=bool)
        assert active.any()
        np.testing.assert_allclose(spliced, plain, rtol=1e-12, atol=1e-14 * np.abs(plain).max())


# ----------------------------------------------------------------- sampling

# Known-answer vectors of Philox4x32-10 published with the generator
# (Salmon, Moraes, Dror & Shaw, SC'11; the Random123 distribution's test
# vectors): counter (c0..c3), key (k0, k1) -> output words.
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answer_vectors(ctr, key, expect):
    """A wrong round constant, Weyl increment, round count or word order
    changes every output word."""
    out = philox.philox4x32(*[np.array([c], dtype=np.uint64) for c in ctr], key[0], key[1])
    assert tuple(int(w[0]) for w in out) == expect


def test_mlp_and_shifted_softplus_worked_example():
    """The network's maps (reading A7: affine maps stored [in][out], shifted
    softplus ln(e^x/2 + 1/2) between layers, none after the last), worked by
    hand for x = (1, -2), W1 = [[1/2, -1], [2, 1/4]], b1 = (1/10, -3/10),
    W2 = [[1], [-2]], b2 = (7/10):
      a = x W1 + b1 = (1/2 - 4 + 1/10, -1 - 1/2 - 3/10) = (-17/5, -9/5)
      h = ssp(a) = (ln((e^-3.4 + 1)/2), ln((e^-1.8 + 1)/2))
        = (-0.66031871013507980, -0.54016957003387118)
      y = h W2 + b2 = h_1 - 2 h_2 + 7/10 = 1.1200204299326626.
    A transposed map, an activation after the last layer or an unshifted
    softplus fails it; so do ssp(0) != 0, ssp'(0) != 1/2 and a large-x
    limit other than x - ln 2."""
    from oracle.ansatz import _mlp, ssp
    x = torch.tensor([[1.0, -2.0]], dtype=DT)
    W1 = torch.tensor([[0.5, -1.0], [2.0, 0.25]], dtype=DT)
    b1 = torch.tensor([0.1, -0.3], dtype=DT)
    W2 = torch.tensor([[1.0], [-2.0]], dtype=DT)
    b2 = torch.tensor([0.7], dtype=DT)
    y = _mlp(x, [(W1, b1), (W2, b2)])
    assert abs(float(y[0, 0]) - 1.1200204299326626) < 1e-14
    z = torch.tensor([0.0, 40.0, -3.4, -1.8], dtype=DT, requires_grad=True)
    v = ssp(z)
    assert float(v[0].detach()) == 0.0
    assert abs(float(v[1].detach()) - (40.0 - math.log(2.0))) < 1e-13
    np.testing.assert_allclose(v[2:].detach().numpy(), [-0.66031871013507980, -0.54016957003387118], rtol=1e-14)
    (g,) = torch.autograd.grad(v[0], z)
    assert abs(float(g[0]) - 0.5) < 1e-15


def _golden_features():
    from fractions import Fraction
    import os
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "features_k4_rc10.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        d, k, mu, sig, x, val = line.split()
        rows.append((Fraction(d), int(k), Fraction(mu), Fraction(sig), Fraction(x), float(val)))
    return rows


def test_features_match_hand_worked_table():
    """e_k(d) for K = 4, r_c = 10 against the table worked by hand from the
    paper's e_k, mu_k and sigma_k (tests/golden/features_k4_rc10.txt).  The
    table's own arithmetic is checked in exact fractions first; then the
    oracle must reproduce every entry.  A wrong 1/7, a q_k instead of q_k^2,
    a missing d^2 envelope or an endpoint-inclusive q grid fails it."""
    from fractions import Fraction
    rows = _golden_features()
    assert len(rows) == 12
    for d, k, mu, sig, x, val in rows:
        q = Fraction(k, 5)
        assert mu == 10 * q * q and sig == (1 + 10 * q) / 7
        assert x == -d - (d - mu) ** 2 / sig ** 2
        assert abs(float(d * d) * math.exp(float(x)) / val - 1) < 1e-15
    sysd = {"K": 4, "r_c": 10.0}
    ds = sorted({r[0] for r in rows})
    e = features(sysd, torch.tensor([float(d) for d in ds], dtype=DT)).numpy()
    for d, k, _, _, _, val in rows:
        assert abs(e[ds.index(d), k - 1] / val - 1) < 1e-13, (d, k)


def test_philox_normals_are_standard_and_reproducible():
    a = philox.normals(7, np.arange(20000), 3, 12)
    b = philox.normals(7, np.arange(20000), 3, 12)
    np.testing.assert_array_equal(a, b)
    assert abs(a.mean()) < 5e-3 and abs(a.std() - 1) < 5e-3
    c = philox.normals(8, np.arange(20000), 3, 12)
    assert abs(np.corrcoef(a.reshape(-1), c.reshape(-1))[0, 1]) < 5e-3
    u = philox.accept_uniform(7, np.arange(200000), 3, 12)
    assert 0 < u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 3e-3


def test_metropolis_samples_hydrogen_density():
    """|psi|^2 = exp(-2r) has <r> = 3/2 and <r^2> = 3 (sampling of Eq.
    monte-carlo); the Gaussian proposal must reproduce them."""
    S = synth.hydrogen_like_sto(1.0, 1.0)
    o = Oracle(S)
    W = 2048
    r = sampling.init_walkers(S, W, seed=5)
    lp, _ = o.eval_logpsi(r)
    r, lp, acc = sampling.metropolis(o, r, lp, 60, 0.5, seed=5, step0=0)
    rs = []
    for k in range(8):
        r, lp, _ = sampling.metropolis(o, r, lp, 10, 0.5, seed=5, step0=60 + 10 * k)
        rs.append(np.linalg.norm(r[:, 0], axis=-1))
    rs = np.concatenate(rs)
    assert abs(rs.mean() - 1.5) < 0.04
    assert abs((rs ** 2).mean() - 3.0) < 0.15


def _langevin_chain(S, W, tau, seed, burn, blocks):
    o = Oracle(S)
    r = sampling.init_walkers(S, W, seed=seed)
    lp, _, g = o.value_and_grad(r)
    r, lp, g, _ = sampling.langevin(o, r, lp, g, burn, tau, seed=seed, step0=0)
    rs, acc = [], []
    for k in range(blocks):
        r, lp, g, a = sampling.langevin(o, r, lp, g, 10, tau, seed=seed, step0=burn + 10 * k)
        rs.append(np.linalg.norm(r[:, 0], axis=-1))
        acc.append(a.mean() / 10)
    return np.concatenate(rs), float(np.mean(acc))


@pytest.mark.parametrize("tau", [0.3, 1.0])
def test_langevin_samples_gaussian_density(tau):
    """psi = exp(-alpha r^2): |psi|^2 is a Gaussian of variance 1/(4 alpha)
    per axis, so <r> = sqrt(2 / (pi alpha)) and <r^2> = 3 / (4 alpha).  With
    tau = 1 the drift step 2 alpha tau r is longer than r, so the clipping
    at the nucleus acts on every move and the Hastings ratio must carry it."""
    alpha = 0.7
    rs, _ = _langevin_chain(synth.single_gto(1.0, alpha), 2048, tau, 5, 40, 6)
    assert abs(rs.mean() - np.sqrt(2 / (np.pi * alpha))) < 0.02
    assert abs((rs ** 2).mean() - 3 / (4 * alpha)) < 0.04


def test_langevin_samples_hydrogen_density():
    """|psi|^2 = exp(-2r): <r> = 3/2, <r^2> = 3 under the Langevin chain."""
    rs, acc = _langevin_chain(synth.hydrogen_like_sto(1.0, 1.0), 2048, 0.1, 6, 40, 6)
    assert abs(rs.mean() - 1.5) < 0.04
    assert abs((rs ** 2).mean() - 3.0) < 0.15
    assert acc > 0.95


def test_langevin_drift_direction_raises_acceptance():
    """With the drift along +grad ln|psi| the proposal nearly follows |psi|^2
    (acceptance 1 - O(tau^3/2)); the same chain with the drift reversed,
    planted here in the oracle, still samples correctly but accepts far less.
    Pins the sign of the drift, which the moments alone cannot see."""
    S = synth.hydrogen_like_sto(1.0, 1.0)
    _, acc = _langevin_chain(S, 1024, 0.1, 6, 20, 1)
    orig = sampling.clipped_drift
    sampling.clipped_drift = lambda s_, r_, g_, t_: -orig(s_, r_, g_, t_)
    try:
        _, acc_rev = _langevin_chain(S, 1024, 0.1, 6, 20, 1)
    finally:
        sampling.clipped_drift = orig
    assert acc > 0.97 and acc_rev < 0.8


def test_langevin_small_step_always_accepts():
    """As tau -> 0 the Hastings ratio tends to 1: every move is accepted."""
    S = synth.be()
    o = Oracle(S)
    r = sampling.init_walkers(S, 16, seed=3)
    lp, _, g = o.value_and_grad(r)
    _, _, _, acc = sampling.langevin(o, r, lp, g, 2, 1e-6, seed=3, step0=0)
    assert np.all(acc == 2)


def test_clipped_drift_never_passes_a_nucleus():
    """The drift displacement is never longer than the distance from the
    electron to its nearest nucleus, and is unchanged where it is shorter."""
    S = synth.h10()
    rng = np.random.default_rng(8)
    r = sampling.init_walkers(S, 64, seed=8)
    g = rng.normal(0, 5.0, r.shape)
    c = sampling.clipped_drift(S, r, g, 0.5)
    d = np.linalg.norm(r[:, :, None, :] - np.asarray(S["R"])[None, None], axis=-1).min(-1)
    lc = np.linalg.norm(c, axis=-1)
    assert np.all(lc <= d * (1 + 1e-12))
    short = np.linalg.norm(0.5 * g, axis=-1) <= d
    np.testing.assert_allclose(c[short], 0.5 * g[short], rtol=0, atol=0)


def _lih_scan_eloc(o, xs):
    r0, e, d, _, _ = synth.lih_scan()
    r = np.repeat(r0[None], len(xs), 0).copy()
    r[:, e, :] = r0[e] + np.asarray(xs, dtype=float)[:, None] * d
    return o.local_energy(r)[0]


def test_lih_scan_local_energy_through_coalescences():
    """The LiH scan (Results, one-dimensional scan): with the nuclear cusp
    splice and the electronic cusp factor gamma, E_loc of the moving electron
    converges at the Li nucleus and at the opposite-spin electron.  Without
    the splice it diverges like -Z/delta at the nucleus, and without gamma like
    +1/delta at the electron: the cusps, not the network, remove those poles."""
    deltas = np.array([1e-2, 1e-3, 1e-4])
    on = Oracle(synth.lih())
    for centre in (0.0, 2.0):
        for side in (1.0, -1.0):
            E = _lih_scan_eloc(on, centre + side * deltas)
            assert np.all(np.isfinite(E))
            assert abs(E[2] - E[1]) < abs(E[1] - E[0]) + 1e-9  # contracting: a limit exists
            assert abs(E[2] - E[1]) < 0.1 * max(1.0, abs(E[1]))
    no_cusp = Oracle(synth.lih(use_cusp=0))
    E = _lih_scan_eloc(no_cusp, deltas)
    assert abs(E[2] * deltas[2] + 3.0) < 0.01  # E_loc ~ -Z / delta, Z = 3
    no_gamma = Oracle(synth.lih(use_gamma=0))
    E = _lih_scan_eloc(no_gamma, 2.0 + deltas)
    assert abs(E[2] * deltas[2] - 1.0) < 0.01  # E_loc ~ +1 / delta


def test_ablation_without_jastrow_and_backflow_is_the_determinant_sum():
    """no_jastrow and no_backflow with gamma off leave
    psi = sum_p c_p det[phi(r_up)]_p det[phi(r_dn)]_p (Eq. ansatz with J = 0,
    f = 1), checked against numpy determinants of the orbital matrices; the
    removed heads get zero gradient."""
    S = synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=4, D=32, K=16, L=2, seed=7,
                          use_gamma=0, no_jastrow=1, no_backflow=1)
    o = Oracle(S)
    r = _pts(16, 4, seed=8)
    lp, sg = o.eval_logpsi(r)
    import torch as _torch
    phi = o.orbitals(_torch.as_tensor(r)).numpy()
    nu = S["n_up"]
    psi = np.zeros(len(r))
    for p, c in enumerate(S["ci"]):
        du = np.linalg.det(phi[:, :nu][:, :, S["occ_up"][p]])
        dd = np.linalg.det(phi[:, nu:][:, :, S["occ_dn"][p]])
        psi += c * du * dd
    np.testing.assert_allclose(lp, np.log(np.abs(psi)), rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(sg, np.sign(psi))
    g = o.grad_logpsi(r, np.ones(len(r)))
    sh = synth.param_shapes(S["D"], S["Zd"], S["K"], S["L"], len(S["Z"]), S["mo_coeffs"].shape[1])
    off = 0
    for name, shape in sh:
        n = int(np.prod(shape))
        if name.startswith("eta.") or name.startswith("kappa."):
            assert np.all(g[off:off + n] == 0), name
        off += n


def test_adamw_closed_forms():
    """With zero moments the first AdamW step moves every parameter by
    lr (g / (|g| + eps) + wd theta); with a constant gradient the bias
    corrections make every later step the same size.  Weight decay alone
    (g = 0) shrinks theta by the factor 1 - lr wd."""
    from oracle import optim
    rng = np.random.default_rng(3)
    th, g = rng.normal(size=50), rng.normal(size=50)
    lr, wd, eps = 0.01, 0.05, 1e-8
    m = v = np.zeros(50)
    x = th
    for t in range(1, 6):
        xn, m, v = optim.adamw_step(x, g, m, v, t, lr, wd=wd, eps=eps)
        np.testing.assert_allclose(xn, x - lr * (g / (np.abs(g) + eps) + wd * x), rtol=1e-12, atol=1e-15)
        x = xn
    xz, _, _ = optim.adamw_step(th, np.zeros(50), np.zeros(50), np.zeros(50), 1, lr, wd=wd, eps=eps)
    np.testing.assert_allclose(xz, th * (1 - lr * wd), rtol=1e-15)
    assert optim.learning_rate(200, 0.01, 200) == 0.005


# ----------------------------------------------------------------- clipping

def test_clipping_window_and_smoothness():
    E = np.concatenate([RNG.normal(-14.6, 0.3, 1000), [50.0, -200.0, 1e4]])
    out = oclip.clip_local_energy(E)
    m = np.median(E)
    L = 5 * np.mean(np.abs(E - m))
    inside = np.abs(E - m) <= L
    np.testing.assert_array_equal(out[inside], E[inside])
    assert np.all(np.abs(out[~inside] - m) < np.abs(E[~inside] - m))
    # continuity and unit slope at the window edge
    for sgn in (1, -1):
        e0 = m + sgn * L
        probe = np.concatenate([E, [e0 - 1e-7, e0 + 1e-7]])
        # the probes barely move median and mean deviation; recompute window
        o2 = oclip.clip_local_energy(probe)
        slope = (o2[-1] - o2[-2]) / 2e-7
        assert abs(slope - 1) < 1e-3


def test_clipping_hand_worked_even_count():
    """Six energies (-2, -1, 1, 2, 3, 100), worked by hand from the clipping
    rule (Methods, ansatz optimization) with the even-count median read as
    the mean of the two middle values: m = (1 + 2)/2 = 3/2; the deviations
    7/2, 5/2, 1/2, 1/2, 3/2, 197/2 sum to 107, so d = 107/6 and the window
    is L = 5 d = 535/6; only 100 lies outside (deviation 197/2 > 535/6) and
    becomes m + L (1 + ln((197/2)/(535/6))) = 3/2 + (535/6)(1 + ln(591/535)).
    The loss weights of Eq. (trainig) are 2 (E' - mean E') / 6."""
    E = np.array([-2.0, -1.0, 1.0, 2.0, 3.0, 100.0])
    out = oclip.clip_local_energy(E)
    expect = E.copy()
    expect[5] = 1.5 + (535.0 / 6.0) * (1.0 + math.log(591.0 / 535.0))
    np.testing.assert_allclose(out, expect, rtol=1e-15, atol=1e-13)
    cot = oclip.loss_cotangent(out)
    np.testing.assert_allclose(cot, 2.0 * (expect - expect.sum() / 6.0) / 6.0, rtol=1e-14, atol=1e-15)
    assert abs(cot.sum()) < 1e-13


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("make", [synth.be, synth.h10])
def test_parameter_gradient_matches_finite_differences(make):
    """grad_theta ln|psi| (Eq. trainig needs only this) against central
    differences on 16 seeded parameter indices."""
    S = make()
    o = Oracle(S)
    r = synth.random_walkers(S, 3, 4)
    cot = np.array([0.7, -1.3, 0.4])
    g = o.grad_logpsi(r, cot)
    flat = synth.flatten_params(S)
    idx = np.random.default_rng(3).choice(len(flat), 16, replace=False)
    h = 1e-5
    for k in idx:
        vals = []
        for s in (1, -1):
            fl = flat.copy()
            fl[k] += s * h
            S2 = synth.with_params(S, synth.unflatten_params(S, fl))
            vals.append((Oracle(S2).eval_logpsi(r)[0] * cot).sum())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_network_with_constant_filters_reduces_to_partner_counts():
    """With every filter's last map zeroed (W2 = 0, b2 = c) each filter is a
    constant, so electron i's messages are counts of its partners times a
    row shared by a spin class: x takes one row for up and one for down
    electrons, J is one number for every configuration and f one row per
    spin.  This pins the channel assignment (same spin, opposite spin,
    nuclei), the exclusion of i from its own sums and the layer recursion
    of the interaction layers (Methods, PauliNet extension of SchNet)."""
    sysd = synth.make_system([3.0, 2.0], [[0, 0, 0], [0, 0, 1.5]], lambda z: {0: 2, 1: 1}, n_det=2, D=8, K=4,
                             L=2, seed=11, Zd=4)
    rng = np.random.default_rng(12)
    P = {k: np.array(v, dtype=np.float64) for k, v in sysd["params"].items()}
    for n in range(sysd["L"]):
        for c in ("same", "anti", "nuc"):
            P[f"w{n}.{c}.W2"] = np.zeros_like(P[f"w{n}.{c}.W2"])
            P[f"w{n}.{c}.b2"] = rng.normal(0.0, 0.5, size=P[f"w{n}.{c}.b2"].shape)
    sysd = dict(sysd)
    sysd["params"] = P
    comp = Oracle(sysd).components(synth.random_walkers(sysd, 12, 3))

    def ssp(x):
        return np.logaddexp(x, 0.0) - np.log(2.0)

    def mlp(x, name):
        for k in (1, 2, 3):
            x = x @ P[f"{name}.W{k}"] + P[f"{name}.b{k}"]
            if k < 3:
                x = ssp(x)
        return x

    nu, nd = sysd["n_up"], sysd["n_dn"]
    xu = xd = P["x0"]
    for n in range(sysd["L"]):
        hu, hd = xu @ P[f"h{n}.W"] + P[f"h{n}.b"], xd @ P[f"h{n}.W"] + P[f"h{n}.b"]
        cs, ca, cn = (P[f"w{n}.{c}.b2"] for c in ("same", "anti", "nuc"))
        g = lambda c, z: z @ P[f"g{n}.{c}.W"] + P[f"g{n}.{c}.b"]
        zn = g("nuc", cn * P["Y"].sum(0))
        xu, xd = (xu + g("same", cs * (nu - 1) * hu) + g("anti", ca * nd * hd) + zn,
                  xd + g("same", cs * (nd - 1) * hd) + g("anti", ca * nu * hu) + zn)
    J = mlp(nu * xu + nd * xd, "eta")[0]
    fu, fd = 1.0 + mlp(xu, "kappa"), 1.0 + mlp(xd, "kappa")
    np.testing.assert_allclose(comp["J"], J, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(comp["f"][:, :nu], np.broadcast_to(fu, comp["f"][:, :nu].shape), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(comp["f"][:, nu:], np.broadcast_to(fd, comp["f"][:, nu:].shape), rtol=1e-12, atol=1e-12)
    assert abs(fu - fd).max() > 1e-6  # the spin classes differ far beyond the tolerance: a swapped channel shows
