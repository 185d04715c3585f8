"""Seeded synthetic inputs: molecular systems, network weights and walkers.

This module only draws numbers.  It holds none of the method's arithmetic: no
orbital evaluation, no network, no determinant, no derivative.  Both the CUDA
path (through the binding) and the CPU oracle take their inputs from here.

A system is a plain dict of numpy arrays:

  Z [M] f64, R [M,3] f64                 nuclear charges and positions (bohr)
  shell_center [S] i32, shell_l [S] i32  l = 0,1,2 Cartesian Gaussian shells;
                                         l = -1 is a Slater 1s function exp(-zeta r)
  shell_nprim [S] i32, prim_exp [P], prim_coef [P]
                                         contracted radial part sum_k d_k exp(-a_k r^2)
                                         (the coefficients are used as given; no
                                         normalisation is implied)
  mo_coeffs [n_b, n_orb] f64             basis-function-major
  n_up, n_dn, occ_up [n_det, n_up] i32, occ_dn [n_det, n_dn] i32, ci [n_det] f64
  net: D, Zd, K, L, r_c                  network sizes (Table 2 of the paper)
  params: dict name -> array             network weights (see ``param_shapes``)
  no_jastrow, no_backflow                ablation switches (J = 0 / f = 1)
  use_cusp, use_gamma                    switches for the nuclear cusp correction
                                         and the electronic cusp factor

Basis-function order: shells in order; within a shell the Cartesian
components are (1) for l=0, (x, y, z) for l=1 and (xx, xy, xz, yy, yz, zz) for
l=2.
"""

from __future__ import annotations

import math

import numpy as np

CART = {
    -1: [(0, 0, 0)],
    0: [(0, 0, 0)],
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)],
}


def n_basis(sys):
    return int(sum(len(CART[int(l)]) for l in sys["shell_l"]))


def param_shapes(D, Zd, K, L, M, n_orb):
    """Ordered (name, shape) list of the flat parameter vector.

    Linear maps are stored [in, out] (y = x @ W + b).  Hidden widths follow the
    reading max(d_in, d_out): the filter nets w are K -> max(K, Zd) -> Zd, the
    heads eta and kappa are D -> D -> D -> (1 | n_orb).
    """
    Hw = max(K, Zd)
    out = [("x0", (D,)), ("Y", (M, Zd))]
    for n in range(L):
        out += [(f"h{n}.W", (D, Zd)), (f"h{n}.b", (Zd,))]
        for c in ("same", "anti", "nuc"):
            out += [(f"w{n}.{c}.W1", (K, Hw)), (f"w{n}.{c}.b1", (Hw,)),
                    (f"w{n}.{c}.W2", (Hw, Zd)), (f"w{n}.{c}.b2", (Zd,))]
        for c in ("same", "anti", "nuc"):
            out += [(f"g{n}.{c}.W", (Zd, D)), (f"g{n}.{c}.b", (D,))]
    out += [("eta.W1", (D, D)), ("eta.b1", (D,)), ("eta.W2", (D, D)), ("eta.b2", (D,)),
            ("eta.W3", (D, 1)), ("eta.b3", (1,))]
    out += [("kappa.W1", (D, D)), ("kappa.b1", (D,)), ("kappa.W2", (D, D)),
            ("kappa.b2", (D,)), ("kappa.W3", (D, n_orb)), ("kappa.b3", (n_orb,))]
    return out


def n_params(sys):
    return int(sum(int(np.prod(s)) for _, s in param_shapes(
        sys["D"], sys["Zd"], sys["K"], sys["L"], len(sys["Z"]), sys["mo_coeffs"].shape[1])))


def flatten_params(sys):
    """Concatenate the parameter dict in ``param_shapes`` order (row-major)."""
    shapes = param_shapes(sys["D"], sys["Zd"], sys["K"], sys["L"], len(sys["Z"]),
                          sys["mo_coeffs"].shape[1])
    return np.concatenate([np.asarray(sys["params"][k], dtype=np.float64).reshape(-1)
                           for k, _ in shapes])


def unflatten_params(sys, flat):
    shapes = param_shapes(sys["D"], sys["Zd"], sys["K"], sys["L"], len(sys["Z"]),
                          sys["mo_coeffs"].shape[1])
    out, o = {}, 0
    for k, s in shapes:
        n = int(np.prod(s))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def random_params(rng, D, Zd, K, L, M, n_orb, scale=0.1):
    """All weights and biases drawn N(0, scale^2)."""
    return {k: rng.normal(0.0, scale, size=s) for k, s in param_shapes(D, Zd, K, L, M, n_orb)}


def zero_params(D, Zd, K, L, M, n_orb):
    return {k: np.zeros(s) for k, s in param_shapes(D, Zd, K, L, M, n_orb)}


def _shells_for_atom(rng, center, spec, lo=0.1, hi=20.0):
    """spec: dict l -> number of contracted shells.  Each l gets a geometric
    exponent ladder over [lo, hi] with n_l + 2 primitives; shell c contracts
    primitives c, c+1, c+2 with seeded positive coefficients."""
    out = []
    for l in sorted(spec):
        ns = spec[l]
        if ns == 0:
            continue
        exps = np.geomspace(hi, lo, ns + 2)
        for c in range(ns):
            e = exps[c:c + 3].copy()
            d = rng.uniform(0.5, 1.5, size=3)
            out.append((center, l, e, d))
    return out


def _pack_shells(shells):
    sc = np.array([s[0] for s in shells], dtype=np.int32)
    sl = np.array([s[1] for s in shells], dtype=np.int32)
    sn = np.array([len(s[2]) for s in shells], dtype=np.int32)
    pe = np.concatenate([np.asarray(s[2], dtype=np.float64) for s in shells])
    pc = np.concatenate([np.asarray(s[3], dtype=np.float64) for s in shells])
    return dict(shell_center=sc, shell_l=sl, shell_nprim=sn, prim_exp=pe, prim_coef=pc)


def _orthonormal(rng, n_b, n_orb):
    """Columns orthonormal in the Euclidean sense (QR of a Gaussian matrix)."""
    A = rng.normal(size=(n_b, n_orb))
    Q, Rm = np.linalg.qr(A)
    return Q * np.sign(np.diag(Rm))[None, :]


def _determinants(rng, n_det, n_up, n_dn, n_orb):
    """Determinant 0 is aufbau; the others are distinct seeded single or double
    excitations inside the n_orb orbitals.  c_0 = 1, c_p ~ N(0, 0.1^2)."""
    base_u = list(range(n_up))
    base_d = list(range(n_dn))
    seen = {(tuple(base_u), tuple(base_d))}
    dets = [(base_u, base_d)]
    tries = 0
    while len(dets) < n_det:
        tries += 1
        if tries > 100000:
            raise ValueError("cannot draw enough distinct determinants")
        u, d = list(base_u), list(base_d)
        level = 1 if rng.random() < 0.5 else 2
        for _ in range(level):
            spin = rng.integers(0, 2) if n_dn > 0 else 0
            occ = u if spin == 0 else d
            if len(occ) == 0:
                continue
            virt = [m for m in range(n_orb) if m not in occ]
            if not virt:
                continue
            k = int(rng.integers(0, len(occ)))
            occ[k] = int(virt[int(rng.integers(0, len(virt)))])
        key = (tuple(u), tuple(d))
        if key in seen:
            continue
        seen.add(key)
        dets.append((u, d))
    occ_up = np.array([d[0] for d in dets], dtype=np.int32).reshape(n_det, n_up)
    occ_dn = np.array([d[1] for d in dets], dtype=np.int32).reshape(n_det, n_dn)
    ci = np.concatenate([[1.0], rng.normal(0.0, 0.1, size=n_det - 1)])
    return occ_up, occ_dn, ci


def make_system(Z, R, atom_spec, n_det, D, K, L, seed, r_c=10.0, Zd=None,
                n_orb=None, n_up=None, n_dn=None, use_cusp=1, use_gamma=1, no_jastrow=0, no_backflow=0):
    """Seeded neutral system.  atom_spec(Z_I) -> {l: n_shells}."""
    rng = np.random.default_rng(seed)
    Z = np.asarray(Z, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    N = int(round(Z.sum()))
    n_up = (N + 1) // 2 if n_up is None else n_up
    n_dn = N - n_up if n_dn is None else n_dn
    shells = []
    for I, z in enumerate(Z):
        shells += _shells_for_atom(rng, I, atom_spec(z))
    sysd = _pack_shells(shells)
    sysd.update(Z=Z, R=R)
    n_b = n_basis(sysd)
    if n_orb is None:
        n_orb = n_up if n_det == 1 else min(n_b, n_up + 4)
    Zd = D // 2 if Zd is None else Zd
    sysd["mo_coeffs"] = _orthonormal(rng, n_b, n_orb)
    occ_up, occ_dn, ci = _determinants(rng, n_det, n_up, n_dn, n_orb)
    sysd.update(n_up=n_up, n_dn=n_dn, occ_up=occ_up, occ_dn=occ_dn, ci=ci,
                D=D, Zd=Zd, K=K, L=L, r_c=float(r_c), use_cusp=int(use_cusp),
                use_gamma=int(use_gamma), cusp_phi0=None, no_jastrow=int(no_jastrow), no_backflow=int(no_backflow))
    sysd["params"] = random_params(rng, D, Zd, K, L, len(Z), n_orb)
    return sysd


def electron_nuclei(sys):
    """Nucleus assigned to each electron for walker initialisation: the list of
    nucleus indices repeated Z_I times; up electron k takes entry 2k, down
    electron k entry 2k+1 (spins alternate), wrapping around for ions."""
    lst = []
    for I, z in enumerate(sys["Z"]):
        lst += [I] * int(round(z))
    if not lst:
        lst = [0]
    n_up, n_dn = sys["n_up"], sys["n_dn"]
    up = [lst[(2 * k) % len(lst)] for k in range(n_up)]
    dn = [lst[(2 * k + 1) % len(lst)] for k in range(n_dn)]
    return np.array(up + dn, dtype=np.int64)


def random_walkers(sys, W, seed, width=1.0):
    """Electrons drawn N(R_I, width^2 I_3) around their assigned nuclei."""
    rng = np.random.default_rng(seed)
    nuc = electron_nuclei(sys)
    R = sys["R"][nuc]
    return R[None, :, :] + width * rng.normal(size=(W, len(nuc), 3))


# ---------------------------------------------------------------------------
# The workloads (seeded, shaped like the paper's systems).

def _spec_h(z):
    return {0: 3}


def h2(seed=0):
    """H2: Z=1 at +-0.7 bohr on z, 1 up 1 down, 1 determinant, 3 s shells per
    atom, D=32, L=2, K=16, r_c=10."""
    return make_system([1.0, 1.0], [[0, 0, -0.7], [0, 0, 0.7]], _spec_h, n_det=1,
                       D=32, K=16, L=2, seed=seed)


def be(seed=0):
    """Be atom: Z=4, 2 up 2 down, 4 determinants, 4s+2p shells (10 functions),
    D=64, L=3, K=32."""
    return make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=4,
                       D=64, K=32, L=3, seed=seed)


def h10(seed=0):
    """Linear H10, spacing 1.8 bohr, 5 up 5 down, 16 determinants, 3 s shells
    per atom (30 functions), D=64, L=3, K=32."""
    R = [[0, 0, 1.8 * (k - 4.5)] for k in range(10)]
    return make_system([1.0] * 10, R, _spec_h, n_det=16, D=64, K=32, L=3, seed=seed)


def n2(seed=0):
    """N2-shaped: two Z=7 nuclei 2.068 bohr apart, 7 up 7 down, 32
    determinants, 4s4p2d Cartesian shells per atom (28 functions), D=128, L=4,
    K=32."""
    return make_system([7.0, 7.0], [[0, 0, -1.034], [0, 0, 1.034]],
                       lambda z: {0: 4, 1: 4, 2: 2}, n_det=32, D=128, K=32, L=4, seed=seed)


def lih(seed=0, use_cusp=1, use_gamma=1):
    """LiH-shaped: Li (Z=3) at the origin and H at 3.015 bohr on the x axis,
    2 up 2 down electrons, 4 determinants; Li 4s2p shells, H 3 s shells; D=64,
    L=3, K=32."""
    return make_system([3.0, 1.0], [[0, 0, 0], [3.015, 0, 0]], lambda z: {0: 4, 1: 2} if z >= 3 else _spec_h(z),
                       n_det=4, D=64, K=32, L=3, seed=seed, use_cusp=use_cusp, use_gamma=use_gamma)


def lih_scan():
    """The one-dimensional scan of the LiH results: on the x axis, from the
    left, the Li nucleus, a spin-up electron (x = 1.0), a spin-down electron
    (x = 2.0) and the H nucleus; the second spin-down electron off the axis;
    the second spin-up electron (index 1, electrons are ordered up first) moves
    along x.  Returns (r0 [4][3], electron, direction, t0, t1)."""
    r0 = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [1.1, 1.3, 0.6]])
    return r0, 1, np.array([1.0, 0.0, 0.0]), -1.5, 4.5


WORKLOADS = {
    "h2": dict(make=h2, W=1024),
    "be": dict(make=be, W=4096, n_steps=100, sigma=0.2),
    "h10": dict(make=h10, W=8192),
    "n2": dict(make=n2, W=16384),
}


def serving_system(seed, max_nuclei=6, zmax=10, box=6.0, min_sep=1.0, D=64, K=32, L=3):
    """A random neutral molecule for the serving stream: 1-6 nuclei with Z in
    1..10 (total electrons 2..30), nuclei uniform in a 6-bohr box at least
    1 bohr apart, 1-32 determinants.  Z<=2 atoms get 3 s shells, heavier atoms
    4s3p."""
    rng = np.random.default_rng(seed)
    while True:
        M = int(rng.integers(1, max_nuclei + 1))
        Z = rng.integers(1, zmax + 1, size=M).astype(np.float64)
        if 2 <= Z.sum() <= 30:
            break
    R = []
    while len(R) < M:
        p = rng.uniform(-box / 2, box / 2, size=3)
        if all(np.linalg.norm(p - q) >= min_sep for q in R):
            R.append(p)
    spec = lambda z: {0: 3} if z <= 2 else {0: 4, 1: 3}
    N = int(Z.sum())
    n_up = (N + 1) // 2
    n_det_max = 32
    n_det = int(rng.integers(1, n_det_max + 1))
    if n_up == 1 and N - n_up <= 1:
        n_det = min(n_det, 4)
    sub = int(rng.integers(0, 2**31 - 1))
    for attempt in range(8):
        try:
            return make_system(Z, np.array(R), spec, n_det=n_det, D=D, K=K, L=L, seed=sub + attempt)
        except ValueError:
            n_det = max(1, n_det // 2)
    return make_system(Z, np.array(R), spec, n_det=1, D=D, K=K, L=L, seed=sub)


def serving_stream(n_jobs=2000, master_seed=2024, rate_per_s=50.0, wmin=256, wmax=16384):
    """Poisson arrivals of jobs; job i uses seed hash(master_seed, i)."""
    rng = np.random.default_rng(master_seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_jobs))
    jobs = []
    for i in range(n_jobs):
        s = int(np.random.SeedSequence([master_seed, i]).generate_state(1)[0])
        jr = np.random.default_rng(s)
        W = int(round(math.exp(jr.uniform(math.log(wmin), math.log(wmax)))))
        kind = "eloc" if jr.random() < 0.5 else "sweep"
        jobs.append(dict(arrival=float(t[i]), seed=s, W=W, kind=kind, n_steps=10, sigma=0.2))
    return jobs


# ---------------------------------------------------------------------------
# Special systems with closed-form answers (single-electron and product states).

def _special(Z, R, shells, n_up, n_dn, mo, occ_up, occ_dn, ci, D=8, K=4, L=1,
             use_cusp=0, use_gamma=1):
    sysd = _pack_shells(shells)
    sysd.update(Z=np.asarray(Z, dtype=np.float64), R=np.asarray(R, dtype=np.float64).reshape(-1, 3))
    n_orb = mo.shape[1]
    sysd.update(mo_coeffs=np.asarray(mo, dtype=np.float64), n_up=n_up, n_dn=n_dn,
                occ_up=np.asarray(occ_up, dtype=np.int32).reshape(len(ci), n_up),
                occ_dn=np.asarray(occ_dn, dtype=np.int32).reshape(len(ci), n_dn),
                ci=np.asarray(ci, dtype=np.float64), D=D, Zd=D // 2, K=K, L=L, r_c=10.0,
                use_cusp=use_cusp, use_gamma=use_gamma, cusp_phi0=None)
    sysd["params"] = zero_params(D, D // 2, K, L, len(Z), n_orb)
    return sysd


def hydrogen_like_sto(Z=1.0, zeta=1.0):
    """One electron, psi = exp(-zeta r) around a nucleus of charge Z; the
    network weights are zero (J = 0, backflow f = 1)."""
    return _special([Z], [[0, 0, 0]], [(0, -1, [zeta], [1.0])], 1, 0, np.ones((1, 1)),
                    [[0]], np.zeros((1, 0)), [1.0])


def sto_beside_bare_nuclei(ZA=1.0, zeta=1.0, bare=((2.0, (0.0, 0.0, 1.7)),)):
    """One electron in exp(-zeta r_A) on a nucleus A of charge ZA at the
    origin, next to further nuclei (charge, position) that carry no basis
    function; the network weights are zero."""
    Z = [ZA] + [b[0] for b in bare]
    R = [[0.0, 0.0, 0.0]] + [list(b[1]) for b in bare]
    return _special(Z, R, [(0, -1, [zeta], [1.0])], 1, 0, np.ones((1, 1)), [[0]], np.zeros((1, 0)), [1.0])


def single_gto(Z=1.0, alpha=0.7):
    """One electron in a single s Gaussian exp(-alpha r^2)."""
    return _special([Z], [[0, 0, 0]], [(0, 0, [alpha], [1.0])], 1, 0, np.ones((1, 1)),
                    [[0]], np.zeros((1, 0)), [1.0])


def single_cartesian_gto(Z=1.0, alpha=0.7, l=1, component=0, coefs=(1.0,)):
    """One electron in one Cartesian component x^a y^b z^c sum_k d_k
    exp(-alpha_k r^2) of an l-shell (components in the order of CART[l]);
    alpha a number or one exponent per coefficient d_k."""
    alphas = list(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (len(coefs),)))
    mo = np.zeros((len(CART[l]), 1))
    mo[component, 0] = 1.0
    return _special([Z], [[0, 0, 0]], [(0, l, alphas, list(coefs))], 1, 0, mo, [[0]], np.zeros((1, 0)), [1.0])


def helium_like_product(Z=2.0, zeta=1.6875, use_gamma=0):
    """Two electrons (1 up, 1 down) in exp(-zeta r1) exp(-zeta r2); the
    network is off, the electronic cusp factor off unless use_gamma."""
    return _special([Z], [[0, 0, 0]], [(0, -1, [zeta], [1.0])], 1, 1, np.ones((1, 1)),
                    [[0]], [[0]], [1.0], use_gamma=use_gamma)


def two_orbital_product(Z=3.0, zetas=(2.7, 0.9), coefs=(1.3, 0.6), mo=((0.8, 0.3), (0.5, 1.1))):
    """Two Slater 1s functions d_b exp(-zeta_b r) on one nucleus, two
    molecular orbitals phi_mu = sum_b mo[b][mu] chi_b, the up electron in
    orbital 0 and the down electron in orbital 1; the network and the
    electronic cusp factor are off."""
    shells = [(0, -1, [zetas[0]], [coefs[0]]), (0, -1, [zetas[1]], [coefs[1]])]
    return _special([Z], [[0, 0, 0]], shells, 1, 1, np.asarray(mo, dtype=np.float64), [[0]], [[1]], [1.0],
                    use_gamma=0)


def with_params(sys, params):
    out = dict(sys)
    out["params"] = params
    return out
