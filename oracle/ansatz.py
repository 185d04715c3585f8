"""PauliNet ansatz, local energy and parameter gradient -- plain torch float64
on the CPU (test infrastructure only; see the package docstring).

Everything here follows the paper's definitions directly, vectorised over
walkers only:
  psi(r) = exp(gamma + J) sum_p c_p det[phi~_up] det[phi~_dn],
  phi~_{mu i} = phi_mu(r_i) f_{mu i}                     Eq. (ansatz)
  gamma = sum_{i<j} -c_ij / (1 + r_ij), c = 1/2 (anti), 1/4 (same)  Methods
  e_k(r) = r^2 exp(-r - (r - mu_k)^2 / sigma_k^2),
  mu_k = r_c q_k^2, sigma_k = (1 + r_c q_k) / 7        Methods (distance features)
  SchNet iteration with channels same/anti/nuc           Methods (PauliNet SchNet)
  J = eta(sum_i x_i), f_i = 1 + kappa(x_i)               Results (Jastrow/backflow)
  E_loc = -1/2 (lap ln|psi| + |grad ln|psi||^2) + V      Eq. (monte-carlo)
  grad_theta L = 2 E[(E_loc - L) grad_theta ln|psi|]     Eq. (trainig)

Readings of points the paper leaves open:
q_k = k/(K+1) (open interval); shifted softplus activation; hidden widths
max(d_in, d_out); biases on every linear map; no activation after a last
layer; f = 1 + kappa(x); one x0 for all electrons; c_ij = 1/4 same spin,
1/2 opposite spin; electrons ordered up first.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from paper_1909_08423_gb300 import synth

from . import cusp as _cusp

DT = torch.float64
LN2 = math.log(2.0)


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


# --------------------------------------------------------------------------
# orbitals


def basis_values(sys, r):
    """chi_b(r_i) for every basis function: [W, N, n_b].  Cartesian Gaussians
    x^a y^b z^c sum_k d_k exp(-alpha_k |r - R_c|^2); Slater 1s d exp(-zeta |r - R_c|)."""
    R = _t(sys["R"])
    out = []
    o = 0
    for s in range(len(sys["shell_l"])):
        c = int(sys["shell_center"][s])
        l = int(sys["shell_l"][s])
        npr = int(sys["shell_nprim"][s])
        ex = _t(sys["prim_exp"][o:o + npr])
        co = _t(sys["prim_coef"][o:o + npr])
        o += npr
        v = r - R[c]
        r2 = (v * v).sum(-1)
        if l == -1:
            out.append(co[0] * torch.exp(-ex[0] * torch.sqrt(r2)))
            continue
        rad = (co * torch.exp(-ex * r2[..., None])).sum(-1)
        for (a, b, cc) in synth.CART[l]:
            out.append(v[..., 0] ** a * v[..., 1] ** b * v[..., 2] ** cc * rad)
    return torch.stack(out, -1)


def _s_rows(sys, I):
    """Basis indices and primitive slices of the l=0 Gaussian shells on I."""
    rows = []
    b = 0
    o = 0
    for s in range(len(sys["shell_l"])):
        l = int(sys["shell_l"][s])
        npr = int(sys["shell_nprim"][s])
        if l == 0 and int(sys["shell_center"][s]) == I:
            rows.append((b, o, npr))
        o += npr
        b += 1 if l <= 0 else (3 if l == 1 else 6)
    return rows


class Model:
    """Holds a system dict and its derived cusp tables."""

    def __init__(self, sys):
        self.sys = sys
        self.N = sys["n_up"] + sys["n_dn"]
        self.C = _t(sys["mo_coeffs"])
        self.cusp = _cusp.cusp_tables(sys, self._orbital_at) if sys["use_cusp"] else None

    def _orbital_at(self, p):
        r = _t(p).reshape(1, 1, 3)
        return (basis_values(self.sys, r) @ self.C).reshape(-1).numpy()

    # -- phi_mu(r_i) with the nuclear cusp splice ---------------------------
    def orbitals(self, r):
        sys = self.sys
        phi = basis_values(sys, r) @ self.C
        if self.cusp is None:
            return phi
        R = _t(sys["R"])
        for I, tab in enumerate(self.cusp):
            if not tab["active"].any():
                continue
            rc = tab["rc"]
            d = torch.linalg.norm(r - R[I], dim=-1)
            inside = d < rc
            dc = torch.clamp(d, max=rc)
            phis = torch.zeros_like(phi)
            for (b, o, npr) in _s_rows(sys, I):
                ex = _t(sys["prim_exp"][o:o + npr])
                co = _t(sys["prim_coef"][o:o + npr])
                rad = (co * torch.exp(-ex * (dc * dc)[..., None])).sum(-1)
                phis = phis + rad[..., None] * self.C[b]
            a = _t(tab["a"])
            p = a[:, 0] + dc[..., None] * (a[:, 1] + dc[..., None] * (a[:, 2] + dc[..., None] * (a[:, 3] + dc[..., None] * a[:, 4])))
            repl = _t(tab["C"]) + _t(tab["sgn"]) * torch.exp(p)
            new = phi - phis + repl
            mask = inside[..., None] & torch.as_tensor(tab["active"])[None, None, :]
            phi = torch.where(mask, new, phi)
        return phi


# --------------------------------------------------------------------------
# network


def ssp(x):
    """Shifted softplus ln(exp(x)/2 + 1/2) = x/2 + ln cosh(x/2): one smooth
    expression, so that autograd gives its derivative, the logistic
    function, at every x (x = 0 included)."""
    return 0.5 * x + torch.log(torch.cosh(0.5 * x))


def features(sys, d):
    """e_k(d) for k = 1..K: [..., K]."""
    K = sys["K"]
    rc = sys["r_c"]
    q = torch.arange(1, K + 1, dtype=DT) / (K + 1)
    mu = rc * q * q
    sig = (1.0 + rc * q) / 7.0
    d = d[..., None]
    return d * d * torch.exp(-d - (d - mu) ** 2 / sig ** 2)


def _mlp(x, Ws):
    """Affine maps with ssp between them (none after the last)."""
    for k, (W, b) in enumerate(Ws):
        x = x @ W + b
        if k + 1 < len(Ws):
            x = ssp(x)
    return x


def params_to_torch(sys, params=None, requires_grad=False):
    p = sys["params"] if params is None else params
    return {k: _t(v).clone().requires_grad_(requires_grad) for k, v in p.items()}


def pair_lists(sys):
    N = sys["n_up"] + sys["n_dn"]
    spin = [0] * sys["n_up"] + [1] * sys["n_dn"]
    pi, pj = [], []
    for i in range(N):
        for j in range(N):
            if i != j:
                pi.append(i)
                pj.append(j)
    same = [spin[i] == spin[j] for i, j in zip(pi, pj)]
    return (torch.tensor(pi, dtype=torch.long), torch.tensor(pj, dtype=torch.long),
            torch.tensor(same, dtype=torch.bool))


def network(sys, P, r):
    """J [W] and backflow f [W, N, n_orb] from the SchNet-style iteration."""
    Wn, N = r.shape[0], r.shape[1]
    D, Zd, L = sys["D"], sys["Zd"], sys["L"]
    R = _t(sys["R"])
    pi, pj, same = pair_lists(sys)
    x = P["x0"].expand(Wn, N, D)
    den = torch.linalg.norm(r[:, :, None, :] - R[None, None], dim=-1)   # [W,N,M]
    e_en = features(sys, den)
    if len(pi):
        dee = torch.linalg.norm(r[:, pi] - r[:, pj], dim=-1)             # [W,P]
        e_ee = features(sys, dee)
    for n in range(L):
        h = x @ P[f"h{n}.W"] + P[f"h{n}.b"]                              # [W,N,Zd]
        z = {}
        for c, sel in (("same", same), ("anti", ~same)):
            zc = torch.zeros(Wn, N, Zd, dtype=DT)
            if len(pi) and bool(sel.any()):
                w = _mlp(e_ee[:, sel], [(P[f"w{n}.{c}.W1"], P[f"w{n}.{c}.b1"]),
                                        (P[f"w{n}.{c}.W2"], P[f"w{n}.{c}.b2"])])
                zc = zc.index_add(1, pi[sel], w * h[:, pj[sel]])
            z[c] = zc
        wn = _mlp(e_en, [(P[f"w{n}.nuc.W1"], P[f"w{n}.nuc.b1"]),
                         (P[f"w{n}.nuc.W2"], P[f"w{n}.nuc.b2"])])          # [W,N,M,Zd]
        z["nuc"] = (wn * P["Y"][None, None]).sum(2)
        x = x + sum(z[c] @ P[f"g{n}.{c}.W"] + P[f"g{n}.{c}.b"] for c in ("same", "anti", "nuc"))
    # ablation variants (Results, single/multiple determinants with and
    # without backflow): a removed head is J = 0 or f = 1
    J = _mlp(x.sum(1), [(P["eta.W1"], P["eta.b1"]), (P["eta.W2"], P["eta.b2"]),
                        (P["eta.W3"], P["eta.b3"])])[..., 0]
    f = 1.0 + _mlp(x, [(P["kappa.W1"], P["kappa.b1"]), (P["kappa.W2"], P["kappa.b2"]),
                       (P["kappa.W3"], P["kappa.b3"])])
    if sys.get("no_jastrow", 0):
        J = torch.zeros_like(J)
    if sys.get("no_backflow", 0):
        f = torch.ones_like(f)
    return J, f


def gamma(sys, r):
    """Electronic cusp factor sum_{i<j} -c_ij / (1 + r_ij)."""
    N = sys["n_up"] + sys["n_dn"]
    spin = [0] * sys["n_up"] + [1] * sys["n_dn"]
    g = torch.zeros(r.shape[0], dtype=DT)
    if not sys["use_gamma"]:
        return g
    for i in range(N):
        for j in range(i + 1, N):
            c = 0.25 if spin[i] == spin[j] else 0.5
            g = g - c / (1.0 + torch.linalg.norm(r[:, i] - r[:, j], dim=-1))
    return g


def potential(sys, r):
    """Coulomb V = sum_{i<j} 1/r_ij - sum_{iI} Z_I/r_iI + sum_{I<J} Z_I Z_J/R_IJ."""
    Z = _t(sys["Z"])
    R = _t(sys["R"])
    N = r.shape[1]
    V = torch.zeros(r.shape[0], dtype=DT)
    for i in range(N):
        for j in range(i + 1, N):
            V = V + 1.0 / torch.linalg.norm(r[:, i] - r[:, j], dim=-1)
        V = V - (Z / torch.linalg.norm(r[:, i, None, :] - R[None], dim=-1)).sum(-1)
    for I in range(len(Z)):
        for J in range(I + 1, len(Z)):
            V = V + Z[I] * Z[J] / torch.linalg.norm(R[I] - R[J])
    return V


def slater(sys, phit):
    """Per determinant: ln|det up| + ln|det dn| and the product of signs."""
    nu, nd = sys["n_up"], sys["n_dn"]
    ld, sg = [], []
    for p in range(len(sys["ci"])):
        s_tot = torch.ones(phit.shape[0], dtype=DT)
        l_tot = torch.zeros(phit.shape[0], dtype=DT)
        for rows, occ in ((slice(0, nu), sys["occ_up"][p]), (slice(nu, nu + nd), sys["occ_dn"][p])):
            if len(occ) == 0:
                continue
            A = phit[:, rows][:, :, torch.as_tensor(np.asarray(occ), dtype=torch.long)]
            s, l = torch.linalg.slogdet(A)
            s_tot = s_tot * s
            l_tot = l_tot + l
        ld.append(l_tot)
        sg.append(s_tot)
    return torch.stack(ld, 1), torch.stack(sg, 1)


class Oracle(Model):
    """ln|psi|, sign, E_loc and grad_theta ln|psi| for one system."""

    def logpsi(self, r, P=None):
        sys = self.sys
        P = params_to_torch(sys) if P is None else P
        phi = self.orbitals(r)
        J, f = network(sys, P, r)
        ld, sg = slater(sys, phi * f)
        ci = _t(sys["ci"])
        m = ld.max(1).values
        t = (ci * sg * torch.exp(ld - m[:, None])).sum(1)
        return gamma(sys, r) + J + m + torch.log(torch.abs(t)), torch.sign(t)

    def components(self, r):
        """Intermediate values for stepwise parity: phi, J, f, per-det ld/sign."""
        r = _t(r)
        with torch.no_grad():
            P = params_to_torch(self.sys)
            phi = self.orbitals(r)
            J, f = network(self.sys, P, r)
            ld, sg = slater(self.sys, phi * f)
        return dict(phi=phi.numpy(), J=J.numpy(), f=f.numpy(), ld=ld.numpy(), sign_det=sg.numpy())

    def eval_logpsi(self, r):
        with torch.no_grad():
            lp, s = self.logpsi(_t(r))
        return lp.numpy(), s.numpy()

    def derivatives(self, r):
        """ln|psi|, sign, grad ln|psi| [W,N,3] and lap ln|psi| [W] (exact, by
        reverse-mode autograd: one gradient, then the Hessian diagonal)."""
        r = _t(r).clone().requires_grad_(True)
        lp, s = self.logpsi(r)
        g = torch.autograd.grad(lp.sum(), r, create_graph=True)[0]
        lap = torch.zeros(r.shape[0], dtype=DT)
        N = r.shape[1]
        for i in range(N):
            for a in range(3):
                gi = torch.autograd.grad(g[:, i, a].sum(), r, retain_graph=True)[0]
                lap = lap + gi[:, i, a]
        return lp.detach().numpy(), s.detach().numpy(), g.detach().numpy(), lap.detach().numpy()

    def value_and_grad(self, r):
        """ln|psi|, sign and grad_r ln|psi| [W,N,3] (one reverse-mode gradient);
        the drift of the Langevin sampler."""
        r = _t(r).clone().requires_grad_(True)
        lp, s = self.logpsi(r)
        g = torch.autograd.grad(lp.sum(), r)[0]
        return lp.detach().numpy(), s.detach().numpy(), g.numpy()

    def local_energy(self, r):
        """E_loc = -1/2 (lap ln|psi| + |grad ln|psi||^2) + V, plus ln|psi| and sign."""
        lp, s, g, lap = self.derivatives(r)
        V = potential(self.sys, _t(r)).numpy()
        E = -0.5 * (lap + (g * g).sum((1, 2))) + V
        return E, lp, s

    def grad_logpsi(self, r, cot):
        """sum_w cot_w grad_theta ln|psi_w| as a flat vector in the parameter
        layout of ``synth.param_shapes``."""
        P = params_to_torch(self.sys, requires_grad=True)
        lp, _ = self.logpsi(_t(r), P)
        if lp.requires_grad:  # else no parameter enters psi (every head removed, gamma off)
            (lp * _t(cot)).sum().backward()
        shapes = synth.param_shapes(self.sys["D"], self.sys["Zd"], self.sys["K"], self.sys["L"],
                                    len(self.sys["Z"]), self.sys["mo_coeffs"].shape[1])
        # parameters that do not enter (e.g. same-spin filters with one
        # electron per spin) have zero gradient
        return np.concatenate([(P[k].grad if P[k].grad is not None else torch.zeros_like(P[k])).numpy().reshape(-1)
                               for k, _ in shapes])
