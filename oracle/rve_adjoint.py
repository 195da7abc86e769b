"""Plain FP64 CPU oracle of the adjoint (reverse) sensitivity of the final
homogenised axial stress of a converged load path.

TEST INFRASTRUCTURE ONLY.  Only the test suite may import this module.  It
shares no code with the CUDA path.  The paper has no adjoint; this is the
discrete adjoint of its converged increments (Algorithm 1 at convergence is
the monolithic implicit solution, Section 3.3), written from the Lagrangian
of the discrete problem:

  objective   J = <sigma_N>_11 = (1/V) sum_x sigma_N(x)_11
  increment n residuals, at the converged state (eps_n, abar_n) with the
  local history h_{n-1} = (eps^p_{n-1}, e_{n-1}) (e = eps_p for the Lemaitre
  phase, kappa for the cracking phase, R20):
    mechanics  P (sigma_n - Sigma_bar_n) = 0, eps_n - Ebar_n in V0
               (P = G*, the orthogonal projector onto V0: compatible fields
               whose mean has no strain-controlled component, R7)
    Helmholtz  L_j abar_{n,j} - alpha_{n,j} = 0, L_j a = a + sum_d
               G_d^T (l_j^2 G_d a), G_d a = F^-1(k_d F a) (R15)
    history    h_n = H(eps_n, h_{n-1})
  with sigma, alpha, H from the return map (R8-R11, R20).

Stationarity of J - sum_n <lambda_n, P(sigma_n - Sigma_bar)> - sum_n <mu_n,
L abar_n - alpha_n> with respect to every state gives, from n = N down to 1,
with w_n = (w_sigma, w_alpha, w_h) = (s_n - lambda_n, mu_n, eta_n), s_N =
e_11 / V, s_n = 0 otherwise, eta_N = 0:

    P C_T lambda_n = P [ d(sigma, alpha, h)/d eps ]^T (s_n, mu_n, eta_n),
                                                         lambda_n in V0
    L_j mu_{n,j}   = [ d sigma / d abar_j ]^T (s_n - lambda_n)
    eta_{n-1}      = [ d(sigma, alpha, h)/d h_{n-1} ]^T w_n
    dJ/dtheta     += [ d(sigma, alpha, h)/d theta ]^T w_n
                     - sum_j <mu_{n,j}, (dL_j/dtheta) abar_{n,j}>

The first two are coupled; they are solved by alternating the two solves
(the transposed staggered scheme) until both stop changing.  The per-voxel
Jacobians come from complex-step differentiation (Squire and Trapp 1998) of
a complex-safe restatement of the return map; the derivative of the
cracking variable ||<eps>_+|| uses its closed form <eps>_+ / ||<eps>_+||.

Parameters theta: per phase sigma_y, H, eps_C, eps_R (kappa_C, kappa_R for
the cracking law), the characteristic length l_k of each non-local variable
(its whole row of the l table scales with it, R13), and a per-voxel factor
s(x) on the Young's modulus (K and mu scale with it).
"""
from __future__ import annotations

import math

import numpy as np

from . import rve_oracle as O

PARAMS = ("sigma_y", "H", "eps_C", "eps_R")
S23 = math.sqrt(2.0 / 3.0)
CS_H = 1e-30           # complex-step size


# ================================================== complex-safe local update
def _ramp(abar, ph):
    """D = clamp((abar - c)/(r - c), 0, D_max) with branch tests on the real
    part (derivative 0 on the clamped branches)."""
    D = (abar - ph["eps_C"]) / (ph["eps_R"] - ph["eps_C"])
    D = np.where(D.real < 0.0, 0.0, D)
    return np.where(D.real > ph["D_max"], ph["D_max"], D)


def ppn_cs(e):
    """||<e>_+|| (R20) for Mandel strains e (n, 6), complex step through the
    closed-form gradient <e>_+ / ||<e>_+|| at the real part."""
    er = np.real(e)
    lam, vec = np.linalg.eigh(O.mandel_to_tensor(er))
    lp = np.maximum(lam, 0.0)
    kap = np.sqrt(np.sum(lp * lp, axis=-1))
    if not np.iscomplexobj(e):
        return kap
    Tp = np.einsum("nij,nj,nkj->nik", vec, lp, vec)
    grad = O.tensor_to_mandel(Tp)
    grad = np.where(kap[:, None] > 0.0, grad / np.where(kap > 0.0, kap, 1.0)[:, None], 0.0)
    return kap + 1j * np.sum(grad * np.imag(e), axis=-1)


def local_update(eps6, epsp_n, ep_n, abar, phase, phases, stiff, dparam=None):
    """Return map of every voxel (same equations as rve_oracle.return_map)
    written so that complex inputs carry first derivatives.

    eps6, epsp_n: (V, 6); ep_n: (V,); abar: (J, V); stiff: (V,); all may be
    complex.  dparam: {(phase, name): increment} added to the phase's
    parameter.  Returns sigma (V, 6), alpha (J, V), epsp (V, 6), ep (V,)."""
    Vn = eps6.shape[0]
    J = abar.shape[0]
    cplx = any(np.iscomplexobj(a) for a in (eps6, epsp_n, ep_n, abar, stiff)) or bool(dparam)
    dt = np.complex128 if cplx else np.float64
    sigma = np.zeros((Vn, 6), dtype=dt)
    epsp = np.array(epsp_n, dtype=dt)
    ep = np.array(ep_n, dtype=dt)
    alpha = np.zeros((J, Vn), dtype=dt)
    for q, P in enumerate(phases):
        sel = phase == q
        if not np.any(sel):
            continue
        ph = {k: getattr(P, k) for k in ("sigma_y", "H", "eps_C", "eps_R", "D_max")}
        if dparam:
            for k in PARAMS:
                ph[k] = ph[k] + dparam.get((q, k), 0.0)
        sc = stiff[sel]
        K = P.K * sc
        mu = P.mu * sc
        e = eps6[sel] - epsp_n[sel]
        tr = e[:, 0] + e[:, 1] + e[:, 2]
        dev = e - tr[:, None] * O.IVEC[None, :] / 3.0
        s_tr = 2.0 * mu[:, None] * dev
        sig_eff = K[:, None] * tr[:, None] * O.IVEC[None, :] + s_tr
        D = np.zeros(int(sel.sum()), dtype=dt)
        if P.law == 1:
            qn = np.sqrt(np.sum(s_tr * s_tr, axis=1))
            f = qn - S23 * (ph["sigma_y"] + ph["H"] * ep_n[sel])
            pl = np.real(f) > 0.0
            qs = np.where(pl, qn, 1.0)
            dl = np.where(pl, f / (2.0 * mu + 2.0 * ph["H"] / 3.0), 0.0)
            nhat = np.where(pl[:, None], s_tr / qs[:, None], 0.0)
            epsp[sel] = epsp_n[sel] + dl[:, None] * nhat
            ep[sel] = ep_n[sel] + S23 * dl
            sig_eff = sig_eff - 2.0 * mu[:, None] * dl[:, None] * nhat
            if P.var >= 0:
                D = _ramp(abar[P.var][sel], ph)
                alpha[P.var, sel] = ep[sel]
        elif P.law == 2:
            kn = ppn_cs(e)
            hist = np.real(ep_n[sel]) >= np.real(kn)
            kap = np.where(hist, ep_n[sel], kn)
            ep[sel] = kap
            if P.var >= 0:
                D = _ramp(abar[P.var][sel], ph)
                alpha[P.var, sel] = kap
        sigma[sel] = (1.0 - D)[:, None] * sig_eff
    return sigma, alpha, epsp, ep


# ================================================== per-voxel Jacobian products
class LocalJacobian:
    """Per-voxel derivatives of (sigma, alpha, eps^p, e) at one converged
    state, by complex step along every input direction."""

    def __init__(self, grid, eps_c, epsp_prev, ep_prev, abar, phase, phases, stiff):
        d = grid.d
        self.d = d
        self.comps = O.carried(d)
        self.phases = phases
        self.phase = phase
        eps6 = O.embed(eps_c, d).reshape(-1, 6)
        self.args = (eps6, epsp_prev, ep_prev, abar, phase, phases, stiff)
        self.cols = {}
        Vn = eps6.shape[0]
        J = abar.shape[0]

        def run(key, **pert):
            a = [np.array(x, dtype=np.complex128)
                 if isinstance(x, np.ndarray) and np.issubdtype(x.dtype, np.floating) else x
                 for x in self.args]
            dp = pert.pop("dparam", None)
            for name, (idx, comp) in pert.items():
                pos = {"eps": 0, "epsp": 1, "ep": 2, "abar": 3, "stiff": 6}[name]
                if comp is None:
                    a[pos] = a[pos] + 1j * CS_H
                else:
                    t = a[pos].copy()
                    if name == "abar":
                        t[comp] = t[comp] + 1j * CS_H
                    else:
                        t[:, comp] = t[:, comp] + 1j * CS_H
                    a[pos] = t
            out = local_update(*a, dparam=dp)
            self.cols[key] = tuple(np.imag(o) / CS_H for o in out)

        for c in self.comps:
            run(("eps", c), eps=(None, c))
        for c in range(6):
            run(("epsp", c), epsp=(None, c))
        run(("ep",), ep=(None, None))
        for j in range(J):
            run(("abar", j), abar=(None, j))
        for q in range(len(phases)):
            for k in PARAMS:
                run(("theta", q, k), dparam={(q, k): 1j * CS_H})
        run(("stiff",), stiff=(None, None))
        self.Vn = Vn
        self.J = J

    @staticmethod
    def _contract(col, w):
        ws, wa, wp, we = w
        ds, da, dp, de = col
        return (np.sum(ds * ws, axis=1) + np.sum(da * wa, axis=0) + np.sum(dp * wp, axis=1) + de * we)

    def vjp(self, w):
        """w = (w_sigma (V,6), w_alpha (J,V), w_epsp (V,6), w_e (V,)).
        Returns dict eps (V, nc), epsp (V, 6), ep (V,), abar (J, V),
        theta {(q, name): float}, stiff (V,)."""
        out = {"eps": np.stack([self._contract(self.cols[("eps", c)], w) for c in self.comps], axis=1),
               "epsp": np.stack([self._contract(self.cols[("epsp", c)], w) for c in range(6)], axis=1),
               "ep": self._contract(self.cols[("ep",)], w),
               "abar": np.stack([self._contract(self.cols[("abar", j)], w) for j in range(self.J)]),
               "theta": {(q, k): float(np.sum(self._contract(self.cols[("theta", q, k)], w)))
                         for q in range(len(self.phases)) for k in PARAMS},
               "stiff": self._contract(self.cols[("stiff",)], w)}
        return out


# ============================================================ gradient fields
def willot_grad(a, grid, ks=None):
    """G_d a = F^-1(k_d F a) for d = 0..dim-1 (the R5 corner derivative of a
    real field a of the grid shape); list of real fields."""
    if ks is None:
        ks = O.willot_k(grid)
    ah = O.fft_fields(a, grid)
    return [O.ifft_fields(k * ah, grid).real for k in ks]


# ================================================================ recursion
def forward_states(grid, phase_map, phase_dicts, ell, strain_ctrl, target, opt, stiff=None):
    """Run the load path, keeping for every increment n the converged
    (eps_n, abar_n) and the history h_{n-1} it started from."""
    st = O.make_state(grid, phase_map, O.phases_from_dicts(phase_dicts), ell, stiff)
    states = []
    prev = np.zeros(6)
    for t in np.asarray(target, dtype=np.float64):
        h = (st.epsp.copy(), st.ep.copy())
        O.step_increment(st, strain_ctrl, prev, t, opt)
        states.append(dict(eps=st.eps.copy(), abar=st.abar.copy(), epsp_prev=h[0], ep_prev=h[1]))
        prev = t
    return st, states


def adjoint_gradient(grid, phase_map, phase_dicts, ell, strain_ctrl, target, opt, stiff=None,
                     tol=1e-12, max_outer=200, rtol=1e-14):
    """dJ/dtheta for J = <sigma_N>_11 over the whole load path.

    Returns dict J, theta {(phase, name): value}, ell (J,) (derivative with
    respect to the own-phase length of each variable, the row scaling with
    it), stiff (V,) (per-voxel modulus factor), outer (list of the transposed
    staggered iteration counts)."""
    phases = O.phases_from_dicts(phase_dicts)
    st, states = forward_states(grid, phase_map, phase_dicts, ell, strain_ctrl, target, opt, stiff)
    d = grid.d
    comps = O.carried(d)
    nc = len(comps)
    Vn = grid.V
    sh = grid.shape
    ph = np.asarray(phase_map).reshape(Vn).astype(np.int64)
    sf = np.ones(Vn) if stiff is None else np.asarray(stiff, dtype=np.float64).reshape(Vn)
    ellA = np.asarray(ell, dtype=np.float64)
    J = ellA.shape[0]
    ctrl_c = np.asarray(strain_ctrl, dtype=np.float64)[comps]
    smask = 1.0 - ctrl_c
    ks = O.willot_k(grid)
    ell2 = [(ellA[j][ph] ** 2).reshape(sh) for j in range(J)]
    own = [float(np.max(ellA[j])) for j in range(J)]
    g_theta = {(q, k): 0.0 for q in range(len(phases)) for k in PARAMS}
    g_ell = np.zeros(J)
    g_stiff = np.zeros(Vn)
    eta_p = np.zeros((Vn, 6))
    eta_e = np.zeros(Vn)
    outer = []
    N = len(states)
    for n in range(N - 1, -1, -1):
        s_ = states[n]
        Lj = LocalJacobian(grid, s_["eps"], s_["epsp_prev"], s_["ep_prev"], s_["abar"], ph, phases, sf)
        rm = O.return_map(O.embed(s_["eps"], d), s_["epsp_prev"], s_["ep_prev"], s_["abar"], ph, phases, sf)
        Cc = rm["C"][:, comps][:, :, comps].reshape(sh + (nc, nc))
        seed = np.zeros((Vn, 6))
        if n == N - 1:
            seed[:, 0] = 1.0 / Vn
        lam = np.zeros((Vn, nc))
        mu = np.zeros((J, Vn))

        def A(x):
            return O.G_apply(np.einsum("...ij,...j->...i", Cc, x), grid, smask)

        it = 0
        while True:
            g = Lj.vjp((seed, mu, eta_p, eta_e))["eps"]
            b = O.G_apply(g.reshape(sh + (nc,)), grid, smask)
            lam_new, _ = O.cg(A, b, rtol, 20000)
            lam_new = lam_new.reshape(Vn, nc)
            ws = seed - O.embed(lam_new, d).reshape(Vn, 6)
            bj = Lj.vjp((ws, np.zeros((J, Vn)), np.zeros((Vn, 6)), np.zeros(Vn)))["abar"]
            mu_new = np.zeros((J, Vn))
            for j in range(J):
                x, _ = O.helmholtz_solve(bj[j].reshape(sh), ell2[j], grid, rtol, 20000)
                mu_new[j] = x.reshape(Vn)
            dl = np.max(np.abs(lam_new - lam)) / max(np.max(np.abs(lam_new)), 1e-300)
            dm = np.max(np.abs(mu_new - mu)) / max(np.max(np.abs(mu_new)), 1e-300)
            lam, mu = lam_new, mu_new
            it += 1
            if (dl <= tol and dm <= tol) or it >= max_outer:
                break
        outer.append(it)
        w = (seed - O.embed(lam, d).reshape(Vn, 6), mu, eta_p, eta_e)
        v = Lj.vjp(w)
        for key, val in v["theta"].items():
            g_theta[key] += val
        g_stiff += v["stiff"]
        for j in range(J):
            gm = willot_grad(mu[j].reshape(sh), grid, ks)
            ga = willot_grad(s_["abar"][j].reshape(sh), grid, ks)
            dot = sum(x * y for x, y in zip(gm, ga))
            g_ell[j] -= float(np.sum(2.0 * ell2[j] / own[j] * dot))
        eta_p, eta_e = v["epsp"], v["ep"]
    return dict(J=float(O.homogenized_stress(st)[0]), theta=g_theta, ell=g_ell, stiff=g_stiff,
                outer=outer[::-1])


def branch_signature(grid, phase_map, phase_dicts, states, stiff=None):
    """Per increment and voxel, the branch each non-smooth part of the local
    update took: plastic or elastic (f > 0), the damage ramp's side (below,
    inside, above) and, for the cracking law, history kept or replaced.  Two
    runs with equal signatures are on the same smooth piece."""
    phases = O.phases_from_dicts(phase_dicts)
    ph = np.asarray(phase_map).reshape(-1).astype(np.int64)
    Vn = ph.size
    sf = np.ones(Vn) if stiff is None else np.asarray(stiff, dtype=np.float64).reshape(Vn)
    sig = []
    for s_ in states:
        eps6 = O.embed(s_["eps"], grid.d).reshape(Vn, 6)
        code = np.zeros(Vn, dtype=np.int64)
        for q, P in enumerate(phases):
            sel = ph == q
            e = eps6[sel] - s_["epsp_prev"][sel]
            tr = e[:, 0] + e[:, 1] + e[:, 2]
            dev = e - tr[:, None] * O.IVEC[None, :] / 3.0
            c = np.zeros(int(sel.sum()), dtype=np.int64)
            if P.law == 1:
                qn = 2.0 * P.mu * sf[sel] * np.sqrt(np.sum(dev * dev, axis=1))
                c += (qn - S23 * (P.sigma_y + P.H * s_["ep_prev"][sel]) > 0.0)
            elif P.law == 2:
                c += (s_["ep_prev"][sel] >= ppn_cs(e))
            if P.law in (1, 2) and P.var >= 0:
                D = (s_["abar"][P.var][sel] - P.eps_C) / (P.eps_R - P.eps_C)
                c += 2 * (D > 0.0) + 4 * (D > P.D_max)
            code[sel] = c
        sig.append(code)
    return np.stack(sig)
