"""Gradient of a converged collision solve by the implicit-function theorem (oracle).

Test infrastructure: only the tests and the benchmark's CPU baseline use it.

At v = 0, with y returned as q(M, y) at the converged moments, the outputs of
Algorithm 1 are fixed by the reduced system

    G(D; p) = D - Q_D(D, q(D; p); p) = 0                                (*)

(the number part of Eq. implicitMomentsNodal with y eliminated through
Eq. implicitFluidNodal; Q_D does not depend on I at v = 0).  The other outputs
are explicit functions of the root D:
  - Ye = q_Ye(D; p) and eps = q_eps(D; p), the matter update;
  - T = T(eps, Ye) by the EoS;
  - H = I* / (1 + dtau kappa(D, y)), the first-moment part of
    Eq. implicitMomentsNodal at v = 0.
p collects the step's inputs: the old moments (D*, I*), the old matter state
(Ye*, T*) and the four opacity scale factors.  With frozen matter, y = y* and
q is the identity on y*.

For a loss L = gD . D + gYe Ye + geps eps + gT T + gH . H, write
L_x(D; p) for its value at given D and O = (Ye, eps, T, H) for the explicit
outputs, g_O for their cotangents.  The IFT gives

    lambda = (dG/dD)^-T dL_x/dD,       dL/dp = dL_x/dp - lambda . dG/dp,

with dL_x/dD = gD + g_O . dO/dD and dL_x/dp = g_O . dO/dp.  G and O are
differenced as vectors and contracted afterwards, so each quotient's rounding
is relative to its own output rather than to the whole loss.

Every derivative here but one is a central finite difference of the oracle's
own functions.  The exception is the scale factors: at fixed D the matter state
does not move with them, and every rate in Eq. implicitMomentsNodal is linear in
its own factor, so Q_D = (D* + dtau eta)/(1 + dtau chi) and the first-moment
map I*/(1 + dtau kappa) are ratios of affine functions of each s_k, whose
derivatives are written out (scale_partials).  A difference quotient loses the
small derivatives of weakly coupled species (the heavy flavours' absorption) to
the rounding of Q_D, and at optically thick nodes the adjoint multiplies exactly
those entries by the large lambda of the number-conserving mode.  Differences use the fourth-order central stencil
f' = (8 (f(h) - f(-h)) - (f(2h) - f(-2h))) / (12 h).  Steps in D and D* start
at rel times the entry's natural scale s_j: the change of D_j that moves the
matter state by O(1) relative, s_j = min(1, rho eps / (MeV W3_j),
rho Ye / (m_B |g_s| W2_j)) (1 with frozen matter); a step relative to an
entry of 1e-30 would leave only rounding, and a step of 1e-6 in a bin of large
W3 would move T far enough for curvature to show.  At fixed y the map is a
ratio of functions affine in D whose denominator 1 + dtau chi can vary on a
much smaller scale in bins where dtau K W~ is large, so these steps are then
cut by 4 until two successive estimates agree element by element (to 1e-8
relative, or to their rounding).  The scale factors do not move y at fixed D,
so Q_D and H are ratios of functions affine in s_k whose nonlinearity scale is
at least s_k: their steps start at 1e-3 s_k (refined the same way), which keeps
the rounding of G, amplified by large entries of lambda, far below 1e-9.
"""

import numpy as np

from . import eos
from .constants import C_LIGHT, lepton_numbers
from .opacities import compute_opacities
from .solver import moment_map, matter_map, neutrino_energy_number, compute_rates


def _matter(grid, tables, params, rho, p, D):
    """Matter state y = q(D; p) (or y* with frozen matter), its T and the opacities there."""
    D_star, _, Ye_star, T_star, scale, dt = p
    ns = D_star.shape[0]
    g = lepton_numbers(ns)
    eps_star = eos.specific_energy(rho, T_star, Ye_star)
    y_star = np.array([eps_star, Ye_star])
    if params.frozen_matter:
        y = y_star
    else:
        EN_star = neutrino_energy_number(D_star, grid, g)
        y = matter_map(D, rho, y_star, EN_star, grid, g)
    T, _ = eos.temperature(rho, y[0], y[1])
    op = compute_opacities(grid, tables, rho, T, y[1], scale, params.proc_mask, params.dmin, params.dmax)
    return y, T, op


def _outputs(grid, tables, params, rho, p, D, state=None):
    """(G, Ye, eps, T, H) at moments D for parameters p = (D*, I*, Ye*, T*, scale, dt)."""
    D_star, I_star, _, _, _, dt = p
    y, T, op = state if state is not None else _matter(grid, tables, params, rho, p, D)
    ns, ne = D_star.shape
    M = np.zeros((ns, ne, 4))
    M[:, :, 0] = D
    Ms = np.zeros((ns, ne, 4))
    Ms[:, :, 0] = D_star
    Ms[:, :, 1:] = I_star
    Q = moment_map(M, Ms, op, grid.W2, C_LIGHT * dt)
    return D - Q[:, :, 0], y[1], y[0], T, Q[:, :, 1:]


def scale_partials(grid, tables, params, rho, p, D, state):
    """(dG/ds, dH/ds) at moments D for the four scale factors (EmAb, Iso, NES, Pair), shapes
    (4, ns, ne) and (4, ns, ne, 3), in closed form.  With unit-factor rates (eta_k, chi_k) of each
    process at D and the matter state y of `state`:
        eta = s_0 chi_EmAb D^Eq + s_2 eta_NES + s_3 eta_Pair,  chi = s_0 chi_EmAb + s_2 chi_NES + s_3 chi_Pair,
        kappa = chi + s_1 sigma_Iso,
        dQ_D/ds_k = dtau (d eta/ds_k - Q_D d chi/ds_k) / (1 + dtau chi),
        dH/ds_k = -I* dtau (d kappa/ds_k) / (1 + dtau kappa)^2,
    and G = D - Q_D."""
    D_star, I_star, _, _, scale, dt = p
    _, T, _ = state
    y = state[0]
    dtau = C_LIGHT * dt
    unit = compute_opacities(grid, tables, rho, T, y[1], np.ones(4), params.proc_mask, params.dmin, params.dmax)
    eta_n, chi_n, eta_p, chi_p = compute_rates(D, unit, grid.W2)
    ab, sg = unit["chi_ab"], unit["sig"]
    zero = np.zeros_like(D)
    deta = [ab * unit["deq"], zero, eta_n, eta_p]
    dchi = [ab, zero, chi_n, chi_p]
    dkap = [ab, sg, chi_n, chi_p]
    eta = sum(scale[k] * deta[k] for k in range(4))
    chi = sum(scale[k] * dchi[k] for k in range(4))
    kappa = chi + scale[1] * sg
    QD = (D_star + dtau * eta) / (1.0 + dtau * chi)
    dG = np.stack([-dtau * (deta[k] - QD * dchi[k]) / (1.0 + dtau * chi) for k in range(4)])
    dH = np.stack([-I_star * (dtau * dkap[k] / (1.0 + dtau * kappa) ** 2)[..., None] for k in range(4)])
    return dG, dH


def _stencil(f, h):
    """Fourth-order central difference of the vector function f(t) at t = 0."""
    return (8.0 * (f(h) - f(-h)) - (f(2.0 * h) - f(-2.0 * h))) / (12.0 * h)


def _stencil_refined(f, h, mag, levels=4):
    """_stencil with the step cut by 4 until successive estimates agree elementwise;
    mag[i] is the size of the terms that f[i] is formed from (its rounding scale)."""
    d = _stencil(f, h)
    for _ in range(levels):
        h4 = 0.25 * h
        d2 = _stencil(f, h4)
        noise = 64.0 * np.finfo(float).eps * mag / h4
        if np.all(np.abs(d2 - d) <= 1e-8 * np.abs(d2) + noise):
            return d2
        d, h = d2, h4
    return d


def natural_scale(grid, params, rho, eps, Ye, ns):
    """s[s, q]: the change of D_sq that moves (eps, Ye) by O(1) relative."""
    from .constants import MEV_TO_ERG, M_B
    s = np.ones((ns, grid.ne))
    if params.frozen_matter:
        return s
    g = np.asarray(lepton_numbers(ns), dtype=float)
    s = np.minimum(s, (rho * abs(eps) / (MEV_TO_ERG * grid.W3))[None, :])
    with np.errstate(divide="ignore"):
        sy = rho * abs(Ye) / (M_B * np.abs(g)[:, None] * grid.W2[None, :])
    return np.minimum(s, sy)


def _vec_fn(grid, tables, params, rho):
    def vec(p, Dm, state=None):
        """(G, Ye, eps, T, H) at moments Dm for parameters p, as one vector."""
        G, Ye, eps, T, H = _outputs(grid, tables, params, rho, p, Dm, state)
        return np.concatenate([G.ravel(), [Ye, eps, T], H.ravel()])
    return vec


def _jacobian(grid, tables, params, rho, p0, D, rel):
    """(dG/dD, dO/dD, rounding scale of vec's entries) at moments D, O = (Ye, eps, T, H)."""
    ns, ne = D.shape
    n = ns * ne
    vec = _vec_fn(grid, tables, params, rho)
    y, T0, _ = _matter(grid, tables, params, rho, p0, D)
    sD = natural_scale(grid, params, rho, y[0], y[1], ns).ravel()
    # rounding scale of each entry of vec: G = D - Q_D is formed from terms of size |D|
    H0 = _outputs(grid, tables, params, rho, p0, D)[4]
    mag = np.concatenate([np.abs(D).ravel(), np.abs([y[1], y[0], T0]), np.abs(H0).ravel()]) + 1e-300
    J = np.empty((n, n))
    dO = np.empty((mag.size - n, n))
    Dv = D.ravel()
    for j in range(n):
        def f(t, j=j):
            Dp = Dv.copy()
            Dp[j] += t
            return vec(p0, Dp.reshape(ns, ne))
        d = _stencil_refined(f, rel * sD[j], mag)
        J[:, j] = d[:n]
        dO[:, j] = d[n:]
    return J, dO, mag


def condition_number(grid, tables, params, rho, T_star, Ye_star, D_star, I_star, dt, scale, D, rel=1e-5):
    """2-norm condition number of dG/dD at the converged moments D of one node."""
    p0 = (np.array(D_star, dtype=float), np.array(I_star, dtype=float), float(Ye_star), float(T_star),
          np.array(scale, dtype=float), float(dt))
    J, _, _ = _jacobian(grid, tables, params, rho, p0, np.asarray(D, dtype=float), rel)
    return float(np.linalg.cond(J))


def gradient(grid, tables, params, rho, T_star, Ye_star, D_star, I_star, dt, scale, D,
             gD=None, gYe=0.0, geps=0.0, gT=0.0, gH=None, rel=1e-5):
    """dL/d(D*, I*, Ye*, T*, scale) at the converged moments D of one node.

    Returns a dict with keys D_star (ns, ne), I_star (ns, ne, 3), Ye, T, scale (4,),
    and two diagnostics of how well the gradient is determined: cond, the
    2-norm condition number of dG/dD, and mag, for every entry the sum of the
    absolute terms it is formed from (|g_O| . |dO/dp| + |lambda| . |dG/dp|).
    An error e in the converged D moves an entry by about cond * |e| * mag.
    """
    ns, ne = D.shape
    n = ns * ne
    gD = np.zeros((ns, ne)) if gD is None else np.asarray(gD, dtype=float)
    gH = np.zeros((ns, ne, 3)) if gH is None else np.asarray(gH, dtype=float)
    p0 = (np.array(D_star, dtype=float), np.array(I_star, dtype=float), float(Ye_star), float(T_star),
          np.array(scale, dtype=float), float(dt))
    D = np.asarray(D, dtype=float)

    gO = np.concatenate([[gYe, geps, gT], gH.ravel()])

    vec = _vec_fn(grid, tables, params, rho)
    J, dO, mag = _jacobian(grid, tables, params, rho, p0, D, rel)
    dLx = gD.ravel() + gO @ dO
    lam = np.linalg.solve(J.T, dLx)

    def dL_dp(make, h, state=None, refine=False):
        """(dL_x/dp - lambda . dG/dp, sum of |terms|) for one scalar parameter;
        make(t) returns p with that parameter + t."""
        fp = lambda t: vec(make(t), D, state)  # noqa: E731
        d = _stencil_refined(fp, h, mag) if refine else _stencil(fp, h)
        return gO @ d[n:] - lam @ d[:n], np.abs(gO) @ np.abs(d[n:]) + np.abs(lam) @ np.abs(d[:n])

    def set_entry(idx, index):
        def make(t):
            lst = list(p0)
            if index is None:
                lst[idx] = lst[idx] + t
            else:
                a = lst[idx].copy()
                a[index] += t
                lst[idx] = a
            return tuple(lst)
        return make

    ys = (eos.specific_energy(rho, p0[3], p0[2]), p0[2])
    sDs = natural_scale(grid, params, rho, ys[0], ys[1], ns)
    out, amag = {}, {}
    out["D_star"], amag["D_star"] = np.empty((ns, ne)), np.empty((ns, ne))
    for s in range(ns):
        for q in range(ne):
            out["D_star"][s, q], amag["D_star"][s, q] = dL_dp(set_entry(0, (s, q)), rel * sDs[s, q], refine=True)
    # I* enters neither q nor the opacities: the matter state at D is shared by its perturbations,
    # and G and the outputs are linear in I*
    state = _matter(grid, tables, params, rho, p0, D)
    hI = rel * max(np.max(np.abs(p0[1])), 1e-300)
    out["I_star"], amag["I_star"] = np.empty((ns, ne, 3)), np.empty((ns, ne, 3))
    for s in range(ns):
        for q in range(ne):
            for c in range(3):
                out["I_star"][s, q, c], amag["I_star"][s, q, c] = dL_dp(set_entry(1, (s, q, c)), hI, state)
    out["Ye"], amag["Ye"] = dL_dp(set_entry(2, None), rel * abs(p0[2]))
    out["T"], amag["T"] = dL_dp(set_entry(3, None), rel * abs(p0[3]))
    out["scale"], amag["scale"] = np.empty(4), np.empty(4)
    dGs, dHs = scale_partials(grid, tables, params, rho, p0, D, state)
    for k in range(4):
        t_g, t_h = lam @ dGs[k].ravel(), gH.ravel() @ dHs[k].ravel()
        out["scale"][k] = t_h - t_g
        amag["scale"][k] = np.abs(gH.ravel()) @ np.abs(dHs[k].ravel()) + np.abs(lam) @ np.abs(dGs[k].ravel())
    out["cond"] = float(np.linalg.cond(J))
    out["mag"] = amag
    return out
