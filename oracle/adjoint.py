"""Gradient of a converged collision solve by the implicit-function theorem (oracle).

At v = 0 with y returned as q(M, y) at the converged moments, the outputs
(D, Ye, eps) of Algorithm 1 are fixed by the reduced system

    G(D; p) = D - Q_D(D, q(D; p); p) = 0                                (*)

(the number part of Eq. implicitMomentsNodal with y eliminated through
Eq. implicitFluidNodal; Q_D does not depend on I at v = 0), with
Ye = q_Ye(D; p), eps = q_eps(D; p).  p collects the step's inputs: the old
moments D*, the old state (Ye*, T*) and the four opacity scale factors.  For a
loss L = gD . D + gYe Ye + geps eps the IFT gives

    lambda = (dG/dD)^-T (gD + gYe dYe/dD + geps deps/dD)
    dL/dp  = -lambda . dG/dp + gYe dYe/dp + geps deps/dp.

Every Jacobian here is formed by central finite differences of the oracle's
own residual functions, so this gradient shares no derivative formula with the
CUDA adjoint.  The old first moments I* do not enter (*) or the outputs at
v = 0, so their gradient is zero.
"""

import numpy as np

from . import eos
from .constants import C_LIGHT, lepton_numbers
from .opacities import compute_opacities
from .solver import moment_map, matter_map, neutrino_energy_number


def _parts(grid, tables, params, rho, p, D):
    """(G(D; p), Ye(D; p), eps(D; p)) for parameters p = (D*, Ye*, T*, scale, dt)."""
    D_star, Ye_star, T_star, scale, dt = p
    ns, ne = D_star.shape
    g = lepton_numbers(ns)
    eps_star = eos.specific_energy(rho, T_star, Ye_star)
    y_star = np.array([eps_star, Ye_star])
    EN_star = neutrino_energy_number(D_star, grid, g)
    y = matter_map(D, rho, y_star, EN_star, grid, g)
    T, _ = eos.temperature(rho, y[0], y[1])
    op = compute_opacities(grid, tables, rho, T, y[1], scale, params.proc_mask, params.dmin, params.dmax)
    M = np.zeros((ns, ne, 4))
    M[:, :, 0] = D
    Ms = np.zeros((ns, ne, 4))
    Ms[:, :, 0] = D_star
    Q = moment_map(M, Ms, op, grid.W2, C_LIGHT * dt)
    return D - Q[:, :, 0], y[1], y[0]


def gradient(grid, tables, params, rho, T_star, Ye_star, D_star, dt, scale, D, gD, gYe, geps, rel=1e-6):
    """dL/d(D*, I*, Ye*, T*, scale) at the converged moments D of one node.

    Returns a dict with keys D_star (ns, ne), I_star (ns, ne, 3), Ye, T, scale (4,).
    """
    ns, ne = D.shape
    n = ns * ne
    p0 = (np.array(D_star, dtype=float), float(Ye_star), float(T_star), np.array(scale, dtype=float), float(dt))

    def G_of_D(Dv):
        return _parts(grid, tables, params, rho, p0, Dv.reshape(ns, ne))

    # dG/dD and dYe/dD, deps/dD by central differences
    J = np.empty((n, n))
    dYe = np.empty(n)
    deps = np.empty(n)
    Dv = D.ravel().astype(float)
    for j in range(n):
        h = rel * max(abs(Dv[j]), 1e-8)
        up, dn = Dv.copy(), Dv.copy()
        up[j] += h
        dn[j] -= h
        Gu, Yu, Eu = G_of_D(up)
        Gd, Yd, Ed = G_of_D(dn)
        J[:, j] = (Gu - Gd).ravel() / (2 * h)
        dYe[j] = (Yu - Yd) / (2 * h)
        deps[j] = (Eu - Ed) / (2 * h)
    rhs = np.asarray(gD, dtype=float).ravel() + gYe * dYe + geps * deps
    lam = np.linalg.solve(J.T, rhs)

    def dL_dp(perturb):
        """-lambda . dG/dp + gYe dYe/dp + geps deps/dp for one scalar parameter."""
        (pu, hu), (pd, hd) = perturb(+1), perturb(-1)
        Gu, Yu, Eu = _parts(grid, tables, params, rho, pu, D)
        Gd, Yd, Ed = _parts(grid, tables, params, rho, pd, D)
        h = hu - hd
        return (-lam @ (Gu - Gd).ravel() + gYe * (Yu - Yd) + geps * (Eu - Ed)) / h

    out_D = np.empty((ns, ne))
    for s in range(ns):
        for q in range(ne):
            def pert(sign, s=s, q=q):
                Ds = p0[0].copy()
                h = rel * max(abs(Ds[s, q]), 1e-8)
                Ds[s, q] += sign * h
                return (Ds,) + p0[1:], sign * h
            out_D[s, q] = dL_dp(pert)

    def pert_scalar(idx):
        def pert(sign):
            lst = list(p0)
            h = rel * abs(lst[idx])
            lst[idx] = lst[idx] + sign * h
            return tuple(lst), sign * h
        return pert

    g_Ye = dL_dp(pert_scalar(1))
    g_T = dL_dp(pert_scalar(2))
    g_scale = np.empty(4)
    for k in range(4):
        def pert(sign, k=k):
            sc = p0[3].copy()
            h = rel * max(abs(sc[k]), 1e-3)
            sc[k] += sign * h
            return (p0[0], p0[1], p0[2], sc, p0[4]), sign * h
        g_scale[k] = dL_dp(pert)
    return dict(D_star=out_D, I_star=np.zeros((ns, ne, 3)), Ye=g_Ye, T=g_T, scale=g_scale)
