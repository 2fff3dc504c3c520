"""O(v/c) collision solve (oracle): Algorithm 1 with the velocity-dependent terms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.5 with v != 0, step by step:

* closure: Minerbo's Eddington factor psi(h) (Eq. eddingtonFactorMinerbo) in the
  Eddington tensor k_ij (Eq. eddingtonTensor), K_ij = k_ij D, with flux factor
  h = |I| / D and unit vector n = I / |I|;
* conserved moments of the old state (Eq. conservedToPrimitive):
  N* = D* + v*^i I*_i and G*_j = I*_j + v*^i K_ij(M*);
* moment map Q: Eq. implicitMomentsNodal with lambda = 1 / (1 + |v|) (the
  remark on the step-size parameter), v the velocity of the current matter
  iterate;
* matter map q: Eq. implicitFluidNodal with the Eulerian momentum, energy and
  number densities (Eqs. eulerianMomentumLG, eulerianEnergyLG,
  eulerianNumberLG); the specific internal energy is eps = eps_f - v^2 / 2.

Readings (each also listed in the design notes):

* flat metric at the node, gamma_ij = delta_ij (Cartesian components); v in
  units of c and |v| its Euclidean norm;
* the number density's flux term is v^i I_i (the index printed on I in
  Eq. eulerianNumberLG is garbled);
* units: v_j = v*_j - (F_j - F*_j) MeV / (rho c^2) and eps_f = eps + v^2 c^2 / 2
  in erg/g; the energy and lepton-number updates are those of the v = 0 solve;
* h is clipped to [0, 1], and where |I| = 0 the tensor is delta_ij / 3
  (psi(0) = 1/3, so n drops out);
* Algorithm 3 compares each velocity component's change with tol times
  max(|v*|, v_floor) (a component-wise |v*_j| is zero along any axis the fluid
  does not move on); the outer residual is scaled the same way;
* the returned matter state extends the v = 0 reading y_out = q(M_out): the
  velocity solves v = v* - (F(M_out, v) - F*) MeV / (rho c^2), which is linear
  in v (a 3 x 3 solve), and eps_f and Ye follow with that v, so momentum,
  energy and lepton number are conserved to rounding;
* freeze_velocity keeps v = v* (the first three components of q's right-hand
  side set to zero, as in the deleptonization setup of Sec. 6); with v* = 0 it
  is the v = 0 solve.
"""

import math
import numpy as np

from . import eos
from .constants import C_LIGHT, M_B, MEV_TO_ERG, lepton_numbers
from .opacities import compute_opacities
from .solver import (compute_rates, anderson_weights, check_inner, species_norms,
                     NOT_CONVERGED_INNER, NOT_CONVERGED_OUTER, NONFINITE, EOS_FAIL, TABLE_CLAMP)

C2 = C_LIGHT * C_LIGHT


def eddington_factor(h):
    """Minerbo's Eddington factor, Eq. eddingtonFactorMinerbo."""
    return 1.0 / 3.0 + (2.0 / 15.0) * (3.0 - h + 3.0 * h * h) * h * h


def eddington_tensor(D, I):
    """k_ij of Eq. eddingtonTensor for number moments D (...) and fluxes I (..., 3): (..., 3, 3)."""
    D = np.asarray(D, dtype=float)
    I = np.asarray(I, dtype=float)
    In = np.sqrt(np.sum(I * I, axis=-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        h = np.where(D > 0.0, In / np.where(D > 0.0, D, 1.0), 0.0)
        n = np.where(In[..., None] > 0.0, I / np.where(In > 0.0, In, 1.0)[..., None], 0.0)
    h = np.clip(h, 0.0, 1.0)
    psi = eddington_factor(h)
    eye = np.eye(3)
    return 0.5 * ((1.0 - psi)[..., None, None] * eye
                  + (3.0 * psi - 1.0)[..., None, None] * n[..., :, None] * n[..., None, :])


def rank2(M):
    """K_ij = k_ij D for moments M (..., 4)."""
    return eddington_tensor(M[..., 0], M[..., 1:]) * M[..., 0][..., None, None]


def conserved(M, v):
    """(N, G) = A(M, v) M of Eq. conservedToPrimitive: N = D + v^i I_i, G_j = I_j + v^i K_ij."""
    v = np.asarray(v, dtype=float)
    N = M[..., 0] + M[..., 1:] @ v
    G = M[..., 1:] + np.einsum("i,...ij->...j", v, rank2(M))
    return N, G


def moment_map(M, U_star, op, W2, dtau, v):
    """Q(M, y) of Eq. implicitMomentsNodal for M (ns, ne, 4), old conserved moments U_star = (N*, G*)."""
    v = np.asarray(v, dtype=float)
    D, I = M[:, :, 0], M[:, :, 1:]
    eta_nes, chi_nes, eta_pair, chi_pair = compute_rates(D, op, W2)
    eta = op["chi_ab"] * op["deq"] + eta_nes + eta_pair      # Eqs. emissivityNodal, emissivityEmAbNodal
    chi = op["chi_ab"] + chi_nes + chi_pair                  # Eq. opacityNodal
    kappa = chi + op["sig"]                                  # Eq. transportOpacityNodal
    lam = 1.0 / (1.0 + math.sqrt(float(v @ v)))
    N_star, G_star = U_star
    cD, cI = linear_corrections(M, op, W2) if "phi1_in" in op else (0.0, 0.0)
    Q = np.empty_like(M)
    Q[:, :, 0] = ((1.0 - lam) * D + lam * (N_star - I @ v + dtau * (eta + cD))) / (1.0 + lam * dtau * chi)
    vK = np.einsum("i,...ij->...j", v, rank2(M))
    Q[:, :, 1:] = ((1.0 - lam) * I + lam * (G_star - vK + dtau * cI)) / (1.0 + lam * dtau * kappa)[:, :, None]
    return Q


def linear_corrections(M, op, W2):
    """Linear-order NES and pair terms of the moment equations (Eqs. zerothMomentCollisionTerm_NES,
    firstMomentCollisionTerm_NES, zerothMomentCollisionTerm_Pair, firstMomentCollisionTerm_Pair) with
    <Phi_1 I> of Eqs. linearCorrectionsNES and linearCorrectionsPair by the energy quadrature:
        number: -(A_in - A_out).I + (P_pro - P_ann).I
        flux_j: (1/3)(gamma_ij - 3 K_ij) A_in^i + K_ij A_out^i
                - (1/3)(gamma_ij - 3 K_ij) P_pro^i - K_ij P_ann^i,
    A = <Phi_1^{In/Out} I_s>, P = <Phi_1^{Pro/Ann} I_sbar>, K = k D.  Returns (cD (ns, ne), cI (ns, ne, 3)).
    Reading: they enter Eq. implicitMomentsNodal as explicit additions to dtau eta and to the flux
    numerator, evaluated at the current iterate."""
    D, I = M[:, :, 0], M[:, :, 1:]
    ns = D.shape[0]
    K = rank2(M)
    cD = np.zeros_like(D)
    cI = np.zeros_like(I)
    for s in range(ns):
        sb = s ^ 1
        wI, wIb = W2[:, None] * I[s], W2[:, None] * I[sb]
        A_in, A_out = op["phi1_in"][s] @ wI, op["phi1_out"][s] @ wI
        P_pro, P_ann = op["phi1_pro"][s] @ wIb, op["phi1_ann"][s] @ wIb
        cD[s] = -np.sum((A_in - A_out) * I[s], axis=-1) + np.sum((P_pro - P_ann) * I[s], axis=-1)
        KA = lambda A: np.einsum("qij,qi->qj", K[s], A)  # noqa: E731
        cI[s] = (A_in / 3.0 - KA(A_in)) + KA(A_out) - (P_pro / 3.0 - KA(P_pro)) - KA(P_ann)
    return cD, cI


def eulerian_sums(M, v, grid, g):
    """(F_nu[3], E_nu, N_nu) of Eqs. eulerianMomentumLG, eulerianEnergyLG, eulerianNumberLG (MeV cm^-3, cm^-3)."""
    v = np.asarray(v, dtype=float)
    D, I = M[:, :, 0], M[:, :, 1:]
    W2, W3 = grid.W2[None, :], grid.W3[None, :]
    F = np.sum(W3[:, :, None] * (I + D[:, :, None] * v + np.einsum("k,...jk->...j", v, rank2(M))), axis=(0, 1))
    E = float(np.sum(W3 * (D + 2.0 * (I @ v))))
    N = float(np.sum(np.asarray(g)[:, None] * W2 * (D + I @ v)))
    return F, E, N


def matter_map(M, y, rho, y_star, S_star, grid, g, freeze_velocity=False):
    """q(M, y) of Eq. implicitFluidNodal: y = (v_1, v_2, v_3, eps_f [erg/g], Ye)."""
    F, E, N = eulerian_sums(M, y[:3], grid, g)
    F_s, E_s, N_s = S_star
    v = y_star[:3].copy() if freeze_velocity else y_star[:3] - (F - F_s) * MEV_TO_ERG / (rho * C2)
    eps_f = y_star[3] - (E - E_s) * MEV_TO_ERG / rho
    Ye = y_star[4] - M_B * (N - N_s) / rho
    return np.concatenate([v, [eps_f, Ye]])


def final_matter_state(M, rho, y_star, S_star, grid, g, freeze_velocity=False):
    """y_out with v = v* - (F(M, v) - F*) MeV/(rho c^2) solved exactly (F is affine in v), then eps_f, Ye."""
    if freeze_velocity:
        v = y_star[:3].copy()
    else:
        D, I = M[:, :, 0], M[:, :, 1:]
        W3 = grid.W3[None, :]
        cf = MEV_TO_ERG / (rho * C2)
        F0 = np.sum(W3[:, :, None] * I, axis=(0, 1))
        B = np.sum(W3[:, :, None, None] * (D[:, :, None, None] * np.eye(3) + rank2(M)), axis=(0, 1))
        v = np.linalg.solve(np.eye(3) + cf * B, y_star[:3] - cf * (F0 - S_star[0]))
    _, E, N = eulerian_sums(M, v, grid, g)
    eps_f = y_star[3] - (E - S_star[1]) * MEV_TO_ERG / rho
    Ye = y_star[4] - M_B * (N - S_star[2]) / rho
    return np.concatenate([v, [eps_f, Ye]])


def internal_energy(y):
    """eps = eps_f - v^2 c^2 / 2 (erg/g)."""
    return y[3] - 0.5 * float(y[:3] @ y[:3]) * C2


def scales(y_star, v_floor):
    """Per-component reference of Algorithm 3 and of the outer residual."""
    vs = max(math.sqrt(float(y_star[:3] @ y_star[:3])), v_floor)
    return np.array([vs, vs, vs, abs(y_star[3]), abs(y_star[4])])


def solve_node(grid, tables, params, rho, T_star, Ye_star, v_star, D_star, I_star, dt, scale=(1, 1, 1, 1),
               freeze_velocity=False, v_floor=1e-6):
    """SolveNeutrinoMatterCoupling (Algorithm 1) with O(v/c) terms for one spatial node.

    v_star: (3,) in units of c.  Returns D, I, v, eps (internal), eps_f, Ye, T, n_outer, n_inner, status.
    """
    p = params
    ns = D_star.shape[0]
    g = lepton_numbers(ns)
    dtau = C_LIGHT * dt
    status = 0
    v_star = np.asarray(v_star, dtype=float)
    eps_star = eos.specific_energy(rho, T_star, Ye_star)
    y_star = np.array([v_star[0], v_star[1], v_star[2], eps_star + 0.5 * float(v_star @ v_star) * C2, Ye_star])
    M_star = np.concatenate([D_star[:, :, None], I_star], axis=2).astype(np.float64)
    U_star = conserved(M_star, v_star)
    S_star = eulerian_sums(M_star, v_star, grid, g)
    sc_y = scales(y_star, v_floor)

    y = y_star.copy()
    M = M_star.copy()
    T = T_star
    op = compute_opacities(grid, tables, rho, T, y[4], scale, p.proc_mask, p.dmin, p.dmax)
    if op["clamped"]:
        status |= TABLE_CLAMP
    q_hist, f_hist = [], []
    n_inner = 0
    k = 0
    outer_converged = False
    while not outer_converged:
        k += 1
        if k > 1 and not p.semi_implicit:   # semi-implicit: opacities at y* only
            op = compute_opacities(grid, tables, rho, T, y[4], scale, p.proc_mask, p.dmin, p.dmax)
            if op["clamped"]:
                status |= TABLE_CLAMP
        D_norm = species_norms(M[:, :, 0], grid.W2, p.norm_floor)
        Qh, Fh = [], []
        inner_converged = False
        ell = 0
        while not inner_converged:
            ell += 1
            n_inner += 1
            Qv = moment_map(M, U_star, op, grid.W2, dtau, y[:3])
            Qh.append(Qv)
            Fh.append(Qv - M)
            Qh, Fh = Qh[-p.M_inner:], Fh[-p.M_inner:]
            alpha = anderson_weights(Fh)
            M_new = sum(a * Qj for a, Qj in zip(alpha, Qh))
            inner_converged = check_inner(M_new - M, D_norm, grid.W2, p.tol_inner, p.norm_floor)
            M = M_new
            if not np.all(np.isfinite(M)):
                status |= NONFINITE
                break
            if not inner_converged and ell >= p.max_inner:
                status |= NOT_CONVERGED_INNER
                break
        if p.frozen_matter or status & (NOT_CONVERGED_INNER | NONFINITE):
            break
        qv = matter_map(M, y, rho, y_star, S_star, grid, g, freeze_velocity)
        q_hist.append(qv)
        f_hist.append((qv - y) / sc_y)
        q_hist, f_hist = q_hist[-p.M_outer:], f_hist[-p.M_outer:]
        beta = anderson_weights(f_hist)
        y_new = sum(b * qj for b, qj in zip(beta, q_hist))
        outer_converged = bool(np.all(np.abs(y_new - y) <= p.tol_outer * sc_y))   # Algorithm 3
        y = y_new
        if not np.all(np.isfinite(y)):
            status |= NONFINITE
            break
        if not outer_converged and k >= p.max_outer:
            status |= NOT_CONVERGED_OUTER
            break
        if not outer_converged:
            T_new, ok = eos.temperature(rho, internal_energy(y), y[4])
            if not ok:
                status |= EOS_FAIL
                break
            T = T_new

    if p.frozen_matter:
        y_out, T_out = y_star.copy(), T_star
    elif status & NONFINITE:
        y_out, T_out = y, T
    else:
        y_out = final_matter_state(M, rho, y_star, S_star, grid, g, freeze_velocity) if p.final_q else y
        T_out, ok = eos.temperature(rho, internal_energy(y_out), y_out[4])
        if not ok:
            status |= EOS_FAIL
            T_out = T
    return dict(D=M[:, :, 0].copy(), I=M[:, :, 1:].copy(), v=y_out[:3].copy(), eps=internal_energy(y_out),
                eps_f=float(y_out[3]), Ye=float(y_out[4]), T=float(T_out), n_outer=k, n_inner=n_inner,
                status=status)


def solve(grid, tables, params, inputs, nodes=None, **kw):
    """solve_node over a batch (inputs as for the v = 0 solve plus "v" of shape (N, 3))."""
    N = len(inputs["rho"])
    idx = range(N) if nodes is None else nodes
    res = []
    for n in idx:
        sc = inputs["scale"][n] if inputs.get("scale") is not None else (1.0, 1.0, 1.0, 1.0)
        res.append(solve_node(grid, tables, params, float(inputs["rho"][n]), float(inputs["T"][n]),
                              float(inputs["Ye"][n]), inputs["v"][n], inputs["D"][n], inputs["I"][n],
                              float(inputs["dt"][n]), sc, **kw))
    return res


# ---------------------------------------------------------------------------
# Independent root solve for tiny nodes: damped Newton on R_M = M - Q(M, y),
# R_y = (y - q(M, y)) / scales (Eqs. implicitMomentsNodalFull, implicitFluidNodal).
# ---------------------------------------------------------------------------

def _residual(x, ctx):
    grid, tables, p, rho, U_star, y_star, S_star, g, dtau, scale, sc_y, freeze = ctx
    ns, ne = U_star[0].shape
    nm = ns * ne * 4
    M = x[:nm].reshape(ns, ne, 4)
    y = x[nm:] * sc_y
    T, _ = eos.temperature(rho, internal_energy(y), y[4])
    op = compute_opacities(grid, tables, rho, T, y[4], scale, p.proc_mask, p.dmin, p.dmax)
    RM = M - moment_map(M, U_star, op, grid.W2, dtau, y[:3])
    Ry = (y - matter_map(M, y, rho, y_star, S_star, grid, g, freeze)) / sc_y
    return np.concatenate([RM.ravel(), Ry])


def newton_solve_node(grid, tables, params, rho, T_star, Ye_star, v_star, D_star, I_star, dt,
                      scale=(1, 1, 1, 1), freeze_velocity=False, v_floor=1e-6, max_iter=50, tol=1e-14):
    """Damped Newton with a central-difference Jacobian on the coupled O(v/c) residual."""
    ns, ne = D_star.shape
    g = lepton_numbers(ns)
    dtau = C_LIGHT * dt
    v_star = np.asarray(v_star, dtype=float)
    eps_star = eos.specific_energy(rho, T_star, Ye_star)
    y_star = np.array([v_star[0], v_star[1], v_star[2], eps_star + 0.5 * float(v_star @ v_star) * C2, Ye_star])
    M_star = np.concatenate([D_star[:, :, None], I_star], axis=2).astype(np.float64)
    U_star = conserved(M_star, v_star)
    S_star = eulerian_sums(M_star, v_star, grid, g)
    sc_y = scales(y_star, v_floor)
    ctx = (grid, tables, params, rho, U_star, y_star, S_star, g, dtau, scale, sc_y, freeze_velocity)
    x = np.concatenate([M_star.ravel(), y_star / sc_y])
    r = _residual(x, ctx)
    for _ in range(max_iter):
        n = x.size
        J = np.empty((n, n))
        for j in range(n):
            h = 1e-7 * max(abs(x[j]), 1e-12)
            xp, xm = x.copy(), x.copy()
            xp[j] += h
            xm[j] -= h
            J[:, j] = (_residual(xp, ctx) - _residual(xm, ctx)) / (2 * h)
        dx = np.linalg.solve(J, -r)
        t = 1.0
        while True:
            xn = x + t * dx
            rn = _residual(xn, ctx)
            if np.linalg.norm(rn) < np.linalg.norm(r) or t < 1e-4:
                break
            t *= 0.5
        x, r = xn, rn
        if np.linalg.norm(dx) <= tol * max(1.0, np.linalg.norm(x)):
            break
    nm = ns * ne * 4
    M = x[:nm].reshape(ns, ne, 4)
    y = x[nm:] * sc_y
    return dict(D=M[:, :, 0], I=M[:, :, 1:], v=y[:3], eps_f=float(y[3]), Ye=float(y[4]),
                residual=float(np.linalg.norm(r)))
