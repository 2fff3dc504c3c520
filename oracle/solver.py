"""Nested fixed-point solve of the implicit neutrino--matter coupling (oracle).

Follows Sec. 3.5 step by step:

* rates: Eqs. nesRatesNodal and pairRatesNodal (dense mat-vecs with W2);
* totals: Eqs. emissivityNodal, opacityNodal, transportOpacityNodal,
  emissivityEmAbNodal;
* moment map Q: Eq. implicitMomentsNodal with v = 0, so lambda = 1/(1+|v|) = 1;
* matter map q: Eq. implicitFluidNodal with Eqs. eulerianEnergyLG and
  eulerianNumberLG (v = 0, velocity frozen as in the deleptonization setup);
* Anderson least squares of Algorithm 1 (inner and outer loops);
* CheckConvergence_Inner (Algorithm 2) and CheckConvergence_Outer (Algorithm 3);
* SolveNeutrinoMatterCoupling (Algorithm 1).

Readings of points the paper leaves open (each also listed in the design notes):
* the InnerConverged flag is reset at the start of every outer iteration
  (otherwise no inner iteration would run after the first outer one);
* Algorithm 2's norm: per species, the W2-weighted sum of squares of the
  change is formed separately for D, I^1, I^2, I^3, the largest is taken and
  its square root compared with tol * ||D_s^[k,1]||_W2, where the reference
  norm is floored at norm_floor * sqrt(sum_q W2_q);
* the inner least-squares norm is the plain Euclidean norm over all moments
  of all species; the outer residual is scaled component-wise by |y*|
  because eps and Ye differ by many orders of magnitude;
* the constrained least-squares problem is solved by eliminating the
  constraint (alpha_M = 1 - sum of the others) and calling numpy's lstsq;
* an inner loop that reaches max_inner without converging ends the node
  before its matter update (NOT_CONVERGED_INNER), so a node that does not
  converge costs at most one capped inner loop more than one that does;
* an outer iterate outside the EoS domain (Ye not in (0, 1), or eps outside
  the range of the EoS at that Ye) sets EOS_FAIL and stops the outer loop; the
  returned temperature is then the last one inside the domain;
* semi_implicit=True skips ComputeOpacities after the first outer iteration,
  so every opacity (chi_EmAb, sigma_Iso, D^Eq and the NES and pair kernels)
  stays at the old state y* (the semi-implicit variant of Sec. 3.5); the outer
  loop still iterates y, whose temperature is then used only for the output;
* after outer convergence the returned matter state is q(M, y) evaluated at
  the converged moments, so lepton number and energy are conserved to
  rounding (final_q=True); final_q=False returns the Anderson-mixed iterate
  exactly as Algorithm 1 prints it.
"""

import math
import numpy as np

from . import eos
from .constants import C_LIGHT, M_B, MEV_TO_ERG, lepton_numbers
from .opacities import compute_opacities, EMAB, ISO, NES, PAIR

NOT_CONVERGED_INNER = 1
NOT_CONVERGED_OUTER = 2
NONFINITE = 4
EOS_FAIL = 8
TABLE_CLAMP = 16

ALL_PROCESSES = EMAB | ISO | NES | PAIR


class Params:
    def __init__(self, tol_inner=1e-10, tol_outer=1e-10, M_inner=3, M_outer=3,
                 max_inner=500, max_outer=100, dmin=1e-30, dmax=1.0 - 1e-6,
                 norm_floor=1e-30, proc_mask=ALL_PROCESSES, frozen_matter=False,
                 final_q=True, semi_implicit=False):
        self.tol_inner = tol_inner
        self.tol_outer = tol_outer
        self.M_inner = M_inner
        self.M_outer = M_outer
        self.max_inner = max_inner
        self.max_outer = max_outer
        self.dmin = dmin
        self.dmax = dmax
        self.norm_floor = norm_floor
        self.proc_mask = proc_mask
        self.frozen_matter = frozen_matter
        self.final_q = final_q
        self.semi_implicit = semi_implicit


def compute_rates(D, op, W2):
    """NES and pair emissivities/opacities for moments D[s, q] (Eqs. nesRatesNodal, pairRatesNodal)."""
    ns, ne = D.shape
    eta_nes = np.zeros((ns, ne))
    chi_nes = np.zeros((ns, ne))
    eta_pair = np.zeros((ns, ne))
    chi_pair = np.zeros((ns, ne))
    for s in range(ns):
        sb = s ^ 1
        eta_nes[s] = op["phi_in"][s] @ (W2 * D[s])
        chi_nes[s] = eta_nes[s] + op["phi_out"][s] @ (W2 * (1.0 - D[s]))
        eta_pair[s] = op["phi_pro"][s] @ (W2 * (1.0 - D[sb]))
        chi_pair[s] = eta_pair[s] + op["phi_ann"][s] @ (W2 * D[sb])
    return eta_nes, chi_nes, eta_pair, chi_pair


def moment_map(M, M_star, op, W2, dtau):
    """Q(M, y) of Eq. implicitMomentsNodal at v = 0; M has shape (ns, ne, 4)."""
    D = M[:, :, 0]
    eta_nes, chi_nes, eta_pair, chi_pair = compute_rates(D, op, W2)
    eta = op["chi_ab"] * op["deq"] + eta_nes + eta_pair      # Eqs. emissivityNodal, emissivityEmAbNodal
    chi = op["chi_ab"] + chi_nes + chi_pair                  # Eq. opacityNodal
    kappa = chi + op["sig"]                                  # Eq. transportOpacityNodal
    v_abs = 0.0
    lam = 1.0 / (1.0 + v_abs)
    Q = np.empty_like(M)
    # number equation: N* = D* + v^i I_i = D* at v = 0
    Q[:, :, 0] = ((1.0 - lam) * D + lam * (M_star[:, :, 0] + dtau * eta)) / (1.0 + lam * dtau * chi)
    # number-flux equation: G*_j = I*_j + v^i K_ij = I*_j at v = 0
    for j in range(3):
        Q[:, :, 1 + j] = ((1.0 - lam) * M[:, :, 1 + j] + lam * M_star[:, :, 1 + j]) / (1.0 + lam * dtau * kappa)
    return Q


def neutrino_energy_number(D, grid, g):
    """E_nu (MeV cm^-3) and N_nu (cm^-3) at v = 0 (Eqs. eulerianEnergyLG, eulerianNumberLG)."""
    E = float(np.sum(grid.W3[None, :] * D))
    N = float(np.sum(np.asarray(g)[:, None] * grid.W2[None, :] * D))
    return E, N


def matter_map(D, rho, y_star, EN_star, grid, g):
    """q(M, y) of Eq. implicitFluidNodal at v = 0: returns (eps, Ye)."""
    E, N = neutrino_energy_number(D, grid, g)
    eps = y_star[0] - (E - EN_star[0]) * MEV_TO_ERG / rho
    Ye = y_star[1] - M_B * (N - EN_star[1]) / rho
    return np.array([eps, Ye])


def anderson_weights(F):
    """alpha minimising 0.5 ||sum_j alpha_j F_j||^2 subject to sum_j alpha_j = 1.

    F is a list of residual vectors, oldest first.  With alpha_m = 1 - sum of
    the others the problem is min || F_m + sum_{j<m} alpha_j (F_j - F_m) ||.
    """
    m = len(F)
    if m == 1:
        return np.array([1.0])
    Fm = F[-1].ravel()
    A = np.stack([F[j].ravel() - Fm for j in range(m - 1)], axis=1)
    gamma, *_ = np.linalg.lstsq(A, -Fm, rcond=None)
    return np.concatenate([gamma, [1.0 - np.sum(gamma)]])


def check_inner(dM, D_norm, W2, tol, floor):
    """CheckConvergence_Inner (Algorithm 2) for a change dM of shape (ns, ne, 4)."""
    ns = dM.shape[0]
    for s in range(ns):
        per_moment = np.sum(W2[:, None] * dM[s] ** 2, axis=0)
        dnorm = math.sqrt(float(np.max(per_moment)))
        if not dnorm <= tol * D_norm[s]:
            return False
    return True


def check_outer(dy, y_star, tol):
    """CheckConvergence_Outer (Algorithm 3)."""
    return bool(np.all(np.abs(dy) <= tol * np.abs(y_star)))


def species_norms(D, W2, floor):
    """||D_s||_W2 = sqrt(sum_q W2_q D_sq^2), floored at floor * sqrt(sum W2)."""
    fl = floor * math.sqrt(float(np.sum(W2)))
    return np.maximum(np.sqrt(np.sum(W2[None, :] * D ** 2, axis=1)), fl)


def solve_node(grid, tables, params, rho, T_star, Ye_star, D_star, I_star, dt, scale=(1, 1, 1, 1)):
    """SolveNeutrinoMatterCoupling (Algorithm 1) for one spatial node.

    D_star: (ns, ne); I_star: (ns, ne, 3); dt in s (dtau = c dt).
    Returns a dict with D, I, Ye, eps, T, n_outer, n_inner, status.
    """
    p = params
    ns = D_star.shape[0]
    g = lepton_numbers(ns)
    dtau = C_LIGHT * dt
    status = 0
    eps_star = eos.specific_energy(rho, T_star, Ye_star)
    y_star = np.array([eps_star, Ye_star])
    M_star = np.concatenate([D_star[:, :, None], I_star], axis=2).astype(np.float64)
    EN_star = neutrino_energy_number(M_star[:, :, 0], grid, g)

    y = y_star.copy()                       # y^[1] <- y*
    M = M_star.copy()                       # M^[1,1] <- M*
    T = T_star
    op = compute_opacities(grid, tables, rho, T, y[1], scale, p.proc_mask, p.dmin, p.dmax)
    if op["clamped"]:
        status |= TABLE_CLAMP
    q_hist, f_hist = [], []
    n_inner = 0
    k = 0
    outer_converged = False
    while not outer_converged:
        k += 1
        if k > 1 and not p.semi_implicit:
            op = compute_opacities(grid, tables, rho, T, y[1], scale, p.proc_mask, p.dmin, p.dmax)
            if op["clamped"]:
                status |= TABLE_CLAMP
        D_norm = species_norms(M[:, :, 0], grid.W2, p.norm_floor)   # ||D^[k,1]||
        Qh, Fh = [], []
        inner_converged = False
        ell = 0
        while not inner_converged:
            ell += 1
            n_inner += 1
            Qv = moment_map(M, M_star, op, grid.W2, dtau)
            F = Qv - M
            Qh.append(Qv)
            Fh.append(F)
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
        if p.frozen_matter:
            break
        if status & (NOT_CONVERGED_INNER | NONFINITE):
            # reading: an inner loop stopped at its cap (or a non-finite moment)
            # ends the node before its matter update
            break
        qv = matter_map(M[:, :, 0], rho, y_star, EN_star, grid, g)
        f = (qv - y) / np.abs(y_star)
        q_hist.append(qv)
        f_hist.append(f)
        q_hist, f_hist = q_hist[-p.M_outer:], f_hist[-p.M_outer:]
        beta = anderson_weights(f_hist)
        y_new = sum(b * qj for b, qj in zip(beta, q_hist))
        outer_converged = check_outer(y_new - y, y_star, p.tol_outer)
        y = y_new
        if not np.all(np.isfinite(y)):
            status |= NONFINITE
            break
        if not outer_converged and k >= p.max_outer:
            status |= NOT_CONVERGED_OUTER
            break
        if not outer_converged:
            # reading: an outer iterate outside the EoS domain stops the node
            T_new, ok = eos.temperature(rho, y[0], y[1])
            if not ok:
                status |= EOS_FAIL
                break
            T = T_new

    if p.frozen_matter:
        y_out, T_out = y_star.copy(), T_star
    elif status & NONFINITE:
        y_out = y                  # last matter iterate; T is its temperature
        T_out = T
    else:
        y_out = matter_map(M[:, :, 0], rho, y_star, EN_star, grid, g) if p.final_q else y
        T_out, ok = eos.temperature(rho, y_out[0], y_out[1])
        if not ok:
            status |= EOS_FAIL
            T_out = T          # last temperature inside the EoS domain
    return dict(D=M[:, :, 0].copy(), I=M[:, :, 1:].copy(), eps=float(y_out[0]), Ye=float(y_out[1]),
                T=float(T_out), n_outer=k, n_inner=n_inner, status=status)


def solve(grid, tables, params, inputs, nodes=None):
    """Algorithm 1 node by node over a batch of inputs (dict of arrays)."""
    N = len(inputs["rho"])
    idx = range(N) if nodes is None else nodes
    res = []
    for n in idx:
        sc = inputs["scale"][n] if inputs.get("scale") is not None else (1.0, 1.0, 1.0, 1.0)
        res.append(solve_node(grid, tables, params, float(inputs["rho"][n]), float(inputs["T"][n]),
                              float(inputs["Ye"][n]), inputs["D"][n], inputs["I"][n],
                              float(inputs["dt"][n]), sc))
    return res


# ---------------------------------------------------------------------------
# Independent root solve for tiny nodes: damped Newton on
#   R_M = M - Q(M, y) = 0,  R_y = y - q(M, y) = 0
# (Eq. implicitMomentsNodalFull and Eq. implicitFluidNodal), with a
# central-difference Jacobian.  It shares the maps with Algorithm 1 but none
# of the fixed-point/Anderson logic, so agreement pins the iteration.
# ---------------------------------------------------------------------------

def _residual(x, ctx):
    grid, tables, p, rho, M_star, y_star, EN_star, g, dtau, scale = ctx
    ns, ne = M_star.shape[:2]
    nm = ns * ne * 4
    M = x[:nm].reshape(ns, ne, 4)
    y = x[nm:] * np.abs(y_star)
    T, _ = eos.temperature(rho, y[0], y[1])
    op = compute_opacities(grid, tables, rho, T, y[1], scale, p.proc_mask, p.dmin, p.dmax)
    RM = M - moment_map(M, M_star, op, grid.W2, dtau)
    Ry = (y - matter_map(M[:, :, 0], rho, y_star, EN_star, grid, g)) / np.abs(y_star)
    return np.concatenate([RM.ravel(), Ry])


def newton_solve_node(grid, tables, params, rho, T_star, Ye_star, D_star, I_star, dt,
                      scale=(1, 1, 1, 1), x0=None, max_iter=50, tol=1e-14):
    """Damped Newton with a finite-difference Jacobian on the coupled residual."""
    ns, ne = D_star.shape
    g = lepton_numbers(ns)
    dtau = C_LIGHT * dt
    eps_star = eos.specific_energy(rho, T_star, Ye_star)
    y_star = np.array([eps_star, Ye_star])
    M_star = np.concatenate([D_star[:, :, None], I_star], axis=2).astype(np.float64)
    EN_star = neutrino_energy_number(M_star[:, :, 0], grid, g)
    ctx = (grid, tables, params, rho, M_star, y_star, EN_star, g, dtau, scale)
    x = np.concatenate([M_star.ravel(), np.ones(2)]) if x0 is None else x0.copy()
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
    y = x[nm:] * np.abs(y_star)
    T, _ = eos.temperature(rho, y[0], y[1])
    return dict(D=M[:, :, 0], I=M[:, :, 1:], eps=float(y[0]), Ye=float(y[1]), T=float(T),
                residual=float(np.linalg.norm(r)))
