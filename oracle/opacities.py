"""Opacity and kernel evaluation (oracle): ComputeOpacities of Algorithm 1.

* EmAb and isoenergetic opacities chi_EmAb(eps, rho, T, Ye), sigma_Iso(...):
  tabulated and interpolated tetralinearly (Sec. 2.3, paragraph after
  Eq. linearCorrectionsPair).  The tables hold natural logs on uniform axes in
  (log10 rho, log10 T, Ye); the energy axis is the set of nodal energies of
  the solve's grid, so inside the solve the energy weight is exactly one and
  the interpolation is trilinear; `opacity_at` handles off-node energies
  (linear in ln eps between neighbouring nodes).
* NES and pair kernels: structure functions given on the energy grid and
  interpolated bilinearly in (T, eta) at run time (same paragraph); here the
  T axis is uniform in log10 T and eta is uniform.
* NES kernels obey in-out invariance (Eq. inOutInvarianceNES) and detailed
  balance (Eq. detailedBalanceNES).  The table holds Phi_Out only for
  eps_q >= eps_q' (down-scattering); the other triangle follows from the two
  relations together.
* Pair kernels: the table holds Phi_Ann of the particle of each pair; the
  antiparticle's kernel is its transpose (Eq. inOutInvariancePair) and
  Phi_Pro follows from detailed balance (Eq. detailedBalancePair).
* Emissivity by detailed balance eta_EmAb = chi_EmAb D^Eq (Eq. emissivityEmAbNodal).

Per-node opacity scale factors (EmAb, Iso, NES, Pair) multiply the four
contributions; a process mask switches contributions off.
"""

import math
import numpy as np

from . import eos
from .equilibrium import equilibrium_distribution

EMAB, ISO, NES, PAIR = 1, 2, 4, 8


def _axis(v, lo, hi, n):
    """Cell index and weight on a uniform axis; clamps outside [lo, hi]."""
    x = (v - lo) / (hi - lo) * (n - 1)
    clamped = x < 0.0 or x > n - 1 or not math.isfinite(x)
    x = min(max(x, 0.0), float(n - 1)) if math.isfinite(x) else 0.0
    i = min(int(math.floor(x)), n - 2)
    return i, x - i, clamped


def _trilinear(vals, ir, tr, it, tt, iy, ty):
    out = 0.0
    for a, wa in ((0, 1.0 - tr), (1, tr)):
        for b, wb in ((0, 1.0 - tt), (1, tt)):
            for c, wc in ((0, 1.0 - ty), (1, ty)):
                out = out + wa * wb * wc * vals[:, iy + c, it + b, ir + a, :]
    return out


def interpolate_opacity(table_vals, axes_table, rho, T, Ye):
    """exp of the trilinear interpolant of ln(opacity) at node energies, (ns, ne)."""
    ir, tr, c1 = _axis(math.log10(rho), *axes_table["lrho"])
    it, tt, c2 = _axis(math.log10(T), *axes_table["lT"])
    iy, ty, c3 = _axis(Ye, *axes_table["ye"])
    return np.exp(_trilinear(table_vals, ir, tr, it, tt, iy, ty)), (c1 or c2 or c3)


def opacity_at(tables, which, species, rho, T, Ye, E):
    """Tetralinear interpolation at an arbitrary energy E (MeV).

    which: 0 = chi_EmAb, 1 = sigma_Iso.  Linear in ln E between the two
    neighbouring table energies; E outside the table range is clamped.
    """
    vals = tables["emab"] if which == 0 else tables["iso"]
    en = tables["energies"]
    lv = np.log(en)
    x = min(max(math.log(E), lv[0]), lv[-1])
    j = int(np.searchsorted(lv, x, side="right") - 1)
    j = min(max(j, 0), len(en) - 2)
    te = (x - lv[j]) / (lv[j + 1] - lv[j])
    ir, tr, _ = _axis(math.log10(rho), *tables["lrho"])
    it, tt, _ = _axis(math.log10(T), *tables["lT"])
    iy, ty, _ = _axis(Ye, *tables["ye"])
    sub = vals[species:species + 1]
    lo = _trilinear(sub[..., j:j + 1], ir, tr, it, tt, iy, ty)[0, 0]
    hi = _trilinear(sub[..., j + 1:j + 2], ir, tr, it, tt, iy, ty)[0, 0]
    return math.exp((1.0 - te) * lo + te * hi)


def interpolate_kernel(kvals, tables, T, eta):
    """Bilinear interpolation in (log10 T, eta) of a (., T, eta, ne, ne) kernel table."""
    it, tt, c1 = _axis(math.log10(T), *tables["klT"])
    ie, te, c2 = _axis(eta, *tables["keta"])
    out = ((1.0 - tt) * (1.0 - te) * kvals[:, it, ie]
           + tt * (1.0 - te) * kvals[:, it + 1, ie]
           + (1.0 - tt) * te * kvals[:, it, ie + 1]
           + tt * te * kvals[:, it + 1, ie + 1])
    return out, (c1 or c2)


def nes_kernels(lower, deq):
    """Phi_Out and Phi_In for one species from the down-scattering table `lower`.

    Detailed balance (Eq. detailedBalanceNES) together with in-out invariance
    (Eq. inOutInvarianceNES) gives, for eps_q < eps_q',
        Phi_Out[q, q'] = (b_q' / b_q) Phi_Out[q', q],   b = D^Eq / (1 - D^Eq),
    and Phi_In[q, q'] = Phi_Out[q', q].
    """
    ne = lower.shape[0]
    b = deq / (1.0 - deq)
    q = np.arange(ne)[:, None]
    qp = np.arange(ne)[None, :]
    # out[q, q'] = lower[q, q'] for q >= q';  (b_q' / b_q) lower[q', q] otherwise
    out = np.where(q >= qp, lower, (b[None, :] / b[:, None]) * lower.T)
    phi_in = out.T.copy()
    return out, phi_in


def pair_kernels(ann_particle, deq_s, deq_sbar, particle):
    """Phi_Pro and Phi_Ann for species s with antiparticle sbar.

    Phi_Ann of the antiparticle is the transpose of the particle's
    (Eq. inOutInvariancePair); Phi_Pro = G o Phi_Ann with
    G_qq' = D_q Dbar_q' / ((1 - D_q)(1 - Dbar_q')) (Eq. detailedBalancePair).
    """
    ann = ann_particle if particle else ann_particle.T
    g = np.outer(deq_s / (1.0 - deq_s), deq_sbar / (1.0 - deq_sbar))
    return g * ann, ann.copy()


def compute_opacities(grid, tables, rho, T, Ye, scale, proc_mask, dmin, dmax):
    """Everything Algorithm 1 needs at matter state (rho, T, Ye): the ComputeOpacities step."""
    ns = tables["ns"]
    mu_e, eta_e, mus = eos.chemical_potentials(rho, T, Ye, ns)
    deq = np.array([equilibrium_distribution(grid, mus[s], T, dmin, dmax) for s in range(ns)])
    chi_ab, c1 = interpolate_opacity(tables["emab"], tables, rho, T, Ye)
    sig, c2 = interpolate_opacity(tables["iso"], tables, rho, T, Ye)
    chi_ab = chi_ab * scale[0] * (1.0 if proc_mask & EMAB else 0.0)
    sig = sig * scale[1] * (1.0 if proc_mask & ISO else 0.0)
    ne = grid.ne
    phi_in = np.zeros((ns, ne, ne))
    phi_out = np.zeros((ns, ne, ne))
    phi_pro = np.zeros((ns, ne, ne))
    phi_ann = np.zeros((ns, ne, ne))
    c3 = c4 = False
    if proc_mask & NES:
        lower, c3 = interpolate_kernel(tables["nes"], tables, T, eta_e)
        for s in range(ns):
            phi_out[s], phi_in[s] = nes_kernels(scale[2] * lower[s], deq[s])
    if proc_mask & PAIR:
        ann, c4 = interpolate_kernel(tables["pair"], tables, T, eta_e)
        for s in range(ns):
            sb = s ^ 1
            phi_pro[s], phi_ann[s] = pair_kernels(scale[3] * ann[s // 2], deq[s], deq[sb], s % 2 == 0)
    op = dict(T=T, mu_e=mu_e, eta_e=eta_e, mu=mus, deq=deq, chi_ab=chi_ab, sig=sig,
              phi_in=phi_in, phi_out=phi_out, phi_pro=phi_pro, phi_ann=phi_ann,
              clamped=bool(c1 or c2 or c3 or c4))
    if "nes1" in tables:
        # linear-order kernels (Eqs. linearCorrectionsNES, linearCorrectionsPair); reading: they obey
        # the in-out invariance and detailed-balance relations of the isotropic ones, which hold for
        # every Legendre coefficient of a kernel, and take the same scale factors
        for key in ("phi1_in", "phi1_out", "phi1_pro", "phi1_ann"):
            op[key] = np.zeros((ns, ne, ne))
        if proc_mask & NES:
            lower1, _ = interpolate_kernel(tables["nes1"], tables, T, eta_e)
            for s in range(ns):
                op["phi1_out"][s], op["phi1_in"][s] = nes_kernels(scale[2] * lower1[s], deq[s])
        if proc_mask & PAIR:
            ann1, _ = interpolate_kernel(tables["pair1"], tables, T, eta_e)
            for s in range(ns):
                op["phi1_pro"][s], op["phi1_ann"][s] = pair_kernels(scale[3] * ann1[s // 2], deq[s], deq[s ^ 1],
                                                                    s % 2 == 0)
    return op
