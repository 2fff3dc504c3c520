"""Seeded synthetic inputs: opacity/kernel tables and node states.

This module produces DATA only.  It holds none of the solver's arithmetic (no
equation of state, no Fermi--Dirac projection, no rates), so the CUDA path and
the CPU oracle can both be fed from it without sharing any of the method.

The weaklib/SFHo tables and the supernova profiles used by the paper are not
available; smooth seeded stand-ins with the same structure take their place:

* chi_EmAb and sigma_Iso on a (species, Ye, T, rho, energy) grid of natural
  logs, chi = chi0_s (rho/1e14) (E/10 MeV)^2 g_s(T, Ye) with a seeded
  log-smooth factor g_s in [0.5, 2]; the energy axis is the nodal energy set
  of the grid the tables are made for;
* the NES structure function Phi_Out(T, eta, eps, eps') for eps >= eps'
  (down-scattering half; the solver fills the rest by detailed balance) and
  the pair annihilation kernel Phi_Ann(T, eta, eps, eps') of the particle of
  each particle/antiparticle pair, both positive and smooth in (log T, eta);
* node states along a collapse-shaped profile: rho from 3e14 g/cm^3 at 10 km
  to 1e9 g/cm^3 at 3000 km, T = 40 MeV (r/10 km)^-0.647, Ye from 0.25 to 0.5,
  and occupations of logistic shape with seeded perturbations (up to 30%,
  smaller in the dense core).
"""

import math
import numpy as np

# table axes: (lo, hi, n) on uniform grids
RHO_AXIS = (8.0, 15.0, 32)       # log10 rho [g/cm^3]
T_AXIS = (math.log10(0.5), math.log10(60.0), 32)    # log10 T [MeV]
YE_AXIS = (0.05, 0.6, 16)
KT_AXIS = (math.log10(0.5), math.log10(60.0), 32)   # kernels: log10 T [MeV]
KETA_AXIS = (0.0, 80.0, 32)      # kernels: eta_e = mu_e / T

# opacity normalisations (chi in 1/cm at rho = 1e14, E = 10 MeV)
CHI0 = (3.0e-3, 1.0e-3, 3.0e-9, 3.0e-9)
SIG0 = (2.0e-3, 2.0e-3, 2.0e-3, 2.0e-3)
# NES / pair structure-function scales (cm^2), per species / per pair
NES0 = (4.0e-40, 2.0e-40, 1.0e-40, 1.0e-40)
PAIR0 = (2.0e-40, 1.0e-40)


def _smooth_factor(rng, x, y, amp=math.log(2.0)):
    """exp of a seeded smooth function of x, y in [0, 1], bounded to [e^-amp, e^amp]."""
    a = rng.uniform(-1.0, 1.0, size=4)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=2)
    v = (a[0] * np.sin(math.pi * x + ph[0]) + a[1] * np.cos(2.0 * math.pi * y + ph[1])
         + a[2] * np.sin(math.pi * (x + y)) + a[3] * x * y)
    return np.exp(amp * v / np.sum(np.abs(a)))


def _species_list(ns):
    return [min(s, 2 + (s % 2)) for s in range(ns)]   # 0 nue, 1 anue, heavy -> 2/3


def make_tables(energies, ns, seed=0, linear=False):
    """Synthetic opacity and kernel tables for nodal energies `energies` (MeV); with `linear`, also
    the linear-order kernels Phi_1 of NES and pair ("nes1", "pair1", drawn after the others)."""
    rng = np.random.default_rng(seed)
    en = np.asarray(energies, dtype=np.float64)
    ne = en.size
    lr = np.linspace(*RHO_AXIS)
    lt = np.linspace(*T_AXIS)
    ye = np.linspace(*YE_AXIS)
    xt = (lt - lt[0]) / (lt[-1] - lt[0])
    xy = (ye - ye[0]) / (ye[-1] - ye[0])
    XT, XY = np.meshgrid(xt, xy, indexing="ij")        # (nT, nYe)
    kinds = _species_list(ns)
    emab = np.empty((ns, YE_AXIS[2], T_AXIS[2], RHO_AXIS[2], ne))
    iso = np.empty_like(emab)
    for s in range(ns):
        base_r = (lr - 14.0) * math.log(10.0)                       # ln(rho/1e14)
        base_e = 2.0 * np.log(en / 10.0)                            # ln((E/10)^2)
        for tab, c0 in ((emab, CHI0[kinds[s]]), (iso, SIG0[kinds[s]])):
            gfac = np.log(_smooth_factor(rng, XT, XY)).T            # (nYe, nT)
            tab[s] = (math.log(c0) + gfac[:, :, None, None] + base_r[None, None, :, None]
                      + base_e[None, None, None, :])
    klt = np.linspace(*KT_AXIS)
    ket = np.linspace(*KETA_AXIS)
    T = 10.0 ** klt
    xk = (klt - klt[0]) / (klt[-1] - klt[0])
    xe = (ket - ket[0]) / (ket[-1] - ket[0])
    XK, XE = np.meshgrid(xk, xe, indexing="ij")        # (nkT, neta)
    E, Ep = np.meshgrid(en, en, indexing="ij")         # E = eps_q (row), Ep = eps_q' (column)
    down = np.maximum(E - Ep, 0.0)
    # electron-density proxy: T^2 (eta^3 + pi^2 eta + 2), normalised at T = 10, eta = 5
    dens = ((T[:, None] / 10.0) ** 2 * (ket[None, :] ** 3 + math.pi ** 2 * ket[None, :] + 2.0)
            / (125.0 + 5.0 * math.pi ** 2 + 2.0))
    nes = np.zeros((ns, KT_AXIS[2], KETA_AXIS[2], ne, ne))
    shape = np.exp(-down[None, :, :] / (2.0 * T[:, None, None])) * (E >= Ep)[None, :, :]  # (nkT, ne, ne)
    for s in range(ns):
        amp = NES0[kinds[s]] * dens * _smooth_factor(rng, XK, XE)     # (nkT, neta)
        nes[s] = amp[:, :, None, None] * shape[:, None, :, :]
    npair = (ns + 1) // 2
    pair = np.zeros((npair, KT_AXIS[2], KETA_AXIS[2], ne, ne))
    # asymmetric in (eps, eps') so that a transposed operand changes the answer
    pshape = ((E + Ep) / 20.0) ** 2 * (1.0 + 0.5 * np.tanh((E - Ep) / 20.0))
    for p in range(npair):
        amp = PAIR0[min(p, 1)] * dens * np.exp(-0.1 * ket)[None, :] * _smooth_factor(rng, XK, XE)
        pair[p] = amp[:, :, None, None] * pshape[None, None, :, :]
    out = dict(ns=ns, ne=ne, energies=en.copy(),
               lrho=RHO_AXIS, lT=T_AXIS, ye=YE_AXIS, emab=emab, iso=iso,
               klT=KT_AXIS, keta=KETA_AXIS, nes=nes, pair=pair)
    if linear:
        # linear-order Legendre coefficients Phi_1 of the same kernels: Phi_1 = -c Phi_0 with c a
        # seeded smooth function of (log T, eta) in [0.1, 0.4] (|Phi_1| < Phi_0, a kernel that
        # stays positive over scattering angles)
        out["nes1"] = np.empty_like(nes)
        for s in range(ns):
            c = 0.25 * _smooth_factor(rng, XK, XE, amp=math.log(1.6))
            out["nes1"][s] = -c[:, :, None, None] * nes[s]
        out["pair1"] = np.empty_like(pair)
        for p_ in range(npair):
            c = 0.25 * _smooth_factor(rng, XK, XE, amp=math.log(1.6))
            out["pair1"][p_] = -c[:, :, None, None] * pair[p_]
    return out


def _logistic(e, a, T):
    return 1.0 / (1.0 + np.exp(np.clip((e - a) / T, -700.0, 700.0)))


def _occupations(rng, en, ns, rho, T, Ye, amp=0.3):
    """Occupations of logistic shape around a crude chemical-potential guess.

    The guess is the textbook degenerate-electron Fermi energy
    11.1 MeV (rho Ye / 1e10 g cm^-3)^(1/3) lowered by 1.5 T; it only shapes the
    input spectra and is never used by the solvers.  Each energy bin is
    perturbed by a uniform factor 1 +- amp / (1 + rho / 1e12 g cm^-3): up to 30%
    in the semi-transparent region, small in the thermalised dense core.
    """
    N = rho.size
    ne = en.size
    a_e = 11.1 * (rho * Ye / 1e10) ** (1.0 / 3.0) - 1.5 * T
    D = np.empty((N, ns, ne))
    for s in range(ns):
        a = a_e if s == 0 else (-a_e if s == 1 else np.zeros(N))
        base = _logistic(en[None, :], a[:, None], T[:, None])
        a_r = amp / (1.0 + rho / 1e12)
        pert = 1.0 + a_r[:, None] * rng.uniform(-1.0, 1.0, size=(N, ne))
        D[:, s, :] = np.clip(base * pert, 0.0, 1.0 - 1e-6)
    return D


def profile_states(rng, N, perturb=0.0):
    """rho, T, Ye along a synthetic collapse profile, optionally perturbed."""
    r = 10.0 ** rng.uniform(1.0, math.log10(3000.0), size=N)      # km
    x = np.log10(r / 10.0) / np.log10(300.0)                      # 0 at 10 km, 1 at 3000 km
    lrho = math.log10(3e14) + x * (9.0 - math.log10(3e14))
    rho = 10.0 ** lrho
    T = 40.0 * (r / 10.0) ** -0.647
    Ye = 0.25 + 0.25 * x
    if perturb > 0.0:
        rho = rho * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=N))
        T = T * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=N))
        Ye = Ye * (1.0 + perturb * rng.uniform(-1.0, 1.0, size=N))
    return r, rho, T, Ye


def make_inputs(kind, N, energies, ns, seed=0):
    """Seeded node inputs.

    kind:
      'uniform'     rho log-uniform 1e10..1e14, T uniform 3..30 MeV, Ye 0.1..0.5,
                    D uniform in [0, 1), |I| < D, dt = 1e-6 s
      'profile'     collapse profile, dt = 1e-6 s
      'perturbed'   collapse profile with +-10% perturbations of rho, T, Ye
      'core_tail'   half core (rho > 1e13) and half tail (rho < 1e10) of the
                    profile, dt log-uniform 1e-7..1e-5 s
    """
    rng = np.random.default_rng(seed)
    en = np.asarray(energies, dtype=np.float64)
    ne = en.size
    if kind == "uniform":
        rho = 10.0 ** rng.uniform(10.0, 14.0, size=N)
        T = rng.uniform(3.0, 30.0, size=N)
        Ye = rng.uniform(0.1, 0.5, size=N)
        D = rng.uniform(0.0, 1.0, size=(N, ns, ne))
        nhat = rng.normal(size=(N, ns, ne, 3))
        nhat /= np.linalg.norm(nhat, axis=-1, keepdims=True)
        h = rng.uniform(0.0, 1.0, size=(N, ns, ne, 1))
        I = D[..., None] * h * nhat
        dt = np.full(N, 1e-6)
    else:
        if kind == "core_tail":
            half = N // 2
            r1, rho1, T1, Ye1 = profile_states(rng, 4 * N)
            core = np.nonzero(rho1 > 1e13)[0]
            tail = np.nonzero(rho1 < 1e10)[0]
            ic = rng.choice(core, size=half, replace=True)
            itl = rng.choice(tail, size=N - half, replace=True)
            sel = np.concatenate([ic, itl])
            rng.shuffle(sel)
            r, rho, T, Ye = r1[sel], rho1[sel], T1[sel], Ye1[sel]
            dt = 10.0 ** rng.uniform(-7.0, -5.0, size=N)
        else:
            r, rho, T, Ye = profile_states(rng, N, perturb=0.1 if kind == "perturbed" else 0.0)
            dt = np.full(N, 1e-6)
        D = _occupations(rng, en, ns, rho, T, Ye)
        h = np.tanh(r / 100.0)[:, None, None] * rng.uniform(0.0, 1.0, size=(N, ns, ne))
        I = np.zeros((N, ns, ne, 3))
        I[..., 0] = D * h
    scale = np.ones((N, 4))
    return dict(rho=rho, T=T, Ye=Ye, D=D, I=I, dt=dt, scale=scale)


def make_velocities(kind, N, seed=0, vmax=0.15):
    """Fluid three-velocities (units of c) for the O(v/c) solve; data only.

    "random": isotropic directions, speeds uniform in [0, vmax].  Otherwise an
    infall profile along the x axis (the direction of the profile inputs'
    fluxes), v_x = -2 vmax x / (1 + x^2) with x = r / 100 km (fastest at
    100 km) over r log-uniform in 10-3000 km, plus transverse components of
    1% of vmax.
    """
    rng = np.random.default_rng(seed + 7919)
    if kind == "random":
        d = rng.normal(size=(N, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return d * rng.uniform(0.0, vmax, size=(N, 1))
    x = 10.0 ** rng.uniform(1.0, math.log10(3000.0), size=N) / 100.0
    v = np.zeros((N, 3))
    v[:, 0] = -2.0 * vmax * x / (1.0 + x * x)
    v[:, 1:] = 0.01 * vmax * rng.normal(size=(N, 2))
    return v


def make_interp_points(P, energies, seed=0):
    """Scattered matter states and energies for opacity_interp; data only.

    (rho, T, Ye) uniform in (log10 rho, log10 T, Ye) over the table axes and E
    log-uniform between the lowest and highest node energy, so every lookup is
    an interior, tetralinear one at an unrelated table cell.
    """
    rng = np.random.default_rng(seed + 104729)
    e = np.asarray(energies, dtype=float)
    return dict(rho=10.0 ** rng.uniform(RHO_AXIS[0], RHO_AXIS[1], size=P),
                T=10.0 ** rng.uniform(T_AXIS[0], T_AXIS[1], size=P),
                Ye=rng.uniform(YE_AXIS[0], YE_AXIS[1], size=P),
                E=np.exp(rng.uniform(math.log(e[0]), math.log(e[-1]), size=P)))
