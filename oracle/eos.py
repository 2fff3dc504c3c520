"""Synthetic closed-form equation of state (oracle).

The paper takes thermodynamic quantities from the SFHo table through weaklib and
obtains T from (rho, eps, Ye) by root finding once eps and Ye are updated
(Sec. 3.5.2, paragraph after Eq. eulerianNumberLG).  That table is not
available, so a smooth closed-form EoS stands in for it:

* electrons + positrons: massless ideal Fermi gas, two spin states, exact
  net number density  n_e = (mu^3 + pi^2 T^2 mu) / (3 pi^2 (hbar c)^3)
  and energy density  u_e = (7 pi^2 T^4/60 + T^2 mu^2/2 + mu^4/(4 pi^2)) / (hbar c)^3;
* nucleons: non-degenerate ideal gas, u_N = (3/2) T n_B, n_B = rho / m_B;
* photons: u_gamma = (pi^2/15) T^4 / (hbar c)^3.

Chemical potentials: n_e = rho Ye / m_B fixes mu_e; the neutron-proton
chemical potential difference of a non-degenerate nucleon gas is
mu_hat = T ln((1-Ye)/Ye) + (m_n - m_p); mu_nue = mu_e - mu_hat,
mu_anue = -mu_nue and heavy flavours have mu = 0.  The electron degeneracy
eta_e = mu_e / T indexes the NES and pair kernel tables (Sec. 2.3).
"""

import math
import numpy as np

from .constants import HBARC, M_B, MEV_TO_ERG, DM_NP

PI2 = math.pi ** 2


def electron_chemical_potential(rho, T, Ye):
    """mu_e [MeV]: the unique real root of mu^3 + pi^2 T^2 mu - 3 pi^2 (hbar c)^3 n_e = 0.

    For a depressed cubic x^3 + p x + q = 0 with p > 0 the real root is
    x = -2 sqrt(p/3) sinh( asinh( (3 q / (2 p)) sqrt(3/p) ) / 3 ).
    """
    ne = Ye * rho / M_B
    p = PI2 * T * T
    q = -3.0 * PI2 * HBARC ** 3 * ne
    return -2.0 * math.sqrt(p / 3.0) * math.sinh(math.asinh(1.5 * q / p * math.sqrt(3.0 / p)) / 3.0)


def electron_number_density(mu, T):
    """Net e- minus e+ number density [cm^-3] of the massless gas."""
    return (mu ** 3 + PI2 * T * T * mu) / (3.0 * PI2 * HBARC ** 3)


def energy_density(rho, T, Ye):
    """Total internal energy density [MeV cm^-3] of the synthetic EoS."""
    mu = electron_chemical_potential(rho, T, Ye)
    ue = (7.0 * PI2 * T ** 4 / 60.0 + 0.5 * T * T * mu * mu + mu ** 4 / (4.0 * PI2)) / HBARC ** 3
    un = 1.5 * T * rho / M_B
    ug = PI2 / 15.0 * T ** 4 / HBARC ** 3
    return ue + un + ug


def specific_energy(rho, T, Ye):
    """Specific internal energy eps [erg/g]."""
    return energy_density(rho, T, Ye) * MEV_TO_ERG / rho


T_MIN = 1.0e-3   # MeV, root-finding bracket
T_MAX = 1.0e3


def temperature(rho, eps, Ye):
    """T [MeV] with specific_energy(rho, T, Ye) = eps, by bisection in log T.

    eps is strictly increasing in T at fixed (rho, Ye) (all three gases have a
    positive heat capacity), so the root is unique.  Returns (T, ok); ok is
    False when eps lies outside [eps(T_MIN), eps(T_MAX)] and T is clamped.
    """
    lo, hi = math.log(T_MIN), math.log(T_MAX)
    if not (0.0 < Ye < 1.0) or not math.isfinite(eps):
        return float("nan"), False
    if eps <= specific_energy(rho, T_MIN, Ye):
        return T_MIN, False
    if eps >= specific_energy(rho, T_MAX, Ye):
        return T_MAX, False
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if specific_energy(rho, math.exp(mid), Ye) < eps:
            lo = mid
        else:
            hi = mid
    return math.exp(0.5 * (lo + hi)), True


def chemical_potentials(rho, T, Ye, ns):
    """(mu_e, eta_e, [mu_s for each species]) in MeV."""
    mu_e = electron_chemical_potential(rho, T, Ye)
    mu_hat = T * math.log((1.0 - Ye) / Ye) + DM_NP
    mu_nue = mu_e - mu_hat
    mus = np.zeros(ns)
    mus[0] = mu_nue
    if ns > 1:
        mus[1] = -mu_nue
    return mu_e, mu_e / T, mus
