"""Physical constants for the oracle (units: MeV, cm, g, s; c = k_B = 1).

The paper works in units with c = G = k_B = 1 (Sec. 1) and writes the energy
integration weights with h^3 (Eq. energy_integration_weights); with energies in
MeV the factor becomes (hc)^3.  The average baryon mass m_B (Sec. 2.1) has no
value in the paper; the atomic mass unit is used.
"""

import math

C_LIGHT = 2.99792458e10          # cm / s
HC = 1.23984198e-10              # MeV cm
HBARC = HC / (2.0 * math.pi)     # MeV cm
M_B = 1.66053906660e-24          # g, average baryon mass (atomic mass unit)
MEV_TO_ERG = 1.602176634e-6      # erg / MeV
DM_NP = 1.2933                   # MeV, neutron-proton mass difference

# Lepton numbers g_s (Sec. 2.2): +1 for nu_e, -1 for anti-nu_e, 0 otherwise.
# Species are ordered as particle/antiparticle pairs: (nu_e, anti-nu_e),
# then (nu_x, anti-nu_x) for each heavy flavour.


def lepton_numbers(ns):
    g = [0.0] * ns
    g[0] = 1.0
    if ns > 1:
        g[1] = -1.0
    return g


def partner(s):
    """Index of the antiparticle of species s (pairs are (0,1), (2,3), ...)."""
    return s ^ 1
