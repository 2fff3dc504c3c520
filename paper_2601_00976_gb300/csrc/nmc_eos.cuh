// Synthetic closed-form equation of state on the device (FP64).
//
// Stands in for the tabulated EoS the paper interpolates with weaklib
// (Sec. 3.5.2, paragraph after Eq. eulerianNumberLG): a massless e+e- gas
// (exact Fermi--Dirac moments), a non-degenerate nucleon gas and photons.
//   n_e   = (mu^3 + pi^2 T^2 mu) / (3 pi^2 (hbar c)^3) = rho Ye / m_B
//   u_e   = (7 pi^2 T^4/60 + T^2 mu^2/2 + mu^4/(4 pi^2)) / (hbar c)^3
//   u_N   = 1.5 T rho / m_B,   u_gamma = pi^2 T^4 / (15 (hbar c)^3)
//   eps   = (u_e + u_N + u_gamma) / rho        [erg/g after unit conversion]
//   mu_nue = mu_e - T ln((1-Ye)/Ye) - (m_n - m_p),  mu_anue = -mu_nue, mu_x = 0.
#pragma once

#include "nmc_internal.h"

namespace nmc {

__device__ __forceinline__ double eos_mu_e(double rho, double T, double Ye) {
    const double pi2 = kPi * kPi;
    const double hc3 = kHbarC * kHbarC * kHbarC;
    const double ne = Ye * rho / kMB;
    const double p = pi2 * T * T;
    const double q = -3.0 * pi2 * hc3 * ne;
    // real root of x^3 + p x + q = 0 (p > 0): hyperbolic form of Cardano's solution
    return -2.0 * sqrt(p / 3.0) * sinh(asinh(1.5 * q / p * sqrt(3.0 / p)) / 3.0);
}

// eps(rho, T, Ye) in erg/g and d eps / dT at fixed rho, Ye, given the electron
// chemical potential mu at (rho, T, Ye).
__device__ __forceinline__ void eos_eps_at_mu(double rho, double T, double mu, double* eps, double* deps) {
    const double pi2 = kPi * kPi;
    const double hc3 = kHbarC * kHbarC * kHbarC;
    const double T2 = T * T, mu2 = mu * mu;
    const double ue = (7.0 * pi2 * T2 * T2 / 60.0 + 0.5 * T2 * mu2 + mu2 * mu2 / (4.0 * pi2)) / hc3;
    const double nb = rho / kMB;
    const double ug = pi2 / 15.0 * T2 * T2 / hc3;
    const double f = kMeVErg / rho;
    *eps = (ue + 1.5 * T * nb + ug) * f;
    // mu(T) at fixed n_e: dmu/dT = -(dn/dT)/(dn/dmu) = -2 pi^2 T mu / (3 mu^2 + pi^2 T^2)
    const double dmu = -2.0 * pi2 * T * mu / (3.0 * mu2 + pi2 * T2);
    const double due = (7.0 * pi2 * T2 * T / 15.0 + T * mu2 + (T2 * mu + mu2 * mu / pi2) * dmu) / hc3;
    *deps = (due + 1.5 * nb + 4.0 * pi2 / 15.0 * T2 * T / hc3) * f;
}

__device__ __forceinline__ void eos_eps(double rho, double T, double Ye, double* eps, double* deps) {
    eos_eps_at_mu(rho, T, eos_mu_e(rho, T, Ye), eps, deps);
}

// T with eps(rho, T, Ye) = eps_t: safeguarded Newton in T within [kTMin, kTMax].
// The bracket starts as the whole range without evaluating its ends (a warm
// start from the previous T needs ~3 evaluations); every evaluation narrows it,
// and a Newton step that leaves it is replaced by a geometric bisection.
// eps is strictly increasing in T, so an eps_t outside [eps(kTMin), eps(kTMax)]
// drives the iterate to a range end: *ok = false and T clamped there.
__device__ inline double eos_temperature(double rho, double eps_t, double Ye, double T0, bool* ok) {
    *ok = true;
    if (!(Ye > 0.0 && Ye < 1.0) || !isfinite(eps_t)) {
        *ok = false;
        return isfinite(T0) ? T0 : 1.0;
    }
    double lo = kTMin, hi = kTMax, e, de, f = 0.0;
    double T = (T0 > lo && T0 < hi) ? T0 : sqrt(lo * hi);
    for (int it = 0; it < 300; ++it) {
        eos_eps(rho, T, Ye, &e, &de);
        f = e - eps_t;
        if (f > 0.0) hi = T; else lo = T;
        if (f == 0.0) break;
        double Tn = T - f / de;
        if (!(Tn > lo && Tn < hi)) Tn = hi > 2.0 * lo ? sqrt(lo * hi) : 0.5 * (lo + hi);
        const double d = fabs(Tn - T);
        T = Tn;
        if (d <= 2e-16 * T || hi - lo <= 4e-16 * hi) break;
    }
    if (f > 0.0 && T <= kTMin * (1.0 + 1e-12)) {   // eps_t below eps(kTMin)
        eos_eps(rho, kTMin, Ye, &e, &de);
        if (eps_t <= e) { *ok = false; return kTMin; }
    }
    if (f < 0.0 && T >= kTMax * (1.0 - 1e-12)) {   // eps_t above eps(kTMax)
        eos_eps(rho, kTMax, Ye, &e, &de);
        if (eps_t >= e) { *ok = false; return kTMax; }
    }
    return T;
}

__device__ __forceinline__ double eos_deps_dye(double rho, double T, double Ye) {
    const double pi2 = kPi * kPi;
    const double mu = eos_mu_e(rho, T, Ye);
    const double mu2 = mu * mu, T2 = T * T;
    return kMeVErg / kMB * 3.0 * mu * (mu2 + pi2 * T2) / (3.0 * mu2 + pi2 * T2);
}

// ---- FP32 variants for the mixed-precision path ----
// Densities are carried times (hbar c)^3 (MeV^3) and energy densities times
// (hbar c)^3 (MeV^4), so every intermediate stays inside FP32 range:
// u (hbar c)^3 = 7 pi^2 T^4/60 + T^2 mu^2/2 + mu^4/(4 pi^2) + 1.5 T nb + pi^2 T^4/15.

struct EosScaleF {
    float nb;      // (rho / m_B) (hbar c)^3
    float ne;      // Ye nb
    double k;      // eps [erg/g] = u~ [MeV^4] * k,  k = MeV/erg / ((hbar c)^3 rho)
};

__device__ __forceinline__ EosScaleF eos_scale(double rho, double Ye) {
    const double hc3 = kHbarC * kHbarC * kHbarC;
    EosScaleF s;
    const double nb = rho / kMB * hc3;
    s.nb = (float)nb;
    s.ne = (float)(Ye * nb);
    s.k = kMeVErg / (hc3 * rho);
    return s;
}

__device__ __forceinline__ float eos_mu_e_f(float ne, float T) {
    const float pi2 = (float)(kPi * kPi);
    const float p = pi2 * T * T;
    const float q = -3.0f * pi2 * ne;
    return -2.0f * sqrtf(p / 3.0f) * sinhf(asinhf(1.5f * q / p * sqrtf(3.0f / p)) / 3.0f);
}

// mu_e in FP64 for the mixed path: the FP32 root of the electron cubic
// x^3 + pi^2 T^2 x - 3 pi^2 n_e (hbar c)^3 = 0 and one FP64 Newton step on it,
// which squares its relative error (~1e-7 to ~1e-14) for a handful of FP64
// operations instead of the closed form's FP64 asinh and sinh.
__device__ __forceinline__ double eos_mu_e_refined(double rho, double T, double Ye) {
    const EosScaleF es = eos_scale(rho, Ye);
    const double m0 = eos_mu_e_f(es.ne, (float)T);
    const double pi2T2 = kPi * kPi * T * T;
    const double ned = Ye * rho / kMB * (kHbarC * kHbarC * kHbarC);   // FP64 target
    const double cub = m0 * (m0 * m0 + pi2T2) - 3.0 * kPi * kPi * ned;
    return m0 - cub / (3.0 * m0 * m0 + pi2T2);
}

__device__ __forceinline__ void eos_u_f(const EosScaleF& sc, float T, float* u, float* du) {
    const float pi2 = (float)(kPi * kPi);
    const float mu = eos_mu_e_f(sc.ne, T);
    const float T2 = T * T, mu2 = mu * mu;
    *u = 7.0f * pi2 * T2 * T2 / 60.0f + 0.5f * T2 * mu2 + mu2 * mu2 / (4.0f * pi2) + 1.5f * T * sc.nb +
         pi2 / 15.0f * T2 * T2;
    const float dmu = -2.0f * pi2 * T * mu / (3.0f * mu2 + pi2 * T2);
    *du = 7.0f * pi2 * T2 * T / 15.0f + T * mu2 + (T2 * mu + mu2 * mu / pi2) * dmu + 1.5f * sc.nb +
          4.0f * pi2 / 15.0f * T2 * T;
}

// Temperature for the mixed path: bracketed Newton in FP32 to ~1e-7, then one
// FP64 Newton step on eps(rho, T, Ye) (with mu_e refined from its FP32 root),
// which squares the relative error.
__device__ inline double eos_temperature_mixed(double rho, double eps_t, double Ye, double T0, bool* ok) {
    *ok = true;
    if (!(Ye > 0.0 && Ye < 1.0) || !isfinite(eps_t)) {
        *ok = false;
        return isfinite(T0) ? T0 : 1.0;
    }
    const EosScaleF sc = eos_scale(rho, Ye);
    const float ut = (float)(eps_t / sc.k);
    float lo = (float)kTMin, hi = (float)kTMax, u, du;
    eos_u_f(sc, lo, &u, &du);
    if (ut <= u) { *ok = false; return kTMin; }
    eos_u_f(sc, hi, &u, &du);
    if (ut >= u) { *ok = false; return kTMax; }
    float T = (T0 > kTMin && T0 < kTMax) ? (float)T0 : sqrtf(lo * hi);
    for (int it = 0; it < 100; ++it) {
        eos_u_f(sc, T, &u, &du);
        const float f = u - ut;
        if (f > 0.0f) hi = T; else lo = T;
        if (f == 0.0f) break;
        float Tn = T - f / du;
        if (!(Tn > lo && Tn < hi)) Tn = 0.5f * (lo + hi);
        const float d = fabsf(Tn - T);
        T = Tn;
        if (d <= 2e-7f * T || hi - lo <= 4e-7f * hi) break;
    }
    double Td = T, e, de;
    eos_eps_at_mu(rho, Td, eos_mu_e_refined(rho, Td, Ye), &e, &de);
    const double Tn = Td - (e - eps_t) / de;
    return (Tn > kTMin && Tn < kTMax) ? Tn : Td;
}

}  // namespace nmc
