// Fully polarised LSDA on one orbital density (Eq. 1 evaluates
// E_xc[rho_i, 0]; Sec. III names LSDA exchange with PW92 correlation).
#pragma once

namespace flosic {

// PW92 correlation of the fully polarised electron gas.  At zeta = 1 the
// spin interpolation of Perdew & Wang (Phys. Rev. B 45, 13244 (1992))
// leaves only its ferromagnetic fit
//   eps_c(rs) = -2A(1 + a1 rs) ln(1 + 1/(2A(b1 rs^1/2 + b2 rs + b3 rs^3/2 + b4 rs^2)))
// with the tabulated parameters below (A = 0.015545).
struct Pw92Ferro {
    static constexpr double A = 0.015545;
    static constexpr double a1 = 0.20548;
    static constexpr double b1 = 14.1189;
    static constexpr double b2 = 6.1977;
    static constexpr double b3 = 3.3662;
    static constexpr double b4 = 0.62517;
};

// eps_xc (energy per electron) and v_xc of the occupied spin channel for
// spin densities (n, 0).  Exchange by spin scaling of the Dirac form:
// eps_x = -(3/4) k, v_x = -k with k = (6n/pi)^{1/3}.  Correlation potential
// v_c = eps_c - (rs/3) d eps_c/d rs (the d/dzeta term vanishes at zeta = 1).
// Densities at or below rho_min give zero.
__device__ __forceinline__ void lsda_pol(double n, double rho_min, double& eps, double& v) {
    if (!(n > rho_min)) {
        eps = 0.0;
        v = 0.0;
        return;
    }
    const double k = cbrt(6.0 * n * (1.0 / 3.14159265358979323846));
    const double rs = cbrt(3.0 / (4.0 * 3.14159265358979323846 * n));
    const double srs = sqrt(rs);
    using P = Pw92Ferro;
    const double den = 2.0 * P::A * (P::b1 * srs + P::b2 * rs + P::b3 * rs * srs + P::b4 * rs * rs);
    const double dden = P::A * (P::b1 / srs + 2.0 * P::b2 + 3.0 * P::b3 * srs + 4.0 * P::b4 * rs);
    const double lg = log1p(1.0 / den);
    const double pre = -2.0 * P::A * (1.0 + P::a1 * rs);
    const double ec = pre * lg;
    const double dec = -2.0 * P::A * P::a1 * lg - pre * dden / (den * den + den);
    eps = -0.75 * k + ec;
    v = -k + ec - rs * (1.0 / 3.0) * dec;
}

// The same functional in float32 arithmetic (mixed-precision path; the
// energies are still summed in float64).  One cube root serves both k and
// rs (rs = (3/4pi)^{1/3} / n^{1/3}, k = (6/pi)^{1/3} n^{1/3}); reciprocals and
// the inverse square root use the fast float forms (a few ulp, far below the
// path's 1e-6 Ha target per orbital energy); log1p keeps its accuracy for the
// small arguments of low densities.
__device__ __forceinline__ void lsda_pol_f(float n, float rho_min, float& eps, float& v) {
    if (!(n > rho_min)) {
        eps = 0.0f;
        v = 0.0f;
        return;
    }
    const float cn = cbrtf(n);
    const float k = (float)1.2407009817988002 * cn;                   // (6/pi)^{1/3} n^{1/3}
    const float rs = __fdividef((float)0.62035049089940001, cn);      // (3/(4 pi))^{1/3} / n^{1/3}
    const float irs = rsqrtf(rs);
    const float srs = rs * irs;
    using P = Pw92Ferro;
    const float A = (float)P::A;
    const float den = 2.0f * A * ((float)P::b1 * srs + (float)P::b2 * rs + (float)P::b3 * rs * srs + (float)P::b4 * rs * rs);
    const float dden = A * ((float)P::b1 * irs + 2.0f * (float)P::b2 + 3.0f * (float)P::b3 * srs + 4.0f * (float)P::b4 * rs);
    const float iden = __fdividef(1.0f, den);
    const float lg = log1pf(iden);
    const float pre = -2.0f * A * (1.0f + (float)P::a1 * rs);
    const float ec = pre * lg;
    const float dec = -2.0f * A * (float)P::a1 * lg - __fdividef(pre * dden * iden, 1.0f + den);
    eps = -0.75f * k + ec;
    v = -k + ec - rs * (1.0f / 3.0f) * dec;
}

}  // namespace flosic
