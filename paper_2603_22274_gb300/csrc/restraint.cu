// Standard-state correction of the Boresch restraint: the free energy of
// imposing the six restraint terms on the ligand in its decoupled state, at
// 1 mol/L. The paper adds this analytic term to the simulated legs
// ("Restraints"). With the ligand decoupled, the restraint acts only on the six
// external coordinates, whose volume element is r^2 sin(theta_A) sin(theta_B)
// dr dtheta_A dtheta_B dphi_A dphi_B dphi_C; the restraint's partition function
// is a product of one-dimensional integrals, and
//     dG = -kT ln( Z_r Z_thetaA Z_thetaB Z_phi^3 / (8 pi^2 V0) ),  V0 = 1/(C0 N_A).
// Each integral is taken by composite Simpson over the span where its
// integrand is not negligible (+-40 standard deviations of the Gaussian, cut
// to the coordinate's range).
#include <cmath>

#include "abfe.h"
#include "abfe_internal.cuh"

namespace {

template <class F>
double simpson(F f, double a, double b, int n) {   // n even
    const double h = (b - a) / n;
    double s = f(a) + f(b);
    for (int i = 1; i < n; ++i) s += (i & 1 ? 4.0 : 2.0) * f(a + i * h);
    return s * h / 3.0;
}

constexpr int N_SIMPSON = 40000;

}  // namespace

extern "C" abfe_status abfe_boresch_correction(double kT, double r0, const double* theta0,
                                               double k_r, double k_theta, double k_phi,
                                               double* dG) {
    if (!theta0 || !dG || !(kT > 0) || !(r0 > 0) || !(k_r > 0) || !(k_theta > 0) || !(k_phi > 0) ||
        !(theta0[0] > 0 && theta0[0] < M_PI) || !(theta0[1] > 0 && theta0[1] < M_PI)) {
        abfe::set_free_error("boresch correction: kT, r0, force constants > 0, 0 < theta0 < pi");
        return ABFE_ERR_INVALID_ARG;
    }
    const double sr = std::sqrt(kT / k_r), st = std::sqrt(kT / k_theta), sp = std::sqrt(kT / k_phi);
    const double zr = simpson([&](double r) { return r * r * std::exp(-0.5 * k_r * (r - r0) * (r - r0) / kT); },
                              std::fmax(0.0, r0 - 40 * sr), r0 + 40 * sr, N_SIMPSON);
    double zt[2];
    for (int i = 0; i < 2; ++i) {
        const double t0 = theta0[i];
        zt[i] = simpson([&](double t) { return std::sin(t) * std::exp(-0.5 * k_theta * (t - t0) * (t - t0) / kT); },
                        std::fmax(0.0, t0 - 40 * st), std::fmin(M_PI, t0 + 40 * st), N_SIMPSON);
    }
    const double pm = std::fmin(M_PI, 40 * sp);
    const double zp = simpson([&](double p) { return std::exp(-k_phi * (1.0 - std::cos(p)) / kT); },
                              -pm, pm, N_SIMPSON);
    const double v0 = 1.0e24 / (6.02214076e23 * 1.0e3);   // nm^3 per molecule at 1 mol/L
    *dG = -kT * std::log(zr * zt[0] * zt[1] * zp * zp * zp / (8.0 * M_PI * M_PI * v0));
    return ABFE_OK;
}
