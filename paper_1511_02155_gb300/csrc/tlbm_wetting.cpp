// tlbm_wetting.cpp -- host-side wetting theory of the model: contact angles from
// the wetting parameters h_m, and h_m from target contact angles.
//
// Solid-fluid tension (Sec. Surface Thermodynamics): gamma_sm = I_m + sum_{n != m} J_n,
// with I_m the majority-phase and J_n the minority-phase contribution of each
// component.  Writing E_j = I_j - J_j, the differences that enter Young's
// equation are gamma_sn - gamma_sm = E_n - E_m, and evaluating I_j and J_j at the
// wall roots C_max = (1 + sqrt(1 + 4h/(alpha kappa)))/2 and
// C_min = (1 - sqrt(1 - 4h/(alpha kappa)))/2 gives E_j = -D_j / 12 with
//
//   D_j = [(alpha kappa_j + 4 h_j)^{3/2} - (alpha kappa_j - 4 h_j)^{3/2}] / sqrt(alpha kappa_j).
//
// With gamma_mn = alpha (kappa_m + kappa_n)/6 (Eq. SurfTens), Young's equation
// (Eq. contact angle) becomes
//
//   cos theta_mn = (D_m - D_n) / (2 alpha (kappa_m + kappa_n)),
//
// theta_mn measured through fluid m.  The printed closed form (Eq. invertCA)
// has the opposite sign and lacks the 1/alpha; the form above is the one that
// follows from I_m, J_n and Young's equation as printed.
//
// D_j grows monotonically with h_j on the admissible range |4 h_j| < alpha kappa_j,
// so the inversion is a pair of nested bisections: for a trial D_1 the targets
// fix D_2 and D_3, each D_j gives h_j, and D_1 moves until the gauge
// sum_m h_m / kappa_m = 0 (Eq. Redundancy, zero wall-normal density gradient) holds.
#include <cmath>

#include "../../include/tlbm.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

double D_of_h(double ak, double h) {
    const double a = ak + 4.0 * h, b = ak - 4.0 * h;
    return (a * std::sqrt(a) - b * std::sqrt(b)) / std::sqrt(ak);
}

// largest |D| on the admissible range (h = +-alpha kappa / 4): 2 sqrt(2) alpha kappa
double D_max(double ak) { return 2.0 * std::sqrt(2.0) * ak; }

// h with D_of_h(ak, h) = D, |D| < D_max(ak); bisection to the last bit
double h_of_D(double ak, double D) {
    double lo = -0.25 * ak, hi = 0.25 * ak;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (D_of_h(ak, mid) < D) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

bool args_ok(const double kappa[3], double alpha) {
    if (!kappa || !(alpha > 0) || !std::isfinite(alpha)) return false;
    for (int m = 0; m < 3; ++m)
        if (!(kappa[m] > 0) || !std::isfinite(kappa[m])) return false;
    return true;
}

double clamp1(double c) { return c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c); }

}  // namespace

extern "C" tlbm_status tlbm_contact_angles(const double kappa[3], double alpha, const double h[3],
                                           double theta_deg[3]) {
    if (!args_ok(kappa, alpha) || !h || !theta_deg) return TLBM_ERR_ARG;
    double D[3];
    for (int m = 0; m < 3; ++m) {
        const double ak = alpha * kappa[m];
        if (!std::isfinite(h[m]) || !(std::fabs(4.0 * h[m]) < ak)) return TLBM_ERR_PARAM;
        D[m] = D_of_h(ak, h[m]);
    }
    const int pair[3][2] = {{0, 1}, {1, 2}, {2, 0}};  // theta_12, theta_23, theta_31
    for (int k = 0; k < 3; ++k) {
        const int m = pair[k][0], n = pair[k][1];
        const double c = (D[m] - D[n]) / (2.0 * alpha * (kappa[m] + kappa[n]));
        // |c| <= 1 holds on the admissible range up to rounding
        theta_deg[k] = std::acos(clamp1(c)) * 180.0 / kPi;
    }
    return TLBM_OK;
}

extern "C" tlbm_status tlbm_wetting_from_angles(const double kappa[3], double alpha, double theta12_deg,
                                                double theta13_deg, double h[3]) {
    if (!args_ok(kappa, alpha) || !h) return TLBM_ERR_ARG;
    if (!(theta12_deg > 0 && theta12_deg < 180) || !(theta13_deg > 0 && theta13_deg < 180)) return TLBM_ERR_ARG;
    const double k1 = kappa[0], k2 = kappa[1], k3 = kappa[2];
    const double c12 = std::cos(theta12_deg * kPi / 180.0), c13 = std::cos(theta13_deg * kPi / 180.0);
    // Girifalco-Good: gamma_12 cos theta_12 + gamma_23 cos theta_23 + gamma_31 cos theta_31 = 0,
    // with theta_31 = 180 - theta_13; the third angle must exist
    const double c23 = ((k1 + k3) * c13 - (k1 + k2) * c12) / (k2 + k3);
    if (!(std::fabs(c23) < 1.0)) return TLBM_ERR_PARAM;
    // D_1 - D_2 = 2 alpha (k1 + k2) cos theta_12,  D_1 - D_3 = 2 alpha (k1 + k3) cos theta_13
    const double d12 = 2.0 * alpha * (k1 + k2) * c12, d13 = 2.0 * alpha * (k1 + k3) * c13;
    const double a1 = alpha * k1, a2 = alpha * k2, a3 = alpha * k3;
    double lo = std::fmax(-D_max(a1), std::fmax(d12 - D_max(a2), d13 - D_max(a3)));
    double hi = std::fmin(D_max(a1), std::fmin(d12 + D_max(a2), d13 + D_max(a3)));
    if (!(lo < hi)) return TLBM_ERR_PARAM;
    auto gauge = [&](double D1, double out[3]) {
        out[0] = h_of_D(a1, D1);
        out[1] = h_of_D(a2, D1 - d12);
        out[2] = h_of_D(a3, D1 - d13);
        return out[0] / k1 + out[1] / k2 + out[2] / k3;  // increasing in D1
    };
    double t[3];
    if (gauge(lo, t) > 0.0 || gauge(hi, t) < 0.0) return TLBM_ERR_PARAM;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (gauge(mid, t) < 0.0) lo = mid;
        else hi = mid;
    }
    gauge(0.5 * (lo + hi), t);
    for (int m = 0; m < 3; ++m)
        if (!(std::fabs(4.0 * t[m]) < alpha * kappa[m])) return TLBM_ERR_PARAM;  // at the edge of the range
    // the targets must come back (they do unless the solution sits at the range's edge)
    double th[3];
    if (tlbm_contact_angles(kappa, alpha, t, th) != TLBM_OK) return TLBM_ERR_PARAM;
    if (std::fabs(th[0] - theta12_deg) > 1e-6 || std::fabs((180.0 - th[2]) - theta13_deg) > 1e-6)
        return TLBM_ERR_PARAM;
    for (int m = 0; m < 3; ++m) h[m] = t[m];
    return TLBM_OK;
}
