// qrs_hyper.cu -- host-side choice of the hyper-parameter N (Sec. 4.2).
//
// g(x) = int_0^x f W(f) A(f)^2 df for the isotropic von Karman PSD W (A the
// Eq. 7 aperture filter when the PSD carries one, else 1).  N = 2 m for the
// first m past the largest panel increment (g rises, then saturates) with
// g(m df) - g((m-1) df) < eps_rel g_inf.  Each panel is
// integrated by composite Simpson's rule; g_inf adds geometrically widening
// panels beyond the scan until the integrand has decayed (W ~ f^-11/3).
#include <cmath>
#include <cstdio>

#include "../../include/qrs.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kSimpson = 64;  // sub-intervals per panel (even)

double vk_c() { return std::pow(std::tgamma(11.0 / 6.0), 2.0) / (2.0 * std::pow(kPi, 11.0 / 3.0)) *
                       std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0); }

struct Integrand {
    double c, a, D, d;
    double operator()(double f) const
    {
        double w = c * std::pow(f * f + a, -11.0 / 6.0);
        if (D > 0.0 && f > 0.0) {
            const double xD = kPi * D * f, xd = kPi * d * f;
            const double A = 2.0 * (D * ::j1(xD) - (d > 0.0 ? d * ::j1(xd) : 0.0)) / (kPi * (D * D - d * d) * f);
            w *= A * A;
        }
        return f * w;
    }
};

double simpson(const Integrand& g, double a, double b)
{
    const double h = (b - a) / kSimpson;
    double s = g(a) + g(b);
    for (int i = 1; i < kSimpson; ++i) s += g(a + i * h) * ((i & 1) ? 4.0 : 2.0);
    return s * h / 3.0;
}

}  // namespace

extern "C" qrs_status qrs_choose_n(const qrs_psd* psd, double delta_f, double eps_rel, int32_t n_max, int32_t* n_out,
                                   double* g_out)
{
    if (!psd || !n_out) return QRS_ERR_ARG;
    if (psd->kind != QRS_PSD_VON_KARMAN || !(psd->r0_m > 0.0) || !(psd->L0_m > 0.0)) return QRS_ERR_ARG;
    if (!(delta_f > 0.0) || !(eps_rel > 0.0) || n_max < 2) return QRS_ERR_ARG;
    if (!(psd->ap_D_m >= 0.0) || !(psd->ap_d_m >= 0.0) || (psd->ap_D_m > 0.0 && !(psd->ap_d_m < psd->ap_D_m)))
        return QRS_ERR_ARG;
    const Integrand g{vk_c() * std::pow(psd->r0_m, -5.0 / 3.0), 1.0 / (psd->L0_m * psd->L0_m), psd->ap_D_m,
                      psd->ap_d_m};
    const int64_t m_max = n_max / 2;
    // g_inf: uniform panels over the scan range, then geometric panels
    double g_scan = 0.0;
    for (int64_t m = 1; m <= m_max; ++m) g_scan += simpson(g, (m - 1) * delta_f, m * delta_f);
    double g_inf = g_scan, x = m_max * delta_f;
    for (int k = 0; k < 400 && x < 1e9; ++k) {
        const double x1 = x * 1.25;
        g_inf += simpson(g, x, x1);
        x = x1;
    }
    double gm = 0.0, peak = 0.0;
    for (int64_t m = 1; m <= m_max; ++m) {
        const double inc = simpson(g, (m - 1) * delta_f, m * delta_f);
        gm += inc;
        if (inc < eps_rel * g_inf && inc < peak) {  // on the saturating side of g
            *n_out = (int32_t)(2 * m);
            if (g_out) {
                g_out[0] = gm;
                g_out[1] = g_inf;
                g_out[2] = inc;
            }
            return QRS_OK;
        }
        if (inc > peak) peak = inc;
    }
    return QRS_ERR_ARG;
}
