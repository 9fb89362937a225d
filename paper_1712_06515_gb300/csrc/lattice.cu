// Parameter-space metric and cubic template lattice (Sec. III A: Eqs.
// phase-derivs-metric, metric-spacing-eq).  Host code: the metric is an average over the
// statistic's pairs of products of phase derivatives, computed once per search set-up.
//
// g_ij = 1/2 < d(Phi_K - Phi_L)/d lambda^i d(Phi_K - Phi_L)/d lambda^j > over the pairs of the
// detector-frame statistic (SFT mid-times (k + 1/2) T_sft of an unbroken run, every
// unordered pair of distinct SFTs of the Q detectors within T_max; same-time pairs of two
// detectors have zero phase difference), lambda = (a_p, T_asc, P) of a circular orbit,
// Phi = 2 pi f (t_SSB - a_p sin(Omega (t_SSB - T_asc))).  The lattice spacing per dimension
// is sqrt(mu / g_ii).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

void phase_derivs(double t, double f, double a_p, double tasc, double P, double d[3]) {
    const double Om = 2.0 * M_PI / P;
    const double psi = Om * (t - tasc);
    const double c = std::cos(psi);
    d[0] = -2.0 * M_PI * f * std::sin(psi);
    d[1] = 2.0 * M_PI * f * a_p * Om * c;
    d[2] = 2.0 * M_PI * f * a_p * Om * (t - tasc) * c / P;
}

}  // namespace

extern "C" cc_status crosscorr_metric(double T_obs, double T_sft, double T_max, int32_t Q, double f,
                                      const cc_template* orbit, double t0, double* g) {
    using cc::fail;
    if (!orbit || !g) return fail(CC_ERR_INVALID, "null argument to crosscorr_metric");
    if (!(T_obs > 0) || !(T_sft > 0) || !(T_max >= 0) || Q < 1 || Q > CC_MAX_DET || !(f > 0) ||
        !(orbit->P > 0) || !std::isfinite(T_obs + T_sft + T_max + f + orbit->a_p + orbit->T_asc + t0))
        return fail(CC_ERR_INVALID, "T_obs, T_sft, f, P > 0, T_max >= 0, 1 <= Q <= 4, finite values");
    if (orbit->e != 0.0) return fail(CC_ERR_UNSUPPORTED, "the metric is written for circular orbits");
    const int64_t n = (int64_t)std::floor(T_obs / T_sft);
    if (n < 2) return fail(CC_ERR_INVALID, "fewer than two SFTs");
    const int64_t Rs = (int64_t)std::floor(T_max / T_sft + 1e-9);
    const double tasc = orbit->T_asc - t0;
    std::vector<double> d((size_t)n * 3);
    for (int64_t k = 0; k < n; ++k) phase_derivs((k + 0.5) * T_sft, f, orbit->a_p, tasc, orbit->P, &d[3 * k]);
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double npairs = 0.0;
    for (int64_t lag = 0; lag <= Rs && lag < n; ++lag) {
        const double mult = lag == 0 ? 0.5 * Q * (Q - 1) : (double)Q * Q;
        if (mult == 0.0) continue;
        double sl[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t k = 0; k + lag < n; ++k) {
            double dd[3];
            for (int i = 0; i < 3; ++i) dd[i] = d[3 * k + i] - d[3 * (k + lag) + i];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) sl[3 * i + j] += dd[i] * dd[j];
        }
        for (int i = 0; i < 9; ++i) s[i] += mult * sl[i];
        npairs += mult * (double)(n - lag);
    }
    for (int i = 0; i < 9; ++i) g[i] = 0.5 * s[i] / npairs;
    return CC_OK;
}

extern "C" cc_status crosscorr_lattice(const double* g, double mu, const double* lo, const double* hi,
                                       cc_template* out, int64_t capacity, int64_t* n_out) {
    using cc::fail;
    if (!g || !lo || !hi || !n_out) return fail(CC_ERR_INVALID, "null argument to crosscorr_lattice");
    if (!(mu > 0) || !std::isfinite(mu)) return fail(CC_ERR_INVALID, "mu must be positive");
    std::vector<double> axes[3];
    for (int i = 0; i < 3; ++i) {
        if (!(g[4 * i] > 0) || !(hi[i] >= lo[i]) || !std::isfinite(lo[i] + hi[i]))
            return fail(CC_ERR_INVALID, "g_ii > 0 and lo <= hi required");
        const double dl = std::sqrt(mu / g[4 * i]);
        const int64_t n = (int64_t)std::floor((hi[i] - lo[i]) / dl + 1e-9) + 1;
        if (n > 100000000) return fail(CC_ERR_INVALID, "lattice axis longer than 1e8 points");
        for (int64_t k = 0; k < n; ++k) axes[i].push_back(lo[i] + dl * (double)k);
        if (axes[i].back() < hi[i] - 1e-12 * std::fmax(1.0, std::fabs(hi[i]))) axes[i].push_back(lo[i] + dl * (double)n);
    }
    const int64_t total = (int64_t)axes[0].size() * (int64_t)axes[1].size() * (int64_t)axes[2].size();
    *n_out = total;
    if (!out) return CC_OK;   // size query
    if (capacity < total) return fail(CC_ERR_INVALID, "output capacity below the lattice size");
    int64_t w = 0;
    for (double a : axes[0])
        for (double t : axes[1])
            for (double P : axes[2]) out[w++] = cc_template{a, t, P, 0.0, 0.0};
    return CC_OK;
}
