// Host-side parts of the C ABI: error reporting, the cloud sampler and the
// OF-MLMC estimator (Section 2.4 of the paper).  All FP64; compiled with
// -ffp-contract=off so the sampler's arithmetic rounds identically on x86 and
// Arm hosts.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ofmlmc.h"
#include "internal.h"

namespace ofm {

static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = '\0'; }

}  // namespace ofm

using namespace ofm;

extern "C" const char* ofm_last_error(void) { return g_err; }

extern "C" const char* ofm_version(void) { return "ofmlmc-gb300 1.0 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Cloud sampler.  SplitMix64 (Steele, Lea & Flood 2014): the state advances by
// the golden-ratio increment and each output is the state passed through two
// xor-shift-multiply rounds and a final xor-shift.
// ---------------------------------------------------------------------------
namespace {

struct SplitMix {
    uint64_t s;
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

}  // namespace

extern "C" int ofm_sample_cloud(const ofm_cloud_params* p, uint64_t seed, uint64_t sample_id,
                                ofm_bubble* out) {
    if (!p || !out) return fail(OFM_EINVAL, "ofm_sample_cloud: NULL argument");
    if (p->n_bubbles < 0 || !(p->cloud_radius >= 0.0) || !(p->r_min > 0.0) ||
        !(p->r_max >= p->r_min))
        return fail(OFM_EINVAL, "ofm_sample_cloud: bad cloud parameters");
    SplitMix g{seed ^ (sample_id * 0x9E3779B97F4A7C15ull)};
    const double R = p->cloud_radius;
    const double c = 0.5 * p->domain_L;
    for (int b = 0; b < p->n_bubbles; ++b) {
        double x, y, z;
        for (;;) {
            x = (2.0 * g.unit() - 1.0) * R;
            y = (2.0 * g.unit() - 1.0) * R;
            z = (2.0 * g.unit() - 1.0) * R;
            if (x * x + y * y + z * z <= R * R) break;
        }
        double r;
        if (p->radius_law == OFM_RADII_UNIFORM) {
            r = p->r_min + g.unit() * (p->r_max - p->r_min);
        } else {
            for (int tries = 0;; ++tries) {
                if (tries > 100000000) return fail(OFM_EINVAL, "ofm_sample_cloud: radius law never hits [r_min, r_max]");
                double u1 = g.unit();
                double u2 = g.unit();
                double n = std::sqrt(-2.0 * std::log(1.0 - u1)) * std::cos(2.0 * M_PI * u2);
                r = std::exp(p->ln_mu + p->ln_sigma * n);
                if (p->r_min <= r && r <= p->r_max) break;
            }
        }
        out[b].x = c + x;
        out[b].y = c + y;
        out[b].z = c + z;
        out[b].r = r;
    }
    return OFM_OK;
}

// ---------------------------------------------------------------------------
// Estimator (Section 2.4).
// ---------------------------------------------------------------------------
namespace {

double mean_of(const std::vector<double>& x) {
    double s = 0.0;
    for (double v : x) s += v;
    return s / (double)x.size();
}

double var_of(const std::vector<double>& x) {
    const double m = mean_of(x);
    double s = 0.0;
    for (double v : x) s += (v - m) * (v - m);
    return s / (double)(x.size() - 1);
}

double cov_of(const std::vector<double>& x, const std::vector<double>& y) {
    const double mx = mean_of(x), my = mean_of(y);
    double s = 0.0;
    for (size_t i = 0; i < x.size(); ++i) s += (x[i] - mx) * (y[i] - my);
    return s / (double)(x.size() - 1);
}

// Thomas algorithm for the symmetric tridiagonal system of Eq. (alpha-matvec):
// row l: -cov[l] W[l] a_{l-1} + sigma2[l] (W[l] + W[l+1]) a_l - cov[l+1] W[l+1] a_{l+1}
//        = (l == L-1) ? cov[L] W[L] : 0.
int solve_alpha(int L, const double* sigma2, const double* cov, const double* W, double* alpha) {
    alpha[L] = 1.0;
    if (L == 0) return OFM_OK;
    std::vector<double> a(L), b(L), c(L), d(L);
    for (int l = 0; l < L; ++l) {
        b[l] = sigma2[l] * (W[l + 1] + W[l]);
        a[l] = l > 0 ? -cov[l] * W[l] : 0.0;
        c[l] = l + 1 < L ? -cov[l + 1] * W[l + 1] : 0.0;
        d[l] = l == L - 1 ? cov[L] * W[L] : 0.0;
    }
    for (int l = 1; l < L; ++l) {
        if (b[l - 1] == 0.0) return fail(OFM_ENUMERIC, "ofm_estimate: singular coefficient system");
        const double m = a[l] / b[l - 1];
        b[l] -= m * c[l - 1];
        d[l] -= m * d[l - 1];
    }
    if (b[L - 1] == 0.0) return fail(OFM_ENUMERIC, "ofm_estimate: singular coefficient system");
    alpha[L - 1] = d[L - 1] / b[L - 1];
    for (int l = L - 2; l >= 0; --l) alpha[l] = (d[l] - c[l] * alpha[l + 1]) / b[l];
    return OFM_OK;
}

}  // namespace

namespace {

// Weighted least squares of ln V_l = a + b l over the levels l >= 1 with at
// least two pairs and V_l > 0, weights (M_l - 1)/2 (the inverse of the
// Gaussian error of ln V_l): the posterior mean of (a, b) under flat priors.
int fit_line(int L, const int64_t* M, const double* V, double* a, double* b) {
    double Sw = 0.0, Sx = 0.0, Sy = 0.0, Sxx = 0.0, Sxy = 0.0;
    int used = 0;
    for (int l = 1; l <= L; ++l) {
        if (M[l] < 2 || !(V[l] > 0.0) || !std::isfinite(V[l])) continue;
        const double w = 0.5 * (double)(M[l] - 1), x = (double)l, y = std::log(V[l]);
        Sw += w;
        Sx += w * x;
        Sy += w * y;
        Sxx += w * x * x;
        Sxy += w * x * y;
        ++used;
    }
    if (used < 2) return fail(OFM_EINVAL, "variance fit: needs two levels l >= 1 with at least two pairs");
    const double det = Sw * Sxx - Sx * Sx;
    *b = (Sw * Sxy - Sx * Sy) / det;
    *a = (Sy - *b * Sx) / Sw;
    return OFM_OK;
}

// Steps 3-5 and the estimator; fit = true replaces the covariances of
// Eq. (alpha-matvec) by (sigma2_l + sigma2_{l-1} - V_fit_l)/2.
int estimate_core(int L, const int64_t* M, const double* const* q, const double* W, ofm_estimate_out* out, bool fit,
                  double* V_fit_out) {
    const char* who = fit ? "ofm_estimate_fitted" : "ofm_estimate";
    if (L < 0 || L >= OFM_MAX_LEVELS || !M || !q || !W || !out) return fail(OFM_EINVAL, "%s: bad arguments", who);
    if (fit && L < 1) return fail(OFM_EINVAL, "%s: the fit needs L >= 1", who);
    for (int l = 0; l <= L; ++l) {
        const int64_t need = (fit && l > 0) ? 1 : 2;
        if (M[l] < need || !q[l]) return fail(OFM_EINVAL, "%s: level %d needs >= %lld samples", who, l, (long long)need);
        if (!(W[l] > 0.0)) return fail(OFM_EINVAL, "%s: W[%d] must be > 0", who, l);
    }
    std::memset(out, 0, sizeof(*out));
    std::vector<std::vector<double>> fine(L + 1), coarse(L + 1);
    for (int l = 0; l <= L; ++l) {
        fine[l].resize(M[l]);
        coarse[l].resize(M[l]);
        for (int64_t i = 0; i < M[l]; ++i) {
            fine[l][i] = q[l][2 * i];
            coarse[l][i] = q[l][2 * i + 1];
        }
    }
    for (int l = 0; l <= L; ++l) {
        std::vector<double> pooled = fine[l];
        if (l < L) pooled.insert(pooled.end(), coarse[l + 1].begin(), coarse[l + 1].end());
        // one computed q_l (the finest level's single warm-up pair): no sample variance exists
        out->sigma2[l] = pooled.size() >= 2 ? var_of(pooled) : out->sigma2[l - 1];
        out->cov[l] = (l > 0 && !fit) ? cov_of(fine[l], coarse[l]) : 0.0;
    }
    if (fit) {
        std::vector<double> V(L + 1, 0.0);
        for (int l = 1; l <= L; ++l) {
            if (M[l] < 2) continue;
            std::vector<double> d(M[l]);
            for (int64_t i = 0; i < M[l]; ++i) d[i] = fine[l][i] - coarse[l][i];
            V[l] = var_of(d);
        }
        double a = 0.0, b = 0.0;
        int rc = fit_line(L, M, V.data(), &a, &b);
        if (rc != OFM_OK) return rc;
        for (int l = 1; l <= L; ++l) {
            // clamped so that |Cov| <= sigma_l sigma_{l-1} (positive semi-definite second moments)
            const double sl = std::sqrt(out->sigma2[l]), sm = std::sqrt(out->sigma2[l - 1]);
            const double lo = (sl - sm) * (sl - sm), hi = (sl + sm) * (sl + sm);
            const double vf = std::min(std::max(std::exp(a + b * (double)l), lo), hi);
            out->cov[l] = 0.5 * (out->sigma2[l] + out->sigma2[l - 1] - vf);
            if (V_fit_out) V_fit_out[l] = vf;
        }
        if (V_fit_out) V_fit_out[0] = 0.0;
    }
    int rc = solve_alpha(L, out->sigma2, out->cov, W, out->alpha);
    if (rc != OFM_OK) return rc;
    double mean = 0.0, eps2 = 0.0;
    for (int l = 0; l <= L; ++l) {
        std::vector<double> d(M[l]);
        for (int64_t i = 0; i < M[l]; ++i)
            d[i] = l == 0 ? out->alpha[0] * fine[0][i]
                          : out->alpha[l] * fine[l][i] - out->alpha[l - 1] * coarse[l][i];
        if (M[l] >= 2)
            out->sigma_tilde2[l] = var_of(d);
        else  // from the fitted second moments
            out->sigma_tilde2[l] = out->alpha[l] * out->alpha[l] * out->sigma2[l] +
                                   out->alpha[l - 1] * out->alpha[l - 1] * out->sigma2[l - 1] -
                                   2.0 * out->alpha[l] * out->alpha[l - 1] * out->cov[l];
        mean += mean_of(d);
        eps2 += out->sigma_tilde2[l] / (double)M[l];
    }
    out->mean = mean;
    out->eps2 = eps2;
    return OFM_OK;
}

}  // namespace

extern "C" int ofm_estimate(int L, const int64_t* M, const double* const* q, const double* W,
                            ofm_estimate_out* out) {
    return estimate_core(L, M, q, W, out, false, nullptr);
}

extern "C" int ofm_estimate_fitted(int L, const int64_t* M, const double* const* q, const double* W,
                                   ofm_estimate_out* out, double* V_fit) {
    return estimate_core(L, M, q, W, out, true, V_fit);
}

extern "C" int ofm_fit_level_variances(int L, const int64_t* M, const double* V, double* V_fit, double* coef) {
    if (L < 1 || L >= OFM_MAX_LEVELS || !M || !V || !V_fit)
        return fail(OFM_EINVAL, "ofm_fit_level_variances: bad arguments");
    double a = 0.0, b = 0.0;
    int rc = fit_line(L, M, V, &a, &b);
    if (rc != OFM_OK) return rc;
    V_fit[0] = 0.0;
    for (int l = 1; l <= L; ++l) V_fit[l] = std::exp(a + b * (double)l);
    if (coef) {
        coef[0] = a;
        coef[1] = b;
    }
    return OFM_OK;
}

// Per-level summaries (Section 2.4 needs only means, pooled variances and the
// fine/coarse covariance); pairwise combination after Chan, Golub and LeVeque.
extern "C" int ofm_level_moments_of(const double* pairs, int64_t M, ofm_level_moments* out) {
    if (!out || M < 0 || (M > 0 && !pairs)) return fail(OFM_EINVAL, "ofm_level_moments_of: bad arguments");
    std::memset(out, 0, sizeof(*out));
    out->n = M;
    if (M == 0) return OFM_OK;
    double sf = 0.0, sc = 0.0;
    for (int64_t i = 0; i < M; ++i) {
        sf += pairs[2 * i];
        sc += pairs[2 * i + 1];
    }
    out->mean_f = sf / (double)M;
    out->mean_c = sc / (double)M;
    for (int64_t i = 0; i < M; ++i) {
        const double df = pairs[2 * i] - out->mean_f, dc = pairs[2 * i + 1] - out->mean_c;
        out->m2_f += df * df;
        out->m2_c += dc * dc;
        out->c_fc += df * dc;
    }
    return OFM_OK;
}

extern "C" int ofm_merge_moments(const ofm_level_moments* a, const ofm_level_moments* b, ofm_level_moments* out) {
    if (!a || !b || !out || a->n < 0 || b->n < 0) return fail(OFM_EINVAL, "ofm_merge_moments: bad arguments");
    const ofm_level_moments x = *a, y = *b;
    if (x.n == 0) {
        *out = y;
        return OFM_OK;
    }
    if (y.n == 0) {
        *out = x;
        return OFM_OK;
    }
    const double n = (double)(x.n + y.n);
    const double df = y.mean_f - x.mean_f, dc = y.mean_c - x.mean_c;
    const double w = (double)x.n * (double)y.n / n;
    out->n = x.n + y.n;
    out->mean_f = x.mean_f + df * (double)y.n / n;
    out->mean_c = x.mean_c + dc * (double)y.n / n;
    out->m2_f = x.m2_f + y.m2_f + df * df * w;
    out->m2_c = x.m2_c + y.m2_c + dc * dc * w;
    out->c_fc = x.c_fc + y.c_fc + df * dc * w;
    return OFM_OK;
}

namespace {

// ofm_estimate_moments, with or without step 3's fit (as estimate_core).
int estimate_moments_core(int L, const ofm_level_moments* m, const double* W, ofm_estimate_out* out, bool fit,
                          double* V_fit_out) {
    const char* who = fit ? "ofm_estimate_moments_fitted" : "ofm_estimate_moments";
    if (L < 0 || L >= OFM_MAX_LEVELS || !m || !W || !out) return fail(OFM_EINVAL, "%s: bad arguments", who);
    if (fit && L < 1) return fail(OFM_EINVAL, "%s: the fit needs L >= 1", who);
    for (int l = 0; l <= L; ++l) {
        const int64_t need = (fit && l > 0) ? 1 : 2;
        if (m[l].n < need) return fail(OFM_EINVAL, "%s: level %d needs >= %lld samples", who, l, (long long)need);
        if (!(W[l] > 0.0)) return fail(OFM_EINVAL, "%s: W[%d] must be > 0", who, l);
    }
    std::memset(out, 0, sizeof(*out));
    for (int l = 0; l <= L; ++l) {
        // pooled: fine members of pair l with the coarse members of pair l+1
        ofm_level_moments pooled{m[l].n, m[l].mean_f, 0.0, m[l].m2_f, 0.0, 0.0};
        if (l < L) {
            const ofm_level_moments up{m[l + 1].n, m[l + 1].mean_c, 0.0, m[l + 1].m2_c, 0.0, 0.0};
            ofm_merge_moments(&pooled, &up, &pooled);
        }
        out->sigma2[l] = pooled.n >= 2 ? pooled.m2_f / (double)(pooled.n - 1) : out->sigma2[l - 1];
        out->cov[l] = (l > 0 && !fit) ? m[l].c_fc / (double)(m[l].n - 1) : 0.0;
    }
    if (fit) {
        int64_t M[OFM_MAX_LEVELS];
        double V[OFM_MAX_LEVELS];
        for (int l = 0; l <= L; ++l) {
            M[l] = m[l].n;
            // V[q_l - q_{l-1}] from the co-moments of pair l
            V[l] = (l > 0 && m[l].n >= 2) ? (m[l].m2_f + m[l].m2_c - 2.0 * m[l].c_fc) / (double)(m[l].n - 1) : 0.0;
        }
        double a = 0.0, b = 0.0;
        int rc = fit_line(L, M, V, &a, &b);
        if (rc != OFM_OK) return rc;
        for (int l = 1; l <= L; ++l) {
            const double sl = std::sqrt(out->sigma2[l]), sm = std::sqrt(out->sigma2[l - 1]);
            const double lo = (sl - sm) * (sl - sm), hi = (sl + sm) * (sl + sm);
            const double vf = std::min(std::max(std::exp(a + b * (double)l), lo), hi);
            out->cov[l] = 0.5 * (out->sigma2[l] + out->sigma2[l - 1] - vf);
            if (V_fit_out) V_fit_out[l] = vf;
        }
        if (V_fit_out) V_fit_out[0] = 0.0;
    }
    int rc = solve_alpha(L, out->sigma2, out->cov, W, out->alpha);
    if (rc != OFM_OK) return rc;
    double mean = 0.0, eps2 = 0.0;
    for (int l = 0; l <= L; ++l) {
        const double n1 = (double)(m[l].n - 1), a = out->alpha[l];
        if (l == 0) {
            out->sigma_tilde2[0] = a * a * m[0].m2_f / n1;
            mean += a * m[0].mean_f;
        } else {
            const double b = out->alpha[l - 1];
            if (m[l].n >= 2)
                out->sigma_tilde2[l] = (a * a * m[l].m2_f + b * b * m[l].m2_c - 2.0 * a * b * m[l].c_fc) / n1;
            else  // from the fitted second moments
                out->sigma_tilde2[l] = a * a * out->sigma2[l] + b * b * out->sigma2[l - 1] - 2.0 * a * b * out->cov[l];
            mean += a * m[l].mean_f - b * m[l].mean_c;
        }
        eps2 += out->sigma_tilde2[l] / (double)m[l].n;
    }
    out->mean = mean;
    out->eps2 = eps2;
    return OFM_OK;
}

}  // namespace

extern "C" int ofm_estimate_moments(int L, const ofm_level_moments* m, const double* W, ofm_estimate_out* out) {
    return estimate_moments_core(L, m, W, out, false, nullptr);
}

extern "C" int ofm_estimate_moments_fitted(int L, const ofm_level_moments* m, const double* W, ofm_estimate_out* out,
                                           double* V_fit) {
    return estimate_moments_core(L, m, W, out, true, V_fit);
}

extern "C" int ofm_warmup_samples(int L, const double* W, int64_t* M_out) {
    if (L < 0 || L >= OFM_MAX_LEVELS || !W || !M_out) return fail(OFM_EINVAL, "ofm_warmup_samples: bad arguments");
    for (int l = 0; l <= L; ++l) {
        if (!(W[l] > 0.0)) return fail(OFM_EINVAL, "ofm_warmup_samples: W[%d] must be > 0", l);
        M_out[l] = (int64_t)std::ceil(W[L] / W[l] / std::ldexp(1.0, L - l));
    }
    return OFM_OK;
}

extern "C" int ofm_optimal_samples(int L, const double* st2, const double* W, const int64_t* M_done,
                                   double target, int mode, int64_t* M_out) {
    if (L < 0 || L >= OFM_MAX_LEVELS || !st2 || !W || !M_out || !(target > 0.0) ||
        (mode != OFM_MODE_TOL && mode != OFM_MODE_BUDGET))
        return fail(OFM_EINVAL, "ofm_optimal_samples: bad arguments");
    const int n = L + 1;
    for (int l = 0; l < n; ++l)
        if (!(st2[l] >= 0.0) || !std::isfinite(st2[l]) || !(W[l] > 0.0))
            return fail(OFM_EINVAL, "ofm_optimal_samples: sigma_tilde2[%d] or W[%d] is not a finite positive value", l,
                        l);
    bool fixed[OFM_MAX_LEVELS] = {false};
    for (;;) {
        double rem = mode == OFM_MODE_TOL ? target * target : target;
        double total = 0.0;
        for (int l = 0; l < n; ++l) {
            if (fixed[l])
                rem -= mode == OFM_MODE_TOL ? st2[l] / (double)M_done[l] : (double)M_done[l] * W[l];
            else
                total += std::sqrt(st2[l] * W[l]);
        }
        if (!(rem > 0.0))
            return fail(OFM_EINVAL, "ofm_optimal_samples: target already consumed by kept samples");
        const double t = mode == OFM_MODE_TOL ? std::sqrt(rem) : rem;
        if (total == 0.0) {  // no sampling variance left on the free levels: they need no samples
            for (int l = 0; l < n; ++l) M_out[l] = fixed[l] ? M_done[l] : (M_done ? M_done[l] : 0);
            return OFM_OK;
        }
        bool newly = false;
        for (int l = 0; l < n; ++l) {
            if (fixed[l]) {
                M_out[l] = M_done[l];
                continue;
            }
            double raw = mode == OFM_MODE_TOL ? (1.0 / (t * t)) * std::sqrt(st2[l] / W[l]) * total
                                              : t * std::sqrt(st2[l] / W[l]) / total;
            if (!(raw < 4.0e18))
                return fail(OFM_EINVAL, "ofm_optimal_samples: level %d needs more than 4e18 samples", l);
            M_out[l] = (int64_t)std::ceil(raw);
            if (M_done && M_out[l] < M_done[l]) {
                fixed[l] = true;
                newly = true;
            }
        }
        if (!newly) {
            for (int l = 0; l < n; ++l)
                if (fixed[l]) M_out[l] = M_done[l];
            return OFM_OK;
        }
    }
}

// OF-MLMC with the surrogate of q_L as an extra control variate of the top
// level term (not in the paper): g = h - alpha_{L-1} q_{L-1}, added with
// coefficient beta to the level-(L-1) terms (h on their fine inputs) and
// subtracted from the level-L terms (h on their coarse inputs).  Unbiased for
// fixed alpha and beta; beta minimises sum_l sigma~^2_l / M_l.
extern "C" int ofm_estimate_surrogate(int L, const int64_t* M, const double* const* q, const double* W,
                                      const double* h_top, const double* h_extra, double beta_in,
                                      ofm_estimate_out* out, double* beta_out, double* sigma_tilde2_plain) {
    if (L < 1 || L >= OFM_MAX_LEVELS || !M || !q || !W || !h_top || !h_extra || !out || !beta_out)
        return fail(OFM_EINVAL, "ofm_estimate_surrogate: bad arguments (needs L >= 1)");
    int rc = estimate_core(L, M, q, W, out, false, nullptr);
    if (rc != OFM_OK) return rc;
    if (sigma_tilde2_plain)
        for (int l = 0; l <= L; ++l) sigma_tilde2_plain[l] = out->sigma_tilde2[l];
    const double* al = out->alpha;
    auto term = [&](int l, int64_t i) {
        return l == 0 ? al[0] * q[0][2 * i] : al[l] * q[l][2 * i] - al[l - 1] * q[l][2 * i + 1];
    };
    const int64_t ML = M[L], Mm = M[L - 1];
    std::vector<double> DL(ML), gL(ML), Dm(Mm), gm(Mm);
    for (int64_t i = 0; i < ML; ++i) {
        DL[i] = term(L, i);
        gL[i] = h_top[i] - al[L - 1] * q[L][2 * i + 1];
    }
    for (int64_t j = 0; j < Mm; ++j) {
        Dm[j] = term(L - 1, j);
        gm[j] = h_extra[j] - al[L - 1] * q[L - 1][2 * j];
    }
    double beta = beta_in;
    if (std::isnan(beta_in)) {
        const double den = var_of(gm) / (double)Mm + var_of(gL) / (double)ML;
        const double num = cov_of(DL, gL) / (double)ML - cov_of(Dm, gm) / (double)Mm;
        beta = den > 0.0 ? num / den : 0.0;
    }
    for (int64_t i = 0; i < ML; ++i) DL[i] -= beta * gL[i];
    for (int64_t j = 0; j < Mm; ++j) Dm[j] += beta * gm[j];
    out->sigma_tilde2[L] = var_of(DL);
    out->sigma_tilde2[L - 1] = var_of(Dm);
    double mean = 0.0, e2 = 0.0;
    for (int l = 0; l <= L; ++l) {
        double m;
        if (l == L)
            m = mean_of(DL);
        else if (l == L - 1)
            m = mean_of(Dm);
        else {
            std::vector<double> d(M[l]);
            for (int64_t i = 0; i < M[l]; ++i) d[i] = term(l, i);
            m = mean_of(d);
        }
        mean += m;
        e2 += out->sigma_tilde2[l] / (double)M[l];
    }
    out->mean = mean;
    out->eps2 = e2;
    *beta_out = beta;
    return OFM_OK;
}

extern "C" int ofm_surrogate_cv(const double* D, const double* s_paired, int64_t M, const double* s_extra, int64_t N,
                                double* beta, double* corrected_mean, double* variance) {
    if (!D || !s_paired || !s_extra || M < 2 || N < 1 || !beta || !corrected_mean || !variance)
        return fail(OFM_EINVAL, "ofm_surrogate_cv: bad arguments");
    std::vector<double> d(D, D + M), sp(s_paired, s_paired + M), se(s_extra, s_extra + N);
    const double vs = var_of(sp);
    const double c = cov_of(d, sp);
    const double f = 1.0 + (double)M / (double)N;
    const double b = vs > 0.0 ? c / (vs * f) : 0.0;
    *beta = b;
    *corrected_mean = mean_of(d) + b * (mean_of(se) - mean_of(sp));
    *variance = vs > 0.0 ? (var_of(d) - c * c / (vs * f)) / (double)M : var_of(d) / (double)M;
    return OFM_OK;
}

// ---------------------------------------------------------------------------
// Level-wise kernel density estimate (Section 3.2): the OF-MLMC estimator of
// E[K_b(x - q)] with a Gaussian kernel, each level's pairs with one
// bandwidth, the larger of its two members' solve-the-equation bandwidths
// (Sheather and Jones 1991).
// ---------------------------------------------------------------------------
namespace {

constexpr double kSqrt2Pi = 2.5066282746310002;

// r-th derivative (r = 4 or 6) of the standard normal density: phi(u) He_r(u).
double phi_deriv(double u, int r) {
    const double phi = std::exp(-0.5 * u * u) / kSqrt2Pi, u2 = u * u;
    return r == 4 ? phi * (u2 * u2 - 6.0 * u2 + 3.0) : phi * (u2 * u2 * u2 - 15.0 * u2 * u2 + 45.0 * u2 - 15.0);
}

// psi_r = int f^(r) f estimated with bandwidth g, the pairs i = j left out.
double psi_hat(const std::vector<double>& x, int r, double g) {
    const size_t n = x.size();
    double tot = 0.0;
    for (size_t i = 0; i < n; ++i)
        for (size_t j = i + 1; j < n; ++j) tot += phi_deriv((x[i] - x[j]) / g, r);
    return 2.0 * tot / ((double)n * (double)(n - 1) * std::pow(g, (double)(r + 1)));
}

// Percentile with linear interpolation between order statistics.
double percentile(std::vector<double> v, double p) {
    std::sort(v.begin(), v.end());
    const double pos = p / 100.0 * (double)(v.size() - 1);
    const size_t lo = (size_t)std::floor(pos), hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

double sj_bandwidth(const std::vector<double>& x) {
    const double n = (double)x.size();
    const double sd = std::sqrt(var_of(x));
    const double iqr = (percentile(x, 75.0) - percentile(x, 25.0)) / 1.349;
    const double s = iqr > 0.0 ? std::min(sd, iqr) : sd;
    if (!(s > 0.0)) return 0.0;
    const double rk = 1.0 / (2.0 * std::sqrt(M_PI)), k4 = 3.0 / kSqrt2Pi, k6 = -15.0 / kSqrt2Pi;
    // normal-reference pilots for psi_4 and psi_6
    const double psi6n = -15.0 / (16.0 * std::sqrt(M_PI) * std::pow(s, 7.0));
    const double psi8n = 105.0 / (32.0 * std::sqrt(M_PI) * std::pow(s, 9.0));
    const double a = std::pow(-2.0 * k4 / (psi6n * n), 1.0 / 7.0);
    const double b = std::pow(-2.0 * k6 / (psi8n * n), 1.0 / 9.0);
    // psi_4 > 0 > psi_6 for any smooth density; a pilot estimate of the wrong sign
    // (possible for a small sample) takes its normal-reference value
    double p4a = psi_hat(x, 4, a), p6b = psi_hat(x, 6, b);
    if (!(p4a > 0.0)) p4a = 3.0 / (8.0 * std::sqrt(M_PI) * std::pow(s, 5.0));
    if (!(p6b < 0.0)) p6b = psi6n;
    const double c_g = std::pow(2.0 * k4 / rk * (p4a / -p6b), 1.0 / 7.0);
    auto f = [&](double h) -> double {
        const double p4 = psi_hat(x, 4, c_g * std::pow(h, 5.0 / 7.0));
        if (!(p4 > 0.0)) return HUGE_VAL;   // the pilot resolves no curvature: h is too small
        return std::pow(rk / (n * p4), 0.2) - h;
    };
    const double h0 = std::pow(4.0 / (3.0 * n), 0.2) * s;
    double lo = h0, hi = h0;
    for (int k = 0; k < 200 && f(hi) > 0.0; ++k) hi *= 2.0;
    for (int k = 0; k < 200 && f(lo) < 0.0; ++k) lo *= 0.5;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (f(mid) > 0.0)
            lo = mid;
        else
            hi = mid;
        if (hi - lo <= 1e-10 * hi) break;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

extern "C" int ofm_sj_bandwidth(const double* x, int64_t n, double* h) {
    if (!x || !h || n < 2) return fail(OFM_EINVAL, "ofm_sj_bandwidth: needs n >= 2 samples");
    *h = sj_bandwidth(std::vector<double>(x, x + n));
    return OFM_OK;
}

extern "C" int ofm_level_kde(int L, const int64_t* M, const double* const* q, const double* alpha, const double* x,
                             int64_t n_x, double* density, double* bandwidth) {
    if (L < 0 || L >= OFM_MAX_LEVELS || !M || !q || !alpha || !x || n_x < 0 || !density)
        return fail(OFM_EINVAL, "ofm_level_kde: bad arguments");
    for (int l = 0; l <= L; ++l)
        if (M[l] < 2 || !q[l]) return fail(OFM_EINVAL, "ofm_level_kde: level %d needs >= 2 pairs", l);
    for (int64_t k = 0; k < n_x; ++k) density[k] = 0.0;
    for (int l = 0; l <= L; ++l) {
        std::vector<double> fine(M[l]), coarse(M[l]);
        for (int64_t i = 0; i < M[l]; ++i) {
            fine[i] = q[l][2 * i];
            coarse[i] = q[l][2 * i + 1];
        }
        double b = sj_bandwidth(fine);
        if (l > 0) b = std::max(b, sj_bandwidth(coarse));
        if (bandwidth) bandwidth[l] = b;
        if (!(b > 0.0)) return fail(OFM_ENUMERIC, "ofm_level_kde: level %d has no spread", l);
        const double wf = alpha[l] / ((double)M[l] * b * kSqrt2Pi);
        const double wc = l > 0 ? alpha[l - 1] / ((double)M[l] * b * kSqrt2Pi) : 0.0;
        for (int64_t k = 0; k < n_x; ++k) {
            double sf = 0.0, sc = 0.0;
            for (int64_t i = 0; i < M[l]; ++i) {
                const double uf = (x[k] - fine[i]) / b;
                sf += std::exp(-0.5 * uf * uf);
                if (l > 0) {
                    const double uc = (x[k] - coarse[i]) / b;
                    sc += std::exp(-0.5 * uc * uc);
                }
            }
            density[k] += wf * sf - wc * sc;
        }
    }
    return OFM_OK;
}
