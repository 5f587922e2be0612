// Adaptive OF-MLMC driver over batched GPU solves (Section 2.4.3, steps 1-8).
//
// Each iteration solves every level's new sample pairs in one uneven batch
// (fine and coarse members of a pair share their random input, Section 2.4.1):
// group (N_l, new ids) for the fine members and (N_{l-1}, new ids) for the
// coarse members of level l >= 1, split into several batches only when the
// batch would exceed the memory cap.  Pair costs W_l are the measured mean
// cell-steps of a pair (one sample at l = 0), proportional to device time for
// this kernel.  Pairs with a failed member are excluded (fault-tolerant MLMC).
// Sample id of pair i on level l: (l << 40) | i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "ofmlmc.h"

using ofm::fail;

namespace {

constexpr uint64_t ID_SHIFT = 40;

double qoi_value(const ofm_qoi& q, int which) {
    return which == 0 ? q.p_peak : q.sensor_peak[which - 1];
}

struct LevelData {
    std::vector<double> fine, coarse;  // per computed pair
    std::vector<char> ok;
    double cell_steps = 0.0;           // summed over its pairs
    int64_t computed = 0;              // pairs solved so far (ok or not)
};

// Solve pairs [from[l], to[l]) of every level in as few batches as the memory cap allows.
int solve_pairs(ofm_solver* s, const ofm_cloud_params* cloud, const ofm_run_config* rc, const int64_t* from,
                const int64_t* to, std::vector<LevelData>& lv, double* gpu_ms, cudaStream_t st, size_t cap) {
    const int L = rc->L;
    std::vector<int64_t> lo(from, from + L + 1);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(OFM_ECUDA, "ofm_run: event creation failed");
    int rcode = OFM_OK;
    while (rcode == OFM_OK) {
        // the chunk: as many remaining pairs per level as fit, halving on overflow
        std::vector<int64_t> cnt(L + 1);
        bool any = false;
        for (int l = 0; l <= L; ++l) {
            cnt[l] = to[l] - lo[l];
            any = any || cnt[l] > 0;
        }
        if (!any) break;
        for (;;) {
            std::vector<ofm_group> g;
            std::vector<std::vector<uint64_t>> ids(L + 1);
            for (int l = 0; l <= L; ++l)
                for (int64_t i = 0; i < cnt[l]; ++i) ids[l].push_back(((uint64_t)l << ID_SHIFT) | (uint64_t)(lo[l] + i));
            std::vector<std::vector<ofm_qoi>> qf(L + 1), qc(L + 1);
            for (int l = 0; l <= L; ++l) {
                if (cnt[l] == 0) continue;
                qf[l].resize(cnt[l]);
                ofm_group gf{rc->N[l], (int)cnt[l], ids[l].data(), rc->seed, nullptr, qf[l].data(), nullptr, nullptr};
                g.push_back(gf);
                if (l > 0) {
                    qc[l].resize(cnt[l]);
                    ofm_group gc{rc->N[l - 1], (int)cnt[l], ids[l].data(), rc->seed, nullptr, qc[l].data(), nullptr, nullptr};
                    g.push_back(gc);
                }
            }
            size_t bytes = 0;
            rcode = ofm_batch_workspace_bytes(s, cloud, g.data(), (int)g.size(), &bytes);
            if (rcode != OFM_OK) break;
            if (bytes > cap) {
                // halve the largest count and retry
                int big = 0;
                for (int l = 1; l <= L; ++l)
                    if (cnt[l] * (int64_t)rc->N[l] * rc->N[l] * rc->N[l] > cnt[big] * (int64_t)rc->N[big] * rc->N[big] * rc->N[big])
                        big = l;
                if (cnt[big] <= 1) {
                    rcode = fail(OFM_ENOMEM, "ofm_run: one pair on level %d needs %zu bytes, the cap is %zu", big, bytes, cap);
                    break;
                }
                cnt[big] = (cnt[big] + 1) / 2;
                continue;
            }
            ofm_batch* b = nullptr;
            rcode = ofm_batch_create(&b, s, cloud, g.data(), (int)g.size(), nullptr, 0, st);
            if (rcode != OFM_OK) break;
            cudaEventRecord(e0, st);
            rcode = ofm_batch_init(b);
            int active = 1;
            while (rcode == OFM_OK && active > 0) rcode = ofm_batch_run(b, 1 << 20, &active);
            cudaEventRecord(e1, st);
            if (rcode == OFM_OK) {
                rcode = ofm_batch_qoi(b);
                if (rcode == OFM_ENUMERIC) rcode = OFM_OK;  // failed samples are excluded below
            }
            ofm_batch_destroy(b);
            if (rcode != OFM_OK) break;
            float ms = 0.f;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            *gpu_ms += ms;
            for (int l = 0; l <= L; ++l) {
                for (int64_t i = 0; i < cnt[l]; ++i) {
                    const ofm_qoi& f = qf[l][i];
                    double c = 0.0;
                    bool ok = f.status == 0;
                    double cs = (double)rc->N[l] * rc->N[l] * rc->N[l] * f.n_steps;
                    if (l > 0) {
                        const ofm_qoi& q2 = qc[l][i];
                        ok = ok && q2.status == 0;
                        c = qoi_value(q2, rc->qoi);
                        cs += (double)rc->N[l - 1] * rc->N[l - 1] * rc->N[l - 1] * q2.n_steps;
                    }
                    lv[l].fine.push_back(qoi_value(f, rc->qoi));
                    lv[l].coarse.push_back(c);
                    lv[l].ok.push_back(ok ? 1 : 0);
                    lv[l].cell_steps += cs;
                    lv[l].computed += 1;
                }
                lo[l] += cnt[l];
            }
            break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rcode;
}

}  // namespace

extern "C" int ofm_run(ofm_solver* s, const ofm_cloud_params* cloud, const ofm_run_config* rc, double* pairs_out,
                       uint64_t* ids_out, int64_t pairs_capacity, ofm_run_result* res, void* stream) {
    ofm::clear_error();
    if (!s || !cloud || !rc || !res) return fail(OFM_EINVAL, "ofm_run: NULL argument");
    const int L = rc->L;
    if (L < 0 || L >= OFM_MAX_LEVELS || 2 * L + 1 > OFM_MAX_GROUPS)
        return fail(OFM_EINVAL, "ofm_run: L = %d unsupported (at most %d levels)", L, (OFM_MAX_GROUPS + 1) / 2);
    if (!(rc->target > 0.0) || (rc->mode != OFM_MODE_TOL && rc->mode != OFM_MODE_BUDGET) || rc->max_iterations < 1 ||
        rc->qoi < 0 || rc->qoi > s->cfg.n_sensors)
        return fail(OFM_EINVAL, "ofm_run: bad target, mode, iteration limit or QoI index");
    if (rc->fit_variances && L < 2)
        return fail(OFM_EINVAL, "ofm_run: the variance fit needs two difference levels (L >= 2)");
    for (int l = 0; l <= L; ++l)
        if (rc->N[l] < 8 || (l > 0 && rc->N[l] <= rc->N[l - 1]))
            return fail(OFM_EINVAL, "ofm_run: levels must refine (N[%d] = %d)", l, rc->N[l]);
    std::memset(res, 0, sizeof(*res));
    cudaStream_t st = (cudaStream_t)stream;
    size_t cap = rc->max_batch_bytes;
    if (cap == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(OFM_ECUDA, "cudaMemGetInfo failed");
        cap = (size_t)(0.8 * (double)fr);
    }
    const int min_m = std::max(2, rc->min_samples);
    // step 1: warm-up numbers from the model W_l ~ pair cells x steps ~ N^4 (+ coarse)
    std::vector<double> Wmodel(L + 1);
    for (int l = 0; l <= L; ++l) {
        Wmodel[l] = std::pow((double)rc->N[l], 4.0);
        if (l > 0) Wmodel[l] += std::pow((double)rc->N[l - 1], 4.0);
    }
    std::vector<int64_t> target(L + 1);
    int r = ofm_warmup_samples(L, Wmodel.data(), target.data());
    if (r != OFM_OK) return r;
    for (int l = 0; l <= L; ++l) target[l] = std::max<int64_t>(target[l], min_m);
    if (rc->fit_variances && L >= 3) {
        // the appendix on M_L = 1: levels 1..L-1 carry the fit, the finest keeps Eq. (warmup)'s value
        std::vector<int64_t> w(L + 1);
        ofm_warmup_samples(L, Wmodel.data(), w.data());
        target[L] = w[L];
    }

    std::vector<LevelData> lv(L + 1);
    double gpu_ms = 0.0;
    for (int it = 0; it < rc->max_iterations; ++it) {
        // step 2: solve the missing pairs
        std::vector<int64_t> from(L + 1), to(L + 1);
        for (int l = 0; l <= L; ++l) {
            from[l] = lv[l].computed;
            to[l] = std::max(target[l], lv[l].computed);
        }
        r = solve_pairs(s, cloud, rc, from.data(), to.data(), lv, &gpu_ms, st, cap);
        if (r != OFM_OK) return r;
        res->iterations = it + 1;
        // steps 3-5: indicators, coefficients, errors (on the pairs without failures)
        std::vector<std::vector<double>> rows(L + 1);
        std::vector<int64_t> M(L + 1);
        std::vector<const double*> ptr(L + 1);
        std::vector<double> W(L + 1);
        int64_t failed = 0;
        for (int l = 0; l <= L; ++l) {
            for (size_t i = 0; i < lv[l].fine.size(); ++i) {
                if (!lv[l].ok[i]) {
                    ++failed;
                    continue;
                }
                rows[l].push_back(lv[l].fine[i]);
                rows[l].push_back(lv[l].coarse[i]);
            }
            M[l] = (int64_t)rows[l].size() / 2;
            ptr[l] = rows[l].data();
            W[l] = lv[l].computed > 0 ? lv[l].cell_steps / (double)lv[l].computed : Wmodel[l];
            res->M[l] = M[l];
            res->W[l] = W[l];
        }
        res->failed = failed;
        r = rc->fit_variances ? ofm_estimate_fitted(L, M.data(), ptr.data(), W.data(), &res->est, nullptr)
                              : ofm_estimate(L, M.data(), ptr.data(), W.data(), &res->est);
        if (r != OFM_OK) return r;
        double spent = 0.0;
        for (int l = 0; l <= L; ++l) spent += lv[l].cell_steps;
        res->cell_steps = spent;
        res->gpu_seconds = gpu_ms * 1e-3;
        // step 6: stop?
        if (rc->mode == OFM_MODE_TOL ? std::sqrt(res->est.eps2) <= rc->target : spent >= rc->target) break;
        if (it + 1 == rc->max_iterations) break;   // no iteration left to take step 7's numbers
        // step 7: optimal numbers, keeping what is computed
        std::vector<int64_t> done(L + 1);
        for (int l = 0; l <= L; ++l) done[l] = lv[l].computed;
        r = ofm_optimal_samples(L, res->est.sigma_tilde2, W.data(), done.data(), rc->target, rc->mode, target.data());
        if (r != OFM_OK) return r;
        bool more = false;
        double planned = spent;
        for (int l = 0; l <= L; ++l) {
            more = more || target[l] > done[l];
            planned += (double)(target[l] - done[l]) * W[l];
        }
        if (!more) break;
        if (rc->max_cell_steps > 0.0 && planned > rc->max_cell_steps) {
            res->capped = 1;
            break;
        }
    }
    if (pairs_out || ids_out) {
        int64_t need = 0;
        for (int l = 0; l <= L; ++l) need += res->M[l];
        if (need > pairs_capacity) return fail(OFM_ENOMEM, "ofm_run: pairs_out holds %lld rows, %lld needed",
                                               (long long)pairs_capacity, (long long)need);
        int64_t at = 0;
        for (int l = 0; l <= L; ++l)
            for (size_t i = 0; i < lv[l].fine.size(); ++i)
                if (lv[l].ok[i]) {
                    if (pairs_out) {
                        pairs_out[2 * at] = lv[l].fine[i];
                        pairs_out[2 * at + 1] = lv[l].coarse[i];
                    }
                    if (ids_out) ids_out[at] = ((uint64_t)l << ID_SHIFT) | (uint64_t)i;
                    ++at;
                }
    }
    return OFM_OK;
}
