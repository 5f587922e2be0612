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
#include <limits>
#include <random>
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

// ---------------------------------------------------------------------------
// Surrogate control variate of the top level term.
// ---------------------------------------------------------------------------
struct SurrogateSetup {
    int nearest, steps, hidden, min_pairs;
    float lr;
};

constexpr int SUR_CHUNK = 25;   // Adam steps between two validation checks

// Inputs of the clouds `ids`: the `keep` bubbles nearest the domain centre as
// ofm_cloud_features computes them on the device (scaled by the cloud radius),
// then that cloud's q_{L-1}.  Row-major host matrix n x (4 keep + 1).
int surrogate_inputs(const ofm_cloud_params* cloud, uint64_t seed, const std::vector<uint64_t>& ids,
                     const std::vector<double>& q_coarse, int keep, std::vector<float>& X, cudaStream_t st) {
    const int n = (int)ids.size(), nb = cloud->n_bubbles, d = 4 * keep + 1;
    X.assign((size_t)n * d, 0.0f);
    if (n == 0) return OFM_OK;
    std::vector<ofm_bubble> bub((size_t)n * nb);
    for (int i = 0; i < n; ++i) {
        int r = ofm_sample_cloud(cloud, seed, ids[i], bub.data() + (size_t)i * nb);
        if (r != OFM_OK) return r;
    }
    double* bub_dev = nullptr;
    float* F_dev = nullptr;
    if (cudaMalloc((void**)&bub_dev, bub.size() * sizeof(ofm_bubble)) != cudaSuccess ||
        cudaMalloc((void**)&F_dev, (size_t)n * 4 * keep * sizeof(float)) != cudaSuccess) {
        cudaFree(bub_dev);
        return fail(OFM_ENOMEM, "ofm_run: surrogate input buffers");
    }
    std::vector<float> F((size_t)n * 4 * keep);
    int r = OFM_OK;
    if (cudaMemcpyAsync(bub_dev, bub.data(), bub.size() * sizeof(ofm_bubble), cudaMemcpyHostToDevice, st) != cudaSuccess)
        r = fail(OFM_ECUDA, "ofm_run: surrogate cloud upload");
    if (r == OFM_OK)
        r = ofm_cloud_features(bub_dev, n, nb, keep, cloud->domain_L, cloud->cloud_radius, F_dev, st);
    if (r == OFM_OK && (cudaMemcpyAsync(F.data(), F_dev, F.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        r = fail(OFM_ECUDA, "ofm_run: surrogate feature download");
    cudaFree(bub_dev);
    cudaFree(F_dev);
    if (r != OFM_OK) return r;
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 4 * keep; ++k) X[(size_t)i * d + k] = F[(size_t)i * 4 * keep + k];
        X[(size_t)i * d + 4 * keep] = (float)q_coarse[i];
    }
    return OFM_OK;
}

// Device copy of a host float matrix (freed by the caller).
int upload(const std::vector<float>& h, float** dev, cudaStream_t st) {
    *dev = nullptr;
    if (h.empty()) return OFM_OK;
    if (cudaMalloc((void**)dev, h.size() * sizeof(float)) != cudaSuccess)
        return fail(OFM_ENOMEM, "ofm_run: surrogate buffer of %zu floats", h.size());
    if (cudaMemcpyAsync(*dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(OFM_ECUDA, "ofm_run: surrogate upload");
    return OFM_OK;
}

// Predictions of a network on n host rows (device forward, host result).
int predict(ofm_mlp* net, const std::vector<float>& X, int n, std::vector<double>& y, cudaStream_t st) {
    y.assign(n, 0.0);
    if (n == 0) return OFM_OK;
    float *X_dev = nullptr, *Y_dev = nullptr;
    int r = upload(X, &X_dev, st);
    if (r == OFM_OK && cudaMalloc((void**)&Y_dev, (size_t)n * sizeof(float)) != cudaSuccess)
        r = fail(OFM_ENOMEM, "ofm_run: surrogate output buffer");
    if (r == OFM_OK) r = ofm_mlp_forward(net, X_dev, n, Y_dev, st);
    std::vector<float> yf(n);
    if (r == OFM_OK && (cudaMemcpyAsync(yf.data(), Y_dev, n * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        r = fail(OFM_ECUDA, "ofm_run: surrogate prediction download");
    cudaFree(X_dev);
    cudaFree(Y_dev);
    for (int i = 0; i < n && r == OFM_OK; ++i) y[i] = yf[i];
    return r;
}

// One network trained on the rows `rows` of (X, y) (y: the residual q_L - q_{L-1}): He-initialised weights
// from a seeded generator, inputs and target standardised by the training
// rows' moments, full-batch Adam on the first four fifths of the rows in
// chunks of SUR_CHUNK steps, the parameters with the lowest mean squared
// error on the last fifth kept (early stopping against overfitting the few
// pairs of the finest level).
int train_fold(const std::vector<float>& X, const std::vector<double>& y, int d, const std::vector<int64_t>& rows,
               const SurrogateSetup& su, uint64_t init_seed, ofm_mlp** out, cudaStream_t st) {
    *out = nullptr;
    const int n = (int)rows.size();
    const int n_tr = std::max(2, (int)(0.8 * n)), n_val = n - n_tr;
    std::vector<float> Xtr((size_t)n_tr * d), ytr(n_tr), Xval((size_t)std::max(n_val, 0) * d);
    std::vector<double> yval(std::max(n_val, 0));
    for (int i = 0; i < n; ++i) {
        const float* src = X.data() + (size_t)rows[i] * d;
        if (i < n_tr) {
            std::copy(src, src + d, Xtr.begin() + (size_t)i * d);
            ytr[i] = (float)y[rows[i]];
        } else {
            std::copy(src, src + d, Xval.begin() + (size_t)(i - n_tr) * d);
            yval[i - n_tr] = y[rows[i]];
        }
    }
    // standardisation from the training rows (FP64, M-1)
    std::vector<float> xm(d), xs(d);
    for (int k = 0; k < d; ++k) {
        double m = 0.0, v = 0.0;
        for (int i = 0; i < n_tr; ++i) m += Xtr[(size_t)i * d + k];
        m /= n_tr;
        for (int i = 0; i < n_tr; ++i) v += (Xtr[(size_t)i * d + k] - m) * (Xtr[(size_t)i * d + k] - m);
        xm[k] = (float)m;
        xs[k] = (float)std::sqrt(v / (n_tr - 1));
    }
    double ym = 0.0, yv = 0.0;
    for (int i = 0; i < n_tr; ++i) ym += ytr[i];
    ym /= n_tr;
    for (int i = 0; i < n_tr; ++i) yv += (ytr[i] - ym) * (ytr[i] - ym);
    const float y_mean = (float)ym, y_std = (float)std::max(std::sqrt(yv / (n_tr - 1)), 1e-30);
    ofm_mlp* net = nullptr;
    int r = ofm_mlp_create(&net, d, su.hidden, 3, 1, n_tr, nullptr, 0);
    if (r != OFM_OK) return r;
    int64_t np = 0;
    ofm_mlp_param_count(net, &np);
    std::vector<float> params(np), best;
    {   // He initialisation: N(0, 2/fan_in) weights (Box-Muller on a seeded 64-bit Mersenne Twister), zero biases
        std::mt19937_64 gen(init_seed);
        auto unit = [&]() { return ((double)(gen() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
        int64_t at = 0;
        int fan_in = d;
        for (int layer = 0; layer < 4; ++layer) {
            const int fan_out = layer < 3 ? su.hidden : 1;
            const double sd = std::sqrt(2.0 / fan_in);
            for (int64_t k = 0; k < (int64_t)fan_in * fan_out; ++k) {
                const double u1 = unit(), u2 = unit();
                params[at++] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
            }
            for (int k = 0; k < fan_out; ++k) params[at++] = 0.0f;
            fan_in = fan_out;
        }
    }
    float *Xtr_dev = nullptr, *ytr_dev = nullptr;
    r = ofm_mlp_set_params(net, params.data());
    if (r == OFM_OK) r = ofm_mlp_set_scaling(net, xm.data(), xs.data(), &y_mean, &y_std);
    if (r == OFM_OK) r = upload(Xtr, &Xtr_dev, st);
    if (r == OFM_OK) r = upload(ytr, &ytr_dev, st);
    double best_err = std::numeric_limits<double>::infinity();
    best = params;
    const int chunks = std::max(1, su.steps / SUR_CHUNK);
    for (int c = 0; c < chunks && r == OFM_OK; ++c) {
        r = ofm_mlp_train(net, Xtr_dev, ytr_dev, n_tr, SUR_CHUNK, su.lr, nullptr, st);
        if (r != OFM_OK || n_val == 0) continue;
        std::vector<double> pv;
        r = predict(net, Xval, n_val, pv, st);
        double err = 0.0;
        for (int i = 0; i < n_val; ++i) err += (pv[i] - yval[i]) * (pv[i] - yval[i]);
        if (r == OFM_OK && err < best_err) {
            best_err = err;
            r = ofm_mlp_get_params(net, best.data());
        }
    }
    if (r == OFM_OK && n_val > 0) r = ofm_mlp_set_params(net, best.data());
    cudaFree(Xtr_dev);
    cudaFree(ytr_dev);
    if (r != OFM_OK) {
        ofm_mlp_destroy(net);
        return r;
    }
    *out = net;
    return OFM_OK;
}

// The surrogate's predictions for the level-L pairs (h_top, each by the
// network of the other half) and the level-(L-1) pairs' fine members
// (h_extra, both networks weighted by the other half's share), from the usable
// pairs' ids and values.  Adds its device time to *ms.
int surrogate_predictions(const ofm_cloud_params* cloud, const ofm_run_config* rc, const SurrogateSetup& su,
                          const std::vector<uint64_t>& ids_top, const std::vector<double>& fine_top,
                          const std::vector<double>& coarse_top, const std::vector<uint64_t>& ids_extra,
                          const std::vector<double>& fine_extra, int iteration, std::vector<double>& h_top,
                          std::vector<double>& h_extra, double* ms, cudaStream_t st) {
    const int keep = su.nearest > 0 ? std::min(su.nearest, cloud->n_bubbles) : cloud->n_bubbles;
    const int d = 4 * keep + 1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(OFM_ECUDA, "ofm_run: event creation failed");
    cudaEventRecord(e0, st);
    std::vector<float> Xt, Xe;
    int r = surrogate_inputs(cloud, rc->seed, ids_top, coarse_top, keep, Xt, st);
    if (r == OFM_OK) r = surrogate_inputs(cloud, rc->seed, ids_extra, fine_extra, keep, Xe, st);
    const int64_t M = (int64_t)ids_top.size();
    std::vector<int64_t> fold[2];
    for (int64_t i = 0; i < M; ++i) fold[i & 1].push_back(i);
    // the networks learn the residual q_L - q_{L-1} (its spread is the level
    // difference's, far below q_L's), and predict q_L as q_{L-1} plus it
    std::vector<double> resid(M);
    for (int64_t i = 0; i < M; ++i) resid[i] = fine_top[i] - coarse_top[i];
    ofm_mlp* net[2] = {nullptr, nullptr};
    for (int f = 0; f < 2 && r == OFM_OK; ++f)
        r = train_fold(Xt, resid, d, fold[f], su, rc->seed ^ (0x5DEECE66Dull * (uint64_t)(2 * iteration + f + 1)),
                       &net[f], st);
    h_top.assign(M, 0.0);
    h_extra.assign(ids_extra.size(), 0.0);
    for (int f = 0; f < 2 && r == OFM_OK; ++f) {
        // rows of fold f are predicted by the other fold's network
        std::vector<float> Xf(fold[f].size() * (size_t)d);
        for (size_t i = 0; i < fold[f].size(); ++i)
            std::copy(Xt.begin() + (size_t)fold[f][i] * d, Xt.begin() + (size_t)(fold[f][i] + 1) * d,
                      Xf.begin() + i * d);
        std::vector<double> y;
        r = predict(net[1 - f], Xf, (int)fold[f].size(), y, st);
        for (size_t i = 0; i < fold[f].size() && r == OFM_OK; ++i)
            h_top[fold[f][i]] = coarse_top[fold[f][i]] + y[i];
    }
    for (int f = 0; f < 2 && r == OFM_OK; ++f) {
        // network f predicts the rows of the other fold: weight = the other fold's share
        const double w = (double)fold[1 - f].size() / (double)M;
        std::vector<double> y;
        r = predict(net[f], Xe, (int)ids_extra.size(), y, st);
        for (size_t j = 0; j < y.size() && r == OFM_OK; ++j) h_extra[j] += w * (fine_extra[j] + y[j]);
    }
    for (int f = 0; f < 2; ++f) ofm_mlp_destroy(net[f]);
    cudaEventRecord(e1, st);
    float t = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) *ms += t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
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
    if (rc->surrogate && (L < 1 || rc->fit_variances || rc->surrogate_min_pairs < 0 || rc->surrogate_min_pairs == 1 ||
                          rc->surrogate_nearest < 0 || rc->surrogate_steps < 0 || rc->surrogate_hidden < 0 ||
                          rc->surrogate_hidden > 4096 || rc->surrogate_lr < 0.0 || cloud->n_bubbles < 1))
        return fail(OFM_EINVAL, "ofm_run: the surrogate needs L >= 1, no variance fit, bubbles and valid settings");
    SurrogateSetup su;
    su.min_pairs = rc->surrogate_min_pairs > 0 ? std::max(8, rc->surrogate_min_pairs) : 64;
    su.nearest = rc->surrogate_nearest;
    su.steps = rc->surrogate_steps > 0 ? rc->surrogate_steps : 600;
    su.hidden = rc->surrogate_hidden > 0 ? rc->surrogate_hidden : 256;
    su.lr = rc->surrogate_lr > 0.0 ? (float)rc->surrogate_lr : 1e-3f;
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
    double gpu_ms = 0.0, sur_ms = 0.0;
    std::vector<double> h_top, h_extra;   // the final iteration's surrogate predictions (usable pairs)
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
        res->surrogate_used = 0;
        res->beta = 0.0;
        res->eps2_plain = res->est.eps2;
        for (int l = 0; l <= L; ++l) res->sigma_tilde2_plain[l] = res->est.sigma_tilde2[l];
        h_top.clear();
        h_extra.clear();
        if (rc->surrogate && M[L] >= su.min_pairs && M[L - 1] >= 2) {
            // usable pairs of the two top levels: ids and values
            std::vector<uint64_t> it_ids, ie_ids;
            std::vector<double> ft, ct, fe;
            for (size_t i = 0; i < lv[L].fine.size(); ++i)
                if (lv[L].ok[i]) {
                    it_ids.push_back(((uint64_t)L << ID_SHIFT) | (uint64_t)i);
                    ft.push_back(lv[L].fine[i]);
                    ct.push_back(lv[L].coarse[i]);
                }
            for (size_t i = 0; i < lv[L - 1].fine.size(); ++i)
                if (lv[L - 1].ok[i]) {
                    ie_ids.push_back(((uint64_t)(L - 1) << ID_SHIFT) | (uint64_t)i);
                    fe.push_back(lv[L - 1].fine[i]);
                }
            r = surrogate_predictions(cloud, rc, su, it_ids, ft, ct, ie_ids, fe, it, h_top, h_extra, &sur_ms, st);
            if (r != OFM_OK) return r;
            r = ofm_estimate_surrogate(L, M.data(), ptr.data(), W.data(), h_top.data(), h_extra.data(),
                                       std::numeric_limits<double>::quiet_NaN(), &res->est, &res->beta,
                                       res->sigma_tilde2_plain);
            if (r != OFM_OK) return r;
            res->surrogate_used = 1;
            double e2p = 0.0;
            for (int l = 0; l <= L; ++l) e2p += res->sigma_tilde2_plain[l] / (double)M[l];
            res->eps2_plain = e2p;
        }
        res->surrogate_seconds = sur_ms * 1e-3;
        double spent = 0.0;
        for (int l = 0; l <= L; ++l) spent += lv[l].cell_steps;
        res->cell_steps = spent;
        res->gpu_seconds = (gpu_ms + sur_ms) * 1e-3;
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
        for (int l = 0; l <= L; ++l) {
            int64_t k = 0;   // index among the level's usable pairs
            for (size_t i = 0; i < lv[l].fine.size(); ++i)
                if (lv[l].ok[i]) {
                    if (pairs_out) {
                        pairs_out[2 * at] = lv[l].fine[i];
                        pairs_out[2 * at + 1] = lv[l].coarse[i];
                    }
                    if (ids_out) ids_out[at] = ((uint64_t)l << ID_SHIFT) | (uint64_t)i;
                    if (rc->surrogate_h_out) {
                        double h = std::numeric_limits<double>::quiet_NaN();
                        if (res->surrogate_used && l == L && k < (int64_t)h_top.size()) h = h_top[k];
                        if (res->surrogate_used && l == L - 1 && k < (int64_t)h_extra.size()) h = h_extra[k];
                        rc->surrogate_h_out[at] = h;
                    }
                    ++at;
                    ++k;
                }
        }
    }
    return OFM_OK;
}
