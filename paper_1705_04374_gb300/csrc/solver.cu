// Host side of the C ABI for batched solves: workspace layout, batch
// lifecycle, CUDA-graph step chunks, QoI copy-out.
//
// GPU design
//   * State in HBM as structure of arrays Q[sample][var][z][y][x] (x fastest),
//     three buffers per sample: Q_a, Q_b (ping-pong, because neighbours read
//     the old state while a block writes the new one) and dQ (2N register).
//   * One fused kernel per RK stage.  A block owns an 8x8x8 tile: it stages
//     the tile plus a 3-cell halo along each axis (no corners) into shared
//     memory as primitives, computes every face flux of the tile once (WENO5
//     or WENO3 both sides + HLLC) per direction into shared memory, differences them
//     into per-cell right-hand sides in registers, and applies the 2N update.
//     Per cell and stage, HBM sees only Q, dQ in and Q', dQ out (the first stage reads no dQ,
//     the last writes none).
//   * The last stage's epilogue evaluates the new state's pressure and sound
//     speed and reduces, per tile, the max signal speed (for the next CFL
//     step), the max pressure with its first index, and health bits.  A
//     per-sample finalize kernel combines the tiles in a fixed order, so every
//     reduction is deterministic; time, step and QoI bookkeeping stays on the
//     device in FP64.
//   * Samples of different grids (levels) share the launches: the grid is the
//     concatenation of every group's tiles, and a block finds its group from
//     its index.  Finished samples' blocks exit at once.
//   * Steps are captured in CUDA graphs (chunks of an even number of steps,
//     which keeps the ping-pong parity of every replay the same).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "host_shared.cuh"
#include "internal.h"
#include "ofmlmc.h"
#include "types.cuh"

using ofm::fail;
using namespace ofm::gpu;

namespace {

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t err__ = (call);                                                        \
        if (err__ != cudaSuccess)                                                          \
            return fail(OFM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(err__));     \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t total = 0;
    size_t take(size_t bytes) {
        const size_t off = total;
        total = align_up(total + bytes, 256);
        return off;
    }
};

}  // namespace

struct GroupHost {
    int N, M;
    ofm_qoi* qoi_out;
    double* hist_out;
    double* ahist_out;
    std::vector<int> sens_cells;
    int sens_off[OFM_MAX_SENSORS + 1];
    size_t off_QA, off_QB, off_dQ, off_part, off_sens;
};

struct ofm_batch {
    ofm_solver* solver;
    int precision;
    int n_groups;
    int total_slots;
    int nb;
    GroupHost gh[OFM_MAX_GROUPS];
    unsigned char* ws;
    bool own_ws;
    cudaStream_t user;
    cudaStream_t priv;
    cudaEvent_t ev;
    int* h_active;            // pinned
    long long global_steps;
    long long launches;
    long long total_blocks;
    cudaGraphExec_t chunk;
    bool chunk_ready;
    bool initialised;
    int variant;              // stage-kernel variant; -1 = pick by timing at the first run
    float tune_ms[OFM_N_VARIANTS];  // autotuning times of the variants (two steps each)
    bool profiling;           // steps without graphs, CUDA events around each stage kernel
    cudaEvent_t pev[4];
    double stage_ms;
    long long stage_launches;
    long long h2d_bytes, d2h_bytes;
    Params<double> pd;        // full group table
    Params<float> pf;
    Params<double> pd_s;      // table the stage kernels walk: groups with unfinished samples
    Params<float> pf_s;
    unsigned active_mask;     // groups in the stage table
    size_t off_t, off_dt, off_last, off_done, off_nsteps, off_kout, off_qoi, off_sold, off_hist, off_aold, off_ahist,
        off_active, off_bub;
};

namespace {

void sensor_cells(const ofm_solver* s, int N, GroupHost& g) { sensor_cell_list(s, N, g.sens_cells, g.sens_off); }

template <typename T>
void fill_params(ofm_batch* b, Params<T>& P) {
    std::memset(&P, 0, sizeof(P));
    const ofm_solver_config& c = b->solver->cfg;
    P.n_groups = b->n_groups;
    long long blk = 0;
    int slot = 0;
    for (int g = 0; g < b->n_groups; ++g) {
        GroupHost& gh = b->gh[g];
        GroupDev& G = P.g[g];
        G.N = gh.N;
        G.tpd = gh.N / TS;
        G.tps = G.tpd * G.tpd * G.tpd;
        G.n_samples = gh.M;
        G.slot0 = slot;
        G.block0 = blk;
        G.QA = b->ws + gh.off_QA;
        G.QB = b->ws + gh.off_QB;
        G.dQ = b->ws + gh.off_dQ;
        G.part = (Partial*)(b->ws + gh.off_part);
        G.sens_cells = (const int*)(b->ws + gh.off_sens);
        for (int k = 0; k <= OFM_MAX_SENSORS; ++k) G.sens_off[k] = k <= c.n_sensors ? gh.sens_off[k] : 0;
        G.h = 1.0 / gh.N;
        G.h32 = (float)G.h;
        blk += (long long)G.tps * gh.M;
        slot += gh.M;
    }
    P.total_blocks = blk;
    P.total_slots = slot;
    P.s.t = (double*)(b->ws + b->off_t);
    P.s.dt = (double*)(b->ws + b->off_dt);
    P.s.last = (int*)(b->ws + b->off_last);
    P.s.done = (int*)(b->ws + b->off_done);
    P.s.nsteps = (int*)(b->ws + b->off_nsteps);
    P.s.kout = (int*)(b->ws + b->off_kout);
    P.s.qoi = (DevQoi*)(b->ws + b->off_qoi);
    P.s.sens_old = (double*)(b->ws + b->off_sold);
    P.s.hist = (double*)(b->ws + b->off_hist);
    P.s.alpha_old = (double*)(b->ws + b->off_aold);
    P.s.ahist = (double*)(b->ws + b->off_ahist);
    P.s.n_active = (int*)(b->ws + b->off_active);
    P.s.g_active = (int*)(b->ws + b->off_active + 16);
    P.s.bubbles = (const double*)(b->ws + b->off_bub);
    params_constants(b->solver, b->nb, P);
}

// Stage-kernel table with only the groups in `mask`: same pointers and sample
// slots, tile ranges (block0) re-packed so finished groups launch no blocks.
template <typename T>
void stage_table(const Params<T>& full, unsigned mask, Params<T>& out) {
    out = full;
    int n = 0;
    long long blk = 0;
    for (int g = 0; g < full.n_groups && g < OFM_MAX_GROUPS; ++g) {
        if (!(mask & (1u << g))) continue;
        out.g[n] = full.g[g];
        out.g[n].block0 = blk;
        blk += (long long)full.g[g].tps * full.g[g].n_samples;
        ++n;
    }
    out.n_groups = n;
    out.total_blocks = blk;
}

void set_active_mask(ofm_batch* b, unsigned mask) {
    if (mask == b->active_mask) return;
    b->active_mask = mask;
    if (b->precision == OFM_FP64)   // only the batch's own precision has a table
        stage_table(b->pd, mask, b->pd_s);
    else
        stage_table(b->pf, mask, b->pf_s);
    if (b->chunk_ready) {
        cudaGraphExecDestroy(b->chunk);
        b->chunk_ready = false;
    }
}

template <typename T>
int build_chunk(ofm_batch* b, const Params<T>& Ps, const Params<T>& P) {
    cudaGraph_t graph;
    CUDA_TRY(cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal));
    const long long saved = b->launches;
    for (int k = 0; k < CHUNK_STEPS; ++k) {
        int rc = launch_step(Ps, P, b->variant < 0 ? OFM_VARIANT_TILES : b->variant, k & 1, b->priv, &b->launches);
        if (rc != OFM_OK) {
            cudaStreamEndCapture(b->priv, &graph);
            return rc;
        }
    }
    b->launches = saved;
    CUDA_TRY(cudaStreamEndCapture(b->priv, &graph));
    cudaError_t e = cudaGraphInstantiate(&b->chunk, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(OFM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    b->chunk_ready = true;
    return OFM_OK;
}

int enter(ofm_batch* b) {
    CUDA_TRY(cudaEventRecord(b->ev, b->user));
    CUDA_TRY(cudaStreamWaitEvent(b->priv, b->ev, 0));
    return OFM_OK;
}

int leave(ofm_batch* b) {
    CUDA_TRY(cudaEventRecord(b->ev, b->priv));
    CUDA_TRY(cudaStreamWaitEvent(b->user, b->ev, 0));
    return OFM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int ofm_solver_create(ofm_solver** out, const ofm_solver_config* c) {
    ofm::clear_error();
    if (!out || !c) return fail(OFM_EINVAL, "ofm_solver_create: NULL argument");
    *out = nullptr;
    if (!(c->gamma[0] > 1.0) || !(c->gamma[1] > 1.0) || !(c->pc[0] >= 0.0) || !(c->pc[1] >= 0.0) ||
        !(c->rho0[0] > 0.0) || !(c->rho0[1] > 0.0) || !(c->p_liq > 0.0) || !(c->p_gas > 0.0) ||
        !(c->cfl > 0.0) || !(c->t_end > 0.0) || !(c->weno_eps > 0.0) || !(c->domain_L > 0.0) ||
        !(c->ramp_radius >= 0.0) || !(c->p_cloud >= 0.0) || (c->ramp_radius > 0.0 && !(c->p_cloud > 0.0)))
        return fail(OFM_EINVAL, "ofm_solver_create: non-physical configuration");
    if (c->precision != OFM_FP64 && c->precision != OFM_FP32)
        return fail(OFM_EINVAL, "ofm_solver_create: precision must be OFM_FP64 or OFM_FP32");
    if (c->bc != OFM_BC_TRANSMISSIVE && c->bc != OFM_BC_PERIODIC && c->bc != OFM_BC_CHARACTERISTIC)
        return fail(OFM_EINVAL, "ofm_solver_create: unknown boundary condition");
    if (c->bc == OFM_BC_CHARACTERISTIC && !(c->bc_penalty >= 0.0 && c->bc_penalty <= 1.0))
        return fail(OFM_EINVAL, "ofm_solver_create: bc_penalty must lie in [0, 1]");
    if (c->weno_order != 0 && c->weno_order != 3 && c->weno_order != 5)
        return fail(OFM_EINVAL, "ofm_solver_create: weno_order must be 3 or 5");
    if (c->n_sensors < 0 || c->n_sensors > OFM_MAX_SENSORS || c->n_out_times < 0 || c->max_steps < 1)
        return fail(OFM_EINVAL, "ofm_solver_create: bad sensor / output / step settings");
    ofm_solver* s = new (std::nothrow) ofm_solver;
    if (!s) return fail(OFM_ENOMEM, "ofm_solver_create: out of host memory");
    s->cfg = *c;
    s->p_ref = c->p_liq;
    s->L = c->domain_L;
    s->u_ref = std::sqrt(c->p_liq / 1000.0);
    s->t_ref = s->L / s->u_ref;
    *out = s;
    return OFM_OK;
}

extern "C" void ofm_solver_destroy(ofm_solver* s) { delete s; }

static int check_groups(const ofm_solver* s, const ofm_cloud_params* cloud, const ofm_group* groups,
                        int n_groups) {
    if (!s || !cloud || !groups) return fail(OFM_EINVAL, "NULL solver, cloud or groups");
    if (n_groups < 1 || n_groups > OFM_MAX_GROUPS)
        return fail(OFM_EINVAL, "n_groups must be in [1, %d]", OFM_MAX_GROUPS);
    if (cloud->n_bubbles < 0) return fail(OFM_EINVAL, "n_bubbles < 0");
    long long blocks = 0;
    for (int g = 0; g < n_groups; ++g) {
        const int N = groups[g].N;
        if (N < TS || N > 512 || N % TS != 0)
            return fail(OFM_EINVAL, "group %d: N = %d must be a multiple of %d in [%d, 512]", g, N, TS, TS);
        if (groups[g].n_samples < 1) return fail(OFM_EINVAL, "group %d: n_samples < 1", g);
        if (!groups[g].bubbles && !groups[g].sample_ids)
            return fail(OFM_EINVAL, "group %d: need sample_ids or bubbles", g);
        blocks += (long long)(N / TS) * (N / TS) * (N / TS) * groups[g].n_samples;
    }
    if (blocks > 0x7fffffffLL) return fail(OFM_EINVAL, "too many tiles in one batch");
    // every sample has at least one tile, so at most 2^31 samples; bounding the
    // per-sample bubble and history counts keeps every workspace size below
    // 2^50 bytes, so no byte count can wrap around
    long long samples = 0;
    for (int g = 0; g < n_groups; ++g) samples += groups[g].n_samples;
    const long long hist_per = (long long)s->cfg.n_sensors * s->cfg.n_out_times;
    if ((long long)cloud->n_bubbles * samples > (1LL << 40) || hist_per * samples > (1LL << 40))
        return fail(OFM_ENOMEM, "batch too large: %lld samples with %d bubbles and %lld history values each", samples,
                    cloud->n_bubbles, hist_per);
    return OFM_OK;
}

static void layout(const ofm_solver* s, const ofm_cloud_params* cloud, const ofm_group* groups,
                   int n_groups, ofm_batch* b, Layout& Lo) {
    const size_t es = s->cfg.precision == OFM_FP64 ? 8 : 4;
    int slots = 0;
    for (int g = 0; g < n_groups; ++g) {
        GroupHost& gh = b->gh[g];
        const size_t n3 = (size_t)groups[g].N * groups[g].N * groups[g].N;
        const size_t M = groups[g].n_samples;
        gh.off_QA = Lo.take(M * 7 * n3 * es);
        gh.off_QB = Lo.take(M * 7 * n3 * es);
        gh.off_dQ = Lo.take(M * 7 * n3 * es);
        const size_t tps = n3 / (TS * TS * TS);
        gh.off_part = Lo.take(M * tps * sizeof(Partial));
        sensor_cells(s, groups[g].N, gh);
        gh.off_sens = Lo.take(std::max<size_t>(1, gh.sens_cells.size()) * sizeof(int));
        slots += groups[g].n_samples;
    }
    const size_t S = slots;
    b->off_t = Lo.take(S * 8);
    b->off_dt = Lo.take(S * 8);
    b->off_last = Lo.take(S * 4);
    b->off_done = Lo.take(S * 4);
    b->off_nsteps = Lo.take(S * 4);
    b->off_kout = Lo.take(S * 4);
    b->off_qoi = Lo.take(S * sizeof(DevQoi));
    b->off_sold = Lo.take(S * OFM_MAX_SENSORS * 8);
    b->off_hist = Lo.take(std::max<size_t>(1, S * s->cfg.n_sensors * s->cfg.n_out_times) * 8);
    b->off_aold = Lo.take(S * OFM_MAX_SENSORS * 8);
    b->off_ahist = Lo.take(std::max<size_t>(1, S * s->cfg.n_sensors * s->cfg.n_out_times) * 8);
    b->off_active = Lo.take(16 + sizeof(int) * OFM_MAX_GROUPS);
    b->off_bub = Lo.take(std::max<size_t>(1, S * cloud->n_bubbles * 4) * 8);
}

extern "C" int ofm_batch_workspace_bytes(const ofm_solver* s, const ofm_cloud_params* cloud,
                                         const ofm_group* groups, int n_groups, size_t* bytes) {
    ofm::clear_error();
    int rc = check_groups(s, cloud, groups, n_groups);
    if (rc != OFM_OK) return rc;
    if (!bytes) return fail(OFM_EINVAL, "NULL bytes");
    ofm_batch tmp{};
    Layout Lo;
    layout(s, cloud, groups, n_groups, &tmp, Lo);
    *bytes = Lo.total;
    return OFM_OK;
}

extern "C" int ofm_batch_create(ofm_batch** out, ofm_solver* s, const ofm_cloud_params* cloud,
                                const ofm_group* groups, int n_groups, void* workspace,
                                size_t workspace_bytes, void* stream) {
    ofm::clear_error();
    if (!out) return fail(OFM_EINVAL, "ofm_batch_create: NULL out");
    *out = nullptr;
    int rc = check_groups(s, cloud, groups, n_groups);
    if (rc != OFM_OK) return rc;
    if (((uintptr_t)workspace) % 256 != 0) return fail(OFM_EINVAL, "workspace must be 256-byte aligned");
    ofm_batch* b = new (std::nothrow) ofm_batch();  // value-initialised: every plain field starts at zero
    if (!b) return fail(OFM_ENOMEM, "out of host memory");
    b->solver = s;
    b->precision = s->cfg.precision;
    b->n_groups = n_groups;
    b->nb = cloud->n_bubbles;
    b->ws = nullptr;
    b->own_ws = false;
    b->user = (cudaStream_t)stream;
    b->priv = nullptr;
    b->ev = nullptr;
    b->h_active = nullptr;
    b->global_steps = 0;
    b->launches = 0;
    b->chunk_ready = false;
    b->initialised = false;
    b->profiling = false;
    b->variant = OFM_VARIANT_TILES;
    for (int v = 0; v < OFM_N_VARIANTS; ++v) b->tune_ms[v] = 0.f;
    for (int k = 0; k < 4; ++k) b->pev[k] = nullptr;
    b->stage_ms = 0.0;
    b->stage_launches = 0;
    b->h2d_bytes = 0;
    b->d2h_bytes = 0;
    Layout Lo;
    layout(s, cloud, groups, n_groups, b, Lo);
    int slots = 0;
    for (int g = 0; g < n_groups; ++g) {
        b->gh[g].N = groups[g].N;
        b->gh[g].M = groups[g].n_samples;
        b->gh[g].qoi_out = groups[g].qoi_out;
        b->gh[g].hist_out = groups[g].sensor_hist;
        b->gh[g].ahist_out = groups[g].alpha_hist;
        slots += groups[g].n_samples;
    }
    b->total_slots = slots;
    auto bail = [&](int code) {
        ofm_batch_destroy(b);
        return code;
    };
    if (workspace) {
        if (workspace_bytes < Lo.total)
            return bail(fail(OFM_ENOMEM, "workspace has %zu bytes, the batch needs %zu", workspace_bytes, Lo.total));
        b->ws = (unsigned char*)workspace;
    } else {
        cudaError_t e = cudaMalloc((void**)&b->ws, Lo.total);
        if (e != cudaSuccess) {
            b->ws = nullptr;
            return bail(fail(OFM_ENOMEM, "cudaMalloc(%zu): %s", Lo.total, cudaGetErrorString(e)));
        }
        b->own_ws = true;
    }
    if (cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_active, 16 + sizeof(int) * OFM_MAX_GROUPS) != cudaSuccess)
        return bail(fail(OFM_ECUDA, "stream / event / pinned allocation failed"));
    b->active_mask = 0;
    if (b->precision == OFM_FP64) {
        fill_params(b, b->pd);
        for (int g = 0; g < b->n_groups; ++g)
            if ((rc = group_tensor_maps(b->pd.g[g], sizeof(double))) != OFM_OK) return bail(rc);
        b->pd_s = b->pd;
        b->total_blocks = b->pd.total_blocks;
        if ((rc = set_smem_attrs<double>()) != OFM_OK) return bail(rc);
    } else {
        fill_params(b, b->pf);
        for (int g = 0; g < b->n_groups; ++g)
            if ((rc = group_tensor_maps(b->pf.g[g], sizeof(float))) != OFM_OK) return bail(rc);
        b->pf_s = b->pf;
        b->total_blocks = b->pf.total_blocks;
        if ((rc = set_smem_attrs<float>()) != OFM_OK) return bail(rc);
    }
    // clouds: sampled (or copied) on the host, non-dimensionalised, uploaded
    std::vector<double> bub((size_t)slots * b->nb * 4);
    std::vector<ofm_bubble> tmp(b->nb > 0 ? b->nb : 1);
    size_t at = 0;
    for (int g = 0; g < n_groups; ++g) {
        for (int i = 0; i < groups[g].n_samples; ++i) {
            const ofm_bubble* src;
            if (groups[g].bubbles) {
                src = groups[g].bubbles + (size_t)i * b->nb;
            } else {
                if ((rc = ofm_sample_cloud(cloud, groups[g].seed, groups[g].sample_ids[i], tmp.data())) != OFM_OK)
                    return bail(rc);
                src = tmp.data();
            }
            for (int k = 0; k < b->nb; ++k) {
                bub[at++] = src[k].x / s->L;
                bub[at++] = src[k].y / s->L;
                bub[at++] = src[k].z / s->L;
                bub[at++] = src[k].r / s->L;
            }
        }
    }
    for (int k = 0; k < 4; ++k)
        if (cudaEventCreate(&b->pev[k]) != cudaSuccess) return bail(fail(OFM_ECUDA, "event creation failed"));
    if (enter(b) != OFM_OK) return bail(OFM_ECUDA);
    b->h2d_bytes += (long long)bub.size() * 8;
    if (!bub.empty() &&
        cudaMemcpyAsync(b->ws + b->off_bub, bub.data(), bub.size() * 8, cudaMemcpyHostToDevice, b->priv) != cudaSuccess)
        return bail(fail(OFM_ECUDA, "bubble upload failed"));
    for (int g = 0; g < n_groups; ++g) {
        const std::vector<int>& sc = b->gh[g].sens_cells;
        b->h2d_bytes += (long long)sc.size() * (long long)sizeof(int);
        if (!sc.empty() &&
            cudaMemcpyAsync(b->ws + b->gh[g].off_sens, sc.data(), sc.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->priv) != cudaSuccess)
            return bail(fail(OFM_ECUDA, "sensor upload failed"));
    }
    // host vectors die at return: wait for the copies
    if (cudaStreamSynchronize(b->priv) != cudaSuccess) return bail(fail(OFM_ECUDA, "upload sync failed"));
    *out = b;
    return OFM_OK;
}

extern "C" int ofm_batch_init(ofm_batch* b) {
    ofm::clear_error();
    if (!b) return fail(OFM_EINVAL, "NULL batch");
    int rc = enter(b);
    if (rc != OFM_OK) return rc;
    rc = b->precision == OFM_FP64 ? launch_init(b->pd, b->priv, true, &b->launches) : launch_init(b->pf, b->priv, true, &b->launches);
    if (rc != OFM_OK) return rc;
    b->active_mask = 0;
    set_active_mask(b, (1u << b->n_groups) - 1u);
    b->global_steps = 0;
    b->initialised = true;
    return leave(b);
}

extern "C" int ofm_batch_run(ofm_batch* b, int max_steps, int* n_active) {
    ofm::clear_error();
    if (!b || max_steps < 0) return fail(OFM_EINVAL, "ofm_batch_run: bad arguments");
    if (!b->initialised) return fail(OFM_EINVAL, "ofm_batch_run: call ofm_batch_init first");
    int rc = enter(b);
    if (rc != OFM_OK) return rc;
    int done_steps = 0;
    int active = 1;
    if (b->variant < 0 && !b->profiling && max_steps >= 2 * OFM_N_VARIANTS && (b->global_steps & 1) == 0) {
        // autotune: time two steps of each stage-kernel variant (interleaved)
        // and keep the fastest; the step count stays even
        float t[OFM_N_VARIANTS] = {};
        for (int k = 0; k < 2 * OFM_N_VARIANTS; ++k) {
            const int var = k % OFM_N_VARIANTS;
            CUDA_TRY(cudaEventRecord(b->pev[0], b->priv));
            rc = b->precision == OFM_FP64
                     ? launch_step(b->pd_s, b->pd, var, (int)(b->global_steps & 1), b->priv, &b->launches)
                     : launch_step(b->pf_s, b->pf, var, (int)(b->global_steps & 1), b->priv, &b->launches);
            if (rc != OFM_OK) return rc;
            CUDA_TRY(cudaEventRecord(b->pev[1], b->priv));
            CUDA_TRY(cudaEventSynchronize(b->pev[1]));
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, b->pev[0], b->pev[1]));
            t[var] += ms;
            b->global_steps += 1;
            done_steps += 1;
        }
        int best = 0;
        for (int v = 1; v < OFM_N_VARIANTS; ++v)
            if (t[v] < t[best]) best = v;
        b->variant = best;
        for (int v = 0; v < OFM_N_VARIANTS; ++v) b->tune_ms[v] = t[v];
    }
    const int variant = b->variant < 0 ? OFM_VARIANT_TILES : b->variant;
    while (done_steps < max_steps) {
        if (b->profiling) {
            const int parity = (int)(b->global_steps & 1);
            for (int k = 0; k < 4; ++k) {
                CUDA_TRY(cudaEventRecord(b->pev[k], b->priv));
                if (k == 3) break;
                rc = b->precision == OFM_FP64
                         ? launch_stage(b->pd_s, b->pd, variant, k, k == 1 ? 1 - parity : parity, b->priv, &b->launches)
                         : launch_stage(b->pf_s, b->pf, variant, k, k == 1 ? 1 - parity : parity, b->priv, &b->launches);
                if (rc != OFM_OK) return rc;
            }
            rc = b->precision == OFM_FP64 ? launch_stage(b->pd_s, b->pd, variant, 3, 1 - parity, b->priv, &b->launches)
                                          : launch_stage(b->pf_s, b->pf, variant, 3, 1 - parity, b->priv, &b->launches);
            if (rc != OFM_OK) return rc;
            CUDA_TRY(cudaEventSynchronize(b->pev[3]));
            for (int k = 0; k < 3; ++k) {
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, b->pev[k], b->pev[k + 1]));
                b->stage_ms += ms;
            }
            b->stage_launches += 3;
            b->global_steps += 1;
            done_steps += 1;
        } else if ((b->global_steps & 1) == 0 && max_steps - done_steps >= CHUNK_STEPS) {
            if (!b->chunk_ready) {
                rc = b->precision == OFM_FP64 ? build_chunk(b, b->pd_s, b->pd) : build_chunk(b, b->pf_s, b->pf);
                if (rc != OFM_OK) return rc;
            }
            CUDA_TRY(cudaGraphLaunch(b->chunk, b->priv));
            b->launches += 4 * CHUNK_STEPS;
            b->global_steps += CHUNK_STEPS;
            done_steps += CHUNK_STEPS;
        } else {
            const int parity = (int)(b->global_steps & 1);
            rc = b->precision == OFM_FP64 ? launch_step(b->pd_s, b->pd, variant, parity, b->priv, &b->launches)
                                          : launch_step(b->pf_s, b->pf, variant, parity, b->priv, &b->launches);
            if (rc != OFM_OK) return rc;
            b->global_steps += 1;
            done_steps += 1;
        }
        const size_t cnt_bytes = 16 + sizeof(int) * b->n_groups;
        CUDA_TRY(cudaMemcpyAsync(b->h_active, b->ws + b->off_active, cnt_bytes, cudaMemcpyDeviceToHost, b->priv));
        b->d2h_bytes += (long long)cnt_bytes;
        CUDA_TRY(cudaStreamSynchronize(b->priv));
        active = *b->h_active;
        if (active == 0) break;
        unsigned mask = 0;
        for (int g = 0; g < b->n_groups; ++g)
            if (b->h_active[4 + g] > 0) mask |= 1u << g;
        set_active_mask(b, mask);
    }
    if (n_active) *n_active = active;
    return leave(b);
}

extern "C" int ofm_batch_qoi(ofm_batch* b) {
    ofm::clear_error();
    if (!b || !b->initialised) return fail(OFM_EINVAL, "ofm_batch_qoi: batch not initialised");
    int rc = enter(b);
    if (rc != OFM_OK) return rc;
    rc = b->precision == OFM_FP64 ? launch_totals(b->pd, b->priv, 1, &b->launches)
                                  : launch_totals(b->pf, b->priv, 1, &b->launches);
    if (rc != OFM_OK) return rc;
    const ofm_solver_config& c = b->solver->cfg;
    std::vector<DevQoi> q(b->total_slots);
    std::vector<int> nsteps(b->total_slots), done(b->total_slots);
    std::vector<double> tt(b->total_slots);
    const size_t hist_n = (size_t)b->total_slots * c.n_sensors * c.n_out_times;
    std::vector<double> hist(hist_n), ahist(hist_n);
    CUDA_TRY(cudaMemcpyAsync(q.data(), b->ws + b->off_qoi, q.size() * sizeof(DevQoi), cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaMemcpyAsync(nsteps.data(), b->ws + b->off_nsteps, nsteps.size() * 4, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaMemcpyAsync(done.data(), b->ws + b->off_done, done.size() * 4, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaMemcpyAsync(tt.data(), b->ws + b->off_t, tt.size() * 8, cudaMemcpyDeviceToHost, b->priv));
    bool want_ahist = false;
    for (int g = 0; g < b->n_groups; ++g) want_ahist = want_ahist || b->gh[g].ahist_out != nullptr;
    if (hist_n)
        CUDA_TRY(cudaMemcpyAsync(hist.data(), b->ws + b->off_hist, hist_n * 8, cudaMemcpyDeviceToHost, b->priv));
    if (hist_n && want_ahist)
        CUDA_TRY(cudaMemcpyAsync(ahist.data(), b->ws + b->off_ahist, hist_n * 8, cudaMemcpyDeviceToHost, b->priv));
    b->d2h_bytes += (long long)(q.size() * sizeof(DevQoi) + nsteps.size() * 4 + done.size() * 4 + tt.size() * 8 +
                                hist_n * 8 * (want_ahist ? 2 : 1));
    CUDA_TRY(cudaStreamSynchronize(b->priv));
    const ofm_solver* s = b->solver;
    int any_bad = 0;
    int slot = 0;
    for (int g = 0; g < b->n_groups; ++g) {
        const GroupHost& gh = b->gh[g];
        const int N = gh.N;
        for (int i = 0; i < gh.M; ++i, ++slot) {
            const DevQoi& d = q[slot];
            if (d.status) any_bad = 1;
            if (gh.qoi_out)
                qoi_to_si(s, N, d, done[slot] ? d.t_final : tt[slot], done[slot] ? d.n_steps : nsteps[slot],
                          gh.qoi_out[i]);
            if (gh.hist_out && hist_n) {
                const size_t per = (size_t)c.n_sensors * c.n_out_times;
                for (size_t a = 0; a < per; ++a) gh.hist_out[(size_t)i * per + a] = hist[(size_t)slot * per + a] * s->p_ref;
            }
            if (gh.ahist_out && hist_n) {
                const size_t per = (size_t)c.n_sensors * c.n_out_times;
                for (size_t a = 0; a < per; ++a) gh.ahist_out[(size_t)i * per + a] = ahist[(size_t)slot * per + a];
            }
        }
    }
    rc = leave(b);
    if (rc != OFM_OK) return rc;
    if (any_bad) return fail(OFM_ENUMERIC, "some samples have a non-zero status");
    return OFM_OK;
}

static int locate(ofm_batch* b, int group, int sample, size_t bytes, size_t* off, size_t* n) {
    if (!b || group < 0 || group >= b->n_groups || sample < 0 || sample >= b->gh[group].M)
        return fail(OFM_EINVAL, "bad group / sample");
    const size_t es = b->precision == OFM_FP64 ? 8 : 4;
    const size_t N = b->gh[group].N;
    *n = 7 * N * N * N * es;
    if (bytes != *n) return fail(OFM_EINVAL, "state buffer must have %zu bytes", *n);
    *off = (size_t)sample * (*n);
    return OFM_OK;
}

extern "C" int ofm_batch_copy_state(ofm_batch* b, int group, int sample, void* host_buf, size_t bytes) {
    ofm::clear_error();
    size_t off = 0, n = 0;
    int rc = locate(b, group, sample, bytes, &off, &n);
    if (rc != OFM_OK) return rc;
    if (!host_buf) return fail(OFM_EINVAL, "NULL buffer");
    rc = enter(b);
    if (rc != OFM_OK) return rc;
    // the current state of a sample is in Q_b after an odd number of its own steps
    int ns = 0;
    int slot = 0;
    for (int g = 0; g < group; ++g) slot += b->gh[g].M;
    slot += sample;
    CUDA_TRY(cudaMemcpyAsync(&ns, b->ws + b->off_nsteps + (size_t)slot * 4, 4, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaStreamSynchronize(b->priv));
    const size_t base = (ns & 1) ? b->gh[group].off_QB : b->gh[group].off_QA;
    CUDA_TRY(cudaMemcpyAsync(host_buf, b->ws + base + off, n, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaStreamSynchronize(b->priv));
    return leave(b);
}

extern "C" int ofm_batch_set_state(ofm_batch* b, int group, int sample, const void* host_buf, size_t bytes) {
    ofm::clear_error();
    size_t off = 0, n = 0;
    int rc = locate(b, group, sample, bytes, &off, &n);
    if (rc != OFM_OK) return rc;
    if (!host_buf) return fail(OFM_EINVAL, "NULL buffer");
    if (!b->initialised || b->global_steps != 0)
        return fail(OFM_EINVAL, "ofm_batch_set_state: only between ofm_batch_init and the first step");
    rc = enter(b);
    if (rc != OFM_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(b->ws + b->gh[group].off_QA + off, host_buf, n, cudaMemcpyHostToDevice, b->priv));
    b->h2d_bytes += (long long)n;
    rc = b->precision == OFM_FP64 ? launch_init(b->pd, b->priv, false, &b->launches) : launch_init(b->pf, b->priv, false, &b->launches);
    if (rc != OFM_OK) return rc;
    CUDA_TRY(cudaStreamSynchronize(b->priv));
    return leave(b);
}

extern "C" int ofm_batch_cell_steps(ofm_batch* b, double* cell_steps) {
    ofm::clear_error();
    if (!b || !cell_steps) return fail(OFM_EINVAL, "NULL argument");
    std::vector<int> ns(b->total_slots);
    CUDA_TRY(cudaMemcpyAsync(ns.data(), b->ws + b->off_nsteps, ns.size() * 4, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaStreamSynchronize(b->priv));
    double total = 0.0;
    int slot = 0;
    for (int g = 0; g < b->n_groups; ++g) {
        const double n3 = (double)b->gh[g].N * b->gh[g].N * b->gh[g].N;
        for (int i = 0; i < b->gh[g].M; ++i, ++slot) total += n3 * ns[slot];
    }
    *cell_steps = total;
    return OFM_OK;
}

extern "C" int ofm_batch_kernel_launches(ofm_batch* b, int64_t* launches) {
    if (!b || !launches) return fail(OFM_EINVAL, "NULL argument");
    *launches = b->launches;
    return OFM_OK;
}

extern "C" int ofm_batch_set_profiling(ofm_batch* b, int on) {
    ofm::clear_error();
    if (!b) return fail(OFM_EINVAL, "NULL batch");
    b->profiling = on != 0;
    return OFM_OK;
}

extern "C" int ofm_batch_set_variant(ofm_batch* b, int variant) {
    ofm::clear_error();
    if (!b || variant < -1 || variant >= OFM_N_VARIANTS) return fail(OFM_EINVAL, "bad batch or variant");
    if (variant != b->variant && b->chunk_ready) {
        cudaGraphExecDestroy(b->chunk);
        b->chunk_ready = false;
    }
    b->variant = variant;
    return OFM_OK;
}

extern "C" int ofm_batch_get_variant(ofm_batch* b, int* variant, float* tune_ms) {
    ofm::clear_error();
    if (!b || !variant) return fail(OFM_EINVAL, "NULL argument");
    *variant = b->variant;
    if (tune_ms)
        for (int v = 0; v < OFM_N_VARIANTS; ++v) tune_ms[v] = b->tune_ms[v];
    return OFM_OK;
}

extern "C" int ofm_batch_stage_time(ofm_batch* b, double* total_ms, int64_t* n_launches) {
    ofm::clear_error();
    if (!b || !total_ms || !n_launches) return fail(OFM_EINVAL, "NULL argument");
    *total_ms = b->stage_ms;
    *n_launches = b->stage_launches;
    return OFM_OK;
}

extern "C" int ofm_batch_transfer_bytes(ofm_batch* b, int64_t* h2d, int64_t* d2h) {
    ofm::clear_error();
    if (!b || !h2d || !d2h) return fail(OFM_EINVAL, "NULL argument");
    *h2d = b->h2d_bytes;
    *d2h = b->d2h_bytes;
    return OFM_OK;
}

extern "C" void ofm_batch_destroy(ofm_batch* b) {
    if (!b) return;
    if (b->priv) cudaStreamSynchronize(b->priv);
    for (int k = 0; k < 4; ++k)
        if (b->pev[k]) cudaEventDestroy(b->pev[k]);
    if (b->chunk_ready) cudaGraphExecDestroy(b->chunk);
    if (b->own_ws && b->ws) cudaFree(b->ws);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->priv) cudaStreamDestroy(b->priv);
    delete b;
}

extern "C" int ofm_solve_batch(ofm_solver* s, const ofm_cloud_params* cloud, const ofm_group* groups,
                               int n_groups, void* workspace, size_t workspace_bytes, void* stream) {
    ofm_batch* b = nullptr;
    int rc = ofm_batch_create(&b, s, cloud, groups, n_groups, workspace, workspace_bytes, stream);
    if (rc != OFM_OK) return rc;
    rc = ofm_batch_init(b);
    int active = 1;
    while (rc == OFM_OK && active > 0) rc = ofm_batch_run(b, 1 << 20, &active);
    if (rc == OFM_OK) rc = ofm_batch_qoi(b);
    ofm_batch_destroy(b);
    return rc;
}

extern "C" int ofm_solve_level(ofm_solver* s, const ofm_cloud_params* cloud, int N, int n,
                               const uint64_t* sample_ids, uint64_t seed, ofm_qoi* out, double* sensor_hist,
                               void* workspace, size_t workspace_bytes, void* stream) {
    ofm_group g;
    g.N = N;
    g.n_samples = n;
    g.sample_ids = sample_ids;
    g.seed = seed;
    g.bubbles = nullptr;
    g.qoi_out = out;
    g.sensor_hist = sensor_hist;
    g.alpha_hist = nullptr;
    return ofm_solve_batch(s, cloud, &g, 1, workspace, workspace_bytes, stream);
}
