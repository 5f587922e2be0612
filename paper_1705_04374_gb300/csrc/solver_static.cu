// Allocation-free single-level solve: ofm_solve_level_static.
//
// Some callers cannot call cudaMalloc: a host framework whose caching
// allocator has already reserved the device memory and owns every allocation
// on the device, or a latency-critical loop where cudaMalloc / cudaFree would
// synchronise the device and stall other work.  This entry point allocates no
// device or pinned host memory and creates no streams or events.  Its device
// scratch (the sample states, the 2N registers, the per-tile partial
// reductions, the per-sample records, the uploaded clouds and sensor lists)
// lives in one file-scope __device__ array of OFM_STATIC_SCRATCH_BYTES, which
// every GPU that loads this library holds until the process exits.  It runs
// the same kernels as ofm_solve_level and gives the same results.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (host code cannot use the
// array's name as a device address) and caches it for the device.  Make that
// first call before any stream capture.  The cached address assumes the
// device's primary context lives as long as the process: after
// cudaDeviceReset the module is loaded again and the array may move, so a
// process that resets a device must not call this entry point afterwards.
//
// Every call shares the one array: calls that overlap on the GPU (on
// different streams or host threads) race on it.  Each call re-initialises
// everything it reads (the per-sample records are reset, every partial is
// rewritten before it is read), so nothing carries over between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "host_shared.cuh"
#include "internal.h"
#include "ofmlmc.h"
#include "types.cuh"

using ofm::fail;
using namespace ofm::gpu;

namespace {

static_assert(OFM_STATIC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");

__device__ __align__(256) unsigned char g_scratch[OFM_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
unsigned char* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(OFM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(OFM_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(OFM_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return OFM_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct StaticLayout {
    size_t QA, QB, dQ, part, sens, t, dt, last, done, nsteps, kout, qoi, sold, hist, active, gact, bub, total;
};

StaticLayout static_layout(const ofm_solver* s, int N, int M, int nb, size_t n_sens_cells) {
    const size_t es = s->cfg.precision == OFM_FP64 ? 8 : 4;
    const size_t n3 = (size_t)N * N * N, tps = n3 / (TS * TS * TS), Ms = (size_t)M;
    StaticLayout L;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t o = at;
        at = up256(at + bytes);
        return o;
    };
    L.QA = take(Ms * 7 * n3 * es);
    L.QB = take(Ms * 7 * n3 * es);
    L.dQ = take(Ms * 7 * n3 * es);
    L.part = take(Ms * tps * sizeof(Partial));
    L.sens = take((n_sens_cells ? n_sens_cells : 1) * sizeof(int));
    L.t = take(Ms * 8);
    L.dt = take(Ms * 8);
    L.last = take(Ms * 4);
    L.done = take(Ms * 4);
    L.nsteps = take(Ms * 4);
    L.kout = take(Ms * 4);
    L.qoi = take(Ms * sizeof(DevQoi));
    L.sold = take(Ms * OFM_MAX_SENSORS * 8);
    const size_t n_hist = Ms * s->cfg.n_sensors * s->cfg.n_out_times;
    L.hist = take((n_hist > 0 ? n_hist : 1) * 8);
    L.active = take(16);
    L.gact = take(16);
    const size_t n_bub = Ms * nb;
    L.bub = take((n_bub > 0 ? n_bub : 1) * 32);
    L.total = at;
    return L;
}

template <typename T>
void static_params(const ofm_solver* s, int N, int M, int nb, unsigned char* ws, const StaticLayout& L,
                   const int* sens_off, Params<T>& P) {
    std::memset(&P, 0, sizeof(P));
    const ofm_solver_config& c = s->cfg;
    P.n_groups = 1;
    GroupDev& G = P.g[0];
    G.N = N;
    G.tpd = N / TS;
    G.tps = G.tpd * G.tpd * G.tpd;
    G.n_samples = M;
    G.slot0 = 0;
    G.block0 = 0;
    G.QA = ws + L.QA;
    G.QB = ws + L.QB;
    G.dQ = ws + L.dQ;
    G.part = (Partial*)(ws + L.part);
    G.sens_cells = (const int*)(ws + L.sens);
    for (int k = 0; k <= c.n_sensors; ++k) G.sens_off[k] = sens_off[k];
    G.h = 1.0 / N;
    G.h32 = (float)G.h;
    P.total_blocks = (long long)G.tps * M;
    P.total_slots = M;
    P.s.t = (double*)(ws + L.t);
    P.s.dt = (double*)(ws + L.dt);
    P.s.last = (int*)(ws + L.last);
    P.s.done = (int*)(ws + L.done);
    P.s.nsteps = (int*)(ws + L.nsteps);
    P.s.kout = (int*)(ws + L.kout);
    P.s.qoi = (DevQoi*)(ws + L.qoi);
    P.s.sens_old = (double*)(ws + L.sold);
    P.s.hist = (double*)(ws + L.hist);
    P.s.n_active = (int*)(ws + L.active);
    P.s.g_active = (int*)(ws + L.gact);
    P.s.bubbles = (const double*)(ws + L.bub);
    params_constants(s, nb, P);
}

#define STATIC_TRY(call)                                                                   \
    do {                                                                                   \
        cudaError_t err__ = (call);                                                        \
        if (err__ != cudaSuccess)                                                          \
            return fail(OFM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(err__));     \
    } while (0)

template <typename T>
int run_static(const ofm_solver* s, int N, int M, int nb, unsigned char* ws, const StaticLayout& L,
               const int* sens_off, cudaStream_t st) {
    Params<T> P;
    static_params(s, N, M, nb, ws, L, sens_off, P);
    int rc = group_tensor_maps(P.g[0], sizeof(T));
    if (rc != OFM_OK) return rc;
    rc = set_smem_attrs<T>();
    if (rc != OFM_OK) return rc;
    long long launches = 0;
    rc = launch_init(P, st, true, &launches);
    if (rc != OFM_OK) return rc;
    long long step = 0;
    for (;;) {
        for (int k = 0; k < CHUNK_STEPS; ++k, ++step) {
            rc = launch_step(P, P, OFM_VARIANT_TILES, (int)(step & 1), st, &launches);
            if (rc != OFM_OK) return rc;
        }
        int active = 0;  // pageable host int: no pinned allocation
        STATIC_TRY(cudaMemcpyAsync(&active, ws + L.active, sizeof(int), cudaMemcpyDeviceToHost, st));
        STATIC_TRY(cudaStreamSynchronize(st));
        if (active == 0) break;
    }
    return launch_totals(P, st, 1, &launches);
}

}  // namespace

extern "C" int ofm_solve_level_static(const ofm_solver* s, const ofm_cloud_params* cloud, int N, int n,
                                      const uint64_t* sample_ids, uint64_t seed, ofm_qoi* out,
                                      double* sensor_hist, void* stream) {
    ofm::clear_error();
    if (!s || !cloud || !sample_ids || !out) return fail(OFM_EINVAL, "ofm_solve_level_static: NULL argument");
    if (N < TS || N > 512 || N % TS != 0)
        return fail(OFM_EINVAL, "ofm_solve_level_static: N = %d must be a multiple of %d in [%d, 512]", N, TS, TS);
    if (n < 1 || cloud->n_bubbles < 0) return fail(OFM_EINVAL, "ofm_solve_level_static: bad sample or bubble count");
    const ofm_solver_config& c = s->cfg;
    const int nb = cloud->n_bubbles;

    // sensor membership: the same cells as the batch API's
    std::vector<int> cells;
    int sens_off[OFM_MAX_SENSORS + 1];
    sensor_cell_list(s, N, cells, sens_off);

    // the three state buffers alone bound the sample count; checked by division
    // first, so that the layout's byte counts below cannot wrap around
    const size_t es = c.precision == OFM_FP64 ? 8 : 4;
    const size_t state_bytes = 3 * 7 * (size_t)N * N * N * es;
    if ((size_t)n > OFM_STATIC_SCRATCH_BYTES / state_bytes)
        return fail(OFM_ENOMEM,
                    "ofm_solve_level_static: %d samples on %d^3 need %.4g bytes for their states alone, the static "
                    "array holds %zu (use ofm_solve_level, or fewer / smaller samples)",
                    n, N, (double)n * (double)state_bytes, (size_t)OFM_STATIC_SCRATCH_BYTES);
    const StaticLayout L = static_layout(s, N, n, nb, cells.size());
    if (L.total > OFM_STATIC_SCRATCH_BYTES)
        return fail(OFM_ENOMEM,
                    "ofm_solve_level_static: %d samples on %d^3 need %zu bytes of scratch, the static array holds %zu "
                    "(use ofm_solve_level, or fewer / smaller samples)",
                    n, N, L.total, (size_t)OFM_STATIC_SCRATCH_BYTES);
    unsigned char* ws = nullptr;
    int rc = scratch_address(&ws);
    if (rc != OFM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    // clouds: sampled on the host, non-dimensionalised, copied into the scratch
    std::vector<double> bub((size_t)n * nb * 4);
    std::vector<ofm_bubble> tmp(nb > 0 ? nb : 1);
    size_t at = 0;
    for (int i = 0; i < n; ++i) {
        if ((rc = ofm_sample_cloud(cloud, seed, sample_ids[i], tmp.data())) != OFM_OK) return rc;
        for (int k = 0; k < nb; ++k) {
            bub[at++] = tmp[k].x / s->L;
            bub[at++] = tmp[k].y / s->L;
            bub[at++] = tmp[k].z / s->L;
            bub[at++] = tmp[k].r / s->L;
        }
    }
    if (!bub.empty()) STATIC_TRY(cudaMemcpyAsync(ws + L.bub, bub.data(), bub.size() * 8, cudaMemcpyHostToDevice, st));
    if (!cells.empty())
        STATIC_TRY(cudaMemcpyAsync(ws + L.sens, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice, st));

    rc = c.precision == OFM_FP64 ? run_static<double>(s, N, n, nb, ws, L, sens_off, st)
                                 : run_static<float>(s, N, n, nb, ws, L, sens_off, st);
    if (rc != OFM_OK) return rc;

    std::vector<DevQoi> q(n);
    const size_t per = (size_t)c.n_sensors * c.n_out_times;
    std::vector<double> hist((size_t)n * per);
    STATIC_TRY(cudaMemcpyAsync(q.data(), ws + L.qoi, q.size() * sizeof(DevQoi), cudaMemcpyDeviceToHost, st));
    if (sensor_hist && per)
        STATIC_TRY(cudaMemcpyAsync(hist.data(), ws + L.hist, hist.size() * 8, cudaMemcpyDeviceToHost, st));
    STATIC_TRY(cudaStreamSynchronize(st));
    int any_bad = 0;
    for (int i = 0; i < n; ++i) {
        const DevQoi& d = q[i];
        qoi_to_si(s, N, d, d.t_final, d.n_steps, out[i]);
        if (d.status) any_bad = 1;
        if (sensor_hist && per)
            for (size_t a = 0; a < per; ++a) sensor_hist[(size_t)i * per + a] = hist[(size_t)i * per + a] * s->p_ref;
    }
    if (any_bad) return fail(OFM_ENUMERIC, "some samples have a non-zero status");
    return OFM_OK;
}
