// Batched cloud-collapse solves on one GPU (sm_103a).
//
// The method (Sukys et al. 2017, Sections 2.1-2.2 and 3.1-3.2): the five-
// equation two-phase model with a stiffened-gas isobaric closure, WENO5
// reconstruction of primitive variables, an HLLC flux with an upwind alpha2
// flux and a face velocity for the K div(u) source, a 3-stage low-storage RK
// update and a CFL time step from a max over all cells, plus on-device
// reductions of the quantities of interest.
//
// GPU design
//   * State in HBM as structure of arrays Q[sample][var][z][y][x] (x fastest),
//     three buffers per sample: Q_a, Q_b (ping-pong, because neighbours read
//     the old state while a block writes the new one) and dQ (2N register).
//   * One fused kernel per RK stage.  A block owns an 8x8x8 tile: it stages
//     the tile plus a 3-cell halo along each axis (no corners) into shared
//     memory as primitives, computes every face flux of the tile once (WENO5
//     both sides + HLLC) per direction into shared memory, differences them
//     into per-cell right-hand sides in registers, and applies the 2N update.
//     Per cell and stage, HBM sees only Q, dQ in and Q', dQ out.
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

#include "internal.h"
#include "ofmlmc.h"

using ofm::fail;

namespace {

constexpr int TS = 8;                    // tile edge (cells)
constexpr int HALO = 3;                  // WENO5 needs three cells on each side
constexpr int BX = TS + 2 * HALO;        // staged box edge (14)
constexpr int BOX3 = BX * BX * BX;       // staged box cells (2744, corners unused)
constexpr int NCELL = TS * TS * TS;      // 512 cells per tile
constexpr int NSLAB = HALO * TS * TS;    // 192 cells per halo slab
constexpr int NCROSS = NCELL + 6 * NSLAB;  // 1664 staged cells
constexpr int NFACE = (TS + 1) * TS * TS;  // 576 faces per direction
constexpr int NT = 192;                  // threads per block: 3 faces each per direction
constexpr int CELLS_PER_THREAD = (NCELL + NT - 1) / NT;  // 3
constexpr int CHUNK_STEPS = 8;           // steps per captured graph (even)

static_assert(NFACE % NT == 0, "each thread computes the same number of faces");

template <typename T>
struct Eos {
    T g1, g2, pc1, pc2;   // gamma, p_c (non-dimensional)
    T gi1, gi2;           // 1/(gamma-1)
    T pi1, pi2;           // gamma p_c/(gamma-1)
    T eps;                // WENO epsilon
};

struct Partial {          // per-tile reduction of one state
    double smax;          // max over cells of max_d(|u_d| + c)
    double pmax;          // max pressure
    long long idx;        // first linear index of pmax
    int status;           // OR of health bits
    int pad;
};

struct DevQoi {           // per-sample record, non-dimensional
    double p_peak;
    long long peak_index;
    double p_peak_t;
    double sensor_peak[OFM_MAX_SENSORS];
    double totals0[6];
    double totals_end[6];
    double t_final;
    int n_steps;
    int status;
};

struct GroupDev {
    int N, tpd, tps, n_samples, slot0;
    long long block0;     // first block of this group in the flattened tile grid
    void* QA;
    void* QB;
    void* dQ;
    Partial* part;
    const int* sens_cells;
    int sens_off[OFM_MAX_SENSORS + 1];
    double h;
};

struct SampleDev {
    double* t;
    double* dt;
    int* last;
    int* done;
    int* nsteps;
    int* kout;
    DevQoi* qoi;
    double* sens_old;     // [slot][OFM_MAX_SENSORS]
    double* hist;         // [slot][n_sens][n_out]
    int* n_active;
    const double* bubbles;  // [slot][nb][4], non-dimensional
};

template <typename T>
struct Params {
    int n_groups;
    long long total_blocks;
    GroupDev g[OFM_MAX_GROUPS];
    SampleDev s;
    Eos<T> eos;
    double rkA[3], rkB[3];
    int bc, nb, n_sens, n_out, max_steps, total_slots;
    double t_end, cfl, p_gas, p_liq, rho1, rho2;
};

// Low-storage TVD RK3 (Gottlieb & Shu 1998), Williamson 2N form.
constexpr double RK_A[3] = {0.0, -2.915492524638791, -0.000000093517376};
constexpr double RK_B[3] = {0.924574, 0.287713063186749, 0.626538109512740};

// --------------------------------------------------------------------------
// Closure, reconstruction, Riemann solver
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T clamp01(T a) {
    return a < T(0) ? T(0) : (a > T(1) ? T(1) : a);
}

// Mixture Gamma = sum alpha_k/(g_k - 1), Pi = sum alpha_k g_k pc_k/(g_k - 1)
// (isobaric stiffened-gas closure), alpha2 clamped to [0, 1] for the closure.
template <typename T>
__device__ __forceinline__ void closure(const Eos<T>& e, T a2, T& G, T& Pi) {
    const T a = clamp01(a2);
    const T a1 = T(1) - a;
    G = a1 * e.gi1 + a * e.gi2;
    Pi = a1 * e.pi1 + a * e.pi2;
}

// Q = (a1r1, a2r2, ru, rv, rw, E, a2) -> W = (a1r1, a2r2, u, v, w, p, a2)
template <typename T>
__device__ __forceinline__ void cons2prim(const Eos<T>& e, const T* q, T* w) {
    const T rho = q[0] + q[1];
    const T ir = T(1) / rho;
    const T u = q[2] * ir, v = q[3] * ir, ww = q[4] * ir;
    T G, Pi;
    closure(e, q[6], G, Pi);
    const T ke = T(0.5) * rho * (u * u + v * v + ww * ww);
    w[0] = q[0];
    w[1] = q[1];
    w[2] = u;
    w[3] = v;
    w[4] = ww;
    w[5] = (q[5] - ke - Pi) / G;
    w[6] = q[6];
}

// WENO5 (Jiang & Shu): value at the right face of the cell holding c from the
// averages a..e.  The nonlinear weights d_k/(eps + beta_k)^2 are normalised
// with one division: multiplying all three by the product of the squared
// denominators leaves their ratios unchanged.
template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e, T eps) {
    const T s6 = T(1.0 / 6.0);
    const T q0 = (T(2) * a - T(7) * b + T(11) * c) * s6;
    const T q1 = (-b + T(5) * c + T(2) * d) * s6;
    const T q2 = (T(2) * c + T(5) * d - e) * s6;
    const T k13 = T(13.0 / 12.0);
    T t = a - T(2) * b + c;
    T s = a - T(4) * b + T(3) * c;
    const T b0 = k13 * t * t + T(0.25) * s * s;
    t = b - T(2) * c + d;
    s = b - d;
    const T b1 = k13 * t * t + T(0.25) * s * s;
    t = c - T(2) * d + e;
    s = T(3) * c - T(4) * d + e;
    const T b2 = k13 * t * t + T(0.25) * s * s;
    T e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
    e0 *= e0;
    e1 *= e1;
    e2 *= e2;
    const T w0 = T(0.1) * (e1 * e2);
    const T w1 = T(0.6) * (e0 * e2);
    const T w2 = T(0.3) * (e0 * e1);
    return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

// Face-state admissibility: alpha2 in [0,1], partial densities > 0 and
// p + Pi/(Gamma+1) > 0 (positive squared sound speed).  An inadmissible
// reconstructed state falls back to its cell's value (first order).
template <typename T>
__device__ __forceinline__ bool admissible(const Eos<T>& e, const T* w) {
    if (!(w[6] >= T(0) && w[6] <= T(1))) return false;
    if (!(w[0] > T(0) && w[1] > T(0))) return false;
    T G, Pi;
    closure(e, w[6], G, Pi);
    return w[5] + Pi / (G + T(1)) > T(0);
}

// HLLC flux in direction DIR.  F[0..5]: mass 1, mass 2, momentum x/y/z,
// energy; F[6]: alpha2 flux = alpha2 (upwind by the sign of s*) times the
// face velocity; F[7]: the face velocity (for div u), i.e. the velocity that
// carries mass through the face, u_K + s_K (chi_K - 1), averaged when s* = 0.
template <typename T, int DIR>
__device__ __forceinline__ void hllc(const Eos<T>& e, const T* wl, const T* wr, T* F) {
    const T rL = wl[0] + wl[1], rR = wr[0] + wr[1];
    const T uL = wl[2 + DIR], uR = wr[2 + DIR];
    const T pL = wl[5], pR = wr[5];
    T GL, PiL, GR, PiR;
    closure(e, wl[6], GL, PiL);
    closure(e, wr[6], GR, PiR);
    const T EL = GL * pL + PiL + T(0.5) * rL * (wl[2] * wl[2] + wl[3] * wl[3] + wl[4] * wl[4]);
    const T ER = GR * pR + PiR + T(0.5) * rR * (wr[2] * wr[2] + wr[3] * wr[3] + wr[4] * wr[4]);
    const T cL = sqrt(((GL + T(1)) * pL + PiL) / (GL * rL));
    const T cR = sqrt(((GR + T(1)) * pR + PiR) / (GR * rR));
    const T sL = fmin(uL - cL, uR - cR);
    const T sR = fmax(uL + cL, uR + cR);
    const T ss = (pR - pL + rL * uL * (sL - uL) - rR * uR * (sR - uR)) /
                 (rL * (sL - uL) - rR * (sR - uR));

    T ufL = uL, ufR = uR;
    if (sL < T(0)) {
        const T chi = (sL - uL) / (sL - ss);
        ufL = uL + sL * (chi - T(1));
    }
    if (sR > T(0)) {
        const T chi = (sR - uR) / (sR - ss);
        ufR = uR + sR * (chi - T(1));
    }

    const bool left = ss >= T(0);
    const T m1 = left ? wl[0] : wr[0];
    const T m2 = left ? wl[1] : wr[1];
    const T vx = left ? wl[2] : wr[2];
    const T vy = left ? wl[3] : wr[3];
    const T vz = left ? wl[4] : wr[4];
    const T r = left ? rL : rR;
    const T un = left ? uL : uR;
    const T p = left ? pL : pR;
    const T E = left ? EL : ER;
    const T sK = left ? sL : sR;
    const bool star = left ? (sL < T(0)) : (sR > T(0));

    const T q2 = r * vx, q3 = r * vy, q4 = r * vz;
    T f0 = m1 * un, f1 = m2 * un, f2 = q2 * un, f3 = q3 * un, f4 = q4 * un;
    if (DIR == 0) f2 += p;
    if (DIR == 1) f3 += p;
    if (DIR == 2) f4 += p;
    T f5 = (E + p) * un;
    if (star) {
        const T chi = (sK - un) / (sK - ss);
        const T cr = chi * r;
        const T s2 = DIR == 0 ? cr * ss : cr * vx;
        const T s3 = DIR == 1 ? cr * ss : cr * vy;
        const T s4 = DIR == 2 ? cr * ss : cr * vz;
        const T s5 = chi * (E + (ss - un) * (r * ss + p / (sK - un)));
        f0 = f0 + sK * (chi * m1 - m1);
        f1 = f1 + sK * (chi * m2 - m2);
        f2 = f2 + sK * (s2 - q2);
        f3 = f3 + sK * (s3 - q3);
        f4 = f4 + sK * (s4 - q4);
        f5 = f5 + sK * (s5 - E);
    }
    T uf;
    if (ss > T(0))
        uf = ufL;
    else if (ss < T(0))
        uf = ufR;
    else
        uf = T(0.5) * (ufL + ufR);
    const T a2 = left ? wl[6] : wr[6];
    F[0] = f0;
    F[1] = f1;
    F[2] = f2;
    F[3] = f3;
    F[4] = f4;
    F[5] = f5;
    F[6] = a2 * uf;
    F[7] = uf;
}

// --------------------------------------------------------------------------
// Tile geometry helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ int box_index(int bx, int by, int bz) {
    return ((bz + HALO) * BX + (by + HALO)) * BX + (bx + HALO);
}

// Staged cell i in [0, NCROSS): the tile, then six 3-deep halo slabs
// (x-, x+, y-, y+, z-, z+).  Box coordinates are tile-relative.
__device__ __forceinline__ void cross_decode(int i, int& bx, int& by, int& bz) {
    if (i < NCELL) {
        bx = i & 7;
        by = (i >> 3) & 7;
        bz = i >> 6;
        return;
    }
    const int j = i - NCELL;
    const int slab = j / NSLAB;
    const int r = j - slab * NSLAB;
    const int hi = slab & 1;
    if (slab < 2) {
        const int hx = r % 3, q = r / 3;
        by = q & 7;
        bz = q >> 3;
        bx = hi ? TS + hx : hx - HALO;
    } else if (slab < 4) {
        bx = r & 7;
        const int q = r >> 3;
        const int hy = q % 3;
        bz = q / 3;
        by = hi ? TS + hy : hy - HALO;
    } else {
        bx = r & 7;
        by = (r >> 3) & 7;
        const int hz = r >> 6;
        bz = hi ? TS + hz : hz - HALO;
    }
}

__device__ __forceinline__ int bc_map(int g, int N, int bc) {
    if (bc == OFM_BC_PERIODIC) return g < 0 ? g + N : (g >= N ? g - N : g);
    return g < 0 ? 0 : (g >= N ? N - 1 : g);
}

template <typename T>
struct BlockWork {
    const GroupDev* G;
    int slot, s_local, x0, y0, z0;
};

template <typename T>
__device__ __forceinline__ bool decode_block(const Params<T>& P, long long b, BlockWork<T>& w) {
    int gi = 0;
    while (gi + 1 < P.n_groups && b >= P.g[gi + 1].block0) ++gi;
    const GroupDev& G = P.g[gi];
    const long long local = b - G.block0;
    const int s_local = (int)(local / G.tps);
    const int tile = (int)(local - (long long)s_local * G.tps);
    w.G = &P.g[gi];
    w.s_local = s_local;
    w.slot = G.slot0 + s_local;
    w.x0 = (tile % G.tpd) * TS;
    w.y0 = ((tile / G.tpd) % G.tpd) * TS;
    w.z0 = (tile / (G.tpd * G.tpd)) * TS;
    return true;
}

// --------------------------------------------------------------------------
// Per-cell health / speed / pressure reduction and its block combine
// --------------------------------------------------------------------------
struct Red {
    double smax, pmax;
    long long idx;
    int status;
};

__device__ __forceinline__ void red_init(Red& r) {
    r.smax = 0.0;
    r.pmax = -INFINITY;
    r.idx = 0x7fffffffffffffffLL;
    r.status = 0;
}

__device__ __forceinline__ void red_merge(Red& a, double smax, double pmax, long long idx, int st) {
    a.smax = fmax(a.smax, smax);
    if (pmax > a.pmax || (pmax == a.pmax && idx < a.idx)) {
        a.pmax = pmax;
        a.idx = idx;
    }
    a.status |= st;
}

template <typename T>
__device__ __forceinline__ void red_cell(const Eos<T>& e, const T* q, long long gi, Red& r) {
    T w[7];
    cons2prim(e, q, w);
    int bad = 0;
#pragma unroll
    for (int v = 0; v < 7; ++v)
        if (!isfinite(q[v])) bad |= OFM_ST_NONFINITE;
    if (!isfinite(w[5])) bad |= OFM_ST_NONFINITE;
    T G, Pi;
    closure(e, w[6], G, Pi);
    const T rho = w[0] + w[1];
    const T c2 = ((G + T(1)) * w[5] + Pi) / (G * rho);
    if (!(rho > T(0)) || !(c2 > T(0))) bad |= OFM_ST_NEGATIVE;
    r.status |= bad;
    if (bad) return;
    const T c = sqrt(c2);
    const T s = fmax(fabs(w[2]) + c, fmax(fabs(w[3]) + c, fabs(w[4]) + c));
    r.smax = fmax(r.smax, (double)s);
    if ((double)w[5] > r.pmax) {   // cells arrive in increasing linear index
        r.pmax = (double)w[5];
        r.idx = gi;
    }
}

// Combine a block's per-thread records in a fixed order (warp shuffles, then
// warps in index order) and write one Partial.
__device__ void block_reduce_write(Red r, Partial* out) {
    __shared__ Red sred[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double sm = __shfl_down_sync(0xffffffffu, r.smax, off);
        const double pm = __shfl_down_sync(0xffffffffu, r.pmax, off);
        const long long ix = __shfl_down_sync(0xffffffffu, r.idx, off);
        const int st = __shfl_down_sync(0xffffffffu, r.status, off);
        red_merge(r, sm, pm, ix, st);
    }
    if (lane == 0) sred[warp] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        Red a = sred[0];
        for (int w = 1; w < NT / 32; ++w) red_merge(a, sred[w].smax, sred[w].pmax, sred[w].idx, sred[w].status);
        out->smax = a.smax;
        out->pmax = a.pmax;
        out->idx = a.idx;
        out->status = a.status;
        out->pad = 0;
    }
}

// --------------------------------------------------------------------------
// Kernels
// --------------------------------------------------------------------------

// Per-sample bookkeeping reset.
template <typename T>
__global__ void reset_kernel(const __grid_constant__ Params<T> P) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot == 0) *P.s.n_active = P.total_slots;
    if (slot >= P.total_slots) return;
    P.s.t[slot] = 0.0;
    P.s.dt[slot] = 0.0;
    P.s.last[slot] = 0;
    P.s.done[slot] = 0;
    P.s.nsteps[slot] = 0;
    P.s.kout[slot] = 1;
    DevQoi& q = P.s.qoi[slot];
    q.p_peak = -INFINITY;
    q.peak_index = 0;
    q.p_peak_t = 0.0;
    for (int i = 0; i < OFM_MAX_SENSORS; ++i) q.sensor_peak[i] = 0.0;
    for (int i = 0; i < 6; ++i) q.totals0[i] = q.totals_end[i] = 0.0;
    q.t_final = 0.0;
    q.n_steps = 0;
    q.status = 0;
}

// Initial condition (reading of the smoothing): H = max_b 1/2 (1 - tanh((|x - x_b| - r_b)/h))
// = 1/2 (1 - tanh(min_b (|x - x_b| - r_b)/h)); alpha2 = clamp(H, 1e-6, 1 - 1e-6);
// a1r1 = (1 - alpha2) rho1; a2r2 = alpha2 rho2; p = p_liq + (p_gas - p_liq) H;
// u = 0; E = Gamma p + Pi.  Evaluated in FP64, stored in T.
template <typename T>
__global__ void __launch_bounds__(NT) ic_kernel(const __grid_constant__ Params<T> P) {
    BlockWork<T> bw;
    decode_block(P, blockIdx.x, bw);
    const GroupDev& G = *bw.G;
    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    T* Q = (T*)G.QA + (size_t)bw.s_local * 7 * n3;
    const double* bub = P.s.bubbles + (size_t)bw.slot * P.nb * 4;
    const double h = G.h;
    const double gi1 = 1.0 / ((double)P.eos.g1 - 1.0), gi2 = 1.0 / ((double)P.eos.g2 - 1.0);
    const double pi1 = (double)P.eos.g1 * (double)P.eos.pc1 * gi1;
    const double pi2 = (double)P.eos.g2 * (double)P.eos.pc2 * gi2;
    for (int c = threadIdx.x; c < NCELL; c += NT) {
        const int x = bw.x0 + (c & 7), y = bw.y0 + ((c >> 3) & 7), z = bw.z0 + (c >> 6);
        const double xc = (x + 0.5) * h, yc = (y + 0.5) * h, zc = (z + 0.5) * h;
        double m = INFINITY;
        for (int b = 0; b < P.nb; ++b) {
            const double dx = xc - bub[4 * b], dy = yc - bub[4 * b + 1], dz = zc - bub[4 * b + 2];
            m = fmin(m, sqrt(dx * dx + dy * dy + dz * dz) - bub[4 * b + 3]);
        }
        const double H = P.nb > 0 ? 0.5 * (1.0 - tanh(m / h)) : 0.0;
        const double a2 = fmin(fmax(H, 1e-6), 1.0 - 1e-6);
        const double a1 = 1.0 - a2;
        const double p = P.p_liq + (P.p_gas - P.p_liq) * H;
        const size_t gi = ((size_t)z * N + y) * N + x;
        Q[0 * n3 + gi] = (T)(a1 * P.rho1);
        Q[1 * n3 + gi] = (T)(a2 * P.rho2);
        Q[2 * n3 + gi] = T(0);
        Q[3 * n3 + gi] = T(0);
        Q[4 * n3 + gi] = T(0);
        Q[5 * n3 + gi] = (T)((a1 * gi1 + a2 * gi2) * p + (a1 * pi1 + a2 * pi2));
        Q[6 * n3 + gi] = (T)a2;
    }
}

// Reductions of a stored state (t = 0, or after ofm_batch_set_state).
template <typename T>
__global__ void __launch_bounds__(NT) reduce_kernel(const __grid_constant__ Params<T> P, int parity) {
    BlockWork<T> bw;
    decode_block(P, blockIdx.x, bw);
    const GroupDev& G = *bw.G;
    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    const T* Q = (const T*)(parity ? G.QB : G.QA) + (size_t)bw.s_local * 7 * n3;
    Red r;
    red_init(r);
    for (int c = threadIdx.x; c < NCELL; c += NT) {
        const int x = bw.x0 + (c & 7), y = bw.y0 + ((c >> 3) & 7), z = bw.z0 + (c >> 6);
        const size_t gi = ((size_t)z * N + y) * N + x;
        T q[7];
#pragma unroll
        for (int v = 0; v < 7; ++v) q[v] = Q[v * n3 + gi];
        red_cell(P.eos, q, (long long)gi, r);
    }
    const long long tile = blockIdx.x - G.block0 - (long long)bw.s_local * G.tps;
    block_reduce_write(r, G.part + (size_t)bw.s_local * G.tps + tile);
}

// One RK stage.  parity 0: read Q_a, write Q_b; parity 1: the reverse.
template <typename T, int STAGE>
__global__ void __launch_bounds__(NT) stage_kernel(const __grid_constant__ Params<T> P, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sW = reinterpret_cast<T*>(smem_raw);  // [7][BOX3] primitives
    T* sF = sW + 7 * BOX3;                   // [8][NFACE] face fluxes + face velocity

    BlockWork<T> bw;
    decode_block(P, blockIdx.x, bw);
    if (P.s.done[bw.slot]) return;
    const GroupDev& G = *bw.G;
    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    const size_t soff = (size_t)bw.s_local * 7 * n3;
    const T* __restrict__ Qin = (const T*)(parity ? G.QB : G.QA) + soff;
    T* __restrict__ Qout = (T*)(parity ? G.QA : G.QB) + soff;
    T* __restrict__ dQ = (T*)G.dQ + soff;
    const T dt = (T)P.s.dt[bw.slot];
    const T invh = (T)N;  // h = 1/N exactly, so 1/h is exact
    const Eos<T> e = P.eos;
    const int bc = P.bc;

    // 1. stage the tile and its halo as primitives
    for (int i = threadIdx.x; i < NCROSS; i += NT) {
        int bx, by, bz;
        cross_decode(i, bx, by, bz);
        const int gx = bc_map(bw.x0 + bx, N, bc);
        const int gy = bc_map(bw.y0 + by, N, bc);
        const int gz = bc_map(bw.z0 + bz, N, bc);
        const size_t gi = ((size_t)gz * N + gy) * N + gx;
        T q[7], w[7];
#pragma unroll
        for (int v = 0; v < 7; ++v) q[v] = Qin[v * n3 + gi];
        cons2prim(e, q, w);
        const int bi = box_index(bx, by, bz);
#pragma unroll
        for (int v = 0; v < 7; ++v) sW[v * BOX3 + bi] = w[v];
    }
    __syncthreads();

    T rhs[CELLS_PER_THREAD][7];
    T divu[CELLS_PER_THREAD];
#pragma unroll
    for (int k = 0; k < CELLS_PER_THREAD; ++k) {
        divu[k] = T(0);
#pragma unroll
        for (int v = 0; v < 7; ++v) rhs[k][v] = T(0);
    }

    // 2. faces, direction by direction
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
        const int S = dir == 0 ? 1 : (dir == 1 ? BX : BX * BX);
        for (int f = threadIdx.x; f < NFACE; f += NT) {
            int lx, ly, lz;  // left cell of face f
            if (dir == 0) {
                const int fx = f % 9, q = f / 9;
                lx = fx - 1;
                ly = q & 7;
                lz = q >> 3;
            } else if (dir == 1) {
                lx = f & 7;
                const int q = f >> 3;
                ly = q % 9 - 1;
                lz = q / 9;
            } else {
                lx = f & 7;
                ly = (f >> 3) & 7;
                lz = (f >> 6) - 1;
            }
            const int base = box_index(lx, ly, lz);
            T wl[7], wr[7];
#pragma unroll
            for (int v = 0; v < 7; ++v) {
                const T* Pv = sW + v * BOX3 + base;
                const T m2 = Pv[-2 * S], m1 = Pv[-S], c0 = Pv[0];
                const T p1 = Pv[S], p2 = Pv[2 * S], p3 = Pv[3 * S];
                wl[v] = weno5(m2, m1, c0, p1, p2, e.eps);
                wr[v] = weno5(p3, p2, p1, c0, m1, e.eps);
            }
            if (!admissible(e, wl)) {
#pragma unroll
                for (int v = 0; v < 7; ++v) wl[v] = sW[v * BOX3 + base];
            }
            if (!admissible(e, wr)) {
#pragma unroll
                for (int v = 0; v < 7; ++v) wr[v] = sW[v * BOX3 + base + S];
            }
            T F[8];
            if (dir == 0)
                hllc<T, 0>(e, wl, wr, F);
            else if (dir == 1)
                hllc<T, 1>(e, wl, wr, F);
            else
                hllc<T, 2>(e, wl, wr, F);
#pragma unroll
            for (int v = 0; v < 8; ++v) sF[v * NFACE + f] = F[v];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CELLS_PER_THREAD; ++k) {
            const int c = threadIdx.x + k * NT;
            if (c < NCELL) {
                const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
                int fl, step;
                if (dir == 0) {
                    fl = x + 9 * (y + 8 * z);
                    step = 1;
                } else if (dir == 1) {
                    fl = x + 8 * (y + 9 * z);
                    step = 8;
                } else {
                    fl = x + 8 * (y + 8 * z);
                    step = 64;
                }
#pragma unroll
                for (int v = 0; v < 7; ++v)
                    rhs[k][v] -= (sF[v * NFACE + fl + step] - sF[v * NFACE + fl]) * invh;
                divu[k] += (sF[7 * NFACE + fl + step] - sF[7 * NFACE + fl]) * invh;
            }
        }
        __syncthreads();
    }

    // 3. alpha2 source, 2N update, and (last stage) the new state's reductions
    const T A = (T)P.rkA[STAGE], B = (T)P.rkB[STAGE];
    Red red;
    red_init(red);
#pragma unroll
    for (int k = 0; k < CELLS_PER_THREAD; ++k) {
        const int c = threadIdx.x + k * NT;
        if (c < NCELL) {
            const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
            const int bi = box_index(x, y, z);
            const T p = sW[5 * BOX3 + bi];
            const T a2raw = sW[6 * BOX3 + bi];
            const T a2 = clamp01(a2raw);
            const T a1 = T(1) - a2;
            const T z1 = e.g1 * (p + e.pc1);  // rho_1 c_1^2
            const T z2 = e.g2 * (p + e.pc2);  // rho_2 c_2^2
            const T K = a1 * a2 * (z1 - z2) / (a1 * z2 + a2 * z1);
            rhs[k][6] += (a2raw + K) * divu[k];
            const size_t gi = ((size_t)(bw.z0 + z) * N + (bw.y0 + y)) * N + (bw.x0 + x);
            T qn[7];
#pragma unroll
            for (int v = 0; v < 7; ++v) {
                const T q = Qin[v * n3 + gi];
                T d = dt * rhs[k][v];
                if (STAGE > 0) d = A * dQ[v * n3 + gi] + d;
                dQ[v * n3 + gi] = d;
                qn[v] = q + B * d;
                Qout[v * n3 + gi] = qn[v];
            }
            if (STAGE == 2) red_cell(e, qn, (long long)gi, red);
        }
    }
    if (STAGE == 2) {
        const long long tile = blockIdx.x - G.block0 - (long long)bw.s_local * G.tps;
        block_reduce_write(red, G.part + (size_t)bw.s_local * G.tps + tile);
    }
}

// Pressure at one cell of a stored state (sensor evaluation).
template <typename T>
__device__ double cell_pressure(const Eos<T>& e, const T* Q, size_t n3, long long gi) {
    T q[7], w[7];
#pragma unroll
    for (int v = 0; v < 7; ++v) q[v] = Q[v * n3 + gi];
    cons2prim(e, q, w);
    return (double)w[5];
}

// Per-sample combine of the tile partials and FP64 bookkeeping: time, next
// CFL step (dt = CFL h / max speed, clipped so the last step lands on
// t_end), step count, peak pressure, sensors and their histories.
// first != 0: the t = 0 record.  parity: which buffer holds the new state.
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(const __grid_constant__ Params<T> P, int first, int parity) {
    const int slot = blockIdx.x;
    if (slot >= P.total_slots) return;
    if (P.s.done[slot]) return;
    int gi = 0;
    while (gi + 1 < P.n_groups && slot >= P.g[gi + 1].slot0) ++gi;
    const GroupDev& G = P.g[gi];
    const int s_local = slot - G.slot0;
    const Partial* part = G.part + (size_t)s_local * G.tps;

    Red r;
    red_init(r);
    for (int t = threadIdx.x; t < G.tps; t += blockDim.x)
        red_merge(r, part[t].smax, part[t].pmax, part[t].idx, part[t].status);
    __shared__ Red sred[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double sm = __shfl_down_sync(0xffffffffu, r.smax, off);
        const double pm = __shfl_down_sync(0xffffffffu, r.pmax, off);
        const long long ix = __shfl_down_sync(0xffffffffu, r.idx, off);
        const int st = __shfl_down_sync(0xffffffffu, r.status, off);
        red_merge(r, sm, pm, ix, st);
    }
    if (lane == 0) sred[warp] = r;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x / 32); ++w)
        red_merge(r, sred[w].smax, sred[w].pmax, sred[w].idx, sred[w].status);

    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    const T* Q = (const T*)(parity ? G.QB : G.QA) + (size_t)s_local * 7 * n3;
    double sv[OFM_MAX_SENSORS];
    for (int s = 0; s < P.n_sens; ++s) {
        double acc = 0.0;
        const int a0 = G.sens_off[s], a1 = G.sens_off[s + 1];
        for (int a = a0; a < a1; ++a) acc += cell_pressure(P.eos, Q, n3, G.sens_cells[a]);
        sv[s] = a1 > a0 ? acc / (double)(a1 - a0) : NAN;
    }
    DevQoi& q = P.s.qoi[slot];
    double* old = P.s.sens_old + (size_t)slot * OFM_MAX_SENSORS;
    double* hist = P.s.hist + (size_t)slot * P.n_sens * P.n_out;
    double t;
    int nsteps;
    if (first) {
        q.status = r.status;
        q.p_peak = r.pmax;
        q.peak_index = r.idx;
        q.p_peak_t = 0.0;
        for (int s = 0; s < P.n_sens; ++s) {
            q.sensor_peak[s] = sv[s];
            old[s] = sv[s];
            if (P.n_out > 0) hist[s * P.n_out] = sv[s];
        }
        t = 0.0;
        nsteps = 0;
        P.s.kout[slot] = 1;
    } else {
        const double t_old = P.s.t[slot];
        t = P.s.last[slot] ? P.t_end : t_old + P.s.dt[slot];
        nsteps = P.s.nsteps[slot] + 1;
        q.status |= r.status;
        if (r.pmax > q.p_peak) {
            q.p_peak = r.pmax;
            q.peak_index = r.idx;
            q.p_peak_t = t;
        }
        for (int s = 0; s < P.n_sens; ++s)
            if (sv[s] > q.sensor_peak[s]) q.sensor_peak[s] = sv[s];
        if (P.n_out > 1) {
            int k = P.s.kout[slot];
            while (k < P.n_out) {
                const double tk = ((double)k * P.t_end) / (double)(P.n_out - 1);
                if (tk > t) break;
                const double wgt = (tk - t_old) / (t - t_old);
                for (int s = 0; s < P.n_sens; ++s) hist[s * P.n_out + k] = (1.0 - wgt) * old[s] + wgt * sv[s];
                ++k;
            }
            P.s.kout[slot] = k;
        }
        for (int s = 0; s < P.n_sens; ++s) old[s] = sv[s];
    }
    P.s.t[slot] = t;
    P.s.nsteps[slot] = nsteps;
    bool finished = !(t < P.t_end) || q.status != 0;
    if (!finished && nsteps >= P.max_steps) {
        q.status |= OFM_ST_MAXSTEPS;
        finished = true;
    }
    if (!finished) {
        double dt = P.cfl * G.h / r.smax;
        int last = 0;
        if (t + dt >= P.t_end) {
            dt = P.t_end - t;
            last = 1;
        }
        P.s.dt[slot] = dt;
        P.s.last[slot] = last;
    } else {
        P.s.done[slot] = 1;
        q.t_final = t;
        q.n_steps = nsteps;
        atomicSub(P.s.n_active, 1);
    }
}

// Conserved totals sum Q_v h^3 (v = 0..5) of each sample's current state, in
// FP64 with a fixed summation order.  One block per sample.  which = 0: into
// totals0 (state in Q_a); 1: into totals_end (state in the buffer its own step
// count points to).
template <typename T>
__global__ void __launch_bounds__(256) totals_kernel(const __grid_constant__ Params<T> P, int which) {
    const int slot = blockIdx.x;
    if (slot >= P.total_slots) return;
    int gi = 0;
    while (gi + 1 < P.n_groups && slot >= P.g[gi + 1].slot0) ++gi;
    const GroupDev& G = P.g[gi];
    const int s_local = slot - G.slot0;
    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    const int parity = which ? (P.s.nsteps[slot] & 1) : 0;
    const T* Q = (const T*)(parity ? G.QB : G.QA) + (size_t)s_local * 7 * n3;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (size_t i = threadIdx.x; i < n3; i += blockDim.x)
#pragma unroll
        for (int v = 0; v < 6; ++v) acc[v] += (double)Q[v * n3 + i];
    __shared__ double sacc[6][256];
#pragma unroll
    for (int v = 0; v < 6; ++v) sacc[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int v = 0; v < 6; ++v) sacc[v][threadIdx.x] += sacc[v][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double vol = G.h * G.h * G.h;
        double* dst = which ? P.s.qoi[slot].totals_end : P.s.qoi[slot].totals0;
        for (int v = 0; v < 6; ++v) dst[v] = sacc[v][0] * vol;
    }
}

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

struct ofm_solver {
    ofm_solver_config cfg;
    double p_ref, L, u_ref, t_ref;
};

struct GroupHost {
    int N, M;
    ofm_qoi* qoi_out;
    double* hist_out;
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
    Params<double> pd;
    Params<float> pf;
    size_t off_t, off_dt, off_last, off_done, off_nsteps, off_kout, off_qoi, off_sold, off_hist,
        off_active, off_bub;
};

namespace {

// Sensor membership: cells whose centre lies within max(r, h) of the sensor
// centre (integer-derived coordinates, FP64), listed in increasing linear index.
void sensor_cells(const ofm_solver* s, int N, GroupHost& g) {
    const double h = 1.0 / N;
    g.sens_cells.clear();
    g.sens_off[0] = 0;
    for (int k = 0; k < s->cfg.n_sensors; ++k) {
        const double cx = s->cfg.sensors[k][0] / s->L, cy = s->cfg.sensors[k][1] / s->L;
        const double cz = s->cfg.sensors[k][2] / s->L, r = s->cfg.sensors[k][3] / s->L;
        const double R = r > h ? r : h;
        for (int z = 0; z < N; ++z)
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) {
                    const double dx = (x + 0.5) * h - cx, dy = (y + 0.5) * h - cy, dz = (z + 0.5) * h - cz;
                    if (dx * dx + dy * dy + dz * dz <= R * R) g.sens_cells.push_back((z * N + y) * N + x);
                }
        g.sens_off[k + 1] = (int)g.sens_cells.size();
    }
}

template <typename T>
void fill_params(ofm_batch* b, Params<T>& P) {
    std::memset(&P, 0, sizeof(P));
    const ofm_solver_config& c = b->solver->cfg;
    const double pref = b->solver->p_ref;
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
    P.s.n_active = (int*)(b->ws + b->off_active);
    P.s.bubbles = (const double*)(b->ws + b->off_bub);
    const double g1 = c.gamma[0], g2 = c.gamma[1];
    const double pc1 = c.pc[0] / pref, pc2 = c.pc[1] / pref;
    P.eos.g1 = (T)g1;
    P.eos.g2 = (T)g2;
    P.eos.pc1 = (T)pc1;
    P.eos.pc2 = (T)pc2;
    P.eos.gi1 = (T)(1.0 / (g1 - 1.0));
    P.eos.gi2 = (T)(1.0 / (g2 - 1.0));
    P.eos.pi1 = (T)(g1 * pc1 / (g1 - 1.0));
    P.eos.pi2 = (T)(g2 * pc2 / (g2 - 1.0));
    P.eos.eps = (T)c.weno_eps;
    for (int s = 0; s < 3; ++s) {
        P.rkA[s] = RK_A[s];
        P.rkB[s] = RK_B[s];
    }
    P.bc = c.bc;
    P.nb = b->nb;
    P.n_sens = c.n_sensors;
    P.n_out = c.n_out_times;
    P.max_steps = c.max_steps;
    P.t_end = c.t_end / b->solver->t_ref;
    P.cfl = c.cfl;
    P.p_gas = c.p_gas / pref;
    P.p_liq = c.p_liq / pref;
    P.rho1 = c.rho0[0] / 1000.0;
    P.rho2 = c.rho0[1] / 1000.0;
}

constexpr size_t smem_bytes(size_t elem) { return elem * (7 * BOX3 + 8 * NFACE); }

template <typename T>
int set_smem_attrs() {
    const int bytes = (int)smem_bytes(sizeof(T));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return OFM_OK;
}

template <typename T>
int launch_step(ofm_batch* b, const Params<T>& P, int parity, cudaStream_t st) {
    const size_t sm = smem_bytes(sizeof(T));
    const dim3 grid((unsigned)P.total_blocks);
    stage_kernel<T, 0><<<grid, NT, sm, st>>>(P, parity);
    stage_kernel<T, 1><<<grid, NT, sm, st>>>(P, 1 - parity);
    stage_kernel<T, 2><<<grid, NT, sm, st>>>(P, parity);
    finalize_kernel<T><<<P.total_slots, 256, 0, st>>>(P, 0, 1 - parity);
    b->launches += 4;
    CUDA_TRY(cudaGetLastError());
    return OFM_OK;
}

template <typename T>
int launch_init(ofm_batch* b, const Params<T>& P, cudaStream_t st, bool fill_ic) {
    reset_kernel<T><<<(P.total_slots + 127) / 128, 128, 0, st>>>(P);
    b->launches += 1;
    if (fill_ic) {
        ic_kernel<T><<<(unsigned)P.total_blocks, NT, 0, st>>>(P);
        b->launches += 1;
    }
    reduce_kernel<T><<<(unsigned)P.total_blocks, NT, 0, st>>>(P, 0);
    finalize_kernel<T><<<P.total_slots, 256, 0, st>>>(P, 1, 0);
    totals_kernel<T><<<P.total_slots, 256, 0, st>>>(P, 0);
    b->launches += 3;
    CUDA_TRY(cudaGetLastError());
    return OFM_OK;
}

template <typename T>
int build_chunk(ofm_batch* b, const Params<T>& P) {
    cudaGraph_t graph;
    CUDA_TRY(cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal));
    const long long saved = b->launches;
    for (int k = 0; k < CHUNK_STEPS; ++k) {
        int rc = launch_step(b, P, k & 1, b->priv);
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
        !(c->cfl > 0.0) || !(c->t_end > 0.0) || !(c->weno_eps > 0.0) || !(c->domain_L > 0.0))
        return fail(OFM_EINVAL, "ofm_solver_create: non-physical configuration");
    if (c->precision != OFM_FP64 && c->precision != OFM_FP32)
        return fail(OFM_EINVAL, "ofm_solver_create: precision must be OFM_FP64 or OFM_FP32");
    if (c->bc != OFM_BC_TRANSMISSIVE && c->bc != OFM_BC_PERIODIC)
        return fail(OFM_EINVAL, "ofm_solver_create: unknown boundary condition");
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
    b->off_active = Lo.take(16);
    b->off_bub = Lo.take(std::max<size_t>(1, S * cloud->n_bubbles * 4) * 8);
}

extern "C" int ofm_batch_workspace_bytes(const ofm_solver* s, const ofm_cloud_params* cloud,
                                         const ofm_group* groups, int n_groups, size_t* bytes) {
    ofm::clear_error();
    int rc = check_groups(s, cloud, groups, n_groups);
    if (rc != OFM_OK) return rc;
    if (!bytes) return fail(OFM_EINVAL, "NULL bytes");
    ofm_batch tmp;
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
    ofm_batch* b = new (std::nothrow) ofm_batch;
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
    Layout Lo;
    layout(s, cloud, groups, n_groups, b, Lo);
    int slots = 0;
    for (int g = 0; g < n_groups; ++g) {
        b->gh[g].N = groups[g].N;
        b->gh[g].M = groups[g].n_samples;
        b->gh[g].qoi_out = groups[g].qoi_out;
        b->gh[g].hist_out = groups[g].sensor_hist;
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
        cudaMallocHost((void**)&b->h_active, sizeof(int)) != cudaSuccess)
        return bail(fail(OFM_ECUDA, "stream / event / pinned allocation failed"));
    if (b->precision == OFM_FP64) {
        fill_params(b, b->pd);
        b->total_blocks = b->pd.total_blocks;
        if ((rc = set_smem_attrs<double>()) != OFM_OK) return bail(rc);
    } else {
        fill_params(b, b->pf);
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
    if (enter(b) != OFM_OK) return bail(OFM_ECUDA);
    if (!bub.empty() &&
        cudaMemcpyAsync(b->ws + b->off_bub, bub.data(), bub.size() * 8, cudaMemcpyHostToDevice, b->priv) != cudaSuccess)
        return bail(fail(OFM_ECUDA, "bubble upload failed"));
    for (int g = 0; g < n_groups; ++g) {
        const std::vector<int>& sc = b->gh[g].sens_cells;
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
    rc = b->precision == OFM_FP64 ? launch_init(b, b->pd, b->priv, true) : launch_init(b, b->pf, b->priv, true);
    if (rc != OFM_OK) return rc;
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
    while (done_steps < max_steps) {
        if ((b->global_steps & 1) == 0 && max_steps - done_steps >= CHUNK_STEPS) {
            if (!b->chunk_ready) {
                rc = b->precision == OFM_FP64 ? build_chunk(b, b->pd) : build_chunk(b, b->pf);
                if (rc != OFM_OK) return rc;
            }
            CUDA_TRY(cudaGraphLaunch(b->chunk, b->priv));
            b->launches += 4 * CHUNK_STEPS;
            b->global_steps += CHUNK_STEPS;
            done_steps += CHUNK_STEPS;
        } else {
            const int parity = (int)(b->global_steps & 1);
            rc = b->precision == OFM_FP64 ? launch_step(b, b->pd, parity, b->priv)
                                          : launch_step(b, b->pf, parity, b->priv);
            if (rc != OFM_OK) return rc;
            b->global_steps += 1;
            done_steps += 1;
        }
        const size_t off = b->off_active;
        CUDA_TRY(cudaMemcpyAsync(b->h_active, b->ws + off, sizeof(int), cudaMemcpyDeviceToHost, b->priv));
        CUDA_TRY(cudaStreamSynchronize(b->priv));
        active = *b->h_active;
        if (active == 0) break;
    }
    if (n_active) *n_active = active;
    return leave(b);
}

extern "C" int ofm_batch_qoi(ofm_batch* b) {
    ofm::clear_error();
    if (!b || !b->initialised) return fail(OFM_EINVAL, "ofm_batch_qoi: batch not initialised");
    int rc = enter(b);
    if (rc != OFM_OK) return rc;
    if (b->precision == OFM_FP64)
        totals_kernel<double><<<b->total_slots, 256, 0, b->priv>>>(b->pd, 1);
    else
        totals_kernel<float><<<b->total_slots, 256, 0, b->priv>>>(b->pf, 1);
    b->launches += 1;
    CUDA_TRY(cudaGetLastError());
    const ofm_solver_config& c = b->solver->cfg;
    std::vector<DevQoi> q(b->total_slots);
    std::vector<int> nsteps(b->total_slots), done(b->total_slots);
    std::vector<double> tt(b->total_slots);
    const size_t hist_n = (size_t)b->total_slots * c.n_sensors * c.n_out_times;
    std::vector<double> hist(hist_n);
    CUDA_TRY(cudaMemcpyAsync(q.data(), b->ws + b->off_qoi, q.size() * sizeof(DevQoi), cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaMemcpyAsync(nsteps.data(), b->ws + b->off_nsteps, nsteps.size() * 4, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaMemcpyAsync(done.data(), b->ws + b->off_done, done.size() * 4, cudaMemcpyDeviceToHost, b->priv));
    CUDA_TRY(cudaMemcpyAsync(tt.data(), b->ws + b->off_t, tt.size() * 8, cudaMemcpyDeviceToHost, b->priv));
    if (hist_n)
        CUDA_TRY(cudaMemcpyAsync(hist.data(), b->ws + b->off_hist, hist_n * 8, cudaMemcpyDeviceToHost, b->priv));
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
            if (gh.qoi_out) {
                ofm_qoi& o = gh.qoi_out[i];
                std::memset(&o, 0, sizeof(o));
                o.p_peak = d.p_peak * s->p_ref;
                o.peak_index = d.peak_index;
                const long long k = d.peak_index;
                const double h = 1.0 / N;
                o.p_peak_xyz[0] = ((k % N) + 0.5) * h * s->L;
                o.p_peak_xyz[1] = (((k / N) % N) + 0.5) * h * s->L;
                o.p_peak_xyz[2] = ((k / ((long long)N * N)) + 0.5) * h * s->L;
                const double cx = 0.5 * s->L;
                o.p_peak_dist = std::sqrt((o.p_peak_xyz[0] - cx) * (o.p_peak_xyz[0] - cx) +
                                          (o.p_peak_xyz[1] - cx) * (o.p_peak_xyz[1] - cx) +
                                          (o.p_peak_xyz[2] - cx) * (o.p_peak_xyz[2] - cx));
                o.p_peak_t = d.p_peak_t * s->t_ref;
                for (int k2 = 0; k2 < c.n_sensors; ++k2) o.sensor_peak[k2] = d.sensor_peak[k2] * s->p_ref;
                for (int v = 0; v < 6; ++v) {
                    o.totals0[v] = d.totals0[v];
                    o.totals_end[v] = d.totals_end[v];
                }
                o.t_final = (done[slot] ? d.t_final : tt[slot]) * s->t_ref;
                o.n_steps = done[slot] ? d.n_steps : nsteps[slot];
                o.status = d.status;
            }
            if (gh.hist_out && hist_n) {
                const size_t per = (size_t)c.n_sensors * c.n_out_times;
                for (size_t a = 0; a < per; ++a) gh.hist_out[(size_t)i * per + a] = hist[(size_t)slot * per + a] * s->p_ref;
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
    size_t off, n;
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
    size_t off, n;
    int rc = locate(b, group, sample, bytes, &off, &n);
    if (rc != OFM_OK) return rc;
    if (!host_buf) return fail(OFM_EINVAL, "NULL buffer");
    if (!b->initialised || b->global_steps != 0)
        return fail(OFM_EINVAL, "ofm_batch_set_state: only between ofm_batch_init and the first step");
    rc = enter(b);
    if (rc != OFM_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(b->ws + b->gh[group].off_QA + off, host_buf, n, cudaMemcpyHostToDevice, b->priv));
    rc = b->precision == OFM_FP64 ? launch_init(b, b->pd, b->priv, false) : launch_init(b, b->pf, b->priv, false);
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

extern "C" void ofm_batch_destroy(ofm_batch* b) {
    if (!b) return;
    if (b->priv) cudaStreamSynchronize(b->priv);
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
    return ofm_solve_batch(s, cloud, &g, 1, workspace, workspace_bytes, stream);
}
