// Device code of the solver, included once per precision (see types.cuh).
//
// The method (Sukys et al. 2017, Sections 2.1-2.2 and 3.1-3.2): the five-
// equation two-phase model with a stiffened-gas isobaric closure, WENO5 (or
// the third-order WENO3) reconstruction of primitive variables, an HLLC flux
// with an upwind alpha2 flux and a face velocity for the K div(u) source, a
// 3-stage low-storage RK update and a CFL time step from a max over all
// cells, transmissive, periodic or characteristic far-field ghost cells, plus
// on-device reductions of the quantities of interest.
//
// In double precision the arithmetic follows the FP64 reference's operation
// order exactly and this file is compiled without FMA contraction, so both
// round identically; in single precision it uses cheaper but equivalent forms
// (reciprocal products, one division for the WENO weights, FMA).
#pragma once

#include <type_traits>

#include "internal.h"
#include "types.cuh"

namespace ofm {
namespace gpu {
namespace {

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
    T u, v, ww;
    if constexpr (std::is_same<T, double>::value) {
        u = q[2] / rho;
        v = q[3] / rho;
        ww = q[4] / rho;
    } else {
        const T ir = T(1) / rho;
        u = q[2] * ir;
        v = q[3] * ir;
        ww = q[4] * ir;
    }
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
// averages a..e, ideal weights (1/10, 6/10, 3/10), alpha_k = d_k/(eps + beta_k)^2.
// In single precision the weights are normalised with one division:
// multiplying all three by the product of the squared denominators leaves
// their ratios unchanged.
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
    if constexpr (std::is_same<T, double>::value) {
        const T w0 = T(0.1) / ((eps + b0) * (eps + b0));
        const T w1 = T(0.6) / ((eps + b1) * (eps + b1));
        const T w2 = T(0.3) / ((eps + b2) * (eps + b2));
        return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
    } else {
        T e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
        e0 *= e0;
        e1 *= e1;
        e2 *= e2;
        const T w0 = T(0.1) * (e1 * e2);
        const T w1 = T(0.6) * (e0 * e2);
        const T w2 = T(0.3) * (e0 * e1);
        return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
    }
}

// WENO3 (Jiang & Shu, the third-order option): value at the right face of
// the cell holding b from the averages a, b, c; candidates (3b - a)/2 and
// (b + c)/2, smoothness (b - a)^2 and (c - b)^2, ideal weights (1/3, 2/3).
// Double precision in the FP64 reference's order; single precision with the
// weights multiplied by 3 (eps + beta_0)^2 (eps + beta_1)^2 and one division.
template <typename T>
__device__ __forceinline__ T weno3(T a, T b, T c, T eps) {
    const T q0 = T(0.5) * (T(3) * b - a);
    const T q1 = T(0.5) * (b + c);
    const T b0 = (b - a) * (b - a);
    const T b1 = (c - b) * (c - b);
    if constexpr (std::is_same<T, double>::value) {
        const T w0 = T(1.0 / 3.0) / ((eps + b0) * (eps + b0));
        const T w1 = T(2.0 / 3.0) / ((eps + b1) * (eps + b1));
        return (w0 * q0 + w1 * q1) / (w0 + w1);
    } else {
        T e0 = eps + b0, e1 = eps + b1;
        e0 *= e0;
        e1 *= e1;
        const T w0 = e1, w1 = T(2) * e0;
        return (w0 * q0 + w1 * q1) / (w0 + w1);
    }
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

// The same test in single precision without the division ((Gamma+1) > 0),
// also returning the state's closure for the Riemann solver.
__device__ __forceinline__ bool admissible_f(const Eos<float>& e, const float* w, float& G, float& Pi) {
    closure(e, w[6], G, Pi);
    return w[6] >= 0.0f && w[6] <= 1.0f && w[0] > 0.0f && w[1] > 0.0f && (G + 1.0f) * w[5] + Pi > 0.0f;
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
// Staging layout of the tile and its halo (no corners), rows along x, every
// row starting on a 16-byte boundary so that rows are copied 16 bytes at a
// time.  Rows whose (y, z) both lie in the tile have RW = 16 slots holding
// x = -4..11 (the stencils read x = -3..10; slots 0 and 15 are padding); rows
// of the y- and z-halo slabs hold x = 0..7.  Each of the five regions (the
// tile's rows, the low and high y slab, the low and high z slab) is one dense
// box in (x, y, z) order in the dense layout (stage_slot has both layouts).
constexpr int RW = 16;                                 // slots of a full-width row
constexpr int XOFF = 4;                                // slot of x = 0 in a full-width row
constexpr int ROWS_INT = TS * TS * RW;                 // 1024 slots in full-width rows
constexpr int ROWS_Y = ROWS_INT + 2 * HALO * TS * TS;  // start of z-halo rows (1408)
static_assert(ROWS_Y + 2 * HALO * TS * TS == NCROSS, "staging layout size");

// Two layouts of the same regions.  LAYOUT_DENSE: every region one dense
// box (the tensor copies of the persistent variant land it so).
// LAYOUT_SWZ (the default kernel, staged by per-row cp.async): the 16-byte
// chunks of each 32-slot group of the tile's rows are XOR-permuted by a
// linear function of the group index (rows_xor), and each 16-byte chunk of
// the halo slabs has its own place (c_slab), so that the stencil loads of the
// face runs and far faces spread over the shared-memory banks (a search over
// the kernel's access patterns: 327 instead of 864 wavefronts per tile and
// variable; the x runs, whose lanes read cells of one parity, stay two-way).
// Chunks stay whole and 16-byte aligned, so every copy is unchanged in size.
constexpr int LAYOUT_DENSE = 0, LAYOUT_SWZ = 1;

// XOR mask (in slots) of tile row `row` = z TS + y: bits 2-4 from the XOR of
// (1, 6, 4, 1, 4) over the set bits of row >> 1.
__device__ __forceinline__ int rows_xor(int row) {
    const int g = row >> 1;
    const int s = ((g & 1) ? 1 : 0) ^ ((g & 2) ? 6 : 0) ^ ((g & 4) ? 4 : 0) ^ ((g & 8) ? 1 : 0) ^ ((g & 16) ? 4 : 0);
    return s << 2;
}

// Slot offsets of the halo slabs' chunks in LAYOUT_SWZ, [y slab, z slab][((side
// 3 + layer) 8 + other coordinate) 2 + half], half = x >> 2.
__constant__ short c_slab[2][96] = {
    {
        0, 12, 16, 28, 4, 8, 20, 24, 48, 60, 44, 32, 64, 40, 36, 72,
        56, 52, 68, 104, 88, 76, 108, 96, 136, 100, 120, 84, 128, 140, 80, 92,
        168, 132, 152, 116, 172, 160, 112, 124, 184, 148, 164, 200, 156, 144, 192, 204,
        196, 232, 180, 216, 264, 228, 188, 176, 248, 212, 244, 208, 236, 280, 260, 296,
        312, 276, 240, 224, 220, 272, 268, 256, 328, 292, 324, 288, 304, 252, 336, 284,
        316, 308, 300, 320, 344, 348, 340, 332, 352, 380, 372, 356, 360, 364, 376, 368,
    },
    {
        4, 8, 20, 24, 28, 16, 0, 56, 48, 60, 12, 32, 64, 40, 44, 92,
        96, 88, 128, 76, 120, 52, 72, 36, 68, 104, 152, 84, 100, 184, 116, 136,
        160, 108, 124, 80, 168, 132, 164, 200, 148, 216, 196, 232, 156, 112, 248, 180,
        188, 212, 280, 244, 144, 264, 220, 176, 252, 208, 140, 192, 312, 276, 228, 296,
        240, 172, 328, 260, 284, 272, 224, 204, 236, 256, 316, 304, 288, 268, 308, 344,
        292, 340, 348, 324, 300, 332, 336, 320, 356, 368, 380, 360, 352, 376, 364, 372,
    }};

// Staged slot of cell (x, y, z) of the tile and its halo (no corners): x in
// -4..11 for the tile's rows, 0..7 for the slab rows.
template <int LAYOUT>
__device__ __forceinline__ int stage_slot(int x, int y, int z) {
    const bool yi = (unsigned)y < (unsigned)TS, zi = (unsigned)z < (unsigned)TS;
    if (yi && zi) {
        const int row = z * TS + y;
        const int s = row * RW + XOFF + x;
        return LAYOUT == LAYOUT_SWZ ? s ^ rows_xor(row) : s;
    }
    if (zi) {   // y slab, layer y' = 0..2 (low side: y = -3..-1, high side: y = 8..10)
        const int side = y < 0 ? 0 : 1, hy = y < 0 ? y + HALO : y - TS;
        if (LAYOUT == LAYOUT_SWZ) return ROWS_INT + c_slab[0][((side * HALO + hy) * TS + z) * 2 + (x >> 2)] + (x & 3);
        return ROWS_INT + side * NSLAB + (z * HALO + hy) * TS + x;
    }
    const int side = z < 0 ? 0 : 1, hz = z < 0 ? z + HALO : z - TS;
    if (LAYOUT == LAYOUT_SWZ) return ROWS_Y + c_slab[1][((side * HALO + hz) * TS + y) * 2 + (x >> 2)] + (x & 3);
    return ROWS_Y + side * NSLAB + (hz * TS + y) * TS + x;
}

// Staged slot i in [0, NCROSS) that holds no stencil cell (row padding).
template <int LAYOUT>
__device__ __forceinline__ bool pad_slot(int i) {
    if (i >= ROWS_INT) return false;
    const int u = LAYOUT == LAYOUT_SWZ ? i ^ rows_xor((i >> 5) << 1) : i;   // one mask per 32-slot group
    return (u & (RW - 1)) == 0 || (u & (RW - 1)) == RW - 1;
}

// The per-row table: sRows[(z + HALO) BX + y + HALO] = (slot of x = 0, slot
// of x = 4) of row (y, z).  slot_lo: cells x = 0..7 of any row; slot_x:
// cells x = -4..11 of a tile row (its slots are the dense ones XOR one mask).
__device__ __forceinline__ int slot_lo(const int2* __restrict__ sRows, int y, int z, int x) {
    const int* t = reinterpret_cast<const int*>(sRows) + 2 * ((z + HALO) * BX + y + HALO);
    return t[x >> 2] + (x & 3);
}
__device__ __forceinline__ int row_xmask(const int2* __restrict__ sRows, int y, int z, int& base) {
    base = (z * TS + y) * RW + XOFF;
    return sRows[(z + HALO) * BX + y + HALO].x ^ base;
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
    double smax, cmax, pmax;
    long long idx;
    int status;
};

__device__ __forceinline__ void red_init(Red& r) {
    r.smax = 0.0;
    r.cmax = 0.0;
    r.pmax = -INFINITY;
    r.idx = 0x7fffffffffffffffLL;
    r.status = 0;
}

__device__ __forceinline__ void red_merge(Red& a, double smax, double cmax, double pmax, long long idx, int st) {
    a.smax = fmax(a.smax, smax);
    a.cmax = fmax(a.cmax, cmax);
    if (pmax > a.pmax || (pmax == a.pmax && idx < a.idx)) {
        a.pmax = pmax;
        a.idx = idx;
    }
    a.status |= st;
}

// A thread's running record in the stencil precision: maxima and the first
// maximiser need no wider type (conversion to double is exact and monotone),
// and single-precision compares avoid the slow FP64 pipe in the cell loop.
template <typename T>
struct RedT {
    T smax, cmax, pmax;
    long long idx;
    int status;
};

template <typename T>
__device__ __forceinline__ void red_init(RedT<T>& r) {
    r.smax = T(0);
    r.cmax = T(0);
    r.pmax = -INFINITY;
    r.idx = 0x7fffffffffffffffLL;
    r.status = 0;
}

template <typename T>
__device__ __forceinline__ Red red_widen(const RedT<T>& r) {
    Red o;
    o.smax = (double)r.smax;
    o.cmax = (double)r.cmax;
    o.pmax = (double)r.pmax;
    o.idx = r.idx;
    o.status = r.status;
    return o;
}

template <typename T>
__device__ __forceinline__ void red_cell(const Eos<T>& e, const T* q, long long gi, RedT<T>& r) {
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
    r.smax = fmax(r.smax, s);
    r.cmax = fmax(r.cmax, c);
    if (w[5] > r.pmax) {   // cells arrive in increasing linear index
        r.pmax = w[5];
        r.idx = gi;
    }
}

template <typename T>
__device__ __forceinline__ void red_merge(RedT<T>& a, T smax, T cmax, T pmax, long long idx, int st) {
    a.smax = fmax(a.smax, smax);
    a.cmax = fmax(a.cmax, cmax);
    if (pmax > a.pmax || (pmax == a.pmax && idx < a.idx)) {
        a.pmax = pmax;
        a.idx = idx;
    }
    a.status |= st;
}

// Combine a block's per-thread records in a fixed order (warp shuffles, then
// warps in index order) in the stencil precision and write one Partial
// (widened at the end: the same bits as a reduction in double, since the
// conversion is exact and monotone, without single-lane FP64 compares).
template <typename T>
__device__ void block_reduce_write(RedT<T> r, Partial* out) {
    __shared__ RedT<T> sred[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T sm = __shfl_down_sync(0xffffffffu, r.smax, off);
        const T cm = __shfl_down_sync(0xffffffffu, r.cmax, off);
        const T pm = __shfl_down_sync(0xffffffffu, r.pmax, off);
        const long long ix = __shfl_down_sync(0xffffffffu, r.idx, off);
        const int st = __shfl_down_sync(0xffffffffu, r.status, off);
        red_merge(r, sm, cm, pm, ix, st);
    }
    if (lane == 0) sred[warp] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        RedT<T> a = sred[0];
        for (int w = 1; w < NT / 32; ++w)
            red_merge(a, sred[w].smax, sred[w].cmax, sred[w].pmax, sred[w].idx, sred[w].status);
        const Red o = red_widen(a);
        out->smax = o.smax;
        out->cmax = o.cmax;
        out->pmax = o.pmax;
        out->idx = o.idx;
        out->status = o.status;
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
    if (slot == 0) {
        *P.s.n_active = P.total_slots;
        for (int g = 0; g < P.n_groups; ++g) P.s.g_active[g] = P.g[g].n_samples;
    }
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
// a1r1 = (1 - alpha2) rho1; a2r2 = alpha2 rho2; p = p_l + (p_gas - p_l) H with the
// liquid pressure p_l = p_liq, or with the cloud ramp of Sec. 3.1 (ramp_r0 > 0, r the
// distance from the domain centre) p_l = p_cloud for r <= ramp_r0 and
// p_liq + (p_cloud - p_liq) ramp_r0 / r beyond; u = 0; E = Gamma p + Pi.
// Evaluated in FP64, stored in T.
//
// The minimum over bubbles runs over the tile's candidates only: with B the
// box of the tile's cell centres, a bubble whose surface distance to B from
// below (its distance to B minus r_b) exceeds U, the smallest distance bound
// from above (the farthest corner of B minus r_b), by more than a rounding
// margin is never the nearest for any cell of the tile, and fmin over the rest
// gives the same bits (fmin is exact and order-free on finite values).
constexpr int IC_MAX_CAND = 2048;   // larger clouds take the plain loop over every bubble

template <typename T>
__global__ void __launch_bounds__(NT) ic_kernel(const __grid_constant__ Params<T> P) {
    __shared__ int s_cand[IC_MAX_CAND];
    __shared__ int s_ncand;
    __shared__ double s_umin[NT / 32];
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
    const bool cull = P.nb <= IC_MAX_CAND;
    if (cull) {
        const double lo[3] = {(bw.x0 + 0.5) * h, (bw.y0 + 0.5) * h, (bw.z0 + 0.5) * h};
        const double hi[3] = {(bw.x0 + TS - 0.5) * h, (bw.y0 + TS - 0.5) * h, (bw.z0 + TS - 0.5) * h};
        // U: the smallest upper bound of a bubble's surface distance over the box
        double u = INFINITY;
        for (int b = threadIdx.x; b < P.nb; b += NT) {
            double f2 = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double d = fmax(fabs(bub[4 * b + k] - lo[k]), fabs(bub[4 * b + k] - hi[k]));
                f2 += d * d;
            }
            u = fmin(u, sqrt(f2) - bub[4 * b + 3]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) u = fmin(u, __shfl_xor_sync(0xffffffffu, u, off));
        if ((threadIdx.x & 31) == 0) s_umin[threadIdx.x >> 5] = u;
        if (threadIdx.x == 0) s_ncand = 0;
        __syncthreads();
        double U = s_umin[0];
        for (int w = 1; w < NT / 32; ++w) U = fmin(U, s_umin[w]);
        const double margin = 1e-9;   // far above the rounding of any distance in the unit domain
        for (int b = threadIdx.x; b < P.nb; b += NT) {
            double n2 = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double c = bub[4 * b + k];
                const double d = c < lo[k] ? lo[k] - c : (c > hi[k] ? c - hi[k] : 0.0);
                n2 += d * d;
            }
            if (sqrt(n2) - bub[4 * b + 3] <= U + margin) s_cand[atomicAdd(&s_ncand, 1)] = b;
        }
        __syncthreads();
    }
    const int n_try = cull ? s_ncand : P.nb;
    for (int c = threadIdx.x; c < NCELL; c += NT) {
        const int x = bw.x0 + (c & 7), y = bw.y0 + ((c >> 3) & 7), z = bw.z0 + (c >> 6);
        const double xc = (x + 0.5) * h, yc = (y + 0.5) * h, zc = (z + 0.5) * h;
        double m = INFINITY;
        for (int i = 0; i < n_try; ++i) {
            const int b = cull ? s_cand[i] : i;
            const double dx = xc - bub[4 * b], dy = yc - bub[4 * b + 1], dz = zc - bub[4 * b + 2];
            m = fmin(m, sqrt(dx * dx + dy * dy + dz * dz) - bub[4 * b + 3]);
        }
        const double H = P.nb > 0 ? 0.5 * (1.0 - tanh(m / h)) : 0.0;
        const double a2 = fmin(fmax(H, 1e-6), 1.0 - 1e-6);
        const double a1 = 1.0 - a2;
        double pl = P.p_liq;
        if (P.ramp_r0 > 0.0) {
            const double cx = xc - 0.5 * N * h, cy = yc - 0.5 * N * h, cz = zc - 0.5 * N * h;
            const double r = sqrt(cx * cx + cy * cy + cz * cz);
            pl = r <= P.ramp_r0 ? P.p_cloud : P.p_liq + (P.p_cloud - P.p_liq) * P.ramp_r0 / r;
        }
        const double p = pl + (P.p_gas - pl) * H;
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
    RedT<T> r;
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

// Both WENO5 face states of the face between the cells holding c0 and p1,
// from the six averages m2..p3, in single precision.  Same algebra as the
// textbook form, arranged to share work between the two sides:
//   * first differences d_j and second differences D_j = d_j - d_{j-1};
//   * 4 beta_k = (13/3) D^2 + t^2 with t = D +- 2d or d + d'; scaling every
//     beta and eps by 4 scales every (eps + beta)^2 by 16, which cancels in
//     the normalised weights;
//   * candidates as increments on the cell value: q_k - v = D/3 + d/2,
//     -D/6 + d/2, ...; the weights multiply out the three squared
//     denominators so one division normalises them.
__device__ __forceinline__ void weno5_pair(float m2, float m1, float c0, float p1, float p2, float p3,
                                           float eps4, float& wl, float& wr) {
    const float d0 = m1 - m2, d1 = c0 - m1, d2 = p1 - c0, d3 = p2 - p1, d4 = p3 - p2;
    const float Dm = d1 - d0, D0 = d2 - d1, D1 = d3 - d2, D2 = d4 - d3;
    const float k = 13.0f / 3.0f;
    const float sm = fmaf(k * Dm, Dm, eps4), s0 = fmaf(k * D0, D0, eps4);
    const float s1 = fmaf(k * D1, D1, eps4), s2 = fmaf(k * D2, D2, eps4);
    const float hd2 = 0.5f * d2;
    {   // left state (cell c0), face to its right
        const float t0 = fmaf(2.0f, d1, Dm), t1 = d1 + d2, t2 = fmaf(-2.0f, d2, D1);
        float e0 = fmaf(t0, t0, sm), e1 = fmaf(t1, t1, s0), e2 = fmaf(t2, t2, s1);
        e0 *= e0;
        e1 *= e1;
        e2 *= e2;
        const float a0 = e1 * e2, a1 = 6.0f * (e0 * e2), a2 = 3.0f * (e0 * e1);
        const float q0 = fmaf(Dm, 1.0f / 3.0f, 0.5f * d1);
        const float q1 = fmaf(D0, -1.0f / 6.0f, hd2);
        const float q2 = fmaf(D1, -1.0f / 6.0f, hd2);
        wl = c0 + fmaf(a0, q0, fmaf(a1, q1, a2 * q2)) / (a0 + a1 + a2);
    }
    {   // right state (cell p1, mirrored stencil), face to its left
        const float t0 = fmaf(-2.0f, d3, D2), t1 = d2 + d3, t2 = fmaf(2.0f, d2, D0);
        float e0 = fmaf(t0, t0, s2), e1 = fmaf(t1, t1, s1), e2 = fmaf(t2, t2, s0);
        e0 *= e0;
        e1 *= e1;
        e2 *= e2;
        const float a0 = e1 * e2, a1 = 6.0f * (e0 * e2), a2 = 3.0f * (e0 * e1);
        const float q0 = fmaf(D2, 1.0f / 3.0f, -0.5f * d3);
        const float q1 = fmaf(D1, -1.0f / 6.0f, -hd2);
        const float q2 = fmaf(D0, -1.0f / 6.0f, -hd2);
        wr = p1 + fmaf(a0, q0, fmaf(a1, q1, a2 * q2)) / (a0 + a1 + a2);
    }
}

// HLLC in the face frame (un normal, ut1/ut2 tangential), single precision.
// Output: F[0..1] masses, F[2] normal momentum, F[3..4] tangential momenta,
// F[5] energy, F[6] alpha2 flux, F[7] face velocity.
// (GL, PiL), (GR, PiR): the closure of each side.
__device__ __forceinline__ void hllc_frame(const float* wl, const float* wr, float GL, float PiL, float GR, float PiR,
                                           float* F) {
    const float rL = wl[0] + wl[1], rR = wr[0] + wr[1];
    const float uL = wl[2], uR = wr[2];
    const float pL = wl[5], pR = wr[5];
    const float EL = GL * pL + PiL + 0.5f * rL * (wl[2] * wl[2] + wl[3] * wl[3] + wl[4] * wl[4]);
    const float ER = GR * pR + PiR + 0.5f * rR * (wr[2] * wr[2] + wr[3] * wr[3] + wr[4] * wr[4]);
    const float cL = sqrtf(((GL + 1.0f) * pL + PiL) / (GL * rL));
    const float cR = sqrtf(((GR + 1.0f) * pR + PiR) / (GR * rR));
    const float sL = fminf(uL - cL, uR - cR);
    const float sR = fmaxf(uL + cL, uR + cR);
    const float mL = rL * (sL - uL), mR = rR * (sR - uR);
    const float ss = (pR - pL + uL * mL - uR * mR) / (mL - mR);
    float ufL = uL, ufR = uR;
    if (sL < 0.0f) ufL = uL + sL * ((sL - uL) / (sL - ss) - 1.0f);
    if (sR > 0.0f) ufR = uR + sR * ((sR - uR) / (sR - ss) - 1.0f);
    const bool left = ss >= 0.0f;
    const float* w = left ? wl : wr;
    const float r = left ? rL : rR, un = left ? uL : uR, p = left ? pL : pR, E = left ? EL : ER;
    const float sK = left ? sL : sR;
    const bool star = left ? (sL < 0.0f) : (sR > 0.0f);
    const float m1 = w[0], m2 = w[1], t1 = w[3], t2 = w[4];
    const float qn = r * un, q1 = r * t1, q2 = r * t2;
    float f0 = m1 * un, f1 = m2 * un, fn = qn * un + p, f1t = q1 * un, f2t = q2 * un, f5 = (E + p) * un;
    if (star) {
        const float chi = (sK - un) / (sK - ss);
        const float cm1 = chi - 1.0f;
        const float cr = chi * r;
        f0 += sK * (cm1 * m1);
        f1 += sK * (cm1 * m2);
        fn += sK * (cr * ss - qn);
        f1t += sK * (cm1 * q1);
        f2t += sK * (cm1 * q2);
        f5 += sK * (chi * (E + (ss - un) * (r * ss + p / (sK - un))) - E);
    }
    const float uf = ss > 0.0f ? ufL : (ss < 0.0f ? ufR : 0.5f * (ufL + ufR));
    F[0] = f0;
    F[1] = f1;
    F[2] = fn;
    F[3] = f1t;
    F[4] = f2t;
    F[5] = f5;
    F[6] = (left ? wl[6] : wr[6]) * uf;
    F[7] = uf;
}

// Packed single-precision arithmetic on two independent values at once
// (sm_100 family: one instruction issues both lanes).  Subtraction is a
// multiply-add with -1, which is exact in its product.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }

// WENO5 states of a run of R faces (the arithmetic of run_states_fp32's
// scalar loop) for two variables at once: lane x from Pa, lane y from Pb.
template <int R>
__device__ __forceinline__ void weno5_run2(const float* __restrict__ Pa, const float* __restrict__ Pb,
                                           const int (&idx)[R + 5], float eps4s, float2 (&wl)[R],
                                           float2 (&wr)[R]) {
    const float2 eps4 = f2(eps4s), k = f2(13.0f / 3.0f);
    float2 p[R + 5];
#pragma unroll
    for (int i = 0; i < R + 5; ++i) p[i] = make_float2(Pa[idx[i]], Pb[idx[i]]);
    float2 d[R + 4], D[R + 3], sv[R + 3];
#pragma unroll
    for (int i = 0; i < R + 4; ++i) d[i] = sub2(p[i + 1], p[i]);
#pragma unroll
    for (int i = 0; i < R + 3; ++i) {
        D[i] = sub2(d[i + 1], d[i]);
        sv[i] = fma2(mul2(k, D[i]), D[i], eps4);
    }
#pragma unroll
    for (int j = 2; j <= R + 2; ++j) {   // cell idx[j]
        const float2 tl = fma2(f2(2.0f), d[j - 1], D[j - 2]);
        const float2 tm = add2(d[j - 1], d[j]);
        const float2 th = fma2(f2(-2.0f), d[j], D[j]);
        float2 El = fma2(tl, tl, sv[j - 2]), Em = fma2(tm, tm, sv[j - 1]), Eh = fma2(th, th, sv[j]);
        El = mul2(El, El);
        Em = mul2(Em, Em);
        Eh = mul2(Eh, Eh);
        const float2 X = mul2(Em, Eh), Y6 = mul2(f2(6.0f), mul2(El, Eh)), Z = mul2(El, Em);
        if (j <= R + 1) {   // left state of face j - 2 of the run
            const float2 hd = mul2(f2(0.5f), d[j]);
            const float2 a2 = mul2(f2(3.0f), Z);
            const float2 q0 = fma2(D[j - 2], f2(1.0f / 3.0f), mul2(f2(0.5f), d[j - 1]));
            const float2 q1 = fma2(D[j - 1], f2(-1.0f / 6.0f), hd);
            const float2 q2 = fma2(D[j], f2(-1.0f / 6.0f), hd);
            const float2 num = fma2(X, q0, fma2(Y6, q1, mul2(a2, q2)));
            wl[j - 2] = fma2(num, rcp2(add2(add2(X, Y6), a2)), p[j]);
        }
        if (j >= 3) {       // right state of face j - 3 of the run
            const float2 hd = mul2(f2(0.5f), d[j - 1]);
            const float2 a2 = mul2(f2(3.0f), X);
            const float2 q0 = fma2(D[j], f2(1.0f / 3.0f), mul2(f2(-0.5f), d[j]));
            const float2 q1 = fma2(D[j - 1], f2(-1.0f / 6.0f), mul2(f2(-1.0f), hd));
            const float2 q2 = fma2(D[j - 2], f2(-1.0f / 6.0f), mul2(f2(-1.0f), hd));
            const float2 num = fma2(Z, q0, fma2(Y6, q1, mul2(a2, q2)));
            wr[j - 3] = fma2(num, rcp2(add2(add2(Z, Y6), a2)), p[j]);
        }
    }
}

// One face in single precision: stencil of six staged cells (staged indices
// i6); vo[v] is the staged offset of face-frame variable v (slot 2 the normal
// velocity, 3 and 4 the tangential ones), so the states are reconstructed
// directly in the face frame.  Returns F in the face frame (see hllc_frame).
template <int ORD>
__device__ __forceinline__ void face_fp32(const Eos<float>& e, const float* __restrict__ sW, const int* i6,
                                          const int (&vo)[7], float* F) {
    float wl[7], wr[7];
#pragma unroll
    for (int v = 0; v < 7; ++v) {
        const float* P = sW + vo[v];
        if constexpr (ORD == 3) {
            wl[v] = weno3(P[i6[1]], P[i6[2]], P[i6[3]], e.eps);
            wr[v] = weno3(P[i6[4]], P[i6[3]], P[i6[2]], e.eps);
        } else {
            weno5_pair(P[i6[0]], P[i6[1]], P[i6[2]], P[i6[3]], P[i6[4]], P[i6[5]], 4.0f * e.eps, wl[v], wr[v]);
        }
    }
    float GL, PiL, GR, PiR;
    if (!admissible_f(e, wl, GL, PiL)) {
#pragma unroll
        for (int v = 0; v < 7; ++v) wl[v] = sW[vo[v] + i6[2]];
        closure(e, wl[6], GL, PiL);
    }
    if (!admissible_f(e, wr, GR, PiR)) {
#pragma unroll
        for (int v = 0; v < 7; ++v) wr[v] = sW[vo[v] + i6[3]];
        closure(e, wr[6], GR, PiR);
    }
    hllc_frame(wl, wr, GL, PiL, GR, PiR, F);
}

// Single precision: the WENO5 states of R consecutive faces of one line.
// idx[i] (i = 0..R+4) is the staged index of the line's cell j - 3 + i,
// where face j (between cells j - 1 and j) is the run's first face.  Each
// variable's R + 5 staged values are loaded once, and each of the cells
// j - 1 .. j + R - 1 forms its three smoothness indicators once for the left
// state of the face to its right and the right state of the face to its left
// (the operations of weno5_pair, in its order).  vo as in face_fp32: the
// states come out in the face frame.
template <int R>
__device__ __forceinline__ void run_states_fp32(const Eos<float>& e, const float* __restrict__ sW,
                                                const int (&idx)[R + 5], const int (&vo)[7], float (&wl)[R][7],
                                                float (&wr)[R][7]) {
    const float eps4 = 4.0f * e.eps;
    // the face-frame velocities (2, 3) and (4, 5) in packed pairs (packing the
    // partial densities (0, 1) as well needs more registers than the three
    // resident blocks per SM leave, and the spills cost more than it saves)
    constexpr int V0 = 2;
#pragma unroll
    for (int v = V0; v < 6; v += 2) {
        float2 l2[R], r2[R];
        weno5_run2<R>(sW + vo[v], sW + vo[v + 1], idx, eps4, l2, r2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            wl[r][v] = l2[r].x;
            wl[r][v + 1] = l2[r].y;
            wr[r][v] = r2[r].x;
            wr[r][v + 1] = r2[r].y;
        }
    }
    // alpha2 (variable 6) and the partial densities one at a time
#pragma unroll
    for (int si = 0; si < 1 + V0; ++si) {
        const int v = si == 0 ? 6 : si - 1;
        const float k = 13.0f / 3.0f;
        const float* P = sW + vo[v];
        float p[R + 5];
#pragma unroll
        for (int i = 0; i < R + 5; ++i) p[i] = P[idx[i]];
        float d[R + 4], D[R + 3], sv[R + 3];
#pragma unroll
        for (int i = 0; i < R + 4; ++i) d[i] = p[i + 1] - p[i];
#pragma unroll
        for (int i = 0; i < R + 3; ++i) {
            D[i] = d[i + 1] - d[i];
            sv[i] = fmaf(k * D[i], D[i], eps4);
        }
#pragma unroll
        for (int j = 2; j <= R + 2; ++j) {   // cell idx[j]
            const float tl = fmaf(2.0f, d[j - 1], D[j - 2]);
            const float tm = d[j - 1] + d[j];
            const float th = fmaf(-2.0f, d[j], D[j]);
            float El = fmaf(tl, tl, sv[j - 2]), Em = fmaf(tm, tm, sv[j - 1]), Eh = fmaf(th, th, sv[j]);
            El *= El;
            Em *= Em;
            Eh *= Eh;
            const float X = Em * Eh, Y6 = 6.0f * (El * Eh), Z = El * Em;
            if (j <= R + 1) {   // left state of face j - 2 of the run
                const float hd = 0.5f * d[j];
                const float a2 = 3.0f * Z;
                const float q0 = fmaf(D[j - 2], 1.0f / 3.0f, 0.5f * d[j - 1]);
                const float q1 = fmaf(D[j - 1], -1.0f / 6.0f, hd);
                const float q2 = fmaf(D[j], -1.0f / 6.0f, hd);
                wl[j - 2][v] = p[j] + fmaf(X, q0, fmaf(Y6, q1, a2 * q2)) / (X + Y6 + a2);
            }
            if (j >= 3) {       // right state of face j - 3 of the run
                const float hd = 0.5f * d[j - 1];
                const float a2 = 3.0f * X;
                const float q0 = fmaf(D[j], 1.0f / 3.0f, -0.5f * d[j]);
                const float q1 = fmaf(D[j - 1], -1.0f / 6.0f, -hd);
                const float q2 = fmaf(D[j - 2], -1.0f / 6.0f, -hd);
                wr[j - 3][v] = p[j] + fmaf(Z, q0, fmaf(Y6, q1, a2 * q2)) / (Z + Y6 + a2);
            }
        }
    }
}

// Fluxes of face r of a run from its states (positivity fallback to the cell
// values, then HLLC): F in the face frame (see hllc_frame).
template <int R>
__device__ __forceinline__ void run_flux_fp32(const Eos<float>& e, const float* __restrict__ sW,
                                              const int (&idx)[R + 5], const int (&vo)[7], int r, float (&wl)[7],
                                              float (&wr)[7], float (&F)[8]) {
    float GL, PiL, GR, PiR;
    if (!admissible_f(e, wl, GL, PiL)) {
#pragma unroll
        for (int v = 0; v < 7; ++v) wl[v] = sW[vo[v] + idx[r + 2]];
        closure(e, wl[6], GL, PiL);
    }
    if (!admissible_f(e, wr, GR, PiR)) {
#pragma unroll
        for (int v = 0; v < 7; ++v) wr[v] = sW[vo[v] + idx[r + 3]];
        closure(e, wr[6], GR, PiR);
    }
    hllc_frame(wl, wr, GL, PiL, GR, PiR, F);
}

// One face in double precision, in the FP64 reference's operation order.
template <int DIR, int ORD>
__device__ __forceinline__ void face_fp64(const Eos<double>& e, const double* __restrict__ sW, const int* i6,
                                          double* F) {
    double wl[7], wr[7];
#pragma unroll
    for (int v = 0; v < 7; ++v) {
        const double* P = sW + v * NCROSS;
        const double m1 = P[i6[1]], c0 = P[i6[2]], p1 = P[i6[3]], p2 = P[i6[4]];
        if constexpr (ORD == 3) {
            wl[v] = weno3(m1, c0, p1, e.eps);
            wr[v] = weno3(p2, p1, c0, e.eps);
        } else {
            const double m2 = P[i6[0]], p3 = P[i6[5]];
            wl[v] = weno5(m2, m1, c0, p1, p2, e.eps);
            wr[v] = weno5(p3, p2, p1, c0, m1, e.eps);
        }
    }
    if (!admissible(e, wl)) {
#pragma unroll
        for (int v = 0; v < 7; ++v) wl[v] = sW[v * NCROSS + i6[2]];
    }
    if (!admissible(e, wr)) {
#pragma unroll
        for (int v = 0; v < 7; ++v) wr[v] = sW[v * NCROSS + i6[3]];
    }
    hllc<double, DIR>(e, wl, wr, F);
}

// Asynchronous global -> shared copies (cp.async) of one element, and an L2
// prefetch of a contiguous global range (bulk, no registers or shared memory).
template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// 16 bytes, both addresses 16-byte aligned, cached in L2 only.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void prefetch_l2(const void* gmem, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

// Tensor-memory-accelerator copies (cp.async.bulk.tensor) completing on a
// shared-memory mbarrier, and the barrier operations they need.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous proxy
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of bar: false if it did not complete
// within about a second of the global timer (each try_wait may itself
// suspend the thread for a while; the iteration cap is a second bound).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Per-tile context of one RK stage.  parity 0: read Q_a, write Q_b; 1: the reverse.
template <typename T>
struct TileCtx {
    BlockWork<T> bw;
    const T* Qin;
    T* Qout;
    T* dQ;
};

template <typename T>
__device__ __forceinline__ void tile_ctx(const Params<T>& P, long long b, int parity, TileCtx<T>& c) {
    decode_block(P, b, c.bw);
    const GroupDev& G = *c.bw.G;
    const size_t n3 = (size_t)G.N * G.N * G.N;
    const size_t soff = (size_t)c.bw.s_local * 7 * n3;
    c.Qin = (const T*)(parity ? G.QB : G.QA) + soff;
    c.Qout = (T*)(parity ? G.QA : G.QB) + soff;
    c.dQ = (T*)G.dQ + soff;
}

// Asynchronous copies of a tile's raw Q (tile and halo) into sBuf, all in
// flight at once, in segments of four cells of one row: 16-byte copies (two
// in double precision) wherever the four cells lie in the domain, else one
// copy per halo cell through the boundary map (x halos of tiles on the
// domain's x faces; rows of y and z halos are mapped as a whole).
constexpr int NSEG_INT = TS * TS * 4;                 // full-width rows: 4 segments each
constexpr int NSEG = NSEG_INT + 4 * HALO * TS * 2;     // + y and z halo rows: 2 each (448)

// L2 prefetch of the tile's own dQ rows (stages that read dQ).
template <typename T>
__device__ __forceinline__ void tile_prefetch_dq(const TileCtx<T>& c) {
    const BlockWork<T>& bw = c.bw;
    const int N = bw.G->N;
    const size_t n3 = (size_t)N * N * N;
    for (int r = threadIdx.x; r < 7 * TS * TS; r += NT) {
        const int v = r / (TS * TS), yz = r % (TS * TS);
        const size_t gi = ((size_t)(bw.z0 + yz / TS) * N + (bw.y0 + yz % TS)) * N + bw.x0;
        prefetch_l2(c.dQ + v * n3 + gi, TS * sizeof(T));
    }
}

template <typename T, int STAGE, int LAYOUT>
__device__ __forceinline__ void tile_issue(const Params<T>& P, const TileCtx<T>& c, T* sBuf) {
    const BlockWork<T>& bw = c.bw;
    const int N = bw.G->N;
    const size_t n3 = (size_t)N * N * N;
    const int bc = P.bc;
    for (int u = threadIdx.x; u < NSEG; u += NT) {
        int by, bz, bx0;   // tile-relative row and first x of the segment
        if (u < NSEG_INT) {
            const int row = u >> 2, seg = u & 3;
            by = row & 7;
            bz = row >> 3;
            bx0 = 4 * seg - 4;
        } else {
            constexpr int NSEG_SLAB = 2 * HALO * TS * 2;        // units of the y (then z) halo rows
            const int v = u - NSEG_INT, zs = v >= NSEG_SLAB;
            const int row = (v - zs * NSEG_SLAB) >> 1, h = row % (2 * HALO), r = row / (2 * HALO);
            const int off = h < HALO ? h - HALO : TS + h - HALO;   // -3..-1, 8..10
            bx0 = 4 * (v & 1);
            if (!zs) {
                by = off;
                bz = r;
            } else {
                by = r;
                bz = off;
            }
        }
        const int gy = bc_map(bw.y0 + by, N, bc);
        const int gz = bc_map(bw.z0 + bz, N, bc);
        const size_t grow = ((size_t)gz * N + gy) * N;
        const int si = stage_slot<LAYOUT>(bx0, by, bz);   // a 16-byte chunk: its 4 cells consecutive
        const int gx0 = bw.x0 + bx0;
        if (gx0 >= 0 && gx0 + 4 <= N) {
#pragma unroll
            for (int v = 0; v < 7; ++v)
#pragma unroll
                for (int h = 0; h < (int)sizeof(T) / 4; ++h)
                    cp_async16(sBuf + v * NCROSS + si + 2 * h, c.Qin + v * n3 + grow + gx0 + 2 * h);
        } else {
            // a 4-cell x-halo segment crossing the domain face: its 3 stencil cells
            const int k0 = bx0 < 0 ? 1 : 0, k1 = bx0 < 0 ? 4 : 3;
            for (int k = k0; k < k1; ++k) {
                const int gx = bc_map(gx0 + k, N, bc);
#pragma unroll
                for (int v = 0; v < 7; ++v) cp_async(sBuf + v * NCROSS + si + k, c.Qin + v * n3 + grow + gx);
            }
        }
    }
}

// The tile's halo'd box by tensor copies: per variable the tile's rows with
// their x halos (x0 - 4 .. x0 + 11), the two y slabs and the two z slabs,
// all completing on bar (7 NCROSS elements).  Issued by the lanes 0..6 of
// one warp, lane v for variable v (lane 0 also posts the expected bytes;
// the barrier's phase cannot complete before that arrival).  Boxes that
// reach outside the domain are zero-filled there; the ghost cells are then
// set by tile_clamp_ghosts.  (x0 - 4 and x0 are multiples of four elements,
// so every box starts on a 16-byte boundary.)
template <typename T>
__device__ __forceinline__ void tile_issue_tma(const TileCtx<T>& c, int parity, T* sW, unsigned long long* bar,
                                               int v) {
    const BlockWork<T>& bw = c.bw;
    const CUtensorMap* m = bw.G->tm[parity];
    const int x0 = bw.x0, y0 = bw.y0, z0 = bw.z0, w = 7 * bw.s_local + v;
    if (v == 0) mbar_expect_tx(bar, (unsigned)(7 * NCROSS * sizeof(T)));
    T* d = sW + v * NCROSS;
    tma_load_4d(d, &m[TMA_BOX_INT], x0 - XOFF, y0, z0, w, bar);
    tma_load_4d(d + ROWS_INT, &m[TMA_BOX_YHALO], x0, y0 - HALO, z0, w, bar);
    tma_load_4d(d + ROWS_INT + NSLAB, &m[TMA_BOX_YHALO], x0, y0 + TS, z0, w, bar);
    tma_load_4d(d + ROWS_Y, &m[TMA_BOX_ZHALO], x0, y0, z0 - HALO, w, bar);
    tma_load_4d(d + ROWS_Y + NSLAB, &m[TMA_BOX_ZHALO], x0, y0, z0 + TS, w, bar);
}

// Faces of the tile on the domain boundary (bit 2 axis + side).
template <typename T>
__device__ __forceinline__ unsigned boundary_faces(const BlockWork<T>& bw) {
    const int N = bw.G->N;
    return (bw.x0 == 0 ? 1u : 0u) | (bw.x0 + TS == N ? 2u : 0u) | (bw.y0 == 0 ? 4u : 0u) |
           (bw.y0 + TS == N ? 8u : 0u) | (bw.z0 == 0 ? 16u : 0u) | (bw.z0 + TS == N ? 32u : 0u);
}

// Ghost cells of a tile on the domain boundary after tensor staging (the
// transmissive map: every ghost takes the value of the boundary cell on its
// line), copied from the staged boundary cells; `on` from boundary_faces.
// (Tensor staging lands the dense layout.)
template <typename T>
__device__ __forceinline__ void tile_clamp_ghosts(unsigned on, T* sW) {
    constexpr int PER = HALO * TS * TS;
    const int n_on = __popc(on);
    for (int u = threadIdx.x; u < n_on * PER; u += NT) {
        const int q = u / PER, r = u - q * PER;
        unsigned rest = on;   // face = the q-th set bit of on
        for (int i = 0; i < q; ++i) rest &= rest - 1;
        const int face = __ffs(rest) - 1;
        const int axis = face >> 1, hi = face & 1;
        const int layer = r / (TS * TS), a = (r / TS) % TS, b = r % TS;
        const int off = hi ? TS + layer : -1 - layer, edge = hi ? TS - 1 : 0;
        const int x = axis == 0 ? off : b;
        const int y = axis == 1 ? off : (axis == 0 ? b : a);
        const int z = axis == 2 ? off : a;
        const int dst = stage_slot<LAYOUT_DENSE>(x, y, z);
        const int src = stage_slot<LAYOUT_DENSE>(axis == 0 ? edge : x, axis == 1 ? edge : y, axis == 2 ? edge : z);
#pragma unroll
        for (int v = 0; v < 7; ++v) sW[v * NCROSS + dst] = sW[v * NCROSS + src];
    }
}

template <int LAYOUT>
__device__ __forceinline__ void fill_rows(int2* sRows) {
    for (int i = threadIdx.x; i < BX * BX; i += NT) {
        const int y = i % BX - HALO, z = i / BX - HALO;
        const bool yi = (unsigned)y < (unsigned)TS, zi = (unsigned)z < (unsigned)TS;
        sRows[i] = (yi || zi) ? make_int2(stage_slot<LAYOUT>(0, y, z), stage_slot<LAYOUT>(4, y, z)) : make_int2(-1, -1);
    }
}

// Characteristic far-field ghost (Sec. 3.1, after Poinsot and Lele): the
// slot holds the primitives of the interior cell next to the face (staged
// through the transmissive map); along the outward normal (side s) with
// Z = rho c of that cell, the outgoing characteristic p + Z u_n stays that
// cell's and the incoming p - Z u_n becomes (1 - kappa) of that cell's plus
// kappa of the far field at rest at p_inf.  Rewrites p and the normal
// velocity in place; same operation order as the oracle.
template <typename T>
__device__ __forceinline__ void char_ghost(const Eos<T>& e, T pinf, T kappa, T* sW, int si, int axis, T s) {
    const T rho = sW[si] + sW[NCROSS + si];
    const T p = sW[5 * NCROSS + si];
    T G, Pi;
    closure(e, sW[6 * NCROSS + si], G, Pi);
    const T Z = rho * sqrt(((G + T(1)) * p + Pi) / (G * rho));
    const T un = s * sW[(2 + axis) * NCROSS + si];
    sW[5 * NCROSS + si] = p + T(0.5) * kappa * (pinf - p + Z * un);
    sW[(2 + axis) * NCROSS + si] = s * (un + T(0.5) * kappa * (p - pinf - Z * un) / Z);
}

// The characteristic ghosts of a tile: the three halo layers behind each
// tile face that lies on a domain face (ghosts outside along one axis only,
// the only ones a stencil reads; every layer takes the same state).
template <typename T, int LAYOUT>
__device__ __forceinline__ void tile_char_bc(const Params<T>& P, const BlockWork<T>& bw, T* sW) {
    const int N = bw.G->N;
    const T pinf = (T)P.p_liq, kappa = (T)P.bc_penalty;
    constexpr int PER = HALO * TS * TS;
    for (int u = threadIdx.x; u < 6 * PER; u += NT) {
        const int face = u / PER, r = u - face * PER;
        const int axis = face >> 1, hi = face & 1;
        const int o = axis == 0 ? bw.x0 : (axis == 1 ? bw.y0 : bw.z0);
        if (hi ? (o + TS < N) : (o > 0)) continue;   // an interior tile face
        const int layer = r / (TS * TS), a = (r / TS) % TS, b = r % TS;
        const int off = hi ? TS + layer : -1 - layer;
        const int x = axis == 0 ? off : b;
        const int y = axis == 1 ? off : (axis == 0 ? b : a);
        const int z = axis == 2 ? off : a;
        char_ghost(P.eos, pinf, kappa, sW, stage_slot<LAYOUT>(x, y, z), axis, hi ? T(1) : T(-1));
    }
}

// cons2prim of two cells at once in packed single precision.
__device__ __forceinline__ void cons2prim2(const Eos<float>& e, const float2 (&q)[7], float2 (&w)[7]) {
    const float2 rho = add2(q[0], q[1]);
    const float2 ir = rcp2(rho);
    const float2 u = mul2(q[2], ir), v = mul2(q[3], ir), ww = mul2(q[4], ir);
    const float2 a = make_float2(clamp01(q[6].x), clamp01(q[6].y));
    const float2 a1 = sub2(f2(1.0f), a);
    const float2 G = fma2(a, f2(e.gi2), mul2(a1, f2(e.gi1)));
    const float2 Pi = fma2(a, f2(e.pi2), mul2(a1, f2(e.pi1)));
    const float2 ke = mul2(mul2(f2(0.5f), rho), fma2(u, u, fma2(v, v, mul2(ww, ww))));
    w[0] = q[0];
    w[1] = q[1];
    w[2] = u;
    w[3] = v;
    w[4] = ww;
    w[5] = mul2(sub2(sub2(q[5], ke), Pi), rcp2(G));
    w[6] = q[6];
}

// Raw Q of every staged cell -> primitives, in place.  Single precision: four
// consecutive slots of a row per thread with 16-byte shared-memory accesses,
// as two packed pairs (row padding slots are converted too and never read).
template <typename T, int LAYOUT>
__device__ __forceinline__ void tile_convert(const Eos<T>& e, T* sW) {
    if constexpr (std::is_same<T, float>::value) {
        for (int i4 = threadIdx.x; i4 < NCROSS / 4; i4 += NT) {
            float4 q4[7];
#pragma unroll
            for (int v = 0; v < 7; ++v) q4[v] = *reinterpret_cast<const float4*>(sW + v * NCROSS + 4 * i4);
            float2 q[7], wa[7], wb[7];
#pragma unroll
            for (int v = 0; v < 7; ++v) q[v] = make_float2(q4[v].x, q4[v].y);
            cons2prim2(e, q, wa);
#pragma unroll
            for (int v = 0; v < 7; ++v) q[v] = make_float2(q4[v].z, q4[v].w);
            cons2prim2(e, q, wb);
#pragma unroll
            for (int v = 0; v < 7; ++v)
                *reinterpret_cast<float4*>(sW + v * NCROSS + 4 * i4) = make_float4(wa[v].x, wa[v].y, wb[v].x, wb[v].y);
        }
    } else {
        for (int i = threadIdx.x; i < NCROSS; i += NT) {
            if (pad_slot<LAYOUT>(i)) continue;
            T q[7], w[7];
#pragma unroll
            for (int v = 0; v < 7; ++v) q[v] = sW[v * NCROSS + i];
            cons2prim(e, q, w);
#pragma unroll
            for (int v = 0; v < 7; ++v) sW[v * NCROSS + i] = w[v];
        }
    }
}

// One face of direction dir from the stencil i6, its 8 values (7 fluxes
// and the face velocity) written to dst[v * stride] in the staged variable
// order; ORD = 5 (WENO5) or 3 (WENO3) reconstruction.
template <typename T, int ORD>
__device__ __forceinline__ void face_store(const Eos<T>& e, const T* __restrict__ sW, const int* i6, int dir,
                                           T* __restrict__ dst, int stride) {
    T F[8];
    if constexpr (std::is_same<T, double>::value) {
        if (dir == 0)
            face_fp64<0, ORD>(e, sW, i6, F);
        else if (dir == 1)
            face_fp64<1, ORD>(e, sW, i6, F);
        else
            face_fp64<2, ORD>(e, sW, i6, F);
#pragma unroll
        for (int v = 0; v < 8; ++v) dst[v * stride] = F[v];
    } else {
        const int r1 = dir == 0 ? 3 : (dir == 1 ? 4 : 2);   // staged row of the first tangential velocity
        const int r2 = dir == 0 ? 4 : (dir == 1 ? 2 : 3);   // and of the second
        const int vo[7] = {0, NCROSS, (2 + dir) * NCROSS, r1 * NCROSS, r2 * NCROSS, 5 * NCROSS, 6 * NCROSS};
        face_fp32<ORD>(e, sW, i6, vo, F);
        dst[0] = F[0];
        dst[stride] = F[1];
        dst[(2 + dir) * stride] = F[2];
        dst[r1 * stride] = F[3];
        dst[r2 * stride] = F[4];
        dst[5 * stride] = F[5];
        dst[6 * stride] = F[6];
        dst[7 * stride] = F[7];
    }
}

// The tile cells a thread owns for the accumulation and the update: in
// single precision two x-neighbours (2t, 2t+1), so the update moves 8 bytes
// per global access; in double precision t and t + NT.
template <typename T>
constexpr bool kPairCells = std::is_same<T, float>::value;
template <typename T>
__device__ __forceinline__ int own_cell(int k) {
    if constexpr (kPairCells<T>) return 2 * (int)threadIdx.x + k;
    return (int)threadIdx.x + k * NT;
}

// Right-hand sides of one tile's cells (faces direction by direction,
// per-cell flux differences and the face-velocity divergence), from the
// primitives staged in sW.  Cell k of this thread is own_cell<T>(k).
template <typename T>
struct TileRhs {
    T rhs[CELLS_PER_THREAD][7];
    T divu[CELLS_PER_THREAD];
};

// The far face of every line of the tile (x = 8, y = 8 or z = 8; 64 per
// direction, all three directions), its 8 values (staged variable order) to
// sFb[dir][v][line].
template <typename T, int ORD>
__device__ __forceinline__ void far_faces(const Eos<T>& e, const T* __restrict__ sW, const int2* __restrict__ sRows,
                                          T* __restrict__ sFb) {
    for (int f = threadIdx.x; f < 3 * TS * TS; f += NT) {
        const int dir = f >> 6, line = f & 63, a = line & 7, b = line >> 3;
        int i6[6];
        if (dir == 0) {
            int base;
            const int m = row_xmask(sRows, a, b, base);
#pragma unroll
            for (int k = 0; k < 6; ++k) i6[k] = (base + TS - 3 + k) ^ m;
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k)
                i6[k] = dir == 1 ? slot_lo(sRows, TS - 3 + k, b, a) : slot_lo(sRows, b, TS - 3 + k, a);
        }
        face_store<T, ORD>(e, sW, i6, dir, sFb + dir * 8 * TS * TS + line, TS * TS);
    }
}

// Slot of tile cell c = x + 8 y + 64 z in the accumulation array: bits 3-4
// (the low bits of y) are XORed with (z >> 1) ^ (y >> 2), a permutation
// within each group of 32 cells, so that the y-run stores (lanes x, runs
// y = 0, 2, 4, 6), the z-run updates (lanes x, runs z = 0, 2, 4, 6) and the
// owners' paired reads (x pairs, rows y) each touch 32 distinct banks.
__device__ __forceinline__ int rslot(int c) { return c ^ ((((c >> 7) & 3) ^ ((c >> 5) & 1)) << 3); }

// Single-precision WENO5 faces and right-hand sides of one tile, with no
// staging of near-face fluxes: every thread takes one run of two consecutive
// near faces j, j + 1 of one line per direction, so it holds both faces of
// cell j; the run's neighbour along the line (the next thread in x, eight
// threads on in y and z, so always in the same warp) hands over its first face
// by a warp shuffle, the line's last run takes the far face computed up front.
// Directions y and z add their flux differences to a shared per-cell array
// (y stores, z accumulates, a barrier between them); direction x comes last,
// where a thread's run is its own cell pair (2t, 2t + 1), so it adds its
// differences in registers to the array's y + z sum.  Three barriers per tile
// instead of seven.
__device__ __forceinline__ void tile_faces_direct(const Eos<float>& e, float invh, const float* __restrict__ sW,
                                                  float* __restrict__ sF, const int2* __restrict__ sRows,
                                                  TileRhs<float>& R) {
    float* __restrict__ sR = sF;                   // [8][RSTRIDE]: y + z contributions per cell
    float* __restrict__ sFb = sF + 8 * RSTRIDE;    // [3][8][64]: far faces
    far_faces<float, 5>(e, sW, sRows, sFb);
    __syncthreads();
    const int t = threadIdx.x;
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        const int dir = k == 2 ? 0 : k + 1;   // y, z, then x
        int a, b, j;   // the line's two other coordinates and the run's first face
        if (dir == 0) {
            j = 2 * (t & 3);
            a = (t >> 2) & 7;
            b = t >> 5;
        } else {
            a = t & 7;
            j = 2 * ((t >> 3) & 3);
            b = t >> 5;
        }
        int idx[7];
        if (dir == 0) {
            int base;
            const int m = row_xmask(sRows, a, b, base);
#pragma unroll
            for (int i = 0; i < 7; ++i) idx[i] = (base + j - 3 + i) ^ m;
        } else {
#pragma unroll
            for (int i = 0; i < 7; ++i)
                idx[i] = dir == 1 ? slot_lo(sRows, j - 3 + i, b, a) : slot_lo(sRows, b, j - 3 + i, a);
        }
        const int r1 = dir == 0 ? 3 : (dir == 1 ? 4 : 2);   // staged variable of the first tangential velocity
        const int r2 = dir == 0 ? 4 : (dir == 1 ? 2 : 3);   // and of the second
        const int vo[7] = {0, NCROSS, (2 + dir) * NCROSS, r1 * NCROSS, r2 * NCROSS, 5 * NCROSS, 6 * NCROSS};
        float F0[8], F1[8];
        {
            float wl[2][7], wr[2][7];
            run_states_fp32<2>(e, sW, idx, vo, wl, wr);
            run_flux_fp32<2>(e, sW, idx, vo, 0, wl[0], wr[0], F0);
            run_flux_fp32<2>(e, sW, idx, vo, 1, wl[1], wr[1], F1);
        }
        // face j + 2: the next run's first face, or the line's far face
        const int line = a + 8 * b;
        const bool last = j == TS - 2;
        const int so[8] = {0, 1, 2 + dir, r1, r2, 5, 6, 7};   // staged variable of face-frame value v
        float dA[8], dB[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            float fn = __shfl_down_sync(0xffffffffu, F0[v], dir == 0 ? 1 : 8);
            if (last) fn = sFb[(dir * 8 + so[v]) * (TS * TS) + line];
            dA[v] = F1[v] - F0[v];
            dB[v] = fn - F1[v];
        }
        if (dir == 0) {
            // cells 2t, 2t + 1 (j + 8a + 64b): the thread's own pair, face frame = staged order
            const int cA = rslot(2 * t);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const float2 acc = *reinterpret_cast<const float2*>(sR + v * RSTRIDE + cA);
                const float2 r = fma2(make_float2(dA[v], dB[v]), f2(v < 7 ? -invh : invh), acc);
                if (v < 7) {
                    R.rhs[0][v] = r.x;
                    R.rhs[1][v] = r.y;
                } else {
                    R.divu[0] = r.x;
                    R.divu[1] = r.y;
                }
            }
        } else {
            const int cA = dir == 1 ? a + 8 * j + 64 * b : a + 8 * b + 64 * j;
            const int step = dir == 1 ? 8 : 64;
            const int sA = rslot(cA), sB = rslot(cA + step);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const float s = v < 7 ? -invh : invh;
                float* dst = sR + so[v] * RSTRIDE;
                if (dir == 1) {
                    dst[sA] = dA[v] * s;
                    dst[sB] = dB[v] * s;
                } else {
                    dst[sA] = fmaf(dA[v], s, dst[sA]);
                    dst[sB] = fmaf(dB[v], s, dst[sB]);
                }
            }
            __syncthreads();
        }
    }
}

// Faces staged per direction (double precision in the FP64 reference's
// accumulation order, and single-precision WENO3): the near faces of one
// direction into sF, a barrier, the per-cell differences, a barrier.
template <typename T, int ORD>
__device__ __forceinline__ void tile_faces_staged(const Eos<T>& e, T invh, const T* __restrict__ sW,
                                                  T* __restrict__ sF, const int2* __restrict__ sRows, TileRhs<T>& R) {
    T (&divu)[CELLS_PER_THREAD] = R.divu;
    T (&rhs)[CELLS_PER_THREAD][7] = R.rhs;
#pragma unroll
    for (int k = 0; k < CELLS_PER_THREAD; ++k) {
        divu[k] = T(0);
#pragma unroll
        for (int v = 0; v < 7; ++v) rhs[k][v] = T(0);
    }

    // The far face of every line (x = 8, y = 8 or z = 8; 64 per direction) for
    // all three directions first, into sFb, then per direction the near face
    // of every cell (512, two per thread) into sF, so that every barrier
    // interval holds the same number of faces per thread.
    T* __restrict__ sFb = sF + 8 * NCELL;   // [3][8][64]
    far_faces<T, ORD>(e, sW, sRows, sFb);
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
        for (int c = threadIdx.x; c < NCELL; c += NT) {
            const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
            int i6[6];
            if (dir == 0) {
                int base;
                const int m = row_xmask(sRows, y, z, base);
#pragma unroll
                for (int k = 0; k < 6; ++k) i6[k] = (base + x - 3 + k) ^ m;
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    i6[k] = dir == 1 ? slot_lo(sRows, y - 3 + k, z, x) : slot_lo(sRows, y, z - 3 + k, x);
            }
            face_store<T, ORD>(e, sW, i6, dir, sF + c, NCELL);
        }
        __syncthreads();
        if constexpr (kPairCells<T>) {
            // cells c, c + 1 (x-neighbours): both lanes of each difference at once
            const int c = own_cell<T>(0);
            const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
            const int cd = dir == 0 ? x : (dir == 1 ? y : z);
            const int step = dir == 0 ? 1 : (dir == 1 ? 8 : 64);
            const int line = dir == 0 ? c >> 3 : (dir == 1 ? x + 8 * z : c & 63);
            const float* __restrict__ Fb = sFb + dir * 8 * TS * TS;
            const float2 mih = f2(-(float)invh);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const float2 Fn = *reinterpret_cast<const float2*>(sF + v * NCELL + c);
                float2 Fr;
                if (dir == 0) {
                    Fr.x = sF[v * NCELL + c + 1];
                    Fr.y = x + 1 < TS - 1 ? sF[v * NCELL + c + 2] : Fb[v * TS * TS + line];
                } else {
                    Fr = cd < TS - 1 ? *reinterpret_cast<const float2*>(sF + v * NCELL + c + step)
                                     : *reinterpret_cast<const float2*>(Fb + v * TS * TS + line);
                }
                const float2 dF = sub2(Fr, Fn);
                if (v < 7) {
                    const float2 r = fma2(dF, mih, make_float2(rhs[0][v], rhs[1][v]));
                    rhs[0][v] = r.x;
                    rhs[1][v] = r.y;
                } else {
                    const float2 r = fma2(dF, f2((float)invh), make_float2(divu[0], divu[1]));
                    divu[0] = r.x;
                    divu[1] = r.y;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < CELLS_PER_THREAD; ++k) {
                const int c = own_cell<T>(k);
                if (c < NCELL) {
                    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
                    const int cd = dir == 0 ? x : (dir == 1 ? y : z);
                    const int step = dir == 0 ? 1 : (dir == 1 ? 8 : 64);
                    const int line = dir == 0 ? c >> 3 : (dir == 1 ? x + 8 * z : c & 63);
                    // flux at the cell's far face: the next cell's near face, or the line's far face
                    const T* __restrict__ Fr = cd < TS - 1 ? sF + c + step : sFb + dir * 8 * TS * TS + line;
                    const int sr = cd < TS - 1 ? NCELL : TS * TS;
#pragma unroll
                    for (int v = 0; v < 7; ++v)
                        rhs[k][v] -= (Fr[v * sr] - sF[v * NCELL + c]) * invh;
                    divu[k] += (Fr[7 * sr] - sF[7 * NCELL + c]) * invh;
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int ORD>
__device__ __forceinline__ void tile_faces(const Params<T>& P, const TileCtx<T>& c, const T* __restrict__ sW,
                                           T* __restrict__ sF, const int2* __restrict__ sRows, TileRhs<T>& R) {
    // 1/h, formed as the FP64 reference forms it (single precision: from the host's float h)
    const T invh = T(1) / (std::is_same<T, float>::value ? (T)c.bw.G->h32 : (T)c.bw.G->h);
    if constexpr (std::is_same<T, float>::value && ORD == 5)
        tile_faces_direct(P.eos, invh, sW, sF, sRows, R);
    else
        tile_faces_staged<T, ORD>(P.eos, invh, sW, sF, sRows, R);
}

// Pressure and raw alpha2 of this thread's cells (the alpha2 source term).
template <typename T>
__device__ __forceinline__ void tile_cell_pa(const T* __restrict__ sW, const int2* __restrict__ sRows,
                                             T (&pc)[CELLS_PER_THREAD], T (&ac)[CELLS_PER_THREAD]) {
#pragma unroll
    for (int k = 0; k < CELLS_PER_THREAD; ++k) {
        const int c = own_cell<T>(k);
        if (c < NCELL) {
            const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
            const int si = slot_lo(sRows, y, z, x);
            pc[k] = sW[5 * NCROSS + si];
            ac[k] = sW[6 * NCROSS + si];
        }
    }
}

// alpha2 source, 2N update and, in the last stage, the new state's per-tile
// reductions (reads Q and dQ from global memory; shared memory is not used
// except by the block reduction).
template <typename T, int STAGE>
__device__ __forceinline__ void tile_update(const Params<T>& P, const TileCtx<T>& c, long long tile_index,
                                            TileRhs<T>& R, const T (&pc)[CELLS_PER_THREAD],
                                            const T (&ac)[CELLS_PER_THREAD], T dt) {
    const BlockWork<T>& bw = c.bw;
    const GroupDev& G = *bw.G;
    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    const T* __restrict__ Qin = c.Qin;
    T* __restrict__ Qout = c.Qout;
    T* __restrict__ dQ = c.dQ;
    const Eos<T> e = P.eos;
    T (&rhs)[CELLS_PER_THREAD][7] = R.rhs;
    T (&divu)[CELLS_PER_THREAD] = R.divu;
    const T A = P.rkA_t[STAGE], B = P.rkB_t[STAGE];
    RedT<T> red;
    red_init(red);
    if constexpr (kPairCells<T>) {
        // cells c, c + 1: alpha2 source per cell, then 8-byte loads and stores
        const int c = own_cell<T>(0);
        const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const T p = pc[k];
            const T a2raw = ac[k];
            const T a2 = clamp01(a2raw);
            const T a1 = T(1) - a2;
            const T z1 = e.g1 * (p + e.pc1);  // rho_1 c_1^2
            const T z2 = e.g2 * (p + e.pc2);  // rho_2 c_2^2
            const T K = a1 * a2 * (z1 - z2) / (a1 * z2 + a2 * z1);
            rhs[k][6] += (a2raw + K) * divu[k];
        }
        const size_t gi = ((size_t)(bw.z0 + z) * N + (bw.y0 + y)) * N + (bw.x0 + x);
        float2 qn[7];
#pragma unroll
        for (int v = 0; v < 7; ++v) {
            const float2 q = *reinterpret_cast<const float2*>(Qin + v * n3 + gi);
            float2 d = mul2(f2(dt), make_float2(rhs[0][v], rhs[1][v]));
            if (STAGE > 0) d = fma2(f2(A), *reinterpret_cast<const float2*>(dQ + v * n3 + gi), d);
            if (STAGE < 2) *reinterpret_cast<float2*>(dQ + v * n3 + gi) = d;
            qn[v] = fma2(f2(B), d, q);
            *reinterpret_cast<float2*>(Qout + v * n3 + gi) = qn[v];
        }
        if (STAGE == 2) {
            T q0[7], q1[7];
#pragma unroll
            for (int v = 0; v < 7; ++v) {
                q0[v] = qn[v].x;
                q1[v] = qn[v].y;
            }
            red_cell(e, q0, (long long)gi, red);
            red_cell(e, q1, (long long)gi + 1, red);
            const long long tile = tile_index - G.block0 - (long long)bw.s_local * G.tps;
            block_reduce_write(red, G.part + (size_t)bw.s_local * G.tps + tile);
        }
    } else {
#pragma unroll
        for (int k = 0; k < CELLS_PER_THREAD; ++k) {
            const int c = own_cell<T>(k);
            if (c < NCELL) {
                const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
                const T p = pc[k];
                const T a2raw = ac[k];
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
                    // the last stage's register is dead: the next step's first stage (A = 0)
                    // overwrites it without reading it
                    if (STAGE < 2) dQ[v * n3 + gi] = d;
                    qn[v] = q + B * d;
                    Qout[v * n3 + gi] = qn[v];
                }
                if (STAGE == 2) red_cell(e, qn, (long long)gi, red);
            }
        }
        if (STAGE == 2) {
            const long long tile = tile_index - G.block0 - (long long)bw.s_local * G.tps;
            block_reduce_write(red, G.part + (size_t)bw.s_local * G.tps + tile);
        }
    }
}


// One tile: faces, source, update.
template <typename T, int STAGE, int ORD>
__device__ __forceinline__ void tile_body(const Params<T>& P, const TileCtx<T>& c, long long tile_index,
                                          const T* __restrict__ sW, T* __restrict__ sF,
                                          const int2* __restrict__ sRows, T dt) {
    TileRhs<T> R;
    tile_faces<T, ORD>(P, c, sW, sF, sRows, R);
    T pc[CELLS_PER_THREAD], ac[CELLS_PER_THREAD];
    tile_cell_pa(sW, sRows, pc, ac);
    tile_update<T, STAGE>(P, c, tile_index, R, pc, ac, dt);
}

// One RK stage, one block per tile (ORD: WENO order, 5 or 3).
template <typename T, int STAGE, int ORD>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? BLOCKS_FP32 : 1)
    stage_kernel(const __grid_constant__ Params<T> P, int parity) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // [7][NCROSS] primitives (staged as raw Q)
    T* sW = reinterpret_cast<T*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    T* sF = sW + 7 * NCROSS;                 // face fluxes + face velocities (NFLUX)
    int2* sRows = reinterpret_cast<int2*>(sF + NFLUX);  // [BX][BX] per-row slot table
    TileCtx<T> c;
    tile_ctx(P, blockIdx.x, parity, c);
    // the finished-sample flag is read while the copies are issued (they only
    // read the sample's own state); a finished tile returns once none is left
    // in flight.  (Staging by tensor copies measured 0.6-1 % slower here: one
    // launch keeps three tiles per SM in flight either way, and the per-row
    // copies need no barrier set-up; the persistent variant uses them.)
    // The update reads dQ straight from global memory: an L2 prefetch of the
    // tile's dQ rows issued with the copies made the single-precision kernel
    // 4 % slower (12.60 against 12.11 ms per launch on 512 x 64^3, same bits);
    // the double-precision kernel, bound by its FP64 pipe, keeps it.
    const int done = P.s.done[c.bw.slot];
    __shared__ T s_dt;   // the sample's time step, converted once per block
    if (threadIdx.x == 0) s_dt = (T)P.s.dt[c.bw.slot];
    tile_issue<T, STAGE, LAYOUT_SWZ>(P, c, sW);
    if (sizeof(T) == 8 && STAGE > 0) tile_prefetch_dq(c);
    fill_rows<LAYOUT_SWZ>(sRows);
    cp_async_wait_all();
    if (done) return;
    __syncthreads();
    tile_convert<T, LAYOUT_SWZ>(P.eos, sW);
    if (P.bc == OFM_BC_CHARACTERISTIC) {
        __syncthreads();
        tile_char_bc<T, LAYOUT_SWZ>(P, c.bw, sW);
    }
    __syncthreads();
    tile_body<T, STAGE, ORD>(P, c, (long long)blockIdx.x, sW, sF, sRows, s_dt);
}

// One RK stage, persistent blocks (three per SM in single precision, one
// staging buffer each): each block walks tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...  Once a tile's faces are done and its pressure and alpha2
// are in registers, one thread issues the next tile's tensor copies into the
// staging buffer and the block then performs the current tile's update, so
// the update's global loads and stores overlap the next tile's copies.
// Finished samples' tiles are staged but not computed.  Same arithmetic as
// stage_kernel.  (Periodic boundaries: per-row cp.async staging, the next
// tile's copies issued the same way.)
template <typename T, int STAGE, int ORD>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? BLOCKS_FP32 : 1)
    stage_kernel_persistent(const __grid_constant__ Params<T> P, int parity) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar;
    T* sW = reinterpret_cast<T*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    T* sF = sW + 7 * NCROSS;
    int2* sRows = reinterpret_cast<int2*>(sF + NFLUX);
    const bool tma = P.bc != OFM_BC_PERIODIC;
    fill_rows<LAYOUT_DENSE>(sRows);   // the layout the tensor copies land
    if (tma && threadIdx.x == 0) mbar_init(&s_bar, 1);
    __syncthreads();   // the barrier is initialised before any thread waits on it
    const long long stride = gridDim.x;
    long long t = blockIdx.x;
    int done = 1;
    if (t < P.total_blocks) {
        TileCtx<T> c;
        tile_ctx(P, t, parity, c);
        done = P.s.done[c.bw.slot];
        if (!tma) {
            tile_issue<T, STAGE, LAYOUT_DENSE>(P, c, sW);
            if (STAGE > 0) tile_prefetch_dq(c);
        } else if (threadIdx.x < 7)
            tile_issue_tma(c, parity, sW, &s_bar, (int)threadIdx.x);
    }
    unsigned phase = 0;
    while (t < P.total_blocks) {
        TileRhs<T> R;
        T pc[CELLS_PER_THREAD], ac[CELLS_PER_THREAD];
        {
            TileCtx<T> c;
            tile_ctx(P, t, parity, c);
            if (tma) {
                if (STAGE > 0 && !done) tile_prefetch_dq(c);
                const bool ok = mbar_wait_bounded(&s_bar, phase);
                if (__syncthreads_or(!ok)) {   // a wait ran out: abandon the sample, leave the device usable
                    if (threadIdx.x == 0) atomicOr(&P.s.qoi[c.bw.slot].status, OFM_ST_TIMEOUT);
                    return;
                }
                phase ^= 1u;
                if (!done) tile_clamp_ghosts(boundary_faces(c.bw), sW);
            } else {
                cp_async_wait_all();
            }
            if (!done) {
                __syncthreads();
                tile_convert<T, LAYOUT_DENSE>(P.eos, sW);
                if (P.bc == OFM_BC_CHARACTERISTIC) {
                    __syncthreads();
                    tile_char_bc<T, LAYOUT_DENSE>(P, c.bw, sW);
                }
                __syncthreads();
                tile_faces<T, ORD>(P, c, sW, sF, sRows, R);
                tile_cell_pa(sW, sRows, pc, ac);
            }
        }
        __syncthreads();   // every read of sW is done
        // the tile's context is formed again below rather than kept in registers through the faces
        asm volatile("" : "+l"(t));
        const long long tn = t + stride;
        int done_n = 1;
        if (tn < P.total_blocks) {
            TileCtx<T> cn;
            tile_ctx(P, tn, parity, cn);
            done_n = P.s.done[cn.bw.slot];
            if (!tma) {
                tile_issue<T, STAGE, LAYOUT_DENSE>(P, cn, sW);
                if (STAGE > 0) tile_prefetch_dq(cn);
            } else if (threadIdx.x < 7) {
                // the block's generic-proxy accesses of sW come before the copies' writes
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                tile_issue_tma(cn, parity, sW, &s_bar, (int)threadIdx.x);
            }
        }
        if (!done) {
            TileCtx<T> c;
            tile_ctx(P, t, parity, c);
            tile_update<T, STAGE>(P, c, t, R, pc, ac, (T)P.s.dt[c.bw.slot]);
        }
        t = tn;
        done = done_n;
    }
    if (!tma) cp_async_wait_all();
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
        red_merge(r, part[t].smax, part[t].cmax, part[t].pmax, part[t].idx, part[t].status);
    __shared__ Red sred[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double sm = __shfl_down_sync(0xffffffffu, r.smax, off);
        const double cm = __shfl_down_sync(0xffffffffu, r.cmax, off);
        const double pm = __shfl_down_sync(0xffffffffu, r.pmax, off);
        const long long ix = __shfl_down_sync(0xffffffffu, r.idx, off);
        const int st = __shfl_down_sync(0xffffffffu, r.status, off);
        red_merge(r, sm, cm, pm, ix, st);
    }
    if (lane == 0) sred[warp] = r;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x / 32); ++w)
        red_merge(r, sred[w].smax, sred[w].cmax, sred[w].pmax, sred[w].idx, sred[w].status);

    const int N = G.N;
    const size_t n3 = (size_t)N * N * N;
    const T* Q = (const T*)(parity ? G.QB : G.QA) + (size_t)s_local * 7 * n3;
    double sv[OFM_MAX_SENSORS], sa[OFM_MAX_SENSORS];
    for (int s = 0; s < P.n_sens; ++s) {
        double acc = 0.0, acca = 0.0;
        const int a0 = G.sens_off[s], a1 = G.sens_off[s + 1];
        for (int a = a0; a < a1; ++a) {
            acc += cell_pressure(P.eos, Q, n3, G.sens_cells[a]);
            acca += (double)Q[6 * n3 + G.sens_cells[a]];
        }
        sv[s] = a1 > a0 ? acc / (double)(a1 - a0) : NAN;
        sa[s] = a1 > a0 ? acca / (double)(a1 - a0) : NAN;
    }
    DevQoi& q = P.s.qoi[slot];
    double* old = P.s.sens_old + (size_t)slot * OFM_MAX_SENSORS;
    double* hist = P.s.hist + (size_t)slot * P.n_sens * P.n_out;
    double* aold = P.s.ahist ? P.s.alpha_old + (size_t)slot * OFM_MAX_SENSORS : nullptr;
    double* ahist = P.s.ahist ? P.s.ahist + (size_t)slot * P.n_sens * P.n_out : nullptr;
    double t;
    int nsteps;
    if (first) {
        q.status = r.status;
        q.p_peak = r.pmax;
        q.peak_index = r.idx;
        q.p_peak_t = 0.0;
        q.c_max = r.cmax;
        for (int s = 0; s < P.n_sens; ++s) {
            q.sensor_alpha0[s] = q.sensor_alpha_min[s] = sa[s];
            q.sensor_alpha_min_t[s] = 0.0;
            q.sensor_peak[s] = sv[s];
            old[s] = sv[s];
            if (P.n_out > 0) hist[s * P.n_out] = sv[s];
            if (ahist) {
                aold[s] = sa[s];
                if (P.n_out > 0) ahist[s * P.n_out] = sa[s];
            }
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
        if (r.cmax > q.c_max) q.c_max = r.cmax;
        for (int s = 0; s < P.n_sens; ++s) {
            if (sv[s] > q.sensor_peak[s]) q.sensor_peak[s] = sv[s];
            if (sa[s] < q.sensor_alpha_min[s]) {
                q.sensor_alpha_min[s] = sa[s];
                q.sensor_alpha_min_t[s] = t;
            }
        }
        if (P.n_out > 1) {
            int k = P.s.kout[slot];
            while (k < P.n_out) {
                const double tk = ((double)k * P.t_end) / (double)(P.n_out - 1);
                if (tk > t) break;
                const double wgt = (tk - t_old) / (t - t_old);
                for (int s = 0; s < P.n_sens; ++s) {
                    hist[s * P.n_out + k] = (1.0 - wgt) * old[s] + wgt * sv[s];
                    if (ahist) ahist[s * P.n_out + k] = (1.0 - wgt) * aold[s] + wgt * sa[s];
                }
                ++k;
            }
            P.s.kout[slot] = k;
        }
        for (int s = 0; s < P.n_sens; ++s) {
            old[s] = sv[s];
            if (aold) aold[s] = sa[s];
        }
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
        atomicSub(P.s.g_active + gi, 1);
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


#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t err__ = (call);                                                        \
        if (err__ != cudaSuccess)                                                          \
            return ofm::fail(OFM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(err__)); \
    } while (0)

}  // namespace

template <typename T, int ORD>
int set_smem_attrs_order() {
    const int bytes = (int)smem_bytes(sizeof(T));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel<T, 0, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel<T, 1, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel<T, 2, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel_persistent<T, 0, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel_persistent<T, 1, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bytes));
    CUDA_TRY(cudaFuncSetAttribute(stage_kernel_persistent<T, 2, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bytes));
    return OFM_OK;
}

template <typename T>
int set_smem_attrs() {
    const int rc = set_smem_attrs_order<T, 5>();
    return rc != OFM_OK ? rc : set_smem_attrs_order<T, 3>();
}

// Grid of the persistent variant: resident blocks per SM (three in single,
// one in double precision) times the SM count, never more than the tiles.
template <typename T>
unsigned persistent_grid(const Params<T>& P) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (long long)sms * (sizeof(T) == 4 ? BLOCKS_FP32 : 1);
    return (unsigned)(P.total_blocks < want ? P.total_blocks : want);
}

template <typename T, int STAGE, int ORD>
void launch_one_stage_order(const Params<T>& P, int variant, int parity, cudaStream_t st) {
    if (variant == OFM_VARIANT_PERSISTENT)
        stage_kernel_persistent<T, STAGE, ORD><<<persistent_grid(P), NT, smem_bytes(sizeof(T)), st>>>(P, parity);
    else
        stage_kernel<T, STAGE, ORD><<<(unsigned)P.total_blocks, NT, smem_bytes(sizeof(T)), st>>>(P, parity);
}

template <typename T, int STAGE>
void launch_one_stage(const Params<T>& P, int variant, int parity, cudaStream_t st) {
    if (P.total_blocks <= 0) return;  // every group finished
    if (P.weno_order == 3)
        launch_one_stage_order<T, STAGE, 3>(P, variant, parity, st);
    else
        launch_one_stage_order<T, STAGE, 5>(P, variant, parity, st);
}

template <typename T>
int launch_step(const Params<T>& Ps, const Params<T>& Pf, int variant, int parity, cudaStream_t st,
                long long* launches) {
    launch_one_stage<T, 0>(Ps, variant, parity, st);
    launch_one_stage<T, 1>(Ps, variant, 1 - parity, st);
    launch_one_stage<T, 2>(Ps, variant, parity, st);
    finalize_kernel<T><<<Pf.total_slots, 256, 0, st>>>(Pf, 0, 1 - parity);
    *launches += 4;
    CUDA_TRY(cudaGetLastError());
    return OFM_OK;
}

template <typename T>
int launch_stage(const Params<T>& Ps, const Params<T>& Pf, int variant, int stage, int parity, cudaStream_t st,
                 long long* launches) {
    if (stage == 0)
        launch_one_stage<T, 0>(Ps, variant, parity, st);
    else if (stage == 1)
        launch_one_stage<T, 1>(Ps, variant, parity, st);
    else if (stage == 2)
        launch_one_stage<T, 2>(Ps, variant, parity, st);
    else
        finalize_kernel<T><<<Pf.total_slots, 256, 0, st>>>(Pf, 0, parity);
    *launches += 1;
    CUDA_TRY(cudaGetLastError());
    return OFM_OK;
}

template <typename T>
int launch_init(const Params<T>& P, cudaStream_t st, bool fill_ic, long long* launches) {
    reset_kernel<T><<<(P.total_slots + 127) / 128, 128, 0, st>>>(P);
    *launches += 1;
    if (fill_ic) {
        ic_kernel<T><<<(unsigned)P.total_blocks, NT, 0, st>>>(P);
        *launches += 1;
    }
    reduce_kernel<T><<<(unsigned)P.total_blocks, NT, 0, st>>>(P, 0);
    finalize_kernel<T><<<P.total_slots, 256, 0, st>>>(P, 1, 0);
    totals_kernel<T><<<P.total_slots, 256, 0, st>>>(P, 0);
    *launches += 3;
    CUDA_TRY(cudaGetLastError());
    return OFM_OK;
}

template <typename T>
int launch_totals(const Params<T>& P, cudaStream_t st, int which, long long* launches) {
    totals_kernel<T><<<P.total_slots, 256, 0, st>>>(P, which);
    *launches += 1;
    CUDA_TRY(cudaGetLastError());
    return OFM_OK;
}

#undef CUDA_TRY

}  // namespace gpu
}  // namespace ofm
