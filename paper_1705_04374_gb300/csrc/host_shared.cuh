// Host-side set-up shared by the batch API (solver.cu) and the
// allocation-free entry point (solver_static.cu): the solver's constants in a
// kernel parameter table, sensor membership, and the conversion of a device
// QoI record to the caller's SI record.  One definition, so a field added to
// the table or the record reaches both entry points.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "ofmlmc.h"
#include "types.cuh"

namespace ofm {
namespace gpu {

// The tensor maps of a group's two state buffers for the stage kernels'
// halo staging: 4-D views (x, y, z, 7 sample + variable) of QA and QB, one
// per staging box shape ([16, 8, 8], [8, 3, 8], [8, 8, 3] cells; the box of
// the tile's rows starts four cells before the tile in x).  Encoded on the
// host through the driver's cuTensorMapEncodeTiled (no allocation).
inline int group_tensor_maps(GroupDev& G, size_t elem) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return ofm::fail(OFM_ECUDA, "the driver does not provide cuTensorMapEncodeTiled");
    const cuuint64_t N = (cuuint64_t)G.N;
    const cuuint64_t dims[4] = {N, N, N, 7ull * (cuuint64_t)G.n_samples};
    const cuuint64_t strides[3] = {N * elem, N * N * elem, N * N * N * elem};
    const cuuint32_t boxes[3][4] = {{(cuuint32_t)(TS + 8), TS, TS, 1}, {TS, HALO, TS, 1}, {TS, TS, HALO, 1}};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    void* bufs[2] = {G.QA, G.QB};
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 3; ++k) {
            const CUresult r = encode(&G.tm[b][k],
                                      elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                                      bufs[b], dims, strides, boxes[k], estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return ofm::fail(OFM_ECUDA, "cuTensorMapEncodeTiled failed (%d) for N = %d, %d samples", (int)r, G.N,
                                 G.n_samples);
        }
    return OFM_OK;
}

// Everything in Params that depends on the solver configuration only
// (non-dimensional EOS constants, RK coefficients, boundary, WENO order,
// sensors, output times, time span, CFL, initial-condition pressures and
// densities).  Group tables and sample pointers are the caller's.
template <typename T>
inline void params_constants(const ofm_solver* s, int nb, Params<T>& P) {
    const ofm_solver_config& c = s->cfg;
    const double pref = s->p_ref;
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
    for (int k = 0; k < 3; ++k) {
        P.rkA[k] = RK_A[k];
        P.rkB[k] = RK_B[k];
        P.rkA_t[k] = (T)RK_A[k];
        P.rkB_t[k] = (T)RK_B[k];
    }
    P.bc = c.bc;
    P.bc_penalty = c.bc_penalty;
    P.weno_order = c.weno_order == 3 ? 3 : 5;
    P.nb = nb;
    P.n_sens = c.n_sensors;
    P.n_out = c.n_out_times;
    P.max_steps = c.max_steps;
    P.t_end = c.t_end / s->t_ref;
    P.cfl = c.cfl;
    P.p_gas = c.p_gas / pref;
    P.p_liq = c.p_liq / pref;
    P.p_cloud = c.p_cloud / pref;
    P.ramp_r0 = c.ramp_radius / c.domain_L;
    P.rho1 = c.rho0[0] / 1000.0;
    P.rho2 = c.rho0[1] / 1000.0;
}

// Sensor membership (Eq. sensor, with the ball widened to one cell): cells
// whose centre lies within max(r, h) of the sensor centre, from
// integer-derived coordinates in FP64, listed per sensor in increasing linear
// index; sens_off[k]..sens_off[k+1] are sensor k's entries of `cells`.
inline void sensor_cell_list(const ofm_solver* s, int N, std::vector<int>& cells, int* sens_off) {
    const double h = 1.0 / N;
    cells.clear();
    sens_off[0] = 0;
    for (int k = 0; k < s->cfg.n_sensors; ++k) {
        const double cx = s->cfg.sensors[k][0] / s->L, cy = s->cfg.sensors[k][1] / s->L;
        const double cz = s->cfg.sensors[k][2] / s->L, r = s->cfg.sensors[k][3] / s->L;
        const double R = r > h ? r : h;
        for (int z = 0; z < N; ++z)
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) {
                    const double dx = (x + 0.5) * h - cx, dy = (y + 0.5) * h - cy, dz = (z + 0.5) * h - cz;
                    if (dx * dx + dy * dy + dz * dz <= R * R) cells.push_back((z * N + y) * N + x);
                }
        sens_off[k + 1] = (int)cells.size();
    }
}

// Device record (non-dimensional) -> SI record of a sample on N^3:
// peak pressure with its cell centre and distance from the domain centre,
// sensor peaks, maximum sound speed, gas-fraction sensors, conserved totals,
// final time t_final_nd and step count.
inline void qoi_to_si(const ofm_solver* s, int N, const DevQoi& d, double t_final_nd, int n_steps, ofm_qoi& o) {
    const ofm_solver_config& c = s->cfg;
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
    o.c_max = d.c_max * s->u_ref;
    for (int k2 = 0; k2 < c.n_sensors; ++k2) {
        o.sensor_alpha0[k2] = d.sensor_alpha0[k2];
        o.sensor_alpha_min[k2] = d.sensor_alpha_min[k2];
        o.sensor_alpha_min_t[k2] = d.sensor_alpha_min_t[k2] * s->t_ref;
    }
    for (int v = 0; v < 6; ++v) {
        o.totals0[v] = d.totals0[v];
        o.totals_end[v] = d.totals_end[v];
    }
    o.t_final = t_final_nd * s->t_ref;
    o.n_steps = n_steps;
    o.status = d.status;
}

}  // namespace gpu
}  // namespace ofm
