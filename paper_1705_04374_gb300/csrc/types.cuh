// Types shared by the host API and the per-precision kernel translation units.
#pragma once

#include <cuda.h>   // CUtensorMap (the staging tensor maps of the state buffers)
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ofmlmc.h"

namespace ofm {
namespace gpu {

constexpr int TS = 8;                    // tile edge (cells)
constexpr int HALO = 3;                  // WENO5 needs three cells on each side
constexpr int BX = TS + 2 * HALO;        // staged box edge (14)
constexpr int NCELL = TS * TS * TS;      // 512 cells per tile
constexpr int NSLAB = HALO * TS * TS;    // 192 cells per halo slab
constexpr int NCROSS = TS * TS * 16 + 4 * NSLAB;  // 1792 staged slots (1664 cells + row padding)
// Single-precision WENO5 accumulates per-cell flux differences in an
// [8][RSTRIDE] array (slots permuted against bank conflicts) instead of
// staging the near faces' fluxes.
constexpr int RSTRIDE = NCELL;
constexpr int NFAR = 3 * 8 * TS * TS;    // far faces of all three directions, 8 values each
constexpr int NFLUX = (8 * RSTRIDE > 8 * NCELL ? 8 * RSTRIDE : 8 * NCELL) + NFAR;  // shared flux values
constexpr int NT = 256;                  // threads per block (measured better than 192 and 256x2)
constexpr int CELLS_PER_THREAD = (NCELL + NT - 1) / NT;  // 2
constexpr int NEAR_RUN = 2;             // FP32: consecutive near faces per thread task (1: one face per task)
constexpr int CHUNK_STEPS = 8;           // steps per captured graph (even)
// resident FP32 stage-kernel blocks per SM: 80 registers per thread (two blocks
// at up to 128 registers measured 10 % slower: latency hiding wins over spills)
constexpr int BLOCKS_FP32 = 3;


template <typename T>
struct Eos {
    T g1, g2, pc1, pc2;   // gamma, p_c (non-dimensional)
    T gi1, gi2;           // 1/(gamma-1)
    T pi1, pi2;           // gamma p_c/(gamma-1)
    T eps;                // WENO epsilon
};

struct Partial {          // per-tile reduction of one state
    double smax;          // max over cells of max_d(|u_d| + c)
    double cmax;          // max over cells of the mixture sound speed c
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
    double c_max;                              // max over time of the max sound speed
    double sensor_alpha0[OFM_MAX_SENSORS];     // sensor gas fractions at t = 0
    double sensor_alpha_min[OFM_MAX_SENSORS];  // their minimum over time
    double sensor_alpha_min_t[OFM_MAX_SENSORS];  // and the first time of it
};

// Box shapes of the halo staging by the tensor memory accelerator (x extent
// first): the tile's rows with their x halos, a y-halo slab, a z-halo slab.
constexpr int TMA_BOX_INT = 0, TMA_BOX_YHALO = 1, TMA_BOX_ZHALO = 2;

struct GroupDev {
    // tm[b][k]: 4-D tiled view (x, y, z, 7 sample + variable) of state buffer
    // b (0: QA, 1: QB) with box shape k
    CUtensorMap tm[2][3];
    int N, tpd, tps, n_samples, slot0;
    long long block0;     // first block of this group in the flattened tile grid
    void* QA;
    void* QB;
    void* dQ;
    Partial* part;
    const int* sens_cells;
    int sens_off[OFM_MAX_SENSORS + 1];
    double h;
    float h32;            // (float)h, converted once on the host (the same rounding as on the device)
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
    double* alpha_old;    // [slot][OFM_MAX_SENSORS] (NULL: no gas-fraction histories)
    double* ahist;        // [slot][n_sens][n_out] gas-fraction histories, or NULL
    int* n_active;
    int* g_active;          // [group] samples not yet finished
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
    T rkA_t[3], rkB_t[3];      // the coefficients in the stencil precision (converted on the host)
    int bc, nb, n_sens, n_out, max_steps, total_slots;
    double t_end, cfl, p_gas, p_liq, rho1, rho2;
    double p_cloud, ramp_r0;   // cloud pressure ramp of the initial condition (ramp_r0 = 0: off)
    double bc_penalty;         // characteristic boundary: far-field weight (far field at p_liq)
    int weno_order;            // 5 (WENO5) or 3 (WENO3)
};

// Low-storage TVD RK3 (Gottlieb & Shu 1998), Williamson 2N form.
constexpr double RK_A[3] = {0.0, -2.915492524638791, -0.000000093517376};
constexpr double RK_B[3] = {0.924574, 0.287713063186749, 0.626538109512740};

// Stage-kernel dynamic shared memory: primitives of the staged cells, face
// fluxes (near faces of one direction or, in single-precision WENO5, the
// per-cell y + z flux differences; far faces of all three directions) and
// the staging layout's per-row slot table
// (FP32: 74.4 KB, three blocks per SM; FP64: 148 KB, one).
// (+128 bytes: the kernels align the staging buffer to 128 bytes for the
// tensor copies.)
constexpr size_t smem_bytes(size_t elem) { return elem * (7 * NCROSS + NFLUX) + 2 * sizeof(int) * BX * BX + 128; }

// Stage-kernel variants: one block per tile, or persistent blocks that issue
// the next tile's copies before the current tile's update.
constexpr int OFM_VARIANT_TILES = 0;
constexpr int OFM_VARIANT_PERSISTENT = 1;
constexpr int OFM_N_VARIANTS = 2;

// Launch wrappers, instantiated for double in kernels_fp64.cu (compiled
// without FMA contraction, in the oracle's operation order) and for float in
// kernels_fp32.cu.  Each returns OFM_OK or OFM_ECUDA and counts its launches.
template <typename T>
int set_smem_attrs();
// Ps: the table the stage kernels walk (finished groups may be left out);
// Pf: the full table (finalize and reductions index samples by slot).
template <typename T>
int launch_step(const Params<T>& Ps, const Params<T>& Pf, int variant, int parity, cudaStream_t st,
                long long* launches);
template <typename T>
int launch_init(const Params<T>& P, cudaStream_t st, bool fill_ic, long long* launches);
// stage 0..2: one RK stage kernel; stage 3: the step's finalize kernel.
template <typename T>
int launch_stage(const Params<T>& Ps, const Params<T>& Pf, int variant, int stage, int parity, cudaStream_t st,
                 long long* launches);
template <typename T>
int launch_totals(const Params<T>& P, cudaStream_t st, int which, long long* launches);

}  // namespace gpu
}  // namespace ofm
