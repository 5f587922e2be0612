/*
 * ofmlmc.h - C ABI of the GB300 library for optimal-fidelity multi-level
 * Monte Carlo (OF-MLMC) of cloud cavitation collapse.
 *
 * Method: Sukys, Rasthofer, Wermelinger, Hadjidoukas, Koumoutsakos,
 * "Optimal fidelity multi-level Monte Carlo for quantification of uncertainty
 * in simulations of cloud cavitation collapse" (2017).
 *
 * Conventions
 *   - Units at this interface are SI (m, Pa, s, kg/m^3).  Internally the
 *     solver is non-dimensional (length L, density 1000 kg/m^3, pressure
 *     p_liq, velocity sqrt(p_liq/1000)).
 *   - Host arrays are owned by the caller.  Device memory is either a
 *     caller-provided workspace (borrowed for the lifetime of the object it
 *     was given to) or allocated by the library when the workspace pointer is
 *     NULL (freed by the matching destroy call).
 *   - Every int-returning call returns OFM_OK (0) or a negative OFM_E* code;
 *     ofm_last_error() gives a message for the calling thread.
 *   - One handle per thread; calls on the same handle must not overlap.
 *   - `stream` arguments are cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Calls order their device work after the work already
 *     queued on that stream.
 */
#ifndef OFMLMC_H
#define OFMLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    OFM_OK = 0,
    OFM_EINVAL = -1,   /* bad argument (sizes, NULL pointers, unsupported grid) */
    OFM_ENOMEM = -2,   /* workspace too small or device allocation failed */
    OFM_ECUDA = -3,    /* a CUDA runtime call failed */
    OFM_ENUMERIC = -4, /* the call completed but some sample's status is non-zero */
    OFM_ETIMEOUT = -5  /* a bounded device-side wait expired */
};

enum { OFM_FP64 = 0, OFM_FP32 = 1 };                      /* stencil storage/arithmetic */
/* Ghost cells: transmissive (nearest interior cell), periodic, or the
 * characteristic far field of Sec. 3.1 (non-reflecting, with a penalty
 * towards the far-field pressure p_liq, after Poinsot and Lele 1992): along
 * the outward normal, with Z = rho c of the interior cell next to the face,
 * the outgoing characteristic p + Z u_n is that cell's and the incoming one
 * p - Z u_n is (1 - bc_penalty) times that cell's plus bc_penalty times the
 * far field at rest, p_liq; partial densities, alpha2 and the tangential
 * velocities are that cell's. */
enum { OFM_BC_TRANSMISSIVE = 0, OFM_BC_PERIODIC = 1, OFM_BC_CHARACTERISTIC = 2 };
enum { OFM_RADII_UNIFORM = 0, OFM_RADII_LOGNORMAL = 1 };  /* cloud radius law */
enum { OFM_MODE_TOL = 0, OFM_MODE_BUDGET = 1 };           /* sample-number optimisation */

/* Per-sample status bits (fault-tolerant MLMC, Section 2.5): a sample with a
 * non-zero status is excluded from estimators. */
enum {
    OFM_ST_NONFINITE = 1, /* NaN/Inf in the state or pressure */
    OFM_ST_NEGATIVE = 2,  /* mixture density or squared sound speed <= 0 */
    OFM_ST_MAXSTEPS = 4,  /* step limit reached before t_end */
    OFM_ST_TIMEOUT = 8    /* a device-side wait for a tile's halo copies ran out
                             (the sample is abandoned, the device stays usable) */
};

#define OFM_MAX_SENSORS 8
#define OFM_MAX_GROUPS 8
#define OFM_MAX_LEVELS 16

/* One spherical bubble; centre and radius in metres. */
typedef struct {
    double x, y, z, r;
} ofm_bubble;

/* Random cloud geometry (Section 3.1): n_bubbles centres uniform in a ball of
 * radius cloud_radius around the domain centre; radii uniform in
 * [r_min, r_max] or log-normal(ln_mu, ln_sigma) truncated to [r_min, r_max].
 * Overlapping bubbles are allowed. */
typedef struct {
    int n_bubbles;
    int radius_law;      /* OFM_RADII_* */
    double cloud_radius; /* m */
    double r_min, r_max; /* m */
    double ln_mu, ln_sigma;
    double domain_L;     /* m, the domain is [0, L]^3 */
} ofm_cloud_params;

/* Flow solver configuration (Sections 2.1-2.2, 3.1). */
typedef struct {
    double gamma[2];  /* stiffened-gas gamma: [0] liquid, [1] gas */
    double pc[2];     /* stiffened-gas p_c [Pa] */
    double rho0[2];   /* initial phase densities [kg/m^3] */
    double p_gas;     /* initial bubble pressure [Pa] */
    double p_liq;     /* initial liquid pressure [Pa] (also the pressure unit) */
    double cfl;       /* Courant number (0.3 in the paper) */
    double t_end;     /* end time [s] */
    double weno_eps;  /* WENO epsilon of the nonlinear weights (non-dimensional) */
    double domain_L;  /* m */
    int precision;    /* OFM_FP64 or OFM_FP32 (FP32 stencil, FP64 reductions) */
    int bc;           /* OFM_BC_* */
    int max_steps;    /* per-sample step limit */
    int n_sensors;    /* <= OFM_MAX_SENSORS */
    double sensors[OFM_MAX_SENSORS][4]; /* centre (x, y, z) and radius [m], Eq. (sensor) */
    int n_out_times;  /* sensor history samples on t_k = k t_end/(n_out_times-1) */
    /* Cloud pressure ramp of the initial condition (Sec. 3.1): with ramp_radius > 0
     * [m] the liquid is at p_cloud [Pa] within ramp_radius of the domain centre and
     * at p_liq + (p_cloud - p_liq) ramp_radius / r at distance r beyond it (the
     * pressure of a liquid at rest around a sphere); 0 = uniform p_liq. */
    double p_cloud;
    double ramp_radius;
    double bc_penalty;  /* OFM_BC_CHARACTERISTIC: weight in [0, 1] of the far field in the incoming
                           characteristic (0 = transmissive, 1 = no reflection of a plane wave
                           leaving along the normal and full penalty); ignored otherwise */
    int weno_order;     /* reconstruction (Jiang & Shu, Sec. 2.2): 5 (or 0) = WENO5, 3 = WENO3 */
} ofm_solver_config;

/* Per-sample quantities of interest (Section 3.2). */
typedef struct {
    double p_peak;          /* max over time (t = 0 and every step) of max over cells of p [Pa] */
    double p_peak_xyz[3];   /* cell centre of the first maximiser (x fastest) [m] */
    double p_peak_t;        /* time of p_peak [s] */
    double p_peak_dist;     /* distance of p_peak_xyz from the domain centre [m] */
    int64_t peak_index;     /* linear cell index of the maximiser */
    double sensor_peak[OFM_MAX_SENSORS]; /* max over time of each sensor [Pa] */
    double totals0[6];      /* sum over cells of Q_0..Q_5 times h^3 at t = 0 (non-dimensional) */
    double totals_end[6];   /* the same at the final time */
    double t_final;         /* [s] */
    int n_steps;
    int status;             /* OFM_ST_* bits */
    double c_max;           /* max over time (t = 0 and every step) of max over cells of the mixture sound speed [m/s] */
    double sensor_alpha0[OFM_MAX_SENSORS];      /* gas-fraction sensors: mean alpha2 over each sensor's cells at t = 0 */
    double sensor_alpha_min[OFM_MAX_SENSORS];   /* their minimum over time (t = 0 and every step) */
    double sensor_alpha_min_t[OFM_MAX_SENSORS]; /* the first time of that minimum [s] (gas-volume collapse time) */
} ofm_qoi;

/* One group of samples on one grid. */
typedef struct {
    int N;                       /* cells per axis: a multiple of 8, 8 <= N <= 512 */
    int n_samples;
    const uint64_t* sample_ids;  /* host [n_samples]; cloud of sample i = (seed, sample_ids[i]) */
    uint64_t seed;
    const ofm_bubble* bubbles;   /* host [n_samples * n_bubbles] or NULL: sample the clouds */
    ofm_qoi* qoi_out;            /* host [n_samples], written by ofm_batch_qoi / ofm_solve_batch */
    double* sensor_hist;         /* host [n_samples][n_sensors][n_out_times] [Pa], or NULL */
    double* alpha_hist;          /* host [n_samples][n_sensors][n_out_times] gas-fraction sensor
                                  * histories (mean alpha2 over each sensor's cells, same output
                                  * times, linear in time between steps), or NULL */
} ofm_group;

typedef struct ofm_solver ofm_solver;
typedef struct ofm_batch ofm_batch;

/* Thread-local message for the last failing call ("" if none). */
const char* ofm_last_error(void);

/* Version string of the library build. */
const char* ofm_version(void);

/* ---------------------------------------------------------------------------
 * Cloud sampler (Section 3.1).  SplitMix64 seeded with
 * seed ^ (sample_id * 0x9E3779B97F4A7C15); uniform doubles from the top 53
 * bits; centres by rejection from the cube [-R, R]^3 (x, y, z per try); then
 * the radius (uniform, or Box-Muller log-normal redrawn until in range).
 * Writes params->n_bubbles bubbles to `out` (host).  Pure host computation.
 * ------------------------------------------------------------------------- */
int ofm_sample_cloud(const ofm_cloud_params* params, uint64_t seed, uint64_t sample_id,
                     ofm_bubble* out);

/* ---------------------------------------------------------------------------
 * Solver handle.  Validates and copies the configuration (non-dimensionalised
 * once).  Allocates no device memory.
 * ------------------------------------------------------------------------- */
int ofm_solver_create(ofm_solver** out, const ofm_solver_config* config);
void ofm_solver_destroy(ofm_solver* solver);

/* Device bytes a batch of these groups needs (states Q, Q', dQ per sample in
 * the configured precision, per-tile partial reductions, per-sample records).
 * Errors: OFM_EINVAL for a bad group table or more than 2^31 - 1 tiles;
 * OFM_ENOMEM when the samples times their bubbles, or times their
 * n_sensors x n_out_times history values, exceed 2^40 (so that no byte count
 * can wrap around; such a batch would not fit any device anyway).  The same
 * checks apply to ofm_batch_create and the calls built on it. */
int ofm_batch_workspace_bytes(const ofm_solver* solver, const ofm_cloud_params* cloud,
                              const ofm_group* groups, int n_groups, size_t* bytes);

/* ---------------------------------------------------------------------------
 * Batched solves of uneven levels (Sections 2.2-2.3 per sample; every group's
 * samples advance together, each with its own CFL time step, in one set of
 * kernel launches per stage).
 *
 * ofm_batch_create: lays out the workspace (device, >= the bytes above; NULL =
 *   allocate), samples or copies the clouds on the host and uploads them.
 * ofm_batch_init:   initial condition, t = 0 reductions and first time step.
 * ofm_batch_run:    advances every unfinished sample by up to max_steps steps
 *   (CUDA-graph-captured chunks); *n_active receives the number of samples
 *   that have not reached t_end (0 when all are done).  Synchronises with the
 *   batch's internal stream once per chunk.
 * ofm_batch_qoi:    copies the QoI records (and the pressure and gas-fraction
 *   sensor histories of the groups that have sensor_hist / alpha_hist buffers)
 *   to the groups' host arrays; returns OFM_ENUMERIC if any sample's status is
 *   non-zero.
 * ofm_batch_copy_state / ofm_batch_set_state: read / overwrite the current
 *   state Q[7][N][N][N] (x fastest, non-dimensional, storage precision) of one
 *   sample; `host_buf` is a host pointer of exactly 7 N^3 elements.  Setting a
 *   state after ofm_batch_init recomputes the sample's t = 0 reductions, so a
 *   caller can start from any state (e.g. to inject a corrupted sample).
 * ------------------------------------------------------------------------- */
int ofm_batch_create(ofm_batch** out, ofm_solver* solver, const ofm_cloud_params* cloud,
                     const ofm_group* groups, int n_groups, void* workspace, size_t workspace_bytes,
                     void* stream);
int ofm_batch_init(ofm_batch* batch);
int ofm_batch_run(ofm_batch* batch, int max_steps, int* n_active);
int ofm_batch_qoi(ofm_batch* batch);
int ofm_batch_copy_state(ofm_batch* batch, int group, int sample, void* host_buf, size_t bytes);
int ofm_batch_set_state(ofm_batch* batch, int group, int sample, const void* host_buf, size_t bytes);
/* Cell-steps (cells x completed RK3 steps, summed over samples) so far. */
int ofm_batch_cell_steps(ofm_batch* batch, double* cell_steps);
/* Number of kernels this batch has launched so far (graph replays count
 * every kernel node). */
int ofm_batch_kernel_launches(ofm_batch* batch, int64_t* launches);
/* Profiling mode (on != 0): later ofm_batch_run steps are launched without
 * graphs, with CUDA events on the batch's stream around each RK-stage kernel;
 * ofm_batch_stage_time returns the accumulated stage-kernel time [ms] and the
 * number of stage launches it covers.  Results are identical in both modes. */
int ofm_batch_set_profiling(ofm_batch* batch, int on);
int ofm_batch_stage_time(ofm_batch* batch, double* total_ms, int64_t* n_launches);
/* Stage-kernel variant: 0 (default) = one block per 8^3 tile; 1 = persistent
 * blocks (three per SM in FP32, one in FP64) with one staging buffer each,
 * issuing the next tile's halo copies (tensor copies; per-row copies with a
 * periodic boundary) before the current tile's update, staging but not
 * computing finished samples' tiles (a copy wait that runs out marks the
 * sample OFM_ST_TIMEOUT); -1 = autotune: the first
 * ofm_batch_run of at least 4 steps times two steps of each variant and keeps
 * the faster.  In FP64 both variants give identical bits; in FP32 they agree
 * to round-off (the compiler may fuse multiply-adds differently in the two
 * kernels), so runs that must be bitwise reproducible keep a fixed variant.
 * get_variant also returns the autotuning times (ms, two steps of each
 * variant; tune_ms holds 2 floats, may be NULL).  Errors: OFM_EINVAL for a
 * variant outside -1..1. */
int ofm_batch_set_variant(ofm_batch* batch, int variant);
int ofm_batch_get_variant(ofm_batch* batch, int* variant, float* tune_ms);
/* Bytes this batch has copied host->device and device->host so far. */
int ofm_batch_transfer_bytes(ofm_batch* batch, int64_t* h2d, int64_t* d2h);
void ofm_batch_destroy(ofm_batch* batch);

/* One call for the whole path: create, init, run to t_end, copy QoIs, destroy. */
int ofm_solve_batch(ofm_solver* solver, const ofm_cloud_params* cloud, const ofm_group* groups,
                    int n_groups, void* workspace, size_t workspace_bytes, void* stream);

/* A single level: ofm_solve_batch with one group. */
int ofm_solve_level(ofm_solver* solver, const ofm_cloud_params* cloud, int N, int n,
                    const uint64_t* sample_ids, uint64_t seed, ofm_qoi* out, double* sensor_hist,
                    void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Allocation-free single-level solve.  The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory, e.g. code
 * running under a framework whose caching allocator already owns the
 * device's memory, or a latency-critical loop in which cudaMalloc/cudaFree
 * would synchronise the device.  It computes exactly what ofm_solve_level
 * computes (same kernels, same results) but allocates no device or pinned
 * memory and creates no streams or events: all device scratch lives in one
 * file-scope __device__ array of OFM_STATIC_SCRATCH_BYTES (32 MiB) that every
 * GPU loading this library holds until the process exits.  Inputs (sample ids,
 * clouds from `cloud`) and outputs (`out`, `sensor_hist`, as in
 * ofm_solve_level) are host arrays owned by the caller.
 *   - Sizes whose scratch would exceed the array are rejected with
 *     OFM_ENOMEM and a message giving the bytes needed (the sample count is
 *     checked against the array by division first, so no byte count can wrap
 *     around and pass the check).  Each sample takes
 *     three state buffers of 7 N^3 values: up to 12 FP32 or 6 FP64 samples on
 *     32^3 fit, one FP32 sample on 64^3, no FP64 sample on 64^3.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and caches it; make that
 *     first call before any stream capture.  The cache assumes the device's
 *     primary context is never reset: after cudaDeviceReset the array may
 *     move, so do not call this entry point again in that process.
 *   - Every call uses the same array and re-initialises what it reads; calls
 *     that overlap on the GPU (other streams or host threads) race on it.
 *   - Synchronises `stream` before returning.
 * ------------------------------------------------------------------------- */
#define OFM_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int ofm_solve_level_static(const ofm_solver* solver, const ofm_cloud_params* cloud, int N, int n,
                           const uint64_t* sample_ids, uint64_t seed, ofm_qoi* out, double* sensor_hist,
                           void* stream);

/* ---------------------------------------------------------------------------
 * OF-MLMC estimator (Section 2.4), host FP64.
 *
 * q[l] points to M[l] rows of (q_l, q_{l-1}) pairs on shared inputs
 * (row-major, 2 doubles per row; the second column is ignored for l = 0).
 * W[l] = cost of one sample (l = 0) or one pair (l > 0).
 * Outputs (arrays of L+1):
 *   alpha        coefficients of Eq. (alpha-matvec), alpha[L] = 1;
 *   sigma2       sample variance of q_l pooled over pair l's fine and pair
 *                l+1's coarse members; cov[l] = sample Cov[q_l, q_{l-1}] of pair l;
 *   sigma_tilde2 sample variance of alpha_l q_l - alpha_{l-1} q_{l-1} (Step 5);
 *   mean         Eq. (ocv-mlmc); eps2 = sum sigma_tilde2/M, Eq. (ocv-mlmc-err).
 * All variances use the M-1 denominator; every level needs M >= 2.
 * ------------------------------------------------------------------------- */
typedef struct {
    double alpha[OFM_MAX_LEVELS];
    double sigma2[OFM_MAX_LEVELS];
    double cov[OFM_MAX_LEVELS];
    double sigma_tilde2[OFM_MAX_LEVELS];
    double mean;
    double eps2;
} ofm_estimate_out;

int ofm_estimate(int L, const int64_t* M, const double* const* q, const double* W,
                 ofm_estimate_out* out);

/* Step 3's optional fit (Section 2.4.3; Section 3.2 fits the level-difference
 * variances with an exponential decay; the appendix on M_L = 1 uses it to
 * start the finest level from one warm-up pair).
 *   ofm_fit_level_variances: V[l] (l = 1..L; V[0] ignored) are the sample
 *     variances of q_l - q_{l-1} over M[l] pairs.  Fits ln V_l = a + b l by
 *     least squares over the levels with M[l] >= 2 and V[l] > 0, each
 *     weighted by (M[l] - 1)/2, the inverse of the Gaussian error of ln V_l:
 *     the posterior mean of (a, b) under flat priors.  Writes
 *     V_fit[l] = exp(a + b l) for l = 1..L, V_fit[0] = 0, and coef = {a, b}
 *     (coef may be NULL).  OFM_EINVAL with fewer than two usable levels.
 *   ofm_estimate_fitted: ofm_estimate with the fitted variances, each
 *     clamped to [(sigma_l - sigma_{l-1})^2, (sigma_l + sigma_{l-1})^2] (so
 *     that |cov_l| <= sigma_l sigma_{l-1}): the covariances of Eq.
 *     (alpha-matvec) become (sigma2_l + sigma2_{l-1} - V_fit_l)/2 and are
 *     returned in out->cov.  Level 0 needs M >= 2, every
 *     level l >= 1 at least one pair; a level whose q_l has a single computed
 *     value takes sigma2_l = sigma2_{l-1}, and a level with one pair takes
 *     sigma_tilde2_l = alpha_l^2 sigma2_l + alpha_{l-1}^2 sigma2_{l-1}
 *     - 2 alpha_l alpha_{l-1} cov_l.  V_fit (L+1 doubles, may be NULL)
 *     receives the fitted level-difference variances.
 * Host FP64 arrays; errors as ofm_estimate plus the fit's. */
int ofm_fit_level_variances(int L, const int64_t* M, const double* V, double* V_fit, double* coef);
int ofm_estimate_fitted(int L, const int64_t* M, const double* const* q, const double* W,
                        ofm_estimate_out* out, double* V_fit);

/* The same estimator from per-level summaries, for pairs spread over several
 * processes (one process per GPU).  Section 2.4 needs only per-level means,
 * pooled variances and the fine/coarse covariance, so each process
 * summarises its own pairs, the summaries are exchanged (a few hundred
 * bytes per level) and combined, and every process evaluates Eqs.
 * (alpha-matvec), (ocv-mlmc) and (ocv-mlmc-err) on the combined summaries.
 *   ofm_level_moments_of: summary of one level's M pairs (row-major (M, 2):
 *     fine, coarse member), two passes over the data; M = 0 gives n = 0.
 *   ofm_merge_moments: summary of the union of two disjoint pair sets
 *     (pairwise update of Chan, Golub and LeVeque); out may alias a or b.
 *   ofm_estimate_moments: ofm_estimate from L+1 summaries (n >= 2 each);
 *     equal to ofm_estimate on the union of the pairs up to round-off.
 * Errors: OFM_EINVAL for NULL pointers, negative counts, n < 2 or W <= 0;
 * OFM_ENUMERIC for a singular coefficient system. */
typedef struct {
    int64_t n;            /* pairs */
    double mean_f, mean_c; /* means of the fine and coarse members */
    double m2_f, m2_c;    /* sums of squared deviations from those means */
    double c_fc;          /* sum of products of the fine and coarse deviations */
} ofm_level_moments;

int ofm_level_moments_of(const double* pairs, int64_t M, ofm_level_moments* out);
int ofm_merge_moments(const ofm_level_moments* a, const ofm_level_moments* b, ofm_level_moments* out);
int ofm_estimate_moments(int L, const ofm_level_moments* moments, const double* W, ofm_estimate_out* out);
/* ofm_estimate_fitted from L+1 summaries (level 0 n >= 2, levels l >= 1
 * n >= 1; V[q_l - q_{l-1}] = (m2_f + m2_c - 2 c_fc)/(n - 1)); equal to
 * ofm_estimate_fitted on the union of the pairs up to round-off.  V_fit as
 * there (may be NULL). */
int ofm_estimate_moments_fitted(int L, const ofm_level_moments* moments, const double* W, ofm_estimate_out* out,
                                double* V_fit);

/* Eq. (M-tol) (mode OFM_MODE_TOL, target = tau, constraint eps_OF <= tau) or
 * Eq. (M-budget) (OFM_MODE_BUDGET, target = budget) with the step-7 rule that
 * keeps already computed samples (M_done may be NULL = none).  OFM_EINVAL for a
 * negative or non-finite sigma_tilde2, W <= 0, a target the kept samples
 * already exceed, or a level that would need more than 4e18 samples. */
int ofm_optimal_samples(int L, const double* sigma_tilde2, const double* W, const int64_t* M_done,
                        double target, int mode, int64_t* M_out);

/* Eq. (warmup): M_l = ceil(W_L / W_l / 2^(L-l)). */
int ofm_warmup_samples(int L, const double* W, int64_t* M_out);

/* ---------------------------------------------------------------------------
 * Adaptive OF-MLMC over GPU solves (Section 2.4.3, steps 1-8).
 * Level l solves on N[l]^3; pair i of level l uses the cloud of sample id
 * (l << 40) | i for both its members (N[l] and N[l-1]).  Step 1 takes the
 * warm-up numbers of Eq. (warmup) from the cost model W_l ~ N_l^4 (+ N_{l-1}^4),
 * raised to min_samples (>= 2: without the optional Bayesian fit of step 3 a
 * variance needs two samples; with it, fit_variances, the finest of L >= 3
 * levels is not raised).  Each iteration solves every level's missing
 * pairs in one uneven batch (split only if it exceeds max_batch_bytes; 0 =
 * 80% of the free device memory), measures the pair costs W_l as mean
 * cell-steps per pair, excludes pairs with a failed member (status != 0),
 * computes the estimator (ofm_estimate, or ofm_estimate_fitted) and stops
 * when eps_OF <= target (tol mode) or the cell-steps spent reach target
 * (budget mode); otherwise, unless
 * it was the last of max_iterations, step 7 re-optimises M_l
 * (ofm_optimal_samples, keeping computed pairs).
 * pairs_out / ids_out (host, may be NULL): the (q_l, q_{l-1}) rows and sample
 * ids of the pairs used, level by level; pairs_capacity rows.
 * ------------------------------------------------------------------------- */
typedef struct {
    int L;                     /* finest level index (levels 0..L, L <= 3) */
    int N[OFM_MAX_LEVELS];     /* grid per level, coarse to fine */
    int mode;                  /* OFM_MODE_TOL or OFM_MODE_BUDGET */
    double target;             /* tau [QoI units] or budget [cell-steps] */
    int qoi;                   /* 0: p_peak; 1 + k: sensor_peak[k] */
    uint64_t seed;
    int max_iterations;
    int min_samples;
    size_t max_batch_bytes;
    double max_cell_steps;     /* safety cap on the total work (0 = none): an iteration that
                                  would exceed it is not started and result.capped is set */
    int fit_variances;         /* 1: step 3's variance fit (ofm_estimate_fitted) in every
                                  iteration; with L >= 3 the finest level keeps the single
                                  warm-up pair of Eq. (warmup) (L < 2 is refused) */
    /* Learned surrogate of q_L as an extra control variate of the top level term
     * (not in the paper; see ofm_estimate_surrogate).  Once level L has
     * surrogate_min_pairs usable pairs, every iteration trains two MLPs
     * (surrogate_hidden x 3 GELU layers, BF16 operands, FP32 accumulation,
     * Adam at surrogate_lr, up to surrogate_steps steps with the parameters of
     * the lowest error on a fifth of the fold held out) on the two halves of
     * the level-L pairs (input: the surrogate_nearest bubbles nearest the domain
     * centre, ofm_cloud_features, and the pair's q_{L-1}; target: the residual
     * q_L - q_{L-1}, so the prediction of q_L is q_{L-1} plus it), predicts
     * each pair with the network of the other half (cross-fitting) and the
     * level-(L-1) pairs' fine members with both, and estimates with
     * ofm_estimate_surrogate; step 7 then takes the modified variances.  Its
     * device time counts in gpu_seconds.  Needs L >= 1 and no variance fit. */
    int surrogate;             /* 1: on */
    int surrogate_min_pairs;   /* 0: 64 */
    int surrogate_nearest;     /* bubbles per cloud in the input (0: all) */
    int surrogate_steps;       /* 0: 600 */
    int surrogate_hidden;      /* 0: 256 */
    double surrogate_lr;       /* 0: 1e-3 */
    double* surrogate_h_out;   /* optional host array (one per returned pair, in pairs_out
                                  order): the prediction used for that pair, NaN where none */
} ofm_run_config;

typedef struct {
    int iterations;
    int64_t M[OFM_MAX_LEVELS];   /* pairs used per level (failed ones excluded) */
    double W[OFM_MAX_LEVELS];    /* mean cell-steps per pair */
    double gpu_seconds;          /* device time of the solves (CUDA events) */
    double cell_steps;           /* total cell-steps solved */
    int64_t failed;              /* pairs excluded */
    int capped;                  /* 1 if max_cell_steps stopped the loop */
    ofm_estimate_out est;        /* final estimator, Eqs. (ocv-mlmc), (ocv-mlmc-err) */
    int surrogate_used;          /* 1 if the final estimator has the surrogate control variate */
    double beta;                 /* its coefficient (0 without) */
    double surrogate_seconds;    /* device time of its training and inference (in gpu_seconds) */
    double eps2_plain;           /* eps^2 of the plain estimator on the final pairs */
    double sigma_tilde2_plain[OFM_MAX_LEVELS];  /* and its level variances */
} ofm_run_result;

int ofm_run(ofm_solver* solver, const ofm_cloud_params* cloud, const ofm_run_config* config, double* pairs_out,
            uint64_t* ids_out, int64_t pairs_capacity, ofm_run_result* result, void* stream);

/* Measured multiply-add rate [TFLOP/s, a multiply-add = 2 flops] of the
 * current device's FP32 (precision OFM_FP32) or FP64 (OFM_FP64) pipes:
 * eight independent register chains per thread, 8 blocks of 256 threads per
 * SM, 3 untimed and 10 timed launches on the given stream, CUDA events.  The
 * ceiling that the stencil kernels' ALU roofline is read against, measured at
 * the clocks the GPU runs at.  The paper has no counterpart.  Errors:
 * OFM_EINVAL for a bad precision or NULL tflops, OFM_ECUDA. */
int ofm_probe_fma_tflops(int precision, double* tflops, void* stream);

/* ---------------------------------------------------------------------------
 * Surrogate control variate (not in the paper).  An MLP s(x) of the cloud
 * geometry x predicts the finest-level QoI; it enters the estimator only as
 * an extra control variate for the top-level term D = q_L - alpha_{L-1} q_{L-1}:
 *   E[D] ~ mean_M(D) + beta (mean_N(s) - mean_M(s)),
 * with s evaluated on the M finest-pair inputs and on N independent extra
 * inputs.  beta = Cov(D, s)/(V[s] (1 + M/N)) minimises the variance, which is
 * then (V[D] - Cov(D, s)^2/(V[s] (1 + M/N)))/M.  The estimate is unbiased for
 * any fixed beta, so a poor surrogate costs variance, never bias.
 * Host FP64; arrays are host pointers; M >= 2, N >= 1.
 * ------------------------------------------------------------------------- */
/* ---------------------------------------------------------------------------
 * OF-MLMC with the surrogate as an extra control variate of the top level
 * term, inside the estimator (not in the paper; it extends Eq. (ocv-mlmc) of
 * Section 2.4.2 by one coefficient).  The surrogate h predicts q_L from a
 * cloud and its q_{L-1}; the control variate is its prediction of the top
 * level term, g = h - alpha_{L-1} q_{L-1}.  Its mean is estimated on the fine
 * members of the level-(L-1) pairs, whose q_{L-1} is computed anyway:
 *   level L-1 terms: alpha_{L-1} q_{L-1} - alpha_{L-2} q_{L-2} + beta g(h_extra)
 *   level L terms:   q_L - alpha_{L-1} q_{L-1} - beta g(h_top)
 * The estimate is unbiased for any fixed alpha and beta (h must not have been
 * trained on the pairs it is evaluated on: cross-fitting), every level stays
 * a mean over its own pairs, so eps2 = sum sigma_tilde2/M and the sample
 * numbers of step 7 (ofm_optimal_samples) apply to the modified variances.
 *   L >= 1; M, q, W as in ofm_estimate (host arrays);
 *   h_top: M[L] predictions on the level-L pairs' inputs (cloud, coarse member);
 *   h_extra: M[L-1] predictions on the level-(L-1) pairs' inputs (cloud, fine member);
 *   beta_in: NaN for the coefficient that minimises eps2 at the current M,
 *            (Cov_L(D_L, g)/M_L - Cov_{L-1}(D_{L-1}, g)/M_{L-1})
 *            / (V_{L-1}[g]/M_{L-1} + V_L[g]/M_L), 0 when g does not vary;
 *            else that fixed beta;
 *   out: alpha, sigma2, cov as in ofm_estimate; sigma_tilde2, mean, eps2 of the
 *        corrected estimator; beta_out: the coefficient used;
 *   sigma_tilde2_plain (may be NULL): L+1 variances of the plain estimator.
 * Errors: OFM_EINVAL (bad sizes, fewer than 2 pairs on a level).
 * ------------------------------------------------------------------------- */
int ofm_estimate_surrogate(int L, const int64_t* M, const double* const* q, const double* W,
                           const double* h_top, const double* h_extra, double beta_in,
                           ofm_estimate_out* out, double* beta_out, double* sigma_tilde2_plain);

int ofm_surrogate_cv(const double* D, const double* s_paired, int64_t M, const double* s_extra, int64_t N,
                     double* beta, double* corrected_mean, double* variance);

/* ---------------------------------------------------------------------------
 * Level-wise kernel density estimate of a QoI (Section 3.2, which estimates
 * the PDFs of its QoIs with level-dependent kernel density estimators whose
 * bandwidth comes from the "solve-the-equation" method of Sheather and Jones,
 * 1991).  Host FP64.
 *   ofm_sj_bandwidth: the solve-the-equation bandwidth of a Gaussian-kernel
 *     KDE of x[n] (n >= 2): h = [R(K)/(n psi_4(g(h)))]^(1/5), psi_r estimated
 *     by sum_{i != j} phi^(r)((x_i - x_j)/g)/(n (n-1) g^(r+1)), the pilot g(h)
 *     from normal-reference pilots (scale min(sd, IQR/1.349); a pilot estimate
 *     of the wrong sign, psi_4 <= 0 or psi_6 >= 0, takes its normal-reference
 *     value), the root by bisection to 1e-10 relative; 0 for a sample without
 *     spread.  O(n^2) per evaluation.
 *   ofm_level_kde: density[k] at x[k] of
 *     f(x) = sum_l (1/M_l) sum_i [alpha_l K_b(x - q_l^i) - alpha_{l-1} K_b(x - q_{l-1}^i)],
 *     K_b the Gaussian kernel, b = b_l the larger of the solve-the-equation
 *     bandwidths of level l's fine and coarse members (bandwidth[l], may be
 *     NULL); pairs q and M as in ofm_estimate, alpha e.g. ofm_estimate's.
 *     It integrates to alpha_L = 1, its first moment is Eq. (ocv-mlmc)'s mean.
 *   Errors: OFM_EINVAL (fewer than 2 pairs on a level), OFM_ENUMERIC (a level
 *   without spread).
 * ------------------------------------------------------------------------- */
int ofm_sj_bandwidth(const double* x, int64_t n, double* h);
int ofm_level_kde(int L, const int64_t* M, const double* const* q, const double* alpha, const double* x,
                  int64_t n_x, double* density, double* bandwidth);

/* ---------------------------------------------------------------------------
 * MLP (the surrogate network): d_in -> hidden (x n_hidden, exact-erf GELU) ->
 * d_out.  Parameters are one FP32 vector: for each layer l, W_l as
 * (fan_in x fan_out) row-major, then b_l (fan_out).  Every GEMM rounds its
 * operands to BF16 (round to nearest even) and accumulates in FP32 on the
 * tensor cores; activations, gradients, master weights and Adam moments are
 * FP32.  Inputs are standardised by (x - x_mean)/x_std and targets by
 * (t - y_mean)/y_std (ofm_mlp_set_scaling; identity until set); the loss is
 * the mean squared error in standardised target space; forward returns
 * de-standardised outputs.  X, T, Y are device pointers, row-major
 * (rows x d_in / d_out).  Training is full-batch Adam (beta 0.9/0.999,
 * eps 1e-8) with n <= max_rows; forward takes any n (chunks of max_rows).
 * All reductions have a fixed order (deterministic).
 * ------------------------------------------------------------------------- */
#define OFM_MLP_MAX_LAYERS 8
#define OFM_MLP_MAX_STEPS 200000
typedef struct ofm_mlp ofm_mlp;
/* Errors: OFM_EINVAL for a size < 1 or more than OFM_MLP_MAX_LAYERS layers;
 * OFM_ENOMEM for a weight matrix or a max_rows x width activation array of
 * more than 2^40 values (no byte count can wrap around). */
int ofm_mlp_workspace_bytes(int d_in, int hidden, int n_hidden, int d_out, int max_rows, size_t* bytes);
int ofm_mlp_create(ofm_mlp** out, int d_in, int hidden, int n_hidden, int d_out, int max_rows, void* workspace,
                   size_t workspace_bytes);
void ofm_mlp_destroy(ofm_mlp* mlp);
int ofm_mlp_param_count(const ofm_mlp* mlp, int64_t* n);
/* Host copies of the parameter vector; set also resets the Adam state. */
int ofm_mlp_set_params(ofm_mlp* mlp, const float* host_params);
int ofm_mlp_get_params(ofm_mlp* mlp, float* host_params);
/* Host arrays of d_in / d_out entries; a zero std leaves that entry unscaled. */
int ofm_mlp_set_scaling(ofm_mlp* mlp, const float* x_mean, const float* x_std, const float* y_mean,
                        const float* y_std);
int ofm_mlp_forward(ofm_mlp* mlp, const float* X, int n, float* Y, void* stream);
/* Loss and gradient (host copies) at the current parameters, without a step. */
int ofm_mlp_gradients(ofm_mlp* mlp, const float* X, const float* T, int n, float* grads_host, float* loss_host,
                      void* stream);
/* `steps` Adam steps (one CUDA graph per step, replayed); the loss before
 * each step goes to loss_hist_host[steps] if not NULL.  Synchronises. */
int ofm_mlp_train(ofm_mlp* mlp, const float* X, const float* T, int n, int steps, float lr, float* loss_hist_host,
                  void* stream);
/* Column mean and standard deviation (M-1) of a device matrix, into device
 * FP64 arrays, fixed summation order. */
int ofm_column_moments(const float* X, int rows, int cols, double* mean_dev, double* std_dev, void* stream);
/* Surrogate inputs: per cloud, its n_keep bubbles nearest the domain centre
 * by the gap between the bubble's surface and the centre, |x_b - L/2| - r_b
 * (ties by index), in that order, each as
 * ((x - L/2)/scale, (y - L/2)/scale, (z - L/2)/scale, r/scale).
 * bubbles_dev: device [n_clouds][n_bubbles][4] doubles (metres);
 * n_keep: 1..n_bubbles (0 = all); X_dev: device [n_clouds][4 n_keep] floats.
 * Errors: OFM_EINVAL for bad sizes, OFM_ECUDA. */
int ofm_cloud_features(const double* bubbles_dev, int n_clouds, int n_bubbles, int n_keep, double domain_L,
                       double scale, float* X_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OFMLMC_H */
