/*
 * Oracle: plain FP64 CPU solver for the cloud-collapse problem of
 * Sukys et al., "Optimal fidelity multi-level Monte Carlo for quantification
 * of uncertainty in simulations of cloud cavitation collapse" (2017).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA path and the timed CPU baseline.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * library and includes none of its headers.
 *
 * What it computes, in the paper's order (Section 2.1-2.2):
 *   - the five-equation model, Eqs. (mass_1)...(vol_frac) with K of Eq. (var_K),
 *     in the quasi-conservative form of Eq. (system): Q = (a1r1, a2r2, ru, rv, rw, E, a2);
 *   - stiffened-gas closure p = (gamma_k-1) rho_k e_k - gamma_k pc_k under the
 *     isobaric assumption, giving the mixture p = (E - 1/2 rho|u|^2 - Pi)/Gamma;
 *   - method of lines, Eq. (ode), on a uniform grid: WENO5 (Jiang-Shu) of the
 *     primitive variables, HLLC fluxes with an upwind alpha2 flux and a face
 *     velocity for div(u), source R7 = (alpha2 + K) div(u);
 *   - 3-stage low-storage RK (Williamson 2N form, TVD coefficients of
 *     Gottlieb & Shu 1998), CFL-limited step from a max over all cells;
 *   - quantities of interest: max pressure and its location, ball-average
 *     pressure sensors (Eq. sensor), conserved totals.
 *
 * Readings of points the paper leaves open (units, WENO eps, wave speeds,
 * the alpha2 flux, positivity fallback, IC smoothing, sensor discretisation)
 * are stated next to the code that takes them.
 *
 * Plain loops, no blocking, no SIMD.  Compiled with -O2 -ffp-contract=off so
 * that x86 and Arm builds round identically.
 *
 * Layout: every field is [var][z][y][x] with x fastest, 7 variables.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 7

/* ------------------------------------------------------------------ */
/* Flop counter (compiled in only with -DORC_COUNT_FLOPS).  Convention:  */
/* add, sub, mul, div, sqrt = 1 each; min/max/compare/abs = 0.           */
/* ------------------------------------------------------------------ */
#ifdef ORC_COUNT_FLOPS
static double orc_flops = 0.0;
#define FL(n) (orc_flops += (double)(n))
#else
#define FL(n) ((void)0)
#endif

double orc_flop_count(void) {
#ifdef ORC_COUNT_FLOPS
    return orc_flops;
#else
    return -1.0;
#endif
}
void orc_flop_reset(void) {
#ifdef ORC_COUNT_FLOPS
    orc_flops = 0.0;
#endif
}

typedef struct {
    int nx, ny, nz;   /* cells per axis */
    int bc;           /* 0: transmissive (nearest interior cell), 1: periodic,
                         2: characteristic far field (see char_ghost) */
    double h;         /* cell width, non-dimensional */
    double gamma1;    /* phase 1 = liquid */
    double gamma2;    /* phase 2 = gas */
    double pc1, pc2;  /* stiffening pressures, non-dimensional */
    double cfl;
    double weno_eps;
    double p_inf;      /* far-field pressure of bc 2, non-dimensional */
    double bc_penalty; /* kappa of bc 2 in [0, 1]: 0 = transmissive, 1 = far field */
    int weno_order;    /* 5 (WENO5) or 3 (WENO3) */
} orc_grid;

/* ------------------------------------------------------------------ */
/* Mixture closure (Section 2.1).                                       */
/* With rho e = sum_k alpha_k rho_k e_k and each phase obeying           */
/* p = (g_k - 1) rho_k e_k - g_k pc_k at a common p:                     */
/*   rho e = Gamma p + Pi,  Gamma = sum alpha_k/(g_k-1),                 */
/*   Pi = sum alpha_k g_k pc_k/(g_k-1).                                  */
/* alpha2 is clamped to [0,1] for the closure only.                      */
/* ------------------------------------------------------------------ */
static double clamp01(double a) { return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a); }

/* The bracketed factors are per-run constants. */
static double mix_gamma(const orc_grid* g, double a2) {
    double a = clamp01(a2);
    FL(4); /* 1 - a, two products by per-run constants, one add */
    return (1.0 - a) * (1.0 / (g->gamma1 - 1.0)) + a * (1.0 / (g->gamma2 - 1.0));
}
static double mix_pi(const orc_grid* g, double a2) {
    double a = clamp01(a2);
    FL(3); /* two products by per-run constants, one add (1 - a shared) */
    return (1.0 - a) * (g->gamma1 * g->pc1 / (g->gamma1 - 1.0))
         + a * (g->gamma2 * g->pc2 / (g->gamma2 - 1.0));
}

/* Q -> W = (a1r1, a2r2, u, v, w, p, a2) */
void orc_prim_from_cons(const orc_grid* g, const double* q, double* w) {
    double rho = q[0] + q[1];
    double u = q[2] / rho, v = q[3] / rho, ww = q[4] / rho;
    double G = mix_gamma(g, q[6]);
    double Pi = mix_pi(g, q[6]);
    double ke = 0.5 * rho * (u * u + v * v + ww * ww);
    FL(1 + 3 + 7 + 3);
    w[0] = q[0];
    w[1] = q[1];
    w[2] = u;
    w[3] = v;
    w[4] = ww;
    w[5] = (q[5] - ke - Pi) / G;
    w[6] = q[6];
}

/* W -> Q */
void orc_cons_from_prim(const orc_grid* g, const double* w, double* q) {
    double rho = w[0] + w[1];
    double G = mix_gamma(g, w[6]);
    double Pi = mix_pi(g, w[6]);
    q[0] = w[0];
    q[1] = w[1];
    q[2] = rho * w[2];
    q[3] = rho * w[3];
    q[4] = rho * w[4];
    q[5] = G * w[5] + Pi + 0.5 * rho * (w[2] * w[2] + w[3] * w[3] + w[4] * w[4]);
    q[6] = w[6];
}

void orc_prim_to_cons_array(const orc_grid* g, const double* W, double* Q, long n) {
    double w[NV], q[NV];
    for (long i = 0; i < n; ++i) {
        for (int v = 0; v < NV; ++v) w[v] = W[v * n + i];
        orc_cons_from_prim(g, w, q);
        for (int v = 0; v < NV; ++v) Q[v * n + i] = q[v];
    }
}

void orc_cons_to_prim_array(const orc_grid* g, const double* Q, double* W, long n) {
    double w[NV], q[NV];
    for (long i = 0; i < n; ++i) {
        for (int v = 0; v < NV; ++v) q[v] = Q[v * n + i];
        orc_prim_from_cons(g, q, w);
        for (int v = 0; v < NV; ++v) W[v * n + i] = w[v];
    }
}

/* Frozen mixture sound speed squared: c^2 = ((Gamma+1) p + Pi)/(Gamma rho),
 * which reduces to g (p + pc)/rho for a pure phase. */
static double sound2(const orc_grid* g, const double* w) {
    double rho = w[0] + w[1];
    double G = mix_gamma(g, w[6]);
    double Pi = mix_pi(g, w[6]);
    FL(6);
    return ((G + 1.0) * w[5] + Pi) / (G * rho);
}

/* ------------------------------------------------------------------ */
/* WENO5 of Jiang & Shu (1996): value at the right face of the cell      */
/* holding c, from the five cell averages a, b, c, d, e (left to right). */
/* Ideal weights (1/10, 6/10, 3/10), alpha_k = d_k/(eps + beta_k)^2.     */
/* The value at the left face of the same cell is the same formula with  */
/* the five averages given in reverse order.                             */
/* ------------------------------------------------------------------ */
double orc_weno5(double a, double b, double c, double d, double e, double eps) {
    double q0 = (2.0 * a - 7.0 * b + 11.0 * c) * (1.0 / 6.0);
    double q1 = (-b + 5.0 * c + 2.0 * d) * (1.0 / 6.0);
    double q2 = (2.0 * c + 5.0 * d - e) * (1.0 / 6.0);
    double t, s;
    t = a - 2.0 * b + c;
    s = a - 4.0 * b + 3.0 * c;
    double b0 = 13.0 / 12.0 * t * t + 0.25 * s * s;
    t = b - 2.0 * c + d;
    s = b - d;
    double b1 = 13.0 / 12.0 * t * t + 0.25 * s * s;
    t = c - 2.0 * d + e;
    s = 3.0 * c - 4.0 * d + e;
    double b2 = 13.0 / 12.0 * t * t + 0.25 * s * s;
    double w0 = 0.1 / ((eps + b0) * (eps + b0));
    double w1 = 0.6 / ((eps + b1) * (eps + b1));
    double w2 = 0.3 / ((eps + b2) * (eps + b2));
    /* candidates 6 + 5 + 5; smoothness 12 + 9 + 12; alphas 3 x 3;
       convex combination 3 mul + 4 add + 1 div */
    FL(16 + 33 + 9 + 8);
    return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

/* ------------------------------------------------------------------ */
/* WENO3 of Jiang & Shu (1996), the paper's third-order option: value at */
/* the right face of the cell holding b from the averages a, b, c.       */
/* Candidates (3b - a)/2 on {a, b} and (b + c)/2 on {b, c}, smoothness   */
/* (b - a)^2 and (c - b)^2, ideal weights (1/3, 2/3),                    */
/* alpha_k = d_k/(eps + beta_k)^2.  The left face of the same cell is   */
/* the same formula with the three averages reversed.                    */
/* ------------------------------------------------------------------ */
double orc_weno3(double a, double b, double c, double eps) {
    double q0 = 0.5 * (3.0 * b - a);
    double q1 = 0.5 * (b + c);
    double b0 = (b - a) * (b - a);
    double b1 = (c - b) * (c - b);
    double w0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
    double w1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
    /* candidates 3 + 2; smoothness 2 x 2; alphas 2 x 3; combination 2 mul + 2 add + 1 div */
    FL(5 + 4 + 6 + 5);
    return (w0 * q0 + w1 * q1) / (w0 + w1);
}

/* Face-state admissibility for the fallback of the positivity reading:
 * alpha2 in [0,1], both partial densities > 0, p + Pi/(Gamma+1) > 0. */
static int admissible(const orc_grid* g, const double* w) {
    if (!(w[6] >= 0.0 && w[6] <= 1.0)) return 0;
    if (!(w[0] > 0.0 && w[1] > 0.0)) return 0;
    double G = mix_gamma(g, w[6]);
    double Pi = mix_pi(g, w[6]);
    FL(3);
    if (!(w[5] + Pi / (G + 1.0) > 0.0)) return 0;
    return 1;
}

int orc_admissible(const orc_grid* g, const double* w) { return admissible(g, w); }

/* Test hook: face sides that fell back to their cell's primitives in this
 * thread since the last reset (one count per inadmissible face state). */
static _Thread_local long orc_fallbacks = 0;
long orc_fallback_count(void) { return orc_fallbacks; }
void orc_fallback_reset(void) { orc_fallbacks = 0; }

/* ------------------------------------------------------------------ */
/* HLLC (Toro et al. 1994) for the five-equation system, direction dir.  */
/* Reading of the alpha2 treatment (Johnsen & Colonius adaptation, not   */
/* printed in the paper): the face velocity u_f is the velocity that     */
/* carries mass through the face in the HLLC flux, and the alpha2 flux   */
/* is alpha2 of the upwind side (by the sign of s*) times u_f.  For      */
/* s* == 0 u_f is the mean of the two one-sided values.                  */
/* Wave speeds (Davis/Einfeldt type): sL = min(uL-cL, uR-cR),            */
/* sR = max(uL+cL, uR+cR).                                               */
/* ------------------------------------------------------------------ */
static void side_state(const orc_grid* g, const double* w, int dir, double* q, double* f,
                       double* rho_o, double* un_o, double* p_o, double* c_o) {
    double rho = w[0] + w[1];
    double un = w[2 + dir];
    double p = w[5];
    double G = mix_gamma(g, w[6]);
    double Pi = mix_pi(g, w[6]);
    double E = G * p + Pi + 0.5 * rho * (w[2] * w[2] + w[3] * w[3] + w[4] * w[4]);
    double c = sqrt(((G + 1.0) * p + Pi) / (G * rho));
    q[0] = w[0];
    q[1] = w[1];
    q[2] = rho * w[2];
    q[3] = rho * w[3];
    q[4] = rho * w[4];
    q[5] = E;
    f[0] = w[0] * un;
    f[1] = w[1] * un;
    f[2] = q[2] * un;
    f[3] = q[3] * un;
    f[4] = q[4] * un;
    f[2 + dir] += p;
    f[5] = (E + p) * un;
    FL(1 + 11 + 7 + 3 + 7 + 2);
    *rho_o = rho;
    *un_o = un;
    *p_o = p;
    *c_o = c;
}

void orc_hllc(const orc_grid* g, const double* wl, const double* wr, int dir, double* F,
              double* uface) {
    double qL[6], qR[6], fL[6], fR[6];
    double rL, uL, pL, cL, rR, uR, pR, cR;
    side_state(g, wl, dir, qL, fL, &rL, &uL, &pL, &cL);
    side_state(g, wr, dir, qR, fR, &rR, &uR, &pR, &cR);
    double sL = fmin(uL - cL, uR - cR);
    double sR = fmax(uL + cL, uR + cR);
    double ss = (pR - pL + rL * uL * (sL - uL) - rR * uR * (sR - uR))
              / (rL * (sL - uL) - rR * (sR - uR));
    FL(4 + 15);

    /* one-sided face velocities u_K + s_K^-/+ (chi_K - 1) */
    double ufL, ufR;
    if (sL >= 0.0) {
        ufL = uL;
    } else {
        double chi = (sL - uL) / (sL - ss);
        ufL = uL + sL * (chi - 1.0);
        FL(6);
    }
    if (sR <= 0.0) {
        ufR = uR;
    } else {
        double chi = (sR - uR) / (sR - ss);
        ufR = uR + sR * (chi - 1.0);
        FL(6);
    }

    if (ss >= 0.0) {
        if (sL >= 0.0) {
            for (int v = 0; v < 6; ++v) F[v] = fL[v];
        } else {
            double chi = (sL - uL) / (sL - ss);
            double qs[6];
            qs[0] = chi * qL[0];
            qs[1] = chi * qL[1];
            qs[2] = chi * rL * wl[2];
            qs[3] = chi * rL * wl[3];
            qs[4] = chi * rL * wl[4];
            qs[2 + dir] = chi * rL * ss;
            qs[5] = chi * (qL[5] + (ss - uL) * (rL * ss + pL / (sL - uL)));
            for (int v = 0; v < 6; ++v) F[v] = fL[v] + sL * (qs[v] - qL[v]);
            FL(3 + 2 + 6 + 9 + 18);
        }
    } else {
        if (sR <= 0.0) {
            for (int v = 0; v < 6; ++v) F[v] = fR[v];
        } else {
            double chi = (sR - uR) / (sR - ss);
            double qs[6];
            qs[0] = chi * qR[0];
            qs[1] = chi * qR[1];
            qs[2] = chi * rR * wr[2];
            qs[3] = chi * rR * wr[3];
            qs[4] = chi * rR * wr[4];
            qs[2 + dir] = chi * rR * ss;
            qs[5] = chi * (qR[5] + (ss - uR) * (rR * ss + pR / (sR - uR)));
            for (int v = 0; v < 6; ++v) F[v] = fR[v] + sR * (qs[v] - qR[v]);
            FL(3 + 2 + 6 + 9 + 18);
        }
    }
    double uf;
    double a2;
    if (ss > 0.0) {
        uf = ufL;
        a2 = wl[6];
    } else if (ss < 0.0) {
        uf = ufR;
        a2 = wr[6];
    } else {
        uf = 0.5 * (ufL + ufR);
        a2 = wl[6];
        FL(2);
    }
    F[6] = a2 * uf;
    FL(1);
    *uface = uf;
}

/* ------------------------------------------------------------------ */
/* Grid helpers                                                         */
/* ------------------------------------------------------------------ */
static long cells(const orc_grid* g) { return (long)g->nx * g->ny * g->nz; }

static int wrap(int i, int n, int bc) {
    if (bc == 1) {
        int r = i % n;
        return r < 0 ? r + n : r;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* ------------------------------------------------------------------ */
/* Characteristic far-field boundary (Sec. 3.1: non-reflecting,          */
/* characteristic boundaries with a penalty towards p_inf, after Poinsot */
/* and Lele 1992), in ghost-cell form.  Along the outward normal n (side */
/* s = +1 at the high face, -1 at the low face) with u_n = s u_axis and  */
/* the acoustic impedance Z = rho c of the interior cell next to the     */
/* face, the outgoing characteristic p + Z u_n is taken from that cell   */
/* and the incoming one p - Z u_n from a blend of that cell (weight      */
/* 1 - kappa) and the far field at rest at p_inf (weight kappa):         */
/*   p_b   = p + kappa/2 (p_inf - p + Z u_n)                             */
/*   u_n,b = u_n + kappa/(2 Z) (p - p_inf - Z u_n).                      */
/* kappa = 0 is the transmissive boundary; kappa = 1 passes a linear     */
/* plane wave leaving along n unchanged (no reflection) and relaxes the  */
/* domain towards p_inf.  Partial densities, alpha2 and the tangential   */
/* velocities are the interior cell's.  Every ghost layer takes this     */
/* state.                                                                */
/* ------------------------------------------------------------------ */
static void char_ghost(const orc_grid* g, const double* wi, int axis, double s, double* wb) {
    for (int v = 0; v < NV; ++v) wb[v] = wi[v];
    const double Z = (wi[0] + wi[1]) * sqrt(sound2(g, wi));
    const double un = s * wi[2 + axis];
    const double k = g->bc_penalty;
    wb[5] = wi[5] + 0.5 * k * (g->p_inf - wi[5] + Z * un);
    wb[2 + axis] = s * (un + 0.5 * k * (wi[5] - g->p_inf - Z * un) / Z);
}

/* ------------------------------------------------------------------ */
/* Right-hand side L(Q) of Eq. (ode):                                    */
/*   rows 1-6: -(1/h) sum_d (F_{+} - F_{-})                              */
/*   row 7:    -(1/h) sum_d (Fa_{+} - Fa_{-}) + (alpha2 + K)(1/h) sum_d  */
/*             (uf_{+} - uf_{-})                                         */
/* with K of Eq. (var_K) from rho_k c_k^2 = g_k (p + pc_k).              */
/* The sum over d runs x, then y, then z.                                */
/* ------------------------------------------------------------------ */
int orc_rhs(const orc_grid* g, const double* Q, double* R) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const int px = nx + 6, py = ny + 6, pz = nz + 6;
    const long n = cells(g);
    const long pn = (long)px * py * pz;
    double* W = (double*)malloc(sizeof(double) * NV * pn);
    double* divu = (double*)calloc((size_t)n, sizeof(double));
    if (!W || !divu) {
        free(W);
        free(divu);
        return -1;
    }
    const double invh = 1.0 / g->h;

    /* primitives of the interior cells */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long c = ((long)k * ny + j) * nx + i;
                double q[NV], w[NV];
                for (int v = 0; v < NV; ++v) q[v] = Q[v * n + c];
                orc_prim_from_cons(g, q, w);
                long pc = ((long)(k + 3) * py + (j + 3)) * px + (i + 3);
                for (int v = 0; v < NV; ++v) W[v * pn + pc] = w[v];
            }
    /* three ghost layers: copies of interior primitives; for bc 2 the     */
    /* ghosts outside along one axis (the only ones a stencil reads) take */
    /* the characteristic state of the interior cell next to the face     */
    for (int k = -3; k < nz + 3; ++k)
        for (int j = -3; j < ny + 3; ++j)
            for (int i = -3; i < nx + 3; ++i) {
                if (k >= 0 && k < nz && j >= 0 && j < ny && i >= 0 && i < nx) continue;
                int ks = wrap(k, nz, g->bc), js = wrap(j, ny, g->bc), is = wrap(i, nx, g->bc);
                long dst = ((long)(k + 3) * py + (j + 3)) * px + (i + 3);
                long src = ((long)(ks + 3) * py + (js + 3)) * px + (is + 3);
                int out_x = i < 0 || i >= nx, out_y = j < 0 || j >= ny, out_z = k < 0 || k >= nz;
                if (g->bc == 2 && out_x + out_y + out_z == 1) {
                    int axis = out_x ? 0 : (out_y ? 1 : 2);
                    int c = out_x ? i : (out_y ? j : k);
                    double wi[NV], wb[NV];
                    for (int v = 0; v < NV; ++v) wi[v] = W[v * pn + src];
                    char_ghost(g, wi, axis, c < 0 ? -1.0 : 1.0, wb);
                    for (int v = 0; v < NV; ++v) W[v * pn + dst] = wb[v];
                } else {
                    for (int v = 0; v < NV; ++v) W[v * pn + dst] = W[v * pn + src];
                }
            }

    for (long c = 0; c < n; ++c)
        for (int v = 0; v < NV; ++v) R[v * n + c] = 0.0;

    const int dims[3] = {nx, ny, nz};
    const long pstride[3] = {1, px, (long)px * py};
    for (int dir = 0; dir < 3; ++dir) {
        const int nd = dims[dir];
        const long st = pstride[dir];
        /* faces f = 0..nd along dir, f between cells f-1 and f */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int idx[3] = {i, j, k};
                    if (idx[dir] != 0) continue; /* walk each line once */
                    double* Fl = (double*)malloc(sizeof(double) * 8 * (nd + 1));
                    for (int f = 0; f <= nd; ++f) {
                        int cl[3] = {i, j, k};
                        cl[dir] = f - 1; /* left cell */
                        long base = ((long)(cl[2] + 3) * py + (cl[1] + 3)) * px + (cl[0] + 3);
                        double wl[NV], wr[NV], wcl[NV], wcr[NV];
                        for (int v = 0; v < NV; ++v) {
                            const double* P = W + v * pn;
                            double m2 = P[base - 2 * st], m1 = P[base - st], c0 = P[base];
                            double p1 = P[base + st], p2 = P[base + 2 * st];
                            if (g->weno_order == 3) {
                                wl[v] = orc_weno3(m1, c0, p1, g->weno_eps);
                                wr[v] = orc_weno3(p2, p1, c0, g->weno_eps);
                            } else {
                                wl[v] = orc_weno5(m2, m1, c0, p1, p2, g->weno_eps);
                                wr[v] = orc_weno5(P[base + 3 * st], p2, p1, c0, m1, g->weno_eps);
                            }
                            wcl[v] = c0;
                            wcr[v] = p1;
                        }
                        if (!admissible(g, wl)) {
                            for (int v = 0; v < NV; ++v) wl[v] = wcl[v];
                            ++orc_fallbacks;
                        }
                        if (!admissible(g, wr)) {
                            for (int v = 0; v < NV; ++v) wr[v] = wcr[v];
                            ++orc_fallbacks;
                        }
                        double F[NV], uf;
                        orc_hllc(g, wl, wr, dir, F, &uf);
                        for (int v = 0; v < NV; ++v) Fl[8 * f + v] = F[v];
                        Fl[8 * f + 7] = uf;
                    }
                    for (int c = 0; c < nd; ++c) {
                        int cc[3] = {i, j, k};
                        cc[dir] = c;
                        long cell = ((long)cc[2] * ny + cc[1]) * nx + cc[0];
                        for (int v = 0; v < NV; ++v)
                            R[v * n + cell] -= (Fl[8 * (c + 1) + v] - Fl[8 * c + v]) * invh;
                        divu[cell] += (Fl[8 * (c + 1) + 7] - Fl[8 * c + 7]) * invh;
                        FL(8 * 3);
                    }
                    free(Fl);
                }
    }

    /* source of the alpha2 row: (alpha2 + K) div u, cell-centred */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long c = ((long)k * ny + j) * nx + i;
                long pc = ((long)(k + 3) * py + (j + 3)) * px + (i + 3);
                double p = W[5 * pn + pc];
                double a2 = clamp01(W[6 * pn + pc]);
                double a1 = 1.0 - a2;
                double z1 = g->gamma1 * (p + g->pc1); /* rho_1 c_1^2 */
                double z2 = g->gamma2 * (p + g->pc2); /* rho_2 c_2^2 */
                double K = a1 * a2 * (z1 - z2) / (a1 * z2 + a2 * z1);
                R[6 * n + c] += (W[6 * pn + pc] + K) * divu[c];
                FL(1 + 4 + 8 + 3);
            }
    free(W);
    free(divu);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Low-storage RK3, Williamson 2N form:                                  */
/*   dQ <- A_s dQ + dt L(Q);  Q <- Q + B_s dQ,  s = 1..3, A_1 = 0.       */
/* Coefficients: the low-storage TVD RK3 of Gottlieb & Shu (1998).       */
/* ------------------------------------------------------------------ */
static const double RK_A[3] = {0.0, -2.915492524638791, -0.000000093517376};
static const double RK_B[3] = {0.924574, 0.287713063186749, 0.626538109512740};

void orc_rk_coefficients(double* A, double* B) {
    for (int s = 0; s < 3; ++s) {
        A[s] = RK_A[s];
        B[s] = RK_B[s];
    }
}

int orc_rk3_step(const orc_grid* g, double* Q, double dt) {
    const long n = cells(g);
    double* dQ = (double*)calloc((size_t)(NV * n), sizeof(double));
    double* R = (double*)malloc(sizeof(double) * NV * n);
    if (!dQ || !R) {
        free(dQ);
        free(R);
        return -1;
    }
    for (int s = 0; s < 3; ++s) {
        if (orc_rhs(g, Q, R) != 0) {
            free(dQ);
            free(R);
            return -1;
        }
        for (long i = 0; i < NV * n; ++i) {
            dQ[i] = RK_A[s] * dQ[i] + dt * R[i];
            Q[i] = Q[i] + RK_B[s] * dQ[i];
        }
        FL((s == 0 ? 4.0 : 5.0) * NV * n); /* stage 1: 0*dQ is not algorithmic */
    }
    free(dQ);
    free(R);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Per-state reductions: max signal speed max_cells max_d(|u_d| + c),    */
/* max pressure and its first index in x-fastest order, health bits.     */
/* ------------------------------------------------------------------ */
enum { ORC_ST_NONFINITE = 1, ORC_ST_NEGATIVE = 2, ORC_ST_MAXSTEPS = 4 };

typedef struct {
    double smax;
    double cmax;   /* max over cells of the mixture sound speed */
    double pmax;
    long argmax;
    int status;
} orc_reduce;

static void reduce_state(const orc_grid* g, const double* Q, orc_reduce* r) {
    const long n = cells(g);
    r->smax = 0.0;
    r->cmax = 0.0;
    r->pmax = -INFINITY;
    r->argmax = 0;
    r->status = 0;
    for (long c = 0; c < n; ++c) {
        double q[NV], w[NV];
        for (int v = 0; v < NV; ++v) q[v] = Q[v * n + c];
        orc_prim_from_cons(g, q, w);
        double c2 = sound2(g, w);
        double rho = w[0] + w[1];
        int bad = 0;
        for (int v = 0; v < NV; ++v)
            if (!isfinite(q[v])) bad |= ORC_ST_NONFINITE;
        if (!isfinite(w[5])) bad |= ORC_ST_NONFINITE;
        if (!(rho > 0.0) || !(c2 > 0.0)) bad |= ORC_ST_NEGATIVE;
        r->status |= bad;
        if (bad) continue;
        double c0 = sqrt(c2);
        double s = fmax(fabs(w[2]) + c0, fmax(fabs(w[3]) + c0, fabs(w[4]) + c0));
        FL(1 + 3 + 1);
        if (s > r->smax) r->smax = s;
        if (c0 > r->cmax) r->cmax = c0;
        if (w[5] > r->pmax) {
            r->pmax = w[5];
            r->argmax = c;
        }
    }
}

double orc_max_speed(const orc_grid* g, const double* Q) {
    orc_reduce r;
    reduce_state(g, Q, &r);
    return r.smax;
}

/* Conserved totals sum_cells Q_v h^3, v = 0..5, Kahan-compensated. */
void orc_totals(const orc_grid* g, const double* Q, double* tot) {
    const long n = cells(g);
    const double vol = g->h * g->h * g->h;
    for (int v = 0; v < 6; ++v) {
        double s = 0.0, comp = 0.0;
        for (long c = 0; c < n; ++c) {
            double y = Q[v * n + c] - comp;
            double t = s + y;
            comp = (t - s) - y;
            s = t;
        }
        tot[v] = s * vol;
    }
}

/* ------------------------------------------------------------------ */
/* Initial condition for a cloud of spheres (reading of the smoothing): */
/*   H(x) = max_b 1/2 (1 - tanh((|x - x_b| - r_b)/h)),                   */
/*   alpha2 = clamp(H, 1e-6, 1 - 1e-6),                                  */
/*   a1r1 = (1 - alpha2) rho1,  a2r2 = alpha2 rho2,                      */
/*   p = p_l(x) + (p_gas - p_l(x)) H,  u = 0,  E = Gamma p + Pi,          */
/* with the liquid pressure p_l = p_liq, or, with the cloud ramp of       */
/* Sec. 3.1 (r0 > 0, distance r from the domain centre): p_l = p_cloud    */
/* for r <= r0 and p_liq + (p_cloud - p_liq) r0 / r beyond (the pressure  */
/* field of a liquid at rest around a sphere, continuous at r0).          */
/* Cell centres x_c = (i + 1/2) h.  bub = nb x (x, y, z, r).             */
/* ------------------------------------------------------------------ */
void orc_init_cloud(const orc_grid* g, const double* bub, int nb, double rho1, double rho2,
                    double p_gas, double p_liq, double p_cloud, double r0, double* Q) {
    const long n = cells(g);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long c = ((long)k * g->ny + j) * g->nx + i;
                double x = (i + 0.5) * g->h, y = (j + 0.5) * g->h, z = (k + 0.5) * g->h;
                double H = 0.0;
                for (int b = 0; b < nb; ++b) {
                    double dx = x - bub[4 * b], dy = y - bub[4 * b + 1], dz = z - bub[4 * b + 2];
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    double hb = 0.5 * (1.0 - tanh((d - bub[4 * b + 3]) / g->h));
                    if (hb > H) H = hb;
                }
                double a2 = H;
                if (a2 < 1e-6) a2 = 1e-6;
                if (a2 > 1.0 - 1e-6) a2 = 1.0 - 1e-6;
                double w[NV], q[NV];
                w[0] = (1.0 - a2) * rho1;
                w[1] = a2 * rho2;
                w[2] = w[3] = w[4] = 0.0;
                double pl = p_liq;
                if (r0 > 0.0) {
                    double cx = x - 0.5 * g->nx * g->h, cy = y - 0.5 * g->ny * g->h, cz = z - 0.5 * g->nz * g->h;
                    double r = sqrt(cx * cx + cy * cy + cz * cz);
                    pl = r <= r0 ? p_cloud : p_liq + (p_cloud - p_liq) * r0 / r;
                }
                w[5] = pl + (p_gas - pl) * H;
                w[6] = a2;
                orc_cons_from_prim(g, w, q);
                for (int v = 0; v < NV; ++v) Q[v * n + c] = q[v];
            }
}

/* ------------------------------------------------------------------ */
/* Sensors, Eq. (sensor): mean pressure over the cells whose centre      */
/* lies within max(r, h) of the sensor centre (reading: the 0.5 mm ball  */
/* is below one cell at every grid used here).                           */
/* ------------------------------------------------------------------ */
static int sensor_cells(const orc_grid* g, const double* s, long* out, int cap) {
    double R = s[3] > g->h ? s[3] : g->h;
    int m = 0;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double dx = (i + 0.5) * g->h - s[0];
                double dy = (j + 0.5) * g->h - s[1];
                double dz = (k + 0.5) * g->h - s[2];
                if (dx * dx + dy * dy + dz * dz <= R * R) {
                    if (m < cap) out[m] = ((long)k * g->ny + j) * g->nx + i;
                    ++m;
                }
            }
    return m;
}

int orc_sensor_cell_count(const orc_grid* g, const double* s) {
    return sensor_cells(g, s, NULL, 0);
}

static double sensor_value(const orc_grid* g, const double* Q, const long* idx, int m) {
    const long n = cells(g);
    double s = 0.0;
    for (int a = 0; a < m; ++a) {
        double q[NV], w[NV];
        for (int v = 0; v < NV; ++v) q[v] = Q[v * n + idx[a]];
        orc_prim_from_cons(g, q, w);
        s += w[5];
    }
    return m > 0 ? s / m : NAN;
}

/* ------------------------------------------------------------------ */
/* One solve to t_end with QoIs (Section 3.2).                           */
/*   dt = CFL h / max speed, clipped to t_end - t (the last step lands    */
/*   exactly on t_end);                                                  */
/*   p_peak = max over t = 0 and every step of max_cells p, first index; */
/*   sensor histories on t_k = k t_end/(K-1), linear in time between     */
/*   steps; sensor peaks = max over steps of the sensor value;           */
/*   c_max = max over t = 0 and every step of max_cells c (Sec. 3.2 maximum */
/*   speed of sound); gas-fraction sensors (Sec. 3.2 alpha sensors): mean   */
/*   alpha2 over the same cells as the pressure sensor, its value at t = 0, */
/*   its minimum over the recorded steps and the first time of that minimum; */
/*   its history on the output times of the pressure sensors (ahist, may be */
/*   NULL), linear in time between steps like theirs.                       */
/* ------------------------------------------------------------------ */
typedef struct {
    double p_peak;
    long peak_index;
    double p_peak_t;
    double sensor_peak[8];
    double totals0[6];
    double totals_end[6];
    int n_steps;
    int status;
    double t_final;
    double c_max;
    double sensor_alpha0[8];
    double sensor_alpha_min[8];
    double sensor_alpha_min_t[8];
} orc_qoi;

static double sensor_alpha(const orc_grid* g, const double* Q, const long* idx, int m) {
    const long n = cells(g);
    double acc = 0.0;
    for (int a = 0; a < m; ++a) acc += Q[6 * n + idx[a]];
    return m > 0 ? acc / m : NAN;
}

int orc_solve(const orc_grid* g, double* Q, double t_end, int max_steps, int n_sensors,
              const double* sensors, int n_out, double* hist, double* ahist, orc_qoi* out) {
    if (n_sensors > 8) return -2;
    long* sidx[8];
    int scount[8];
    for (int s = 0; s < n_sensors; ++s) {
        scount[s] = sensor_cells(g, sensors + 4 * s, NULL, 0);
        sidx[s] = (long*)malloc(sizeof(long) * (scount[s] > 0 ? scount[s] : 1));
        sensor_cells(g, sensors + 4 * s, sidx[s], scount[s]);
    }
    double sv_old[8], sv_new[8], sa_old[8], sa_new[8];
    orc_reduce r;
    reduce_state(g, Q, &r);
    out->status = r.status;
    out->p_peak = r.pmax;
    out->peak_index = r.argmax;
    out->p_peak_t = 0.0;
    orc_totals(g, Q, out->totals0);
    out->c_max = r.cmax;
    for (int s = 0; s < n_sensors; ++s) {
        sv_old[s] = sensor_value(g, Q, sidx[s], scount[s]);
        out->sensor_peak[s] = sv_old[s];
        if (hist && n_out > 0) hist[s * n_out + 0] = sv_old[s];
        out->sensor_alpha0[s] = out->sensor_alpha_min[s] = sa_old[s] = sensor_alpha(g, Q, sidx[s], scount[s]);
        out->sensor_alpha_min_t[s] = 0.0;
        if (ahist && n_out > 0) ahist[s * n_out + 0] = sa_old[s];
    }
    double t = 0.0;
    int nsteps = 0;
    int kout = 1; /* next output time index */
    while (t < t_end && out->status == 0) {
        if (nsteps >= max_steps) {
            out->status |= ORC_ST_MAXSTEPS;
            break;
        }
        double dt = g->cfl * g->h / r.smax;
        int last = 0;
        if (t + dt >= t_end) {
            dt = t_end - t;
            last = 1;
        }
        if (orc_rk3_step(g, Q, dt) != 0) return -1;
        double t_new = last ? t_end : t + dt;
        ++nsteps;
        reduce_state(g, Q, &r);
        out->status |= r.status;
        if (r.pmax > out->p_peak) {
            out->p_peak = r.pmax;
            out->peak_index = r.argmax;
            out->p_peak_t = t_new;
        }
        if (r.cmax > out->c_max) out->c_max = r.cmax;
        for (int s = 0; s < n_sensors; ++s) {
            sv_new[s] = sensor_value(g, Q, sidx[s], scount[s]);
            if (sv_new[s] > out->sensor_peak[s]) out->sensor_peak[s] = sv_new[s];
            double a = sa_new[s] = sensor_alpha(g, Q, sidx[s], scount[s]);
            if (a < out->sensor_alpha_min[s]) {
                out->sensor_alpha_min[s] = a;
                out->sensor_alpha_min_t[s] = t_new;
            }
        }
        if (hist && n_out > 1) {
            while (kout < n_out) {
                double tk = (kout * t_end) / (n_out - 1);
                if (tk > t_new) break;
                double wgt = (tk - t) / (t_new - t);
                for (int s = 0; s < n_sensors; ++s) {
                    hist[s * n_out + kout] = (1.0 - wgt) * sv_old[s] + wgt * sv_new[s];
                    if (ahist) ahist[s * n_out + kout] = (1.0 - wgt) * sa_old[s] + wgt * sa_new[s];
                }
                ++kout;
            }
        }
        for (int s = 0; s < n_sensors; ++s) {
            sv_old[s] = sv_new[s];
            sa_old[s] = sa_new[s];
        }
        t = t_new;
    }
    orc_totals(g, Q, out->totals_end);
    out->n_steps = nsteps;
    out->t_final = t;
    for (int s = 0; s < n_sensors; ++s) free(sidx[s]);
    return 0;
}

/* Plain stepping to t_end without QoIs (used by the Riemann pins). */
int orc_advance(const orc_grid* g, double* Q, double t_end, int max_steps, int* n_steps) {
    double t = 0.0;
    int n = 0;
    while (t < t_end) {
        if (n >= max_steps) return -3;
        double dt = g->cfl * g->h / orc_max_speed(g, Q);
        int last = 0;
        if (t + dt >= t_end) {
            dt = t_end - t;
            last = 1;
        }
        if (orc_rk3_step(g, Q, dt) != 0) return -1;
        t = last ? t_end : t + dt;
        ++n;
    }
    *n_steps = n;
    return 0;
}
