"""Pins of the oracle solver against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
formulas, exact solutions, invariants, or brute force.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import cloud
from oracle import solver as S
from riemann_exact import Side, sample

GAM = (6.12, 1.4)
PC = (34.3, 0.0)


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------- closure (Section 2.1)

@pytest.mark.parametrize("a2,gamma,pc", [(0.0, GAM[0], PC[0]), (1.0, GAM[1], PC[1])])
def test_pure_phase_limit_is_stiffened_gas(a2, gamma, pc):
    """alpha2 = 0 / 1: p = (g - 1) rho e - g pc with rho e = E - rho|u|^2/2."""
    g = S.make_grid(4, gamma=GAM, pc_nd=PC)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u = rng.normal(size=3) * 0.3
        rhoe = rng.uniform(1.0, 50.0) + gamma * pc / (gamma - 1)
        E = rhoe + 0.5 * rho * u @ u
        q = np.array([rho * (1 - a2), rho * a2, *(rho * u), E, a2]).reshape(7, 1)
        w = S.cons_to_prim(g, q).ravel()
        p_text = (gamma - 1.0) * rhoe - gamma * pc
        assert abs(w[5] - p_text) <= 1e-12 * abs(rhoe * gamma)
        assert np.allclose(w[2:5], u, rtol=1e-14, atol=1e-15)


def test_prim_cons_round_trip():
    g = S.make_grid(8, gamma=GAM, pc_nd=PC)
    Wp = W.smooth_periodic_primitives(8, seed=3).reshape(7, -1)
    Q = S.prim_to_cons(g, Wp)
    assert rel(S.cons_to_prim(g, Q), Wp) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_max_speed_uniform_state_is_textbook(axis):
    """Uniform pure-liquid state: max speed = max|u_d| + sqrt(g (p + pc)/rho),
    with the largest velocity component along each axis in turn."""
    n = 4
    g = S.make_grid(n, gamma=GAM, pc_nd=PC)
    Wp = np.zeros((7, n ** 3))
    Wp[0] = 1.0
    Wp[1] = 0.0
    vel = [0.1, 0.2, -0.15]
    vel[axis] = -0.7
    Wp[2], Wp[3], Wp[4] = vel
    Wp[5] = 1.0
    Q = S.prim_to_cons(g, Wp)
    c = math.sqrt(GAM[0] * (1.0 + PC[0]) / 1.0)
    assert abs(S.max_speed(g, Q) - (0.7 + c)) < 1e-12 * c


# ---------------------------------------------------------------- WENO5 (Jiang & Shu)

def test_weno5_exact_on_quadratics():
    """Cell averages of a quadratic give exact face values for any nonlinear weights."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        a, b, c = rng.normal(size=3) * np.array([1.0, 3.0, 10.0])
        avg = lambda i: a + b * i + c * (i * i + 1.0 / 12.0)   # average over [i-1/2, i+1/2]
        exact_r = a + b * 0.5 + c * 0.25                        # f(+1/2)
        exact_l = a - b * 0.5 + c * 0.25                        # f(-1/2)
        v = [avg(i) for i in (-2, -1, 0, 1, 2)]
        scale = abs(a) + abs(b) + abs(c)
        assert abs(S.weno5(*v) - exact_r) < 1e-12 * scale
        assert abs(S.weno5(*v[::-1]) - exact_l) < 1e-12 * scale


def test_weno5_fifth_order_on_smooth_data():
    def err(n):
        h = 1.0 / n
        x = (np.arange(-2, n + 3) + 0.5) * h
        avg = (np.cos(2 * np.pi * (x - 0.5 * h)) - np.cos(2 * np.pi * (x + 0.5 * h))) / (2 * np.pi * h)
        e = 0.0
        for i in range(2, n + 2):
            val = S.weno5(*avg[i - 2:i + 3], eps=1e-40)
            e = max(e, abs(val - np.sin(2 * np.pi * (x[i] + 0.5 * h))))
        return e
    e1, e2 = err(40), err(80)
    assert math.log2(e1 / e2) > 4.5


# ---------------------------------------------------------------- WENO3 (Jiang & Shu, the third-order option)

def test_weno3_exact_on_linear_data():
    """Both candidates reproduce a linear function: any weights give the exact face value."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        a, b = rng.normal(size=2) * np.array([1.0, 5.0])
        v = [a + b * i for i in (-1, 0, 1)]     # averages of a + b x over unit cells
        assert abs(S.weno3(*v) - (a + 0.5 * b)) < 1e-13 * (abs(a) + abs(b))
        assert abs(S.weno3(*v[::-1]) - (a - 0.5 * b)) < 1e-13 * (abs(a) + abs(b))


def test_weno3_ideal_weights_are_third_order_linear_scheme():
    """Symmetric data (equal smoothness of both sub-stencils) gives the ideal weights
    1/3, 2/3, whose combination is exact for the averages of a parabola."""
    for c in (1.0, -2.5, 7.0):
        avg = [c * (i * i + 1.0 / 12.0) for i in (-1, 0, 1)]   # averages of c x^2
        assert abs(S.weno3(*avg) - c * 0.25) < 1e-14 * abs(c)


def test_weno3_third_order_on_smooth_monotone_data():
    def err(n):
        h = 0.5 / n
        x = (np.arange(-1, n + 2) + 0.5) * h
        avg = (np.exp(x + 0.5 * h) - np.exp(x - 0.5 * h)) / h
        return max(abs(S.weno3(*avg[i - 1:i + 2]) - math.exp(x[i] + 0.5 * h)) for i in range(1, n + 1))
    e1, e2 = err(40), err(80)
    assert math.log2(e1 / e2) > 2.6


def test_weno3_takes_the_smooth_side_of_a_step():
    for lo, hi in ((0.0, 1.0), (2.0, -3.0)):
        v = S.weno3(lo, lo, hi)        # step to the right of the cell: the left stencil
        assert abs(v - lo) < 1e-6 * abs(hi - lo)
        v = S.weno3(lo, hi, hi)        # step to the left: the right stencil
        assert abs(v - hi) < 1e-6 * abs(hi - lo)


def test_weno3_solver_keeps_p_and_u_uniform_across_an_interface_and_conserves():
    """The WENO3 option in the solver: the interface invariant and periodic
    conservation hold as for WENO5, and the result differs from WENO5."""
    n = 16
    g = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=1, weno_order=3)
    g5 = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=1)
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    d = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    a2 = np.clip(0.5 * (1 - np.tanh((d - 0.3) * n)), 1e-6, 1 - 1e-6)
    Wp = np.zeros((7, n, n, n))
    Wp[0] = (1 - a2) * 1.0
    Wp[1] = a2 * 0.005
    Wp[2], Wp[3], Wp[4] = 0.5, -0.25, 0.125
    Wp[5] = 1.0
    Wp[6] = a2
    Q = S.prim_to_cons(g, Wp.reshape(7, -1)).reshape(7, n, n, n)
    dt = 0.3 * g.h / S.max_speed(g, Q)
    Q3, Q5 = Q, Q
    for _ in range(6):
        Q3 = S.rk3_step(g, Q3, dt)
        Q5 = S.rk3_step(g5, Q5, dt)
    Wn = S.cons_to_prim(g, Q3.reshape(7, -1))
    assert np.max(np.abs(Wn[5] - 1.0)) < 1e-12
    assert np.max(np.abs(Wn[2] - 0.5)) < 1e-12
    scale = np.array([1.0, 0.005, 1.0, 1.0, 1.0, 40.0])
    assert np.all(np.abs(S.totals(g, Q3) - S.totals(g, Q)) <= 1e-13 * scale)
    assert np.max(np.abs(Q3[6] - Q5[6])) > 1e-4


# ---------------------------------------------------------------- HLLC

def _flux_text(w, d, gamma, pc):
    """Physical flux of the five-equation system from textbook formulas."""
    a2 = w[6]
    rho = w[0] + w[1]
    G = (1 - a2) / (gamma[0] - 1) + a2 / (gamma[1] - 1)
    Pi = (1 - a2) * gamma[0] * pc[0] / (gamma[0] - 1) + a2 * gamma[1] * pc[1] / (gamma[1] - 1)
    u = np.array(w[2:5])
    p = w[5]
    E = G * p + Pi + 0.5 * rho * u @ u
    un = u[d]
    F = np.array([w[0] * un, w[1] * un, rho * u[0] * un, rho * u[1] * un, rho * u[2] * un,
                  (E + p) * un, a2 * un])
    F[2 + d] += p
    return F


def _random_state(rng, a2=None):
    a2 = rng.uniform(0.01, 0.99) if a2 is None else a2
    return np.array([(1 - a2) * rng.uniform(0.8, 1.2), a2 * rng.uniform(0.004, 0.006),
                     *rng.normal(size=3) * 0.5, rng.uniform(0.5, 2.0), a2])


def test_hllc_consistency():
    g = S.make_grid(4, gamma=GAM, pc_nd=PC)
    rng = np.random.default_rng(11)
    for _ in range(30):
        w = _random_state(rng)
        for d in range(3):
            F, uf = S.hllc(g, w, w, d)
            Ft = _flux_text(w, d, GAM, PC)
            assert np.allclose(F, Ft, rtol=1e-12, atol=1e-12 * np.max(np.abs(Ft)))
            assert abs(uf - w[2 + d]) < 1e-12


def test_hllc_isolated_contact_is_exact():
    """Equal p and u, different composition: flux is the upwind physical flux."""
    g = S.make_grid(4, gamma=GAM, pc_nd=PC)
    rng = np.random.default_rng(12)
    for un in (0.3, -0.4, 0.0):
        wl = _random_state(rng, 0.1)
        wr = _random_state(rng, 0.9)
        wl[2:5] = wr[2:5] = [un, 0.1, -0.2]
        wl[5] = wr[5] = 1.3
        F, uf = S.hllc(g, wl, wr, 0)
        up = wl if un >= 0 else wr
        Ft = _flux_text(up, 0, GAM, PC)
        assert np.allclose(F[:6], Ft[:6], rtol=1e-12, atol=1e-12)
        assert abs(uf - un) < 1e-13
        assert abs(F[6] - up[6] * un) < 1e-13


def test_hllc_mirror_symmetry():
    g = S.make_grid(4, gamma=GAM, pc_nd=PC)
    rng = np.random.default_rng(13)
    for _ in range(30):
        wl, wr = _random_state(rng), _random_state(rng)
        F, uf = S.hllc(g, wl, wr, 1)
        ml, mr = wr.copy(), wl.copy()
        ml[3] *= -1
        mr[3] *= -1
        Fm, ufm = S.hllc(g, ml, mr, 1)
        sign = np.ones(7)
        sign[[0, 1, 2, 4, 5, 6]] = -1.0   # mass, tangential momenta, energy, alpha2 flip
        sign[3] = 1.0                      # normal momentum flux is even
        assert np.allclose(Fm, sign * F, rtol=1e-11, atol=1e-12)
        assert abs(ufm + uf) < 1e-12


def test_hllc_face_between_a_state_and_its_mirror_image():
    """Left and right states that are mirror images across the face (normal
    velocity reversed), colliding and separating: by symmetry nothing crosses
    the face but momentum, the face velocity is zero and the normal momentum
    flux is the HLLC star pressure p* = p + rho u (u - s_L) with s* = 0 and
    s_L = -|u| - c (Toro).  With s* = 0 the face velocity is the mean of the
    two one-sided ones, which are exact opposites here, so it is exactly 0."""
    g = S.make_grid(4, gamma=GAM, pc_nd=PC)
    rng = np.random.default_rng(14)
    for _ in range(20):
        w = _random_state(rng)
        for d in range(3):
            for sgn in (1.0, -1.0):      # towards the face from both sides / away from it
                wl = w.copy()
                wl[2 + d] = sgn * (abs(w[2 + d]) + 0.05)
                wr = wl.copy()
                wr[2 + d] = -wl[2 + d]
                F, uf = S.hllc(g, wl, wr, d)
                assert uf == 0.0 and F[6] == 0.0
                a2, rho, u, p = wl[6], wl[0] + wl[1], wl[2 + d], wl[5]
                G = (1 - a2) / (GAM[0] - 1) + a2 / (GAM[1] - 1)
                Pi = (1 - a2) * GAM[0] * PC[0] / (GAM[0] - 1) + a2 * GAM[1] * PC[1] / (GAM[1] - 1)
                c = math.sqrt(((G + 1) * p + Pi) / (G * rho))
                # the vanishing fluxes cancel terms of the size of the one-sided flux and
                # of s_L times the conserved state: bound them by rounding on that scale
                qv = S.prim_to_cons(g, wl.reshape(7, 1)).ravel()
                size = np.abs(_flux_text(wl, d, GAM, PC)) + (abs(u) + c) * np.abs(qv)
                others = [v for v in range(6) if v != 2 + d]
                assert np.all(np.abs(F[others]) <= 1e-14 * size[others]), (F, d, sgn)
                p_star = p + rho * u * (u + abs(u) + c)
                assert abs(F[2 + d] - p_star) <= 1e-13 * (abs(p) + rho * abs(u) * (2 * abs(u) + c))
                assert (F[2 + d] > p) == (sgn > 0)    # compression when colliding


@pytest.mark.parametrize("order", [5, 3])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_rhs_commutes_with_reflections_and_axis_swaps(order, bc):
    """The right-hand side of a random smooth state is equivariant under the
    symmetries of the grid: reflecting the state along an axis (with that
    velocity component reversed) reflects its right-hand side the same way,
    and swapping two axes (with their velocity components) swaps it.  A
    stencil taken in the wrong orientation, a face state from the wrong side,
    or a direction index mixed up breaks one of these."""
    n = 8
    g = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=bc, weno_order=order, bc_penalty=0.7, p_inf=1.1)
    Wp = W.smooth_periodic_primitives(n, seed=21, amp=0.3)
    Q = S.prim_to_cons(g, Wp.reshape(7, -1)).reshape(7, n, n, n)
    R = S.rhs(g, Q).reshape(7, n, n, n)
    scale = np.max(np.abs(R), axis=(1, 2, 3), keepdims=True)
    assert np.all(scale > 1e-3)
    for ax in range(3):                  # grid axis ax is array axis 3 - ax (x fastest)
        sl = [slice(None)] * 4
        sl[3 - ax] = slice(None, None, -1)
        M = Q[tuple(sl)].copy()
        M[2 + ax] *= -1
        want = R[tuple(sl)].copy()
        want[2 + ax] *= -1
        got = S.rhs(g, M).reshape(7, n, n, n)
        assert np.all(np.abs(got - want) <= 1e-12 * scale), (ax, np.max(np.abs(got - want) / scale))
    for a, b in ((0, 1), (1, 2), (0, 2)):
        T = np.swapaxes(Q, 3 - a, 3 - b).copy()
        T[[2 + a, 2 + b]] = T[[2 + b, 2 + a]]
        want = np.swapaxes(R, 3 - a, 3 - b).copy()
        want[[2 + a, 2 + b]] = want[[2 + b, 2 + a]]
        got = S.rhs(g, T).reshape(7, n, n, n)
        assert np.all(np.abs(got - want) <= 1e-12 * scale), ((a, b), np.max(np.abs(got - want) / scale))


# ---------------------------------------------------------------- positivity fallback (reading of Sec. 2.2)

def test_face_admissibility_clauses_and_their_directions():
    """Each clause of the face-state test on its own, on both sides of its
    threshold.  The pressure clause is the positivity of the frozen squared
    sound speed; in the pure-phase limits that is the textbook stiffened-gas
    condition p + p_c > 0 (liquid) and p > 0 (ideal gas)."""
    g = S.make_grid(4, gamma=GAM, pc_nd=PC)
    base = np.array([0.5, 0.0025, 0.1, -0.2, 0.3, 1.0, 0.5])
    assert S.admissible(g, base)

    def with_(i, v, w=base):
        w = w.copy()
        w[i] = v
        return w
    # alpha2 in [0, 1], both ends included
    assert S.admissible(g, with_(6, 0.0)) and S.admissible(g, with_(6, 1.0))
    assert not S.admissible(g, with_(6, -1e-9)) and not S.admissible(g, with_(6, 1.0 + 1e-9))
    # partial densities strictly positive
    for i in (0, 1):
        assert S.admissible(g, with_(i, 1e-12))
        assert not S.admissible(g, with_(i, 0.0)) and not S.admissible(g, with_(i, -1e-9))
    # liquid (alpha2 = 0): p + p_c > 0
    liq = with_(6, 0.0)
    assert S.admissible(g, with_(5, -PC[0] * (1.0 - 1e-9), liq))
    assert not S.admissible(g, with_(5, -PC[0] * (1.0 + 1e-9), liq))
    assert S.admissible(g, with_(5, -0.5 * PC[0], liq))            # tension below p_c is fine
    # gas (alpha2 = 1): p > 0
    gas = with_(6, 1.0)
    assert S.admissible(g, with_(5, 1e-9, gas))
    assert not S.admissible(g, with_(5, 0.0, gas)) and not S.admissible(g, with_(5, -1e-9, gas))
    # velocities never matter
    assert S.admissible(g, np.array([0.5, 0.0025, -40.0, 25.0, 1e3, 1.0, 0.5]))


def _bump_state(nx):
    """1D primitives: a sharp two-cell alpha2 bump (1e-6 outside, 1 - 1e-6 inside)
    on smooth partial densities, velocities and pressure."""
    x = (np.arange(nx) + 0.5) / nx
    two_pi = 2.0 * math.pi
    Wp = np.zeros((7, nx))
    Wp[0] = 1.0 + 0.1 * np.sin(two_pi * x)
    Wp[1] = 0.005 * (1.0 + 0.1 * np.cos(two_pi * x))
    Wp[2] = 0.05 * np.sin(two_pi * x)
    Wp[3] = 0.02 * np.cos(two_pi * x)
    Wp[4] = -0.01 * np.sin(2.0 * two_pi * x)
    Wp[5] = 1.0 + 0.1 * np.cos(two_pi * x)
    Wp[6] = 1e-6
    Wp[6, nx // 2 - 1:nx // 2 + 1] = 1.0 - 1e-6
    return Wp


def _x_rhs_composed(g, Wp, fallback_all=True):
    """Rows 0-6 of the right-hand side of a 1D state along x, composed face by
    face from the pinned WENO5 and HLLC routines and this test's own face
    test (alpha2 in [0, 1], partial densities > 0, p > 0; p + Pi/(Gamma+1) > 0
    follows from p > 0 since Pi >= 0).  An inadmissible face state takes its
    cell's primitives: all seven (fallback_all) or only alpha2.  Returns the
    rows and the number of face states that fell back."""
    nx = Wp.shape[1]
    h = g.h
    cl = lambda i: min(max(i, 0), nx - 1)                     # transmissive ghosts
    P = lambda v, i: Wp[v, cl(i)]

    def ok(w):
        return 0.0 <= w[6] <= 1.0 and w[0] > 0.0 and w[1] > 0.0 and w[5] > 0.0
    F = np.zeros((nx + 1, 7))
    uf = np.zeros(nx + 1)
    n_fb = 0
    for f in range(nx + 1):
        wl = np.array([S.weno5(P(v, f - 3), P(v, f - 2), P(v, f - 1), P(v, f), P(v, f + 1)) for v in range(7)])
        wr = np.array([S.weno5(P(v, f + 2), P(v, f + 1), P(v, f), P(v, f - 1), P(v, f - 2)) for v in range(7)])
        assert min(wl[5], wr[5]) > 0.5                          # the pressure clause is never marginal here
        for w, c in ((wl, f - 1), (wr, f)):
            if not ok(w):
                n_fb += 1
                if fallback_all:
                    w[:] = Wp[:, cl(c)]
                else:
                    w[6] = Wp[6, cl(c)]
        F[f], uf[f] = S.hllc(g, wl, wr, 0)
    R = -(F[1:] - F[:-1]).T * (1.0 / h)
    # alpha2 row: + (alpha2 + K) div u with K of Eq. (var_K), rho_k c_k^2 = g_k (p + pc_k)
    a2 = np.clip(Wp[6], 0.0, 1.0)
    z1, z2 = GAM[0] * (Wp[5] + PC[0]), GAM[1] * (Wp[5] + PC[1])
    K = (1 - a2) * a2 * (z1 - z2) / ((1 - a2) * z2 + a2 * z1)
    R[6] += (Wp[6] + K) * (uf[1:] - uf[:-1]) * (1.0 / h)
    return R, n_fb


def test_rhs_falls_back_to_the_cell_state_for_all_seven_primitives():
    """WENO5 overshoots alpha2 above 1 at the faces inside a sharp two-cell
    bump (the other variables are smooth, so only the alpha2 clause fails).
    The oracle's right-hand side must equal the one composed with every
    primitive of such a face state replaced by its cell's, fall back at
    exactly the same face states, and differ clearly from replacing alpha2
    alone (so the comparison can tell the two apart)."""
    nx = 16
    g = S.make_grid(nx, 1, 1, gamma=GAM, pc_nd=PC)
    Wp = _bump_state(nx)
    Q = S.prim_to_cons(g, Wp)
    S.fallback_reset()
    R = S.rhs(g, Q).reshape(7, nx)
    n_oracle = S.fallback_count()
    Rc, n_fb = _x_rhs_composed(g, Wp)
    assert n_fb > 0 and n_oracle == n_fb
    scale = np.max(np.abs(Rc), axis=1, keepdims=True)
    assert np.all(np.abs(R - Rc) <= 1e-12 * scale)
    Ralpha, _ = _x_rhs_composed(g, Wp, fallback_all=False)
    assert np.max(np.abs(Ralpha - Rc) / scale) > 1e-4


def test_smooth_state_needs_no_fallback():
    g = S.make_grid(8, gamma=GAM, pc_nd=PC, bc=1)
    Q = S.prim_to_cons(g, W.smooth_periodic_primitives(8, seed=5).reshape(7, -1))
    S.fallback_reset()
    S.rhs(g, Q)
    assert S.fallback_count() == 0


# ---------------------------------------------------------------- low-storage RK3

def _butcher():
    A, B = S.rk_coefficients()
    a21 = B[0]
    a31, a32 = B[0] + B[1] * A[1], B[1]
    b = np.array([B[0] + B[1] * A[1] + B[2] * A[2] * A[1], B[1] + B[2] * A[2], B[2]])
    c = np.array([0.0, a21, a31 + a32])
    return A, B, b, c, a32


def test_rk3_order_conditions():
    A, B, b, c, a32 = _butcher()
    assert A[0] == 0.0
    assert abs(b.sum() - 1) < 1e-8
    assert abs(b @ c - 0.5) < 1e-8
    assert abs(b @ (c * c) - 1.0 / 3.0) < 1e-8
    assert abs(b[2] * a32 * c[1] - 1.0 / 6.0) < 1e-8


def test_rk3_linear_amplification():
    A, B = S.rk_coefficients()
    for z in (-0.3, 0.1 + 0.5j, -1.0 + 1.0j):
        y, dy = 1.0, 0.0
        for s in range(3):
            dy = A[s] * dy + z * y
            y = y + B[s] * dy
        assert abs(y - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-8


# ---------------------------------------------------------------- full scheme

def _riemann_run(nx, left, right, gam, pc, t_end, x0=0.5, eps=1e-8):
    g = S.make_grid(nx, 1, 1, gamma=gam, pc_nd=pc, bc=0, h=1.0 / nx)
    x = (np.arange(nx) + 0.5) / nx
    L = x < x0
    Wp = np.zeros((7, nx))
    a2 = np.where(L, eps, 1 - eps)
    Wp[0] = np.where(L, (1 - a2) * left[0], (1 - a2) * left[0])
    Wp[1] = np.where(L, a2 * right[0], a2 * right[0])
    Wp[2] = np.where(L, left[1], right[1])
    Wp[5] = np.where(L, left[2], right[2])
    Wp[6] = a2
    Q = S.prim_to_cons(g, Wp)
    Q, n = S.advance(g, Q.reshape(7, 1, 1, nx), t_end)
    Wn = S.cons_to_prim(g, Q.reshape(7, -1))
    er, eu, ep, _ = sample(Side(*left, gam[0], pc[0]), Side(*right, gam[1], pc[1]), (x - x0) / t_end)
    rho = Wn[0] + Wn[1]
    return (np.mean(np.abs(rho - er)) / np.mean(er), np.mean(np.abs(Wn[5] - ep)) / np.mean(np.abs(ep)),
            np.mean(np.abs(Wn[2] - eu)) / max(np.mean(np.abs(eu)), 1e-300))


def test_riemann_sod_single_gas_converges():
    """Ideal gas on both sides (both phases gamma 1.4, pc 0): Sod's problem."""
    e100 = _riemann_run(100, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (1.4, 1.4), (0.0, 0.0), 0.2)
    e200 = _riemann_run(200, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (1.4, 1.4), (0.0, 0.0), 0.2)
    for a, b in zip(e100, e200):
        assert b < 0.65 * a
    assert max(e200) < 0.025


def test_riemann_water_air_converges():
    """Water at 1e9 Pa against air at 1e5 Pa (ratio 1e4), densities 1000 / 50 kg/m^3."""
    args = ((1.0, 0.0, 100.0), (0.05, 0.0, 0.01), GAM, PC, 0.008)
    e100 = _riemann_run(100, *args)
    e200 = _riemann_run(200, *args)
    for a, b in zip(e100, e200):
        assert b < 0.75 * a
    assert e200[0] < 0.02 and e200[1] < 0.03 and e200[2] < 0.15


def test_mixture_expansion_follows_phase_isentropes():
    """Pins K of Eq. (var_K): in smooth flow each phase of the Kapila model is
    isentropic, rho_k = rho_k0 ((p + pc_k)/(p0 + pc_k))^(1/g_k).  Without the
    K div(u) source the gas density would follow the mixture density instead
    (a few per cent off for this expansion)."""
    nx = 200
    g = S.make_grid(nx, 1, 1, gamma=GAM, pc_nd=PC, bc=0, h=1.0 / nx)
    x = (np.arange(nx) + 0.5) / nx
    a2, r1, r2, p0 = 0.3, 1.0, 0.005, 1.0
    Wp = np.zeros((7, nx))
    Wp[0], Wp[1], Wp[5], Wp[6] = (1 - a2) * r1, a2 * r2, p0, a2
    Wp[2] = np.where(x < 0.5, -0.02, 0.02)
    Q, _ = S.advance(g, S.prim_to_cons(g, Wp).reshape(7, 1, 1, nx), 0.1)
    Wn = S.cons_to_prim(g, Q.reshape(7, -1))
    p, a = Wn[5], Wn[6]
    assert p.min() < 0.97 * p0       # a real expansion happened
    rho2 = Wn[1] / a
    rho1 = Wn[0] / (1 - a)
    iso2 = r2 * ((p + PC[1]) / (p0 + PC[1])) ** (1 / GAM[1])
    iso1 = r1 * ((p + PC[0]) / (p0 + PC[0])) ** (1 / GAM[0])
    assert np.max(np.abs(rho2 / iso2 - 1)) < 1e-3
    assert np.max(np.abs(rho1 / iso1 - 1)) < 1e-4


def test_interface_advection_keeps_p_and_u_uniform():
    """Uniform p and u with an alpha2 / density step stays at uniform p and u.

    The step carries the initial condition's one-cell tanh smoothing; a bare
    step on a bubble only ~5 cells wide drives WENO5 into overshoots that make
    the liquid partial density negative (a known limit of the scheme).
    """
    n = 16
    g = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=1)
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    d = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    a2 = np.clip(0.5 * (1 - np.tanh((d - 0.3) * n)), 1e-6, 1 - 1e-6)
    Wp = np.zeros((7, n, n, n))
    Wp[0] = (1 - a2) * 1.0
    Wp[1] = a2 * 0.005
    Wp[2], Wp[3], Wp[4] = 0.5, -0.25, 0.125
    Wp[5] = 1.0
    Wp[6] = a2
    Q = S.prim_to_cons(g, Wp.reshape(7, -1)).reshape(7, n, n, n)
    dt = 0.3 * g.h / S.max_speed(g, Q)
    for _ in range(10):
        Q = S.rk3_step(g, Q, dt)
    Wn = S.cons_to_prim(g, Q.reshape(7, -1))
    assert np.max(np.abs(Wn[5] - 1.0)) < 1e-12
    assert np.max(np.abs(Wn[2] - 0.5)) < 1e-12
    assert np.max(np.abs(Wn[3] + 0.25)) < 1e-12
    assert np.max(np.abs(Wn[4] - 0.125)) < 1e-12
    assert np.max(np.abs(Wn[6] - a2.ravel())) > 1e-3   # the interface did move


def test_conservation_on_periodic_box():
    n = 8
    g = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=1)
    Q = S.prim_to_cons(g, W.smooth_periodic_primitives(n, seed=5).reshape(7, -1)).reshape(7, n, n, n)
    t0 = S.totals(g, Q)
    dt = 0.3 * g.h / S.max_speed(g, Q)
    for _ in range(4):
        Q = S.rk3_step(g, Q, dt)
    t1 = S.totals(g, Q)
    scale = np.array([1.0, 0.005, 1.0, 1.0, 1.0, 40.0])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)
    assert np.max(np.abs(S.rhs(g, Q)[:6])) > 1e-3   # the fields are not static


def test_centred_bubble_keeps_cube_symmetry():
    n = 12
    sp = W.SolverParams()
    b = np.array([[0.05, 0.05, 0.05, 0.02]])
    Q = S.init_cloud(sp, n, b)
    g = S.grid_from_params(sp, n)
    dt = 0.3 * g.h / S.max_speed(g, Q)
    for _ in range(3):
        Q = S.rk3_step(g, Q, dt)
    # transpose x <-> y swaps the x and y momenta
    T = Q.transpose(0, 1, 3, 2).copy()
    T[[2, 3]] = T[[3, 2]]
    assert rel(T, Q) < 1e-12
    # mirror x -> -x flips the x momentum
    M = Q[:, :, :, ::-1].copy()
    M[2] *= -1
    assert np.max(np.abs(M - Q)) < 1e-12 * np.max(np.abs(Q))
    assert np.max(np.abs(Q[2])) > 1e-6


# ---------------------------------------------------------------- reductions and QoIs

def test_reductions_brute_force():
    n = 6
    g = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=1)
    Wp = W.smooth_periodic_primitives(n, seed=9, amp=0.3).reshape(7, -1)
    Q = S.prim_to_cons(g, Wp)
    a2 = Wp[6]
    G = (1 - a2) / (GAM[0] - 1) + a2 / (GAM[1] - 1)
    Pi = (1 - a2) * GAM[0] * PC[0] / (GAM[0] - 1) + a2 * GAM[1] * PC[1] / (GAM[1] - 1)
    c = np.sqrt(((G + 1) * Wp[5] + Pi) / (G * (Wp[0] + Wp[1])))
    smax = np.max(np.maximum(np.maximum(np.abs(Wp[2]), np.abs(Wp[3])), np.abs(Wp[4])) + c)
    assert abs(S.max_speed(g, Q) - smax) < 1e-12 * smax
    vol = (1.0 / n) ** 3
    assert np.allclose(S.totals(g, Q), Q[:6].sum(axis=1) * vol, rtol=1e-13)


def test_centre_sensor_has_eight_cells_on_even_grids():
    for n in (16, 32, 64):
        g = S.make_grid(n)
        s = np.array([0.5, 0.5, 0.5, 0.005])
        assert S._lib().orc_sensor_cell_count(g, S._p(s)) == 8


def test_solve_time_loop_and_qois():
    w = W.tiny(16, 4)
    b = cloud.sample_cloud(w.cloud, W.BASE_SEED, 3)
    q, hist, Q = S.solve(w.solver, 16, b)
    assert q["status"] == 0
    assert q["t_final"] == w.solver.t_end
    g = S.grid_from_params(w.solver, 16)
    # the peak is at least the final max pressure, and the history ends at the final sensor value
    Wn = S.cons_to_prim(g, Q.reshape(7, -1))
    assert q["p_peak"] >= Wn[5].max() * w.solver.p_liq * (1 - 1e-15)
    k = q["peak_index"]
    assert q["p_peak_xyz"][0] == ((k % 16) + 0.5) / 16 * w.solver.domain_L
    centre = Wn[5].reshape(16, 16, 16)[7:9, 7:9, 7:9].mean() * w.solver.p_liq
    assert abs(hist[0, -1] - centre) < 1e-9 * centre
    # number of steps ~ t_end / dt at CFL 0.3 (the IC at rest has c = 1469.8 m/s in water)
    assert 25 <= q["n_steps"] <= 40


def test_sound_speed_and_gas_fraction_sensor_qois():
    """Liquid at rest (no bubbles): the state stays uniform, so c_max is the
    textbook stiffened-gas sound speed sqrt(gamma (p + p_c) / rho) of the
    liquid (the 1e-6 gas fraction moves it by < 1e-5) and the gas-fraction
    sensors read 1e-6 throughout, with the minimum at t = 0.  One centred
    bubble at 10 MPa: its gas is compressed, so the gas fraction of a sensor
    ball around it falls, its minimum coming later than t = 0."""
    sp = W.SolverParams(sensors=((0.05, 0.05, 0.05, 0.02), W.centre_sensor()[0]))
    q, _, _ = S.solve(sp, 16, np.zeros((0, 4)))
    c_text = math.sqrt(sp.gamma[0] * (sp.p_liq + sp.pc[0]) / sp.rho0[0])
    assert abs(q["c_max"] / c_text - 1) < 1e-5
    assert np.allclose(q["sensor_alpha0"], 1e-6, rtol=1e-9)
    assert np.allclose(q["sensor_alpha_min"], 1e-6, rtol=1e-9)
    assert np.all(q["sensor_alpha_min_t"] == 0.0)
    assert np.allclose(q["alpha_hist"], 1e-6, rtol=1e-9)
    q, _, _ = S.solve(sp, 16, np.array([[0.05, 0.05, 0.05, 0.015]]))
    assert q["status"] == 0
    assert q["sensor_alpha0"][0] > 0.1 and q["sensor_alpha_min"][0] < q["sensor_alpha0"][0]
    assert 0.0 < q["sensor_alpha_min_t"][0] <= q["t_final"]
    assert q["c_max"] >= c_text * (1 - 1e-5)
    # the history starts at the t = 0 value and, interpolating between step values, never
    # goes below their minimum
    ah = q["alpha_hist"]
    assert ah[0, 0] == q["sensor_alpha0"][0] and ah.shape == (2, sp.n_out_times)
    assert np.all(ah[0] >= q["sensor_alpha_min"][0] * (1 - 1e-15)) and ah[0].min() < ah[0, 0]


# ---------------------------------------------------------------- initial condition and sampler

def test_initial_condition_far_and_inside():
    sp = W.SolverParams()
    n = 16
    b = np.array([[0.05, 0.05, 0.05, 0.03]])
    Q = S.init_cloud(sp, n, b)
    g = S.grid_from_params(sp, n)
    Wn = S.cons_to_prim(g, Q.reshape(7, -1)).reshape(7, n, n, n)
    # corner cell: liquid (alpha2 clamped at 1e-6), p = p_liq + (p_gas - p_liq) H
    Hc = 0.5 * (1 - math.tanh((math.sqrt(3) * (0.5 - 0.5 / n) - 0.3) * n))
    assert abs(Wn[6, 0, 0, 0] - 1e-6) < 1e-18
    assert abs(Wn[5, 0, 0, 0] - (1.0 + (2.34e3 / 1e7 - 1.0) * Hc)) < 1e-12
    assert abs(Wn[0, 0, 0, 0] - (1 - 1e-6)) < 1e-15
    # centre cells: gas at p_gas (H = 1/2 (1 - tanh(-r/h)) ~ 1)
    H = 0.5 * (1 - math.tanh((math.sqrt(3) * 0.5 / n - 0.3) * n))
    assert abs(Wn[5, 8, 8, 8] - (1.0 + (2.34e3 / 1e7 - 1.0) * H)) < 1e-12
    assert np.all(Wn[2:5] == 0.0)


def test_sampler_distributions():
    cp = W.cloud_uniform(200)
    b = cloud.sample_cloud(cp, W.BASE_SEED, 0)
    c = 0.5 * cp.domain_L
    r = np.sqrt(((b[:, :3] - c) ** 2).sum(1))
    assert np.all(r <= cp.cloud_radius * (1 + 1e-15))
    assert np.all((b[:, 3] >= cp.r_min) & (b[:, 3] <= cp.r_max))
    # uniform in a ball: E[(r/R)^3] = 1/2
    assert abs(np.mean((r / cp.cloud_radius) ** 3) - 0.5) < 0.07
    lp = W.cloud_paper500()
    b5 = cloud.sample_cloud(lp, 1, 2)
    assert b5.shape == (500, 4)
    assert np.all((b5[:, 3] >= 0.8e-3) & (b5[:, 3] <= 1.2e-3))
    # same (seed, id) -> same cloud; another id -> another cloud
    assert np.array_equal(cloud.sample_cloud(cp, 5, 7), cloud.sample_cloud(cp, 5, 7))
    assert not np.array_equal(cloud.sample_cloud(cp, 5, 7), cloud.sample_cloud(cp, 5, 8))


def test_splitmix64_reference_values():
    """SplitMix64 from seed 0 (Steele, Lea & Flood): first outputs of the published generator."""
    g = cloud.SplitMix64(0, 0)
    assert g.next_u64() == 0xE220A8397B1DCDAF
    assert g.next_u64() == 0x6E789E6AA1B965F4
    assert g.next_u64() == 0x06C45D188009454F


def test_cloud_pressure_ramp_is_harmonic_and_continuous():
    """Sec. 3.1 ramp (no bubbles, so the field is the liquid's alone): the
    cloud pressure inside r0, continuity across r0, a harmonic field beyond it
    (a liquid at rest around a sphere: the 7-point Laplacian is a small
    fraction of the size |b| h^2 / r^3 of the second differences of b/r, which
    a linear or 1/r^2 profile would not give), rising monotonically towards
    p_inf."""
    sp = W.solver_paper500()
    N = 64
    g = S.grid_from_params(sp, N)
    Q = S.init_cloud(sp, N, np.zeros((0, 4)))
    p = S.cons_to_prim(g, Q.reshape(7, -1))[5].reshape(N, N, N) * sp.p_liq     # Pa
    h = sp.domain_L / N
    x = (np.arange(N) + 0.5) * h - 0.5 * sp.domain_L
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    r0 = sp.ramp_radius
    inside = r <= r0
    assert np.allclose(p[inside], sp.p_cloud, rtol=1e-12, atol=0)
    # continuity: cells within half a cell of r0 differ from p_cloud by at most one cell's rise
    rise = (sp.p_liq - sp.p_cloud) * h / r0        # |dp/dr| at r0 times h
    near = np.abs(r - r0) < 0.5 * h
    assert near.any() and np.max(np.abs(p[near] - sp.p_cloud)) <= rise
    # harmonic beyond r0 (all 7 stencil cells in the ramp region)
    core = (slice(1, -1),) * 3
    d2 = [p[2:, 1:-1, 1:-1] - 2 * p[core] + p[:-2, 1:-1, 1:-1],
          p[1:-1, 2:, 1:-1] - 2 * p[core] + p[1:-1, :-2, 1:-1],
          p[1:-1, 1:-1, 2:] - 2 * p[core] + p[1:-1, 1:-1, :-2]]
    lap = d2[0] + d2[1] + d2[2]
    b = abs(sp.p_cloud - sp.p_liq) * r0
    ramp = r[core] > r0 + 2 * h
    scale = b * h * h / r[core] ** 3
    assert np.all(np.abs(lap[ramp]) <= 0.05 * scale[ramp])
    assert np.max(np.abs(d2[0][ramp]) / scale[ramp]) > 0.5     # the scale is the size of the terms
    # monotone rise with r, below p_inf
    order = np.argsort(r[core][ramp])
    pr = p[core][ramp][order]
    assert np.all(np.diff(pr) >= -1e-9 * sp.p_liq) and pr[-1] < sp.p_liq and pr[0] > sp.p_cloud
    # off by default: the uniform liquid pressure
    q0 = S.init_cloud(W.SolverParams(), N, np.zeros((0, 4)))
    p0 = S.cons_to_prim(g, q0.reshape(7, -1))[5]
    assert np.allclose(p0, 1.0, rtol=1e-13)


# ---------------------------------------------------------------- characteristic far-field boundary (Sec. 3.1)

C_LIQ = math.sqrt(GAM[0] * (1.0 + PC[0]))   # liquid sound speed at p = 1, rho = 1 (impedance Z = rho c)


def _liquid(n, p, bc, kappa=1.0, rho=None, u=None):
    g = S.make_grid(n, gamma=GAM, pc_nd=PC, bc=bc, bc_penalty=kappa)
    Wp = np.zeros((7, n, n, n))
    Wp[0] = 1.0 if rho is None else rho
    Wp[5] = p
    if u is not None:
        Wp[2] = u
    return g, S.prim_to_cons(g, Wp.reshape(7, -1)).reshape(7, n, n, n), Wp


def _prim(g, Q):
    n = g.nx
    return S.cons_to_prim(g, Q.reshape(7, -1)).reshape(7, n, n, n)


def test_characteristic_boundary_with_zero_penalty_is_transmissive():
    sp = W.tiny(16, 4).solver
    bub = cloud.sample_cloud(W.tiny(16, 4).cloud, W.BASE_SEED, 3)
    Q0 = S.init_cloud(sp, 16, bub)
    g0 = S.grid_from_params(sp, 16)
    g2 = S.grid_from_params(sp, 16)
    g2.bc, g2.bc_penalty = 2, 0.0
    a, b = Q0, Q0
    dt = 0.3 * g0.h / S.max_speed(g0, Q0)
    for _ in range(2):
        a = S.rk3_step(g0, a, dt)
        b = S.rk3_step(g2, b, dt)
    assert np.array_equal(a, b)


def test_characteristic_boundary_keeps_the_far_field_at_rest():
    g, Q, _ = _liquid(8, 1.0, 2)
    dt = 0.3 * g.h / S.max_speed(g, Q)
    Q1 = Q
    for _ in range(3):
        Q1 = S.rk3_step(g, Q1, dt)
    assert np.array_equal(Q1, Q)


@pytest.mark.parametrize("rho", [1.0, 2.0])
def test_characteristic_boundary_admits_the_far_field_wave_of_linear_acoustics(rho):
    """Liquid at rest at p0 = p_inf - d: each face admits the wave of the
    acoustic Riemann problem against the far field, p0 + d/2 moving inwards
    at d/(2 Z) with the impedance Z = rho c, and the incoming characteristic
    at the face carries p_inf.  At t = L/(4c) the face centres are still
    reached by their own face's wave only.  (At rho = 2 the impedance differs
    from the sound speed, so a boundary that used c for Z would admit a
    wave of the wrong amplitude.)"""
    n, d = 32, 0.01
    p0 = 1.0 - d
    g, Q, _ = _liquid(n, p0, 2, rho=rho)
    c = math.sqrt(GAM[0] * (p0 + PC[0]) / rho)
    Z = rho * c
    Qt, _ = S.advance(g, Q, 0.25 / c)
    Wn = _prim(g, Qt)
    p, u = Wn[5][16, 16, :], Wn[2][16, 16, :]
    for i, sgn in ((0, 1.0), (n - 1, -1.0)):      # low face: wave moves +x; high face: -x
        assert abs((p[i] - p0) / d - 0.5) < 0.03, (i, p[i])
        assert abs(u[i] * sgn * 2.0 * Z / d - 1.0) < 0.03, (i, u[i])
        # incoming characteristic p - Z u_n (u_n outward = -sgn u) equals the far field
        assert abs(p[i] + sgn * Z * u[i] - 1.0) < 0.01 * d
    # the middle of the domain has not been reached by a wave front
    assert abs(p[n // 2] - p0) < 0.05 * d and abs(u[n // 2]) < 0.05 * d / Z


def test_characteristic_boundary_relaxes_the_domain_to_the_far_field_pressure():
    """The penalty term drives the pressure to p_inf (the transmissive
    boundary keeps the initial state for ever)."""
    n, d = 16, 0.01
    for bc, want in ((2, 0.01), (0, None)):
        g, Q, _ = _liquid(n, 1.0 - d, bc)
        Qt, _ = S.advance(g, Q, 3.0 / C_LIQ)
        pm = np.mean(np.abs(_prim(g, Qt)[5] - 1.0)) / d
        if want is None:
            assert abs(pm - 1.0) < 1e-12
        else:
            assert pm < want


def test_characteristic_boundary_lets_an_acoustic_pulse_leave():
    """A Gaussian pressure pulse next to the x = L face: once the direct
    waves have left (t = 1.2 L/c) little acoustic energy is reflected back,
    less than with the transmissive boundary."""
    n, d = 24, 0.01
    x = (np.arange(n) + 0.5) / n
    Zc, Yc, Xc = np.meshgrid(x, x, x, indexing="ij")
    gs = np.exp(-0.5 * (np.sqrt((Xc - 0.85) ** 2 + (Yc - 0.5) ** 2 + (Zc - 0.5) ** 2) / 0.05) ** 2)

    def energy(Wp):
        return np.sum(0.5 * (Wp[5] - 1.0) ** 2 / C_LIQ ** 2 + 0.5 * (Wp[2] ** 2 + Wp[3] ** 2 + Wp[4] ** 2))

    left = {}
    for bc in (2, 0):
        g, _, Wp = _liquid(n, 1.0 + d * gs, bc, rho=1.0 + d * gs / C_LIQ ** 2)
        Q = S.prim_to_cons(g, Wp.reshape(7, -1)).reshape(7, n, n, n)
        Qt, _ = S.advance(g, Q, 1.2 / C_LIQ)
        left[bc] = energy(_prim(g, Qt)) / energy(Wp)
    assert left[2] < 1e-3
    assert left[2] < 0.5 * left[0]


def _qoi_bookkeeping(sp, n, b, Q0=None):
    """Solve with the oracle and check its QoI bookkeeping against a time loop
    written here (CFL steps of the oracle's RK3, the last one clipped to
    t_end): sensor means taken with numpy over the cells whose centre lies
    within max(r, h), their histories by numpy's linear interpolation onto
    t_k = k t_end/(K - 1), the peak pressure with its first (x-fastest) cell
    and first time, the maximum sound speed from the textbook closure, the
    sensor peaks, and the gas-fraction minima with their first times.
    Returns the QoIs and the loop's step values."""
    q, hist, _ = S.solve(sp, n, b, Q0=Q0)
    g = S.grid_from_params(sp, n)
    u = S.Units(sp.domain_L, sp.p_liq)
    t_end = sp.t_end / u.t_ref
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    masks = []
    for sx, sy, sz, r in sp.sensors:
        R = max(r / sp.domain_L, 1.0 / n)
        d2 = (X - sx / sp.domain_L) ** 2 + (Y - sy / sp.domain_L) ** 2 + (Z - sz / sp.domain_L) ** 2
        masks.append(d2 <= R * R)
    gam = sp.gamma
    pc = (sp.pc[0] / u.p_ref, sp.pc[1] / u.p_ref)

    def sensors(Q):
        Wp = S.cons_to_prim(g, Q.reshape(7, -1)).reshape(7, n, n, n)
        a2 = np.clip(Wp[6], 0.0, 1.0)
        G = (1 - a2) / (gam[0] - 1) + a2 / (gam[1] - 1)
        Pi = (1 - a2) * gam[0] * pc[0] / (gam[0] - 1) + a2 * gam[1] * pc[1] / (gam[1] - 1)
        c = np.sqrt(((G + 1) * Wp[5] + Pi) / (G * (Wp[0] + Wp[1])))
        return [Wp[5][m].mean() for m in masks], [Wp[6][m].mean() for m in masks], Wp[5].ravel(), c.max()

    Q = S.init_cloud(sp, n, b) if Q0 is None else Q0
    t, times = 0.0, [0.0]
    p0, a0, pf, cm = sensors(Q)
    ps, als, cms = [p0], [a0], [cm]
    peak, peak_i, peak_t = pf.max(), int(np.argmax(pf)), 0.0     # first maximum, x fastest
    while t < t_end:
        dt = sp.cfl * g.h / S.max_speed(g, Q)
        last = t + dt >= t_end
        if last:
            dt = t_end - t
        Q = S.rk3_step(g, Q, dt)
        t = t_end if last else t + dt
        times.append(t)
        p, a, pf, cm = sensors(Q)
        ps.append(p)
        als.append(a)
        cms.append(cm)
        if pf.max() > peak:                                        # a later equal value keeps the first
            peak, peak_i, peak_t = pf.max(), int(np.argmax(pf)), t
    assert len(times) - 1 == q["n_steps"]
    assert abs(q["p_peak"] - peak * sp.p_liq) <= 1e-12 * q["p_peak"]
    assert q["peak_index"] == peak_i and abs(q["p_peak_t"] - peak_t * u.t_ref) <= 1e-12 * u.t_ref
    assert abs(q["c_max"] - max(cms) * u.u_ref) <= 1e-12 * q["c_max"]
    ps_a, als_a = np.array(ps), np.array(als)
    assert np.allclose(q["sensor_peak"], ps_a.max(axis=0) * sp.p_liq, rtol=1e-12, atol=0)
    assert np.allclose(q["sensor_alpha_min"], als_a.min(axis=0), rtol=1e-12, atol=0)
    first_min = [times[int(np.argmin(als_a[:, s]))] * u.t_ref for s in range(len(sp.sensors))]
    assert np.allclose(q["sensor_alpha_min_t"], first_min, rtol=1e-12, atol=0)
    tk = np.arange(sp.n_out_times) * t_end / (sp.n_out_times - 1)
    for s in range(len(sp.sensors)):
        want_p = np.interp(tk, times, ps_a[:, s]) * sp.p_liq
        want_a = np.interp(tk, times, als_a[:, s])
        assert np.allclose(hist[s], want_p, rtol=1e-12, atol=0)
        assert np.allclose(q["alpha_hist"][s], want_a, rtol=1e-12, atol=0)
    return q, np.array(times) * u.t_ref, ps_a, np.array(cms)


def test_sensor_histories_are_the_step_values_interpolated_onto_the_output_times():
    """The QoI bookkeeping of a cloud solve (4 bubbles on 16^3, two sensors)."""
    sp = W.SolverParams(sensors=(W.centre_sensor()[0], (0.03, 0.05, 0.06, 0.012)), n_out_times=17)
    b = cloud.sample_cloud(W.cloud_uniform(4), W.BASE_SEED, 2)
    _qoi_bookkeeping(sp, 16, b)


def test_qoi_maxima_reached_after_the_initial_state_are_recorded():
    """A converging flow of liquid at uniform pressure: the compression raises
    the pressure, the sound speed and the centre sensor's reading after t = 0,
    so the peak pressure, its time, the maximum sound speed and the sensor
    peak all come from later steps, and are checked against the time loop."""
    sp = W.SolverParams(sensors=W.centre_sensor(), n_out_times=9)
    n = 16
    g = S.grid_from_params(sp, n)
    x = (np.arange(n) + 0.5) / n - 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    env = 0.05 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 0.04)
    a2 = 1e-6
    Wp = np.zeros((7, n, n, n))
    Wp[0] = (1 - a2) * 1.0
    Wp[1] = a2 * sp.rho0[1] / 1000.0
    Wp[2], Wp[3], Wp[4] = -X * env / 0.2, -Y * env / 0.2, -Z * env / 0.2
    Wp[5] = 1.0
    Wp[6] = a2
    Q0 = S.prim_to_cons(g, Wp.reshape(7, -1)).reshape(7, n, n, n)
    q, times, ps, cms = _qoi_bookkeeping(sp, n, np.zeros((0, 4)), Q0=Q0)
    assert q["status"] == 0
    assert q["p_peak"] > 1.05 * sp.p_liq and q["p_peak_t"] > 0.0
    assert q["c_max"] > cms[0] * 1.0001 * S.Units(sp.domain_L, sp.p_liq).u_ref
    assert q["sensor_peak"][0] > 1.05 * ps[0, 0] * sp.p_liq


def test_uniform_state_keeps_the_first_cell_and_the_first_time_of_its_peak():
    """Every cell of a uniform liquid at rest ties for the maximum pressure at
    every step: the peak is the first cell in x-fastest order at t = 0."""
    sp = W.SolverParams(sensors=W.centre_sensor())
    n = 8
    g = S.grid_from_params(sp, n)
    Wp = np.zeros((7, n ** 3))
    Wp[0], Wp[1], Wp[5], Wp[6] = 1.0 - 1e-6, 1e-6 * sp.rho0[1] / 1000.0, 1.0, 1e-6
    Q0 = S.prim_to_cons(g, Wp).reshape(7, n, n, n)
    q, _, Qt = S.solve(sp, n, np.zeros((0, 4)), Q0=Q0)
    assert np.array_equal(Qt, Q0)
    assert q["peak_index"] == 0 and q["p_peak_t"] == 0.0
    assert abs(q["p_peak"] / sp.p_liq - 1.0) < 1e-12   # the primitive -> conserved round trip


def test_sensor_ball_holds_the_cells_within_and_on_its_radius():
    """A sensor centred on a cell centre of a 16^3 grid (h = 1/16, so the
    offsets and radii below are exact binary fractions) holds the cells whose
    integer offset (i, j, k) has i^2 + j^2 + k^2 <= (R/h)^2, R = max(r, h),
    the boundary included: counted here by brute force."""
    n = 16
    g = S.make_grid(n)
    h = 1.0 / n
    for r_over_h, R_over_h in ((0.5, 1), (1.0, 1), (1.5, 1.5), (2.0, 2), (3.0, 3)):
        s = np.array([8.5 * h, 8.5 * h, 5.5 * h, r_over_h * h])
        m = int(math.floor(R_over_h))
        want = sum(1 for i in range(-m, m + 1) for j in range(-m, m + 1) for k in range(-m, m + 1)
                   if i * i + j * j + k * k <= R_over_h * R_over_h)
        assert S._lib().orc_sensor_cell_count(g, S._p(s)) == want, r_over_h
