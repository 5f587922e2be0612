"""The allocation-free entry point ofm_solve_level_static against ofm_solve_level.

ofm_solve_level_static serves callers that cannot allocate device memory (a
framework's caching allocator owns the device, or cudaMalloc would stall a
latency-critical loop): its scratch is a fixed file-scope device array.  It
runs the same kernels as ofm_solve_level, so its QoIs must agree with it to
the FP64 QoI tolerance of the parity tests, on two calls in a row (the second
call reuses the array the first one left behind).  This file is collected
last; it must pass alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04374_gb300 import api  # noqa: E402
from paper_1705_04374_gb300 import native as nv  # noqa: E402

TOL = 1e-9   # the FP64 QoI tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _solve(fn_static: bool, solver, w, N, ids):
    sp = w.solver
    n = len(ids)
    ids_c = (C.c_uint64 * n)(*ids)
    out = (nv.ofm_qoi * n)()
    hist = np.zeros((n, len(sp.sensors), sp.n_out_times))
    hp = hist.ctypes.data_as(C.POINTER(C.c_double))
    cp = api.cloud_params(w.cloud)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = nv.lib()
    if fn_static:
        rc = L.ofm_solve_level_static(solver.h, C.byref(cp), N, n, ids_c, W.BASE_SEED, out, hp, stream)
    else:
        rc = L.ofm_solve_level(solver.h, C.byref(cp), N, n, ids_c, W.BASE_SEED, out, hp, None, 0, stream)
    assert rc == nv.OFM_OK, L.ofm_last_error()
    return out, hist


def _close(a, b):
    return abs(a - b) <= TOL * max(abs(b), 1e-300)


def _same_qoi(a, b, n_sens):
    """Every field of the two QoI records: integers equal, values within TOL
    (sensor fields over the configured sensors)."""
    for name, ctype in nv.ofm_qoi._fields_:
        x, y = getattr(a, name), getattr(b, name)
        if ctype in (C.c_int, C.c_int64):
            assert x == y, name
        elif ctype is C.c_double:
            assert _close(x, y), (name, x, y)
        else:   # fixed-size double arrays
            k = n_sens if name.startswith("sensor_") else len(y)
            assert all(_close(u, v) for u, v in zip(x[:k], y[:k])), (name, list(x[:k]), list(y[:k]))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_entry_point_matches_allocating_one_twice(precision):
    """Eight sensors (centre, +-R/2 on each axis, 0.45 L along x) on 16^3, so
    every field of the record is exercised."""
    w = W.with_solver(W.tiny(16, 4), sensors=W.eight_sensors(0.3 * W.DOMAIN_L))
    solver = api.Solver(w.solver, precision)
    ids = [3, 4, 5]
    ref, ref_hist = _solve(False, solver, w, 16, ids)
    for _ in range(2):
        got, got_hist = _solve(True, solver, w, 16, ids)
        for a, b in zip(got, ref):
            assert a.status == 0 and b.status == 0
            _same_qoi(a, b, len(w.solver.sensors))
        assert np.all(np.abs(got_hist - ref_hist) <= TOL * np.abs(ref_hist))


def test_static_entry_point_rejects_oversized_requests():
    w = W.cfg2("fp32")
    solver = api.Solver(w.solver, "fp32")
    n = 64   # three FP32 state buffers of 7 x 64^3 cells each per cloud: ~1.4 GB
    ids = (C.c_uint64 * n)(*range(n))
    out = (nv.ofm_qoi * n)()
    cp = api.cloud_params(w.cloud)
    rc = nv.lib().ofm_solve_level_static(solver.h, C.byref(cp), 64, n, ids, W.BASE_SEED, out, None,
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == nv.OFM_ENOMEM
    msg = nv.lib().ofm_last_error().decode()
    assert "static array holds" in msg
    need = int(msg.split(" need ")[1].split(" bytes")[0])
    states = n * 3 * 7 * 64 ** 3 * 4
    assert states <= need <= 1.01 * states
