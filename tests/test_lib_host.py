"""CPU tests of the C-ABI library: loads, exports the header's symbols, and its
host-side parts (sampler, estimator, validation) agree with the oracle.
No device work is requested here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import cloud as ocloud
from oracle import estimator as E
from paper_1705_04374_gb300 import api
from paper_1705_04374_gb300 import native as nv

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ofmlmc.h")


def header_functions():
    text = open(HEADER).read()
    return re.findall(r"^\s*(?:const char\*|int|void)\s+(ofm_\w+)\s*\(", text, re.M)


def test_library_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 18
    L = nv.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(nv.SIGNATURES), "binding and header list different functions"


def test_struct_sizes_match_header_layout():
    assert C.sizeof(nv.ofm_bubble) == 32
    assert C.sizeof(nv.ofm_qoi) == 8 * (1 + 3 + 1 + 1 + 1 + 8 + 6 + 6 + 1) + 8 + 8 * (1 + 8 + 8 + 8)
    assert C.sizeof(nv.ofm_estimate_out) == 8 * (4 * 16 + 2)


@pytest.mark.parametrize("cp", [W.cloud_uniform(4), W.cloud_uniform(50), W.cloud_paper500()],
                         ids=["uniform4", "uniform50", "paper500"])
def test_sampler_bitwise_identical_to_oracle(cp):
    for sid in (0, 1, 17, 2 ** 40 + 3):
        a = api.sample_cloud(cp, W.BASE_SEED, sid)
        b = ocloud.sample_cloud(cp, W.BASE_SEED, sid)
        assert a.shape == b.shape
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_estimator_matches_oracle():
    for L, M in ((1, [40, 7]), (3, [300, 50, 9, 3])):
        pairs = W.toy_levels(M, L, 0.4, 0.7, seed=11)
        Wc = [1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, L + 1)]
        a = api.estimate(pairs, Wc)
        b = E.estimate(pairs, Wc)
        for k in ("alpha", "sigma2", "cov", "sigma_tilde2"):
            assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-14), k
        assert abs(a["mean"] - b["mean"]) < 1e-12 * max(1, abs(b["mean"]))
        assert abs(a["eps2"] - b["eps2"]) < 1e-12 * b["eps2"]


def test_fitted_estimator_matches_oracle():
    """ofm_estimate_fitted / ofm_fit_level_variances against the oracle,
    with several pairs on every level and with one pair on the finest."""
    for L, M in ((2, [60, 20, 6]), (3, [300, 50, 9, 3]), (3, [300, 50, 9, 1])):
        pairs = W.toy_levels(M, L, 0.4, 0.7, seed=12)
        Wc = [1.0] + [16.0 ** l + 16.0 ** (l - 1) for l in range(1, L + 1)]
        a = api.estimate(pairs, Wc, fit=True)
        b = E.estimate_fitted(pairs, Wc)
        for k in ("alpha", "sigma2", "cov", "sigma_tilde2"):
            assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-14), (M, k)
        assert np.allclose(a["V_fit"][1:], b["V_fit"][1:], rtol=1e-12, atol=0)
        assert abs(a["mean"] - b["mean"]) < 1e-12 * max(1, abs(b["mean"]))
        assert abs(a["eps2"] - b["eps2"]) < 1e-12 * b["eps2"]
        V = E.diff_variances(pairs)
        fa, fb, vf = api.fit_level_variances(V, M)
        oa, ob, ovf = E.fit_diff_variances(V, M)
        assert abs(fa - oa) < 1e-12 * max(1, abs(oa)) and abs(fb - ob) < 1e-12 * max(1, abs(ob))
        assert np.allclose(vf[1:], ovf[1:], rtol=1e-12, atol=0)
    # fewer than two usable difference levels, or a level-0 with one sample
    with pytest.raises(nv.OfmError):
        api.estimate(W.toy_levels([20, 20, 1], 2, 0.4, 0.7, seed=1), [1.0, 17.0, 272.0], fit=True)
    with pytest.raises(nv.OfmError):
        api.estimate(W.toy_levels([1, 20, 20], 2, 0.4, 0.7, seed=1), [1.0, 17.0, 272.0], fit=True)
    with pytest.raises(nv.OfmError):
        api.fit_level_variances([0.0, 0.3, -1.0], [0, 5, 5])
    # few pairs: the clamped fit agrees with the oracle where the clamp acts
    Wc = [4096.0, 69632.0, 397312.0, 1380352.0]
    for seed in (6, 26, 95):
        pairs = W.toy_levels([43, 5, 2, 1], 3, 0.4, 0.7, seed=seed)
        a = api.estimate(pairs, Wc, fit=True)
        b = E.estimate_fitted(pairs, Wc)
        for k in ("alpha", "cov", "sigma_tilde2", "V_fit"):
            assert np.allclose(a[k][1:], b[k][1:], rtol=1e-11, atol=1e-13), (seed, k)
        assert np.all(a["sigma_tilde2"] >= 0.0)


def test_fitted_summary_estimator_matches_oracle_on_the_union():
    """ofm_estimate_moments_fitted on per-part summaries merged pairwise equals
    the oracle's fitted estimator on all pairs (one finest pair included)."""
    Wc = [1.0, 17.0, 272.0, 4352.0]
    for M in ([300, 50, 9, 3], [300, 50, 9, 1]):
        pairs = W.toy_levels(M, 3, 0.4, 0.7, seed=31)
        moms = []
        for p in pairs:
            cut = p.shape[0] // 2
            a, b = api.level_moments(p[:cut]), api.level_moments(p[cut:])
            moms.append(api.merge_moments(a, b))
        got = api.estimate_moments(moms, Wc, fit=True)
        ref = E.estimate_fitted(pairs, Wc)
        for k in ("alpha", "sigma2", "cov", "sigma_tilde2"):
            assert np.allclose(got[k], ref[k], rtol=1e-10, atol=1e-13), (M, k)
        assert np.allclose(got["V_fit"][1:], ref["V_fit"][1:], rtol=1e-10, atol=0)
        assert abs(got["mean"] - ref["mean"]) < 1e-10 * max(1.0, abs(ref["mean"]))
        assert abs(got["eps2"] - ref["eps2"]) < 1e-10 * ref["eps2"]


def test_run_configuration_is_validated_before_any_device_work():
    """ofm_run refuses bad configurations on the host (no stream or device is touched)."""
    L = nv.lib()
    s = api.Solver(W.SolverParams(sensors=W.centre_sensor()), "fp32")
    cp = api.cloud_params(W.cloud_uniform(4))
    res = nv.ofm_run_result()

    def run(**kw):
        cfg = nv.ofm_run_config()
        base = dict(L=2, mode=nv.OFM_MODE_TOL, target=1.0, qoi=0, seed=1, max_iterations=1, min_samples=2)
        base.update(kw)
        levels = base.pop("N", [8, 16, 24])
        for k, v in base.items():
            setattr(cfg, k, v)
        for i, n in enumerate(levels):
            cfg.N[i] = n
        return L.ofm_run(s.h, C.byref(cp), C.byref(cfg), None, None, 0, C.byref(res), None)

    assert run(L=1, N=[8, 16], fit_variances=1) == nv.OFM_EINVAL      # the fit needs two difference levels
    assert b"variance fit" in L.ofm_last_error()
    assert run(N=[16, 8, 24]) == nv.OFM_EINVAL                          # levels must refine
    assert run(target=0.0) == nv.OFM_EINVAL
    assert run(qoi=5) == nv.OFM_EINVAL                                  # one sensor configured
    assert run(max_iterations=0) == nv.OFM_EINVAL


def test_optimal_samples_rejects_invalid_variances_and_overflow():
    for st2 in ([1.0, -0.1], [1.0, float("nan")]):
        with pytest.raises(nv.OfmError):
            api.optimal_samples(st2, [1.0, 17.0], 0.1, "tol")
    with pytest.raises(nv.OfmError):
        api.optimal_samples([1.0, 0.5], [1.0, 17.0], 1e-12, "tol")


def test_optimal_and_warmup_samples_match_oracle():
    st2 = [1.0, 0.2, 0.04, 0.01]
    Wc = [1.0, 17.0, 272.0, 4352.0]
    for tau in (0.05, 0.01, 0.003):
        assert list(api.optimal_samples(st2, Wc, tau, "tol")) == list(E.optimal_M(st2, Wc, tau, "tol"))
    for B in (1e4, 3e6):
        assert list(api.optimal_samples(st2, Wc, B, "budget")) == list(E.optimal_M(st2, Wc, B, "budget"))
    done = [200000, 10, 1, 1]
    assert list(api.optimal_samples(st2, Wc, 0.01, "tol", done)) == \
        list(E.optimal_M_keep(st2, Wc, done, 0.01, "tol"))
    assert list(api.warmup_samples([16.0 ** l for l in range(4)])) == [512, 64, 8, 1]
    assert list(api.warmup_samples(Wc)) == list(E.warmup_M(Wc))


def test_invalid_arguments_are_rejected_on_the_host():
    L = nv.lib()
    cfg = api.solver_config(W.SolverParams(), "fp64")
    cfg.cfl = -1.0
    h = C.c_void_p()
    assert L.ofm_solver_create(C.byref(h), C.byref(cfg)) == nv.OFM_EINVAL
    assert b"non-physical" in L.ofm_last_error()
    cfg = api.solver_config(W.SolverParams(), "fp64")
    cfg.ramp_radius, cfg.p_cloud = 0.02, 0.0          # a ramp needs a cloud pressure
    assert L.ofm_solver_create(C.byref(h), C.byref(cfg)) == nv.OFM_EINVAL
    for bc, kappa in ((3, 1.0), (nv.OFM_BC_CHARACTERISTIC, 1.5), (nv.OFM_BC_CHARACTERISTIC, -0.1)):
        cfg = api.solver_config(W.SolverParams(bc=bc, bc_penalty=kappa), "fp64")
        assert L.ofm_solver_create(C.byref(h), C.byref(cfg)) == nv.OFM_EINVAL, (bc, kappa)
    cfg = api.solver_config(W.SolverParams(weno_order=4), "fp64")
    assert L.ofm_solver_create(C.byref(h), C.byref(cfg)) == nv.OFM_EINVAL
    cfg = api.solver_config(W.SolverParams(bc=nv.OFM_BC_CHARACTERISTIC, bc_penalty=0.25), "fp64")
    assert L.ofm_solver_create(C.byref(h), C.byref(cfg)) == nv.OFM_OK
    L.ofm_solver_destroy(h)
    # estimator needs two samples per level
    with pytest.raises(nv.OfmError):
        api.estimate([np.zeros((1, 2)), np.zeros((5, 2))], [1.0, 2.0])
    # grid sizes must be multiples of the tile edge
    s = api.Solver(W.SolverParams(), "fp32")
    g = api.make_group(W.SolverParams(), 20, [0], 1)
    cp = api.cloud_params(W.cloud_uniform(2))
    garr = (nv.ofm_group * 1)(g.c)
    n = C.c_size_t()
    assert L.ofm_batch_workspace_bytes(s.h, C.byref(cp), garr, 1, C.byref(n)) == nv.OFM_EINVAL


def test_workspace_size_accounts_for_three_state_buffers():
    sp = W.SolverParams()
    L = nv.lib()
    for prec, es in (("fp64", 8), ("fp32", 4)):
        s = api.Solver(sp, prec)
        g = api.make_group(sp, 64, list(range(3)), 1)
        cp = api.cloud_params(W.cloud_uniform(20))
        garr = (nv.ofm_group * 1)(g.c)
        n = C.c_size_t()
        nv.check(L.ofm_batch_workspace_bytes(s.h, C.byref(cp), garr, 1, C.byref(n)), "ws")
        state = 3 * 3 * 7 * 64 ** 3 * es
        assert state <= n.value < state * 1.05


def test_workspace_holds_both_sensor_histories():
    """Each sample's pressure and gas-fraction histories (n_sensors x n_out_times
    doubles each) are part of the workspace."""
    L = nv.lib()
    cp = api.cloud_params(W.cloud_uniform(4))

    def bytes_for(n_out):
        sp = W.SolverParams(sensors=W.eight_sensors(0.03), n_out_times=n_out)
        s = api.Solver(sp, "fp32")
        garr = (nv.ofm_group * 1)(api.make_group(sp, 16, list(range(5)), 1).c)
        n = C.c_size_t()
        nv.check(L.ofm_batch_workspace_bytes(s.h, C.byref(cp), garr, 1, C.byref(n)), "ws")
        return n.value

    grow = bytes_for(1001) - bytes_for(1)
    hist = 5 * 8 * 1000 * 8                     # samples x sensors x added output times x 8 bytes
    assert 2 * hist <= grow <= 2 * hist + 4096  # two histories, allocation rounding


def test_surrogate_cv_host_matches_oracle():
    from paper_1705_04374_gb300 import surrogate as S
    rng = np.random.default_rng(0)
    D = rng.normal(size=50)
    sp = D * 0.8 + rng.normal(size=50) * 0.3
    se = rng.normal(size=400) * 0.9
    a, b = S.surrogate_cv(D, sp, se), E.surrogate_cv(D, sp, se)
    for k in ("beta", "mean", "var"):
        assert abs(a[k] - b[k]) <= 1e-13 * max(1.0, abs(b[k]))


def test_zero_variance_needs_no_samples_in_the_library():
    assert list(api.optimal_samples([0.0, 0.0], [1.0, 16.0], 0.1, "tol", [5, 3])) == [5, 3]
    assert list(api.optimal_samples([0.0, 0.0], [1.0, 16.0], 1e3, "budget")) == [0, 0]


def test_summary_estimator_matches_oracle_and_pair_estimator():
    """ofm_level_moments_of / ofm_merge_moments / ofm_estimate_moments against
    the oracle's summaries and against ofm_estimate on the union of the pairs."""
    L, a, b = 2, 0.5, 1.0
    pairs = W.toy_levels([300, 40, 9], L, a, b, seed=11)
    Wl = [1.0, 17.0, 272.0]
    for p in pairs:
        got, ref = api.level_moments(p), E.level_moments(p)
        assert got[0] == ref[0] and np.allclose(got[1:], ref[1:], rtol=1e-13, atol=0)
        half = len(p) // 3
        m = api.merge_moments(api.level_moments(p[:half]), api.level_moments(p[half:]))
        r = E.merge_moments(E.level_moments(p[:half]), E.level_moments(p[half:]))
        assert m[0] == r[0] and np.allclose(m[1:], r[1:], rtol=1e-13, atol=0)
    assert api.level_moments(np.zeros((0, 2))) == (0, 0.0, 0.0, 0.0, 0.0, 0.0)
    est = api.estimate_moments([api.level_moments(p) for p in pairs], Wl)
    ref = E.estimate_from_moments([E.level_moments(p) for p in pairs], Wl)
    whole = api.estimate(pairs, Wl)
    for k in ("alpha", "sigma2", "cov", "sigma_tilde2"):
        assert np.allclose(est[k], ref[k], rtol=1e-12, atol=1e-15), k
        assert np.allclose(est[k], whole[k], rtol=1e-11, atol=1e-14), k
    assert abs(est["mean"] - whole["mean"]) <= 1e-12 * abs(whole["mean"])
    with pytest.raises(nv.OfmError):
        api.estimate_moments([api.level_moments(pairs[0][:1])], [1.0])   # one sample: no variance


def test_binding_structs_match_the_c_header(tmp_path):
    """Every struct of the ABI: size and field offsets from a C compiler reading
    include/ofmlmc.h equal the ctypes layout of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {name: cls for name, cls in vars(nv).items()
               if isinstance(cls, type) and issubclass(cls, C.Structure) and name.startswith("ofm_")}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ofmlmc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for line in out:
        if line:
            name, field, val = line.split()
            got[(name, field)] = int(val)
    assert len(structs) >= 8
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_product_code_never_touches_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it,
    no CUDA or C++ source of the library calls or loads it, the public header
    declares none of it, and the library does not link it."""
    root = os.path.dirname(os.path.dirname(__file__))
    pkg = os.path.join(root, "paper_1705_04374_gb300")
    py_use = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|liborc|oracle\.(solver|estimator|mlp|cloud)", re.M)
    c_use = re.compile(r"liborc|\borc_\w+\s*\(|#include\s+[<\"][^>\"]*oracle")
    offenders = []
    for d, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(d, f)
            if f.endswith(".py") and py_use.search(open(path).read()):
                offenders.append(path)
            elif f.endswith((".cu", ".cuh", ".cpp", ".h")) and c_use.search(open(path).read()):
                offenders.append(path)
    assert not offenders, offenders
    assert "orc_" not in open(HEADER).read()
    lib = nv.lib()
    assert not hasattr(lib, "orc_solve") and not hasattr(lib, "orc_rk3_step")


def test_oracle_shares_no_code_with_the_library():
    """The oracle neither imports the package nor includes its headers or sources."""
    root = os.path.dirname(os.path.dirname(__file__))
    odir = os.path.join(root, "oracle")
    for f in os.listdir(odir):
        path = os.path.join(odir, f)
        if f.endswith(".py"):
            text = open(path).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1705_04374_gb300", text, re.M), f
            assert "libofmlmc" not in text, f
        elif f.endswith((".c", ".h")):
            assert not re.search(r"#include\s+[<\"][^>\"]*(ofmlmc|csrc|paper_1705)", open(path).read()), f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library the binding raises; there is no fallback path."""
    monkeypatch.setattr(nv, "_lib", None)
    monkeypatch.setattr(nv, "LIB_PATH", str(tmp_path / "libofmlmc.so"))
    with pytest.raises(ImportError):
        nv.lib()
    with pytest.raises(ImportError):
        api.Solver(W.SolverParams())


@pytest.mark.parametrize("precision,N,fits", [("fp32", 32, 12), ("fp64", 32, 6), ("fp32", 64, 1), ("fp64", 64, 0)])
def test_static_entry_point_capacity(precision, N, fits):
    """The allocation-free entry point's size check runs on the host before any
    device call: `fits` samples on N^3 pass it, one more is rejected with
    OFM_ENOMEM (three state buffers of 7 N^3 values per sample in a 32 MiB
    array).  Without a GPU the accepted size fails later, at the device."""
    import ctypes as C
    sp = W.SolverParams(sensors=W.centre_sensor())
    s = api.Solver(sp, precision)
    cp = api.cloud_params(W.cloud_uniform(4))
    for n, rejected in ((fits, False), (fits + 1, True)):
        if n == 0:
            continue
        ids = (C.c_uint64 * n)(*range(n))
        out = (nv.ofm_qoi * n)()
        rc = nv.lib().ofm_solve_level_static(s.h, C.byref(cp), N, n, ids, W.BASE_SEED, out, None, None)
        assert (rc == nv.OFM_ENOMEM) == rejected, (n, rc, nv.lib().ofm_last_error())


@pytest.mark.parametrize("precision,N,n", [("fp64", 512, 2**31 - 1), ("fp64", 512, 2**30), ("fp32", 504, 10**9),
                                            ("fp32", 8, 2**31 - 1), ("fp32", 8, 781)])
def test_static_entry_point_rejects_huge_sample_counts(precision, N, n):
    """Sample counts whose byte count would not fit a 64-bit size (n times
    three state buffers of 7 N^3 values reaches 2^64 on the finest grids) are
    rejected with OFM_ENOMEM before any byte count is formed, so no wrapped
    size can pass the 32 MiB check.  The ids array is never read on this path."""
    import ctypes as C
    sp = W.SolverParams(sensors=W.centre_sensor())
    s = api.Solver(sp, precision)
    cp = api.cloud_params(W.cloud_uniform(4))
    ids = (C.c_uint64 * 1)(0)
    out = (nv.ofm_qoi * 1)()
    rc = nv.lib().ofm_solve_level_static(s.h, C.byref(cp), N, n, ids, W.BASE_SEED, out, None, None)
    assert rc == nv.OFM_ENOMEM, (rc, nv.lib().ofm_last_error())
    assert b"need" in nv.lib().ofm_last_error()


def test_static_entry_point_rejects_oversized_histories():
    """One sample on 8^3 with eight sensors and 2^31 - 1 output times needs
    ~1.4e11 bytes of history: rejected with OFM_ENOMEM on the host."""
    import ctypes as C
    sp = W.SolverParams(sensors=W.eight_sensors(0.02), n_out_times=2**31 - 1)
    s = api.Solver(sp, "fp32")
    cp = api.cloud_params(W.cloud_uniform(4))
    ids = (C.c_uint64 * 1)(0)
    out = (nv.ofm_qoi * 1)()
    rc = nv.lib().ofm_solve_level_static(s.h, C.byref(cp), 8, 1, ids, W.BASE_SEED, out, None, None)
    assert rc == nv.OFM_ENOMEM, (rc, nv.lib().ofm_last_error())


def test_static_entry_point_rejects_a_request_whose_byte_count_wraps():
    """2^30 FP64 samples on 512^3, one sensor, no bubbles and 1,475,084,226
    output times: every per-sample byte count is then a multiple of 256 and
    their sum a multiple of 2^34, so the unchecked total is 2 x 2^64 + 1280
    bytes and wraps to 1280, under the 32 MiB of the array.  The sample
    count is rejected (OFM_ENOMEM) before any byte count is formed."""
    import ctypes as C
    sp = W.SolverParams(sensors=W.centre_sensor(), n_out_times=1475084226)
    s = api.Solver(sp, "fp64")
    cp = api.cloud_params(W.cloud_uniform(0))
    ids = (C.c_uint64 * 1)(0)
    out = (nv.ofm_qoi * 1)()
    rc = nv.lib().ofm_solve_level_static(s.h, C.byref(cp), 512, 2**30, ids, W.BASE_SEED, out, None, None)
    assert rc == nv.OFM_ENOMEM, (rc, nv.lib().ofm_last_error())


@pytest.mark.parametrize("n_bubbles,n_out,n_samples", [(0, 2**30, 2**28), (2**31 - 1, 65, 2**28 + 1),
                                                       (4, 65, 2**31 - 1)])
def test_batch_workspace_size_never_wraps(n_bubbles, n_out, n_samples):
    """ofm_batch_workspace_bytes returns an error instead of a wrapped byte
    count: 2^28 samples with 8 sensors x 2^30 output times make a history of
    exactly 2^64 bytes (a wrapped count of 0); 2^28 + 1 samples of 2^31 - 1
    bubbles make a cloud table of just over 2^64 bytes; 2^31 - 1 samples of
    8^3 (within the tile limit) carry more than 2^40 history values.  The
    benchmark's size (512 samples on 64^3) is still computed.  Only the group
    table is read on this path."""
    import ctypes as C
    sp = W.SolverParams(sensors=W.eight_sensors(0.02), n_out_times=n_out)
    s = api.Solver(sp, "fp32")
    cloud = W.cloud_uniform(4)
    cp = api.cloud_params(cloud)
    cp.n_bubbles = n_bubbles
    ids = (C.c_uint64 * 1)(0)
    g = nv.ofm_group()
    g.N = 8
    g.n_samples = n_samples
    g.sample_ids = ids
    nbytes = C.c_size_t(0)
    rc = nv.lib().ofm_batch_workspace_bytes(s.h, C.byref(cp), C.byref(g), 1, C.byref(nbytes))
    assert rc in (nv.OFM_ENOMEM, nv.OFM_EINVAL), (rc, nbytes.value)
    # the benchmark's size is still computed, and it is at least its three state buffers
    sp = W.SolverParams(sensors=W.eight_sensors(0.02))
    s = api.Solver(sp, "fp32")
    cp = api.cloud_params(W.cloud_uniform(20))
    ids = (C.c_uint64 * 512)(*range(512))
    g = nv.ofm_group()
    g.N = 64
    g.n_samples = 512
    g.sample_ids = ids
    assert nv.lib().ofm_batch_workspace_bytes(s.h, C.byref(cp), C.byref(g), 1, C.byref(nbytes)) == nv.OFM_OK
    assert nbytes.value >= 3 * 512 * 7 * 64**3 * 4


@pytest.mark.parametrize("d_in,hidden,d_out,rows", [(2**31 - 1, 2**31 - 1, 1, 1), (2000, 2**31 - 1, 1, 1),
                                                    (201, 1024, 1, 2**31 - 1)])
def test_mlp_workspace_size_never_wraps(d_in, hidden, d_out, rows):
    """Four parameter-sized buffers of (2^31 - 1)^2 floats sum past 2^64
    bytes: ofm_mlp_workspace_bytes returns OFM_ENOMEM for that and the other
    oversized networks instead of a wrapped count, and still sizes the
    surrogate's own shapes (2001 inputs, 3 x 256, 65,536 rows)."""
    import ctypes as C
    nbytes = C.c_size_t(0)
    rc = nv.lib().ofm_mlp_workspace_bytes(d_in, hidden, 3, d_out, rows, C.byref(nbytes))
    assert rc == nv.OFM_ENOMEM, (rc, nbytes.value)
    assert nv.lib().ofm_mlp_workspace_bytes(2001, 256, 3, 1, 65536, C.byref(nbytes)) == nv.OFM_OK
    assert nbytes.value >= 4 * 4 * (2001 * 256 + 2 * 256 * 256 + 256)


def test_surrogate_estimator_matches_oracle():
    """ofm_estimate_surrogate against the oracle on a toy hierarchy with a
    nonlinear surrogate: optimal and fixed beta."""
    rng = np.random.default_rng(9)
    M = [150, 50, 16]
    pairs = W.toy_levels(M, 2, 0.5, 0.6, seed=9)
    ht = 0.7 * pairs[2][:, 1] + 0.2 * np.tanh(pairs[2][:, 1]) + 0.01 * rng.normal(size=M[2])
    he = 0.7 * pairs[1][:, 0] + 0.2 * np.tanh(pairs[1][:, 0]) + 0.01 * rng.normal(size=M[1])
    Wl = [1.0, 6.0, 40.0]
    for beta in (None, 0.4, 0.0):
        got = api.estimate_surrogate(pairs, Wl, ht, he, beta=beta)
        ref = E.estimate_surrogate(pairs, Wl, ht, he, beta=beta)
        assert got["beta"] == pytest.approx(ref["beta"], rel=1e-12, abs=1e-15)
        for k in ("alpha", "sigma_tilde2", "sigma_tilde2_plain"):
            assert np.allclose(got[k], ref[k], rtol=1e-12, atol=0), k
        assert got["mean"] == pytest.approx(ref["mean"], rel=1e-13)
        assert got["eps2"] == pytest.approx(ref["eps2"], rel=1e-12)
    with pytest.raises(nv.OfmError):
        api.estimate_surrogate(pairs[:1], Wl[:1], ht, he)


def test_level_kde_matches_oracle():
    """ofm_sj_bandwidth and ofm_level_kde against the oracle (Sec. 3.2's
    level-wise density): the bandwidths to the bisection's 1e-10 (sums in
    another order may move a bisection step), the density accordingly."""
    from oracle import kde as K
    pairs = W.toy_levels([300, 120, 40], 2, 0.5, 0.6, seed=12)
    for x in (pairs[0][:, 0], np.random.default_rng(1).gamma(2.0, size=200)):
        assert api.sj_bandwidth(x) == pytest.approx(K.sj_bandwidth(x), rel=1e-9)
    alpha = [0.9, 1.2, 1.0]
    xs = np.linspace(-6, 8, 57)
    f, bw = api.level_kde(pairs, alpha, xs)
    fr, bwr = K.level_kde(pairs, alpha, xs)
    assert np.allclose(bw, bwr, rtol=1e-9)
    assert np.allclose(f, fr, rtol=1e-7, atol=1e-9 * np.max(np.abs(fr)))
    with pytest.raises(nv.OfmError):
        api.sj_bandwidth([1.0])
