"""GPU MLP surrogate kernels against the FP64 oracle.

Tolerances.  BF16 keeps 8 significant bits (unit roundoff u = 2^-9 ~ 2e-3).
Against an oracle that rounds the same GEMM operands to BF16 and computes in
FP64, the GPU differs only by FP32 accumulation (~1e-6) and by rare one-ulp
flips where an FP32 activation sits on a BF16 rounding boundary: relative L2
<= 2e-3 for outputs and gradients.  Against the plain FP64 oracle (no BF16),
each of the four GEMM layers adds ~2u of relative noise: <= 3e-2.

Element by element (each element against |its reference| plus 1e-2 of the
largest reference element): without flips the error is FP32 accumulation,
~1e-7 (measured 1.7e-7 to 7.5e-6 on the narrow networks).  A flip moves one
operand by one BF16 ulp (<= 2^-8 of it); in a weight gradient that changes
the column it feeds by ~2^-8/sqrt(rows) of its size, ~3e-4 on 130 rows, and
more on elements near zero, which the floor judges on the layer's scale:
measured 4.2e-3 (outputs) and 4.3e-2 (first-layer weight gradient) on the
200 -> 256 x 3 network.  Bounds: 2e-2 for outputs, 0.15 for gradients, and
relative L2 per row and per column of every weight gradient <= 1e-2 (a wrong
row or column gives ~1 there).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import cloud as ocloud
from oracle import estimator as E
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04374_gb300 import surrogate as S  # noqa: E402

ELEM_FWD = 2e-2
ELEM_GRAD = 0.15
ROWCOL_GRAD = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def init_params(rng, sizes):
    return [(rng.normal(size=(a, b)) * math.sqrt(2.0 / a), rng.normal(size=b) * 0.05)
            for a, b in zip(sizes[:-1], sizes[1:])]


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


def rel_elem(a, b, floor=1e-2):
    """Largest element-wise error, each relative to its reference element
    plus a floor of `floor` times the largest reference magnitude (so that
    elements near zero are judged on the vector's scale)."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / (np.abs(b) + floor * max(np.max(np.abs(b)), 1e-300))))


def setup_net(d_in, hidden, n_hidden, d_out, rows, seed=0, max_rows=None):
    rng = np.random.default_rng(seed)
    sizes = [d_in] + [hidden] * n_hidden + [d_out]
    P = init_params(rng, sizes)
    vec = omlp.flatten(P).astype(np.float32)
    P32 = omlp.unflatten(vec.astype(np.float64), sizes)
    net = S.MLP(d_in, hidden, n_hidden, d_out, max_rows or rows)
    net.set_params(vec)
    X = rng.normal(size=(rows, d_in)).astype(np.float32)
    T = (np.sin(X[:, :d_out] * 1.3) + 0.1 * X[:, d_out:2 * d_out] ** 2).astype(np.float32)
    return net, P32, sizes, X, T


@pytest.mark.parametrize("shape", [(40, 64, 2, 1, 50), (200, 256, 3, 1, 130), (37, 48, 3, 3, 77)])
def test_forward_matches_oracle(shape):
    d_in, hidden, nh, d_out, rows = shape
    net, P, sizes, X, T = setup_net(d_in, hidden, nh, d_out, rows)
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Xd = X.astype(np.float64)
    y_lowp, _ = omlp.forward(P, Xd, lowp=True)
    y_fp64, _ = omlp.forward(P, Xd)
    assert rel_l2(Y, y_lowp) < 2e-3
    assert rel_l2(Y, y_fp64) < 3e-2
    e = rel_elem(Y, y_lowp)
    print(f"\nforward {shape}: element-wise error vs the BF16-operand oracle {e:.2e}")
    assert e < ELEM_FWD
    net.close()


def test_forward_in_chunks_equals_single_pass():
    net, P, sizes, X, T = setup_net(30, 64, 3, 1, 300, max_rows=300)
    Xt = torch.from_numpy(X).cuda()
    Y1 = net.forward(Xt).cpu().numpy()
    params = net.get_params()
    net2 = S.MLP(30, 64, 3, 1, max_rows=64)
    net2.set_params(params)
    Y2 = net2.forward(Xt).cpu().numpy()
    assert np.array_equal(Y1, Y2)   # rows are independent: chunking changes nothing
    net.close()
    net2.close()


@pytest.mark.parametrize("shape", [(40, 64, 2, 1, 50), (200, 256, 3, 1, 130)])
def test_gradients_match_oracle(shape):
    d_in, hidden, nh, d_out, rows = shape
    net, P, sizes, X, T = setup_net(d_in, hidden, nh, d_out, rows, seed=1)
    g, loss = net.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    Xd, Td = X.astype(np.float64), T.astype(np.float64)
    for lowp, tol in ((True, 2e-3), (False, 3e-2)):
        y, cache = omlp.forward(P, Xd, lowp=lowp)
        G = omlp.backward(P, cache, y, Td, lowp=lowp)
        gref = omlp.flatten(G)
        assert rel_l2(g, gref) < tol, (lowp, rel_l2(g, gref))
        # and layer by layer
        ggpu = omlp.unflatten(g.astype(np.float64), sizes)
        for li, ((gw, gb), (rw, rb)) in enumerate(zip(ggpu, G)):
            assert rel_l2(gw, rw) < tol and rel_l2(gb, rb) < tol
            if lowp:   # element by element, and row by row / column by column, against the BF16-operand oracle
                ew, eb = rel_elem(gw, rw), rel_elem(gb, rb)
                er = max(rel_l2(gw[i], rw[i]) for i in range(rw.shape[0]))
                ec = max(rel_l2(gw[:, j], rw[:, j]) for j in range(rw.shape[1]))
                print(f"\ngradients {shape} layer {li}: element-wise error W {ew:.2e} b {eb:.2e}, "
                      f"worst row {er:.2e}, worst column {ec:.2e}")
                assert ew < ELEM_GRAD and eb < ELEM_GRAD
                assert er < ROWCOL_GRAD and ec < ROWCOL_GRAD
        assert abs(loss - omlp.mse_loss(y, Td)) < tol * omlp.mse_loss(y, Td)
    net.close()


def test_adam_step_matches_oracle_update():
    net, P, sizes, X, T = setup_net(24, 32, 3, 1, 40, seed=2)
    p0 = net.get_params().astype(np.float64)
    Xt, Tt = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    g, _ = net.gradients(Xt, Tt)
    net.train(Xt, Tt, steps=1, lr=1e-3)
    p1 = net.get_params().astype(np.float64)
    Pp = omlp.unflatten(p0, sizes)
    G = omlp.unflatten(g.astype(np.float64), sizes)
    opt = omlp.Adam(Pp, lr=1e-3)
    ref = omlp.flatten(opt.step(Pp, G))
    assert np.max(np.abs(p1 - ref)) < 1e-6 * max(1.0, np.max(np.abs(p0)))
    net.close()


def test_training_tracks_oracle_and_reduces_loss():
    net, P, sizes, X, T = setup_net(16, 64, 3, 1, 256, seed=3)
    Xt, Tt = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    hist = net.train(Xt, Tt, steps=200, lr=3e-3)
    assert hist[-1] < 0.3 * hist[0]
    # oracle (BF16 operands) with the same full-batch steps
    opt = omlp.Adam(P, lr=3e-3)
    Pp = P
    losses = []
    for _ in range(20):
        y, cache = omlp.forward(Pp, X.astype(np.float64), lowp=True)
        losses.append(omlp.mse_loss(y, T.astype(np.float64)))
        Pp = opt.step(Pp, omlp.backward(Pp, cache, y, T.astype(np.float64), lowp=True))
    assert np.max(np.abs(hist[:20] - np.array(losses)) / np.array(losses)) < 2e-2
    net.close()


def test_training_is_deterministic():
    outs = []
    for _ in range(2):
        net, P, sizes, X, T = setup_net(16, 64, 3, 1, 128, seed=4)
        net.train(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), steps=20, lr=1e-3)
        outs.append(net.get_params())
        net.close()
    assert np.array_equal(outs[0], outs[1])


def test_scaling_is_applied_and_undone():
    net, P, sizes, X, T = setup_net(8, 32, 2, 1, 64, seed=5)
    xm, xs = X.mean(0), X.std(0) * 2.0
    ym, ys = np.array([0.3], np.float32), np.array([2.5], np.float32)
    net.set_scaling(xm, xs, ym, ys)
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Xs = (X.astype(np.float64) - xm) / xs.astype(np.float64)
    y_ref, _ = omlp.forward(P, Xs.astype(np.float32).astype(np.float64), lowp=True)
    assert rel_l2(Y, y_ref * 2.5 + 0.3) < 2e-3
    net.close()


def test_cloud_features_match_oracle_bitwise():
    cp = W.cloud_uniform(50)
    ids = list(range(17))
    bub = np.stack([ocloud.sample_cloud(cp, 7, i) for i in ids])
    Xg = S.cloud_features(torch.from_numpy(bub).cuda(), 50, cp.domain_L, cp.cloud_radius).cpu().numpy()
    for i in ids:
        ref = omlp.cloud_features(bub[i], cp.domain_L, cp.cloud_radius).astype(np.float32)
        assert np.array_equal(Xg[i], ref)
    # the 3 nearest bubbles only
    Xk = S.cloud_features(torch.from_numpy(bub).cuda(), 50, cp.domain_L, cp.cloud_radius, 3).cpu().numpy()
    assert Xk.shape == (len(ids), 12)
    for i in ids:
        assert np.array_equal(Xk[i], omlp.cloud_features(bub[i], cp.domain_L, cp.cloud_radius, 3).astype(np.float32))


def test_column_moments_match_numpy():
    rng = np.random.default_rng(6)
    X = rng.normal(size=(333, 70)).astype(np.float32) * 3 + 1
    m, s = S.column_moments(torch.from_numpy(X).cuda())
    Xd = X.astype(np.float64)
    assert np.allclose(m.cpu().numpy(), Xd.mean(0), rtol=1e-12, atol=1e-12)
    assert np.allclose(s.cpu().numpy(), Xd.std(0, ddof=1), rtol=1e-12)


def test_trained_surrogate_reduces_estimator_variance():
    """A learnable QoI of the cloud geometry: the trained network used as an
    extra control variate cuts the variance of the top-level term, and the
    corrected estimate stays unbiased."""
    cp = W.cloud_uniform(20)
    rng = np.random.default_rng(8)

    def geom_qoi(b):   # a smooth function of the cloud: volume of the 5 bubbles nearest the centre
        f = omlp.cloud_features(b, cp.domain_L, cp.cloud_radius).reshape(-1, 4)
        return float(np.sum(f[:5, 3] ** 3) * 100.0)

    n_train, M, N = 4096, 64, 2048
    clouds = [ocloud.sample_cloud(cp, 11, i) for i in range(n_train + M + N)]
    q = np.array([geom_qoi(b) for b in clouds])
    noise = rng.normal(size=q.size) * 0.05 * q.std()
    D = q + noise
    bub = torch.from_numpy(np.stack(clouds)).cuda()
    X = S.cloud_features(bub, 20, cp.domain_L, cp.cloud_radius)
    m, s = S.column_moments(X[:n_train])
    net = S.MLP(80, 256, 3, 1, max_rows=n_train)
    p = omlp.flatten(init_params(np.random.default_rng(9), net.sizes)).astype(np.float32)
    net.set_params(p)
    net.set_scaling(m.cpu().numpy(), s.cpu().numpy(), np.array([D[:n_train].mean()]), np.array([D[:n_train].std()]))
    T = torch.from_numpy(D[:n_train, None].astype(np.float32)).cuda()
    hist = net.train(X[:n_train], T, steps=300, lr=1e-3)
    assert hist[-1] < 0.1 * hist[0]
    sv = net.forward(X[n_train:]).cpu().numpy().ravel().astype(np.float64)
    assert np.corrcoef(sv, D[n_train:])[0, 1] > 0.7      # it generalises to unseen clouds
    Dm = D[n_train:n_train + M]
    out = S.surrogate_cv(Dm, sv[:M], sv[M:])
    ref = E.surrogate_cv(Dm, sv[:M], sv[M:])
    assert abs(out["mean"] - ref["mean"]) < 1e-12 * abs(ref["mean"]) and abs(out["beta"] - ref["beta"]) < 1e-12
    plain_var = np.var(Dm, ddof=1) / M
    assert out["var"] < 0.5 * plain_var
    net.close()


def test_surrogate_of_solver_qois_cuts_level_variance():
    """On the solver's own samples: centre-sensor peak pressures of 2048 clouds
    (20 bubbles, 16^3, FP32) and a network on the geometry of each cloud's
    bubble nearest the centre.  Trained on 1024 clouds, it predicts the other
    1024 well, and as an extra control variate it cuts the variance of the
    plain sample mean by more than half."""
    from paper_1705_04374_gb300 import api
    cp = W.cloud_uniform(20)
    sp = W.SolverParams(sensors=W.centre_sensor())
    s = api.Solver(sp, "fp32")
    ids = list(range(2048))
    g = api.make_group(sp, 16, ids, W.BASE_SEED)
    b = api.Batch(s, cp, [g])
    b.init()
    while b.run(1 << 20) > 0:
        pass
    b.qoi(allow_bad=True)
    q = np.array([d["sensor_peak"][0] for d in g.qoi_dicts(1)])
    b.close()
    bub = torch.from_numpy(np.stack([api.sample_cloud(cp, W.BASE_SEED, i) for i in ids])).cuda()
    X = S.cloud_features(bub, 20, cp.domain_L, cp.cloud_radius, 1)
    n = 1024
    m, sd = S.column_moments(X[:n])
    net = S.MLP(4, 256, 3, 1, max_rows=n)
    net.set_params(omlp.flatten(init_params(np.random.default_rng(9), net.sizes)).astype(np.float32))
    net.set_scaling(m.cpu().numpy(), sd.cpu().numpy(), np.array([q[:n].mean()]), np.array([q[:n].std()]))
    net.train(X[:n], torch.from_numpy(q[:n, None].astype(np.float32)).cuda(), steps=600, lr=1e-3)
    sv = net.forward(X[n:]).cpu().numpy().ravel().astype(np.float64)
    net.close()
    assert np.corrcoef(sv, q[n:])[0, 1] > 0.8
    M = 256                                   # the plain mean of M samples, and N further clouds
    out = S.surrogate_cv(q[n:n + M], sv[:M], sv[M:])
    assert out["var"] < 0.5 * np.var(q[n:n + M], ddof=1) / M
