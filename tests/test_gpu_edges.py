"""Edge cases of the GPU path: clouds without bubbles (a state at rest must
stay exactly at rest), and the largest grid with sample offsets beyond 2^31
elements (64-bit indexing), against the same cloud solved alone."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04374_gb300 import api  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cloud_without_bubbles_stays_at_rest(precision):
    """No bubbles: uniform liquid at p_liq, u = 0.  Every WENO difference is
    zero, both sides of every face are equal and the fluxes cancel exactly, so
    the state is unchanged bit for bit and the peak pressure is p_liq at every
    step up to t_end."""
    w = W.tiny(16, 0)
    sp = w.solver
    s = api.Solver(sp, precision)
    g = api.make_group(sp, 16, [0, 1], W.BASE_SEED)
    b = api.Batch(s, w.cloud, [g])
    b.init()
    Q0 = b.state(0, 0).copy()
    while b.run(64) > 0:
        pass
    b.qoi()
    assert np.array_equal(b.state(0, 0), Q0)
    for d in g.qoi_dicts(1):
        assert d["status"] == 0 and d["n_steps"] > 0
        assert abs(d["p_peak"] - sp.p_liq) <= (1e-12 if precision == "fp64" else 1e-5) * sp.p_liq
    b.close()


def test_largest_grid_with_offsets_beyond_2_31_elements():
    """Four samples on 512^3 in FP32 (the fourth starts 2.8e9 elements into
    each state buffer): one step of the fourth equals the same cloud solved
    alone, bit for bit."""
    free, _ = torch.cuda.mem_get_info()
    need = 5 * 3 * 7 * 512 ** 3 * 4
    if free < need * 1.1:
        pytest.skip("not enough device memory")
    w = W.tiny(16, 20)
    sp = w.solver
    s = api.Solver(sp, "fp32")
    ids = [0, 1, 2, 3]
    g = api.make_group(sp, 512, ids, W.BASE_SEED)
    b = api.Batch(s, w.cloud, [g])
    b.init()
    b.run(1)
    together = b.state(0, 3)
    b.close()
    del b
    torch.cuda.empty_cache()
    g1 = api.make_group(sp, 512, [3], W.BASE_SEED)
    b1 = api.Batch(s, w.cloud, [g1])
    b1.init()
    b1.run(1)
    alone = b1.state(0, 0)
    b1.close()
    assert np.array_equal(together, alone)
    assert np.isfinite(alone).all()
