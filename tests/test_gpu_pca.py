"""GPU data-derived metric (Sec. 3.1, principal component analysis) against
the oracle's, and the paper's data pipeline end to end: Eq. (9) data, the
PCA metric, the prescribed top rotation."""
import numpy as np
import pytest

import dd_inputs as I
from oracle import dd as odd
from oracle import metric

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_00357_gb300 as P  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    P.build()
    c = P.dd_create(0)
    yield c
    P.dd_destroy(c)


def test_pca_metric_matches_oracle(ctx):
    """Eq. (9) data: the GPU metric equals the oracle's FP64 PCA metric; host
    and device input give the same bits, and so does a second call."""
    data = I.make_dataset(300000, I.EQ9_LAW, seed=2)
    Cg = P.dd_pca_metric(ctx, data)
    Co = metric.pca_metric(data.astype(np.float64))
    assert np.allclose(Cg, Co, rtol=1e-9, atol=1e-9 * np.abs(Co).max())
    Cd = P.dd_pca_metric(ctx, torch.from_numpy(data).cuda())
    assert np.array_equal(Cg, Cd)
    assert np.array_equal(Cg, P.dd_pca_metric(ctx, data))
    assert np.allclose(Cg, Cg.T, rtol=0, atol=0)


def test_pca_metric_of_linear_data(ctx):
    """Data on sig = C0 eps with a non-isotropic SPD C0, stored in float32:
    GPU and oracle agree to rounding, and both return C0 to the storage
    precision."""
    rng = np.random.default_rng(7)
    B = rng.normal(size=(6, 6))
    C0 = B @ B.T + 6 * np.eye(6)
    eps = rng.uniform(-1e-3, 1e-3, (40000, 6)) * np.array([1, 2, 3, 0.5, 0.7, 1.3])
    data = np.ascontiguousarray(np.concatenate([eps, eps @ C0.T], axis=1).astype(np.float32))
    Cg = P.dd_pca_metric(ctx, data)
    Co = metric.pca_metric(data.astype(np.float64))
    assert np.allclose(Cg, Co, rtol=1e-8, atol=1e-8 * np.abs(Co).max())
    assert np.allclose(Cg, C0, rtol=1e-4, atol=1e-4 * np.abs(C0).max())


def test_pca_metric_rejects_degenerate_strains(ctx):
    """All strains on one axis: the principal strain block is singular."""
    data = np.zeros((1000, 12), np.float32)
    data[:, 0] = np.linspace(-1e-3, 1e-3, 1000)
    data[:, 6] = 2.0 * data[:, 0]
    with pytest.raises(P.DDError):
        P.dd_pca_metric(ctx, data)


@pytest.mark.parametrize("n_el", [3, 4])
def test_paper_pipeline_matches_oracle(ctx, n_el):
    """The paper's setup at small size: data from Eq. (9), the metric from
    the GPU's principal component analysis, the top face turned by 2 degrees;
    the GPU DD solve (exact search) equals the oracle's with the same metric."""
    data = I.make_dataset(20000, I.EQ9_LAW, seed=3)
    C = P.dd_pca_metric(ctx, data)
    assert np.allclose(C, metric.pca_metric(data.astype(np.float64)), rtol=1e-9, atol=1e-9 * np.abs(C).max())
    load = I.top_rotation(2.0)
    init = I.initial_association(8 * n_el ** 3, len(data), seed=4)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r = P.dd_solve(ds, ctx, n_el, load, init_idx=init)
    finally:
        P.dd_free_dataset(ds)
    o = odd.DDProblem(data, C, n_el, load).solve(init)
    assert r.converged == o.converged and r.iters == o.iters
    assert np.array_equal(r.idx, o.idx)
    assert np.allclose(r.u, o.u, rtol=0, atol=1e-6 * np.abs(o.u).max())
    assert np.allclose(r.d2_pd, o.d2_after_pd, rtol=1e-6)
