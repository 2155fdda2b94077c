"""GPU k-nearest-neighbour graph and greedy walk (Sec. 4.4) against the
oracle's restatement, through the C ABI."""
import numpy as np
import pytest

import dd_inputs as I
from oracle import knng, metric

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_00357_gb300 as P  # noqa: E402

C = I.isotropic_C()


@pytest.fixture(scope="module")
def ctx():
    P.build()
    c = P.dd_create(0)
    yield c
    P.dd_destroy(c)


def test_graph_at_fd_one_is_exact(ctx):
    """8 coarse cells of 8 leaves: every cell and leaf is a candidate, so the
    build at f_d = 1 is the exact k-NN graph (equal rows up to near-ties at
    the k-th place, equal sorted distances)."""
    data = I.make_dataset(3000, I.NONLINEAR, seed=41)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=64, ann_levels=2, seed=3, knn_k=12, knn_fd=1.0)
    try:
        assert P.dd_dataset_knn_k(ds) == 12
        g = P.dd_dataset_knn_graph(ds, ctx)
    finally:
        P.dd_free_dataset(ds)
    Z = metric.to_z(data.astype(np.float64), C)
    go = knng.knn_graph(Z, 12)
    dg = np.array([((Z[g[i]] - Z[i]) ** 2).sum(1) for i in range(len(Z))])
    do = np.array([((Z[go[i]] - Z[i]) ** 2).sum(1) for i in range(len(Z))])
    assert np.all(g >= 0) and np.all(g != np.arange(len(Z))[:, None])
    assert np.allclose(dg, do, rtol=1e-5, atol=0)
    same = np.array([set(g[i]) == set(go[i]) for i in range(len(Z))])
    # rows may differ only where the k-th and (k+1)-th distances nearly tie
    g13 = knng.knn_graph(Z, 13)
    d12 = ((Z[g13[:, 11]] - Z) ** 2).sum(1)
    d13 = ((Z[g13[:, 12]] - Z) ** 2).sum(1)
    near = np.abs(d13 - d12) <= 1e-5 * d12
    assert np.all(same | near)
    print(f"rows equal: {same.mean():.4f}")


@pytest.mark.parametrize("k", [40, 75, 128])
def test_wide_graph_at_fd_one_is_exact(ctx, k):
    """k above 32: the list spans several registers per lane; the build at
    f_d = 1 still gives the exact k-NN graph, and a walk over k neighbours
    matches the oracle's."""
    data = I.make_dataset(2500, I.NONLINEAR, seed=49)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=64, ann_levels=2, seed=3, knn_k=k, knn_fd=1.0)
    try:
        g = P.dd_dataset_knn_graph(ds, ctx)
        y = I.make_states(400, I.NONLINEAR, seed=50, spread=0.1)
        prev = np.random.default_rng(7).integers(0, len(data), len(y)).astype(np.int32)
        idx, d2, st = walk(ctx, ds, y, prev)
    finally:
        P.dd_free_dataset(ds)
    Z = metric.to_z(data.astype(np.float64), C)
    go = knng.knn_graph(Z, k)
    dg = np.array([((Z[g[i]] - Z[i]) ** 2).sum(1) for i in range(len(Z))])
    do = np.array([((Z[go[i]] - Z[i]) ** 2).sum(1) for i in range(len(Z))])
    assert np.allclose(dg, do, rtol=1e-5, atol=0)
    same = np.mean([set(g[i]) == set(go[i]) for i in range(len(Z))])
    assert same >= 0.99
    oi, od, osec, omv, oev = knng.walk_all(Z, g, metric.to_z(y, C), prev)
    assert np.mean(idx == oi) >= 0.98 and abs(st.moves - omv.sum()) <= 0.02 * omv.sum() + 5


def test_small_data_set_pads_rows(ctx):
    """N - 1 < k: every other point is a neighbour, the rest of a row is -1."""
    data = I.make_dataset(20, I.LINEAR, seed=42)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=4, ann_levels=2, seed=3, knn_k=32, knn_fd=1.0)
    try:
        g = P.dd_dataset_knn_graph(ds, ctx)
    finally:
        P.dd_free_dataset(ds)
    Z = metric.to_z(data.astype(np.float64), C)
    go = knng.knn_graph(Z, 32)
    assert np.all(g[:, 19:] == -1) and np.all(go[:, 19:] == -1)
    assert all(set(g[i, :19]) == set(range(20)) - {i} for i in range(20))
    dg = np.array([((Z[g[i, :19]] - Z[i]) ** 2).sum(1) for i in range(20)])
    assert np.all(np.diff(dg, axis=1) >= -1e-6 * dg[:, 1:])        # nearest first


@pytest.fixture(scope="module")
def graphset(ctx):
    data = I.make_dataset(20000, I.NONLINEAR, seed=43)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=256, ann_levels=2, seed=5, knn_k=16, knn_fd=0.6)
    g = P.dd_dataset_knn_graph(ds, ctx)
    yield data, ds, g
    P.dd_free_dataset(ds)


def walk(ctx, ds, y, prev=None, f_s=0):
    idx = np.full(len(y), -7, np.int32)
    d2 = np.full(len(y), -1.0)
    st = P.dd_project_nearest(ds, ctx, y, idx, d2, mode=P.DD_SEARCH_KNNG, f_s=f_s,
                              prev_idx=None if prev is None else np.ascontiguousarray(prev, np.int32))
    return idx, d2, st


@pytest.mark.parametrize("f_s", [0, 1, 3])
def test_walk_matches_oracle(ctx, graphset, f_s):
    """Same graph, same starts: the GPU walk (FP32 distances) and the oracle's
    (FP64) agree but for near-ties, and every GPU answer is a valid end of a
    walk (no neighbour nearer unless stopped by f_s, never worse than the
    start); the FP64 Eq. (3) distance of the answer is reported."""
    data, ds, g = graphset
    Z = metric.to_z(data.astype(np.float64), C)
    y = I.make_states(800, I.NONLINEAR, seed=44, spread=0.1)
    zq = metric.to_z(y, C)
    prev = np.random.default_rng(5).integers(0, len(data), len(y)).astype(np.int32)
    idx, d2, st = walk(ctx, ds, y, prev, f_s)
    oi, od, osec, omv, oev = knng.walk_all(Z, g, zq, prev, f_s)
    same = idx == oi
    print(f"f_s={f_s}: agree {same.mean():.4f}, moves gpu {st.moves} oracle {omv.sum()}")
    assert same.mean() >= 0.98
    dg = ((Z[idx] - zq) ** 2).sum(1)
    assert np.all(dg <= ((Z[prev] - zq) ** 2).sum(1) * (1 + 1e-6))
    if f_s == 0:
        for i in np.nonzero(~same)[0]:
            assert np.all(((Z[g[idx[i]]] - zq[i]) ** 2).sum(1) >= dg[i] * (1 - 1e-5))
    assert abs(st.moves - omv.sum()) <= 0.02 * max(omv.sum(), 1) + 5
    assert st.distances == pytest.approx(oev.sum(), rel=0.02)
    assert np.allclose(metric.local_d2(y, data[idx].astype(np.float64), C), d2, rtol=1e-10)


def test_walk_without_previous_neighbour(ctx, graphset):
    """Without prev_idx the walk of query i starts at data point
    SplitMix64(i) mod N (the first output of SplitMix64 seeded with i)."""
    data, ds, g = graphset
    Z = metric.to_z(data.astype(np.float64), C)
    y = I.make_states(300, I.NONLINEAR, seed=45, spread=0.05)
    zq = metric.to_z(y, C)
    starts = np.array([I._fmix64_int(i + I.GAMMA) % len(data) for i in range(len(y))])
    idx, d2, st = walk(ctx, ds, y)
    oi = knng.walk_all(Z, g, zq, starts)[0]
    assert np.mean(idx == oi) >= 0.98


def test_walk_on_complete_graph_is_exact(ctx):
    """Every point linked to all others (N = 33, k = 32): the walk returns the
    exact nearest point from any start."""
    data = I.make_dataset(33, I.NONLINEAR, seed=46)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=4, ann_levels=2, seed=3, knn_k=32, knn_fd=1.0)
    try:
        y = I.make_states(500, I.NONLINEAR, seed=47, spread=0.3)
        prev = np.random.default_rng(6).integers(0, 33, len(y)).astype(np.int32)
        idx, d2, st = walk(ctx, ds, y, prev)
    finally:
        P.dd_free_dataset(ds)
    from gpu_util import assert_nn_parity
    assert_nn_parity(idx, d2, data, y, C)


def test_graph_solve_and_batch(ctx, graphset):
    """A DD solve driven by the graph walk converges (association unchanged
    or distance stalled), is never worse than its first iteration, and two
    solves stepped together reproduce the stand-alone solves bit for bit."""
    data, ds, g = graphset
    loads = [I.load_case("tension", 1e-3), I.load_case("torsion", 1e-3)]
    alone = [P.dd_solve(ds, ctx, 3, L, mode=P.DD_SEARCH_KNNG, seed=9, max_iter=100) for L in loads]
    both = P.dd_solve_batch(ds, ctx, [3, 3], loads, mode=P.DD_SEARCH_KNNG, seed=9, max_iter=100)
    for a, b in zip(alone, both):
        assert a.converged and a.iters >= 2
        assert a.d2_pd[-1] <= a.d2_pd[0]
        assert a.iters == b.iters
        assert np.array_equal(a.idx, b.idx) and np.array_equal(a.u, b.u)
    # the exact-search solve from the same association for scale
    ex = P.dd_solve(ds, ctx, 3, loads[0], seed=9)
    print(f"graph solve d2 {alone[0].d2_pd[-1]:.4e} ({alone[0].iters} it), exact {ex.d2_pd[-1]:.4e} ({ex.iters} it)")
    assert alone[0].d2_pd[-1] <= 2.0 * ex.d2_pd[-1]


def test_graph_errors(ctx):
    data = I.make_dataset(500, I.LINEAR, seed=48)
    with pytest.raises(P.DDError):       # the graph needs the two-level tree
        P.dd_load_dataset(ctx, data, C, ann_nlist=16, ann_levels=1, knn_k=8)
    with pytest.raises(P.DDError):       # k at most 128
        P.dd_load_dataset(ctx, data, C, ann_nlist=16, ann_levels=2, knn_k=129)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=16, ann_levels=2)
    try:
        y = I.make_states(4, I.LINEAR, seed=1, spread=0.1)
        with pytest.raises(P.DDError):   # no graph built
            walk(ctx, ds, y)
        with pytest.raises(P.DDError):
            P.dd_solver_create(ds, ctx, 2, I.load_case("tension", 1e-3), mode=P.DD_SEARCH_KNNG)
    finally:
        P.dd_free_dataset(ds)
