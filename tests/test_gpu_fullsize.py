"""Full-size sampled parity: the 10^8-point data set of the 32^3 workload,
all 262 144 material-point queries through the kernels as benchmarked, a
sample checked against the oracle's streaming brute force (which regenerates
the data set itself from the seed, chunk by chunk)."""
import numpy as np
import pytest

import dd_inputs as I
from oracle import metric, nn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_00357_gb300 as P  # noqa: E402

C = I.isotropic_C()
W = I.WORKLOADS["cube32_N1e8_ann"]


@pytest.fixture(scope="module")
def big():
    P.build()
    ctx = P.dd_create(0)
    raw = torch.empty((W.N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, W.law, C, seed=W.seed)
    # 512 cells of 512 leaves, about 380 points per leaf (the benchmark's
    # leaf size at 10^9 points)
    ds = P.dd_load_dataset(ctx, raw, C, borrow=True, build_fp16=True, ann_nlist=1 << 18, ann_levels=2, seed=1)
    y = I.make_states(W.m, W.law, seed=41, spread=0.02)
    sample = np.random.default_rng(4).choice(W.m, 12, replace=False)
    oi, od = nn.nn_stream(W.law, W.seed, W.N, C, metric.to_z(y[sample], C))
    yield ctx, ds, y, sample, oi, od
    P.dd_free_dataset(ds)
    del raw
    P.dd_destroy(ctx)


def run(ctx, ds, y, **kw):
    yd = torch.from_numpy(y).cuda()
    idx = torch.empty(len(y), dtype=torch.int32, device="cuda")
    d2 = torch.empty(len(y), dtype=torch.float64, device="cuda")
    st = P.dd_project_nearest(ds, ctx, yd, idx, d2, **kw)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy(), st


def test_exact_fp32_full_size(big):
    ctx, ds, y, sample, oi, od = big
    idx, d2, st = run(ctx, ds, y, mode=P.DD_SEARCH_EXACT_FP32)
    assert np.array_equal(idx[sample], oi)
    assert np.allclose(d2[sample], 2 * od, rtol=1e-9)
    print(f"exact N=1e8, m={len(y)}: uncertified {st.uncertified}, scan {st.scan_ms:.1f} ms")


def test_ann_tree_fd_one_full_size(big):
    ctx, ds, y, sample, oi, od = big
    prev = np.random.default_rng(5).integers(0, W.N, len(sample)).astype(np.int32)
    idx, d2, st = run(ctx, ds, np.ascontiguousarray(y[sample]), mode=P.DD_SEARCH_ANN, f_d=1.0,
                      prev_idx=torch.from_numpy(prev).cuda())
    assert np.array_equal(idx, oi)
    assert np.allclose(d2, 2 * od, rtol=1e-9)


@pytest.fixture(scope="module")
def exact_solve(big):
    ctx, ds, y, sample, oi, od = big
    return P.dd_solve(ds, ctx, W.n_el, I.load_case("tension", 1e-3), mode=P.DD_SEARCH_EXACT_TC, seed=W.seed,
                      max_iter=60)


def test_ann_solve_within_1e3_of_exact_full_size(big, exact_solve):
    """The DD solution driven by the approximate search (tree, f_d from 0.3
    to 0.8 over 5 iterations, the benchmark schedule) ends at most 1e-3 relative above, in global
    distance (Eq. 2) of the solution driven by the certified exact search, on
    the 32^3 cube with the 10^8-point data set, from the same initial
    association."""
    ctx, ds, y, sample, oi, od = big
    L = I.load_case("tension", 1e-3)
    exact = exact_solve
    ann = P.dd_solve(ds, ctx, W.n_el, L, mode=P.DD_SEARCH_ANN, f_d0=0.3, f_d_final=0.8, ramp_iters=5,
                     seed=W.seed, max_iter=60)
    de, da = float(exact.d2_pd[-1]), float(ann.d2_pd[-1])
    print(f"exact: {exact.iters} iterations, d2 {de:.6e}; approximate: {ann.iters} iterations, d2 {da:.6e}, "
          f"relative difference {abs(da - de) / de:.2e}")
    assert exact.converged and ann.converged
    # the DD iteration is non-convex: a different search may end at a lower
    # fixed point, which is no loss of accuracy; the bar is 1e-3 above
    assert da <= (1 + 1e-3) * de


def test_graph_solve_full_size(big, exact_solve):
    """The DD solve driven by the greedy walk in the k-NN graph (Sec. 4.4;
    k = 128 built at f_d = 0.8, at most 2 node changes per walk) on the 32^3
    cube with 10^8 points ends within 1 % above the certified exact-search
    solution, from the same initial association (bounded walks may end at a
    better fixed point), and the walk evaluates a few hundred neighbours per
    query, not the millions of points of a scan."""
    ctx, ds, y, sample, oi, od = big
    Wg = I.WORKLOADS["cube32_N1e8_knng"]
    raw = torch.empty((W.N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, W.law, C, seed=W.seed)
    dg = P.dd_load_dataset(ctx, raw, C, borrow=True, ann_nlist=1 << 17, ann_levels=2, seed=1,
                           knn_k=Wg.extra["knn_k"], knn_fd=Wg.extra["knn_fd"])
    try:
        g = P.dd_solve(dg, ctx, W.n_el, I.load_case("tension", 1e-3), mode=P.DD_SEARCH_KNNG, f_s=Wg.extra["f_s"],
                       seed=W.seed, max_iter=200)
    finally:
        P.dd_free_dataset(dg)
        del raw
    de, dgr = float(exact_solve.d2_pd[-1]), float(g.d2_pd[-1])
    print(f"exact d2 {de:.6e}; graph walk: {g.iters} iterations, d2 {dgr:.6e}, relative {(dgr - de) / de:+.2e}, "
          f"{g.distances / W.m / g.iters:.0f} distances per query and iteration")
    assert g.converged and dgr <= 1.01 * de
    assert g.distances / W.m / g.iters < 1000


def test_paper_problem_ann_within_1e3_of_exact():
    """The paper's own problem (Sec. 3.1: 20^3 cube, top face turned by 2
    degrees, data from the law of Eq. (9) with strains in [-0.025, 0.025],
    the metric from the data's principal components) with 10^8 points: the
    DD solution driven by the approximate search (f_d 0.4 -> 0.8 over 5
    iterations) ends at most 1e-3 relative above, in global distance (Eq. 2), the one
    driven by the certified exact search, from the same initial association;
    the tensor-core exact search is checked on a sample of the final states
    against the oracle's streaming brute force."""
    Wr = I.WORKLOADS["cube20_N1e8_rot2_ann"]
    fd0, fdf, ramp = Wr.extra["schedule"]
    ctx = P.dd_create(0)
    raw = torch.empty((Wr.N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, Wr.law, I.isotropic_C(Wr.law.E, Wr.law.nu), seed=Wr.seed)
    Cp = P.dd_pca_metric(ctx, raw)          # the data-derived metric of Sec. 3.1
    ds = P.dd_load_dataset(ctx, raw, Cp, borrow=True, build_fp16=True, ann_nlist=1 << 18, ann_levels=2, seed=1)
    try:
        L = I.load_case(*Wr.loads[0])
        init = I.initial_association(Wr.m, Wr.N, seed=Wr.seed)
        exact = P.dd_solve(ds, ctx, Wr.n_el, L, mode=P.DD_SEARCH_EXACT_TC, init_idx=init, max_iter=60)
        ann = P.dd_solve(ds, ctx, Wr.n_el, L, mode=P.DD_SEARCH_ANN, f_d0=fd0, f_d_final=fdf, ramp_iters=ramp,
                         init_idx=init, max_iter=60)
        y = np.concatenate([exact.eps, exact.sig], axis=1)
        sample = np.random.default_rng(5).choice(Wr.m, 8, replace=False)
        oi, od = nn.nn_stream(Wr.law, Wr.seed, Wr.N, Cp, metric.to_z(y[sample], Cp))
        got = raw[torch.from_numpy(exact.idx[sample].astype(np.int64)).cuda()].cpu().numpy().astype(np.float64)
    finally:
        P.dd_free_dataset(ds)
        del raw
        P.dd_destroy(ctx)
    de, da = float(exact.d2_pd[-1]), float(ann.d2_pd[-1])
    print(f"exact: {exact.iters} iterations, d2 {de:.6e}; approximate: {ann.iters} iterations, d2 {da:.6e}, "
          f"relative difference {abs(da - de) / de:+.2e}")
    assert exact.converged and ann.converged
    # the DD iteration is non-convex: a different search may end at a lower
    # fixed point, which is no loss of accuracy; the bar is 1e-3 above
    assert da <= (1 + 1e-3) * de
    # at convergence the final association is the exact projection of the
    # final P_C states (equal index, or an FP64 near-tie within 1e-6)
    dg = ((metric.to_z(got, Cp) - metric.to_z(y[sample], Cp)) ** 2).sum(1)
    assert np.all((exact.idx[sample] == oi) | (np.abs(dg - od) <= 1e-6 * od))
    # the top nodes carry the prescribed turn u = (R - I)(x - x_c, y - y_c, 0)
    n = Wr.n_el + 1
    top = exact.u.reshape(n, n, n, 3)[-1]                  # node (i, j, k): i fastest
    x = np.linspace(0.0, 1.0, n)[None, :] - 0.5
    yy = np.linspace(0.0, 1.0, n)[:, None] - 0.5
    c, s_ = np.cos(np.radians(2.0)), np.sin(np.radians(2.0))
    assert np.allclose(top[..., 0], (c - 1) * x - s_ * yy, rtol=0, atol=1e-15)
    assert np.allclose(top[..., 1], s_ * x + (c - 1) * yy, rtol=0, atol=1e-15)
    assert np.all(top[..., 2] == 0.0)
