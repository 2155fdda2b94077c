"""GPU tensor-core (tcgen05) exact projection and DD solve against the oracle."""
import numpy as np
import pytest

import dd_inputs as I
from gpu_util import assert_nn_parity, oracle_nn
from oracle import dd as odd

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


def project(ctx, ds, y, certify=True, terms=0, d2nd=None):
    m = len(y)
    yd = torch.from_numpy(y).cuda()
    idx = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
    st = P.dd_project_nearest(ds, ctx, yd, idx, d2, mode=P.DD_SEARCH_EXACT_TC, certify=certify, tc_terms=terms,
                              d2nd=d2nd)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy(), st


@pytest.mark.parametrize("terms", [3, 2])
@pytest.mark.parametrize("N", [1, 100, 128, 129, 4097, 30000])
def test_tc_certified_ragged(ctx, N, terms):
    """Three FP16 products per distance (split query and data) and two
    (split data, single FP16 query, window widened by the query's rounding
    term): both the exact nearest point, and the second-distance bound below
    the true second distance."""
    data = I.make_dataset(N, I.NONLINEAR, seed=N + 1)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    try:
        for m, spread in ((1, 0.05), (127, 0.02), (129, 0.3), (3000, 2.0)):
            y = I.make_states(m, I.NONLINEAR, seed=7 * m + N, spread=spread)
            d2nd = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
            idx, d2, st = project(ctx, ds, y, terms=terms, d2nd=d2nd)
            assert_nn_parity(idx, d2, data, y, C)
            if N > 1:
                _, _, b2 = oracle_nn(data, y, C)
                assert np.all(d2nd.cpu().numpy() <= b2 * (1 + 1e-9))
    finally:
        P.dd_free_dataset(ds)


def test_tc_planted_and_ties(ctx):
    data = I.make_dataset(9000, I.LINEAR, seed=5)
    data[8000] = data[3]
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    try:
        y = data[[3, 8000, 8999, 0, 4096]].astype(np.float64)
        idx, d2, _ = project(ctx, ds, y)
        assert idx.tolist() == [3, 3, 8999, 0, 4096]
        assert np.all(d2 == 0.0)
    finally:
        P.dd_free_dataset(ds)


def test_tc_topk_mode_reports_accuracy(ctx):
    """Single FP16 term, best 8 scores rescored in FP64 (no certificate):
    most queries exact, every answer one of the near neighbours."""
    data = I.make_dataset(50000, I.LINEAR, seed=2)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    try:
        y = I.make_states(4096, I.LINEAR, seed=3, spread=0.05)
        idx, d2, st = project(ctx, ds, y, certify=False)
        i1, b1, b2 = oracle_nn(data, y, C)
        exact = np.mean(idx == i1)
        rel = (d2 - b1) / b1
        print(f"top-k FP16: exact {exact:.4f}, max rel distance excess {rel.max():.3e}")
        assert exact >= 0.9
        assert np.all(rel >= -1e-12)
        # the answer's FP64 distance is its true distance
        from oracle import metric
        assert np.allclose(metric.local_d2(y, data[idx].astype(np.float64), C), d2, rtol=1e-10)
    finally:
        P.dd_free_dataset(ds)


@pytest.mark.parametrize("terms", [0, 3, 2])
def test_tc_full_size_sampled(ctx, terms):
    """32 768 queries x 10^6 points (the 16^3 workload's sizes): the tuned
    variant (0), three and two FP16 products per distance, on sampled
    queries against the oracle."""
    N, m = 1_000_000, 32768
    raw = torch.empty((N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, I.LINEAR, C, seed=0)
    ds = P.dd_load_dataset(ctx, raw, C, borrow=True, build_fp16=True)
    try:
        y = I.make_states(m, I.LINEAR, seed=5, spread=0.05)
        project(ctx, ds, y, terms=terms)                     # tunes / warms up
        idx, d2, st = project(ctx, ds, y, terms=terms)
        sample = np.random.default_rng(1).choice(m, 192, replace=False)
        data = I.make_dataset(N, I.LINEAR, seed=0)
        assert_nn_parity(idx[sample], d2[sample], data, y[sample], C)
        print(f"terms {terms}: uncertified {st.uncertified} of {m}, scan {st.scan_ms:.3f} ms, call {st.ms:.3f} ms")
        assert st.uncertified <= m // 50
    finally:
        P.dd_free_dataset(ds)


def test_tc_solve_matches_oracle(ctx):
    W = I.WORKLOADS["cube4_N1e4_exact_fp64"]
    data = I.make_dataset(W.N, W.law, seed=W.seed)
    load = I.load_case(*W.loads[0])
    init = I.initial_association(W.m, W.N, seed=W.seed)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    try:
        r = P.dd_solve(ds, ctx, W.n_el, load, mode=P.DD_SEARCH_EXACT_TC, init_idx=init)
    finally:
        P.dd_free_dataset(ds)
    o = odd.DDProblem(data, C, W.n_el, load).solve(init)
    assert r.converged and r.iters == o.iters
    assert np.array_equal(r.idx, o.idx)
    assert np.allclose(r.u, o.u, rtol=0, atol=1e-6 * np.abs(o.u).max())


def test_stepwise_solver_equals_solve(ctx):
    data = I.make_dataset(5000, I.LINEAR, seed=4)
    load = I.load_case("bending", 1e-3)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    try:
        r = P.dd_solve(ds, ctx, 3, load, mode=P.DD_SEARCH_EXACT_TC, seed=3)
        sv = P.dd_solver_create(ds, ctx, 3, load, mode=P.DD_SEARCH_EXACT_TC, seed=3)
        n0 = P.dd_launch_count(ctx)
        infos = []
        while not P.dd_solver_done(sv):
            infos.append(P.dd_solver_step(sv, ctx))
        assert P.dd_launch_count(ctx) > n0
        r2 = P.dd_solver_result(sv, ctx)
        P.dd_solver_free(sv)
    finally:
        P.dd_free_dataset(ds)
    assert r2.iters == r.iters == len(infos) and r2.converged
    assert np.array_equal(r2.idx, r.idx) and np.array_equal(r2.u, r.u)
    assert infos[-1].changed == 0 and infos[-1].done
