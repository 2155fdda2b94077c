"""Serving loop: requests admitted as memory frees up, stepped together, each
result the same as the solve run alone."""
import time

import numpy as np
import pytest

import dd_inputs as I

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


def requests(k, seed=0):
    out = []
    for r in range(k):
        edge = 2 + (r * 7) % 4
        out.append((edge, I.random_load(seed, r, 1e-4, 2e-3), 100 + r))
    return out


@pytest.mark.parametrize("budget", [0, 1])
def test_served_results_equal_standalone(ctx, budget):
    data = I.make_dataset(15000, I.NONLINEAR, seed=31)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=32, seed=4)
    reqs = requests(7)
    kw = dict(mode=P.DD_SEARCH_ANN, f_d0=0.0, f_d_final=0.6, ramp_iters=5, max_iter=80)
    try:
        alone = [P.dd_solve(ds, ctx, e, L, seed=sd, **kw) for e, L, sd in reqs]
        # budget 1 byte: one solve at a time (admission waits for room)
        srv = P.dd_server_start(ds, ctx, state_budget=budget, **kw)
        tickets = []
        for i, (e, L, sd) in enumerate(reqs):
            tickets.append(P.dd_server_submit(srv, e, L, seed=sd))
            if i % 3 == 1:
                time.sleep(0.02)     # arrivals while others are on the GPU
        got = [P.dd_server_poll(srv, ctx, t, timeout_s=120.0) for t in tickets]
        st = P.dd_server_get_stats(srv)
        P.dd_server_stop(srv)
    finally:
        P.dd_free_dataset(ds)
    assert st.completed == len(reqs)
    if budget:
        assert st.max_active == 1
    else:
        assert st.max_active > 1
    for (res, lat), a in zip(got, alone):
        assert lat > 0
        assert res.iters == a.iters and np.array_equal(res.idx, a.idx)
        assert np.allclose(res.u, a.u, rtol=0, atol=1e-9 * np.abs(a.u).max())


def test_bad_request_fails_alone(ctx):
    data = I.make_dataset(3000, I.LINEAR, seed=32)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        srv = P.dd_server_start(ds, ctx)
        good = P.dd_server_submit(srv, 2, I.load_case("tension", 1e-3), seed=1)
        bad = P.dd_server_submit(srv, 0, I.load_case("tension", 1e-3), seed=1)
        r_good = P.dd_server_poll(srv, ctx, good, timeout_s=60.0)
        with pytest.raises(P.DDError):
            P.dd_server_poll(srv, ctx, bad, timeout_s=60.0)
        P.dd_server_stop(srv)
    finally:
        P.dd_free_dataset(ds)
    assert r_good[0].converged
