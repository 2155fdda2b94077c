"""Batched steps captured as CUDA graphs: a replayed step gives the same
results as the eager step, and a graph is recaptured when a workspace it
uses has moved."""
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


def run_batch(ds, ctx, n_els, loads, between=None, **kw):
    """Step solvers created for n_els/loads together until all are done;
    returns (results, infos per step).  between(step) runs after each step."""
    svs = [P.dd_solver_create(ds, ctx, k, L, **kw) for k, L in zip(n_els, loads)]
    steps = []
    try:
        while True:
            act = [s for s in svs if not P.dd_solver_done(s)]
            if not act:
                break
            steps.append(P.dd_solvers_step(act, ctx))
            if between:
                between(len(steps))
        return [P.dd_solver_result(s, ctx) for s in svs], steps
    finally:
        for s in svs:
            P.dd_solver_free(s)


@pytest.mark.parametrize("mode", [P.DD_SEARCH_EXACT_FP32, P.DD_SEARCH_EXACT_TC])
def test_replayed_steps_equal_eager_single_solve(ctx, mode):
    """One solve through dd_solvers_step (graph from the second step on) is bit
    for bit the stand-alone eager dd_solve: same kernels, same order."""
    data = I.make_dataset(15000, I.NONLINEAR, seed=31)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    L = I.load_case("bending", 1e-3)
    try:
        ref = P.dd_solve(ds, ctx, 4, L, mode=mode, seed=2)
        (got,), steps = run_batch(ds, ctx, [4], [L], mode=mode, seed=2)
    finally:
        P.dd_free_dataset(ds)
    assert got.iters == ref.iters >= 3
    assert [s[0].graph for s in steps[:2]] == [0, 1]
    assert all(s[0].graph == 1 for s in steps[1:])
    assert np.array_equal(got.idx, ref.idx)
    assert np.array_equal(got.u, ref.u)
    assert np.array_equal(got.d2_pd, ref.d2_pd)
    assert np.array_equal(got.cg_iters, ref.cg_iters)


def test_replay_counts_launches(ctx):
    """The launch counter grows by the kernels of the captured step on every
    replay, as much as the eager first step of the same list launches."""
    data = I.make_dataset(6000, I.LINEAR, seed=32)
    ds = P.dd_load_dataset(ctx, data, C)
    loads = [I.load_case("tension", 1e-3), I.load_case("shear", 1e-3)]
    svs = [P.dd_solver_create(ds, ctx, k, L, seed=4, max_iter=6) for k, L in zip([3, 4], loads)]
    per_step, graph = [], []
    try:
        while not any(P.dd_solver_done(s) for s in svs):
            c0 = P.dd_launch_count(ctx)
            infos = P.dd_solvers_step(svs, ctx)
            per_step.append(P.dd_launch_count(ctx) - c0)
            graph.append(infos[0].graph)
    finally:
        for s in svs:
            P.dd_solver_free(s)
        P.dd_free_dataset(ds)
    assert len(per_step) >= 3 and graph[:3] == [0, 1, 1]
    assert per_step[0] > 0
    assert per_step == [per_step[0]] * len(per_step)   # eager step 1 == every replay


def test_recapture_after_workspace_moves(ctx):
    """A large projection between steps regrows the search workspaces the
    captured graph points into; the next step must capture again and the
    solves must still match their stand-alone results."""
    data = I.make_dataset(10000, I.NONLINEAR, seed=33)
    ds = P.dd_load_dataset(ctx, data, C)
    loads = [I.load_case("torsion", 1e-3), I.load_case("tension", 2e-3)]
    big = torch.from_numpy(I.make_states(200_000, I.NONLINEAR, seed=9, spread=0.05)).cuda()
    idx = torch.empty(len(big), dtype=torch.int32, device="cuda")
    d2 = torch.empty(len(big), dtype=torch.float64, device="cuda")

    def grow(k):
        if k == 3:
            P.dd_project_nearest(ds, ctx, big, idx, d2)
            torch.cuda.synchronize()

    try:
        alone = [P.dd_solve(ds, ctx, k, L, seed=7) for k, L in zip([3, 5], loads)]
        mixed, steps = run_batch(ds, ctx, [3, 5], loads, between=grow, seed=7)
    finally:
        P.dd_free_dataset(ds)
    assert len(steps) > 4
    for a, b in zip(mixed, alone):
        assert a.iters == b.iters
        assert np.array_equal(a.idx, b.idx)
        assert np.allclose(a.u, b.u, rtol=0, atol=1e-9 * np.abs(b.u).max())
