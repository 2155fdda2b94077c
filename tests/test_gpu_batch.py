"""Several solves stepped together (one CG launch, one search) give the same
results as each solve alone."""
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


def same(a, b, tol=1e-9):
    assert a.iters == b.iters and a.converged == b.converged
    assert np.array_equal(a.idx, b.idx)
    assert np.allclose(a.u, b.u, rtol=0, atol=tol * np.abs(b.u).max())
    assert np.allclose(a.d2_pd, b.d2_pd, rtol=1e-9)


@pytest.mark.parametrize("mode", [P.DD_SEARCH_EXACT_FP32, P.DD_SEARCH_EXACT_TC])
def test_batch_of_uneven_meshes_equals_single_solves(ctx, mode):
    data = I.make_dataset(12000, I.NONLINEAR, seed=21)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    n_els = [2, 5, 3, 4]
    loads = [I.load_case(n, 1e-3) for n in ("tension", "shear", "bending", "torsion")]
    try:
        alone = [P.dd_solve(ds, ctx, k, L, mode=mode, seed=1) for k, L in zip(n_els, loads)]
        mixed = P.dd_solve_batch(ds, ctx, n_els, loads, mode=mode, seed=1)
    finally:
        P.dd_free_dataset(ds)
    for a, b in zip(mixed, alone):
        same(a, b)


def test_batch_ann_equals_single_solves(ctx):
    data = I.make_dataset(20000, I.NONLINEAR, seed=22)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=48, seed=2)
    n_els = [3, 4]
    loads = [I.load_case("torsion", 1e-3), I.load_case("tension", 2e-3)]
    kw = dict(mode=P.DD_SEARCH_ANN, f_d0=0.0, f_d_final=0.6, ramp_iters=6, seed=3, max_iter=60)
    try:
        alone = [P.dd_solve(ds, ctx, k, L, **kw) for k, L in zip(n_els, loads)]
        mixed = P.dd_solve_batch(ds, ctx, n_els, loads, **kw)
    finally:
        P.dd_free_dataset(ds)
    for a, b in zip(mixed, alone):
        same(a, b)


def test_solvers_step_staggered(ctx):
    """Solves that start at different times (as in a serving loop) still
    reproduce their stand-alone results."""
    data = I.make_dataset(8000, I.LINEAR, seed=23)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        L1, L2 = I.load_case("tension", 1e-3), I.load_case("torsion", 1e-3)
        r1 = P.dd_solve(ds, ctx, 3, L1, seed=5)
        r2 = P.dd_solve(ds, ctx, 4, L2, seed=6)
        a = P.dd_solver_create(ds, ctx, 3, L1, seed=5)
        b = P.dd_solver_create(ds, ctx, 4, L2, seed=6)
        P.dd_solver_step(a, ctx)                      # a runs alone first
        while not (P.dd_solver_done(a) and P.dd_solver_done(b)):
            act = [s for s in (a, b) if not P.dd_solver_done(s)]
            P.dd_solvers_step(act, ctx)
        ra, rb = P.dd_solver_result(a, ctx), P.dd_solver_result(b, ctx)
        P.dd_solver_free(a)
        P.dd_solver_free(b)
    finally:
        P.dd_free_dataset(ds)
    same(ra, r1)
    same(rb, r2)
