"""GPU DD solve (Eq. 8) against the FP64 oracle's direct-solve iteration."""
import numpy as np
import pytest

import dd_inputs as I
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


def compare(r, o, rtol_u=1e-6):
    assert r.converged == o.converged
    assert r.iters == o.iters
    assert np.array_equal(r.idx, o.idx)
    scale = np.abs(o.u).max()
    assert np.allclose(r.u, o.u, rtol=0, atol=rtol_u * scale)
    assert np.allclose(r.eps, o.eps, rtol=0, atol=rtol_u * np.abs(o.eps).max())
    assert np.allclose(r.sig, o.sig, rtol=0, atol=rtol_u * np.abs(o.sig).max())
    assert np.allclose(r.d2_pd, o.d2_after_pd, rtol=1e-6)
    assert np.allclose(r.d2_pc, o.d2_after_pc, rtol=1e-6)


def test_cube4_N1e4_exact_matches_oracle(ctx):
    """4^3 cube, N = 10^4 linear data, tension 1e-3, seed 0: iterate until the
    association stops changing."""
    W = I.WORKLOADS["cube4_N1e4_exact_fp64"]
    data = I.make_dataset(W.N, W.law, seed=W.seed)
    load = I.load_case(*W.loads[0])
    init = I.initial_association(W.m, W.N, seed=W.seed)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r = P.dd_solve(ds, ctx, W.n_el, load, init_idx=init)
    finally:
        P.dd_free_dataset(ds)
    o = odd.DDProblem(data, C, W.n_el, load).solve(init)
    compare(r, o)
    assert r.converged


@pytest.mark.parametrize("case", ["shear", "bending", "torsion"])
def test_load_cases_match_oracle(ctx, case):
    data = I.make_dataset(4000, I.NONLINEAR, seed=2)
    load = I.load_case(case, 1e-3)
    init = I.initial_association(8 * 27, len(data), seed=4)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r = P.dd_solve(ds, ctx, 3, load, init_idx=init)
    finally:
        P.dd_free_dataset(ds)
    o = odd.DDProblem(data, C, 3, load).solve(init)
    compare(r, o)


def test_monotone_distance_and_library_init(ctx):
    data = I.make_dataset(6000, I.LINEAR, seed=9)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r = P.dd_solve(ds, ctx, 3, I.load_case("tension", 1e-3), seed=0)
    finally:
        P.dd_free_dataset(ds)
    # the library's own initial association is the same SplitMix64 draw
    o = odd.DDProblem(data, C, 3, I.load_case("tension", 1e-3)).solve(I.initial_association(216, 6000, seed=0))
    compare(r, o)
    tol = 1e-12 * r.d2_pc[0]
    assert np.all(r.d2_pd <= r.d2_pc + tol) and np.all(r.d2_pc[1:] <= r.d2_pd[:-1] + tol)


def test_mixed_precision_cg_matches_fp64_cg(ctx):
    """FP32 Krylov steps inside FP64 refinement meet the same FP64 residual
    test as the FP64 CG: same associations, displacements within 1e-9."""
    data = I.make_dataset(6000, I.NONLINEAR, seed=5)
    load = I.load_case("torsion", 1e-3)
    init = I.initial_association(8 * 64, len(data), seed=5)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r64 = P.dd_solve(ds, ctx, 4, load, init_idx=init, cg_mode=1)
        rmx = P.dd_solve(ds, ctx, 4, load, init_idx=init, cg_mode=0)
    finally:
        P.dd_free_dataset(ds)
    assert r64.iters == rmx.iters and np.array_equal(r64.idx, rmx.idx)
    assert np.allclose(rmx.u, r64.u, rtol=0, atol=1e-9 * np.abs(r64.u).max())
    assert np.allclose(rmx.eta, r64.eta, rtol=0, atol=1e-9 * np.abs(r64.eta).max() + 1e-300)


@pytest.mark.parametrize("n_el,deg", [(3, 0.1), (4, 0.1), (5, 2.0), (6, 0.1)])
def test_top_rotation_matches_oracle(ctx, n_el, deg):
    """The paper's own boundary-value problem: the top face turned by a
    prescribed angle about the vertical axis (non-homogeneous Dirichlet
    values for u, homogeneous for eta), bottom clamped.  Meshes with even and
    odd element counts (both multigrid coarsenings with a fixed top)."""
    data = I.make_dataset(5000, I.LINEAR, seed=11)
    load = I.top_rotation(deg)
    init = I.initial_association(8 * n_el ** 3, len(data), seed=12)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r = P.dd_solve(ds, ctx, n_el, load, init_idx=init)
    finally:
        P.dd_free_dataset(ds)
    o = odd.DDProblem(data, C, n_el, load).solve(init)
    compare(r, o)


def test_top_rotation_mixed_cg_matches_fp64_cg(ctx):
    data = I.make_dataset(6000, I.NONLINEAR, seed=13)
    load = I.top_rotation(0.5)
    init = I.initial_association(8 * 64, len(data), seed=14)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        r64 = P.dd_solve(ds, ctx, 4, load, init_idx=init, cg_mode=1)
        rmx = P.dd_solve(ds, ctx, 4, load, init_idx=init, cg_mode=0)
    finally:
        P.dd_free_dataset(ds)
    assert r64.iters == rmx.iters and np.array_equal(r64.idx, rmx.idx)
    assert np.allclose(rmx.u, r64.u, rtol=0, atol=1e-9 * np.abs(r64.u).max())


def test_rotation_with_traction_is_rejected(ctx):
    data = I.make_dataset(500, I.LINEAR, seed=1)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        bad = I.Load(t0=(0.0, 0.0, 1e-3), rot_z=0.01)
        with pytest.raises(P.DDError):
            P.dd_solve(ds, ctx, 3, bad)
    finally:
        P.dd_free_dataset(ds)


@pytest.fixture(scope="module")
def cfg1_oracle():
    """The exact DD solve of the 16^3 cube on 10^6 linear-law points (Eq. 8
    with the brute-force P_D and the direct P_C), seed 0, tension 1e-3:
    minutes of host work, done once for the modes below."""
    W = I.WORKLOADS["cube16_N1e6_exact"]
    data = I.make_dataset(W.N, W.law, seed=W.seed)
    load = I.load_case(*W.loads[0])
    init = I.initial_association(W.m, W.N, seed=W.seed)
    o = odd.DDProblem(data, C, W.n_el, load).solve(init)
    return W, data, load, init, o


@pytest.mark.parametrize("mode", ["fp32", "tc"])
def test_cube16_N1e6_exact_solve_matches_oracle(ctx, cfg1_oracle, mode):
    """The 16^3 / 10^6-point workload end to end: the certified FP32 scan and
    the certified split-FP16 tensor-core scan give the oracle's associations
    at every iteration and its displacements within 1e-6."""
    W, data, load, init, o = cfg1_oracle
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=(mode == "tc"))
    try:
        md = P.DD_SEARCH_EXACT_TC if mode == "tc" else P.DD_SEARCH_EXACT_FP32
        r = P.dd_solve(ds, ctx, W.n_el, load, mode=md, init_idx=init, max_iter=200)
    finally:
        P.dd_free_dataset(ds)
    print(f"cube16 N=1e6 {mode}: {r.iters} iterations (oracle {o.iters}), "
          f"{r.uncertified} FP64 re-searches")
    compare(r, o)
    assert r.converged
