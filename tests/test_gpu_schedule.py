"""Accuracy schedules of Eq. (11) on the GPU: the global-distance rule follows
the oracle's rule on the solve's own distance history, its limit tau = 1 and
the local rule's limit tau = 0 are the plain ramp bit for bit, and the local
rule gives the same solves stepped alone, batched and replayed as a graph."""
import numpy as np
import pytest

import dd_inputs as I
from oracle import schedule as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_00357_gb300 as P  # noqa: E402

C = I.isotropic_C()
KW = dict(mode=P.DD_SEARCH_ANN, f_d0=0.1, f_d_final=0.7, ramp_iters=6, max_iter=60)


@pytest.fixture(scope="module")
def env():
    P.build()
    ctx = P.dd_create(0)
    data = I.make_dataset(40000, I.NONLINEAR, seed=61)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=256, ann_levels=2, seed=5)
    yield ctx, ds
    P.dd_free_dataset(ds)
    P.dd_destroy(ctx)


def stepped(ds, ctx, n_el, load, seed, **kw):
    sv = P.dd_solver_create(ds, ctx, n_el, load, seed=seed, **kw)
    infos = []
    try:
        while not P.dd_solver_done(sv):
            infos.append(P.dd_solver_step(sv, ctx))
        return P.dd_solver_result(sv, ctx), infos
    finally:
        P.dd_solver_free(sv)


def same(a, b):
    return a.iters == b.iters and np.array_equal(a.idx, b.idx) and np.array_equal(a.u, b.u)


@pytest.mark.parametrize("tau", [0.02, 0.2])
def test_global_rule_follows_the_oracle(env, tau):
    ctx, ds = env
    r, infos = stepped(ds, ctx, 4, I.load_case("torsion", 1e-3), 3, fd_rule=1, fd_tau=tau, **KW)
    f_ref = S.global_rule(KW["f_d0"], KW["f_d_final"], KW["ramp_iters"], tau,
                          [i.d2_pc for i in infos], [i.d2_pd for i in infos])
    got = np.array([i.f_d for i in infos], np.float32)
    assert np.array_equal(got, np.array(f_ref[:len(infos)], np.float32))
    print(f"tau={tau}: f_d {got.tolist()}, {r.iters} iterations")
    assert r.converged


def test_global_rule_tau_one_is_the_ramp(env):
    ctx, ds = env
    L = I.load_case("tension", 1e-3)
    a = P.dd_solve(ds, ctx, 4, L, seed=5, **KW)
    b = P.dd_solve(ds, ctx, 4, L, seed=5, fd_rule=1, fd_tau=1.0, **KW)
    assert same(a, b)


def test_local_rule_tau_zero_is_the_ramp(env):
    ctx, ds = env
    L = I.load_case("shear", 1e-3)
    a = P.dd_solve(ds, ctx, 4, L, seed=6, **KW)
    b = P.dd_solve(ds, ctx, 4, L, seed=6, fd_rule=2, fd_tau=0.0, **KW)
    assert same(a, b)


def test_local_rule_alone_batched_and_replayed(env):
    """The local rule fills every point's f_d from the solve's own distances:
    the same in a stand-alone solve, in a batched step and in its graph."""
    ctx, ds = env
    loads = [I.load_case("tension", 1e-3), I.load_case("bending", 1e-3)]
    kw = dict(fd_rule=2, fd_tau=1.0, **KW)
    alone = [P.dd_solve(ds, ctx, 4, L, seed=7, **kw) for L in loads]
    svs = [P.dd_solver_create(ds, ctx, 4, L, seed=7, **kw) for L in loads]
    graph = []
    try:
        while not all(P.dd_solver_done(s) for s in svs):
            act = [s for s in svs if not P.dd_solver_done(s)]
            graph.append(P.dd_solvers_step(act, ctx)[0].graph)
        both = [P.dd_solver_result(s, ctx) for s in svs]
    finally:
        for s in svs:
            P.dd_solver_free(s)
    assert sum(graph) > 0
    for a, b in zip(alone, both):
        assert same(a, b)
    # the rule acts: the plain ramp takes another path
    ramp = P.dd_solve(ds, ctx, 4, loads[0], seed=7, **KW)
    assert not same(alone[0], ramp)
