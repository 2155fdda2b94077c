"""The k nearest data points through dd_project_nearest (topk_out): exact
modes against the oracle's sorted brute force (Eq. 7 for the k best), and
the uncertified tensor-core top-k form with its error reported."""
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


@pytest.fixture(scope="module")
def ctx():
    P.build()
    c = P.dd_create(0)
    yield c
    P.dd_destroy(c)


_ORACLE = {}


def oracle_topk(data, y, k):
    """The oracle's sorted brute force, computed once per query set."""
    key = (len(data), len(y), float(y[0, 0]))
    if key not in _ORACLE or _ORACLE[key][0].shape[1] < k:
        _ORACLE[key] = nn.nn_topk(metric.to_z(data.astype(np.float64), C), metric.to_z(y, C), max(k, 8))
    oi, od = _ORACLE[key]
    return oi[:, :k], od[:, :k]


@pytest.fixture(scope="module")
def dset(ctx):
    data = I.make_dataset(23457, I.NONLINEAR, seed=41)      # ragged: not a multiple of any tile
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    yield data, ds
    P.dd_free_dataset(ds)


def topk(ctx, ds, y, k, mode, certify=True, device=False):
    m = len(y)
    if device:
        yy = torch.from_numpy(y).cuda()
        idx = torch.full((m,), -7, dtype=torch.int32, device="cuda")
        d2 = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
        tk = torch.full((m, k), -7, dtype=torch.int32, device="cuda")
        tkd = torch.full((m, k), -1.0, dtype=torch.float64, device="cuda")
        d2nd = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
        st = P.dd_project_nearest(ds, ctx, yy, idx, d2, mode=mode, certify=certify, topk_out=tk, topk_d2=tkd,
                                  d2nd=d2nd)
        torch.cuda.synchronize()
        return [t.cpu().numpy() for t in (idx, d2, tk, tkd, d2nd)] + [st]
    idx = np.full(m, -7, np.int32)
    d2 = np.full(m, -1.0)
    tk = np.full((m, k), -7, np.int32)
    tkd = np.full((m, k), -1.0)
    d2nd = np.full(m, -1.0)
    st = P.dd_project_nearest(ds, ctx, y, idx, d2, mode=mode, certify=certify, topk_out=tk, topk_d2=tkd, d2nd=d2nd)
    return idx, d2, tk, tkd, d2nd, st


def check_exact_topk(tk, tkd, oi, od, data, y):
    """Distances equal the oracle's sorted ones (Eq. 3 units = 2 x mapped);
    indices equal wherever the neighbouring distances are separated by more
    than 1e-6 relative, else the GPU's point has the oracle's distance."""
    k = tk.shape[1]
    ref = 2 * od[:, :k]
    assert np.allclose(tkd, ref, rtol=1e-9, atol=0)
    pad = np.isinf(ref)
    assert np.all(tk[pad] == -1)
    gap = np.ones_like(ref, dtype=bool)
    rel = np.diff(ref, axis=1) > 1e-6 * ref[:, 1:]
    gap[:, 1:] &= rel
    gap[:, :-1] &= rel
    assert np.array_equal(tk[gap & ~pad], oi[:, :k][gap & ~pad])
    amb = ~gap & ~pad
    if amb.any():
        q, e = np.nonzero(amb)
        dg = metric.local_d2(y[q], data[tk[q, e]].astype(np.float64), C)
        assert np.allclose(dg, ref[q, e], rtol=1e-9)


@pytest.mark.parametrize("mode", ["fp32", "tc"])
@pytest.mark.parametrize("k", [1, 2, 5, 8])
@pytest.mark.parametrize("m", [1, 1000, 3001])
def test_exact_topk_matches_oracle(ctx, dset, mode, k, m):
    data, ds = dset
    md = P.DD_SEARCH_EXACT_FP32 if mode == "fp32" else P.DD_SEARCH_EXACT_TC
    y = I.make_states(m, I.NONLINEAR, seed=42 + m, spread=0.1)
    idx, d2, tk, tkd, d2nd, st = topk(ctx, ds, y, k, md, device=(m == 1000))
    oi, od = oracle_topk(data, y, max(k, 2))
    check_exact_topk(tk, tkd, oi, od, data, y)
    assert np.array_equal(idx, tk[:, 0]) and np.array_equal(d2, tkd[:, 0])
    if k >= 2:
        assert np.allclose(d2nd, 2 * od[:, 1], rtol=1e-9)           # the exact second distance
    else:
        assert np.all(d2nd <= 2 * od[:, 1] * (1 + 1e-9))              # a lower bound
    print(f"{mode} k={k} m={m}: re-searched in FP64 {st.uncertified}")


def test_topk_fewer_points_than_k(ctx):
    data = I.make_dataset(5, I.LINEAR, seed=1)
    ds = P.dd_load_dataset(ctx, data, C, build_fp16=True)
    try:
        y = I.make_states(37, I.LINEAR, seed=2, spread=0.2)
        oi, od = nn.nn_topk(metric.to_z(data.astype(np.float64), C), metric.to_z(y, C), 8)
        for md in (P.DD_SEARCH_EXACT_FP32, P.DD_SEARCH_EXACT_TC):
            _, _, tk, tkd, _, _ = topk(ctx, ds, y, 8, md)
            check_exact_topk(tk, tkd, oi, od, data, y)
            assert np.all(tk[:, 5:] == -1) and np.all(np.isinf(tkd[:, 5:]))
    finally:
        P.dd_free_dataset(ds)


def test_tensor_core_topk_form_error_reported(ctx, dset):
    """The single-FP16 tensor-core scan (certify = 0) keeps the best 8 scores
    per data range and rescored them in FP64: the sorted list can only be as
    far as or farther than the exact k nearest, position by position; its
    agreement with the exact top-k is reported."""
    data, ds = dset
    k = 4
    y = I.make_states(2000, I.NONLINEAR, seed=47, spread=0.1)
    _, _, tk, tkd, _, _ = topk(ctx, ds, y, k, P.DD_SEARCH_EXACT_TC, certify=False)
    oi, od = oracle_topk(data, y, k)
    ref = 2 * od
    assert np.all(np.diff(tkd, axis=1) >= 0)
    assert np.all(tkd >= ref * (1 - 1e-9))
    dg = metric.local_d2(np.repeat(y, k, axis=0), data[tk.reshape(-1)].astype(np.float64), C).reshape(-1, k)
    assert np.allclose(dg, tkd, rtol=1e-9)
    exact_sets = np.mean([set(a) == set(b) for a, b in zip(tk.tolist(), oi.tolist())])
    excess = np.mean((tkd - ref) / ref)
    print(f"tensor-core top-{k} (one FP16 term): exact set {exact_sets:.4f}, nearest exact "
          f"{np.mean(tk[:, 0] == oi[:, 0]):.4f}, mean relative distance excess {excess:.2e}")
    assert np.mean(tk[:, 0] == oi[:, 0]) >= 0.9


def test_topk_argument_errors(ctx, dset):
    data, ds = dset
    y = I.make_states(10, I.NONLINEAR, seed=3, spread=0.1)
    idx = np.zeros(10, np.int32)
    for bad in (dict(topk_out=np.zeros((10, 9), np.int32)),
                dict(topk_out=np.zeros((10, 2), np.int32), mode=P.DD_SEARCH_ANN)):
        with pytest.raises(P.DDError) as e:
            P.dd_project_nearest(ds, ctx, y, idx, **bad)
        assert e.value.status in (P.DD_ERR_ARG, P.DD_ERR_STATE)
