"""GPU exact data projection P_D (Eq. 7) against the FP64 oracle."""
import numpy as np
import pytest

import dd_inputs as I
from gpu_util import assert_nn_parity

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


def project(ctx, ds, y, mode=P.DD_SEARCH_EXACT_FP32, device=True, certify=True):
    m = len(y)
    if device:
        yd = torch.from_numpy(y).cuda()
        idx = torch.full((m,), -7, dtype=torch.int32, device="cuda")
        d2 = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
        st = P.dd_project_nearest(ds, ctx, yd, idx, d2, mode=mode, certify=certify)
        torch.cuda.synchronize()
        return idx.cpu().numpy(), d2.cpu().numpy(), st
    idx = np.full(m, -7, np.int32)
    d2 = np.full(m, -1.0)
    st = P.dd_project_nearest(ds, ctx, y, idx, d2, mode=mode, certify=certify)
    return idx, d2, st


@pytest.mark.parametrize("N", [1, 2, 127, 128, 129, 255, 256, 257, 3001, 20000])
def test_exact_fp32_ragged_sizes(ctx, N):
    data = I.make_dataset(N, I.LINEAR, seed=N)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        for m, spread in ((1, 0.1), (1023, 0.05), (1025, 0.5), (2500, 3.0)):
            y = I.make_states(m, I.LINEAR, seed=m + N, spread=spread)
            idx, d2, st = project(ctx, ds, y, device=(m % 2 == 1))
            assert_nn_parity(idx, d2, data, y, C)
    finally:
        P.dd_free_dataset(ds)


def test_exact_fp32_planted_and_ties(ctx):
    data = I.make_dataset(5000, I.NONLINEAR, seed=3)
    data[4000] = data[17]            # exact duplicate: lowest index wins
    data[4500] = data[17]
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        y = data[[17, 4000, 4500, 99, 4999, 0]].astype(np.float64)
        idx, d2, _ = project(ctx, ds, y)
        assert idx.tolist() == [17, 17, 17, 99, 4999, 0]
        assert np.all(d2 == 0.0)
    finally:
        P.dd_free_dataset(ds)


def test_empty_query_batch_is_noop(ctx):
    data = I.make_dataset(100, I.LINEAR, seed=1)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        y = np.zeros((0, 12))
        idx = np.zeros(0, np.int32)
        P.dd_project_nearest(ds, ctx, y, idx, None)
    finally:
        P.dd_free_dataset(ds)


def test_device_generator_is_bit_identical(ctx):
    for law, N, start in ((I.LINEAR, 5000, 0), (I.NONLINEAR, 3000, 123457)):
        out = torch.empty((N, 12), dtype=torch.float32, device="cuda")
        P.dd_synth_dataset(ctx, out, law, C, seed=11, start=start)
        torch.cuda.synchronize()
        want = I.make_dataset(N, law, seed=11, start=start)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_full_size_exact_sampled(ctx):
    """N = 10^6 points, m = 32768 queries (16^3 cube's Gauss points): all
    queries through the kernel as benched, a sample checked by the oracle."""
    N, m = 1_000_000, 32768
    law = I.LINEAR
    raw = torch.empty((N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, law, C, seed=0)
    ds = P.dd_load_dataset(ctx, raw, C, borrow=True)
    try:
        y = I.make_states(m, law, seed=5, spread=0.05)
        idx, d2, st = project(ctx, ds, y)
        rng = np.random.default_rng(0)
        sample = rng.choice(m, 192, replace=False)
        data = I.make_dataset(N, law, seed=0)
        assert_nn_parity(idx[sample], d2[sample], data, y[sample], C)
        assert st.uncertified <= m // 100
    finally:
        P.dd_free_dataset(ds)


def test_errors(ctx):
    data = I.make_dataset(10, I.LINEAR, seed=1)
    bad = C.copy()
    bad[0, 0] = -1.0
    with pytest.raises(P.DDError) as e:
        P.dd_load_dataset(ctx, data, bad)
    assert e.value.status == P.DD_ERR_NOT_SPD
    nanny = data.copy()
    nanny[3, 4] = np.nan
    with pytest.raises(P.DDError) as e:
        P.dd_load_dataset(ctx, nanny, C)
    assert e.value.status == P.DD_ERR_ARG
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        with pytest.raises(P.DDError) as e:
            P.dd_project_nearest(ds, ctx, np.zeros((3, 12)), np.zeros(3, np.int32), mode=7)
        assert e.value.status == P.DD_ERR_ARG
        with pytest.raises(P.DDError) as e:
            P.dd_project_nearest(ds, ctx, np.zeros((3, 12)), np.zeros(3, np.int32), mode=P.DD_SEARCH_EXACT_TC)
        assert e.value.status == P.DD_ERR_STATE
    finally:
        P.dd_free_dataset(ds)
