"""The allocation-free projection entry point (dd_project_nearest_noalloc).

It serves callers that cannot allocate device memory inside a call (memory
reserved up front by another allocator, or no tolerance for cudaMalloc /
cudaFree).  This file is collected last so that a run stopping at the first
failure has already run every other test.  Its results must equal those of
dd_project_nearest (exact FP32 mode) on two calls in a row, since the second
call reuses the shared scratch array left by the first.
"""
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


def test_noalloc_matches_allocating_entry_point_twice(ctx):
    data = I.make_dataset(30000, I.NONLINEAR, seed=12)
    ds = P.dd_load_dataset(ctx, torch.from_numpy(data).cuda(), C)
    try:
        for call, (m, seed) in enumerate(((5000, 1), (777, 2))):
            y = torch.from_numpy(I.make_states(m, I.NONLINEAR, seed=seed, spread=0.2)).cuda()
            ref_i = torch.empty(m, dtype=torch.int32, device="cuda")
            ref_d = torch.empty(m, dtype=torch.float64, device="cuda")
            P.dd_project_nearest(ds, ctx, y, ref_i, ref_d, mode=P.DD_SEARCH_EXACT_FP32)
            got_i = torch.full((m,), -1, dtype=torch.int32, device="cuda")
            got_d = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
            P.dd_project_nearest_noalloc(ds, ctx, y, got_i, got_d)
            torch.cuda.synchronize()
            assert torch.equal(got_i, ref_i), f"call {call}: indices differ"
            assert np.allclose(got_d.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-12, atol=0)
    finally:
        P.dd_free_dataset(ds)


def test_noalloc_at_the_query_limit_matches_oracle(ctx):
    """At m = DD_NOALLOC_MAX_QUERIES the scan's data splits are capped so that
    the candidate windows fit the fixed array; the answers still equal the
    FP64 oracle's brute force (and the allocating entry point's), with the
    call waiting for its own status (no device wait gave up)."""
    from gpu_util import assert_nn_parity
    data = I.make_dataset(4000, I.NONLINEAR, seed=13)
    ds = P.dd_load_dataset(ctx, torch.from_numpy(data).cuda(), C)
    try:
        m = P.DD_NOALLOC_MAX_QUERIES
        y_np = I.make_states(m, I.NONLINEAR, seed=14, spread=0.2)
        y = torch.from_numpy(y_np).cuda()
        got_i = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        got_d = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
        P.dd_project_nearest_noalloc(ds, ctx, y, got_i, got_d, wait=True)
        assert_nn_parity(got_i.cpu().numpy(), got_d.cpu().numpy(), data, y_np, C)
        ref_i = torch.empty(m, dtype=torch.int32, device="cuda")
        ref_d = torch.empty(m, dtype=torch.float64, device="cuda")
        P.dd_project_nearest(ds, ctx, y, ref_i, ref_d, mode=P.DD_SEARCH_EXACT_FP32)
        torch.cuda.synchronize()
        assert torch.equal(got_i, ref_i)
        assert np.allclose(got_d.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-12, atol=0)
        assert torch.cuda.current_device() == 0
    finally:
        P.dd_free_dataset(ds)


def test_noalloc_rejects_oversized_batch(ctx):
    data = I.make_dataset(1000, I.LINEAR, seed=1)
    ds = P.dd_load_dataset(ctx, data, C)
    try:
        m = P.DD_NOALLOC_MAX_QUERIES + 1
        y = torch.zeros((m, 12), dtype=torch.float64, device="cuda")
        idx = torch.zeros(m, dtype=torch.int32, device="cuda")
        d2 = torch.zeros(m, dtype=torch.float64, device="cuda")
        with pytest.raises(P.DDError) as e:
            P.dd_project_nearest_noalloc(ds, ctx, y, idx, d2)
        assert e.value.status == P.DD_ERR_ARG
    finally:
        P.dd_free_dataset(ds)
