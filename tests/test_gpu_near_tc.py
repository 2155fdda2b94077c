"""The tensor-core nearest-centroid passes (cell ranking of the search, the
k-means assignment of the tree build to the cells) and the shared-memory
leaf sums give exactly the answers of the ALU kernels they replace: a
partition built with them equals, centroid for centroid and point for point,
the one built on the ALU from the same data and seed, and searches on the
two give the same indices and distances, including queries so far out that
the tensor-core scores cannot settle them (those rows are finished by the
ALU kernel)."""
import numpy as np
import pytest

import dd_inputs as I
from oracle import metric

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


def pair(ctx, data, **kw):
    a = P.dd_load_dataset(ctx, data, C, ann_alu=False, **kw)
    b = P.dd_load_dataset(ctx, data, C, ann_alu=True, **kw)
    return a, b


def export(ctx, ds, two):
    cl, cent, rad = P.dd_dataset_ann_index(ds, ctx)
    out = [cl, cent, rad]
    if two:
        L2, ccent, crad = P.dd_dataset_ann_cells(ds, ctx)
        out += [np.array([L2]), ccent, crad]
    return out


def search(ctx, ds, y, f_d, prev):
    yd = torch.from_numpy(y).cuda()
    idx = torch.empty(len(y), dtype=torch.int32, device="cuda")
    d2 = torch.empty(len(y), dtype=torch.float64, device="cuda")
    P.dd_project_nearest(ds, ctx, yd, idx, d2, mode=P.DD_SEARCH_ANN, f_d=f_d,
                         prev_idx=None if prev is None else torch.from_numpy(prev).cuda())
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy()


def states(n, seed, far=0):
    y = I.make_states(n, I.NONLINEAR, seed=seed, spread=0.1)
    if far:   # states far outside the data (out of the FP16 operand range)
        y[:far] *= 1e4
    return np.ascontiguousarray(y)


# (levels, N, nlist): 128 cells of 128 leaves (one centroid tile); 256
# cells of 256 leaves (two tiles); one level of 1000 clusters (a partial
# last tile)
CASES = [(2, 200_000, 128 * 128), (2, 300_000, 256 * 256), (1, 60_000, 1000)]


@pytest.mark.parametrize("levels,n,nlist", CASES)
def test_partition_and_search_equal_alu(ctx, levels, n, nlist):
    data = I.make_dataset(n, I.NONLINEAR, seed=31)
    a, b = pair(ctx, data, ann_nlist=nlist, ann_levels=levels, seed=3)
    try:
        ea, eb = export(ctx, a, levels == 2), export(ctx, b, levels == 2)
        for x, z in zip(ea, eb):
            assert np.array_equal(x, z)
        print(f"levels {levels}, N {n}, nlist {nlist}: build rows left to the ALU "
              f"{P.dd_dataset_ann_build_fallback(a)}")
        assert P.dd_dataset_ann_build_fallback(b) == 0
        y = states(3000, seed=32, far=40)
        prev = np.random.default_rng(6).integers(0, n, len(y)).astype(np.int32)
        for f_d, pv in [(0.0, None), (0.4, prev), (0.8, prev), (1.0, None)]:
            ia, da = search(ctx, a, y, f_d, pv)
            ib, db = search(ctx, b, y, f_d, pv)
            assert np.array_equal(ia, ib), f"f_d {f_d}: indices differ"
            assert np.array_equal(da, db), f"f_d {f_d}: distances differ"
    finally:
        P.dd_free_dataset(a)
        P.dd_free_dataset(b)


def test_assignment_is_nearest_centroid(ctx):
    """Each point of a one-level partition belongs to a cluster whose
    centroid is nearest up to FP32 rounding of the expanded score (checked
    in FP64 against all centroids)."""
    data = I.make_dataset(40_000, I.NONLINEAR, seed=33)
    ds = P.dd_load_dataset(ctx, data, C, ann_nlist=300, seed=2)
    try:
        cl, cent, rad = P.dd_dataset_ann_index(ds, ctx)
        Z = metric.to_z(data.astype(np.float64), C)
        # scores |c|^2 - 2 c.z of every point against every centroid
        s = (cent ** 2).sum(1)[None, :] - 2.0 * Z @ cent.T
        best = s.min(1)
        got = s[np.arange(len(Z)), cl]
        scale = (cent ** 2).sum(1).max() + 2.0 * np.sqrt((Z ** 2).sum(1)) * np.sqrt((cent ** 2).sum(1).max())
        assert np.all(got - best <= 1e-5 * scale)
    finally:
        P.dd_free_dataset(ds)


def test_tied_centroids_are_finished_on_the_alu(ctx):
    """Forty distinct points, each repeated 500 times: the k-means build
    starts from many identical centroids, so most points have more tied
    nearest cells than the tensor-core list holds; those rows go to the ALU
    kernel, and the partition and the searches still equal the ALU-only
    build's (ties to the lower index)."""
    base = I.make_dataset(40, I.NONLINEAR, seed=35)
    data = np.ascontiguousarray(np.repeat(base, 500, axis=0))
    a, b = pair(ctx, data, ann_nlist=1000, seed=3)
    try:
        print(f"tied centroids: build rows left to the ALU {P.dd_dataset_ann_build_fallback(a)}")
        assert P.dd_dataset_ann_build_fallback(a) > 0
        for x, z in zip(export(ctx, a, False), export(ctx, b, False)):
            assert np.array_equal(x, z)
        y = states(500, seed=36)
        for f_d in (0.0, 0.8):
            ia, da = search(ctx, a, y, f_d, None)
            ib, db = search(ctx, b, y, f_d, None)
            assert np.array_equal(ia, ib) and np.array_equal(da, db)
    finally:
        P.dd_free_dataset(a)
        P.dd_free_dataset(b)
