"""Pins of oracle.metric: Eq. (3) and the mapped coordinates of Sec. 3.2."""
import numpy as np

import dd_inputs as I
from oracle import metric as M


def random_spd(rng, n=6):
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def test_isotropic_spectrum_closed_form():
    E, nu = 1.0, 0.3
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    C = I.isotropic_C(E, nu)
    Ch, Cmh = M.metric_roots(C)
    want = np.sort(np.sqrt([3 * lam + 2 * mu, 2 * mu, 2 * mu, mu, mu, mu]))
    assert np.allclose(np.sort(np.linalg.eigvalsh(Ch)), want, rtol=1e-13)
    assert np.allclose(np.sort(np.linalg.eigvalsh(Cmh)), np.sort(1 / want), rtol=1e-13)


def test_root_identities():
    rng = np.random.default_rng(0)
    for C in (I.isotropic_C(), random_spd(rng), random_spd(rng)):
        Ch, Cmh = M.metric_roots(C)
        assert np.allclose(Ch @ Ch, C, rtol=0, atol=1e-13 * np.abs(C).max())
        assert np.allclose(Ch @ Cmh, np.eye(6), atol=1e-13)
        assert np.allclose(Ch, Ch.T, atol=1e-14 * np.abs(Ch).max())


def test_mapped_distance_is_half_eq3():
    rng = np.random.default_rng(1)
    for C in (I.isotropic_C(), random_spd(rng)):
        y = rng.standard_normal((50, 12))
        z = rng.standard_normal((50, 12))
        dq = M.to_z(y, C) - M.to_z(z, C)
        assert np.allclose((dq * dq).sum(1), 0.5 * M.local_d2(y, z, C), rtol=1e-12)


def test_local_d2_hand_value():
    C = 2.0 * np.eye(6)
    y = np.zeros((1, 12)); z = np.zeros((1, 12))
    y[0, 0] = 1.0          # d eps = e_1 -> C de.de = 2
    y[0, 7] = 2.0          # d sig = 2 e_2 -> C^-1 ds.ds = 4 / 2 = 2
    assert np.isclose(M.local_d2(y, z, C)[0], 4.0)


def test_rejects_non_spd():
    C = I.isotropic_C(); C[0, 0] = -1.0
    try:
        M.metric_roots(C)
    except ValueError:
        return
    raise AssertionError("non-SPD metric accepted")


def test_pca_metric_recovers_a_linear_law():
    """Data on sig = C0 eps (C0 SPD, not isotropic, strains from a
    non-isotropic distribution): the principal subspace is {(x, C0 x)} and
    the PCA metric is C0 itself."""
    rng = np.random.default_rng(3)
    B = rng.normal(size=(6, 6))
    C0 = B @ B.T + 6 * np.eye(6)
    eps = rng.uniform(-1, 1, (5000, 6)) * np.array([1, 2, 3, 0.5, 0.7, 1.3]) + 0.2
    data = np.concatenate([eps, eps @ C0.T], axis=1)
    C = M.pca_metric(data)
    assert np.allclose(C, C0, rtol=1e-9, atol=1e-9 * np.abs(C0).max())
    # invariant to the order of the data
    assert np.allclose(M.pca_metric(data[::-1]), C, rtol=1e-12, atol=0)


def test_pca_metric_of_the_papers_law():
    """Eq. (9) data (strains in [-0.025, 0.025]^6): the PCA metric is
    symmetric positive definite, stiffer than the law's tangent at zero
    strain (the cubic terms stiffen), and nearly isotropic (the cube of
    strains is symmetric under axis permutations)."""
    law = I.EQ9_LAW
    data = I.make_dataset(200000, law, seed=1).astype(np.float64)
    C = M.pca_metric(data)
    assert np.allclose(C, C.T)
    w = np.linalg.eigvalsh(C)
    assert w.min() > 0
    C_lin = I.isotropic_C(law.E, law.nu)
    assert np.all(np.diag(C) > np.diag(C_lin))
    assert np.allclose(np.diag(C)[:3], np.diag(C)[:3].mean(), rtol=0.02)
    assert np.allclose(np.diag(C)[3:], np.diag(C)[3:].mean(), rtol=0.02)
