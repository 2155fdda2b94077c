"""Pins of the seeded input generators (dd_inputs)."""
import os

import numpy as np

import dd_inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    got = I.draws(1234567, np.arange(5)).tolist()
    assert got == want


def test_dataset_is_counter_based():
    law = I.LINEAR
    full = I.make_dataset(3000, law, seed=7, chunk=1000)
    part = I.make_dataset(500, law, seed=7, start=1234)
    assert np.array_equal(full[1234:1734], part)
    other = I.make_dataset(500, law, seed=8, start=1234)
    assert not np.array_equal(other, part)


def test_dataset_linear_law():
    law = I.LINEAR
    d = I.make_dataset(20000, law, seed=0).astype(np.float64)
    eps, sig = d[:, :6], d[:, 6:]
    assert eps.min() >= law.eps_lo - 1e-9 and eps.max() <= law.eps_hi + 1e-9
    # mean of a uniform on [lo, hi] and its variance (hi-lo)^2/12
    assert abs(eps.mean()) < 2e-5
    assert abs(eps.var() / ((law.eps_hi - law.eps_lo) ** 2 / 12) - 1) < 0.02
    C = I.isotropic_C(law.E, law.nu)
    noise = sig - eps @ C.T
    assert abs(noise.mean()) < 2e-7
    assert abs(noise.std() / law.noise_std - 1) < 0.02   # float32 storage adds ~1e-10


def test_dataset_nonlinear_law():
    law = I.NONLINEAR
    d = I.make_dataset(5000, law, seed=3).astype(np.float64)
    eps, sig = d[:, :6], d[:, 6:]
    C = I.isotropic_C(law.E, law.nu)
    fac = 1 + law.beta * np.linalg.norm(eps, axis=1)
    noise = sig - (eps @ C.T) * fac[:, None]
    assert abs(noise.std() / law.noise_std - 1) < 0.03


def test_irwin_hall_moments():
    w = I.draws(I.stream_key(5, 9), np.arange(6 * 200000).reshape(-1, 6))
    g = I.irwin_hall(w)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1) < 0.01
    assert g.min() >= -6 and g.max() <= 6


def test_isotropic_C():
    C = I.isotropic_C(1.0, 0.3)
    lam, mu = 0.3 / (1.3 * 0.4), 1 / 2.6
    assert np.isclose(C[0, 0], lam + 2 * mu) and np.isclose(C[0, 1], lam) and np.isclose(C[3, 3], mu)
    # uniaxial stress: compliance gives eps_xx = 1/E, eps_yy = -nu/E
    e = np.linalg.solve(C, np.array([1.0, 0, 0, 0, 0, 0]))
    assert np.allclose(e[:3], [1.0, -0.3, -0.3])


def test_initial_association_range():
    a = I.initial_association(100000, 777, seed=0)
    assert a.dtype == np.int32 and a.min() >= 0 and a.max() < 777
    assert len(np.unique(a)) == 777


def test_load_cases():
    assert I.load_case("tension", 2.0).t0 == (0.0, 0.0, 2.0)
    L = I.random_load(0, 3, 1e-4, 2e-3)
    mag = np.linalg.norm(L.t0)
    assert 1e-4 <= mag <= 2e-3


def test_c_generator_bit_identical():
    from dd_inputs import cgen
    for law, start in ((I.LINEAR, 0), (I.NONLINEAR, 987654)):
        a = I.make_dataset(4000, law, seed=3, start=start)
        b = cgen.make_dataset(4000, law, seed=3, start=start)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
