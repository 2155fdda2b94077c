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
    for law, start in ((I.LINEAR, 0), (I.NONLINEAR, 987654), (I.EQ9_LAW, 55555)):
        a = I.make_dataset(4000, law, seed=3, start=start)
        b = cgen.make_dataset(4000, law, seed=3, start=start)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def voigt_to_tensor(e):
    """Strain tensor from Voigt strains with engineering shears."""
    return np.array([[e[0], e[5] / 2, e[4] / 2], [e[5] / 2, e[1], e[3] / 2], [e[4] / 2, e[3] / 2, e[2]]])


def stress_to_voigt(S):
    return np.array([S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[0, 2], S[0, 1]])


def test_eq9_law_is_the_papers_formula():
    """With lam = mu = E/2 (E = 1000) and beta = alpha = 500 the generator's
    law is E (eps + alpha eps^3 + 0.5 (tr eps + alpha (tr eps)^3) I) of
    Eq. (9), eps^3 the matrix cube of the strain tensor, written out here
    with numpy's matrix power."""
    law = I.EQ9_LAW
    Cm = I.isotropic_C(law.E, law.nu)
    assert np.isclose(Cm[0, 1], 500.0) and np.isclose(Cm[3, 3], 500.0)
    rng = np.random.default_rng(0)
    eps = rng.uniform(-0.025, 0.025, (50, 6))
    got = I.law_stress(law, eps)
    E, alpha = 1000.0, 500.0
    for k in range(len(eps)):
        T = voigt_to_tensor(eps[k])
        tr = np.trace(T)
        S = E * (T + alpha * np.linalg.matrix_power(T, 3) + 0.5 * (tr + alpha * tr ** 3) * np.eye(3))
        assert np.allclose(got[k], stress_to_voigt(S), rtol=1e-12, atol=1e-12)


def test_eq9_law_closed_forms_and_isotropy():
    law = I.EQ9_LAW
    lam = mu = 500.0
    beta = law.beta
    x, gam = 0.02, 0.03
    s = I.law_stress(law, np.array([[x, 0, 0, 0, 0, 0], [0, 0, 0, 0, 0, gam]]))
    g = x + beta * x ** 3
    assert np.allclose(s[0], [(lam + 2 * mu) * g, lam * g, lam * g, 0, 0, 0], rtol=1e-14)
    h = gam / 2
    assert np.allclose(s[1], [0, 0, 0, 0, 0, 2 * mu * (h + beta * h ** 3)], rtol=1e-14, atol=1e-15)
    # an isotropic tensor function: rotating the strain rotates the stress
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    e = rng.uniform(-0.025, 0.025, 6)
    Te = voigt_to_tensor(e)
    Tr = Q @ Te @ Q.T
    er = np.array([Tr[0, 0], Tr[1, 1], Tr[2, 2], 2 * Tr[1, 2], 2 * Tr[0, 2], 2 * Tr[0, 1]])
    s0, s1 = I.law_stress(law, np.stack([e, er]))
    S0 = np.array([[s0[0], s0[5], s0[4]], [s0[5], s0[1], s0[3]], [s0[4], s0[3], s0[2]]])
    assert np.allclose(stress_to_voigt(Q @ S0 @ Q.T), s1, rtol=1e-12, atol=1e-12)
