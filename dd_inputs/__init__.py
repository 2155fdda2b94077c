"""Seeded synthetic inputs for the data-driven (DD) solver workloads.

This module only *describes and draws* problem inputs: material data sets,
query states, initial data associations, the metric tensor and the workload
definitions (mesh size, loads, data law).  It holds no step of the DD method
itself (no distance, no projection, no finite-element operator), so both the
FP64 oracle and the CUDA path can consume its outputs without sharing any of
the method's arithmetic.

Random numbers come from a counter-based generator: the SplitMix64 output
function of Steele, Lea & Flood, "Fast splittable pseudorandom number
generators" (OOPSLA 2014), applied to ``key + (n + 1) * GAMMA``.  Draw ``n`` of
a stream can therefore be produced independently of every other draw, which is
what lets a device-side generator build the same billion-point data set in
place.  Every floating-point step below is a single correctly rounded IEEE
operation (+, -, *, sqrt, float64 -> float32) taken in a fixed order, with no
fused multiply-add, so a second implementation that follows the same order is
bit-identical.  Gaussian noise uses the Irwin-Hall sum of twelve uniforms minus
six (mean 0, variance 1), whose integer sum is exact.

Data-set draw layout, point ``j`` uses counters ``64*j + s``:
  s = 0..5   strain component i: u = (x >> 11) * 2**-53,  eps_i = lo + (hi-lo)*u
  s = 8..43  noise of stress component i uses s = 8 + 6*i + r, r = 0..5; the
             twelve 32-bit halves of those six words are summed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

STREAM_DATA = 1
STREAM_STATES = 2
STREAM_ASSOC = 3

DRAWS_PER_POINT = 64


def _fmix64_int(x: int) -> int:
    x &= _MASK
    x ^= x >> 30
    x = (x * _M1) & _MASK
    x ^= x >> 27
    x = (x * _M2) & _MASK
    x ^= x >> 31
    return x


def stream_key(seed: int, stream: int) -> int:
    """Key of one random stream: fmix(fmix(seed + GAMMA) + stream)."""
    return _fmix64_int((_fmix64_int((seed + GAMMA) & _MASK) + stream) & _MASK)


def _fmix64(x: np.ndarray) -> np.ndarray:
    x = x ^ (x >> np.uint64(30))
    x = x * np.uint64(_M1)
    x = x ^ (x >> np.uint64(27))
    x = x * np.uint64(_M2)
    return x ^ (x >> np.uint64(31))


def draws(key: int, counters: np.ndarray) -> np.ndarray:
    """uint64 draw for every counter n: fmix(key + (n + 1) * GAMMA) mod 2**64."""
    with np.errstate(over="ignore"):
        c = np.asarray(counters, dtype=np.uint64)
        return _fmix64(np.uint64(key) + (c + np.uint64(1)) * np.uint64(GAMMA))


def uniform53(x: np.ndarray) -> np.ndarray:
    """Top 53 bits of a uint64 draw as a float64 in [0, 1) (exact)."""
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def irwin_hall(words: np.ndarray) -> np.ndarray:
    """Standard-normal stand-in from 6 uint64 words (last axis): sum of the
    twelve 32-bit halves scaled to [0,12), minus 6.  Exact in float64."""
    lo = (words & np.uint64(0xFFFFFFFF)).sum(axis=-1, dtype=np.uint64)
    hi = (words >> np.uint64(32)).sum(axis=-1, dtype=np.uint64)
    s = (lo + hi).astype(np.int64) - (6 << 32)
    return s.astype(np.float64) * (2.0 ** -32)


# ----------------------------------------------------------------------------
# Material: isotropic Voigt stiffness (engineering shear strains).
# ----------------------------------------------------------------------------
def isotropic_C(E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """6x6 Voigt stiffness of an isotropic solid, order (xx,yy,zz,yz,xz,xy),
    acting on engineering shear strains.  Used both as the data law and as
    the metric tensor of the local distance."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2.0 * mu
        C[3 + i, 3 + i] = mu
    return C


def _matvec_ordered(C: np.ndarray, e: np.ndarray) -> np.ndarray:
    """(C e) with each row summed left to right, one rounding per op."""
    out = np.empty_like(e)
    for i in range(6):
        acc = C[i, 0] * e[:, 0]
        for k in range(1, 6):
            acc = acc + C[i, k] * e[:, k]
        out[:, i] = acc
    return out


def _norm_ordered(e: np.ndarray) -> np.ndarray:
    acc = e[:, 0] * e[:, 0]
    for k in range(1, 6):
        acc = acc + e[:, k] * e[:, k]
    return np.sqrt(acc)


@dataclass(frozen=True)
class DataLaw:
    """Synthetic material law sampled into a data set.

    kind="linear":     sigma = C eps + noise
    kind="nonlinear":  sigma = C eps (1 + beta*|eps|) + noise   (|eps|: 2-norm
                       of the Voigt 6-vector as stored)
    kind="eq9":        the isotropic cubic law of Eq. (9),
                       sigma = 2 mu (eps + beta eps^3) + lam (tr eps + beta (tr eps)^3) I,
                       eps^3 the tensor power, lam and mu the Lame constants of
                       C (with lam = mu = E/2 and beta = alpha this is the
                       paper's E (eps + alpha eps^3 + 0.5 (tr eps + alpha (tr eps)^3) I)
    eps components i.i.d. uniform in [eps_lo, eps_hi]; noise i.i.d. per stress
    component, std ``noise_std`` (Irwin-Hall).
    """
    kind: str = "linear"
    eps_lo: float = -2e-3
    eps_hi: float = 2e-3
    noise_std: float = 1e-5
    beta: float = 50.0
    E: float = 1.0
    nu: float = 0.3

    @property
    def code(self) -> int:
        return {"linear": 0, "nonlinear": 1, "eq9": 2}[self.kind]


def _eq9_stress(C: np.ndarray, e: np.ndarray, beta: float) -> np.ndarray:
    """Stress of the cubic law (kind "eq9") in Voigt order, tensor shear
    stresses; every operation rounded once, in a fixed order shared with the
    C and device copies of the generator."""
    lam, mu = C[0, 1], C[3, 3]
    a, b, c = e[:, 0], e[:, 1], e[:, 2]
    d, g, f = 0.5 * e[:, 3], 0.5 * e[:, 4], 0.5 * e[:, 5]      # tensor shears e23, e13, e12
    # P = E E
    p11 = (a * a + f * f) + g * g
    p22 = (f * f + b * b) + d * d
    p33 = (g * g + d * d) + c * c
    p23 = (f * g + b * d) + d * c
    p13 = (a * g + f * d) + g * c
    p12 = (a * f + f * b) + g * d
    # Q = P E
    q11 = (p11 * a + p12 * f) + p13 * g
    q22 = (p12 * f + p22 * b) + p23 * d
    q33 = (p13 * g + p23 * d) + p33 * c
    q23 = (p12 * g + p22 * d) + p23 * c
    q13 = (p11 * g + p12 * d) + p13 * c
    q12 = (p11 * f + p12 * b) + p13 * d
    tr = (a + b) + c
    h = lam * (tr + beta * ((tr * tr) * tr))
    m2 = 2.0 * mu
    return np.stack([h + m2 * (a + beta * q11), h + m2 * (b + beta * q22), h + m2 * (c + beta * q33),
                     m2 * (d + beta * q23), m2 * (g + beta * q13), m2 * (f + beta * q12)], axis=1)


def law_stress(law: DataLaw, eps: np.ndarray) -> np.ndarray:
    """Noise-free stress of the law at strains eps [n, 6] (float64)."""
    C = isotropic_C(law.E, law.nu)
    if law.kind == "eq9":
        return _eq9_stress(C, eps, law.beta)
    s = _matvec_ordered(C, eps)
    if law.kind == "nonlinear":
        s = s * (1.0 + law.beta * _norm_ordered(eps))[:, None]
    return s


def make_dataset(N: int, law: DataLaw, seed: int = 0, start: int = 0,
                 chunk: int = 1 << 20) -> np.ndarray:
    """Points ``start .. start+N-1`` of the seeded data set, float32 [N, 12]:
    columns 0..5 strain (Voigt, engineering shear), 6..11 stress."""
    C = isotropic_C(law.E, law.nu)
    key = stream_key(seed, STREAM_DATA)
    out = np.empty((N, 12), dtype=np.float32)
    width = law.eps_hi - law.eps_lo
    for c0 in range(0, N, chunk):
        n = min(chunk, N - c0)
        j = np.arange(start + c0, start + c0 + n, dtype=np.uint64)
        base = j * np.uint64(DRAWS_PER_POINT)
        ctr_e = base[:, None] + np.arange(6, dtype=np.uint64)[None, :]
        eps = law.eps_lo + width * uniform53(draws(key, ctr_e))
        ctr_n = base[:, None, None] + (np.uint64(8) + np.arange(36, dtype=np.uint64)).reshape(1, 6, 6)
        g = irwin_hall(draws(key, ctr_n))
        s = law_stress(law, eps)
        sig = s + law.noise_std * g
        out[c0:c0 + n, :6] = eps.astype(np.float32)
        out[c0:c0 + n, 6:] = sig.astype(np.float32)
    return out


def make_states(m: int, law: DataLaw, seed: int, spread: float,
                scale: float | None = None) -> np.ndarray:
    """Query states y = (eps, sig), float64 [m, 12]: points of ``law`` (noise
    free) displaced by uniform perturbations of relative size ``spread`` of
    the strain range, in both strain and stress.  spread=0 lies on the law,
    large spread moves the states far off the data manifold, as in the first
    DD iterations."""
    C = isotropic_C(law.E, law.nu)
    key = stream_key(seed, STREAM_STATES)
    j = np.arange(m, dtype=np.uint64)[:, None] * np.uint64(32)
    u = uniform53(draws(key, j + np.arange(18, dtype=np.uint64)[None, :]))
    width = law.eps_hi - law.eps_lo
    eps = law.eps_lo + width * u[:, :6]
    s = law_stress(law, eps)
    a = spread * width if scale is None else scale
    eps = eps + a * (u[:, 6:12] - 0.5)
    s = s + a * float(np.abs(C).max()) * (u[:, 12:18] - 0.5)
    return np.concatenate([eps, s], axis=1)


def initial_association(m: int, N: int, seed: int = 0) -> np.ndarray:
    """Random initial data point of every material point (uniform, int32):
    draw(e) mod N."""
    key = stream_key(seed, STREAM_ASSOC)
    x = draws(key, np.arange(m, dtype=np.uint64))
    return (x % np.uint64(N)).astype(np.int32)


# ----------------------------------------------------------------------------
# Boundary-value problem: unit cube, clamped bottom, traction on the top face
# t(x, y) = t0 + tx*(x - cx) + ty*(y - cy), (cx, cy) the top-face centre.
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Load:
    t0: tuple = (0.0, 0.0, 0.0)
    tx: tuple = (0.0, 0.0, 0.0)
    ty: tuple = (0.0, 0.0, 0.0)
    rot_z: float = 0.0        # prescribed rotation of the top face about the vertical axis (radians)


def load_case(name: str, t: float) -> Load:
    """Top-face load cases on a unit cube: tension, shear, bending, torsion."""
    if name == "tension":
        return Load(t0=(0.0, 0.0, t))
    if name == "shear":
        return Load(t0=(t, 0.0, 0.0))
    if name == "bending":      # t_z = t (2x - 1)
        return Load(tx=(0.0, 0.0, 2.0 * t))
    if name == "torsion":      # t = 2t (-(y - 1/2), x - 1/2, 0)
        return Load(tx=(0.0, 2.0 * t, 0.0), ty=(-2.0 * t, 0.0, 0.0))
    if name == "rotation":     # prescribed top rotation, t in degrees
        return top_rotation(t)
    raise ValueError(name)


def top_rotation(theta_deg: float) -> Load:
    """The top face turned rigidly by theta_deg degrees about the vertical
    axis through its centre, the bottom clamped, no traction (the paper's
    own boundary-value problem, a 2 degree torsion)."""
    return Load(rot_z=math.radians(theta_deg))


def random_load(seed: int, r: int, tmin: float, tmax: float) -> Load:
    """Uniform top traction of magnitude U[tmin, tmax] along a uniformly
    random direction (request r of a serving stream)."""
    key = stream_key(seed, 100 + r)
    u = uniform53(draws(key, np.arange(3, dtype=np.uint64)))
    mag = tmin + (tmax - tmin) * u[0]
    cz = 2.0 * u[1] - 1.0
    phi = 2.0 * math.pi * u[2]
    sz = math.sqrt(max(0.0, 1.0 - cz * cz))
    return Load(t0=(mag * sz * math.cos(phi), mag * sz * math.sin(phi), mag * cz))


def serve_requests(seed: int, n: int, edge_min: int, edge_max: int, t_min: float, t_max: float,
                   rate: float):
    """Serving stream: for request r, a cube edge uniform in {edge_min..edge_max}
    (elements), a random load (random_load) and an arrival time of a Poisson
    process of the given rate (exponential gaps from uniform draws)."""
    key = stream_key(seed, 99)
    u = uniform53(draws(key, np.arange(2 * n, dtype=np.uint64))).reshape(n, 2)
    edges = edge_min + np.minimum((u[:, 0] * (edge_max - edge_min + 1)).astype(np.int64), edge_max - edge_min)
    gaps = -np.log1p(-u[:, 1]) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    return [(int(edges[r]), random_load(seed, r, t_min, t_max), int(arrivals[r] * 1e6) / 1e6, 1000 + r)
            for r in range(n)]


@dataclass(frozen=True)
class Workload:
    name: str
    n_el: int                 # elements per cube edge
    N: int                    # data points
    law: DataLaw
    loads: tuple = (("tension", 1e-3),)
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:       # material (Gauss) points per solve
        return 8 * self.n_el ** 3


LINEAR = DataLaw("linear", -2e-3, 2e-3, 1e-5)
NONLINEAR = DataLaw("nonlinear", -5e-3, 5e-3, 1e-5)
# the strain range of the paper's torsion data (Sec. 3.1: [-0.025, 0.025]),
# with a milder stiffening (the factor 1 + beta |eps| stays below 1.6)
TORSION_LAW = DataLaw("nonlinear", -0.025, 0.025, 1e-5, beta=10.0)
# the paper's law, Eq. (9): E = 1000, alpha = 500, i.e. Lame constants
# lam = mu = 500 (isotropic C with E' = 1250, nu = 0.25), no noise
EQ9_LAW = DataLaw("eq9", -0.025, 0.025, 0.0, beta=500.0, E=1250.0, nu=0.25)

WORKLOADS = {
    "cube4_N1e4_exact_fp64": Workload("cube4_N1e4_exact_fp64", 4, 10_000, LINEAR),
    "cube16_N1e6_exact": Workload("cube16_N1e6_exact", 16, 1_000_000, LINEAR),
    "cube32_N1e8_ann": Workload("cube32_N1e8_ann", 32, 100_000_000, NONLINEAR),
    "cube32_N1e9_ann_4loads": Workload(
        "cube32_N1e9_ann_4loads", 32, 1_000_000_000, NONLINEAR,
        loads=(("tension", 1e-3), ("shear", 1e-3), ("bending", 1e-3), ("torsion", 1e-3))),
    # profiling cases of a few GB: the tree search (with --ann-levels 2) and
    # the 32^3 constraint projection with a small data set
    "cube16_N3e7_ann": Workload("cube16_N3e7_ann", 16, 30_000_000, NONLINEAR),
    "cube32_N3e7_ann": Workload("cube32_N3e7_ann", 32, 30_000_000, NONLINEAR),
    "cube32_N1e7_knng": Workload("cube32_N1e7_knng", 32, 10_000_000, NONLINEAR,
                                 extra={"knn_k": 128, "knn_fd": 0.8, "f_s": 2}),
    # the greedy walk in the k-NN graph (Sec. 4.4) on the 10^8-point data set
    "cube32_N1e8_knng": Workload("cube32_N1e8_knng", 32, 100_000_000, NONLINEAR,
                                 extra={"knn_k": 128, "knn_fd": 0.8, "f_s": 2}),
    # (the search is cheap in the latter)
    "cube32_N1e5_exact": Workload("cube32_N1e5_exact", 32, 100_000, NONLINEAR),
    # the paper's own problem (Sec. 3.1): 20^3 cube, top face turned by 2
    # degrees, 64 000 material points, data from the law of Eq. (9), the
    # metric from the data's principal components; approximate-search
    # schedule f_d 0.4 -> 0.8 over 5 iterations (f_d0, f_d_final, ramp)
    "cube20_N1e9_rot2_ann": Workload("cube20_N1e9_rot2_ann", 20, 1_000_000_000, EQ9_LAW,
                                     loads=(("rotation", 2.0),),
                                     extra={"schedule": (0.4, 0.8, 5), "metric": "pca"}),
    "cube20_N1e8_rot2_ann": Workload("cube20_N1e8_rot2_ann", 20, 100_000_000, EQ9_LAW,
                                     loads=(("rotation", 2.0),),
                                     extra={"schedule": (0.4, 0.8, 5), "metric": "pca"}),
    "serve_N1e7": Workload("serve_N1e7", 0, 10_000_000, NONLINEAR,
                           extra={"requests": 512, "edge_min": 4, "edge_max": 24,
                                  "t_min": 1e-4, "t_max": 2e-3}),
}
