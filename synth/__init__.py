"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the method itself: it only draws the random
feature parameters (the ELM-FBPINN hidden weights of Eq. (2), which the method
freezes after drawing them, Sec. 2.1) and describes the workloads (problem sizes,
manufactured-solution coefficients).  Both the oracle and the GPU library receive
the same arrays produced here, so they see bit-identical inputs.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Output i of a stream seeded with s is
mix(s + (i+1)*0x9E3779B97F4A7C15) with the published 64-bit finaliser; a double in
[0,1) is the top 53 bits times 2^-53.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1

# problem kinds
PDE_POISSON = 0   # -Laplace(u) = f, Dirichlet data on every face
PDE_HEAT = 1      # u_t - kappa * Laplace_x(u) = f, last coordinate is time;
                  # Dirichlet data on spatial faces, initial data on t = lo
PDE_OSC = 2       # m u'' + mu u' + k u = f in 1D (time), u and u' given at t = lo

# activations of the subdomain networks
ACT_TANH, ACT_SIGMOID, ACT_SIN = 0, 1, 2

# manufactured-solution families
FAM_SINPROD = 0       # u = sum_m c_m prod_i sin(k_mi pi x_i)         (Poisson)
FAM_HEAT_SINPROD = 1  # u = sum_m c_m exp(-kappa pi^2 |k_m|^2 t) prod_i sin(k_mi pi x_i)  (heat)
FAM_PARAM5 = 2        # f = sin(a pi x) sin(b pi y) + c sin(d pi x + e pi y), g = 0, no closed form
FAM_OSC = 3           # damped oscillator with u(lo) = 1, u'(lo) = 0; fparams = (m, mu, k)

MAX_MODES = 8


def splitmix64_u64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + i * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_unit(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): top 53 bits of each output times 2^-53."""
    return (splitmix64_u64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class Problem:
    """One ELM-FBPINN problem instance on the box prod_i [lo_i, hi_i].

    Fields mirror the paper's knobs (Sec. 4.2): S subdomains per dimension,
    overlap ratio delta (subdomain width / centre spacing), K features per
    subdomain, and a regular cell-centred interior collocation grid of n points
    per dimension.  Boundary rows use the interior grid of the other
    dimensions on each face.
    """
    dim: int
    pde: int
    S: Sequence[int]
    delta: float
    K: int
    n: Sequence[int]
    family: int
    coef: Sequence[float] = ()
    waves: Sequence[Sequence[float]] = ()
    fparams: Sequence[float] = ()
    kappa: float = 0.0
    lo: Sequence[float] = (0.0, 0.0, 0.0)
    hi: Sequence[float] = (1.0, 1.0, 1.0)
    lam: Sequence[float] = (1.0, 1.0)
    R: float = 5.0          # feature parameters drawn from U(-R, R)
    seed: int = 0
    n_test: Sequence[int] = ()   # test grid (cell-centred) per dimension
    name: str = ""
    depth: int = 1          # h of Eq. (2): h - 1 hidden layers of K units before the features
    act: int = ACT_TANH     # activation of every layer
    hard_bc: float = 0.0    # > 0: the hard-constraint ansatz of the Laplace problem with this factor
    init: str = "range"     # "range": weights U(-R/2, R/2), biases U(-R, R); "lecun": uniform LeCun

    @property
    def params_per_subdomain(self) -> int:
        """Doubles of one subdomain network: the output layer (K rows of
        w_1..w_n, b, n = dim for h = 1, else K), then each hidden layer's
        weights (K x n_in, row-major) and biases (K)."""
        n_last = self.dim if self.depth <= 1 else self.K
        c = self.K * (n_last + 1)
        nin = self.dim
        for _ in range(1, max(1, self.depth)):
            c += self.K * (nin + 1)
            nin = self.K
        return c

    @property
    def J(self) -> int:
        return int(np.prod([int(s) for s in self.S[: self.dim]]))

    def fam_vector(self) -> np.ndarray:
        """Family coefficients packed as 64 doubles.

        FAM_SINPROD / FAM_HEAT_SINPROD: slot 4m is c_m, slots 4m+1..4m+3 the
        wave numbers k_m (one per spatial dimension).  FAM_PARAM5: slots 0..4
        are (a, b, c, d, e).
        """
        v = np.zeros(64, dtype=np.float64)
        if self.family in (FAM_SINPROD, FAM_HEAT_SINPROD):
            assert len(self.coef) <= MAX_MODES
            for m, (c, k) in enumerate(zip(self.coef, self.waves)):
                v[4 * m] = c
                for i, kk in enumerate(k):
                    v[4 * m + 1 + i] = kk
        else:
            v[: len(self.fparams)] = self.fparams
        return v

    @property
    def n_modes(self) -> int:
        return len(self.coef) if self.family in (FAM_SINPROD, FAM_HEAT_SINPROD) else 0


def feature_params(p: Problem, seed: Optional[int] = None) -> np.ndarray:
    """Random network parameters: shape (J, K, dim+1), (w_1..w_d, b) per
    feature, for one-layer networks with the "range" draw; else (J, P) with P
    = p.params_per_subdomain in the layout described there.

    The features act on the input normalised to [-1, 1] over the subdomain
    (x - mu) / sig (sig the half-width).  Workloads state "weights U(-R, R)
    scaled by 1/subdomain width": a raw weight U(-R, R) / (2 sig) on x is a
    weight U(-R, R) / 2 on the normalised input, which is what is stored;
    biases are U(-R, R).
    Draw order: subdomain j (lexicographic, dimension 0 fastest), then feature k,
    then w_1..w_d, then b; each value is R * (2u - 1) with u from SplitMix64.
    "lecun": every weight and bias of a layer with n inputs is drawn from
    U(-sqrt(3/n), sqrt(3/n)) (uniform LeCun initialisation, Sec. 4.2, read as
    applying to the biases too), in the layout order.
    """
    s = p.seed if seed is None else seed
    if p.depth <= 1 and p.init == "range":
        n = p.J * p.K * (p.dim + 1)
        u = splitmix64_unit(s, n)
        v = (p.R * (2.0 * u - 1.0)).reshape(p.J, p.K, p.dim + 1)
        v[:, :, : p.dim] *= 0.5
        return v
    P = p.params_per_subdomain
    u = splitmix64_unit(s, p.J * P).reshape(p.J, P)
    lim = np.empty(P)
    n_last = p.dim if p.depth <= 1 else p.K
    lim[: p.K * (n_last + 1)] = math.sqrt(3.0 / n_last)
    o, nin = p.K * (n_last + 1), p.dim
    for _ in range(1, max(1, p.depth)):
        lim[o: o + p.K * (nin + 1)] = math.sqrt(3.0 / nin)
        o += p.K * (nin + 1)
        nin = p.K
    v = lim * (2.0 * u - 1.0)
    if p.depth <= 1:
        return v.reshape(p.J, p.K, p.dim + 1)
    return v


# ---------------------------------------------------------------------------
# Workloads.  Sizes follow the published workload descriptions.  Readings of
# ambiguous items: the overlap ratio (subdomain width over centre spacing) is
# 1 + the stated overlap fraction; collocation points are cell-centred uniform
# grids; boundary points lie on each face at the interior grid's cell-centred
# coordinates in the other dimensions (so no point sits on a corner).
# ---------------------------------------------------------------------------

def poisson1d(S=20, K=100, n=1600, delta=1.3, R=5.0, seed=0, n_test=1000) -> Problem:
    """1D Poisson -u'' = f on [0,1], u = sin(2 pi x) + 0.1 sin(50 pi x)."""
    return Problem(dim=1, pde=PDE_POISSON, S=[S], delta=delta, K=K, n=[n],
                   family=FAM_SINPROD, coef=[1.0, 0.1], waves=[[2.0], [50.0]],
                   R=R, seed=seed, n_test=[n_test], name=f"poisson1d_S{S}_K{K}_n{n}")


def poisson2d(S=20, K=300, n=None, delta=1.25, R=8.0, seed=0, n_test=400) -> Problem:
    """2D Poisson on [0,1]^2, u = sin2pix sin2piy + 0.05 sin30pix sin30piy.

    Interior grid: the paper's collocation rule S * ceil(K^(1/d)) points per
    dimension (Sec. 4.2), 360 for S = 20, K = 300, which keeps the global
    system tall; n = 200 gives the literal 200 x 200 grid of the workload
    description (an underdetermined system, kept as a parity case)."""
    if n is None:
        n = S * int(math.ceil(K ** 0.5 - 1e-12))
    return Problem(dim=2, pde=PDE_POISSON, S=[S, S], delta=delta, K=K, n=[n, n],
                   family=FAM_SINPROD, coef=[1.0, 0.05], waves=[[2.0, 2.0], [30.0, 30.0]],
                   R=R, seed=seed, n_test=[n_test, n_test], name=f"poisson2d_S{S}_K{K}_n{n}")


def heat3d(S=10, K=500, n=100, delta=1.2, R=5.0, kappa=0.01, k=6.0, seed=0, n_test=50) -> Problem:
    """(2+1)D heat u_t = kappa Lap u, u = exp(-2 kappa pi^2 k^2 t) sin(k pi x) sin(k pi y)."""
    return Problem(dim=3, pde=PDE_HEAT, S=[S, S, S], delta=delta, K=K, n=[n, n, n],
                   family=FAM_HEAT_SINPROD, coef=[1.0], waves=[[k, k]], kappa=kappa,
                   R=R, seed=seed, n_test=[n_test] * 3, name=f"heat3d_S{S}_K{K}_n{n}")


def oscillator(S=20, K=8, delta=2.9, omega0=60.0, mu=4.0, m=1.0, seed=0, act=ACT_TANH, depth=1) -> Problem:
    """The damped harmonic oscillator of Sec. 4.1: m u'' + mu u' + k u = 0 on
    [0, 1], u(0) = 1, u'(0) = 0, k = m omega0^2 (m = 1, mu = 4, omega0 = 60 in
    the paper's baseline), S subdomains at overlap ratio delta, K features,
    S ceil(K) interior collocation points (Sec. 4.2), uniform LeCun features,
    test points 50 S (Sec. 4.3)."""
    return Problem(dim=1, pde=PDE_OSC, S=[S], delta=delta, K=K, n=[S * K], family=FAM_OSC,
                   fparams=[m, mu, m * omega0 * omega0], seed=seed, n_test=[50 * S], init="lecun", act=act,
                   depth=depth, name=f"oscillator_w{omega0:g}_S{S}_K{K}")


def laplace_multiscale(n_scales=3, S=16, K=16, delta=2.9, seed=0, act=ACT_TANH, depth=1) -> Problem:
    """The multi-scale Laplace problem of Sec. 4.1: -Lap u = f on [0,1]^2,
    u = 0 on the boundary, u = (1/n) sum_i sin(w_i pi x) sin(w_i pi y) with
    w_i = 2^i (i = 1..n), by the hard-constraint ansatz with factor w_n (no
    boundary rows); S x S subdomains, overlap ratio delta, K features, S
    ceil(sqrt K) collocation points per dimension, 6 S test points per
    dimension (Sec. 4.4)."""
    import math as _m
    n = S * int(_m.ceil(K ** 0.5 - 1e-12))
    coef = [1.0 / n_scales] * n_scales
    waves = [[2.0 ** i, 2.0 ** i] for i in range(1, n_scales + 1)]
    return Problem(dim=2, pde=PDE_POISSON, S=[S, S], delta=delta, K=K, n=[n, n], family=FAM_SINPROD, coef=coef,
                   waves=waves, seed=seed, n_test=[6 * S, 6 * S], init="lecun", act=act, depth=depth,
                   hard_bc=2.0 ** n_scales, name=f"laplace_n{n_scales}_S{S}_K{K}")


def batched_instance(i: int, S_range=(8, 24), K_range=(100, 400), p_range=(40, 200),
                     delta=1.25, R=5.0) -> Problem:
    """Instance i of the batched 2D Poisson family: seeded S, K, points per
    subdomain spacing p and four separable sine modes with wave numbers
    U[1, 20] and amplitudes U[0.5, 1]."""
    seed = 1000 + i
    u = splitmix64_unit(seed, 16, offset=1 << 40)   # disjoint from the feature stream
    S = int(S_range[0] + math.floor(u[0] * (S_range[1] - S_range[0] + 1)))
    K = int(K_range[0] + math.floor(u[1] * (K_range[1] - K_range[0] + 1)))
    p = int(p_range[0] + math.floor(u[2] * (p_range[1] - p_range[0] + 1)))
    coef = [0.5 + 0.5 * u[3 + m] for m in range(4)]
    waves = [[1.0 + 19.0 * u[7 + 2 * m], 1.0 + 19.0 * u[8 + 2 * m]] for m in range(4)]
    n = (S - 1) * p
    return Problem(dim=2, pde=PDE_POISSON, S=[S, S], delta=delta, K=K, n=[n, n],
                   family=FAM_SINPROD, coef=coef, waves=waves, R=R, seed=seed,
                   n_test=[200, 200], name=f"batch{i}_S{S}_K{K}_p{p}")


def param5(a, b, c, d, e, S=20, K=300, n=200, delta=1.25, R=8.0, seed=0, n_test=400) -> Problem:
    """2D Poisson family f = sin(a pi x) sin(b pi y) + c sin(d pi x + e pi y), g = 0."""
    return Problem(dim=2, pde=PDE_POISSON, S=[S, S], delta=delta, K=K, n=[n, n],
                   family=FAM_PARAM5, fparams=[a, b, c, d, e], R=R, seed=seed,
                   n_test=[n_test, n_test], name="param5")


def param5_context(fp) -> np.ndarray:
    """(a, b, c, d, e) scaled by their ranges' upper ends to O(1) network inputs."""
    a, b, c, d, e = fp
    return np.array([a / 12.0, b / 12.0, c / 0.5, d / 30.0, e / 30.0], dtype=np.float32)


def param5_amplitude_scale(fp) -> float:
    """pi^2 (a^2 + b^2): the inverse amplitude of the dominant part of the
    solution (-Laplace sin(a pi x) sin(b pi y) = pi^2 (a^2 + b^2) sin sin),
    used to bring the family's solutions to a common scale."""
    a, b = fp[0], fp[1]
    return float(np.pi ** 2 * (a * a + b * b))


def param5_draw(seed: int) -> List[float]:
    """(a, b, c, d, e) with a, b ~ U[1,12], c ~ U[0,0.5], d, e ~ U[10,30]."""
    u = splitmix64_unit(seed, 5, offset=1 << 41)
    return [1 + 11 * u[0], 1 + 11 * u[1], 0.5 * u[2], 10 + 20 * u[3], 10 + 20 * u[4]]
