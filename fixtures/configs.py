"""The five synthetic workloads (stand-ins for the paper's SuiteSparse/FreeFem++ set).

The paper's matrices (its Table 1) are not available; these PDE matrices have the
same character (SPD, 2D and 3D, large condition numbers, DBBD by nested dissection,
tens of subdomains) at the sizes listed below:

0. poisson2d_64   : 2D 5-point Poisson 64x64 (n=4096), a=1, 4 subdomains, k=16, p=10.
1. lognormal3d_64 : 3D 7-point, 64^3 (n=262144), lognormal a (ell=8 cells, sigma=2),
                    32 subdomains, k=64, p=16.
2. aniso2d_batch  : 64 independent 2D 5-point anisotropic problems, side N ~ U{100..400},
                    anisotropy ratio r log-uniform in [1, 1e3], angle theta ~ U[0, pi),
                    K_xx = cos^2 + sin^2 / r, K_yy = sin^2 + cos^2 / r (mixed term dropped),
                    subdomains ~ U{8, 16, 32, 64}, k=32, p=8.
3. lognormal2d_256: 2D 5-point 256x256 (n=65536), lognormal a with ell ~ U[4, 16],
                    sigma ~ U[1, 3] per field seed, 16 subdomains, k=48, p=8.
4. aniso3d_128    : 3D 7-point 128^3 (n=2097152), axis scales (1, 1, 1e-3), lognormal a
                    (sigma=1.5, ell=8 cells), 256 subdomains, k=128, p=32.

All right-hand sides are b = A x* with x* ~ N(0, 1); sketches are N(0, 1).
"""

from dataclasses import dataclass, field

import numpy as np

from .fields import lognormal_grid_field
from .grids import diffusion_matrix, grid_coords
from .partition import interior_nd_order, nd_partition
from .seeds import rng_for

CONFIGS = {
    0: dict(name="poisson2d_64", shape=(64, 64), nsub=4, k=16, p=10, field=None),
    1: dict(name="lognormal3d_64", shape=(64, 64, 64), nsub=32, k=64, p=16,
            field=dict(ell=8.0, sigma=2.0)),
    2: dict(name="aniso2d_batch", count=64, nsub_choices=(8, 16, 32, 64), side=(100, 400),
            ratio=(1.0, 1e3), k=32, p=8, field=None),
    3: dict(name="lognormal2d_256", shape=(256, 256), nsub=16, k=48, p=8,
            field=dict(ell=(4.0, 16.0), sigma=(1.0, 3.0))),
    4: dict(name="aniso3d_128", shape=(128, 128, 128), nsub=256, k=128, p=32,
            axis_scale=(1.0, 1.0, 1e-3), field=dict(ell=8.0, sigma=1.5)),
}

EPS_INNER = 0.1   # inner block-CG relative tolerance (paper: eps_{S_I} = 0.1)
RTOL = 1e-8       # outer PCG relative tolerance


@dataclass
class Problem:
    name: str
    shape: tuple
    A: object                 # scipy.sparse.csr_matrix, float64, sorted indices
    part: np.ndarray          # int32, subdomain id or -1 for Gamma
    boxes: list               # (lo, hi) inclusive grid bounds of each subdomain
    nsub: int
    k: int
    p: int
    eps_inner: float = EPS_INNER
    rtol: float = RTOL
    coef: np.ndarray = None
    coords: np.ndarray = None
    meta: dict = field(default_factory=dict)
    leaf: int = 16
    _perm: np.ndarray = None

    @property
    def perm(self):
        """int64 elimination order of the interior nodes, block by block (geometric nested
        dissection inside each subdomain box), computed on first use."""
        if self._perm is None:
            self._perm = interior_nd_order(self.shape, self.boxes, self.leaf)
        return self._perm

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def gamma(self):
        """Interface node ids in increasing order (the order of Gamma-sized vectors)."""
        return np.nonzero(self.part < 0)[0]

    @property
    def n_gamma(self):
        return int((self.part < 0).sum())

    @property
    def s(self):
        return self.k + self.p


def _build(name, shape, nsub, k, p, coef=None, axis_scale=None, leaf=16, meta=None):
    A = diffusion_matrix(shape, coef, axis_scale)
    part, boxes = nd_partition(shape, nsub)
    return Problem(name=name, shape=tuple(shape), A=A, part=part, boxes=boxes, nsub=nsub,
                   k=k, p=p, coef=coef, coords=grid_coords(shape), meta=meta or {}, leaf=leaf)


def make_problem(config: int, index: int = 0):
    """Problem ``index`` of configuration ``config`` (index > 0 only for configs 2 and 3)."""
    c = CONFIGS[config]
    if config == 2:
        return problem_from_spec(batched_problem_specs()[index])
    shape = c["shape"]
    coef = None
    meta = {}
    if c["field"] is not None:
        rng = rng_for(config, index, "field")
        ell, sigma = c["field"]["ell"], c["field"]["sigma"]
        if isinstance(ell, tuple):
            ell = float(rng.uniform(*ell))
            sigma = float(rng.uniform(*sigma))
        coef = lognormal_grid_field(shape, ell, sigma, rng)
        meta = dict(ell=ell, sigma=sigma)
    return _build(c["name"], shape, c["nsub"], c["k"], c["p"], coef,
                  c.get("axis_scale"), meta=meta)


def batched_problem_specs(count=None):
    """Drawn parameters of the independent anisotropic 2D problems of configuration 2."""
    c = CONFIGS[2]
    count = c["count"] if count is None else count
    rng = rng_for(2, 0, "draw")
    specs = []
    for i in range(c["count"]):
        side = int(rng.integers(c["side"][0], c["side"][1] + 1))
        ratio = float(np.exp(rng.uniform(np.log(c["ratio"][0]), np.log(c["ratio"][1]))))
        theta = float(rng.uniform(0.0, np.pi))
        nsub = int(rng.choice(c["nsub_choices"]))
        specs.append(dict(index=i, side=side, ratio=ratio, theta=theta, nsub=nsub,
                          k=c["k"], p=c["p"]))
    return specs[:count]


def problem_from_spec(spec):
    th, r = spec["theta"], spec["ratio"]
    kxx = np.cos(th) ** 2 + np.sin(th) ** 2 / r
    kyy = np.sin(th) ** 2 + np.cos(th) ** 2 / r
    side = spec["side"]
    return _build("aniso2d_%d" % spec["index"], (side, side), spec["nsub"], spec["k"],
                  spec["p"], None, (kxx, kyy), meta=dict(spec))


def make_rhs(problem: Problem, config: int, index: int = 0):
    """(x_star, b) with x_star ~ N(0, 1) and b = A x_star."""
    x = rng_for(config, index, "xstar").standard_normal(problem.n)
    return x, problem.A @ x


def make_sketch(n_gamma: int, s: int, config: int, index: int = 0):
    """Gaussian sketch G (n_gamma x s, row-major float64) for parity runs."""
    return rng_for(config, index, "sketch").standard_normal((n_gamma, s))


def make_probe(rows: int, cols: int, config: int, index: int = 0):
    """Seeded N(0, 1) block (rows x cols) to probe an operator at full size."""
    return rng_for(config, index, "probe").standard_normal((rows, cols))


def sample_rows(n: int, count: int, config: int, index: int = 0):
    """Sorted distinct seeded row indices in [0, n) at which full-size outputs are compared."""
    rng = rng_for(config, index, "sample")
    return np.sort(rng.choice(n, size=min(count, n), replace=False))
