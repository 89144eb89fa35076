"""Seeded synthetic inputs for the additive sweeping preconditioner workloads.

This module is shared by the CPU oracle tests, the GPU tests and the benchmark.
It holds no arithmetic of the method itself (no PML profiles, no discretization,
no solver): only the velocity fields c(x), the right-hand sides f(x), the
problem parameters and the seeds.  Everything is returned as numpy arrays in
the grid ordering used throughout the project:

* 2D arrays are indexed ``a[i2-1, i1-1]`` (x1 fastest, the column-major
  ordering of the paper's Section 3.1), 3D arrays ``a[i3-1, i2-1, i1-1]``,
  1D arrays ``a[i-1]``; grid node ``i`` sits at ``x = i*h`` with
  ``h = 1/(n+1)`` (Sections 2 and 3.1).
* A batch of right-hand sides is stacked on a trailing axis:
  ``f[i2-1, i1-1, r]`` (point-major, right-hand side fastest).

The paper gives no parameters for its velocity fields and sources (Section
3.2 and Section 4.2 describe them in words and their figures are missing), so
the recipes below are the synthetic stand-ins; each one is named after what
it is and its sizes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem",
    "grid_nodes",
    "gaussian_source",
    "lens_velocity",
    "layered_velocity",
    "bump_velocity",
    "constant_velocity",
    "problem_2d_n127_const",
    "problem_2d_n511_lens",
    "problem_2d_n1023_layered",
    "problem_3d_n95_bump",
    "serving_stream",
    "small_problem",
]


@dataclasses.dataclass
class Problem:
    """One Helmholtz solve request: geometry, frequency, PML and layer sizes.

    ``c`` is the velocity on the grid nodes (shape ``(n,)*dim`` in the
    ordering described in the module docstring) and ``f`` the batch of
    right-hand sides with a trailing right-hand-side axis.
    """

    name: str
    dim: int
    n: int
    omega: float
    pml: int  # gamma: PML width eta = gamma*h
    b: int  # interior layer width (grid columns along the sweep axis)
    c: np.ndarray
    f: np.ndarray
    pml_aux: int | None = None  # width of the auxiliary PMLs (default gamma)
    C: float = 20.0  # PML strength constant
    tol: float = 1e-6
    restart: int = 40
    seed: int | None = None

    @property
    def gamma_aux(self) -> int:
        return self.pml if self.pml_aux is None else self.pml_aux

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[-1])


def grid_nodes(n: int, dim: int) -> list[np.ndarray]:
    """Coordinates of the interior nodes, one array per axis, broadcastable.

    Returns ``[x1, x2, ...]`` shaped for the array ordering of this module
    (x1 varies along the last numpy axis).
    """
    h = 1.0 / (n + 1)
    t = np.arange(1, n + 1, dtype=np.float64) * h
    out = []
    for ax in range(dim):
        shape = [1] * dim
        shape[dim - 1 - ax] = n
        out.append(t.reshape(shape))
    return out


def gaussian_source(n: int, dim: int, centre, width: float) -> np.ndarray:
    """f(x) = exp(-|x - centre|^2 / (2 width^2)) sampled at the grid nodes."""
    xs = grid_nodes(n, dim)
    r2 = np.zeros((n,) * dim, dtype=np.float64)
    for ax in range(dim):
        r2 = r2 + (xs[ax] - centre[ax]) ** 2
    return np.exp(-r2 / (2.0 * width * width))


def wave_packet(n: int, dim: int, centre, direction, omega: float, c_typ: float = 1.0,
                width: float | None = None) -> np.ndarray:
    """Gaussian wave packet (the paper's second force family, Section 3.2/4.2):
    envelope exp(-|x - centre|^2 / (2 s^2)) times the plane wave
    exp(i k d.(x - centre)) with k = omega / c_typ and unit direction d.  The
    paper gives no envelope width; s defaults to one wavelength 2 pi / k."""
    k = omega / c_typ
    s = width if width is not None else 2.0 * math.pi / k
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    xs = grid_nodes(n, dim)
    r2 = np.zeros((n,) * dim, dtype=np.float64)
    phase = np.zeros((n,) * dim, dtype=np.float64)
    for ax in range(dim):
        dx = xs[ax] - centre[ax]
        r2 = r2 + dx * dx
        phase = phase + d[ax] * dx
    return np.exp(-r2 / (2.0 * s * s)) * np.exp(1j * k * phase)


def constant_velocity(n: int, dim: int, value: float = 1.0) -> np.ndarray:
    return np.full((n,) * dim, value, dtype=np.float64)


def lens_velocity(n: int, dim: int = 2) -> np.ndarray:
    """Converging lens: c(x) = 4/3 * (1 - 0.5 exp(-32 |x - (1/2,..)|^2))."""
    xs = grid_nodes(n, dim)
    r2 = sum((x - 0.5) ** 2 for x in xs)
    return (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * r2)) * np.ones((n,) * dim)


def bump_velocity(n: int, dim: int = 3, height: float = 0.3) -> np.ndarray:
    """Constant c=1 plus a Gaussian bump: c = 1 + height*exp(-32|x-(1/2,..)|^2)."""
    xs = grid_nodes(n, dim)
    r2 = sum((x - 0.5) ** 2 for x in xs)
    return (1.0 + height * np.exp(-32.0 * r2)) * np.ones((n,) * dim)


def layered_velocity(n: int, seed: int, layers: int = 16, lo: float = 0.8,
                     hi: float = 1.2, smooth_h: float = 3.0, dim: int = 2) -> np.ndarray:
    """Random horizontal layers along the sweep axis (the last axis x_d).

    ``layers`` equal bands along x_d, each with a velocity drawn uniformly
    from [lo, hi] by numpy's PCG64 generator seeded with ``seed``; the band
    profile is then smoothed along x_d by a Gaussian filter of standard
    deviation ``smooth_h * h`` truncated at three standard deviations, with
    clamped (edge-replicating) ends.  The field is constant along the other
    axes.
    """
    rng = np.random.default_rng(seed)
    vals = rng.uniform(lo, hi, size=layers)
    i = np.arange(n)
    band = np.minimum((i * layers) // n, layers - 1)
    prof = vals[band]
    half = int(math.ceil(3.0 * smooth_h))
    k = np.arange(-half, half + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (k / smooth_h) ** 2)
    ker /= ker.sum()
    padded = np.concatenate([np.full(half, prof[0]), prof, np.full(half, prof[-1])])
    sm = np.convolve(padded, ker, mode="valid")
    assert sm.shape == (n,)
    shape = [n] + [1] * (dim - 1)
    return np.broadcast_to(sm.reshape(shape), (n,) * dim).astype(np.float64).copy()


def _stack(fs) -> np.ndarray:
    return np.stack(fs, axis=-1).astype(np.complex128)


def problem_2d_n127_const() -> Problem:
    """2D plain FP64 case: n=127 (h=1/128), omega=16*pi, c=1, PML 12, b=4,
    one Gaussian point source of width 2h at (x1, x2) = (0.5, 0.2)."""
    n = 127
    h = 1.0 / (n + 1)
    f = gaussian_source(n, 2, (0.5, 0.2), 2 * h)
    return Problem("2d_n127_const", 2, n, 16 * math.pi, 12, 4,
                   constant_velocity(n, 2), _stack([f]))


def problem_2d_n511_lens() -> Problem:
    """2D n=511, omega=64*pi, smooth lens velocity, PML 16, b=4, one Gaussian
    source of width 2h at (0.5, 0.2)."""
    n = 511
    h = 1.0 / (n + 1)
    f = gaussian_source(n, 2, (0.5, 0.2), 2 * h)
    return Problem("2d_n511_lens", 2, n, 64 * math.pi, 16, 4,
                   lens_velocity(n, 2), _stack([f]))


def problem_2d_n1023_layered(nrhs: int = 32, seed: int = 1504, source: str = "point") -> Problem:
    """2D n=1023, omega=128*pi, 16 random smoothed horizontal layers, PML 20,
    b=4, ``nrhs`` sources at seeded positions drawn uniformly from the physical
    square [gamma*h, 1-gamma*h]^2: Gaussian point sources of width 2h
    (``source="point"``) or Gaussian wave packets of one wavelength with seeded
    directions (``source="packet"``)."""
    n, gamma = 1023, 20
    h = 1.0 / (n + 1)
    omega = 128 * math.pi
    c = layered_velocity(n, seed, dim=2)
    rng = np.random.default_rng(seed + 1)
    lo, hi = gamma * h, 1.0 - gamma * h
    pos = rng.uniform(lo, hi, size=(nrhs, 2))
    if source == "point":
        fs = [gaussian_source(n, 2, tuple(p), 2 * h) for p in pos]
    elif source == "packet":
        ang = rng.uniform(0.0, 2.0 * math.pi, size=nrhs)
        fs = [wave_packet(n, 2, tuple(p), (math.cos(a), math.sin(a)), omega) for p, a in zip(pos, ang)]
    else:
        raise ValueError(source)
    return Problem("2d_n1023_layered" + ("" if source == "point" else "_packets"), 2, n, omega, gamma, 4, c,
                   _stack(fs), seed=seed)


def problem_3d_n95_bump() -> Problem:
    """3D n=95, omega=48*pi, c = 1 + 0.3 Gaussian bump at the centre, PML 8,
    slab width b=4, one Gaussian source (width 2h) at (0.5, 0.5, 0.25)."""
    n = 95
    h = 1.0 / (n + 1)
    f = gaussian_source(n, 3, (0.5, 0.5, 0.25), 2 * h)
    return Problem("3d_n95_bump", 3, n, 48 * math.pi, 8, 4, bump_velocity(n, 3), _stack([f]))


def small_problem(dim: int, n: int, omega: float, pml: int, b: int, velocity: str = "const",
                  nrhs: int = 1, seed: int = 7, pml_aux: int | None = None,
                  C: float = 20.0, source: str = "point") -> Problem:
    """A small seeded case for parity tests (several layers, ragged last layer).

    ``velocity`` is one of ``const``, ``lens``, ``layered``, ``bump``;
    sources are Gaussians of width 2h at seeded positions in the physical box.
    """
    h = 1.0 / (n + 1)
    if velocity == "const":
        c = constant_velocity(n, dim)
    elif velocity == "lens":
        c = lens_velocity(n, dim)
    elif velocity == "layered":
        c = layered_velocity(n, seed, dim=dim)
    elif velocity == "bump":
        c = bump_velocity(n, dim)
    else:
        raise ValueError(velocity)
    rng = np.random.default_rng(seed)
    lo, hi = pml * h, 1.0 - pml * h
    fs = []
    for _ in range(nrhs):
        p = rng.uniform(lo, hi, size=dim)
        if source == "point":
            fs.append(gaussian_source(n, dim, tuple(p), 2 * h))
        else:  # wave packet with a seeded direction
            d = rng.standard_normal(dim)
            fs.append(wave_packet(n, dim, tuple(p), tuple(d), omega))
    return Problem(f"{dim}d_n{n}_{velocity}", dim, n, omega, pml, b, c, _stack(fs),
                   pml_aux=pml_aux, C=C, seed=seed)


SERVING_PML = {255: 14, 511: 16, 1023: 20}


def serving_stream(num_requests: int = 2000, seed: int = 2016, rate_hz: float = 50.0,
                   sizes=(255, 511, 1023), velocity_pool: int = 64):
    """Poisson-arriving 2D requests.

    Each request draws n from ``sizes``, uses omega = n*pi/8 (16 points per
    wavelength at c=1), the PML width for that n, b=4, a layered velocity
    whose seed comes from a pool of ``velocity_pool`` seeds (so that factor
    caches can hit), and 1-8 Gaussian sources.  Returns a list of dicts with
    the arrival time in seconds and the parameters; fields are generated on
    demand with :func:`materialize`.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(num_requests):
        t += rng.exponential(1.0 / rate_hz)
        n = int(rng.choice(sizes))
        vseed = int(rng.integers(0, velocity_pool))
        nrhs = int(rng.integers(1, 9))
        src_seed = int(rng.integers(0, 2**31 - 1))
        reqs.append({"id": i, "t": t, "n": n, "omega": n * math.pi / 8.0,
                     "pml": SERVING_PML[n], "b": 4, "velocity_seed": vseed,
                     "nrhs": nrhs, "source_seed": src_seed})
    return reqs


def materialize(req: dict) -> Problem:
    """Build the velocity and right-hand sides of one serving request."""
    n, gamma = req["n"], req["pml"]
    h = 1.0 / (n + 1)
    c = layered_velocity(n, 10_000 + req["velocity_seed"], dim=2)
    rng = np.random.default_rng(req["source_seed"])
    lo, hi = gamma * h, 1.0 - gamma * h
    fs = [gaussian_source(n, 2, tuple(rng.uniform(lo, hi, size=2)), 2 * h)
          for _ in range(req["nrhs"])]
    return Problem(f"serve_{req['id']}", 2, n, req["omega"], gamma, req["b"], c, _stack(fs),
                   seed=req["velocity_seed"])
