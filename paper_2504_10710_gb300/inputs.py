"""Seeded synthetic workloads for the GLL Poisson solver.

This module only *describes* problems: a structured element grid on the unit
square/cube, a smooth deformation map, a right-hand side f and Dirichlet data g
given as closed-form functions of the physical coordinates, all with seeded
random parameters.  It contains none of the solver's arithmetic: no quadrature,
no basis, no operator.  The caller supplies the undeformed node positions
(wherever its own GLL nodes put them) and gets back physical coordinates and
nodal samples of f and g.  Both the CUDA path and the CPU oracle consume the
same workload objects, so their inputs agree up to the rounding of their own
node computations.

Sign convention: the solver treats -Laplace(u) = f (weak form of Sec. 2.1,
integral of grad u . grad v = integral of f v), so a manufactured solution u
comes with f = -Laplace(u).

Workloads (seeds are numpy.random.default_rng(2504_10710 + 1000*cfg + i)):
  * ``square_sine``      4x4 undeformed elements, p=4, u = sin(pi x) sin(pi y).
  * ``terrain2d``        64x64 elements, p=8, y' = y + A sin(2 pi x)(1-y), A=0.1,
                         f = sum of 16 seeded Fourier modes, seeded smooth g.
  * ``terrain3d``        16^3 elements, p=7,
                         z' = z + 0.15 sin(2 pi x) cos(2 pi y)(1-z), 32 seeded
                         right-hand sides, g = 0.
  * ``table1_problem1``  one element, -Laplace(u) = 1, u = 0 on the boundary.
  * ``table1_problem3``  one element, u = sin(8 pi / (x + y + pi/10)).
  * ``random2d/3d``      any element grid / order / amplitude, for parity tests.
  * ``batch_uneven``     independent 2-D problems, n x n elements with n ~ U{4..64},
                         p ~ U{4..12}, amplitude ~ U(0, 0.2), terrain2d generators.
  * ``serving_stream``   Poisson arrivals over a pool of 2-D (batch_uneven
                         distribution) and 3-D (n^3, n ~ U{8..32}, p ~ U{4..8})
                         meshes, several seeded right-hand sides per mesh.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np

SEED_BASE = 2504_10710


def rng_for(cfg_id: int, i: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + 1000 * cfg_id + i)


@dataclass
class Workload:
    """A problem description: grid, map, f and g (closed forms, seeded)."""

    name: str
    dim: int
    nelem: tuple          # elements per physical axis (x, y[, z])
    order: int            # GLL order p of the finest level
    map: Callable         # (X, Y[, Z]) undeformed -> tuple of physical coords
    rhs: Sequence[Callable]  # one f(x, y[, z]) per right-hand side
    dirichlet: Callable   # g(x, y[, z]); only boundary samples are used
    exact: Callable | None = None  # exact solution when manufactured
    params: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return len(self.rhs)

    def grid_shape(self, order: int | None = None) -> tuple:
        """Global node array shape, slowest axis first: (Nz, Ny, Nx)."""
        p = self.order if order is None else order
        return tuple(self.nelem[a] * p + 1 for a in reversed(range(self.dim)))

    def ndof(self) -> int:
        return int(np.prod(self.grid_shape()))

    # ---- sampling helpers (the caller provides the 1-D node positions) ----
    def undeformed_nodes(self, ref_nodes: np.ndarray) -> list[np.ndarray]:
        """Global undeformed coordinates from reference nodes in [-1, 1].

        Returns one array per physical axis, each of the global grid shape,
        for the unit square/cube split into ``nelem`` equal elements.
        """
        p = len(ref_nodes) - 1
        lines = []
        for a in range(self.dim):
            E = self.nelem[a]
            t = np.empty(E * p + 1)
            for e in range(E):
                t[e * p:(e + 1) * p + 1] = (e + 0.5 * (np.asarray(ref_nodes) + 1.0)) / E
            t[0], t[-1] = 0.0, 1.0
            lines.append(t)
        # meshgrid with 'ij' indexing in slowest-first order
        grids = np.meshgrid(*[lines[a] for a in reversed(range(self.dim))], indexing="ij")
        return [grids[self.dim - 1 - a] for a in range(self.dim)]

    def coords(self, ref_nodes: np.ndarray) -> np.ndarray:
        """Physical coordinates, shape (dim, *grid)."""
        und = self.undeformed_nodes(ref_nodes)
        return np.stack(self.map(*und))

    def sample_rhs(self, coords: np.ndarray) -> np.ndarray:
        """f samples, shape (nrhs, *grid)."""
        return np.stack([f(*coords) for f in self.rhs])

    def sample_dirichlet(self, coords: np.ndarray) -> np.ndarray:
        return np.asarray(self.dirichlet(*coords), dtype=np.float64)


# --------------------------------------------------------------------------
# maps
# --------------------------------------------------------------------------
def terrain2d_map(amp: float):
    def m(X, Y):
        return X, Y + amp * np.sin(2 * np.pi * X) * (1.0 - Y)
    return m


def terrain3d_map(amp: float):
    def m(X, Y, Z):
        return X, Y, Z + amp * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * (1.0 - Z)
    return m


def identity_map(*X):
    return X


# --------------------------------------------------------------------------
# right-hand sides and Dirichlet data
# --------------------------------------------------------------------------
_CHUNK = 1 << 20


def _sine_harmonics(t: np.ndarray, kmax: int, out: np.ndarray, tmp: np.ndarray) -> np.ndarray:
    """out[k] = sin(pi k t) for k = 0..kmax by the recurrence
    sin((k+1) a) = 2 cos(a) sin(k a) - sin((k-1) a), a = pi t (in place)."""
    n = t.size
    h = out[:, :n]
    c2 = tmp[:n]
    h[0] = 0.0
    np.multiply(t, np.pi, out=c2)
    np.sin(c2, out=h[1])
    np.cos(c2, out=c2)
    c2 *= 2.0
    for k in range(2, kmax + 1):
        np.multiply(c2, h[k - 1], out=h[k])
        h[k] -= h[k - 2]
    return h


def _fourier_sum(coords, a, ks, kmax):
    """sum_k a[k] prod_axis sin(pi ks[k, axis] x_axis), evaluated in chunks
    of nodes with the sine harmonics of each coordinate tabulated once
    (buffers reused across chunks)."""
    shape = np.shape(coords[0])
    flat = [np.ascontiguousarray(c, dtype=np.float64).reshape(-1) for c in coords]
    out = np.empty(flat[0].size, dtype=np.float64)
    ch = min(_CHUNK, max(1, out.size))
    tabs = [np.empty((kmax + 1, ch)) for _ in flat]
    tmp, term = np.empty(ch), np.empty(ch)
    for s0 in range(0, out.size, ch):
        n = min(out.size, s0 + ch) - s0
        h = [_sine_harmonics(c[s0:s0 + n], kmax, tb, tmp) for c, tb in zip(flat, tabs)]
        acc = out[s0:s0 + n]
        acc[:] = 0.0
        t = term[:n]
        for k in range(len(a)):
            np.multiply(h[0][ks[k][0]], a[k], out=t)
            for ax in range(1, len(flat)):
                t *= h[ax][ks[k][ax]]
            acc += t
    return out.reshape(shape)


def fourier_rhs_2d(rng: np.random.Generator, nmodes: int = 16, kmax: int = 8):
    """f = sum of nmodes products sin(pi m x) sin(pi n y), a ~ N(0, 1),
    m, n ~ U{1..kmax}."""
    a = rng.standard_normal(nmodes)
    m = rng.integers(1, kmax + 1, nmodes)
    n = rng.integers(1, kmax + 1, nmodes)
    ks = np.stack([m, n], axis=1)

    def f(x, y):
        return _fourier_sum((x, y), a, ks, kmax)
    return f, dict(a=a.tolist(), m=m.tolist(), n=n.tolist())


def fourier_rhs_3d(rng: np.random.Generator, nmodes: int = 16, kmax: int = 8):
    """f = sum of nmodes products sin(pi k1 x) sin(pi k2 y) sin(pi k3 z),
    a ~ N(0, 1), k ~ U{1..kmax}^3."""
    a = rng.standard_normal(nmodes)
    ks = rng.integers(1, kmax + 1, (nmodes, 3))

    def f(x, y, z):
        return _fourier_sum((x, y, z), a, ks, kmax)
    return f, dict(a=a.tolist(), k=ks.tolist())


def smooth_dirichlet_2d(rng: np.random.Generator, nmodes: int = 4):
    b = rng.standard_normal(nmodes)
    c = rng.integers(0, 4, nmodes)
    d = rng.integers(0, 4, nmodes)
    th = rng.uniform(0.0, 2 * np.pi, nmodes)

    def g(x, y):
        out = np.zeros_like(x, dtype=np.float64)
        for k in range(nmodes):
            out += b[k] * np.cos(np.pi * (c[k] * x + d[k] * y) + th[k])
        return out
    return g, dict(b=b.tolist(), c=c.tolist(), d=d.tolist(), theta=th.tolist())


def smooth_dirichlet_3d(rng: np.random.Generator, nmodes: int = 4):
    b = rng.standard_normal(nmodes)
    c = rng.integers(0, 4, (nmodes, 3))
    th = rng.uniform(0.0, 2 * np.pi, nmodes)

    def g(x, y, z):
        out = np.zeros_like(x, dtype=np.float64)
        for k in range(nmodes):
            out += b[k] * np.cos(np.pi * (c[k, 0] * x + c[k, 1] * y + c[k, 2] * z) + th[k])
        return out
    return g, dict(b=b.tolist(), c=c.tolist(), theta=th.tolist())


def _zero(*x):
    return np.zeros_like(x[0], dtype=np.float64)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def square_sine() -> Workload:
    """4x4 undeformed elements, p = 4; u = sin(pi x) sin(pi y), g = 0."""
    def u(x, y):
        return np.sin(np.pi * x) * np.sin(np.pi * y)

    def f(x, y):
        return 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)
    return Workload("square_sine_4x4_p4", 2, (4, 4), 4, identity_map, [f], _zero, exact=u)


def terrain2d(nelem: int = 64, order: int = 8, amp: float = 0.1) -> Workload:
    """Terrain-deformed unit square, 16 random Fourier modes, random smooth g."""
    f, fp = fourier_rhs_2d(rng_for(1, 0))
    g, gp = smooth_dirichlet_2d(rng_for(1, 1))
    return Workload(f"terrain2d_{nelem}x{nelem}_p{order}", 2, (nelem, nelem), order,
                    terrain2d_map(amp), [f], g, params=dict(amp=amp, f=fp, g=gp))


def terrain3d(nelem: int = 16, order: int = 7, nrhs: int = 32, amp: float = 0.15) -> Workload:
    """Hex mesh with a deformed bottom face, ``nrhs`` seeded right-hand sides, g = 0."""
    fs = []
    fps = []
    for j in range(nrhs):
        f, fp = fourier_rhs_3d(rng_for(2, j))
        fs.append(f)
        fps.append(fp)
    return Workload(f"terrain3d_{nelem}^3_p{order}_x{nrhs}", 3, (nelem,) * 3, order,
                    terrain3d_map(amp), fs, _zero, params=dict(amp=amp, f=fps))


def table1_problem1(order: int) -> Workload:
    """Single element on [0,1]^2, -Laplace(u) = 1 (the paper's Lap u = -1), g = 0."""
    def f(x, y):
        return np.ones_like(x, dtype=np.float64)
    return Workload(f"table1_p1_p{order}", 2, (1, 1), order, identity_map, [f], _zero)


def table1_problem3(order: int) -> Workload:
    """Single element, u = sin(8 pi / (x + y + pi/10)), non-homogeneous Dirichlet."""
    c = np.pi / 10.0

    def u(x, y):
        return np.sin(8 * np.pi / (x + y + c))

    def f(x, y):
        s = x + y + c
        # Laplace(u) = 2 * u''(s) with u(s) = sin(8 pi / s)
        d2 = (-(64 * np.pi ** 2) / s ** 4 * np.sin(8 * np.pi / s)
              + (16 * np.pi) / s ** 3 * np.cos(8 * np.pi / s))
        return -2.0 * d2
    return Workload(f"table1_p3_p{order}", 2, (1, 1), order, identity_map, [f], u, exact=u)


def random2d(nelem: Sequence[int], order: int, amp: float = 0.1, seed: int = 0,
             nrhs: int = 1) -> Workload:
    """Deformed 2-D grid of any size for parity tests (cfg2 map and generators)."""
    fs = [fourier_rhs_2d(rng_for(7, 2 * seed + 17 * j))[0] for j in range(nrhs)]
    g, _ = smooth_dirichlet_2d(rng_for(7, 2 * seed + 1))
    ne = tuple(int(n) for n in nelem)
    return Workload(f"random2d_{ne[0]}x{ne[1]}_p{order}_s{seed}", 2, ne, order,
                    terrain2d_map(amp), fs, g, params=dict(amp=amp, seed=seed))


def random3d(nelem: Sequence[int], order: int, amp: float = 0.15, seed: int = 0,
             nrhs: int = 1) -> Workload:
    """Deformed 3-D grid of any size for parity tests (cfg3 map and generators)."""
    fs = [fourier_rhs_3d(rng_for(8, 2 * seed + 17 * j))[0] for j in range(nrhs)]
    g, _ = smooth_dirichlet_3d(rng_for(8, 2 * seed + 1))
    ne = tuple(int(n) for n in nelem)
    return Workload(f"random3d_{'x'.join(map(str, ne))}_p{order}_s{seed}", 3, ne, order,
                    terrain3d_map(amp), fs, g, params=dict(amp=amp, seed=seed))


def batch_uneven(count: int = 256) -> list[Workload]:
    """Independent 2-D problems of uneven size for batched solves: problem i
    draws n ~ U{4..64} (n x n elements), p ~ U{4..12} and an amplitude
    A ~ U(0, 0.2) of the terrain2d map, then a right-hand side and Dirichlet
    data from the terrain2d generators (seeds 2504_10710 + 3000 + i)."""
    out = []
    for i in range(count):
        rng = rng_for(3, i)
        n = int(rng.integers(4, 65))
        p = int(rng.integers(4, 13))
        amp = float(rng.uniform(0.0, 0.2))
        f, fp = fourier_rhs_2d(rng)
        g, gp = smooth_dirichlet_2d(rng)
        out.append(Workload(f"batch{i}_{n}x{n}_p{p}_a{amp:.3f}", 2, (n, n), p, terrain2d_map(amp), [f], g,
                            params=dict(amp=amp, f=fp, g=gp)))
    return out


def serving_stream(nreq: int = 2000, rate: float = 200.0, pool2d: int = 16, pool3d: int = 8,
                   nmax3d: int = 32, rhs_per_mesh: int = 4, seed: int = 0):
    """Poisson-arrival request stream of the serving workload.

    A pool of meshes drawn from the serving distributions: ``pool2d`` 2-D
    meshes from the batch_uneven generator (n ~ U{4..64}, n x n elements,
    p ~ U{4..12}, amplitude ~ U(0, 0.2)) and ``pool3d`` 3-D meshes with
    n ~ U{8..nmax3d} (n^3 elements), p ~ U{4..8} and the terrain3d map at
    amplitude 0.15; the largest 3-D draw is replaced by n = nmax3d, p = 8 so
    that the pool covers the top of the range.  Every mesh carries
    ``rhs_per_mesh`` seeded right-hand sides (16 Fourier modes) and seeded
    smooth Dirichlet data.  Then ``nreq`` requests, half 2-D and half 3-D in
    a seeded order, each on a mesh drawn uniformly from its half of the pool
    with one of that mesh's right-hand sides, arrival gaps exponential with
    mean 1/rate (seeds 2504_10710 + 5000 + i).

    Returns (meshes, requests): meshes a list of Workload (one right-hand
    side function per seeded RHS), requests a list of (arrival_s,
    mesh_index, rhs_index)."""
    rng = rng_for(5, seed)
    meshes = []
    for i in range(pool2d):
        r = rng_for(5, 1000 + i)
        n = int(r.integers(4, 65))
        p = int(r.integers(4, 13))
        amp = float(r.uniform(0.0, 0.2))
        fs = [fourier_rhs_2d(r)[0] for _ in range(rhs_per_mesh)]
        g, _ = smooth_dirichlet_2d(r)
        meshes.append(Workload(f"serve2d{i}_{n}x{n}_p{p}_a{amp:.3f}", 2, (n, n), p, terrain2d_map(amp), fs, g,
                               params=dict(amp=amp)))
    draws = []
    for i in range(pool3d):
        r = rng_for(5, 2000 + i)
        draws.append((int(r.integers(8, nmax3d + 1)), int(r.integers(4, 9)), r))
    big = max(range(pool3d), key=lambda i: draws[i][0] ** 3 * draws[i][1] ** 3) if pool3d else None
    for i, (n, p, r) in enumerate(draws):
        if i == big:
            n, p = nmax3d, 8
        fs = [fourier_rhs_3d(r)[0] for _ in range(rhs_per_mesh)]
        g, _ = smooth_dirichlet_3d(r)
        meshes.append(Workload(f"serve3d{i}_{n}^3_p{p}", 3, (n, n, n), p, terrain3d_map(0.15), fs, g,
                               params=dict(amp=0.15)))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    kinds = rng.permutation(np.arange(nreq) % 2)          # 0: 2-D, 1: 3-D
    reqs = []
    for k in range(nreq):
        if kinds[k] == 0 or pool3d == 0:
            mi = int(rng.integers(0, pool2d))
        else:
            mi = pool2d + int(rng.integers(0, pool3d))
        reqs.append((float(arrivals[k]), mi, int(rng.integers(0, rhs_per_mesh))))
    return meshes, reqs


def random_field(shape, seed: int) -> np.ndarray:
    """Seeded N(0,1) nodal field, e.g. a vector to apply an operator to."""
    return np.random.default_rng(SEED_BASE + 9000 + seed).standard_normal(shape)
