"""Seeded synthetic inputs for the hierarchical solver: sparse matrices, grid
coordinates and right-hand sides.

This module holds none of the solver's arithmetic.  It only builds the linear
systems the paper solves in Sec. 5.1 (seven-point Poisson, variable-coefficient
Poisson, and the nonsymmetric/indefinite problems of Sec. 5.3 stand-ins) and the
random right-hand sides, so that the CUDA path and the CPU oracle are fed the
same bytes.

Conventions
-----------
* Unknowns are the cells of an ``nx x ny (x nz)`` grid in lexicographic order,
  x fastest: ``idx = i + nx*(j + ny*k)``.
* Matrices are returned as CSR with int64 ``rowptr``, int32 ``col`` (sorted,
  diagonal included) and float64 ``val``.
* Coordinates are the integer cell indices as float64, shape ``(n, dim)``.
* Homogeneous Dirichlet boundary: a row simply drops its exterior neighbours.
* Right-hand sides have shape ``(nrhs, n)`` C-contiguous, which is the
  column-major ``n x nrhs`` layout (leading dimension ``n``) the library uses.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Problem:
    name: str
    n: int
    rowptr: np.ndarray  # int64 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]
    coords: np.ndarray  # float64 [n, dim]
    symmetric: bool
    spd: bool
    grid: tuple

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    def dense(self) -> np.ndarray:
        """Dense copy (small problems only)."""
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            lo, hi = self.rowptr[i], self.rowptr[i + 1]
            a[i, self.col[lo:hi]] = self.val[lo:hi]
        return a

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _grid_coords(shape):
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    out = np.empty((n, len(shape)), dtype=np.float64)
    stride = 1
    for d, s in enumerate(shape):
        out[:, d] = (idx // stride) % s
        stride *= s
    return out


def _stencil_csr(shape, diag, offdiag):
    """Assemble a 2*dim+1 point stencil on a grid.

    ``diag``: float64 array of length n.  ``offdiag(d, s, lo_idx)`` returns the
    coefficients coupling cell ``lo_idx`` (flat index array) with its neighbour
    in direction ``d`` (``s=+1`` means the +x_d neighbour, ``s=-1`` the -x_d
    neighbour) for all cells whose neighbour exists.
    """
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[:d])) for d in range(dim)]
    idx = np.arange(n, dtype=np.int64)
    # per-axis integer coordinates
    coord = []
    rem = idx.copy()
    for d in range(dim):
        coord.append(rem % shape[d])
        rem //= shape[d]
    rows, cols, vals = [idx], [idx], [np.asarray(diag, dtype=np.float64)]
    for d in range(dim):
        for s in (-1, +1):
            ok = (coord[d] + s >= 0) & (coord[d] + s < shape[d])
            r = idx[ok]
            rows.append(r)
            cols.append(r + s * strides[d])
            vals.append(np.asarray(offdiag(d, s, r), dtype=np.float64))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return n, rowptr, cols.astype(np.int32), vals


def poisson(shape) -> Problem:
    """Unscaled (2*dim+1)-point Dirichlet Laplacian: diagonal 2*dim, off -1."""
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    nn, rp, c, v = _stencil_csr(shape, np.full(n, 2.0 * dim), lambda d, s, r: -np.ones(len(r)))
    return Problem(f"poisson{dim}d_{'x'.join(map(str, shape))}", nn, rp, c, v,
                   _grid_coords(shape), True, True, shape)


def _face_harmonic(shape, a):
    """Face coefficients from cell coefficients: harmonic mean 2ab/(a+b)."""
    shape = tuple(shape)
    strides = [int(np.prod(shape[:d])) for d in range(len(shape))]

    def off(d, s, r):
        ai = a[r]
        aj = a[r + s * strides[d]]
        return -(2.0 * ai * aj / (ai + aj))
    return off


def _diffusion(shape, a, name) -> Problem:
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    off = _face_harmonic(shape, a)
    # diagonal: sum of face coefficients; a Dirichlet boundary face uses the
    # cell's own coefficient (ghost cell with the same coefficient, zero value)
    diag = np.zeros(n)
    idx = np.arange(n, dtype=np.int64)
    coord, rem = [], idx.copy()
    for d in range(dim):
        coord.append(rem % shape[d])
        rem //= shape[d]
    strides = [int(np.prod(shape[:d])) for d in range(dim)]
    for d in range(dim):
        for s in (-1, +1):
            ok = (coord[d] + s >= 0) & (coord[d] + s < shape[d])
            diag[idx[ok]] += -off(d, s, idx[ok])
            diag[idx[~ok]] += a[idx[~ok]]
    nn, rp, c, v = _stencil_csr(shape, diag, off)
    return Problem(name, nn, rp, c, v, _grid_coords(shape), True, True, shape)


def vc_diffusion(shape, seed: int, log10_range: float = 3.0) -> Problem:
    """Variable-coefficient diffusion, cell coefficient 10**U(-r, r) i.i.d."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(-log10_range, log10_range, size=n)
    return _diffusion(shape, a, f"vcdiff{len(shape)}d_{'x'.join(map(str, shape))}")


def high_contrast(shape, seed: int, sigma_cells: float = 4.0) -> Problem:
    """The quantized high-contrast field of Sec. 5.1: uniform field, Gaussian
    blur of deviation 4h, then 1e2 where the blurred value exceeds 0.5, else
    1e-2.  Face coefficients are harmonic means."""
    from scipy.ndimage import gaussian_filter
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed)
    # field stored with axis 0 = x (fastest in the flat index), so reverse
    u = rng.uniform(0.0, 1.0, size=shape[::-1])
    u = gaussian_filter(u, sigma=sigma_cells, mode="reflect")
    a = np.where(u > 0.5, 1e2, 1e-2).reshape(-1)
    return _diffusion(shape, a, f"hcdiff{len(shape)}d_{'x'.join(map(str, shape))}")


def convection_diffusion(shape, peclet: float = 10.0) -> Problem:
    """-nu Lap u + v . grad u with v = (1,..,1), first-order upwind, scaled by
    h^2/nu.  Cell Peclet number Pe = |v_d| h / nu.  Diagonal 2*dim + dim*Pe,
    upwind (-x_d side) neighbour -(1+Pe), downwind neighbour -1: a
    nonsymmetric M-matrix."""
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    pe = float(peclet)
    nn, rp, c, v = _stencil_csr(
        shape, np.full(n, 2.0 * dim + dim * pe),
        lambda d, s, r: np.full(len(r), -(1.0 + pe) if s < 0 else -1.0))
    return Problem(f"convdiff{dim}d_{'x'.join(map(str, shape))}", nn, rp, c, v,
                   _grid_coords(shape), False, False, shape)


def helmholtz(shape, k2: float) -> Problem:
    """(-Lap - k^2) on the unscaled stencil: diagonal 2*dim - k2 (indefinite
    for k2 above the smallest Laplacian eigenvalue)."""
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    nn, rp, c, v = _stencil_csr(shape, np.full(n, 2.0 * dim - k2), lambda d, s, r: -np.ones(len(r)))
    return Problem(f"helmholtz{dim}d_{'x'.join(map(str, shape))}", nn, rp, c, v,
                   _grid_coords(shape), True, False, shape)


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides with entries uniform in [-1, 1]; shape (nrhs, n)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(nrhs, n)))


# The workloads the library is measured and tested on.  Each entry gives the
# problem constructor, the leaf (cluster) size and the solver settings.
def workload(name: str):
    """Return (problem, settings dict) for a named workload."""
    w = {
        # 2D 5-point Poisson 64x64, clusters of 64, eps 1e-3, one RHS, PCG
        "poisson2d_64": (lambda: poisson((64, 64)), dict(leaf=64, eps=1e-3, nrhs=1, krylov="pcg", rhs_seed=1000)),
        # 3D 7-point Poisson 64^3, clusters of 128, eps 1e-2, PCG
        "poisson3d_64": (lambda: poisson((64, 64, 64)), dict(leaf=128, eps=1e-2, nrhs=1, krylov="pcg", rhs_seed=1001)),
        "poisson3d_32": (lambda: poisson((32, 32, 32)), dict(leaf=128, eps=1e-2, nrhs=1, krylov="pcg", rhs_seed=1001)),
        "poisson3d_16": (lambda: poisson((16, 16, 16)), dict(leaf=64, eps=1e-2, nrhs=1, krylov="pcg", rhs_seed=1001)),
        "vcdiff3d_96": (lambda: vc_diffusion((96, 96, 96), seed=2002), dict(leaf=128, eps=1e-2, nrhs=1, krylov="pcg", rhs_seed=1002, equilibrate=1)),
        "convdiff3d_64": (lambda: convection_diffusion((64, 64, 64), 10.0), dict(leaf=128, eps=1e-2, nrhs=1, krylov="gmres", rhs_seed=1002)),
        "poisson3d_128": (lambda: poisson((128, 128, 128)), dict(leaf=128, eps=1e-2, nrhs=8, krylov="gmres", rhs_seed=1003)),
        # the paper's indefinite Helmholtz problem (Sec. 5.1): -Lap - k^2 at
        # 32 grid points per wavelength, GMRES to 1e-3
        "helmholtz3d_64": (lambda: helmholtz((64, 64, 64), helmholtz_k2(32.0)), dict(leaf=128, eps=1e-2, nrhs=1, krylov="gmres", rhs_seed=1004, tol=1e-3)),
        "helmholtz3d_32": (lambda: helmholtz((32, 32, 32), helmholtz_k2(32.0)), dict(leaf=128, eps=1e-2, nrhs=1, krylov="gmres", rhs_seed=1004, tol=1e-3)),
    }[name]
    return w[0](), dict(w[1])


def helmholtz_k2(points_per_wavelength: float) -> float:
    """k^2 h^2 of the unscaled Helmholtz stencil for a wavelength of the given
    number of grid spacings: k h = 2 pi / points_per_wavelength."""
    return (2.0 * np.pi / points_per_wavelength) ** 2


def sample_of(name: str, shape) -> Problem:
    """The problem family of workload `name` on a smaller grid (the bounded
    sample the CPU oracle is timed on)."""
    shape = tuple(int(x) for x in shape)
    if name.startswith("poisson"):
        return poisson(shape)
    if name.startswith("vcdiff"):
        return vc_diffusion(shape, seed=2002)
    if name.startswith("convdiff"):
        return convection_diffusion(shape, 10.0)
    if name.startswith("helmholtz"):
        return helmholtz(shape, helmholtz_k2(32.0))
    raise KeyError(name)


# The serving stream: six matrix families (2D Poisson 32^2, 128^2, 512^2; 3D
# Poisson 16^3, 64^3; 3D high-contrast diffusion 32^3, factored as S A S
# with the diagonal equilibration: its 1e4 coefficient contrast otherwise
# costs definiteness at this eps), eps 1e-2, mixed precision.  Families are drawn uniformly, 1-32 right-hand sides each,
# exponential inter-arrival times (Poisson arrivals).
SERVING_FAMILIES = {
    "poisson2d_32": (lambda: poisson((32, 32)), dict(leaf=64)),
    "poisson2d_128": (lambda: poisson((128, 128)), dict(leaf=64)),
    "poisson2d_512": (lambda: poisson((512, 512)), dict(leaf=64)),
    "poisson3d_16": (lambda: poisson((16, 16, 16)), dict(leaf=64)),
    "poisson3d_64": (lambda: poisson((64, 64, 64)), dict(leaf=128)),
    "hcdiff3d_32": (lambda: high_contrast((32, 32, 32), seed=5), dict(leaf=128, equilibrate=1)),
}


def serving_stream(n_requests: int = 2000, rate: float = 200.0, seed: int = 3000,
                   families=None, max_rhs: int = 32):
    """Requests (arrival time s, family, nrhs, rhs seed) of a Poisson stream."""
    fams = list(families or SERVING_FAMILIES)
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    fam = rng.integers(0, len(fams), size=n_requests)
    nrhs = rng.integers(1, max_rhs + 1, size=n_requests)
    return [(float(t[i]), fams[int(fam[i])], int(nrhs[i]), seed * 10007 + i)
            for i in range(n_requests)]
