"""Seeded synthetic array workloads.

Conventions shared by every consumer of these inputs:

* Work in wavelength units: lambda = 1, wavenumber k = 2*pi.
* A cell is 0.5 x 0.5 wavelengths.  The array has nx columns and ny rows of
  cells; cell (ix, iy) has linear index iy*nx + ix (rows on the upper level,
  columns on the lower level, bases inside a cell on the lowest level, as in
  the paper's Sec. II-A with N[2] = ny, N[1] = nx, N[0] = b).
* A current vector holds element (ix, iy, p) at (iy*nx + ix)*b + p.
* Generator blocks are returned as a complex128 array of shape
  (2*ny-1, 2*nx-1, b, b); gen[j + ny - 1, i + nx - 1, p, q] = T[i, j][p, q]
  is the coupling seen by basis p of a cell offset by (i, j) cells from the
  cell that holds source basis q.

Synthetic generator recipe (a stand-in for the paper's RWG impedance blocks,
whose meshes are not available): basis centroids c_p are drawn uniformly in
[0, 0.5)^2 with numpy's PCG64 ``default_rng(seed)`` as ``random((b, 2))``
(x then y for p = 0 .. b-1), the same centroids in every cell, and

    T[i, j][p, q] = exp(-1j*k*R) / (4*pi*R),
    R = max(|c_p + 0.5*(i, j) - c_q|, 0.05),

with the self term 1 + 0.5j added to the diagonal of T[0, 0] after the clamp.
The result is reciprocal: T[-i, -j] = T[i, j]^T.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CELL = 0.5          # cell pitch in wavelengths
R_MIN = 0.05        # distance clamp in wavelengths
K0 = 2.0 * np.pi    # wavenumber for lambda = 1
SELF_TERM = 1.0 + 0.5j


def centroids(b: int, seed: int) -> np.ndarray:
    """Basis centroids of one cell, shape (b, 2), uniform in [0, 0.5)^2."""
    rng = np.random.default_rng(seed)
    return rng.random((b, 2)) * CELL


def generator_blocks(nx: int, ny: int, b: int, seed: int) -> np.ndarray:
    """Synthetic Green's-function generator blocks (see module docstring)."""
    c = centroids(b, seed)
    gen = np.empty((2 * ny - 1, 2 * nx - 1, b, b), dtype=np.complex128)
    ii = np.arange(-(nx - 1), nx, dtype=np.float64)
    # dx[i, p, q] = c_p.x + 0.5 i - c_q.x
    dx = c[None, :, 0, None] + CELL * ii[:, None, None] - c[None, None, :, 0]
    for jj, j in enumerate(range(-(ny - 1), ny)):
        dy = c[:, 1, None] + CELL * j - c[None, :, 1]          # (p, q)
        r = np.sqrt(dx * dx + dy[None, :, :] ** 2)
        r = np.maximum(r, R_MIN)
        gen[jj] = np.exp(-1j * K0 * r) / (4.0 * np.pi * r)
    gen[ny - 1, nx - 1][np.diag_indices(b)] += SELF_TERM
    return gen


def generator_blocks_torch(nx: int, ny: int, b: int, seed: int, device="cuda"):
    """The synthetic generators of ``generator_blocks`` synthesised with torch
    (binary64) on ``device``: same centroids, same formula, for large batches
    where numpy synthesis would dominate.  Returns a complex128 tensor."""
    import torch
    c = torch.from_numpy(centroids(b, seed)).to(device)
    ii = torch.arange(-(nx - 1), nx, dtype=torch.float64, device=device)
    jj = torch.arange(-(ny - 1), ny, dtype=torch.float64, device=device)
    dx = c[None, None, :, 0, None] + CELL * ii[None, :, None, None] - c[None, None, None, :, 0]
    dy = c[None, None, :, 1, None] + CELL * jj[:, None, None, None] - c[None, None, None, :, 1]
    r = torch.clamp(torch.sqrt(dx * dx + dy * dy), min=R_MIN)
    gen = torch.polar(1.0 / (4.0 * np.pi * r), -K0 * r)
    idx = torch.arange(b, device=device)
    gen[ny - 1, nx - 1, idx, idx] += SELF_TERM
    return gen.contiguous()


def random_generator_blocks(nx: int, ny: int, b: int, seed: int,
                            diag_shift: complex = 0.0) -> np.ndarray:
    """Non-reciprocal complex Gaussian generators (T[-i,-j] != T[i,j]^T).

    Used to catch transposition and offset-sign mistakes that symmetric
    synthetic generators would hide.  ``diag_shift`` is added to the diagonal
    of T[0, 0] (handy to make a well-conditioned solve test).
    """
    rng = np.random.default_rng(seed)
    shape = (2 * ny - 1, 2 * nx - 1, b, b)
    gen = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    if diag_shift:
        gen[ny - 1, nx - 1][np.diag_indices(b)] += diag_shift
    return gen


def periodic_generator_blocks(nx: int, ny: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """b = 1 generators that are periodic in both offsets.

    Returns (gen, c) where c is a random complex (nx, ny) table and
    T[i, j] = c[i mod nx, j mod ny].  The resulting two-level Toeplitz
    matrix is block circulant with circulant blocks.
    """
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((nx, ny)) + 1j * rng.standard_normal((nx, ny))
    gen = np.empty((2 * ny - 1, 2 * nx - 1, 1, 1), dtype=np.complex128)
    for j in range(-(ny - 1), ny):
        for i in range(-(nx - 1), nx):
            gen[j + ny - 1, i + nx - 1, 0, 0] = c[i % nx, j % ny]
    return gen, c


def port_index(nx: int, b: int, ix: int, iy: int, basis: int = 0) -> int:
    """Vector index of basis ``basis`` of cell (ix, iy)."""
    return (iy * nx + ix) * b + basis


def port_excitations(nx: int, ny: int, b: int, cells=None) -> np.ndarray:
    """Delta-gap excitations: one column per listed cell, 1 at its basis 0.

    ``cells`` is a list of (ix, iy); default is every cell in raster order
    (the embedded-element-pattern workload).  Returns an (N, ncols)
    complex128 array in column-major use (column c is V[:, c]).
    """
    if cells is None:
        cells = [(ix, iy) for iy in range(ny) for ix in range(nx)]
    n = nx * ny * b
    v = np.zeros((n, len(cells)), dtype=np.complex128)
    for c, (ix, iy) in enumerate(cells):
        v[port_index(nx, b, ix, iy), c] = 1.0
    return v


def centre_excitation(nx: int, ny: int, b: int) -> np.ndarray:
    """Single delta-gap at basis 0 of the centre cell (nx//2, ny//2)."""
    return port_excitations(nx, ny, b, [(nx // 2, ny // 2)])[:, 0]


def random_port_excitations(nx: int, ny: int, b: int, ncols: int, seed: int) -> np.ndarray:
    """Columns with CN(0,1) amplitudes on every cell's port basis (basis 0)."""
    rng = np.random.default_rng(seed)
    n = nx * ny * b
    v = np.zeros((n, ncols), dtype=np.complex128)
    amp = (rng.standard_normal((nx * ny, ncols)) + 1j * rng.standard_normal((nx * ny, ncols))) / np.sqrt(2.0)
    v[np.arange(nx * ny) * b, :] = amp
    return v


def random_vectors(n: int, ncols: int, seed: int) -> np.ndarray:
    """Dense CN(0,1) vectors, shape (n, ncols)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))) / np.sqrt(2.0)


@dataclass
class ArraySpec:
    nx: int
    ny: int
    b: int
    seed: int
    nrhs: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.b


def uneven_batch_specs(count: int = 64, master_seed: int = 3) -> list[ArraySpec]:
    """The uneven batch: nx, ny ~ U{8..40}, b in {24, 60, 96}, nrhs ~ U{1..16}.

    Drawn from ``default_rng(master_seed)`` in the order nx[], ny[], b[],
    nrhs[]; array a uses centroid seed 1000*master_seed + a.  Its right-hand
    sides are port excitations of the first nrhs cells in raster order.
    """
    rng = np.random.default_rng(master_seed)
    nx = rng.integers(8, 41, count)
    ny = rng.integers(8, 41, count)
    b = rng.choice(np.array([24, 60, 96]), count)
    nrhs = rng.integers(1, 17, count)
    return [ArraySpec(int(nx[a]), int(ny[a]), int(b[a]), 1000 * master_seed + a, int(nrhs[a]))
            for a in range(count)]


# Named workloads: sizes and seeds of the five benchmark configurations.
CONFIGS = {
    "tiny": dict(nx=4, ny=4, b=12, seed=0, tol=1e-10, restart=50),
    "precision": dict(nx=30, ny=30, b=60, seed=1, tol=1e-8, restart=50),
    "multi_rhs": dict(nx=30, ny=30, b=60, seed=1, tol=1e-8, restart=50, nrhs=900),
    "uneven": dict(count=64, master_seed=3, tol=1e-8),
    "learned": dict(nx=40, ny=40, b=96, seed=4, test_seed=5, tol=1e-8, ntrain=2000, ntest=50),
}
