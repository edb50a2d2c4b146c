"""Pins for the CPU oracle: each test ties an oracle function to something
other than itself -- a value the paper prints, a library routine that a
special case reduces to, a closed form, or an invariant of the mathematics.
"""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from workloads import arrays

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sections(name):
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                out[cur] = []
            else:
                out[cur].append(line.split())
    return out


def _scalar_gen(t):
    """gen for nx = len(t)//2 + 1, ny = 1, b = 1 from a dict offset -> value."""
    nx = (len(t) + 1) // 2
    gen = np.zeros((1, 2 * nx - 1, 1, 1), dtype=np.complex128)
    for k, v in t.items():
        gen[0, k + nx - 1, 0, 0] = v
    return gen


def _rng_complex(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------
# Worked example of Sec. II-B (golden values printed in the paper)
# ----------------------------------------------------------------------------

def test_worked_example_assembly_matches_eq_T():
    g = _sections("worked_example_scalar.txt")
    rng = np.random.default_rng(10)
    t = {k: complex(*rng.standard_normal(2)) for k in range(-2, 3)}
    z = oracle.assemble(_scalar_gen(t))
    expect = np.array([[t[int(k)] for k in row] for row in g["T"]])
    np.testing.assert_array_equal(z, expect)


def test_worked_example_first_column_matches_eq_cT1():
    g = _sections("worked_example_scalar.txt")
    rng = np.random.default_rng(11)
    t = {k: complex(*rng.standard_normal(2)) for k in range(-2, 3)}
    c1 = oracle.wrap_first_column(_scalar_gen(t), mx=5, my=1)[0, :, 0, 0]
    expect = np.array([t[int(k)] for k in g["c1"][0]])
    np.testing.assert_array_equal(c1, expect)
    # Eq. (scalarC): the circulant with that first column is the printed C(T)
    cmat = scipy.linalg.circulant(c1)
    expect_c = np.array([[t[int(k)] for k in row] for row in g["C"]])
    np.testing.assert_array_equal(cmat, expect_c)
    # Eq. (circmult): C(T)[u; 0] = [T u; gamma]
    u = _rng_complex(rng, 3)
    z = oracle.assemble(_scalar_gen(t))
    np.testing.assert_allclose((cmat @ np.concatenate([u, np.zeros(2)]))[:3], z @ u, rtol=1e-14)


def test_two_level_structure_matches_paper():
    g = _sections("two_level_structure.txt")
    rng = np.random.default_rng(12)
    gen = _rng_complex(rng, 3, 3, 1, 1)   # nx = ny = 2, b = 1

    def t(s):
        i, j = (int(v) for v in s.split(","))
        return gen[j + 1, i + 1, 0, 0]

    z = oracle.assemble(gen)
    np.testing.assert_array_equal(z, np.array([[t(s) for s in row] for row in g["Z"]]))
    c1 = oracle.wrap_first_column(gen, mx=3, my=3)[:, :, 0, 0].reshape(-1)
    np.testing.assert_array_equal(c1, np.array([t(s) for s in g["C1"][0]]))


# ----------------------------------------------------------------------------
# Special cases that reduce to library routines
# ----------------------------------------------------------------------------

def test_one_level_scalar_is_scipy_toeplitz():
    rng = np.random.default_rng(13)
    nx = 7
    t = {k: complex(*rng.standard_normal(2)) for k in range(-(nx - 1), nx)}
    col = [t[k] for k in range(nx)]
    row = [t[-k] for k in range(nx)]
    np.testing.assert_array_equal(oracle.assemble(_scalar_gen(t)), scipy.linalg.toeplitz(col, row))


def test_two_level_scalar_is_block_toeplitz_of_toeplitz():
    rng = np.random.default_rng(14)
    nx, ny = 3, 4
    gen = _rng_complex(rng, 2 * ny - 1, 2 * nx - 1, 1, 1)

    def lower(j):   # T_j^[1] as a scipy Toeplitz matrix over the x offsets
        col = [gen[j + ny - 1, i + nx - 1, 0, 0] for i in range(nx)]
        row = [gen[j + ny - 1, -i + nx - 1, 0, 0] for i in range(nx)]
        return scipy.linalg.toeplitz(col, row)

    expect = np.block([[lower(m - n) for n in range(ny)] for m in range(ny)])
    np.testing.assert_array_equal(oracle.assemble(gen), expect)


def test_single_cell_is_dense_gemv():
    rng = np.random.default_rng(15)
    gen = _rng_complex(rng, 1, 1, 9, 9)
    x = _rng_complex(rng, 9, 3)
    np.testing.assert_allclose(oracle.matvec(gen, x), gen[0, 0] @ x, rtol=1e-13, atol=1e-13)


def test_block_one_level_matches_scipy_block_toeplitz():
    """ny = 1: a 1-level block Toeplitz matrix (Eq. Tblock, L = 1)."""
    rng = np.random.default_rng(16)
    nx, b = 5, 3
    gen = _rng_complex(rng, 1, 2 * nx - 1, b, b)
    expect = np.block([[gen[0, m - n + nx - 1] for n in range(nx)] for m in range(nx)])
    np.testing.assert_array_equal(oracle.assemble(gen), expect)


# ----------------------------------------------------------------------------
# Closed form: b = 1 doubly circulant case (Sec. II-B, diagonalisation by DFT)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny", [(5, 4), (3, 3), (1, 6), (8, 2)])
def test_bccb_eigenpairs(nx, ny):
    gen, c = arrays.periodic_generator_blocks(nx, ny, seed=17)
    lam = np.fft.fft2(c)                                  # library closed form
    ix = np.tile(np.arange(nx), ny)
    iy = np.repeat(np.arange(ny), nx)
    modes = np.stack([np.exp(2j * np.pi * (kx * ix / nx + ky * iy / ny))
                      for ky in range(ny) for kx in range(nx)], axis=1)
    lam_col = np.array([lam[kx, ky] for ky in range(ny) for kx in range(nx)])
    y = oracle.matvec(gen, modes)
    np.testing.assert_allclose(y, modes * lam_col[None, :], rtol=0, atol=1e-12 * np.abs(lam).max())


# ----------------------------------------------------------------------------
# Invariants
# ----------------------------------------------------------------------------

def test_matvec_agrees_with_dense_and_rows():
    rng = np.random.default_rng(18)
    gen = arrays.random_generator_blocks(3, 2, 4, seed=19)
    z = oracle.assemble(gen)
    x = _rng_complex(rng, z.shape[0], 3)
    y = oracle.matvec(gen, x)
    np.testing.assert_allclose(y, z @ x, rtol=1e-13, atol=1e-13)
    rows = np.array([0, 5, 17, z.shape[0] - 1])
    np.testing.assert_allclose(oracle.matvec_rows(gen, x[:, 1], rows), (z @ x[:, 1])[rows], rtol=1e-13)


def test_reciprocal_generators_give_symmetric_z():
    gen = arrays.generator_blocks(3, 4, 5, seed=20)
    z = oracle.assemble(gen)
    np.testing.assert_allclose(z, z.T, rtol=1e-13, atol=1e-15)
    rng = np.random.default_rng(21)
    x, y = _rng_complex(rng, z.shape[0]), _rng_complex(rng, z.shape[0])
    assert abs(x @ oracle.matvec(gen, y) - y @ oracle.matvec(gen, x)) < 1e-12 * np.linalg.norm(z)


def test_linearity():
    rng = np.random.default_rng(22)
    gen = arrays.random_generator_blocks(4, 3, 3, seed=23)
    n = 4 * 3 * 3
    x, y = _rng_complex(rng, n), _rng_complex(rng, n)
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    np.testing.assert_allclose(oracle.matvec(gen, a * x + b * y),
                               a * oracle.matvec(gen, x) + b * oracle.matvec(gen, y), rtol=1e-12, atol=1e-12)


def test_shift_invariance():
    """Moving a source by one cell moves the field by one cell (interior)."""
    rng = np.random.default_rng(24)
    nx, ny, b = 5, 4, 3
    gen = arrays.random_generator_blocks(nx, ny, b, seed=25)
    x = np.zeros(nx * ny * b, dtype=np.complex128)
    xs = np.zeros_like(x)
    src = _rng_complex(rng, b)
    x[(1 * nx + 1) * b:(1 * nx + 2) * b] = src          # cell (1, 1)
    xs[(2 * nx + 2) * b:(2 * nx + 3) * b] = src         # cell (2, 2)
    y = oracle.matvec(gen, x).reshape(ny, nx, b)
    ys = oracle.matvec(gen, xs).reshape(ny, nx, b)
    np.testing.assert_allclose(ys[1:, 1:], y[:-1, :-1], rtol=1e-14, atol=0)


def test_generator_reciprocity_and_self_term():
    nx, ny, b = 3, 2, 6
    gen = arrays.generator_blocks(nx, ny, b, seed=26)
    for j in range(-(ny - 1), ny):
        for i in range(-(nx - 1), nx):
            np.testing.assert_allclose(gen[-j + ny - 1, -i + nx - 1], gen[j + ny - 1, i + nx - 1].T, rtol=1e-13)
    t00 = gen[ny - 1, nx - 1]
    # diagonal: R clamped at 0.05 -> exp(-j 2 pi 0.05)/(4 pi 0.05) + 1 + 0.5j
    d = np.exp(-1j * 2 * np.pi * 0.05) / (4 * np.pi * 0.05) + 1 + 0.5j
    np.testing.assert_allclose(np.diag(t00), d, rtol=1e-15)


# ----------------------------------------------------------------------------
# Circulant embedding spectrum: convolution identity against the pinned product
# ----------------------------------------------------------------------------

def _mlfft_numpy(gen, x, mx, my):
    """Pad (Eq. xc2), 2-D DFT, per-bin block product (Eq. multL), inverse, crop."""
    nx, ny, b = (gen.shape[1] + 1) // 2, (gen.shape[0] + 1) // 2, gen.shape[2]
    u = np.zeros((my, mx, b), dtype=np.complex128)
    u[:ny, :nx] = x.reshape(ny, nx, b)
    uh = np.fft.fft2(u, axes=(0, 1))
    gh = oracle.spectrum(gen, mx, my)
    vh = np.einsum("yxpq,yxq->yxp", gh, uh)
    v = np.fft.ifft2(vh, axes=(0, 1))
    return v[:ny, :nx].reshape(-1)


@pytest.mark.parametrize("extra", [0, 1, 4])
def test_spectrum_convolution_identity(extra):
    nx, ny, b = 4, 3, 5
    gen = arrays.random_generator_blocks(nx, ny, b, seed=27)
    rng = np.random.default_rng(28)
    x = _rng_complex(rng, nx * ny * b)
    y = _mlfft_numpy(gen, x, 2 * nx - 1 + extra, 2 * ny - 1 + extra)
    np.testing.assert_allclose(y, oracle.matvec(gen, x), rtol=1e-12, atol=1e-12)


def test_spectrum_too_small_grid_is_rejected():
    gen = arrays.random_generator_blocks(4, 3, 2, seed=29)
    with pytest.raises(ValueError):
        oracle.wrap_first_column(gen, mx=6, my=5)


# ----------------------------------------------------------------------------
# DFT and LU
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 15, 59, 60, 79, 80])
def test_dft_matches_numpy(n):
    rng = np.random.default_rng(30 + n)
    x = _rng_complex(rng, n)
    np.testing.assert_allclose(oracle.dft(x, -1), np.fft.fft(x), rtol=1e-13, atol=1e-13 * np.sqrt(n))
    np.testing.assert_allclose(oracle.dft(x, +1), np.fft.ifft(x) * n, rtol=1e-13, atol=1e-13 * np.sqrt(n))


def test_dft_closed_forms():
    n = 12
    x = np.zeros(n, dtype=np.complex128)
    x[0] = 1.0
    np.testing.assert_allclose(oracle.dft(x), np.ones(n), atol=1e-18)
    x = np.exp(2j * np.pi * 3 * np.arange(n) / n)
    e = np.zeros(n)
    e[3] = n
    np.testing.assert_allclose(oracle.dft(x), e, atol=1e-13)


def test_lu_solve_matches_numpy():
    rng = np.random.default_rng(40)
    a = _rng_complex(rng, 30, 30)
    b = _rng_complex(rng, 30, 4)
    x = oracle.lu_solve(a, b)
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(a @ x, b, atol=1e-12)


def test_lu_solve_needs_pivoting():
    a = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    np.testing.assert_allclose(oracle.lu_solve(a, np.array([2.0, 3.0])), [3.0, 2.0])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lu_solve(np.zeros((2, 2)), np.ones(2))


# ----------------------------------------------------------------------------
# GMRES (textbook properties) and the block-Jacobi preconditioner
# ----------------------------------------------------------------------------

def test_gmres_terminates_within_n_steps():
    rng = np.random.default_rng(41)
    n = 14
    a = _rng_complex(rng, n, n) + 4 * np.eye(n)
    b = _rng_complex(rng, n)
    x, info = oracle.gmres(lambda v: a @ v, b, tol=1e-12, restart=n, max_iters=n)
    assert info["converged"] and info["iters"] <= n
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-9, atol=1e-10)


def test_gmres_distinct_eigenvalues():
    rng = np.random.default_rng(42)
    n = 20
    s = _rng_complex(rng, n, n) + 5 * np.eye(n)
    lam = np.array([1.0 + 1j, -2.0, 3.0 - 0.5j])[np.arange(n) % 3]
    a = s @ np.diag(lam) @ np.linalg.inv(s)
    b = _rng_complex(rng, n)
    x, info = oracle.gmres(lambda v: a @ v, b, tol=1e-9, restart=10, max_iters=10)
    assert info["converged"] and info["iters"] <= 3


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_gmres_minimises_over_krylov_space(k):
    rng = np.random.default_rng(43)
    n = 16
    a = _rng_complex(rng, n, n) + 3 * np.eye(n)
    b = _rng_complex(rng, n)
    kry = np.stack([np.linalg.matrix_power(a, i) @ b for i in range(k)], axis=1)
    q, _ = np.linalg.qr(kry)
    y, *_ = np.linalg.lstsq(a @ q, b, rcond=None)
    best = np.linalg.norm(b - a @ (q @ y)) / np.linalg.norm(b)
    _, info = oracle.gmres(lambda v: a @ v, b, tol=1e-30, restart=k, max_iters=k)
    assert abs(info["relres"] - best) <= 1e-10 * max(best, 1e-3)


@pytest.mark.parametrize("side", ["left", "right"])
def test_gmres_exact_preconditioner_one_step(side):
    rng = np.random.default_rng(44)
    n = 10
    a = _rng_complex(rng, n, n) + 3 * np.eye(n)
    ainv = np.linalg.inv(a)
    b = _rng_complex(rng, n)
    x, info = oracle.gmres(lambda v: a @ v, b, tol=1e-10, restart=5, max_iters=5,
                           precond=lambda v: ainv @ v, side=side)
    assert info["converged"] and info["iters"] == 1


def test_block_jacobi_inverse():
    nx, ny, b = 3, 2, 4
    gen = arrays.random_generator_blocks(nx, ny, b, seed=45, diag_shift=3.0)
    rng = np.random.default_rng(46)
    x = _rng_complex(rng, nx * ny * b, 2)
    z = oracle.block_jacobi_apply(gen, x)
    t00 = gen[ny - 1, nx - 1]
    back = np.concatenate([t00 @ z[c * b:(c + 1) * b] for c in range(nx * ny)])
    np.testing.assert_allclose(back, x, rtol=1e-12, atol=1e-12)
    g1 = arrays.random_generator_blocks(1, 1, 6, seed=47, diag_shift=2.0)
    v = _rng_complex(rng, 6)
    np.testing.assert_allclose(oracle.block_jacobi_apply(g1, v), np.linalg.solve(oracle.assemble(g1), v), rtol=1e-12)


def test_tiny_config_gmres_matches_lu():
    cfg = arrays.CONFIGS["tiny"]
    nx, ny, b = cfg["nx"], cfg["ny"], cfg["b"]
    gen = arrays.generator_blocks(nx, ny, b, cfg["seed"])
    v = arrays.port_excitations(nx, ny, b, [(1, 1)])[:, 0]
    z = oracle.assemble(gen)
    x_lu = oracle.lu_solve(z, v)
    x, info = oracle.gmres(lambda u: oracle.matvec(gen, u), v, tol=cfg["tol"],
                           restart=cfg["restart"], max_iters=2000)
    assert info["converged"]
    assert oracle.relres(gen, v, x)[0] <= cfg["tol"]
    assert np.linalg.norm(x - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
