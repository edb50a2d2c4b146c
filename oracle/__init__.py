"""CPU oracle for the MLFFT-accelerated two-level block-Toeplitz solver.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The solver library
(``paper_2506_20350_gb300``) never imports, links or calls it, and this
package imports nothing from the solver: the two share only the seeded input
generators in ``workloads``.

Every function computes the plain definition of what it names, in IEEE
binary64 (numpy complex128 or the C file ``bttb_oracle.c`` next to this one),
and cites the passage of the paper it follows.  The O(N^2) products, the
dense assembly, the dense LU and the naive DFT live in C because pure Python
loops would take hours at the benchmark sizes; the C code is the same
definition written out with plain loops.

Parity status of each function (what pins it is in tests/test_oracle.py):
  assemble, matvec, matvec_rows  -- pinned: worked example (Eq. T), scipy
      Toeplitz special cases, closed-form BCCB eigenvalues, symmetry.
  wrap_first_column, spectrum    -- pinned: worked example c1 (Eq. cT1),
      convolution identity against the pinned matvec.
  lu_solve                       -- pinned: numpy.linalg.solve, residual.
  dft                            -- pinned: numpy.fft, closed forms.
  gmres                          -- pinned: exact termination in <= N steps,
      k distinct eigenvalues, residual-estimate identity.  Iteration counts
      on the synthetic matrices are reported, not pinned (the paper's
      convergence figure is missing).
  block_jacobi_apply             -- pinned: P_K (P_K^{-1} x) = x, nx=ny=1 case.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bttb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``bttb_oracle.c`` into ``liboracle.so`` (gcc, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.c_void_p
            lib.oracle_assemble.argtypes = [ctypes.c_int] * 3 + [dp, dp]
            lib.oracle_matvec.argtypes = [ctypes.c_int] * 3 + [dp, dp, ctypes.c_long, dp, ctypes.c_long, ctypes.c_int]
            lib.oracle_matvec_rows.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp, ctypes.c_int, dp]
            lib.oracle_lu_solve.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_lu_solve.restype = ctypes.c_int
            lib.oracle_dft.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _dims(gen: np.ndarray):
    if gen.ndim != 4 or gen.shape[2] != gen.shape[3]:
        raise ValueError("gen must have shape (2ny-1, 2nx-1, b, b)")
    ny = (gen.shape[0] + 1) // 2
    nx = (gen.shape[1] + 1) // 2
    return nx, ny, gen.shape[2]


# --------------------------------------------------------------------------
# The matrix and its product (Sec. II-A, Eq. (Tblock), L = 2)
# --------------------------------------------------------------------------

def assemble(gen: np.ndarray) -> np.ndarray:
    """Dense Z with Z[(m*b+p), (n*b+q)] = T[ix_m-ix_n, iy_m-iy_n][p, q] (Eq. Tblock)."""
    nx, ny, b = _dims(gen)
    g = np.ascontiguousarray(gen, dtype=np.complex128)
    n = nx * ny * b
    z = np.empty((n, n), dtype=np.complex128)
    _load().oracle_assemble(nx, ny, b, _ptr(g), _ptr(z))
    return z


def matvec(gen: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = Z x by the O(N^2) definition, streamed from the generator table.

    ``x`` is (N,) or (N, k); returns the same shape.
    """
    nx, ny, b = _dims(gen)
    g = np.ascontiguousarray(gen, dtype=np.complex128)
    n = nx * ny * b
    squeeze = x.ndim == 1
    xs = np.asarray(x, dtype=np.complex128).reshape(n, -1)
    xc = np.ascontiguousarray(xs.T)       # column c contiguous
    k = xc.shape[0]
    yc = np.empty_like(xc)
    _load().oracle_matvec(nx, ny, b, _ptr(g), _ptr(xc), n, _ptr(yc), n, k)
    y = yc.T
    return y[:, 0].copy() if squeeze else np.ascontiguousarray(y)


def matvec_rows(gen: np.ndarray, x: np.ndarray, rows) -> np.ndarray:
    """Entries ``rows`` of Z x (one vector), by the same O(N) per-row sum."""
    nx, ny, b = _dims(gen)
    g = np.ascontiguousarray(gen, dtype=np.complex128)
    xv = np.ascontiguousarray(x, dtype=np.complex128).reshape(-1)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(r.shape[0], dtype=np.complex128)
    _load().oracle_matvec_rows(nx, ny, b, _ptr(g), _ptr(xv), _ptr(r), r.shape[0], _ptr(out))
    return out


def relres(gen: np.ndarray, v: np.ndarray, i: np.ndarray) -> np.ndarray:
    """Per-column ||V - Z I||_2 / ||V||_2 with the oracle product."""
    v2 = np.asarray(v).reshape(v.shape[0], -1)
    i2 = np.asarray(i).reshape(i.shape[0], -1)
    r = v2 - matvec(gen, i2)
    return np.linalg.norm(r, axis=0) / np.linalg.norm(v2, axis=0)


# --------------------------------------------------------------------------
# Circulant embedding and its spectrum (Sec. II-B/C)
# --------------------------------------------------------------------------

def wrap_first_column(gen: np.ndarray, mx: int, my: int) -> np.ndarray:
    """First block column C_1^[2] of the two-level circulant embedding.

    Eq. (cT1), (circL1) and (circL2): offsets 0..N-1 keep their position and
    offsets -N+1..-1 are appended after them, i.e. offset n sits at slot
    n mod M on each level; the padded slots N..M-N hold zero blocks.
    Returns an array of shape (my, mx, b, b), slot (sy, sx).
    """
    nx, ny, b = _dims(gen)
    if mx < 2 * nx - 1 or my < 2 * ny - 1:
        raise ValueError("embedding needs M >= 2N-1 on each level")
    c1 = np.zeros((my, mx, b, b), dtype=np.complex128)
    for j in range(-(ny - 1), ny):
        for i in range(-(nx - 1), nx):
            c1[j % my, i % mx] = gen[j + ny - 1, i + nx - 1]
    return c1


def spectrum(gen: np.ndarray, mx: int, my: int) -> np.ndarray:
    """Block spectrum F^[2] C_1^[2] (Eq. multL, F^[2] of Eq. F2), shape (my, mx, b, b).

    Bin (ky, kx) holds the b x b block  sum_{sy,sx} C1[sy,sx] e^{-2 pi i (ky sy/my + kx sx/mx)}.
    numpy's FFT is the library step for the two DFT levels.
    """
    return np.fft.fft2(wrap_first_column(gen, mx, my), axes=(0, 1))


# --------------------------------------------------------------------------
# Direct solve and DFT
# --------------------------------------------------------------------------

def lu_solve(a: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Dense complex LU with partial pivoting; solves a X = rhs."""
    n = a.shape[0]
    aa = np.ascontiguousarray(a, dtype=np.complex128).copy()
    squeeze = rhs.ndim == 1
    r = np.ascontiguousarray(np.asarray(rhs, dtype=np.complex128).reshape(n, -1)).copy()
    info = _load().oracle_lu_solve(n, _ptr(aa), _ptr(r), r.shape[1])
    if info != 0:
        raise np.linalg.LinAlgError(f"zero pivot at step {info - 1}")
    return r[:, 0] if squeeze else r


def dft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Naive DFT X[k] = sum_t x[t] exp(sign 2 pi i k t / n) in long double."""
    xv = np.ascontiguousarray(x, dtype=np.complex128).reshape(-1)
    out = np.empty_like(xv)
    _load().oracle_dft(xv.shape[0], _ptr(xv), _ptr(out), int(sign))
    return out


# --------------------------------------------------------------------------
# Preconditioner and Krylov solver (Sec. III-B and III-C)
# --------------------------------------------------------------------------

def block_jacobi_apply(gen: np.ndarray, x: np.ndarray) -> np.ndarray:
    """P_K^{-1} x for the block-Jacobi preconditioner of Sec. III-B.

    P_K is block diagonal with the self block R_0 = T[0,0] of every cell;
    one factorisation of R_0 serves every cell (numpy's solve is the library
    step).  ``x`` is (N,) or (N, k).
    """
    nx, ny, b = _dims(gen)
    t00 = gen[ny - 1, nx - 1]
    squeeze = x.ndim == 1
    xs = np.asarray(x, dtype=np.complex128).reshape(nx * ny, b, -1)
    z = np.stack([np.linalg.solve(t00, xs[c]) for c in range(nx * ny)])
    z = z.reshape(nx * ny * b, -1)
    return z[:, 0] if squeeze else z


def gmres(apply_a, b: np.ndarray, tol: float, restart: int, max_iters: int,
          x0: np.ndarray | None = None, precond=None, side: str = "left",
          true_residual=None):
    """Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations.

    Follows the textbook algorithm (Saad, Iterative Methods for Sparse
    Linear Systems, Alg. 6.9 / 9.4-9.5) that the paper hands its matvec and
    preconditioner to (Sec. III-C).  x0 = 0 unless given.  Convergence is
    judged on the true relative residual ||b - A x|| / ||b|| computed with
    ``true_residual`` (default: ``apply_a``) at the end of each cycle; a
    cycle ends after ``restart`` steps or when the rotation estimate of the
    (preconditioned) residual reaches the target.  ``precond`` applies
    P^{-1}; ``side`` is "left" (P^{-1} A x = P^{-1} b, the paper's choice)
    or "right" (A P^{-1} u = b, x = P^{-1} u).

    Returns (x, info) with info = dict(iters, relres, converged, history).
    """
    n = b.shape[0]
    true_residual = true_residual or apply_a
    m_inv = precond if precond is not None else (lambda v: v)
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), dict(iters=0, relres=0.0, converged=True, history=[])
    history = []
    iters = 0
    while True:
        r = b - true_residual(x)
        rel = np.linalg.norm(r) / bnorm
        history.append(rel)
        if rel <= tol:
            return x, dict(iters=iters, relres=rel, converged=True, history=history)
        if iters >= max_iters:
            return x, dict(iters=iters, relres=rel, converged=False, history=history)
        z = m_inv(r) if side == "left" else r
        beta = np.linalg.norm(z)
        target = tol * (np.linalg.norm(m_inv(b)) if side == "left" else bnorm)
        basis = [z / beta]
        h = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.float64)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(restart):
            if side == "left":
                w = m_inv(apply_a(basis[j]))
            else:
                w = apply_a(m_inv(basis[j]))
            for i in range(j + 1):                      # modified Gram-Schmidt
                h[i, j] = np.vdot(basis[i], w)
                w = w - h[i, j] * basis[i]
            h[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                          # earlier rotations
                a0, a1 = h[i, j], h[i + 1, j]
                h[i, j] = cs[i] * a0 + sn[i] * a1
                h[i + 1, j] = -np.conj(sn[i]) * a0 + cs[i] * a1
            a0, a1 = h[j, j], h[j + 1, j]
            rho = np.sqrt(abs(a0) ** 2 + abs(a1) ** 2)
            if abs(a0) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a0) / rho
                sn[j] = (a0 / abs(a0)) * np.conj(a1) / rho
            h[j, j] = cs[j] * a0 + sn[j] * a1
            h[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            hnext = abs(a1)
            if abs(g[j + 1]) <= target or hnext == 0.0 or iters >= max_iters:
                break
            basis.append(w / hnext)
        y = np.zeros(k, dtype=np.complex128)              # back substitution
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(h[i, i + 1:k], y[i + 1:k])) / h[i, i]
        d = sum(y[i] * basis[i] for i in range(k))
        x = x + (d if side == "left" else m_inv(d))
