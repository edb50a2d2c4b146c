"""GB300 solver for two-level block-Toeplitz MoM systems Z I = V.

Python binding of ``libbttb`` (C ABI in ``include/bttb.h``).  The functions
below carry the C names and only marshal arguments: every step of the
product and of the solver runs in the library's CUDA kernels.  PyTorch is used
for device memory and streams.  There is no fallback: if ``libbttb.so`` is
missing, every entry point raises ImportError.

Vector convention: a multi-vector with k columns is a C-contiguous tensor of
shape (k, N) (column c of the paper's V is row c here), element (ix, iy, p) of
a column at (iy*nx + ix)*b + p.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# BTTB_LIB_CHECKED=1 in the environment loads the bounds-checked build instead (tests of the checks).
LIB_PATH = os.path.join(HERE, "libbttb_checked.so" if os.environ.get("BTTB_LIB_CHECKED") == "1" else "libbttb.so")

BTTB_C64, BTTB_C128 = 0, 1
BTTB_MV_FP64, BTTB_MV_FP32, BTTB_MV_FP64_NATIVE, BTTB_MV_TC_3XTF32, BTTB_MV_TC_BF16X3 = 0, 1, 2, 3, 4
BTTB_PC_NONE, BTTB_PC_BLOCK_JACOBI, BTTB_PC_LEARNED = 0, 1, 2
BTTB_GMRES_NO_GRAPH, BTTB_GMRES_GLOBAL, BTTB_GMRES_CGS2 = 1, 2, 4
BTTB_OK, BTTB_NOT_CONVERGED, BTTB_BREAKDOWN = 0, 1, 2
BTTB_ERR_INVALID_ARG, BTTB_ERR_CUDA, BTTB_ERR_OOM = -1, -2, -3
BTTB_ERR_NO_GENERATORS, BTTB_ERR_TIMEOUT, BTTB_ERR_NONFINITE, BTTB_ERR_SINGULAR = -4, -5, -6, -7

BTTB_K_BLOCK_PRODUCT, BTTB_K_FFT, BTTB_K_ALL, BTTB_K_BLOCK_PRODUCT_PREC = 0, 1, 2, 16
BTTB_DEBUG_WAIT_LIMIT_NS, BTTB_DEBUG_WITHHOLD_ARRIVAL, BTTB_DEBUG_PRODUCT_ROUTE, BTTB_DEBUG_ROUTE_TAKEN = 1, 2, 3, 4
BTTB_DEBUG_FUSED_SHAPE, BTTB_DEBUG_FUSED_CLUSTER = 5, 6

EXPORTS = ("bttb_plan_create", "bttb_plan_grid", "bttb_set_generators", "bttb_matvec",
           "bttb_gmres_solve", "bttb_block_jacobi_apply", "bttb_get_spectrum_bin",
           "bttb_profile", "bttb_profile_read", "bttb_matvec_noalloc",
           "bttb_batch_create", "bttb_batch_plan", "bttb_batch_set_generators", "bttb_batch_autotune",
           "bttb_batch_gmres_solve", "bttb_batch_destroy",
           "bttb_learned_create", "bttb_learned_param_count", "bttb_learned_params", "bttb_learned_apply",
           "bttb_learned_gradients", "bttb_learned_train_step", "bttb_plan_set_learned", "bttb_learned_destroy",
           "bttb_plan_autotune", "bttb_plan_debug", "bttb_plan_workspace_bytes", "bttb_plan_destroy",
           "bttb_last_error", "bttb_check_report", "bttb_check_probe")


class BttbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bttb error {code}: {msg}")
        self.code = code


class GmresOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("pc", ctypes.c_int), ("inner", ctypes.c_int), ("use_x0", ctypes.c_int),
                ("host_io", ctypes.c_int), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_len", ctypes.c_int), ("flags", ctypes.c_int)]


class KernelStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_long), ("bytes", ctypes.c_double)]


class ColResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("cycles", ctypes.c_int),
                ("relres_true", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbttb.so (built by ``paper_2506_20350_gb300.build``) and declare its C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2506_20350_gb300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, ci, cl = ctypes.c_void_p, ctypes.c_int, ctypes.c_long
    lib.bttb_plan_create.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ctypes.c_uint, vp]
    lib.bttb_plan_grid.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.bttb_set_generators.argtypes = [vp, vp, ci, ci]
    lib.bttb_matvec.argtypes = [vp, vp, vp, ci, cl, ci, ci]
    lib.bttb_gmres_solve.argtypes = [vp, vp, vp, ci, cl, ctypes.POINTER(GmresOpts), ctypes.POINTER(ColResult)]
    lib.bttb_block_jacobi_apply.argtypes = [vp, vp, vp, ci, cl, ci]
    lib.bttb_get_spectrum_bin.argtypes = [vp, ci, ci, ctypes.POINTER(ctypes.c_double)]
    lib.bttb_profile.argtypes = [vp, ci]
    lib.bttb_profile_read.argtypes = [vp, ci, ctypes.POINTER(KernelStats)]
    lib.bttb_matvec_noalloc.argtypes = [ci, ci, ci, vp, vp, vp, ci, cl, vp]
    pi = ctypes.POINTER(ci)
    lib.bttb_batch_create.argtypes = [ctypes.POINTER(vp), ci, pi, pi, pi, pi, ctypes.c_uint]
    lib.bttb_batch_plan.argtypes = [vp, ci, ctypes.POINTER(vp)]
    lib.bttb_batch_set_generators.argtypes = [vp, ci, vp, ci, ci]
    lib.bttb_batch_autotune.argtypes = [vp, ci, pi]
    lib.bttb_batch_gmres_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(cl),
                                           ctypes.POINTER(GmresOpts), ctypes.POINTER(ColResult)]
    lib.bttb_batch_destroy.argtypes = [vp]
    lib.bttb_learned_create.argtypes = [ctypes.POINTER(vp), vp, ci, ci, ci, ctypes.c_ulonglong]
    lib.bttb_learned_param_count.argtypes = [vp]
    lib.bttb_learned_params.argtypes = [vp, vp, ci]
    lib.bttb_learned_apply.argtypes = [vp, vp, vp, ci, cl, ci]
    lib.bttb_learned_gradients.argtypes = [vp, vp, vp, ci, cl, vp, ctypes.POINTER(ctypes.c_double)]
    lib.bttb_learned_train_step.argtypes = [vp, vp, vp, ci, cl, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.bttb_plan_set_learned.argtypes = [vp, vp]
    lib.bttb_learned_destroy.argtypes = [vp]
    lib.bttb_plan_autotune.argtypes = [vp, ci, ci, pi]
    lib.bttb_plan_debug.argtypes = [vp, ci, ctypes.c_longlong]
    lib.bttb_check_report.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]
    lib.bttb_check_probe.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
    lib.bttb_plan_workspace_bytes.argtypes = [vp]
    lib.bttb_plan_workspace_bytes.restype = ctypes.c_size_t
    lib.bttb_plan_destroy.argtypes = [vp]
    lib.bttb_last_error.argtypes = [vp]
    lib.bttb_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("bttb_plan_workspace_bytes", "bttb_last_error", "bttb_learned_param_count"):
            getattr(lib, name).restype = ci
    lib.bttb_learned_param_count.restype = cl
    _lib = lib
    return lib


def _check(rc: int, plan=None, soft_ok: bool = False) -> int:
    if rc < 0 or (rc > 0 and not soft_ok):
        msg = load_library().bttb_last_error(plan).decode()
        raise BttbError(rc, msg)
    return rc


def _ptr(t) -> int:
    """Address of a torch tensor or numpy array."""
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------- C names

def bttb_plan_create(nx: int, ny: int, b: int, max_rhs: int = 1, prec_mask: int = 0, stream=None):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.bttb_plan_create(ctypes.byref(h), nx, ny, b, max_rhs, prec_mask, _stream_handle(stream)))
    return h


def bttb_plan_grid(plan) -> tuple[int, int]:
    mx, my = ctypes.c_int(), ctypes.c_int()
    _check(load_library().bttb_plan_grid(plan, ctypes.byref(mx), ctypes.byref(my)), plan)
    return mx.value, my.value


def bttb_set_generators(plan, gen) -> None:
    """gen: complex128/complex64 array or tensor of shape (2ny-1, 2nx-1, b, b), host or device."""
    is_host = not (hasattr(gen, "is_cuda") and gen.is_cuda)
    if hasattr(gen, "is_contiguous"):
        assert gen.is_contiguous()
        dt = BTTB_C128 if str(gen.dtype) == "torch.complex128" else BTTB_C64
    else:
        import numpy as np
        assert gen.flags["C_CONTIGUOUS"]
        dt = BTTB_C128 if gen.dtype == np.complex128 else BTTB_C64
    _check(load_library().bttb_set_generators(plan, _ptr(gen), dt, int(is_host)), plan)


def bttb_matvec(plan, x, y, nrhs: int, ld: int, dtype: int, prec: int) -> None:
    _check(load_library().bttb_matvec(plan, _ptr(x), _ptr(y), nrhs, ld, dtype, prec), plan)


def bttb_block_jacobi_apply(plan, x, z, nrhs: int, ld: int, dtype: int) -> None:
    _check(load_library().bttb_block_jacobi_apply(plan, _ptr(x), _ptr(z), nrhs, ld, dtype), plan)


def bttb_gmres_solve(plan, V, I, nrhs: int, ld: int, opts: GmresOpts) -> tuple[int, list[ColResult]]:
    res = (ColResult * nrhs)()
    rc = load_library().bttb_gmres_solve(plan, _ptr(V), _ptr(I), nrhs, ld, ctypes.byref(opts), res)
    _check(rc, plan, soft_ok=True)
    return rc, list(res)


def bttb_get_spectrum_bin(plan, ky: int, kx: int, b: int):
    import numpy as np
    out = np.empty((b, b), dtype=np.complex128)
    _check(load_library().bttb_get_spectrum_bin(plan, ky, kx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           plan)
    return out


def bttb_profile(plan, enable) -> None:
    """enable: False/0 off, True/1 on, 2 also times every kernel inside captured GMRES cycles."""
    _check(load_library().bttb_profile(plan, int(enable)), plan)


def bttb_profile_read(plan, which: int) -> KernelStats:
    st = KernelStats()
    _check(load_library().bttb_profile_read(plan, which, ctypes.byref(st)), plan)
    return st


def bttb_matvec_noalloc(nx: int, ny: int, b: int, gen, x, y, nrhs: int, ld: int, stream=None) -> None:
    """Allocation-free FP64 product for small arrays (see include/bttb.h); all tensors on the device."""
    _check(load_library().bttb_matvec_noalloc(nx, ny, b, _ptr(gen), _ptr(x), _ptr(y), nrhs, ld,
                                              _stream_handle(stream)))


def _ints(vals):
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


def bttb_batch_create(nx, ny, b, nrhs, prec_mask: int = 0):
    h = ctypes.c_void_p()
    _check(load_library().bttb_batch_create(ctypes.byref(h), len(nx), _ints(nx), _ints(ny), _ints(b), _ints(nrhs),
                                            prec_mask))
    return h


def bttb_batch_plan(batch, index: int):
    h = ctypes.c_void_p()
    _check(load_library().bttb_batch_plan(batch, index, ctypes.byref(h)))
    return h


def bttb_batch_set_generators(batch, index: int, gen) -> None:
    bttb_set_generators(bttb_batch_plan(batch, index), gen)


def bttb_batch_autotune(batch, count: int, reps: int = 5) -> list[int]:
    out = (ctypes.c_int * count)()
    _check(load_library().bttb_batch_autotune(batch, reps, out))
    return list(out)


def bttb_batch_gmres_solve(batch, Vs, Is, lds, opts: GmresOpts) -> tuple[int, list[ColResult]]:
    n = len(Vs)
    total = sum(v.shape[0] for v in Vs)
    res = (ColResult * total)()
    vp = (ctypes.c_void_p * n)(*[_ptr(v) for v in Vs])
    ip = (ctypes.c_void_p * n)(*[_ptr(i) for i in Is])
    ld = (ctypes.c_long * n)(*lds)
    rc = load_library().bttb_batch_gmres_solve(batch, vp, ip, ld, ctypes.byref(opts), res)
    _check(rc, None, soft_ok=True)
    return rc, list(res)


def bttb_batch_destroy(batch) -> None:
    if batch:
        _check(load_library().bttb_batch_destroy(batch))


def bttb_learned_create(plan, rank: int = 16, channels: int = 64, max_cols: int = 64, seed: int = 0):
    h = ctypes.c_void_p()
    _check(load_library().bttb_learned_create(ctypes.byref(h), plan, rank, channels, max_cols, seed), plan)
    return h


def bttb_learned_param_count(learned) -> int:
    return int(load_library().bttb_learned_param_count(learned))


def bttb_learned_params(learned, host_array, to_host: bool) -> None:
    """host_array: C-contiguous float32 numpy array of param_count entries."""
    _check(load_library().bttb_learned_params(learned, _ptr(host_array), int(bool(to_host))))


def bttb_learned_apply(learned, r, z, ncols: int, ld: int, dtype: int) -> None:
    _check(load_library().bttb_learned_apply(learned, _ptr(r), _ptr(z), ncols, ld, dtype))


def bttb_learned_gradients(learned, r, e, ncols: int, ld: int, grad_host=None) -> float:
    loss = ctypes.c_double(0.0)
    g = _ptr(grad_host) if grad_host is not None else None
    _check(load_library().bttb_learned_gradients(learned, _ptr(r), _ptr(e), ncols, ld, g, ctypes.byref(loss)))
    return loss.value


def bttb_learned_train_step(learned, r, e, ncols: int, ld: int, lr: float, want_loss: bool = True):
    loss = ctypes.c_double(0.0)
    _check(load_library().bttb_learned_train_step(learned, _ptr(r), _ptr(e), ncols, ld, lr,
                                                  ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def bttb_plan_set_learned(plan, learned) -> None:
    _check(load_library().bttb_plan_set_learned(plan, learned), plan)


def bttb_learned_destroy(learned) -> None:
    if learned:
        _check(load_library().bttb_learned_destroy(learned))


def bttb_plan_autotune(plan, nrhs: int = 1, reps: int = 5) -> int:
    """FFT batch-chunk width chosen for products of nrhs columns."""
    out = ctypes.c_int(0)
    _check(load_library().bttb_plan_autotune(plan, nrhs, reps, ctypes.byref(out)), plan)
    return out.value


def bttb_plan_debug(plan, what: int, value: int) -> int:
    """Test hooks: BTTB_DEBUG_WAIT_LIMIT_NS, _WITHHOLD_ARRIVAL, _PRODUCT_ROUTE, _ROUTE_TAKEN (returns the route)."""
    return _check(load_library().bttb_plan_debug(plan, what, value), plan, soft_ok=True)


def bttb_check_report():
    """(checked, hits, first_bad_address): checked is False for the normal build (hits 0)."""
    h, f = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    rc = load_library().bttb_check_report(ctypes.byref(h), ctypes.byref(f))
    if rc < 0:
        _check(rc)
    return rc == 1, int(h.value), int(f.value)


def bttb_check_probe() -> int:
    """Checked build only: the failed checks counted by one deliberate read one element past a buffer
    (the check skips the read)."""
    h = ctypes.c_ulonglong(0)
    _check(load_library().bttb_check_probe(ctypes.byref(h)))
    return int(h.value)


def bttb_plan_workspace_bytes(plan) -> int:
    return int(load_library().bttb_plan_workspace_bytes(plan))


def bttb_plan_destroy(plan) -> None:
    if plan:
        _check(load_library().bttb_plan_destroy(plan))


def bttb_last_error(plan=None) -> str:
    return load_library().bttb_last_error(plan).decode()


# ---------------------------------------------------------------- convenience

def gmres_opts(tol=1e-8, restart=50, max_iters=5000, pc=BTTB_PC_NONE, inner=BTTB_MV_FP64, use_x0=False,
               host_io=False, history=None, flags=0) -> GmresOpts:
    o = GmresOpts()
    o.tol, o.restart, o.max_iters, o.pc, o.inner, o.flags = tol, restart, max_iters, pc, inner, flags
    o.use_x0, o.host_io = int(bool(use_x0)), int(bool(host_io))
    if history is not None:
        o.history = history.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.history_len = history.shape[0]
    return o


class Batch:
    """Owner of a bttb_batch: independent arrays of uneven sizes solved concurrently."""

    def __init__(self, specs, prec_mask=0):
        """specs: sequence of (nx, ny, b, nrhs)."""
        self.specs = [tuple(int(v) for v in s) for s in specs]
        nx, ny, b, k = zip(*self.specs)
        self.handle = bttb_batch_create(nx, ny, b, k, prec_mask)

    def set_generators(self, index, gen):
        bttb_batch_set_generators(self.handle, index, gen)

    def autotune(self, reps=5):
        return bttb_batch_autotune(self.handle, len(self.specs), reps)

    def solve(self, Vs, Is=None, **kw):
        """Vs[i]: (nrhs_i, N_i) complex128 device tensors; returns (Is, rc, results)."""
        import torch
        if Is is None:
            Is = [torch.zeros_like(v) for v in Vs]
        lds = [v.shape[1] for v in Vs]
        rc, res = bttb_batch_gmres_solve(self.handle, Vs, Is, lds, gmres_opts(**kw))
        return Is, rc, res

    def close(self):
        if getattr(self, "handle", None):
            bttb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owner of a bttb_plan handle (destroyed on close / garbage collection)."""

    def __init__(self, nx, ny, b, max_rhs=1, prec_mask=0, stream=None):
        self.nx, self.ny, self.b, self.max_rhs = nx, ny, b, max_rhs
        self.n = nx * ny * b
        self.handle = bttb_plan_create(nx, ny, b, max_rhs, prec_mask, stream)
        self.mx, self.my = bttb_plan_grid(self.handle)

    def set_generators(self, gen):
        bttb_set_generators(self.handle, gen)

    def matvec(self, x, y=None, prec=BTTB_MV_FP64):
        """x: (k, N) or (N,) complex tensor on the GPU; returns y = Z x of the same shape."""
        import torch
        xs = x.reshape(-1, self.n)
        if y is None:
            y = torch.empty_like(xs)
        dt = BTTB_C128 if xs.dtype == torch.complex128 else BTTB_C64
        bttb_matvec(self.handle, xs, y, xs.shape[0], self.n, dt, prec)
        return y.reshape(x.shape)

    def block_jacobi(self, x):
        import torch
        xs = x.reshape(-1, self.n)
        z = torch.empty_like(xs)
        dt = BTTB_C128 if xs.dtype == torch.complex128 else BTTB_C64
        bttb_block_jacobi_apply(self.handle, xs, z, xs.shape[0], self.n, dt)
        return z.reshape(x.shape)

    def solve(self, V, I=None, **kw):
        """V: (k, N) complex128 (GPU tensor, or host tensor with host_io=True)."""
        import torch
        vs = V.reshape(-1, self.n)
        if I is None:
            I = torch.zeros_like(vs)
        opts = gmres_opts(**kw)
        rc, res = bttb_gmres_solve(self.handle, vs, I, vs.shape[0], self.n, opts)
        return I.reshape(V.shape), rc, res

    def spectrum_bin(self, ky, kx):
        return bttb_get_spectrum_bin(self.handle, ky, kx, self.b)

    def autotune(self, nrhs=1, reps=5):
        return bttb_plan_autotune(self.handle, nrhs, reps)

    def workspace_bytes(self):
        return bttb_plan_workspace_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            bttb_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Learned:
    """Owner of a bttb_learned object (the learned correction of a plan).

    Parameters as a dict of numpy arrays with the shapes of the C layout:
    B (bins, rank, b) complex, A (bins, b, rank) complex, W1 (ch, 2*rank, 3, 3),
    c1 (ch,), W2 (ch, ch, 3, 3), c2 (ch,), W3 (2*rank, ch, 3, 3), c3 (2*rank,).
    """

    def __init__(self, plan: "Plan", rank=16, channels=64, max_cols=64, seed=0):
        self.plan, self.rank, self.channels, self.max_cols = plan, rank, channels, max_cols
        self.bins = plan.mx * plan.my
        self.handle = bttb_learned_create(plan.handle, rank, channels, max_cols, seed)
        self.count = bttb_learned_param_count(self.handle)

    def _shapes(self):
        R, C, b, bins = self.rank, self.channels, self.plan.b, self.bins
        return [("B", (bins, R, b), True), ("A", (bins, b, R), True), ("W1", (C, 2 * R, 3, 3), False),
                ("c1", (C,), False), ("W2", (C, C, 3, 3), False), ("c2", (C,), False),
                ("W3", (2 * R, C, 3, 3), False), ("c3", (2 * R,), False)]

    def unflatten(self, flat):
        import numpy as np
        out, o = {}, 0
        for name, shape, cplx in self._shapes():
            cnt = int(np.prod(shape)) * (2 if cplx else 1)
            v = flat[o:o + cnt]
            o += cnt
            out[name] = (v[0::2] + 1j * v[1::2]).reshape(shape) if cplx else v.reshape(shape).copy()
        return out

    def flatten(self, params):
        import numpy as np
        parts = []
        for name, shape, cplx in self._shapes():
            v = np.asarray(params[name]).reshape(-1)
            if cplx:
                w = np.empty(2 * v.size, dtype=np.float32)
                w[0::2], w[1::2] = v.real, v.imag
                parts.append(w)
            else:
                parts.append(v.astype(np.float32))
        return np.ascontiguousarray(np.concatenate(parts))

    def get_params(self):
        import numpy as np
        flat = np.empty(self.count, dtype=np.float32)
        bttb_learned_params(self.handle, flat, True)
        return self.unflatten(flat)

    def set_params(self, params):
        flat = self.flatten(params)
        assert flat.size == self.count
        bttb_learned_params(self.handle, flat, False)

    def apply(self, r):
        """M(r) for (k, N) device columns (complex64 or complex128)."""
        import torch
        rs = r.reshape(-1, self.plan.n)
        z = torch.empty_like(rs)
        dt = BTTB_C128 if rs.dtype == torch.complex128 else BTTB_C64
        bttb_learned_apply(self.handle, rs, z, rs.shape[0], self.plan.n, dt)
        return z.reshape(r.shape)

    def gradients(self, r, e):
        """(loss, grads dict) for complex64 device pairs (k, N)."""
        import numpy as np
        g = np.empty(self.count, dtype=np.float32)
        loss = bttb_learned_gradients(self.handle, r, e, r.shape[0], self.plan.n, g)
        return loss, self.unflatten(g)

    def train_step(self, r, e, lr=1e-3, want_loss=True):
        return bttb_learned_train_step(self.handle, r, e, r.shape[0], self.plan.n, lr, want_loss)

    def attach(self):
        bttb_plan_set_learned(self.plan.handle, self.handle)

    def close(self):
        if getattr(self, "handle", None):
            bttb_learned_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
