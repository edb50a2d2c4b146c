"""bttb_matvec_noalloc: the FP64 product for callers that cannot allocate.

Some callers cannot call cudaMalloc (a host application that only lets
plug-ins use memory reserved at load time, code running under CUDA graph
capture, a process whose allocator is owned by someone else), so they cannot
create a plan.  bttb_matvec_noalloc takes the generator blocks, the input and
the output from the caller and keeps everything else in a fixed file-scope
device array.  These tests check it against the oracle's O(N^2) product and
against the plan-based bttb_matvec on two calls in a row (a different problem
each time, so the second call runs on the scratch contents the first one
left), within the FP64 tolerance of the other parity tests; with one to four
columns and with five to eight (the two FFT forms of the product); that a
repeated call allocates no device memory; and that non-finite generators are
not detected (the call does not synchronise: they come out as a non-finite y).
The file is collected last and passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

import oracle
from workloads import arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def bt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20350_gb300 import build
    build.build()
    import paper_2506_20350_gb300 as m
    m.load_library()
    return m


def _noalloc(bt, nx, ny, b, gen_dev, x_dev, y_dev, k):
    stream = torch.cuda.current_stream().cuda_stream
    return bt.load_library().bttb_matvec_noalloc(nx, ny, b, gen_dev.data_ptr(), x_dev.data_ptr(), y_dev.data_ptr(),
                                                 k, nx * ny * b, ctypes.c_void_p(stream))


def _close(a, r):
    return (np.linalg.norm(a - r) <= FP64_TOL * np.linalg.norm(r)
            and np.abs(a - r).max() <= FP64_TOL * np.abs(r).max())


@pytest.mark.parametrize("case", [[(4, 4, 12, 2, 0), (5, 3, 7, 3, 1)], [(6, 5, 16, 1, 2), (4, 4, 12, 4, 3)],
                                  [(5, 4, 12, 6, 4), (3, 5, 10, 8, 5)]])
def test_noalloc_matches_oracle_and_plan_product_twice(bt, case):
    for nx, ny, b, k, seed in case:
        gen = arrays.random_generator_blocks(nx, ny, b, seed=200 + seed)
        rng = np.random.default_rng(300 + seed)
        x = rng.standard_normal((k, nx * ny * b)) + 1j * rng.standard_normal((k, nx * ny * b))
        xd = torch.from_numpy(x).cuda()
        gd = torch.from_numpy(gen).cuda()
        y_new = torch.full_like(xd, np.nan)
        rc = _noalloc(bt, nx, ny, b, gd, xd, y_new, k)
        assert rc == bt.BTTB_OK, bt.bttb_last_error()
        plan = bt.Plan(nx, ny, b, max_rhs=k)
        plan.set_generators(gen)
        y_ref = plan.matvec(xd)
        torch.cuda.synchronize()
        a = y_new.cpu().numpy()
        assert _close(a, oracle.matvec(gen, x.T).T), (nx, ny, b, k)
        assert _close(a, y_ref.cpu().numpy()), (nx, ny, b, k)
        plan.close()


def test_noalloc_repeated_call_allocates_nothing(bt):
    """Once a shape has run (its kernels loaded), another call leaves the device's free memory unchanged."""
    nx, ny, b, k = 4, 4, 12, 6
    gen = arrays.random_generator_blocks(nx, ny, b, seed=210)
    rng = np.random.default_rng(310)
    x = rng.standard_normal((k, nx * ny * b)) + 1j * rng.standard_normal((k, nx * ny * b))
    xd, gd = torch.from_numpy(x).cuda(), torch.from_numpy(gen).cuda()
    y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
    assert _noalloc(bt, nx, ny, b, gd, xd, y1, k) == bt.BTTB_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _noalloc(bt, nx, ny, b, gd, xd, y2, k) == bt.BTTB_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.equal(y1, y2)
    assert _close(y2.cpu().numpy(), oracle.matvec(gen, x.T).T)


def test_noalloc_does_not_detect_non_finite_generators(bt):
    """The call returns once its work is queued, so it cannot report device-side findings: a NaN in the
    generators gives BTTB_OK and a non-finite y (a plan's bttb_set_generators would reject them)."""
    nx, ny, b, k = 4, 3, 6, 1
    gen = arrays.random_generator_blocks(nx, ny, b, seed=211)
    gen[1, 2, 0, 3] = np.nan
    x = torch.ones((k, nx * ny * b), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(bt, nx, ny, b, torch.from_numpy(gen).cuda(), x, y, k) == bt.BTTB_OK
    torch.cuda.synchronize()
    assert not torch.isfinite(torch.view_as_real(y)).all()


def test_noalloc_rejects_sizes_beyond_its_scratch(bt):
    lib = bt.load_library()
    nx, ny, b = 30, 30, 60                      # the 30x30 spectrum alone exceeds the fixed scratch
    x = torch.zeros(1, nx * ny * b, dtype=torch.complex128, device="cuda")
    g = torch.zeros(1, dtype=torch.complex128, device="cuda")
    rc = lib.bttb_matvec_noalloc(nx, ny, b, g.data_ptr(), x.data_ptr(), x.data_ptr(), 1, nx * ny * b, None)
    assert rc == bt.BTTB_ERR_INVALID_ARG
    assert "scratch" in bt.bttb_last_error()
