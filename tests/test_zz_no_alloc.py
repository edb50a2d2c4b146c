"""bttb_matvec_noalloc: the FP64 product for callers that cannot allocate.

Some callers cannot call cudaMalloc (a host application that only lets
plug-ins use memory reserved at load time, code running under CUDA graph
capture, a process whose allocator is owned by someone else), so they cannot
create a plan.  bttb_matvec_noalloc takes the generator blocks, the input and
the output from the caller and keeps everything else in a fixed file-scope
device array.  This test checks it against the plan-based bttb_matvec on two
calls in a row (a different problem each time, so the second call runs on the
scratch contents the first one left), within the FP64 tolerance of the other
parity tests.  It is collected last and passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

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
    rc = bt.load_library().bttb_matvec_noalloc(nx, ny, b, gen_dev.data_ptr(), x_dev.data_ptr(), y_dev.data_ptr(),
                                                k, nx * ny * b, ctypes.c_void_p(stream))
    assert rc == bt.BTTB_OK, bt.bttb_last_error()


@pytest.mark.parametrize("case", [[(4, 4, 12, 2, 0), (5, 3, 7, 3, 1)], [(6, 5, 16, 1, 2), (4, 4, 12, 4, 3)]])
def test_noalloc_matches_plan_product_twice(bt, case):
    for nx, ny, b, k, seed in case:
        gen = arrays.random_generator_blocks(nx, ny, b, seed=200 + seed)
        rng = np.random.default_rng(300 + seed)
        x = rng.standard_normal((k, nx * ny * b)) + 1j * rng.standard_normal((k, nx * ny * b))
        xd = torch.from_numpy(x).cuda()
        gd = torch.from_numpy(gen).cuda()
        y_new = torch.full_like(xd, np.nan)
        _noalloc(bt, nx, ny, b, gd, xd, y_new, k)
        plan = bt.Plan(nx, ny, b, max_rhs=k)
        plan.set_generators(gen)
        y_ref = plan.matvec(xd)
        torch.cuda.synchronize()
        a, r = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.linalg.norm(a - r) <= FP64_TOL * np.linalg.norm(r)
        assert np.abs(a - r).max() <= FP64_TOL * np.abs(r).max()
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(bt):
    lib = bt.load_library()
    nx, ny, b = 30, 30, 60                      # the 30x30 spectrum alone exceeds the fixed scratch
    x = torch.zeros(1, nx * ny * b, dtype=torch.complex128, device="cuda")
    g = torch.zeros(1, dtype=torch.complex128, device="cuda")
    rc = lib.bttb_matvec_noalloc(nx, ny, b, g.data_ptr(), x.data_ptr(), x.data_ptr(), 1, nx * ny * b, None)
    assert rc == bt.BTTB_ERR_INVALID_ARG
    assert "scratch" in bt.bttb_last_error()
