"""Failure paths and input range of the GMRES solver, on the GPU, through the C ABI.

None of these tests faults or hangs the GPU.  The timeout test uses the
library's own test hook: one warp of one block-product launch withholds an
mbarrier arrival, its bounded wait runs out after 1 ms, the kernel supplies
the arrival, drains its copies and returns, and the solve reports
BTTB_ERR_TIMEOUT.  Every solve that succeeds is checked with the oracle's
product (the true relative residual ||V - Z I|| / ||V|| in binary64).
"""
import numpy as np
import pytest

import oracle
from workloads import arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20350_gb300 import build
    build.build()
    import paper_2506_20350_gb300 as m
    m.load_library()
    return m


@pytest.fixture(scope="module")
def tiny():
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    v = arrays.port_excitations(nx, ny, b, [(1, 1)])[:, 0]
    return nx, ny, b, gen, v


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("scale", [1e-30, 1e-25, 1e25, 1e30])
def test_scaled_right_hand_side(bt, tiny, scale):
    """Double-float has binary32's exponent range; the solver scales each column of V by a power of two
    first, so V * 1e-30 .. V * 1e30 solve like V: BTTB_OK, the oracle's residual at tol, and I scaled."""
    nx, ny, b, gen, v = tiny
    plan = bt.Plan(nx, ny, b, max_rhs=1)
    plan.set_generators(gen)
    tol = 1e-10
    I1, rc1, _ = plan.solve(_dev(v[None, :]), tol=tol, restart=50)
    Is, rcs, res = plan.solve(_dev(scale * v[None, :]), tol=tol, restart=50)
    assert rc1 == bt.BTTB_OK and rcs == bt.BTTB_OK
    a, a1 = Is.cpu().numpy()[0], I1.cpu().numpy()[0]
    assert np.all(np.isfinite(a)) and np.abs(a).max() > 0.0
    rel = oracle.relres(gen, scale * v, a)[0]
    assert rel <= tol and res[0].relres_true <= tol, (rel, res[0].relres_true)
    # same problem up to the scale: the two solutions agree to the solve's accuracy
    assert np.linalg.norm(a / scale - a1) <= 1e-8 * np.linalg.norm(a1)
    plan.close()


def test_columns_of_very_different_scale_in_one_solve(bt, tiny):
    """Per-column scaling: columns at 1e-30, 1 and 1e30 in one batched solve all reach tol (binary32 inner
    products, FP64-class refinement)."""
    nx, ny, b, gen, v = tiny
    scales = np.array([1e-30, 1.0, 1e30])
    V = scales[:, None] * v[None, :]
    plan = bt.Plan(nx, ny, b, max_rhs=3)
    plan.set_generators(gen)
    tol = 1e-10
    I, rc, res = plan.solve(_dev(V), tol=tol, restart=50, inner=bt.BTTB_MV_FP32)
    assert rc == bt.BTTB_OK
    rel = oracle.relres(gen, V.T, I.cpu().numpy().T)
    assert np.all(rel <= tol), rel
    plan.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_right_hand_side(bt, tiny, bad):
    """A NaN or Inf in V: the device norm of V is non-finite and the solve returns BTTB_ERR_NONFINITE."""
    nx, ny, b, gen, v = tiny
    plan = bt.Plan(nx, ny, b, max_rhs=1)
    plan.set_generators(gen)
    vb = v.copy()
    vb[7] = bad
    with pytest.raises(bt.BttbError) as e:
        plan.solve(_dev(vb[None, :]), tol=1e-10, restart=50)
    assert e.value.code == bt.BTTB_ERR_NONFINITE
    # the plan still works afterwards
    I, rc, _ = plan.solve(_dev(v[None, :]), tol=1e-10, restart=50)
    assert rc == bt.BTTB_OK and oracle.relres(gen, v, I.cpu().numpy()[0])[0] <= 1e-10
    plan.close()


def test_zero_right_hand_side_gives_zero_solution(bt, tiny):
    """V = 0 has the solution I = 0, whatever the initial guess; the other column is solved as usual."""
    nx, ny, b, gen, v = tiny
    plan = bt.Plan(nx, ny, b, max_rhs=2)
    plan.set_generators(gen)
    V = np.stack([np.zeros_like(v), v])
    x0 = torch.ones((2, plan.n), dtype=torch.complex128, device="cuda")
    I, rc, res = plan.solve(_dev(V), I=x0, tol=1e-10, restart=50, use_x0=True)
    assert rc == bt.BTTB_OK
    a = I.cpu().numpy()
    assert np.all(a[0] == 0.0)
    assert oracle.relres(gen, v, a[1])[0] <= 1e-10
    assert res[0].status == bt.BTTB_OK and res[0].relres_true == 0.0
    plan.close()


def test_happy_breakdown_on_an_eigenvector(bt):
    """b = 1, periodic generators: Z is block circulant with Fourier modes as eigenvectors (Sec. II-B).  With
    V a mode, the Krylov space is exhausted after one step (a happy breakdown): the solve ends with BTTB_OK
    and I = V / lambda, with no NaN from the zero subdiagonal."""
    nx, ny = 5, 4
    gen, c = arrays.periodic_generator_blocks(nx, ny, seed=9)
    lam = np.fft.fft2(c)
    kx, ky = np.unravel_index(np.argmax(np.abs(lam)), lam.shape)
    ix = np.tile(np.arange(nx), ny)
    iy = np.repeat(np.arange(ny), nx)
    mode = np.exp(2j * np.pi * (kx * ix / nx + ky * iy / ny))
    plan = bt.Plan(nx, ny, 1, max_rhs=1)
    plan.set_generators(gen)
    for flags in (0, 4):                    # delayed CGS2 (default) and two-pass CGS2
        I, rc, res = plan.solve(_dev(mode[None, :]), tol=1e-12, restart=20, flags=flags)
        a = I.cpu().numpy()[0]
        assert rc == bt.BTTB_OK and np.all(np.isfinite(a))
        assert res[0].iters <= 2, res[0].iters  # delayed CGS2 sees the zero subdiagonal one step later
        np.testing.assert_allclose(a, mode / lam[kx, ky], rtol=0, atol=1e-12 * np.abs(mode / lam[kx, ky]).max())
    plan.close()


@pytest.mark.parametrize("route", [1, 3, 4])
def test_timeout_is_reported_and_the_plan_recovers(bt, tiny, route):
    """A block-product launch that withholds an mbarrier arrival (the warp-per-bin kernel of the strided
    route, the fused level-2 kernel, and the whole-product persistent kernel, whose other CTAs then also
    pass its later grid barriers): the bounded wait (1 ms here) runs out, the kernel drains its copies and
    returns, and the solve returns BTTB_ERR_TIMEOUT.  The same plan and a fresh plan then solve normally."""
    nx, ny, b, gen, v = tiny
    plan = bt.Plan(nx, ny, b, max_rhs=1)
    plan.set_generators(gen)
    bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, route)
    bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_WAIT_LIMIT_NS, 1_000_000)
    bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_WITHHOLD_ARRIVAL, 1)
    with pytest.raises(bt.BttbError) as e:
        plan.solve(_dev(v[None, :]), tol=1e-10, restart=50)
    assert e.value.code == bt.BTTB_ERR_TIMEOUT
    torch.cuda.synchronize()                # the context is still usable
    bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_WAIT_LIMIT_NS, 0)
    I, rc, _ = plan.solve(_dev(v[None, :]), tol=1e-10, restart=50)
    assert rc == bt.BTTB_OK and oracle.relres(gen, v, I.cpu().numpy()[0])[0] <= 1e-10
    fresh = bt.Plan(nx, ny, b, max_rhs=1)
    fresh.set_generators(gen)
    I2, rc2, _ = fresh.solve(_dev(v[None, :]), tol=1e-10, restart=50)
    assert rc2 == bt.BTTB_OK and oracle.relres(gen, v, I2.cpu().numpy()[0])[0] <= 1e-10
    with pytest.raises(bt.BttbError) as e:
        bt.bttb_plan_debug(plan.handle, 99, 0)
    assert e.value.code == bt.BTTB_ERR_INVALID_ARG
    fresh.close()
    plan.close()
