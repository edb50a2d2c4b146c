"""Solves with hundreds of right-hand sides (Sec. III-C) through the C ABI.

With many columns (or one long global column) the delayed-CGS2 reduction runs
chunk-major: one CTA covers a chunk of every basis vector and streams the
basis through shared memory.  On a 152-SM GPU the sizes below select that
layout (chunk groups x columns >= 2 x SMs) for both the per-column and the
global solve; the single-column solves they are compared with use the
vector-major layout.  Every solve must reach the requested residual as
measured with the oracle's product.
"""
import numpy as np
import pytest

import oracle
from workloads import arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX, NY, B = 16, 16, 12          # N = 3072: 12 reduction chunks of 256 entries, 2 chunk groups per column


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
def problem():
    gen = arrays.generator_blocks(NX, NY, B, seed=41)
    v = arrays.port_excitations(NX, NY, B).T.copy()             # 256 columns
    return gen, v


@pytest.mark.parametrize("pc", [0, 1])
def test_all_ports_per_column(bt, problem, pc):
    gen, v = problem
    tol = 1e-8
    plan = bt.Plan(NX, NY, B, max_rhs=v.shape[0])
    plan.set_generators(gen)
    sol, rc, res = plan.solve(torch.from_numpy(v).cuda(), tol=tol, restart=30, inner=bt.BTTB_MV_FP32, pc=pc)
    assert rc == bt.BTTB_OK, bt.bttb_last_error()
    x = sol.cpu().numpy()
    rr = oracle.relres(gen, v.T, x.T)
    assert np.all(rr <= tol), rr.max()
    np.testing.assert_allclose([r.relres_true for r in res], rr, rtol=1e-6, atol=1e-14)
    for col in (0, 101, 255):
        s1, _, r1 = plan.solve(torch.from_numpy(v[col:col + 1].copy()).cuda(), tol=tol, restart=30,
                               inner=bt.BTTB_MV_FP32, pc=pc)
        x1 = s1.cpu().numpy()[0]
        assert np.linalg.norm(x[col] - x1) <= 1e-6 * np.linalg.norm(x1)
        assert abs(r1[0].iters - res[col].iters) <= 2
    plan.close()


def test_all_ports_global(bt, problem):
    gen, v = problem
    tol = 1e-8
    plan = bt.Plan(NX, NY, B, max_rhs=v.shape[0])
    plan.set_generators(gen)
    sol, rc, res = plan.solve(torch.from_numpy(v).cuda(), tol=tol, restart=30, inner=bt.BTTB_MV_FP32,
                              flags=bt.BTTB_GMRES_GLOBAL)
    assert rc == bt.BTTB_OK, bt.bttb_last_error()
    rr = oracle.relres(gen, v.T, sol.cpu().numpy().T)
    assert np.all(rr <= tol), rr.max()
    assert len({r.iters for r in res}) == 1
    plan.close()
