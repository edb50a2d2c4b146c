"""Global GMRES for many right-hand sides (Sec. III-C, Eq. (ZIVvec)) through the C ABI.

Global GMRES on k columns is plain GMRES on the stacked system
(I (x) Z) vec(I) = vec(V).  After a fixed number of steps from x0 = 0 its
iterate is the unique minimiser of the residual over that Krylov space, so it
must match the oracle's textbook GMRES run on the stacked operator (built from
the oracle's O(N^2) product) to the accuracy of the FP64-class arithmetic.
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


def _stacked_oracle(gen, V, steps):
    """Oracle GMRES on vec(I) after `steps` Arnoldi steps (no restart)."""
    k, n = V.shape

    def apply(v):
        return oracle.matvec(gen, v.reshape(k, n).T).T.reshape(-1)

    x, info = oracle.gmres(apply, V.reshape(-1), tol=1e-300, restart=steps, max_iters=steps)
    return x.reshape(k, n), info


@pytest.mark.parametrize("steps", [4, 11])
def test_global_iterate_matches_oracle(bt, steps):
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    k = 5
    V = arrays.random_port_excitations(nx, ny, b, k, seed=90).T.copy()
    ref, _ = _stacked_oracle(gen, V, steps)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    Vd = torch.from_numpy(V).cuda()
    I, rc, res = plan.solve(Vd, tol=1e-14, restart=50, max_iters=steps, flags=bt.BTTB_GMRES_GLOBAL)
    assert rc == bt.BTTB_NOT_CONVERGED
    assert all(r.iters == steps for r in res)
    got = I.cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-10, err
    # one Krylov space per column gives a different iterate after the same number of steps
    Ip, _, _ = plan.solve(Vd, tol=1e-14, restart=50, max_iters=steps)
    assert np.linalg.norm(Ip.cpu().numpy() - ref) / np.linalg.norm(ref) > 1e-6
    plan.close()


@pytest.mark.parametrize("pc,inner", [(0, 0), (1, 1)])
def test_global_solve_reaches_tol(bt, pc, inner):
    nx, ny, b, k, tol = 8, 7, 12, 9, 1e-8
    gen = arrays.generator_blocks(nx, ny, b, seed=91)
    V = arrays.port_excitations(nx, ny, b, [(i % nx, i // nx) for i in range(0, 3 * k, 3)]).T.copy()
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    I, rc, res = plan.solve(torch.from_numpy(V).cuda(), tol=tol, restart=20, max_iters=3000, pc=pc, inner=inner,
                            flags=bt.BTTB_GMRES_GLOBAL)
    assert rc == bt.BTTB_OK
    rel = oracle.relres(gen, V.T, I.cpu().numpy().T)
    assert np.all(rel <= tol), rel
    assert len({r.iters for r in res}) == 1                   # one Krylov space: same count for all
    np.testing.assert_allclose([r.relres_true for r in res], rel, rtol=1e-6, atol=1e-14)
    plan.close()


def test_global_with_single_column_is_plain_gmres(bt):
    c = arrays.CONFIGS["tiny"]
    gen = arrays.generator_blocks(c["nx"], c["ny"], c["b"], c["seed"])
    plan = bt.Plan(c["nx"], c["ny"], c["b"], max_rhs=1)
    plan.set_generators(gen)
    V = torch.from_numpy(arrays.centre_excitation(c["nx"], c["ny"], c["b"])[None, :].copy()).cuda()
    Ig, _, rg = plan.solve(V, tol=1e-10, flags=bt.BTTB_GMRES_GLOBAL)
    Ip, _, rp = plan.solve(V, tol=1e-10)
    assert rg[0].iters == rp[0].iters
    assert torch.equal(Ig, Ip)
    plan.close()
