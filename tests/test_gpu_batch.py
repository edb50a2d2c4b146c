"""Batches of independent arrays of uneven sizes, solved concurrently."""
import numpy as np
import pytest

import oracle
from workloads import arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPECS = [(3, 4, 8, 2), (6, 2, 12, 1), (5, 5, 7, 3), (2, 7, 24, 1), (4, 4, 12, 4)]


@pytest.fixture(scope="module")
def bt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20350_gb300 import build
    build.build()
    import paper_2506_20350_gb300 as m
    m.load_library()
    return m


def _problem(i, spec):
    nx, ny, b, k = spec
    gen = arrays.generator_blocks(nx, ny, b, seed=500 + i)
    cells = [(c % nx, c // nx) for c in range(k)]
    v = arrays.port_excitations(nx, ny, b, cells).T.copy()
    return gen, v


def test_uneven_batch_matches_oracle_and_single_plans(bt):
    probs = [_problem(i, s) for i, s in enumerate(SPECS)]
    batch = bt.Batch(SPECS)
    for i, (gen, _) in enumerate(probs):
        batch.set_generators(i, gen)
    vs = [torch.from_numpy(v).cuda() for _, v in probs]
    sols, rc, res = batch.solve(vs, tol=1e-9, restart=20, inner=bt.BTTB_MV_FP32)
    assert rc == bt.BTTB_OK, bt.bttb_last_error()
    assert len(res) == sum(s[3] for s in SPECS)
    off = 0
    for i, ((gen, v), s) in enumerate(zip(probs, sols)):
        x = s.cpu().numpy()
        rr = oracle.relres(gen, v.T, x.T)
        assert np.all(rr <= 1e-9), (i, rr)
        for c in range(v.shape[0]):
            assert res[off + c].status == bt.BTTB_OK
            assert abs(res[off + c].relres_true - rr[c]) <= 1e-3 * 1e-9 + 1e-12
        off += v.shape[0]
        # the same array through a plan of its own gives the same bits
        nx, ny, b, k = SPECS[i]
        plan = bt.Plan(nx, ny, b, max_rhs=k)
        plan.set_generators(gen)
        xs, _, _ = plan.solve(vs[i], tol=1e-9, restart=20, inner=bt.BTTB_MV_FP32)
        assert torch.equal(xs, s)
        plan.close()
    batch.close()


def test_autotune_keeps_results(bt):
    probs = [_problem(i, s) for i, s in enumerate(SPECS)]
    batch = bt.Batch(SPECS)
    for i, (gen, _) in enumerate(probs):
        batch.set_generators(i, gen)
    vs = [torch.from_numpy(v).cuda() for _, v in probs]
    before, _, _ = batch.solve(vs, tol=1e-9, restart=20, inner=bt.BTTB_MV_FP32)
    widths = batch.autotune(reps=2)
    assert len(widths) == len(SPECS) and all(w in (2, 4, 8, 16, 32, 64) for w in widths)
    after, rc, _ = batch.solve(vs, tol=1e-9, restart=20, inner=bt.BTTB_MV_FP32)
    assert rc == bt.BTTB_OK
    for a, c in zip(before, after):
        assert torch.equal(a, c)          # the tuned form and chunk width change scheduling, not arithmetic
    batch.close()


def test_torch_generator_synthesis_matches_numpy(bt):
    g_np = arrays.generator_blocks(4, 3, 6, seed=9)
    g_t = arrays.generator_blocks_torch(4, 3, 6, seed=9, device="cuda").cpu().numpy()
    np.testing.assert_allclose(g_t, g_np, rtol=1e-13, atol=1e-15)


def test_batch_products_match_oracle_and_single_plans(bt):
    """A plan inside a batch runs products of few columns with both FFT levels fused in one kernel each
    way; a lone plan runs binary32 products as strided passes.  Both agree with the oracle, and bit for bit
    with each other (the same butterflies in the same order)."""
    batch = bt.Batch(SPECS)
    for i, spec in enumerate(SPECS):
        nx, ny, b, k = spec
        gen = arrays.random_generator_blocks(nx, ny, b, seed=700 + i)
        batch.set_generators(i, gen)
        rng = np.random.default_rng(i)
        n = nx * ny * b
        x = (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))).astype(np.complex64)
        ref = oracle.matvec(gen, x.T.astype(np.complex128)).T
        xd = torch.from_numpy(x).cuda()
        yb = torch.empty_like(xd)
        ph = bt.bttb_batch_plan(batch.handle, i)
        bt.bttb_matvec(ph, xd, yb, k, n, bt.BTTB_C64, bt.BTTB_MV_FP32)
        torch.cuda.synchronize()
        err = np.linalg.norm(yb.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (spec, err)
        plan = bt.Plan(nx, ny, b, max_rhs=k)
        plan.set_generators(gen)
        ys = plan.matvec(xd, prec=bt.BTTB_MV_FP32)
        assert torch.equal(ys, yb), spec
        plan.close()
    batch.close()
