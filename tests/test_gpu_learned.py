"""Parity of the learned Fourier-domain correction (through the C ABI) with the
CPU oracle (oracle/learned.py), and its use inside flexible GMRES.

The CUDA path reads bfloat16 copies of B, A and the convolution weights (the
biases stay binary32) and accumulates in binary32, with binary32 FFTs and a
binary32 block-Jacobi part.  The oracle therefore gets the same bfloat16-rounded
parameters and runs in binary64; the remaining difference is binary32 rounding.
An output of M(r) passes through a few dozen accumulation steps, so outputs and
the loss are compared at TOL = 2e-4 relative (max-norm and 2-norm).  A weight
gradient sums products over every grid position, column and tap of the
minibatch (thousands of binary32 terms, in per-chunk partial sums), so the
gradients are compared at GRAD_TOL = 1e-3 relative, norm-wise per parameter
group.
"""
import numpy as np
import pytest

import oracle
from oracle import learned as olearned
from workloads import arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def bt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20350_gb300 import build
    build.build()
    import paper_2506_20350_gb300 as m
    m.load_library()
    return m


def bf16_round(x):
    """Round binary32 values to bfloat16 (nearest, ties to even), returned as binary32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _rounded(lrn, params):
    """The parameters as the kernels see them: B, A, W* through bfloat16, biases binary32."""
    flat = lrn.flatten(params)
    p = lrn.unflatten(flat)
    out = {}
    for k, v in p.items():
        if k.startswith("c"):
            out[k] = v.astype(np.float64)
        elif np.iscomplexobj(v):
            out[k] = bf16_round(v.real).astype(np.float64) + 1j * bf16_round(v.imag).astype(np.float64)
        else:
            out[k] = bf16_round(v).astype(np.float64)
    return out


def _random_params(lrn, rng, scale_ab=0.3, scale_w=0.15):
    shapes = dict((n, s) for n, s, _ in lrn._shapes())
    p = {}
    for k, s in shapes.items():
        if k in ("A", "B"):
            p[k] = (rng.standard_normal(s) + 1j * rng.standard_normal(s)) * scale_ab
        else:
            p[k] = rng.standard_normal(s) * scale_w
    return p


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SHAPES = [
    # nx, ny, b, rank, channels, columns
    (5, 4, 12, 8, 16, 3),
    (6, 5, 20, 16, 64, 37),
]


@pytest.mark.parametrize("nx,ny,b,rank,ch,k", SHAPES)
def test_apply_matches_oracle(bt, nx, ny, b, rank, ch, k):
    gen = arrays.generator_blocks(nx, ny, b, seed=70)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    lrn = bt.Learned(plan, rank=rank, channels=ch, max_cols=k, seed=71)
    params = _random_params(lrn, np.random.default_rng(72))
    lrn.set_params(params)
    rp = _rounded(lrn, params)
    rng = np.random.default_rng(73)
    r = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
    ref = oracle.block_jacobi_apply(gen, r.T).T + olearned.forward(gen, rp, r, plan.mx, plan.my)
    for dt in (torch.complex64, torch.complex128):
        z = lrn.apply(torch.from_numpy(r).to(dt).cuda()).cpu().numpy()
        err = np.abs(z - ref).max() / np.abs(ref).max()
        assert err <= TOL and _rel(z, ref) <= TOL, (dt, err)
    # the correction itself is a sizeable part of M(r): the test sees it
    f = olearned.forward(gen, rp, r, plan.mx, plan.my)
    assert np.linalg.norm(f) > 0.1 * np.linalg.norm(ref)
    lrn.close()
    plan.close()


@pytest.mark.parametrize("nx,ny,b,rank,ch,k", SHAPES)
def test_gradients_match_oracle(bt, nx, ny, b, rank, ch, k):
    gen = arrays.generator_blocks(nx, ny, b, seed=74)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    lrn = bt.Learned(plan, rank=rank, channels=ch, max_cols=k, seed=75)
    params = _random_params(lrn, np.random.default_rng(76))
    lrn.set_params(params)
    rp = _rounded(lrn, params)
    rng = np.random.default_rng(77)
    r = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
    e = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
    rd = torch.from_numpy(r).to(torch.complex64).cuda()
    ed = torch.from_numpy(e).to(torch.complex64).cuda()
    # the kernels read the inputs in binary32: give the oracle the same rounding of them
    r32 = rd.cpu().numpy().astype(np.complex128)
    e32 = ed.cpu().numpy().astype(np.complex128)
    loss_ref, g_ref = olearned.loss_and_grads(gen, rp, r32, e32, plan.mx, plan.my)
    loss, g = lrn.gradients(rd, ed)
    assert abs(loss - loss_ref) <= TOL * loss_ref, (loss, loss_ref)
    for name in ("B", "A", "W1", "c1", "W2", "c2", "W3", "c3"):
        assert _rel(g[name], g_ref[name]) <= GRAD_TOL, (name, _rel(g[name], g_ref[name]))
    lrn.close()
    plan.close()


def test_adam_step_updates_master_and_lowers_loss(bt):
    nx, ny, b, k = 6, 5, 12, 8
    gen = arrays.generator_blocks(nx, ny, b, seed=78)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    lrn = bt.Learned(plan, rank=8, channels=16, max_cols=k, seed=79)
    rng = np.random.default_rng(80)
    e = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
    r = oracle.matvec(gen, e.T).T
    rd = torch.from_numpy(r).to(torch.complex64).cuda()
    ed = torch.from_numpy(e).to(torch.complex64).cuda()
    p0 = np.empty(lrn.count, dtype=np.float32)
    bt.bttb_learned_params(lrn.handle, p0, True)
    l0, g0 = lrn.gradients(rd, ed)
    lr = 1e-3
    l_first = lrn.train_step(rd, ed, lr=lr)
    assert abs(l_first - l0) <= 1e-6 * l0           # same minibatch, same weights
    p1 = np.empty(lrn.count, dtype=np.float32)
    bt.bttb_learned_params(lrn.handle, p1, True)
    # first Adam step: w1 = w0 - lr * g/(|g| + eps) elementwise (bias-corrected moments)
    gflat = lrn.flatten(g0)
    expect = p0 - lr * gflat / (np.abs(gflat) + 1e-8)
    np.testing.assert_allclose(p1, expect, rtol=1e-5, atol=1e-7)
    for _ in range(30):
        last = lrn.train_step(rd, ed, lr=lr)
    assert last < 0.9 * l0
    lrn.close()
    plan.close()


def test_invalid_arguments(bt):
    plan = bt.Plan(4, 4, 12, max_rhs=2)
    with pytest.raises(bt.BttbError):
        bt.Learned(plan, rank=12, channels=64, max_cols=2)     # rank not in {8, 16, 32}
    with pytest.raises(bt.BttbError):
        bt.Learned(plan, rank=16, channels=48, max_cols=2)
    plan.set_generators(arrays.generator_blocks(4, 4, 12, seed=0))
    lrn = bt.Learned(plan, rank=8, channels=16, max_cols=2)
    x = torch.zeros((3, plan.n), dtype=torch.complex64, device="cuda")
    with pytest.raises(bt.BttbError):
        lrn.apply(x)                                            # more columns than max_cols
    V = torch.zeros((1, plan.n), dtype=torch.complex128, device="cuda")
    V[0, 0] = 1.0
    with pytest.raises(bt.BttbError):
        plan.solve(V, pc=bt.BTTB_PC_LEARNED)                    # nothing attached yet
    lrn.close()
    plan.close()


def _pairs(plan, V, snapshots):
    """(residual, exact correction) pairs from partial solves of the plain solver,
    each pair scaled so that the residual has unit norm."""
    x_star, rc, _ = plan.solve(V, tol=1e-11, restart=50, max_iters=3000)
    assert rc == 0
    rs, es = [], []
    for j in snapshots:
        if j == 0:
            xj = torch.zeros_like(V)
        else:
            xj, _, _ = plan.solve(V, tol=1e-14, restart=50, max_iters=j)
        r = V - plan.matvec(xj)
        e = x_star - xj
        nr = torch.linalg.vector_norm(r, dim=1, keepdim=True)
        rs.append(r / nr)
        es.append(e / nr)
    return torch.cat(rs).to(torch.complex64).contiguous(), torch.cat(es).to(torch.complex64).contiguous()


def test_trained_correction_in_fgmres(bt):
    """Trained on pairs from the plain solver, the learned preconditioner lowers the
    held-out loss below block-Jacobi's and, inside flexible GMRES, solves held-out
    right-hand sides to the requested true residual in fewer iterations than P_K."""
    nx, ny, b = 12, 12, 24
    gen = arrays.generator_blocks(nx, ny, b, seed=4)
    plan = bt.Plan(nx, ny, b, max_rhs=64)
    plan.set_generators(gen)
    Vtr = torch.from_numpy(arrays.random_port_excitations(nx, ny, b, 48, seed=4).T.copy()).cuda()
    Vte = torch.from_numpy(arrays.random_port_excitations(nx, ny, b, 8, seed=5).T.copy()).cuda()
    rtr, etr = _pairs(plan, Vtr, (0, 5, 15, 40))
    rte, ete = _pairs(plan, Vte, (0, 10))
    lrn = bt.Learned(plan, rank=16, channels=32, max_cols=64, seed=6)
    loss_bj = lrn.gradients(rte, ete)[0]         # f starts near zero: about P_K's own loss
    gen_t = torch.Generator().manual_seed(7)
    for step in range(400):
        idx = torch.randperm(rtr.shape[0], generator=gen_t)[:64].cuda()
        lrn.train_step(rtr[idx].contiguous(), etr[idx].contiguous(), lr=2e-3, want_loss=False)
    loss_te = lrn.gradients(rte, ete)[0]
    assert loss_te < 0.8 * loss_bj, (loss_te, loss_bj)
    lrn.attach()
    tol = 1e-8
    _, rc_bj, res_bj = plan.solve(Vte, tol=tol, restart=50, max_iters=2000, pc=bt.BTTB_PC_BLOCK_JACOBI)
    I_l, rc_l, res_l = plan.solve(Vte, tol=tol, restart=50, max_iters=2000, pc=bt.BTTB_PC_LEARNED)
    assert rc_bj == 0 and rc_l == 0
    assert all(r.relres_true <= tol for r in res_l)
    rel = oracle.relres(gen, Vte.cpu().numpy().T, I_l.cpu().numpy().T)
    assert np.all(rel <= tol), rel
    it_bj = sum(r.iters for r in res_bj)
    it_l = sum(r.iters for r in res_l)
    assert it_l < it_bj, (it_l, it_bj)
    bt.bttb_plan_set_learned(plan.handle, None)
    lrn.close()
    plan.close()
