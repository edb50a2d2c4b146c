"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the FP64 product (double-float or binary64) within 1e-12 relative
of the oracle, the binary32 product within 1e-5 relative, every solve at the
requested relative residual as measured with the oracle's product.
"""
import numpy as np
import pytest

import oracle
from workloads import arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def bt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_20350_gb300 import build
    build.build()
    import paper_2506_20350_gb300 as m
    m.load_library()
    return m


def _dev(x_kn):
    return torch.from_numpy(np.ascontiguousarray(x_kn)).cuda()


def _rand(rng, k, n):
    return rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))


def _check(y, ref, tol, what=""):
    scale = np.abs(ref).max()
    err_inf = np.abs(y - ref).max() / scale
    err_2 = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err_inf <= tol and err_2 <= tol, f"{what}: max-rel {err_inf:.3e}, norm-rel {err_2:.3e} (tol {tol})"
    return err_2


ALL_PRECS = (1 << 0) | (1 << 1) | (1 << 2)


# ------------------------------------------------------------------ products

def test_tiny_product_all_precisions(bt):
    c = arrays.CONFIGS["tiny"]
    gen = arrays.generator_blocks(c["nx"], c["ny"], c["b"], c["seed"])
    plan = bt.Plan(c["nx"], c["ny"], c["b"], max_rhs=3, prec_mask=ALL_PRECS)
    plan.set_generators(gen)
    assert (plan.mx, plan.my) == (8, 8)
    x = _rand(np.random.default_rng(1), 3, plan.n)
    ref = oracle.matvec(gen, x.T).T
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, "df64")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64_NATIVE).cpu().numpy(), ref, FP64_TOL, "binary64")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref, FP32_TOL, "binary32")
    x32 = _dev(x.astype(np.complex64))
    _check(plan.matvec(x32, prec=bt.BTTB_MV_FP32).cpu().numpy(), oracle.matvec(gen, x.astype(np.complex64).T).T,
           FP32_TOL, "binary32 c64 io")


@pytest.mark.parametrize("nx,ny,b,k", [
    (5, 3, 7, 3),      # odd b, ragged chunks
    (1, 1, 5, 1),      # single cell: dense GEMV
    (1, 6, 3, 2),      # one column of cells
    (7, 1, 4, 1),      # one row: 1-level block Toeplitz
    (2, 2, 1, 5),      # scalar blocks, two contraction groups
    (13, 9, 16, 2),    # grid 25 x 18: radix 5, 3, 2
    (33, 5, 24, 1),    # grid 72 x 9
    (4, 3, 96, 2),     # wide blocks: the spectrum is streamed in column chunks
    (3, 2, 256, 1),    # largest b
])
def test_product_random_generators(bt, nx, ny, b, k):
    gen = arrays.random_generator_blocks(nx, ny, b, seed=100 + nx + ny + b)
    plan = bt.Plan(nx, ny, b, max_rhs=k, prec_mask=ALL_PRECS)
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(2), k, plan.n)
    ref = oracle.matvec(gen, x.T).T
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, "df64")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64_NATIVE).cpu().numpy(), ref, FP64_TOL, "binary64")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref, FP32_TOL, "binary32")


@pytest.mark.parametrize("nx,ny,b,k", [
    (5, 3, 7, 20),     # odd b, one 64-column tile (partial)
    (4, 4, 12, 65),    # two tiles, the second with one column
    (3, 3, 33, 130),   # three row warps' layout (rw = 2), three tiles
    (3, 2, 96, 70),    # widest multi-RHS layout (rw = 3)
    (5, 4, 60, 70),    # 4 x 4 register tiles (b <= 64), even b: 16-byte row-pair loads
    (3, 3, 64, 129),   # largest b of the 4 x 4 tiles, a one-column third tile
    (4, 3, 45, 17),    # odd b between 32 and 64: row-by-row loads, second row pairs partly valid
])
def test_multi_rhs_product_binary32(bt, nx, ny, b, k):
    """k > 8 right-hand sides take the tiled per-bin GEMM (binary32)."""
    gen = arrays.random_generator_blocks(nx, ny, b, seed=300 + b + k)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(7), k, plan.n)
    ref = oracle.matvec(gen, x.T).T
    y = plan.matvec(_dev(x.astype(np.complex64)), prec=bt.BTTB_MV_FP32).cpu().numpy()
    _check(y, ref, FP32_TOL, "multi-RHS binary32")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, "multi-RHS df64")


@pytest.mark.parametrize("nx,ny,b,k", [(5, 4, 60, 16), (6, 5, 60, 70), (4, 3, 64, 130), (7, 6, 12, 65),
                                        (3, 5, 1, 33), (4, 4, 37, 20), (5, 3, 96, 40), (4, 4, 60, 9),
                                        (3, 3, 2, 17), (4, 2, 30, 31), (6, 4, 24, 97)])
def test_tensor_core_product(bt, nx, ny, b, k):
    """BTTB_MV_TC_3XTF32: the per-bin GEMM on the tensor cores (3xTF32) for >= 16 columns and b <= 64:
    tcgen05 MMAs on TMA-fed tiles for even b (one to four K blocks of the 2b-row embedding, partial last
    column tiles), warp-level MMAs for odd b; binary32 elsewhere (b = 96, k = 9); binary32-level accuracy."""
    gen = arrays.random_generator_blocks(nx, ny, b, seed=400 + b + k)
    plan = bt.Plan(nx, ny, b, max_rhs=k, prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_TC_3XTF32))
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(8), k, plan.n)
    ref = oracle.matvec(gen, x.T).T
    y = plan.matvec(_dev(x.astype(np.complex64)), prec=bt.BTTB_MV_TC_3XTF32).cpu().numpy()
    _check(y, ref, FP32_TOL, "tensor-core product")


@pytest.mark.parametrize("ny", [1, 2, 3, 5, 8, 13, 20, 31, 40])
def test_product_fft_lengths_along_y(bt, ny):
    """The y level of both FFT forms: a product of 2 columns (both levels fused in one kernel each way) and
    of 6 columns (strided passes) on the same vectors, each against the oracle."""
    nx, b = 7, 5
    gen = arrays.random_generator_blocks(nx, ny, b, seed=600 + ny)
    plan = bt.Plan(nx, ny, b, max_rhs=6, prec_mask=ALL_PRECS)
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(ny), 6, plan.n)
    ref = oracle.matvec(gen, x.T).T
    for k in (2, 6):
        for prec, tol in ((bt.BTTB_MV_FP64, FP64_TOL), (bt.BTTB_MV_FP64_NATIVE, FP64_TOL)):
            _check(plan.matvec(_dev(x[:k]), prec=prec).cpu().numpy(), ref[:k], tol, f"prec {prec} k={k} my={plan.my}")
        _check(plan.matvec(_dev(x[:k].astype(np.complex64)), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref[:k], FP32_TOL,
               f"binary32 k={k} my={plan.my}")
    plan.close()


@pytest.mark.parametrize("nx", list(range(1, 41)))
def test_product_every_fft_length(bt, nx):
    """nx = 1..40 makes the plan pick every padded length smallest_5smooth(2 nx - 1) up to 80 (1, 3, 5, 8,
    9, 12, 15, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48, 50, 54, 60, 64, 72, 75, 80): every radix-2/3/4/5
    stage combination of the FFT passes, forward and inverse, checked through the product."""
    ny, b = 2, 3
    gen = arrays.random_generator_blocks(nx, ny, b, seed=500 + nx)
    plan = bt.Plan(nx, ny, b, max_rhs=2, prec_mask=ALL_PRECS)
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(nx), 2, plan.n)
    ref = oracle.matvec(gen, x.T).T
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, f"df64 mx={plan.mx}")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64_NATIVE).cpu().numpy(), ref, FP64_TOL, f"binary64 mx={plan.mx}")
    _check(plan.matvec(_dev(x.astype(np.complex64)), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref, FP32_TOL,
           f"binary32 mx={plan.mx}")
    plan.close()


@pytest.mark.parametrize("inner", ["tf32x3", "bf16x3"])
def test_tensor_core_ir_solve(bt, inner):
    """GMRES-IR with tensor-core inner products (3xTF32 and split-BF16x3) reaches the FP64-class residual on
    every column."""
    nx, ny, b = 8, 6, 12
    gen = arrays.generator_blocks(nx, ny, b, seed=32)
    v = arrays.port_excitations(nx, ny, b).T.copy()          # 48 columns
    pr = bt.BTTB_MV_TC_3XTF32 if inner == "tf32x3" else bt.BTTB_MV_TC_BF16X3
    plan = bt.Plan(nx, ny, b, max_rhs=v.shape[0], prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << pr))
    plan.set_generators(gen)
    sol, rc, res = plan.solve(_dev(v), tol=1e-8, restart=30, inner=pr)
    assert rc == bt.BTTB_OK, bt.bttb_last_error()
    rr = oracle.relres(gen, v.T, sol.cpu().numpy().T)
    assert np.all(rr <= 1e-8), rr.max()


def test_multi_rhs_solve_all_ports(bt):
    """Every element's port excitation (the embedded-element-pattern workload), IR per column."""
    nx, ny, b = 8, 6, 12
    gen = arrays.generator_blocks(nx, ny, b, seed=31)
    v = arrays.port_excitations(nx, ny, b).T.copy()          # 48 columns
    plan = bt.Plan(nx, ny, b, max_rhs=v.shape[0])
    plan.set_generators(gen)
    sol, rc, res = plan.solve(_dev(v), tol=1e-8, restart=30, inner=bt.BTTB_MV_FP32)
    assert rc == bt.BTTB_OK, bt.bttb_last_error()
    rr = oracle.relres(gen, v.T, sol.cpu().numpy().T)
    assert np.all(rr <= 1e-8), rr.max()
    assert all(r.status == bt.BTTB_OK for r in res)
    # each column agrees with its own single-column solve
    for col in (0, 17, 47):
        s1, _, _ = plan.solve(_dev(v[col:col + 1]), tol=1e-8, restart=30, inner=bt.BTTB_MV_FP32)
        x1 = s1.cpu().numpy()[0]
        assert np.linalg.norm(sol.cpu().numpy()[col] - x1) <= 1e-6 * np.linalg.norm(x1)


def test_product_padded_leading_dimension_and_groups(bt):
    nx, ny, b, k = 6, 4, 10, 9          # 9 columns -> three passes of the block product
    gen = arrays.random_generator_blocks(nx, ny, b, seed=7)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    n = plan.n
    ld = n + 13
    x = _rand(np.random.default_rng(3), k, ld)
    xd = _dev(x)
    yd = torch.full_like(xd, 7.0 + 7.0j)
    bt.bttb_matvec(plan.handle, xd, yd, k, ld, bt.BTTB_C128, bt.BTTB_MV_FP64)
    y = yd.cpu().numpy()
    ref = oracle.matvec(gen, x[:, :n].T).T
    _check(y[:, :n], ref, FP64_TOL, "ld-padded")
    assert np.all(y[:, n:] == 7.0 + 7.0j), "product wrote past N in a padded column"
    bt.bttb_matvec(plan.handle, xd, yd, 0, ld, bt.BTTB_C128, bt.BTTB_MV_FP64)   # empty call is a no-op


def test_largest_grid(bt):
    nx, ny, b = 1024, 2, 2                # grid side 2048, the maximum
    gen = arrays.random_generator_blocks(nx, ny, b, seed=8)
    plan = bt.Plan(nx, ny, b)
    plan.set_generators(gen)
    assert plan.mx == 2048
    x = _rand(np.random.default_rng(4), 1, plan.n)
    _check(plan.matvec(_dev(x)).cpu().numpy(), oracle.matvec(gen, x.T).T, FP64_TOL, "largest grid")


@pytest.mark.parametrize("nx,ny", [(5, 4), (3, 3), (6, 1)])
def test_bccb_eigenpairs_on_gpu(bt, nx, ny):
    gen, c = arrays.periodic_generator_blocks(nx, ny, seed=9)
    lam = np.fft.fft2(c)
    ix = np.tile(np.arange(nx), ny)
    iy = np.repeat(np.arange(ny), nx)
    modes = np.stack([np.exp(2j * np.pi * (kx * ix / nx + ky * iy / ny)) for ky in range(ny) for kx in range(nx)])
    lam_row = np.array([lam[kx, ky] for ky in range(ny) for kx in range(nx)])
    plan = bt.Plan(nx, ny, 1, max_rhs=nx * ny)
    plan.set_generators(gen)
    y = plan.matvec(_dev(modes)).cpu().numpy()
    assert np.abs(y - lam_row[:, None] * modes).max() <= 1e-12 * np.abs(lam).max()


def test_spectrum_matches_oracle(bt):
    nx, ny, b = 5, 3, 4
    gen = arrays.random_generator_blocks(nx, ny, b, seed=11)
    plan = bt.Plan(nx, ny, b, prec_mask=ALL_PRECS)
    plan.set_generators(gen)
    ref = oracle.spectrum(gen, plan.mx, plan.my) / (plan.mx * plan.my)
    for ky in range(plan.my):
        for kx in range(plan.mx):
            got = plan.spectrum_bin(ky, kx)
            assert np.abs(got - ref[ky, kx]).max() <= 1e-13 * np.abs(ref).max()
    plan_df = bt.Plan(nx, ny, b)
    plan_df.set_generators(gen)
    got = plan_df.spectrum_bin(1, 2)
    assert np.abs(got - ref[1, 2]).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("route", [1, 2, 3, 4])
@pytest.mark.parametrize("nx,ny,b,k", [
    (5, 4, 12, 1),     # grid 9 x 8: clusters of 8, two bases per CTA
    (6, 5, 16, 2),     # two columns
    (7, 3, 33, 3),     # odd b: even chunk widths, ragged last chunk; three columns
    (4, 6, 60, 4),     # four columns, b = 60
    (9, 8, 96, 1),     # three rows per lane in the block product
    (3, 2, 5, 1),      # b < Q: CTAs without bases
    (12, 2, 24, 2),    # grid 24 x 3: more bins than CTAs of a column
])
def test_product_routes(bt, route, nx, ny, b, k):
    """The four forms of a one-to-four-column product (four strided passes; the two-level FFT in one
    cluster kernel each way; the level-1 passes around the fused level-2 transform + block product; all of
    it as phases of one persistent kernel) give the oracle's product to the precision's tolerance; a form
    that does not fit falls back.  Every form gives the strided route's bits (the same butterflies and the
    same per-lane accumulation of the block product)."""
    gen = arrays.random_generator_blocks(nx, ny, b, seed=500 + nx + ny + b + k)
    plan = bt.Plan(nx, ny, b, max_rhs=k)
    plan.set_generators(gen)
    bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, route)
    x = _rand(np.random.default_rng(9), k, plan.n)
    ref = oracle.matvec(gen, x.T).T
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, f"df64 route {route}")
    _check(plan.matvec(_dev(x.astype(np.complex64)), prec=bt.BTTB_MV_FP32).cpu().numpy(),
           oracle.matvec(gen, x.astype(np.complex64).T).T, FP32_TOL, f"binary32 route {route}")
    _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref, FP32_TOL, f"binary32 c128 io {route}")
    if route != 1:
        ys = {}
        for r in (1, route):
            bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, r)
            ys[r] = (plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(),
                     plan.matvec(_dev(x.astype(np.complex64)), prec=bt.BTTB_MV_FP32).cpu().numpy())
        assert np.array_equal(ys[1][0], ys[route][0]) and np.array_equal(ys[1][1], ys[route][1])
    plan.close()


# split-BF16x3: each binary32 factor is h + l with h = bf16(x), l = bf16(x - h) (round to nearest), and the
# product drops l*l' and the remainders x - h - l (each at most 2^-18 |x|): at most 3 * 2^-18 = 1.1e-5
# relative per product term, and a sum of such terms with independent rounding has a norm-wise relative
# error of about 2^-18 * sqrt(3) = 6.6e-6 -- inside the 1e-5 bar of the tensor-core products.
BF16X3_TOL = 1e-5


@pytest.mark.parametrize("nx,ny,b,k", [(5, 4, 60, 16), (6, 5, 60, 70), (4, 3, 64, 130), (7, 6, 12, 65),
                                        (4, 2, 30, 31), (6, 4, 24, 97), (4, 4, 37, 20)])
def test_tensor_core_bf16x3_product(bt, nx, ny, b, k):
    """BTTB_MV_TC_BF16X3: the per-bin GEMM on the tcgen05 tensor cores in split-BF16x3 (kind::f16, bfloat16
    operands, binary32 accumulation in tensor memory) for even b <= 64 and >= 16 columns; binary32 for odd b."""
    gen = arrays.random_generator_blocks(nx, ny, b, seed=450 + b + k)
    plan = bt.Plan(nx, ny, b, max_rhs=k, prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_TC_BF16X3))
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(18), k, plan.n)
    ref = oracle.matvec(gen, x.T).T
    y = plan.matvec(_dev(x.astype(np.complex64)), prec=bt.BTTB_MV_TC_BF16X3).cpu().numpy()
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= BF16X3_TOL, err
    assert np.abs(y - ref).max() <= 4 * BF16X3_TOL * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_tensor_core_all_ports_product_sampled(bt, prec):
    """900 columns (every element's port excitation plus random amplitudes) of the 30x30, b=60 array through
    the tensor-core per-bin GEMM: sampled columns against the oracle's O(N^2) product."""
    c = arrays.CONFIGS["precision"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    pr = bt.BTTB_MV_TC_3XTF32 if prec == "tf32x3" else bt.BTTB_MV_TC_BF16X3
    k = nx * ny
    plan = bt.Plan(nx, ny, b, max_rhs=k, prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << pr))
    plan.set_generators(gen)
    rng = np.random.default_rng(19)
    x = (rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))).astype(np.complex64)
    y = plan.matvec(_dev(x), prec=pr).cpu().numpy()
    cols = [0, 1, 449, 898, 899]
    ref = oracle.matvec(gen, x[cols].astype(np.complex128).T).T
    err = np.linalg.norm(y[cols] - ref) / np.linalg.norm(ref)
    assert err <= (FP32_TOL if prec == "tf32x3" else BF16X3_TOL), err
    plan.close()


# ------------------------------------------------------------------ full size

@pytest.fixture(scope="module")
def precision_case(bt):
    c = arrays.CONFIGS["precision"]
    gen = arrays.generator_blocks(c["nx"], c["ny"], c["b"], c["seed"])
    plan = bt.Plan(c["nx"], c["ny"], c["b"], max_rhs=1, prec_mask=ALL_PRECS)
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(5), 1, plan.n)
    ref = oracle.matvec(gen, x.T).T           # O(N^2) brute force, 2.9e9 complex MACs
    return c, gen, plan, x, ref


def test_full_size_product(bt, precision_case):
    c, gen, plan, x, ref = precision_case
    assert (plan.mx, plan.my) == (60, 60)
    e64 = _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, "df64 30x30")
    e64n = _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64_NATIVE).cpu().numpy(), ref, FP64_TOL, "binary64 30x30")
    e32 = _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref, FP32_TOL, "binary32 30x30")
    print(f"30x30 b=60 product error vs oracle: df64 {e64:.2e}, binary64 {e64n:.2e}, binary32 {e32:.2e}")


@pytest.mark.parametrize("route", [1, 2, 3, 4])
def test_full_size_product_routes(bt, precision_case, route):
    """Every form of the 30x30, b=60 product against the O(N^2) oracle, double-float and binary32."""
    c, gen, plan, x, ref = precision_case
    bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, route)
    try:
        _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref, FP64_TOL, f"df64 route {route}")
        _check(plan.matvec(_dev(x), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref, FP32_TOL, f"binary32 route {route}")
    finally:
        bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, 0)


@pytest.mark.parametrize("prec_name", ["BTTB_MV_TC_3XTF32", "BTTB_MV_TC_BF16X3"])
def test_full_size_tensor_core_product(bt, prec_name):
    """The tcgen05 per-bin GEMM at full size: the 30x30, b=60 array (3600 bins) times 128 columns (four tiles
    of 32), columns at the tile edges and in between checked on 300 sampled rows each against the oracle's
    O(N) row sums, to the tensor-core tolerance relative to the column's largest entry."""
    c = arrays.CONFIGS["precision"]
    gen = arrays.generator_blocks(c["nx"], c["ny"], c["b"], c["seed"])
    prec = getattr(bt, prec_name)
    plan = bt.Plan(c["nx"], c["ny"], c["b"], max_rhs=128, prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << prec))
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(12), 128, plan.n)
    y = plan.matvec(_dev(x.astype(np.complex64)), prec=prec).cpu().numpy()
    rows = np.unique(np.concatenate([np.arange(0, 60), plan.n - 1 - np.arange(60),
                                     np.random.default_rng(13).integers(0, plan.n, 180)]))
    for col in (0, 31, 32, 77, 127):
        ref = oracle.matvec_rows(gen, x[col].astype(np.complex64), rows)
        scale = np.abs(y[col]).max()
        assert np.abs(y[col][rows] - ref).max() <= 4 * BF16X3_TOL * scale, (prec_name, col)
    plan.close()


def test_full_size_sampled_rows(bt, precision_case):
    c, gen, plan, x, ref = precision_case
    y = plan.matvec(_dev(x)).cpu().numpy()[0]
    rows = np.unique(np.concatenate([np.arange(0, 60), plan.n - 1 - np.arange(60),
                                     np.random.default_rng(6).integers(0, plan.n, 200)]))
    sampled = oracle.matvec_rows(gen, x[0], rows)
    assert np.abs(y[rows] - sampled).max() <= FP64_TOL * np.abs(ref).max()


# ------------------------------------------------------------------ solves

def test_tiny_solve_matches_lu(bt):
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    cells = [(1, 1), (0, 0), (3, 2)]
    v = arrays.port_excitations(nx, ny, b, cells).T.copy()
    plan = bt.Plan(nx, ny, b, max_rhs=3)
    plan.set_generators(gen)
    sol, rc, res = plan.solve(_dev(v), tol=c["tol"], restart=c["restart"])
    assert rc == bt.BTTB_OK
    x = sol.cpu().numpy()
    x_lu = oracle.lu_solve(oracle.assemble(gen), v.T).T
    rr = oracle.relres(gen, v.T, x.T)
    for col in range(3):
        assert res[col].status == bt.BTTB_OK
        assert rr[col] <= c["tol"], rr
        assert abs(res[col].relres_true - rr[col]) <= 1e-3 * c["tol"] + 1e-12 * rr[col]
        assert np.linalg.norm(x[col] - x_lu[col]) <= 1e-8 * np.linalg.norm(x_lu[col])


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_precision_solve(bt, precision_case, inner):
    c, gen, plan, _, _ = precision_case
    v = arrays.centre_excitation(c["nx"], c["ny"], c["b"])[None, :]
    hist = np.zeros(64)
    prec = bt.BTTB_MV_FP64 if inner == "fp64" else bt.BTTB_MV_FP32
    sol, rc, res = plan.solve(_dev(v), tol=c["tol"], restart=c["restart"], inner=prec, history=hist)
    assert rc == bt.BTTB_OK, bt.bttb_last_error()
    rr = oracle.relres(gen, v.T, sol.cpu().numpy().T)[0]
    print(f"30x30 solve inner={inner}: {res[0].iters} iterations, {res[0].cycles} cycles, oracle relres {rr:.3e}")
    assert rr <= c["tol"]


@pytest.mark.parametrize("pc", ["none", "bj"])
def test_graph_and_host_driven_solves_agree(bt, pc):
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    v = arrays.port_excitations(nx, ny, b, [(1, 1), (2, 3)]).T.copy()
    plan = bt.Plan(nx, ny, b, max_rhs=2)
    plan.set_generators(gen)
    kw = dict(tol=1e-10, restart=7, inner=bt.BTTB_MV_FP32,
              pc=bt.BTTB_PC_BLOCK_JACOBI if pc == "bj" else bt.BTTB_PC_NONE)
    s1, rc1, r1 = plan.solve(_dev(v), **kw)
    s2, rc2, r2 = plan.solve(_dev(v), flags=bt.BTTB_GMRES_NO_GRAPH, **kw)
    bt.bttb_profile(plan.handle, True)                   # graph rebuilt with timing nodes
    s3, rc3, r3 = plan.solve(_dev(v), **kw)
    st = bt.bttb_profile_read(plan.handle, bt.BTTB_K_BLOCK_PRODUCT)
    bt.bttb_profile(plan.handle, False)
    assert rc3 == bt.BTTB_OK and torch.equal(s1, s3)
    assert st.launches > 0 and st.ms > 0 and st.bytes > 0
    assert rc1 == rc2 == bt.BTTB_OK
    assert [x.iters for x in r1] == [x.iters for x in r2]
    assert torch.equal(s1, s2)
    rr = oracle.relres(gen, v.T, s1.cpu().numpy().T)
    assert np.all(rr <= 1e-10)


def test_block_jacobi_apply_matches_oracle(bt):
    nx, ny, b = 4, 3, 12
    gen = arrays.generator_blocks(nx, ny, b, seed=12)
    plan = bt.Plan(nx, ny, b, max_rhs=2)
    plan.set_generators(gen)
    x = _rand(np.random.default_rng(13), 2, plan.n)
    z = plan.block_jacobi(_dev(x)).cpu().numpy()
    _check(z, oracle.block_jacobi_apply(gen, x.T).T, FP32_TOL, "block-Jacobi")


def test_block_jacobi_solve(bt):
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    v = arrays.port_excitations(nx, ny, b, [(1, 1)]).T.copy()
    plan = bt.Plan(nx, ny, b)
    plan.set_generators(gen)
    _, _, res0 = plan.solve(_dev(v), tol=c["tol"])
    sol, rc, res = plan.solve(_dev(v), tol=c["tol"], pc=bt.BTTB_PC_BLOCK_JACOBI)
    assert rc == bt.BTTB_OK
    assert oracle.relres(gen, v.T, sol.cpu().numpy().T)[0] <= c["tol"]
    assert res[0].iters <= res0[0].iters


def test_host_io_and_initial_guess(bt):
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    v = arrays.port_excitations(nx, ny, b, [(2, 1)]).T.copy()
    plan = bt.Plan(nx, ny, b)
    plan.set_generators(gen)
    vh = torch.from_numpy(v)
    ih = torch.zeros_like(vh)
    _, rc, res = plan.solve(vh, ih, tol=1e-10, host_io=True)
    assert rc == bt.BTTB_OK
    assert oracle.relres(gen, v.T, ih.numpy().T)[0] <= 1e-10
    x_lu = torch.from_numpy(oracle.lu_solve(oracle.assemble(gen), v.T).T.copy()).cuda()
    _, rc, res = plan.solve(_dev(v), x_lu.clone(), tol=1e-10, use_x0=True)
    assert rc == bt.BTTB_OK and res[0].iters == 0


# ------------------------------------------------------------------ failure paths (host-side)

def test_not_converged_status(bt):
    c = arrays.CONFIGS["tiny"]
    gen = arrays.generator_blocks(c["nx"], c["ny"], c["b"], c["seed"])
    v = arrays.port_excitations(c["nx"], c["ny"], c["b"], [(1, 1)]).T.copy()
    plan = bt.Plan(c["nx"], c["ny"], c["b"])
    plan.set_generators(gen)
    sol, rc, res = plan.solve(_dev(v), tol=1e-12, max_iters=3, restart=50)
    assert rc == bt.BTTB_NOT_CONVERGED and res[0].status == bt.BTTB_NOT_CONVERGED
    assert res[0].iters == 3
    rr = oracle.relres(gen, v.T, sol.cpu().numpy().T)[0]
    assert abs(res[0].relres_true - rr) <= 1e-9


def test_error_codes(bt):
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    plan = bt.Plan(nx, ny, b, max_rhs=1)
    x = _dev(np.ones((1, plan.n), dtype=np.complex128))
    with pytest.raises(bt.BttbError) as e:
        plan.matvec(x)
    assert e.value.code == bt.BTTB_ERR_NO_GENERATORS
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    bad = gen.copy()
    bad[2, 3, 1, 1] = np.nan
    with pytest.raises(bt.BttbError) as e:
        plan.set_generators(bad)
    assert e.value.code == bt.BTTB_ERR_NONFINITE
    plan.set_generators(gen)
    with pytest.raises(bt.BttbError) as e:
        bt.bttb_matvec(plan.handle, x, x.clone(), 2, plan.n, bt.BTTB_C128, bt.BTTB_MV_FP64)
    assert e.value.code == bt.BTTB_ERR_INVALID_ARG
    with pytest.raises(bt.BttbError) as e:
        bt.bttb_matvec(plan.handle, x, x.clone(), 1, plan.n, bt.BTTB_C128, bt.BTTB_MV_FP64_NATIVE)
    assert e.value.code == bt.BTTB_ERR_INVALID_ARG           # copy not kept by this plan
    zero_self = gen.copy()
    zero_self[ny - 1, nx - 1] = 0.0
    plan.set_generators(zero_self)
    with pytest.raises(bt.BttbError) as e:
        plan.solve(x, pc=bt.BTTB_PC_BLOCK_JACOBI)
    assert e.value.code == bt.BTTB_ERR_SINGULAR
