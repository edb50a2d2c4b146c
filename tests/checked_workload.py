"""Workload for the bounds-checked build (run in a child process by test_gpu_checked.py with
BTTB_LIB_CHECKED=1): products in every form and precision, the many-column GEMMs, the solver variants,
the block-Jacobi apply and the allocation-free product, each checked against the oracle; then it prints
the failed-check count of the whole run as one JSON line."""
import ctypes
import json
import sys

import numpy as np
import torch

import oracle
import paper_2506_20350_gb300 as bt
from workloads import arrays

FP64_TOL, FP32_TOL = 1e-12, 1e-5


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


def main():
    assert bt.bttb_check_report()[0], "not the bounds-checked library"
    out = {"probe_hits": bt.bttb_check_probe()}
    _, h0, _ = bt.bttb_check_report()
    errs = {}
    rng = np.random.default_rng(3)
    all_prec = (1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_FP32) | (1 << bt.BTTB_MV_FP64_NATIVE)
    # one-to-four-column products in every form, odd and even b, ragged grids
    for nx, ny, b, k in [(5, 4, 12, 1), (7, 3, 33, 3), (4, 6, 60, 2), (9, 8, 96, 1), (3, 2, 5, 1)]:
        gen = arrays.random_generator_blocks(nx, ny, b, seed=nx + ny + b)
        plan = bt.Plan(nx, ny, b, max_rhs=k, prec_mask=all_prec)
        plan.set_generators(gen)
        x = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
        ref = oracle.matvec(gen, x.T).T
        for route in (1, 2, 3, 4):
            bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, route)
            errs[f"df64 {nx}x{ny} b{b} k{k} r{route}"] = (rel(plan.matvec(dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref), FP64_TOL)
            errs[f"f32 {nx}x{ny} b{b} k{k} r{route}"] = (rel(plan.matvec(dev(x), prec=bt.BTTB_MV_FP32).cpu().numpy(), ref), FP32_TOL)
        errs[f"f64n {nx}x{ny} b{b} k{k}"] = (rel(plan.matvec(dev(x), prec=bt.BTTB_MV_FP64_NATIVE).cpu().numpy(), ref), FP64_TOL)
        plan.close()
    # many columns: the binary32 GEMM and the tensor-core GEMMs (tcgen05 for even b <= 64)
    for nx, ny, b, k in [(4, 3, 12, 20), (3, 3, 33, 70), (4, 4, 60, 40)]:
        gen = arrays.random_generator_blocks(nx, ny, b, seed=40 + b + k)
        mask = (1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_FP32) | (1 << bt.BTTB_MV_TC_3XTF32) | (1 << bt.BTTB_MV_TC_BF16X3)
        plan = bt.Plan(nx, ny, b, max_rhs=k, prec_mask=mask)
        plan.set_generators(gen)
        x = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
        ref = oracle.matvec(gen, x.T).T
        x32 = dev(x.astype(np.complex64))
        for prec, name in ((bt.BTTB_MV_FP32, "f32"), (bt.BTTB_MV_TC_3XTF32, "tf32x3"), (bt.BTTB_MV_TC_BF16X3, "bf16x3")):
            errs[f"{name} {nx}x{ny} b{b} k{k}"] = (rel(plan.matvec(x32, prec=prec).cpu().numpy(), ref), FP32_TOL)
        errs[f"df64 multi {nx}x{ny} b{b} k{k}"] = (rel(plan.matvec(dev(x), prec=bt.BTTB_MV_FP64).cpu().numpy(), ref), FP64_TOL)
        plan.close()
    # solves: delayed CGS2 (few and many columns), two-pass CGS2, IR, block-Jacobi, global GMRES
    c = arrays.CONFIGS["tiny"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    for k, kw in [(1, {}), (3, {"inner": bt.BTTB_MV_FP32}), (2, {"flags": bt.BTTB_GMRES_CGS2}),
                  (2, {"pc": bt.BTTB_PC_BLOCK_JACOBI}), (12, {"inner": bt.BTTB_MV_FP32}),
                  (3, {"flags": bt.BTTB_GMRES_GLOBAL})]:
        plan = bt.Plan(nx, ny, b, max_rhs=k)
        plan.set_generators(gen)
        V = rng.standard_normal((k, plan.n)) + 1j * rng.standard_normal((k, plan.n))
        I, rc, res = plan.solve(dev(V), tol=1e-10, restart=20, **kw)
        Ih = I.cpu().numpy()
        if kw.get("flags") == bt.BTTB_GMRES_GLOBAL:    # global GMRES: the block residual, Frobenius norm
            r = np.linalg.norm(V - oracle.matvec(gen, Ih.T).T) / np.linalg.norm(V)
        else:
            r = float(np.max(oracle.relres(gen, V.T, Ih.T)))
        errs[f"solve k{k} {kw}"] = (float(r), 1e-10 if rc == bt.BTTB_OK else -1.0)
        if kw.get("pc") == bt.BTTB_PC_BLOCK_JACOBI:
            z = torch.empty_like(dev(V))
            bt.bttb_block_jacobi_apply(plan.handle, dev(V), z, k, plan.n, bt.BTTB_C128)
            torch.cuda.synchronize()
        plan.close()
    # the allocation-free product
    x = rng.standard_normal((1, nx * ny * b)) + 1j * rng.standard_normal((1, nx * ny * b))
    y = torch.zeros((1, nx * ny * b), dtype=torch.complex128, device="cuda")
    gd, xd = dev(gen), dev(x)
    stream = torch.cuda.current_stream().cuda_stream
    rc = bt.load_library().bttb_matvec_noalloc(nx, ny, b, gd.data_ptr(), xd.data_ptr(), y.data_ptr(), 1, nx * ny * b,
                                               ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    errs["noalloc"] = (rel(y.cpu().numpy(), oracle.matvec(gen, x.T).T), FP64_TOL if rc == 0 else -1.0)
    _, h1, first = bt.bttb_check_report()
    out["hits"] = h1 - h0
    out["first"] = first
    out["bad"] = {k: v for k, v in errs.items() if not (v[1] > 0 and v[0] <= v[1])}
    out["cases"] = len(errs)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
