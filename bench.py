#!/usr/bin/env python
"""Benchmark of the MLFFT block-Toeplitz product inside GMRES on GB300.

Workload (the 30 x 30 array, b = 60, N = 54,000 unknowns, synthetic Green's
function generators with centroid seed 1, mx = my = 60): one step is one
GMRES(50)-IR solve of the centre-element delta-gap excitation to a true
relative residual of 1e-8 -- binary32 products inside each restart cycle,
double-float (FP64-class) residual, Arnoldi and updates.

Reported:
  value        FFT-product throughput inside the solve: algorithmic bytes of
               every product the step ran (spectrum planes read once + x in +
               y out per product) / measured step time, summed over ranks.
  roofline     the dominant kernel (the binary32 block product), measured live
               with CUDA events on the plan's stream over the timed steps.
  gmres        plain FP64 (double-float) GMRES time to 1e-8 vs the IR step.
  e2e          the same step through the C ABI with host buffers (H2D of V,
               D2H of I inside the timed region).
  cpu_baseline the CPU oracle's O(N^2) product timed on the host cores.
  multi_rhs    all 900 port excitations of the same array in one batched solve.
  uneven_batch 64 independent arrays of uneven size solved concurrently.
  learned_preconditioner
               the 40 x 40, b = 96 array: training of the learned correction
               on 2000 plain-solver pairs, then 50 held-out excitations with
               plain GMRES, block-Jacobi FGMRES and learned FGMRES.
  (BTTB_BENCH_SKIP_MULTI / _UNEVEN / _LEARNED leave a leg out.)

``--impl reference`` times the CPU oracle as it stands on this workload:
each step is one brute-force product (a bounded sample of the solve).
Multi-GPU (torchrun): every rank solves its own replica; no collective is on
the data path (weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BTTB FFT-matvec GB/s (% HBM peak); GMRES time to 1e-8 rel. residual vs FP64"
WORKLOAD = "30x30 array, b=60, N=54000, centre-element delta gap, GMRES(50)-IR to 1e-8"
FALLBACK_HBM = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # the autotuner times the product forms; under a profiler that serialises launches its choice differs
    # from the unprofiled one, so a profiling run can pin the form it wants to see (1..4, as
    # BTTB_DEBUG_PRODUCT_ROUTE; 0: the tuned choice)
    ap.add_argument("--product-form", type=int, choices=[0, 1, 2, 3, 4], default=0)
    return ap.parse_args()


def dist_setup(use_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(x: float, world: int, op: str = "max") -> float:
    """MAX or SUM of a per-rank scalar over all ranks (a CUDA tensor under NCCL, a CPU one under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    return reduce_over_ranks(x, world, "max")


def job_rate(units: float, seconds: float, world: int) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return reduce_over_ranks(units, world, "sum") / reduce_over_ranks(seconds, world, "max")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def product_bytes(nx, ny, b, mx, my, prec):
    """Algorithmic bytes of one FFT product: spectrum planes once, x in, y out."""
    bins, n = mx * my, nx * ny * b
    if prec == "fp32":
        return bins * b * b * 8 + 2 * n * 8
    return bins * b * b * 16 + 2 * n * 16         # double-float planes or binary64 copy


def kernel_digest(src_name: str) -> str | None:
    """Digest of the code lines (comments excluded) of the kernel an ncu capture in profiles/ measured:
    the block-product kernel template and its launch configuration (contract.cu), or the whole fused
    level-2 kernel file (ycontract.cu).  Comment edits keep a capture valid; code edits void it."""
    src = os.path.join(ROOT, "paper_2506_20350_gb300", "csrc", src_name)
    text = open(src).read()
    if src_name == "contract.cu":
        try:
            a = text.index("// KC: right-hand sides per launch")
            b = text.index("template <class A>\nconstexpr int prec_of()")
            c = text.index("static int launch_contract_impl(")
            d = text.index("\n}\n", c)
        except ValueError:
            return None
        text = text[a:b] + "\n" + text[c:d]
    code = [ln for ln in text.splitlines() if not ln.strip().startswith("//")]
    return hashlib.sha1("\n".join(code).encode()).hexdigest()[:12]


def traffic_from_profiles(kernel_key: str, src_name: str):
    """ncu DRAM bytes per launch recorded in profiles/, if the kernel source is unchanged."""
    digest = kernel_digest(src_name)
    path = os.path.join(ROOT, "profiles", "contract_traffic.txt")
    if digest is None or not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel_key and f[2] == digest:
            return float(f[1])
    return None


def cpu_oracle_product_time(gen, n, budget_s=12.0):
    import oracle
    x = (np.random.default_rng(0).standard_normal(n) + 1j * np.random.default_rng(1).standard_normal(n))
    oracle.matvec(gen, x)                 # warm (loads and builds the C oracle)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.matvec(gen, x)
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return (time.perf_counter() - t0) / reps, reps


class HostMlfft:
    """The paper's multilevel-FFT product restated on the host cores (Sec. II-C, III-A, App. B), the second
    CPU baseline: the spectrum of the wrapped first block column once (Eq. (circL2)), then per product the
    zero padding of Eq. (xc2), the 2-level DFT (level 1 along the cells of a row, then level 2 along the
    rows, App. B), the per-bin b x b block product of Eq. (multL), the inverse and the crop.  scipy.fft
    with workers = the host's cores; numpy's batched matmul for the per-bin product; complex128."""

    def __init__(self, gen, nx, ny, b, mx, my, workers):
        import scipy.fft as sfft
        self.fft, self.nx, self.ny, self.b, self.mx, self.my, self.w = sfft, nx, ny, b, mx, my, workers
        c1 = np.zeros((my, mx, b, b), dtype=np.complex128)
        for j in range(-(ny - 1), ny):
            for i in range(-(nx - 1), nx):
                c1[j % my, i % mx] = gen[j + ny - 1, i + nx - 1]
        g = sfft.fft(c1, axis=1, workers=workers)
        g = sfft.fft(g, axis=0, workers=workers) / (mx * my)
        self.G = np.ascontiguousarray(g.reshape(my * mx, b, b))          # bin-major b x b blocks

    def matvec(self, x):
        """y = Z x for x of shape (N,) or (N, k)."""
        nx, ny, b, mx, my, w = self.nx, self.ny, self.b, self.mx, self.my, self.w
        k = 1 if x.ndim == 1 else x.shape[1]
        u = np.zeros((my, mx, b, k), dtype=np.complex128)
        u[:ny, :nx] = x.reshape(ny, nx, b, k)
        u = self.fft.fft(u[:ny], n=mx, axis=1, workers=w)                 # level 1 on the ny nonzero rows
        u = self.fft.fft(u, n=my, axis=0, workers=w)                      # level 2 (rows ny.. are zero)
        v = np.matmul(self.G, u.reshape(my * mx, b, k)).reshape(my, mx, b, k)
        v = self.fft.ifft(v, axis=0, workers=w)[:ny] * my
        v = self.fft.ifft(v, axis=1, workers=w)[:, :nx] * mx
        return v.reshape(-1) if x.ndim == 1 else v.reshape(-1, k)


def host_mlfft_baseline(gen, nx, ny, b, mx, my, gmres_iters, cores, budget_s=10.0):
    """Time the host MLFFT product on this workload (bounded sample) and a CPU GMRES(50) of the 4x4, b=12
    array to 1e-10 with it; the 30x30 solve time is the per-product time times the products a solve needs."""
    import oracle
    from workloads import arrays
    t0 = time.perf_counter()
    hm = HostMlfft(gen, nx, ny, b, mx, my, cores)
    setup_s = time.perf_counter() - t0
    n = nx * ny * b
    x = np.random.default_rng(0).standard_normal(n) + 1j * np.random.default_rng(1).standard_normal(n)
    y = hm.matvec(x)
    rows = np.random.default_rng(2).choice(n, size=8, replace=False)
    ref = oracle.matvec_rows(gen, x, rows)
    err = float(np.abs(y[rows] - ref).max() / np.abs(ref).max())
    t0, reps = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s or reps < 2:
        hm.matvec(x)
        reps += 1
    per = (time.perf_counter() - t0) / reps
    c = arrays.CONFIGS["tiny"]
    gt = arrays.generator_blocks(c["nx"], c["ny"], c["b"], c["seed"])
    ht = HostMlfft(gt, c["nx"], c["ny"], c["b"], 8, 8, cores)
    vt = arrays.port_excitations(c["nx"], c["ny"], c["b"], [(1, 1)])[:, 0]
    t0 = time.perf_counter()
    xt, info = oracle.gmres(ht.matvec, vt, tol=c["tol"], restart=50, max_iters=5000)
    tiny_s = time.perf_counter() - t0
    tiny_rel = float(oracle.relres(gt, vt, xt)[0])
    return {"kind": "paper_method_host", "cores": cores, "setup_s": setup_s, "product_ms": per * 1e3,
            "product_gbs": product_bytes(nx, ny, b, mx, my, "fp64") / per / 1e9, "reps": reps,
            "sampled_rows_rel_err_vs_oracle": err,
            "solve_30x30_fp64_s_estimate": per * gmres_iters,
            "solve_estimate_basis": f"{gmres_iters} products (the FP64 GMRES iterations and residuals on the GPU)",
            "tiny_4x4_b12_gmres_s": tiny_s, "tiny_iters": int(info["iters"]), "tiny_relres_oracle": tiny_rel,
            "sample": f"{reps} host MLFFT products of the 30x30 b=60 array (scipy.fft, workers={cores}, "
                      "numpy batched matmul per bin)"}


def oracle_relres_sampled(gen, V, I, cols):
    """Relative residuals of the sampled columns, with the oracle's O(N^2) product (binary64)."""
    import oracle
    v = np.ascontiguousarray(V[:, cols])
    i = np.ascontiguousarray(I[:, cols])
    return [float(r) for r in oracle.relres(gen, v, i)]


def run_reference(args):
    rank, world, _ = dist_setup(False)
    if rank != 0:
        return
    from workloads import arrays
    c = arrays.CONFIGS["precision"]
    nx, ny, b = c["nx"], c["ny"], c["b"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    import oracle
    n = nx * ny * b
    x = np.random.default_rng(0).standard_normal(n) + 0j
    for _ in range(args.warmup):
        oracle.matvec(gen, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.matvec(gen, x)
    dt = (time.perf_counter() - t0) / args.steps
    mx = my = 60
    val = product_bytes(nx, ny, b, mx, my, "fp64") / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "one O(N^2) brute-force FP64 product of the 30x30 b=60 matrix per step (2.9e9 complex MACs)"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: one product per step)", "nx": nx, "ny": ny, "b": b},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def learned_leg(dev, stream):
    """The learned Fourier-domain preconditioner on the 40x40, b=96 array: 2000
    (residual, exact correction) pairs from 500 seeded random port excitations
    (plain-solver iterates after 0, 10, 40 and 80 steps; exact solutions to
    1e-10), GPU training, then 50 held-out excitations solved to 1e-8 by plain
    GMRES, block-Jacobi FGMRES and learned FGMRES."""
    import torch

    import paper_2506_20350_gb300 as bt
    from workloads import arrays

    c = arrays.CONFIGS["learned"]
    nx, ny, b, tol = c["nx"], c["ny"], c["b"], c["tol"]
    ntr_rhs, snaps, chunk = c["ntrain"] // 4, (0, 10, 40, 80), 50
    t_all = time.perf_counter()
    plan = bt.Plan(nx, ny, b, max_rhs=64, prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_FP32), stream=stream)
    g = arrays.generator_blocks_torch(nx, ny, b, c["seed"], device=dev)
    plan.set_generators(g)
    gen_host = g.cpu().numpy()                # for the oracle's residual checks of sampled columns
    del g
    n = plan.n
    t0 = time.perf_counter()
    rs, es = [], []
    with torch.cuda.stream(stream):
        vtr = arrays.random_port_excitations(nx, ny, b, ntr_rhs, seed=c["seed"])
        for c0 in range(0, ntr_rhs, chunk):
            V = torch.from_numpy(vtr[:, c0:c0 + chunk].T.copy()).to(dev)
            xs, rc, _ = plan.solve(V, tol=1e-10, restart=50, max_iters=4000, pc=bt.BTTB_PC_BLOCK_JACOBI,
                                   inner=bt.BTTB_MV_FP32)
            for j in snaps:
                xj = torch.zeros_like(V) if j == 0 else plan.solve(V, tol=1e-14, restart=50, max_iters=j)[0]
                r = V - plan.matvec(xj)
                nr = torch.linalg.vector_norm(r, dim=1, keepdim=True)
                rs.append((r / nr).to(torch.complex64))
                es.append(((xs - xj) / nr).to(torch.complex64))
        rtr, etr = torch.cat(rs).contiguous(), torch.cat(es).contiguous()
        del rs, es, vtr
    torch.cuda.synchronize()
    pairs_s = time.perf_counter() - t0
    npairs = rtr.shape[0]
    lrn = bt.Learned(plan, rank=16, channels=64, max_cols=64, seed=c["seed"])
    plan.autotune(c["ntest"], 3)              # FFT chunk width for the 50-column products and applications
    Vte = torch.from_numpy(arrays.random_port_excitations(nx, ny, b, c["ntest"], seed=c["test_seed"]).T.copy()).to(dev)
    steps, batch, lr = 1500, 64, 1e-3
    gen_t = torch.Generator().manual_seed(c["seed"])
    with torch.cuda.stream(stream):
        loss0 = lrn.gradients(rtr[:64], etr[:64])[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s_ in range(steps):
            idx = torch.randperm(npairs, generator=gen_t)[:batch].to(dev)
            lrn.train_step(rtr[idx].contiguous(), etr[idx].contiguous(), lr=lr, want_loss=False)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        loss1 = lrn.gradients(rtr[:64], etr[:64])[0]
        # held-out loss on the test excitations' first residuals (r = V, exact correction Z^-1 V)
        xs_te, _, _ = plan.solve(Vte, tol=1e-10, restart=50, max_iters=4000, pc=bt.BTTB_PC_BLOCK_JACOBI,
                                 inner=bt.BTTB_MV_FP32)
        nr = torch.linalg.vector_norm(Vte, dim=1, keepdim=True)
        rte = (Vte / nr).to(torch.complex64).contiguous()
        ete = (xs_te / nr).to(torch.complex64).contiguous()
        lrn2 = lrn.gradients(rte, ete)[0]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lrn.apply(rte)
        ev0.record(stream)
        for _ in range(10):
            lrn.apply(rte)
        ev1.record(stream)
    torch.cuda.synchronize()
    apply_ms = ev0.elapsed_time(ev1) / 10
    del rtr, etr
    lrn.attach()
    res = {}
    for name, pc, inner in (("plain_fp64", bt.BTTB_PC_NONE, bt.BTTB_MV_FP64),
                            ("plain_ir", bt.BTTB_PC_NONE, bt.BTTB_MV_FP32),
                            ("block_jacobi_fp64", bt.BTTB_PC_BLOCK_JACOBI, bt.BTTB_MV_FP64),
                            ("block_jacobi_ir", bt.BTTB_PC_BLOCK_JACOBI, bt.BTTB_MV_FP32),
                            ("learned_fp64", bt.BTTB_PC_LEARNED, bt.BTTB_MV_FP64),
                            ("learned_ir", bt.BTTB_PC_LEARNED, bt.BTTB_MV_FP32)):
        with torch.cuda.stream(stream):
            plan.solve(Vte, tol=tol, restart=50, max_iters=2, pc=pc, inner=inner)     # graph + buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            Isol, rc, rr = plan.solve(Vte, tol=tol, restart=50, max_iters=5000, pc=pc, inner=inner)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = [x.iters for x in rr]
        res[name] = {"solve_ms": dt * 1e3, "status_ok": sum(x.status == bt.BTTB_OK for x in rr),
                     "iters_mean": float(np.mean(its)), "iters_max": max(its),
                     "relres_true_max": max(x.relres_true for x in rr)}
        if name in ("learned_ir", "block_jacobi_ir"):
            samp = [0, c["ntest"] // 2, c["ntest"] - 1]
            res[name]["oracle_relres_max_sampled"] = max(oracle_relres_sampled(
                gen_host, Vte.cpu().numpy().T, Isol.cpu().numpy().T, samp))
    base = res["plain_fp64"]["solve_ms"]
    for v in res.values():
        v["speedup_vs_plain_fp64"] = base / v["solve_ms"]
    # what the network must save to pay back its pairs and training: solves of 50 excitations until the
    # learned IR solve's saving over block-Jacobi IR covers them
    saved_ms = res["block_jacobi_ir"]["solve_ms"] - res["learned_ir"]["solve_ms"]
    bt.bttb_plan_set_learned(plan.handle, None)
    out = {"workload": f"{nx}x{ny} b={b}, N={n}, grid {plan.mx}x{plan.my}; {c['ntest']} held-out random "
                       f"port excitations (seed {c['test_seed']}) to {tol:g}",
           "network": "per-bin rank-16 complex encode/decode + 3 circular 3x3 convs (32->64->64->32 ch), "
                      "bf16 weights, fp32 accumulate",
           "params": lrn.count, "training_pairs": npairs, "pairs_s": pairs_s,
           "train_steps": steps, "batch": batch, "lr": lr, "train_s": train_s,
           "train_ms_per_step": train_s * 1e3 / steps, "loss_train_before": loss0, "loss_train_after": loss1,
           "loss_heldout_first_residual": lrn2, "apply_ms_50_columns": apply_ms,
           "amortised_s": pairs_s + train_s, "saved_ms_per_solve_vs_block_jacobi_ir": saved_ms,
           "break_even_solves": (pairs_s + train_s) * 1e3 / saved_ms if saved_ms > 0 else None,
           "solves": res, "leg_s": time.perf_counter() - t_all}
    lrn.close()
    plan.close()
    return out


def run_ours(args):
    import torch

    import paper_2506_20350_gb300 as bt
    from workloads import arrays

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    rank, world, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = arrays.CONFIGS["precision"]
    nx, ny, b, tol, restart = c["nx"], c["ny"], c["b"], c["tol"], c["restart"]
    gen = arrays.generator_blocks(nx, ny, b, c["seed"])
    stream = torch.cuda.Stream(device=dev)
    all_prec = (1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_FP32) | (1 << bt.BTTB_MV_FP64_NATIVE)
    plan = bt.Plan(nx, ny, b, max_rhs=1, prec_mask=all_prec, stream=stream)
    plan.set_generators(gen)
    fft_width = plan.autotune(1, 30)          # product form and FFT batch-chunk width for one-column products
    if args.product_form:
        bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, args.product_form)
    n, mx, my = plan.n, plan.mx, plan.my
    v_host = arrays.centre_excitation(nx, ny, b)[None, :].copy()
    V = torch.from_numpy(v_host).to(dev)
    I = torch.zeros_like(V)
    b64 = product_bytes(nx, ny, b, mx, my, "fp64")
    b32 = product_bytes(nx, ny, b, mx, my, "fp32")
    torch.cuda.synchronize()          # inputs were built on the default stream; the plan runs on its own

    def solve(inner=bt.BTTB_MV_FP32, pc=bt.BTTB_PC_NONE, Vt=V, It=I, host_io=False, flags=0):
        with torch.cuda.stream(stream):
            if not host_io:
                It.zero_()
            _, rc, res = plan.solve(Vt, It, tol=tol, restart=restart, inner=inner, pc=pc, host_io=host_io,
                                    flags=flags)
        if rc != bt.BTTB_OK:
            raise RuntimeError(f"solve failed rc={rc}: {bt.bttb_last_error()}")
        return res[0]

    def step_bytes(r, inner):
        inner_b = b32 if inner == bt.BTTB_MV_FP32 else b64
        return r.iters * inner_b + (r.cycles + 1) * b64

    for _ in range(args.warmup):
        solve()
    # ---------------- timed region (no per-kernel events: they would split the graphs' PDL chains)
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total_bytes, iters, cycles, relres = 0.0, [], [], []
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("ir_step")
        r = solve()
        torch.cuda.nvtx.range_pop()
        total_bytes += step_bytes(r, bt.BTTB_MV_FP32)
        iters.append(r.iters)
        cycles.append(r.cycles)
        relres.append(r.relres_true)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world)
    # ---------------- the same K steps again with CUDA events around every block product (roofline)
    bt.bttb_profile(plan.handle, True)
    torch.cuda.synchronize()
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        solve()
    ev3.record(stream)
    torch.cuda.synchronize()
    ms_prof = ev2.elapsed_time(ev3)
    bt.bttb_profile(plan.handle, False)
    st32 = bt.bttb_profile_read(plan.handle, bt.BTTB_K_BLOCK_PRODUCT_PREC + bt.BTTB_MV_FP32)
    st64 = bt.bttb_profile_read(plan.handle, bt.BTTB_K_BLOCK_PRODUCT_PREC + bt.BTTB_MV_FP64)
    stfft = bt.bttb_profile_read(plan.handle, bt.BTTB_K_FFT)
    stall = bt.bttb_profile_read(plan.handle, bt.BTTB_K_ALL)
    # with the plan's tuned forms, before the form sweep below
    # per-kernel breakdown of one host-driven IR solve (CUDA events around every launch)
    bt.bttb_profile(plan.handle, True)
    solve(flags=bt.BTTB_GMRES_NO_GRAPH)
    kids = {"fft_passes": bt.BTTB_K_FFT, "gs_dots": 3, "gs_update": 4, "norm_givens": 5, "normalise_advance": 6,
            "block_product_fp32": bt.BTTB_K_BLOCK_PRODUCT_PREC + bt.BTTB_MV_FP32,
            "block_product_doublefloat": bt.BTTB_K_BLOCK_PRODUCT_PREC + bt.BTTB_MV_FP64}
    breakdown, hd = {}, {}
    for name, kid in kids.items():
        st = hd[name] = bt.bttb_profile_read(plan.handle, kid)
        breakdown[name] = {"launches": st.launches, "avg_us": st.ms * 1e3 / max(st.launches, 1),
                           "total_ms": st.ms}
    bt.bttb_profile(plan.handle, False)
    value = job_rate(total_bytes, ms / 1e3, world) / 1e9
    ms_step = ms_max / args.steps

    # end to end through the C ABI with host buffers (every rank; whole-job rate as for the value)
    vh = torch.from_numpy(v_host).pin_memory()
    ih = torch.zeros_like(vh).pin_memory()
    solve(Vt=vh, It=ih, host_io=True)
    e2e_bytes = 0.0
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = solve(Vt=vh, It=ih, host_io=True)
        e2e_bytes += step_bytes(r, bt.BTTB_MV_FP32)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = job_rate(e2e_bytes, e2e_s, world) / 1e9
    e2e_s = max_over_ranks(e2e_s, world)

    if rank != 0:
        barrier(world)
        return
    # ---------------- comparison arms (rank 0, untimed for the headline)
    def timed(fn, reps):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            out.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(out))

    fp64_res = solve(inner=bt.BTTB_MV_FP64)
    fp64_ms = timed(lambda: solve(inner=bt.BTTB_MV_FP64), 5)
    # GMRES whose products are IEEE binary64 (DFMA) end to end; Arnoldi, residuals and updates double-float
    f64n_res = solve(inner=bt.BTTB_MV_FP64_NATIVE)
    f64n_ms = timed(lambda: solve(inner=bt.BTTB_MV_FP64_NATIVE), 5)
    ir_ms = timed(lambda: solve(inner=bt.BTTB_MV_FP32), 5)
    ir_oracle = oracle_relres_sampled(gen, v_host.T, I.cpu().numpy().T, [0])[0]     # I: the last IR solution
    bj_res = solve(inner=bt.BTTB_MV_FP32, pc=bt.BTTB_PC_BLOCK_JACOBI)
    bj_ms = timed(lambda: solve(inner=bt.BTTB_MV_FP32, pc=bt.BTTB_PC_BLOCK_JACOBI), 5)

    x = torch.randn(1, n, dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    x32 = x.to(torch.complex64)
    y32 = torch.empty_like(x32)
    mv = {}
    route_names = {1: "strided_passes", 2: "fused_fft2", 3: "fused_y", 4: "persistent"}
    for name, prec, xx, yy, dt, nb in [("fp64_doublefloat", bt.BTTB_MV_FP64, x, y, bt.BTTB_C128, b64),
                                      ("fp32", bt.BTTB_MV_FP32, x32, y32, bt.BTTB_C64, b32),
                                      ("fp64_native", bt.BTTB_MV_FP64_NATIVE, x, y, bt.BTTB_C128, b64)]:
        entry = {}
        for route in (0, 1, 2, 3, 4):
            bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, route)
            taken = bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_ROUTE_TAKEN, (prec << 8) | 1)
            if route and taken != route:
                continue                                    # that form does not apply to this precision
            reps = 30
            with torch.cuda.stream(stream):
                for _ in range(3):
                    bt.bttb_matvec(plan.handle, xx, yy, 1, n, dt, prec)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    bt.bttb_matvec(plan.handle, xx, yy, 1, n, dt, prec)
                e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps
            rec = {"us": t * 1e3, "gbs": nb / (t / 1e3) / 1e9, "route": route_names[taken]}
            if route == 0:
                entry.update(rec)
            else:
                entry.setdefault("by_route", {})[route_names[route]] = rec
        mv[name] = entry
    plan.autotune(1, 30)                      # the sweep forced each form: restore the tuned ones
    if args.product_form:
        bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_PRODUCT_ROUTE, args.product_form)
    ir_route = route_names[bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_ROUTE_TAKEN, (bt.BTTB_MV_FP32 << 8) | 1)]
    df_route = route_names[bt.bttb_plan_debug(plan.handle, bt.BTTB_DEBUG_ROUTE_TAKEN, (bt.BTTB_MV_FP64 << 8) | 1)]


    # multi-RHS: every element's port excitation of the same array (900 columns), one batched IR solve
    multi = None
    if os.environ.get("BTTB_BENCH_SKIP_MULTI") is None:
        kall = nx * ny
        vm = torch.from_numpy(arrays.port_excitations(nx, ny, b).T.copy()).to(dev)
        im = torch.zeros_like(vm)
        planm = bt.Plan(nx, ny, b, max_rhs=kall, prec_mask=(1 << bt.BTTB_MV_FP64) | (1 << bt.BTTB_MV_FP32) |
                        (1 << bt.BTTB_MV_TC_3XTF32) | (1 << bt.BTTB_MV_TC_BF16X3), stream=stream)
        planm.set_generators(gen)
        torch.cuda.synchronize()
        width = planm.autotune(kall, 3)                       # FFT chunk width for 900-column products
        with torch.cuda.stream(stream):
            planm.solve(vm, im, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32, max_iters=2)   # graph + buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            im.zero_()
            torch.cuda.nvtx.range_push("multi_solve")
            _, rcm, resm = planm.solve(vm, im, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32)
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        mt = time.perf_counter() - t0
        its = [r.iters for r in resm]
        cols = [0, kall // 2, kall - 1]
        vm_h, im_h = vm.cpu().numpy().T, im.cpu().numpy().T
        multi_oracle = oracle_relres_sampled(gen, vm_h, im_h, cols)
        multi = {"columns": kall, "solve_ms": mt * 1e3, "ms_per_column": mt * 1e3 / kall,
                 "oracle_relres_sampled": dict(zip(map(str, cols), multi_oracle)),
                 "oracle_relres_max_sampled": max(multi_oracle),
                 "status_ok": sum(r.status == bt.BTTB_OK for r in resm), "iters_max": max(its),
                 "iters_mean": float(np.mean(its)), "relres_true_max": max(r.relres_true for r in resm),
                 "speedup_vs_fp64_column_by_column": fp64_ms * kall / (mt * 1e3),
                 "workspace_gb": planm.workspace_bytes() / 1e9, "fft_chunk_width": width}
        # per-kernel breakdown of the first cycle (restart steps), event nodes around every kernel
        bt.bttb_profile(planm.handle, 2)
        with torch.cuda.stream(stream):
            im.zero_()
            planm.solve(vm, im, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32, max_iters=restart)
        torch.cuda.synchronize()
        vec_bytes = nx * ny * b * 16 * kall                  # one double-float Krylov vector of every column
        # algorithmic traffic of one cycle: the reduction of step j reads q_0..q_{j-1}, u and x (plus the
        # closing reduction: the basis and u); the update reads q_0..q_{j-1}, u, x and writes q_j, u_{j+1}
        cyc_bytes = {3: vec_bytes * (sum(j + 2 for j in range(restart)) + restart + 1),
                     4: vec_bytes * sum(j + 4 for j in range(restart))}
        cyc = {}
        for name, kid in {"fft_passes": bt.BTTB_K_FFT, "gs_dots": 3, "gs_update": 4,
                          "block_product_fp32": bt.BTTB_K_BLOCK_PRODUCT_PREC + bt.BTTB_MV_FP32}.items():
            st = bt.bttb_profile_read(planm.handle, kid)
            cyc[name] = {"launches": st.launches, "total_ms": st.ms}
            if kid in cyc_bytes and st.ms > 0:
                cyc[name]["achieved_gbs"] = cyc_bytes[kid] / (st.ms / 1e3) / 1e9
        bt.bttb_profile(planm.handle, 0)
        multi["first_cycle_breakdown"] = cyc
        # the paper's global GMRES: one Krylov space over vec(I), Frobenius inner products
        with torch.cuda.stream(stream):
            planm.solve(vm, im, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32, max_iters=2,
                        flags=bt.BTTB_GMRES_GLOBAL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            im.zero_()
            _, rcg, resg = planm.solve(vm, im, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32,
                                       flags=bt.BTTB_GMRES_GLOBAL)
        torch.cuda.synchronize()
        gt = time.perf_counter() - t0
        glob_oracle = oracle_relres_sampled(gen, vm_h, im.cpu().numpy().T, cols)
        multi["global_gmres_ir"] = {"solve_ms": gt * 1e3, "iters": resg[0].iters,
                                    "oracle_relres_max_sampled": max(glob_oracle),
                                    "status_ok": sum(r.status == bt.BTTB_OK for r in resg),
                                    "relres_true_max": max(r.relres_true for r in resg),
                                    "speedup_vs_fp64_column_by_column": fp64_ms * kall / (gt * 1e3)}
        # the per-bin GEMM of one 900-column product: binary32 FMA kernel vs the tcgen05 tensor-core kernel
        # (3xTF32, split-BF16x3); CUDA events around the block-product launches, 5 products each
        xm = torch.randn(kall, n, dtype=torch.complex64, device=dev)
        ym = torch.empty_like(xm)
        gemm = {}
        for name, pr in (("fp32_fma", bt.BTTB_MV_FP32), ("tc_3xtf32", bt.BTTB_MV_TC_3XTF32),
                         ("tc_bf16x3", bt.BTTB_MV_TC_BF16X3)):
            with torch.cuda.stream(stream):
                bt.bttb_matvec(planm.handle, xm, ym, kall, n, bt.BTTB_C64, pr)
            torch.cuda.synchronize()
            bt.bttb_profile(planm.handle, 1)
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                for _ in range(5):
                    bt.bttb_matvec(planm.handle, xm, ym, kall, n, bt.BTTB_C64, pr)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) / 5
            bt.bttb_profile(planm.handle, 0)
            st_ = bt.bttb_profile_read(planm.handle, bt.BTTB_K_BLOCK_PRODUCT_PREC + pr)
            gemm[name] = {"block_product_ms": st_.ms / max(st_.launches, 1), "product_ms": wall * 1e3,
                          "algorithmic_gbs": st_.bytes / (st_.ms / 1e3) / 1e9 if st_.ms > 0 else None,
                          "useful_tflops": 8.0 * mx * my * b * b * kall / (st_.ms / max(st_.launches, 1) / 1e3) / 1e12
                          if st_.ms > 0 else None}
        multi["per_bin_gemm_900_columns"] = gemm
        del xm, ym
        # the all-ports solve with tensor-core inner products (the batched per-column GMRES-IR)
        for name, pr in (("tc_3xtf32_ir", bt.BTTB_MV_TC_3XTF32), ("tc_bf16x3_ir", bt.BTTB_MV_TC_BF16X3)):
            with torch.cuda.stream(stream):
                planm.solve(vm, im, tol=tol, restart=restart, inner=pr, max_iters=2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                im.zero_()
                _, rct, rest = planm.solve(vm, im, tol=tol, restart=restart, inner=pr)
            torch.cuda.synchronize()
            tt = time.perf_counter() - t0
            tco = oracle_relres_sampled(gen, vm_h, im.cpu().numpy().T, cols)
            multi[name] = {"solve_ms": tt * 1e3, "status_ok": sum(r.status == bt.BTTB_OK for r in rest),
                           "iters_max": max(r.iters for r in rest),
                           "relres_true_max": max(r.relres_true for r in rest),
                           "oracle_relres_max_sampled": max(tco),
                           "speedup_vs_fp32_ir": mt / tt,
                           "speedup_vs_fp64_column_by_column": fp64_ms * kall / (tt * 1e3)}
        del vm, im
        planm.close()
        torch.cuda.empty_cache()

    # uneven batch: 64 independent arrays (nx, ny ~ U{8..40}, b in {24, 60, 96}, 1..16 port excitations)
    uneven = None
    if os.environ.get("BTTB_BENCH_SKIP_UNEVEN") is None:
        specs = arrays.uneven_batch_specs()
        batch = bt.Batch([(s.nx, s.ny, s.b, s.nrhs) for s in specs])
        vs = []
        for i, sp in enumerate(specs):
            g = arrays.generator_blocks_torch(sp.nx, sp.ny, sp.b, sp.seed, device=dev)
            batch.set_generators(i, g)
            del g
            cells = [(c % sp.nx, c // sp.nx) for c in range(sp.nrhs)]
            vs.append(torch.from_numpy(arrays.port_excitations(sp.nx, sp.ny, sp.b, cells).T.copy()).to(dev))
        widths = batch.autotune(reps=3)
        batch.solve(vs, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32, max_iters=2)     # graphs + buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Is_u, rcu, resu = batch.solve(vs, tol=tol, restart=restart, inner=bt.BTTB_MV_FP32)
        torch.cuda.synchronize()
        ut = time.perf_counter() - t0
        # sampled columns re-measured with the oracle: the first column of three arrays
        samp = [0, len(specs) // 2, len(specs) - 1]
        uneven_oracle = []
        for i in samp:
            sp = specs[i]
            gi = arrays.generator_blocks(sp.nx, sp.ny, sp.b, sp.seed)
            uneven_oracle += oracle_relres_sampled(gi, vs[i].cpu().numpy().T, Is_u[i].cpu().numpy().T, [0])
        # the same arrays one after another: plain FP64 GMRES, and the batch's own precision (binary32
        # products, FP64-class refinement) -- the second isolates the gain of running the arrays concurrently
        plans = [bt.bttb_batch_plan(batch.handle, i) for i in range(len(specs))]

        def sequential(inner):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(len(specs)):
                out = torch.zeros_like(vs[i])
                bt.bttb_gmres_solve(plans[i], vs[i], out, vs[i].shape[0], vs[i].shape[1],
                                    bt.gmres_opts(tol=tol, restart=restart, inner=inner))
            torch.cuda.synchronize()
            return time.perf_counter() - t0

        st = sequential(bt.BTTB_MV_FP64)
        seq_ir = sequential(bt.BTTB_MV_FP32)
        its = [r.iters for r in resu]
        uneven = {"arrays": len(specs), "columns": len(resu), "solve_ms": ut * 1e3,
                  "status_ok": sum(r.status == bt.BTTB_OK for r in resu), "iters_max": max(its),
                  "iters_mean": float(np.mean(its)), "relres_true_max": max(r.relres_true for r in resu),
                  "oracle_relres_sampled_arrays": samp, "oracle_relres_max_sampled": max(uneven_oracle),
                  "sequential_fp64_ms": st * 1e3, "speedup_vs_sequential_fp64": st / ut,
                  "sequential_ir_ms": seq_ir * 1e3, "speedup_vs_sequential_ir": seq_ir / ut,
                  "fft_chunk_widths": {str(w): widths.count(w) for w in sorted(set(widths))},
                  "unknowns_total": int(sum(s.nx * s.ny * s.b * s.nrhs for s in specs))}
        del vs
        batch.close()
        torch.cuda.empty_cache()

    learned = None
    if os.environ.get("BTTB_BENCH_SKIP_LEARNED") is None:
        learned = learned_leg(dev, stream)
        torch.cuda.empty_cache()

    peak, peak_kind = measured_peaks()
    # the block products of the host-driven solve: each launch bracketed by CUDA events on the plan's stream
    # with nothing else in flight (event nodes inside the captured graphs also time the broken
    # programmatic-dependent-launch overlap, which depends on the neighbouring kernels' shapes)
    h32, h64 = hd["block_product_fp32"], hd["block_product_doublefloat"]
    ach32 = h32.bytes / (h32.ms / 1e3) / 1e9 if h32.ms > 0 else 0.0
    ach64 = h64.bytes / (h64.ms / 1e3) / 1e9 if h64.ms > 0 else 0.0
    if ir_route == "fused_y":
        kname = ("ycontract_kernel<F32,1> (level-2 FFT + binary32 block product of 3600 bins x 60x60 + inverse "
                 "level-2 FFT, one cluster kernel)")
        traffic = traffic_from_profiles("ycontract_f32_30x30_b60", "ycontract.cu")
    else:
        kname = "contract_kernel<F32> (binary32 block product, 3600 bins x 60x60)"
        traffic = traffic_from_profiles("contract_f32_30x30_b60", "contract.cu")
    roofline = {"kernel": kname, "product_route": ir_route,
                "bound": "hbm", "achieved": ach32, "peak": peak, "unit": "GB/s",
                "frac": ach32 / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                "whole_product": {
                    "note": "one whole FFT product (x in, spectrum planes once, y out: 209.1 MB double-float, "
                            "104.5 MB binary32) / its CUDA-event time, 30 back-to-back products",
                    "fp64_doublefloat": {"achieved": mv["fp64_doublefloat"]["gbs"],
                                         "frac": mv["fp64_doublefloat"]["gbs"] / peak,
                                         "us": mv["fp64_doublefloat"]["us"], "route": mv["fp64_doublefloat"]["route"]},
                    "fp32": {"achieved": mv["fp32"]["gbs"], "frac": mv["fp32"]["gbs"] / peak,
                             "us": mv["fp32"]["us"], "route": mv["fp32"]["route"]}},
                "traffic": traffic, "algorithmic_bytes_per_launch": h32.bytes / max(h32.launches, 1),
                "avg_launch_us": h32.ms * 1e3 / max(h32.launches, 1), "launches": h32.launches,
                "share_of_step": st32.ms / ms_prof if ms_prof > 0 else None,
                "timing": "CUDA events around each block-product launch on the plan's stream, over one solve of "
                          "the same step run launch by launch (no graphs) with the tuned forms; the second "
                          "window of the K steps with event nodes inside the graphs gives "
                          f"{st32.ms * 1e3 / max(st32.launches, 1):.2f} us per launch (graph_window_avg_us) "
                          f"and took {ms_prof / args.steps:.2f} ms per step against {ms / args.steps:.2f} ms "
                          "unprofiled",
                "graph_window_avg_us": st32.ms * 1e3 / max(st32.launches, 1),
                "doublefloat_product": {"achieved": ach64, "frac": ach64 / peak, "launches": h64.launches,
                                        "avg_launch_us": h64.ms * 1e3 / max(h64.launches, 1)},
                "fft_passes": {"ms_per_step": stfft.ms / args.steps, "launches": stfft.launches,
                               "achieved_gbs": stfft.bytes / (stfft.ms / 1e3) / 1e9 if stfft.ms > 0 else 0.0}}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        t_cpu, reps = cpu_oracle_product_time(gen, n)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": b64 / t_cpu / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"{reps} brute-force O(N^2) FP64 products of the same matrix ({t_cpu:.2f} s each); "
                         "bytes counted as for one FFT product"}
        cpu["mlfft_host"] = host_mlfft_baseline(gen, nx, ny, b, mx, my, fp64_res.iters + fp64_res.cycles + 1,
                                                os.cpu_count() or 1)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 products + df64 (double-float) residual/Arnoldi",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "b": b, "grid": [mx, my], "seed": c["seed"],
                   "fft_chunk_width": fft_width, "product_forms": {"fp32": ir_route, "fp64": df_route},
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: every product streams the 104-207 MB spectrum"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": n * 16,
                "ms_per_step": e2e_s * 1e3 / args.steps},
        "gpu_launches": stall.launches,
        "clocks": clk,
        "gmres": {"comparator": "fp64_ms is GMRES with double-float (FP64-class) products, Arnoldi and "
                                "residuals; binary64_products_ms runs the products in IEEE binary64 (DFMA); "
                                "every speedup_* divides fp64_ms",
                  "ir_ms": ir_ms, "fp64_ms": fp64_ms, "speedup_ir_vs_fp64": fp64_ms / ir_ms,
                  "binary64_products_ms": f64n_ms, "binary64_products_iters": f64n_res.iters,
                  "binary64_products_relres_true": f64n_res.relres_true,
                  "speedup_ir_vs_binary64_products": f64n_ms / ir_ms,
                  "ir_iters": iters[0], "ir_cycles": cycles[0], "fp64_iters": fp64_res.iters,
                  "ir_relres_true": max(relres), "fp64_relres_true": fp64_res.relres_true,
                  "ir_oracle_relres": ir_oracle, "block_jacobi_ir_ms": bj_ms, "block_jacobi_ir_iters": bj_res.iters,
                  "speedup_bj_ir_vs_fp64": fp64_ms / bj_ms},
        "matvec": mv,
        "step_breakdown_host_driven": breakdown,
        "multi_rhs": multi,
        "uneven_batch": uneven,
        "learned_preconditioner": learned,
    }
    print(json.dumps(line), flush=True)
    barrier(world)
    plan.close()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
