#!/usr/bin/env python
"""Benchmark: eigenvalues + eigenvectors of an n = 32768 symmetric tridiagonal
(d, e ~ U[-1, 1], seed 0) on one GB300, through the library's C ABI.

One step = one full tdc_syev_tridiag solve (tear, leaves, and every merge level:
deflation, secular roots, Loewner z, norms, eigenvector product, placement, deflated
copy, sign normalisation).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n 32768] [--gen uniform|graded|normal|toeplitz] [--path fp64|ozaki|hss|auto]

Under torchrun (N > 1) every rank solves its own replica (the solve does not shard
across GPUs; see the design notes), the timed region is bracketed by barriers, the
maximum over ranks is reported and value = seconds per solve for the whole job
(step time / N).  --impl reference times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n=32768 eig+vecs time (s); merge Q·U eff. TFLOP/s vs peak; at stated orth/resid"
PATHS = {"fp64": 0, "ozaki": 1, "hss": 2, "auto": 3}
# FP64 on GB300 runs on the SIMT FP64 pipe: 2 DFMA per clock per SM (ncu's
# sm__sass_thread_inst_executed_op_dfma_pred_on peak), 152 SMs, 2 flops per FMA
GB300_SMS = 152
DFMA_PER_CLK_SM = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--gen", default="uniform", choices=["uniform", "graded", "normal", "toeplitz"])
    ap.add_argument("--path", default="fp64", choices=list(PATHS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--leaf", type=int, default=8,
                    help="leaf order of the DC tree (8: fastest at n = 32768; the library default is 32)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the few-deflation and batched context measurements")
    ap.add_argument("--no-tune", action="store_true", help="skip the FP64 tile-shape autotuning")
    ap.add_argument("--direct", action="store_true",
                    help="time direct tdc_syev_tridiag calls instead of replays of a captured plan")
    return ap.parse_args()


def make_input(gen, n, seed=0):
    import workloads as W
    if gen == "uniform":
        return W.uniform_tridiag(n, seed)
    if gen == "graded":
        return W.graded_tridiag(n, seed)
    if gen == "normal":
        return W.normal_tridiag(n, seed)
    return W.toeplitz_121(n)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count()


def time_oracle(gen, n, leaf):
    """Seconds of one CPU-oracle solve (oracle.dc.dc_eig as it stands) of the workload's
    matrix of order n."""
    from oracle import dc
    d, e = make_input(gen, n, 0)
    t0 = time.perf_counter()
    dc.dc_eig(d, e, leaf=leaf)
    return time.perf_counter() - t0


def cpu_oracle_fit(gen, n_full, leaf, sizes=(8192, 16384)):
    """A bounded CPU-oracle sample: solves of orders `sizes` (seed 0, same distribution),
    timed once each (the CPU has no warm-up effect), and the time at n_full from the
    power law t = c n^p through the two largest points (p fitted, not assumed)."""
    import math
    ts = [time_oracle(gen, n, leaf) for n in sizes]
    p = math.log(ts[-1] / ts[-2]) / math.log(sizes[-1] / sizes[-2])
    value = ts[-1] * (n_full / sizes[-1]) ** p
    sample = ("oracle dc_eig at n=" + ", ".join(f"{n}: {t:.2f} s" for n, t in zip(sizes, ts))
              + f" ({gen}, seed 0, leaf {leaf}); fitted exponent p={p:.3f}; value = t({sizes[-1]}) x "
              f"({n_full}/{sizes[-1]})^p")
    return value, {"sizes": list(sizes), "seconds": ts, "exponent": p}, sample, _oracle_threads()


def workload_config(args):
    """The `config` of both arms' lines (the workload: matrix, order, product path, leaf)."""
    return {"workload": f"tridiag eig+vecs n={args.n}, {args.gen} seed 0, leaf {args.leaf}, path {args.path}",
            "n": args.n, "gen": args.gen, "path": args.path, "leaf": args.leaf,
            "l2": "inputs and eigenvector buffers (8.6 GB each at n=32768) far exceed L2",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def sampled_accuracy(torch, d, e, lam, q, ncol=32, seed=1):
    """Orthogonality of `ncol` sampled eigenvectors against all of them (max |Q^T q_s - e_s|)
    and their scaled residual ||T q - lambda q||_F / (sqrt(ncol/n) n eps ||T||_1),
    eps = 2^-52, computed with torch on the GPU from the definitions."""
    import numpy as np
    n = len(d)
    ncol = min(ncol, n)
    sel = np.random.Generator(np.random.PCG64(seed)).choice(n, ncol, replace=False)
    idx = torch.tensor(sel, device=q.device)
    qs = q[:, idx]
    gram = q.t() @ qs
    gram[idx, torch.arange(ncol, device=q.device)] -= 1.0
    dt = torch.tensor(d, device=q.device)
    et = torch.tensor(e, device=q.device)
    tq = dt[:, None] * qs
    if n > 1:
        tq[:-1] += et[:, None] * qs[1:]
        tq[1:] += et[:, None] * qs[:-1]
    r = tq - qs * lam[idx][None, :]
    row = dt.abs().clone()
    if n > 1:
        row[:-1] += et.abs()
        row[1:] += et.abs()
    tnorm = float(row.max())
    return {"orth_max_sampled": float(gram.abs().max()),
            "resid_scaled_sampled": float(torch.linalg.norm(r)) / (ncol / n) ** 0.5 / (n * 2.0 ** -52 * tnorm)}


def profiled_solve(api, _lib, lib, torch, d, e, path, exact=None, **kw):
    """One warm-up and one timed solve with per-phase events; returns a summary."""
    import ctypes
    n = len(d)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    o = _lib.default_opts(path=PATHS[path], **kw)
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    q = api.fortran_empty(n, n, "cuda")
    api.syev_tridiag(dt, et, opts=o, out=(lam, q))
    torch.cuda.synchronize()
    lib.tdc_profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.syev_tridiag(dt, et, opts=o, out=(lam, q), check=False)
    e1.record()
    e1.synchronize()
    p = _lib.TdcProfile()
    lib.tdc_profile_end(ctypes.byref(p))
    prod_ms = p.ms[5] + p.ms[8] + p.ms[9]
    out = {"ms": e0.elapsed_time(e1), "product_ms": prod_ms,
           "product_eff_fp64_tflops": p.product_flops / (prod_ms * 1e-3) / 1e12 if prod_ms else 0.0,
           "product_algorithmic_flops": p.product_flops}
    if p.ms[8]:
        out["split_gemm_ms"] = p.ms[8]
        out["split_operand_split_ms"] = p.ms[9]
        out["split_gemm_bf16_tflops"] = p.split_tensor_flops / (p.ms[8] * 1e-3) / 1e12
    out["phases_ms"] = {nm: round(p.ms[i], 3) for i, nm in enumerate(_lib.PHASES)}
    if p.sg_gemm_ms > 0:             # the dense split GEMM kernel (HSS products): bf16 slice-pair rate
        pk, src = peaks()
        rate = p.sg_tensor_flops / (p.sg_gemm_ms * 1e-3) / 1e12
        peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        out["sg_gemm"] = {"kernel": "k_sg_gemm (split-precision tcgen05 GEMM, all HSS products)", "ms": p.sg_gemm_ms,
                          "bf16_tflops": rate, "peak": peak, "frac": rate / peak,
                          "peak_source": f"{src} bf16 sustained",
                          "flops_basis": "launch-time sizes (device-held ranks below them count as zeros)"}
    if p.ms[10] > 0:                 # HSS: the sampling's FP64-equivalent rate (4 K^2 (r + p) flops, split GEMM)
        out["hss"] = {"sampling_flops": p.hss_sampling_flops,
                      "sampling_fp64_equivalent_tflops": p.hss_sampling_flops / (p.ms[10] * 1e-3) / 1e12,
                      "regrowths": int(p.hss_regrowths), "dense_fallbacks": int(p.hss_fallbacks)}
    out["K_total"] = int(p.K_total)
    out["secular_fp64_evals_per_root"] = p.secular_evals / max(int(p.K_total), 1)
    out["accuracy"] = sampled_accuracy(torch, d, e, lam, q)
    if exact is not None:           # closed-form eigenvalues: max |error| / (n eps ||T||)
        lh = lam.cpu().numpy()
        tn = float(max(abs(d).max() + 2 * abs(e).max(), 1e-300))
        out["accuracy"]["eig_err_scaled_closed_form"] = float(abs(lh - exact).max()) / (n * 2.0 ** -52 * tn)
    del q
    torch.cuda.empty_cache()
    return out


def context_measurements(api, _lib, lib, torch):
    """Context runs beside the headline:
    - the few-deflation case tridiag(1,2,1) (Examples 2-3) with each product form;
    - the headline matrix and the graded matrix of the same configuration on the split
      product, with their accuracy (error per result);
    - the paper's example matrices at n = 30000 (Clement, Hermite, tridiag(1,2,1), SHT of
      Example 4) on the split product, with per-phase times (a Table 2 analog) and the
      closed-form eigenvalues where there are any;
    - a sweep of the AUTO path's K threshold (HSS above it, split product below);
    - the batched configuration (ragged problems, autotuned tiles, graph replay)."""
    import numpy as np
    import workloads as W
    ctx = {}
    d, e = W.toeplitz_121(32768)
    k = np.arange(1, 32769)
    ctx["toeplitz_32768_split"] = profiled_solve(api, _lib, lib, torch, d, e, "ozaki",
                                                 exact=2.0 - 2.0 * np.cos(k * np.pi / 32769))
    ctx["toeplitz_32768_split_7slices"] = profiled_solve(api, _lib, lib, torch, d, e, "ozaki", ozaki_slices=7,
                                                         exact=2.0 - 2.0 * np.cos(k * np.pi / 32769))
    ctx["toeplitz_32768_hss"] = profiled_solve(api, _lib, lib, torch, d, e, "hss",
                                               exact=2.0 - 2.0 * np.cos(k * np.pi / 32769))
    ctx["toeplitz_32768_auto"] = profiled_solve(api, _lib, lib, torch, d, e, "auto",
                                                exact=2.0 - 2.0 * np.cos(k * np.pi / 32769))
    d, e = W.uniform_tridiag(32768, 0)
    ctx["uniform_32768_split"] = profiled_solve(api, _lib, lib, torch, d, e, "ozaki")
    d, e = W.graded_tridiag(32768, 0)
    ctx["graded_32768_fp64"] = profiled_solve(api, _lib, lib, torch, d, e, "fp64")
    ctx["graded_32768_split"] = profiled_solve(api, _lib, lib, torch, d, e, "ozaki")
    d, e = W.toeplitz_121(16384)
    k = np.arange(1, 16385)
    ex = 2.0 - 2.0 * np.cos(k * np.pi / 16385)
    ctx["toeplitz_16384_fp64"] = profiled_solve(api, _lib, lib, torch, d, e, "fp64", exact=ex)
    ctx["toeplitz_16384_split"] = profiled_solve(api, _lib, lib, torch, d, e, "ozaki", exact=ex)
    ctx["toeplitz_16384_hss"] = profiled_solve(api, _lib, lib, torch, d, e, "hss", exact=ex)
    # HSS with 256-leaves and 64 starting samples (grown where a rank reaches them): less
    # work in the sampling and the IDs, a looser residual
    ctx["toeplitz_16384_hss_leaf256_rp64"] = profiled_solve(api, _lib, lib, torch, d, e, "hss", exact=ex,
                                                            hss_leaf=256, hss_rp=64)
    d, e = W.normal_tridiag(16384, 0)
    ctx["normal_16384_fp64"] = profiled_solve(api, _lib, lib, torch, d, e, "fp64")
    ctx["normal_16384_hss"] = profiled_solve(api, _lib, lib, torch, d, e, "hss")
    n = 30000
    ex_clement = np.arange(-(n - 1), n, 2, dtype=np.float64)
    for name, (d, e), ex in (("clement", W.clement(n), ex_clement),
                             ("hermite", W.hermite(n), None),
                             ("toeplitz", W.toeplitz_121(n), 2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))),
                             ("sht", W.sht(n), None)):
        ctx[f"paper_{name}_30000_split"] = profiled_solve(api, _lib, lib, torch, d, e, "ozaki", exact=ex)
    d, e = W.toeplitz_121(16384)
    sweep = {}
    for kt in (2048, 4096, 8192, 16385):
        r = profiled_solve(api, _lib, lib, torch, d, e, "auto", k_threshold=kt)
        sweep[str(kt)] = {"ms": r["ms"], "accuracy": r["accuracy"]}
    ctx["auto_k_threshold_sweep_toeplitz_16384"] = sweep
    # batched: 4096 problems, n log-uniform in [32, 2048], d, e ~ N(0, 1)
    sizes, probs = W.batched_normal(4096, seed=0)
    plan = api.BatchedPlan(sizes, opts={"path": PATHS["fp64"]})
    d_cat, e_cat = plan.pack([p[0] for p in probs], [p[1] for p in probs])
    lam, q = plan.outputs()
    shapes = plan.autotune(d_cat, e_cat, lam, q)
    plan.capture(d_cat, e_cat, lam, q)
    for _ in range(2):
        plan.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        plan.replay()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # per-phase times of one direct (non-graph) execute of the same plan
    import ctypes
    torch.cuda.synchronize()
    lib.tdc_profile_begin()
    plan.execute(d_cat, e_cat, lam, q)
    torch.cuda.synchronize()
    p = _lib.TdcProfile()
    lib.tdc_profile_end(ctypes.byref(p))
    ctx["batched_4096_phases_ms"] = {nm: round(p.ms[i], 3) for i, nm in enumerate(_lib.PHASES) if p.ms[i] > 0}
    if p.secular_flops > 0 and p.ms[2] > 0:
        ctx["batched_4096_secular"] = {"algorithmic_tflop": p.secular_flops / 1e12,
                                       "achieved_tflops": p.secular_flops / (p.ms[2] * 1e-3) / 1e12,
                                       "fp64_evals_per_root": p.secular_evals / max(p.K_total, 1)}
    ctx["batched_4096"] = {"ms": ms, "problems_per_s": 4096 / (ms * 1e-3), "sum_n": int(sizes.sum()),
                           "status_nonzero": int((plan.status != 0).sum()),
                           "tile_shapes": ",".join(map(str, shapes)),
                           "launch": "one launch per phase per tree level, captured in a CUDA graph"}
    # the same batch as ONE persistent kernel launch (each CTA takes whole problems from a
    # work queue, largest first), captured in a graph and replayed
    lam_p, q_p = plan.outputs()
    plan.capture(d_cat, e_cat, lam_p, q_p, persistent=True)
    for _ in range(2):
        plan.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.replay()
    e1.record()
    e1.synchronize()
    ms_p = e0.elapsed_time(e1) / reps
    ctx["batched_4096_persistent"] = {"ms": ms_p, "problems_per_s": 4096 / (ms_p * 1e-3),
                                      "status_nonzero": int((plan.status != 0).sum()),
                                      "max_abs_lambda_diff_vs_level_launches": float((lam_p - lam).abs().max()),
                                      "launch": "one persistent kernel (after 4 memsets), captured in a CUDA graph"}
    del lam_p, q_p
    # the same batch with the split-precision product for merges of order 256 and up
    # (level form; the persistent kernel keeps the FP64 product)
    plan_s = api.BatchedPlan(sizes, opts={"path": PATHS["ozaki"]})
    lam_s, q_s = plan_s.outputs()
    plan_s.autotune(d_cat, e_cat, lam_s, q_s)
    plan_s.capture(d_cat, e_cat, lam_s, q_s)
    for _ in range(2):
        plan_s.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        plan_s.replay()
    e1.record()
    e1.synchronize()
    ms_s = e0.elapsed_time(e1) / reps
    ctx["batched_4096_split"] = {"ms": ms_s, "problems_per_s": 4096 / (ms_s * 1e-3),
                                 "status_nonzero": int((plan_s.status != 0).sum()),
                                 "max_abs_lambda_diff_vs_fp64": float((lam_s - lam).abs().max()),
                                 "launch": "one launch per phase per tree level, captured in a CUDA graph"}
    del plan_s, lam_s, q_s
    del plan, q, lam
    torch.cuda.empty_cache()
    ctx["backward_batched_64x4096"] = backward_measurement(api, _lib, lib, torch)
    return ctx


def backward_measurement(api, _lib, lib, torch, batch=64, n=4096, m=64):
    """The differentiable configuration: 64 problems of n = 4096 (d, e ~ N(0, 1)), loss
    sum_i w_i lambda_i + ||Q[:, :64]^T G||_F^2 per problem.  Times the batched forward
    (graph replay of the batched plan) and the batched backward to (d, e); the backward's
    work is 2 products of n x n x 64 per problem (Q^T Qbar_S, then Q M_S: 4 n^2 64 flops)
    plus the band sums of the lambda term (6 n^2 flops), on the FP64 pipe."""
    import numpy as np
    import workloads as W
    sizes = np.full(batch, n, dtype=np.int64)
    ds = [W.normal_tridiag(n, 500 + p)[0] for p in range(batch)]
    es = [W.normal_tridiag(n, 500 + p)[1] for p in range(batch)]
    plan = api.BatchedPlan(sizes, opts={"path": PATHS["fp64"]})
    d_cat, e_cat = plan.pack(ds, es)
    lam, q = plan.outputs()
    plan.autotune(d_cat, e_cat, lam, q)
    plan.capture(d_cat, e_cat, lam, q)
    for _ in range(2):
        plan.replay()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    plan.replay()
    f1.record()
    f1.synchronize()
    fwd_ms = f0.elapsed_time(f1)
    w = torch.tensor(np.concatenate([W.gaussian(n, 900 + p) for p in range(batch)]), device="cuda")
    gq = torch.zeros_like(q)
    for p in range(batch):
        G = torch.tensor(W.gaussian((n, m), 1000 + p), device="cuda")
        qp = q[p * n * n:(p + 1) * n * n].view(n, n).t()
        gq[p * n * n:(p + 1) * n * n].view(n, n).t()[:, :m] = 2.0 * G @ (G.t() @ qp[:, :m])
    api.syev_backward_batched(sizes, lam, q, w, gq, max_cols=m)
    torch.cuda.synchronize()
    reps = 3
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    for _ in range(reps):
        gd, ge = api.syev_backward_batched(sizes, lam, q, w, gq, max_cols=m)
    b1.record()
    b1.synchronize()
    bw_ms = b0.elapsed_time(b1) / reps
    # the same backward with its two products on the split-precision tensor-core path
    so = {"path": PATHS["ozaki"]}
    gd_s, ge_s = api.syev_backward_batched(sizes, lam, q, w, gq, max_cols=m, opts=so)
    torch.cuda.synchronize()
    b0.record()
    for _ in range(reps):
        gd_s, ge_s = api.syev_backward_batched(sizes, lam, q, w, gq, max_cols=m, opts=so)
    b1.record()
    b1.synchronize()
    bw_split_ms = b0.elapsed_time(b1) / reps
    gscale = max(torch.max(torch.abs(gd)).item(), torch.max(torch.abs(ge)).item())
    split_err = max(torch.max(torch.abs(gd_s - gd)).item(), torch.max(torch.abs(ge_s - ge)).item()) / gscale
    flops = batch * (4.0 * n * n * m + 6.0 * n * n)
    out = {"forward_ms": fwd_ms, "backward_ms": bw_ms, "problems": batch, "n": n, "loss_columns": m,
           "backward_split_products_ms": bw_split_ms,
           "backward_split_max_rel_diff_vs_fp64": split_err,
           "backward_algorithmic_flops": flops,
           "backward_fp64_tflops": flops / (bw_ms * 1e-3) / 1e12,
           "note": "backward timed with its one stream synchronization (the column count) inside"}
    del plan, q, lam, gq, d_cat, e_cat
    torch.cuda.empty_cache()
    return out


def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        else:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(torch):
    """(NUMA node, its CPUs) of the current GPU's PCI device, or (None, None).  Page-locked
    host buffers allocated by a thread on those CPUs are placed in that node's memory
    (first touch), next to the GPU's host link."""
    import subprocess
    try:
        idx = torch.cuda.current_device()
        out = subprocess.run(["nvidia-smi", "-i", str(idx), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, bus, rest = out.split(":")
        bdf = f"{int(dom, 16):04x}:{bus.lower()}:{rest.lower()}"
        node = int(open(f"/sys/bus/pci/devices/{bdf}/numa_node").read())
        if node < 0:
            return None, None
        return node, _cpulist(open(f"/sys/devices/system/node/node{node}/cpulist").read())
    except Exception:
        return None, None


# DRAM traffic of the FP64 product kernel, from a small case that ncu can capture
# within its size rule: one solve of tridiag U[-1, 1], n = 8192, leaf 8 (a few GB on the
# device), DRAM bytes read + written by the three k_gemm_fp64 launches of its top three
# tree levels, divided by those levels' algorithmic bytes (Q_sel read + U written, the
# per-level product_min_bytes that the same run records).  The capture and its command
# are summarised under profiles/.  The product reads each selected column of Q once
# and writes each output column once whatever n is, so the ratio carries over to
# n = 32768, where the traffic per launch is the ratio times the algorithmic bytes per
# launch.  A kernel whose source files (all of them) have changed since the capture
# reports no traffic.
TRAFFIC_RATIO = {
    # the top three levels (7-9) at n = 8192, leaf 8: DRAM 728832 + 379136 + 326400 bytes read,
    # 0 written, against 9043968 + 9388032 + 9175040 algorithmic bytes (the working set stays in L2)
    "k_gemm_fp64": (1434368 / 27607040,
                    (("paper_1612_07526_gb300/csrc/gemm_fp64.cu", "77ca22faebba88f56e0fdf2de8ee79efeddd6d3d6dce1dd896dc2f7353fe1bd2"),
                     ("paper_1612_07526_gb300/csrc/tdc_gemm_tile.cuh", "836078dcdb591b869d10646d2f2d04fd2b39f4e23d3551a8b68be960f55b228d"))),
}


def measured_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch of `kernel` (the captured ratio times the algorithmic bytes
    per launch), or None without a capture of the current source."""
    import hashlib
    rec = TRAFFIC_RATIO.get(kernel)
    if rec is None or not alg_bytes_per_launch:
        return None
    ratio, sources = rec
    for src, sha in sources:                   # every file holding the kernel's code, unchanged
        try:
            with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), src), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != sha:
                    return None
        except OSError:
            return None
    return ratio * alg_bytes_per_launch


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (the job's time is the slowest replica's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_solve(step_ms_max, world):
    """Replicas: each of `world` ranks solves one problem per step, so the job solves
    `world` problems in the slowest rank's step time."""
    return step_ms_max / 1000.0 / world


def run_reference(args, rank):
    """The reference arm: the CPU oracle (as it stands) solves the workload's full-size
    matrix once on the host's cores.  One solve takes minutes, so the arm times exactly
    one step whatever --steps / --warmup say (a CPU run has no warm-up effect) and
    reports it with steps = 1, warmup = 0."""
    if rank != 0:
        return
    t = time_oracle(args.gen, args.n, args.leaf)
    cores = _oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": t, "unit": "s", "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "steps_requested": args.steps, "warmup_requested": args.warmup,
        "ms_per_step": t * 1000.0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": workload_config(args),
        "cpu_baseline": {"value": t, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"the whole workload: one oracle dc_eig solve at n={args.n} ({args.gen}, seed 0, "
                                   f"leaf {args.leaf}), timed once (no warm-up effect on the CPU)"},
        "e2e": {"value": t, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import ctypes

    import numpy as np
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import _lib, api

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    lib = _lib.load()
    n = args.n
    d, e = make_input(args.gen, n, 0)
    dt = torch.tensor(d, device="cuda")
    et = torch.tensor(e, device="cuda")
    opts = _lib.default_opts(path=PATHS[args.path], leaf=args.leaf)
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    q = api.fortran_empty(n, n, "cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        api.syev_tridiag(dt, et, opts=opts, check=False, status=status, out=(lam, q), stream=stream)

    # The timed step is one whole solve.  By default it is the replay of a CUDA graph of
    # tdc_batched_plan_execute for this one problem (the public entry for repeated solves
    # of a fixed size: the plan is built, autotuned and captured once, then every step
    # replays the same kernels on device-resident inputs); --direct times direct
    # tdc_syev_tridiag calls, with their per-call host work and launches.
    shapes = None
    plan = None
    if args.direct or args.path not in ("fp64", "ozaki"):   # plans cover the dense product paths
        if not args.no_tune and args.path in ("fp64", "ozaki"):
            shapes = api.autotune(dt, et, opts=opts, stream=stream)     # one-time setup, before warm-up
        timed = step
    else:
        del q
        torch.cuda.empty_cache()
        plan = api.BatchedPlan([n], opts=opts)
        e_cat = torch.zeros(n, dtype=torch.float64, device="cuda")
        if n > 1:
            e_cat[:n - 1] = et
        lam, q_flat = plan.outputs()
        q = q_flat.view(n, n).t()                                       # column-major n x n
        if not args.no_tune and args.path in ("fp64", "ozaki"):
            shapes = plan.autotune(dt, e_cat, lam, q_flat)
        plan.capture(dt, e_cat, lam, q_flat)
        timed = plan.replay
    for _ in range(args.warmup):
        timed()
    barrier()
    bits = (int((plan.status != 0).sum()) if plan is not None
            else lib.tdc_read_status(api._vp(status), api._stream(stream)))
    if bits:
        raise SystemExit(f"device status {bits} during warm-up")

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            timed()
        ev1.record(stream)
        ev1.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = max_over_ranks(ms, dist, "cuda")
    bits = (int(plan.status.abs().sum()) if plan is not None
            else lib.tdc_read_status(api._vp(status), api._stream(stream)))
    # per-phase times, launch and work counts: the same solves again, outside the timed
    # region, with CUDA events around every phase (direct executes of the same plan)
    torch.cuda.synchronize()
    lib.tdc_profile_begin()
    for _ in range(args.steps):
        if plan is not None:
            plan.execute(dt, e_cat, lam, q_flat, stream=stream)
        else:
            step()
    torch.cuda.synchronize()
    prof = _lib.TdcProfile()
    lib.tdc_profile_end(ctypes.byref(prof))
    direct_ms = None
    if plan is not None:
        # context: the same solve as direct calls (plan build and launches per call)
        q_direct = api.fortran_empty(n, n, "cuda")
        lam_direct = torch.empty(n, dtype=torch.float64, device="cuda")
        o_direct = _lib.default_opts(path=PATHS[args.path], leaf=args.leaf)
        api.syev_tridiag(dt, et, opts=o_direct, out=(lam_direct, q_direct), stream=stream)
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(args.steps):
            api.syev_tridiag(dt, et, opts=o_direct, check=False, out=(lam_direct, q_direct), stream=stream)
        d1.record(stream)
        d1.synchronize()
        direct_ms = d0.elapsed_time(d1) / args.steps
        del q_direct, lam_direct
        torch.cuda.empty_cache()

    # accuracy of the last solve (sampled columns; the full checks live in the tests)
    acc = {}
    if rank == 0:
        acc = sampled_accuracy(torch, d, e, lam, q)
        acc["status"] = int(bits)

    step_kind = ("direct tdc_syev_tridiag calls" if plan is None else
                 "replay of a captured CUDA graph of the one-problem batched plan")
    if plan is not None:
        del plan, e_cat, q_flat
    del lam, q
    torch.cuda.empty_cache()

    # end to end through the host-memory entry point (pinned buffers)
    e2e = None
    if not args.no_e2e:
        # host buffers in the memory of the GPU's own NUMA node, as a deployment would
        # place them (numactl); the node is recorded with the result
        node, cpus = gpu_local_cpus(torch)
        old_aff = os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus & old_aff or cpus)
        # a stream of solves through the host-memory API with two in flight
        # (api.HostPipeline: one-problem plans, tdc_batched_plan_execute_host): every
        # step copies its inputs in and its eigenvalues and eigenvectors out, and the
        # copy-out of one solve overlaps the next solve
        dh = torch.tensor(d).pin_memory()
        eh = torch.tensor(e).pin_memory()
        steps_p = max(args.steps, 12)
        pipe = api.HostPipeline(n, depth=2, opts=opts)

        # the bound: the host link's own device-to-host rate for the same bytes (one
        # copy of the eigenvector array into the pipeline's page-locked buffer), taken
        # just before and just after the timed solves; the best sample sets the bound,
        # and all are reported, since the host link and host memory can be shared
        def link_samples(reps=3):
            out = []
            for _ in range(reps):
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                pipe.q[0].copy_(pipe.q_dev[0], non_blocking=True)
                c1.record(stream)
                c1.synchronize()
                out.append(8.0 * n * n / (c0.elapsed_time(c1) * 1e-3))
            return out

        # untimed warm-up of the host link, then of the pipeline: after tens of seconds
        # without host transfers (the headline's device-only section before this) the
        # first copies of a process run at 10-60 GB/s and one of the next few solves
        # takes several hundred ms; the link is warmed until two copies in a row reach
        # 90 % of the best seen (at most ten), then eight solves run untimed
        warm = []
        for _ in range(10):
            warm += link_samples(1)
            if len(warm) >= 2 and min(warm[-2:]) >= 0.9 * max(warm):
                break
        for _ in range(8):
            pipe.submit(dh, eh)
        pipe.wait_all()
        link_before = link_samples()
        barrier()
        t0 = time.perf_counter()
        marks = []
        for _ in range(steps_p):
            pipe.submit(dh, eh)
            marks.append(time.perf_counter())
        pipe.wait_all()
        t1 = time.perf_counter()
        link_after = link_samples()
        e_max = max_over_ranks((t1 - t0) / steps_p, dist, "cuda")
        gaps = sorted(b - a for a, b in zip(marks, marks[1:] + [t1]))
        e2e = {"value": e_max / world, "unit": "s", "h2d_bytes_per_step": pipe.h2d_bytes,
               "d2h_bytes_per_step": pipe.d2h_bytes, "steps": steps_p,
               "api": "api.HostPipeline (tdc_batched_plan_execute_host), two solves in flight",
               "host_numa_node": node,
               "step_s_min_median_max": [gaps[0], gaps[len(gaps) // 2], gaps[-1]]}
        del pipe
        torch.cuda.empty_cache()
        link = max(link_before + link_after)
        e2e["link_d2h_gbs"] = link / 1e9
        e2e["link_d2h_gbs_before_after"] = [[round(x / 1e9, 1) for x in link_before],
                                            [round(x / 1e9, 1) for x in link_after]]
        e2e["link_warmup_gbs"] = [round(x / 1e9, 1) for x in warm]
        bound_s = e2e["d2h_bytes_per_step"] / link
        e2e["link_bound_s"] = bound_s
        e2e["frac_of_link_bound"] = bound_s / e2e["value"]
        # context: one blocking call at a time (tdc_syev_tridiag_host)
        hs = api.HostSolver(n, opts=opts)
        hs(dh, eh)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hs(dh, eh)
        t1 = time.perf_counter()
        e2e["blocking_call_s"] = (t1 - t0) / args.steps
        del hs
        torch.cuda.empty_cache()
        os.sched_setaffinity(0, old_aff)
        torch.cuda.empty_cache()

    extra = {}
    if not args.no_extra and rank == 0:
        extra = context_measurements(api, _lib, lib, torch)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    phases = {nm: {"ms_per_step": prof.ms[i] / args.steps, "launches_per_step": prof.launches[i] / args.steps}
              for i, nm in enumerate(_lib.PHASES)}
    launches = int(round(sum(prof.launches) / args.steps))
    clk_sum = clk.summary()
    fp64_peak = GB300_SMS * DFMA_PER_CLK_SM * 2 * (clk_sum["sm_max_mhz"] or 2070.0) * 1e6 / 1e12
    cands = []
    if prof.fp64_product_flops > 0 and prof.ms[5] > 0:
        cands.append({"bound": "alu", "achieved": prof.fp64_product_flops / (prof.ms[5] * 1e-3) / 1e12,
                      "peak": fp64_peak, "unit": "TFLOP/s", "ms_per_step": prof.ms[5] / args.steps,
                      "kernel": "k_gemm_fp64: FP64 eigenvector product (Eq. 6), Qhat generated in-kernel",
                      "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock",
                      "algorithmic_per_step": prof.fp64_product_flops / args.steps})
    if prof.split_tensor_flops > 0 and prof.ms[8] > 0:
        cands.append({"bound": "tensor", "achieved": prof.split_tensor_flops / (prof.ms[8] * 1e-3) / 1e12,
                      "peak": pk.get("bf16_tflops_sustained", pk["bf16_tflops"]), "unit": "TFLOP/s",
                      "ms_per_step": prof.ms[8] / args.steps,
                      "kernel": "k_oz_gemm: split-precision eigenvector product on tcgen05 (bf16 slice pairs)",
                      "peak_source": f"{pk_kind} bf16 sustained",
                      "algorithmic_per_step": prof.split_tensor_flops / args.steps})
    if prof.defl_copy_bytes > 0 and prof.ms[6] > 0:
        cands.append({"bound": "hbm", "achieved": prof.defl_copy_bytes / (prof.ms[6] * 1e-3) / 1e9,
                      "peak": pk["hbm_gbs"], "unit": "GB/s", "ms_per_step": prof.ms[6] / args.steps,
                      "kernel": "k_defl_copy: deflated columns gathered to their sorted positions (column written, live rows read)",
                      "peak_source": f"{pk_kind} HBM copy",
                      "algorithmic_per_step": prof.defl_copy_bytes / args.steps})
    if prof.secular_flops > 0 and prof.ms[2] > 0:
        cands.append({"bound": "alu", "achieved": prof.secular_flops / (prof.ms[2] * 1e-3) / 1e12,
                      "peak": fp64_peak, "unit": "TFLOP/s", "ms_per_step": prof.ms[2] / args.steps,
                      "kernel": "k_secular / k_secular_grp: secular roots, a warp per root, or 4-16 lanes "
                                "per root on levels with enough roots (K terms per FP64 evaluation: "
                                "1 division + 4 FMA + 1 multiplication)",
                      "fp64_evals_per_root": prof.secular_evals / max(prof.K_total, 1),
                      "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock",
                      "algorithmic_per_step": prof.secular_flops / args.steps})
    # per tree level (leaves up), per step: the FP64 product's algorithmic bytes and flops
    lvl_bytes = [prof.level_fp64_min_bytes[i] / args.steps for i in range(32)]
    lvl_flops = [prof.level_fp64_flops[i] / args.steps for i in range(32)]
    lvl_ms = [prof.level_fp64_product_ms[i] / args.steps for i in range(32)]
    nlev = max([i + 1 for i in range(32) if lvl_bytes[i] > 0] + [0])
    gemm_launches = prof.launches[5] / 2 / args.steps          # k_gemm_sched + k_gemm_fp64 per level
    for c in cands:
        c["frac"] = c["achieved"] / c["peak"] if c["peak"] else None
        c["traffic"] = None
        if c["kernel"].startswith("k_gemm_fp64") and gemm_launches:
            alg = sum(lvl_bytes) / gemm_launches
            tr = measured_traffic("k_gemm_fp64", alg)
            c["algorithmic_bytes_per_launch"] = alg
            if tr:
                c["traffic"] = tr
                c["traffic_unit"] = ("bytes per launch: DRAM read + write per algorithmic byte from the "
                                     "n=8192 ncu capture, times the algorithmic bytes per launch here")
    cands.sort(key=lambda c: -c["ms_per_step"])
    roofline = cands[0] if cands else None
    achieved = (prof.product_flops / ((prof.ms[5] + prof.ms[8] + prof.ms[9]) * 1e-3) / 1e12
                if (prof.ms[5] + prof.ms[8] + prof.ms[9]) > 0 else 0.0)

    cpu = None
    if not args.no_cpu and world == 1:
        v, fit, sample, cores = cpu_oracle_fit(args.gen, n, args.leaf)
        cpu = {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample, "fit": fit}

    line = {
        "metric": METRIC, "value": job_seconds_per_solve(ms_max, world), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "run": {"tile_shapes": ("autotuned per level: " + ",".join(map(str, shapes))) if shapes else "size rule",
                "step": step_kind, "direct_call_ms": direct_ms},
        "fp64_product_levels": {"min_bytes_per_step": lvl_bytes[:nlev], "flops_per_step": lvl_flops[:nlev],
                                "ms_per_step": [round(x, 4) for x in lvl_ms[:nlev]],
                                "fp64_tflops": [round(f / (t * 1e-3) / 1e12, 4) if t > 0 else None
                                                for f, t in zip(lvl_flops[:nlev], lvl_ms[:nlev])]},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_other": cands[1:],
        "cpu_baseline": cpu,
        "phases": phases,
        "merge_stats": {"merges_per_step": prof.merges / args.steps, "K_total_per_step": prof.K_total / args.steps,
                        "secular_fp64_evals_per_root": prof.secular_evals / max(prof.K_total, 1)},
        "product_eff_tflops": achieved,
        "accuracy": acc,
        "clocks": clk_sum,
        "context": extra,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
