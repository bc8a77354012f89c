#!/usr/bin/env python3
"""Benchmark of the mixed-precision staggered CG (Sec. 3 of the paper) on one GB300.

A step is one solve of (4 m^2 - D_eo D_oe) x = b to a true FP64 residual of
1e-10 on a 20^3 x 64 lattice (the paper's production shape; synthetic SU(3)
links exp(0.4 i H), m = 0.01, one complex-Gaussian source), FP32 inner
iteration with FP64 reliable updates, through the C ABI (libstag.so).

Printed (rank 0, one JSON line):
  value       CG GFLOP/s = 1212 flop x V/2 sites x iterations / solve time,
              inputs resident in HBM, CUDA events on the solver's stream,
              L2 flushed (256 MiB write) before every timed solve;
  e2e         the same metric through the C ABI with the source in pinned host
              memory and the solution copied back, copies inside the timing;
  roofline    the slower of the two CG kernels against the measured HBM copy
              bandwidth (and, in `nominal`, against ~8 TB/s);
  cpu_baseline the FP64 CPU oracle's CG on a bounded sample of the workload
              (all cores and one thread), and in `configs` the oracle on the
              other configurations (full CGs on 8^4 and 16^3x32, operator
              timings, an extrapolated 48^3x96 solve).
Extra keys give time-to-solution of the mixed, FP16/BF16-storage and plain FP64
solves on the same GPU.

--impl reference times the CPU oracle as the reference arm.
Multi-GPU (torchrun): independent replicas, each rank its own source (weak
scaling); no data-path collective.
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOP/s & HBM GB/s; CG time-to-1e-10 residual, mixed/batched vs FP64"
FLOP_PER_SITE_ITER = 1212     # 2 x 570 (two half operators) + 12 (mass) + 5 x 12 (BLAS-1)
DSLASH_FLOP_PER_SITE = 570    # 8 x 66 (SU(3) x vector) + 7 x 6 (accumulation)
PAPER_TX_CG_GFLOPS = 107.7    # Titan X, mixed CG, 20^3 x 64, one GPU (Table 2 of the paper)
HBM_NOMINAL_GBS = 8000.0      # nominal HBM3e bandwidth (~8 TB/s); the roofline's peak is the measured copy
L2_FLUSH_BYTES = 256 << 20
# NPR contraction per hypercube, as the kernel computes it: the 120 path
# averages W(A, D), A < D (the rest are adjoints or 1), at |A xor D| = n from n
# products with a step link -- 32 copies at n = 1, 48 x 2 + 32 x 3 + 8 x 4 = 224
# products of 3x3 complex matrices (27 complex multiply-adds = 216 flop each)
# for n >= 2 -- and 256 terms of two colour contractions (2 x 12 complex
# multiply-adds) and their product: 224*216 + 256*(24*8 + 6)
NPR_FLOP_PER_HYPERCUBE = 224 * 216 + 256 * (24 * 8 + 6)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lattice", default="20,20,20,64")
    ap.add_argument("--mass", type=float, default=0.01)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    ap.add_argument("--links", default="recon12", choices=["full", "recon12"],
                    help="storage of the reduced-precision links (the FP64 copy is always full)")
    ap.add_argument("--masses", default=None,
                    help="comma-separated masses solved together with every source (overrides --mass; "
                         "the 12-source x 4-mass workload: --nrhs 12 --masses 0.01,0.02,0.03,0.05)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="sources solved together in one call (the 48^3x96 workload uses 16)")
    ap.add_argument("--seed-config", type=int, default=1,
                    help="config number of the input seeds (1000 * config + stream)")
    ap.add_argument("--no-extras", action="store_true",
                    help="profiling runs: skip the comparison solves, the e2e leg and the CPU baseline")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched / 48^3x96 extras (config 2, ragged, config 4, HBM-bound kernels)")
    ap.add_argument("--probe", default=None, choices=["npr", "hyp"],
                    help="time only the NPR contraction or the HYP smearing on --lattice (profiling runs); "
                         "prints one JSON line")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def link_mb(L, prec, links):
    """MB of the inner-precision link field (both parities, 4 directions)."""
    cb = {"fp64": 16, "fp32": 8, "fp16": 4, "bf16": 4}[prec]
    return 4 * math.prod(L) * (6 if links == "recon12" else 9) * cb / 1e6


def mass_str(mass):
    return ",".join(f"{m:g}" for m in mass) if isinstance(mass, (list, tuple)) else f"{mass:g}"


def l2_note(L, prec, links, l2_persisting):
    """What the L2 holds during the timed solves (the launch form decides)."""
    mb = link_mb(L, prec, links)
    head = "flushed before every timed solve (256 MiB write); "
    if l2_persisting == "vectors":
        return head + (f"during the solve the Krylov vectors r, x, p, t are an L2 access-policy window whose "
                       f"lines persist; the links ({mb:.0f} MB) stream; persisting lines are released after "
                       "every solve")
    if l2_persisting in (True, "links"):
        return head + (f"during the solve the inner-precision links ({mb:.0f} MB) are an L2 access-policy "
                       "window whose lines persist (set-aside ~85 MB of the 129 MB L2), so most of the two "
                       "link passes per iteration hit L2; the vectors stream; persisting lines are released "
                       "after every solve")
    return head + (f"the links ({mb:.0f} MB) and vectors stream through L2 with no persistence window")


def workload_config(L, mass, tol, prec, links="full", nrhs=1, l2_persisting=False):
    return {
        "link_storage": ("reconstruct-12 (rows 0, 1 stored; row 2 = conj(row0 x row1) in registers)"
                         if links == "recon12" else "full 3x3") + f" at {prec.upper()}; FP64 copy full",
        "workload": f"{L[0]}^3x{L[3]} even-odd staggered CG, {prec.upper()} inner iteration, "
                    f"FP64 reliable updates (delta=0.1), m={mass_str(mass)}, {nrhs} RHS, true residual {tol:g}"
        if L[0] == L[1] == L[2] else f"{L} staggered CG",
        "lattice": list(L),
        "links": "reunitarised exp(0.4 i H), synthetic (stands in for the MILC 20^3x64 ensemble)",
        "mass": mass,
        "tol": tol,
        "inner_precision": prec,
        "reliable_update": "f64",
        "l2": l2_note(L, prec, links, l2_persisting),
        "graph": "one CUDA graph launch per solve (conditional WHILE/IF nodes)",
    }


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the single-system FP32 CG kernels (the
    traffic figures of an ncu capture stand only for the code they measured)."""
    h = hashlib.sha256()
    for f in ("stag_kernels.cuh", "dslash_p32.cu", "dslash_inst.cuh"):
        with open(os.path.join(ROOT, "paper_1511_00088_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(key):
    """DRAM bytes per launch of `key` from the committed ncu summary, when it was
    taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    cur = kernel_source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == key and parts[1] == cur:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def whole_job(dist, ms_step, flops_step, device):
    """Whole-job numbers of the replicas: the step time is the slowest rank's
    (max over ranks), the work is every rank's (sum); without a process group
    the rank's own.  Returns (ms_per_step, flops_per_step, GFLOP/s)."""
    flops_all = flops_step
    if dist is not None:
        import torch
        t = torch.tensor([ms_step], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
        f = torch.tensor([flops_step], device=device, dtype=torch.float64)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
        flops_all = float(f.item())
    return ms_step, flops_all, flops_all / (ms_step * 1e-3) / 1e9


def sum_over_ranks(dist, value, device):
    """A throughput summed over the replicas (None stays None)."""
    if dist is None or value is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_oracle_sample(L, U, b, mass, budget_s, threads=1):
    """The FP64 oracle's CG for a bounded number of iterations on this workload,
    single-threaded or (threads = 0: every host core) with the all-core build
    (only the operator's per-site loop parallel; results bit-identical).
    Returns (GFLOP/s, iterations, seconds, threads used)."""
    import oracle

    def run():
        t = time.perf_counter()
        oracle.mdagm(L, U, mass, b)
        t1 = time.perf_counter() - t
        n = max(2, int(budget_s / max(t1, 1e-3)))
        t = time.perf_counter()
        _, st, it, _ = oracle.cg(L, U, mass, b, tol=1e-300, maxiter=n)
        return it, time.perf_counter() - t

    if threads == 1:
        used = 1
        it, dt = run()
    else:
        with oracle.threads(threads) as th:
            used = th.count()
            it, dt = run()
    Ve = (L[0] * L[1] * L[2] * L[3]) // 2
    # the oracle also recomputes the true residual once (one more operator application)
    gflops = FLOP_PER_SITE_ITER * Ve * it / dt / 1e9
    return gflops, it, dt, used


def cpu_oracle_configs(fp64_iters_48x96):
    """The FP64 CPU oracle on the machine's host cores, per configuration: a full
    CG on 8^4 (one thread and all cores), the half operator and M^dag M on
    20^3x64, a full CG on 16^3x32 (m = 0.02, all cores), and on 48^3x96 one
    M^dag M plus 10 CG iterations, extrapolated to a whole solve by the GPU FP64
    solve's iteration count (a full CPU solve there would take hours).  A
    baseline only: the oracle is plain, untuned code."""
    import oracle
    import torch

    from paper_1511_00088_gb300 import synth
    out = {}

    def cg_run(L, U, b, m, tol=1e-10, maxiter=100000):
        t = time.perf_counter()
        _, st, it, _ = oracle.cg(L, U, m, b, tol=tol, maxiter=maxiter)
        dt = time.perf_counter() - t
        Ve = synth.volume(L) // 2
        return {"s": dt, "iters": int(it), "GFLOP/s": FLOP_PER_SITE_ITER * Ve * it / dt / 1e9}

    with oracle.threads(0) as th:
        cores = th.count()
    L = (8, 8, 8, 8)
    U = synth.random_links(L, 0.3, synth.seed_for(0, 1))
    b = synth.gaussian_vector(synth.volume(L) // 2, synth.seed_for(0, 2))
    c0 = {"one_thread": cg_run(L, U, b, 0.05)}
    with oracle.threads(0):
        c0["all_cores"] = cg_run(L, U, b, 0.05)
    out["config0_8^4_m0.05_fp64_cg_to_1e-10"] = c0
    L = (20, 20, 20, 64)
    Ve = synth.volume(L) // 2
    U = synth.random_links(L, 0.4, synth.seed_for(1, 1))
    b = synth.gaussian_vector(Ve, synth.seed_for(1, 2))
    c1 = {}
    for label, n in (("one_thread", 1), ("all_cores", 0)):
        with oracle.threads(n) if n != 1 else contextlib.nullcontext():
            t = time.perf_counter()
            oracle.dslash_oe(L, U, b)
            t1 = time.perf_counter() - t
            t = time.perf_counter()
            oracle.mdagm(L, U, 0.01, b)
            t2 = time.perf_counter() - t
        c1[label] = {"dslash_oe_ms": 1e3 * t1, "dslash_oe_GFLOP/s": 570 * Ve / t1 / 1e9,
                     "mdagm_ms": 1e3 * t2, "mdagm_GFLOP/s": (2 * 570 + 12) * Ve / t2 / 1e9}
    out["config1_20^3x64_operator"] = c1
    L = (16, 16, 16, 32)
    U = synth.random_links(L, 0.4, synth.seed_for(3, 1))
    b = synth.gaussian_vector(synth.volume(L) // 2, synth.seed_for(3, 2))
    with oracle.threads(0):
        out["config3_16^3x32_m0.02_fp64_cg_to_1e-10"] = {"all_cores": cg_run(L, U, b, 0.02)}
    if fp64_iters_48x96:
        L = (48, 48, 48, 96)
        Ve = synth.volume(L) // 2
        Ud = synth.random_links_device(L, 0.4, synth.seed_for(4, 1), device="cuda")
        U = Ud.cpu().numpy()
        del Ud
        torch.cuda.empty_cache()
        b = synth.gaussian_vector(Ve, synth.seed_for(4, 2))
        with oracle.threads(0):
            t = time.perf_counter()
            oracle.mdagm(L, U, 0.005, b)
            t_m = time.perf_counter() - t
            r10 = cg_run(L, U, b, 0.005, tol=1e-300, maxiter=10)
        per_it = r10["s"] / max(r10["iters"], 1)
        out["config4_48^3x96_m0.005"] = {
            "all_cores": {"mdagm_s": t_m, "cg_10_iterations_s": r10["s"], "GFLOP/s": r10["GFLOP/s"]},
            "extrapolated_one_source_s": per_it * fp64_iters_48x96,
            "extrapolated_16_sources_s": 16 * per_it * fp64_iters_48x96,
            "iterations_used": fp64_iters_48x96}
        del U
    return out, cores


def timed_solve(ctx, srcs, masses, prec, tol, maxiter, stream):
    """One solve timed with CUDA events on the solver's stream, after an
    untimed 16-iteration call that tunes the launch form and builds the graph.
    Returns a dict of time, iterations and worst true residual."""
    import torch

    from paper_1511_00088_gb300 import stag
    ctx.cg_solve(srcs, masses, tol=tol, maxiter=16, precision=prec, allow_not_converged=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xs, st, it, tr = ctx.cg_solve(srcs, masses, tol=tol, maxiter=maxiter, precision=prec,
                                  allow_not_converged=True)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    Ve = ctx.Ve
    return {"ms": ms, "systems": len(it), "iters_max": int(max(it)), "iters_sum": int(sum(it)),
            "true_res_max": float(max(tr)), "status": stag.status_name(st),
            "TFLOP/s": FLOP_PER_SITE_ITER * Ve * float(sum(it)) / (ms * 1e-3) / 1e12,
            "launch_form": ctx.solve_form()}


def batched_extras(stream, hbm):
    """Driver-visible numbers of the batched workloads and the HBM-bound
    lattice: 12 sources x 4 masses on 20^3x64 (FP32 and FP16/BF16 Krylov
    vectors, FP32 reconstruct-12 links), the ragged batch of four lattices in
    one graph, and on 48^3x96 the two CG kernels at one source (links far
    larger than L2: algorithmic bytes / time is DRAM-honest there) and the
    16-source m = 0.005 solve against one FP64 single-source solve."""
    import torch

    from paper_1511_00088_gb300 import stag, synth
    out = {}
    tol = 1e-10
    V32 = stag.STAG_FP32
    # configuration 2: 12 sources x 4 masses on 20^3 x 64
    L = (20, 20, 20, 64)
    V = synth.volume(L)
    U = torch.from_numpy(synth.random_links(L, 0.4, synth.seed_for(2, 1))).cuda()
    bs = [torch.from_numpy(synth.gaussian_vector(V // 2, synth.seed_for(2, 100 + r))).cuda() for r in range(12)]
    masses = [0.01, 0.02, 0.03, 0.05]
    c2 = {}
    with stag.Context(L, recon12=True, stream=stream.cuda_stream) as ctx:
        ctx.links_upload(U)
        for name, p in (("fp32", V32), ("fp32_links_fp16_vectors", V32 | stag.STAG_VEC_FP16),
                        ("fp32_links_bf16_vectors", V32 | stag.STAG_VEC_BF16)):
            c2[name] = timed_solve(ctx, bs, masses, p, tol, 40000, stream)
        c2["fp64_one_system_m0.01"] = timed_solve(ctx, bs[:1], masses[:1], stag.STAG_FP64, tol, 40000, stream)
        # the same 48 systems by the multi-shift CG (the 4 masses of a source on
        # one Krylov space, then each refined from that solution)
        ctx.cg_solve_multishift(bs, masses, tol=tol, maxiter=16, precision=V32, allow_not_converged=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st, it, tr = ctx.cg_solve_multishift(bs, masses, tol=tol, maxiter=40000, precision=V32,
                                                allow_not_converged=True)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        c2["fp32_multishift"] = {"ms": ms, "systems": len(it), "iters_max": int(max(it)),
                                 "iters_sum": int(sum(it)), "true_res_max": float(max(tr)),
                                 "status": stag.status_name(st)}
        # the full-lattice equation M x = b (one source, m = 0.01) and HYP smearing of the field
        bfull = torch.from_numpy(synth.gaussian_vector(V, synth.seed_for(2, 300))).cuda()
        ctx.solve_full([bfull], [0.01], tol=tol, maxiter=16, precision=V32, allow_not_converged=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, st, it, tr = ctx.solve_full([bfull], [0.01], tol=tol, maxiter=40000, precision=V32)
        e1.record(stream)
        e1.synchronize()
        out["full_lattice_solve_20x64_m0.01"] = {"ms": e0.elapsed_time(e1), "iters": int(it[0]),
                                                 "true_res": float(tr[0]), "status": stag.status_name(st)}
        H = ctx.hyp_smear(U)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.hyp_smear(U, out=H)
        e1.record(stream)
        e1.synchronize()
        out["hyp_smear_20x64_fp64"] = {"ms": e0.elapsed_time(e1), "links": 4 * V}
        del H
        # the NPR one-colour-trace four-fermion contraction (Sec. 4, FP64) on the
        # same field: four Gaussian colour-vector fields, spin-taste (S1,F1,S2,F2)
        # = (15, 0, 15, 0); flops by the kernel's arithmetic per hypercube
        fs = [torch.from_numpy(synth.gaussian_vector(V, synth.seed_for(2, 400 + k))).cuda() for k in range(4)]
        ctx.npr_contract((15, 0, 15, 0), *fs)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.npr_contract((15, 0, 15, 0), *fs)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out["npr_contraction_20x64_fp64"] = {"ms": ms, "hypercubes": V // 16,
                                             "GFLOP/s": NPR_FLOP_PER_HYPERCUBE * (V // 16) / (ms * 1e-3) / 1e9,
                                             "flop_per_hypercube": NPR_FLOP_PER_HYPERCUBE}
    out["config2_12src_x_4mass_20x64"] = c2
    del U, bs
    # the ragged batch: one source x the 4 masses on each of four lattices, one graph
    ctxs, batch = [], []
    try:
        for n, Lr in enumerate([(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (20, 20, 20, 64)]):
            Vr = synth.volume(Lr)
            c = stag.Context(Lr, recon12=True, stream=stream.cuda_stream)
            c.links_upload(torch.from_numpy(synth.random_links(Lr, 0.4, synth.seed_for(2, 10 * n + 1))).cuda())
            ctxs.append(c)
            batch.append((c, [torch.from_numpy(synth.gaussian_vector(Vr // 2, synth.seed_for(2, 10 * n + 2)))
                              .cuda()], masses))
        stag.cg_solve_ragged(batch, tol=tol, maxiter=16, precision=V32, allow_not_converged=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st, its, trs = stag.cg_solve_ragged(batch, tol=tol, maxiter=40000, precision=V32,
                                               allow_not_converged=True)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        flop = sum(FLOP_PER_SITE_ITER * c.Ve * float(sum(it)) for c, it in zip(ctxs, its))
        out["ragged_4_lattices_4_masses"] = {
            "lattices": [list(c.dims) for c in ctxs], "sites": sum(c.V for c in ctxs), "ms": ms,
            "iters_max": int(max(max(it) for it in its)), "true_res_max": float(max(max(t) for t in trs)),
            "status": stag.status_name(st), "TFLOP/s": flop / (ms * 1e-3) / 1e12}
    finally:
        for c in ctxs:
            c.close()
    # 48^3 x 96: HBM-bound kernels and configuration 4
    L = (48, 48, 48, 96)
    V = synth.volume(L)
    U = synth.random_links_device(L, 0.4, synth.seed_for(4, 1), device="cuda")
    with stag.Context(L, recon12=True, stream=stream.cuda_stream) as ctx:
        ctx.links_upload(U)
        del U
        kern = {}
        for name, p in (("fp32", V32), ("fp32_links_bf16_vectors", V32 | stag.STAG_VEC_BF16)):
            for kk in (0, 1):
                ms_k, by_k = ctx.time_cg_kernel(kk, p, nlaunch=50)
                gbs = by_k / (ms_k * 1e-3) / 1e9
                kern[f"{name}_k{kk + 1}"] = {"ms_per_launch": ms_k, "algorithmic_bytes_per_launch": by_k,
                                            "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm}
        out["hbm_bound_48x96_one_source"] = kern
        bs = [torch.from_numpy(synth.gaussian_vector(V // 2, synth.seed_for(4, 2 + r))).cuda() for r in range(16)]
        c4 = {"mixed_fp32_r12_16src": timed_solve(ctx, bs, [0.005], V32, tol, 40000, stream),
              "fp64_one_source": timed_solve(ctx, bs[:1], [0.005], stag.STAG_FP64, tol, 40000, stream)}
        c4["speedup_per_source_vs_fp64"] = c4["fp64_one_source"]["ms"] / (c4["mixed_fp32_r12_16src"]["ms"] / 16)
        out["config4_48x96_16src_m0.005"] = c4
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    from paper_1511_00088_gb300 import synth
    L = tuple(int(v) for v in args.lattice.split(","))
    V = synth.volume(L)
    U = synth.random_links(L, 0.4, synth.seed_for(1, 1))
    b = synth.gaussian_vector(V // 2, synth.seed_for(1, 2))
    vals, times = [], []
    for i in range(args.warmup + args.steps):
        g, it, dt, used = cpu_oracle_sample(L, U, b, args.mass, 6.0, threads=0)
        if i >= args.warmup:
            vals.append(g)
            times.append(dt)
    value = statistics.mean(vals)
    sample = (f"{it} FP64 CG iterations of the CPU oracle per step on the {L} field, {used} threads "
              f"(all host cores; the operator's per-site loop in parallel)")
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": workload_config(L, args.mass, args.tol, "fp64"),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": used, "kind": "oracle",
                         "sample": sample, "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1511_00088_gb300 import build as B
    from paper_1511_00088_gb300 import stag, synth

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    stag.load()
    prec = stag.PRECISIONS[args.precision]
    L = tuple(int(v) for v in args.lattice.split(","))
    V = synth.volume(L)
    Ve = V // 2
    cfg = args.seed_config
    if V > (1 << 22):  # the numpy eigendecomposition is slow at this size: same recipe on the GPU
        Ud = synth.random_links_device(L, 0.4, synth.seed_for(cfg, 1), device="cuda")
        U = None
    else:
        U = synth.random_links(L, 0.4, synth.seed_for(cfg, 1))
        Ud = torch.from_numpy(U).cuda()
    nrhs = args.nrhs
    masses = [float(m) for m in args.masses.split(",")] if args.masses else [args.mass]
    nsys = nrhs * len(masses)
    bs = [synth.gaussian_vector(Ve, synth.seed_for(cfg, 2 + rank * nrhs + r)) for r in range(nrhs)]
    b = bs[0]
    stream = torch.cuda.current_stream()
    ctx = stag.Context(L, recon12=(args.links == "recon12"), stream=stream.cuda_stream)
    ctx.links_upload(Ud)
    bds = [torch.from_numpy(v).cuda() for v in bs]
    xds = [torch.empty_like(bds[0]) for _ in range(nsys)]
    bd, xd = bds[0], xds[0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def solve():
        xs, st, it, tr = ctx.cg_solve(bds, masses, tol=args.tol, maxiter=50000,
                                      precision=prec, xs=xds)
        return [int(v) for v in it], float(max(tr))

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    dev_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    clocks = ClockSampler(dev_index)
    clocks.start()
    total_ms, iters, updates, launches, res, step_ms = 0.0, [], [], 0, [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, tr = solve()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        total_ms += step_ms[-1]
        _, nu, _ = ctx.solve_stats(0)
        passes, ups = ctx.solve_counters()
        unroll = ctx.solve_form()["iterations_per_pass"]
        iters.append(it)
        updates.append(nu)
        res.append(tr)
        # one pack per source and mass, init + its finalize, one unpack per
        # system; per loop pass 2 CG kernels per iteration and one finalize
        # (the multi-RHS form: a finalize after each CG kernel); per update
        # step 5 kernels
        per_pass = 4 * unroll if ctx.solve_form()["kernels"] == "k_cg_nrhs" else 2 * unroll + 1
        launches += 2 * nsys + 2 + per_pass * passes + 5 * ups
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    form = ctx.solve_form()
    ms_step = total_ms / args.steps
    flops_step = FLOP_PER_SITE_ITER * Ve * statistics.mean(sum(i) for i in iters)
    ms_step, flops_all, value = whole_job(dist, ms_step, flops_step, "cuda")

    # end to end through the C ABI with host buffers (pinned), copies inside
    bhs = [torch.from_numpy(v).pin_memory() for v in bs]
    xhs = [torch.empty_like(bhs[0]).pin_memory() for _ in range(nsys)]
    e2e_ms, e2e_it = [], []
    for k in range(0 if args.no_extras else max(1, min(args.steps, 5))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t = time.perf_counter()
        xs, st, it, tr = ctx.cg_solve(bhs, masses, tol=args.tol, maxiter=50000,
                                      precision=prec, xs=xhs)
        e2e_ms.append(1e3 * (time.perf_counter() - t))
        e2e_it.append(int(sum(it)))
    e2e_ms_step = statistics.mean(e2e_ms) if e2e_ms else None
    e2e_value = (FLOP_PER_SITE_ITER * Ve * statistics.mean(e2e_it) / (e2e_ms_step * 1e-3) / 1e9
                 if e2e_ms else None)
    e2e_value = sum_over_ranks(dist, e2e_value, "cuda")

    # the two CG kernels, timed alternately as the iteration runs them (CUDA
    # events between launches); the roofline is reported for the slower one
    hbm, peak_kind = peaks()
    # the key names the workload the kernels ran: a capture's traffic stands only
    # for the same kernels on the same lattice and number of systems
    tag = f"{args.precision}{'_r12' if args.links == 'recon12' else ''}_{'x'.join(map(str, L))}"
    if nsys > 1:
        tag += f"_{nsys}sys_{form['kernels']}"
    kern = []
    for kk, what in ((0, "t = D_oe r + beta t_old, |t|^2"),
                     (1, "p = r + beta p; r -= alpha (4m^2 p - D_eo t); x += alpha p; |r|^2, Re<r,p>")):
        ms_k, by_k = ctx.time_cg_kernel(kk, prec, nlaunch=100)
        kern.append({"kernel": f"{form['kernels']} CG kernel {kk + 1}: {what} ({args.precision}, links {args.links}, "
                               f"{nsys} systems)",
                     "key": f"cg_k{kk + 1}_{tag}", "ms_per_launch": ms_k, "algorithmic_bytes_per_launch": by_k,
                     "achieved": by_k / (ms_k * 1e-3) / 1e9})
    dom = max(kern, key=lambda d: d["ms_per_launch"])
    other = kern[1 - kern.index(dom)]
    traffic = ncu_traffic(dom["key"])
    roof = {"bound": "hbm", "achieved": dom["achieved"], "peak": hbm, "unit": "GB/s",
            "frac": dom["achieved"] / hbm, "traffic": traffic, "peak_source": peak_kind,
            # the nominal figure (~8 TB/s HBM3e) beside the measured copy peak
            "nominal": {"peak": HBM_NOMINAL_GBS, "frac": dom["achieved"] / HBM_NOMINAL_GBS},
            # the ncu DRAM bytes of one launch over its live time: the DRAM side
            # of the effective (algorithmic) fraction, the rest being L2 hits
            "dram_gbs": traffic / (dom["ms_per_launch"] * 1e-3) / 1e9 if traffic else None,
            "dram_frac": traffic / (dom["ms_per_launch"] * 1e-3) / 1e9 / hbm if traffic else None,
            "kernel": dom["kernel"],
            "ms_per_launch": dom["ms_per_launch"],
            "algorithmic_bytes_per_launch": dom["algorithmic_bytes_per_launch"],
            "other_kernel": {"kernel": other["kernel"], "ms_per_launch": other["ms_per_launch"],
                             "achieved": other["achieved"], "frac": other["achieved"] / hbm,
                             "traffic": ncu_traffic(other["key"])}}

    extras = {}
    if not args.no_extras and rank == 0:
        # single-source solves of the first source at the other precisions (with
        # several sources: the FP64 and FP32 single-source references only)
        # fp16 / bf16: FP32 links (the bench's link format) with the Krylov
        # vectors p, D_oe p stored at FP16 / BF16; *_links: the links
        # themselves rounded to FP16 / BF16 (vectors FP32) -- BF16 links stall
        # at small masses, so that leg is capped at 5000 iterations
        cmp = ((("fp64", stag.STAG_FP64, 30000), ("fp32", stag.STAG_FP32, 30000),
                ("fp16", stag.STAG_FP32 | stag.STAG_VEC_FP16, 30000),
                ("bf16", stag.STAG_FP32 | stag.STAG_VEC_BF16, 30000),
                ("fp16_links", stag.STAG_FP16, 30000), ("bf16_links", stag.STAG_BF16, 5000))
               if nsys == 1 else (("fp64", stag.STAG_FP64, 30000), ("fp32", stag.STAG_FP32, 30000)))
        for name, p, cap in cmp:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xs, st, it, tr = ctx.cg_solve([bd], masses[:1], tol=args.tol, maxiter=cap, precision=p,
                                          xs=[xd], allow_not_converged=True)
            e1.record(stream)
            e1.synchronize()
            _, nu, _ = ctx.solve_stats(0)
            extras[f"cg_{name}"] = {"ms": e0.elapsed_time(e1), "iters": int(it[0]),
                                    "reliable_updates": nu, "true_res": float(tr[0]),
                                    "status": stag.status_name(st)}
        for name, p in ((("fp64", stag.STAG_FP64), ("fp16", stag.STAG_FP16), ("bf16", stag.STAG_BF16))
                        if nsys == 1 else ()):
            m, by = ctx.time_dslash(p, nlaunch=50)
            extras[f"dslash_{name}"] = {"ms": m, "GB/s": by / (m * 1e-3) / 1e9,
                                        "GFLOP/s": DSLASH_FLOP_PER_SITE * Ve / (m * 1e-3) / 1e9}
        # FP64 single-source time over the timed solve's time per source
        extras["mixed_vs_fp64_speedup"] = extras["cg_fp64"]["ms"] / (total_ms / args.steps / nsys)
        if not args.no_batched and nsys == 1 and L == (20, 20, 20, 64):
            extras["batched"] = batched_extras(stream, hbm)

    cpu = None
    if ws == 1 and rank == 0 and not args.no_extras:
        if U is None:
            U = Ud.cpu().numpy()
        g1, it1, dt1, _ = cpu_oracle_sample(L, U, b, masses[0], 10.0, threads=1)
        g, it, dt, used = cpu_oracle_sample(L, U, b, masses[0], 10.0, threads=0)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": used, "kind": "oracle", "nproc": os.cpu_count(),
               "sample": f"{it} FP64 CG iterations of the CPU oracle on the same {L} field "
                         f"({dt:.1f} s, {used} threads: the operator's per-site loop in parallel)",
               "single_thread": {"value": g1, "unit": "GFLOP/s", "cores": 1,
                                 "sample": f"{it1} FP64 CG iterations ({dt1:.1f} s, one thread)"}}
        if "batched" in extras:
            c4 = extras["batched"].get("config4_48x96_16src_m0.005", {}).get("fp64_one_source", {})
            cpu["configs"], _ = cpu_oracle_configs(c4.get("iters_max"))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / PAPER_TX_CG_GFLOPS,
            "dtype": "f32" if args.precision == "fp32" else args.precision.replace("fp", "f"),
            "data": "synthetic",
            "config": workload_config(L, masses, args.tol, args.precision, args.links, nrhs,
                                      form["l2_persisting"]),
            "time_to_solution_ms": ms_step,
            "time_to_solution_ms_best": min(step_ms), "time_to_solution_ms_median": statistics.median(step_ms),
            "iters": iters[-1] if nsys > 1 else iters[-1][0],
            "reliable_updates": updates[-1],
            "true_res": max(res),
            "e2e": {"value": e2e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": 48 * Ve * nrhs,
                    "d2h_bytes_per_step": 48 * Ve * nsys, "ms_per_step": e2e_ms_step},
            "gpu_launches": launches,
            "launch_form": form,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_probe(args):
    """--probe: time one FP64 side workload of the paper on --lattice: the NPR
    contraction (Sec. 4; spin-taste (15, 0, 15, 0), four Gaussian fields) or
    the HYP smearing of the field (Sec. 3's smeared links)."""
    import torch

    from paper_1511_00088_gb300 import build as B
    from paper_1511_00088_gb300 import stag, synth
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    B.build()
    stag.load()
    L = tuple(int(v) for v in args.lattice.split(","))
    V = synth.volume(L)
    U = (synth.random_links_device(L, 0.4, synth.seed_for(2, 1), device="cuda") if V > (1 << 22)
         else torch.from_numpy(synth.random_links(L, 0.4, synth.seed_for(2, 1))).cuda())
    stream = torch.cuda.current_stream()
    with stag.Context(L, stream=stream.cuda_stream) as ctx:
        ctx.links_upload(U)
        if args.probe == "npr":
            fs = [torch.from_numpy(synth.gaussian_vector(V, synth.seed_for(2, 400 + k))).cuda() for k in range(4)]
            op = lambda: ctx.npr_contract((15, 0, 15, 0), *fs)  # noqa: E731
        else:
            H = torch.empty_like(U)
            op = lambda: ctx.hyp_smear(U, out=H)  # noqa: E731
        for _ in range(args.warmup):
            op()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            op()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
    line = {"probe": args.probe, "lattice": list(L), "ms": ms, "steps": args.steps, "warmup": args.warmup}
    if args.probe == "npr":
        line["GFLOP/s"] = NPR_FLOP_PER_HYPERCUBE * (V // 16) / (ms * 1e-3) / 1e9
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.probe:
        return run_probe(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
