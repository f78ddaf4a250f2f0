#!/usr/bin/env python
"""Benchmark of the GB300 photoacoustic operator: FISTA at 128^2 x 64 depths x 256 samples.

Workload (one step): a 100-iteration non-negative least-squares FISTA
reconstruction (Eq. 12-15) of one synthetic vessel volume, 128 x 128 voxels
zero-padded to 256 x 256, 64 depths, 256 time samples, dx = 50 um, dt = 10 ns,
c = 1500 m/s, data y = H p0 + 5 % Gaussian noise. Every iteration applies H
and H* once (one A+A^T pair), so `value` is FISTA iterations/s = pairs/s of
the whole job (all ranks). The impulse-response library is generated on the
device from the k-space solution (real spectra: the real-even table path).

Also reported: the bare A+A^T pair rate, the plain single-precision path
(complex64 table, same kernels otherwise), a live CUDA-event roofline of the
dominant kernel (the depth contraction), an end-to-end rate through the C ABI
with host buffers, the clocks seen while timing, and the CPU oracle's rate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--mode freq-shard]
Under torchrun every rank reconstructs its own volume (independent problems,
weak scaling, no collective on the data path); rank 0 prints one JSON line.
With --mode freq-shard the ranks instead share one reconstruction: each holds
1/N of the table's rows, 1/N of the depth slices and 1/N of the time samples,
with an all-to-all of slice spectra (NCCL) at each stage boundary (strong
scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A+Aᵀ pairs/s & FISTA it/s at 128²×64z×256t vs plain FP32; serve p50/p99"
N, NZ, NT, P = 128, 64, 256, 256
DX, DT, C0 = 50e-6, 10e-9, 1500.0
MZ, Z0 = 256, 1
ITERS = 100
WORKLOAD = (f"FISTA-{ITERS} NNLS, {N}x{N} (padded {P}x{P}) x {NZ} depths x {NT} samples, "
            f"dx={DX * 1e6:.0f}um dt={DT * 1e9:.0f}ns, vessel phantom + 5% noise")


def folded_table_bytes(radial: bool = True) -> int:
    """Bytes of the benchmark's resident library: real f32 spectra of the
    256 x 256 grid stored in chunks of 32 rows, 4 depths per 16-byte group (the
    plan's layout). One row per D4 representative {|kx|, |ky|}, or (radial)
    one row per group of representatives with equal kx^2 + ky^2 (the k-space
    library depends on |k| only)."""
    h = P // 2
    reps = [(a, b) for a in range(h + 1) for b in range(a, h + 1)]
    chunks = (len(reps) + 31) // 32
    if radial:  # radii grouped by their number of representatives, 32 radii per chunk
        per_radius = {}
        for a, b in reps:
            per_radius[a * a + b * b] = per_radius.get(a * a + b * b, 0) + 1
        sizes = {}
        for m in per_radius.values():
            sizes[m] = sizes.get(m, 0) + 1
        chunks = min(chunks, sum((n + 31) // 32 for n in sizes.values()))
    return chunks * NT * ((NZ + 3) // 4) * 32 * 16


def bench_config() -> dict:
    """`config` of the JSON line; both arms print this same dict."""
    tb = folded_table_bytes() / 1e9
    td4 = folded_table_bytes(radial=False) / 1e9
    return {"workload": WORKLOAD,
            "table": f"real f32 spectra generated on device, one stored row per group of D4 "
                     f"representatives {{|kx|,|ky|}} with equal kx^2+ky^2 ({tb:.2f} GB; "
                     f"{td4:.2f} GB with one row per representative)",
            "l2": f"no flush: the table streamed every pass is {tb:.2f} GB > 129 MB L2",
            "per_rank": "one volume per rank"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="wall time of the CPU-oracle sample")
    ap.add_argument("--mode", default="volumes", choices=["volumes", "freq-shard"],
                    help="volumes: one independent volume per rank; freq-shard: one volume "
                         "with the operator split over the ranks by frequency rows")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="arrival window of the serving measurement (0 = skip)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist


def max_over_ranks(value: float, world: int, device) -> float:
    """Largest value over all ranks (the job's wall time is the slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
                 "200", "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        for line in open(path):
            f = line.strip().strip("|").split("|")
            if len(f) >= 2 and f[0].strip() == kernel:
                return float(f[1])
    except (OSError, ValueError):
        pass
    return None


# ----------------------------------------------------------------------------- workload
def make_inputs(seed: int):
    """Phantom and 5 % noise (host, float64) for one volume."""
    from paper_2603_28150_gb300 import synth
    p0 = synth.vessel_phantom(N, NZ, seed=seed)
    noise = synth.gaussian_field((NT, N, N), seed=seed + 1000)
    return p0, noise


def events_ms(fn, reps: int) -> float:
    import torch
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def graph_ms(fn, reps: int, replays: int = 5) -> float:
    """Device time of one call of `fn`, from `reps` calls captured in one CUDA
    graph and replayed (no host launch overhead between the calls)."""
    import torch
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            for _ in range(reps):
                fn()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(replays):
        g.replay()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / (reps * replays)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2603_28150_gb300 import Medium, Plan

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")
    med = Medium(C0, DX, DX, DX, DT, MZ, Z0)
    plan = Plan(N, N, NZ, NT, P, P, medium=med)
    info = plan.info()
    p0, noise = make_inputs(seed=rank)
    p0_d = torch.tensor(p0, dtype=torch.float32, device=dev)
    clean = plan.forward(p0_d)
    sigma = 0.05 * float(torch.sqrt(torch.mean(clean.double() ** 2)))
    y = (clean + sigma * torch.tensor(noise, dtype=torch.float32, device=dev)).contiguous()
    v0 = torch.ones((NZ, N, N), dtype=torch.float32, device=dev)
    L = 1.01 * plan.power_norm(v0, 50)

    x = torch.empty((NZ, N, N), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        plan.fista(y, x=x, iters=ITERS, L=L)
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(s)
        rep = None
        for _ in range(args.steps):
            _, rep = plan.fista(y, x=x, iters=ITERS, L=L)
        e1.record(s)
        torch.cuda.synchronize()
    barrier(world)
    t_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = t_ms / args.steps
    value = world * args.steps * ITERS / (t_ms / 1e3)
    launches = rep["kernels_per_iter"] * ITERS * args.steps

    # bare A + A^T pairs (gradient of Eq. 15, device buffers)
    g = torch.empty_like(x)
    pair_ms = events_ms(lambda: plan.gradient(p0_d, y, out=g, resid=False), 20)

    # dominant kernel: the depth contraction, timed alone with CUDA events
    Kp = info["bins_padded"]
    Xb = torch.zeros((NZ, Kp), dtype=torch.complex64, device=dev)
    Yb = torch.zeros((NT, Kp), dtype=torch.complex64, device=dev)
    plan.stage_contract(Xb, Yb)  # warm
    fwd_ms = events_ms(lambda: plan.stage_contract(Xb, Yb), 20)
    adj_ms = events_ms(lambda: plan.stage_contract(Yb, Xb, adjoint=True), 20)
    K = info["bins"]
    assert info["table_bytes"] == folded_table_bytes() and info["radial"] == 1
    d4_bytes = folded_table_bytes(radial=False)
    # algorithmic bytes of one application: the stored table once, plus the
    # operator's input and output (rho 4 B per voxel, d 4 B per sample); the
    # spectra X and Y between the stages are implementation traffic
    rho_b, d_b = NZ * N * N * 4, NT * N * N * 4
    algo = info["table_bytes"] + rho_b + d_b
    algo_spectra = info["table_bytes"] + (NZ + NT) * K * 8  # table + X in + Y out (complex64)
    kname = "k_fold_fwd" if info["folded"] else "k_contract_fwd"
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured"
    if not hbm:
        hbm, peak_src = 6800.0, "fallback"
    achieved = algo / (fwd_ms / 1e3) / 1e9
    iter_bytes = 2 * algo + 5 * rho_b  # A + A^T + the FISTA step's vectors

    # every stage of one A + A^T pair on its own (20 calls in a CUDA graph,
    # CUDA events around the replays), with its algorithmic bytes (inputs +
    # outputs, + the table for the contractions)
    slab_z = torch.empty((NZ, N, N), dtype=torch.float32, device=dev).uniform_()
    slab_t = torch.empty((NT, N, N), dtype=torch.float32, device=dev).uniform_()
    Sz = torch.empty((NZ, P // 2 + 1, P), dtype=torch.complex64, device=dev)
    St = torch.empty((NT, P // 2 + 1, P), dtype=torch.complex64, device=dev)
    oz, ot = torch.empty_like(slab_z), torch.empty_like(slab_t)
    plan.stage_spectrum(slab_z, out=Sz)
    plan.stage_spectrum(slab_t, out=St)
    stage = {}
    for name, fn, nbytes in (
            ("a2_spectrum_depths", lambda: plan.stage_spectrum(slab_z, out=Sz), NZ * (N * N * 4 + K * 8)),
            ("a3_contract_fwd", lambda: plan.stage_contract(Xb, Yb), algo_spectra),
            ("a4_image_times", lambda: plan.stage_image(St, out=ot), NT * (N * N * 4 + K * 8)),
            ("a5_spectrum_times", lambda: plan.stage_spectrum(slab_t, out=St), NT * (N * N * 4 + K * 8)),
            ("a6_contract_adj", lambda: plan.stage_contract(Yb, Xb, adjoint=True), algo_spectra),
            ("a7_image_depths", lambda: plan.stage_image(Sz, out=oz), NZ * (N * N * 4 + K * 8))):
        ms = graph_ms(fn, 20)
        stage[name] = {"us": ms * 1e3, "gbs": nbytes / (ms / 1e3) / 1e9,
                       "frac_hbm": nbytes / (ms / 1e3) / 1e9 / hbm}

    # plain single-precision path: complex64 table, one volume at a time
    plan_c = Plan(N, N, NZ, NT, P, P, medium=med, force_complex=True)
    xc = torch.empty_like(x)
    plan_c.fista(y, x=xc, iters=ITERS, L=L)
    plain_ms = events_ms(lambda: plan_c.fista(y, x=xc, iters=ITERS, L=L), max(2, args.steps // 4))
    plain_pair_ms = events_ms(lambda: plan_c.gradient(p0_d, y, out=g, resid=False), 20)
    plan_c.close()

    # end to end through the C ABI: pinned host y in, host x out, every step
    y_h = y.cpu().pin_memory()
    x_h = torch.empty((NZ, N, N), dtype=torch.float32).pin_memory()
    plan.fista(y_h, x=x_h, iters=ITERS, L=L)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(2, args.steps // 4)
    for _ in range(e2e_steps):
        plan.fista(y_h, x=x_h, iters=ITERS, L=L)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = world * e2e_steps * ITERS / e2e_s

    out = {
        "metric": METRIC, "value": value, "unit": "FISTA it/s (= A+Aᵀ pairs/s)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(),
        "fista_it_per_s": value,
        "pairs_per_s": world * 1e3 / pair_ms,
        "plain_fp32": {"table": "complex64", "fista_it_per_s": world * ITERS * 1e3 / plain_ms,
                       "pairs_per_s": world * 1e3 / plain_pair_ms,
                       "speedup_real_even": plain_ms / ms_per_step},
        "roofline": {"bound": "hbm", "kernel": kname,
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_src,
                     "traffic": profiled_traffic(kname),
                     "algorithmic_bytes": algo,
                     "algorithmic": "stored table once + rho + d per application",
                     "table": "one stored row per radius group of D4 representatives",
                     "vs_d4_table": {
                         "note": "rate a one-row-per-representative table would have to stream "
                                 "at to give the same times (what radial sharing buys)",
                         "bytes": d4_bytes + rho_b + d_b,
                         "frac": (d4_bytes + rho_b + d_b) / (fwd_ms / 1e3) / 1e9 / hbm,
                         "adjoint_frac": (d4_bytes + rho_b + d_b) / (adj_ms / 1e3) / 1e9 / hbm},
                     "launch_ms": fwd_ms,
                     "adjoint_launch_ms": adj_ms,
                     "adjoint_frac": algo / (adj_ms / 1e3) / 1e9 / hbm,
                     "adjoint_traffic": profiled_traffic(kname.replace("fwd", "adj")),
                     "incl_spectra": {
                         "note": "also crediting the spectra X in and Y out of the kernel",
                         "bytes": algo_spectra,
                         "frac": algo_spectra / (fwd_ms / 1e3) / 1e9 / hbm,
                         "adjoint_frac": algo_spectra / (adj_ms / 1e3) / 1e9 / hbm},
                     "iteration": {
                         "note": "whole FISTA iteration: 2 x (table + rho + d) + 5 x rho",
                         "bytes": iter_bytes, "ms": ms_per_step / ITERS,
                         "frac": iter_bytes / (ms_per_step / ITERS / 1e3) / 1e9 / hbm}},
        "e2e": {"value": e2e_value, "unit": "FISTA it/s (= A+Aᵀ pairs/s)",
                "h2d_bytes_per_step": int(y_h.numel() * 4),
                "d2h_bytes_per_step": int(x_h.numel() * 4)},
        "gpu_launches": launches,
        "stages": stage,
        "clocks": clk.summary(),
        "L": L,
        "resid2_last": rep["resid2_last"],
    }
    plan.close()
    out["batched_16"] = run_batched(dev)
    samples = out["batched_16"].pop("_samples")
    if args.serve_seconds > 0:
        out["serve"] = run_serve(args.serve_seconds, seed=rank)
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, samples)
        if out["cpu_baseline"]:
            out["batched_16"]["rel_l2_vs_oracle"] = out["cpu_baseline"].pop("batched_vs_oracle")
    return out


# ----------------------------------------------------------------------------- batching
BATCH_T, BATCH_Z = (150, 400), 40  # sampled outputs of the batched workload


def run_batched(dev):
    """16 volumes sharing one library at 128^2 (padded 256^2) x 128 depths x 512
    samples: one batched H and one batched H* per step, contraction on the
    tcgen05 tensor cores (split BF16, FP32 accumulate) vs the CUDA-core path."""
    import numpy as np
    import torch

    from paper_2603_28150_gb300 import Medium, Plan
    B, nz, nt = 16, 128, 512
    plan = Plan(N, N, nz, nt, P, P, max_batch=B, medium=Medium(C0, DX, DX, DX, DT, 512, Z0),
                bf16_split=True)
    info = plan.info()
    from paper_2603_28150_gb300 import synth
    rho = torch.tensor(np.stack([synth.vessel_phantom(N, nz, seed=s) for s in range(B)]),
                       dtype=torch.float32, device=dev)
    d = plan.forward(rho)
    res = {"workload": f"{B} volumes (vessel phantoms, seeds 0..{B - 1}), {N}x{N} "
                       f"(padded {P}x{P}) x {nz} depths x {nt} samples",
           "tensor_tables_gb": info["tensor_table_bytes"] / 1e9}
    K = info["bins"]
    # algorithmic bytes of one batched application: one direction's tiles +
    # the operator's input and output; also with the spectra X, Y
    algo = info["tensor_table_bytes"] / 2 + B * (nz + nt) * N * N * 4
    algo_spectra = info["tensor_table_bytes"] / 2 + B * (nz + nt) * K * 8
    # the FFT stages of one batched H and H* on their own, to separate the
    # contractions out of the operator times
    sz = torch.rand((B * nz, N, N), device=dev)
    st = torch.rand((B * nt, N, N), device=dev)
    Sz = torch.empty((B * nz, P // 2 + 1, P), dtype=torch.complex64, device=dev)
    St = torch.empty((B * nt, P // 2 + 1, P), dtype=torch.complex64, device=dev)
    fft_fwd = graph_ms(lambda: plan.stage_spectrum(sz, out=Sz), 2) + \
        graph_ms(lambda: plan.stage_image(St, out=st), 2)
    fft_adj = graph_ms(lambda: plan.stage_spectrum(st, out=St), 2) + \
        graph_ms(lambda: plan.stage_image(Sz, out=sz), 2)
    del sz, st, Sz, St
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    # the tensor-core contraction alone, live, on spectra already in its
    # representative-slot layout (as the operator runs it)
    srow = 4 * ((info["table_rows"] + 31) // 32 * 32)
    Xs = torch.zeros((B, nz, srow), dtype=torch.complex64, device=dev)
    Ys = torch.zeros((B, nt, srow), dtype=torch.complex64, device=dev)
    plan.set_tensor_batch(2)
    plan.stage_contract_slots(Xs, Ys, B)
    cf_ms = events_ms(lambda: plan.stage_contract_slots(Xs, Ys, B), 5)
    ca_ms = events_ms(lambda: plan.stage_contract_slots(Ys, Xs, B, adjoint=True), 5)
    plan.check()
    del Xs, Ys
    outs = {}
    dd = d.clone()
    r2 = torch.empty_like(rho)
    for mode, mb in (("tensor", 2), ("cuda_core", 0)):
        plan.set_tensor_batch(mb)
        outs[mode] = (plan.forward(rho).double(), plan.adjoint(dd).double())
        a_ms = events_ms(lambda: plan.forward(rho, out=d), 5)
        at_ms = events_ms(lambda: plan.adjoint(dd, out=r2), 5)
        res[mode] = {"volume_pairs_per_s": B * 1e3 / (a_ms + at_ms), "A_ms": a_ms, "AT_ms": at_ms}
        if mode == "tensor":
            res[mode].update({
                "contract_fwd_ms": cf_ms, "contract_adj_ms": ca_ms,
                "contract_fwd_frac_hbm": algo / (cf_ms / 1e3) / 1e9 / hbm,
                "contract_adj_frac_hbm": algo / (ca_ms / 1e3) / 1e9 / hbm,
                "contract_fwd_frac_hbm_incl_spectra": algo_spectra / (cf_ms / 1e3) / 1e9 / hbm,
                "contract_adj_frac_hbm_incl_spectra": algo_spectra / (ca_ms / 1e3) / 1e9 / hbm,
                # the FFT stages in the slot layout: operator minus its contraction;
                # beside them the same stages in the bin layout, timed alone
                "fft_slot_layout_ms_per_direction": [a_ms - cf_ms, at_ms - ca_ms],
                "fft_bin_layout_ms_per_direction": [fft_fwd, fft_adj]})
    plan.check()
    plan.close()
    # sampled tensor-path outputs for the FP64 oracle comparison of the host
    # leg (H at two time samples and H* at one depth, every volume)
    res["_samples"] = {"t": BATCH_T, "z": BATCH_Z, "nz": nz, "nt": nt,
                       "H": outs["tensor"][0][:, list(BATCH_T)].cpu().numpy(),
                       "Hs": outs["tensor"][1][:, BATCH_Z].cpu().numpy(),
                       "d_in": dd.cpu().numpy()}
    # per-volume relative l2 of the split-BF16 outputs against the FP32
    # CUDA-core path on the same inputs
    err = {}
    for i, name in enumerate(("H", "H*")):
        t, c = outs["tensor"][i], outs["cuda_core"][i]
        e = [float((t[v] - c[v]).norm() / c[v].norm()) for v in range(B)]
        err[name] = {"max": max(e), "median": float(np.median(e)), "per_volume": e}
    res["rel_l2_vs_fp32_path"] = err
    res["speedup"] = res["tensor"]["volume_pairs_per_s"] / res["cuda_core"]["volume_pairs_per_s"]
    return res


# ----------------------------------------------------------------------------- serving
SERVE_GEOMS = [(64, 32, 128), (128, 64, 256), (256, 128, 512)]  # n, nz, nt; padded 2n
SERVE_RATE, SERVE_ITERS, SERVE_BUDGET, SERVE_SLOTS = 20.0, 50, 150 << 30, 16


def run_serve(seconds: float, seed: int = 0):
    """Poisson arrivals (20/s) of FISTA-50 requests over the three grids, same
    trace through the continuous-batching server (real-even tables, 16 slots per
    grid, 150 GB budget) and through the plain path (complex64 tables, one
    request at a time). Each arm gets `seconds` of arrivals plus 10 s to drain;
    requests still open then are reported as unfinished (with a lower bound on
    the p99 that includes them)."""
    import numpy as np
    import torch

    from paper_2603_28150_gb300 import synth
    from paper_2603_28150_gb300.serve import (CudaEngine, Geometry, Request, Server,
                                              poisson_arrivals, serve_one_at_a_time)
    geoms = [Geometry(n, nz, nt, 2 * n, C0, DX, DT) for n, nz, nt in SERVE_GEOMS]
    srv = Server(geoms, SERVE_BUDGET, SERVE_SLOTS, engine_factory=CudaEngine)
    engines = {g.key: srv._engine_for(g.key) for g in geoms}
    pool = {}
    for g in geoms:  # 3 noisy data sets per grid, reused round-robin
        eng = engines[g.key]
        pool[g.key] = []
        for s in range(3):
            p0 = torch.tensor(synth.vessel_phantom(g.n, g.nz, seed=seed * 10 + s),
                              dtype=torch.float32, device="cuda")
            d = eng.plan.forward(p0)
            nz = torch.tensor(synth.gaussian_field(tuple(d.shape), 900 + s), dtype=torch.float32,
                              device="cuda")
            pool[g.key].append((d + 0.05 * d.pow(2).mean().sqrt() * nz).contiguous())
    rng = np.random.default_rng(seed)
    arr = poisson_arrivals(SERVE_RATE, seconds, seed=seed)
    keys = [geoms[int(rng.integers(0, len(geoms)))].key for _ in arr]

    def trace():
        return [Request(i, k, pool[k][i % 3], SERVE_ITERS, 0.0, float(t))
                for i, (t, k) in enumerate(zip(arr, keys))]

    torch.cuda.synchronize()
    rep = srv.run(trace(), drain_seconds=10.0)
    rep["gpu_launches"] = sum(e.kernels for e in engines.values())
    rep["memory_gb"] = srv.used / 1e9
    srv.close()
    # plain path: complex64 tables, one request at a time
    plain = {}
    for g in geoms:
        e = CudaEngine(g, 1, force_complex=True)
        plain[g.key] = (e.plan, e.L)
    torch.cuda.synchronize()
    base = serve_one_at_a_time(plain, trace(), drain_seconds=10.0)
    for p, _ in plain.values():
        p.close()
    return {"workload": f"Poisson {SERVE_RATE:.0f} req/s for {seconds:.0f} s, FISTA-{SERVE_ITERS}, "
                        "grids 64²x32x128 / 128²x64x256 / 256²x128x512 (padded 2x), uniform mix",
            "batched": rep, "plain_one_at_a_time": base}


# ----------------------------------------------------------------------------- CPU oracle
def _mem_available_bytes() -> int:
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def _oracle_nt() -> int:
    """Time samples the oracle sample keeps: all of them when the complex128
    full-plane library (plus working copies) fits in a quarter of the free
    host memory, else the largest power of two that does."""
    per_t = NZ * P * P * 16
    budget = _mem_available_bytes() // 4
    nt = NT
    while nt > 8 and nt * per_t > budget:
        nt //= 2
    return nt


def _oracle_problem(nt: int):
    """The oracle's FFT-form operator on the same transverse grid and depths
    (nt time samples), with a complex128 full-plane library filled quickly
    (timing does not depend on its values)."""
    import numpy as np

    import oracle
    from paper_2603_28150_gb300 import synth
    g = oracle.Grid.square(N, NZ, nt, pad=P)
    Hf = synth.timing_spectra(NZ, nt, P, P, seed=0)
    op = oracle.Operator(g, Hf=Hf)
    p0, noise = make_inputs(seed=0)
    y = op.A(p0)
    y = y + 0.05 * float(np.sqrt(np.mean(y ** 2))) * noise[:nt]
    return op, y


def _oracle_rate(op, y, seconds: float):
    """(iterations, wall seconds) of FP64 oracle FISTA iterations run for about
    `seconds` (at least one)."""
    import numpy as np

    import oracle
    x_prev = np.zeros(op.obj_shape)
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.fista(op, y, 1.0, iters=1, x0=x_prev)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return n, time.perf_counter() - t0


def _spatial_cfg1(seconds: float):
    """A + A^T pairs/s of the oracle's direct spatial form (Eq. 7 and Eq. 11
    summed as written) beside its FFT form, at 32^2 -> 64^2, 16 depths, 64
    samples (the spatial form is O(N^4 Nz Nt): only this size is timed)."""
    import numpy as np

    import oracle
    from paper_2603_28150_gb300 import synth
    g = oracle.Grid.square(32, 16, 64)
    h = synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=0)
    rho = synth.blobs(g.nx, g.ny, g.nz, count=8, seed=0)
    out = {"workload": "32^2 -> 64^2 x 16 depths x 64 samples, one A + A^T pair"}
    for form in ("spatial", "fft"):
        op = oracle.Operator(g, h=h, form=form)
        t0 = time.perf_counter()
        n = 0
        while True:
            op.AT(op.A(rho))
            n += 1
            if time.perf_counter() - t0 >= seconds / 2:
                break
        out[f"{form}_pairs_per_s"] = n / (time.perf_counter() - t0)
    return out


def batched_vs_oracle(samples: dict) -> dict:
    """Per-volume relative l2 of the batched split-BF16 outputs against the FP64
    oracle (closed-form library of the same medium) at the sampled time
    samples of H rho and the sampled depth of H* d."""
    import numpy as np

    import oracle
    from paper_2603_28150_gb300 import synth
    nz, nt = samples["nz"], samples["nt"]
    g = oracle.Grid.square(N, nz, nt)
    med = oracle.Medium(C0, DX, DX, DX, DT)
    B = samples["H"].shape[0]
    Ht = oracle.table_kspace_closed(g, med, 512, z0=Z0, t_idx=list(samples["t"]))
    gt = oracle.Grid(N, N, nz, len(samples["t"]), P, P)
    eH = [oracle.rel_l2(samples["H"][v], oracle.forward_fft(Ht, synth.vessel_phantom(N, nz, seed=v), gt))
          for v in range(B)]
    del Ht
    Hz = oracle.table_kspace_closed(g, med, 512, z0=Z0, z_idx=[samples["z"]])
    gz = oracle.Grid(N, N, 1, nt, P, P)
    eA = [oracle.rel_l2(samples["Hs"][v], oracle.adjoint_fft(Hz, samples["d_in"][v], gz)[0])
          for v in range(B)]
    summ = lambda e: {"max": max(e), "median": float(np.median(e)), "per_volume": e}  # noqa: E731
    return {"H": dict(summ(eH), at_t=list(samples["t"])),
            "H*": dict(summ(eA), at_z=samples["z"]),
            "note": "FP64 oracle, closed-form library of the same medium, at the sampled "
                    "outputs; inputs: the vessel phantoms (H) and the batched H output (H*)"}


def cpu_baseline(seconds: float, batched_samples: dict | None = None):
    """FISTA iterations of the FP64 oracle on the host cores, bounded to about
    `seconds` of wall time (at least one iteration), on all cores and on one;
    plus the direct spatial form's rate at the smallest configuration; plus
    (given the batched workload's sampled outputs) their error against the
    oracle."""
    import oracle
    if seconds <= 0:
        return None
    nt = _oracle_nt()
    op, y = _oracle_problem(nt)
    cores = oracle.get_threads()
    n, dt = _oracle_rate(op, y, seconds)
    oracle.set_threads(1)
    try:
        n1, dt1 = _oracle_rate(op, y, seconds / 2)
        spatial = _spatial_cfg1(seconds / 2)
    finally:
        oracle.set_threads(cores)
    scale = nt / NT  # the oracle's cost is linear in nt (contraction and time-slice FFTs)
    note = "" if nt == NT else (f"; run with {nt} of {NT} time samples (host memory) and scaled "
                                f"by {nt}/{NT}")
    return {"value": n / dt * scale, "unit": "FISTA it/s (= A+Aᵀ pairs/s)",
            "cores": cores, "kind": "oracle",
            "sample": f"{n} FP64 FISTA iterations (FFT form, complex128 full-plane library) of the "
                      f"{N}x{N}x{NZ}x{nt} problem in {dt:.1f} s{note}",
            "one_core": {"value": n1 / dt1 * scale, "cores": 1,
                         "sample": f"{n1} iterations in {dt1:.1f} s"},
            "spatial_form_cfg1_one_core": spatial,
            "batched_vs_oracle": batched_vs_oracle(batched_samples) if batched_samples else None}


# ----------------------------------------------------------------------------- sharded
class _SelfExchange:
    """The exchange of a single rank: every chunk stays where it is."""

    def all_to_all(self, send):
        return send

    def sum(self, value, device):
        return value


def run_shard(args, world, rank, local):
    """FISTA-100 of one volume with the operator split over the ranks: each
    rank keeps 1/N of the folded table's rows (the stored operator scales as
    1/N per GPU), 1/N of the depth slices and 1/N of the time samples; the
    slice spectra cross ranks in one all-to-all per stage boundary."""
    import numpy as np
    import torch

    from paper_2603_28150_gb300 import Medium, Plan
    from paper_2603_28150_gb300.shard import DistExchange, ShardedOperator
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")
    if NZ % world or NT % world:
        raise SystemExit(f"--mode freq-shard needs N dividing {NZ} and {NT}")
    plan = Plan(N, N, NZ, NT, P, P, medium=Medium(C0, DX, DX, DX, DT, MZ, Z0), shard=(rank, world))
    info = plan.shard_info()
    sop = ShardedOperator(plan, DistExchange() if world > 1 else _SelfExchange())
    zr, tr = NZ // world, NT // world
    p0, noise = make_inputs(seed=0)
    clean = sop.forward(torch.tensor(p0[rank * zr:(rank + 1) * zr], dtype=torch.float32, device=dev))
    sigma = 0.05 * float(np.sqrt(sop.ex.sum(plan.dot(clean, clean), dev) / (NT * N * N)))
    y = clean.clone()
    plan.axpby(y, torch.tensor(noise[rank * tr:(rank + 1) * tr], dtype=torch.float32, device=dev),
               sigma, 1.0)
    L = 1.01 * sop.power_norm(torch.ones((zr, N, N), dtype=torch.float32, device=dev), 50)
    for _ in range(args.warmup):
        sop.fista(y, L, ITERS)
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(s)
        for _ in range(args.steps):
            _, hist = sop.fista(y, L, ITERS)
        e1.record(s)
        torch.cuda.synchronize()
    barrier(world)
    t_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    value = args.steps * ITERS / (t_ms / 1e3)
    return {
        "metric": METRIC, "value": value, "unit": "FISTA it/s (= A+Aᵀ pairs/s)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(bench_config(), per_rank="1/N of one volume's table rows, depth slices and "
                                                "time samples (frequency shards)"),
        "mode": "freq-shard",
        "shard": {"rows_per_rank": info["rows_per_rank"], "slot_width": info["slot_width"],
                  "table_bytes_per_rank": plan.info()["table_bytes"]},
        # per iteration: stage i (2 kernels), stage ii (1), stage iii with the
        # residual (3), stage i (2), stage ii (1), stage iii (2), FISTA step (1)
        "gpu_launches": 12 * ITERS * args.steps,
        "clocks": clk.summary(), "L": L, "resid2_last": hist[-1],
    }


def run_reference(args, world, rank):
    """The CPU oracle as the reference arm: each step one FP64 FISTA iteration."""
    if rank != 0:
        return None
    import numpy as np

    import oracle
    nt = _oracle_nt()
    op, y = _oracle_problem(nt)
    x = np.zeros(op.obj_shape)
    for _ in range(args.warmup):
        oracle.fista(op, y, 1.0, iters=1, x0=x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fista(op, y, 1.0, iters=1, x0=x)
    dt = time.perf_counter() - t0
    v = args.steps / dt * nt / NT
    unit = "FISTA it/s (= A+Aᵀ pairs/s)"
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": unit,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(),
        "cpu_baseline": {"value": v, "unit": unit, "kind": "oracle", "cores": oracle.get_threads(),
                         "sample": f"{args.steps} FP64 FISTA iterations of the oracle (FFT form, "
                                   f"complex128 full-plane library, {nt} of {NT} time samples, "
                                   f"rate scaled by {nt}/{NT})" if nt != NT else
                                   f"{args.steps} FP64 FISTA iterations of the oracle (FFT form, "
                                   f"complex128 full-plane library)"},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
    elif args.mode == "freq-shard":
        out = run_shard(args, world, rank, local)
    else:
        out = run_ours(args, world, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
