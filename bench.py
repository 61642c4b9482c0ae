#!/usr/bin/env python3
"""Throughput of batched FSSCS-RM decoding of polar codes on GB300.

Workload (one step): PC(1024, 512) with CRC-16 (0x1021), Bhattacharyya
frozen set at 0 dB design SNR, stack depth D = 32, visit cap L = 32, fast
Rate-0/Rate-1/REP/SPC nodes, 1,048,576 BPSK/AWGN frames at each of
Eb/N0 = 1.5, 2.0, 2.5 and 3.0 dB: four decode launches of 1,048,576 frames.
Inputs are synthetic (seeded), encoded on the GPU and resident in HBM when
the timed region starts; each launch reads 4 GiB of LLRs, far more than the
129 MB L2, so no flush is needed between launches.

Prints ONE JSON line (rank 0).  Metric: decoded message bits per second
(496 per frame; the CRC bits are not counted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Other workloads (--workload; each prints its own line): mixed (2,000,000
frames of mixed codes and depths in one launch, against per-configuration
launches), serve (Poisson arrivals, continuous batching against
one-size-per-launch batching), gsc (genie-aided SC loss and gradient over
per-stage scales), paper (the paper's decoder setting: systematic
PC(1024,512), CRC-24C, D = 8192, L = 8, 524,288 frames at each of 0 ... 3 dB).

Multi-GPU (torchrun, one process per GPU): every rank decodes its own
frames (seed offset by rank) with no collective on the data path (weak
scaling); the timed region is bracketed by barriers and the slowest rank's
time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(N=1024, K=512, crc=16, D=32, L=32, fast=True, frames=1 << 20, ebn0=(1.5, 2.0, 2.5, 3.0), seed=2,
                design_snr_db=0.0, systematic=False)
# the decoder setting of the paper's experiments (Sec. 5): PC(1024,512) with
# CRC-24C, stack depth 8192, visit cap 8, systematic encoding; the frozen set
# comes from the Bhattacharyya construction (the paper uses the 5G sequence)
PAPER = dict(N=1024, K=512, crc=24, D=8192, L=8, fast=True, frames=1 << 19, ebn0=(0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0),
             seed=6, design_snr_db=0.0, systematic=True)
# the paper's own FSSCS-RM figures at those points (Sec. 5, throughput and FER
# plots): Mb/s of information bits per CPU thread on a Ryzen 5 1600, and FER
PAPER_FSSCS_RM = dict(mbps_per_thread=(0.169, 0.182, 0.232, 0.343, 0.449, 0.620, 0.925),
                      fer=(9.81e-1, 8.11e-1, 3.54e-1, 6.08e-2, 3.68e-3, 1.10e-4, None))
ALU_LANES_PER_SM = 128  # FP32/INT32 lanes per SM (4 partitions x 32)


def workload_name(w=WORKLOAD) -> str:
    sysd = "systematic " if w.get("systematic") else ""
    return (f"{sysd}PC({w['N']},{w['K']}) CRC-{w['crc']} FSSCS-RM D={w['D']} L={w['L']} fast nodes, "
            f"{w['frames']} frames x Eb/N0 {'/'.join(str(e) for e in w['ebn0'])} dB")


def bytes_per_frame(w=WORKLOAD) -> int:
    """Algorithmic DRAM bytes of one frame: LLRs in, packed message + pm + status out."""
    kmsg = w["K"] - w["crc"]
    return 4 * w["N"] + 4 * ((kmsg + 31) // 32) + 4 + 1


def rank_seed(rank: int, w=WORKLOAD) -> int:
    return int(w["seed"]) + 1000 * int(rank)


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


def profiled_values(kernel_src: str, key: str, ebn0s) -> list[float] | None:
    """Per-Eb/N0 values (DRAM bytes per frame, issue-slot utilisation) from the
    committed ncu summary, if it was taken on the current kernel source (its
    sha256 is recorded in the summary) and covers every point; else None."""
    path = os.path.join(ROOT, "profiles", "scs_decode_pc1024_traffic.txt")
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
        if kv.get("kernel_sha256") != sha:
            return None
        return [float(kv[f"{key}_{e}"]) for e in ebn0s]
    except Exception:
        return None


def profiled_traffic(kernel_src: str, ebn0s) -> list[float] | None:
    return profiled_values(kernel_src, "dram_bytes_per_frame", ebn0s)


def reduce_max(value: float, world: int) -> float:
    """Largest value over ranks (the slowest rank's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int) -> float:
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows), power_w_max=max(power) if power else None)


# --------------------------------------------------------------- inputs
def make_gpu_inputs(ps, plan, frames: int, rank: int, w=WORKLOAD):
    """Messages and noise from the seeded generators (host), encoded by the
    GPU encoder, BPSK/AWGN LLRs formed on the GPU in float32 with the same
    three rounded steps as workloads.bpsk_awgn_llr."""
    import numpy as np
    import torch

    import workloads as W

    seed = rank_seed(rank, w)
    kmsg = w["K"] - w["crc"]
    msg = W.message_bits(seed, frames, kmsg)
    d_msg = torch.from_numpy(ps.pack_bits(msg)).cuda()
    del msg
    d_cw = torch.empty((frames, plan.words), dtype=torch.int32, device="cuda")
    ps.polar_encode_batch(plan, d_msg, d_cw)
    shifts = torch.arange(32, dtype=torch.int32, device="cuda")
    x = torch.empty((frames, w["N"]), dtype=torch.float32, device="cuda")
    step = 1 << 16
    for lo in range(0, frames, step):
        bits = (d_cw[lo:lo + step].unsqueeze(-1) >> shifts) & 1
        x[lo:lo + step] = 1.0 - 2.0 * bits.reshape(-1, w["N"]).to(torch.float32)
    del d_cw
    z = torch.from_numpy(W.awgn_noise(seed, frames, w["N"])).cuda()
    llrs = []
    for e in w["ebn0"]:
        s, k = W.channel_constants(W.sigma_from_ebn0(e, w["K"] / w["N"]))
        y = torch.mul(z, float(s))
        y = torch.add(x, y)
        llrs.append(torch.mul(y, float(k)))
        del y
    del z, x
    torch.cuda.synchronize()
    return llrs, d_msg


def oracle_sample_inputs(frames: int, rank: int, w=WORKLOAD):
    """The first `frames` frames of each point's batch, built on the host with
    the oracle's encoder (CPU baseline / reference arm only)."""
    import oracle
    import workloads as W

    seed = rank_seed(rank, w)
    fr = oracle.construct(w["N"], w["K"], w["design_snr_db"])
    kmsg = w["K"] - w["crc"]
    msg = W.message_bits(seed, frames, kmsg)
    cw = oracle.encode_batch(msg, w["N"], w["K"], fr, w["crc"], systematic=bool(w.get("systematic")))
    z = W.awgn_noise(seed, frames, w["N"])
    llrs = [W.bpsk_awgn_llr(cw, z, W.sigma_from_ebn0(e, w["K"] / w["N"])) for e in w["ebn0"]]
    return fr, msg, llrs


def run_oracle(fr, llrs, threads: int, w=WORKLOAD):
    import oracle

    t0 = time.perf_counter()
    outs = [oracle.scs_decode_batch(l, w["N"], w["K"], fr, fast=w["fast"], D=w["D"], L=w["L"], crc_len=w["crc"],
                                    threads=threads, systematic=bool(w.get("systematic"))) for l in llrs]
    return time.perf_counter() - t0, outs


# ------------------------------------------------------------ reference arm
def bench_reference(args, rank: int, world: int) -> None:
    """The CPU oracle as it stands, timed on the host cores: each step decodes a
    bounded sample (the first frames of every point) of the same workload."""
    if rank != 0:
        return
    import numpy as np

    sample = args.ref_frames
    threads = os.cpu_count() or 1
    w = dict(WORKLOAD, systematic=bool(args.systematic))
    fr, msg, llrs = oracle_sample_inputs(sample, 0, w)
    for _ in range(args.warmup):
        run_oracle(fr, llrs, threads, w)
    times = []
    for _ in range(args.steps):
        dt, outs = run_oracle(fr, llrs, threads, w)
        times.append(dt)
    kmsg = WORKLOAD["K"] - WORKLOAD["crc"]
    total = sum(times)
    bits = kmsg * sample * len(WORKLOAD["ebn0"]) * args.steps
    value = bits / total / 1e9
    fer = {str(e): float(np.mean(np.any(o[0] != msg, axis=1))) for e, o in zip(WORKLOAD["ebn0"], outs)}
    desc = f"oracle on {sample} frames per Eb/N0 point ({sample * len(WORKLOAD['ebn0'])} frames per step), {threads} host threads"
    line = {"impl": "reference", "metric": "decoded info Gbit/s", "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(w), "sample": desc, "fer_sample": fer},
            "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm
def bench_ours(args, rank: int, world: int, local_rank: int, base=WORKLOAD) -> None:
    import numpy as np
    import torch

    import paper_1809_03606_gb300 as ps

    torch.cuda.set_device(local_rank)
    ps.load(build_if_missing=True)
    w = dict(base, systematic=bool(args.systematic) or bool(base["systematic"]))
    if args.frames:
        w["frames"] = int(args.frames)
    B, N, K, crc, D, L = w["frames"], w["N"], w["K"], w["crc"], w["D"], w["L"]
    kmsg = K - crc
    npts = len(w["ebn0"])
    fr = ps.polar_construct(N, K, w["design_snr_db"])
    plan = ps.Plan(N, K, fr, fast_nodes=w["fast"], crc=crc, systematic=w["systematic"])
    llrs, d_msg = make_gpu_inputs(ps, plan, B, rank, w)
    outs = [(torch.empty((B, plan.msg_words), dtype=torch.int32, device="cuda"),
             torch.empty(B, dtype=torch.float32, device="cuda"), torch.empty(B, dtype=torch.int8, device="cuda"))
            for _ in range(npts)]
    stream = torch.cuda.current_stream()

    def step(events=None):
        for p in range(npts):
            if events is not None:
                events[p][0].record(stream)
            ps.scs_decode_batch(plan, llrs[p], D, L, *outs[p], stream=stream)
            if events is not None:
                events[p][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # per-frame counters from one untimed launch per point (decoding is deterministic)
    ops_pt, iters_pt, sw_pt, fer_pt, fail_pt = [], [], [], [], []
    stats = torch.empty((B, 4), dtype=torch.int32, device="cuda")
    for p in range(npts):
        info, pm, st = outs[p]
        ps.scs_decode_batch(plan, llrs[p], D, L, info, pm, st, stats, stream=stream)
        torch.cuda.synchronize()
        s64 = stats.to(torch.int64) & 0xFFFFFFFF
        ops_pt.append(int(s64[:, 2].sum().item()))
        iters_pt.append(float(s64[:, 0].double().mean().item()))
        sw_pt.append(float(s64[:, 1].double().mean().item()))
        fer_pt.append(float((info != d_msg).any(dim=1).double().mean().item()))
        fail_pt.append(float((st != 0).double().mean().item()))
    del stats

    sampler = ClockSampler(local_rank) if rank == 0 else None
    launch_events = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(npts)]
                     for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.__enter__()
    barrier(world)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        step(launch_events[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    if sampler:
        sampler.__exit__(None, None, None)
    elapsed_ms = t_start.elapsed_time(t_end)
    launch_ms = [[launch_events[k][p][0].elapsed_time(launch_events[k][p][1]) for p in range(npts)]
                 for k in range(args.steps)]
    elapsed_ms = reduce_max(elapsed_ms, world)
    ms_per_step = elapsed_ms / args.steps
    frames_all = reduce_sum(float(B * npts * args.steps), world)
    value = frames_all * kmsg / (elapsed_ms / 1e3) / 1e9

    # roofline of the decode kernel over the step: the slower of counted ALU
    # operations at the FP32/INT32 lane peak and algorithmic bytes at HBM BW
    peaks = measured_peaks()
    info_dev = ps.polar_device_info()
    sms = info_dev["sm_count"]
    alu_peak = sms * ALU_LANES_PER_SM * peaks["sm_max_mhz"] * 1e6  # lane-ops/s
    hbm_peak = peaks["hbm_gbs"] * 1e9
    kernel_s = sum(sum(r) for r in launch_ms) / args.steps / 1e3  # per step
    bytes_step = B * npts * bytes_per_frame(w)
    ops_step = float(sum(ops_pt))
    t_alu, t_hbm = ops_step / alu_peak, bytes_step / hbm_peak
    traffic_pf = profiled_traffic(os.path.join(ROOT, "paper_1809_03606_gb300", "csrc", "scs_decode.cu"), w["ebn0"])
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": ops_step / kernel_s / 1e12, "peak": alu_peak / 1e12, "unit": "Top/s"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_step / kernel_s / 1e9, "peak": hbm_peak / 1e9, "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes per launch (ncu), averaged over the step's launches like `achieved`
    roof["traffic"] = None if traffic_pf is None else float(sum(traffic_pf)) * B / npts
    roof["peak_source"] = (f"{peaks['source']}: {sms} SMs x {ALU_LANES_PER_SM} lanes x {peaks['sm_max_mhz']:.0f} MHz"
                           if roof["bound"] == "alu" else f"{peaks['source']} HBM copy bandwidth")
    # what bounds the kernel in practice: its own instruction issue (ncu,
    # same kernel source), next to the lane-op fraction above
    issue = profiled_values(os.path.join(ROOT, "paper_1809_03606_gb300", "csrc", "scs_decode.cu"), "issue_active_pct",
                            w["ebn0"])
    roof["issue_slots_busy"] = None if issue is None else statistics.mean(issue) / 100.0
    per_point = []
    for p, e in enumerate(w["ebn0"]):
        ms = statistics.mean(launch_ms[k][p] for k in range(args.steps))
        ta, th = ops_pt[p] / alu_peak, B * bytes_per_frame(w) / hbm_peak
        per_point.append({"ebn0_db": e, "ms": ms, "info_gbps": B * kmsg / (ms / 1e3) / 1e9, "fer": fer_pt[p],
                          "crc_fail_rate": fail_pt[p], "pops_per_frame": iters_pt[p], "switches_per_frame": sw_pt[p],
                          "ops_per_frame": ops_pt[p] / B, "bound": "alu" if ta >= th else "hbm",
                          "roofline_frac": max(ta, th) / (ms / 1e3)})

    e2e = None
    if not args.no_e2e:
        e2e = bench_e2e(ps, plan, llrs, w, args, world)
    mixed = None
    if base is WORKLOAD and world == 1 and not args.no_mixed:
        # the batching claim (config 3 of the workload) beside the sweep: the
        # batched path against per-configuration launches on the same frames
        del llrs, outs
        torch.cuda.empty_cache()
        mixed = measure_mixed(args, MIXED["frames"], rank, local_rank, steps=3, warmup=1, with_roofline=False)
    subsystems = None
    if base is WORKLOAD and world == 1 and not args.no_extras:
        subsystems = measure_subsystems(args, rank, local_rank)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_frames, w)
    clocks = sampler.summary() if sampler else None

    if rank == 0:
        config = {"workload": workload_name(w), "frames_per_step_per_gpu": B * npts,
                  "message_bits_per_frame": kmsg,
                  "l2": f"inputs larger than L2 ({B * w['N'] * 4 / 2**30:.1f} GiB of LLRs per launch)",
                  "parallelism": f"frames sharded over {world} GPU(s), no data-path collective",
                  "per_point": per_point}
        if base is PAPER:
            config["paper_fsscs_rm_context"] = {
                "note": "the paper's CPU figures (5G-sequence frozen set, one Ryzen 5 1600 thread); context only",
                "per_point": [{"ebn0_db": e, "paper_mbps_per_thread": t, "paper_fer": f,
                               "this_gpu_mbps": pp["info_gbps"] * 1e3, "this_fer": pp["fer"]}
                              for e, t, f, pp in zip(w["ebn0"], PAPER_FSSCS_RM["mbps_per_thread"],
                                                     PAPER_FSSCS_RM["fer"], per_point)]}
        line = {"metric": "decoded info Gbit/s", "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": npts * args.steps,
                "clocks": clocks}
        if mixed is not None:
            line["mixed"] = mixed
        if subsystems is not None:
            line["subsystems"] = subsystems
        print(json.dumps(line), flush=True)


def bench_e2e(ps, plan, llrs, w, args, world: int):
    """Same metric through the C ABI with host buffers: every step copies its
    LLRs from pinned host memory and reads the results back, in chunks whose
    copies overlap the decodes of earlier chunks; consecutive chunks decode on
    two streams, so the tail of one launch overlaps the next.  Each chunk has
    its own device buffer (up to 16 GiB of them), so the copy stream runs
    ahead during the long low-Eb/N0 decodes and the copies of the short
    high-Eb/N0 ones are already done when they start.  (Chunks of a whole
    Eb/N0 point on two buffers measured slower: a 4 GiB copy does not hide
    behind the short decode of the 3.0 dB point.)"""
    import torch

    B, N = w["frames"], w["N"]
    npts = len(llrs)
    chunk = min(B, 1 << 18)
    nchunks = npts * ((B + chunk - 1) // chunk)
    nbuf = max(2, min(nchunks, (16 << 30) // (chunk * N * 4)))
    host = []
    for l in llrs:
        h = torch.empty((B, N), dtype=torch.float32, pin_memory=True)
        h.copy_(l)
        host.append(h)
    out_host = [(torch.empty((B, plan.msg_words), dtype=torch.int32, pin_memory=True),
                 torch.empty(B, dtype=torch.float32, pin_memory=True), torch.empty(B, dtype=torch.int8, pin_memory=True))
                for _ in range(npts)]
    dbuf = [torch.empty((chunk, N), dtype=torch.float32, device="cuda") for _ in range(nbuf)]
    dout = [(torch.empty((chunk, plan.msg_words), dtype=torch.int32, device="cuda"),
             torch.empty(chunk, dtype=torch.float32, device="cuda"), torch.empty(chunk, dtype=torch.int8, device="cuda"))
            for _ in range(nbuf)]
    copy_s = torch.cuda.Stream()
    comp = [torch.cuda.Stream(), torch.cuda.Stream()]
    ready = [torch.cuda.Event() for _ in range(nbuf)]
    free = [torch.cuda.Event() for _ in range(nbuf)]
    for j, e in enumerate(free):
        e.record(comp[j & 1])

    def one_step():
        i = 0
        for p in range(npts):
            for lo in range(0, B, chunk):
                hi = min(B, lo + chunk)
                j = i % nbuf
                with torch.cuda.stream(copy_s):
                    copy_s.wait_event(free[j])
                    dbuf[j][: hi - lo].copy_(host[p][lo:hi], non_blocking=True)
                    ready[j].record(copy_s)
                cs = comp[i & 1]
                with torch.cuda.stream(cs):
                    cs.wait_event(ready[j])
                    o = [t[: hi - lo] for t in dout[j]]
                    ps.scs_decode_batch(plan, dbuf[j][: hi - lo], w["D"], w["L"], *o, stream=cs)
                    for src, dst in zip(o, out_host[p]):
                        dst[lo:hi].copy_(src, non_blocking=True)
                    free[j].record(cs)
                i += 1

    steps = max(1, min(args.steps, 3))
    one_step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    dt = reduce_max(time.perf_counter() - t0, world)
    barrier(world)
    kmsg = w["K"] - w["crc"]
    frames = reduce_sum(float(B * npts * steps), world)
    h2d = B * N * 4 * npts
    d2h = B * (4 * plan.msg_words + 4 + 1) * npts
    del host, out_host, dbuf, dout
    return {"value": frames * kmsg / dt / 1e9, "unit": "Gbit/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": steps, "chunk_frames": chunk, "device_buffers": nbuf}


# ------------------------------------------------------ mixed-batch workload
MIXED = dict(frames=2_000_000, seed=3, crc=8, design_snr_db=0.0)


def make_mixed_inputs(ps, frames: int, rank: int, w=MIXED):
    """Per-frame (N, K, D, Eb/N0) draws of the mixed workload, messages and
    noise per code from the seeded generators, GPU encoding, and per-frame
    float32 channel LLRs packed in frame order."""
    import numpy as np
    import torch

    import workloads as W

    seed = int(w["seed"]) + 1000 * rank
    draw = W.mixed_frames(seed, frames)
    Ns, Ks, Ds, eb = draw["N"], draw["K"], draw["D"], draw["ebn0_db"]
    keys = sorted(set(zip(Ns.tolist(), Ks.tolist())))
    plans = [ps.Plan(N, K, ps.polar_construct(N, K, w["design_snr_db"]), fast_nodes=True, crc=w["crc"]) for N, K in keys]
    code_of = {k: i for i, k in enumerate(keys)}
    idx = np.array([code_of[(int(n), int(k))] for n, k in zip(Ns, Ks)], np.int32)
    llr_off = np.concatenate([[0], np.cumsum(Ns)[:-1]]).astype(np.int64)
    words = np.array([plans[i].msg_words for i in idx], np.int64)
    info_off = np.concatenate([[0], np.cumsum(words)[:-1]]).astype(np.int64)
    flat = torch.empty(int(Ns.sum()), dtype=torch.float32, device="cuda")
    msg_flat = torch.zeros(int(words.sum()), dtype=torch.int32, device="cuda")
    for ci, (N, K) in enumerate(keys):
        sel = np.nonzero(idx == ci)[0]
        if sel.size == 0:
            continue
        plan = plans[ci]
        msg = W.message_bits(seed * 97 + ci, sel.size, K - w["crc"])
        d_msg = torch.from_numpy(ps.pack_bits(msg)).cuda()
        d_cw = torch.empty((sel.size, plan.words), dtype=torch.int32, device="cuda")
        ps.polar_encode_batch(plan, d_msg, d_cw)
        shifts = torch.arange(32, dtype=torch.int32, device="cuda")
        x = 1.0 - 2.0 * ((d_cw.unsqueeze(-1) >> shifts) & 1).reshape(sel.size, -1)[:, :N].to(torch.float32)
        z = torch.from_numpy(W.awgn_noise(seed * 97 + ci, sel.size, N)).cuda()
        sig = np.array([W.sigma_from_ebn0(e, K / N) for e in eb[sel]])
        s32 = torch.from_numpy(sig.astype(np.float32)).cuda()[:, None]
        k32 = torch.from_numpy((2.0 / (sig * sig)).astype(np.float32)).cuda()[:, None]
        llr = torch.mul(torch.add(x, torch.mul(z, s32)), k32)
        offs = torch.from_numpy(llr_off[sel]).cuda()
        flat[(offs[:, None] + torch.arange(N, device="cuda")[None, :]).reshape(-1)] = llr.reshape(-1)
        woffs = torch.from_numpy(info_off[sel]).cuda()
        msg_flat[(woffs[:, None] + torch.arange(plan.msg_words, device="cuda")[None, :]).reshape(-1)] = d_msg.reshape(-1)
        del x, z, llr, d_cw
    torch.cuda.synchronize()
    return dict(plans=plans, keys=keys, idx=idx, D=Ds.astype(np.int32), llr=flat, llr_off=llr_off, info_off=info_off,
                words=words, msg=msg_flat, Ns=Ns, Ks=Ks)


def measure_mixed(args, B: int, rank: int, local_rank: int, steps: int, warmup: int, with_roofline: bool) -> dict:
    """The mixed batch (config 3 of the workload) three ways on the same
    frames: split by stack rows into two persistent launches on two streams
    (scs_decode_mixed_split, tuned, replayed from one captured CUDA graph),
    one persistent launch (scs_decode_mixed, graph-replayed), and one launch
    per (code, D) configuration; all three must give identical outputs."""
    import numpy as np
    import torch

    import paper_1809_03606_gb300 as ps

    m = make_mixed_inputs(ps, B, rank)
    pset = ps.PlanSet(m["plans"])
    fr = np.zeros((B, 4), np.int32)
    fr[:, 0] = m["idx"]
    fr[:, 1] = m["D"]
    fr[:, 2] = m["D"]  # L = D
    frames = torch.from_numpy(fr).cuda()
    Dmax = int(fr[:, 1].max())
    llr_off = torch.from_numpy(m["llr_off"]).cuda()
    info_off = torch.from_numpy(m["info_off"]).cuda()
    info = torch.zeros_like(m["msg"])
    pm = torch.empty(B, dtype=torch.float32, device="cuda")
    st = torch.empty(B, dtype=torch.int8, device="cuda")
    order = torch.from_numpy(ps.polar_mixed_order(pset, fr)).cuda() if not args.no_lpt else None  # longest first
    sorder_np, n_two = ps.polar_mixed_split_order(pset, fr)
    sorder = torch.from_numpy(sorder_np).cuda()
    margs = (pset, frames, Dmax, m["llr"], llr_off, info, info_off, pm, st)
    ps.scs_decode_mixed(*margs, order=order)
    torch.cuda.synchronize()
    nsample = min(B, 200_000)
    sfr = fr[:nsample]
    tune_order = torch.from_numpy(ps.polar_mixed_order(pset, sfr)).cuda() if not args.no_lpt else None
    sample = (pset, frames[:nsample], Dmax, m["llr"], llr_off[:nsample], info, info_off[:nsample], pm[:nsample],
              st[:nsample])
    wpb, chunk = ps.scs_tune_mixed(*sample, order=tune_order)
    # first calls on a side stream (set tables, split streams), then capture
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        ps.scs_decode_mixed(*margs, stream=stream, order=order)
        ps.scs_decode_mixed_split(pset, frames, sorder, n_two, Dmax, m["llr"], llr_off, info, info_off, pm, st,
                                  stream=stream)
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    graph_one = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_one):
        ps.scs_decode_mixed(*margs, order=order)
    graph_split = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_split):
        ps.scs_decode_mixed_split(pset, frames, sorder, n_two, Dmax, m["llr"], llr_off, info, info_off, pm, st)

    # per-configuration launches: frames grouped by (code, D), each group's
    # LLR rows gathered into its own contiguous buffer (outside the timing)
    groups = {}
    for b in range(B):
        groups.setdefault((int(m["idx"][b]), int(m["D"][b])), []).append(b)
    per = []
    for (ci, d), bs in sorted(groups.items()):
        plan = m["plans"][ci]
        bs_t = torch.from_numpy(np.asarray(bs, np.int64)).cuda()
        offs = torch.from_numpy(m["llr_off"][bs]).cuda()
        x = m["llr"][(offs[:, None] + torch.arange(plan.N, device="cuda")[None, :])].contiguous()
        per.append((plan, d, x, bs_t, torch.empty((len(bs), plan.msg_words), dtype=torch.int32, device="cuda"),
                    torch.empty(len(bs), dtype=torch.float32, device="cuda"),
                    torch.empty(len(bs), dtype=torch.int8, device="cuda")))

    def run_per_config():
        for plan, d, x, bs_t, i_, p_, s_ in per:
            ps.scs_decode_batch(plan, x, d, d, i_, p_, s_)

    def timed(fn, n):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.__enter__()
    ms_one = timed(graph_one.replay, steps)
    pm_one, st_one, info_one = pm.clone(), st.clone(), info.clone()
    ms_split = timed(graph_split.replay, steps)
    ms_per = timed(run_per_config, steps)
    if sampler:
        sampler.__exit__(None, None, None)
    # identical outputs: per-configuration results scattered back in frame order
    pm_per = torch.empty_like(pm)
    st_per = torch.empty_like(st)
    for plan, d, x, bs_t, i_, p_, s_ in per:
        pm_per[bs_t] = p_
        st_per[bs_t] = s_
    same = bool(torch.equal(pm_per.view(torch.int32), pm.view(torch.int32)) and torch.equal(st_per, st) and
                torch.equal(pm_one.view(torch.int32), pm.view(torch.int32)) and torch.equal(st_one, st) and
                torch.equal(info_one, info))
    kmsg = torch.from_numpy((m["Ks"] - MIXED["crc"]).astype(np.int64)).sum().item()
    out = {"frames": B, "codes": len(m["keys"]), "two_row_frames": int(n_two),
           "batched_ms": ms_split, "batched": "two persistent launches split by stack rows, two streams, one graph",
           "single_launch_ms": ms_one, "per_config_ms": ms_per, "per_config_launches": len(per),
           "ratio": ms_per / ms_split, "ratio_single_launch": ms_per / ms_one, "outputs_identical": same,
           "gbps": kmsg / (ms_split / 1e3) / 1e9, "per_config_gbps": kmsg / (ms_per / 1e3) / 1e9,
           "tuned": {"warps_per_block": wpb, "frames_per_claim": chunk},
           "crc_fail_rate": float((st != 0).double().mean().item()),
           "clocks": sampler.summary() if sampler else None}
    if with_roofline:
        # counted operations (one untimed launch with counters) and algorithmic
        # bytes against the same peaks as the sweep
        stats = torch.empty((B, 4), dtype=torch.int32, device="cuda")
        ps.scs_decode_mixed_split(pset, frames, sorder, n_two, Dmax, m["llr"], llr_off, info, info_off, pm, st,
                                  stats=stats)
        torch.cuda.synchronize()
        ops_step = float((stats[:, 2].to(torch.int64) & 0xFFFFFFFF).sum().item())
        del stats
        bytes_step = float(sum(4 * int(n) for n in m["Ns"]) + 4 * int(m["words"].sum()) + 5 * B)
        peaks = measured_peaks()
        sms = ps.polar_device_info()["sm_count"]
        alu_peak = sms * ALU_LANES_PER_SM * peaks["sm_max_mhz"] * 1e6
        t_alu, t_hbm = ops_step / alu_peak, bytes_step / (peaks["hbm_gbs"] * 1e9)
        if t_alu >= t_hbm:
            roof = {"bound": "alu", "achieved": ops_step / (ms_split / 1e3) / 1e12, "peak": alu_peak / 1e12,
                    "unit": "Top/s"}
        else:
            roof = {"bound": "hbm", "achieved": bytes_step / (ms_split / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["traffic"] = None
        out["roofline"] = roof
        err = 0
        info_np = info.cpu().numpy()
        msg_np = m["msg"].cpu().numpy()
        for b in range(0, B, max(1, B // 20000)):
            lo = int(m["info_off"][b])
            err += int(not np.array_equal(info_np[lo:lo + m["words"][b]], msg_np[lo:lo + m["words"][b]]))
        out["fer_sampled"] = err / len(range(0, B, max(1, B // 20000)))
    del m, per
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def bench_mixed(args, rank: int, world: int, local_rank: int) -> None:
    """The mixed workload on its own line: the batched path (two launches split
    by stack rows, one graph) against one launch and per-configuration launches."""
    import torch

    import paper_1809_03606_gb300 as ps

    torch.cuda.set_device(local_rank)
    ps.load(build_if_missing=True)
    B = int(args.frames) if args.frames else MIXED["frames"]
    r = measure_mixed(args, B, rank, local_rank, args.steps, args.warmup, with_roofline=True)
    cpu = mixed_cpu_baseline(args.cpu_frames * 4) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    if rank == 0:
        cfg = {"workload": f"{B} mixed frames: N in {{128..2048}}, K/N in {{1/4,1/3,1/2,2/3,3/4}}, "
                           f"D in {{8,16,32,64}}, L = D, CRC-8, Eb/N0 ~ U[1,4] dB, shuffled"}
        cfg.update({k: v for k, v in r.items() if k not in ("roofline", "clocks", "gbps")})
        line = {"metric": "decoded info Gbit/s (mixed batch)", "value": r["gbps"], "unit": "Gbit/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["batched_ms"],
                "higher_is_better": True, "dtype": "f32", "data": "synthetic", "config": cfg,
                "roofline": r["roofline"], "cpu_baseline": cpu, "clocks": r["clocks"]}
        print(json.dumps(line), flush=True)


# ------------------------------------------------ genie-aided SC (gradient)
GSC = dict(N=1024, K=512, crc=0, frames=65536, ebn0=(2.0,), seed=4, design_snr_db=0.0, train_steps=200, lr=0.02,
           fer_frames=1 << 18)


def bench_gsc(args, rank: int, world: int, local_rank: int) -> None:
    """Genie-aided SC with ten per-stage min-sum scales: forward + reverse
    kernel throughput on 65,536 PC(1024,512) frames at 2.0 dB, a training run
    of the scales with Adam, and the learned scales fed back into the
    PC(1024,512) CRC-16 stack decoder (D = L = 32) against unit scales."""
    import numpy as np
    import torch

    import paper_1809_03606_gb300 as ps

    torch.cuda.set_device(local_rank)
    ps.load(build_if_missing=True)
    g = dict(GSC)
    if args.frames:
        g["frames"] = int(args.frames)
    B, N, K = g["frames"], g["N"], g["K"]
    n = N.bit_length() - 1
    fr = ps.polar_construct(N, K, g["design_snr_db"])
    plan = ps.Plan(N, K, fr, fast_nodes=False)
    llrs, d_msg = make_gpu_inputs(ps, plan, B, rank, g)
    x = llrs[0]
    import workloads as W

    msg = W.message_bits(rank_seed(rank, g), B, K)
    u = torch.from_numpy(ps.u_from_messages(plan, msg)).cuda()
    del msg
    ones = torch.ones(n, dtype=torch.float32, device="cuda")

    def step():
        return ps.gsc_loss_grad(plan, x, u, ones)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.__enter__()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__(None, None, None)
    ms = e0.elapsed_time(e1) / args.steps
    ms = reduce_max(ms, world)
    # roofline: counted operations per frame (forward 4 per node pair and
    # stage: min-sum 2, scale 1, g 1; reverse 7: two adjoint selects, two
    # products, the g adjoint, the scale-gradient product and sum; 8 per
    # information leaf: loss and seed) against the lane-op peak, and LLR plus
    # transmitted-bit bytes against the HBM bandwidth
    ops_frame = 11 * n * (N // 2) + 8 * K
    bytes_frame = 4 * N + N // 8
    peaks = measured_peaks()
    sms = ps.polar_device_info()["sm_count"]
    alu_peak = sms * ALU_LANES_PER_SM * peaks["sm_max_mhz"] * 1e6
    if ops_frame / alu_peak >= bytes_frame / (peaks["hbm_gbs"] * 1e9):
        roof = {"bound": "alu", "achieved": ops_frame * B / (ms / 1e3) / 1e12, "peak": alu_peak / 1e12, "unit": "Top/s"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_frame * B / (ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    cpu = gsc_cpu_baseline(g, g["frames"]) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    # training the scales (Adam), then the learned scales in the stack decoder
    sc = torch.ones(n, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([sc], lr=g["lr"])
    loss0 = None
    for _ in range(g["train_steps"]):
        opt.zero_grad()
        loss = ps.genie_sc_loss(x, sc, u, plan)
        loss.backward()
        opt.step()
        loss0 = loss.item() if loss0 is None else loss0
    loss1 = ps.genie_sc_loss(x, sc.detach(), u, plan).item()
    learned = sc.detach().cpu().numpy().astype(np.float32)

    w = dict(WORKLOAD)
    w["frames"] = g["fer_frames"]
    w["ebn0"] = (2.0,)
    dplan = ps.Plan(w["N"], w["K"], ps.polar_construct(w["N"], w["K"], w["design_snr_db"]), fast_nodes=True,
                    crc=w["crc"])
    dl, dmsg = make_gpu_inputs(ps, dplan, w["frames"], rank, w)
    fer = {}
    for name, scales in (("unit", None), ("learned", learned)):
        dplan.set_scales(scales)
        info, pm, st = ps.decode(dplan, dl[0], w["D"], w["L"])
        torch.cuda.synchronize()
        fer[name] = float((info != dmsg).any(dim=1).double().mean().item())
    dplan.set_scales(None)
    # the same scales in the plain bit-level decoder of PC(256,128), D = 16,
    # L = 4, no CRC, at 2.5 dB: a tree of 8 stages takes the scales learned for
    # stages 0 .. 7 (child nodes of 1 .. 128 values)
    c1 = dict(N=256, K=128, crc=0, D=16, L=4, frames=g["fer_frames"], ebn0=(2.5,), seed=1, design_snr_db=0.0)
    n1 = c1["N"].bit_length() - 1
    p1 = ps.Plan(c1["N"], c1["K"], ps.polar_construct(c1["N"], c1["K"], c1["design_snr_db"]), fast_nodes=False)
    l1, m1 = make_gpu_inputs(ps, p1, c1["frames"], rank, c1)
    fer1 = {}
    for name, scales in (("unit", None), ("learned", learned[:n1].copy())):
        p1.set_scales(scales)
        info, pm, st = ps.decode(p1, l1[0], c1["D"], c1["L"])
        torch.cuda.synchronize()
        fer1[name] = float((info != m1).any(dim=1).double().mean().item())
    p1.set_scales(None)
    del l1, m1
    if rank == 0:
        line = {"metric": "genie-aided SC forward+backward frames/s", "value": B * world / (ms / 1e3),
                "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{B} frames of PC({N},{K}) at {g['ebn0'][0]} dB, genie-aided SC with {n} "
                                       f"per-stage scales, loss and d loss/d scales per step",
                           "loss_unit_scales": loss0, "loss_learned": loss1, "train_steps": g["train_steps"],
                           "learned_scales": [round(float(v), 5) for v in learned],
                           "scs_fer_check": {"workload": f"PC({w['N']},{w['K']}) CRC-{w['crc']} D={w['D']} "
                                                         f"L={w['L']}, {w['frames']} frames at 2.0 dB",
                                             "fer_unit_scales": fer["unit"], "fer_learned_scales": fer["learned"]},
                           "plain_scs_fer_check": {"workload": f"PC({c1['N']},{c1['K']}) bit-level, no CRC, "
                                                               f"D={c1['D']} L={c1['L']}, {c1['frames']} frames at "
                                                               f"{c1['ebn0'][0]} dB, scales of stages 0..{n1 - 1}",
                                                   "fer_unit_scales": fer1["unit"],
                                                   "fer_learned_scales": fer1["learned"]}},
                "roofline": roof, "cpu_baseline": cpu, "clocks": sampler.summary() if sampler else None}
        print(json.dumps(line), flush=True)


def gsc_cpu_baseline(g, frames: int = 4096):
    """The double-precision oracle's loss and gradient on a bounded sample of
    the gradient workload (host-made frames), in frames/s, on all host cores."""
    import numpy as np

    import oracle
    import workloads as W

    threads = os.cpu_count() or 1
    N, K = g["N"], g["K"]
    fr = oracle.construct(N, K, g["design_snr_db"])
    msg = W.message_bits(int(g["seed"]) + 77, frames, K)
    cw = oracle.encode_batch(msg, N, K, fr, 0)
    llr = W.bpsk_awgn_llr(cw, W.awgn_noise(int(g["seed"]) + 77, frames, N), W.sigma_from_ebn0(g["ebn0"][0], K / N))
    u = np.zeros((frames, N), np.uint8)
    u[:, fr == 0] = msg
    scales = np.ones(N.bit_length() - 1)
    parts = np.array_split(np.arange(frames), threads)
    from concurrent.futures import ThreadPoolExecutor

    def run(idx):
        if idx.size:
            oracle.gsc_loss_grad(llr[idx].astype(np.float64), u[idx], fr, scales)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, parts))
    dt = time.perf_counter() - t0
    return {"value": frames / dt, "unit": "frames/s", "cores": threads, "kind": "oracle",
            "sample": f"{frames} host-made frames, loss and gradient in double precision, wall time {dt:.2f} s "
                      f"on {threads} host threads"}


def mixed_cpu_baseline(frames: int, w=MIXED):
    """The oracle on a bounded sample of the mixed workload: the first
    `frames` (N, K, D, Eb/N0) draws, with messages, encodings and LLRs made on
    the host per code, decoded frame by frame on all host cores."""
    import numpy as np

    import oracle
    import workloads as W

    threads = os.cpu_count() or 1
    draw = W.mixed_frames(int(w["seed"]), frames)
    jobs = []
    for (N, K) in sorted(set(zip(draw["N"].tolist(), draw["K"].tolist()))):
        sel = np.nonzero((draw["N"] == N) & (draw["K"] == K))[0]
        fr = oracle.construct(N, K, w["design_snr_db"])
        seed = int(w["seed"]) * 31 + N * 7 + K
        msg = W.message_bits(seed, sel.size, K - w["crc"])
        cw = oracle.encode_batch(msg, N, K, fr, w["crc"])
        sig = np.array([W.sigma_from_ebn0(float(e), K / N) for e in draw["ebn0_db"][sel]])
        llr = W.bpsk_awgn_llr(cw, W.awgn_noise(seed, sel.size, N), sig)
        jobs += [(llr[j], N, K, fr, int(draw["D"][b])) for j, b in enumerate(sel)]
    from concurrent.futures import ThreadPoolExecutor

    def run(j):
        llr, N, K, fr, D = j
        oracle.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=D, crc_len=w["crc"])

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, jobs))
    dt = time.perf_counter() - t0
    bits = sum(j[2] - w["crc"] for j in jobs)
    return {"value": bits / dt / 1e9, "unit": "Gbit/s", "cores": threads, "kind": "oracle",
            "sample": f"first {frames} draws of the mixed workload (host-made frames), decode-only wall time "
                      f"{dt:.2f} s on {threads} host threads"}


# ------------------------------------------------------------ served workload
SERVE = dict(rate=5e6, seconds=10.0, pool=1 << 18, seed=5, arena_bytes=2 << 30, interval_s=2e-3, compare_seconds=0.5)


def bench_serve(args, rank: int, world: int, local_rank: int) -> None:
    """Poisson arrivals drawn from the mixed workload's code/D/Eb-N0 mix,
    served by the continuous-batching engine and by the one-size-per-launch
    baseline on the same request stream; p50/p99 latency and throughput."""
    import numpy as np
    import torch

    import paper_1809_03606_gb300 as ps
    import workloads as W

    torch.cuda.set_device(local_rank)
    ps.load(build_if_missing=True)
    rate = float(args.serve_rate or SERVE["rate"])
    seconds = float(args.serve_seconds or SERVE["seconds"])
    m = make_mixed_inputs(ps, SERVE["pool"], rank, dict(MIXED, seed=SERVE["seed"]))
    pool = m["llr"].cpu().numpy()
    pool_off = m["llr_off"]
    pset = ps.PlanSet(m["plans"])
    P = SERVE["pool"]
    kmsg_pool = (m["Ks"] - MIXED["crc"]).astype(np.int64)

    def stream(rate_hz, dur, seed):
        arr = W.poisson_arrivals(seed, rate_hz, dur)
        R = arr.size
        p = np.arange(R) % P
        req = np.stack([m["idx"][p], m["D"][p], m["D"][p], p], axis=1).astype(np.int32)
        return req, arr, p

    def summarize(out, arr, p):
        lat = out["latency"]
        ok = np.isfinite(lat)
        t_end = out["report"]["seconds_to_last_completion"]
        R = arr.size
        bits = float(kmsg_pool[p[ok]].sum())
        res = {"requests": int(R), "completed": int(ok.sum()), "seconds": t_end,
                "throughput_req_s": float(ok.sum()) / t_end if t_end > 0 else None,
                "info_gbps": bits / t_end / 1e9 if t_end > 0 else None,
                "p50_ms": float(np.percentile(lat[ok], 50) * 1e3) if ok.any() else None,
                "p99_ms": float(np.percentile(lat[ok], 99) * 1e3) if ok.any() else None,
                "report": out["report"]}
        svc = out.get("service")
        if svc is not None and ok.any():
            wait_ = lat[ok] - svc[ok]
            res.update({"p50_service_ms": float(np.percentile(svc[ok], 50) * 1e3),
                        "p99_service_ms": float(np.percentile(svc[ok], 99) * 1e3),
                        "p50_wait_ms": float(np.percentile(wait_, 50) * 1e3),
                        "p99_wait_ms": float(np.percentile(wait_, 99) * 1e3)})
        return res

    arena = SERVE["arena_bytes"] // 4
    wait = max(60.0, 4 * seconds)
    # below saturation: a short sweep
    sweep = []
    for r_hz in (2e5, 5e5, 1e6, 1.5e6):
        req, arr, p = stream(r_hz, min(2.0, seconds), SERVE["seed"] + int(r_hz))
        out = ps.polar_serve(pset, req, arr, pool, pool_off, arena, wait_s=wait)
        sweep.append(dict(offered_req_s=r_hz, rc=out["rc"], **{k: v for k, v in summarize(out, arr, p).items() if k != "report"}))
    # the configured load served in full; both engines on the same prefix of it
    req, arr, p = stream(rate, seconds, SERVE["seed"])
    served = ps.polar_serve(pset, req, arr, pool, pool_off, arena, wait_s=wait)
    s_sum = summarize(served, arr, p)
    cut = int(np.searchsorted(arr, SERVE["compare_seconds"]))
    sp = ps.polar_serve(pset, req[:cut], arr[:cut], pool, pool_off, arena, wait_s=wait)
    bp = ps.polar_serve_baseline(pset, req[:cut], arr[:cut], pool, pool_off, arena, interval_s=SERVE["interval_s"],
                                 wait_s=20 * wait)
    same = bool(np.array_equal(sp["pm"].view(np.uint32), bp["pm"].view(np.uint32)) and
                np.array_equal(sp["status"], bp["status"]))
    sp_sum, b_sum = summarize(sp, arr[:cut], p[:cut]), summarize(bp, arr[:cut], p[:cut])
    if rank == 0:
        line = {"metric": "served decode: info Gbit/s with p50/p99 request latency", "value": s_sum["info_gbps"],
                "unit": "Gbit/s", "n_gpus": world, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"Poisson arrivals {rate:.3g} requests/s for {seconds:g} s, each request a "
                                       f"frame of the mixed-batch mix (pool of {P} frames cycled)",
                           "arena_bytes": SERVE["arena_bytes"], "served": s_sum,
                           "compare_prefix_seconds": SERVE["compare_seconds"], "served_prefix": sp_sum,
                           "one_size_per_launch_prefix": dict(b_sum, interval_s=SERVE["interval_s"]),
                           "identical_outputs": same, "load_sweep": sweep}}
        print(json.dumps(line), flush=True)


def measure_subsystems(args, rank: int, local_rank: int) -> dict:
    """Compact measurements of the other workloads, for the default line: the
    genie-aided SC gradient step (65,536 frames), one sweep of the paper's
    decoder setting (7 x 2^19 frames, memory stack), and a short serving run
    (1 s of 5 M req/s Poisson arrivals, the first 0.5 s through both engines
    with identical outputs, and 1 s at 0.5 M req/s split into waiting and
    service time)."""
    import numpy as np
    import torch

    import paper_1809_03606_gb300 as ps
    import workloads as W

    out = {}
    # genie-aided SC: forward + reverse with unit scales
    g = dict(GSC)
    N, K = g["N"], g["K"]
    n = N.bit_length() - 1
    plan = ps.Plan(N, K, ps.polar_construct(N, K, g["design_snr_db"]), fast_nodes=False)
    llrs, _ = make_gpu_inputs(ps, plan, g["frames"], rank, g)
    msg = W.message_bits(rank_seed(rank, g), g["frames"], K)
    u = torch.from_numpy(ps.u_from_messages(plan, msg)).cuda()
    ones = torch.ones(n, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ps.gsc_loss_grad(plan, llrs[0], u, ones)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        ps.gsc_loss_grad(plan, llrs[0], u, ones)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    out["gsc"] = {"workload": f"{g['frames']} frames of PC({N},{K}) at 2.0 dB, forward + reverse, {n} stage scales",
                  "ms_per_step": ms, "frames_per_s": g["frames"] / (ms / 1e3)}
    del llrs, u
    torch.cuda.empty_cache()

    # the paper's decoder setting: one warm-up and two timed sweeps
    w = dict(PAPER)
    fr = ps.polar_construct(w["N"], w["K"], w["design_snr_db"])
    plan = ps.Plan(w["N"], w["K"], fr, fast_nodes=w["fast"], crc=w["crc"], systematic=w["systematic"])
    llrs, d_msg = make_gpu_inputs(ps, plan, w["frames"], rank, w)
    B = w["frames"]
    res = [(torch.empty((B, plan.msg_words), dtype=torch.int32, device="cuda"),
            torch.empty(B, dtype=torch.float32, device="cuda"), torch.empty(B, dtype=torch.int8, device="cuda"))
           for _ in llrs]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in llrs]
    for rep in range(3):
        for p_, x in enumerate(llrs):
            if rep:
                ev[p_][0].record()
            ps.scs_decode_batch(plan, x, w["D"], w["L"], *res[p_])
            if rep:
                ev[p_][1].record()
        torch.cuda.synchronize()
        if rep == 1:
            ms1 = [e[0].elapsed_time(e[1]) for e in ev]
    ms2 = [e[0].elapsed_time(e[1]) for e in ev]
    pt_ms = [min(a, b) for a, b in zip(ms1, ms2)]
    kmsg = w["K"] - w["crc"]
    fer = [float((r[0] != d_msg).any(dim=1).double().mean().item()) for r in res]
    out["paper"] = {"workload": workload_name(w), "info_gbps": len(llrs) * B * kmsg / (sum(pt_ms) / 1e3) / 1e9,
                    "ms_per_sweep": sum(pt_ms),
                    "per_point": [{"ebn0_db": e, "ms": t, "info_gbps": B * kmsg / (t / 1e3) / 1e9, "fer": f}
                                  for e, t, f in zip(w["ebn0"], pt_ms, fer)]}
    del llrs, res, d_msg
    torch.cuda.empty_cache()

    # serving: continuous batching against one size per launch on the same stream
    m = make_mixed_inputs(ps, SERVE["pool"], rank, dict(MIXED, seed=SERVE["seed"]))
    pool = m["llr"].cpu().numpy()
    pset = ps.PlanSet(m["plans"])
    P = SERVE["pool"]
    kmsg_pool = (m["Ks"] - MIXED["crc"]).astype(np.int64)
    arena = SERVE["arena_bytes"] // 4

    def stream(rate_hz, dur, seed):
        arr = W.poisson_arrivals(seed, rate_hz, dur)
        p_ = np.arange(arr.size) % P
        req = np.stack([m["idx"][p_], m["D"][p_], m["D"][p_], p_], axis=1).astype(np.int32)
        return req, arr, p_

    def summary(o, p_):
        lat = o["latency"]
        ok = np.isfinite(lat)
        t_end = o["report"]["seconds_to_last_completion"]
        r = {"requests": int(lat.size), "completed": int(ok.sum()),
             "throughput_req_s": float(ok.sum()) / t_end if t_end > 0 else None,
             "info_gbps": float(kmsg_pool[p_[ok]].sum()) / t_end / 1e9 if t_end > 0 else None,
             "p50_ms": float(np.percentile(lat[ok], 50) * 1e3), "p99_ms": float(np.percentile(lat[ok], 99) * 1e3)}
        svc = o.get("service")
        if svc is not None:
            r["p99_service_ms"] = float(np.percentile(svc[ok], 99) * 1e3)
            r["p99_wait_ms"] = float(np.percentile((lat - svc)[ok], 99) * 1e3)
        return r

    req, arr, p_ = stream(SERVE["rate"], 1.0, SERVE["seed"])
    full = ps.polar_serve(pset, req, arr, pool, m["llr_off"], arena, wait_s=60.0)
    cut = int(np.searchsorted(arr, SERVE["compare_seconds"]))
    sp = ps.polar_serve(pset, req[:cut], arr[:cut], pool, m["llr_off"], arena, wait_s=60.0)
    bp = ps.polar_serve_baseline(pset, req[:cut], arr[:cut], pool, m["llr_off"], arena,
                                 interval_s=SERVE["interval_s"], wait_s=600.0)
    same = bool(np.array_equal(sp["pm"].view(np.uint32), bp["pm"].view(np.uint32)) and
                np.array_equal(sp["status"], bp["status"]))
    lreq, larr, lp = stream(5e5, 1.0, SERVE["seed"] + 7)
    low = ps.polar_serve(pset, lreq, larr, pool, m["llr_off"], arena, wait_s=60.0)
    out["serving"] = {"workload": "Poisson arrivals from the mixed mix (pool of 262,144 frames cycled)",
                      "offered_5M_req_s_for_1s": summary(full, p_),
                      "prefix_0.5s": {"continuous_batching": summary(sp, p_[:cut]),
                                      "one_size_per_launch": summary(bp, p_[:cut]), "identical_outputs": same},
                      "offered_0.5M_req_s_for_1s": summary(low, lp),
                      "rc": [int(full["rc"]), int(sp["rc"]), int(bp["rc"]), int(low["rc"])]}
    del m, pool
    torch.cuda.empty_cache()
    return out


def cpu_baseline(frames: int, w=WORKLOAD):
    import os as _os

    threads = _os.cpu_count() or 1
    fr, msg, llrs = oracle_sample_inputs(frames, 0, w)
    dt, _ = run_oracle(fr, llrs, threads, w)
    kmsg = w["K"] - w["crc"]
    nf = frames * len(llrs)
    return {"value": nf * kmsg / dt / 1e9, "unit": "Gbit/s", "cores": threads, "kind": "oracle",
            "sample": f"first {frames} frames of each of the {len(llrs)} Eb/N0 points ({nf} frames), "
                      f"decode-only wall time {dt:.2f} s on {threads} host threads"}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["sweep", "mixed", "serve", "gsc", "paper"], default="sweep",
                    help="sweep: the PC(1024,512) Eb/N0 sweep (default); mixed: the 2M-frame mixed batch; "
                         "serve: Poisson-arrival serving; gsc: genie-aided SC gradient and learned scales; "
                         "paper: the paper's decoder setting (CRC-24C, D = 8192, L = 8) over 0-3 dB")
    ap.add_argument("--serve-rate", type=float, default=0.0, help="serve workload: arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=0.0, help="serve workload: seconds of arrivals")
    ap.add_argument("--frames", type=int, default=0,
                    help="frames per Eb/N0 point (default 1048576; paper workload 524288; gsc 65536)")
    ap.add_argument("--cpu-frames", type=int, default=8192, help="oracle sample per point for cpu_baseline")
    ap.add_argument("--ref-frames", type=int, default=1024, help="oracle sample per point per step (reference arm)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-lpt", action="store_true", help="mixed workload: claim frames in batch order")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="sweep: skip the mixed-batch comparison object")
    ap.add_argument("--no-extras", action="store_true",
                    help="sweep: skip the compact gradient, paper-setting and serving measurements")
    ap.add_argument("--systematic", action="store_true", help="sweep: systematic encoding and decoding")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if args.impl == "ours":
            import torch

            torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    try:
        if args.impl == "reference":
            bench_reference(args, rank, world)
        elif args.workload == "mixed":
            bench_mixed(args, rank, world, local_rank)
        elif args.workload == "serve":
            bench_serve(args, rank, world, local_rank)
        elif args.workload == "gsc":
            bench_gsc(args, rank, world, local_rank)
        elif args.workload == "paper":
            bench_ours(args, rank, world, local_rank, base=PAPER)
        else:
            bench_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
