"""Benchmark: raw emulated frames per second of the batched emulation path.

One step = one pass of the whole path (interpreter for F frames with TIA
logging, rasteriser, preprocessing, on-device reset) over every env of the
workload.  Default workload: 4096 envs over 8 seeded 4 KB sprite cartridges,
frame skip 4, 84x84x4 luma stack output, uniform random actions.

Timing: W untimed warm-up steps, then K steps each timed on the device with
CUDA events on the step's stream; L2 is flushed (a 256 MB write) before every
timed step, outside the events.  value = envs * F * K / (sum of step times),
max over ranks.  e2e = the same metric through the host-buffer entry point
(actions copied in, observations, rewards and dones copied out every step).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--form plain|batched] [--config 2]
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

METRIC = "raw emulated frames/sec on 1 GB300 vs plain GPU path and CPU oracle; p50/p99 step ms"
SM_COUNT, SMSP_PER_SM, SM_MAX_MHZ = 152, 4, 2070.0

# Warp instructions issued per env-frame by the interpreter kernel (with the
# split form: its CPU and TIA warps together) and DRAM bytes per env-step,
# from the ncu captures summarised in profiles/interpreter_batched_sprite4096.md (smsp__inst_executed.sum and
# dram__bytes_read.sum + dram__bytes_write.sum of one launch, divided by its
# 16384 env-frames / 4096 env-steps), keyed by (workload config, form, envs
# per warp, tia_warps).  They hold for the interpreter version captured there; a key
# without an entry reports achieved = null.
INTERP_WARP_INST_PER_ENV_FRAME = {(2, "batched", 32, 2): 424750280 / 16384}
INTERP_DRAM_BYTES_PER_ENV_STEP = {(2, "batched", 32, 2): (1278720 + 112128) / 4096}
# Algorithmic bytes of the fused rasterise + preprocess kernel per env-step,
# besides 4 bytes per logged TIA write: snapshots and record counts of the two
# rendered frames (2 x 64 + 2 x 8), the three older stack planes read from the
# ring, the 84x84x4 stack written out, the new plane written to the ring and
# the ring head.
FUSED_FIXED_BYTES_PER_ENV_STEP = 2 * 64 + 2 * 8 + 3 * 7056 + 4 * 7056 + 7056 + 1
# DRAM bytes per env-step of the fused kernel from the capture summarised in
# profiles/raster_preprocess_fused_sprite4096.md.
FUSED_DRAM_BYTES_PER_ENV_STEP = {2: (109457408 + 94802688) / 4096}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--form", default="batched", choices=["plain", "batched"])
    p.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5])
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-clients", type=int, default=64)
    p.add_argument("--n-envs", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--envs-per-warp", type=int, default=0)
    p.add_argument("--envs-per-block", type=int, default=0)
    p.add_argument("--warps-per-frame", type=int, default=0)
    p.add_argument("--tia-warps", type=int, default=0, choices=[0, 1, 2])
    return p.parse_args()


_REDUCE_DEVICE = "cuda"


def dist_setup(backend: str = "nccl"):
    """Replicas: one process per GPU from torchrun's environment.  Only the
    timing and the whole-job frame count cross ranks (no collective touches
    the emulation path)."""
    global _REDUCE_DEVICE
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    _REDUCE_DEVICE = "cuda" if backend == "nccl" else "cpu"
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return ws, rank, local


def replica_env_keys(n_envs: int, rank: int):
    """Env keys of a rank's replica of the workload: disjoint across ranks."""
    import numpy as np
    return np.arange(n_envs, dtype=np.uint32) + np.uint32(rank * n_envs)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_REDUCE_DEVICE)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_REDUCE_DEVICE)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def cpu_oracle_rate(w, seconds, seed=77, max_envs=512):
    """The oracle timed on the host cores on a bounded sample of the workload:
    the first `max_envs` envs (same cartridges, keys and actions), stepped
    until `seconds` of wall time have passed."""
    import numpy as np

    from oracle import OracleEnvs
    from paper_1907_08467_gb300 import synth
    n = min(max_envs, w.n_envs)
    idx = np.linspace(0, w.n_envs - 1, n).astype(np.int64)
    cores = os.cpu_count() or 1
    o = OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms], [r.gameover_addr for r in w.roms],
                   [w.env_rom[i] for i in idx], luma=synth.luma_table(), env_key=idx, seed=w.seed,
                   sticky=w.sticky, output_mode=w.output_mode, frameskip=w.frameskip)
    acts = synth.actions(seed, 4096, w.n_envs)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds and steps < 4096:
        o.step(acts[steps][idx], n_threads=cores)
        steps += 1
    dt = time.perf_counter() - t0
    frames = n * w.frameskip * steps
    return {"value": frames / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} of {w.n_envs} envs (same cartridges, keys, actions) x {steps} steps, "
                      f"{frames} frames in {dt:.1f} s on {cores} threads"}


def reference_arm(args, w, ws, rank):
    """The oracle as the reference arm: timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    sample_seconds = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    import numpy as np

    from oracle import OracleEnvs
    from paper_1907_08467_gb300 import synth
    n = min(256, w.n_envs)
    idx = np.linspace(0, w.n_envs - 1, n).astype(np.int64)
    cores = os.cpu_count() or 1
    o = OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms], [r.gameover_addr for r in w.roms],
                   [w.env_rom[i] for i in idx], luma=synth.luma_table(), env_key=idx, seed=w.seed,
                   sticky=w.sticky, output_mode=w.output_mode, frameskip=w.frameskip)
    acts = synth.actions(78, 100000, n)
    s = 0
    for _ in range(args.warmup):
        o.step(acts[s], n_threads=cores)
        s += 1
    times, frames = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        k = 0
        while True:
            o.step(acts[s], n_threads=cores)
            s += 1
            k += 1
            if time.perf_counter() - t0 >= sample_seconds / 4 or k >= 64:
                break
        times.append(time.perf_counter() - t0)
        frames += n * w.frameskip * k
    total = sum(times)
    val = frames / total
    sample = f"{n} of {w.n_envs} envs x {s} steps on {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "n_envs": w.n_envs, "frameskip": w.frameskip, "sample_envs": n},
        "cpu_baseline": {"value": val, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def serve_bench(args, ws, rank, local):
    """Serving loop: N native client threads (closed loop, Exp(2 ms) think
    time) open sessions of U{1..2048} envs on the 32 banked cartridges, step
    them (stacks, rewards and dones back to pinned host memory) and close
    them; admission under a 40 GB device budget.  value = aggregate emulated
    frames/s over the run; p50/p99 = request latency (submit to outputs in
    place)."""
    import torch

    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.server import AtariServer
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle has no serving loop; the serving "
                              "workload is measured against the plain and batched GPU paths"}), flush=True)
        return
    torch.cuda.set_device(local)
    w = synth.workload(3, n_envs=32)
    clients, max_envs = args.serve_clients, 2048
    srv = AtariServer.from_roms(w.roms, budget_bytes=40 << 30, max_slots=clients * max_envs, sticky=True,
                                seed=w.seed)
    warm = srv.loadgen(n_clients=clients, seconds=max(1.0, float(args.warmup)), think_mean_ms=2.0, min_envs=1,
                       max_envs=max_envs, session_steps_mean=100, seed=1000 + rank, want_obs=True)
    clocks = ClockSampler(local)
    barrier(ws)
    l0 = srv.stats()["launches"]
    clocks.start()
    r = srv.loadgen(n_clients=clients, seconds=args.serve_seconds, think_mean_ms=2.0, min_envs=1,
                    max_envs=max_envs, session_steps_mean=100, seed=1 + rank, want_obs=True)
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    value = allreduce_sum(r["frames"], ws) / allreduce_max(r["seconds"], ws)
    if rank == 0:
        reqs = max(1, r["requests"])
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": r["requests"],
            "warmup": warm["requests"], "ms_per_step": r["mean_ms"], "p50_step_ms": r["p50_ms"],
            "p99_step_ms": r["p99_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic (seeded cartridges, client actions and arrivals)",
            "config": {"workload": f"serving: {clients} clients, sessions U{{1..{max_envs}}} envs on 32 banked "
                                   "4k/f8/f6 roms, sticky, closed loop Exp(2 ms) think, geometric sessions "
                                   "(mean 100 steps), 40 GB budget",
                       "seconds": r["seconds"], "budget_bytes": st["budget_bytes"], "capacity": st["capacity"],
                       "per_env_bytes": st["per_env_bytes"], "parallelism": f"replicas x{ws}",
                       "l2": "inputs (slots of all admitted sessions) far larger than L2"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": r["h2d_bytes"] // reqs,
                    "d2h_bytes_per_step": r["d2h_bytes"] // reqs},
            "serving": {"requests": r["requests"], "sessions": r["sessions"], "ticks": r["ticks"],
                        "mean_tick_envs": r["mean_tick_envs"], "latency_ms": {"p50": r["p50_ms"], "p99": r["p99_ms"],
                                                                              "max": r["max_ms"], "mean": r["mean_ms"]},
                        "admission_wait_ms": {"p50": r["admit_p50_ms"], "p99": r["admit_p99_ms"]}},
            "gpu_launches": int(st["launches"] - l0), "clocks": clk, "roofline": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_setup()
    from paper_1907_08467_gb300 import synth
    if args.config == 4:
        serve_bench(args, ws, rank, local)
        return
    w = synth.workload(args.config, n_envs=args.n_envs)
    if args.impl == "reference":
        reference_arm(args, w, ws, rank)
        return
    import numpy as np
    import torch

    from paper_1907_08467_gb300.env import FORM_BATCHED, FORM_PLAIN, AtariEnv
    torch.cuda.set_device(local)
    form = FORM_BATCHED if args.form == "batched" else FORM_PLAIN
    # replicas: each rank runs the whole workload with its own env keys
    env_key = replica_env_keys(w.n_envs, rank)
    env = AtariEnv([r.data for r in w.roms], [(r.score_addr, r.gameover_addr) for r in w.roms], w.env_rom,
                   luma=synth.luma_table(), env_key=env_key, frameskip=w.frameskip, sticky=w.sticky,
                   output_mode=w.output_mode, form=form, seed=w.seed, envs_per_warp=args.envs_per_warp,
                   envs_per_block=args.envs_per_block, raster_warps_per_frame=args.warps_per_frame,
                   tia_warps=args.tia_warps)
    K, W = args.steps, args.warmup
    acts = torch.from_numpy(synth.actions(100 + rank, K + W, w.n_envs)).cuda()
    obs, rew, done = env.alloc_outputs()
    inference = args.config == 5
    if inference:
        # inference-path loop: the policy picks every action on the device and
        # each step appends the newest plane and reward to a 5-deep ring
        weights = torch.from_numpy(synth.policy_weights(w.seed).view(np.int16)).cuda()
        ring = torch.zeros((5, w.n_envs, 84 * 84), dtype=torch.uint8, device="cuda")
        ring_r = torch.zeros((5, w.n_envs), dtype=torch.float32, device="cuda")
        obs.zero_()
        pol_act = torch.empty(w.n_envs, dtype=torch.uint8, device="cuda")
        t_ring = [0]

        def do_step(a):
            env.rollout(weights, 1, obs, pol_act, rew, done, ring, ring_r, ring_start=t_ring[0])
            t_ring[0] += 1
    else:
        def do_step(a):
            env.step(a, obs, rew, done)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for s in range(W):
        do_step(acts[s])
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    instr = 0
    logrec = 0
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for s in range(K):
        flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        do_step(acts[W + s])
        ev[s][1].record(stream)
        a, b = env.counters()
        instr += a
        logrec += b
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    barrier(ws)
    clk = clocks.stop()
    # second pass, same launch configuration, CUDA events around every kernel
    # (the batched form launches its kernels directly instead of replaying
    # the captured graph while profiling)
    prof_steps = max(3, min(K, 10))
    pacts = torch.from_numpy(synth.actions(300 + rank, prof_steps, w.n_envs)).cuda()
    env.profile_read()
    env.profile(True)
    for s in range(prof_steps):
        flush.fill_(s & 0xFF)
        do_step(pacts[s])
    torch.cuda.synchronize()
    env.profile(False)
    prof = env.profile_read()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_s = sum(step_ms) / 1000.0
    total_s_max = allreduce_max(total_s, ws)
    frames = w.n_envs * w.frameskip * K
    frames_all = allreduce_sum(frames, ws)
    value = frames_all / total_s_max
    ms_sorted = sorted(step_ms)
    p50 = ms_sorted[len(ms_sorted) // 2]
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(round(0.99 * (len(ms_sorted) - 1))))]
    gpu_launches = int(round(sum(v[1] for v in prof.values()) * K / prof_steps))

    # e2e through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e and not inference:
        ha = torch.from_numpy(synth.actions(200 + rank, 8 + K, w.n_envs)).pin_memory()
        ho = torch.empty(env.obs_shape(), dtype=torch.uint8).pin_memory()
        hr = torch.empty(w.n_envs, dtype=torch.int32).pin_memory()
        hd = torch.empty(w.n_envs, dtype=torch.uint8).pin_memory()
        for s in range(3):
            env.step_host(ha[s], ho, hr, hd)
        barrier(ws)
        t0 = time.perf_counter()
        for s in range(K):
            env.step_host(ha[3 + s], ho, hr, hd)
        dt = allreduce_max(time.perf_counter() - t0, ws)
        e2e = {"value": frames_all / dt, "unit": "frames/s", "h2d_bytes_per_step": int(ha[0].numel()),
               "d2h_bytes_per_step": int(ho.numel() + hr.numel() * 4 + hd.numel())}

    # roofline of the dominant kernel (the interpreter): issue-slot use
    interp_ms, interp_n = prof.get("interpreter", (0.0, 0))
    roof = None
    if interp_n:
        dur = interp_ms / interp_n / 1000.0
        shape_key = (args.config, args.form, env.launch_shape()[0], env.launch_shape()[4])
        per = INTERP_WARP_INST_PER_ENV_FRAME.get(shape_key)
        peak = SM_COUNT * SMSP_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
        ach = per * w.n_envs * w.frameskip / dur / 1e9 if per else None
        tb = INTERP_DRAM_BYTES_PER_ENV_STEP.get(shape_key)
        roof = {"bound": "alu", "kernel": "interpreter", "achieved": ach, "peak": peak, "unit": "Gwarp-inst/s",
                "frac": (ach / peak) if ach else None, "traffic": tb * w.n_envs if tb else None,
                "launch_ms": dur * 1000.0,
                "share_of_step": interp_ms / max(1e-9, sum(v[0] for v in prof.values())),
                "m6502_inst_per_s": instr / total_s / 1e6 if instr else None,
                "peak_source": "152 SMs x 4 schedulers x 2070 MHz (issue slots)"}
    # the fused rasterise + preprocess kernel against HBM (its design bound)
    roof2 = None
    fused_ms, fused_n = prof.get("fused_raster_preprocess", (0.0, 0))
    if fused_n and not inference:
        dur = fused_ms / fused_n / 1000.0
        per_step = FUSED_FIXED_BYTES_PER_ENV_STEP + 4.0 * (logrec / K if K else 0.0) / w.n_envs
        hbm = load_peaks().get("hbm_gbs")
        ach = per_step * w.n_envs / dur / 1e9
        tb = FUSED_DRAM_BYTES_PER_ENV_STEP.get(args.config)
        roof2 = {"bound": "hbm", "kernel": "fused_raster_preprocess", "achieved": ach,
                 "peak": hbm if hbm else 6800.0, "unit": "GB/s", "frac": ach / (hbm if hbm else 6800.0),
                 "traffic": tb * w.n_envs if tb else None, "algorithmic_bytes_per_env_step": per_step,
                 "launch_ms": dur * 1000.0,
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if hbm else "fallback 6.8 TB/s"}
    kernels = {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]} for k, v in prof.items()}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": 1000.0 * total_s_max / K, "p50_step_ms": p50, "p99_step_ms": p99,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded cartridges and actions)",
            "config": {"workload": w.name + (" (policy + step + ring per step)" if inference else ""),
                       "n_envs": w.n_envs, "n_roms": len(w.roms), "frameskip": w.frameskip,
                       "output": "84x84x4 uint8 stack" if w.output_mode == 1 else "210x160 palette frame",
                       "form": args.form, "l2": "flushed (256 MB write) before each timed step",
                       "launch_shape": dict(zip(["envs_per_warp", "envs_per_block", "warps_per_frame", "grid",
                                                 "tia_warps"], env.launch_shape())),
                       "parallelism": f"replicas x{ws}"},
            "e2e": e2e, "roofline": roof, "roofline_fused": roof2, "kernels": kernels, "gpu_launches": gpu_launches,
            "m6502_inst_per_step": instr / K if K else None, "tia_log_records_per_step": logrec / K if K else None,
            "wall_s": wall, "clocks": clk, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
