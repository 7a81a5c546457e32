"""Benchmark: raw emulated frames per second of the batched emulation path.

One step = one pass of the whole path (interpreter for F frames with TIA
logging, rasteriser, preprocessing, on-device reset) over every env of the
workload.  Default workload (the largest single-GPU configuration): 32768
envs over 32 seeded banked cartridges (12 x 4 KB, 10 x F8, 10 x F6), sticky
actions p = 1/4 from each env's Philox stream, frame skip 4, 84x84x4 luma
stack output, uniform random actions.

Timing: W untimed warm-up steps, then K steps each timed on the device with
CUDA events on the step's stream; L2 is flushed (a 256 MB write) before every
timed step, outside the events.  value = envs * F * K / (sum of step times),
max over ranks.  In the same process the plain one-launch-per-kernel form is
timed the same way on the same workload ("plain"), and e2e repeats the
batched step through the host-buffer entry point (actions copied in,
observations, rewards and dones copied out every step).  Unless --no-extras,
the line also carries short runs of the inference-path loop (16384 envs,
policy + step + ring append per step) and of the serving loop.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--form plain|batched] [--config 1|2|3|4|5]
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "raw emulated frames/sec on 1 GB300 vs plain GPU path and CPU oracle; p50/p99 step ms"
SM_COUNT, SMSP_PER_SM, SM_MAX_MHZ = 152, 4, 2070.0

# Warp instructions the interpreter kernel issues per emulated 6502
# instruction (its CPU and TIA warps together in the split form), and its DRAM
# bytes per env-step, from one ncu capture per (kernel, envs per warp,
# workload config): smsp__inst_executed.sum and dram__bytes_read.sum +
# dram__bytes_write.sum of one launch, divided by the 6502 instructions that
# launch executed (counted by the kernel itself) and by its env-steps.  The
# bench multiplies the ratio by the instructions executed in the profiled
# launches, counted live, and divides by their live CUDA-event duration.
# A shape captured on another workload is used with its source named; a shape
# never captured reports achieved = null.
INTERP_CAPTURES = {
    # (kernel, envs per warp, opcode dispatch, config): (warp-inst per executed 6502 instruction, DRAM bytes per env-step)
    ("k_interp_split", 32, 1, 3): (2234457806 / 433965025, (13179648 + 114831104) / 32768),
    ("k_interp_split", 32, 2, 3): (2213124575 / 433965025, (13961216 + 124522240) / 32768),
    ("k_interp_split", 32, 1, 2): (445471194 / 94159103, (1266688 + 88064) / 4096),
    ("k_interp_split", 32, 2, 2): (442946243 / 94159103, (1260288 + 104192) / 4096),
}
# Algorithmic bytes of the fused rasterise + preprocess kernel per env-step,
# besides 4 bytes per logged TIA write: snapshots and record counts of the two
# rendered frames (2 x 64 + 2 x 8), the three older stack planes read from the
# ring, the 84x84x4 stack written out, the new plane written to the ring and
# the ring head.
FUSED_FIXED_BYTES_PER_ENV_STEP = 2 * 64 + 2 * 8 + 3 * 7056 + 4 * 7056 + 7056 + 1
# Warp instructions per env-step of the fused kernel (it is bound by issue,
# not HBM), from the same captures: smsp__inst_executed.sum / env-steps.
FUSED_WARP_INST_PER_ENV_STEP = {3: 5979554498 / 32768, 2: 711969603 / 4096}
# DRAM bytes per env-step of the fused kernel, from an ncu capture per config.
FUSED_DRAM_BYTES_PER_ENV_STEP = {3: (863958016 + 1106787000) / 32768, 2: (109476096 + 94397696) / 4096}


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--form", default="batched", choices=["plain", "batched"])
    p.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 4, 5])
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-clients", type=int, default=64)
    p.add_argument("--n-envs", type=int, default=None)
    p.add_argument("--idle-skip", type=int, default=1, choices=[0, 1],
                   help="batched form: retire RIOT-timer wait-loop iterations at once (1) or run each (0)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--extra-serve-seconds", type=float, default=15.0)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--envs-per-warp", type=int, default=0)
    p.add_argument("--envs-per-block", type=int, default=0)
    p.add_argument("--warps-per-frame", type=int, default=0)
    p.add_argument("--tia-warps", type=int, default=0, choices=[0, 1, 2])
    p.add_argument("--grouping", type=int, default=0, choices=[0, 1, 2])
    p.add_argument("--dispatch", type=int, default=0, choices=[0, 1, 2])
    p.add_argument("--divergence", action="store_true",
                   help="divergence study: frames/s and lockstep lane efficiency per window of steps from one shared "
                        "start state per cartridge, beside a run from the usual random start states and the oracle "
                        "on the host from the same shared start")
    p.add_argument("--window", type=int, default=10)
    p.add_argument("--sweep", default=None,
                   help="comma-separated env counts: frames/s and frames/s per env of the batched and plain forms "
                        "and of the oracle at each count (paper Section 4, Fig. 2)")
    p.add_argument("--capture", action="store_true",
                   help="profiling run: W + K plain steps, no timing; prints each step's instructions retired and "
                        "TIA writes logged (the counts an ncu capture of one of these launches is divided by)")
    return p.parse_args(argv)


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


def cpu_model() -> str:
    """The host CPU's model name (lscpu on Arm hosts, /proc/cpuinfo on x86)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_for(w, idx):
    from oracle import OracleEnvs
    from paper_1907_08467_gb300 import synth
    return OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms], [r.gameover_addr for r in w.roms],
                      [w.env_rom[i] for i in idx], luma=synth.luma_table(), env_key=idx, seed=w.seed,
                      sticky=w.sticky, output_mode=w.output_mode, frameskip=w.frameskip)


def cpu_oracle_rate(w, seconds, seed=77, max_envs=512):
    """The oracle timed on the host cores on a bounded sample of the workload:
    `max_envs` envs spread evenly over the batch (same cartridges, keys and
    actions), stepped until `seconds` of wall time have passed."""
    import numpy as np

    from paper_1907_08467_gb300 import synth
    n = min(max_envs, w.n_envs)
    idx = np.linspace(0, w.n_envs - 1, n).astype(np.int64)
    cores = os.cpu_count() or 1
    o = _oracle_for(w, idx)
    acts = synth.actions(seed, 4096, w.n_envs)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds and steps < 4096:
        o.step(acts[steps][idx], n_threads=cores)
        steps += 1
    dt = time.perf_counter() - t0
    frames = n * w.frameskip * steps
    return {"value": frames / dt, "unit": "frames/s", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{n} of {w.n_envs} envs (same cartridges, keys, actions) x {steps} steps, "
                      f"{frames} frames in {dt:.1f} s on {cores} threads"}


def reference_arm(args, w, ws, rank):
    """The oracle as the reference arm: timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    sample_seconds = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    import numpy as np

    from paper_1907_08467_gb300 import synth
    n = min(256, w.n_envs)
    idx = np.linspace(0, w.n_envs - 1, n).astype(np.int64)
    cores = os.cpu_count() or 1
    o = _oracle_for(w, idx)
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
        "cpu_baseline": {"value": val, "unit": "frames/s", "cores": cores, "cpu_model": cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def serve_run(seconds, clients, warmup_s, rank):
    """Serving loop: native client threads (closed loop, Exp(2 ms) think time)
    open sessions of U{1..2048} envs on the 32 banked cartridges, step them
    (stacks, rewards and dones back to pinned host memory) and close them;
    admission under a 40 GB device budget.  Returns the loop's statistics."""
    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.server import AtariServer
    w = synth.workload(3, n_envs=32)
    max_envs = 2048
    srv = AtariServer.from_roms(w.roms, budget_bytes=40 << 30, max_slots=clients * max_envs, sticky=True,
                                seed=w.seed)
    warm = srv.loadgen(n_clients=clients, seconds=warmup_s, think_mean_ms=2.0, min_envs=1,
                       max_envs=max_envs, session_steps_mean=100, seed=1000 + rank, want_obs=True)
    l0 = srv.stats()["launches"]
    r = srv.loadgen(n_clients=clients, seconds=seconds, think_mean_ms=2.0, min_envs=1,
                    max_envs=max_envs, session_steps_mean=100, seed=1 + rank, want_obs=True)
    st = srv.stats()
    srv.close()
    r["warmup_requests"] = warm["requests"]
    r["launches"] = int(st["launches"] - l0)
    r["stats"] = st
    return r


def serve_bench(args, ws, rank, local):
    import torch
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle has no serving loop; the serving "
                              "workload is measured against the plain and batched GPU paths"}), flush=True)
        return
    torch.cuda.set_device(local)
    clients, max_envs = args.serve_clients, 2048
    clocks = ClockSampler(local)
    barrier(ws)
    clocks.start()
    r = serve_run(args.serve_seconds, clients, max(1.0, float(args.warmup)), rank)
    clk = clocks.stop()
    st = r["stats"]
    value = allreduce_sum(r["frames"], ws) / allreduce_max(r["seconds"], ws)
    if rank == 0:
        reqs = max(1, r["requests"])
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": r["requests"],
            "warmup": r["warmup_requests"], "ms_per_step": r["mean_ms"], "p50_step_ms": r["p50_ms"],
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
            "serving": _serving_summary(r),
            "gpu_launches": r["launches"], "clocks": clk, "roofline": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _serving_summary(r):
    return {"requests": r["requests"], "sessions": r["sessions"], "ticks": r["ticks"],
            "seconds": r["seconds"], "frames_per_s": r["frames"] / max(1e-9, r["seconds"]),
            "mean_tick_envs": r["mean_tick_envs"],
            "latency_ms": {"p50": r["p50_ms"], "p99": r["p99_ms"], "max": r["max_ms"], "mean": r["mean_ms"]},
            "admission_wait_ms": {"p50": r["admit_p50_ms"], "p99": r["admit_p99_ms"]}}


def make_env(w, form, args, rank):
    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.env import AtariEnv
    kw = dict(envs_per_warp=args.envs_per_warp, envs_per_block=args.envs_per_block,
              raster_warps_per_frame=args.warps_per_frame, tia_warps=args.tia_warps, idle_skip=args.idle_skip)
    if args.grouping:
        kw["grouping"] = args.grouping
    if args.dispatch:
        kw["dispatch"] = args.dispatch
    # replicas: each rank runs the whole workload with its own env keys
    return AtariEnv([r.data for r in w.roms], [(r.score_addr, r.gameover_addr) for r in w.roms], w.env_rom,
                    luma=synth.luma_table(), env_key=replica_env_keys(w.n_envs, rank), frameskip=w.frameskip,
                    sticky=w.sticky, output_mode=w.output_mode, form=form, seed=w.seed, **kw)


def timed_steps(do_step, acts, K, W, flush, ws, clocks=None):
    """W warm-up steps, then K steps each bracketed by CUDA events on the
    current stream, with an L2 flush before each (outside the events).
    Returns the step times in ms and the wall time of the timed loop."""
    import torch
    stream = torch.cuda.current_stream()
    for s in range(W):
        do_step(acts[s])
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t_wall = time.perf_counter()
    for s in range(K):
        flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        do_step(acts[W + s])
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    barrier(ws)
    clk = clocks.stop() if clocks else None
    return [e0.elapsed_time(e1) for e0, e1 in ev], wall, clk


def percentiles(ms):
    s = sorted(ms)
    return s[len(s) // 2], s[min(len(s) - 1, int(round(0.99 * (len(s) - 1))))]


def profile_pass(env, do_step, acts, flush):
    """Same launch configuration with CUDA events around every kernel (the
    batched form launches its kernels directly instead of replaying the
    captured graph while profiling), and the kernels' own counters of 6502
    instructions retired and TIA writes logged per step."""
    import torch
    env.profile_read()
    env.profile(True)
    instr = logrec = rounds = 0
    for s in range(acts.shape[0]):
        flush.fill_(s & 0xFF)
        do_step(acts[s])
        a, b, c = env.counters()
        instr += a
        logrec += b
        rounds += c
    torch.cuda.synchronize()
    env.profile(False)
    k = acts.shape[0]
    return env.profile_read(), instr / k, logrec / k, rounds / k


def interp_roofline(prof, instr_per_step, kernel, lanes, dispatch, config, n_envs, frameskip):
    """Issue-slot roofline of the interpreter (plain integer and control work:
    no tensor-core or FLOP peak applies)."""
    ms, n = prof.get("interpreter", (0.0, 0))
    if not n:
        return None
    dur = ms / n / 1000.0
    peak = SM_COUNT * SMSP_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    cap = INTERP_CAPTURES.get((kernel, lanes, dispatch, config))
    src = f"ncu capture of {kernel}, {lanes} envs/warp, dispatch {dispatch}, this workload"
    if cap is None:
        other = [(k, v) for k, v in INTERP_CAPTURES.items() if k[:3] == (kernel, lanes, dispatch)]
        if other:
            cap = other[0][1]
            src = f"ncu capture of {kernel}, {lanes} envs/warp, dispatch {dispatch}, workload config {other[0][0][3]}"
    ach = cap[0] * instr_per_step / dur / 1e9 if cap else None
    return {"bound": "alu", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "Gwarp-inst/s",
            "frac": (ach / peak) if ach else None, "traffic": cap[1] * n_envs if cap else None,
            "launch_ms": dur * 1000.0,
            "share_of_step": ms / max(1e-9, sum(v[0] for v in prof.values())),
            "m6502_inst_per_launch": instr_per_step,
            "m6502_inst_per_s": instr_per_step / dur,
            "warp_inst_per_m6502_inst": cap[0] if cap else None, "ratio_source": src if cap else None,
            "env_frames_per_launch": n_envs * frameskip,
            "peak_source": "152 SMs x 4 schedulers x 2070 MHz (issue slots)"}


def fused_roofline(prof, logrec_per_step, config, n_envs):
    ms, n = prof.get("fused_raster_preprocess", (0.0, 0))
    if not n:
        return None
    dur = ms / n / 1000.0
    per_step = FUSED_FIXED_BYTES_PER_ENV_STEP + 4.0 * logrec_per_step / n_envs
    hbm = load_peaks().get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    ach = per_step * n_envs / dur / 1e9
    tb = FUSED_DRAM_BYTES_PER_ENV_STEP.get(config)
    wi = FUSED_WARP_INST_PER_ENV_STEP.get(config)
    issue_peak = SM_COUNT * SMSP_PER_SM * SM_MAX_MHZ * 1e6 / 1e9
    return {"bound": "hbm", "kernel": "fused_raster_preprocess", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": tb * n_envs if tb else None, "algorithmic_bytes_per_env_step": per_step,
            "launch_ms": dur * 1000.0,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if hbm else "fallback 6.8 TB/s",
            # what binds it in practice: issue slots (same method as the interpreter's roofline)
            "issue": {"achieved": wi * n_envs / dur / 1e9 if wi else None, "peak": issue_peak,
                      "unit": "Gwarp-inst/s", "frac": wi * n_envs / dur / 1e9 / issue_peak if wi else None,
                      "warp_inst_per_env_step": wi}}


def inference_run(args, rank, flush):
    """Inference-path loop: 16384 envs over 16 sprite cartridges; each step
    the policy kernel picks every action from the stack, the env steps, and
    the newest plane and reward go to a 5-deep ring, all on the device."""
    import numpy as np
    import torch

    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.env import FORM_BATCHED
    w = synth.workload(5)
    env = make_env(w, FORM_BATCHED, args, rank)
    weights = torch.from_numpy(synth.policy_weights(w.seed).view(np.int16)).cuda()
    ring = torch.zeros((5, w.n_envs, 84 * 84), dtype=torch.uint8, device="cuda")
    ring_r = torch.zeros((5, w.n_envs), dtype=torch.float32, device="cuda")
    obs, rew, done = env.alloc_outputs()
    obs.zero_()
    act = torch.empty(w.n_envs, dtype=torch.uint8, device="cuda")
    t = [0]

    def do_step(_):
        env.rollout(weights, 1, obs, act, rew, done, ring, ring_r, ring_start=t[0])
        t[0] += 1
    K, W = args.steps, args.warmup
    ms, wall, _ = timed_steps(do_step, [None] * (K + W), K, W, flush, 1)
    prof, _, _, _ = profile_pass(env, do_step, np.zeros((3, 1)), flush)
    env.close()
    p50, p99 = percentiles(ms)
    return {"workload": w.name + " (policy + step + ring per step)", "n_envs": w.n_envs,
            "value": w.n_envs * w.frameskip * K / (sum(ms) / 1000.0), "unit": "frames/s", "steps": K,
            "ms_per_step": sum(ms) / K, "p50_step_ms": p50, "p99_step_ms": p99,
            "kernels": {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]} for k, v in prof.items()}}


def divergence_run(args, w, rank):
    """Paper Section 4, Fig. 3 and its CPU counterpart in the appendix: start
    every env of a cartridge from the same state (its first cached start
    state) and follow frames/s and the fraction of lanes executing per
    lockstep issue round window by window as random actions drive the envs
    apart; the same for a run from the usual random start states, and the
    oracle's frames/s on the host from the same shared start (a bounded env
    sample)."""
    import numpy as np
    import torch

    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.env import FORM_BATCHED
    S, win = args.steps, max(1, args.window)
    acts = torch.from_numpy(synth.actions(900 + rank, S, w.n_envs)).cuda()
    score = [r.score_addr for r in w.roms]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def gpu_curve(shared):
        env = make_env(w, FORM_BATCHED, args, rank)
        if shared:
            st = synth.shared_start_states(env.state().cpu().numpy(), env.cache().cpu().numpy(), w.env_rom, score)
            env.set_state(torch.from_numpy(st).cuda())
        obs, rew, done = env.alloc_outputs()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(S)]
        cnt = []
        stream = torch.cuda.current_stream()
        for s in range(S):
            flush.fill_(s & 0xFF)
            ev[s][0].record(stream)
            env.step(acts[s], obs, rew, done)
            ev[s][1].record(stream)
            cnt.append(env.counters())
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        shape = env.launch_shape()
        env.close()
        out = []
        for a in range(0, S - win + 1, win):
            t = sum(ms[a:a + win]) / 1000.0
            ins = sum(c[0] for c in cnt[a:a + win])
            rnd = sum(c[2] for c in cnt[a:a + win])
            out.append({"steps": [a, a + win], "frames_per_s": w.n_envs * w.frameskip * win / t,
                        "lockstep_lane_efficiency": ins / rnd if rnd else None,
                        "m6502_inst_per_env_frame": ins / (w.n_envs * w.frameskip * win)})
        return out, shape

    shared, shape = gpu_curve(True)
    random_start, _ = gpu_curve(False)
    # the oracle from the same shared start on a bounded sample of the envs
    from oracle import OracleEnvs
    n = min(256, w.n_envs)
    idx = np.linspace(0, w.n_envs - 1, n).astype(np.int64)
    o = OracleEnvs([r.data for r in w.roms], score, [r.gameover_addr for r in w.roms], [w.env_rom[i] for i in idx],
                   luma=synth.luma_table(), env_key=idx, seed=w.seed, sticky=w.sticky, output_mode=w.output_mode,
                   frameskip=w.frameskip)
    o.set_state(synth.shared_start_states(o.state(), o.cache(), [w.env_rom[i] for i in idx], score))
    ha = acts.cpu().numpy()
    cores = os.cpu_count() or 1
    oracle_curve = []
    t_budget = time.perf_counter() + max(5.0, args.cpu_seconds)
    for a in range(0, S - win + 1, win):
        t0 = time.perf_counter()
        for s in range(a, a + win):
            o.step(ha[s][idx], n_threads=cores)
        oracle_curve.append({"steps": [a, a + win], "frames_per_s": n * w.frameskip * win / (time.perf_counter() - t0)})
        if time.perf_counter() > t_budget:
            break
    return {"divergence": {
        "workload": w.name, "n_envs": w.n_envs, "window_steps": win, "steps": S,
        "launch_shape": shape_dict(shape),
        "shared_start": shared, "random_start": random_start,
        "oracle_shared_start": {"envs": n, "cores": cores, "cpu_model": cpu_model(), "windows": oracle_curve},
        "l2": "flushed (256 MB write) before each step"}}


def shape_dict(shape):
    """launch_shape() as named fields (the grouping word also carries the
    compact-dispatch flag, 4)."""
    e, b, wpf, grid, tia, g = shape
    return {"envs_per_warp": e, "envs_per_block": b, "warps_per_frame": wpf, "grid": grid, "tia_warps": tia,
            "grouping": g & 3, "dispatch": 2 if g & 4 else 1}


def sweep_run(args, config, counts, rank):
    """Frames/s and frames/s per env against the number of envs (the paper's
    Fig. 2 and its FPS-per-env discussion in Section 4): the batched form
    (autotuned at each count), the plain form, and the oracle on the host
    cores (a bounded sample at the larger counts), same cartridges and keys."""
    import numpy as np
    import torch

    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.env import FORM_BATCHED, FORM_PLAIN
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, W = max(3, args.steps), max(3, args.warmup)
    rows = []
    cores = os.cpu_count() or 1
    for n in counts:
        w = synth.workload(config, n_envs=n)
        acts = torch.from_numpy(synth.actions(700 + rank, K + W, n)).cuda()
        row = {"n_envs": n}
        for name, form in (("batched", FORM_BATCHED), ("plain", FORM_PLAIN)):
            env = make_env(w, form, args, rank)
            obs, rew, done = env.alloc_outputs()
            ms, _, _ = timed_steps(lambda a: env.step(a, obs, rew, done), acts, K, W, flush, 1)
            fps = n * w.frameskip * K / (sum(ms) / 1000.0)
            row[name] = {"frames_per_s": fps, "frames_per_s_per_env": fps / n, "ms_per_step": sum(ms) / K}
            if form == FORM_BATCHED:
                row[name]["launch_shape"] = shape_dict(env.launch_shape())
            env.close()
        m = min(n, 256)
        idx = np.linspace(0, n - 1, m).astype(np.int64)
        o = _oracle_for(w, idx)
        ha = acts.cpu().numpy()
        t0, k = time.perf_counter(), 0
        while k < K + W and (k < 3 or time.perf_counter() - t0 < 3.0):
            o.step(ha[k][idx], n_threads=cores)
            k += 1
        ofps = m * w.frameskip * k / (time.perf_counter() - t0)
        row["oracle"] = {"frames_per_s": ofps, "envs_timed": m, "cores": cores,
                         "note": "rate of the timed sample; the oracle's rate does not grow with more envs than cores"}
        rows.append(row)
    return {"sweep": {"workload": synth.workload(config).name.split(",")[0], "config": config, "steps": K,
                      "cpu_model": cpu_model(), "rows": rows, "l2": "flushed (256 MB write) before each step"}}


def kernel_name(env, form):
    if form == "plain":
        return "k_interp_plain"
    return "k_interp_split" if env.launch_shape()[4] == 2 else "k_interp_batched"


def main(argv=None):
    args = parse(argv)
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

    from paper_1907_08467_gb300.env import FORM_BATCHED, FORM_PLAIN
    torch.cuda.set_device(local)
    K, W = args.steps, args.warmup
    if args.divergence:
        res = divergence_run(args, w, rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    if args.sweep:
        res = sweep_run(args, args.config, [int(x) for x in args.sweep.split(",")], rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    inference = args.config == 5

    if inference:
        res = inference_run(args, rank, flush)
        value = allreduce_sum(res["value"], ws)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": res["ms_per_step"], "p50_step_ms": res["p50_step_ms"],
                "p99_step_ms": res["p99_step_ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded cartridges and policy weights)",
                "config": {"workload": res["workload"], "n_envs": res["n_envs"], "parallelism": f"replicas x{ws}",
                           "l2": "flushed (256 MB write) before each timed step"},
                "kernels": res["kernels"], "e2e": None, "roofline": None, "cpu_baseline": None,
                "gpu_launches": int(sum(v["launches"] for v in res["kernels"].values()) * K / 3)}), flush=True)
        return

    form = FORM_BATCHED if args.form == "batched" else FORM_PLAIN
    env = make_env(w, form, args, rank)
    acts = torch.from_numpy(synth.actions(100 + rank, K + W, w.n_envs)).cuda()
    obs, rew, done = env.alloc_outputs()
    if args.capture:
        counts = []
        for s in range(W + K):
            env.step(acts[s], obs, rew, done)
            counts.append(env.counters())
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"capture": w.name, "kernel": kernel_name(env, args.form),
                              "launch_shape": shape_dict(env.launch_shape()), "n_envs": w.n_envs,
                              "m6502_inst_per_step": [c[0] for c in counts],
                              "tia_log_records_per_step": [c[1] for c in counts],
                              "lane_rounds_per_step": [c[2] for c in counts]}), flush=True)
        return

    def do_step(a):
        env.step(a, obs, rew, done)
    step_ms, wall, clk = timed_steps(do_step, acts, K, W, flush, ws, ClockSampler(local))
    prof_steps = max(3, min(K, 10))
    pacts = torch.from_numpy(synth.actions(300 + rank, prof_steps, w.n_envs)).cuda()
    prof, instr, logrec, lane_rounds = profile_pass(env, do_step, pacts, flush)
    total_s_max = allreduce_max(sum(step_ms) / 1000.0, ws)
    frames_all = allreduce_sum(w.n_envs * w.frameskip * K, ws)
    value = frames_all / total_s_max
    p50, p99 = percentiles(step_ms)
    gpu_launches = int(round(sum(v[1] for v in prof.values()) * K / prof_steps))
    shape = env.launch_shape()
    kern = kernel_name(env, args.form)

    # e2e through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        ha = torch.from_numpy(synth.actions(200 + rank, 3 + K, w.n_envs)).pin_memory()
        ho = torch.empty(env.obs_shape(), dtype=torch.uint8).pin_memory()
        hr = torch.empty(w.n_envs, dtype=torch.int32).pin_memory()
        hd = torch.empty(w.n_envs, dtype=torch.uint8).pin_memory()
        for s in range(3):
            env.step_host(ha[s], ho, hr, hd)
        barrier(ws)
        t0 = time.perf_counter()
        host_ms = []
        for s in range(K):
            t1 = time.perf_counter()
            env.step_host(ha[3 + s], ho, hr, hd)
            host_ms.append((time.perf_counter() - t1) * 1e3)
        dt = allreduce_max(time.perf_counter() - t0, ws)
        hp50, hp99 = percentiles(host_ms)
        e2e = {"value": frames_all / dt, "unit": "frames/s", "h2d_bytes_per_step": int(ha[0].numel()),
               "d2h_bytes_per_step": int(ho.numel() + hr.numel() * 4 + hd.numel()),
               "p50_step_ms": hp50, "p99_step_ms": hp99}
    roof = interp_roofline(prof, instr, kern, shape[0], shape_dict(shape)["dispatch"], args.config, w.n_envs,
                           w.frameskip)
    if roof and lane_rounds:
        # fraction of a warp's lanes executing per lockstep issue round
        roof["lockstep_lane_efficiency"] = instr / lane_rounds
    roof2 = fused_roofline(prof, logrec, args.config, w.n_envs)
    kernels = {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]} for k, v in prof.items()}
    env.close()
    del env, obs, rew, done

    # the plain one-launch-per-kernel form on the same workload, timed the same way
    plain = None
    if args.form == "batched" and not args.no_plain:
        penv = make_env(w, FORM_PLAIN, args, rank)
        pobs, prew, pdone = penv.alloc_outputs()
        pms, _, _ = timed_steps(lambda a: penv.step(a, pobs, prew, pdone), acts, K, W, flush, ws)
        pprof, _, _, _ = profile_pass(penv, lambda a: penv.step(a, pobs, prew, pdone), pacts[:3], flush)
        penv.close()
        del penv, pobs, prew, pdone
        pval = frames_all / allreduce_max(sum(pms) / 1000.0, ws)
        q50, q99 = percentiles(pms)
        plain = {"value": pval, "unit": "frames/s", "ms_per_step": sum(pms) / K, "p50_step_ms": q50,
                 "p99_step_ms": q99,
                 "kernels": {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]} for k, v in pprof.items()},
                 "batched_over_plain": value / pval}

    extras = None
    if rank == 0 and ws == 1 and args.config == 3 and not args.no_extras:
        torch.cuda.empty_cache()
        inf = inference_run(args, rank, flush)
        del flush
        torch.cuda.empty_cache()
        srv = serve_run(args.extra_serve_seconds, args.serve_clients, 2.0, rank)
        extras = {"inference_loop": inf, "serving": {
            "workload": f"{args.serve_clients} clients, sessions U{{1..2048}} envs on the 32 banked cartridges, "
                        "closed loop Exp(2 ms) think time, 40 GB budget",
            **_serving_summary(srv), "gpu_launches": srv["launches"]}}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": 1000.0 * total_s_max / K, "p50_step_ms": p50, "p99_step_ms": p99,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded cartridges and actions)",
            "config": {"workload": w.name, "n_envs": w.n_envs, "n_roms": len(w.roms), "frameskip": w.frameskip,
                       "sticky": bool(w.sticky),
                       "output": "84x84x4 uint8 stack" if w.output_mode == 1 else "210x160 palette frame",
                       "form": args.form, "l2": "flushed (256 MB write) before each timed step",
                       "launch_shape": shape_dict(shape),
                       "timer_wait_skip": bool(args.idle_skip) and args.form == "batched",
                       "parallelism": f"replicas x{ws}"},
            "plain": plain, "e2e": e2e, "roofline": roof, "roofline_fused": roof2, "kernels": kernels,
            "gpu_launches": gpu_launches, "m6502_inst_per_step": instr, "tia_log_records_per_step": logrec,
            "wall_s": wall, "clocks": clk, "cpu_baseline": cpu, "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
