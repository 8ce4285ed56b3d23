"""Benchmark of the batched rigid-body step: env-steps/s on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config arm]
                    [--impl ours|reference] [--n-per-call 1]

A timed "step" is one call of the public entry point ms_step advancing every
env of the configuration by --n-per-call physics steps (all stages:
broadphase, narrowphase, colouring, prep, solve, integration).  Inputs are
the seeded synthetic scenes of scenegen, resident on the GPU; L2 is flushed
(256 MB write) before every timed step, outside the timed events.  Prints
one JSON line (rank 0).  Under torchrun every rank runs its own batch of the
configuration (weak scaling, no collective in the step).

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on the host cores for the same configuration and metric.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen  # noqa: E402

METRIC = "env-steps/s on 1 B300, batched vs plain at oracle tol; served p50/p99 latency"
WORKLOADS = {
    "arm": "7-DoF capsule arm + 2 prismatic box fingers + cube on a plane, 4096 envs "
           "(dt 0.01 s, 4 substeps, 8+1 iterations, PD kp 1000 kd 100, targets N(0,0.3) per step)",
    "small": "plane + 1 box + 3 spheres, 64 envs (dt 0.01 s, 4 substeps, 8+1 iterations)",
    "clutter": "1-32 boxes/spheres/capsules in a 5-box bin, 16384 envs (dt 0.01 s, 4 substeps, 8+1)",
    "hand": "16-DoF capsule hand holding a cube, 4096 envs (dt 1/120 s, 8 substeps, 16+1 iterations)",
    "hulls": "1-12 convex hulls (6-12 points, from a pool of 128) dropped into the 5-box bin, 4096 envs "
             "(dt 0.01 s, 4 substeps, 8+1 iterations)",
    "mixed": "arm (9 joints), hand (16 joints) and clutter (no joint) envs interleaved in one batch, 4096 envs "
             "(dt 0.01 s, 4 substeps, 8+1 iterations, capacities 704 pairs / 384 contacts)",
    "pick": "the arm envs driven by the pick task, 4096 envs: delta joint-position controller on normalised "
            "actions, and per step a record of reward, grasp / tcp / table flags, tcp and cube positions, "
            "joint coordinates and targets (dt 0.01 s, 4 substeps, 8+1 iterations)",
}

# FLOP weights per counted operation of the oracle (the step's algorithmic work model)
FLOP_WEIGHTS = {
    "row_solve_2dyn": 61, "row_solve_1dyn": 31, "rows_prep": 40, "body_inertia": 45,
    "body_integrate": 40, "warm_apply": 25, "pairs_tested": 10,
    "np_ss": 20, "np_sc": 40, "np_sb": 60, "np_sp": 15, "np_cc": 120, "np_cb": 300, "np_cp": 30,
    "np_bb": 1000, "np_bp": 150, "np_sh": 400, "np_xh": 500, "np_hp": 150,
    # the hull SAT's own work: a face-vertex projection (6 flop), an edge pair's
    # Gauss-map test (2 cross products' worth and 4 dot products, 20 flop)
    "sat_face_vert": 6, "sat_edge_pair": 20, "np_ch": 2000,
}
FP32_LANES_PER_SM = 128

# --variants: the optional solver variants on (damping, restitution, warm start)
VARIANT_PARAMS = dict(linear_damping=0.5, angular_damping=0.3, bounce_threshold=0.5, warm_start=1)
VARIANT_RESTITUTION = 0.4


def make_workload(name, variants=False, **kw):
    sc = scenegen.make_scene(name, **kw)
    if variants:
        sc.params = dict(sc.params, **VARIANT_PARAMS)
        sc.bodies = sc.bodies.copy()
        sc.bodies["restitution"] = VARIANT_RESTITUTION
    return sc

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from one ncu capture of the bench command (profiles/), keyed
# by workload and tuning.  Valid only while the kernel sources hash to the
# recorded value; otherwise the bench reports traffic null.
NCU_TRAFFIC = {
    ("arm", "4,1,0"): {"bytes": 1.80493e+07, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<4, lean, dynamic>"},
    ("arm", "8,1,0"): {"bytes": 3.04064e+07, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<8, lean, dynamic>"},
    ("arm", "8,2,0"): {"bytes": 3.02684e+07, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<8, lean, dynamic>"},
    ("clutter", "16,4,0"): {"bytes": 5.51108e+08, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, dynamic, no joints>"},
    ("clutter", "16,8,0"): {"bytes": 5.5136e+08, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, dynamic, no joints>"},
    ("clutter", "16,8,2"): {"bytes": 5.51332e+08, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, dynamic, no joints>"},
    ("hand", "8,4,2"): {"bytes": 3.33629e+07, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<8, lean, dynamic>"},
    ("hulls", "16,8,0"): {"bytes": 2.958e+08, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, dynamic, hulls, no joints>"},
    ("hulls", "16,8,2"): {"bytes": 2.95881e+08, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, dynamic, hulls, no joints>"},
    ("mixed", "16,4,2"): {"bytes": 3.39876e+07, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, dynamic>"},
    ("pick", "8,1,0"): {"bytes": 3.09965e+07, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<8, full, dynamic>"},
    ("small", "16,2,0"): {"bytes": 179712, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<16, lean, capacity slots, no joints>"},
    ("small", "32,2,0"): {"bytes": 187648, "kernel_sha": "d66443322403c88d", "kernel": "k_fused<32, lean, capacity slots, no joints>"},
}
KERNEL_SOURCES = ("ms_fused.cu", "ms_stages.cuh", "ms_narrow.cuh", "ms_math.cuh", "ms_internal.h", "../build.py")


def kernel_sha():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2410_00425_b300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(name, tuning, variants=False):
    if variants:
        return None
    key = (name, None if not tuning else "%d,%d,%d" % (tuning["lanes_per_env"], tuning["warps_per_cta"],
                                                       tuning["rows_in_smem"]))
    rec = NCU_TRAFFIC.get(key)
    if rec is None or rec["kernel_sha"] != kernel_sha():
        return None
    return rec["bytes"]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def algorithmic_flops_per_env_step(name, warmup, steps, sample_envs=32, variants=False):
    """Oracle op counters x fixed FLOP weights, counted over the same window
    of steps the timed region covers (after `warmup` steps) on the first
    `sample_envs` envs of the workload (per-env seeding: the same envs)."""
    import oracle
    sc = make_workload(name, variants, n_envs=min(sample_envs, scenegen.CONFIG_SIZES[name]))
    o = oracle.Oracle(sc)
    th = os.cpu_count() or 1
    if sc.task is not None:
        o.set_task(sc.task)
    stepper = o.step_task if sc.task is not None else o.step
    if warmup:
        stepper(warmup, actions=sc.actions(0, warmup), threads=th)
    c0 = o.counters()
    n = max(1, min(steps, 200))
    stepper(n, actions=sc.actions(warmup, n), threads=th)
    c1 = o.counters()
    c = {k: c1[k] - c0[k] for k in c1}
    flops = sum(FLOP_WEIGHTS[k] * c[k] for k in FLOP_WEIGHTS)
    return flops / (sc.n_envs * n), c


class ClockSampler:
    """SM clock and clock-event reasons while the timed region runs: NVML
    read-only queries every 2 ms from a thread (the device matched by PCI bus
    id), else nvidia-smi at its 50 ms minimum.  Nothing is set."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.nvml = None
        self.samples = []          # (sm_mhz, max_mhz, set of reason names)
        self.stop = threading.Event()

    def _nvml_handle(self):
        """The NVML handle of this process's CUDA device: by UUID, else by PCI
        bus id, else by index (NVML ignores CUDA_VISIBLE_DEVICES)."""
        import pynvml
        import torch
        pynvml.nvmlInit()
        p = torch.cuda.get_device_properties(self.index)
        uuid = getattr(p, "uuid", None)
        if uuid is not None:
            u = str(uuid)
            for cand in (u if u.startswith("GPU-") else "GPU-" + u, u):
                try:
                    return pynvml, pynvml.nvmlDeviceGetHandleByUUID(cand.encode())
                except Exception:
                    pass
        try:
            bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
            return pynvml, pynvml.nvmlDeviceGetHandleByPciBusId(bus.encode())
        except Exception:
            return pynvml, pynvml.nvmlDeviceGetHandleByIndex(self.index)

    def _poll_nvml(self):
        nv, h = self.nvml
        mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        while not self.stop.is_set():
            sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
            bits = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
            self.samples.append((float(sm), float(mx), {k for k, v in self.REASONS.items() if bits & v}))
            self.stop.wait(0.002)

    def _read_smi(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or self.stop.is_set():
                continue
            try:
                self.samples.append((float(f[1]), float(f[2]),
                                     {n for n, v in zip(self.REASONS, f[5:9]) if v.lower() == "active"}))
            except ValueError:
                continue

    def __enter__(self):
        try:
            self.nvml = self._nvml_handle()
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
        except Exception:
            self.nvml = None
            try:
                self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "50"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.t = threading.Thread(target=self._read_smi, daemon=True)
            except OSError:
                self.t = None
        if self.t is not None:
            self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [x[0] for x in self.samples]
        reasons = set().union(*[x[2] for x in self.samples])
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(x[1] for x in self.samples),
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvml" if self.nvml else "nvidia-smi",
                "window": "the settling, warm-up and timed steps of the batched timing (one kernel, one load)"}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        # the step has no collective: gloo carries only the barrier and the
        # max over ranks of the timed region
        dist.init_process_group("gloo")
    return ws, rank, local


def reduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_rate(name, n_envs, settle, steps, variants=False, threads=None):
    """The oracle as it stands, timed on the host cores: one oracle over the
    first n_envs envs of the workload (per-env seeding: the same envs the
    GPU steps), advanced `settle` steps untimed, then `steps` steps timed one
    call each.  Returns (env-steps/s, seconds per step list, threads)."""
    import oracle
    sc = make_workload(name, variants, n_envs=n_envs)
    o = oracle.Oracle(sc)
    th = threads or os.cpu_count() or 1
    task = sc.task is not None
    if task:
        o.set_task(sc.task)
    acts = sc.actions(0, settle + steps)

    def adv(k0, n):
        a = None if acts is None else np.ascontiguousarray(acts[k0:k0 + n])
        if task:
            o.step_task(n, actions=a, threads=th)
        else:
            o.step(n, actions=a, threads=th)
    if settle:
        adv(0, settle)
    times = []
    for k in range(steps):
        t0 = time.perf_counter()
        adv(settle + k, 1)
        times.append(time.perf_counter() - t0)
    return n_envs * steps / sum(times), times, th


def oracle_sample_envs(name):
    """Envs of the bounded oracle sample of a workload (about 10-30 s of
    CPU work for the default run; rates extrapolate linearly in envs)."""
    return min(scenegen.CONFIG_SIZES[name], 1024)


def time_cpu_baseline(name, settle, steps, one_core=False, variants=False):
    """cpu_baseline of the JSON line: the oracle on every host core on the
    bounded sample at the same settled state as the GPU timing, and on one
    core on a sixteenth of it."""
    n = oracle_sample_envs(name)
    v, times, th = oracle_rate(name, n, settle, steps, variants)
    out = {"value": v, "unit": "env-steps/s", "cores": th, "kind": "oracle",
           "sample": f"{n} envs of the {name} workload, {settle} settling steps, then {steps} timed steps "
                     f"(one call each), FP64, {th} threads ({sum(times):.2f} s timed)"}
    if one_core:
        n1 = max(1, n // 16)
        v1, t1, _ = oracle_rate(name, n1, settle, steps, variants, threads=1)
        out["value_1core"] = v1
        out["sample_1core"] = f"{n1} envs, {settle} settling + {steps} timed steps, 1 thread ({sum(t1):.2f} s timed)"
    return out


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle on the host cores, same metric and
    the same bounded sample and settled state as the cpu_baseline of the
    GPU line.  Each timed step advances the sample by one step."""
    if rank != 0:
        return
    E = scenegen.CONFIG_SIZES[args.config]
    n = oracle_sample_envs(args.config)
    v, times, th = oracle_rate(args.config, n, args.settle + args.warmup, args.steps, args.variants)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * E / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scenegen scenes)",
            "config": {"workload": WORKLOADS[args.config], "n_envs": E, "n_per_call": 1,
                       "settle_steps": args.settle, "l2": "not applicable (CPU)",
                       "variants": (dict(VARIANT_PARAMS, restitution=VARIANT_RESTITUTION) if args.variants
                                    else None)},
            "cpu_baseline": {"value": v, "unit": "env-steps/s", "cores": th, "kind": "oracle",
                             "sample": f"{n} of {E} envs, {args.settle + args.warmup} untimed steps, then "
                                       f"{args.steps} timed steps of one call each, {th} threads"},
            "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_run(rate, duration, merge, seed=5, n_sessions=128, budget=120 << 30, pools=None, life_mean=50.0,
              max_inflight=32, openers=4):
    """Open-loop Poisson load on the step server.

    Sessions own 1..1024 envs (log-uniform) of a scene type drawn uniformly
    from {arm, clutter, hand}, live for a geometric number of requests (mean
    life_mean, an episode) and are replaced by fresh sessions; each request
    steps its session once with fresh drive targets.  A closed session's
    replacement is opened by one of `openers` client threads (session
    creation, admission and upload are part of the served work).  Returns
    latency percentiles (host arrival -> completion) and the env-steps/s the
    server sustained."""
    import queue as _q
    from paper_2410_00425_b300.server import Server
    g = np.random.default_rng(seed)
    types = ["arm", "clutter", "hand"]
    if pools is None:
        pools = {t: scenegen.make_scene(t, n_envs=1024) for t in types}
    act_pool = {t: (pools[t].actions(0, 8) if pools[t].n_act else None) for t in types}
    srv = Server(budget, merge=merge, max_inflight=max_inflight)
    g_open = np.random.default_rng(seed + 1)      # the opener thread's own generator

    def new_session(g):
        t = types[int(g.integers(0, 3))]
        n = int(np.exp(g.uniform(0.0, np.log(1024.0))))
        n = max(1, min(1024, n))
        a0 = int(g.integers(0, 1024 - n + 1))
        sc = pools[t].subset(range(a0, a0 + n))
        sid = srv.open(sc)
        life = int(g.geometric(1.0 / life_mean))
        return sid, t, a0, n, life

    active = []
    for _ in range(n_sessions):
        s_ = new_session(g)
        if s_[0] is not None:
            active.append(list(s_))
    repl = _q.Queue()
    closing = _q.Queue()
    stop = threading.Event()
    # replacement sessions are cut from the pools before the timed region, so
    # the opener thread only makes the (GIL-free) library calls
    spare = []
    for _ in range(int(rate * duration / max(life_mean, 1.0) * 1.5) + 64):
        t = types[int(g_open.integers(0, 3))]
        n = max(1, min(1024, int(np.exp(g_open.uniform(0.0, np.log(1024.0))))))
        a0 = int(g_open.integers(0, 1024 - n + 1))
        spare.append((t, a0, n, pools[t].subset(range(a0, a0 + n)), int(g_open.geometric(1.0 / life_mean))))

    open_s = []
    spare_it = iter(spare)
    spare_mu = threading.Lock()

    def opener():
        while not stop.is_set():
            try:
                sid = closing.get(timeout=0.05)
            except _q.Empty:
                continue
            srv.close_session(sid)
            with spare_mu:
                nxt_spare = next(spare_it, None)
            if nxt_spare is not None:
                t, a0, n, sc, life = nxt_spare
                t_open = time.perf_counter()
                sid2 = srv.open(sc)
                open_s.append(time.perf_counter() - t_open)
                if sid2 is not None:
                    repl.put([sid2, t, a0, n, life])
    # the arrival loop and the openers share the interpreter: switch often
    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(2e-4)
    ths = [threading.Thread(target=opener, daemon=True) for _ in range(max(1, openers))]
    for th in ths:
        th.start()
    # warm-up: one request per session (first launches, graph capture)
    for s_ in active:
        srv.submit(s_[0], None)
    srv.drain()
    srv.reset_stats()
    t0 = time.perf_counter()
    nxt = t0
    submitted = 0
    arrivals = no_session = 0
    saturated = False
    next_check = t0 + 0.5
    while True:
        nxt += g.exponential(1.0 / rate)
        if nxt - t0 > duration:
            break
        if nxt > next_check:
            # open loop: stop if the server falls more than 2 s of arrivals behind
            next_check += 0.5
            if submitted - srv.stats()["requests_done"] > 2.0 * rate:
                saturated = True
                break
        while True:                      # sleep to the arrival, spin the last 0.2 ms
            left = nxt - time.perf_counter()
            if left <= 0:
                break
            if left > 3e-4:
                time.sleep(left - 2e-4)
        while not repl.empty():
            active.append(repl.get())
        arrivals += 1
        if not active:
            no_session += 1              # every session is being replaced: the arrival is lost
            continue
        k = int(g.integers(0, len(active)))
        sid, t, a0, n, life = active[k]
        ap = act_pool[t]
        srv.submit(sid, None if ap is None else ap[submitted % 8, a0:a0 + n])
        submitted += 1
        active[k][4] -= 1
        if active[k][4] <= 0:
            closing.put(sid)
            active.pop(k)
    srv.drain()
    wall = time.perf_counter() - t0
    st = srv.stats()
    stop.set()
    for th in ths:
        th.join()
    sys.setswitchinterval(old_switch)
    srv.close()
    return {"rate_req_s": rate, "duration_s": duration, "merge": merge, "arrivals": arrivals,
            "lost_no_session": no_session, "requests": int(st["requests_done"]),
            "session_opens": len(open_s), "open_ms_p50": 1e3 * float(np.median(open_s)) if open_s else None,
            "launches": int(st["launches"]), "p50_ms": 1e3 * st["p50"], "p99_ms": 1e3 * st["p99"],
            "mean_ms": 1e3 * st["mean"], "env_steps_per_s": st["env_steps"] / wall,
            "sessions_admitted": int(st["sessions_admitted"]), "sessions_rejected": int(st["sessions_rejected"]),
            "graph_captures": int(st["graph_captures"]), "launch_p50_ms": 1e3 * st["launch_p50"],
            "launch_p99_ms": 1e3 * st["launch_p99"], "launch_max_ms": 1e3 * st["launch_max"],
            "queue_p50_ms": 1e3 * st["queue_p50"], "queue_p99_ms": 1e3 * st["queue_p99"],
            "stage_p99_ms": 1e3 * st["stage_p99"], "stage_max_ms": 1e3 * st["stage_max"], "life_mean": life_mean,
            "max_inflight": max_inflight, "sessions": n_sessions, "openers": openers, "saturated": saturated}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--settle", type=int, default=100,
                    help="untimed calls before the warm-up: every timing starts from the settled workload")
    ap.add_argument("--config", default="arm", choices=sorted(WORKLOADS))
    ap.add_argument("--n-per-call", type=int, default=1)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default=None, help="force the launch shape G,W,R (skips the autotuner)")
    ap.add_argument("--serve", action="store_true", help="serving sweep only (rates x merge modes)")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000", help="arrival rates (requests/s) of --serve")
    ap.add_argument("--serve-life", type=float, default=50.0, help="mean session lifetime (requests) of --serve")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-render", action="store_true", help="skip the camera-rendering measurement")
    ap.add_argument("--variants", action="store_true",
                    help="velocity damping, restitution and warm starting across steps on")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    from paper_2410_00425_b300 import Batch, build
    build.build()
    if args.serve:
        if rank == 0:
            torch.cuda.set_device(local)
            pools = {t: scenegen.make_scene(t, n_envs=1024) for t in ("arm", "clutter", "hand")}
            rates = [int(r) for r in args.serve_rates.split(",")]
            runs = [serve_run(r, args.serve_seconds, m, pools=pools, life_mean=args.serve_life)
                    for r in rates for m in (True, False)]
            print(json.dumps({"metric": "served step latency (host arrival -> completion), env-steps/s",
                              "unit": "ms", "n_gpus": 1, "higher_is_better": False,
                              "config": {"workload": "step server: Poisson arrivals, sessions of 1-1024 envs "
                                                     "of arm/clutter/hand, geometric lifetime mean %g requests, "
                                                     "120 GB HBM budget" % args.serve_life},
                              "runs": runs}), flush=True)
        return
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    name = args.config
    E = scenegen.CONFIG_SIZES[name]
    sc = make_workload(name, args.variants, seed=None if rank == 0 else 1000 + rank)
    n = args.n_per_call
    S = args.settle                 # untimed calls that bring the workload to its steady state
    total_calls = S + args.warmup + args.steps
    acts_np = sc.actions(0, n * total_calls)
    acts = None if acts_np is None else torch.from_numpy(acts_np).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def act(i):
        return None if acts is None else acts[i * n:(i + 1) * n]

    def settle(bb):
        """The first S calls, untimed (batched path; the plain path gives
        bit-identical states), so every timing starts from the same settled
        state: arms on the floor and at the cube, objects landed."""
        with torch.cuda.stream(stream):
            for i in range(S):
                bb.step(act(i), n, stream=stream, out=None)
        stream.synchronize()

    b = Batch(sc)
    if sc.task is not None:
        b.set_task(sc.task, stream=stream)
    tuning = None
    if args.tuning:
        G, W, R = (int(x) for x in args.tuning.split(","))
        b.set_tuning(G, W, R)
        tuning = b.tuning()
    elif not args.no_autotune:
        # tune on the settled state (arms moving, objects landed and in
        # contact), not on the initial poses: the trials restore this state
        # after each candidate (tuned on the falling phase, the hulls
        # workload picked a launch shape 1.5x slower over the run)
        settle(b)
        tuning = b.autotune(n, cache_path=os.path.join(ROOT, "paper_2410_00425_b300", "tuning_cache.json"),
                            stream=stream)
    else:
        tuning = b.tuning()
    b.close()

    def new_batch():
        bb = Batch(sc)
        if sc.task is not None:
            bb.set_task(sc.task, stream=stream)
        return bb

    def timed(plain, launches_per_call):
        bb = new_batch()
        if not plain and tuning:
            bb.set_tuning(tuning["lanes_per_env"], tuning["warps_per_cta"], tuning["rows_in_smem"])
        rec = (torch.empty((n, E, bb.record_len()), dtype=torch.float32, device=dev)
               if sc.task is not None else None)
        clk = ClockSampler(local)
        clk.__enter__()
        settle(bb)
        with torch.cuda.stream(stream):
            for i in range(args.warmup):
                bb.step(act(S + i), n, stream=stream, plain=plain, out=rec)
        stream.synchronize()
        times = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier(ws)
        torch.cuda.synchronize()
        try:
            for i in range(args.steps):
                flush.fill_(float(i))                      # L2 flush, outside the events
                stream.wait_stream(torch.cuda.current_stream())
                ev[i][0].record(stream)
                bb.step(act(S + args.warmup + i), n, stream=stream, plain=plain, out=rec)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
        finally:
            clk.__exit__(None, None, None)
        barrier(ws)
        times = [a.elapsed_time(z) for a, z in ev]
        code, status = bb.sync()
        bb.close()
        return sum(times) / 1e3, times, clk.summary(), code, launches_per_call * args.steps

    from paper_2410_00425_b300 import _ffi as _ffi_peak
    fp32_flops, _, fp32_s = _ffi_peak.ms_measure_fp32_peak(0.5)
    fp32_peak = fp32_flops / 1e12
    t_b, times_b, clocks, code, launches = timed(False, 1)
    t_b = reduce_max(t_b, ws)
    value = ws * E * n * args.steps / t_b
    plain_value = None
    if not args.no_plain:
        p = sc.params
        # launches per step: begin, narrow, colour; per substep prep, warm start
        # (not on the first substep without warm_start), sweeps, integrate, end; check
        lp = n * (3 + p["substeps"] * (4 + p["pos_iters"] + p["vel_iters"]) + 1 - (0 if p.get("warm_start") else 1))
        t_p, _, _, _, _ = timed(True, lp)
        t_p = reduce_max(t_p, ws)
        plain_value = ws * E * n * args.steps / t_p

    # e2e: host actions in (pinned), state out to pinned host, every step
    # (with a task: the records -- observations and rewards -- instead of the state)
    bb = new_batch()
    if tuning:
        bb.set_tuning(tuning["lanes_per_env"], tuning["warps_per_cta"], tuning["rows_in_smem"])
    # one C-ABI call per step (ms_step_host): pinned host actions in, pinned
    # host state (or the task records) out, both copies on the stream
    h_act = None if acts_np is None else torch.from_numpy(acts_np).pin_memory()
    task = sc.task is not None
    h_state = torch.empty((bb.NB, 13), dtype=torch.float32).pin_memory()
    h_rec = torch.empty((n, E, bb.record_len()), dtype=torch.float32).pin_memory() if task else None

    def e2e_step(j):
        a = None if h_act is None else h_act[j * n:(j + 1) * n]
        bb.step_host(a, n, h_rec if task else h_state, records=task, stream=stream)
    settle(bb)
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            e2e_step(S + i)
    stream.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            e2e_step(S + args.warmup + i)
    e1.record(stream)
    stream.synchronize()
    t_e = reduce_max(e0.elapsed_time(e1) / 1e3, ws)
    bb.close()
    h2d = 0 if h_act is None else n * E * sc.n_act * 4
    d2h = (h_rec.numel() if task else h_state.numel()) * 4

    # batched camera rendering (one 128 x 128 camera per env): the render
    # launch alone, and step + render per iteration (sim + render rate)
    render = None
    if not args.no_render:
        from paper_2410_00425_b300 import _ffi
        bb = new_batch()
        if tuning:
            bb.set_tuning(tuning["lanes_per_env"], tuning["warps_per_cta"], tuning["rows_in_smem"])
        cam = scenegen.default_camera(name)
        bb.set_camera(cam, scenegen.body_colors(sc))
        Hc, Wc = cam["height"], cam["width"]
        o_rgba = torch.empty((E, Hc, Wc, 4), dtype=torch.uint8, device=dev)
        o_depth = torch.empty((E, Hc, Wc), dtype=torch.float32, device=dev)
        o_seg = torch.empty((E, Hc, Wc), dtype=torch.int16, device=dev)
        rec = (torch.empty((n, E, bb.record_len()), dtype=torch.float32, device=dev)
               if sc.task is not None else None)
        reps = min(args.steps, 50)
        settle(bb)
        with torch.cuda.stream(stream):
            for i in range(args.warmup):
                bb.step(act(S + i), n, stream=stream, out=rec)
                _ffi.ms_render(bb.h, o_rgba, o_depth, o_seg, stream)
        stream.synchronize()
        ev_r = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        ev_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for i in range(reps):
            flush.fill_(float(i))
            stream.wait_stream(torch.cuda.current_stream())
            ev_r[i][0].record(stream)
            _ffi.ms_render(bb.h, o_rgba, o_depth, o_seg, stream)
            ev_r[i][1].record(stream)
        for i in range(reps):
            flush.fill_(float(i))
            stream.wait_stream(torch.cuda.current_stream())
            ev_s[i][0].record(stream)
            bb.step(act(S + args.warmup + i), n, stream=stream, out=rec)
            _ffi.ms_render(bb.h, o_rgba, o_depth, o_seg, stream)
            ev_s[i][1].record(stream)
        torch.cuda.synchronize()
        t_r = statistics.mean(a.elapsed_time(z) for a, z in ev_r) / 1e3
        t_s = statistics.mean(a.elapsed_time(z) for a, z in ev_s) / 1e3
        bb.close()
        # algorithmic bytes per launch: the images written (4 + 4 + 2 B per
        # pixel) plus each body's pose, shape and colour read (60 B)
        rbytes = E * Hc * Wc * 10 + int(sc.body_off[-1]) * 60
        hbm = float(load_peaks().get("hbm_gbs", 6400.0))
        render = {"renders_per_s": E / t_r, "ms_per_render": 1e3 * t_r, "image": f"{Wc}x{Hc} RGBA8 + depth + seg",
                  "sim_render_env_steps_per_s": E * n / t_s, "ms_per_step_and_render": 1e3 * t_s,
                  "roofline": {"bound": "hbm", "achieved": rbytes / t_r / 1e9, "peak": hbm, "unit": "GB/s",
                               "frac": rbytes / t_r / 1e9 / hbm, "bytes_per_launch": rbytes,
                               "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
                  "l2": "flushed before every timed launch"}

    if rank != 0:
        return
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    unit_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    fl, _ = algorithmic_flops_per_env_step(name, (S + args.warmup) * n, args.steps * n, variants=args.variants)
    kernel_s = statistics.mean(times_b) / 1e3
    achieved = fl * E * n / kernel_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_b / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scenegen scenes)",
        "config": {"workload": WORKLOADS[name], "n_envs": E, "n_per_call": n, "path": "batched",
                   "settle_steps": S * n, "tuning": tuning, "l2": "flushed (256 MB write) before every timed step",
                   "variants": (dict(VARIANT_PARAMS, restitution=VARIANT_RESTITUTION) if args.variants else None)},
        "plain_value": plain_value,
        "batched_over_plain": None if not plain_value else value / plain_value,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": ncu_traffic(name, tuning, args.variants),
                     "peak_note": f"measured FP32 FMA rate of this GPU (ms_measure_fp32_peak: 8 dependent-FMA "
                                  f"chains per thread, full occupancy, {fp32_s:.2f} s); from unit counts "
                                  f"{props.multi_processor_count} SMs x 128 lanes x 2 x {sm_max:.0f} MHz = "
                                  f"{unit_tflops:.1f} TFLOP/s",
                     "flops_per_env_step": fl},
        "e2e": {"value": ws * E * n * args.steps / t_e, "unit": "env-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "status": code,
        "device": props.name,
    }
    if render is not None:
        line["render"] = render
    if not args.no_serve:
        pools = {t: scenegen.make_scene(t, n_envs=1024) for t in ("arm", "clutter", "hand")}
        # 2k requests/s: latency at load; 10k requests/s: over capacity, the
        # env-steps/s each mode sustains (its latencies grow with the run)
        line["served"] = {"merged": serve_run(2000, 4.0, True, pools=pools),
                          "one_launch_per_request": serve_run(2000, 4.0, False, pools=pools),
                          "overload_10k_merged": serve_run(10000, 3.0, True, pools=pools),
                          "overload_10k_one_launch_per_request": serve_run(10000, 3.0, False, pools=pools)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = time_cpu_baseline(name, S * n + args.warmup, 100, one_core=True,
                                                 variants=args.variants)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
