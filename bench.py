#!/usr/bin/env python
"""Benchmark of the GB300 state-vector hot path; prints ONE JSON line.

Workload (one step): the 20-qubit hardware-efficient ansatz, 8 layers of
per-qubit RY, RZ and a CNOT ring (480 gates, 320 parameters), complex64,
batch 1: state preparation, evolution and the expectation of sum_i Z_i.

value = amplitude-GB/s: the bytes of every full-state pass the kernels make
(a read and a write of 2^n complex64 amplitudes per pass, the write-only
state preparation counted once) divided by the device time of the step.  The
gate-equivalent figure (every gate counted as one full read+write sweep,
whatever the implementation moves) is reported beside it under its own key.
L2 is flushed (a 512 MiB write) between timed steps.

Extra objects on the line: the dominant kernel's roofline, the CPU oracle
baseline (timed in fresh processes) with the headline result's error against
it, the end-to-end figure through the public API with host buffers, SM clocks
sampled during the timed region, the HBM-bound single-gate sweep at 30
qubits, and fused vs plain batched forward+adjoint gradients (12 qubits x 4096
samples) and the other configurations.

--impl reference runs the FP64 CPU oracle on the same workload and prints the
same line with "impl": "reference".
"""
import argparse
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

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "amplitude-GB/s vs HBM peak; batched fwd+adjoint grads/s vs plain path at 1e-4"
UNIT = "GB/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return None


NOMINAL_HBM_GBS = 8000.0    # GB300 HBM3e nominal bandwidth, for the fraction beside the measured one


def gate_pass_bytes(n, gates, amp=8):
    """Gate-equivalent bytes: one full read+write sweep per gate."""
    return len(gates) * 2 * (1 << n) * amp


def oracle_pass_bytes(n, ngates, nterms, amp=16):
    """Amplitude bytes of the passes the oracle makes in one step: one full
    read+write sweep of its complex128 state per gate, and per Pauli term a
    copy, the Pauli string applied to the copy and the inner product (three
    passes)."""
    return (ngates + 3 * nterms) * 2 * (1 << n) * amp


def touched_bytes(n, g, amp=8):
    """Bytes the per-gate sweep kernel must move for one gate."""
    full = 2 * (1 << n) * amp
    if g.kind in ("cnot", "cz", "cp", "crx", "cry", "crz"):
        return full // 2
    return full


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def throttled(clocks) -> bool:
    """Whether a clock record disqualifies the run it was taken in: a
    hardware or thermal slowdown, or SM clocks well below their maximum with
    no reason reported (a leftover clock lock).  A power cap is kept."""
    if any(r in THROTTLE_REASONS for r in clocks.get("reasons", [])):
        return True
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.85 * mx and not clocks.get("reasons"))


def any_rank(flag: bool, world: int, dist, device) -> bool:
    """flag on any rank (every rank gets the same answer)."""
    if world <= 1 or dist is None:
        return bool(flag)
    import torch
    t = torch.tensor([1.0 if flag else 0.0], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return bool(t.item() > 0)


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
_ORACLE_TIMER = r"""
import json, sys, time
import oracle, workloads as W
oracle.build()
wl = W.config_c2()
budget = float(sys.argv[1])
def step():
    st = oracle.run(wl.n, wl.gates, wl.params)
    oracle.expect(wl.n, st, wl.observables)
t0 = time.perf_counter(); step(); per = time.perf_counter() - t0
steps = max(1, int(budget / max(per, 1e-6)))
t0 = time.perf_counter()
for _ in range(steps):
    step()
print(json.dumps({"steps": steps, "seconds": time.perf_counter() - t0, "cores": oracle.num_threads()}))
"""


def oracle_timing(budget_s, threads=None):
    """Full oracle steps (480-gate forward + <sum Z>) of the headline workload
    in a fresh process (nothing else of this process competes for the cores),
    as many as fit the time budget (at least one); threads=1 holds OpenMP to
    one core."""
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    out = subprocess.run([sys.executable, "-c", _ORACLE_TIMER, str(budget_s)], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        tail = out.stderr.strip().splitlines()
        return {"unavailable": tail[-1][:160] if tail else "failed"}
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_line_values(wl, steps, seconds):
    """The oracle's figures in the line's units: amplitude-GB/s of the passes
    it makes, gate-equivalent GB/s and ms per step."""
    nterms = sum(len(o) for o in wl.observables)
    return {"value": oracle_pass_bytes(wl.n, len(wl.gates), nterms) * steps / seconds / 1e9,
            "gate_equivalent": gate_pass_bytes(wl.n, wl.gates) * steps / seconds / 1e9,
            "ms_per_step": 1e3 * seconds / steps}


def cpu_leg(wl, budget_s, gpu_state, gpu_expect):
    """The oracle beside the GPU: timed on all host cores and on one core
    (fresh processes), and the headline result's error against it (the final
    state's max-abs amplitude error, the relative error of <sum Z>)."""
    allc = oracle_timing(budget_s)
    if "unavailable" in allc:
        return {"unavailable": allc["unavailable"]}, None
    one = oracle_timing(max(2.0, budget_s / 3), threads=1)
    v = oracle_line_values(wl, allc["steps"], allc["seconds"])
    cpu = {"value": v["value"], "unit": UNIT, "cores": allc["cores"], "kind": "oracle",
           "sample": (f"{allc['steps']} full steps (480-gate forward + <sum Z>) in {allc['seconds']:.1f} s on "
                      f"{allc['cores']} threads, in a fresh process; one thread: "
                      + (f"{oracle_line_values(wl, one['steps'], one['seconds'])['value']:.2f} GB/s"
                         if "steps" in one else "unavailable")),
           "ms_per_step": v["ms_per_step"], "gate_equivalent": v["gate_equivalent"]}
    if "steps" in one:
        o1 = oracle_line_values(wl, one["steps"], one["seconds"])
        cpu["single_thread_value"] = o1["value"]
        cpu["single_thread_ms_per_step"] = o1["ms_per_step"]
    import oracle
    oracle.build()
    ref = oracle.run(wl.n, wl.gates, wl.params)
    e_ref = float(oracle.expect(wl.n, ref, wl.observables)[0, 0])
    amp_err = float(np.max(np.abs(gpu_state.reshape(-1) - ref.reshape(-1))))
    e_err = abs(float(gpu_expect) - e_ref)
    errors = {"state_max_abs": amp_err, "state_tol": 1e-5,
              "expect_sum_z": float(gpu_expect), "expect_sum_z_oracle": e_ref,
              "expect_abs": e_err, "expect_rel": e_err / max(abs(e_ref), 1e-300), "expect_tol_rel": 1e-4,
              "against": "FP64 oracle, same seeded parameters"}
    return cpu, errors


def max_over_ranks(ms, world, dist, device):
    """The job's time: the slowest replica's (all ranks receive it)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, bytes_step, steps, ms):
    """Whole-job GB/s: every replica moves bytes_step per step."""
    return world * bytes_step * steps / (ms / 1e3) / 1e9


def reference_arm(args, rank, world):
    """The oracle on the host cores, as the reference arm."""
    if rank != 0:
        return
    wl = W.config_c2()
    import oracle
    oracle.build()
    # bounded steps: each step is a full forward + expectation when K*W fits
    # ~3 minutes, else a prefix of the gate list (the unit stays per gate).
    t0 = time.perf_counter()
    st = oracle.run(wl.n, wl.gates, wl.params)
    oracle.expect(wl.n, st, wl.observables)
    full = time.perf_counter() - t0
    total_steps = args.steps + args.warmup
    frac = min(1.0, 180.0 / max(total_steps * full, 1e-9))
    ng = max(1, int(len(wl.gates) * frac))
    gates = wl.gates[:ng]
    for _ in range(args.warmup):
        s = oracle.run(wl.n, gates, wl.params)
        oracle.expect(wl.n, s, wl.observables)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = oracle.run(wl.n, gates, wl.params)
        oracle.expect(wl.n, s, wl.observables)
    dt = time.perf_counter() - t0
    nterms = sum(len(o) for o in wl.observables)
    value = oracle_pass_bytes(wl.n, len(gates), nterms) * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "gate_equivalent": {"value": gate_pass_bytes(wl.n, gates) * args.steps / dt / 1e9, "unit": UNIT},
        "value_definition": "amplitude bytes of the passes the oracle makes (one complex128 read+write sweep per "
                            "gate, three per Pauli term) / step time",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
        "data": "synthetic",
        "config": {"workload": "c2_hea20_c64", "nqubits": 20, "layers": 8, "gates": len(wl.gates),
                   "params": wl.nparams, "batch": 1, "gates_per_step": ng},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} steps of the first {ng} of {len(wl.gates)} gates + <sum Z>"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def our_arm(args, rank, world, dist):
    import torch
    import paper_2512_18995_gb300 as dq
    from paper_2512_18995_gb300 import build as dqbuild

    dqbuild.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device(f"cuda:{local}")
    ctx = dq.Context(local, path={"auto": dq.PATH_AUTO, "plain": dq.PATH_PLAIN, "fused": dq.PATH_FUSED}[args.path])
    hbm_peak, peak_kind = peaks()

    wl = W.config_c2()
    n = wl.n
    circ = dq.Circuit(n, wl.gates, nparams=wl.nparams)
    obs = dq.Observables(wl.observables)
    params = torch.tensor(wl.params, dtype=torch.float64, device=device)
    state = torch.empty((1, 1 << n), dtype=torch.complex64, device=device)
    expect = torch.empty((1, 1), dtype=torch.float64, device=device)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)
    ctx.set_graphs(not args.no_graphs)   # before tuning: the tuner times the way the context runs
    if args.path != "plain":
        ctx.plan_autotune(circ, state)

    def step():
        ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=state, expect_out=expect)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed():
        launches0 = ctx.launch_count
        with ClockSampler(local) as clk:
            barrier()
            for i in range(args.steps):
                flush.zero_()
                starts[i].record()
                step()
                ends[i].record()
            barrier()
        ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world, dist, device)
        return ms, ctx.launch_count - launches0, clk.summary()

    ms, launches, clocks = timed()
    # a run that saw thermal or hardware slowdown (or clocks far below their
    # maximum with no reason given) is measured once more, on every rank
    if any_rank(throttled(clocks), world, dist, device):
        first = clocks
        ms, launches, clocks = timed()
        clocks["remeasured_after"] = {"reasons": first["reasons"], "sm_mhz": first["sm_mhz"]}
    # per-kernel launches and device-time shares: a traced repetition of the
    # same timed steps.  With graphs on, the per-launch CUDA events are nodes of
    # the replayed graph (recorded on the launching stream); the first two
    # traced steps (run once, then captured) are left out.  The event nodes add
    # time of their own, so only the shares are taken from this run: the
    # dominant kernel's duration is its share of the untraced step time.
    ctx.set_tracing(True)
    for _ in range(2):
        flush.zero_()
        step()
    base = ctx.trace()
    for i in range(args.steps):
        flush.zero_()
        step()
    trace = {k: (v[0] - base.get(k, (0, 0.0))[0], v[1] - base.get(k, (0, 0.0))[1]) for k, v in ctx.trace().items()}
    trace = {k: v for k, v in trace.items() if v[0] > 0}
    ctx.set_tracing(False)
    passes = forward_passes(ctx, circ, torch.complex64)
    per_launch = kernel_bytes(n, wl.gates, passes)
    bytes_step = sum(per_launch.get(k, 0) * c for k, (c, _) in trace.items()) / args.steps
    if "k_sweep" in trace:
        bytes_step += sum(touched_bytes(n, g) for g in wl.gates if g.kind != "swap")
    value = job_value(world, bytes_step, args.steps, ms)
    gate_equiv = job_value(world, gate_pass_bytes(n, wl.gates), args.steps, ms)
    traced_total = sum(v[1] for v in trace.values())
    kname, (klaunch, kms) = max(trace.items(), key=lambda kv: kv[1][1])
    share = kms / traced_total
    launches_step = klaunch / args.steps
    avg_ms = share * (ms / args.steps) / launches_step
    kbytes = per_launch[kname] if kname in per_launch else 2 * (1 << n) * 8
    if kname == "k_sweep":
        kbytes = sum(touched_bytes(n, g) for g in wl.gates if g.kind != "swap") / launches_step
    achieved = kbytes / (avg_ms / 1e3) / 1e9
    tuned = ctx.plan_tuned(circ)
    traffic = recorded_traffic(kname, tuned if kname == "k_tile_fwd_jit" else None)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic.get("bytes"), "peak_kind": peak_kind,
                "frac_of_nominal_8TBps": achieved / NOMINAL_HBM_GBS,
                "launches": launches_step, "avg_launch_us": 1e3 * avg_ms, "bytes_per_launch": kbytes,
                "share_of_step": share, "passes_per_step": passes,
                "timing": "untraced step time x the kernel's share of a traced repetition of the same steps",
                "traffic_source": traffic.get("source"),
                "tile_shape": {"k": tuned[0], "low": tuned[1], "M": tuned[2]},
                "note": "20-qubit state (8 MiB) is L2-resident within a step"}
    kernels_step = {k: {"launches": c / args.steps, "share": t / traced_total} for k, (c, t) in trace.items()}

    # the last step's result, for the error against the oracle (cpu leg)
    torch.cuda.synchronize()
    final_state = state.detach().cpu().numpy().astype(np.complex128)
    final_expect = float(expect.cpu().item())

    # end to end through the public API with host buffers: dq_forward_host
    # copies the parameters in from pinned host memory, runs the step, copies
    # <sum Z> back and synchronises, every step (one graph replay a step)
    host_params = torch.tensor(wl.params, dtype=torch.float64).pin_memory()
    host_expect = torch.empty((1, 1), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    for _ in range(2):   # same buffers as the timed loop (graph captured)
        ctx.forward_host(circ, host_params, obs, 1, torch.complex64, expect_out=host_expect)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.forward_host(circ, host_params, obs, 1, torch.complex64, expect_out=host_expect)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * bytes_step * e2e_steps / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": int(host_params.numel() * 8), "d2h_bytes_per_step": 8,
           "call": "dq_forward_host, pinned host buffers", "ms_per_step": 1e3 * e2e_s / e2e_steps,
           "expect_sum_z": float(host_expect[0, 0])}

    extras = {}
    if not args.no_extras:
        runs = {
            "hbm_sweep": lambda: hbm_sweep(ctx, device, hbm_peak, peak_kind),
            "grads": lambda: batched_grads(ctx, device),
            "dense_block": lambda: dense_block(ctx, device, hbm_peak, peak_kind),
            "dense_planner": lambda: dense_planner(ctx, device, hbm_peak, peak_kind),
            "uneven_batch": lambda: uneven_batch(ctx, device),
            "qft_tfim30": lambda: qft_tfim30(ctx, device),
            "qcnn": lambda: qcnn_batch(ctx, device),
            "trotter30": lambda: trotter30(ctx, device),
            "sample30": lambda: sample30(ctx, device, hbm_peak, peak_kind),
            "hessian": lambda: hessian_hea(ctx, device),
            "density": lambda: density_noisy(ctx, device),
        }
        pick = list(runs) if args.extras == "all" else [x for x in args.extras.split(",") if x]
        for name in pick:
            extras[name] = runs[name]()
        ctx.set_path({"auto": dq.PATH_AUTO, "plain": dq.PATH_PLAIN, "fused": dq.PATH_FUSED}[args.path])

    if rank == 0:
        cpu, errors = None, None
        if world == 1 and not args.no_cpu:
            cpu, errors = cpu_leg(wl, args.cpu_budget, final_state, final_expect)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "c2_hea20_c64", "nqubits": n, "layers": 8, "gates": len(wl.gates),
                       "params": wl.nparams, "batch": 1, "path": args.path, "graphs": not args.no_graphs,
                       "l2": "flushed between steps (512 MiB write)", "parallelism": f"replicas x{world}"},
            "value_definition": "amplitude bytes of the full-state passes the kernels make "
                                "(2 * 2^n * 8 B per pass, the state preparation 2^n * 8 B) / step time",
            "gate_equivalent": {"value": gate_equiv, "unit": UNIT,
                                "definition": "480 gates x one read+write sweep of 2^20 complex64 each / step time"},
            "roofline": roofline, "kernels_per_step": kernels_step, "cpu_baseline": cpu,
            "errors_vs_oracle": errors, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()


def forward_passes(ctx, circ, dtype):
    """Forward tile passes of the schedule the fused path runs for circ (the
    autotuned configuration, else the library's default), or None."""
    from paper_2512_18995_gb300 import _lib
    k, low, m = ctx.plan_tuned(circ, dtype)
    if not k:
        return None
    try:
        return len(_lib.tile_schedule(circ, k, low, m, _lib.dtype_code(dtype)))
    except Exception:
        return None


def kernel_bytes(n, gates, passes, amp=8):
    """Algorithmic amplitude bytes per launch of the kernels of the headline
    step: a tile pass reads and writes the state once, the persistent
    multi-pass kernel does so once per pass, the state preparation writes it
    once, a per-gate expectation pass reads it once."""
    full = (1 << n) * amp
    out = {"k_tile_fwd": 2 * full, "k_tile_fwd_jit": 2 * full, "k_init_zero": full, "k_bind_init": full,
           "k_expect": full}
    if passes:
        out["k_tile_multi"] = 2 * full * passes
    return out


def source_fingerprint(files, extra=b""):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2512_18995_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    h.update(extra)
    return h.hexdigest()[:16]


# DRAM traffic per launch recorded from one ncu capture of the kernel (the
# profile summary states the figure and the fingerprint of the sources the
# capture was built from); reported only while those sources are unchanged.
# The specialised passes are fingerprinted by what they are compiled from:
# the generated source of the headline schedule and the device headers it
# includes.
JIT_FWD_HEADERS = ["dq_tile_fwd.cuh", "dq_engine.cuh", "dq_tma.cuh", "dq_common.cuh", "dq_devterm.h"]
TRAFFIC_RECORDS = {
    "k_tile_multi": ("k_tile_multi_c2_hea20.md", ["k_tile.cu", "dq_engine.cuh", "dq_tma.cuh", "dq_common.cuh"]),
    "k_tile_fwd": ("k_tile_fwd_c2_hea20.md", ["k_tile.cu", "dq_engine.cuh", "dq_tma.cuh", "dq_common.cuh"]),
    "k_tile_fwd_jit": ("k_tile_fwd_jit_c2_hea20.md", JIT_FWD_HEADERS),
}


def headline_jit_source(shape=None):
    """The generated source of the headline circuit's specialised forward
    passes for tile shape (k, low, M) (default: the shape its tuner picks on
    a GB300, 12 / 5 / 4)."""
    import paper_2512_18995_gb300 as dq
    from paper_2512_18995_gb300 import _lib
    wl = W.config_c2()
    k, low, M = shape if shape and shape[0] else (12, 5, 4)
    return _lib.jit_source(dq.Circuit(wl.n, wl.gates, nparams=wl.nparams), k, low, M).encode()


def traffic_fingerprint(kname, shape=None):
    rec = TRAFFIC_RECORDS[kname]
    return source_fingerprint(rec[1], headline_jit_source(shape) if kname == "k_tile_fwd_jit" else b"")


def recorded_traffic(kname, shape=None):
    rec = TRAFFIC_RECORDS.get(kname)
    if not rec:
        return {}
    path = os.path.join(ROOT, "profiles", rec[0])
    if not os.path.exists(path):
        return {}
    import re
    found = re.findall(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+sources:\s*([0-9a-f]{16})", open(path).read())
    if not found:
        return {}
    fp = traffic_fingerprint(kname, shape)
    for bytes_, fp_rec in found:   # one record per captured schedule
        if fp_rec == fp:
            return {"bytes": float(bytes_), "source": f"profiles/{rec[0]}"}
    return {"source": f"profiles/{rec[0]} (stale: no capture of the kernels as built now)"}


def hbm_sweep(ctx, device, hbm_peak, peak_kind, n=30, reps=3):
    """Single one-qubit gate sweeps on an 8 GiB state (far beyond L2)."""
    import torch
    import paper_2512_18995_gb300 as dq
    ctx.set_path(dq.PATH_PLAIN)
    try:
        state = torch.empty((1, 1 << n), dtype=torch.complex64, device=device)
    except RuntimeError:
        return None
    ctx.state_init(state, n)
    targets = [0, 1, 3, 7, 12, 18, 24, 29]
    gates = [W.Gate("ry", (q,), angle=0.3 + 0.01 * q) for q in targets]
    circ = dq.Circuit(n, gates)
    ctx.apply_circuit(circ, None, state)
    torch.cuda.synchronize()
    ctx.set_tracing(True)
    for _ in range(reps):
        ctx.apply_circuit(circ, None, state)
    tr = ctx.trace()
    ctx.set_tracing(False)
    cnt, tot = tr["k_sweep"]
    per_ms = tot / cnt
    gbs = 2 * (1 << n) * 8 / (per_ms / 1e3) / 1e9
    del state
    torch.cuda.empty_cache()
    return {"n": n, "kernel": "k_sweep", "launches": cnt, "avg_launch_ms": per_ms, "GB/s": gbs,
            "peak": hbm_peak, "frac_of_measured_copy": gbs / hbm_peak, "peak_kind": peak_kind,
            "frac_of_nominal_8TBps": gbs / NOMINAL_HBM_GBS, "targets": targets}


def dense_block(ctx, device, hbm_peak, peak_kind, n=30, reps=4):
    """Tensor-core dense 64 x 64 complex block on the six lowest-order qubits
    of an 8 GiB complex64 state: HBM GB/s and three-pass TF32 FLOP/s."""
    import torch
    try:
        state = torch.empty((1, 1 << n), dtype=torch.complex64, device=device)
    except RuntimeError:
        return None
    ctx.state_init(state, n)
    U = torch.from_numpy(W.random_unitary(6, 6)).to(device)
    ctx.apply_dense(n, U, state)
    torch.cuda.synchronize()
    ctx.set_tracing(True)
    for _ in range(reps):
        ctx.apply_dense(n, U, state)
    tr = ctx.trace()
    ctx.set_tracing(False)
    cnt, tot = tr["k_dense"]
    per_ms = tot / cnt
    rows = 1 << (n - 6)
    gbs = 2 * (1 << n) * 8 / (per_ms / 1e3) / 1e9
    tflops = 3 * 2 * 128 * 128 * rows / (per_ms / 1e3) / 1e12
    # TF32 dense peak: the measured bf16 GEMM peak times the nominal TF32/BF16 ratio (1.1 / 2.25)
    bf16 = bf16_peak()
    tf32_peak = bf16 * (1.1 / 2.25) if bf16 else 1900.0 * (1.1 / 2.25)
    del state
    torch.cuda.empty_cache()
    return {"n": n, "kernel": "k_dense", "launches": cnt, "avg_launch_ms": per_ms, "GB/s": gbs,
            "hbm_frac_of_measured_copy": gbs / hbm_peak, "hbm_frac_of_nominal_8TBps": gbs / NOMINAL_HBM_GBS,
            "peak_kind": peak_kind, "tflops_tf32x3": tflops,
            "tf32_peak": tf32_peak, "tensor_frac": tflops / tf32_peak,
            "tf32_peak_kind": "measured bf16 x nominal tf32/bf16" if bf16 else "fallback bf16 x nominal tf32/bf16"}


def dense_planner(ctx, device, hbm_peak, peak_kind, n=28, layers=6):
    """Dense blocks chosen by the planner on a forward-only call: 28 qubits
    (2 GiB complex64), a brick wall of two-qubit gates on the six
    lowest-order wires (six layers: RY, RZ on each wire, a CNOT chain and
    CZ/CRY couplings -- 144 gates in one run) between two RY/RZ + CNOT-ring
    layers on all wires.  Time with dense blocks on vs tile passes only."""
    import torch
    import paper_2512_18995_gb300 as dq
    w = list(range(n - 6, n))
    gates = W.hea_layers(n, 1)
    p = 2 * n
    for _ in range(layers):
        for q in w:
            gates += [W.Gate("ry", (q,), param=p), W.Gate("rz", (q,), param=p + 1)]
            p += 2
        gates += [W.Gate("cnot", (a, b)) for a, b in zip(w[:-1], w[1:])]
        gates += [W.Gate("cz", (w[0], w[5])), W.Gate("cry", (w[2], w[4]), param=p), W.Gate("cry", (w[5], w[1]),
                                                                                            param=p + 1)]
        p += 2
    gates += W.hea_layers(n, 1, first_param=p)
    p += 2 * n
    circ = dq.Circuit(n, gates, nparams=p)
    params = torch.tensor(W.uniform_array(W._seed(28), p, 0.0, 2 * np.pi), device=device)
    obs = dq.Observables([W.obs_sum_z(n)])
    try:
        st = torch.empty((1, 1 << n), dtype=torch.complex64, device=device)
    except RuntimeError as exc:
        return {"skipped": str(exc)[:120]}
    ctx.set_path(dq.PATH_FUSED)
    ctx.plan_autotune(circ, st)
    out = {"workload": f"dense_brickwall{n}_c64", "gates": len(gates), "run_gates": 17 * layers}
    for name, mode in (("tiles_only", 0), ("dense_blocks", 1)):
        ctx.set_option(dq.OPT_DENSE_BLOCKS, mode)
        ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=st)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=st)
        b.record()
        torch.cuda.synchronize()
        out[name] = {"ms_per_step": a.elapsed_time(b) / 3}
        if mode == 1:
            ctx.set_tracing(True)
            ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=st)
            out[name]["kernels"] = {k: [v[0], round(v[1], 3)] for k, v in ctx.trace().items()}
            ctx.set_tracing(False)
    ctx.set_option(dq.OPT_DENSE_BLOCKS, 2)
    ctx.set_path(dq.PATH_AUTO)
    out["speedup"] = out["tiles_only"]["ms_per_step"] / out["dense_blocks"]["ms_per_step"]
    del st
    ctx.release_workspace()
    torch.cuda.empty_cache()
    return out


def qft_tfim30(ctx, device):
    """30 qubits (8 GiB complex64 per vector): QFT then 10 RY/RZ + CNOT-ring
    layers (600 parameters), open-chain TFIM energy and all 600 gradients,
    the fused path vs the per-gate path (one warm-up and one timed call each)."""
    import torch
    import paper_2512_18995_gb300 as dq
    wl = W.config_c5(30)
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    obs = dq.Observables(wl.observables)
    params = torch.tensor(wl.params, device=device)
    out = {}
    for name, path, jit in (("fused", dq.PATH_FUSED, 1), ("fused_interpreted", dq.PATH_FUSED, 0),
                            ("plain", dq.PATH_PLAIN, 0)):
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        try:
            ctx.forward_grad(circ, params, obs, 1, torch.complex64)   # warm-up (and the passes' compile)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.forward_grad(circ, params, obs, 1, torch.complex64)
            b.record()
            torch.cuda.synchronize()
        except RuntimeError as exc:   # not enough device memory
            ctx.set_path(dq.PATH_AUTO)
            ctx.set_option(dq.OPT_JIT, 2)
            return {"skipped": str(exc)[:120]}
        ms = a.elapsed_time(b)
        out[name] = {"ms_per_step": ms, "grads_per_s": wl.nparams / (ms / 1e3)}
        if name == "fused":
            ctx.set_tracing(True)
            ctx.forward_grad(circ, params, obs, 1, torch.complex64)
            out[name]["kernel_ms"] = {k: [v[0], round(v[1], 2)] for k, v in ctx.trace().items()}
            ctx.set_tracing(False)
    ctx.set_path(dq.PATH_AUTO)
    ctx.set_option(dq.OPT_JIT, 2)
    ctx.release_workspace()
    torch.cuda.empty_cache()
    out["speedup"] = out["plain"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["workload"] = "c5_qft_tfim30_c64"
    out["fused_note"] = "forward and reverse tile passes as run-time specialised kernels (DQ_OPT_JIT = 1)"
    return out


def trotter30(ctx, device, steps=5):
    """Trotterised TFIM quench on 30 qubits (8 GiB complex64): `steps`
    second-order Trotter steps (RX half steps and RZZ on every bond of the
    periodic chain, fixed angles) from |0...0>, then <H>; fused path vs
    per-gate path.  Gate-equivalent bandwidth counts one read and one write
    of the state per gate of the circuit as written (RZZ counted once)."""
    import torch
    import paper_2512_18995_gb300 as dq
    n = 30
    gates = W.tfim_trotter_gates(n, steps)
    circ = dq.Circuit(n, gates, nparams=0)
    H = dq.Observables([[W.pauli_term(-1.0, {i: "Z", (i + 1) % n: "Z"}) for i in range(n)]
                        + [W.pauli_term(-1.2, {i: "X"}) for i in range(n)]])
    out = {}
    # fused: tile passes compiled per circuit (DQ_OPT_JIT = 1; the compile is
    # part of the untimed warm-up call); fused_interpreted: the interpreting kernels
    for name, path, jit in (("fused", dq.PATH_FUSED, 1), ("fused_interpreted", dq.PATH_FUSED, 0),
                            ("plain", dq.PATH_PLAIN, 0)):
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        try:
            ctx.forward_grad(circ, None, H, 1, torch.complex64, want_grad=False)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.forward_grad(circ, None, H, 1, torch.complex64, want_grad=False)
            b.record()
            torch.cuda.synchronize()
        except RuntimeError as exc:   # not enough device memory
            ctx.set_path(dq.PATH_AUTO)
            ctx.set_option(dq.OPT_JIT, 2)
            return {"skipped": str(exc)[:120]}
        ms = a.elapsed_time(b)
        out[name] = {"ms_per_step": ms,
                     "gate_equiv_GBps": len(gates) * 2 * (8 << n) / (ms / 1e3) / 1e9}
    ctx.set_path(dq.PATH_AUTO)
    ctx.set_option(dq.OPT_JIT, 2)
    ctx.release_workspace()
    torch.cuda.empty_cache()
    out["speedup"] = out["plain"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["workload"] = f"tfim_trotter30_{steps}steps_c64"
    out["gates"] = len(gates)
    return out


def sample30(ctx, device, hbm_peak, peak_kind, n=30, shots=1 << 20, reps=3):
    """2^20 shots from a 30-qubit complex64 state (8 GiB): one streaming pass
    for the cumulative sums, then per shot a search over group prefixes, a
    search of up to 1024 chunk prefixes and a scan of one 32-amplitude chunk.
    Algorithmic HBM bytes: the state once, the chunk prefixes written (8 B per
    32 amplitudes) and 256 B of amplitudes per shot."""
    import torch
    try:
        gen = torch.Generator(device=device).manual_seed(30)
        st = torch.randn((1, 1 << n), dtype=torch.complex64, device=device, generator=gen)
        out = torch.empty((1, shots), dtype=torch.int64, device=device)
        ctx.sample(n, st, shots, seed=1, out=out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for r in range(reps):
            ctx.sample(n, st, shots, seed=2 + r, out=out)
        b.record()
        torch.cuda.synchronize()
    except RuntimeError as exc:
        return {"skipped": str(exc)[:120]}
    ms = a.elapsed_time(b) / reps
    nbytes = (8 << n) + (8 << (n - 5)) + shots * 32 * 8
    ctx.set_tracing(True)
    ctx.sample(n, st, shots, seed=9, out=out)
    kernels = {k: round(v[1], 3) for k, v in ctx.trace().items()}
    ctx.set_tracing(False)
    del st, out
    ctx.release_workspace()
    torch.cuda.empty_cache()
    return {"workload": "sample_30q_1Mshots_c64", "ms_per_call": ms, "shots_per_s": shots / (ms / 1e3),
            "GBps": nbytes / (ms / 1e3) / 1e9, "frac_of_measured_copy": nbytes / (ms / 1e3) / 1e9 / hbm_peak,
            "frac_of_nominal_8TBps": nbytes / (ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
            "peak_kind": peak_kind, "kernel_ms": kernels}


def hessian_workload(n=22, layers=2):
    """The layered ansatz of the gradient-and-Hessian benchmark at 22 qubits:
    2 layers of RY/RZ + CNOT ring (88 parameters), <sum_i Z_i>."""
    g = W.hea_layers(n, layers)
    p = W.uniform_array(W._seed(22), 2 * n * layers, 0.0, 2 * np.pi)
    return W.Workload(f"hessian_hea{n}x{layers}_c64", n, "c64", 1, g, p.size, p, False, 0, None,
                      [W.obs_sum_z(n)], True, False)


def _arms():
    import paper_2512_18995_gb300 as dq
    # fused: passes compiled per circuit (DQ_OPT_JIT = 1, the compile falls in
    # the untimed warm-up call); fused_interpreted: the interpreting kernels
    return (("fused", dq.PATH_FUSED, 1), ("fused_interpreted", dq.PATH_FUSED, 0), ("plain", dq.PATH_PLAIN, 0))


def hessian_hea(ctx, device):
    """Full 88 x 88 Hessian of <sum Z> for the 22-qubit, 2-layer ansatz: 176
    shifted points of the fused forward + adjoint as one batch, vs the same
    on the per-gate path."""
    import torch
    import paper_2512_18995_gb300 as dq
    wl = hessian_workload()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
    obs = dq.Observables(wl.observables)
    params = torch.tensor(wl.params, device=device)
    out = {}
    for name, path, jit in _arms():
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        try:
            ctx.hessian(circ, params, obs, want_grad=False)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.hessian(circ, params, obs, want_grad=False)
            b.record()
            torch.cuda.synchronize()
        except RuntimeError as exc:
            ctx.set_path(dq.PATH_AUTO)
            ctx.set_option(dq.OPT_JIT, 2)
            return {"skipped": str(exc)[:120]}
        ms = a.elapsed_time(b)
        out[name] = {"ms_per_hessian": ms, "entries_per_s": wl.nparams ** 2 / (ms / 1e3)}
        if name == "fused":
            ctx.set_tracing(True)
            ctx.hessian(circ, params, obs, want_grad=False)
            out[name]["kernel_ms"] = {k: [v[0], round(v[1], 3)] for k, v in ctx.trace().items()}
            ctx.set_tracing(False)
    ctx.set_path(dq.PATH_AUTO)
    ctx.set_option(dq.OPT_JIT, 2)
    ctx.release_workspace()
    torch.cuda.empty_cache()
    out["speedup"] = out["plain"]["ms_per_hessian"] / out["fused"]["ms_per_hessian"]
    out["workload"] = wl.name
    return out


def density_gates(n=13, layers=4, p=0.01):
    """Layered ansatz (RY, RZ, CNOT ring) with a depolarizing channel of
    probability p on every qubit after each layer."""
    g = []
    for l in range(layers):
        g += W.hea_layers(n, 1, first_param=2 * n * l)
        g += [W.Gate("depolarizing", (q,), angle=p) for q in range(n)]
    return g


def density_noisy(ctx, device, n=13, layers=4):
    """Noisy 13-qubit circuit as a density matrix (a 26-qubit vectorised
    register, 512 MiB complex64): forward evolution and <sum Z>, fused vs
    per-gate path."""
    import torch
    import paper_2512_18995_gb300 as dq
    gates = density_gates(n, layers)
    circ = dq.Circuit(n, gates, nparams=2 * n * layers)
    obs = dq.Observables([W.obs_sum_z(n)])
    params = torch.tensor(W.uniform_array(W._seed(13), 2 * n * layers, 0.0, 2 * np.pi), device=device)
    out = {}
    for name, path, jit in _arms():
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        try:
            ctx.density_forward(circ, params, obs, 1, torch.complex64)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.density_forward(circ, params, obs, 1, torch.complex64)
            b.record()
            torch.cuda.synchronize()
        except RuntimeError as exc:
            ctx.set_path(dq.PATH_AUTO)
            ctx.set_option(dq.OPT_JIT, 2)
            return {"skipped": str(exc)[:120]}
        out[name] = {"ms_per_step": a.elapsed_time(b)}
    ctx.set_path(dq.PATH_AUTO)
    out["speedup"] = out["plain"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["workload"] = f"density_hea{n}x{layers}_depolarizing_c64"
    out["gates"] = len(gates)
    # gradients of the same kind of circuit at 10 qubits, 2 layers (40 parameters,
    # 80 shifted density rows of 2^20 amplitudes)
    ng, lg = 10, 2
    gg = density_gates(ng, lg)
    cg = dq.Circuit(ng, gg, nparams=2 * ng * lg)
    og = dq.Observables([W.obs_sum_z(ng)])
    pg = torch.tensor(W.uniform_array(W._seed(10), 2 * ng * lg, 0.0, 2 * np.pi), device=device)
    grad = {}
    for name, path, jit in _arms():
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        ctx.density_grad(cg, pg, og, dtype=torch.complex64)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.density_grad(cg, pg, og, dtype=torch.complex64)
        b.record()
        torch.cuda.synchronize()
        grad[name] = {"ms_per_gradient": a.elapsed_time(b)}
    ctx.set_path(dq.PATH_AUTO)
    ctx.set_option(dq.OPT_JIT, 2)
    grad["speedup"] = grad["plain"]["ms_per_gradient"] / grad["fused"]["ms_per_gradient"]
    grad["workload"] = f"density_grad_hea{ng}x{lg}_depolarizing_c64"
    out["grad"] = grad
    return out


def qcnn_batch(ctx, device, batch=4096, steps=5):
    """The 12-qubit QCNN (RY encodings, RXX/RYY convolutions, CRY pooling; 33
    parameters, 21 features per row) on 4096 rows: <Z_0>, gradients with
    respect to the parameters and to every feature; fused vs per-gate path."""
    import torch
    import paper_2512_18995_gb300 as dq
    gates, npar, nfeat = W.qcnn_gates(12)
    circ = dq.Circuit(12, gates, nparams=npar, nfeatures=nfeat)
    obs = dq.Observables([W.obs_z(0)])
    params = torch.tensor(W.uniform_array(71, npar, 0.0, 2 * np.pi), device=device)
    data = torch.tensor(W.uniform_array(72, batch * nfeat, -np.pi, np.pi).reshape(batch, nfeat), device=device)
    out = {}
    for name, path, jit in _arms():
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        for _ in range(2):
            ctx.forward_grad(circ, params, obs, batch, torch.complex64, data=data)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            ctx.forward_grad(circ, params, obs, batch, torch.complex64, data=data)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": ms, "grads_per_s": batch * (npar + nfeat) / (ms / 1e3)}
    ctx.set_path(dq.PATH_AUTO)
    ctx.set_option(dq.OPT_JIT, 2)
    out["speedup"] = out["plain"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["workload"] = "qcnn12x4096_c64"
    return out


def uneven_batch(ctx, device, steps=3):
    """1024 circuits of 8..16 qubits and depth 10..40 (own parameters each):
    expectations and per-circuit adjoint gradients, the persistent uneven-
    batch kernel vs the per-gate path run circuit after circuit."""
    import torch
    import paper_2512_18995_gb300 as dq
    circs = W.config_c4(1024)
    dcs = [dq.Circuit(n, g, nparams=len(a)) for n, g, a in circs]
    params = torch.tensor(np.concatenate([a for _, _, a in circs]), device=device)
    obs = dq.Observables([W.obs_zz01_x0()])
    out = {}
    tuned = None
    for name, path in (("fused_default_launch", dq.PATH_FUSED), ("fused", dq.PATH_FUSED),
                       ("plain", dq.PATH_PLAIN)):
        ctx.set_path(path)
        if name == "fused":
            tuned = ctx.batch_autotune(dcs, params, obs, torch.complex64)
        ctx.batch_forward_grad(dcs, params, obs, torch.complex64)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            ctx.batch_forward_grad(dcs, params, obs, torch.complex64)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": ms, "circuits_per_s": len(circs) / (ms / 1e3)}
    ctx.set_path(dq.PATH_AUTO)
    out["fused"]["tuned_launch"] = {"qubits_in_shared_memory": tuned[0], "threads_per_circuit": tuned[1],
                                    "ctas_per_sm": tuned[2], "scratch_mib_in_flight": tuned[3]}
    out["speedup"] = out["plain"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["workload"] = "c4_uneven1024_c64"
    return out


def batched_grads(ctx, device, steps=5):
    """12 qubits x 4096 encoded samples, 6 layers (144 shared params):
    forward + adjoint gradient, fused path vs plain per-gate path."""
    import torch
    import paper_2512_18995_gb300 as dq
    wl = W.config_c3()
    circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams, nfeatures=wl.nfeatures)
    obs = dq.Observables(wl.observables)
    params = torch.tensor(wl.params, device=device)
    data = torch.tensor(wl.data, device=device)
    out = {}
    # fused: the autotuner picks the interpreting or the specialised
    # whole-row kernel (the latter compiled on first use); fused_interpreted
    # forces the interpreting kernel
    for name, path, jit in (("fused", dq.PATH_FUSED, 2), ("fused_interpreted", dq.PATH_FUSED, 0),
                            ("plain", dq.PATH_PLAIN, 0)):
        ctx.set_path(path)
        ctx.set_option(dq.OPT_JIT, jit)
        if name == "fused":
            tune = torch.empty((wl.batch, 1 << wl.n), dtype=torch.complex64, device=device)
            ctx.plan_autotune(circ, tune)
            del tune
        for _ in range(2):
            ctx.forward_grad(circ, params, obs, wl.batch, torch.complex64, data=data)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            ctx.forward_grad(circ, params, obs, wl.batch, torch.complex64, data=data)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": ms, "grads_per_s": wl.batch * wl.nparams / (ms / 1e3)}
        if name == "fused":
            ctx.set_tracing(True)
            ctx.forward_grad(circ, params, obs, wl.batch, torch.complex64, data=data)
            out[name]["kernel_ms"] = {k: [v[0], round(v[1], 3)] for k, v in ctx.trace().items()}
            ctx.set_tracing(False)
    ctx.set_path(dq.PATH_AUTO)
    ctx.set_option(dq.OPT_JIT, 2)
    out["speedup"] = out["plain"]["ms_per_step"] / out["fused"]["ms_per_step"]
    out["workload"] = "c3_qml12x4096_c64"
    return out


def profile_case(args):
    """Run one kernel family's workload a few times (for ncu captures): no
    JSON line, a one-line timing summary only."""
    import torch
    import paper_2512_18995_gb300 as dq
    from paper_2512_18995_gb300 import build as dqbuild
    dqbuild.build()
    dev = torch.device("cuda:0")
    ctx = dq.Context(0)
    iters = args.warmup + args.steps
    t0 = time.perf_counter()
    if args.profile_case == "c2":            # the headline step as the bench runs it (autotuned schedule)
        wl = W.config_c2()
        circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
        obs = dq.Observables(wl.observables)
        params = torch.tensor(wl.params, device=dev)
        st = torch.empty((1, 1 << wl.n), dtype=torch.complex64, device=dev)
        e = torch.empty((1, 1), dtype=torch.float64, device=dev)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        if args.tile:
            # under a profiler the tuner's timings change its choice: pin the
            # shape the bench's own tuned run reports (roofline.tile_shape),
            # with specialised passes
            k, low, M = (int(x) for x in args.tile.split(","))
            ctx.plan_set_tile(circ, k, low, M, jit=True)
        else:
            ctx.plan_autotune(circ, st)
        for _ in range(args.warmup):
            ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=st, expect_out=e)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()          # profilers started with capture off record from here
        for _ in range(args.steps):
            flush.zero_()
            ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=st, expect_out=e)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("tuned (k, low, M):", ctx.plan_tuned(circ), flush=True)
    elif args.profile_case == "tile":        # C2 forward on the fused tile path
        wl = W.config_c2()
        ctx.set_path(dq.PATH_FUSED)
        circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
        obs = dq.Observables(wl.observables)
        params = torch.tensor(wl.params, device=dev)
        st = torch.empty((1, 1 << wl.n), dtype=torch.complex64, device=dev)
        for _ in range(iters):
            ctx.forward_grad(circ, params, obs, 1, torch.complex64, want_grad=False, state_out=st)
    elif args.profile_case == "wsv":         # C3 fused forward + adjoint (--jit 1: the specialised whole-row kernel)
        wl = W.config_c3()
        ctx.set_path(dq.PATH_FUSED)
        if args.jit >= 0:
            ctx.set_option(dq.OPT_JIT, args.jit)
        circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams, nfeatures=wl.nfeatures)
        obs = dq.Observables(wl.observables)
        params = torch.tensor(wl.params, device=dev)
        data = torch.tensor(wl.data, device=dev)
        for _ in range(iters):
            ctx.forward_grad(circ, params, obs, wl.batch, torch.complex64, data=data)
    elif args.profile_case == "c4":          # uneven batch: 1024 circuits of 8..16 qubits, fwd + adjoint
        circs = W.config_c4(1024)
        dcs = [dq.Circuit(n, g, nparams=len(a)) for n, g, a in circs]
        params = torch.tensor(np.concatenate([a for _, _, a in circs]), device=dev)
        obs = dq.Observables([W.obs_zz01_x0()])
        ctx.set_path(dq.PATH_FUSED)
        for _ in range(iters):
            ctx.batch_forward_grad(dcs, params, obs, torch.complex64)
    elif args.profile_case == "sweep":       # one-qubit sweeps on a 2 GiB state
        n = 28
        ctx.set_path(dq.PATH_PLAIN)
        st = torch.empty((1, 1 << n), dtype=torch.complex64, device=dev)
        ctx.state_init(st, n)
        circ = dq.Circuit(n, [W.Gate("ry", (q,), angle=0.3) for q in (0, 7, 14, 21, 27)])
        for _ in range(iters):
            ctx.apply_circuit(circ, None, st)
    elif args.profile_case == "dense":       # tensor-core dense block on a 512 MiB state
        n = 26
        st = torch.empty((1, 1 << n), dtype=torch.complex64, device=dev)
        ctx.state_init(st, n)
        U = torch.from_numpy(W.random_unitary(6, 6)).to(dev)
        for _ in range(iters):
            ctx.apply_dense(n, U, st)
    elif args.profile_case == "c5":          # QFT + layers, forward + adjoint, 26 qubits, specialised passes
        wl = W.config_c5(26)
        ctx.set_path(dq.PATH_FUSED)
        ctx.set_option(dq.OPT_JIT, 1)
        circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
        obs = dq.Observables(wl.observables)
        params = torch.tensor(wl.params, device=dev)
        for _ in range(iters):
            ctx.forward_grad(circ, params, obs, 1, torch.complex64)
    elif args.profile_case == "sample":      # 2^18 shots from a 26-qubit state (512 MiB)
        n = 26
        gen = torch.Generator(device=dev).manual_seed(26)
        st = torch.randn((1, 1 << n), dtype=torch.complex64, device=dev, generator=gen)
        out = torch.empty((1, 1 << 18), dtype=torch.int64, device=dev)
        for i in range(iters):
            ctx.sample(n, st, 1 << 18, seed=i, out=out)
    elif args.profile_case == "hessian":     # 22-qubit, 2-layer ansatz Hessian (88 parameters)
        wl = hessian_workload()
        circ = dq.Circuit(wl.n, wl.gates, nparams=wl.nparams)
        obs = dq.Observables(wl.observables)
        params = torch.tensor(wl.params, device=dev)
        for _ in range(iters):
            ctx.hessian(circ, params, obs, want_grad=False)
    torch.cuda.synchronize()
    print(f"profile case {args.profile_case}: {iters} iterations in {time.perf_counter() - t0:.3f} s, "
          f"{ctx.launch_count} launches", flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", choices=["auto", "plain", "fused"], default="auto")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="all", help="comma-separated extra workloads to run (default: all)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graphs", action="store_true", help="issue kernels one by one (no CUDA-graph replay)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--jit", type=int, default=-1, help="profile cases: DQ_OPT_JIT value (default: the library's)")
    ap.add_argument("--tile", default="", help="profile case c2: pin the tile shape k,low,M (specialised passes)")
    ap.add_argument("--traffic-fingerprint", action="store_true",
                    help="print the source fingerprint of each kernel with a recorded DRAM traffic figure")
    ap.add_argument("--profile-case", choices=["c2", "tile", "wsv", "c4", "sweep", "c5", "dense", "sample", "hessian"],
                    default=None,
                    help="run one kernel family's workload for profiling and exit")
    args = ap.parse_args()
    if args.traffic_fingerprint:
        for kname in TRAFFIC_RECORDS:
            print(kname, traffic_fingerprint(kname, tuple(int(x) for x in args.tile.split(",")) if args.tile else None))
        return
    if args.profile_case:
        profile_case(args)
        return
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend="nccl")
    our_arm(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
