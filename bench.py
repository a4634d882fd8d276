"""Throughput of exact negacyclic polynomial multiplication on GB300.

Workload (the headline configuration): independent products c = a * b in
Z_q[X]/(X^N + 1) with N = 2^16 and q the largest 60-bit prime with
q = 1 mod 2^17, operands uniform in [0, q), `--batch` products per step
(default 1024: 1 GiB of operands, larger than L2, so no flush is needed
between steps).

One step = one pm_polymul call over the batch (forward NTTs of a and b,
Barrett pointwise product, inverse NTT), timed with CUDA events on its
stream.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the plain C implementation under
oracle/) on a bounded sample of the same workload on the host cores.
Multi-GPU: one replica per rank (the products are independent), launched by
torch.distributed.run; the value is the units of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "negacyclic polymults/sec (N=2^16, 60-bit q) and % of HBM/INT-mul roofline"


def mulmods_per_polymul(log2n: int) -> int:
    """Algorithmic modular products of Eq. 2: 3 NTTs of N/2 log2 N butterflies
    plus N pointwise products."""
    n = 1 << log2n
    return 3 * (n // 2) * log2n + n


def rows_kernel_mulmods(log2n: int, row_log: int = 12) -> int:
    """Modular products done by the row kernel of the split path for one unit:
    the in-row forward stages on a and b (12 for rows of 4096 words, 10 for
    rows of 1024), the pointwise product and as many inverse in-row stages."""
    n = 1 << log2n
    rows_stages = min(row_log, log2n)
    return 2 * rows_stages * (n // 2) + n + rows_stages * (n // 2)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons; only samples
    taken inside the timed window (wall clock) are summarised."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_index: int, period_ms: int = 20):
        self.dev = device_index
        self.period = period_ms
        self.proc = None
        self.samples = []  # (wall time, fields)
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), parts))

    def window(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(2 * self.period / 1000)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [p for (t, p) in self.samples
                if self.t0 is None or (self.t0 <= t <= self.t1 + self.period / 1000)]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        pw = [v for v in (num(r[3]) for r in rows) if v is not None]
        reasons = sorted({self.NAMES[i] for r in rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_min_mhz": min(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    return rank, ws, local, dist


def replica_seed(rank: int) -> int:
    """Input seed of one replica: every rank multiplies its own operands."""
    from paper_2209_01290_gb300 import inputs
    return inputs.seed_for(1) + 1000 * rank


def replica_max(x: float, dist) -> float:
    """Max over ranks of a per-rank float (the slowest replica decides the
    job's time); the identity without a process group.  NCCL groups reduce on
    the current CUDA device, others (gloo) on the host."""
    if dist is None:
        return x
    import torch
    dev = f"cuda:{torch.cuda.current_device()}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput under weak scaling: all ranks' products over the
    slowest rank's time."""
    return world * units_per_rank * steps / (max_ms * 1e-3)


def cpu_baseline(log2n: int, qs, psis, seconds: float = 12.0):
    """The oracle's scalar-NTT product on the host cores, on a bounded sample
    of the workload: as many products as keep every core busy for about
    `seconds` of wall time."""
    import oracle
    from paper_2209_01290_gb300 import inputs
    cores = os.cpu_count() or 1
    n = 1 << log2n
    a, b = inputs.operand_pair(inputs.seed_for(1) + 77, qs, cores, n)
    a2, b2 = a.reshape(-1, n), b.reshape(-1, n)
    t0 = time.perf_counter()
    oracle.polymul_ntt_batch(a2[:1], b2[:1], qs, psis, nthreads=1)  # probe one
    one = time.perf_counter() - t0
    per_thread = max(1, int(seconds / max(one, 1e-6)))
    units = min(cores * per_thread, cores * 256)
    reps = max(1, units // a2.shape[0])
    A = np.concatenate([a2] * reps)[:units]
    B = np.concatenate([b2] * reps)[:units]
    t0 = time.perf_counter()
    oracle.polymul_ntt_batch(A, B, qs, psis, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": "polymuls/s", "cores": cores, "kind": "oracle",
            "sample": f"{units} products at N=2^{log2n} (oracle textbook-NTT product, "
                      f"{cores} threads, {dt:.2f} s wall, about {dt * cores:.0f} core-s)"}


def run_reference(args):
    rank, ws, local, dist = _dist()
    if rank != 0:
        return 0
    # the oracle's own parameter search: this arm maps no GPU library
    import oracle
    from paper_2209_01290_gb300 import inputs
    n = 1 << args.log2n
    qs = oracle.find_primes(n, args.limbs, 60)
    psis = [oracle.find_psi(q, n) for q in qs]
    cores = os.cpu_count() or 1
    per_step = cores  # one product per core per step
    a, b = inputs.operand_pair(inputs.seed_for(1), qs, max(1, per_step // args.limbs), n)
    A, B = a.reshape(-1, n)[:per_step], b.reshape(-1, n)[:per_step]
    for _ in range(args.warmup):
        oracle.polymul_ntt_batch(A[:1], B[:1], qs, psis, nthreads=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.polymul_ntt_batch(A, B, qs, psis, nthreads=cores)
    dt = time.perf_counter() - t0
    value = A.shape[0] * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "polymuls/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"N=2^{args.log2n} negacyclic products, 60-bit q, "
                               f"{A.shape[0]} products per step (bounded CPU sample)"},
        "cpu_baseline": {"value": value, "unit": "polymuls/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{A.shape[0]} products per step x {args.steps} steps"},
        "e2e": {"value": value, "unit": "polymuls/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    rank, ws, local, dist = _dist()
    if dist is not None:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.cuda.current_device()
    from paper_2209_01290_gb300 import Plan, capi, inputs

    log2n, n, L = args.log2n, 1 << args.log2n, args.limbs
    npoly = max(1, args.batch // L)
    units = npoly * L
    qs, psis = capi.pm_find_params(log2n, L, 60)
    plan = Plan(n, qs, psis, device=dev, fused=args.fused)
    stream = torch.cuda.Stream(device=dev)
    plan.reserve(npoly, stream=stream)

    a, b = inputs.operand_pair(replica_seed(rank), qs, npoly, n)
    ha = torch.from_numpy(a.view(np.int64)).pin_memory()
    hb = torch.from_numpy(b.view(np.int64)).pin_memory()
    hc = torch.empty_like(ha).pin_memory()
    with torch.cuda.stream(stream):
        da = ha.to(dev, non_blocking=True)
        db = hb.to(dev, non_blocking=True)
        dc = torch.empty_like(da)
    stream.synchronize()

    peak_mulmod, peak_imad = capi.pm_measure_peaks(dev)
    if args.variant == "split":
        capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT, row_ops=args.row_ops)
    elif args.variant == "persistent":
        capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_PERSISTENT, args.ctas_per_sm,
                          args.lag_fwd, args.lag_inv, row_ops=args.row_ops)
    tuning = capi.pm_plan_get_tuning(plan.handle)
    persistent = tuning.variant == capi.PM_VARIANT_PERSISTENT and log2n >= 13

    # ---- warm-up
    for _ in range(args.warmup):
        plan.polymul(da, db, out=dc, stream=stream)
    stream.synchronize()

    # per-step phase events (recorded by the library on `stream`)
    nphase = 4 if (log2n >= 14 and not persistent) else 2
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nphase)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for e in [x for row in ev for x in row] + [start, end]:
        e.record(stream)  # torch creates the CUDA event on first record
    stream.synchronize()
    sampler = ClockSampler(dev, period_ms=10)  # a 4096-product step is ~8 ms: 10 ms sampling
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.5)  # let the sampler attach before the timed region
    t_wall0 = time.time()
    start.record(stream)
    for k in range(args.steps):
        capi.pm_plan_set_phase_events(plan.handle, [e.cuda_event for e in ev[k]])
        plan.polymul(da, db, out=dc, stream=stream)
    end.record(stream)
    stream.synchronize()
    sampler.window(t_wall0, time.time())
    clocks = sampler.stop()
    capi.pm_plan_set_phase_events(plan.handle, [])
    torch.cuda.synchronize(dev)
    elapsed_ms = replica_max(start.elapsed_time(end), dist)
    if dist is not None:
        dist.barrier()
    phase_ms = [[ev[k][i].elapsed_time(ev[k][i + 1]) for i in range(nphase - 1)]
                for k in range(args.steps)]
    avg_phase = [sum(p[i] for p in phase_ms) / args.steps for i in range(nphase - 1)]

    value = replica_value(units, args.steps, elapsed_ms, ws)

    # ---- end to end through the C ABI with host buffers: each step timed on
    # its own (pm_polymul_host returns once the result is in host memory);
    # the median step, since the host link is shared with other jobs and a
    # single disturbed step would otherwise set the figure
    e2e_steps = max(3, min(7, args.steps))
    plan.polymul_host(ha, hb, hc, da, db, dc, stream=stream)  # warm
    torch.cuda.synchronize(dev)
    e2e_each = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        plan.polymul_host(ha, hb, hc, da, db, dc, stream=stream)
        e2e_each.append(time.perf_counter() - t0)
    e2e_dt = replica_max(float(np.median(e2e_each)), dist)
    e2e_value = replica_value(units, 1, e2e_dt * 1e3, ws)
    e2e_range = [replica_value(units, 1, replica_max(x, dist) * 1e3, ws)
                 for x in (max(e2e_each), min(e2e_each))]

    # ---- roofline: the dominant kernel (rows, or the single fused kernel)
    if persistent:
        dom_idx, dom_name = 0, "k_persist (whole polymul, one persistent launch)"
        dom_mulmods = mulmods_per_polymul(log2n) * units
    elif log2n >= 14:
        dom_idx = 1
        # the row kernel the library picks for this batch (row_ops 0 resolved)
        row_ops = capi.pm_plan_resolve_tuning(plan.handle, npoly).row_ops
        dom_name = {2: "k_rows2<POLYMUL> (in-row stages of a and b together, Barrett pointwise, "
                       "inverse in-row stages)",
                    3: "k_rows_lat<POLYMUL> (1024 threads per row, radix-4 passes)",
                    1: "k_rows<POLYMUL> (in-row stages + Barrett pointwise)",
                    4: "k_wrows<POLYMUL> (1024-word rows: 10 in-row stages of a and b in "
                       "radix-4 passes, Barrett pointwise, 10 inverse in-row stages; row "
                       "twiddles staged in shared memory)"}[row_ops]
        dom_mulmods = rows_kernel_mulmods(log2n, 10 if row_ops == 4 else 12) * units
    else:
        dom_idx, dom_name = 0, "single-launch polymul"
        dom_mulmods = mulmods_per_polymul(log2n) * units
    dom_ms = avg_phase[dom_idx]
    achieved = dom_mulmods / (dom_ms * 1e-3)
    step_mulmod_rate = mulmods_per_polymul(log2n) * units / (elapsed_ms / args.steps * 1e-3)

    line = {
        "metric": METRIC, "value": value, "unit": "polymuls/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"N=2^{log2n} negacyclic polymul, q = largest 60-bit prime "
                               f"= 1 mod 2^{log2n + 1} ({L} limb(s)), {units} independent "
                               f"products per step, uniform coefficients",
                   "N": n, "limbs": L, "products_per_step": units,
                   "operand_bytes_per_step": units * n * 8 * 3,
                   "l2": "inputs (%.2f GiB) larger than L2, no flush" % (units * n * 16 / 2**30),
                   "parallelism": f"replicas x{ws}",
                   "algorithm": "Alg. 8 fused" if args.fused else "Eq. 2 (Alg. 6 / 4 / 7)",
                   "launch": tuning.as_dict()},
        "gpu_launches": (3 if (log2n >= 14 and not persistent) else 1) * args.steps,
        "phase_ms": {"col_fwd": avg_phase[0], "rows": avg_phase[1], "col_inv": avg_phase[2]}
        if nphase == 4 else {"single_launch": avg_phase[0]},
        "roofline": {"bound": "alu", "kernel": dom_name, "achieved": achieved / 1e12,
                     "peak": peak_mulmod / 1e12, "unit": "Tmulmod/s",
                     "frac": achieved / peak_mulmod,
                     "traffic": kernel_traffic(dom_name.split(" ")[0], log2n, units,
                                               args.fused, persistent),
                     "peak_source": "measured register-resident 60-bit Shoup mulmod rate "
                                    "(pm_measure_peaks, same process)",
                     "imad_peak_tops": peak_imad / 1e12,
                     "step_frac": step_mulmod_rate / peak_mulmod,
                     "mulmods_per_polymul": mulmods_per_polymul(log2n)},
        "e2e": {"value": e2e_value, "unit": "polymuls/s",
                "h2d_bytes_per_step": 2 * units * n * 8, "d2h_bytes_per_step": units * n * 8,
                "steps": e2e_steps, "statistic": "median step",
                "min_max": e2e_range},
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(log2n, qs, psis, seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def kernel_sources_sha1(unit: str = "pm_wide.cu") -> str:
    """Hash of the translation unit that builds the kernel (`unit` and the
    headers it includes from the source folder, recursively), with comments
    and whitespace removed, so that a comment edit, or an edit of another
    kernel or of host code, keeps a captured figure."""
    import hashlib
    import re
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2209_01290_gb300",
                        "csrc")
    seen, todo = set(), [unit]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo += re.findall(r'#include\s+"([^"]+)"', fh.read())
    h = hashlib.sha1()
    for f in sorted(seen):
        with open(os.path.join(csrc, f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", "", code, flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        code = re.sub(r"\s+", "", code)
        h.update(f.encode() + b"\0" + code.encode())
    return h.hexdigest()


def kernel_traffic(kernel: str, log2n: int, units: int, fused: bool, persistent: bool):
    """DRAM bytes (read + write) per launch of the dominant kernel, from the
    committed ncu figure in profiles/traffic.json scaled by the units this
    launch processes; None when there is no figure for this kernel and N or
    the kernel sources changed since it was captured."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "traffic.json")
    if persistent or fused or not os.path.exists(path):
        return None
    with open(path) as fh:
        table = json.load(fh)
    ent = table.get(f"{kernel} N=2^{log2n}")
    if not ent or ent.get("source_sha1") != kernel_sources_sha1():
        return None
    return ent["dram_bytes_per_unit"] * units


# ------------------------------------------------------------------ workloads
# Secondary measurements for the other configurations (one JSON line each);
# the default workload above is the headline.

def _flush_l2(buf):
    buf.add_(1)  # writes 256 MiB: larger than the 129 MB L2


def _sizes(args):
    """log2 N values of the sweep workloads (fused, word32)."""
    return [int(x) for x in args.sizes.split(",")]


def _time_each(fn, reps, stream, flush=None):
    """Device time of fn() on `stream`, one event pair per call.  The L2
    flush runs on the same stream, before the start event, so that it is
    finished (and not competing for HBM) when the timed work starts."""
    import torch
    out = []
    for _ in range(reps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def run_workload(args):
    import torch
    from paper_2209_01290_gb300 import Plan, Queue, capi, inputs
    dev = torch.cuda.current_device()
    st = torch.cuda.Stream(device=dev)
    flushbuf = torch.zeros(32 << 20, dtype=torch.int64, device=dev)
    lines = []
    if args.workload == "c1":
        n = 1 << 12
        qs, psis = capi.pm_find_params(12, 1, 60)
        plan = Plan(n, qs, psis)
        a, b = inputs.operand_pair(inputs.seed_for(0), qs, 1, n)
        da = torch.from_numpy(a.view(np.int64)).to(dev)
        db = torch.from_numpy(b.view(np.int64)).to(dev)
        dc = torch.empty_like(da)
        g = plan.graph_polymul(da, db, dc)
        for _ in range(args.warmup):
            g.launch(st)
        st.synchronize()
        lat = _time_each(lambda: g.launch(st), max(args.steps, 50), st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(1000):
            g.launch(st)
        e1.record(st)
        st.synchronize()
        lines.append({"workload": "c1: one N=2^12 product, graph-launched", "metric": "latency",
                      "p50_us": 1e3 * float(np.median(lat)), "p99_us": 1e3 * float(np.percentile(lat, 99)),
                      "back_to_back_polymuls_per_s": 1000 / (e0.elapsed_time(e1) * 1e-3)})
    elif args.workload == "c2sweep":
        for log2n in [x for x in _sizes(args) if x >= 13]:
            n = 1 << log2n
            qs, psis = capi.pm_find_params(log2n, 1, 60)
            plan = Plan(n, qs, psis)
            a, b = inputs.operand_pair(inputs.seed_for(1) + log2n, qs, 1, n)
            da = torch.from_numpy(a.view(np.int64)).to(dev)
            db = torch.from_numpy(b.view(np.int64)).to(dev)
            dc = torch.empty_like(da)
            plan.reserve(1, stream=st)
            res = {"workload": f"c2: N=2^{log2n}, single product", "N": n}
            for name, fn in [("polymul", lambda: plan.polymul(da, db, out=dc, stream=st)),
                             ("ntt_fwd", lambda: plan.ntt_fwd_(dc, stream=st)),
                             ("ntt_inv", lambda: plan.ntt_inv_(dc, stream=st))]:
                for _ in range(args.warmup):
                    fn()
                t = _time_each(fn, 30, st, flush=lambda: _flush_l2(flushbuf))
                res[name + "_us_median"] = 1e3 * float(np.median(t))
            # batched throughput (about 1 GiB of operands)
            P = max(1, (1 << 26) // n)
            A = inputs.uniform_limbs_torch(log2n, qs, P, n, device=dev)
            B = inputs.uniform_limbs_torch(log2n + 100, qs, P, n, device=dev)
            C = torch.empty_like(A)
            plan.reserve(P, stream=st)
            for _ in range(args.warmup):
                plan.polymul(A, B, out=C, stream=st)
            t = _time_each(lambda: plan.polymul(A, B, out=C, stream=st), 10, st)
            res["batched_products"] = P
            res["batched_polymuls_per_s"] = P / (float(np.median(t)) * 1e-3)
            lines.append(res)
    elif args.workload == "c3":
        log2n, L = 16, 32
        n = 1 << log2n
        qs, psis = capi.pm_find_params(log2n, L, 60)
        plan = Plan(n, qs, psis)
        A = inputs.uniform_limbs_torch(inputs.seed_for(2), qs, 1, n, device=dev)
        B = inputs.uniform_limbs_torch(inputs.seed_for(2) + 1, qs, 1, n, device=dev)
        C = torch.empty_like(A)
        res = {"workload": "c3: N=2^16, 32 RNS limbs (32 distinct 60-bit primes), one product per limb",
               "l2": "256 MiB written between iterations"}
        for vname, variant in [("split", capi.PM_VARIANT_SPLIT), ("persistent", capi.PM_VARIANT_PERSISTENT)]:
            capi.pm_plan_tune(plan.handle, variant, 4, 32, 64)  # lags: measured best on C3
            g = plan.graph_polymul(A, B, C)
            for _ in range(args.warmup):
                g.launch(st)
            t = _time_each(lambda: g.launch(st), 30, st, flush=lambda: _flush_l2(flushbuf))
            res[f"graph_{vname}_us_median"] = 1e3 * float(np.median(t))
            g.close()
        # 32 plain launches: one single-limb plan and call per limb
        single = [Plan(n, [qs[l]], [psis[l]]) for l in range(L)]
        for p1 in single:
            p1.reserve(1, stream=st)
        def per_limb():
            for l in range(L):
                single[l].polymul(A[:, l], B[:, l], out=C[:, l], stream=st)
        for _ in range(args.warmup):
            per_limb()
        t = _time_each(per_limb, 30, st, flush=lambda: _flush_l2(flushbuf))
        res["per_limb_launches_us_median"] = 1e3 * float(np.median(t))
        best = min(v for k, v in res.items() if k.startswith("graph_"))
        res["batched_speedup_vs_per_limb"] = res["per_limb_launches_us_median"] / best
        res["polymuls_per_s_batched"] = L / (best * 1e-6)
        lines.append(res)
    elif args.workload == "c4":
        shapes = inputs.uneven_shapes(inputs.seed_for(3), njobs=args.c4_jobs)
        plans, jobs = {}, []
        units = 0
        for j, sh in enumerate(shapes):
            key = (sh.log2n, sh.nlimbs)
            if key not in plans:
                q_, p_ = capi.pm_find_params(sh.log2n, sh.nlimbs, 60)
                plans[key] = Plan(1 << sh.log2n, q_, p_)
            plan = plans[key]
            a = inputs.uniform_limbs_torch(inputs.seed_for(3) + 2 * j, plan.qs, 1, 1 << sh.log2n, device=dev)
            b = inputs.uniform_limbs_torch(inputs.seed_for(3) + 2 * j + 1, plan.qs, 1, 1 << sh.log2n, device=dev)
            jobs.append((plan, a, b, torch.empty_like(a)))
            units += sh.nlimbs
        t_mode = {}
        for mname, mode in [("persistent", capi.PM_UNEVEN_PERSISTENT),
                            ("grouped", capi.PM_UNEVEN_GROUPED)]:
            q = Queue(dev, mode=mode)
            for _ in range(args.warmup):
                q.polymul_uneven(jobs, stream=st)
            q.sync(st)
            t_mode[mname] = float(np.median(_time_each(lambda: q.polymul_uneven(jobs, stream=st),
                                                       10, st)))
            q.close()
        t1 = [min(t_mode.values())]
        for plan in plans.values():
            plan.reserve(1, stream=st)
        def per_job():
            for plan, a, b, c in jobs:
                plan.polymul(a, b, out=c, stream=st)
        for _ in range(args.warmup):
            per_job()
        t2 = _time_each(per_job, 10, st)
        mm = sum(mulmods_per_polymul(sh.log2n) * sh.nlimbs for sh in shapes)
        lines.append({"workload": f"c4: {args.c4_jobs} uneven jobs, N in 2^12..2^17, 1..48 limbs",
                      "units": units, "operand_gib": sum((1 << sh.log2n) * sh.nlimbs for sh in shapes) * 8 / 2**30,
                      "persistent_one_launch_ms_median": t_mode["persistent"],
                      "grouped_launches_ms_median": t_mode["grouped"],
                      "per_job_launches_ms_median": float(np.median(t2)),
                      "best_speedup_vs_per_job": float(np.median(t2)) / float(np.median(t1)),
                      "best_polymuls_per_s": units / (float(np.median(t1)) * 1e-3),
                      "best_tmulmod_per_s": mm / (float(np.median(t1)) * 1e-3) / 1e12})
    elif args.workload == "c5":
        lines.append(run_serving(args, dev))
    elif args.workload == "reductions":
        for bits in (30, 60, 62):
            q = capi.pm_find_params(12, 1, bits)[0][0]
            r = capi.pm_reduction_rates(dev, q)
            lines.append({"workload": f"reduction study, {bits}-bit q", "q": q,
                          "unit": "G reductions/s (register-resident)",
                          **{k: round(v / 1e9, 1) for k, v in r.items()}})
    elif args.workload == "tom":
        # batched stand-alone NTTs: 2^15 transforms of 2^16 points (16 GiB)
        log2n, count = 16, args.tom_count
        n = 1 << log2n
        qs, psis = capi.pm_find_params(log2n, 1, 60)
        plan = Plan(n, qs, psis)
        X = inputs.uniform_limbs_torch(inputs.seed_for(5), qs, count, n, device=dev)
        res = {"workload": f"batched stand-alone NTT: {count} transforms of 2^{log2n} points, 60-bit q",
               "gib": count * n * 8 / 2**30}
        for name, fn in [("ntt_fwd", lambda: plan.ntt_fwd_(X, stream=st)),
                         ("ntt_inv", lambda: plan.ntt_inv_(X, stream=st))]:
            fn()
            t = _time_each(fn, 3, st)
            ms = float(np.median(t))
            res[name + "_ms"] = ms
            res[name + "_us_per_ntt"] = ms * 1e3 / count
            res[name + "_tmulmod_per_s"] = count * (n // 2) * log2n / (ms * 1e-3) / 1e12
        lines.append(res)
    elif args.workload == "fused":
        # Eq. 2 vs Algorithm 8 products, batched (~1 GiB of operands per
        # step) for N = 2^12 .. 2^17; the two plans alternate step by step
        for log2n in _sizes(args):
            n = 1 << log2n
            qs, psis = capi.pm_find_params(log2n, 1, 60)
            plans = {"eq2": Plan(n, qs, psis), "alg8": Plan(n, qs, psis, fused=True)}
            P = args.products or max(1, (1 << 26) // n)
            A = inputs.uniform_limbs_torch(log2n, qs, P, n, device=dev)
            B = inputs.uniform_limbs_torch(log2n + 100, qs, P, n, device=dev)
            C = torch.empty_like(A)
            res = {"workload": f"Eq. 2 vs Alg. 8 products, N=2^{log2n}, {P} per step", "N": n,
                   "products": P}
            times = {k: [] for k in plans}
            for p in plans.values():
                p.reserve(P, stream=st)
                for _ in range(args.warmup):
                    p.polymul(A, B, out=C, stream=st)
            for _ in range(10):
                for k, p in plans.items():
                    times[k] += _time_each(lambda: p.polymul(A, B, out=C, stream=st), 1, st)
            for k in plans:
                ms = float(np.median(times[k]))
                res[k + "_ms"] = ms
                res[k + "_polymuls_per_s"] = P / (ms * 1e-3)
            res["alg8_speedup"] = res["eq2_ms"] / res["alg8_ms"]
            lines.append(res)
    elif args.workload == "word32":
        # 30-bit primes: 32-bit words (PM_PLAN_WORD32) vs the same primes in
        # 64-bit words; batched products (~1 GiB of 64-bit operands per step)
        for log2n in _sizes(args):
            n = 1 << log2n
            qs, psis = capi.pm_find_params(log2n, 1, 30)
            P = args.products or max(1, (1 << 26) // n)
            A = inputs.uniform_limbs_torch(log2n, qs, P, n, device=dev)
            B = inputs.uniform_limbs_torch(log2n + 100, qs, P, n, device=dev)
            A32, B32 = A.to(torch.int32), B.to(torch.int32)
            C, C32 = torch.empty_like(A), torch.empty_like(A32)
            p64, p32 = Plan(n, qs, psis), Plan(n, qs, psis, word32=True)
            res = {"workload": f"30-bit primes, N=2^{log2n}, {P} products per step", "N": n,
                   "products": P, "q": qs[0]}
            for name, plan, x, y, z in [("w64", p64, A, B, C), ("w32", p32, A32, B32, C32)]:
                plan.reserve(P, stream=st)
                for _ in range(args.warmup):
                    plan.polymul(x, y, out=z, stream=st)
                t = _time_each(lambda: plan.polymul(x, y, out=z, stream=st), 10, st)
                ms = float(np.median(t))
                res[name + "_ms"] = ms
                res[name + "_polymuls_per_s"] = P / (ms * 1e-3)
                tf = _time_each(lambda: plan.ntt_fwd_(z, stream=st), 10, st)
                res[name + "_ntt_fwd_us_per_ntt"] = float(np.median(tf)) * 1e3 / P
            res["same_products"] = bool(torch.equal(C32.to(torch.int64) & 0xFFFFFFFF, C))
            res["w32_speedup"] = res["w64_ms"] / res["w32_ms"]
            lines.append(res)
    for line in lines:
        print(json.dumps(line), flush=True)
    return 0


def run_serving(args, dev):
    """Poisson request stream through the continuous-batching server."""
    import threading
    import torch
    from paper_2209_01290_gb300 import Plan, capi, inputs
    rate, seconds = args.serve_rate, args.serve_seconds
    choices, weights, max_l = (13, 15, 16), (0.3, 0.4, 0.3), 32
    reqs = inputs.poisson_requests(inputs.seed_for(4), rate, seconds, choices, weights, max_l)
    plans, pool = {}, {}
    for ln in choices:
        for L in range(1, max_l + 1):
            qs, psis = capi.pm_find_params(ln, L, 60)
            plans[(ln, L)] = Plan(1 << ln, qs, psis, device=dev)
            a = inputs.uniform_limbs_torch(ln * 100 + L, qs, 1, 1 << ln, device=dev)
            b = inputs.uniform_limbs_torch(ln * 100 + L + 50, qs, 1, 1 << ln, device=dev)
            pool[(ln, L)] = (a, b)
    torch.cuda.synchronize(dev)
    srv = capi.pm_server_create(dev, args.serve_budget_gb << 30, 0, 2)
    ids = [0] * len(reqs)
    lag = [0.0] * len(reqs)
    submitted = threading.Event()
    n_sub = [0]

    def producer():
        # submit every request whose arrival time has passed, then sleep (the
        # GIL is free for the consumer); the library stamps each submission,
        # so the latencies are measured from the actual submit time
        t0 = time.perf_counter()
        i = 0
        while i < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival_s <= now:
                r = reqs[i]
                a, b = pool[(r.log2n, r.nlimbs)]
                ids[i] = capi.pm_server_submit(srv, plans[(r.log2n, r.nlimbs)].handle,
                                               a.data_ptr(), b.data_ptr(), 1)
                lag[i] = time.perf_counter() - t0 - r.arrival_s
                i += 1
                n_sub[0] = i
            if i < len(reqs):
                time.sleep(min(1e-4, max(0.0, reqs[i].arrival_s - (time.perf_counter() - t0))))
        submitted.set()

    lat = []
    th = threading.Thread(target=producer)
    t_start = time.perf_counter()
    th.start()
    sys.setswitchinterval(1e-4)  # the two threads hand the GIL over often
    for i in range(len(reqs)):
        while n_sub[0] <= i:
            time.sleep(1e-4)
        _, l_us = capi.pm_server_wait(srv, ids[i], 600000)
        lat.append(l_us)
        capi.pm_server_release(srv, ids[i])
    t_end = time.perf_counter()
    th.join()
    st = capi.pm_server_get_stats(srv)
    capi.pm_server_destroy(srv)
    units = sum(r.nlimbs for r in reqs)
    mm = sum(mulmods_per_polymul(r.log2n) * r.nlimbs for r in reqs)
    span = t_end - t_start
    lat = np.array(lat)
    workload = (f"c5: Poisson {rate:.0f} req/s for {seconds:.0f} s, N in 2^13/2^15/2^16 "
                f"(0.3/0.4/0.3), 1..32 limbs, device-resident operands, "
                f"{args.serve_budget_gb} GB budget")
    # the headline line's shape: metric / value / unit ... config, with the
    # latency percentiles beside the throughput
    return {"metric": "serving: request latency p50/p99 and polymuls/s under Poisson arrivals",
            "value": units / span, "unit": "polymuls/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload, "rate_per_s": rate, "seconds": seconds,
                       "budget_gb": args.serve_budget_gb, "max_inflight": 2},
            "latency_us": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "workload": workload,
            "requests": len(reqs), "latency_p50_us": float(np.percentile(lat, 50)),
            "latency_p99_us": float(np.percentile(lat, 99)),
            "latency_max_us": float(lat.max()),
            "achieved_requests_per_s": len(reqs) / span, "offered_requests_per_s": rate,
            "achieved_polymuls_per_s": units / span, "achieved_tmulmod_per_s": mm / span / 1e12,
            "generator_lag_p99_us": float(np.percentile(np.array(lag), 99) * 1e6),
            "batches": st["batches"], "mean_batch": st["batched_requests"] / max(1, st["batches"]),
            "max_batch": st["max_batch"], "arena_peak_gib": st["arena_peak_bytes"] / 2**30,
            "max_batches_in_flight": st["max_inflight"],
            "max_batches_overlapping_on_device": st["max_device_overlap"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--log2n", type=int, default=16)
    ap.add_argument("--limbs", type=int, default=1)
    ap.add_argument("--batch", type=int, default=4096,
                    help="products per step (default: 4096 products of N=2^16, 6 GiB of "
                         "operands and result per step)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", default="default", choices=["default", "split", "persistent"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "c1", "c2sweep", "c3", "c4", "c5", "reductions", "tom",
                             "fused", "word32"])
    ap.add_argument("--sizes", default="12,13,14,15,16,17",
                    help="log2 N values for --workload fused / word32 / c2sweep (>= 13)")
    ap.add_argument("--products", type=int, default=0,
                    help="products per step for --workload fused / word32 (0: ~1 GiB)")
    ap.add_argument("--fused", action="store_true",
                    help="headline products by Algorithm 8 (PM_PLAN_FUSED)")
    ap.add_argument("--tom-count", type=int, default=1 << 15)
    ap.add_argument("--c4-jobs", type=int, default=512,
                    help="jobs of --workload c4 (512; fewer for a profiler capture)")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--ctas-per-sm", type=int, default=4)
    ap.add_argument("--row-ops", type=int, default=0,
                    help="launch choice with --variant split/persistent (pm_tuning.row_ops; "
                         "5: tensor-copy column tiles)")
    ap.add_argument("--lag-fwd", type=int, default=8)
    ap.add_argument("--lag-inv", type=int, default=16)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "headline":
        return run_workload(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
