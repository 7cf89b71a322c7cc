"""Benchmark of the RSKA hot path on one GB300 (or N independent replicas).

Workload (the paper's Sec. 5 recipe at scale): A 20000 x 10000 i.i.d. N(0,1)
float32 (800 MB, larger than L2), xhat with 200 N(0,1) nonzeros, b = A xhat
plus noise uniform on the sphere of radius 1% of ||A xhat||, lambda = 2,
eta = 1024, t = alpha^*(eta) (Corollary 1, uniform weights, sigma_max from
the Marchenko-Pastur edge).  One step = one solve from z = 0 for 300
iterations (one persistent kernel launch, past the noise plateau).

Metric: row-updates/s = eta * iterations / second (duplicates counted),
whole job.  Also reported: the roofline of the persistent kernel against the
measured HBM copy bandwidth, the end-to-end rate through the public API with
host buffers, a naive per-iteration PyTorch RSKA on the same GPU, time to
1e-6 relative error on the 1000 x 500 configuration, and the FP64 CPU oracle
timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, S, ETA, LAM, NOISE, ITERS = 20000, 10000, 200, 1024, 2.0, 0.01, 300
PSEED, SEED = 1001, 0
WORKLOAD = "rska_single_20000x10000_eta1024"
METRIC = "RSKA row-updates/s (20000x10000 Gaussian, eta=1024, t=alpha*)"
UNIT = "row-updates/s"


def alpha_star_mp(m, n, eta):
    s2 = (np.sqrt(m) + np.sqrt(n)) ** 2
    return float(eta / (1.0 + (eta - 1) * s2 / (m * n)))


T_STEP = alpha_star_mp(M, N, ETA)


def config_dict():
    return {"workload": WORKLOAD, "m": M, "n": N, "nnz": S, "noise": NOISE, "lambda": LAM,
            "eta": ETA, "t": round(T_STEP, 4), "iters_per_step": ITERS,
            "l2": "inputs larger than L2 (A is 800 MB; rows are sampled at random)",
            "parallelism": "replicas"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_group(world):
    """One process per GPU: a process group only for the barrier and the
    maximum over ranks of the timed region (no data-path collective)."""
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


def barrier(world):
    import torch.distributed as dist
    if world > 1 and dist.is_initialized():
        dist.barrier()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {"mrhs_tmem_kernel": ["rska_mrhs_tmem.cu", "rska_tc.cuh", "rska_device.cuh"],
                  "rska_rows_kernel": ["rska_rows.cu", "rska_device.cuh"],
                  "rska_persistent_kernel": ["rska_solve.cu", "rska_device.cuh"],
                  "unrolled_bwd_rows_kernel": ["rska_unrolled.cu", "rska_device.cuh"],
                  "rska_batched_kernel": ["rska_batched.cu", "rska_device.cuh"]}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2203_10838_gb300", "csrc")
    for fn in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, iters=ITERS):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel's source or the iterations of one launch changed since the
    counters were taken."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash(kernel) or d.get("iters_per_launch") != iters:
        return None
    return d.get("dram_bytes_per_launch")


def committed_traffic_ratio(kernel):
    """DRAM bytes per algorithmic byte of `kernel` from the committed ncu
    summary of a smaller launch of the same kernel, or None when the kernel's
    source changed since the counters were taken.  Used where the benchmark's
    own launch is too large to capture and traffic grows in proportion to the
    row updates processed."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash(kernel):
        return None
    return d.get("dram_bytes_per_algorithmic_byte")


class _NvmlClocks:
    """SM clock and clock-event reasons read through NVML (ctypes, read-only)
    every millisecond on a background thread."""

    SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL, HW_POWER_BRAKE = 0x4, 0x8, 0x20, 0x40, 0x80

    def __init__(self, index: int, bus_id):
        import ctypes
        import threading
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        rc = 1
        if bus_id:
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus_id.encode(), ctypes.byref(self.h))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        ok = self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0
        self.max_mhz = mx.value if ok else None
        self.samples = []
        self.run = True
        self.t = threading.Thread(target=self._loop, daemon=True)
        self.t.start()

    def _loop(self):
        ct = self.ct
        mhz, rs = ct.c_uint(0), ct.c_ulonglong(0)
        while self.run:
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0 and \
                    self.reasons_fn(self.h, ct.byref(rs)) == 0:
                self.samples.append((mhz.value, rs.value))
            time.sleep(0.001)

    def stop(self):
        self.run = False
        self.t.join(timeout=5)
        self.lib.nvmlShutdown()
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"],
                    "samples": 0, "source": "nvml"}
        reasons = set()
        names = [(self.HW_SLOWDOWN, "hw_slowdown"), (self.HW_THERMAL, "hw_thermal_slowdown"),
                 (self.SW_THERMAL, "sw_thermal_slowdown"), (self.SW_POWER_CAP, "sw_power_cap"),
                 (self.HW_POWER_BRAKE, "hw_power_brake_slowdown")]
        for _, r in self.samples:
            for bit, name in names:
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml, 1 ms"}


class ClockSampler:
    """Clock and throttle sampling during the timed region: NVML every
    millisecond when libnvidia-ml loads, else nvidia-smi every 20 ms."""

    def __init__(self, index: int):
        self.nv = None
        bus_id = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(index)
            bus_id = "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:
            bus_id = None
        try:
            self.nv = _NvmlClocks(index, bus_id)
            return
        except Exception:
            self.nv = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        sel = [f"--id={bus_id}"] if bus_id else [f"--id={index}"]
        try:
            self.p = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.nv is not None:
            return self.nv.stop()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows), "source": "nvidia-smi, 20 ms"}


# --------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# --------------------------------------------------------------------------
def oracle_rate(prob, seconds=10.0, max_iters=300, chunk=5):
    """Time the oracle on a bounded sample of the workload: iterations of the
    same problem from z = 0 until `seconds` have passed."""
    import oracle
    A = prob.A[:, :N]
    b = prob.b.astype(np.float64)
    t0 = time.perf_counter()
    nu = oracle.row_norms(A)
    thr, alias = oracle.alias_build(nu)
    setup_s = time.perf_counter() - t0
    z = np.zeros(N)
    done = 0
    t0 = time.perf_counter()
    while done < max_iters:
        z = oracle.rska(A, b, LAM, ETA, T_STEP, SEED, chunk, k0=done, z0=z, tables=(nu, thr, alias))
        done += chunk
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return ETA * done / el, done, el, setup_s


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from synth import gaussian_problem
    prob = gaussian_problem(M, N, S, seed=PSEED, noise=NOISE)
    per_step = []
    total_iters = 0
    for i in range(args.warmup + args.steps):
        secs = args.ref_seconds if i >= args.warmup else min(1.0, args.ref_seconds)
        rate, iters, el, _ = oracle_rate(prob, seconds=secs, max_iters=ITERS)
        if i >= args.warmup:
            per_step.append((rate, iters, el))
            total_iters += iters
    tot_time = sum(el for _, _, el in per_step)
    value = ETA * total_iters / tot_time
    sample = (f"{total_iters} iterations of the {M}x{N} eta={ETA} workload over {args.steps} "
              f"steps (~{args.ref_seconds:.0f} s each, bounded sample of the {ITERS}-iteration "
              f"step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot_time / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def naive_torch_rska(torch, A, b, tau, lam, t, eta, n):
    """Plain per-iteration PyTorch RSKA (index_select + mv + where): the
    'plain RSKA on the same GPU' comparator.  Not the product path."""
    nu = (A[:, :n].double() ** 2).sum(1).float()
    z = torch.zeros(n, device=A.device)
    for k in range(tau.shape[0]):
        x = torch.sign(z) * torch.clamp(z.abs() - lam, min=0.0)
        rows = A.index_select(0, tau[k])[:, :n]
        r = rows @ x - b.index_select(0, tau[k])
        c = (t / eta) * r / nu.index_select(0, tau[k])
        z = z - rows.t() @ c
    return z


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2203_10838_gb300 import build
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2203_10838_gb300.rska import Solver
    from synth import gaussian_problem

    prob = gaussian_problem(M, N, S, seed=PSEED + rank, noise=NOISE)
    A_host = torch.from_numpy(prob.A).pin_memory()
    b_host = torch.from_numpy(prob.b).pin_memory()
    A = A_host.to(dev)
    b = b_host.to(dev)
    stream = torch.cuda.current_stream(dev)
    sol = Solver(A, b, LAM, ETA, T_STEP, SEED, n=N, stream=stream)

    def step():
        sol.reset()
        sol.solve(ITERS)

    # warm-up
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    # timed region: per-launch events around the persistent kernel
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        sol.reset()
        ev[i][0].record(stream)
        sol.solve(ITERS)
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(bq) for a, bq in ev]
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    updates = ETA * ITERS * args.steps * world
    value = updates / (total_ms / 1000.0)

    # final accuracy of the timed solve (FP64 on the device)
    xh = torch.from_numpy(prob.xhat.astype(np.float32)).to(dev)
    rel_res, rel_err = sol.metrics(xh)

    # roofline of the dominant kernel
    hbm_peak, peak_kind = load_peaks()
    alg_bytes = ITERS * ETA * (4.0 * N + 12.0) + 8.0 * N
    avg_launch_s = statistics.mean(launch_ms) / 1000.0
    achieved = alg_bytes / avg_launch_s / 1e9
    kname = "rska_rows_kernel" if sol.query("kernel") == 2 else "rska_persistent_kernel"
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": committed_traffic(kname),
            "peak_kind": f"{peak_kind} (copy bandwidth)", "kernel": kname,
            "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1000.0,
            "grid": sol.query("grid"), "rows_resident": sol.query("rows_resident")}

    # end to end through the public API with host buffers.  One context is
    # made from the pinned host buffers before the loop (rska_setup_host: it
    # allocates the library's device copy of A once); every step then loads the
    # step's problem from pinned host memory into it (rska_load_host: H2D in
    # row chunks overlapped with the FP64 row norms and the sum of W, then the
    # alias table), solves, and reads x back to pinned host memory.
    e2e = None
    e2e_steps = 0 if args.skip_e2e else max(3, min(args.steps, 10))
    torch.cuda.synchronize(dev)
    x_host = torch.empty(N, dtype=torch.float32).pin_memory()
    if e2e_steps:
        # the two host-visible parts of a step add up to it: the load call
        # (returns once A, b and the tables are on the device) and the time
        # from the solve call to x in pinned host memory (the asynchronous
        # solve, then the copy); the device time of the solve is reported
        # beside them
        parts = {"load_with_h2d_ms": 0.0, "solve_then_d2h_ms": 0.0, "solve_device_ms": 0.0}
        inside = {"h2d_norms_w_ms": 0.0, "alias_table_ms": 0.0}
        c_first = time.perf_counter()
        s2 = Solver(A_host, b_host, LAM, ETA, T_STEP, SEED, n=N, stream=stream)
        first_setup = {"setup_ms": (time.perf_counter() - c_first) * 1000.0,
                       "alloc_ms": s2.query("setup_alloc_us") / 1000.0,
                       "h2d_norms_w_ms": s2.query("setup_norms_us") / 1000.0,
                       "alias_table_ms": s2.query("setup_alias_us") / 1000.0}
        s2.solve(ITERS)   # warm the path once
        s2.get_x()
        torch.cuda.synchronize(dev)
        e0 = time.perf_counter()
        for _ in range(e2e_steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            c_load = time.perf_counter()
            s2.load_host(A_host, b_host)
            load_s = time.perf_counter() - c_load
            inside["h2d_norms_w_ms"] += s2.query("setup_norms_us") / 1000.0
            inside["alias_table_ms"] += s2.query("setup_alias_us") / 1000.0
            c_solve = time.perf_counter()
            ev[0].record(stream)
            s2.solve(ITERS)
            ev[1].record(stream)
            xd, _ = s2.get_x()
            x_host.copy_(xd, non_blocking=True)
            torch.cuda.synchronize(dev)
            parts["load_with_h2d_ms"] += load_s * 1000.0
            parts["solve_device_ms"] += ev[0].elapsed_time(ev[1])
            parts["solve_then_d2h_ms"] += (time.perf_counter() - c_solve) * 1000.0
        e2e_s = (time.perf_counter() - e0) / e2e_steps
        s2.close()
        e2e = {"value": ETA * ITERS * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(A_host.numel() * 4 + b_host.numel() * 4),
               "d2h_bytes_per_step": int(N * 4),
               "includes": "per step: rska_load_host of A and b from pinned host memory into a "
                           "context made once by rska_setup_host (H2D in row chunks overlapped "
                           "with the FP64 row norms and the sum of W, then the alias table), "
                           f"the {ITERS}-iteration solve, D2H of x",
               "parts_ms_per_step": {k: v / e2e_steps for k, v in parts.items()},
               "load_inside_ms_per_step": {k: v / e2e_steps for k, v in inside.items()},
               "h2d_gbs_link_bound": (A_host.numel() * 4) / (inside["h2d_norms_w_ms"] / e2e_steps
                                                              / 1000.0) / 1e9,
               "first_setup": first_setup}

    # plain per-iteration PyTorch RSKA on the same GPU (comparator)
    plain = None
    if not args.skip_plain:
        K_plain = 50
        tau = sol.get_indices(0, K_plain).long()
        naive_torch_rska(torch, A, b, tau[:3], LAM, T_STEP, ETA, N)
        torch.cuda.synchronize(dev)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        naive_torch_rska(torch, A, b, tau, LAM, T_STEP, ETA, N)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        plain_rate = ETA * K_plain / (p0.elapsed_time(p1) / 1000.0)
        plain = {"value": plain_rate, "unit": UNIT, "impl": "torch index_select+mv loop",
                 "speedup_of_fused": (value / world) / plain_rate}

    # time to 1e-6 relative error on the 1000 x 500 configuration
    tta = None
    if not args.skip_tta:
        p1c = gaussian_problem(1000, 500, 25, seed=1000)
        A1 = torch.from_numpy(p1c.A).to(dev)
        b1 = torch.from_numpy(p1c.b).to(dev)
        xh1 = torch.from_numpy(p1c.xhat.astype(np.float32)).to(dev)
        t1 = alpha_star_mp(1000, 500, 10)
        with Solver(A1, b1, 1.0, 10, t1, 0, n=500, stream=stream) as s1:
            s1.solve_until(20000, 100, 1e-6, xhat=xh1)   # warm-up
            s1.reset()
            torch.cuda.synchronize(dev)
            c0 = time.perf_counter()
            iters, err = s1.solve_until(200000, 100, 1e-6, xhat=xh1)
            tt_s = time.perf_counter() - c0
            tta_kernel = {1: "rska_persistent_kernel", 2: "rska_rows_kernel",
                          3: "rska_small_kernel"}[s1.query("kernel")]
        # the roof of this configuration: A (2 MB) stays in L2, so the measured
        # L2 read bandwidth (in-repo probe over a 16 MB buffer) bounds it
        from paper_2203_10838_gb300.rska import rska_probe_l2_read
        ctas = 2 * torch.cuda.get_device_properties(dev).multi_processor_count
        pbuf = torch.ones((16 << 20) // 4, dtype=torch.float32, device=dev)
        psink = torch.zeros(ctas, dtype=torch.float32, device=dev)
        rska_probe_l2_read(pbuf, 2, ctas, psink, stream=stream)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        rska_probe_l2_read(pbuf, 8, ctas, psink, stream=stream)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        l2_gbs = ctas * 8 * pbuf.numel() * 4 / (q0.elapsed_time(q1) / 1000.0) / 1e9
        c1_bytes = float(iters) * 10 * (4 * 500 + 12)
        c1_gbs = c1_bytes / tt_s / 1e9
        tta = {"config": "1000x500, 25 nnz, lambda=1, eta=10, t=alpha*", "tol": 1e-6,
               "iterations": iters, "ms": tt_s * 1000.0, "rel_err": err,
               "check_every": 100, "kernel": tta_kernel,
               "roofline": {"bound": "l2", "achieved": c1_gbs, "peak": l2_gbs, "unit": "GB/s",
                            "frac": c1_gbs / l2_gbs,
                            "peak_kind": "measured in this run (rska_probe_l2_read, 16 MB "
                                         "buffer, L2-cached loads)",
                            "note": "row bytes of the iterations over the whole time to 1e-6 "
                                    "(FP64 checks included); latency-bound: 20 KB per iteration"}}

    # batch-size sweep of the same system (the eta axis of Sec. 5.2 at scale)
    sweep = None
    if not args.skip_sweep:
        sweep = []
        from paper_2203_10838_gb300.rska import KERNEL
        for eta_s, kern in [(e, k) for e in (1, 16, 64, 256, 1024) for k in ("rows", "column")]:
            K_s = {1: 4000, 16: 4000, 64: 2000, 256: 800, 1024: 300}[eta_s]
            with Solver(A, b, LAM, eta_s, alpha_star_mp(M, N, eta_s), SEED, n=N,
                        stream=stream) as ss:
                ss.set_option("kernel", KERNEL[kern])
                ss.solve(min(200, K_s))
                q0 = torch.cuda.Event(enable_timing=True)
                q1 = torch.cuda.Event(enable_timing=True)
                q0.record(stream)
                ss.solve(K_s)
                q1.record(stream)
                torch.cuda.synchronize(dev)
                ms = q0.elapsed_time(q1)
                us_it = 1000.0 * ms / K_s
                gbs = K_s * eta_s * (4.0 * N + 12.0) / (ms / 1000.0) / 1e9
                sweep.append({"eta": eta_s, "kernel": kern, "grid": ss.query("grid"),
                              "us_per_iter": us_it,
                              "row_updates_per_s": eta_s * K_s / (ms / 1000.0),
                              "hbm_frac": gbs / hbm_peak})

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        rate, iters, el, _ = oracle_rate(prob, seconds=args.ref_seconds, max_iters=ITERS)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{iters} iterations of this workload from z=0 ({el:.1f} s, FP64, "
                         "single thread)"}

    # the step of Corollary 1 from a power-iteration estimate of sigma_max^2
    # (outside the timed region), beside the Marchenko-Pastur value the
    # workload uses
    step = lb = None
    if not args.skip_plain:
        s2, f2, al = sol.sigma_max2(30, 0)
        step = {"t_used": T_STEP, "t_rule": "alpha*(eta) with sigma_max^2 ~ (sqrt m + sqrt n)^2",
                "power_iteration": {"iters": 30, "sigma_max2": s2, "fro2": f2, "alpha_star": al}}
        # the eta -> infinity limit: linearized Bregman, one full sweep of A per
        # iteration; per-iteration time from the difference of two runs (the
        # call is synchronous and allocates its index list), and the iteration
        # complexity factor H(eta) = 1/L(alpha^*) of the mini-batch remark
        walls = []
        for kk in (5, 15):
            torch.cuda.synchronize(dev)
            c0 = time.perf_counter()
            sol.linearized_bregman(kk, 1.0 / s2)
            walls.append(time.perf_counter() - c0)
        lb_us = (walls[1] - walls[0]) / 10 * 1e6
        srat = s2 / f2
        H = lambda e: 2.0 / e + 2.0 * (1.0 - 1.0 / e) * srat
        rska_us = total_ms / args.steps / ITERS * 1000.0
        lb = {"us_per_iter": lb_us, "rows_per_iter": M,
              "rska_us_per_iter": rska_us,
              "H": {str(e): H(e) for e in (1, 16, 64, 256, 1024)} | {"inf": 2.0 * srat},
              "predicted_time_ratio_rska_over_lb":
                  (H(ETA) * rska_us) / (2.0 * srat * lb_us) if lb_us > 0 else None}
    sol.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                # per step: fill_shrink_kernel (reset), presample_kernel, the solve kernel
                "clocks": clk, "gpu_launches": 3 * args.steps,
                "accuracy": {"rel_residual": rel_res, "rel_error": rel_err,
                             "after_iterations": ITERS},
                "plain_rska_gpu": plain, "time_to_accuracy": tta, "eta_sweep": sweep,
                "step": step, "linearized_bregman": lb}
        return line
    return None


# --------------------------------------------------------------------------
# batched workload: 4096 independent systems, each to 1e-6 relative residual
# --------------------------------------------------------------------------
BATCH_P, BATCH_ETA, BATCH_T, BATCH_LAM, BATCH_TOL, BATCH_SEED = 4096, 32, 16.0, 1.0, 1e-6, 2024
# Iteration cap per problem.  About one problem in eight of this set has a
# nonzero of xhat far below lambda; sparse Kaczmarz then stalls for a very long
# time at a relative residual of 1e-6 .. 1e-3 (the FP64 oracle shows the same
# plateau), so the step runs every problem to 1e-6 or to this cap, and the line
# reports how many reached 1e-6.
BATCH_MAX_ITERS = 20000


def run_batched(args):
    import torch

    from paper_2203_10838_gb300 import build
    from synth import batched_problem_set
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    dev = torch.device("cuda", local)
    build.build()
    from paper_2203_10838_gb300.rska import BatchSolver, Solver
    from paper_2203_10838_gb300.shard import gather_by_unit, problem_shards
    from synth import batched_sizes
    t0 = time.perf_counter()
    P_all = args.batch_p
    if args.shard:
        # one fixed problem set split across the ranks (strong scaling): this
        # rank generates and solves only its share, each problem with its
        # index stream id in the whole set
        ms_all, ns_all = batched_sizes(P_all, BATCH_SEED)
        shards = problem_shards(ms_all, ns_all, BATCH_ETA, world)
        units = shards[rank]
        A, a_off, m, n, lda, b, b_off, xhats = batched_problem_set(P_all, BATCH_SEED,
                                                                   subset=units)
    else:
        # replicas (weak scaling): every rank solves its own full problem set
        shards = None
        units = list(range(P_all))
        A, a_off, m, n, lda, b, b_off, xhats = batched_problem_set(P_all, BATCH_SEED + rank)
    P = len(units)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    Ad = torch.from_numpy(A).to(dev)
    bd = torch.from_numpy(b).to(dev)
    torch.cuda.synchronize(dev)
    h2d_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    bs = BatchSolver(Ad, bd, a_off, m, n, lda, b_off, BATCH_LAM, BATCH_ETA, BATCH_T, BATCH_SEED,
                     stream=stream)
    if args.shard:
        bs.set_stream_ids(units)
    setup_s = time.perf_counter() - t0
    # --iters K: every problem runs exactly K iterations (no stopping test)
    max_iters = args.iters if args.iters is not None else BATCH_MAX_ITERS
    tol = 0.0 if args.iters is not None else BATCH_TOL
    for _ in range(max(1, args.warmup)):
        bs.solve(max_iters, tol=tol)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    clocks = ClockSampler(local)
    ev0.record(stream)
    for _ in range(args.steps):
        bs.solve(max_iters, tol=tol)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    from paper_2203_10838_gb300.shard import max_over_ranks
    ms_step = max_over_ranks(ms_step, dev)
    iters, rr = bs.results()
    bs.close()
    # time to 1e-6 of the problems that reach it: the same problems (same
    # data, same index streams) re-run as a batch of their own
    conv = None
    if tol > 0 and not args.shard:
        sel = np.nonzero(rr <= BATCH_TOL)[0]
        if len(sel) > 0:
            with BatchSolver(Ad, bd, a_off[sel], m[sel], n[sel], lda[sel], b_off[sel], BATCH_LAM,
                             BATCH_ETA, BATCH_T, BATCH_SEED, stream=stream) as bc:
                bc.set_stream_ids(sel)
                bc.solve(max_iters, tol=tol)
                torch.cuda.synchronize(dev)
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                bc.solve(max_iters, tol=tol)
                c1.record(stream)
                torch.cuda.synchronize(dev)
                it_c, rr_c = bc.results()
            conv = {"problems": int(len(sel)), "ms": c0.elapsed_time(c1),
                    "all_reach_tol": bool((rr_c <= BATCH_TOL).all()),
                    "iterations_total": int(it_c.sum()),
                    "row_updates_per_s": float(it_c.sum()) * BATCH_ETA / (c0.elapsed_time(c1) / 1000.0),
                    "note": "the problems of the set that reach 1e-6 within the cap, re-run as one "
                            "batch with their own index streams"}
    hbm_peak, peak_kind = load_peaks()
    row_bytes = float((iters * BATCH_ETA * (4.0 * n + 12.0)).sum())
    ratio = committed_traffic_ratio("rska_batched_kernel")
    traffic = None if ratio is None else ratio * row_bytes   # this rank's launch
    achieved = row_bytes / (ms_step / 1000.0) / 1e9   # this rank's own rows
    if args.shard:
        # per-problem results of every rank (after the timed region)
        by_p = gather_by_unit(units, list(zip(iters.tolist(), rr.tolist())), world)
        iters_all = np.array([by_p[p][0] for p in range(P_all)], dtype=np.int64)
        rr_all = np.array([by_p[p][1] for p in range(P_all)])
        ms_all_, ns_all_ = batched_sizes(P_all, BATCH_SEED)
        updates = float(iters_all.sum()) * BATCH_ETA
        value = updates / (ms_step / 1000.0)
        row_bytes_all = float((iters_all * BATCH_ETA * (4.0 * ns_all_ + 12.0)).sum())
        achieved = row_bytes_all / (ms_step / 1000.0) / 1e9 / world   # per GPU
        iters, rr = iters_all, rr_all
    else:
        updates = float(iters.sum()) * BATCH_ETA
        value = updates / (ms_step / 1000.0) * world
    # per-problem comparator: the single-system solver looped over a subset
    sub = list(range(0, P, max(1, P // 32)))
    if args.shard:
        sub = []   # the sharded run reports the split, not the comparators
    t_loop = 0.0
    for p in (sub if args.mode != "kernel" else []):
        mp, np_, lp = int(m[p]), int(n[p]), int(lda[p])
        Ap = Ad[int(a_off[p]):int(a_off[p]) + mp * lp].view(mp, lp)
        bp = bd[int(b_off[p]):int(b_off[p]) + mp]
        torch.cuda.synchronize(dev)
        c0 = time.perf_counter()
        with Solver(Ap, bp, BATCH_LAM, BATCH_ETA, BATCH_T, BATCH_SEED, n=np_, stream=stream) as sp:
            sp.solve_until(max_iters, -(-mp // BATCH_ETA), tol) if tol > 0 else sp.solve(max_iters)
        t_loop += time.perf_counter() - c0
    loop_all_s = t_loop * P / len(sub) if (args.mode != "kernel" and sub) else None
    cpu = None
    if not args.skip_cpu and sub:
        # one problem per host thread: the C oracle is reentrant and ctypes
        # releases the GIL for the length of each call
        from concurrent.futures import ThreadPoolExecutor

        import oracle
        oracle.build()
        cores = min(os.cpu_count() or 1, len(sub))

        def one(p):
            mp, np_, lp = int(m[p]), int(n[p]), int(lda[p])
            Ap = A[int(a_off[p]):int(a_off[p]) + mp * lp].reshape(mp, lp)[:, :np_]
            bp = b[int(b_off[p]):int(b_off[p]) + mp].astype(np.float64)
            K = int(iters[p])
            oracle.rska(Ap, bp, BATCH_LAM, BATCH_ETA, BATCH_T, BATCH_SEED, K, problem=p)
            return K * BATCH_ETA

        c0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            done_updates = sum(ex.map(one, sub))
        el = time.perf_counter() - c0
        cpu = {"value": done_updates / el, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the {len(sub)}-problem subset (every {max(1, P // 32)}th problem), one "
                         f"problem per thread on {cores} threads, each run for the iterations "
                         f"the GPU needed: {done_updates // BATCH_ETA} iterations in {el:.1f} s"}
    line = {"metric": (f"batched RSKA: {P_all} Gaussian systems to 1e-6 relative residual"
                       if tol > 0
                       else f"batched RSKA: {P_all} Gaussian systems, {max_iters} iterations each"),
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if args.shard else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"rska_batched_{P_all}", "P": P_all,
                       "m": "log-uniform [200, 4000]", "n": "m/2 rounded to 8", "eta": BATCH_ETA,
                       "t": BATCH_T, "lambda": BATCH_LAM, "tol": tol,
                       "A_bytes_this_rank": int(A.nbytes),
                       "parallelism": "sharded" if args.shard else "replicas"},
            "partition": ({"problems_per_rank": [len(sh) for sh in shards],
                           "rule": "longest estimated work first (n^2 + m n / eta) to the least "
                                   "loaded rank", "slowest_rank_ms": ms_step}
                          if args.shard else None),
            "time_to_all_stopped_ms": ms_step,
            "converged_subset_to_tol": conv,
            "converged": int((rr <= BATCH_TOL).sum()), "max_iters": max_iters,
            "stalled_at_cap": int((rr > BATCH_TOL).sum()) if tol > 0 else None,
            "rel_residual_deciles_of_stalled": (np.quantile(rr[rr > BATCH_TOL], [0.1, 0.5, 0.9]).tolist()
                                                if tol > 0 and (rr > BATCH_TOL).any() else None),
            "iterations_total": int(iters.sum()),
            "iterations_max": int(iters.max()),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic,
                         "traffic_how": (None if ratio is None else
                                         f"{ratio:.4f} DRAM bytes per algorithmic byte from an ncu "
                                         "capture of the 256-problem launch, times this launch's "
                                         "algorithmic bytes"),
                         "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "kernel": "rska_batched_kernel",
                         "note": "row bytes of all iterations; exact residual checks not counted"},
            "plain_per_problem_gpu": None if loop_all_s is None else {"value_s_extrapolated": loop_all_s,
                                      "impl": f"single-system solver looped, {len(sub)}-problem "
                                              f"subset scaled to {P}; each problem runs "
                                              "rska_solve_until with the exact FP64 relative "
                                              "residual every ceil(m/eta) iterations, to 1e-6 or "
                                              "the same iteration cap",
                                      "speedup_of_batched": loop_all_s / (ms_step / 1000.0)},
            "prep": {"generate_s": gen_s, "h2d_s": h2d_s, "setup_s": setup_s},
            "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": args.steps}   # one rska_batched_kernel per solve
    return line if rank == 0 else None


# --------------------------------------------------------------------------
# unrolled workload: 64 problems, K = 200 iterations, forward + adjoint
# --------------------------------------------------------------------------
U_P, U_M, U_N, U_NNZ, U_K, U_ETA, U_CK, U_LAM, U_T, U_SEED = 64, 2048, 1024, 50, 200, 64, 20, 1.0, 32.0, 11


def naive_unrolled_torch(torch, A, b, lam, t, tau, inv_nu, eta):
    """Unrolled RSKA written with torch ops and differentiated by autograd:
    the comparator for the hand-written adjoint (not the product path)."""
    z = torch.zeros(A.shape[1], device=A.device)
    for k in range(tau.shape[0]):
        x = torch.sign(z) * torch.relu(z.abs() - lam)
        rows = A.index_select(0, tau[k])
        r = rows @ x - b.index_select(0, tau[k])
        z = z - (t / eta) * (rows.t() @ (r * inv_nu.index_select(0, tau[k])))
    return torch.sign(z) * torch.relu(z.abs() - lam)


def run_unrolled(args):
    import torch

    from paper_2203_10838_gb300 import build
    from synth import gaussian_problem, pack_batch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    dev = torch.device("cuda", local)
    build.build()
    from paper_2203_10838_gb300.rska import Solver, Unrolled
    probs = [gaussian_problem(U_M, U_N, U_NNZ, seed=700 + i + 1000 * rank, noise=0.01)
             for i in range(U_P)]
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    Ad = torch.from_numpy(A).to(dev)
    stream = torch.cuda.current_stream(dev)
    un = Unrolled(Ad, a_off, m, n, lda, b_off, U_ETA, U_SEED, U_K, U_CK, stream=stream)
    bd = torch.from_numpy(b).to(dev).requires_grad_(True)
    lam = torch.full((U_P,), U_LAM, device=dev, requires_grad=True)
    t = torch.full((U_P,), U_T, device=dev, requires_grad=True)
    xhat = torch.zeros(int(un.x_off[-1]), device=dev)
    for p, pr in enumerate(probs):
        xhat[int(un.x_off[p]):int(un.x_off[p]) + pr.n] = torch.from_numpy(pr.xhat.astype(np.float32))

    def step():
        bd.grad = lam.grad = t.grad = None
        x = un(bd, lam, t)
        loss = 0.5 * ((x - xhat) ** 2).sum()
        loss.backward()
        return loss

    # events on the solver's stream around each forward (b gather + forward
    # kernel) and each adjoint launch (one backward kernel) of the timed steps
    spans = {"fwd": [], "bwd": []}
    timing = [False]

    def timed(raw, key):
        def call(*xs):
            if not timing[0]:
                return raw(*xs)
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
            out = raw(*xs)
            ev[1].record(stream)
            spans[key].append(ev)
            return out
        return call

    un.forward_raw = timed(un.forward_raw, "fwd")
    un.backward_raw = timed(un.backward_raw, "bwd")

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    timing[0] = True
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    timing[0] = False
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    fwd_ms = sum(a.elapsed_time(b) for a, b in spans["fwd"]) / len(spans["fwd"])
    bwd_ms = sum(a.elapsed_time(b) for a, b in spans["bwd"]) / len(spans["bwd"])
    from paper_2203_10838_gb300.shard import max_over_ranks
    ms = max_over_ranks(ms, dev)
    fwd_ms = max_over_ranks(fwd_ms, dev)
    bwd_ms = max_over_ranks(bwd_ms, dev)
    # rows read: K forward, K - K/c recompute, K adjoint steps of eta rows each
    bwd_rows = U_P * U_ETA * ((U_K - U_K // U_CK) + U_K)
    row_reads = U_P * U_ETA * U_K + bwd_rows
    value = row_reads / (ms / 1000.0) * world
    hbm_peak, peak_kind = load_peaks()
    # the dominant kernel is the adjoint launch (recompute + adjoint steps)
    achieved = bwd_rows * (4.0 * U_N) / (bwd_ms / 1000.0) / 1e9
    fwd_gbs = U_P * U_ETA * U_K * (4.0 * U_N) / (fwd_ms / 1000.0) / 1e9
    step_gbs = row_reads * (4.0 * U_N) / (ms / 1000.0) / 1e9
    # naive torch autograd comparator on 4 problems, scaled to 64
    sub = 4 if args.mode != "kernel" else 0
    t_naive = 0.0
    for p in range(sub):
        pr = probs[p]
        Ap = torch.from_numpy(pr.A[:, :pr.n].copy()).to(dev)
        bp = torch.from_numpy(pr.b).to(dev).requires_grad_(True)
        nu = (Ap.double() ** 2).sum(1)
        inv_nu = (1.0 / nu).float()
        with Solver(torch.from_numpy(pr.A).to(dev), torch.from_numpy(pr.b).to(dev), U_LAM, U_ETA,
                    U_T, U_SEED, n=pr.n) as sp:
            tau = sp.get_indices(0, U_K).long()   # problem 0's stream; timing only
        lam1 = torch.tensor(U_LAM, device=dev, requires_grad=True)
        t1 = torch.tensor(U_T, device=dev, requires_grad=True)
        xh = torch.from_numpy(pr.xhat.astype(np.float32)).to(dev)
        torch.cuda.synchronize(dev)
        c0 = time.perf_counter()
        xk = naive_unrolled_torch(torch, Ap, bp, lam1, t1, tau, inv_nu, U_ETA)
        (0.5 * ((xk - xh) ** 2).sum()).backward()
        torch.cuda.synchronize(dev)
        t_naive += time.perf_counter() - c0
    naive_ms = 1000.0 * t_naive * U_P / sub if sub else None
    un.close()
    # the FP64 oracle (forward, then the reverse sweep over all stored z_k) on
    # one host core, problem by problem, expressed in this line's unit: the
    # row reads the GPU's checkpointed schedule makes per problem
    cpu = None
    if rank == 0 and args.mode != "kernel" and not args.skip_cpu:
        import oracle
        oracle.build()
        c0 = time.perf_counter()
        done = 0
        for p in range(U_P):
            pr = probs[p]
            Ap = np.ascontiguousarray(pr.A[:, :pr.n])
            nu = oracle.row_norms(Ap)
            thr, alias = oracle.alias_build(nu)
            tau = oracle.sample(thr, alias, seed=U_SEED, eta=U_ETA, k0=0, K=U_K, problem=p)
            oracle.unrolled_grad(Ap, pr.b.astype(np.float64), U_LAM, U_T, U_ETA, tau,
                                 pr.xhat.astype(np.float32).astype(np.float64), nu=nu)
            done += 1
            if time.perf_counter() - c0 > args.ref_seconds:
                break
        el = time.perf_counter() - c0
        cpu = {"value": row_reads / U_P * done / el, "unit": "row-reads/s", "cores": 1,
               "kind": "oracle",
               "sample": f"loss and gradient of {done} of the {U_P} problems (K = {U_K}, FP64, "
                         f"single thread, {el:.1f} s), counted in the GPU schedule's row reads "
                         f"per problem"}
    line = {"metric": "unrolled RSKA forward + adjoint (64 x 2048x1024, K=200, eta=64)",
            "value": value, "unit": "row-reads/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "rska_unrolled_64x2048x1024", "P": U_P, "m": U_M, "n": U_N,
                       "K": U_K, "eta": U_ETA, "ckpt": U_CK, "lambda": U_LAM, "t": U_T},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": committed_traffic("unrolled_bwd_rows_kernel", U_K),
                         "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "kernel": "unrolled_bwd_rows_kernel", "launch_ms": bwd_ms,
                         "algorithmic_bytes": bwd_rows * 4.0 * U_N},
            "forward": {"launch_ms": fwd_ms, "achieved_gbs": fwd_gbs,
                        "frac": fwd_gbs / hbm_peak,
                        "kernels": "unrolled_gather_b_kernel + unrolled_fwd_rows_kernel"},
            "step_row_bytes_gbs": step_gbs,
            "naive_torch_autograd_ms_extrapolated": naive_ms,
            "speedup_vs_naive_autograd": naive_ms / ms if naive_ms else None,
            "cpu_baseline": cpu, "clocks": clk,
            # per step: unrolled_gather_b_kernel, unrolled_fwd_rows_kernel, unrolled_bwd_rows_kernel
            "gpu_launches": 3 * args.steps}
    return line if rank == 0 else None


# --------------------------------------------------------------------------
# shared-A multi-RHS workload on the tensor cores
# --------------------------------------------------------------------------
MR_M, MR_N, MR_R, MR_S, MR_ETA, MR_T, MR_LAM, MR_K, MR_PSEED, MR_SEED = (
    16384, 8192, 512, 400, 256, 128.0, 1.0, 128, 1, 0)


def run_mrhs(args):
    import torch

    from paper_2203_10838_gb300 import build
    from synth import multi_rhs_problem
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_group(world)
    dev = torch.device("cuda", local)
    build.build()
    from paper_2203_10838_gb300.rska import MultiRHS, Solver
    from paper_2203_10838_gb300.shard import gather_by_unit, rhs_shards
    t0 = time.perf_counter()
    if args.shard:
        # one A with R right-hand sides split across the ranks (strong
        # scaling): A is replicated, each rank takes a contiguous block of
        # right-hand sides, every rank draws the same tau from the same seed
        p = multi_rhs_problem(MR_M, MR_N, MR_R, MR_S, seed=MR_PSEED)
        r0, r1 = rhs_shards(MR_R, world)[rank]
    else:
        p = multi_rhs_problem(MR_M, MR_N, MR_R, MR_S, seed=MR_PSEED + rank)
        r0, r1 = 0, MR_R
    R_loc = r1 - r0
    gen_s = time.perf_counter() - t0
    A16_host = torch.from_numpy(p.A16.view(np.int16)).pin_memory()
    B_host = torch.from_numpy(np.ascontiguousarray(p.B[r0:r1])).pin_memory()
    A = A16_host.to(dev).view(torch.bfloat16)
    B = B_host.to(dev)
    stream = torch.cuda.current_stream(dev)
    h = MultiRHS(A, B, MR_LAM, MR_ETA, MR_T, MR_SEED, n=MR_N, stream=stream)
    if args.mrhs_form != "auto":
        from paper_2203_10838_gb300.rska import MRHS_FORM
        h.set_option("form", MRHS_FORM[args.mrhs_form])
    form = h.query("form")

    def step():
        h.reset()
        h.solve(MR_K)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    form = h.query("form")   # the schedule the timed steps ran (the autotuner may have picked it)
    ms = e0.elapsed_time(e1) / args.steps
    from paper_2203_10838_gb300.shard import max_over_ranks
    ms = max_over_ranks(ms, dev)
    updates = MR_ETA * R_loc * MR_K   # this rank's row-updates per step
    # whole job: sharded ranks split the 512 right-hand sides, replicas each run all of them
    value = (MR_ETA * MR_R * MR_K if args.shard else updates * world) / (ms / 1000.0)
    flops = 4.0 * MR_ETA * MR_N * R_loc * MR_K   # the two products, multiply-add = 2 flops
    achieved = flops / (ms / 1000.0) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    if args.mode == "kernel":
        h.close()
        return ({"metric": "shared-A multi-RHS RSKA (kernel-only run for profiling)",
                 "ms_per_step": ms, "iters_per_step": MR_K, "tflops": achieved}
                if rank == 0 else None)
    # accuracy of the timed solve: relative residual and error per right-hand side (FP64)
    x, _ = h.get_x()
    A64 = A.double()
    B64 = torch.from_numpy(np.ascontiguousarray(p.B64[r0:r1])).to(dev)
    res = (x.double() @ A64[:, :MR_N].t()) - B64
    rr = (res.norm(dim=1) / B64.norm(dim=1)).cpu().numpy()
    xh = torch.from_numpy(np.ascontiguousarray(p.Xhat[r0:r1])).to(dev)
    re = ((x.double() - xh).norm(dim=1) / xh.norm(dim=1)).cpu().numpy()
    del A64, res, B64
    if args.shard:
        by_j = gather_by_unit(range(r0, r1), list(zip(rr.tolist(), re.tolist())), world)
        rr = np.array([by_j[j][0] for j in range(MR_R)])
        re = np.array([by_j[j][1] for j in range(MR_R)])
    terms = h.query("terms")
    terms_update = h.query("terms_update")
    ksplit = h.query("ksplit")
    from paper_2203_10838_gb300.rska import decode_schedule
    tuned_code = h.query("tuned_code")
    schedule = {"chosen_by": "autotuner (rska_mrhs_tune, first long solve)" if tuned_code else
                "pinned by --mrhs-form",
                **decode_schedule(tuned_code if tuned_code else
                                  (2 | (h.query("gather_sched") << 17) if form == 2 else
                                   1 | (h.query("ksplit_used") << 8) | (h.query("pdl") << 16))),
                "tuned_us_per_iter": h.query("tuned_ns") / 1000.0 if tuned_code else None}
    # end to end through the public API: H2D of A and B, setup, K iterations, D2H of X
    torch.cuda.synchronize(dev)
    c0 = time.perf_counter()
    A_e = A16_host.to(dev, non_blocking=True).view(torch.bfloat16)
    B_e = B_host.to(dev, non_blocking=True)
    with MultiRHS(A_e, B_e, MR_LAM, MR_ETA, MR_T, MR_SEED, n=MR_N, stream=stream) as he:
        he.set_option("form", form)
        he.solve(MR_K)
        xe = he.get_x()[0].cpu()
    e2e_s = time.perf_counter() - c0
    del A_e, B_e
    # comparator: the single-system GPU solver looped over right-hand sides
    A32 = torch.from_numpy(p.A).to(dev)
    sub = 4
    torch.cuda.synchronize(dev)
    c0 = time.perf_counter()
    for j in range(sub):
        with Solver(A32, B[j].contiguous(), MR_LAM, MR_ETA, MR_T, MR_SEED, n=MR_N,
                    stream=stream) as sp:
            sp.solve(MR_K)
            sp.get_x()
    torch.cuda.synchronize(dev)
    loop_s = (time.perf_counter() - c0) * MR_R / sub
    del A32
    h.close()
    cpu = None
    if not args.skip_cpu:
        import oracle
        oracle.build()
        A_np = np.ascontiguousarray(p.A[:, :MR_N])
        nu = oracle.row_norms(A_np)
        thr, alias = oracle.alias_build(nu)
        Kc = 8
        tau = oracle.sample(thr, alias, seed=MR_SEED, eta=MR_ETA, k0=0, K=Kc)
        c0 = time.perf_counter()
        done = 0
        for j in range(MR_R):
            oracle.rska_fixed(A_np, p.B[j].astype(np.float64), MR_LAM, MR_T, MR_ETA, tau, nu=nu)
            done += 1
            if time.perf_counter() - c0 > args.ref_seconds:
                break
        el = time.perf_counter() - c0
        cpu = {"value": done * Kc * MR_ETA / el, "unit": "row-updates/s", "cores": 1,
               "kind": "oracle",
               "sample": f"{Kc} iterations on each of the first {done} right-hand sides "
                         f"({el:.1f} s, FP64, single thread)"}
    line = {"metric": "shared-A multi-RHS RSKA row-updates/s (16384x8192 BF16 A, 512 RHS, "
                      "eta=256)",
            "value": value, "unit": "row-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
            "dtype": "bf16 operands, f32 accumulate", "data": "synthetic",
            "config": {"workload": "rska_mrhs_16384x8192_R512", "m": MR_M, "n": MR_N, "R": MR_R,
                       "nnz": MR_S, "eta": MR_ETA, "t": MR_T, "lambda": MR_LAM,
                       "iters_per_step": MR_K, "terms": terms, "terms_update": terms_update,
                       "form": {1: "staged", 2: "persistent"}[form],
                       "schedule": schedule,
                       "ksplit": ksplit if form == 1 else None,
                       "l2": "A is 256 MB (> L2); rows of A are sampled at random",
                       "parallelism": "sharded" if args.shard else "replicas"},
            "partition": ({"rhs_per_rank": [b - a for a, b in rhs_shards(MR_R, world)],
                           "rule": "contiguous blocks of right-hand sides; A replicated, one "
                                   "index stream", "slowest_rank_ms": ms}
                          if args.shard else None),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": (committed_traffic("mrhs_tmem_kernel", MR_K)
                                     if form == 2 else None),
                         "peak_kind": "measured cuBLAS bf16, sustained",
                         "kernel": ("mrhs_tmem_kernel (one persistent launch per step; the "
                                    "step's time includes the index draw before it)"
                                    if form == 2 else
                                    "whole iteration (gather, residual GEMM, scale, update GEMM)"),
                         "flops_per_iteration": 4.0 * MR_ETA * MR_N * MR_R,
                         "executed_mma_flops_factor": (terms + terms_update) / 2.0,
                         # the other roof: DRAM bytes of a launch (committed ncu
                         # figure) over the step time, against the HBM copy peak
                         "hbm": (None if form != 2 or committed_traffic("mrhs_tmem_kernel", MR_K) is None
                                 else {"gbs": committed_traffic("mrhs_tmem_kernel", MR_K) / (ms / 1000.0) / 1e9,
                                       "frac": committed_traffic("mrhs_tmem_kernel", MR_K) / (ms / 1000.0)
                                       / 1e9 / load_peaks()[0],
                                       "binds": "tensor pipe (Z^T stays in tensor memory; DRAM carries "
                                                "only the sampled rows of A)"})},
            "accuracy": {"rel_residual_median": float(np.median(rr)),
                         "rel_residual_max": float(rr.max()),
                         "rel_error_median": float(np.median(re)),
                         "after_iterations": MR_K},
            "e2e": {"value": updates / e2e_s, "unit": "row-updates/s",
                    "h2d_bytes_per_step": int(p.A16.nbytes + B_host.numel() * 4),
                    "d2h_bytes_per_step": int(xe.numel() * 4),
                    "includes": "H2D of A (BF16) and B, setup (FP64 norms + alias table), "
                                "K iterations, D2H of X"},
            "plain_per_rhs_gpu": {"value_s_extrapolated": loop_s,
                                  "impl": "single-system solver (FP32 copy of the BF16 A) looped "
                                          "over 4 right-hand sides, scaled to 512",
                                  "speedup_of_mrhs": loop_s / (ms / 1000.0)},
            # per step: the index draw and one persistent kernel, or per
            # iteration gather, two products and the scale kernel (+ the draw
            # and the output kernel per step)
            "gpu_launches": (2 * args.steps if form == 2 else 4 * MR_K * args.steps + 2 * args.steps),
            "prep": {"generate_s": gen_s},
            "cpu_baseline": cpu, "clocks": clk}
    return line if rank == 0 else None


# --------------------------------------------------------------------------
# time to the noise plateau on the 20000 x 10000 system, eta x t sweep
# --------------------------------------------------------------------------
PLATEAU_ROW_UPDATES = 2_000_000   # per (eta, t) run: 100 checks of m row-updates each
PLATEAU_ETAS = (1, 16, 64, 256, 1024)


def plateau_of(errs):
    """(plateau, reached) of one error curve: the median of its last quarter
    of checks, reached when it and the previous quarter's median are within
    5% of each other (the curve has flattened; a rising curve is not) and it
    is at most half the first check's error (a curve that never moved, as
    with a step far too small for its eta, has no plateau yet)."""
    e = np.asarray(errs, dtype=np.float64)
    q = max(1, len(e) // 4)
    last, prev = np.median(e[-q:]), np.median(e[-2 * q:-q])
    flat = np.isfinite(last) and np.isfinite(prev) and prev <= 1.05 * last and last <= 1.05 * prev
    return float(last), bool(flat and last <= 0.5 * e[0])


def run_plateau(args):
    """With 1% noise the error of RSKA levels off at a horizon set by the noise
    (Sec. 4, the noisy-data theorem) instead of reaching 1e-6, so on the
    20000 x 10000 system the time-to-accuracy measure is the time to reach
    1.05x the plateau of each run.  Sweep: eta in {1, 16, 64, 256, 1024}, t in
    {1, alpha*(eta), eta} (Corollary 1 with sigma_max^2 from the power
    iteration); the same budget of row-updates per run, checked every
    ceil(m/eta) iterations (one check costs one pass over A, about what m/eta
    iterations read).  Solve time is timed with CUDA events around each solve
    chunk on the solver's stream (checks excluded, their count reported)."""
    import torch

    from paper_2203_10838_gb300 import build
    from synth import gaussian_problem
    rank, world, local = dist_env()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    from paper_2203_10838_gb300.rska import Solver
    prob = gaussian_problem(M, N, S, seed=PSEED, noise=NOISE)
    A = torch.from_numpy(prob.A).to(dev)
    b = torch.from_numpy(prob.b).to(dev)
    xh = torch.from_numpy(prob.xhat.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    with Solver(A, b, LAM, 1, 1.0, SEED, n=N, stream=stream) as probe:
        s2, f2, _ = probe.sigma_max2(30, 0)
    clocks = ClockSampler(local)
    runs = []
    for eta in PLATEAU_ETAS:
        a_star = eta / (1.0 + (eta - 1) * s2 / f2)
        ts = sorted({1.0, a_star, float(eta)})
        C = -(-M // eta)
        n_chunks = max(1, PLATEAU_ROW_UPDATES // (C * eta))
        for t in ts:
            with Solver(A, b, LAM, eta, t, SEED, n=N, stream=stream) as sol:
                sol.solve(min(C, 50))        # warm-up, then start over
                sol.reset()
                ms_chunks, errs, res = [], [], []
                for _ in range(n_chunks):
                    ev = (torch.cuda.Event(enable_timing=True),
                          torch.cuda.Event(enable_timing=True))
                    ev[0].record(stream)
                    sol.solve(C)
                    ev[1].record(stream)
                    rr, re = sol.metrics(xh)    # synchronises
                    ms_chunks.append(ev[0].elapsed_time(ev[1]))
                    errs.append(re)
                    res.append(rr)
            plat, reached = plateau_of(errs)
            first = next((j for j, e in enumerate(errs) if e <= 1.05 * plat), None)
            cum = np.cumsum(ms_chunks)
            runs.append({"eta": eta, "t": t,
                         "t_kind": "alpha*" if t == a_star else ("1" if t == 1.0 else "eta"),
                         "check_every": C, "checks": n_chunks,
                         "us_per_iter": float(cum[-1] / (C * n_chunks) * 1000.0),
                         "final_rel_err": errs[-1], "final_rel_res": res[-1],
                         "plateau_rel_err": plat, "plateau_reached": reached,
                         "iters_to_plateau": (first + 1) * C if reached else None,
                         "ms_to_plateau": float(cum[first]) if reached else None,
                         "_errs": errs, "_cum": cum.tolist()})
    clk = clocks.stop()
    # a common target: 1.05x the lowest plateau any run reached
    best = min((r["plateau_rel_err"] for r in runs if r["plateau_reached"]), default=None)
    for r in runs:
        j = (next((j for j, e in enumerate(r["_errs"]) if e <= 1.05 * best), None)
             if best is not None else None)
        r["iters_to_common_target"] = (j + 1) * r["check_every"] if j is not None else None
        r["ms_to_common_target"] = r["_cum"][j] if j is not None else None
        del r["_errs"], r["_cum"]
    head = next(r for r in runs if r["eta"] == ETA and r["t_kind"] == "alpha*")
    line = {"metric": f"time to the noise plateau ({M}x{N}, 1% noise, eta={ETA}, t=alpha*)",
            "value": head["ms_to_plateau"], "unit": "ms", "n_gpus": 1, "steps": 1,
            "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rska_plateau_{M}x{N}", "m": M, "n": N, "nnz": S,
                       "lambda": LAM, "noise": NOISE, "row_updates_per_run": PLATEAU_ROW_UPDATES,
                       "sigma_max2": s2, "fro2": f2,
                       "plateau_rule": "median of the last quarter of checks, reached when "
                                       "within 5% of the previous quarter's; time to the first "
                                       "check at or below 1.05x it"},
            "common_target_rel_err": 1.05 * best if best is not None else None,
            "sweep": runs, "clocks": clk,
            # per timed solve chunk: the pre-sampler and the solve kernel (each
            # chunk of ceil(m/eta) iterations fits one pre-sample of 2^21 draws)
            "gpu_launches": 2 * sum(r["checks"] for r in runs)}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-tta", action="store_true")
    ap.add_argument("--skip-sweep", action="store_true")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "unrolled", "mrhs", "plateau"])
    ap.add_argument("--mode", default="full", choices=["full", "kernel"],
                    help="kernel: only the timed persistent-kernel steps (for profiling)")
    ap.add_argument("--batch-p", type=int, default=BATCH_P,
                    help="batched workload: number of problems (default 4096)")
    ap.add_argument("--shard", action="store_true",
                    help="batched / mrhs: split one problem set (one set of right-hand sides) "
                         "across the ranks instead of running a replica per rank")
    ap.add_argument("--mrhs-form", default="auto", choices=["auto", "staged", "persistent"],
                    help="mrhs: the form of the iteration (default: the library's choice)")
    ap.add_argument("--no-forms", action="store_true",
                    help="single workload: leave out the batched, unrolled and multi-RHS keys")
    ap.add_argument("--iters", type=int, default=None,
                    help="iterations per step (default 300; profiling uses fewer)")
    args = ap.parse_args()
    global ITERS
    if args.iters is not None:
        ITERS = args.iters
    if args.mode == "kernel":
        args.skip_cpu = args.skip_plain = args.skip_tta = args.skip_e2e = True
        args.skip_sweep = True
    else:
        args.skip_e2e = False
    if args.impl == "reference":
        return run_reference(args)
    runners = {"single": run_gpu, "batched": run_batched, "unrolled": run_unrolled,
               "mrhs": run_mrhs, "plateau": run_plateau}
    line = runners[args.workload](args)
    _, world, _ = dist_env()
    if (line is not None and args.workload == "single" and args.mode == "full"
            and not args.no_forms and world == 1):
        # the other forms of the path, each in its own timed region with its
        # own clocks, at their full per-problem sizes
        line.update(run_other_forms(args))
    if line is not None:
        print(json.dumps(line), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
    return 0


def run_other_forms(args):
    """The batched (4096 systems to 1e-6), unrolled (64 x 2048 x 1024 forward +
    adjoint) and shared-A multi-RHS (16384 x 8192, 512 right-hand sides)
    workloads, each with a few timed steps, returned as extra keys of the
    single-system line.  Device memory is released between them."""
    import copy

    import torch
    out = {}
    plan = [("batched", run_batched, 2, 1), ("unrolled", run_unrolled, 10, 3),
            ("mrhs", run_mrhs, 5, 3)]
    for key, fn, steps, warmup in plan:
        sub = copy.copy(args)
        sub.steps, sub.warmup, sub.workload, sub.shard, sub.iters = steps, warmup, key, False, None
        sub.batch_p = BATCH_P
        t0 = time.perf_counter()
        res = fn(sub)
        if res is not None:
            res["wall_s"] = time.perf_counter() - t0
        out[key] = res
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    sys.exit(main())
