"""Benchmark: full-definition reconstruction of the 32-qubit chain workload
(approximate QFT with controlled phases up to qubit distance 4 and Ry input
angles, cut into 4 subcircuits of 11 qubits by K = 12 wire cuts, 4 per
boundary) on GB300: 2^32 float32 probabilities (16 GiB) per step.

One step = attribution of the four subcircuits' variant tensors (float64,
resident in HBM) + the pairwise contraction chain of Eq. 1 on the
split-precision tensor-core path (FP16 hi/lo operands, three products, every
cut term evaluated), with the FP64 total.  The 16 GiB output is larger than
L2, so no flush is needed between steps.  The line carries the total
variation against the FP64 oracle on 2^20 sampled outputs of the timed
result.

With N > 1 ranks (torchrun), one reconstruction is split by rows of its last
contraction (the high output bits): each rank writes its 1/N of the output,
with no data exchange; the FP64 totals are summed over the ranks.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
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

METRIC = "reconstructed probs/sec (FD) and DD bins/sec at 1 GB300, TV<=1e-6; % of roofline"
WORKLOAD = ("fd_chain_aqft32: 32-qubit AQFT (controlled phases to qubit distance 4, input Ry), 4 subcircuits "
            "of 11 qubits in a chain, K=12 (4 cuts per boundary) -> 2^32 probabilities, every cut term")
TWO_SUB_WORKLOAD = ("fd_two_sub_supremacy30_bridged: 5x6 supremacy-family depth 10 with the couplers across "
                    "one split bridged, K=4, subcircuits 17+17 -> 2^30 probabilities")


_T0 = time.perf_counter()


def _log(msg):
    """Progress line on stderr (elapsed seconds, peak host RSS)."""
    import resource
    rss = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1024
    print(f"[bench {time.perf_counter() - _T0:7.1f}s rss {rss:7.0f} MB] {msg}", file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], bf16_tflops=d["bf16_tflops"],
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained", d["bf16_tflops"]), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback")


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, clock
    event reasons, power).  Nothing here changes a GPU setting."""
    SM = 1
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
        except Exception:
            uuid = None
        ok = False
        if uuid:
            u = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            ok = self.lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(self.h)) == 0
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device_index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        self.sm_max = float(v.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(v)) == 0 \
            else None

    def sample(self):
        c = self.c
        mhz, mw, r = c.c_uint(), c.c_uint(), c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, c.byref(mhz)) != 0:
            return None
        self.reasons_fn(self.h, c.byref(r))
        self.lib.nvmlDeviceGetPowerUsage(self.h, c.byref(mw))
        return float(mhz.value), int(r.value), mw.value / 1000.0


class ClockSampler:
    """SM clock and clock event reasons sampled DURING the timed region: a
    thread polls NVML (read-only, through ctypes) every millisecond, so even
    a region of a few tens of milliseconds gets samples; without NVML,
    nvidia-smi every 200 ms (which may see none in a short region)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_s=0.001):
        self.index = index
        self.period = period_s
        self.proc = None
        self.nvml = None
        self.samples = []
        self.path = os.path.join(tempfile.gettempdir(), f"cutqc_clocks_{os.getpid()}.csv")
        try:
            self.nvml = _Nvml(index)
        except Exception:
            self.nvml = None

    def _poll(self):
        while not self._stop.is_set():
            s = self.nvml.sample()
            if s is not None:
                self.samples.append(s)
            self._stop.wait(self.period)

    def __enter__(self):
        if self.nvml is not None:
            import threading
            self._stop = threading.Event()
            self.samples = []
            first = self.nvml.sample()
            if first is not None:
                self.samples.append(first)
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
            return self
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.nvml is not None:
            self._stop.set()
            self._thread.join(timeout=5)
            last = self.nvml.sample()
            if last is not None:
                self.samples.append(last)
            return
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.nvml is not None:
            if not self.samples:
                return {"sm_mhz": None, "sm_max_mhz": self.nvml.sm_max, "reasons": ["unsampled"]}
            reasons = set()
            for _, r, _ in self.samples:
                for bit, nm in _Nvml.REASONS.items():
                    if r & bit:
                        reasons.add(nm)
            return {"sm_mhz": statistics.median(s[0] for s in self.samples), "sm_max_mhz": self.nvml.sm_max,
                    "sm_min_mhz": min(s[0] for s in self.samples), "reasons": sorted(reasons),
                    "power_w_max": max(s[2] for s in self.samples), "samples": len(self.samples),
                    "source": "nvml, 1 ms"}
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 200 ms"}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)    # the rank's GPU current before NCCL binds to it
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    from paper_2205_05836_gb300.shard import max_over_ranks as mor
    return mor(x)


def profiled_traffic(kernel_src, summary):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, summary)).read()
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()
    except OSError:
        return None
    m = re.search(r"sha256: ([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    if not m or not t or m.group(1) != sha:
        return None
    return int(t.group(1))


class ChainOracle:
    """FP64 oracle data for the 32-qubit chain, computed once: attribution of
    the four subcircuits, then the edges inside the pairs (C0, C1) and (C2,
    C3) summed for all their outputs (oracle.fd.contract_pair); an output is
    then Eq. 1 over the four edges between the pairs (oracle.fd.entries).
    Timings of each part are kept for the CPU baseline."""

    def __init__(self, w):
        from oracle import attribution, fd
        self.w = w
        subs = w.subcircuits
        var = w.variants()
        t0 = time.perf_counter()
        self.A = [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
                  for s, v in zip(subs, var)]
        t1 = time.perf_counter()
        self.L, self.eL = fd.contract_pair(self.A[0], subs[0].edges, self.A[1], subs[1].edges)
        self.R, self.eR = fd.contract_pair(self.A[2], subs[2].edges, self.A[3], subs[3].edges)
        t2 = time.perf_counter()
        self.t_attr, self.t_pairs = t1 - t0, t2 - t1

    def entries(self, idx, order_kron=True):
        from oracle import fd
        subs = self.w.subcircuits
        parts = fd.split_kron_index(idx, [s.o for s in subs]) if order_kron else \
            fd.split_original_index(idx, [s.out_qubit for s in subs])
        pairs = [(parts[0] << subs[1].o) | parts[1], (parts[2] << subs[3].o) | parts[3]]
        return fd.entries([self.L, self.R], [self.eL, self.eR], self.w.K, pairs)


def cpu_baseline(oracle, budget_s=15.0, chunk=1 << 16):
    """The FP64 oracle as it stands on the host cores for the whole-job rate:
    attribution and the two pair sums (full, prorated over the 2^32 outputs)
    plus Eq. 1 at contiguous outputs until the budget is spent."""
    n_total = 2 ** oracle.w.n
    done, t_rec = 0, 0.0
    while t_rec < budget_s and done < n_total:
        idx = np.arange(done, min(done + chunk, n_total), dtype=np.int64)
        t1 = time.perf_counter()
        oracle.entries(idx)
        t_rec += time.perf_counter() - t1
        done += len(idx)
    t_setup = oracle.t_attr + oracle.t_pairs
    t = t_rec + t_setup * done / n_total
    return dict(value=done / t, unit="probs/s", cores=_threads(), kind="oracle",
                sample=f"FP64 oracle on the 32-qubit chain: attribution of the four subcircuits and the edge sums "
                       f"inside the pairs (C0,C1), (C2,C3) (full, {t_setup:.1f} s, prorated over 2^32 outputs) + "
                       f"Eq. 1 over the 4 middle edges at the first {done} outputs in Kronecker order "
                       f"({t_rec:.1f} s)")


def _threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count()


def chain_config(w, ws=1, r0=0, r1=None):
    """The bench line's `config` for the 32-qubit chain, the same dict in
    both arms: the workload and its shape (the last contraction: rows of the
    first subcircuit pair, columns of the second, cut terms between them),
    how L2 is handled between steps, and the parallelism."""
    subs = w.subcircuits
    half = len(subs) // 2
    edges_lo = {e for s in subs[:half] for e in s.edges}
    edges_hi = {e for s in subs[half:] for e in s.edges}
    rows = 1 << sum(s.o for s in subs[:half])
    cols = 1 << sum(s.o for s in subs[half:])
    r1 = rows if r1 is None else r1
    return {"workload": WORKLOAD, "n_qubits": w.n, "cuts": w.K,
            "subcircuit_widths": [s.w for s in subs], "subcircuit_outputs": [s.o for s in subs],
            "last_contraction": [rows, cols, 4 ** len(edges_lo & edges_hi)],
            "l2": "output 16 GiB > L2 each step; no flush",
            "parallelism": f"{ws} rank(s), each writing rows [{r0}, {r1}) of the last contraction"
                           if ws > 1 else "one GPU"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same workload and
    metric; each step a bounded sample of Eq. 1 at contiguous outputs (the
    attribution and pair sums, done once, are prorated into every step)."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    from workloads.configs import fd_chain
    w = fd_chain()
    oracle = ChainOracle(w)
    budget = max(0.5, args.ref_budget / max(1, args.steps))
    for _ in range(args.warmup):
        cpu_baseline(oracle, budget_s=min(0.5, budget))
    vals, step_s = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        vals.append(cpu_baseline(oracle, budget_s=budget))
        step_s.append(time.perf_counter() - t0)
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "probs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.median(step_s) * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": chain_config(w),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "probs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "full_job_s_at_this_rate": 2 ** w.n / v,
            "note": "each timed step is a bounded sample of the job (ms_per_step is its wall time); value is the "
                    "whole-job rate of the samples, the attribution and pair sums prorated"}
    print(json.dumps(line), flush=True)


def _graph(fn, stream, warmup):
    """Warm fn up on a side stream, then capture it into a CUDA graph."""
    import torch
    side = torch.cuda.Stream(stream.device)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(warmup):
            fn()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def _time_graph(g, stream, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run(args):
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc as cq
    from paper_2205_05836_gb300.shard import row_range
    from workloads.configs import fd_chain
    _log("library built")
    w = fd_chain()
    subs = w.subcircuits
    var_host = w.variants()
    _log("variants simulated")
    var = [torch.from_numpy(v).to(dev) for v in var_host]
    att = [torch.empty((1 << s.o, 4 ** (len(s.in_local) + len(s.out_local))), dtype=torch.float32, device=dev)
           for s in subs]
    att_ws = [torch.empty(max(1, cq.cutqc_attribute_workspace_size(s)), dtype=torch.uint8, device=dev) for s in subs]
    rows, cols = cq.cutqc_fd_shape(subs)
    r0, r1 = row_range(rows, ws, rank)
    n_all = 1 << w.n
    n_out = (r1 - r0) * cols
    out = torch.empty(max(1, n_out), dtype=torch.float32, device=dev)
    prec = {"tc": cq.PREC_FP16X3_TC, "tc_prune": cq.PREC_FP16X3_TC_PRUNE, "simt": cq.PREC_FP32_SIMT}[args.precision]
    fd_ws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, prec)), dtype=torch.uint8, device=dev)
    total = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    att_side = [torch.cuda.Stream(dev) for _ in range(2)]

    def attribute_all(outs=att):
        # the subcircuits' attributions are independent: the two middle ones
        # (the large variant tensors) go to two side streams of their own,
        # the end ones stay on the caller's stream; all joined before FD
        cur = torch.cuda.current_stream(dev)
        fork = torch.cuda.Event()
        fork.record(cur)
        joins = []
        for i, side in zip((1, 2), att_side):
            side.wait_event(fork)
            with torch.cuda.stream(side):
                cq.cutqc_attribute(subs[i], var[i], out=outs[i], ws=att_ws[i])
            ev = torch.cuda.Event()
            ev.record(side)
            joins.append(ev)
        for i in (0, 3):
            cq.cutqc_attribute(subs[i], var[i], out=outs[i], ws=att_ws[i])
        for ev in joins:
            cur.wait_event(ev)

    def reconstruct(dst=out, tot=total, events=None):
        tot.zero_()
        if n_out > 0:
            cq.cutqc_reconstruct_fd(subs, att, cq.ORDER_KRON, prec, row_begin=r0, row_end=r1, out=dst,
                                    sum_out=tot, ws=fd_ws, input_events=events)

    def attribute_and_reconstruct(dst=out, tot=total):
        # each pair's subcircuits attributed on a side stream of its own (C2
        # and C3, then C1 and C0); the reconstruction, issued at once, starts
        # each contraction when its own inputs are written
        # (cutqc_fd_input_events) instead of after all four
        cur = torch.cuda.current_stream(dev)
        fork = torch.cuda.Event()
        fork.record(cur)
        sa, sb = att_side
        sa.wait_event(fork)
        sb.wait_event(fork)
        ev = [torch.cuda.Event() for _ in subs]
        with torch.cuda.stream(sa):
            for i in (2, 3):
                cq.cutqc_attribute(subs[i], var[i], out=att[i], ws=att_ws[i])
                ev[i].record(sa)
        with torch.cuda.stream(sb):
            for i in (1, 0):
                cq.cutqc_attribute(subs[i], var[i], out=att[i], ws=att_ws[i])
                ev[i].record(sb)
        reconstruct(dst, tot, events=ev)
        cur.wait_stream(sa)
        cur.wait_stream(sb)

    def step():
        attribute_and_reconstruct()

    # the contraction's work-item size, autotuned on this data (outputs must
    # be bit-identical across the candidates); set before the graphs capture
    # the launches
    tuned = None
    if ws == 1 and prec != cq.PREC_FP32_SIMT:
        from paper_2205_05836_gb300.tune import tune_fd
        attribute_all()
        best, trials = tune_fd(subs, att, prec, out=out, ws=fd_ws)
        tuned = {"tiles_per_item": best, "trials_ms": {str(t): round(m, 4) for m, t, same in trials if same},
                 "all_identical": all(same for _, _, same in trials)}
        _log(f"work-item size tuned: {best}")

    # one step = one replay of a CUDA graph holding every launch of the step
    # (host argument checks run once, at capture); the library's launch
    # counter across the capture gives the kernels per step
    n0 = cq.cutqc_kernel_launches()
    graph = _graph(step, stream, args.warmup)
    launches_per_step = (cq.cutqc_kernel_launches() - n0) // (args.warmup + 1)
    g_att = _graph(attribute_all, stream, 1)
    g_fd = _graph(reconstruct, stream, 1)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, ws, dev)
    tot_all = total.clone()
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(tot_all)            # the FP64 totals of the ranks' row ranges
    sum_err = abs(tot_all.item() - 1.0)
    status = cq.cutqc_device_status()
    _log("timed steps done")

    # per-kernel timing on the stream the kernels run on: the attribution and
    # the FD sequence as graph replays; the dominant kernel (the last
    # contraction's tcgen05 GEMM) with events the library records around its
    # launch (eager calls, same stream)
    att_ms, fd_ms, gemm_ms = [], [], []
    for _ in range(max(3, min(args.steps, 10))):
        att_ms.append(_time_graph(g_att, stream, 1))
        fd_ms.append(_time_graph(g_fd, stream, 1))
        gs, ge = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cq.cutqc_fd_timing_events(gs, ge)
        reconstruct()
        torch.cuda.synchronize()
        gemm_ms.append(gs.elapsed_time(ge))
    att_ms, fd_ms, gemm_ms = (statistics.median(x) for x in (att_ms, fd_ms, gemm_ms))
    graph.replay()              # the timed output again (the eager calls rewrote it identically)
    torch.cuda.synchronize()

    pk = peaks()
    from workloads.cutting import contraction_plan
    _, alg_flops_all = contraction_plan([s.o for s in subs], [set(s.edges) for s in subs])
    # the last contraction: rows x cols outputs over 4^(cuts between the
    # pairs) terms; operands read once, 4 B written per probability
    k_last = 4 ** 4
    gemm_out_bytes = 4.0 * n_out
    gemm_in_bytes = 4.0 * k_last * ((r1 - r0) + cols)
    gemm_bytes = gemm_out_bytes + gemm_in_bytes
    gemm_flops = 2.0 * n_out * k_last
    achieved = gemm_bytes / (gemm_ms * 1e-3) / 1e9
    fd_bytes = 4.0 * n_out + sum(a.numel() * 4 for a in att)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"],
                "traffic": profiled_traffic("paper_2205_05836_gb300/csrc/gemm_tc_pair.cu",
                                            "profiles/tc_pair_gemm_fd_chain.md"),
                "kernel": "tc_pair_gemm_kernel (tcgen05, SM pairs): the last contraction of the chain, "
                          f"{r1 - r0} x {cols} outputs over {k_last} cut terms, one launch",
                "kernel_ms": gemm_ms, "algorithmic_bytes": gemm_bytes,
                "algorithmic_bytes_per_unit": "4 B written per probability + the two operands read once",
                "hbm_bound_ms": gemm_bytes / (pk["hbm_gbs"] * 1e9) * 1e3,
                "tensor_bound_ms_1pass": gemm_flops / (pk["bf16_tflops"] * 1e12) * 1e3,
                "tensor_bound_ms_executed": 3 * gemm_flops / (pk["bf16_tflops"] * 1e12) * 1e3,
                "executed_tflops": 3 * gemm_flops / (gemm_ms * 1e-3) / 1e12,
                "peak_source": pk["source"] + " (copy bandwidth; fp16 dense rate = bf16 rate)",
                "fd_sequence": {"ms": fd_ms, "algorithmic_bytes": fd_bytes,
                                "frac": fd_bytes / (fd_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                                "note": "all three contractions with their operand preps"},
                "step_frac": fd_bytes / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                "attribution_ms": att_ms}
    value = n_all / (ms * 1e-3) if ws > 1 else n_out / (ms * 1e-3)

    # total variation of the timed output against the FP64 oracle on 2^20
    # seeded uniformly sampled outputs of this rank's rows
    tv = None
    if rank == 0 and not args.no_tv:
        oracle = ChainOracle(w)
        rng = np.random.default_rng(2024)
        idx = np.unique(rng.integers(r0 * cols, r1 * cols, size=1 << 20))
        got = out[torch.from_numpy(idx - r0 * cols).to(dev)].cpu().numpy().astype(np.float64)
        ref = oracle.entries(idx)
        err = np.abs(got - ref)
        tv = {"tv_estimate": 0.5 * n_out * float(err.mean()), "max_abs_error": float(err.max()),
              "samples": int(len(idx)), "gate": 1e-6,
              "how": "0.5 * outputs * mean |GPU - FP64 oracle| over seeded uniform samples of the timed output"}
        _log("sampled TV against the oracle done")
    else:
        oracle = None

    # end to end through the C ABI from pinned host buffers: every step
    # uploads its variants, attributes, reconstructs and downloads its whole
    # output and FP64 total.  Two device output buffers let the download of
    # step i (a copy stream) overlap the upload and compute of step i + 1.
    host_var = [torch.from_numpy(v).pin_memory() for v in var_host]
    host_out = torch.empty(max(1, n_out), dtype=torch.float32, pin_memory=True)
    host_total = torch.zeros(1, dtype=torch.float64, pin_memory=True)
    dev_out = [out, torch.empty_like(out)]
    dev_total = [total, torch.zeros_like(total)]
    h2d = sum(v.numel() * v.element_size() for v in host_var)
    d2h = n_out * 4 + 8
    copy_stream = torch.cuda.Stream(dev)
    copied = [None, None]

    def e2e_step(i):
        b = i % 2
        if copied[b] is not None:
            stream.wait_event(copied[b])           # the previous download of this buffer is done
        for hv, v in zip(host_var, var):
            v.copy_(hv, non_blocking=True)
        attribute_and_reconstruct(dev_out[b], dev_total[b])
        done = torch.cuda.Event()
        done.record(stream)
        copy_stream.wait_event(done)
        with torch.cuda.stream(copy_stream):
            host_out.copy_(dev_out[b], non_blocking=True)
            host_total.copy_(dev_total[b], non_blocking=True)
            copied[b] = torch.cuda.Event()
            copied[b].record(copy_stream)
    e2e_step(0)
    e2e_step(1)
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 4))
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    stream.wait_stream(copy_stream)
    g1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(g0.elapsed_time(g1) / e2e_steps, ws, dev)
    del host_out, dev_out
    _log("end-to-end steps done")

    line = {"metric": METRIC, "value": value, "unit": "probs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None,
            "dtype": "f32 (FP16x3 split tensor-core products, FP32 accumulate)" if prec else "f32",
            "data": "synthetic",
            "config": chain_config(w, ws, r0, r1), "precision": args.precision, "tuned": tuned,
            "sum_p_error": sum_err, "tv": tv, "device_status": status,
            "roofline": roofline, "clocks": clk.summary(),
            "e2e": {"value": (n_all if ws > 1 else n_out) / (e2e_ms * 1e-3), "unit": "probs/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": "bound by the device-to-host copy of the output"},
            "gpu_launches": args.steps * launches_per_step, "gpu_launches_per_step": launches_per_step}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(oracle or ChainOracle(w), budget_s=args.ref_budget)
        _log("cpu baseline done")
    if rank == 0 and not args.no_extras:
        del graph, g_att, g_fd
        line["fd_chain_variants"] = chain_variant_extras(dev, cq, subs, att, out, total, r0, r1, ms)
        del out, fd_ws, host_var
        torch.cuda.empty_cache()
        _log("FD chain variants done")
        line["fd_two_sub"] = fd_two_sub_extras(dev, cq)
        torch.cuda.empty_cache()
        _log("FD two-subcircuit extras done")
        line["dd_batched"] = dd_extras(dev, cq)
        tc = dd_extras(dev, cq, precision=1)
        line["dd_batched"]["split_precision"] = {
            "graph_ms": tc["graph_ms"], "bins_per_s": tc["bins_per_s"],
            "root_sum_error": max(c["root_sum_error"] for c in tc["circuits"]),
            "options": {c["circuit"]: c["options"] for c in tc["circuits"]}}
        _log("DD extras done")
        torch.cuda.empty_cache()
        line["dd_dense"] = dd_dense_extras(dev, cq)
        torch.cuda.empty_cache()
        _log("DD dense extras done")
        line["finite_shots"] = finite_shot_extras(dev, cq)
        _log("finite-shot extras done")
        line["learned"] = learned_extras(dev, cq)
        _log("cut-scorer extras done")
    if rank == 0:
        print(json.dumps(line), flush=True)


def chain_variant_extras(dev, cq, subs, att, out, total, r0, r1, headline_ms, steps=10, warmup=3):
    """The same chain with cut-term pruning (the last contraction skips cut
    terms whose summed L1 bound is <= 2^-30) and on FP32 CUDA cores (the
    speed-up of the tensor-core path), each as a graph of the reconstruction
    alone; the headline's own reconstruction timed the same way beside them."""
    import torch
    stream = torch.cuda.current_stream(dev)
    res = {}
    pk = peaks()
    alg_bytes = 4.0 * out.numel() + sum(a.numel() * 4 for a in att)
    for name, prec in (("tc", cq.PREC_FP16X3_TC), ("tc_prune", cq.PREC_FP16X3_TC_PRUNE), ("simt", cq.PREC_FP32_SIMT)):
        fws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, prec)), dtype=torch.uint8, device=dev)

        def rec():
            total.zero_()
            cq.cutqc_reconstruct_fd(subs, att, cq.ORDER_KRON, prec, row_begin=r0, row_end=r1, out=out,
                                    sum_out=total, ws=fws)
        g = _graph(rec, stream, warmup)
        g.replay()
        torch.cuda.synchronize()
        k = 3 if name == "simt" else steps
        with ClockSampler(dev.index or 0) as clk:
            ms = _time_graph(g, stream, k)
        res[name] = {"ms": ms, "probs_per_s": out.numel() / (ms * 1e-3),
                     "hbm_frac": alg_bytes / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                     "sum_p_error": abs(total.item() - 1.0), "clocks": clk.summary()}
        del g, fws
    res["tc_prune"]["note"] = "last contraction skips cut terms whose summed L1 bound is <= 2^-30 (not the headline)"
    res["speedup_tc_over_simt"] = res["simt"]["ms"] / res["tc"]["ms"]
    res["speedup_tc_prune_over_simt"] = res["simt"]["ms"] / res["tc_prune"]["ms"]
    res["note"] = "reconstruction only (no attribution); tc = the headline's arithmetic"
    return res


def fd_two_sub_extras(dev, cq, steps=10, warmup=3):
    """The 30-qubit two-subcircuit workload (5 x 6 supremacy family, depth 10,
    the couplers across one split bridged so that K = 4; subcircuits 17 + 17,
    2^30 outputs): attribution + one tcgen05 contraction per step, timed as a
    graph; the contraction's own time with the library's events."""
    import torch
    from workloads.configs import fd_two_sub
    w = fd_two_sub()
    subs = w.subcircuits
    var = [torch.from_numpy(v).to(dev) for v in w.variants()]
    att = [torch.empty((1 << s.o, 4 ** (len(s.in_local) + len(s.out_local))), dtype=torch.float32, device=dev)
           for s in subs]
    aws = [torch.empty(max(1, cq.cutqc_attribute_workspace_size(s)), dtype=torch.uint8, device=dev) for s in subs]
    n_out = 1 << w.n
    out = torch.empty(n_out, dtype=torch.float32, device=dev)
    fws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, cq.PREC_FP16X3_TC)), dtype=torch.uint8,
                      device=dev)
    total = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        for s, v, a, b in zip(subs, var, att, aws):
            cq.cutqc_attribute(s, v, out=a, ws=b)
        total.zero_()
        cq.cutqc_reconstruct_fd(subs, att, cq.ORDER_KRON, cq.PREC_FP16X3_TC, out=out, sum_out=total, ws=fws)
    from paper_2205_05836_gb300.tune import tune_fd
    step()
    best, trials = tune_fd(subs, att, cq.PREC_FP16X3_TC, out=out, ws=fws)
    g = _graph(step, stream, warmup)
    g.replay()
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        ms = _time_graph(g, stream, steps)
    gemm = []
    for _ in range(5):
        gs, ge = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cq.cutqc_fd_timing_events(gs, ge)
        step()
        torch.cuda.synchronize()
        gemm.append(gs.elapsed_time(ge))
    gemm_ms = statistics.median(gemm)
    cq.cutqc_fd_set_tiles_per_item(0)
    pk = peaks()
    M, N = 1 << subs[0].o, 1 << subs[1].o
    Kg = 4 ** w.K
    gbytes = 4.0 * n_out + 4.0 * Kg * (M + N)
    return {"workload": TWO_SUB_WORKLOAD, "n_qubits": w.n, "cuts": w.K, "gemm": [M, N, Kg], "tiles_per_item": best,
            "tiles_per_item_trials_ms": {str(t): round(m, 4) for m, t, same in trials if same},
            "ms_per_step": ms, "probs_per_s": n_out / (ms * 1e-3), "sum_p_error": abs(total.item() - 1.0),
            "roofline": {"bound": "hbm", "kernel": "tc_pair_gemm_kernel, one launch", "kernel_ms": gemm_ms,
                         "algorithmic_bytes": gbytes, "achieved": gbytes / (gemm_ms * 1e-3) / 1e9,
                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gbytes / (gemm_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                         "traffic": profiled_traffic("paper_2205_05836_gb300/csrc/gemm_tc_pair.cu",
                                                     "profiles/tc_pair_gemm_fd_two_sub.md"),
                         "tensor_bound_ms_executed": 3 * 2.0 * n_out * Kg / (pk["bf16_tflops"] * 1e12) * 1e3},
            "clocks": clk.summary()}


def learned_extras(dev, cq, n_circuits=10000, train_steps=4000, batch=1024):
    """Cut scorer at scale: training set from seeded random circuits of 20-60
    qubits (labels: exact contraction cost of candidate cuts), GPU training
    by the library's kernels, then cut proposal for a 100-qubit BV circuit
    (subcircuits <= 20 qubits) against the local cut search, and dynamic
    definition on the proposed cut down to the hidden string."""
    import math
    import torch
    from paper_2205_05836_gb300.scorer import propose_cut
    from workloads import circuits as C
    from workloads.cutting import contraction_cost, search_cut
    from workloads.features import training_set, training_set_parallel
    from workloads.simulate import simulate_variants
    t0 = time.perf_counter()
    x, t, _ = training_set_parallel(n_circuits, 4, seed=0, workers=min(8, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    _log(f"training set: {len(t)} samples from {n_circuits} circuits in {gen_s:.1f} s")
    xv, tv, _ = training_set(200, 8, seed=99)
    net = cq.MLP(seed=0)
    X, T = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    net.fit(X, T, steps=20, batch=batch, lr=1e-3, seed=1)       # warm-up
    net = cq.MLP(seed=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.fit(X, T, steps=train_steps, batch=batch, lr=1e-3, seed=0)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    loss = net.loss.item()
    pv = net.forward(torch.from_numpy(xv).to(dev)).cpu().numpy()
    val_mse = float(((pv - tv) ** 2).mean())
    # inference latency: 4096 candidates in one forward
    xq = torch.from_numpy(np.ascontiguousarray(np.resize(xv, (4096, xv.shape[1])))).to(dev)
    for _ in range(3):
        net.forward(xq)
    torch.cuda.synchronize()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record()
    for _ in range(20):
        net.forward(xq)
    i1.record()
    torch.cuda.synchronize()
    infer_ms = i0.elapsed_time(i1) / 20

    _log("scorer trained")
    n, w_max = 100, 20
    c = C.bv(n, 5)
    t0 = time.perf_counter()
    searched = search_cut(c, w_max, -(-(n + 8) // w_max), restarts=4, seed=5)
    search_s = time.perf_counter() - t0
    mlp_only, info0 = propose_cut(c, w_max, net, n_candidates=4096, n_exact=8, seed=0)
    cut, info = propose_cut(c, w_max, net, n_candidates=4096, n_exact=8, seed=0, check_restarts=4)
    subs = cut.subcircuits
    att = [cq.cutqc_attribute(s, torch.from_numpy(simulate_variants(s)).to(dev)) for s in subs]
    M = 16
    R = math.ceil(n / M)
    cq.cutqc_dd_run(subs, att, n, M, R, 1, 0)        # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    jobs, bins = cq.cutqc_dd_run(subs, att, n, M, R, 1, 0)
    torch.cuda.synchronize()
    dd_s = time.perf_counter() - t0
    last = jobs[-1]
    b = bins[last.bins_offset:last.bins_offset + (1 << last.n_active)].cpu().numpy()
    top = int(np.argmax(b))
    bits = last.zoom()
    for j in range(last.n_active):
        bits[last.active[j]] = (top >> j) & 1
    exact = [bits.get(q, -1) for q in range(n - 1)] == c.meta["hidden"] and bits.get(n - 1) == 1
    return {"train_circuits": n_circuits, "train_samples": int(len(t)), "train_set_seconds": gen_s,
            "train_steps": train_steps, "batch": batch, "train_ms": train_ms,
            "train_samples_per_s": train_steps * batch / (train_ms * 1e-3), "final_loss": loss,
            "val_mse": val_mse, "val_label_var": float(tv.var()), "infer_4096_ms": infer_ms,
            "bv100": {"mlp_cut_log2_cost": math.log2(contraction_cost(mlp_only)), "mlp_cut_K": mlp_only.K,
                      "mlp_seconds": info0["seconds"], "feasible_candidates": info0["feasible"],
                      "with_search_check": {"log2_cost": math.log2(contraction_cost(cut)), "K": cut.K,
                                            "fallback": info["fallback"], "seconds": info["seconds"]},
                      "searched_cut_log2_cost": math.log2(contraction_cost(searched)), "searched_cut_K": searched.K,
                      "search_seconds": search_s, "dd_recursions": len(jobs), "dd_seconds": dd_s,
                      "bitstring_exact": bool(exact), "p_top": float(b[top])}}


def dd_alg_bytes(subs, jobs):
    """Algorithmic bytes of a set of DD bin jobs: each job reads the slice of
    every attributed tensor whose zoomed output bits equal its zoom (all 4^k
    columns of those rows, float32) and writes its 2^active bins (float32);
    the merged tensors in between are small and L2-resident."""
    tot = 0
    for j in jobs:
        zoom = j.zoom()
        for s in subs:
            z = sum(1 for q in s.out_qubit if q in zoom)
            k = len(s.in_local) + len(s.out_local)
            tot += (1 << (s.o - z)) * 4 ** k * 4
        tot += (1 << j.n_active) * 4
    return tot


def dd_extras(dev, cq, M=16, R=6, T=4, reps=5, precision=0):
    """Dynamic definition on the three blocked brick-wall circuits (40, 50
    and 60 qubits, subcircuits <= 15 qubits): Algorithm 1 level by level
    (breadth first), 16 active qubits per recursion, the top-4 bins of each
    level expanded in the next.  All levels of all three circuits are
    enqueued without host synchronisation (the selection runs on the device)
    and captured in one CUDA graph; bins/s = bins of one replay / its time.
    Launch shapes per circuit are chosen by the autotuner (tune.py) first.
    precision: bin reconstruction in FP32 (0) or on the split-precision
    tensor-core path (1)."""
    import torch
    from paper_2205_05836_gb300.tune import tune_dd
    from workloads.configs import dd_batched
    runs = []
    for w in dd_batched():
        _log(f"DD {w.name}")
        subs = w.subcircuits
        att = [cq.cutqc_attribute(s, torch.from_numpy(v).to(dev)) for s, v in zip(subs, w.variants())]
        ws = torch.empty(cq.cutqc_dd_run_workspace_size(subs, w.n, M, T), dtype=torch.uint8, device=dev)
        opt, trials = tune_dd(subs, att, w.n, M, R, T, precision=precision)
        jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, att, w.n, M, R, T, max_jobs=64, ws=ws, options=opt)
        runs.append((w, subs, att, jobs, n_jobs, bins, ws, opt, trials))
    torch.cuda.synchronize()
    # one graph: the three circuits' runs on three streams (independent work)
    side = torch.cuda.Stream(dev)
    streams = [torch.cuda.Stream(dev) for _ in runs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        fork = torch.cuda.Event()
        fork.record(side)
        joins = []
        for st, (w, subs, att, jobs, n_jobs, bins, ws, opt, trials) in zip(streams, runs):
            st.wait_event(fork)
            with torch.cuda.stream(st):
                cq.cutqc_dd_run_async(subs, att, w.n, M, R, T, jobs=jobs, n_jobs=n_jobs, bins=bins, ws=ws,
                                      options=opt)
                ev = torch.cuda.Event()
                ev.record(st)
                joins.append(ev)
        for ev in joins:
            side.wait_event(ev)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    out, tot_bins, tot_bytes = [], 0, 0
    for w, subs, att, jobs, n_jobs, bins, ws, opt, trials in runs:
        js = cq.dd_jobs_from_device(jobs, n_jobs)
        nb = sum(1 << j.n_active for j in js)
        tot_bins += nb
        tot_bytes += dd_alg_bytes(subs, js)
        out.append({"circuit": w.name, "n": w.n, "subcircuits": len(subs), "K": w.K, "jobs": len(js), "bins": nb,
                    "root_sum_error": abs(js[0].bin_sum - 1.0), "options": opt,
                    "tuning_ms": {f"{o['merge_ctas']}/{o['topk_threads']}": round(ms, 4) for ms, o, ok in trials if ok}})
    pk = peaks()
    res = {"M": M, "R": R, "T": T, "strategy": "bfs", "precision": "tc" if precision else "fp32",
           "circuits": out, "graph_ms": ms, "bins_per_s": tot_bins / (ms * 1e-3),
           "algorithmic_bytes": tot_bytes,
           "graph_roofline": {"bound": "hbm", "achieved": tot_bytes / (ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": tot_bytes / (ms * 1e-3) / 1e9 / pk["hbm_gbs"]},
           "note": "all levels of the three circuits in one captured CUDA graph (one stream per circuit); "
                   "selection on the device"}
    if precision == 0:
        # the headline DD rate is the persistent launch's when it reproduced
        # the level launches' records and bins; both rates are kept
        pers = dd_batch_extras(dev, cq, runs, M, R, T, tot_bins, reps)
        pers["roofline"] = {"bound": "hbm", "achieved": tot_bytes / (pers["ms"] * 1e-3) / 1e9,
                            "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": tot_bytes / (pers["ms"] * 1e-3) / 1e9 / pk["hbm_gbs"],
                            "algorithmic_bytes": tot_bytes,
                            "note": "per job: the zoomed slice of every attributed tensor read once + 4 B per "
                                    "bin written; the launch is bound by its phases' barrier and dependency "
                                    "latency, not by bytes"}
        res["persistent"] = pers
        res["level_launches_bins_per_s"] = res["bins_per_s"]
        if pers["matches_level_by_level"] and pers["device_status"] == 0:
            res["bins_per_s"] = pers["bins_per_s"]
            res["ms"] = pers["ms"]
            res["headline"] = "persistent launch"
            res["note"] = ("bins_per_s / ms: all levels of the three circuits in one persistent cooperative launch; "
                           "graph_ms / level_launches_bins_per_s: the same runs as one captured CUDA graph of "
                           "level launches (one stream per circuit); selection on the device in both")
    return res


def dd_batch_extras(dev, cq, runs, M, R, T, tot_bins, reps):
    """The same three circuits in ONE persistent cooperative launch
    (cutqc_dd_batch_*, launch shapes from tune.py), captured in a graph and
    replayed; its records and bins must equal the level-by-level run's."""
    import torch
    from paper_2205_05836_gb300.tune import tune_dd_batch
    bruns = [cq.dd_batch_run(subs, att, w.n, M, R, T, max_jobs=64) for w, subs, att, *_ in runs]
    opt, trials = tune_dd_batch(bruns)
    batch = cq.cutqc_dd_batch_create(bruns, opt)
    side = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        batch.launch(side)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    same = True
    for (w, subs, att, jobs, n_jobs, bins, *_), b in zip(runs, bruns):
        ref = cq.dd_jobs_from_device(jobs, n_jobs)
        got = cq.dd_jobs_from_device(b["jobs"], b["n_jobs"])
        same &= len(ref) == len(got) and all(
            (x.parent, x.parent_bin, list(x.top_idx)) == (y.parent, y.parent_bin, list(y.top_idx)) and
            torch.equal(bins[x.bins_offset:x.bins_offset + (1 << x.n_active)],
                        b["bins"][y.bins_offset:y.bins_offset + (1 << y.n_active)]) for x, y in zip(ref, got))
    info = batch.info()
    return {"ms": ms, "bins_per_s": tot_bins / (ms * 1e-3), "options": opt, "phases": info["phases"],
            "ops": info["ops"], "ctas": info["ctas"], "matches_level_by_level": bool(same),
            "device_status": cq.cutqc_device_status(), "clocks": clk.summary(),
            "tuning_ms": {f"{o['ctas_per_sm']}/{o['topk_chunk']}/{o['narrow_max_n']}": round(t, 4)
                          for t, o, ok in trials if ok},
            "tuning_key": "ctas_per_sm/topk_chunk/narrow_max_n",
            "gpu_launches_per_replay": 1,
            "note": "one cooperative launch (and one memset) for all levels of the three circuits; "
                    "grid barriers between phases"}


def finite_shot_extras(dev, cq, shots=(10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6), seed=7):
    """The paper's shot-based mode on the 8-qubit brick-wall workload: every
    subcircuit variant sampled with S shots (seeded multinomial), attributed
    and reconstructed on the GPU, and Eq. 3 (chi^2) against the reconstruction
    from exact variants (which the tests pin to the uncut circuit's exact
    distribution).  Beside it, chi^2 of the uncut circuit sampled directly
    with the same total number of shots (no device noise in either)."""
    import torch
    from workloads.configs import fd_plain
    from workloads.simulate import sample_distribution, sample_variants
    w = fd_plain()
    subs = w.subcircuits
    exact = w.variants()

    def rec(vs):
        att = [cq.cutqc_attribute(s, torch.from_numpy(v).to(dev)) for s, v in zip(subs, vs)]
        out, _ = cq.cutqc_reconstruct_fd(subs, att, cq.ORDER_ORIGINAL, cq.PREC_FP16X3_TC)
        return out.double()

    def chi2(a, b):       # Eq. 3 over the terms with a_i + b_i != 0
        s = a + b
        m = s != 0
        return float(((a[m] - b[m]) ** 2 / s[m]).sum())

    def clip(a):          # Eq. 3 is for distributions: negatives to 0, total 1
        a = a.clamp(min=0)
        return a / a.sum()
    truth = rec(exact)
    runs = sum(v.shape[0] * v.shape[1] for v in exact)
    res = {"workload": w.name, "n_qubits": w.n, "cuts": w.K, "variant_runs": int(runs), "per_shots": {}}
    for i, S in enumerate(shots):
        a = rec([sample_variants(v, S, seed + 10 * i + j) for j, v in enumerate(exact)])
        direct = torch.from_numpy(sample_distribution(truth.cpu().numpy(), S * runs, seed + 10 * i + 9)).to(dev)
        res["per_shots"][str(S)] = {"chi2_cut": chi2(clip(a), truth),
                                    "chi2_direct_same_total_shots": chi2(direct, truth),
                                    "tv_cut": 0.5 * float((a - truth).abs().sum()),
                                    "tv_direct_same_total_shots": 0.5 * float((direct - truth).abs().sum()),
                                    "negative_mass": float(-a[a < 0].sum())}
    res["note"] = "chi2_cut: the reconstruction with negative entries clipped to 0 and renormalised"
    return res


def dd_dense_extras(dev, cq, M=30, T=4, reps=5):
    """One dense recursion (the paper's per-recursion workload of 2^30 bins):
    the 60-qubit blocked brick-wall circuit (5 subcircuits <= 15 qubits,
    K = 6), qubits 0..29 active, 30..59 merged; merge, bin reconstruction
    and top-T selection as one captured CUDA graph, FP32 and split-precision
    tensor cores; bins/s = 2^30 / time."""
    import torch
    from workloads.configs import dd_batched
    w = [x for x in dd_batched() if x.n == 60][0]
    subs = w.subcircuits
    att = [cq.cutqc_attribute(s, torch.from_numpy(v).to(dev)) for s, v in zip(subs, w.variants())]
    ws = torch.empty(cq.cutqc_dd_run_workspace_size(subs, w.n, M, T), dtype=torch.uint8, device=dev)
    bins = torch.empty(1 << M, dtype=torch.float32, device=dev)
    res = {"circuit": w.name, "n": w.n, "subcircuits": len(subs), "K": w.K, "active": M, "bins": 1 << M, "T": T}
    for name, prec in (("fp32", 0), ("tc", 1)):
        opt = {"precision": prec}
        jobs, n_jobs, _ = cq.cutqc_dd_run_async(subs, att, w.n, M, 1, T, max_jobs=4, bins=bins, ws=ws, options=opt)
        torch.cuda.synchronize()
        side = torch.cuda.Stream(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            cq.cutqc_dd_run_async(subs, att, w.n, M, 1, T, jobs=jobs, n_jobs=n_jobs, bins=bins, ws=ws, options=opt)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index or 0) as clk:
            e0.record()
            for _ in range(reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        js = cq.dd_jobs_from_device(jobs, n_jobs)
        res[name] = {"ms": ms, "bins_per_s": (1 << M) / (ms * 1e-3), "root_sum_error": abs(js[0].bin_sum - 1.0),
                     "top_idx": [int(i) for i in js[0].top_idx[:T]], "clocks": clk.summary()}
        del g
    pk = peaks()
    alg = dd_alg_bytes(subs, js)
    res["algorithmic_bytes"] = alg
    res["hbm_bound_ms"] = alg / (pk["hbm_gbs"] * 1e9) * 1e3
    for name in ("fp32", "tc"):
        a = alg / (res[name]["ms"] * 1e-3) / 1e9
        res[name]["roofline"] = {"bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                 "frac": a / pk["hbm_gbs"]}
    res["speedup_tc_over_fp32"] = res["fp32"]["ms"] / res["tc"]["ms"]
    res["note"] = "algorithmic bytes: the attributed tensors read once + 4 B per bin written"
    return res


def run_profile_case(args):
    """The benchmark's kernels once after one warm-up pass, for ncu.
    Workloads: fd_two_sub -- a row slice (args.profile_rows rows of the last
    contraction, 1 GiB of output at 2048) of the 30-qubit two-subcircuit
    reconstruction; fd_chain -- the whole 32-qubit chain (2^32 outputs, 16
    GiB: for one-pass launch lists only); fd_chain_slice -- a row slice of
    the chain's last contraction; dd_dense -- one 2^30-bin recursion of the
    60-qubit DD circuit; dd_batched -- Algorithm 1 on the three DD circuits
    (16 active qubits, top 4, breadth first); dd_persistent -- the same as
    one persistent launch (cutqc_dd_batch_*)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc as cq
    prec = {"tc": cq.PREC_FP16X3_TC, "tc_prune": cq.PREC_FP16X3_TC_PRUNE, "simt": cq.PREC_FP32_SIMT}[args.precision]
    wl = args.profile_workload
    info = {"profile_case": wl, "precision": args.precision}
    if wl in ("fd_two_sub", "fd_chain", "fd_chain_slice"):
        from workloads.configs import fd_chain, fd_two_sub
        w = fd_two_sub() if wl == "fd_two_sub" else fd_chain()
        subs = w.subcircuits
        var = [torch.from_numpy(v).cuda() for v in w.variants()]
        ranged = wl != "fd_chain"
        out = None
        if not ranged:
            out = torch.empty(1 << w.n, dtype=torch.float32, device="cuda")
        ws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, prec)), dtype=torch.uint8, device="cuda")
        total = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            att = [cq.cutqc_attribute(s, v) for s, v in zip(subs, var)]
            total.zero_()
            if ranged:
                out, _ = cq.cutqc_reconstruct_fd(subs, att, cq.ORDER_KRON, prec, row_begin=0,
                                                 row_end=args.profile_rows, ws=ws, sum_out=total)
            else:
                cq.cutqc_reconstruct_fd(subs, att, cq.ORDER_KRON, prec, out=out, ws=ws, sum_out=total)
        torch.cuda.synchronize()
        info.update({"workload": w.name, "rows": args.profile_rows if ranged else None, "outputs": out.numel(),
                     "sum": total.item()})
    elif wl == "dd_dense":
        from workloads.configs import dd_batched
        w = [x for x in dd_batched() if x.n == 60][0]
        subs = w.subcircuits
        att = [cq.cutqc_attribute(s, torch.from_numpy(v).cuda()) for s, v in zip(subs, w.variants())]
        ws = torch.empty(cq.cutqc_dd_run_workspace_size(subs, w.n, 30, 4), dtype=torch.uint8, device="cuda")
        bins = torch.empty(1 << 30, dtype=torch.float32, device="cuda")
        for _ in range(2):
            jobs, n_jobs, _ = cq.cutqc_dd_run_async(subs, att, w.n, 30, 1, 4, max_jobs=4, bins=bins, ws=ws,
                                                    options={"precision": prec})
        js = cq.dd_jobs_from_device(jobs, n_jobs)
        info.update({"workload": w.name, "bins": 1 << 30, "bin_sum": js[0].bin_sum})
    elif wl == "dd_persistent":
        from workloads.configs import dd_batched
        runs = []
        for w in dd_batched():
            subs = w.subcircuits
            att = [cq.cutqc_attribute(s, torch.from_numpy(v).cuda()) for s, v in zip(subs, w.variants())]
            runs.append(cq.dd_batch_run(subs, att, w.n, 16, 6, 4, max_jobs=64))
        batch = cq.cutqc_dd_batch_create(runs)
        for _ in range(2):
            batch.launch()
        torch.cuda.synchronize()
        # per-phase durations of the last launch (SM cycles of CTA 0 between barriers)
        info.update({"workload": [w.name for w in dd_batched()], "batch": batch.info(),
                     "phases": batch.phases(), "device_status": cq.cutqc_device_status()})
    else:
        from workloads.configs import dd_batched
        runs = []
        for w in dd_batched():
            subs = w.subcircuits
            att = [cq.cutqc_attribute(s, torch.from_numpy(v).cuda()) for s, v in zip(subs, w.variants())]
            ws = torch.empty(cq.cutqc_dd_run_workspace_size(subs, w.n, 16, 4), dtype=torch.uint8, device="cuda")
            runs.append((w, subs, att, ws))
        for _ in range(2):
            for w, subs, att, ws in runs:
                cq.cutqc_dd_run_async(subs, att, w.n, 16, 6, 4, max_jobs=64, ws=ws, options={"precision": prec})
        torch.cuda.synchronize()
        info.update({"workload": [r[0].name for r in runs]})
    print(json.dumps(info))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tc", choices=["tc", "tc_prune", "simt"])
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tv", action="store_true", help="skip the sampled TV of the timed output")
    ap.add_argument("--no-extras", action="store_true", help="skip the DD and cut-scorer measurements")
    ap.add_argument("--profile-case", action="store_true",
                    help="run the kernels once on a row slice (for ncu) and exit")
    ap.add_argument("--profile-rows", type=int, default=2048)
    ap.add_argument("--profile-workload", default="fd_two_sub",
                    choices=["fd_two_sub", "fd_chain", "fd_chain_slice", "dd_dense", "dd_batched", "dd_persistent"])
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
