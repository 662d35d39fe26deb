"""SpKAdd benchmark (one JSON line on rank 0).

Default workload: k = 32 Erdos-Renyi matrices of 2^20 x 2^20, exactly 16
distinct uniform rows per column, int32 indices, fp64 values uniform on
[-1, 1] (about 5.4e8 input nonzeros, 6.4 GB).  One step = the whole hot path
on one batch: spkadd_plan (column binning) + spkadd_symbolic (per-column
distinct-row counts, scan, nnz(B) readback) + output allocation +
spkadd_numeric (accumulate + sort + write B) + spkadd_destroy.

value     input nonzeros per second over all ranks, inputs resident in HBM.
e2e       the same metric through the same C ABI with inputs in pinned host
          memory: every step copies the inputs host->device and B
          device->host inside the timed region (step i+1's input copy
          overlaps step i's compute and output copy).
roofline  for the numeric kernel (the dominant one): algorithmic bytes per
          launch / its CUDA-event duration, against the measured HBM copy
          bandwidth.
cpu_baseline  the CPU oracle (oracle/spk_oracle.c, OpenMP) timed on this
          host on a bounded sample of the same workload.

--impl reference times the oracle alone (the reference arm of this repo is
the oracle; no GPU work).  Under torchrun every rank runs its own instance
(weak scaling, no data-path collective); timings are reduced with MAX.
"""
from __future__ import annotations

import argparse
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

import torch  # noqa: E402

METRIC = "SpKAdd input nnz/s & HBM GB/s vs roofline; batched/served p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    # name: (family, k, m, n, d or scale, dtype)
    "er_k32_m2p20_d16_f64": dict(family="er", k=32, m=1 << 20, n=1 << 20, d=16, dtype=torch.float64),
    "rmat_k64_s20_ef16_f32": dict(family="rmat", k=64, scale=20, ef=16, dtype=torch.float32),
    # profiling case: the R-MAT workload at scale 18 (2.6e8 input nnz, 2 GB, still > L2)
    "rmat_k64_s18_ef16_f32": dict(family="rmat", k=64, scale=18, ef=16, dtype=torch.float32),
    "er_k4_m1024_d8_f64int": dict(family="er", k=4, m=1024, n=1024, d=8, dtype=torch.float64, value_kind="int8"),
    # profiling case: the default workload with a quarter of the columns (1.6 GB of input, still > L2)
    "er_k32_m2p20_n2p18_d16_f64": dict(family="er", k=32, m=1 << 20, n=1 << 18, d=16, dtype=torch.float64),
}
DEFAULT_WORKLOAD = "er_k32_m2p20_d16_f64"
RMAT_WORKLOAD = "rmat_k64_s20_ef16_f32"


def make_inputs(w, device, seed, n_override=None):
    import synth

    if w["family"] == "er":
        n = n_override or w["n"]
        A = synth.er(w["k"], w["m"], n, w["d"], seed=seed, dtype=w["dtype"],
                     value_kind=w.get("value_kind", "uniform"), device=device)
        return A, w["m"]
    if w["family"] == "rmat":
        A = synth.rmat(w["k"], w["scale"], w["ef"], seed=seed, dtype=w["dtype"], device=device)
        return A, 1 << w["scale"]
    raise ValueError(w["family"])


def shuffle_within_columns(A, seed):
    """The same matrices with every input column's (row, value) pairs in random order."""
    out = []
    g = torch.Generator(device=A[0][0].device)
    g.manual_seed(seed + 7919)
    for cp, ri, va in A:
        cpl = cp.to(torch.int64)
        col = torch.repeat_interleave(torch.arange(cp.numel() - 1, device=cp.device), cpl[1:] - cpl[:-1])
        key = col.to(torch.float64) + 0.5 * torch.rand(ri.numel(), generator=g, device=cp.device, dtype=torch.float64)
        perm = torch.argsort(key)
        out.append((cp, ri[perm].contiguous(), va[perm].contiguous()))
    return out


def algorithmic_bytes(k, n, nnz_in, nnz_out, vbytes):
    """Read every input once (rows, values, column pointers), write B once."""
    return nnz_in * (4 + vbytes) + k * (n + 1) * 4 + nnz_out * (4 + vbytes) + (n + 1) * 8


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("hbm_gbs"):
            return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("spk_warp.cu", "spk_common.cuh"):
        with open(os.path.join(ROOT, "paper_2112_10223_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(workload):
    """ncu DRAM bytes per launch of the numeric kernel, if captured for the current source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload)
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        with open(self.file.name) as f:
            rows = [r.strip().split(", ") for r in f if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        loaded = [x for x in sm if mx and x > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(A, cols):
    """A bounded sample of the workload for the CPU oracle: every
    (n / cols)-th column of the same inputs, copied to host memory."""
    import synth

    n = A[0][0].numel() - 1
    stride = max(1, n // max(cols, 1))
    idx = torch.arange(0, n, stride, dtype=torch.int64)[:cols]
    sub = synth.take_columns(A, idx)
    return [tuple(t.cpu() for t in a) for a in sub], stride


def time_oracle(A, threads=0, repeat=1, min_seconds=0.0):
    """Mean time of the oracle on A over `repeat` runs, or over as many runs as
    it takes to reach min_seconds of CPU work (at most 8)."""
    import oracle

    An = [tuple(t.numpy() for t in a) for a in A]
    oracle.add(An, threads=threads)  # warm (page faults, build)
    ts = []
    while len(ts) < repeat or (sum(ts) < min_seconds and len(ts) < 8):
        t0 = time.perf_counter()
        oracle.add(An, threads=threads)
        ts.append(time.perf_counter() - t0)
    nnz = sum(a[1].numel() for a in A)
    return nnz, sum(ts) / len(ts), oracle.threads_used(threads), len(ts)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def reduce_max(x, world):
    if world == 1:
        return x
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def reference_sample(args):
    """The oracle's bounded sample of the workload: a list of problems (inputs
    on the host), a description, and the value dtype."""
    import synth

    dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    if args.workload in WORKLOADS:
        w = WORKLOADS[args.workload]
        A, _ = make_inputs(w, dev, seed=args.seed)
        S, stride = oracle_sample(A, args.oracle_cols)
        nnz = sum(a[1].numel() for a in S)
        return [S], f"every {stride}-th column of the workload: {len(S[0][0]) - 1} columns, {nnz} input nnz per step", \
            "f64" if w["dtype"] == torch.float64 else "f32"
    if args.workload == STREAM_WORKLOAD:  # the summed result of all 64 inputs, on a column sample
        A = synth.spgemm_like(64, 1 << 18, 1 << 18, 32, seed=args.seed, dtype=torch.float32, device=dev)
        S, stride = oracle_sample(A, min(args.oracle_cols, 1 << 14))
        nnz = sum(a[1].numel() for a in S)
        return [S], f"every {stride}-th column of the 64 inputs: {nnz} input nnz per step", "f32"
    # batched / served workloads: the instances in seed order, up to about 3e7 input nnz
    if args.workload == BATCH_WORKLOAD:
        params = synth.batch_instance_params(args.batch_count, seed=args.seed)
    else:
        params = synth.batch_instance_params(args.serve_requests, seed=args.seed, k_range=(2, 512),
                                             mn_range=(1 << 10, 1 << 18))
    probs, nnz = [], 0
    for p in params:  # in seed order, every instance that still fits the budget
        if nnz + synth.instance_nnz_estimate(p) > 3e7:
            continue
        A, _ = synth.instance(p, "cpu")
        probs.append(A)
        nnz += sum(a[1].numel() for a in A)
    return probs, (f"{len(probs)} instances of the workload, in seed order those that fit a 3e7-nnz budget "
                   f"({nnz} input nnz per step)"), "f32+f64"


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle on a bounded sample, rank 0 only."""
    if rank != 0:
        return
    probs, sample, dtype = reference_sample(args)
    nnz = sum(a[1].numel() for A in probs for a in A)
    cores = 1

    def once():
        nonlocal cores
        t = 0.0
        for A in probs:
            _, ti, cores, _ = time_oracle(A, repeat=1)
            t += ti
        return t

    for _ in range(args.warmup):
        once()
    ts = [once() for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    val = nnz / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": {"workload": args.workload},
        "cpu_baseline": {"value": val, "unit": "nnz/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def step_fn(spk, A, m, n, dtype, dev, stream, opts, method, ev=None, want_info=False):
    """One step of the hot path on resident inputs: plan, (symbolic, B
    allocation, numeric) or (B allocation, one pass), destroy.  `ev` brackets
    the dominant kernel work (the numeric phase, or the one-pass launch)."""
    h = spk.spkadd_plan(A, m, stream=stream, options=opts)
    cp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    if method == "onepass":
        cap = sum(a[1].numel() for a in A)
        ri = torch.empty(cap, dtype=torch.int32, device=dev)
        va = torch.empty(cap, dtype=dtype, device=dev)
        if ev is not None:
            ev[0].record(stream)
        nnz = spk.spkadd_onepass(h, cp, ri, va)
        if ev is not None:
            ev[1].record(stream)
    else:
        nnz = spk.spkadd_symbolic(h)
        ri = torch.empty(nnz, dtype=torch.int32, device=dev)
        va = torch.empty(nnz, dtype=dtype, device=dev)
        if ev is not None:
            ev[0].record(stream)
        spk.spkadd_numeric(h, cp, ri, va)
        if ev is not None:
            ev[1].record(stream)
    info = spk.spkadd_get_info(h) if want_info else None  # (synchronises: never inside the timed region)
    spk.spkadd_destroy(h)
    return nnz, info


def timed_steps(spk, A, m, n, dtype, dev, stream, opts, method, steps, warmup, world, rank, clocks=False):
    """W untimed steps, then exactly K timed steps bracketed by a barrier and a
    synchronize; returns (seconds per step (MAX over ranks), dominant-kernel ms
    per step (CUDA events on the launching stream), nnz(B), info, clocks)."""
    nnz, info = None, None
    for i in range(max(warmup, 1)):
        nnz, inf = step_fn(spk, A, m, n, dtype, dev, stream, opts, method, want_info=(i == 0))
        info = inf or info
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if clocks and rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        step_fn(spk, A, m, n, dtype, dev, stream, opts, method, events[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = sampler.stop() if sampler else None
    barrier(world)
    elapsed = reduce_max(t0.elapsed_time(t1) / 1e3, world)
    kern_ms = reduce_max(sum(a.elapsed_time(b) for a, b in events) / steps, world)
    return elapsed / steps, kern_ms, nnz, info, clk


def cpu_baseline_of(A, cols, min_seconds=10.0):
    S, stride = oracle_sample(A, cols)
    nz_s, t_s, cores, reps = time_oracle(S, min_seconds=min_seconds)
    return {"value": nz_s / t_s, "unit": "nnz/s", "cores": cores, "kind": "oracle",
            "sample": f"every {stride}-th column of the workload ({len(S[0][0]) - 1} columns, {nz_s} input nnz), "
                      f"{reps} runs of {t_s:.2f} s each"}


def pairwise_tree(A, m):
    """The 2-way tree of Sec. II-B (the paper's "2-way Tree" / "MKL Tree"
    comparison systems) on this GPU: inputs added in pairs, level by level,
    each addition done by cuSPARSE (csrgeam2, reached through torch.add on
    sparse CSR tensors: a CSC matrix is the CSR form of its transpose).
    Returns (col_ptr, row_idx, val) of the sum."""
    import warnings

    warnings.filterwarnings("ignore", message="Sparse CSR tensor support is in beta state")
    n = A[0][0].numel() - 1
    level = [torch.sparse_csr_tensor(cp, ri, va, size=(n, m), check_invariants=False) for cp, ri, va in A]
    while len(level) > 1:
        nxt = [torch.add(level[i], level[i + 1]) for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    B = level[0]
    return B.crow_indices(), B.col_indices(), B.values()


def time_pairwise_tree(A, m, ours, steps, warmup):
    """Per-step time of pairwise_tree on resident inputs (CUDA events), and
    whether its result equals ours (indices exactly, values within the parity
    tolerance)."""
    for _ in range(max(warmup, 1)):
        B = pairwise_tree(A, m)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        B = pairwise_tree(A, m)
    e1.record()
    torch.cuda.synchronize()
    cp, ri, va = ours
    same_idx = (B[0].numel() == cp.numel() and bool(torch.equal(B[0].to(torch.int64), cp))
                and bool(torch.equal(B[1].to(torch.int32), ri)))
    tol = 1e-12 if va.dtype == torch.float64 else 1e-5
    same_val = same_idx and bool(((B[2].to(torch.float64) - va.to(torch.float64)).abs()
                                  <= tol * len(A) * (va.to(torch.float64).abs() + 1)).all())
    return e0.elapsed_time(e1) / steps, same_idx, same_val


def kernel_label(info, method):
    if method == "onepass" and info.get("onepass"):
        return "k_warp_onepass (spkadd_onepass)"
    if info["cols_cta"] + info["cols_heavy"] == 0:
        return "k_warp_col<numeric> (spkadd_numeric)"
    return ("spkadd_numeric: k_warp_col<numeric> and the thread-block items' kernel "
            "(k_num_compact or k_num_bitmap)")


def run_ours(args, world, rank, local):
    import paper_2112_10223_gb300 as spk

    spk.library()  # fails loudly if the CUDA library was not built
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    w = WORKLOADS[args.workload]
    A, m = make_inputs(w, dev, seed=args.seed + rank)
    opts = None
    if args.unordered or args.unsorted_output or args.block_accumulator:
        if args.unordered:  # rows shuffled inside every input column; the library told so
            A = shuffle_within_columns(A, args.seed + rank)
        opts = spk.default_options(input_order=1 if args.unordered else 0, sort_mode=2 if args.unsorted_output else 0,
                                   block_accumulator=args.block_accumulator)
    k = len(A)
    n = A[0][0].numel() - 1
    dtype = w["dtype"]
    vbytes = 8 if dtype == torch.float64 else 4
    nnz_in = sum(a[1].numel() for a in A)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    t_step, kern_ms, nnz_out, info, clk = timed_steps(spk, A, m, n, dtype, dev, stream, opts, args.method,
                                                      args.steps, args.warmup, world, rank, clocks=True)
    launches_per_step = info["kernel_launches"]
    peak, peak_src = read_peaks()
    alg = algorithmic_bytes(k, n, nnz_in, nnz_out, vbytes)

    # The other method on the same inputs (context line: which path is faster here).
    other = None
    if args.compare_methods:
        om = "onepass" if args.method == "twopass" else "twopass"
        o_step, o_kern, _, o_info, _ = timed_steps(spk, A, m, n, dtype, dev, stream, opts, om, args.steps,
                                                   args.warmup, world, rank)
        other = {"method": om, "ms_per_step": o_step * 1e3, "value": world * nnz_in / o_step,
                 "step_frac": alg / o_step / 1e9 / peak, "kernel_ms": o_kern, "kernel": kernel_label(o_info, om),
                 "onepass_used": bool(o_info.get("onepass"))}

    # Context for Sec. II-C's claim that k-way beats 2-way: the same sum as a
    # pairwise tree of cuSPARSE additions on this GPU.
    tree = None
    if args.pairwise_tree and args.workload == DEFAULT_WORKLOAD and not args.unordered:
        ours = spk.spkadd(A, m, method=args.method)
        t_ms, same_idx, same_val = time_pairwise_tree(A, m, ours, max(2, args.steps // 3), 2)
        del ours
        torch.cuda.empty_cache()
        tree = {"system": "pairwise tree of cuSPARSE csrgeam2 additions (torch.add on sparse CSR), "
                          f"{k - 1} additions in {math.ceil(math.log2(max(k, 2)))} levels",
                "ms_per_step": t_ms, "value": world * nnz_in / (t_ms / 1e3), "unit": "nnz/s",
                "kway_speedup": t_ms / (t_step * 1e3), "same_indices": same_idx, "same_values": same_val}

    cpu_sample, cpu_stride = (oracle_sample(A, args.oracle_cols) if rank == 0 and world == 1
                              and args.oracle_cols > 0 else (None, None))
    # e2e: host buffers through the same C ABI, copies inside the timed region.
    # Steps are pipelined the way a streaming caller would run them: step
    # i+1's inputs go host->device on their own stream (into the other of two
    # device buffer sets) while step i computes and its result goes
    # device->host on the compute stream.
    e2e = None
    if args.e2e_steps > 0:
        host = [tuple(t.cpu().pin_memory() for t in a) for a in A]
        h2d = sum(t.numel() * t.element_size() for a in host for t in a)
        out_cp = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
        out_ri = torch.empty(nnz_out, dtype=torch.int32, pin_memory=True)
        out_va = torch.empty(nnz_out, dtype=dtype, pin_memory=True)
        d2h = (n + 1) * 8 + nnz_out * (4 + vbytes)
        del A
        torch.cuda.empty_cache()
        s_in = torch.cuda.Stream(device=dev)
        s_c = torch.cuda.Stream(device=dev)
        bufs = [[tuple(torch.empty_like(t, device=dev) for t in a) for a in host] for _ in range(2)]

        def e2e_run(steps):
            ev_in = [torch.cuda.Event() for _ in range(steps)]
            ev_done = [torch.cuda.Event() for _ in range(steps)]

            def copy_in(i):
                with torch.cuda.stream(s_in):
                    if i >= 2:
                        s_in.wait_event(ev_done[i - 2])  # buffer set i % 2 is free again
                    for dst, src in zip(bufs[i % 2], host):
                        for d, s_ in zip(dst, src):
                            d.copy_(s_, non_blocking=True)
                    ev_in[i].record(s_in)

            copy_in(0)
            for i in range(steps):
                if i + 1 < steps:
                    copy_in(i + 1)
                s_c.wait_event(ev_in[i])
                with torch.cuda.stream(s_c):
                    hh = spk.spkadd_plan(bufs[i % 2], m, stream=s_c, options=opts)
                    nz = spk.spkadd_symbolic(hh)
                    cp = torch.empty(n + 1, dtype=torch.int64, device=dev)
                    ri = torch.empty(nz, dtype=torch.int32, device=dev)
                    va = torch.empty(nz, dtype=dtype, device=dev)
                    spk.spkadd_numeric(hh, cp, ri, va)
                    out_cp.copy_(cp, non_blocking=True)
                    out_ri[:nz].copy_(ri, non_blocking=True)
                    out_va[:nz].copy_(va, non_blocking=True)
                    spk.spkadd_destroy(hh)
                    ev_done[i].record(s_c)
            torch.cuda.synchronize()

        e2e_run(2)
        barrier(world)
        t0 = time.perf_counter()
        e2e_run(args.e2e_steps)
        te = reduce_max(time.perf_counter() - t0, world)
        e2e = {"value": world * nnz_in * args.e2e_steps / te, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "pipelining": "step i+1's H2D overlaps step i's compute and D2H (two streams, two input buffers)"}
        del bufs, host
    else:
        del A
    torch.cuda.empty_cache()

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and args.oracle_cols > 0:
        nz_s, t_s, cores, reps = time_oracle(cpu_sample, min_seconds=10.0)
        cpu = {"value": nz_s / t_s, "unit": "nnz/s", "cores": cores, "kind": "oracle",
               "sample": f"every {cpu_stride}-th column of the workload ({len(cpu_sample[0][0]) - 1} columns, "
                         f"{nz_s} input nnz), {reps} runs of {t_s:.2f} s each"}

    # The skewed R-MAT workload (k = 64, scale 20, fp32) in the same run, as a
    # second line under its own key: the default invocation measures both
    # single-instance workloads that the roofline target names.
    extra = {}
    if args.extra_rmat and args.workload == DEFAULT_WORKLOAD:
        wr = WORKLOADS[RMAT_WORKLOAD]
        R, mr = make_inputs(wr, dev, seed=args.seed + rank)
        kr, nr = len(R), R[0][0].numel() - 1
        nnz_r = sum(a[1].numel() for a in R)
        r_step, r_kern, r_nnz, r_info, r_clk = timed_steps(spk, R, mr, nr, wr["dtype"], dev, stream, None, "twopass",
                                                           args.steps, args.warmup, world, rank, clocks=True)
        alg_r = algorithmic_bytes(kr, nr, nnz_r, r_nnz, 4)
        extra[RMAT_WORKLOAD] = {
            "value": world * nnz_r / r_step, "unit": "nnz/s", "ms_per_step": r_step * 1e3, "steps": args.steps,
            "warmup": args.warmup, "dtype": "f32",
            "config": {"workload": RMAT_WORKLOAD, "k": kr, "m": mr, "n": nr, "nnz_in": nnz_r, "nnz_out": r_nnz,
                       "cf": nnz_r / max(r_nnz, 1)},
            "hbm_gbs_step": alg_r / r_step / 1e9,
            "roofline": {"kernel": kernel_label(r_info, "twopass"), "bound": "hbm",
                         "achieved": alg_r / (r_kern / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg_r / (r_kern / 1e3) / 1e9 / peak, "peak_source": peak_src, "traffic": None,
                         "algorithmic_bytes": alg_r, "launch_ms": r_kern, "step_frac": alg_r / r_step / 1e9 / peak},
            "cpu_baseline": (cpu_baseline_of(R, args.oracle_cols // 4) if rank == 0 and world == 1
                             and args.oracle_cols > 0 else None),
            "clocks": r_clk, "gpu_launches": r_info["kernel_launches"] * args.steps,
            "classes": {x: r_info[x] for x in ("cols_warp", "cols_cta", "cols_heavy", "windows", "windows_split")},
        }
        del R
        torch.cuda.empty_cache()

    if rank != 0:
        return
    achieved = alg / (kern_ms / 1e3) / 1e9
    step_gbs = alg / t_step / 1e9
    out = {
        "metric": METRIC, "value": world * nnz_in / t_step, "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if vbytes == 8 else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "k": k, "m": m, "n": n, "nnz_in": nnz_in, "nnz_out": nnz_out,
                   "cf": nnz_in / max(nnz_out, 1), "l2": "inputs exceed the 129 MB L2; no flush between steps",
                   "parallelism": f"{world} independent instance(s), one per GPU", "seed": args.seed,
                   "method": args.method,
                   "input_order": "rows shuffled inside columns" if args.unordered else "sorted",
                   "output_order": "any order inside a column" if args.unsorted_output else "sorted",
                   "block_accumulator": ("automatic", "flat bitmap", "compact word table")[args.block_accumulator]},
        "hbm_gbs_step": step_gbs,
        "roofline": {"kernel": kernel_label(info, args.method), "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                     "traffic": read_traffic(args.workload), "algorithmic_bytes": alg,
                     "launch_ms": kern_ms, "step_frac": step_gbs / peak},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
        "classes": {x: info[x] for x in ("cols_warp", "cols_cta", "cols_heavy", "windows", "windows_split",
                                         "cols_unique")},
    }
    if other:
        out["other_method"] = other
    if tree:
        out["pairwise_tree"] = tree
    out.update(extra)
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Batched workload: 4096 independent instances (k log-uniform on [2, 256],
# m = n log-uniform on [2^10, 2^16], per-column length L_j uniform on
# [4, 64], half ER / half SpGEMM-like, dtype fp32 or fp64 with probability
# 1/2, seed 0).  About 1.1e11 input nonzeros in total: more than HBM holds,
# so instances run in seed order as memory-sized waves, each wave one batch
# (one set of launches for all its instances).  Compared with one spkadd
# call per instance on the same inputs.
# ---------------------------------------------------------------------------
BATCH_WORKLOAD = "batch4096_k2-256_mn2p10-2p16_L4-64"


def _instance_bytes(p):
    import synth

    sv = 8 if p["dtype"] == torch.float64 else 4
    nz = synth.instance_nnz_estimate(p)
    n = p.get("n", p["m"])
    return 2 * nz * (4 + sv) + 96 * n + 64 * p["k"]  # inputs, B (<= inputs), workspace


def plan_waves(params, budget):
    waves, cur, used = [], [], 0
    for q, p in enumerate(params):
        b = _instance_bytes(p)
        if cur and used + b > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(q)
        used += b
    if cur:
        waves.append(cur)
    return waves


def _descriptors(probs):
    """Flat descriptor arrays of instances whose k inputs are rows of one (k, tot) buffer each."""
    import numpy as np

    ks, ms, ns, nnz, cps, ris, vas, dts = [], [], [], [], [], [], [], []
    for A, m in probs:
        k = len(A)
        cp, ri, va = A[0]
        tot = ri.numel()
        ks.append(k)
        ms.append(m)
        ns.append(cp.numel() - 1)
        dts.append(va.dtype)
        nnz.append(np.full(k, tot, dtype=np.int64))
        cps.append(np.full(k, cp.data_ptr(), dtype=np.uint64))
        ris.append(np.uint64(ri.data_ptr()) + np.arange(k, dtype=np.uint64) * np.uint64(tot * 4))
        vas.append(np.uint64(va.data_ptr()) + np.arange(k, dtype=np.uint64) * np.uint64(tot * va.element_size()))
    cat = np.concatenate
    return dict(k=np.asarray(ks, dtype=np.int32), m=np.asarray(ms), n=np.asarray(ns), nnz=cat(nnz), cp=cat(cps),
                ri=cat(ris), va=cat(vas), dtypes=dts)


def batch_once(spk, desc, dev, stream, options=None):
    """One batch: plan, symbolic, one flat allocation per output array, numeric, destroy."""
    import numpy as np

    h = spk.spkadd_batch_plan_raw(desc["k"], desc["m"], desc["n"], desc["nnz"], desc["cp"], desc["ri"], desc["va"],
                                  desc["dtypes"], stream=stream, options=options)
    nnz = np.asarray(spk.spkadd_batch_symbolic(h), dtype=np.int64)
    n1 = desc["n"].astype(np.int64) + 1
    is64 = np.asarray([d == torch.float64 for d in desc["dtypes"]])
    cp = torch.empty(int(n1.sum()), dtype=torch.int64, device=dev)
    ri = torch.empty(max(int(nnz.sum()), 1), dtype=torch.int32, device=dev)
    v64 = torch.empty(max(int(nnz[is64].sum()), 1), dtype=torch.float64, device=dev)
    v32 = torch.empty(max(int(nnz[~is64].sum()), 1), dtype=torch.float32, device=dev)

    def offs(sizes):
        o = np.zeros(sizes.size, dtype=np.uint64)
        o[1:] = np.cumsum(sizes[:-1]).astype(np.uint64)
        return o

    a_cp = np.uint64(cp.data_ptr()) + offs(n1) * np.uint64(8)
    a_ri = np.uint64(ri.data_ptr()) + offs(nnz) * np.uint64(4)
    a_va = np.zeros(nnz.size, dtype=np.uint64)
    a_va[is64] = np.uint64(v64.data_ptr()) + offs(nnz[is64]) * np.uint64(8)
    a_va[~is64] = np.uint64(v32.data_ptr()) + offs(nnz[~is64]) * np.uint64(4)
    spk.spkadd_batch_numeric_raw(h, a_cp, a_ri, a_va)
    info = spk.spkadd_get_info(h)
    spk.spkadd_destroy(h)
    return (cp, ri, v64, v32, nnz, a_cp, a_ri, a_va), info


def run_batch(args, world, rank, local):
    import numpy as np

    import paper_2112_10223_gb300 as spk
    import synth

    spk.library()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    params = synth.batch_instance_params(args.batch_count, seed=args.seed + rank)
    est = np.asarray([synth.instance_nnz_estimate(p) for p in params], dtype=np.float64)
    edges = np.quantile(est, np.linspace(0, 1, 11))
    decile = np.clip(np.searchsorted(edges, est, side="right") - 1, 0, 9)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * args.batch_mem_frac)
    waves = plan_waves(params, budget)

    tot = dict(nnz=0, bytes=0, t_batch=0.0, t_req=0.0, launches=0, instances=0)
    dec = [dict(instances=0, nnz=0, t_batch=0.0, t_req=0.0) for _ in range(10)]
    lat_req = []
    tuned = None
    tune_log = []
    wave_log = []
    verified = 0
    oracle_nnz, oracle_t, oracle_cores = 0, 0.0, 0
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    for wi, wave in enumerate(waves):
        probs = [synth.instance(params[q], device=dev) for q in wave]
        torch.cuda.synchronize()
        desc = _descriptors(probs)
        nnz_in = np.asarray([len(A) * A[0][1].numel() for A, _ in probs], dtype=np.int64)
        if tuned is None:  # the library's autotuner picks the options on the first wave
            from paper_2112_10223_gb300 import autotune

            cache = args.autotune_cache or os.path.join(tempfile.mkdtemp(), "autotune.json")
            tuner = autotune.Autotuner(cache_path=cache)
            t0 = time.perf_counter()
            opt = autotune.tune_batch(desc, device=dev, tuner=tuner, repeats=1)
            tune_s = time.perf_counter() - t0
            tuned = {f: int(getattr(opt, f)) for f in autotune.DEFAULTS}
            rec = tuner.last
            tune_log = {"chosen": tuned, "tuning_s": tune_s, "cached": rec["cached"],
                        "timed_candidates": rec["timed"], "candidates": rec["candidates"]}
        opt = spk.default_options(**tuned)
        for _ in range(args.warmup):
            batch_once(spk, desc, dev, stream, opt)
        torch.cuda.synchronize()
        tb = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            res, info = batch_once(spk, desc, dev, stream, opt)
            torch.cuda.synchronize()
            tb.append(time.perf_counter() - t0)
        t_batch = sum(tb) / len(tb)
        nnz_out = res[4]
        tot["launches"] += info["kernel_launches"] * args.steps
        # per-size-decile batches
        for d in range(10):
            sel = [i for i, q in enumerate(wave) if decile[q] == d]
            if not sel:
                continue
            sub = _descriptors([probs[i] for i in sel])
            batch_once(spk, sub, dev, stream, opt)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch_once(spk, sub, dev, stream, opt)
            torch.cuda.synchronize()
            dec[d]["t_batch"] += time.perf_counter() - t0
        # one call per instance, in seed order, each waited for
        spk.spkadd(probs[0][0], probs[0][1])
        torch.cuda.synchronize()
        t_req_wave = 0.0
        for i, (A, m) in enumerate(probs):
            t0 = time.perf_counter()
            spk.spkadd(A, m, options=opt)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            lat_req.append(t)
            tot["t_req"] += t
            t_req_wave += t
            q = wave[i]
            dec[decile[q]]["t_req"] += t
            dec[decile[q]]["instances"] += 1
            dec[decile[q]]["nnz"] += int(nnz_in[i])
        wave_log.append({"wave": wi, "instances": len(wave), "first_instance": wave[0], "nnz_in": int(nnz_in.sum()),
                         "batch_ms": t_batch * 1e3, "per_request_ms": t_req_wave * 1e3,
                         "nnz_per_s": float(nnz_in.sum()) / t_batch, "speedup": t_req_wave / t_batch})
        # verification of a few instances against the oracle (not timed)
        if rank == 0 and args.batch_verify > 0:
            import oracle

            # a size-stratified sample: instances evenly spaced in the wave's size order
            by_size = sorted(range(len(wave)), key=lambda i: nnz_in[i])
            nv = min(args.batch_verify, len(by_size))
            picks = sorted({by_size[round(q * (len(by_size) - 1) / max(nv - 1, 1))] for q in range(nv)})
            cp_all, ri_all, v64, v32 = res[0], res[1], res[2], res[3]
            for i in picks:
                A, m = probs[i]
                An = [tuple(t.cpu().numpy() for t in a) for a in A]
                t0 = time.perf_counter()
                want = oracle.add(An)
                oracle_t += time.perf_counter() - t0
                oracle_nnz += int(nnz_in[i])
                oracle_cores = oracle.threads_used(0)
                n = desc["n"][i]
                o_cp = int((res[5][i] - np.uint64(cp_all.data_ptr())) // np.uint64(8))
                o_ri = int((res[6][i] - np.uint64(ri_all.data_ptr())) // np.uint64(4))
                vbuf = v64 if A[0][2].dtype == torch.float64 else v32
                o_va = int((res[7][i] - np.uint64(vbuf.data_ptr())) // np.uint64(vbuf.element_size()))
                nz = int(nnz_out[i])
                got_cp = cp_all[o_cp:o_cp + n + 1].cpu().numpy()
                got_ri = ri_all[o_ri:o_ri + nz].cpu().numpy()
                got_va = vbuf[o_va:o_va + nz].cpu().numpy().astype(np.float64)
                tol = 1e-12 if A[0][2].dtype == torch.float64 else 1e-5
                ok = (np.array_equal(got_cp, want["col_ptr"]) and np.array_equal(got_ri, want["row_idx"])
                      and bool(np.all(np.abs(got_va - want["val"]) <= tol * want["abs_sum"])))
                if not ok:
                    raise SystemExit(f"batch parity failed for instance {wave[i]}")
                verified += 1
        alg = 0
        for i, (A, m) in enumerate(probs):
            sv = A[0][2].element_size()
            n = A[0][0].numel() - 1
            alg += algorithmic_bytes(len(A), n, int(nnz_in[i]), int(nnz_out[i]), sv)
        tot["nnz"] += int(nnz_in.sum())
        tot["bytes"] += alg
        tot["t_batch"] += t_batch
        tot["instances"] += len(wave)
        del probs, desc, res
        torch.cuda.empty_cache()
    clk = clocks.stop() if clocks else None
    if rank != 0:
        return
    peak, peak_src = read_peaks()
    achieved = tot["bytes"] / tot["t_batch"] / 1e9
    lat = sorted(lat_req)
    out = {
        "metric": METRIC, "value": tot["nnz"] / tot["t_batch"], "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot["t_batch"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "instances": tot["instances"], "nnz_in": tot["nnz"],
                   "waves": len(waves), "wave_budget_bytes": budget, "seed": args.seed,
                   "l2": "every wave's inputs exceed the 129 MB L2; no flush"},
        "roofline": {"kernel": "whole batch (all phases)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
                     "algorithmic_bytes": tot["bytes"]},
        "batch": {
            "autotune": tune_log,
            "instances_per_s": tot["instances"] / tot["t_batch"],
            "per_request": {"nnz_per_s": tot["nnz"] / tot["t_req"], "instances_per_s": tot["instances"] / tot["t_req"],
                            "seconds": tot["t_req"], "p50_ms": lat[len(lat) // 2] * 1e3,
                            "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3},
            "speedup_vs_per_request": tot["t_req"] / tot["t_batch"],
            "deciles": [{"decile": d, "instances": x["instances"], "nnz_in": x["nnz"],
                         "batch_ms": x["t_batch"] * 1e3, "per_request_ms": x["t_req"] * 1e3,
                         "speedup": (x["t_req"] / x["t_batch"]) if x["t_batch"] > 0 else None}
                        for d, x in enumerate(dec)],
            "verified_instances": verified,
            "waves": wave_log,
            # Wave 0 is the longest seed-order prefix of the instances whose
            # inputs fit one wave's budget, run as one batch (one set of launches).
            "prefix_single_launch": wave_log[0] if wave_log else None,
        },
        "cpu_baseline": ({"value": oracle_nnz / oracle_t, "unit": "nnz/s", "cores": oracle_cores, "kind": "oracle",
                          "sample": f"{verified} verified instances, {oracle_nnz} input nnz, {oracle_t:.2f} s"}
                         if oracle_t > 0 else None),
        "e2e": None,
        "clocks": clk,
        "gpu_launches": tot["launches"],
    }
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Served workload: Poisson arrivals of requests drawn like the batched workload
# but with k log-uniform on [2, 512] and m = n log-uniform on [2^10, 2^18].
# The inputs of every request stay on the device before it arrives, and all
# requests of the full stream (about 2.9e12 input nonzeros) do not fit HBM,
# so requests reuse the inputs of a pool: the longest prefix of the seeded
# stream whose inputs fit the pool budget.  Request r computes the sum of pool
# entry r mod G.  The capacity C (requests/s) is the pool run as one burst; the
# trace runs at fractions of C, with continuous batching and with one batch
# per request, and every request's output digest is checked against the same
# problem computed alone.
# ---------------------------------------------------------------------------
SERVE_WORKLOAD = "serve_k2-512_mn2p10-2p18_L4-64"


def run_serve(args, world, rank, local):
    import numpy as np

    import paper_2112_10223_gb300 as spk
    import synth
    from paper_2112_10223_gb300.serve import Request, Server, output_digest

    spk.library()
    if rank != 0:
        return
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    params = synth.batch_instance_params(args.serve_requests, seed=args.seed, k_range=(2, 512),
                                         mn_range=(1 << 10, 1 << 18))
    free, _ = torch.cuda.mem_get_info()
    pool_budget = int(free * args.serve_pool_frac)
    pool, used = [], 0
    for q, p in enumerate(params):  # the longest seed-order prefix that fits: an unbiased sample
        if len(pool) >= args.serve_pool_max:
            break
        b = synth.instance_nnz_estimate(p) * (4 + (8 if p["dtype"] == torch.float64 else 4))
        if used + b > pool_budget:
            break
        A, m = synth.instance(p, device=dev)
        pool.append((A, m, q))
        used += sum(a[1].numel() * (4 + a[2].element_size()) for a in A) + A[0][0].numel() * 4
    torch.cuda.synchronize()
    G = len(pool)
    pool_nnz = [sum(a[1].numel() for a in A) for A, _, _ in pool]
    # Alone results of every pool entry (digest only).
    alone = []
    for A, m, _ in pool:
        alone.append(output_digest(spk.spkadd(A, m)))
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.8)

    def trace(rate, count, seed):
        rng = np.random.default_rng(seed)
        t = np.cumsum(rng.exponential(1.0 / rate, size=count)) if rate > 0 else np.zeros(count)
        return [Request(r, pool[r % G][0], pool[r % G][1], arrival=float(t[r]), tag=r % G) for r in range(count)]

    # Capacity: the pool as one burst (all arrive at 0), after one warm-up burst.
    Server(dev, budget).run(trace(0, G, 1))
    burst = Server(dev, budget).run(trace(0, G, 1))
    cap = G / burst.seconds
    burst1 = Server(dev, budget, batching=False).run(trace(0, G, 1))
    cap1 = G / burst1.seconds

    results = []
    R = args.serve_requests
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for frac in args.serve_rates:
        rate = frac * cap
        st_b = Server(dev, budget).run(trace(rate, R, 100 + int(frac * 100)))
        st_1 = Server(dev, budget, batching=False).run(trace(rate, R, 100 + int(frac * 100)))
        results.append({"load": frac, "rate_per_s": rate, "batched": st_b.summary(), "per_request": st_1.summary()})
    clk = clocks.stop()

    # Alone vs mix: every request of a trace at the highest load, digests compared.
    bad = []
    tol = {torch.float64: 1e-12, torch.float32: 1e-5}

    def check(r):
        d = output_digest(r.out)
        a = alone[r.tag]
        scale = max(a[3], 1e-300)
        if d[0] != a[0] or d[1] != a[1] or abs(d[2] - a[2]) > tol[r.dtype] * max(scale, 1.0) * 4:
            bad.append(r.rid)

    vr = max(args.serve_rates) * cap
    Server(dev, budget, on_done=check).run(trace(vr, R, 999))
    if bad:
        raise SystemExit(f"alone-vs-mix digest mismatch for requests {bad[:10]}")

    hi = results[-1]
    out = {
        "metric": METRIC, "value": hi["batched"]["nnz_per_s"], "unit": "nnz/s", "n_gpus": world,
        "steps": len(args.serve_rates), "warmup": 1, "ms_per_step": hi["batched"]["seconds"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "requests_per_trace": R, "pool_instances": G,
                   "pool_input_nnz": int(sum(pool_nnz)),
                   "pool_budget_bytes": pool_budget, "serve_budget_bytes": budget, "seed": args.seed},
        "serve": {"capacity_req_per_s": cap, "capacity_per_request_req_per_s": cap1,
                  "burst_batches": burst.batches, "loads": results,
                  "alone_vs_mix": {"requests": R, "load": max(args.serve_rates), "mismatches": len(bad)}},
        "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
        "gpu_launches": None,
    }
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Streamed workload: partial products arriving in batches (sparse SUMMA's
# stage results, Sec. IV; inputs added batch by batch, Sec. V).  k = 64
# SpGEMM-like inputs of 2^18 x 2^18 with 32 rows per column (fp32) are added
# into a running sum 8 at a time (one 9-way SpKAdd per batch), against the
# one-shot 64-way sum and fully pairwise accumulation on the same inputs.
# ---------------------------------------------------------------------------
STREAM_WORKLOAD = "stream_spgemm_k64_g8_m2p18_L32_f32"


def run_stream(args, world, rank, local):
    import paper_2112_10223_gb300 as spk
    import synth

    spk.library()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    k, m, L, G = 64, 1 << 18, 32, 8
    dtype, vbytes = torch.float32, 4
    A = synth.spgemm_like(k, m, m, L, seed=args.seed + rank, dtype=dtype, device=dev)
    n = m
    nnz_in = sum(a[1].numel() for a in A)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def streamed(group):
        s = spk.SpkaddStream(m, n, dtype=dtype, stream=stream)
        nnz_b = [0]
        for i in range(0, k, group):
            nnz_b.append(s.add(A[i:i + group]))
        out = s.result()
        q = s.query()
        s.close()
        return out, nnz_b, q["kernel_launches"]

    def timed(fn, steps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            res = fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return reduce_max(t0.elapsed_time(t1) / 1e3 / steps, world), res

    for _ in range(max(args.warmup, 1)):
        streamed(G)
        spk.spkadd(A, m)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t_stream, (out_s, nnz_b, launches) = timed(lambda: streamed(G), args.steps)
    clk = clocks.stop() if clocks else None
    t_one, out_1 = timed(lambda: spk.spkadd(A, m), args.steps)
    t_pair, (out_p, _, _) = timed(lambda: streamed(1), 1)
    # The streamed and pairwise sums against the one-shot sum: indices bit-exact,
    # values within the fp32 bound (each addition rounds once either way).
    absum = spk.spkadd([(a[0], a[1], a[2].abs()) for a in A], m)[2]
    for name, o in (("streamed", out_s), ("pairwise", out_p)):
        if not (torch.equal(o[0], out_1[0]) and torch.equal(o[1], out_1[1])):
            raise SystemExit(f"{name} indices differ from the one-shot sum")
        if bool(((o[2].double() - out_1[2].double()).abs() > 2e-5 * absum.double()).any()):
            raise SystemExit(f"{name} values outside tolerance of the one-shot sum")
    nnz_out = int(out_1[1].numel())
    # Algorithmic bytes of the streamed step: every add reads its inputs and the
    # running sum once and writes the new sum once; the result is copied once.
    alg = 0
    for j, i in enumerate(range(0, k, G)):
        add_in = sum(a[1].numel() for a in A[i:i + G])
        alg += algorithmic_bytes(G + 1, n, add_in + nnz_b[j], nnz_b[j + 1], vbytes)
    alg += 2 * (nnz_out * (4 + vbytes)) + (n + 1) * (4 + 8)
    cpu = None
    if rank == 0 and world == 1 and args.oracle_cols > 0:
        sample, stride = oracle_sample(A, min(args.oracle_cols, 1 << 14))
        s_nnz, s_t, cores, runs = time_oracle(sample, min_seconds=10.0)
        cpu = {"value": s_nnz / s_t, "unit": "nnz/s", "cores": cores, "kind": "oracle",
               "sample": f"every {stride}-th column ({s_nnz} input nnz), {runs} runs of {s_t:.2f} s each"}
    if rank != 0:
        return
    peak, peak_src = read_peaks()
    achieved = alg / t_stream / 1e9
    out = {
        "metric": METRIC, "value": world * nnz_in / t_stream, "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_stream * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": STREAM_WORKLOAD, "k": k, "m": m, "n": n, "rows_per_column": L, "batches": k // G,
                   "inputs_per_batch": G, "nnz_in": nnz_in, "nnz_out": nnz_out, "seed": args.seed,
                   "l2": "inputs (4.3 GB) exceed the 129 MB L2; no flush between steps"},
        "roofline": {"kernel": "whole streamed step (all adds)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
                     "algorithmic_bytes": alg},
        "stream": {"streamed_ms": t_stream * 1e3, "one_shot_ms": t_one * 1e3, "pairwise_ms": t_pair * 1e3,
                   "streamed_over_one_shot": t_stream / t_one, "pairwise_over_one_shot": t_pair / t_one,
                   "inputs_resident": {"streamed": G, "one_shot": k, "pairwise": 1},
                   "nnz_B_after_each_add": nnz_b[1:],
                   "verified": "streamed and pairwise sums equal the one-shot sum (indices bit-exact, values "
                               "within 2e-5 of sum|terms|)"},
        "cpu_baseline": cpu,
        "e2e": None,
        "clocks": clk,
        "gpu_launches": launches * args.steps,
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [BATCH_WORKLOAD, SERVE_WORKLOAD, STREAM_WORKLOAD],
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--oracle-cols", type=int, default=1 << 20,
                    help="columns of the CPU oracle's sample (every (n / cols)-th column)")
    ap.add_argument("--info", action="store_true")
    ap.add_argument("--method", choices=["twopass", "onepass"], default="twopass",
                    help="twopass: spkadd_symbolic + spkadd_numeric; onepass: spkadd_onepass")
    ap.add_argument("--no-compare-methods", dest="compare_methods", action="store_false",
                    help="skip timing the other method on the same inputs")
    ap.add_argument("--no-pairwise-tree", dest="pairwise_tree", action="store_false",
                    help="skip timing the cuSPARSE pairwise-tree sum beside the k-way path")
    ap.add_argument("--no-extra-rmat", dest="extra_rmat", action="store_false",
                    help="skip the R-MAT line that the default workload's run adds")
    ap.add_argument("--unordered", action="store_true",
                    help="shuffle rows inside every input column and run with input_order = 1")
    ap.add_argument("--unsorted-output", action="store_true", help="run with sort_mode = 2 (B's columns unsorted)")
    ap.add_argument("--block-accumulator", type=int, default=0, choices=(0, 1, 2),
                    help="thread-block items' accumulator: 0 automatic, 1 flat bitmap, 2 compact word table")
    ap.add_argument("--batch-count", type=int, default=4096, help="instances of the batched workload")
    ap.add_argument("--batch-mem-frac", type=float, default=0.55, help="device memory share of one wave")
    ap.add_argument("--autotune-cache", default=None,
                    help="autotuner cache file (default: tune afresh into a temporary cache)")
    ap.add_argument("--batch-verify", type=int, default=32,
                    help="instances per wave checked against the oracle (evenly spaced in size order)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per served trace")
    ap.add_argument("--serve-pool-frac", type=float, default=0.3, help="device memory share of the input pool")
    ap.add_argument("--serve-pool-max", type=int, default=512, help="most distinct requests in the input pool")
    ap.add_argument("--serve-rates", type=lambda x: [float(v) for v in x.split(",")], default=[0.5, 0.7, 0.9],
                    help="loads as fractions of the measured capacity")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == BATCH_WORKLOAD:
        run_batch(args, world, rank, local)
    elif args.workload == SERVE_WORKLOAD:
        run_serve(args, world, rank, local)
    elif args.workload == STREAM_WORKLOAD:
        run_stream(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
