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
          device->host inside the timed region.
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


def time_oracle(A, threads=0, repeat=1):
    import oracle

    An = [tuple(t.numpy() for t in a) for a in A]
    oracle.add(An, threads=threads)  # warm (page faults, build)
    ts = []
    for _ in range(repeat):
        t0 = time.perf_counter()
        oracle.add(An, threads=threads)
        ts.append(time.perf_counter() - t0)
    nnz = sum(a[1].numel() for a in A)
    return nnz, min(ts), oracle.threads_used(threads)


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


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle on a bounded sample, rank 0 only."""
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    A, _ = make_inputs(w, dev, seed=args.seed)
    S, stride = oracle_sample(A, args.oracle_cols)
    del A
    nnz = sum(a[1].numel() for a in S)
    for _ in range(args.warmup):
        time_oracle(S, repeat=1)
    ts = []
    cores = 1
    for _ in range(args.steps):
        _, t, cores = time_oracle(S, repeat=1)
        ts.append(t)
    t = sum(ts) / len(ts)
    val = nnz / t
    sample = f"every {stride}-th column of the workload: {len(S[0][0]) - 1} columns, {nnz} input nnz per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w["dtype"] == torch.float64 else "f32",
        "data": "synthetic", "config": {"workload": args.workload},
        "cpu_baseline": {"value": val, "unit": "nnz/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args, world, rank, local):
    import paper_2112_10223_gb300 as spk

    spk.library()  # fails loudly if the CUDA library was not built
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    w = WORKLOADS[args.workload]
    A, m = make_inputs(w, dev, seed=args.seed + rank)
    k = len(A)
    n = A[0][0].numel() - 1
    vbytes = 8 if w["dtype"] == torch.float64 else 4
    nnz_in = sum(a[1].numel() for a in A)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def step(ev=None):
        h = spk.spkadd_plan(A, m, stream=stream)
        nnz = spk.spkadd_symbolic(h)
        cp = torch.empty(n + 1, dtype=torch.int64, device=dev)
        ri = torch.empty(nnz, dtype=torch.int32, device=dev)
        va = torch.empty(nnz, dtype=w["dtype"], device=dev)
        if ev is not None:
            ev[0].record(stream)
        spk.spkadd_numeric(h, cp, ri, va)
        if ev is not None:
            ev[1].record(stream)
        info = spk.spkadd_get_info(h) if args.info else None
        spk.spkadd_destroy(h)
        return nnz, info

    nnz_out, info = None, None
    for _ in range(max(args.warmup, 1)):
        nnz_out, _ = step()
    # launches per step, from one untimed step
    h = spk.spkadd_plan(A, m, stream=stream)
    spk.spkadd_symbolic(h)
    cp0 = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ri0 = torch.empty(nnz_out, dtype=torch.int32, device=dev)
    va0 = torch.empty(nnz_out, dtype=w["dtype"], device=dev)
    spk.spkadd_numeric(h, cp0, ri0, va0)
    info = spk.spkadd_get_info(h)
    spk.spkadd_destroy(h)
    del cp0, ri0, va0
    launches_per_step = info["kernel_launches"]

    num_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(num_events[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    barrier(world)
    elapsed = reduce_max(t_start.elapsed_time(t_end) / 1e3, world)
    num_ms = [a.elapsed_time(b) for a, b in num_events]
    num_avg = reduce_max(sum(num_ms) / len(num_ms), world)

    cpu_sample, cpu_stride = (oracle_sample(A, args.oracle_cols) if rank == 0 and world == 1
                              and args.oracle_cols > 0 else (None, None))
    # e2e: host buffers through the same C ABI, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        host = [tuple(t.cpu().pin_memory() for t in a) for a in A]
        h2d = sum(t.numel() * t.element_size() for a in host for t in a)
        out_cp = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
        out_ri = torch.empty(nnz_out, dtype=torch.int32, pin_memory=True)
        out_va = torch.empty(nnz_out, dtype=w["dtype"], pin_memory=True)
        d2h = (n + 1) * 8 + nnz_out * (4 + vbytes)

        def e2e_step():
            Ad = [tuple(t.to(dev, non_blocking=True) for t in a) for a in host]
            hh = spk.spkadd_plan(Ad, m, stream=stream)
            nz = spk.spkadd_symbolic(hh)
            cp = torch.empty(n + 1, dtype=torch.int64, device=dev)
            ri = torch.empty(nz, dtype=torch.int32, device=dev)
            va = torch.empty(nz, dtype=w["dtype"], device=dev)
            spk.spkadd_numeric(hh, cp, ri, va)
            out_cp.copy_(cp, non_blocking=True)
            out_ri[:nz].copy_(ri, non_blocking=True)
            out_va[:nz].copy_(va, non_blocking=True)
            spk.spkadd_destroy(hh)
            del Ad

        del A
        torch.cuda.empty_cache()
        e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        te = reduce_max(time.perf_counter() - t0, world)
        e2e = {"value": world * nnz_in * args.e2e_steps / te, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}
    else:
        del A

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and args.oracle_cols > 0:
        S = cpu_sample
        nz_s, t_s, cores = time_oracle(S)
        cpu = {"value": nz_s / t_s, "unit": "nnz/s", "cores": cores, "kind": "oracle",
               "sample": f"every {cpu_stride}-th column of the workload: {len(S[0][0]) - 1} columns, "
                         f"{nz_s} input nnz, {t_s:.2f} s"}

    if rank != 0:
        return
    peak, peak_src = read_peaks()
    alg = algorithmic_bytes(k, n, nnz_in, nnz_out, vbytes)
    achieved = alg / (num_avg / 1e3) / 1e9
    step_gbs = alg / (elapsed / args.steps) / 1e9
    out = {
        "metric": METRIC, "value": world * nnz_in * args.steps / elapsed, "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if vbytes == 8 else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "k": k, "m": m, "n": n, "nnz_in": nnz_in, "nnz_out": nnz_out,
                   "cf": nnz_in / max(nnz_out, 1), "l2": "inputs exceed the 129 MB L2; no flush between steps",
                   "parallelism": f"{world} independent instance(s), one per GPU", "seed": args.seed},
        "hbm_gbs_step": step_gbs,
        "roofline": {"kernel": "k_warp_col<numeric> (spkadd_numeric)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                     "traffic": read_traffic(args.workload), "algorithmic_bytes": alg,
                     "launch_ms": num_avg, "step_frac": step_gbs / peak},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
        "classes": {x: info[x] for x in ("cols_warp", "cols_cta", "cols_heavy", "windows", "windows_split",
                                         "cols_unique")},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--oracle-cols", type=int, default=1 << 19)
    ap.add_argument("--info", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
