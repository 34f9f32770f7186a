#!/usr/bin/env python3
"""Benchmark: half-stored M-scheme Hamiltonian nonzeros built per second.

One step = the whole construction path on one synthetic workload: basis
enumeration (sub-determinants, partner ranges, neighbour lists), the count
pass, the row-pointer scan and the fill pass (columns and values), with the
two-body table already resident in HBM.  value = nonzeros of all ranks'
steps / device time of those steps.  L2 is flushed (a 256 MiB write) between
timed steps.

Default workload: 4 protons + 4 neutrons, Nmax = 6, 2M = 0, one seeded
synthetic two-body table (PCG64 seed 0, N(0,1) float32 per entry): dimension
2,217,754, 924,863,410 stored nonzeros.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank builds the same workload on its own GPU
(replicas, weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hamiltonian nonzeros built/sec (% HBM roofline); gradient/forward time ratio"
WORKLOADS = {
    "4p4n_nmax6": dict(Z=4, N=4, Nmax=6, twoM=0, seed=0),
    "3p3n_nmax6": dict(Z=3, N=3, Nmax=6, twoM=0, seed=100),
    "4p4n_nmax4": dict(Z=4, N=4, Nmax=4, twoM=0, seed=0),
    "3p3n_nmax2": dict(Z=3, N=3, Nmax=2, twoM=0, seed=0),
    "3p4n_nmax4": dict(Z=3, N=4, Nmax=4, twoM=1, seed=0),   # 8.0 M stored nonzeros: mid-size ncu captures
}
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_NNZ = 8            # int32 column + float32 value written by the fill


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="4p4n_nmax6", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched-fill and Lanczos side measurements")
    ap.add_argument("--extra", choices=["all", "batched", "lanczos"], default="all",
                    help="which side measurements to run (default all)")
    ap.add_argument("--sets", type=int, default=1,
                    help="K two-body tables (seeds seed..seed+K-1); K > 1 times the batched fill "
                         "(interleaved tables, element-major values)")
    ap.add_argument("--cpu-rows", type=int, default=60000, help="rows in the oracle's timed sample")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun, every rank builds the whole matrix (default: each rank fills its "
                         "row shard of about equal nonzeros)")
    return ap.parse_args()


def workload_name(w):
    return f"{w['Z']}p{w['N']}n_nmax{w['Nmax']}_2M{w['twoM']}_plain_build_seed{w['seed']}"


# ---------------------------------------------------------------- helpers

def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def write_only_gbs(dev, st, nbytes=4 << 30, reps=5):
    """Write-only streaming bandwidth of this GPU, the second roofline
    denominator next to the measured copy: a float32 fill of a buffer larger
    than L2 (16-byte stores), CUDA events on the launching stream, best of
    `reps`.  Measurement only; no part of the construction path."""
    import torch
    buf = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
    buf.fill_(0.0)
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        buf.fill_(1.0)
        b.record(st)
        torch.cuda.synchronize()
        best = max(best, buf.numel() * 4 / (a.elapsed_time(b) * 1e-3) / 1e9)
    del buf
    torch.cuda.empty_cache()
    return best


def fill_traffic(fill_source_sha):
    """DRAM bytes per fill launch from the committed ncu summary, if it was taken
    on the current fill kernel (same source hash); else None."""
    p = os.path.join(ROOT, "profiles", "fill_4p4n_nmax6.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != fill_source_sha:
        return None
    return float(m.group(1))


def kernel_source_sha():
    """Hash of what the fill kernel compiles from -- ham.cu, ham_common.cuh and
    the device structs it reads (DevSpecies, DevBasis) -- with comments and
    blank space removed, so that only a change of that code invalidates a
    recorded capture."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1412_5989_gb300", "csrc")
    parts = [open(os.path.join(csrc, f)).read() for f in ("ham.cu", "ham_common.cuh")]
    hdr = open(os.path.join(csrc, "cih_internal.h")).read()
    parts += re.findall(r"struct (?:DevSpecies|DevBasis) \{.*?\n\};", hdr, flags=re.S)
    for src in parts:
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rate(w, rows_n, seed=1):
    """The CPU oracle, as it stands, on a bounded sample of rows of the same
    workload: (nnz/s, nnz in sample, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_1412_5989_gb300 import synth
    S = oracle.Space(w["Z"], w["N"], w["Nmax"], w["twoM"])
    t = synth.tbme_table(S.tbme_len, w["seed"])
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(S.dim, size=min(rows_n, S.dim), replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    cnt, off, col, val = S.rows(rows, t)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return float(cnt.sum()) / dt, int(cnt.sum()), dt, threads, len(rows)


def oracle_rate_one_thread(workload, rows_n, seed=2, timeout=900):
    """The same oracle sample on one host thread: a child process started with
    OMP_NUM_THREADS=1 (the OpenMP runtime reads it once per process).  Returns
    (nnz/s, nnz in sample, seconds, threads)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r, n, dt, th, rows = bench.oracle_rate(bench.WORKLOADS[%r], %d, seed=%d); "
            "print(json.dumps([r, n, dt, th]))") % (ROOT, workload, rows_n, seed)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=timeout, check=True)
    r, n, dt, th = json.loads(out.stdout.strip().splitlines()[-1])
    return float(r), int(n), float(dt), int(th)


def max_over_ranks(x, world, device=None):
    """The largest value of x over the ranks (replicas report the slowest)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_step, total_ms):
    """Units all ranks processed per second: each replica runs `steps` steps of
    `units_per_step` units; the job takes the slowest rank's time."""
    return world * steps * units_per_step / (total_ms * 1e-3)


def sharded_rate(steps, units_total, total_ms):
    """Units per second when the ranks split one matrix: each step builds
    `units_total` units between them; the job takes the slowest rank's time."""
    return steps * units_total / (total_ms * 1e-3)


def rank_rows(rowptr_host, world, rank):
    """This rank's rows of a row-sharded build: shards of about equal stored
    nonzeros (cih_shard_rows).  Returns (r0, r1, nonzeros in the shard)."""
    from paper_1412_5989_gb300 import cih
    b = cih.shard_bounds(rowptr_host, world)
    r0, r1 = int(b[rank]), int(b[rank + 1])
    return r0, r1, int(rowptr_host[r1]) - int(rowptr_host[r0])


def side_measurements(args, dev, st, flush, peak, cih, synth, sp, rowptr, col, val, nnz):
    """Measurements beside the headline (not part of `value`): the batched fill
    (4+4 Nmax=4, K=64 tables, element-major values) and Lanczos iterations on
    the step's matrix.  CUDA events on the launching stream, L2 flushed."""
    import torch

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {}
    if args.extra in ("all", "batched"):
        out.update(batched_fill_measurement(dev, st, peak, cih, synth, timed))
    if args.extra in ("all", "lanczos"):
        out.update(lanczos_measurement(args, dev, st, cih, synth, sp, rowptr, col, val, nnz))
    return out


def batched_fill_measurement(dev, st, peak, cih, synth, timed):
    """4+4 Nmax=4, K = 64 tables: the batched fill and Lanczos on the 64 matrices."""
    import torch
    out = {}
    K = 64
    Bk = cih.Basis(4, 4, 4, 0)
    T = torch.from_numpy(synth.tbme_tables(Bk.tbme_len, range(K))).to(dev)
    til = cih.tbme_interleave(T)
    rp4, n4 = Bk.count()
    c4 = torch.empty(n4, dtype=torch.int32, device=dev)
    v4 = torch.empty((n4, K), dtype=torch.float32, device=dev)
    ms = timed(lambda: Bk.fill_batched(rp4, n4, til, K, col=c4, val=v4))
    Bk.check()
    gbs = n4 * (4 + 4 * K) / (ms * 1e-3) / 1e9
    out["batched_fill"] = {"workload": "4p4n_nmax4_2M0_K64_seeds0-63", "layout": "interleaved tables, element-major values",
                           "nnz_half": n4, "sets": K, "fill_ms": ms, "values_per_s": n4 * K / (ms * 1e-3),
                           "achieved_gbs": gbs, "frac_of_hbm_peak": gbs / peak}
    def lanczos_k(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        Bk.lanczos(rp4, c4, v4, nev=1, max_iter=iters, tol=1e-300, want_vectors=False, element_major=True)
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    lanczos_k(2)
    t1, t11 = lanczos_k(1), lanczos_k(11)
    out["batched_fill"]["lanczos_64_sets"] = {"setup_ms": t1, "ms_per_iteration": (t11 - t1) / 10}
    del c4, v4, T, til
    Bk.close()
    return out


def lanczos_measurement(args, dev, st, cih, synth, sp, rowptr, col, val, nnz):
    """Lanczos on the step's matrix: a fixed number of iterations (no convergence test passes)."""
    import torch
    out = {}
    Bl = cih.Basis(*sp)
    Bl.count_into(rowptr)
    Bl.fill(rowptr, nnz, torch.from_numpy(synth.tbme_table(Bl.tbme_len, 0)).to(dev), col=col, val=val)
    def lanczos_ms(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        Bl.lanczos(rowptr, col[:nnz], val[:, :nnz], nev=1, max_iter=iters, tol=1e-300, want_vectors=False)
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    lanczos_ms(2)
    t1, t41 = lanczos_ms(1), lanczos_ms(41)
    out["lanczos"] = {"workload": args.workload, "setup_ms": t1, "ms_per_iteration": (t41 - t1) / 40,
                      "note": "40 further iterations (one product reading each stored nonzero once, two "
                              "Gram-Schmidt passes, host tridiagonal step) after a one-iteration call"}
    # the product alone through its entry point (cih_ham_spmv): the bound pass
    # (values, 4 B per nonzero) and the product (column + value, 8 B per
    # nonzero), x read and y written once
    g = torch.Generator().manual_seed(10)
    x = torch.randn(Bl.dim, dtype=torch.float64, generator=g)
    x = (x / torch.linalg.vector_norm(x)).to(dev)
    v1 = val[:, :nnz]
    Bl.spmv(rowptr, col[:nnz], v1, x)
    reps = 5
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        Bl.spmv(rowptr, col[:nnz], v1, x)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    byts = 12 * nnz + 16 * Bl.dim
    out["lanczos"]["spmv_call"] = {"ms": ms, "algorithmic_bytes": byts, "achieved_gbs": byts / (ms * 1e-3) / 1e9,
                                   "note": "L2 not flushed between the 5 calls; the matrix (8 B per nonzero) "
                                           "is far larger than L2"}
    Bl.close()
    return out


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank):
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_rate(w, max(50, args.cpu_rows // 20))
    rates, times, nnzs = [], [], 0
    threads = rows = 0
    for k in range(args.steps):
        r, n, dt, threads, rows = oracle_rate(w, args.cpu_rows // 4, seed=10 + k)
        rates.append(r)
        times.append(dt)
        nnzs += n
    value = nnzs / sum(times)
    sample = (f"{rows} random rows per step (of {args.workload}), count + fill by the oracle's plain "
              f"row walk, OpenMP over rows")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": workload_name(w), "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1412_5989_gb300 import cih, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    w = WORKLOADS[args.workload]
    sp = (w["Z"], w["N"], w["Nmax"], w["twoM"])

    K = max(1, args.sets)
    B0 = cih.Basis(*sp)
    dim, tl = B0.dim, B0.tbme_len
    tbme_h = synth.tbme_table(tl, w["seed"])
    tbme = torch.from_numpy(tbme_h).to(dev)
    rowptr, nnz = B0.count()
    # under torchrun: this rank's row shard (default), or the whole matrix (replicas)
    sharded = world > 1 and not args.replicas
    if sharded and K > 1:
        raise SystemExit("the row-sharded build runs one table (--sets 1)")
    r0, r1, nnz_s = rank_rows(rowptr.cpu().numpy(), world, rank) if sharded else (0, dim, nnz)
    col = torch.empty(max(nnz_s, 1), dtype=torch.int32, device=dev)
    if K == 1:
        val = torch.empty((1, max(nnz_s, 1)), dtype=torch.float32, device=dev)
    else:                                                    # K tables, interleaved once (not timed)
        til = cih.tbme_interleave(torch.from_numpy(synth.tbme_tables(tl, range(w["seed"], w["seed"] + K))).to(dev))
        val = torch.empty((max(nnz, 1), K), dtype=torch.float32, device=dev)
    bytes_per_nnz = 4 + 4 * K                                # int32 column + K float32 values
    B0.close()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(ev):
        ev[0].record(st)
        B = cih.Basis(*sp)                                   # basis + neighbour lists
        ev[1].record(st)
        B.count_into(rowptr)                                 # count + scan
        ev[2].record(st)
        if sharded:
            B.fill_rows(rowptr, r0, r1, tbme, nnz_s=nnz_s, col=col, val=val)   # this rank's rows
        elif K == 1:
            B.fill(rowptr, nnz, tbme, col=col, val=val)      # fill: columns + values
        else:
            B.fill_batched(rowptr, nnz, til, K, col=col, val=val)
        ev[3].record(st)
        return B

    def new_events(n=4):
        return [torch.cuda.Event(enable_timing=True) for _ in range(n)]

    for _ in range(args.warmup):
        B = step(new_events())
        torch.cuda.synchronize()
        B.check()
        B.close()
    assert int(rowptr[-1].item()) == nnz

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = cih.kernel_launches()
    t_step, t_basis, t_count, t_fill = [], [], [], []
    for _ in range(args.steps):
        flush.fill_(1)                                        # evict L2 between steps (not timed)
        ev = new_events()
        B = step(ev)
        torch.cuda.synchronize()
        t_step.append(ev[0].elapsed_time(ev[3]))
        t_basis.append(ev[0].elapsed_time(ev[1]))
        t_count.append(ev[1].elapsed_time(ev[2]))
        t_fill.append(ev[2].elapsed_time(ev[3]))
        B.close()
    launches = cih.kernel_launches() - launches0
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(t_step), world, dev)
    if world > 1:
        torch.distributed.barrier()
    value = sharded_rate(args.steps, nnz, total_ms) if sharded else whole_job_rate(world, args.steps, nnz, total_ms)

    # gradient / forward time ratio: adjoint over the same structure with a
    # normalised vector, against the fill pass
    Bg = cih.Basis(*sp)
    Bg.count_into(rowptr)
    psi = torch.rand(dim, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    psi /= psi.norm()
    Bg.tbme_grad(rowptr, psi)
    torch.cuda.synchronize()
    tg = []
    for _ in range(max(1, min(args.steps, 3))):
        a, b = new_events(2)
        a.record(st)
        Bg.tbme_grad(rowptr, psi)
        b.record(st)
        torch.cuda.synchronize()
        tg.append(a.elapsed_time(b))
    Bg.close()
    grad_ratio = statistics.median(tg) / statistics.median(t_fill)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e and K == 1 and not sharded:
        # end to end through the library's host-memory call: tables from pinned
        # host memory, the matrix back to pinned host memory, copies inside
        tb_pin = torch.from_numpy(tbme_h).pin_memory()
        col_h = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
        val_h = torch.empty((1, nnz), dtype=torch.float32, pin_memory=True)
        rp_h = torch.empty(dim + 1, dtype=torch.int64, pin_memory=True)
        te = []
        for k in range(args.warmup + args.steps):
            flush.fill_(1)
            a, b = new_events(2)
            torch.cuda.synchronize()
            a.record(st)
            B = cih.Basis(*sp)
            n_h = B.build_to_host(tb_pin, rp_h, col_h, val_h)
            b.record(st)
            torch.cuda.synchronize()
            assert n_h == nnz
            if k >= args.warmup:
                te.append(a.elapsed_time(b))
            B.close()
        e_ms = max_over_ranks(sum(te) / len(te), world, dev)
        d2h = int(nnz * BYTES_PER_NNZ + (dim + 1) * 8)
        # the link in the same run: the matrix's bytes device -> the same pinned
        # host buffers, one copy per array, CUDA events (best of 3)
        link = []
        for _ in range(3):
            a, b = new_events(2)
            torch.cuda.synchronize()
            a.record(st)
            col_h.copy_(col[:nnz], non_blocking=True)
            val_h.copy_(val[:, :nnz], non_blocking=True)
            rp_h.copy_(rowptr, non_blocking=True)
            b.record(st)
            torch.cuda.synchronize()
            link.append(a.elapsed_time(b))
        link_gbs = d2h / (min(link) * 1e-3) / 1e9
        floor_ms = statistics.median(t_basis) + statistics.median(t_count) + min(link)
        e2e = {"value": whole_job_rate(world, 1, nnz, e_ms), "unit": "nnz/s", "call": "cih_ham_build_host",
               "h2d_bytes_per_step": int(tl * 4), "d2h_bytes_per_step": d2h, "ms": e_ms,
               "link_gbs": link_gbs, "floor_ms": floor_ms, "frac_of_link_floor": floor_ms / e_ms,
               "floor": "basis + count (device, this run) + the matrix's device-to-host copy at link_gbs "
                        "(pinned, measured in this run); the fill overlaps the copies"}
        del col_h, val_h

    peak, peak_kind = measured_peak()
    extra = {} if (args.no_extra or K > 1 or sharded) else side_measurements(args, dev, st, flush, peak, cih, synth, sp, rowptr, col, val, nnz)
    fill_ms = statistics.median(t_fill)
    achieved = nnz_s * bytes_per_nnz / (fill_ms * 1e-3) / 1e9
    wpeak = write_only_gbs(dev, st)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": "k_rows<W,1,K1> (fill)" if K == 1 else f"k_rows<W,1> (batched fill, K={K})",
                "algorithmic_bytes_per_launch": nnz_s * bytes_per_nnz,
                "traffic": fill_traffic(kernel_source_sha()) if (args.workload == "4p4n_nmax6" and K == 1
                                                                  and not sharded) else None,
                "write_only_peak": wpeak, "frac_of_write_only": achieved / wpeak,
                "write_only_source": "float32 fill of a 4 GiB buffer on this GPU, best of 5, CUDA events"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and K == 1:
        r, n, dt, threads, rows = oracle_rate(w, args.cpu_rows)
        cpu = {"value": r, "unit": "nnz/s", "cores": threads, "kind": "oracle",
               "sample": f"{rows} random rows of {args.workload} ({n} nonzeros, {dt:.1f} s): count + fill by "
                         f"the oracle's plain row walk, OpenMP over rows"}
        rows1 = max(50, args.cpu_rows // 25)
        try:
            r1, n1, dt1, th1 = oracle_rate_one_thread(args.workload, rows1)
            cpu["one_thread"] = {"value": r1, "unit": "nnz/s", "cores": th1,
                                 "sample": f"{rows1} other random rows ({n1} nonzeros, {dt1:.1f} s), same walk"}
        except (subprocess.SubprocessError, OSError, ValueError, IndexError) as e:
            cpu["one_thread"] = {"value": None, "error": str(e)[:200]}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(w), "dim": dim, "nnz_half": nnz, "tbme_entries": tl,
                       "tbme_sets": K, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": (f"row shards of about equal nonzeros over {world} GPUs (basis and "
                                       f"count on every rank, no collective on the data path)") if sharded
                       else ("replicas" if world > 1 else "single GPU")},
            "stages_ms": {"basis": statistics.median(t_basis), "count_scan": statistics.median(t_count),
                          "fill": fill_ms, "adjoint": statistics.median(tg)},
            "grad_fwd_ratio": grad_ratio,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            **extra,
            "clocks": clocks,
        }), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
