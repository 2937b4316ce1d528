#!/usr/bin/env python
"""Benchmark of the TREES epoch step on B300.

One step = one complete run of the fib(34) task tree (no sequential cutoff)
through the persistent scheduler: every epoch of the task vector, forks,
joins and the per-epoch grid barrier, from the root task to the empty stack.
The JSON line reports tasks/s (valid task executions, joins included) with
microseconds per epoch, the roofline of the persistent kernel, the clocks seen,
an end-to-end figure through the C ABI with host-side input/output, and the
CPU oracle timed on this host.  Secondary workloads (fib(34) with a leaf
cutoff of 12, mergesort of 2^26 keys, BFS on R-MAT scale 22) and the
V1/V-infinity fit of T_P = V1*T1/P + Vinf*Tinf ride along in the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--quick]

Multi-GPU: the run shards nothing (one task tree per GPU), so N>1 runs N
independent replicas (weak scaling) with no collective on the data path.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tasks/sec & µs/epoch (fib, sort, BFS); batched jobs/sec, p99 latency vs plain"
FIB_N = 34
FLUSH_BYTES = 256 << 20  # > 126 MB L2
FFT_LG, FFT_LEAF, FFT_CUTOFF = 24, 16, 0  # 2^24 points; 16-point leaves; every combine a map
SSSP_SLOTS_PER_VERTEX = 3  # task-vector slots per vertex for SSSP (relax tasks per reached vertex are measured below)
EPOCH_OVER_FLOOR_TARGET = 3.5  # target: fib(34) microseconds per epoch within 3.5x the bare grid-barrier floor
CLOCK_WARM_S = 1.0  # the clock sampler runs through at least this much warm-up of the timed step


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="headline only (no secondary workloads / fit)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--clock-warm-s", type=float, default=CLOCK_WARM_S,
                    help="least seconds of headline warm-up steps the clock sampler sees before the timed steps")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file for the autotuner's choices (default: tune afresh every run)")
    ap.add_argument("--profile-case", default=None,
                    help="PROGRAM:SIZE[:BLOCK[:SLOTS_PER_THREAD[:SCHEDULER]]] -- run one small case twice and exit "
                         "(for ncu): fib:N, sort:LOG2KEYS, bfs:RMAT_SCALE, sssp:RMAT_SCALE, fft:LOG2POINTS")
    return ap.parse_args()


def profile_case(spec):
    """One small workload run twice (a warm-up and the captured launch)."""
    import numpy as np
    import torch
    import paper_1608_00571_b300 as T
    from paper_1608_00571_b300 import gen
    parts = spec.split(":")
    prog, size = parts[0], int(parts[1])
    bs = int(parts[2]) if len(parts) > 2 else 1024
    tpt = int(parts[3]) if len(parts) > 3 else 2
    sched = {"persistent": 0, "graph": 1, "hostloop": 2}[parts[4]] if len(parts) > 4 else 0
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    keep = []
    if prog == "fib":
        a, b = 0, 1
        for _ in range(size + 1):
            a, b = b, a + b
        ctx = T.trees_create(2 * a + 1024, T.trees_default_config(block_size=bs, tasks_per_thread=tpt, map_capacity=1, scheduler=sched))
        job = T.make_job(T.TREES_PROG_FIB, n=size)
    elif prog == "sort":
        n = 1 << size
        kd = torch.from_numpy(gen.keys_u32(1, n).view(np.int32)).cuda()
        sc = torch.empty_like(kd)
        keep += [kd, sc]
        ctx = T.trees_create(max(4 * n // 1024, 1024),
                             T.trees_default_config(block_size=bs, tasks_per_thread=tpt, scheduler=sched))
        job = T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=kd, scratch=sc)
    elif prog == "bfs":
        row_ptr, col, _ = gen.rmat(size, 16, seed=2)
        rp, cl = torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda()
        lv = torch.empty(row_ptr.size - 1, dtype=torch.int32, device="cuda")
        keep += [rp, cl, lv]
        ctx = T.trees_create(row_ptr.size + 1024,
                             T.trees_default_config(block_size=bs, tasks_per_thread=tpt, scheduler=sched))
        job = T.make_job(T.TREES_PROG_BFS, n=0, row_ptr=rp, col=cl, level=lv, nv=row_ptr.size - 1)
    elif prog == "sssp":
        row_ptr, col, _ = gen.rmat(size, 16, seed=2)
        w = gen.weights(3, row_ptr, col)
        nv = row_ptr.size - 1
        rp, cl = torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda()
        wt = torch.from_numpy(w.view(np.int32)).cuda()
        dist = torch.empty(nv, dtype=torch.int64, device="cuda")
        sched_t = torch.empty(nv, dtype=torch.int32, device="cuda")
        keep += [rp, cl, wt, dist, sched_t]
        ctx = T.trees_create(3 * nv + 1024,
                             T.trees_default_config(block_size=bs, tasks_per_thread=tpt, scheduler=sched))
        job = T.make_job(T.TREES_PROG_SSSP, n=0, row_ptr=rp, col=cl, weight=wt, nv=nv, dist=dist, sched=sched_t)
    elif prog == "fft":
        n = 1 << size
        xi = torch.from_numpy(gen.signal(1, n).view(np.float32)).cuda()
        xo = torch.empty_like(xi)
        keep += [xi, xo]
        job = T.make_job(T.TREES_PROG_FFT, n=n, leaf=FFT_LEAF, cutoff=FFT_CUTOFF, fft_in=xi, fft_out=xo)
        ctx = T.trees_create(T.trees_job_slots(job)[0],
                             T.trees_default_config(block_size=bs, tasks_per_thread=tpt, scheduler=sched))
    else:
        raise SystemExit(f"unknown profile case {spec}")
    for _ in range(2):
        T.trees_run(ctx, job, s)
        st = T.trees_sync(ctx)
        if st != T.TREES_OK:
            raise SystemExit(f"status {st}")
    print(prog, size, T.trees_stats(ctx))
    T.trees_destroy(ctx)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def source_hash():
    """Hash of the kernel sources: the library's csrc/ and the engine headers
    under include/trees_impl/."""
    h = hashlib.sha256()
    for d in (os.path.join(ROOT, "paper_1608_00571_b300", "csrc"), os.path.join(ROOT, "include", "trees_impl")):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "20", "-i", str(dev)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.tmp.flush()
        with open(self.tmp.name) as f:
            rows = [r.split(",") for r in f.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for i, nm in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ algorithmic bytes

def fib_alg_bytes(stats, trace):
    """Minimum TV traffic of the fib task tree with the SoA layout (u32 code,
    u32 arg, u32 link, u64 result): an internal fib task reads code+arg (8 B),
    writes two children (16 B) and rewrites itself as a join (code+link, 8 B);
    a leaf reads 8 B and emits (result 8 B + code 4 B); a sum join reads
    code+link (8 B) and two child results (16 B) and emits (12 B); a dead entry
    launched in a join epoch is read once (4 B)."""
    joins = stats["joins"]
    fib_tasks = stats["tasks"] - joins
    leaves = fib_tasks - joins
    dead = sum(t["hi"] - t["lo"] - t["valid"] for t in trace)
    return 32 * joins + 20 * leaves + 36 * joins + 4 * dead


def sort_alg_bytes(n, leaf=1024):
    """Each key is read and written once per level: the leaf sort plus one
    merge per level of the split tree."""
    levels = 0
    m = n
    while m > leaf:
        m = (m + 1) // 2
        levels += 1
    return (levels + 1) * 2 * 4 * n


def bfs_alg_bytes(row_ptr, level):
    """Adjacency (4 B) and one level probe (4 B) per scanned edge, plus per
    reached vertex its row offsets (8 B), level write (4 B), TV entry written
    and read (16 B), retirement (4 B) and its map descriptor written and read
    (16 B)."""
    import numpy as np
    reached = level >= 0
    deg = np.diff(row_ptr)
    edges = int(deg[reached].sum())
    nreach = int(reached.sum())
    return 8 * edges + 48 * nreach, edges


def sssp_alg_bytes(row_ptr, reached, tasks):
    """Per scanned edge its column (4 B), weight (4 B) and the neighbour's
    distance probe (8 B); per relax task its TV entry written and read (16 B),
    retirement (4 B), row offsets (8 B), its map descriptor written and read
    (16 B), its own distance (8 B) and the fork dedupe word (4 B).  Edges are
    counted once per reached vertex: a lower bound when vertices are relaxed
    again."""
    import numpy as np
    edges = int(np.diff(row_ptr)[reached].sum())
    return 16 * edges + 56 * tasks, edges


def fft_alg_bytes(n, leaf):
    """Bytes the FFT task tree must move: the leaves read x and write X once
    (16 B per point), every combine level reads and writes X once more (16 B
    per point per level, log2(n / leaf) levels).  Task-vector and map
    descriptor traffic (under 1 % here) is left out."""
    levels = max(0, n.bit_length() - leaf.bit_length())
    return 16 * n * (1 + levels), levels


NQUEENS_SOLUTIONS = {1: 1, 2: 0, 3: 0, 4: 2, 5: 10, 6: 4, 7: 40, 8: 92, 9: 352, 10: 724, 11: 2680}


def bfs_certificate(row_ptr, col, src, level):
    """True when level holds the BFS levels from src of a symmetric graph:
    level[src] = 0, no edge from a reached vertex leads to an unreached one
    or skips a level (level[u] <= level[v] + 1), and every other reached
    vertex has a neighbour one level closer.  Chunked over edges."""
    import numpy as np
    nv = row_ptr.shape[0] - 1
    if level[src] != 0:
        return False
    has_parent = np.zeros(nv, dtype=bool)
    step = 1 << 24
    for e0 in range(0, col.shape[0], step):
        e1 = min(e0 + step, col.shape[0])
        s_of = np.searchsorted(row_ptr, np.arange(e0, e1), side="right") - 1
        ls, lu = level[s_of], level[col[e0:e1]]
        ok = ls >= 0
        if not ((lu[ok] >= 0) & (lu[ok] <= ls[ok] + 1)).all():
            return False
        has_parent[col[e0:e1][ok][lu[ok] == ls[ok] + 1]] = True
    reached = level >= 0
    reached[src] = False
    return bool(has_parent[reached].all())


def dft_samples(x, ks):
    """X[k] = sum_j x[j] exp(-2 pi i j k / n) for the indices ks, by direct
    summation in fp64 (the angle from j*k mod n)."""
    import numpy as np
    n = x.shape[0]
    j = np.arange(n, dtype=np.int64)
    xx = x.astype(np.complex128)
    return np.array([np.sum(xx * np.exp(-2j * np.pi * ((j * int(k)) % n) / n)) for k in ks])


def sssp_certificate(row_ptr, col, weight, src, dist, level):
    """True when dist are exactly the shortest distances: dist[src] = 0, no
    edge shortens any distance, every other reached vertex has an incoming edge
    that attains its distance, and the reached set is BFS's (weights >= 1, so
    there are no zero-weight cycles and these conditions characterise the
    shortest distances).  Chunked over edges to bound host memory."""
    import numpy as np
    inf = np.iinfo(np.uint64).max
    nv = row_ptr.shape[0] - 1
    if dist[src] != 0 or not np.array_equal(dist != inf, level >= 0):
        return False
    tight = np.zeros(nv, dtype=bool)
    step = 1 << 24
    for e0 in range(0, col.shape[0], step):
        e1 = min(e0 + step, col.shape[0])
        s_of = np.searchsorted(row_ptr, np.arange(e0, e1), side="right") - 1
        ds, du = dist[s_of], dist[col[e0:e1]]
        ok = ds != inf
        cand = ds[ok] + weight[e0:e1][ok].astype(np.uint64)
        if not (du[ok] <= cand).all():
            return False
        tight[col[e0:e1][ok][du[ok] == cand]] = True
    reached = dist != inf
    reached[src] = False
    return bool(tight[reached].all())


# ------------------------------------------------------------ multi-rank

def reduce_max_ms(total_ms, dist, device):
    """The timed region's length as the slowest rank saw it (max over ranks)."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, tasks_per_step, total_ms):
    """Whole-job throughput: every rank runs `steps` replicas of the task tree."""
    return world * steps * tasks_per_step / (total_ms / 1000.0)


# ------------------------------------------------------------ runners

def timed_runs(T, torch, ctx, job, steps, warmup, stream, flush=None, setup=None):
    """Runs `job` warmup+steps times; returns per-step device ms (CUDA events
    on the launching stream), flushing L2 between steps."""
    times = []
    for i in range(warmup + steps):
        if setup is not None:
            setup()
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        T.trees_run(ctx, job, stream)
        b.record(stream)
        st = T.trees_sync(ctx)
        if st != T.TREES_OK:
            raise RuntimeError(f"run failed with status {st}")
        b.synchronize()
        if i >= warmup:
            times.append(a.elapsed_time(b))
    return times


def vfit(T, torch, stream, cfg, solo_slots):
    """V1 and V-infinity of T_P = V1*T1/P + Vinf*Tinf (Sec. 1, Sec. 3), fitted
    per epoch: each epoch e of fib(34) is one step of the critical path
    (Tinf counts epochs), so its duration is modelled as
    dt_e = V1 * valid_e / P + Vinf, with valid_e the tasks it ran (its share
    of T1) and P the SMs working.  Runs the tuned block shape on P = 1/4,
    1/2 and all of the SMs (trace on, per-epoch end times from globaltimer)
    and fits the epochs that close with a grid barrier by least squares.
    Epochs of at most `solo_slots` slots run in one block under block
    barriers, so the model's P does not apply to them: their mean duration
    is reported beside the fit as the solo-epoch Vinf."""
    import numpy as np
    job = T.make_job(T.TREES_PROG_FIB, n=FIB_N)
    rows, ys, solo, per_p = [], [], [], {}
    probe = T.trees_create(1024, cfg)
    full_grid, _, sms = T.trees_geometry(probe)
    T.trees_destroy(probe)
    per_sm = max(1, full_grid // sms)
    for frac in (4, 2, 1):
        P = max(1, sms // frac)
        c = T.trees_create(20_000_000, T.trees_default_config(
            block_size=cfg.block_size, tasks_per_thread=cfg.tasks_per_thread, grid_blocks=P * per_sm, trace=1,
            map_capacity=1))
        try:
            timed_runs(T, torch, c, job, 2, 1, stream)
            tr = T.trees_trace(c)
        finally:
            T.trees_destroy(c)
        pr, py = [], []
        for a, b in zip(tr, tr[1:]):
            dt_us = (b["t_ns"] - a["t_ns"]) / 1000.0
            if b["hi"] - b["lo"] <= solo_slots:
                solo.append(dt_us)
            else:
                pr.append([b["valid"] / P, 1.0])
                py.append(dt_us)
        rows += pr
        ys += py
        A1, y1 = np.array(pr), np.array(py)
        c1, *_ = np.linalg.lstsq(A1, y1, rcond=None)
        per_p[str(P)] = {"V1_us_per_task_per_SM": float(c1[0]), "Vinf_us_per_epoch": float(c1[1]),
                         "grid_epochs": len(py)}
    A, y = np.array(rows), np.array(ys)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - A @ coef
    r2 = 1.0 - float((res ** 2).sum() / ((y - y.mean()) ** 2).sum())
    return {"model": "per grid-barrier epoch: dt = V1 * valid / P + Vinf (P = SMs working)",
            "V1_us_per_task_per_SM": float(coef[0]), "Vinf_us_per_epoch": float(coef[1]), "r2": r2,
            "rms_residual_us": float(np.sqrt((res ** 2).mean())), "max_abs_residual_us": float(np.abs(res).max()),
            "points": len(ys), "per_P": per_p, "solo_epoch_mean_us": float(np.mean(solo)) if solo else None,
            "solo_epochs_per_run": len(solo) // 3,
            "P": f"SMs: {sms // 4}, {sms // 2}, {sms} ({per_sm} block(s) of {cfg.block_size} threads per SM)"}


def batch_and_serve(T, torch, np, gen, stream):
    """The batched configuration: 4096 jobs (seed 42) in one persistent launch
    against one job per launch, then Poisson arrivals (seed 43) at 0.5x and
    0.9x of the batched throughput served by continuous batching and by one
    job per launch."""
    kind, param, kseed = gen.jobs(42, 4096)
    jobs, pristine, work = [], [], []
    for i in range(4096):
        if kind[i] == gen.JOB_FIB:
            jobs.append(T.make_job(T.TREES_PROG_FIB, n=int(param[i])))
        elif kind[i] == gen.JOB_NQUEENS:
            jobs.append(T.make_job(T.TREES_PROG_NQUEENS, n=int(param[i])))
        else:
            k = torch.from_numpy(gen.keys_u32(int(kseed[i]), int(param[i])).view(np.int32)).cuda()
            d, sc = torch.empty_like(k), torch.empty_like(k)
            pristine.append(k)
            work.append(d)
            jobs.append(T.make_job(T.TREES_PROG_MERGESORT, n=int(param[i]), keys=d, scratch=sc))
            jobs[-1]._keep = (d, sc)

    def reset():
        for k, d in zip(pristine, work):
            d.copy_(k)
        torch.cuda.synchronize()

    segs = [T.trees_job_slots(j)[0] for j in jobs]
    # each sort job's expected output: its input sorted on the device (as unsigned values)
    want = [torch.sort(k.to(torch.int64) & 0xFFFFFFFF).values for k in pristine]

    def sorts_ok():
        return all(torch.equal(d.to(torch.int64) & 0xFFFFFFFF, w) for d, w in zip(work, want))

    out = {}
    best = None
    per_bs = {}
    for bs in (256, 512, 1024):  # the batch kernel's block size, tuned here
        cfg_b = T.trees_default_config(block_size=bs, map_capacity=1 << 22)
        ctx = T.trees_create(sum(segs) + 1024, cfg_b)
        times = []
        for rep in range(3):
            reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            T.trees_batch_run(ctx, jobs, segs, stream)
            b.record(stream)
            status, res, steps = T.trees_batch_results(ctx, 4096)
            assert status == T.TREES_OK and all(r["status"] == T.TREES_OK for r in res)
            times.append(a.elapsed_time(b))
        assert sorts_ok(), f"batched sorts (block size {bs}) differ from their sorted inputs"
        T.trees_destroy(ctx)
        per_bs[bs] = min(times)
        if best is None or min(times) < best[0]:
            best = (min(times), bs, res, steps)
    bms, bs, res, steps = best
    cfg = T.trees_default_config(block_size=bs, map_capacity=1 << 22)
    # spot checks against closed forms and the known N-Queens counts (OEIS A000170)
    for i, r in enumerate(res):
        if kind[i] == gen.JOB_NQUEENS:
            assert r["result"] == NQUEENS_SOLUTIONS[int(param[i])]
        elif kind[i] == gen.JOB_FIB:
            assert r["epochs"] == 2 * int(param[i]) - 1
    tasks = sum(r["tasks"] for r in res)
    out["batched"] = {"jobs": 4096, "ms": bms, "jobs_per_s": 4096 / (bms / 1000), "steps": steps,
                      "tasks": tasks, "tasks_per_s": tasks / (bms / 1000), "block_size": bs,
                      "ms_by_block_size": per_bs}
    # one job per launch, back to back
    reset()
    solo = T.trees_create(max(segs) + 1024, T.trees_default_config(block_size=bs, map_capacity=1 << 22))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in jobs:
        T.trees_run(solo, j, stream)
        assert T.trees_sync(solo) == T.TREES_OK
    pms = 1000 * (time.perf_counter() - t0)
    T.trees_destroy(solo)
    out["one_job_per_launch"] = {"jobs": 4096, "ms": pms, "jobs_per_s": 4096 / (pms / 1000)}
    # served: continuous batching vs one job per launch, same arrivals
    batched_rate = 4096 / (bms / 1000)
    serve = {}
    for frac in (0.5, 0.9):
        rate = frac * batched_rate
        arr = gen.poisson_arrivals(43, 4096, rate)
        row = {"rate_jobs_per_s": rate}
        for mode, plain in (("continuous", False), ("one_job_per_launch", True)):
            reset()
            srv = T.trees_server_create(sum(segs) + 1024, 4096, 4, cfg)
            t0 = time.perf_counter()
            lat, rr = T.trees_server_replay(srv, jobs, arr, segs, plain=plain, stream=stream)
            wall = time.perf_counter() - t0
            _, _, launches = T.trees_server_stats(srv)
            T.trees_server_destroy(srv)
            assert all(r["status"] == T.TREES_OK for r in rr)
            lat_ms = np.array(lat) * 1000
            row[mode] = {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                         "mean_ms": float(lat_ms.mean()), "jobs_per_s": 4096 / wall,
                         "launches": int(launches) if not plain else 4096}
        serve[f"{frac}x_batched"] = row
    out["served"] = serve
    return out


def host_cpu():
    """The host's logical CPU count and CPU model (first "model name" of /proc/cpuinfo)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _timed_repeats(fn, seconds):
    """Calls fn() until `seconds` have passed (at least once); returns (calls, elapsed s)."""
    t0 = time.perf_counter()
    runs = 0
    while True:
        fn()
        runs += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            return runs, dt


def cpu_fib_rate(seconds):
    """fib(34) by the oracle's plain recursion (the sequential program of
    Sec. 6.2's comparison, one host core): jobs/s and calls/s."""
    import oracle
    v, calls = oracle.fib(FIB_N)
    assert v == 5702887
    runs, dt = _timed_repeats(lambda: oracle.fib(FIB_N), seconds)
    return runs / dt, calls


def cpu_baseline(seconds, gpu_tasks_per_job, extra=None):
    """The oracle on one host core.  Headline: fib(34) by the plain recursion,
    converted to the headline's unit as (fib(34) jobs/s) x (task executions
    per fib(34) job as the task vector machine counts them), so both arms
    divide the same work by their time.  Secondary: the oracle's sequential
    TVM simulator on fib(34), and the plain recursions of the other
    workloads (`extra`, timed by the caller next to their GPU runs)."""
    import oracle
    jobs_per_s, calls = cpu_fib_rate(min(seconds, 3.0))
    sim_runs, sim_dt = _timed_repeats(lambda: oracle.tvm_run(oracle.FIB, fib_n=FIB_N), min(seconds, 2.0))
    out = {"value": jobs_per_s * gpu_tasks_per_job, "unit": "tasks/s", "cores": 1, "kind": "oracle",
           "sample": f"fib({FIB_N}) by the oracle's plain recursion (oracle.fib, {calls} calls per job), repeated "
                     f"for ~{min(seconds, 3.0):.0f} s on one host core; value = jobs/s x {gpu_tasks_per_job} task "
                     f"executions per fib({FIB_N}) job",
           "fib34_jobs_per_s": jobs_per_s, "fib34_calls_per_s": jobs_per_s * calls,
           "tvm_simulator": {"value": sim_runs * gpu_tasks_per_job / sim_dt, "unit": "tasks/s",
                             "sample": f"{sim_runs} runs of the oracle's sequential TVM simulator on fib({FIB_N})"},
           **host_cpu()}
    if extra:
        out["workloads"] = extra
    return out


def cpu_sort_rate(seconds):
    """The oracle's recursive top-down mergesort (1024-key leaves) on a
    bounded sample: 2^24 splitmix64 keys, repeated for about `seconds`."""
    import numpy as np
    import oracle
    from paper_1608_00571_b300 import gen
    n = 1 << 24
    keys = gen.keys_u32(1, n)
    runs, dt = _timed_repeats(lambda: oracle.mergesort(keys), seconds)
    return {"keys_per_s": runs * n / dt, "sample": f"{runs} oracle.mergesort runs on 2^24 keys (seed 1), "
                                                   f"one core", "cores": 1}


def cpu_bfs_rate(row_ptr, col, seconds):
    """The oracle's FIFO-queue BFS on the R-MAT scale-22 graph from vertex 0."""
    import oracle
    box = {}

    def one():
        box["r"] = oracle.bfs(row_ptr, col, 0)[1]
    runs, dt = _timed_repeats(one, seconds)
    return {"ms": 1000 * dt / runs, "reached_per_s": box["r"] * runs / dt,
            "sample": f"{runs} oracle.bfs runs on R-MAT 22, one core", "cores": 1}


def cpu_nqueens_rate(seconds):
    """The oracle's backtracking N-Queens(11) (166,926 row tasks)."""
    import oracle
    v, rows, joins = oracle.nqueens(11)
    assert v == 2680
    runs, dt = _timed_repeats(lambda: oracle.nqueens(11), seconds)
    return {"jobs_per_s": runs / dt, "row_tasks_per_s": runs * rows / dt,
            "sample": f"{runs} oracle.nqueens(11) runs, one core", "cores": 1}


FIB34_TASKS = 27682393  # task executions of the fib(34) tree (fib tasks + joins), the TVM's count


def run_reference(args, rank, world):
    """The reference arm: the oracle's plain recursive fib(34) on one host
    core, one fib(34) job per step, reported in the headline's unit."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    v, calls = oracle.fib(FIB_N)
    assert v == 5702887
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r, _ = oracle.fib(FIB_N)
        dt = time.perf_counter() - t0
        assert r == 5702887
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * FIB34_TASKS / total
    sim_t0 = time.perf_counter()
    oracle.tvm_run(oracle.FIB, fib_n=FIB_N)
    sim_dt = time.perf_counter() - sim_t0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
            "data": "synthetic", "config": {"workload": f"fib({FIB_N}) uint64 task tree, no sequential cutoff",
                                            "n": FIB_N, "cutoff": 0},
            "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed fib({FIB_N}) jobs by the oracle's plain recursion "
                                       f"({calls} calls each); value = jobs/s x {FIB34_TASKS} task executions "
                                       f"per job",
                             "tvm_simulator": {"value": FIB34_TASKS / sim_dt, "unit": "tasks/s",
                                               "sample": "one run of the oracle's sequential TVM simulator"},
                             **host_cpu()},
            "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    import paper_1608_00571_b300 as T
    from paper_1608_00571_b300 import build as tbuild
    from paper_1608_00571_b300 import gen

    tbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    stream = torch.cuda.current_stream()
    hbm_peak, peak_kind = measured_peaks()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    tuned = {}

    def tune(job, cap, key, base=None):
        best, ms, cands = T.trees_autotune(job, cap, base, 2, args.tune_cache, key)
        tuned[key] = {"block_size": best.block_size, "tasks_per_thread": best.tasks_per_thread,
                      "scheduler": ["persistent", "graph", "hostloop"][best.scheduler], "ms": ms,
                      "candidates": len(cands)}
        return best

    # ---------------- headline: fib(34), autotuned configuration
    job = T.make_job(T.TREES_PROG_FIB, n=FIB_N)
    cfg = tune(job, 20_000_000, f"fib:n={FIB_N}:cutoff=0", T.trees_default_config(map_capacity=1))
    ctx = T.trees_create(20_000_000, cfg)
    # the clock record covers the warm-up (at least CLOCK_WARM_S of the same step, and at least W steps)
    # and the timed region: a timed region of a few milliseconds is shorter than the sampling interval
    clocks = ClockSampler(local)
    t_w0 = time.perf_counter()
    nwarm = 0
    while nwarm < args.warmup or time.perf_counter() - t_w0 < args.clock_warm_s:
        timed_runs(T, torch, ctx, job, 0, 1, stream, flush)
        nwarm += 1
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    times = timed_runs(T, torch, ctx, job, args.steps, 0, stream, flush)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    stats = T.trees_stats(ctx)
    grid, bs = stats["grid_blocks"], stats["block_size"]
    sms = T.trees_geometry(ctx)[2]
    result = T.trees_result(ctx, 0)
    assert result == 5702887, result
    total_ms = reduce_max_ms(sum(times), dist, "cuda")
    tasks = stats["tasks"]
    ms_step = total_ms / args.steps
    value = job_value(world, args.steps, tasks, total_ms)
    us_epoch = 1000.0 * ms_step / stats["epochs"]
    floor_us = T.trees_barrier_floor(ctx, 20000, stream)
    T.trees_destroy(ctx)

    # per-epoch trace (counts are deterministic) for the algorithmic bytes
    tctx = T.trees_create(20_000_000, T.trees_default_config(block_size=1024, trace=1, map_capacity=1))
    T.trees_run(tctx, job, stream)
    assert T.trees_sync(tctx) == T.TREES_OK
    trace = T.trees_trace(tctx)
    T.trees_destroy(tctx)
    alg = fib_alg_bytes(stats, trace)
    achieved = alg / (ms_step / 1000.0) / 1e9
    traffic = ncu_traffic(f"fib34_persistent_{cfg.block_size}x{cfg.tasks_per_thread}"
                          if cfg.scheduler == T.TREES_SCHED_PERSISTENT else "none")

    # ---------------- end to end through the C ABI: host input, host result
    ectx = T.trees_create(20_000_000, cfg)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.trees_fib(ectx, FIB_N, 0, stream)  # the root task travels host->device in the launch
        st = T.trees_sync(ectx)
        r = T.trees_result(ectx, 0)          # device->host read of the result
        dt = time.perf_counter() - t0
        assert st == T.TREES_OK and r == 5702887
        if i >= args.warmup:
            e2e_times.append(dt)
    T.trees_destroy(ectx)
    e2e_value = world * args.steps * tasks / sum(e2e_times)

    line = {
        "metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
        "config": {"workload": f"fib({FIB_N}) uint64 task tree, no sequential cutoff", "n": FIB_N, "cutoff": 0,
                   "scheduler": ["persistent", "graph", "hostloop"][cfg.scheduler], "block_size": bs,
                   "tasks_per_thread": cfg.tasks_per_thread, "grid_blocks": grid, "sms": sms,
                   "l2": "flushed between steps (256 MiB device write)"},
        "headline2": None,  # mergesort of 2^26 keys, filled in below (kept near the front of the line)
        "us_per_epoch": us_epoch, "epochs": stats["epochs"], "tasks_per_step": tasks,
        "barrier_floor_us": floor_us, "epoch_over_floor": us_epoch / floor_us,
        "epoch_over_floor_target": EPOCH_OVER_FLOOR_TARGET,
        "epoch_over_floor_met": us_epoch / floor_us <= EPOCH_OVER_FLOOR_TARGET,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)",
                     "algorithmic_bytes_per_launch": alg,
                     "kernel": f"k_persistent<{bs},{cfg.tasks_per_thread},PM_FIB>"},
        "clocks": {**clk, "window": f"{nwarm} warm-up steps ({time.perf_counter() - t_w0 - wall:.2f} s, "
                                    f"same step) and the {args.steps} timed steps"},
        "wall_s_timed_region": wall,
        "e2e": {"value": e2e_value, "unit": "tasks/s", "h2d_bytes_per_step": 12, "d2h_bytes_per_step": 8},
        # per step: k_setup + the persistent kernel, or k_setup + 4 kernels per epoch in the graph
        "gpu_launches": args.steps * (2 if cfg.scheduler == T.TREES_SCHED_PERSISTENT else 1 + 4 * stats["epochs"]),
    }

    cpu_extra = {}
    if not args.quick:
        workloads = {}
        # fib(34) with a leaf cutoff of 12
        j2 = T.make_job(T.TREES_PROG_FIB, n=FIB_N, cutoff=12)
        c2 = T.trees_create(200_000, tune(j2, 200_000, f"fib:n={FIB_N}:cutoff=12", T.trees_default_config(map_capacity=1)))
        t2 = timed_runs(T, torch, c2, j2, 10, 2, stream, flush)
        s2 = T.trees_stats(c2)
        assert T.trees_result(c2, 0) == 5702887
        T.trees_destroy(c2)
        m2 = statistics.mean(t2)
        workloads["fib34_cutoff12"] = {"ms": m2, "tasks": s2["tasks"], "epochs": s2["epochs"],
                                       "tasks_per_s": s2["tasks"] / (m2 / 1000), "us_per_epoch": 1000 * m2 / s2["epochs"],
                                       "bound": "alu (leaves run the naive recursion in-thread)"}
        # mergesort of 2^26 uint32 keys
        n = 1 << 26
        keys = gen.keys_u32(1, n)
        src = torch.from_numpy(keys.view(np.int32)).cuda()
        kd = torch.empty_like(src)
        sc = torch.empty_like(src)
        j3 = T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=kd, scratch=sc)
        kd.copy_(src)
        c3 = T.trees_create(1 << 18, tune(j3, 1 << 18, "mergesort:n=2^26"))
        t3 = timed_runs(T, torch, c3, j3, 5, 1, stream, None, setup=lambda: kd.copy_(src))
        s3 = T.trees_stats(c3)
        T.trees_destroy(c3)
        ok3 = bool(np.array_equal(kd.cpu().numpy().view(np.uint32), np.sort(keys)))
        assert ok3, "mergesort 2^26: output differs from numpy's sort"
        m3 = statistics.mean(t3)
        ab3 = sort_alg_bytes(n)
        workloads["mergesort_2^26"] = {"ms": m3, "tasks": s3["tasks"], "epochs": s3["epochs"],
                                       "tasks_per_s": s3["tasks"] / (m3 / 1000), "us_per_epoch": 1000 * m3 / s3["epochs"],
                                       "keys_per_s": n / (m3 / 1000), "sorted_equal_numpy": ok3,
                                       "roofline": {"bound": "hbm", "achieved": ab3 / (m3 / 1000) / 1e9,
                                                    "peak": hbm_peak, "unit": "GB/s",
                                                    "frac": ab3 / (m3 / 1000) / 1e9 / hbm_peak,
                                                    "algorithmic_bytes": ab3}}
        del src, kd, sc
        line["headline2"] = {"workload": "mergesort of 2^26 uint32 keys (splitmix64 seed 1), 1024-key leaves",
                             "ms": m3, "tasks_per_s": s3["tasks"] / (m3 / 1000), "keys_per_s": n / (m3 / 1000),
                             "us_per_epoch": 1000 * m3 / s3["epochs"],
                             "hbm_frac": ab3 / (m3 / 1000) / 1e9 / hbm_peak, "sorted_equal_numpy": ok3}
        if rank == 0:
            cpu_extra["mergesort"] = cpu_sort_rate(min(args.cpu_seconds, 6.0))
        # BFS on R-MAT scale 22
        row_ptr, col, info = gen.rmat(22, 16, seed=2)
        rp = torch.from_numpy(row_ptr).cuda()
        cl = torch.from_numpy(col).cuda()
        lv = torch.empty(row_ptr.size - 1, dtype=torch.int32, device="cuda")
        j4 = T.make_job(T.TREES_PROG_BFS, n=0, row_ptr=rp, col=cl, level=lv, nv=row_ptr.size - 1)
        c4 = T.trees_create(1 << 23, tune(j4, 1 << 23, "bfs:rmat22"))
        t4 = timed_runs(T, torch, c4, j4, 5, 1, stream, flush)
        s4 = T.trees_stats(c4)
        T.trees_destroy(c4)
        level = lv.cpu().numpy()
        ok4 = bfs_certificate(row_ptr, col, 0, level)
        assert ok4, "BFS R-MAT 22: the level certificate fails"
        m4 = statistics.mean(t4)
        ab4, edges = bfs_alg_bytes(row_ptr, level)
        workloads["bfs_rmat22"] = {"ms": m4, "tasks": s4["tasks"], "epochs": s4["epochs"],
                                   "tasks_per_s": s4["tasks"] / (m4 / 1000), "us_per_epoch": 1000 * m4 / s4["epochs"],
                                   "edges_scanned": edges, "teps": edges / (m4 / 1000), "levels_certified": ok4,
                                   "graph": {k: info[k] for k in ("nv", "m", "generated")},
                                   "roofline": {"bound": "hbm", "achieved": ab4 / (m4 / 1000) / 1e9, "peak": hbm_peak,
                                                "unit": "GB/s", "frac": ab4 / (m4 / 1000) / 1e9 / hbm_peak,
                                                "algorithmic_bytes": ab4}}
        if rank == 0:
            cpu_extra["bfs_rmat22"] = cpu_bfs_rate(row_ptr, col, 1.5)
        # SSSP on the same graph, symmetric weights in [1, 255] (Sec. 6.3's worklist relaxation as tasks)
        weight = gen.weights(3, row_ptr, col)
        wt = torch.from_numpy(weight.view(np.int32)).cuda()
        nv = row_ptr.size - 1
        dist_t = torch.empty(nv, dtype=torch.int64, device="cuda")
        sched_t = torch.empty(nv, dtype=torch.int32, device="cuda")
        j5 = T.make_job(T.TREES_PROG_SSSP, n=0, row_ptr=rp, col=cl, weight=wt, nv=nv, dist=dist_t, sched=sched_t)
        cap5 = SSSP_SLOTS_PER_VERTEX * nv
        c5 = T.trees_create(cap5, tune(j5, cap5, "sssp:rmat22"))
        t5 = timed_runs(T, torch, c5, j5, 5, 1, stream, flush)
        s5 = T.trees_stats(c5)
        T.trees_destroy(c5)
        sssp_dist = dist_t.cpu().numpy().view(np.uint64)
        ok5 = sssp_certificate(row_ptr, col, weight, 0, sssp_dist, level)
        assert ok5, "SSSP R-MAT 22: the shortest-path certificate fails"
        m5 = statistics.mean(t5)
        ab5, edges5 = sssp_alg_bytes(row_ptr, level >= 0, s5["tasks"])
        workloads["sssp_rmat22"] = {"ms": m5, "tasks": s5["tasks"], "epochs": s5["epochs"],
                                    "tasks_per_s": s5["tasks"] / (m5 / 1000), "us_per_epoch": 1000 * m5 / s5["epochs"],
                                    "relax_tasks_per_reached_vertex": s5["tasks"] / max(int((level >= 0).sum()), 1),
                                    "edges_scanned_lower_bound": edges5,
                                    "distances_certified_shortest": ok5, "weights": "[1, 255], seed 3",
                                    "roofline": {"bound": "hbm", "achieved": ab5 / (m5 / 1000) / 1e9,
                                                 "peak": hbm_peak, "unit": "GB/s",
                                                 "frac": ab5 / (m5 / 1000) / 1e9 / hbm_peak,
                                                 "algorithmic_bytes": ab5, "note": "lower bound (edges once per vertex)"}}
        del rp, cl, lv, wt, dist_t, sched_t
        # FFT of 2^24 complex fp32 points (Sec. 6.2, Fig. 6): radix-2 tasks, every combine a map
        n6 = 1 << FFT_LG
        x6 = gen.signal(1, n6)
        xi6 = torch.from_numpy(x6.view(np.float32)).cuda()
        xo6 = torch.empty_like(xi6)
        j6 = T.make_job(T.TREES_PROG_FFT, n=n6, leaf=FFT_LEAF, cutoff=FFT_CUTOFF, fft_in=xi6, fft_out=xo6)
        cap6 = T.trees_job_slots(j6)[0]
        cfg6 = tune(j6, cap6, f"fft:n=2^{FFT_LG}:leaf={FFT_LEAF}:cutoff={FFT_CUTOFF}")
        c6 = T.trees_create(cap6, cfg6)
        t6 = timed_runs(T, torch, c6, j6, 5, 1, stream, flush)
        s6 = T.trees_stats(c6)
        T.trees_destroy(c6)
        X6 = xo6.cpu().numpy().view(np.complex64).astype(np.complex128)
        ks = np.array([0, 1, n6 // 3, n6 - 1])
        norm_X = np.sqrt(n6) * np.linalg.norm(x6.astype(np.complex128))  # Parseval
        rel = 24 * 8 * 2.0 ** -24 / (1 - 24 * 8 * 2.0 ** -24)           # radix-2 fp32 error bound
        ok6 = bool(np.all(np.isfinite(X6)) and abs(np.linalg.norm(X6) - norm_X) <= rel * norm_X and
                   np.all(np.abs(X6[ks] - dft_samples(x6, ks)) <= rel * norm_X))
        assert ok6, "FFT 2^24: an output is not finite or outside the radix-2 error bound"
        m6 = statistics.mean(t6)
        ab6, lv6 = fft_alg_bytes(n6, FFT_LEAF)
        workloads[f"fft_2^{FFT_LG}"] = {
            "ms": m6, "tasks": s6["tasks"], "epochs": s6["epochs"], "maps": s6["maps"],
            "tasks_per_s": s6["tasks"] / (m6 / 1000), "us_per_epoch": 1000 * m6 / s6["epochs"],
            "points_per_s": n6 / (m6 / 1000), "gflops_5nlogn": 5 * n6 * FFT_LG / (m6 / 1000) / 1e9,
            "leaf": FFT_LEAF, "cutoff": FFT_CUTOFF, "dtype": "complex fp32", "combine_levels": lv6,
            "sampled_outputs_within_bound": ok6,
            "roofline": {"bound": "hbm", "achieved": ab6 / (m6 / 1000) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ab6 / (m6 / 1000) / 1e9 / hbm_peak, "algorithmic_bytes": ab6,
                         "traffic": ncu_traffic(f"fft{FFT_LG}_persistent_{cfg6.block_size}x{cfg6.tasks_per_thread}"
                                                if cfg6.scheduler == T.TREES_SCHED_PERSISTENT else "none"),
                         "kernel": f"k_persistent<{cfg6.block_size},{cfg6.tasks_per_thread},PM_FFT>"}}
        del xi6, xo6
        # a user task program through the SDK (examples/chunk_sum.cu): the sum of 2^26 keys, arity-8 forks,
        # leaves of 4096 keys reduced by one block each (a user map)
        import ctypes
        ex = os.path.join(ROOT, "paper_1608_00571_b300", "examples")
        prog = ctypes.CDLL(tbuild.build_program(os.path.join(ex, "chunk_sum.cu"),
                                                os.path.join(ex, "libchunk_sum.so"))).trees_chunk_sum
        n7, chunk7, arity7 = 1 << 26, 4096, 8
        keys7 = gen.keys_u32(7, n7)
        kd7 = torch.from_numpy(keys7.view(np.int32)).cuda()
        j7 = T.make_job(T.TREES_PROG_USER, user_program=prog, user_type=1, user_a0=0, user_a1=n7,
                        user_ptr=(kd7,), user_val=(chunk7, arity7))
        cap7 = 4 * (n7 // chunk7) + 1024  # leaves of at least chunk/arity keys, plus their ancestors
        cfg7 = tune(j7, cap7, f"user:chunk_sum:n=2^26:chunk={chunk7}:arity={arity7}")
        c7 = T.trees_create(cap7, cfg7)
        t7 = timed_runs(T, torch, c7, j7, 5, 2, stream, flush)
        s7 = T.trees_stats(c7)
        ok7 = T.trees_result(c7, 0) == int(keys7.astype(np.uint64).sum())
        assert ok7, "user program: the sum differs from numpy's"
        T.trees_destroy(c7)
        m7 = statistics.mean(t7)
        ab7 = 4 * n7
        workloads["user_chunk_sum_2^26"] = {
            "ms": m7, "tasks": s7["tasks"], "epochs": s7["epochs"], "maps": s7["maps"],
            "keys_per_s": n7 / (m7 / 1000), "sum_equal_numpy": ok7, "chunk": chunk7, "arity": arity7,
            "config": f"{cfg7.block_size} threads x {cfg7.tasks_per_thread} slots, persistent (tuned; user programs "
                      "run under the persistent scheduler only)",
            "roofline": {"bound": "hbm", "achieved": ab7 / (m7 / 1000) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ab7 / (m7 / 1000) / 1e9 / hbm_peak, "algorithmic_bytes": ab7}}
        del kd7
        line["workloads"] = workloads
        # graph-relaunch and host-loop schedulers on the headline workload
        sch = {}
        for name, sid in (("graph", T.TREES_SCHED_GRAPH), ("hostloop", T.TREES_SCHED_HOSTLOOP)):
            cx = T.trees_create(20_000_000, T.trees_default_config(block_size=cfg.block_size, scheduler=sid,
                                                                  tasks_per_thread=cfg.tasks_per_thread,
                                                                  map_capacity=1))
            tt = timed_runs(T, torch, cx, job, 5, 1, stream, flush)
            T.trees_destroy(cx)
            mm = statistics.mean(tt)
            sch[name] = {"ms": mm, "us_per_epoch": 1000 * mm / stats["epochs"], "tasks_per_s": tasks / (mm / 1000)}
        sch["persistent"] = {"ms": ms_step, "us_per_epoch": us_epoch, "tasks_per_s": tasks / (ms_step / 1000)}
        line["schedulers"] = sch
        line["vfit"] = vfit(T, torch, stream, cfg, 2 * cfg.block_size * cfg.tasks_per_thread)
        line["batch_serve"] = batch_and_serve(T, torch, np, gen, stream)
    line["autotune"] = tuned

    if rank == 0:
        cpu_extra["nqueens11"] = cpu_nqueens_rate(1.0)
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, tasks, cpu_extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
