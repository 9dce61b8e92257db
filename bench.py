#!/usr/bin/env python3
"""Throughput benchmark of the annealed p-dit sweep (one JSON line on stdout).

Workload (default): dense symmetric QAP, N = 100, D and F off-diagonal entries
uniform in 0..99 (seeded, synthetic), 4096 replicas, 10000 sweeps, linear
beta schedule 0 -> beta_max. One step = one complete anneal of that workload
through the C ABI: Fisher-Yates initial permutations, influence tables,
10000 sweeps, best-so-far tracking and the final reduction to the best
permutation. Metric: p-dit updates per second (one update = one location's
Eq. 5 draw; N x replicas x sweeps per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1: one process per GPU (torchrun); rank r runs replicas r*R..(r+1)*R-1
(weak scaling, no collective in the timed region); value = all ranks'
updates / max-over-ranks time.
--impl reference: the CPU oracle on this host's cores (rank 0 only).

Other workloads: --workload n100a (general form), c256 (two-level flow),
n256 (largest size), dense --dense-n N, n30, n12; --mode cupim (concurrent
updates); --workload ragged (time to 1% gap, batched vs one launch per
instance); --workload served (continuous batching: capacity, p50/p99).
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

from paper_2605_24408_gb300 import instances as G  # noqa: E402
from paper_2605_24408_gb300 import multi  # noqa: E402

WORKLOADS = {
    # name: (instance, replicas, sweeps, schedule)
    "n100": ("n100", 4096, 10000, "linear"),
    "n30": ("n30", 1024, 5000, "geometric"),
    "n12": ("n12", 64, 1000, "linear"),
    "n100a": ("n100a", 4096, 10000, "linear"),
    "c256": ("c256", 4096, 2000, "linear"),
    "n256": ("n256", 2048, 1000, "linear"),
    "dense": ("dense", 2048, 1000, "linear"),  # N from --dense-n
}
WORKLOAD_TEXT = {
    "n100": "dense symmetric QAP N=100 (D, F uniform 0..99)",
    "n100a": "dense asymmetric QAP N=100 (every entry of D and F independent uniform 0..99, zero diagonals)",
    "n256": "dense symmetric QAP N=256 (D, F uniform 0..99): influence tables in global memory",
    "dense": "dense symmetric QAP (D, F uniform 0..99) of the size given by --dense-n",
    "c256": "two-level flow N=256 (flow 1 between every pair of a 92-facility subset, 0 elsewhere; "
            "D dense symmetric uniform 1..99): the structure of the paper's tai256c, synthetic values",
}
METRIC = "p-dit updates/s"
L2_FLUSH_BYTES = 512 << 20
SMEM_BYTES_PER_CLK = 128  # shared-memory bandwidth per SM per clock (32 banks x 4 B)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dot_kernel_n100_traffic.json")
# the n100 kernel's own sources; the stored DRAM counters also record the
# kernel and the launch shape they were taken with, and all must match to be
# reported
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2605_24408_gb300", "csrc", f)
                  for f in ("pdit_sweep.cuh", "pdit_dot.cu")]


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dot_parts(replicas: int, slots: int, sweeps: int, pt: bool = False) -> int:
    """Parts the library splits each replica's sweeps into for one
    dot-kernel launch of `sweeps` sweeps: 1 while the replicas fill whole
    rounds of the resident slots, else up to 16 parts of at least 8 sweeps
    (anneal and fixed modes; more where a part would exceed 1000 sweeps) or
    of one sweep (a PT launch, one exchange period)."""
    if replicas <= slots or replicas % slots == 0:
        return 1
    k = max(min(16, sweeps if pt else sweeps // 8), -(-sweeps // 1000))  # parts of at most 1000 sweeps
    return max(1, min(k, (1 << 30) // replicas))


def dot_kernel_name(maxk: int, wpr: int, n: int, parts: int = 1) -> str:
    """The dot kernel instantiation a launch runs: the third parameter is the
    row stride in 16-byte chunks where it is compiled in (four locations per
    thread, one warp per replica, 7-chunk rows: N = 97..112), else 0; the
    fourth is 1 for a call split into parts."""
    nch = 7 if (maxk, wpr) == (4, 1) and product_stride(n) == 16 * 7 else 0
    return "dot_kernel<%d,%d,%d,%d>" % (maxk, wpr, nch, 1 if parts > 1 else 0)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def method_bytes_per_update(n: int, accept_frac: float, general: bool = False) -> float:
    """Algorithmic shared-memory bytes per p-dit update of the method as
    written (every accepted swap rewrites the table): 4 (4N) for the gathers
    (row, column, p-diagonal, permutation, int32) plus, per accepted swap,
    8 N^2 (table read and write) + 8 N (the two factor vectors; four for the
    rank-2 update of the general form)."""
    return 4 * (4 * n) + accept_frac * (8 * n * n + (16 if general else 8) * n)


def algorithmic_bytes_per_update(n: int, dt_bytes: int, accept_frac: float, pending: int = 1,
                                 general: bool = False) -> float:
    """Shared-memory bytes one update must move in this design.
    Immediate table updates (pending = 1):
      gather, every update: p[j], I[i][p(j)], I[j][p(i)], h[j] as int32, plus
      D[i][j] and F[p(i)][p(j)] at the staged width dt: 16 N + 2 N dt;
      accepted swap: read+write of the N x N int32 table (8 N^2), two D rows
      and two F rows (4 N dt), the column factor written once (4 N), the
      p-diagonal read and written (8 N).
    Deferred updates (pending = 4 or 16 terms, pending / 4 packed words):
    the gather also reads the packed factors u[j], v[p(j)] (+8 N per word);
    an accepted swap writes one byte of each packed factor per entry (2 N),
    reads two D rows and two F rows (4 N dt) and p, h (12 N), and 1 / pending
    of a table rewrite (8 N^2 / pending).
    General form: the gather also reads D[j][i] and F[p(j)][p(i)] (+2 N dt);
    a swap reads D and F columns as well (+4 N dt) and carries two rank-1
    terms (two factor vectors; two of the four pending slots, so half a table
    rewrite per swap when deferred)."""
    if pending <= 1:
        gather = 16 * n + 2 * n * dt_bytes
        swap = 8 * n * n + 4 * n * dt_bytes + 12 * n
        if general:
            gather += 2 * n * dt_bytes
            swap += 4 * n * dt_bytes + 4 * n
    else:
        words = pending // 4  # packed words per entry, read by both queries
        gather = 16 * n + 8 * n * words + 2 * n * dt_bytes
        swap = 8 * n * n / pending + 4 * n * dt_bytes + 16 * n
        if general:
            gather += 2 * n * dt_bytes
            swap += 8 * n * n / pending + 4 * n * dt_bytes + 4 * n
    return gather + accept_frac * swap


def product_stride(n: int) -> int:
    """Row stride in bytes of D and of the permuted flow matrix in the
    dot-product kernel: 16 bytes x the smallest odd number >= n / 16."""
    s16 = (n + 15) // 16
    return 16 * (s16 + 1 - s16 % 2)


def product_bytes_per_update(n: int, accept_frac: float) -> float:
    """Shared-memory bytes one update moves in the dot-product kernel
    (row stride S): for every candidate its row of D and its row of the
    permuted flow matrix Q (2 N S), the updating location's two rows (2 S),
    D[i][j] and Q[i][j] (2 N) and h[i] (4); per accepted swap the p-diagonal
    update reads two D rows and two Q rows (4 N) and writes h (4 N), the two
    Q rows are exchanged (4 S: read and written) and so are two columns
    (4 N), and p moves (16)."""
    S = product_stride(n)
    return 2 * n * S + 2 * S + 2 * n + 4 + accept_frac * (12 * n + 4 * S + 16)


def product_dp4a_per_update(n: int) -> int:
    """dp4a operations per update of the dot-product kernel: two dot
    products of S / 4 words for each of the N candidates."""
    return 2 * n * (product_stride(n) // 4)


def class_bytes_per_update(n: int, dt_bytes: int, accept_frac: float) -> float:
    """Shared-memory bytes per update of the flow-class kernel: per candidate
    p[j], G[j] and the swap energy written then read back (int32), x[p(j)]
    (1 byte) and D[i][j] (dt): (17 + dt) N; per accepted swap at most (only
    swaps across the classes move G) two D rows and G read and written:
    2 N dt + 8 N."""
    return (17 + dt_bytes) * n + accept_frac * (2 * n * dt_bytes + 8 * n)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline(D, F, beta, n: int, sweeps: int, mode: str, gpu: dict) -> dict:
    """The CPU oracle as it stands, one replica per host core over the full
    schedule (a bounded sample of the workload's replicas), timed; then,
    untimed, the parity sample of the same leg (parity_sample)."""
    import oracle as O

    cores = host_cores()
    t = time.perf_counter()
    O.anneal(D, F, beta, sweeps, 0, 0, cores, threads=cores)
    dt = time.perf_counter() - t
    return {"value": cores * n * sweeps / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": "%d of the replicas (ids 0..%d), all %d sweeps, one per core; %.1f s"
                      % (cores, cores - 1, sweeps, dt),
            "parity_sample": parity_sample(D, F, beta, sweeps, mode, gpu)}


def parity_sample(D, F, beta, sweeps: int, mode: str, gpu: dict, reps: int = 4) -> dict:
    """The oracle on replicas 0..reps-1 of the workload (outside every timed
    region): their best costs, best sweeps and accepted counts must equal the
    GPU's; also the number of draws that fell within 1e-6 of a boundary of the
    exact double-precision Eq. 5 CDF (where an ideal sampler might have chosen
    another outcome)."""
    import oracle as O

    r = O.anneal(D, F, beta, sweeps, 0, 0, reps, threads=reps, near=True,
                 mode="cupim" if mode == "cupim" else "anneal")
    same = (np.array_equal(gpu["replica_best_cost"][:reps], r["best_cost"]) and
            np.array_equal(gpu["replica_best_sweep"][:reps], r["best_sweep"]) and
            np.array_equal(gpu["replica_accepted"][:reps], r["accepted"]))
    draws = reps * sweeps * D.shape[0]
    return {"replicas": reps, "bit_exact": bool(same), "draws": draws,
            "near_boundary_draws": int(r["near_boundary"].sum()),
            "near_boundary_fraction": float(r["near_boundary"].sum()) / draws}


def run_reference(args, wl):
    """--impl reference: the CPU oracle on this host, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    inst, replicas, sweeps, kind = WORKLOADS[wl]
    D, F = G.named(inst)
    n = D.shape[0]
    beta_full = O.beta_schedule(kind, sweeps, O.beta_max(D, F))
    sub = max(1, sweeps // 1000)
    beta = np.ascontiguousarray(beta_full[::sub])
    s_steps = len(beta)
    cores = host_cores()
    upd = cores * n * s_steps

    def step(k):
        O.anneal(D, F, beta, s_steps, 1000 + k, 0, cores, threads=cores)

    for k in range(args.warmup):
        step(k)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        step(args.warmup + k)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = upd * args.steps / tot
    sample = ("per step: %d replicas (one per core) x %d sweeps, the %d-sweep schedule taken every "
              "%d-th sweep (same beta range)" % (cores, s_steps, sweeps, sub))
    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "%s: N=%d, %d replicas x %d sweeps, %s beta" % (wl, n, replicas, sweeps, kind),
                       "global_batch": replicas, "seq_len": n, "parallelism": "cpu threads",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ragged_optima():
    """{k: optimum} for the ragged instances with N <= 12, brute-forced over
    all N! permutations and stored under tests/golden (empty if absent)."""
    out = {}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "ragged_optima.txt")) as fh:
            for line in fh:
                f = line.split()
                if f and not line.startswith("#"):
                    out[int(f[0])] = int(f[2])
    except OSError:
        pass
    return out


def run_ragged(args):
    """Ragged multi-instance batch: K instances, N uniform in 12..256 (half grid
    D with 30% flow density, half dense 0..99), R replicas and S linear sweeps
    each. (A) one batched, graph-captured run to the end: throughput and each
    instance's final best. Targets T_k = floor(1.01 C*_k) with C*_k the best
    cost of an independent reference run of instance k (bench_targets/
    ragged.json: 4x replicas, 2x sweeps, another seed), or for N <= 12 the
    brute-force optimum (tests/golden/ragged_optima.txt); without those
    files, C*_k = the final best of run (A), said so in the line. Time to reach
    every target with each instance's replicas stopping once its target is
    reached: (B) batched, (C) one single-instance launch after another."""
    import torch

    from paper_2605_24408_gb300 import build as B
    from paper_2605_24408_gb300 import pdit as P

    torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", 0)
    K, R, S = args.instances, args.ragged_replicas, args.ragged_sweeps
    qs, betas, sizes = [], [], []
    for k in range(K):
        n = G.ragged_size(k, 0)
        D, F = G.ragged_instance(k, n, 0)
        q = P.Qap(D, F)
        qs.append(q)
        sizes.append(n)
        betas.append(torch.from_numpy(P.pdit_beta_schedule("linear", S, P.pdit_beta_max(q))).to(dev))
    # autotune one instance per distinct size, reuse its shape for the others
    tuned = {}
    t0 = time.perf_counter()
    if not args.no_autotune:
        for k, q in enumerate(qs):
            n = sizes[k]
            if n not in tuned:
                mid = torch.full((4,), float(betas[k][S // 2].item()), dtype=torch.float32, device=dev)
                wpr, pk = P.pdit_autotune(q, R, mid, 4)
                shp = P.pdit_launch_shape(q, R)
                tuned[n] = (wpr, pk, shp["replicas_per_cta"],
                            P.PDIT_PLACE_SHARED if shp["tables_in_smem"] else P.PDIT_PLACE_GLOBAL,
                            shp["influence"])
            else:
                wpr, pk, rpc, place, infl = tuned[n]
                P.pdit_set_warps_per_replica(q, wpr)
                P.pdit_set_replicas_per_cta(q, rpc)
                if infl == "products":
                    P.pdit_set_influence(q, P.PDIT_INFLUENCE_PRODUCTS)
                else:
                    P.pdit_set_influence(q, P.PDIT_INFLUENCE_TABLE)
                    P.pdit_set_pending_swaps(q, pk)
                    P.pdit_set_table_placement(q, place)
    tune_s = time.perf_counter() - t0
    items = [dict(qap=q, replicas=R, sweeps=S, beta=betas[k], seed=0, instance_id=k) for k, q in enumerate(qs)]
    stream = torch.cuda.Stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
        stream.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1000.0

    full = P.Batch(items, graph=True)
    with torch.cuda.stream(stream):
        full.run(stream)  # capture + first run
    stream.synchronize()
    t_full = timed(lambda: full.run(stream))
    best = [int(o["best_cost"].item()) for o in full.out]
    updates = sum(n * R * S for n in sizes)
    ref, target_source = None, "1.01 x the final best of the full batched run (same random streams)"
    try:
        with open(os.path.join(ROOT, "bench_targets", "ragged.json")) as fh:
            tr = json.load(fh)["targets"]
        if len(tr) >= K and all(tr[k]["k"] == k and tr[k]["n"] == sizes[k] for k in range(K)):
            ref = [int(tr[k]["best"]) for k in range(K)]
            target_source = ("1.01 x the best of an independent reference run per instance "
                             "(bench_targets/ragged.json: 1024 replicas x 4000 sweeps, seed 1)")
    except (OSError, ValueError, KeyError):
        pass
    goal = list(ref if ref is not None else best)
    # N <= 12: the brute-force optimum over all N! permutations, where stored
    n_exact = 0
    for k, opt in ragged_optima().items():
        if k < K and sizes[k] <= 12:
            goal[k] = opt
            n_exact += 1
    if n_exact:
        target_source += "; the brute-force optimum for the %d instance(s) with N <= 12" % n_exact
    # gap <= 1%: best - C* <= 0.01 C*, in integers best <= floor(1.01 C*)
    targets = [torch.tensor([c + c // 100], dtype=torch.int64, device=dev) for c in goal]
    titems = [dict(it, target=targets[k]) for k, it in enumerate(items)]
    bt = P.Batch(titems, stop_at_target=True, graph=True)
    with torch.cuda.stream(stream):
        bt.run(stream)
    stream.synchronize()
    t_batched = timed(lambda: bt.run(stream))
    reached_b = sum(int(o["reach_sweep"].item()) < S for o in bt.out)
    # plain: one launch per instance, in sequence, same targets and stopping
    ws = []
    for k, q in enumerate(qs):
        o = P.opts(replicas=R, sweeps=S, seed=0, instance_id=k, beta=betas[k].data_ptr(),
                   stream=stream.cuda_stream, stop_at_target=1, target=targets[k].data_ptr())
        w = torch.empty(P.pdit_workspace_bytes(q, o), dtype=torch.uint8, device=dev)
        outs = {"best_perm": torch.empty(q.n, dtype=torch.int32, device=dev),
                "best_cost": torch.empty(1, dtype=torch.int64, device=dev),
                "reach_ns": torch.empty(1, dtype=torch.int64, device=dev),
                "reach_sweep": torch.empty(1, dtype=torch.int32, device=dev)}
        o.workspace, o.workspace_bytes = w.data_ptr(), w.numel()
        for key, t in outs.items():
            setattr(o, key, t.data_ptr())
        ws.append((o, w, outs))

    def plain():
        for k, q in enumerate(qs):
            P.pdit_anneal_ex(q, ws[k][0])

    with torch.cuda.stream(stream):
        plain()
    stream.synchronize()
    t_plain = timed(plain)
    reached_p = sum(int(w[2]["reach_sweep"].item()) < S for w in ws)
    classes, wsb = full.info()
    line = {"metric": "time-to-1%-gap, ragged batch", "value": t_batched, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "int32",
            "config": {"workload": "ragged: %d instances, N uniform 12..256 (even k grid D + 30%% flow "
                                   "1..10, odd k dense 0..99), %d replicas x %d linear sweeps each"
                                   % (K, R, S),
                       "target": target_source,
                       "autotune": not args.no_autotune, "autotune_s": tune_s,
                       "shape_classes": classes, "workspace_bytes": wsb},
            "batched_s": t_batched, "plain_s": t_plain, "speedup": t_plain / t_batched,
            "instances_reached": {"batched": reached_b, "plain": reached_p, "of": K},
            "full_run_vs_targets": None if ref is None else {
                "within_1pct": sum(b <= c + c // 100 for b, c in zip(best, ref)),
                "better_than_target": sum(b < c for b, c in zip(best, ref)),
                "median_gap": float(np.median([(b - c) / c for b, c in zip(best, ref)]))},
            "full_run": {"seconds": t_full, "updates": updates, "updates_per_s": updates / t_full}}
    print(json.dumps(line), flush=True)
    for q in qs:
        q.close()


def run_served(args):
    """Serving with continuous batching. Request r: N uniform in 20..200 from
    r, the ragged generator keyed by r, 512 replicas, 2000 linear sweeps.
    (1) capacity: a closed burst of requests; (2) an open-loop Poisson stream
    at a fraction of that capacity for a fixed window: p50/p99 latency (submit
    to result) and solves/s. The configured 200 requests/s is reported as the
    offered load beside the capacity."""
    import threading

    import torch

    from paper_2605_24408_gb300 import build as B
    from paper_2605_24408_gb300 import pdit as P

    torch.cuda.set_device(0)
    B.build()
    R, S = args.serve_replicas, args.serve_sweeps
    reqs = {}

    def instance(rid):
        if rid not in reqs:
            reqs[rid] = G.request_instance(rid)
        return reqs[rid]

    def drain(srv, tickets, producer=None):
        while True:
            a, q = srv.tick()
            if (producer is None or not producer.is_alive()) and a == 0 and q == 0:
                break
        out = []
        for rid, t in tickets.items():
            st, _, cost, lat = srv.result(t)
            out.append((rid, st, cost, lat))
        return out

    # (1) capacity: a burst submitted at once
    srv = P.Server(device_budget_bytes=args.serve_budget_gb << 30, slice_sweeps=args.serve_slice,
                   max_active=args.serve_max_active)
    burst = args.serve_burst
    for rid in range(burst):
        instance(rid)
    t0 = time.perf_counter()
    tickets = {rid: srv.submit(*instance(rid), R, S, 0, rid) for rid in range(burst)}
    res = drain(srv, tickets)
    t_burst = time.perf_counter() - t0
    srv.close()
    capacity = burst / t_burst
    upd = sum(instance(rid)[0].shape[0] * R * S for rid in range(burst))
    # the same burst as one single-instance call after another (qap_create,
    # pdit_anneal, qap_destroy per request), each result checked against the
    # served one
    served = {rid: cost for rid, st, cost, _ in res}
    t0 = time.perf_counter()
    for rid in range(burst):
        Dr, Fr = instance(rid)
        with P.Qap(Dr, Fr) as qr:
            br = torch.from_numpy(P.pdit_beta_schedule("linear", S, P.pdit_beta_max(qr))).cuda()
            out = P.anneal_device(qr, R, br, S, 0, instance_id=rid)
            c = int(out["best_cost"].item())
        if c != served[rid]:
            raise SystemExit("served and single-call results differ for request %d" % rid)
    t_plain = time.perf_counter() - t0
    # (2) open-loop Poisson arrivals at a fraction of capacity
    lam = args.serve_load * capacity
    gaps = -np.log(1.0 - G.hash_unit(7, 91, np.arange(100000, dtype=np.uint64))) / lam
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < args.serve_window]
    base = 1000
    for k in range(len(arrivals)):
        instance(base + k)
    srv = P.Server(device_budget_bytes=args.serve_budget_gb << 30, slice_sweeps=args.serve_slice,
                   max_active=args.serve_max_active)
    tickets = {}

    def producer():
        start = time.perf_counter()
        for k, at in enumerate(arrivals):
            delay = at - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            tickets[base + k] = srv.submit(*instance(base + k), R, S, 0, base + k)

    th = threading.Thread(target=producer)
    t0 = time.perf_counter()
    th.start()
    res2 = drain(srv, tickets, th)
    th.join()
    t_open = time.perf_counter() - t0
    srv.close()
    lats = np.array([r[3] for r in res2 if r[1] == 2])
    # the single-instance rate beside it: the n100 workload's shape (dense N =
    # 100, 4096 replicas) for 1000 sweeps
    Dn, Fn = G.named("n100")
    with P.Qap(Dn, Fn) as qn:
        bn = torch.from_numpy(P.pdit_beta_schedule("linear", 1000, P.pdit_beta_max(qn))).cuda()
        P.anneal_device(qn, 4096, bn, 1000, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.anneal_device(qn, 4096, bn, 1000, 0)
        e1.record()
        torch.cuda.synchronize()
        single = 100 * 4096 * 1000 / (e0.elapsed_time(e1) / 1000.0)
    line = {"metric": "p50/p99 latency, served stream", "value": float(np.percentile(lats, 50)) if len(lats) else None,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "int32",
            "config": {"workload": "served: request r -> N uniform 20..200 (ragged generator keyed by r), "
                                   "%d replicas x %d linear sweeps per request" % (R, S),
                       "slice_sweeps": args.serve_slice, "max_active": args.serve_max_active,
                       "device_budget_gb": args.serve_budget_gb},
            "capacity": {"burst_requests": burst, "seconds": t_burst, "solves_per_s": capacity,
                         "updates_per_s": upd / t_burst,
                         "single_instance_n100_updates_per_s": single,
                         "fraction_of_single_instance": upd / t_burst / single,
                         "one_call_per_request_seconds": t_plain,
                         "one_call_per_request_solves_per_s": burst / t_plain,
                         "speedup_over_one_call_per_request": t_plain / t_burst},
            "open_loop": {"arrival_rate_per_s": lam, "load_fraction_of_capacity": args.serve_load,
                          "window_s": args.serve_window, "requests": int(len(arrivals)),
                          "completed": int(len(lats)), "p50_s": float(np.percentile(lats, 50)) if len(lats) else None,
                          "p99_s": float(np.percentile(lats, 99)) if len(lats) else None,
                          "solves_per_s": len(lats) / t_open},
            "offered_rate_configured_per_s": 200.0,
            "offered_over_capacity": 200.0 / capacity}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n100", choices=sorted(WORKLOADS) + ["ragged", "served"])
    ap.add_argument("--serve-replicas", type=int, default=512)
    ap.add_argument("--serve-sweeps", type=int, default=2000)
    ap.add_argument("--serve-slice", type=int, default=100)
    ap.add_argument("--serve-max-active", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=int, default=16)
    ap.add_argument("--serve-burst", type=int, default=24)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-window", type=float, default=20.0)
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--ragged-replicas", type=int, default=256)
    ap.add_argument("--ragged-sweeps", type=int, default=2000)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--wpr", type=int, default=0,
                    help="warps per replica (0: the library's choice)")
    ap.add_argument("--no-class-update", action="store_true",
                    help="run two-level-flow instances with the table kernels")
    ap.add_argument("--mode", default="anneal", choices=["anneal", "cupim", "pt"],
                    help="sequential p-dit sweeps (the paper's PIM) or concurrent updates (its CUPIM)")
    ap.add_argument("--pk", type=int, default=0,
                    help="pending rank-1 terms held before a table rewrite (0: the library's choice)")
    ap.add_argument("--rpc", type=int, default=0,
                    help="replicas per CTA at most (0: the library's choice)")
    ap.add_argument("--dense-n", type=int, default=180, help="size of the 'dense' workload")
    ap.add_argument("--influence", default="auto", choices=["auto", "table", "products"],
                    help="influence entries: the library's choice, the incrementally updated table, "
                         "or dot products of byte rows (no table)")
    ap.add_argument("--place", type=int, default=0, choices=[0, 1, 2],
                    help="influence tables: 0 library's choice, 1 shared memory, 2 global memory")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="override the workload's sweep count (smaller cases for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args, args.workload if args.workload in WORKLOADS else "n100")
    if args.workload == "ragged":
        return run_ragged(args)
    if args.workload == "served":
        return run_served(args)

    import torch

    from paper_2605_24408_gb300 import build as B
    from paper_2605_24408_gb300 import pdit as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()

    inst, replicas, sweeps, kind = WORKLOADS[args.workload]
    if args.sweeps > 0:
        sweeps = args.sweeps
    D, F = G.dense_instance(args.dense_n, 0) if inst == "dense" else G.named(inst)
    n = D.shape[0]
    q = P.Qap(D, F)
    if args.no_class_update:
        P.pdit_set_class_update(q, False)
    class_path = (P.pdit_instance_form(q) == P.PDIT_FORM_FLOW_CLASSES and not args.no_class_update
                  and args.mode != "cupim")
    if args.wpr:
        P.pdit_set_warps_per_replica(q, args.wpr)
    if args.pk:
        P.pdit_set_pending_swaps(q, args.pk)
    if args.rpc:
        P.pdit_set_replicas_per_cta(q, args.rpc)
    if args.place:
        P.pdit_set_table_placement(q, args.place)
    infl = {"auto": P.PDIT_INFLUENCE_AUTO, "table": P.PDIT_INFLUENCE_TABLE,
            "products": P.PDIT_INFLUENCE_PRODUCTS}[args.influence]
    if args.mode == "cupim" and infl == P.PDIT_INFLUENCE_AUTO:
        infl = P.PDIT_INFLUENCE_TABLE  # concurrent updates run the table kernels: report their shape
    P.pdit_set_influence(q, infl)
    pt = args.mode == "pt"
    ladder = 10
    if pt:
        # the paper's mode: sets of 10 rungs on a ladder from its beta-range
        # selection (trial runs; untimed), exchange every 4 sweeps, timeout 100
        replicas -= replicas % ladder
        lo, hi, _ = P.pdit_beta_range(q)
        beta = P.pdit_beta_ladder(lo, hi, ladder)
    shape = P.pdit_launch_shape(q, replicas)
    if not pt:
        beta = P.pdit_beta_schedule(kind, sweeps, P.pdit_beta_max(q))
    dev = torch.device("cuda", local)
    dbeta = torch.from_numpy(beta).to(dev)
    base = rank * replicas
    stream = torch.cuda.current_stream(dev)
    outs = {"best_perm": torch.empty(n, dtype=torch.int32, device=dev),
            "best_cost": torch.empty(1, dtype=torch.int64, device=dev),
            "replica_accepted": torch.empty(replicas, dtype=torch.int64, device=dev),
            "replica_best_cost": torch.empty(replicas, dtype=torch.int64, device=dev),
            "replica_best_sweep": torch.empty(replicas, dtype=torch.int32, device=dev),
            "status": torch.zeros(1, dtype=torch.int32, device=dev)}
    mode_code = {"anneal": P.PDIT_MODE_ANNEAL, "cupim": P.PDIT_MODE_CUPIM, "pt": P.PDIT_MODE_PT}[args.mode]
    o = P.opts(replicas=replicas, sweeps=sweeps, seed=0, replica_base=base, beta=dbeta.data_ptr(),
               stream=stream.cuda_stream, mode=mode_code, ladder_len=ladder if pt else 0,
               exchange_period=4, timeout_periods=100)
    ws = torch.empty(P.pdit_workspace_bytes(q, o), dtype=torch.uint8, device=dev)
    o.workspace, o.workspace_bytes = ws.data_ptr(), ws.numel()
    for k, t in outs.items():
        setattr(o, k, t.data_ptr())
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # on-chip peaks of this GPU (a few milliseconds, before the timed region)
    try:
        peaks = P.pdit_probe_peaks(4000)
    except P.PditError:
        peaks = None

    def step():
        P.pdit_anneal_ex(q, o)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    status = int(outs["status"].item())
    if status != 0:
        raise SystemExit("device audit failed: status %d" % status)
    upd_rank = n * replicas * sweeps
    value = world * upd_rank * args.steps / (tot_ms / 1000.0)
    accepted = int(outs["replica_accepted"].sum().item())
    accept_frac = accepted / upd_rank

    # final answer over ranks (outside the timed region)
    best_cost = int(outs["best_cost"].item())
    rep_best = outs["replica_best_cost"].cpu().numpy()
    best_replica = base + multi.rank_winner(rep_best)
    if dist is not None:
        best_cost, best_replica, _ = multi.rank_result(rep_best, outs["best_perm"].cpu().numpy(), base, dev)

    # end to end, the whole user call per step: qap_create (H2D of D and F from
    # host memory), pdit_anneal (H2D of beta, D2H of the result), qap_destroy
    hD = torch.from_numpy(np.ascontiguousarray(D, np.int32)).pin_memory()
    hF = torch.from_numpy(np.ascontiguousarray(F, np.int32)).pin_memory()
    hbeta = torch.from_numpy(beta).pin_memory()
    hperm = torch.empty(n, dtype=torch.int32).pin_memory()
    hcost = torch.empty(1, dtype=torch.int64).pin_memory()
    e2e_t = []
    e2e_clocks = Clocks(local)
    e2e_clocks.start()
    for k in range(args.e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qe = P.qap_create_host_ptrs(n, hD.data_ptr(), hF.data_ptr())
        for setter, v in ((P.pdit_set_warps_per_replica, args.wpr), (P.pdit_set_pending_swaps, args.pk),
                          (P.pdit_set_replicas_per_cta, args.rpc), (P.pdit_set_table_placement, args.place),
                          (P.pdit_set_influence, infl)):
            if v:
                setter(qe, v)
        if args.no_class_update:
            P.pdit_set_class_update(qe, False)
        if args.mode == "anneal":
            rc = P.pdit_anneal_host_ptrs(qe, replicas, hbeta.data_ptr(), sweeps, 0, hperm.data_ptr(),
                                         hcost.data_ptr())
        else:
            # pdit_anneal runs the sequential sweep; other modes go through
            # pdit_anneal_ex with the host copies inside the timed region
            ebeta = hbeta.to(dev, non_blocking=True)
            eperm = torch.empty(n, dtype=torch.int32, device=dev)
            ecost = torch.empty(1, dtype=torch.int64, device=dev)
            eo = P.opts(replicas=replicas, sweeps=sweeps, seed=0, beta=ebeta.data_ptr(),
                        stream=stream.cuda_stream, mode=mode_code, ladder_len=ladder if pt else 0,
                        exchange_period=4, timeout_periods=100,
                        best_perm=eperm.data_ptr(), best_cost=ecost.data_ptr())
            P.pdit_anneal_ex(qe, eo)
            rc = 0
            hperm.copy_(eperm, non_blocking=True)
            hcost.copy_(ecost, non_blocking=True)
            torch.cuda.synchronize()
        qe.close()
        t1 = time.perf_counter()
        if rc != 0:
            raise SystemExit("pdit_anneal failed: %s" % P.strerror(rc))
        if k > 0:  # the first call also loads the kernels
            e2e_t.append(t1 - t0)
    e2e_clk = e2e_clocks.stop()
    e2e_val = world * upd_rank * len(e2e_t) / sum(e2e_t) if e2e_t else None
    if e2e_t and dist is None and int(hcost[0]) != int(outs["best_cost"].item()):
        raise SystemExit("host-buffer and device-buffer results differ")

    # roofline of the sweep kernel: shared-memory bound
    props = torch.cuda.get_device_properties(dev)
    dt_bytes = 1 if max(abs(int(D.max())), abs(int(F.max()))) <= 127 else 2
    general = not (np.array_equal(D, D.T) and np.array_equal(F, F.T))
    bpu = method_bytes_per_update(n, accept_frac, general)
    bpu_design = algorithmic_bytes_per_update(n, dt_bytes, accept_frac, shape["pending_swaps"], general)
    basis = (("16 N + A (8 N^2 + 16 N): the method's traffic with a rank-2 table rewrite per accepted swap "
              "(general form)") if general else
             "16 N + A (8 N^2 + 8 N): the method's traffic with a table rewrite per accepted swap")
    kname = "sweep_kernel<int8,%d,%d,%s,%d>" % (shape["candidates_per_thread"], shape["warps_per_replica"],
                                                "smem" if shape["tables_in_smem"] else "global",
                                                shape["pending_swaps"])
    products = shape.get("influence") == "products" and not class_path
    alu = None
    kernel_s = tot_ms / 1000.0 / args.steps
    if class_path:
        # the flow-class kernel keeps no table: its own traffic is the figure
        bpu = bpu_design = class_bytes_per_update(n, dt_bytes, accept_frac)
        basis = ("(17 + dt) N + A (2 N dt + 8 N): the flow-class kernel's gathers plus, per accepted "
                 "swap, at most two D rows and the G vector (A counts swaps within a class too)")
        kname = "class_kernel<int8,%d,%d>" % (shape["candidates_per_thread"], shape["warps_per_replica"])
    elif products:
        # no table: the kernel's own traffic is the design figure; the
        # method's figure stays the basis of `achieved`
        bpu_design = product_bytes_per_update(n, accept_frac)
        parts = dot_parts(replicas, shape["ctas"] * shape["replicas_per_cta"], 4 if pt else sweeps, pt)
        kname = dot_kernel_name(shape["candidates_per_thread"], shape["warps_per_replica"], n, parts)
        dp4a = product_dp4a_per_update(n)
        alu = {"op": "dp4a", "per_update": dp4a, "achieved_ops_per_s": dp4a * upd_rank / kernel_s}
    achieved = bpu * upd_rank / kernel_s / 1e9
    sm_mhz = clk.get("sm_mhz") or 0.0
    sms = props.multi_processor_count
    if peaks and sm_mhz:
        peak = sms * peaks["smem_bytes_per_clk_sm"] * sm_mhz * 1e6 / 1e9
        peak_source = ("measured: pdit_probe_peaks %.1f B/clk/SM (conflict-free 128-bit ld.shared) x %d SMs x "
                       "median SM clock under load (%s MHz)" % (peaks["smem_bytes_per_clk_sm"], sms, sm_mhz))
        if alu is not None:
            alu["peak_ops_per_s"] = sms * peaks["dp4a_ops_per_clk_sm"] * sm_mhz * 1e6
            alu["frac"] = alu["achieved_ops_per_s"] / alu["peak_ops_per_s"]
            alu["peak_source"] = "measured: pdit_probe_peaks %.1f dp4a/clk/SM x %d SMs x %s MHz" % (
                peaks["dp4a_ops_per_clk_sm"], sms, sm_mhz)
    else:
        peak = sms * SMEM_BYTES_PER_CLK * sm_mhz * 1e6 / 1e9 if sm_mhz else None
        peak_source = "derived: %d SMs x %d B/clk x median SM clock under load (%s MHz)" % (
            sms, SMEM_BYTES_PER_CLK, sm_mhz)
    traffic = None
    try:
        # the stored DRAM counters describe the default workload's kernel only
        if args.workload == "n100" and args.mode == "anneal" and not (args.wpr or args.pk or args.rpc or args.place):
            with open(TRAFFIC_FILE) as fh:
                tr = json.load(fh)
            if tr.get("kernel") == kname and tr.get("source_sha") == kernel_source_sha() and \
                    tr.get("launch") == shape:
                traffic = tr.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass

    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "%s%s: %s" % (args.workload, (" N=%d" % n) if inst == "dense" else "",
                                             WORKLOAD_TEXT[args.workload])
                   if args.workload in WORKLOAD_TEXT else args.workload,
                   "mode": args.mode,
                   "update": "flow classes" if class_path else ("dot products" if products else "table"),
                   "replicas_per_gpu": replicas, "sweeps": sweeps, "schedule": "pt ladder" if pt else kind, "seed": 0,
                   "global_batch": replicas * world, "seq_len": n,
                   "parallelism": "replicas sharded over %d GPU(s)" % world,
                   "l2": "flushed between timed steps (512 MiB write)",
                   "accept_fraction": accept_frac, "best_cost": best_cost, "best_replica": best_replica,
                   "launch": shape},
        "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": 8 * n * n + 4 * len(beta),
                "d2h_bytes_per_step": 4 * n + 8 + 4,
                "call": "qap_create + pdit_anneal + qap_destroy from pinned host buffers",
                "steps": len(e2e_t),
                "clocks": {"sm_mhz": e2e_clk.get("sm_mhz"), "reasons": e2e_clk.get("reasons")}},
        # per step: sweep kernel + final reduction; PT mode: the rung set-up,
        # one sweep kernel per exchange period (4 sweeps), one exchange kernel
        # per completed period, the final reduction
        "gpu_launches": args.steps * ((2 + -(-sweeps // 4) + sweeps // 4) if pt else 2),
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons"), "samples": clk.get("samples")},
        "roofline": {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if peak else None, "traffic": traffic,
                     "kernel": kname,
                     "bytes_per_update": bpu,
                     "bytes_per_update_basis": basis,
                     "design_bytes_per_update": bpu_design,
                     "design_frac": (bpu_design * upd_rank / kernel_s / 1e9 / peak) if peak else None,
                     "peak_source": peak_source, "alu": alu},
        "wall_s_timed_region": wall,
    }
    if pt:
        line["config"]["beta"] = "ladder of %d rungs from the beta-range selection, exchange every 4 sweeps, " \
                                 "top-rung timeout 100 periods; the CPU-baseline leg is omitted in this mode " \
                                 "(the oracle splits work by whole ladders; PT parity is in the GPU tests)" % ladder
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not pt:
        gpu = {k: outs[k].cpu().numpy() for k in ("replica_best_cost", "replica_best_sweep", "replica_accepted")}
        line["cpu_baseline"] = cpu_baseline(D, F, beta, n, sweeps, args.mode, gpu)
    if rank == 0:
        print(json.dumps(line), flush=True)
    q.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
