"""Targets of the ragged-batch time-to-1%-gap benchmark (bench.py --workload
ragged), written once to ragged.json beside this script.

For every instance k of the benchmark's batch (N uniform in 12..256, the
ragged generator keyed by k and seed 0) the target is the best cost of a
reference run that the benchmark's own runs never see: the same instance
annealed with 4x the replicas (1024), 2x the sweeps (4000, linear 0 ->
beta_max) and another random stream (seed 1). The benchmark then counts an
instance as solved when its best is within 1% of that target. These are
benchmark targets, not expected values: no test compares against them.

    python bench_targets/make_ragged.py            # on a GPU, about ten minutes
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2605_24408_gb300 import instances as G  # noqa: E402

OUT = os.path.join(HERE, "ragged.json")


def main():
    import torch

    from paper_2605_24408_gb300 import build as B
    from paper_2605_24408_gb300 import pdit as P

    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--replicas", type=int, default=1024)
    ap.add_argument("--sweeps", type=int, default=4000)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", 0)
    qs, items, sizes = [], [], []
    for k in range(args.instances):
        n = G.ragged_size(k, 0)
        D, F = G.ragged_instance(k, n, 0)
        q = P.Qap(D, F)
        beta = torch.from_numpy(P.pdit_beta_schedule("linear", args.sweeps, P.pdit_beta_max(q))).to(dev)
        qs.append(q)
        sizes.append(n)
        items.append(dict(qap=q, replicas=args.replicas, sweeps=args.sweeps, beta=beta, seed=args.seed,
                          instance_id=k))
    t0 = time.perf_counter()
    b = P.Batch(items)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        b.run(stream)
    stream.synchronize()
    secs = time.perf_counter() - t0
    best = [int(o["best_cost"].item()) for o in b.out]
    rec = {"what": "ragged-batch targets: best cost of a reference run per instance",
           "instances": "k = 0..%d, N = ragged_size(k, 0), ragged_instance(k, N, 0)" % (args.instances - 1),
           "reference_run": {"replicas": args.replicas, "sweeps": args.sweeps, "schedule": "linear 0 -> beta_max",
                             "seed": args.seed, "instance_id": "k", "seconds": secs},
           "targets": [{"k": k, "n": sizes[k], "best": best[k]} for k in range(args.instances)]}
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
    print("wrote %s (%d instances, %.0f s)" % (OUT, args.instances, secs))
    for q in qs:
        q.close()


if __name__ == "__main__":
    main()
