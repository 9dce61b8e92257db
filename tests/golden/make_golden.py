"""Writes the stored expected values under tests/golden/ that are too slow to
recompute in every test run. Calls only the CPU oracle (and the seeded
instance generator for its inputs).

    python tests/golden/make_golden.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2605_24408_gb300 import instances as G  # noqa: E402


def n12_optimum():
    D, F = G.named("n12")
    t = time.time()
    best, perm, cnt = O.brute_force(D, F)
    with open(os.path.join(HERE, "n12_optimum.txt"), "w") as fh:
        fh.write("# Brute-force minimum of Eq. 1 over all 12! permutations of the 3x4-grid\n")
        fh.write("# instance (instances.named('n12', seed=0)); written by make_golden.py\n")
        fh.write("# in %.0f s with oracle.brute_force.\n" % (time.time() - t))
        fh.write("optimum %d\n" % best)
        fh.write("perm %s\n" % ",".join(str(int(x)) for x in perm))
        fh.write("optimal_permutations %d\n" % cnt)


def ragged_optima(instances=256):
    """Brute-force optima of the ragged-batch instances with N <= 12 (the
    time-to-1%-gap target for those sizes; larger ones take the best of a
    long reference run instead)."""
    rows = []
    t = time.time()
    for k in range(instances):
        n = G.ragged_size(k, 0)
        if n > 12:
            continue
        D, F = G.ragged_instance(k, n, 0)
        best, perm, cnt = O.brute_force(D, F)
        rows.append((k, n, best, cnt))
    with open(os.path.join(HERE, "ragged_optima.txt"), "w") as fh:
        fh.write("# Brute-force minimum of Eq. 1 over all N! permutations of every instance\n")
        fh.write("# with N <= 12 among the %d of the ragged batch (instances.ragged_instance(k,\n" % instances)
        fh.write("# ragged_size(k, 0), 0)); written by make_golden.py in %.0f s with\n" % (time.time() - t))
        fh.write("# oracle.brute_force. Columns: k n optimum optimal_permutations\n")
        for k, n, best, cnt in rows:
            fh.write("%d %d %d %d\n" % (k, n, best, cnt))


if __name__ == "__main__":
    n12_optimum()
    ragged_optima()
