"""Pins of the concurrent-update conflict rule and of the final tie rule.

GPU-CUPIM Algorithm section: after every location has proposed a swap from
a snapshot of the swap energies, conflicts go to the larger energy decrease,
ties to the lower p-dit index, and losers stay. Hardware and Data Reporting
Details: the result is the best over the independent duplicates (reading R6:
ties to the lowest replica).

The instance below (N = 6, found by a search, then worked by hand) has a
conflict decided by the energy order, an equal-energy tie between two
initiating locations, and a pair proposed from both ends. With beta so
large that every weight but the minimum's is zero, each location proposes
the argmin of its row of swap energies (Eq. 5 in the beta -> infinity
limit), so the outcome of one iteration follows from the energy matrix
alone. The energy matrix is recomputed here from Eq. 1 by brute force.

Hand working (location space; p0 is the oracle's Fisher-Yates start for
seed 7, replica 0):

  proposals  0->2 (-6)  1->4 (-18)  2->1 (-16)  3->2 (-6)  4->1 (-18)  5->1 (-10)
  ascending by energy change, ties to the lower initiator:
    (1,4) -18  accept: 1 and 4 free
    (4,1) -18  the same pair from the other end: 4 and 1 taken, not again
    (2,1) -16  1 taken: loses, location 2 stays
    (5,1) -10  1 taken: loses
    (0,2)  -6  accept: 0 and 2 free
    (3,2)  -6  2 taken: loses (the tie with (0,2) went to location 0)
  applied: (1,4) then (0,2): p = [4, 0, 5, 3, 2, 1], E = 72, 2 accepted.

The plausible mistakes give other states (also worked by hand):
  descending order:          (0,2), (3,2) tie -> (0,2); then (5,1); (2,1) x;
                             (1,4) x -> p = [4, 1, 5, 3, 0, 2]
  ties to the higher index:  (1,4); (3,2) wins the -6 tie -> [5, 0, 3, 4, 2, 1]
  a both-ends pair twice:    (1,4) and (4,1) both applied (cancel); (0,2)
                             -> [4, 2, 5, 3, 0, 1]
"""

import numpy as np

import oracle as O

D = np.array([[0, 1, 1, 1, 3, 3],
              [1, 0, 2, 0, 0, 1],
              [1, 2, 0, 2, 3, 3],
              [1, 0, 2, 0, 2, 1],
              [3, 0, 3, 2, 0, 1],
              [3, 1, 3, 1, 1, 0]], dtype=np.int32)
F = np.array([[0, 3, 2, 3, 2, 2],
              [3, 0, 1, 1, 3, 1],
              [2, 1, 0, 1, 1, 0],
              [3, 1, 1, 0, 3, 1],
              [2, 3, 1, 3, 0, 3],
              [2, 1, 0, 1, 3, 0]], dtype=np.int32)
SEED = 7
P0 = [5, 2, 4, 3, 0, 1]
DE = [[0, 4, -6, 4, 12, 4],
      [4, 0, -16, -4, -18, -10],
      [-6, -16, 0, -6, 8, 8],
      [4, -4, -6, 0, -2, 0],
      [12, -18, 8, -2, 0, -2],
      [4, -10, 8, 0, -2, 0]]
PROPOSALS = {0: 2, 1: 4, 2: 1, 3: 2, 4: 1, 5: 1}
EXPECTED = [4, 0, 5, 3, 2, 1]
WRONG = {"descending": [4, 1, 5, 3, 0, 2],
         "ties_to_higher": [5, 0, 3, 4, 2, 1],
         "pair_twice": [4, 2, 5, 3, 0, 1]}
BIG_BETA = np.float32(1e30)


def eq1(p):
    """Eq. 1 written out: sum_ij D_ij F_p(i)p(j)."""
    p = np.asarray(p)
    return int((D.astype(np.int64) * F.astype(np.int64)[np.ix_(p, p)]).sum())


def swapped(p, i, j):
    q = list(p)
    q[i], q[j] = q[j], q[i]
    return q


def test_fixture_energies_by_brute_force():
    assert O.init_perm(6, SEED, 0, 0).tolist() == P0
    E0 = eq1(P0)
    de = [[eq1(swapped(P0, i, j)) - E0 if i != j else 0 for j in range(6)] for i in range(6)]
    assert de == DE
    # every row has one minimum (the stay outcome counts as 0), so at large
    # beta each location's proposal is that row's argmin
    for i in range(6):
        row = np.array(DE[i])
        assert (row == row.min()).sum() == 1
        assert int(row.argmin()) == PROPOSALS[i]


def test_large_beta_proposals_are_row_argmins():
    E0 = eq1(P0)
    for i in range(6):
        r = O.update_draw(SEED, 0, 0, 0, i)
        j, dE, w, _ = O.choose(D, F, P0, i, float(BIG_BETA), r)
        assert j == PROPOSALS[i]
        assert dE.tolist() == DE[i]
        assert eq1(swapped(P0, i, j)) - E0 == DE[i][j]


def test_conflicts_follow_the_rule():
    r = O.anneal(D, F, np.array([BIG_BETA], np.float32), 1, SEED, 0, 1, mode="cupim", tables=True)
    assert r["final_perm"][0].tolist() == EXPECTED
    assert int(r["final_cost"][0]) == eq1(EXPECTED) == 72
    assert int(r["accepted"][0]) == 2
    assert int(r["best_cost"][0]) == 72 and int(r["best_sweep"][0]) == 0
    # the table left behind is Eq. 2 of the final state
    assert np.array_equal(r["tables"][0], O.influence(D, F, EXPECTED))
    # the fixture tells the plausible mistakes apart
    for name, wrong in WRONG.items():
        assert wrong != EXPECTED, name
        assert sorted(wrong) == list(range(6)), name


def test_argmin_best_ties_go_to_the_lowest_replica():
    lib = O.lib()
    cases = [([9, 4, 6, 4, 4], 1), ([3, 3, 3], 0), ([5], 0), ([7, 8, 2, 2], 2),
             ([-1, -5, -5, 0, -5], 1), ([2 ** 40, 2 ** 40 - 1, 2 ** 40 - 1], 1)]
    for vals, want in cases:
        a = np.array(vals, dtype=np.int64)
        assert lib.oracle_argmin_best(len(a), a) == want, vals


def test_anneal_winner_is_lowest_tied_replica():
    # four replicas started at beta = 0 on an instance whose cost is the same
    # for every permutation (F = all ones off the diagonal): every best cost
    # ties, so the winner must be replica 0
    n = 5
    Dm = np.ones((n, n), np.int32) - np.eye(n, dtype=np.int32)
    r = O.anneal(Dm, Dm, np.zeros(3, np.float32), 3, 1, 0, 4)
    assert len(set(r["best_cost"].tolist())) == 1
    assert r["winner"] == 0
