"""Pins of the oracle's general form (D or F not symmetric, any diagonal):
Eq. 2 taken with both of its terms and Eq. 3 as printed. Pinned against the
plain definition of Eq. 1 (hand-worked values and brute-force recomputation),
a closed form of Eq. 2, and an exact reduction to the symmetric form, which
test_oracle_pins.py pins on its own. No GPU needed."""

import itertools

import numpy as np
import pytest

import oracle as O
from paper_2605_24408_gb300 import instances as G


def _asym(n, lo, hi, seed, diag=True):
    """Independent entries (no symmetry), drawn from the seeded hash."""
    idx = np.arange(n * n, dtype=np.uint64)
    M = G.hash_int(seed, 901, idx, lo, hi).reshape(n, n)
    if not diag:
        M[np.arange(n), np.arange(n)] = 0
    return M.astype(np.int32)


def test_cost_hand_worked_asymmetric_example():
    # E(p) = sum_ij D[i][j] F[p(i)][p(j)], worked by hand:
    # identity: 1*7 + 2*0 + 3*1 + 4*2 + 5*0 + 6*3 = 36
    # p = (1, 2, 0): D01 F12 + D02 F10 + D10 F21 + D12 F20 + D20 F01 + D21 F02
    #              = 1*2 + 2*1 + 3*3 + 4*0 + 5*7 + 6*0 = 48
    D = np.array([[0, 1, 2], [3, 0, 4], [5, 6, 0]], np.int32)
    F = np.array([[0, 7, 0], [1, 0, 2], [0, 3, 0]], np.int32)
    assert O.cost(D, F, [0, 1, 2]) == 36
    assert O.cost(D, F, [1, 2, 0]) == 48
    assert O.general_form(D, F)
    # Eq. 3 between the two: p = (1, 2, 0) is not one swap away from the
    # identity, but (1, 0, 2) is:
    # E(1,0,2) = D01 F10 + D02 F12 + D10 F01 + D12 F02 + D20 F21 + D21 F20
    #          = 1*1 + 2*2 + 3*7 + 4*0 + 5*3 + 6*0 = 41
    assert O.cost(D, F, [1, 0, 2]) == 41
    Ip = O.influence_eq2(D, F, [0, 1, 2])
    assert O.delta_e_eq3(D, F, [0, 1, 2], Ip, 0, 1) == 41 - 36


def test_eq2_table_closed_form():
    # sum_m Ip[m][p(m)] = -2 E(p) for any D, F (each product of Eq. 1 appears
    # once in each of Eq. 2's two terms).
    for n, seed in [(5, 1), (8, 2), (13, 3)]:
        D, F = _asym(n, -20, 40, seed), _asym(n, -9, 30, seed + 50)
        for rep in range(4):
            p = O.init_perm(n, seed, 0, rep)
            Ip = O.influence_eq2(D, F, p)
            assert int(Ip[np.arange(n), p].sum()) == -2 * O.cost(D, F, p)


@pytest.mark.parametrize("n", [2, 3, 4, 7, 9])
@pytest.mark.parametrize("diag", [False, True])
def test_eq3_general_equals_brute_recomputation(n, diag):
    D, F = _asym(n, -15, 60, 10 + n, diag), _asym(n, -7, 25, 20 + n, diag)
    for rep in range(3):
        p = O.init_perm(n, 3, 1, rep)
        Ip = O.influence_eq2(D, F, p)
        e0 = O.cost(D, F, p)
        for i, j in itertools.product(range(n), range(n)):
            q = p.copy()
            q[i], q[j] = q[j], q[i]
            assert O.delta_e_eq3(D, F, p, Ip, i, j) == O.cost(D, F, q) - e0


def test_general_form_incremental_tables_and_costs():
    n = 11
    D, F = _asym(n, 0, 50, 5), _asym(n, 0, 20, 6)
    beta = O.beta_schedule("linear", 25, O.beta_max(D, F))
    r = O.anneal(D, F, beta, 25, 7, 0, 6, tables=True)
    assert r["general"]
    for k in range(6):
        fp, bp = r["final_perm"][k], r["best_perm"][k]
        assert sorted(fp) == list(range(n)) and sorted(bp) == list(range(n))
        assert r["final_cost"][k] == O.cost(D, F, fp)
        assert r["best_cost"][k] == O.cost(D, F, bp)
        assert np.array_equal(r["tables"][k], O.influence_eq2(D, F, fp))
    assert r["accepted"].min() > 0


def test_general_form_on_symmetric_input_matches_symmetric_form():
    # For symmetric D and F, Eq. 2's table is -2 I and Eq. 3 gives the same
    # exact energies, so the two forms follow the same trajectory.
    D, F = G.named("n12")
    beta = O.beta_schedule("linear", 30, O.beta_max(D, F))
    a = O.anneal(D, F, beta, 30, 4, 0, 5, tables=True)
    b = O.anneal(D, F, beta, 30, 4, 0, 5, tables=True, form="general")
    assert not a["general"] and b["general"]
    for key in ("final_perm", "final_cost", "best_perm", "best_cost", "best_sweep", "accepted"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(b["tables"], -2 * a["tables"])


@pytest.mark.parametrize("side", ["F", "D"])
def test_one_sided_asymmetry_reduces_to_symmetric_form(side):
    # With D symmetric, E(D, F) = E(D, F + F^T) / 2 for every permutation, so
    # every swap energy is exactly half; (float)(2k) * (beta / 2) rounds the
    # same as (float)k * beta, so the general-form run on (D, F) at beta equals
    # the symmetric-form run on (D, F + F^T) at beta / 2, draw for draw. The
    # same holds with the roles of D and F exchanged.
    n = 10
    S = G.random_symmetric(n, 0, 30, seed=8, tag=3)
    A = _asym(n, 0, 25, 9, diag=False)
    if side == "F":
        D, F, Ds, Fs = S, A, S, A + A.T
    else:
        D, F, Ds, Fs = A, S, A + A.T, S
    assert O.general_form(D, F) and not O.general_form(Ds, Fs)
    beta = O.beta_schedule("linear", 40, O.beta_max(D, F))
    r = O.anneal(D, F, beta, 40, 12, 0, 6)
    s = O.anneal(Ds, Fs, (beta / np.float32(2)).astype(np.float32), 40, 12, 0, 6)
    for key in ("final_perm", "best_perm", "best_sweep", "accepted"):
        assert np.array_equal(r[key], s[key]), key
    assert np.array_equal(2 * r["best_cost"], s["best_cost"])
    # beta_max halves the mean positive swap energy's reciprocal exactly
    assert O.beta_max(D, F) == 2 * O.beta_max(Ds, Fs)


def test_general_form_reaches_brute_force_optimum():
    n = 8
    D, F = _asym(n, 0, 9, 31, diag=True), _asym(n, 0, 9, 32, diag=True)
    opt, perm, _ = O.brute_force(D, F)
    assert O.cost(D, F, perm) == opt
    beta = O.beta_schedule("linear", 200, O.beta_max(D, F))
    r = O.anneal(D, F, beta, 200, 1, 0, 16, threads=4)
    assert (r["best_cost"] >= opt).all()
    assert r["cost"] == opt


def test_general_form_pt_and_cupim_invariants():
    n = 9
    D, F = _asym(n, -5, 30, 41), _asym(n, 0, 12, 42)
    ladder = O.beta_grid(4, 0.001, 0.2)
    r = O.anneal(D, F, ladder, 24, 3, 0, 8, mode="pt", ladder_len=4, tables=True)
    c = O.anneal(D, F, O.beta_schedule("linear", 24, O.beta_max(D, F)), 24, 3, 0, 4,
                 mode="cupim", tables=True)
    for res in (r, c):
        for k in range(len(res["final_cost"])):
            fp = res["final_perm"][k]
            assert res["final_cost"][k] == O.cost(D, F, fp)
            assert res["best_cost"][k] == O.cost(D, F, res["best_perm"][k])
            assert np.array_equal(res["tables"][k], O.influence_eq2(D, F, fp))
