"""GPU parity of the dot-product kernel (pdit_set_influence PRODUCTS): the
influence entries of every swap energy formed as 8-bit dot products of rows
of D and of the flow matrix permuted to location order, with no influence
table. Every replica's final and best permutation, costs, best sweep and
accepted count must equal the CPU oracle's (which keeps the table of Eq. 2 and
updates it incrementally), bit for bit, over sizes that span one to eight
candidates per thread and ragged tails, every compiled thread mapping, zero
and nonzero diagonals, negative entries, the sequential modes, resume, and
the time-to-target bookkeeping."""

import numpy as np
import pytest

import oracle as O
from paper_2605_24408_gb300 import instances as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24408_gb300 import build as B

    B.build()
    torch.cuda.set_device(0)


def P():
    from paper_2605_24408_gb300 import pdit

    return pdit


def run_products(D, F, beta, sweeps, seed, R, wpr=0, **kw):
    p = P()
    with p.Qap(D, F) as q:
        p.pdit_set_class_update(q, False)  # tiny instances can look like two-level flows
        p.pdit_set_influence(q, p.PDIT_INFLUENCE_PRODUCTS)
        if wpr:
            p.pdit_set_warps_per_replica(q, wpr)
        shape = p.pdit_launch_shape(q, R)
        assert shape["influence"] == "products"
        dbeta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda()
        out = p.anneal_device(q, R, dbeta, sweeps, seed, per_replica=True, **kw)
        torch.cuda.synchronize()
        res = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    res["shape"] = shape
    return res


def check_equal(g, r, rep_slice=slice(None)):
    assert int(g["status"][0]) == 0
    assert np.array_equal(g["replica_final_perm"][rep_slice], r["final_perm"])
    assert np.array_equal(g["replica_final_cost"][rep_slice], r["final_cost"])
    assert np.array_equal(g["replica_best_perm"][rep_slice], r["best_perm"])
    assert np.array_equal(g["replica_best_cost"][rep_slice], r["best_cost"])
    assert np.array_equal(g["replica_best_sweep"][rep_slice], r["best_sweep"])
    assert np.array_equal(g["replica_accepted"][rep_slice], r["accepted"])


def schedule(D, F, kind, sweeps):
    return O.beta_schedule(kind, sweeps, O.beta_max(D, F))


@pytest.mark.parametrize("n", [2, 3, 12, 31, 32, 33, 63, 64, 65, 99, 100, 101, 127, 128, 129, 190, 255, 256])
def test_sizes_dense(n):
    D, F = G.dense_instance(n, seed=n + 40)
    S = 8 if n > 128 else 20
    beta = schedule(D, F, "linear", S)
    R = 9
    g = run_products(D, F, beta, S, 3, R)
    r = O.anneal(D, F, beta, S, 3, 0, R, threads=R)
    check_equal(g, r)


@pytest.mark.parametrize("n,wpr", [(100, 1), (100, 2), (100, 4), (200, 2), (200, 4), (200, 8), (60, 1), (20, 1)])
def test_every_compiled_mapping(n, wpr):
    D, F = G.dense_instance(n, seed=n + 7)
    S = 6
    beta = schedule(D, F, "geometric", S)
    g = run_products(D, F, beta, S, 5, 7, wpr=wpr)
    assert g["shape"]["warps_per_replica"] == wpr
    r = O.anneal(D, F, beta, S, 5, 0, 7, threads=7)
    check_equal(g, r)


def test_named_workloads_sampled():
    for name, R, S, kind in [("n12", 64, 1000, "linear"), ("n30", 256, 600, "geometric")]:
        D, F = G.named(name)
        beta = schedule(D, F, kind, S)
        g = run_products(D, F, beta, S, 0, R)
        r = O.anneal(D, F, beta, S, 0, 0, R, threads=8)
        check_equal(g, r)
    D, F = G.named("n100")
    beta = schedule(D, F, "linear", 300)
    g = run_products(D, F, beta, 300, 0, 300)
    for lo, hi in [(0, 3), (297, 300)]:
        r = O.anneal(D, F, beta, 300, 0, lo, hi, threads=3)
        check_equal(g, r, slice(lo, hi))


@pytest.mark.parametrize("n", [10, 77, 140])
def test_negative_values_and_nonzero_diagonals(n):
    D = G.random_symmetric(n, -60, 70, seed=n, tag=3, diag=True)
    F = G.random_symmetric(n, -127, 127, seed=n, tag=4, diag=True)
    beta = schedule(D, F, "linear", 10)
    g = run_products(D, F, beta, 10, 9, 6)
    r = O.anneal(D, F, beta, 10, 9, 0, 6, threads=6)
    check_equal(g, r)


def test_fixed_beta_and_parallel_tempering():
    D, F = G.dense_instance(70, seed=4)
    bm = O.beta_max(D, F)
    rbeta = np.array([bm * f for f in (0.0, 0.1, 0.5, 1.0, 3.0, 30.0)], np.float32)
    g = run_products(D, F, rbeta, 12, 2, 6, mode=P().PDIT_MODE_FIXED)
    r = O.anneal(D, F, rbeta, 12, 2, 0, 6, threads=6, mode="fixed")
    check_equal(g, r)
    ladder = O.beta_schedule("geometric", 5, bm)
    g = run_products(D, F, ladder, 22, 6, 10, mode=P().PDIT_MODE_PT, ladder_len=5, exchange_period=4,
                     timeout_periods=2)
    r = O.anneal(D, F, ladder, 22, 6, 0, 10, threads=10, mode="pt", ladder_len=5, period=4, timeout=2)
    check_equal(g, r)
    assert np.array_equal(g["replica_rung"], r["rung"])


def test_resume_continues_bit_identically():
    D, F = G.dense_instance(100, seed=8)
    beta = schedule(D, F, "linear", 30)
    p = P()
    R = 20
    with p.Qap(D, F) as q:
        p.pdit_set_class_update(q, False)
        p.pdit_set_influence(q, p.PDIT_INFLUENCE_PRODUCTS)
        dbeta = torch.from_numpy(beta).cuda()
        first = p.anneal_device(q, R, dbeta, 30, 4, per_replica=True, sweep_end=13)
        rest = p.anneal_device(q, R, dbeta, 30, 4, per_replica=True, sweep_begin=13, resume=True,
                               workspace=first["workspace"])
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in rest.items() if k != "workspace"}
    r = O.anneal(D, F, beta, 30, 4, 0, R, threads=8)
    check_equal(g, r)


def test_zero_sweeps_and_beta_extremes():
    D, F = G.dense_instance(40, seed=1)
    g = run_products(D, F, np.zeros(0, np.float32), 0, 7, 5)
    r = O.anneal(D, F, np.zeros(0, np.float32), 0, 7, 0, 5)
    check_equal(g, r)
    for b in (0.0, 1e30):
        beta = np.full(5, b, np.float32)
        g = run_products(D, F, beta, 5, 7, 5)
        r = O.anneal(D, F, beta, 5, 7, 0, 5, threads=5)
        check_equal(g, r)


def test_target_bookkeeping_matches_the_oracle():
    D, F = G.named("n30")
    beta = schedule(D, F, "geometric", 200)
    R = 32
    r = O.anneal(D, F, beta, 200, 1, 0, R, threads=8)
    target = int(np.sort(r["best_cost"])[R // 2])
    ro = O.anneal(D, F, beta, 200, 1, 0, R, threads=8, target=target)
    tg = torch.tensor([target], dtype=torch.int64, device="cuda")
    g = run_products(D, F, beta, 200, 1, R, target=tg)
    check_equal(g, r)
    assert int(g["reach_sweep"][0]) == int(ro["reach_sweep"].min())


def test_auto_choice_and_table_knobs():
    """Automatic choice: products for a symmetric byte-valued instance, the
    table once a table knob is set, for entries beyond a byte, for the
    general form and for the concurrent-update mode; results equal."""
    p = P()
    D, F = G.dense_instance(100, seed=3)
    beta = schedule(D, F, "linear", 10)
    dbeta = torch.from_numpy(beta).cuda()
    outs = []
    for knob in (None, "table", "pk", "place"):
        with p.Qap(D, F) as q:
            if knob == "table":
                p.pdit_set_influence(q, p.PDIT_INFLUENCE_TABLE)
            elif knob == "pk":
                p.pdit_set_pending_swaps(q, 1)
            elif knob == "place":
                p.pdit_set_table_placement(q, p.PDIT_PLACE_SHARED)
            shape = p.pdit_launch_shape(q, 64)
            assert shape["influence"] == ("products" if knob is None else "table")
            out = p.anneal_device(q, 12, dbeta, 10, 2, per_replica=True)
            torch.cuda.synchronize()
            outs.append({k: v.cpu().numpy() for k, v in out.items() if k != "workspace"})
    r = O.anneal(D, F, beta, 10, 2, 0, 12, threads=12)
    for g in outs:
        check_equal(g, r)
    wide = G.random_symmetric(50, 0, 300, seed=2, tag=9)
    with p.Qap(wide, wide) as q:
        assert p.pdit_launch_shape(q, 64)["influence"] == "table"
        p.pdit_set_influence(q, p.PDIT_INFLUENCE_PRODUCTS)
        with pytest.raises(p.PditError):
            p.pdit_launch_shape(q, 64)


def test_resume_across_kernels():
    """A call with the dot kernel continued by the table kernels (and the
    reverse) on the same workspace: the state the two keep between calls is
    the same, so the continuation equals one uninterrupted oracle run."""
    D, F = G.dense_instance(90, seed=12)
    beta = schedule(D, F, "linear", 24)
    p = P()
    R = 12
    r = O.anneal(D, F, beta, 24, 6, 0, R, threads=8)
    for first, second in ((p.PDIT_INFLUENCE_PRODUCTS, p.PDIT_INFLUENCE_TABLE),
                          (p.PDIT_INFLUENCE_TABLE, p.PDIT_INFLUENCE_PRODUCTS)):
        with p.Qap(D, F) as q:
            p.pdit_set_class_update(q, False)
            dbeta = torch.from_numpy(beta).cuda()
            p.pdit_set_influence(q, first)
            a = p.anneal_device(q, R, dbeta, 24, 6, per_replica=True, sweep_end=10)
            p.pdit_set_influence(q, second)
            b = p.anneal_device(q, R, dbeta, 24, 6, per_replica=True, sweep_begin=10, resume=True,
                                workspace=a["workspace"])
            torch.cuda.synchronize()
            g = {k: v.cpu().numpy() for k, v in b.items() if k != "workspace"}
        check_equal(g, r)


def test_pt_resume_across_kernels():
    """Parallel tempering in two calls, the first with one kernel and the
    second with the other; within each call the dot kernel keeps its permuted
    flow matrices from one exchange period to the next. The rung assignment
    and every replica's state equal one uninterrupted oracle run."""
    D, F = G.dense_instance(64, seed=21)
    bm = O.beta_max(D, F)
    ladder = O.beta_schedule("geometric", 4, bm)
    p = P()
    R, S, cut = 12, 26, 10
    r = O.anneal(D, F, ladder, S, 8, 0, R, threads=R, mode="pt", ladder_len=4, period=3, timeout=2)
    kw = dict(mode=p.PDIT_MODE_PT, ladder_len=4, exchange_period=3, timeout_periods=2)
    for first, second in ((p.PDIT_INFLUENCE_PRODUCTS, p.PDIT_INFLUENCE_TABLE),
                          (p.PDIT_INFLUENCE_TABLE, p.PDIT_INFLUENCE_PRODUCTS),
                          (p.PDIT_INFLUENCE_PRODUCTS, p.PDIT_INFLUENCE_PRODUCTS)):
        with p.Qap(D, F) as q:
            p.pdit_set_class_update(q, False)
            dbeta = torch.from_numpy(ladder).cuda()
            p.pdit_set_influence(q, first)
            # room for either kernel's tables: the second call may need more
            ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
            a = p.anneal_device(q, R, dbeta, S, 8, per_replica=True, sweep_end=cut, workspace=ws, **kw)
            p.pdit_set_influence(q, second)
            b = p.anneal_device(q, R, dbeta, S, 8, per_replica=True, sweep_begin=cut, resume=True,
                                workspace=a["workspace"], **kw)
            torch.cuda.synchronize()
            g = {k: v.cpu().numpy() for k, v in b.items() if k != "workspace"}
        check_equal(g, r)
        assert np.array_equal(g["replica_rung"], r["rung"])


def _slots(p, q):
    """Resident replica slots of the dot kernel on this GPU (CTAs x replicas
    per CTA when the replicas exceed what fits at once)."""
    shape = p.pdit_launch_shape(q, 1 << 20)
    return shape["ctas"] * shape["replicas_per_cta"]


@pytest.mark.parametrize("n,S,kind", [(40, 40, "linear"), (100, 24, "geometric"), (13, 16, "linear")])
def test_more_replicas_than_slots_runs_in_parts(n, S, kind):
    """With more replicas than resident slots (not a whole number of rounds)
    each replica's sweeps run as several work units of one launch, each part
    resuming from the state the previous part published. Replicas of the
    first and of the last round equal the oracle's."""
    D, F = G.dense_instance(n, seed=n + 11)
    beta = schedule(D, F, kind, S)
    p = P()
    with p.Qap(D, F) as q:
        p.pdit_set_class_update(q, False)
        p.pdit_set_influence(q, p.PDIT_INFLUENCE_PRODUCTS)
        R = _slots(p, q) + 37
        dbeta = torch.from_numpy(beta).cuda()
        out = p.anneal_device(q, R, dbeta, S, 5, per_replica=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    for lo, hi in [(0, 3), (R - 40, R - 37), (R - 3, R)]:
        r = O.anneal(D, F, beta, S, 5, lo, hi, threads=3)
        check_equal(g, r, slice(lo, hi))
    assert int(g["best_cost"][0]) <= int(g["replica_best_cost"].min())


def test_parts_with_resume_and_fixed_beta():
    """Parts inside a resumed call (the range [sweep_begin, sweep_end) split)
    and in fixed-beta mode: still the oracle's results."""
    D, F = G.dense_instance(48, seed=3)
    p = P()
    S = 30
    beta = schedule(D, F, "linear", S)
    with p.Qap(D, F) as q:
        p.pdit_set_class_update(q, False)
        R = _slots(p, q) + 5
        dbeta = torch.from_numpy(beta).cuda()
        a = p.anneal_device(q, R, dbeta, S, 9, per_replica=True, sweep_end=17)
        b = p.anneal_device(q, R, dbeta, S, 9, per_replica=True, sweep_begin=17, resume=True,
                            workspace=a["workspace"])
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in b.items() if k != "workspace"}
        bm = O.beta_max(D, F)
        fb = np.array([bm * (0.2 + 0.01 * (i % 50)) for i in range(R)], np.float32)
        f = p.anneal_device(q, R, torch.from_numpy(fb).cuda(), 16, 4, per_replica=True, mode=p.PDIT_MODE_FIXED)
        torch.cuda.synchronize()
        gf = {k: v.cpu().numpy() for k, v in f.items() if k != "workspace"}
    for lo, hi in [(0, 2), (R - 2, R)]:
        r = O.anneal(D, F, beta, S, 9, lo, hi, threads=2)
        check_equal(g, r, slice(lo, hi))
        rf = O.anneal(D, F, fb[lo:hi], 16, 4, lo, hi, threads=2, mode="fixed")  # beta of the k-th replica
        check_equal(gf, rf, slice(lo, hi))


def test_parallel_tempering_in_parts():
    """Parallel tempering with more replicas than slots: each exchange
    period's launch runs every replica's sweeps as one-sweep parts. Ladders
    of the first and of the last round, with their rungs, equal the
    oracle's."""
    D, F = G.dense_instance(40, seed=17)
    bm = O.beta_max(D, F)
    L = 5
    ladder = O.beta_schedule("geometric", L, bm)
    p = P()
    S = 13
    with p.Qap(D, F) as q:
        p.pdit_set_class_update(q, False)
        R = -(-(_slots(p, q) + 37) // L) * L
        out = p.anneal_device(q, R, torch.from_numpy(ladder).cuda(), S, 3, per_replica=True,
                              mode=p.PDIT_MODE_PT, ladder_len=L, exchange_period=4, timeout_periods=2)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    for lo, hi in [(0, L), (R - L, R)]:
        r = O.anneal(D, F, ladder, S, 3, lo, hi, threads=L, mode="pt", ladder_len=L, period=4, timeout=2)
        check_equal(g, r, slice(lo, hi))
        assert np.array_equal(g["replica_rung"][lo:hi], r["rung"])


def test_resume_from_a_whole_call_into_parts():
    """A short call (too few sweeps to split) continued by a longer one that
    is split into parts, on the first call's workspace: the workspace does not
    depend on the sweep range, and the continuation equals one uninterrupted
    oracle run."""
    D, F = G.dense_instance(40, seed=29)
    S, cut = 40, 6
    beta = schedule(D, F, "linear", S)
    p = P()
    with p.Qap(D, F) as q:
        p.pdit_set_class_update(q, False)
        R = _slots(p, q) + 5
        dbeta = torch.from_numpy(beta).cuda()
        a = p.anneal_device(q, R, dbeta, S, 4, per_replica=True, sweep_end=cut)
        b = p.anneal_device(q, R, dbeta, S, 4, per_replica=True, sweep_begin=cut, resume=True,
                            workspace=a["workspace"])
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in b.items() if k != "workspace"}
    for lo, hi in [(0, 2), (R - 2, R)]:
        r = O.anneal(D, F, beta, S, 4, lo, hi, threads=2)
        check_equal(g, r, slice(lo, hi))
