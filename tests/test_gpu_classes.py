"""GPU parity of the flow-class kernel (two-level flow, Methods section's
tai256c paragraph): every replica's permutations, costs, best sweep and
accepted-move count equal the oracle's plain run (which keeps the full
table), and equal the table kernels' results on the same handle."""

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


def gpu_run(D, F, beta, sweeps, seed, R, wpr=0, classes=True, expect_form=None, **kw):
    p = P()
    with p.Qap(D, F) as q:
        if expect_form is not None:
            assert p.pdit_instance_form(q) == expect_form
        p.pdit_set_class_update(q, classes)
        if wpr:
            p.pdit_set_warps_per_replica(q, wpr)
        dbeta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda()
        out = p.anneal_device(q, R, dbeta, sweeps, seed, per_replica=True, **kw)
        torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}


def check_equal(g, r):
    assert int(g["status"][0]) == 0
    for gk, rk in [("replica_final_perm", "final_perm"), ("replica_final_cost", "final_cost"),
                   ("replica_best_perm", "best_perm"), ("replica_best_cost", "best_cost"),
                   ("replica_best_sweep", "best_sweep"), ("replica_accepted", "accepted")]:
        assert np.array_equal(g[gk], r[rk]), gk


def schedule(D, F, sweeps, scale=1.0):
    return O.beta_schedule("linear", sweeps, O.beta_max(D, F)) * np.float32(scale)


def test_forms_are_detected():
    p = P()
    cases = [(G.flow_class_instance(20, 7, seed=1), p.PDIT_FORM_FLOW_CLASSES),
             (G.flow_class_instance(20, 7, seed=1, f0=3, f=-2, fdiag=9), p.PDIT_FORM_FLOW_CLASSES),
             (G.flow_class_instance(20, 0, seed=1, f0=5), p.PDIT_FORM_FLOW_CLASSES),
             (G.dense_instance(20, seed=1), p.PDIT_FORM_SYMMETRIC),
             (G.asymmetric_instance(20, seed=1), p.PDIT_FORM_GENERAL)]
    D, F = G.flow_class_instance(20, 7, seed=1)
    Dd = D.copy()
    Dd[3, 3] = 1  # D's diagonal must be zero for the class form
    cases.append(((Dd, F), p.PDIT_FORM_SYMMETRIC))
    F3 = F.copy()
    F3[0, 1] = F3[1, 0] = 2  # a third flow value
    cases.append(((D, F3), p.PDIT_FORM_SYMMETRIC))
    for (A, B), form in cases:
        with p.Qap(A, B) as q:
            assert p.pdit_instance_form(q) == form


@pytest.mark.parametrize("n,k", [(2, 1), (2, 2), (3, 2), (12, 5), (31, 10), (33, 33), (64, 20), (100, 36),
                                 (129, 50), (200, 71), (256, 92), (256, 0), (256, 255)])
def test_sizes_and_class_sizes(n, k):
    D, F = G.flow_class_instance(n, k, seed=n + k)
    sweeps = 8
    beta = schedule(D, F, sweeps, 0.5)
    g = gpu_run(D, F, beta, sweeps, 3, 6, expect_form=P().PDIT_FORM_FLOW_CLASSES)
    r = O.anneal(D, F, beta, sweeps, 3, 0, 6, threads=6)
    check_equal(g, r)


@pytest.mark.parametrize("wpr", [1, 2, 4, 8])
def test_every_thread_mapping_and_table_path_agree(wpr):
    D, F = G.flow_class_instance(256, 92, seed=7, f0=2, f=3, fdiag=5)
    beta = schedule(D, F, 6)
    g = gpu_run(D, F, beta, 6, 11, 5, wpr=wpr)
    t = gpu_run(D, F, beta, 6, 11, 5, classes=False)
    r = O.anneal(D, F, beta, 6, 11, 0, 5, threads=5)
    check_equal(g, r)
    check_equal(t, r)


@pytest.mark.parametrize("lo,hi", [(0, 99), (0, 3000), (-500, 500)])
def test_value_ranges(lo, hi):
    D, F = G.flow_class_instance(60, 25, seed=4, lo=lo, hi=hi, f0=-1, f=2)
    beta = schedule(D, F, 20)
    g = gpu_run(D, F, beta, 20, 9, 8)
    r = O.anneal(D, F, beta, 20, 9, 0, 8, threads=8)
    check_equal(g, r)


def test_long_anneal_resume_and_fixed_beta():
    D, F = G.flow_class_instance(90, 30, seed=2)
    beta = schedule(D, F, 60)
    r = O.anneal(D, F, beta, 60, 4, 0, 12, threads=6)
    check_equal(gpu_run(D, F, beta, 60, 4, 12), r)
    p = P()
    with p.Qap(D, F) as q:
        dbeta = torch.from_numpy(beta).cuda()
        first = p.anneal_device(q, 12, dbeta, 60, 4, sweep_end=25, per_replica=True)
        ws = first["workspace"]
        second = p.anneal_device(q, 12, dbeta, 60, 4, sweep_begin=25, resume=True, workspace=ws,
                                 per_replica=True)
        torch.cuda.synchronize()
        assert np.array_equal(second["replica_best_cost"].cpu().numpy(), r["best_cost"])
        assert np.array_equal(second["replica_final_perm"].cpu().numpy(), r["final_perm"])
        assert int(second["status"].item()) == 0
    bm = O.beta_max(D, F)
    betas = np.float32([bm * f for f in (0.0, 0.1, 1.0, 10.0)])
    g = gpu_run(D, F, betas, 30, 12, 4, mode=2)
    r = O.anneal(D, F, betas, 30, 12, 0, 4, mode="fixed", threads=4)
    check_equal(g, r)


def test_parallel_tempering():
    D, F = G.flow_class_instance(70, 25, seed=3)
    bm = O.beta_max(D, F)
    L = 5
    ladder = np.float32([bm * 0.05 * (20.0 ** (q / (L - 1))) for q in range(L)])
    g = gpu_run(D, F, ladder, 26, 5, 20, mode=1, ladder_len=L, exchange_period=4, timeout_periods=2)
    r = O.anneal(D, F, ladder, 26, 5, 0, 20, mode="pt", ladder_len=L, period=4, timeout=2, threads=4)
    check_equal(g, r)
    assert np.array_equal(g["replica_rung"], r["rung"])


def test_table_dump_and_concurrent_mode_use_the_table_kernels():
    D, F = G.flow_class_instance(40, 15, seed=6)
    beta = schedule(D, F, 10)
    g = gpu_run(D, F, beta, 10, 2, 4, tables=True)
    r = O.anneal(D, F, beta, 10, 2, 0, 4, threads=4, tables=True)
    check_equal(g, r)
    assert np.array_equal(g["tables"].astype(np.int64), r["tables"])
    g = gpu_run(D, F, beta, 10, 2, 4, mode=3)
    r = O.anneal(D, F, beta, 10, 2, 0, 4, mode="cupim", threads=4)
    check_equal(g, r)


def test_stop_at_target_on_the_class_path():
    D, F = G.flow_class_instance(80, 30, seed=9)
    beta = schedule(D, F, 300)
    p = P()
    with p.Qap(D, F) as q:
        dbeta = torch.from_numpy(beta).cuda()
        full = p.anneal_device(q, 32, dbeta, 300, 5, per_replica=True)
        torch.cuda.synchronize()
        target = int(full["best_cost"].item() * 1.02)
        dt = torch.tensor([target], dtype=torch.int64, device="cuda")
        early = p.anneal_device(q, 32, dbeta, 300, 5, target=dt, stop_at_target=True, per_replica=True)
        torch.cuda.synchronize()
        assert int(early["best_cost"].item()) <= target
        assert 0 <= int(early["reach_sweep"].item()) < 300
        assert int(early["replica_accepted"].sum().item()) < int(full["replica_accepted"].sum().item())
        # without stopping, the first sweep at which any replica reaches the
        # target is the oracle's
        noted = p.anneal_device(q, 32, dbeta, 300, 5, target=dt, per_replica=True)
        torch.cuda.synchronize()
    r = O.anneal(D, F, beta, 300, 5, 0, 32, threads=8, target=target)
    assert int(noted["reach_sweep"].item()) == int(r["reach_sweep"].min())
