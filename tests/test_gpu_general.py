"""GPU parity for the general QAP form (D or F not symmetric, any diagonal):
the CUDA path keeps the two-term table T of Eq. 2 (T = -Ip, the oracle's
table negated) and applies each swap as a rank-2 update; every replica's
permutations, costs, best sweep, accepted-move count and table must equal the
oracle's. Integers, so the bar is bit-exact."""

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


def gpu_run(D, F, beta, sweeps, seed, R, tables=False, wpr=0, pk=0, **kw):
    p = P()
    with p.Qap(D, F) as q:
        if wpr:
            p.pdit_set_warps_per_replica(q, wpr)
        if pk:
            p.pdit_set_pending_swaps(q, pk)
        dbeta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda()
        out = p.anneal_device(q, R, dbeta, sweeps, seed, per_replica=True, tables=tables, **kw)
        torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}


def check_equal(g, r, tables=False):
    assert r["general"]
    assert int(g["status"][0]) == 0
    assert np.array_equal(g["replica_final_perm"], r["final_perm"])
    assert np.array_equal(g["replica_final_cost"], r["final_cost"])
    assert np.array_equal(g["replica_best_perm"], r["best_perm"])
    assert np.array_equal(g["replica_best_cost"], r["best_cost"])
    assert np.array_equal(g["replica_best_sweep"], r["best_sweep"])
    assert np.array_equal(g["replica_accepted"], r["accepted"])
    if tables:
        assert np.array_equal(g["tables"].astype(np.int64), -r["tables"])


def schedule(D, F, sweeps, scale=1.0):
    return O.beta_schedule("linear", sweeps, O.beta_max(D, F)) * np.float32(scale)


@pytest.mark.parametrize("n", [2, 3, 5, 12, 31, 33, 64, 65, 100, 129, 190, 256])
@pytest.mark.parametrize("diag", [False, True])
def test_sizes(n, diag):
    D, F = G.asymmetric_instance(n, seed=n, diag=diag)
    sweeps = 5 if n > 150 else 10
    beta = schedule(D, F, sweeps, 0.4)
    g = gpu_run(D, F, beta, sweeps, 7, 4, tables=True)
    r = O.anneal(D, F, beta, sweeps, 7, 0, 4, threads=4, tables=True)
    check_equal(g, r, tables=True)


MAPPINGS = [(40, 1, 1), (40, 2, 1), (40, 1, 4), (40, 2, 4), (100, 1, 1), (100, 4, 1), (100, 2, 4),
            (100, 4, 4), (129, 2, 1), (129, 8, 4), (200, 4, 1), (200, 8, 4), (256, 1, 1), (256, 8, 1),
            (256, 2, 4), (256, 8, 4), (256, 8, 16), (200, 4, 16)]


@pytest.mark.parametrize("n,wpr,pk", MAPPINGS)
def test_every_thread_mapping(n, wpr, pk):
    """Immediate rank-2 updates (1) and deferred ones (4 or 16 pending terms =
    two or eight swaps), shared- and global-memory tables."""
    D, F = G.asymmetric_instance(n, seed=n + 3)
    beta = schedule(D, F, 5, 0.5)
    g = gpu_run(D, F, beta, 5, 13, 3, tables=True, wpr=wpr, pk=pk)
    r = O.anneal(D, F, beta, 5, 13, 0, 3, threads=3, tables=True)
    check_equal(g, r, tables=True)


@pytest.mark.parametrize("n,lo,hi,fmax,diag", [(20, -9, 9, 9, True), (40, 0, 300, 50, False),
                                               (40, -300, 300, 50, True), (60, 0, 30000, 12, False),
                                               (30, 0, 40000, 20, False), (24, -2000, 2000, 50, True)])
def test_value_ranges_signs_and_diagonals(n, lo, hi, fmax, diag):
    """int8 / int16 / int32 staging with the odd-word row stride."""
    D = G.asymmetric(n, lo, hi, seed=n + 1, tag=5, diag=diag)
    F = G.asymmetric(n, max(lo, -fmax), fmax, seed=n + 2, tag=6, diag=diag)
    beta = schedule(D, F, 12)
    g = gpu_run(D, F, beta, 12, 3, 5, tables=True)
    r = O.anneal(D, F, beta, 12, 3, 0, 5, threads=5, tables=True)
    check_equal(g, r, tables=True)


@pytest.mark.parametrize("side", ["D", "F"])
def test_one_sided_asymmetry(side):
    n = 48
    S = G.random_symmetric(n, 0, 60, seed=2, tag=3)
    A = G.asymmetric(n, 0, 60, seed=4, tag=7)
    D, F = (A, S) if side == "D" else (S, A)
    beta = schedule(D, F, 20)
    g = gpu_run(D, F, beta, 20, 9, 6, tables=True)
    r = O.anneal(D, F, beta, 20, 9, 0, 6, threads=6, tables=True)
    check_equal(g, r, tables=True)


def test_longer_anneal_with_deferred_flush_boundaries():
    D, F = G.asymmetric_instance(30, seed=1, diag=True)
    beta = schedule(D, F, 41)
    g = gpu_run(D, F, beta, 41, 5, 8, tables=True, pk=4)
    r = O.anneal(D, F, beta, 41, 5, 0, 8, threads=8, tables=True)
    check_equal(g, r, tables=True)


def test_parallel_tempering_fixed_beta_and_cupim():
    D, F = G.asymmetric_instance(37, seed=2)
    bm = O.beta_max(D, F)
    L = 5
    ladder = np.float32([bm * 0.05 * (20.0 ** (q / (L - 1))) for q in range(L)])
    g = gpu_run(D, F, ladder, 22, 5, 20, mode=1, ladder_len=L, exchange_period=4, timeout_periods=2)
    r = O.anneal(D, F, ladder, 22, 5, 0, 20, mode="pt", ladder_len=L, period=4, timeout=2, threads=4)
    check_equal(g, r)
    assert np.array_equal(g["replica_rung"], r["rung"])
    betas = np.float32([bm * f for f in (0.0, 0.1, 1.0, 10.0)])
    g = gpu_run(D, F, betas, 30, 12, 4, mode=2)
    r = O.anneal(D, F, betas, 30, 12, 0, 4, mode="fixed", threads=4)
    check_equal(g, r)
    beta = schedule(D, F, 12)
    g = gpu_run(D, F, beta, 12, 31, 5, tables=True, mode=3)
    r = O.anneal(D, F, beta, 12, 31, 0, 5, mode="cupim", threads=5, tables=True)
    check_equal(g, r, tables=True)


def test_beta_max_and_host_entry_point():
    p = P()
    D, F = G.asymmetric_instance(50, seed=8, diag=True)
    with p.Qap(D, F) as q:
        assert p.pdit_beta_max(q) == O.beta_max(D, F)
        beta = schedule(D, F, 30)
        perm, cost = p.pdit_anneal(q, 12, beta, 30, 4)
    r = O.anneal(D, F, beta, 30, 4, 0, 12, threads=6)
    assert cost == r["cost"] and np.array_equal(perm, r["perm"])
    assert cost == O.cost(D, F, perm)


def test_batch_mixing_symmetric_and_general_instances():
    p = P()
    insts = [G.ragged_instance(0, 40, seed=1), G.asymmetric_instance(40, seed=2),
             G.asymmetric_instance(130, seed=3, diag=True), G.dense_instance(100, seed=4),
             G.asymmetric_instance(12, seed=5)]
    qs = [p.Qap(D, F) for D, F in insts]
    items = []
    for k, ((D, F), q) in enumerate(zip(insts, qs)):
        beta = torch.from_numpy(schedule(D, F, 8)).cuda()
        items.append(dict(qap=q, replicas=4 + k, sweeps=8, beta=beta, seed=50 + k, instance_id=k))
    b = p.Batch(items)
    b.run()
    torch.cuda.synchronize()
    for k, it in enumerate(items):
        D, F = insts[k]
        r = O.anneal(D, F, it["beta"].cpu().numpy(), 8, it["seed"], 0, it["replicas"], inst=k, threads=4)
        assert int(b.out[k]["best_cost"].item()) == r["cost"]
        assert np.array_equal(b.out[k]["best_perm"].cpu().numpy(), r["perm"])
    b.close()
    for q in qs:
        q.close()


def test_qaplib_file_end_to_end(tmp_path):
    """Read an instance file, anneal it, write and re-read the solution."""
    p = P()
    A, B = G.asymmetric_instance(27, seed=11, diag=True)
    f = tmp_path / "a27.dat"
    f.write_text("27\n\n" + "\n".join(" ".join(map(str, r)) for r in A) + "\n\n" +
                 "\n".join(" ".join(map(str, r)) for r in B) + "\n")
    D, F = p.read_qaplib(str(f))
    beta = schedule(D, F, 60)
    with p.Qap(D, F) as q:
        perm, cost = p.pdit_anneal(q, 16, beta, 60, 2)
    r = O.anneal(A, B, beta, 60, 2, 0, 16, threads=8)
    assert cost == r["cost"] and np.array_equal(perm, r["perm"])
    sln = tmp_path / "a27.sln"
    p.write_qaplib_solution(str(sln), perm, cost)
    c2, p2 = p.read_qaplib_solution(str(sln))
    assert c2 == cost and np.array_equal(p2, perm) and O.cost(A, B, p2) == cost


def test_resume_is_bit_identical_to_one_run():
    D, F = G.asymmetric_instance(60, seed=12, diag=True)
    beta = schedule(D, F, 40)
    r = O.anneal(D, F, beta, 40, 6, 0, 10, threads=5, tables=True)
    p = P()
    with p.Qap(D, F) as q:
        dbeta = torch.from_numpy(beta).cuda()
        first = p.anneal_device(q, 10, dbeta, 40, 6, sweep_end=17, per_replica=True)
        second = p.anneal_device(q, 10, dbeta, 40, 6, sweep_begin=17, resume=True, workspace=first["workspace"],
                                 per_replica=True, tables=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in second.items() if k != "workspace"}
    check_equal(g, r, tables=True)


def test_concurrent_updates_with_global_tables():
    D, F = G.asymmetric_instance(256, seed=14)
    beta = schedule(D, F, 4)
    g = gpu_run(D, F, beta, 4, 8, 3, tables=True, mode=3)
    r = O.anneal(D, F, beta, 4, 8, 0, 3, mode="cupim", threads=3, tables=True)
    check_equal(g, r, tables=True)
