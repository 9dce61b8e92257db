"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element on the same seeded inputs: every replica's final and best
permutation, costs, best sweep, accepted-move count, and the influence tables.
Integers, so the bar is bit-exact."""

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
        dbeta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda() if len(beta) else \
            torch.zeros(1, dtype=torch.float32, device="cuda")
        out = p.anneal_device(q, R, dbeta, sweeps, seed, per_replica=True, tables=tables, **kw)
        torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}


def check_equal(g, r, rep_slice=slice(None), tables=False):
    assert int(g["status"][0]) == 0
    assert np.array_equal(g["replica_final_perm"][rep_slice], r["final_perm"])
    assert np.array_equal(g["replica_final_cost"][rep_slice], r["final_cost"])
    assert np.array_equal(g["replica_best_perm"][rep_slice], r["best_perm"])
    assert np.array_equal(g["replica_best_cost"][rep_slice], r["best_cost"])
    assert np.array_equal(g["replica_best_sweep"][rep_slice], r["best_sweep"])
    assert np.array_equal(g["replica_accepted"][rep_slice], r["accepted"])
    if tables:
        assert np.array_equal(g["tables"][rep_slice].astype(np.int64), r["tables"])


def schedule(D, F, kind, sweeps):
    return O.beta_schedule(kind, sweeps, O.beta_max(D, F))


# --- the named workloads -----------------------------------------------------

def test_n12_full_config_all_replicas(record_property):
    """3x4 grid, 64 replicas, 1000 linear sweeps: every replica bit-exact. The
    oracle also counts the draws within 1e-6 of a boundary of the exact
    double-precision Eq. 5 CDF (draws an ideal sampler might have resolved
    differently); they are reported and must stay rare."""
    D, F = G.named("n12")
    beta = schedule(D, F, "linear", 1000)
    g = gpu_run(D, F, beta, 1000, 0, 64, tables=True)
    r = O.anneal(D, F, beta, 1000, 0, 0, 64, threads=8, tables=True, near=True)
    check_equal(g, r, tables=True)
    assert int(g["best_cost"][0]) == r["cost"] == 564  # the 12! brute-force optimum
    assert np.array_equal(g["best_perm"], r["perm"])
    draws = 64 * 1000 * 12
    near = int(r["near_boundary"].sum())
    record_property("near_boundary_draws", "%d of %d" % (near, draws))
    assert near < 1e-3 * draws


def test_n9_sibling_reaches_brute_force_optimum():
    D, F = G.named("n9")
    opt, _, _ = O.brute_force(D, F)
    beta = schedule(D, F, "linear", 1000)
    g = gpu_run(D, F, beta, 1000, 0, 64)
    r = O.anneal(D, F, beta, 1000, 0, 0, 64, threads=8)
    check_equal(g, r)
    assert int(g["best_cost"][0]) == opt


def test_n30_full_config_sampled_replicas():
    """5x6 grid, 1024 replicas, 5000 geometric sweeps: the GPU runs all of them,
    the oracle recomputes a sample of replicas one by one."""
    D, F = G.named("n30")
    beta = schedule(D, F, "geometric", 5000)
    g = gpu_run(D, F, beta, 5000, 0, 1024)
    for lo, hi in [(0, 6), (509, 512), (1019, 1024)]:
        r = O.anneal(D, F, beta, 5000, 0, lo, hi, threads=8)
        check_equal(g, r, slice(lo, hi))
    assert (g["replica_best_cost"] >= g["best_cost"][0]).all()


def test_n100_full_config_sampled_replicas():
    """Dense N=100, 4096 replicas, 10000 linear sweeps (the throughput
    workload, same launch path as the benchmark): sampled replicas bit-exact."""
    D, F = G.named("n100")
    beta = schedule(D, F, "linear", 10000)
    g = gpu_run(D, F, beta, 10000, 0, 4096)
    for lo, hi in [(0, 2), (4094, 4096)]:
        r = O.anneal(D, F, beta, 10000, 0, lo, hi, threads=2)
        check_equal(g, r, slice(lo, hi))
    w = int(np.argmin(g["replica_best_cost"]))
    assert int(g["best_cost"][0]) == int(g["replica_best_cost"][w])
    assert O.cost(D, F, g["best_perm"]) == int(g["best_cost"][0])


# --- sizes across tiles, ragged tails and both table placements ---------------

SIZES = [2, 3, 5, 12, 31, 32, 33, 37, 63, 64, 65, 97, 100, 128, 129, 150, 190, 200, 256]


@pytest.mark.parametrize("n", SIZES)
def test_sizes_dense(n):
    D, F = G.dense_instance(n, seed=n)
    sweeps = 6 if n > 150 else 12
    beta = schedule(D, F, "linear", sweeps) * np.float32(0.3)
    R = 5
    g = gpu_run(D, F, beta, sweeps, 11, R, tables=True)
    r = O.anneal(D, F, beta, sweeps, 11, 0, R, threads=5, tables=True)
    check_equal(g, r, tables=True)


MAPPINGS = [(30, 1, 1), (30, 1, 4), (40, 1, 1), (40, 2, 1), (40, 1, 4), (40, 2, 4), (100, 1, 1),
            (100, 2, 1), (100, 4, 1), (100, 1, 4), (100, 2, 4), (100, 4, 4), (129, 1, 1), (129, 2, 4),
            (129, 4, 1), (129, 8, 4), (190, 8, 1), (190, 4, 4), (256, 1, 1), (256, 2, 1), (256, 4, 1),
            (256, 8, 1), (200, 1, 4), (256, 2, 4), (256, 4, 4), (256, 8, 4), (256, 8, 16), (256, 1, 16),
            (200, 2, 16), (230, 4, 16)]


@pytest.mark.parametrize("n,wpr,pk", MAPPINGS)
def test_every_thread_mapping(n, wpr, pk):
    """Every warps-per-replica shape, with immediate (1) or deferred (4)
    table updates, gives the oracle's results."""
    D, F = G.dense_instance(n, seed=n + 7)
    sweeps = 5
    beta = schedule(D, F, "linear", sweeps) * np.float32(0.5)
    g = gpu_run(D, F, beta, sweeps, 21, 4, tables=True, wpr=wpr, pk=pk)
    r = O.anneal(D, F, beta, sweeps, 21, 0, 4, threads=4, tables=True)
    check_equal(g, r, tables=True)


def test_deferred_updates_long_run_with_flush_boundaries():
    """Deferred updates over many accepted swaps, sweeps ending mid-batch,
    resumed calls: still bit-exact."""
    D, F = G.named("n30")
    beta = schedule(D, F, "linear", 37)
    g = gpu_run(D, F, beta, 37, 5, 10, tables=True, pk=4)
    r = O.anneal(D, F, beta, 37, 5, 0, 10, threads=5, tables=True)
    check_equal(g, r, tables=True)


@pytest.mark.parametrize("n,lo,hi,fmax,diag", [(20, -9, 9, 9, True), (40, 0, 300, 50, False),
                                               (40, -300, 300, 50, True), (70, 0, 40000, 20, False),
                                               (24, -2000, 2000, 50, True)])
def test_value_ranges_signs_and_diagonals(n, lo, hi, fmax, diag):
    """int8 / int16 / int32 staging of D and F, negative entries, nonzero diagonals."""
    D = G.random_symmetric(n, lo, hi, seed=n + 1, tag=1, diag=diag)
    F = G.random_symmetric(n, max(lo, -fmax), fmax, seed=n + 2, tag=2, diag=diag)
    bm = O.beta_max(D, F)
    beta = O.beta_schedule("linear", 15, bm)
    g = gpu_run(D, F, beta, 15, 3, 6, tables=True)
    r = O.anneal(D, F, beta, 15, 3, 0, 6, threads=6, tables=True)
    check_equal(g, r, tables=True)


@pytest.mark.parametrize("n", [12, 45, 110])
def test_ragged_grid_instances(n):
    D, F = G.ragged_instance(0, n, seed=5)
    beta = schedule(D, F, "linear", 10)
    g = gpu_run(D, F, beta, 10, 9, 7, tables=True)
    r = O.anneal(D, F, beta, 10, 9, 0, 7, threads=7, tables=True)
    check_equal(g, r, tables=True)


# --- degenerate and special cases ------------------------------------------------

def test_zero_sweeps_returns_initial_permutations():
    D, F = G.named("n30")
    g = gpu_run(D, F, np.zeros(0, np.float32), 0, 4, 9, tables=True)
    r = O.anneal(D, F, np.zeros(1, np.float32), 0, 4, 0, 9, tables=True)
    check_equal(g, r, tables=True)
    assert (g["replica_best_sweep"] == -1).all()


def test_beta_zero_and_huge_beta():
    D, F = G.named("n30")
    for val in [0.0, 1e30]:
        beta = np.full(8, val, np.float32)
        g = gpu_run(D, F, beta, 8, 1, 6)
        r = O.anneal(D, F, beta, 8, 1, 0, 6, threads=6)
        check_equal(g, r)


def test_single_replica_and_seed_high_bits():
    D, F = G.named("n12")
    beta = schedule(D, F, "linear", 50)
    seed = 0xDEADBEEF12345678
    g = gpu_run(D, F, beta, 50, seed, 1)
    r = O.anneal(D, F, beta, 50, seed, 0, 1)
    check_equal(g, r)


def test_instance_id_and_replica_base_shard_the_replica_space():
    """Replicas keyed by (instance id, global replica id): a shard run with
    replica_base = 40 equals replicas 40.. of one big run, and the oracle."""
    D, F = G.named("n30")
    beta = schedule(D, F, "linear", 20)
    big = gpu_run(D, F, beta, 20, 2, 64, instance_id=3)
    part = gpu_run(D, F, beta, 20, 2, 24, instance_id=3, replica_base=40)
    for key in ["replica_final_perm", "replica_best_cost", "replica_accepted", "replica_best_sweep"]:
        assert np.array_equal(big[key][40:], part[key])
    r = O.anneal(D, F, beta, 20, 2, 40, 46, inst=3, threads=6)
    check_equal(part, r, slice(0, 6))


def test_resume_is_bit_identical_to_one_run():
    D, F = G.named("n30")
    S = 40
    beta = schedule(D, F, "geometric", S)
    full = gpu_run(D, F, beta, S, 6, 33)
    p = P()
    with p.Qap(D, F) as q:
        dbeta = torch.from_numpy(beta).cuda()
        a = p.anneal_device(q, 33, dbeta, S, 6, sweep_end=17, per_replica=True)
        b = p.anneal_device(q, 33, dbeta, S, 6, sweep_begin=17, resume=True,
                            workspace=a["workspace"], per_replica=True)
        torch.cuda.synchronize()
    for key in ["replica_final_perm", "replica_best_cost", "replica_best_perm", "replica_best_sweep",
                "replica_accepted"]:
        assert np.array_equal(b[key].cpu().numpy(), full[key])
    assert int(b["best_cost"].item()) == int(full["best_cost"][0])


def test_host_buffer_entry_point_matches():
    D, F = G.named("n30")
    beta = schedule(D, F, "linear", 200)
    p = P()
    with p.Qap(D, F) as q:
        perm, cost = p.pdit_anneal(q, 96, beta, 200, 13)
        assert abs(p.pdit_beta_max(q) - O.beta_max(D, F)) <= 1e-12 * O.beta_max(D, F)
    r = O.anneal(D, F, beta, 200, 13, 0, 96, threads=8)
    assert cost == r["cost"] and np.array_equal(perm, r["perm"])


def test_invalid_options_are_rejected():
    p = P()
    D, F = G.named("n12")
    with p.Qap(D, F) as q:
        beta = torch.ones(4, device="cuda")
        with pytest.raises(p.PditError) as e:
            p.anneal_device(q, 0, beta, 4, 1)
        assert e.value.code == p.PDIT_EINVAL
        with pytest.raises(p.PditError):
            p.anneal_device(q, 4, beta, 4, 1, sweep_begin=2)  # sweep_begin without resume
        with pytest.raises(p.PditError):
            p.anneal_device(q, 30, beta, 4, 1, mode=p.PDIT_MODE_PT, ladder_len=7)  # 30 % 7 != 0


# --- parallel tempering ------------------------------------------------------------

@pytest.mark.parametrize("n,timeout", [(12, 3), (30, 100), (70, 2)])
def test_parallel_tempering_matches_oracle(n, timeout):
    D, F = (G.named("n12") if n == 12 else G.named("n30") if n == 30 else G.dense_instance(70, 1))
    bm = O.beta_max(D, F)
    L = 10
    ladder = np.float32([bm * 0.05 * (20.0 ** (q / (L - 1))) for q in range(L)])
    R, S = 40, 42
    g = gpu_run(D, F, ladder, S, 5, R, mode=1, ladder_len=L, exchange_period=4, timeout_periods=timeout)
    r = O.anneal(D, F, ladder, S, 5, 0, R, mode="pt", ladder_len=L, period=4, timeout=timeout, threads=4)
    check_equal(g, r)
    assert np.array_equal(g["replica_rung"], r["rung"])


# --- fixed beta per replica and the beta-range selection ------------------------

def test_fixed_beta_mode_matches_oracle():
    D, F = G.named("n30")
    bm = O.beta_max(D, F)
    betas = np.float32([bm * f for f in (0.0, 0.01, 0.1, 0.5, 1.0, 3.0, 10.0, 30.0)])
    g = gpu_run(D, F, betas, 40, 12, 8, mode=2)
    r = O.anneal(D, F, betas, 40, 12, 0, 8, mode="fixed", threads=8)
    check_equal(g, r)


def test_beta_range_selection_matches_oracle():
    D, F = G.named("n30")
    p = P()
    with p.Qap(D, F) as q:
        lo, hi, curve = p.pdit_beta_range(q, points=16, replicas_per_point=4, sweeps=100, seed=5)
    olo, ohi, omean, grid = O.beta_range(D, F, points=16, rpp=4, sweeps=100, seed=5)
    assert np.array_equal(curve, omean)
    assert lo == olo and hi == ohi
    assert lo <= hi


# --- concurrent updates (GPU-CUPIM) -----------------------------------------------

@pytest.mark.parametrize("name,n,wpr,pk", [("n12", 12, 0, 0), ("n30", 30, 0, 0), ("dense", 100, 4, 4),
                                          ("dense", 100, 2, 1), ("dense", 100, 1, 4), ("dense", 150, 0, 0),
                                          ("dense", 256, 0, 0)])
def test_cupim_matches_oracle(name, n, wpr, pk):
    D, F = G.named(name) if name != "dense" else G.dense_instance(n, seed=n)
    S = 12
    beta = schedule(D, F, "linear", S)
    g = gpu_run(D, F, beta, S, 31, 6, tables=True, wpr=wpr, pk=pk, mode=3)
    r = O.anneal(D, F, beta, S, 31, 0, 6, mode="cupim", threads=6, tables=True)
    check_equal(g, r, tables=True)


@pytest.mark.parametrize("wpr,pk", [(0, 0), (1, 1), (1, 4)])
def test_cupim_hand_worked_conflicts(wpr, pk):
    """The hand-worked conflict case of the oracle's pins (N = 6, beta so
    large that each location proposes its row's argmin): an energy-ordered
    conflict, an equal-energy tie between two initiators and a pair proposed
    from both ends; the GPU applies the same two swaps."""
    from tests import test_oracle_cupim_rule as C

    beta = np.array([C.BIG_BETA], np.float32)
    g = gpu_run(C.D, C.F, beta, 1, C.SEED, 1, tables=True, wpr=wpr, pk=pk, mode=3)
    r = O.anneal(C.D, C.F, beta, 1, C.SEED, 0, 1, mode="cupim", tables=True)
    check_equal(g, r, tables=True)
    assert g["replica_final_perm"][0].tolist() == C.EXPECTED
    assert int(g["replica_accepted"][0]) == 2


# --- launch-shape knobs and the autotuner ------------------------------------------

@pytest.mark.parametrize("n,g", [(100, 1), (100, 3), (256, 1), (256, 3)])
def test_replicas_per_cta_does_not_change_results(n, g):
    D, F = G.dense_instance(n, seed=n + 9)
    beta = schedule(D, F, "linear", 6) * np.float32(0.5)
    p = P()
    with p.Qap(D, F) as q:
        p.pdit_set_replicas_per_cta(q, g)
        assert p.pdit_launch_shape(q, 64)["replicas_per_cta"] <= g
        dbeta = torch.from_numpy(beta).cuda()
        out = p.anneal_device(q, 9, dbeta, 6, 4, per_replica=True)
        torch.cuda.synchronize()
        g_out = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    r = O.anneal(D, F, beta, 6, 4, 0, 9, threads=9)
    check_equal(g_out, r)


@pytest.mark.parametrize("n", [40, 230])
def test_autotune_keeps_results_and_reports_a_shape(n):
    D, F = G.dense_instance(n, seed=n + 2)
    beta = schedule(D, F, "linear", 8)
    p = P()
    with p.Qap(D, F) as q:
        dbeta = torch.from_numpy(beta).cuda()
        wpr, pk = p.pdit_autotune(q, 32, dbeta, 4)
        shape = p.pdit_launch_shape(q, 32)
        assert shape["warps_per_replica"] == wpr and shape["pending_swaps"] == pk
        assert wpr in (1, 2, 4, 8) and pk in (1, 4, 16)
        out = p.anneal_device(q, 7, dbeta, 8, 3, per_replica=True)
        torch.cuda.synchronize()
        g_out = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    r = O.anneal(D, F, beta, 8, 3, 0, 7, threads=7)
    check_equal(g_out, r)


def test_wide_values_at_a_single_replica_size_stay_in_shared_memory():
    """N = 150 with D up to 300 (int16 staging; swap factors do not fit a
    byte, so no pending terms): one table fits shared memory next to D and F,
    and without pending terms the tables stay there."""
    n = 150
    D = G.random_symmetric(n, 0, 300, seed=5, tag=1)
    F = G.random_symmetric(n, 0, 50, seed=6, tag=2)
    p = P()
    with p.Qap(D, F) as q:
        shape = p.pdit_launch_shape(q, 64)
        assert shape["tables_in_smem"] == 1 and shape["pending_swaps"] == 1
    beta = schedule(D, F, "linear", 6)
    g = gpu_run(D, F, beta, 6, 2, 4, tables=True)
    r = O.anneal(D, F, beta, 6, 2, 0, 4, threads=4, tables=True)
    check_equal(g, r, tables=True)


def test_very_many_replicas_sampled():
    """200,000 replicas in one call (the work queue and every per-replica
    offset at scale): sampled replicas, the last one included, equal the
    oracle's runs of the same global replica ids."""
    D, F = G.named("n12")
    R, sweeps = 200_000, 3
    beta = schedule(D, F, "linear", sweeps)
    g = gpu_run(D, F, beta, sweeps, 21, R)
    for r0 in (0, 65_535, 123_457, R - 3):
        r = O.anneal(D, F, beta, sweeps, 21, r0, r0 + 3, threads=3)
        sl = slice(r0, r0 + 3)
        assert np.array_equal(g["replica_final_perm"][sl], r["final_perm"])
        assert np.array_equal(g["replica_best_cost"][sl], r["best_cost"])
        assert np.array_equal(g["replica_accepted"][sl], r["accepted"])
    assert int(g["best_cost"][0]) == int(g["replica_best_cost"].min())


# --- launches split into parts (more replicas than resident slots) ----------

@pytest.mark.parametrize("kind,n,mode,S", [("sym", 40, 0, 24), ("asym", 36, 0, 24), ("sym", 40, 3, 24),
                                           ("sym", 200, 0, 16), ("asym", 150, 0, 16)])
def test_table_kernels_in_parts(kind, n, mode, S):
    """The table kernels with more replicas than resident slots. With tables
    in shared memory each replica's sweeps run as parts (work units of one
    launch) that resume from the state, table included, the previous part
    published; tables in global memory (N = 150, 200) take whole calls.
    Replicas of the first and of the last round, their final tables
    included, equal the oracle's; symmetric and general form, sequential and
    concurrent updates."""
    D, F = (G.dense_instance(n, seed=n + 5) if kind == "sym" else G.asymmetric_instance(n, seed=n + 5))
    beta = schedule(D, F, "linear", S)
    p = P()
    with p.Qap(D, F) as q:
        p.pdit_set_influence(q, p.PDIT_INFLUENCE_TABLE)
        shape = p.pdit_launch_shape(q, 1 << 20)
        R = shape["ctas"] * shape["replicas_per_cta"] + 7
        dbeta = torch.from_numpy(beta).cuda()
        out = p.anneal_device(q, R, dbeta, S, 2, per_replica=True, tables=True, mode=mode)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    m = {0: "anneal", 3: "cupim"}[mode]
    for lo, hi in [(0, 2), (R - 9, R - 7), (R - 2, R)]:
        r = O.anneal(D, F, beta, S, 2, lo, hi, threads=2, tables=True, mode=m)
        if r["general"]:
            r["tables"] = -r["tables"]  # the oracle keeps Eq. 2's sign; the kernels its negation
        check_equal(g, r, slice(lo, hi), tables=True)
