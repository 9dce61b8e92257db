"""Multi-instance batches (one persistent launch per kernel shape, optionally
captured as a CUDA graph) and the time-to-target bookkeeping: every
instance's result equals its single-instance call and the oracle."""

import numpy as np
import pytest

import oracle as O
from paper_2605_24408_gb300 import instances as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24408_gb300 import build as B
    from paper_2605_24408_gb300 import pdit

    B.build()
    torch.cuda.set_device(0)
    return pdit


SIZES = [12, 30, 45, 100, 101, 150, 200, 256]


def _instances():
    out = []
    for k, n in enumerate(SIZES):
        D, F = G.ragged_instance(k, n, seed=3)
        out.append((D, F))
    return out


def _items(P, qs, insts, sweeps=12):
    items = []
    for k, ((D, F), q) in enumerate(zip(insts, qs)):
        beta = O.beta_schedule("linear", sweeps, O.beta_max(D, F))
        items.append(dict(qap=q, replicas=5 + k, sweeps=sweeps, beta=torch.from_numpy(beta).cuda(),
                          seed=100 + k, instance_id=k))
    return items


def test_batch_matches_single_instance_calls_and_oracle(P):
    insts = _instances()
    qs = [P.Qap(D, F) for D, F in insts]
    items = _items(P, qs, insts)
    b = P.Batch(items)
    classes, ws = b.info()
    assert classes >= 2 and ws > 0
    b.run()
    torch.cuda.synchronize()
    for k, it in enumerate(items):
        single = P.anneal_device(qs[k], it["replicas"], it["beta"], it["sweeps"], it["seed"],
                                 instance_id=it["instance_id"])
        torch.cuda.synchronize()
        assert int(b.out[k]["best_cost"].item()) == int(single["best_cost"].item())
        assert torch.equal(b.out[k]["best_perm"], single["best_perm"])
        # every size, up to N = 256 (both kernel families, several shapes)
        D, F = insts[k]
        r = O.anneal(D, F, it["beta"].cpu().numpy(), it["sweeps"], it["seed"], 0, it["replicas"],
                     inst=it["instance_id"], threads=8)
        assert int(b.out[k]["best_cost"].item()) == r["cost"]
        assert np.array_equal(b.out[k]["best_perm"].cpu().numpy(), r["perm"])
    b.close()
    for q in qs:
        q.close()


def test_batch_graph_replays_identically(P):
    insts = _instances()[:5]
    qs = [P.Qap(D, F) for D, F in insts]
    items = _items(P, qs, insts, sweeps=8)
    plain = P.Batch(items)
    plain.run()
    torch.cuda.synchronize()
    want = [(int(o["best_cost"].item()), o["best_perm"].clone()) for o in plain.out]
    g = P.Batch(items, graph=True)
    s = torch.cuda.Stream()
    for _ in range(2):
        with torch.cuda.stream(s):
            g.run(s)
        s.synchronize()
        for k, o in enumerate(g.out):
            assert int(o["best_cost"].item()) == want[k][0]
            assert torch.equal(o["best_perm"], want[k][1])
    g.close()
    plain.close()
    for q in qs:
        q.close()


def test_reach_sweep_matches_oracle_single_and_batched(P):
    D, F = G.named("n30")
    sweeps, R, seed = 40, 6, 17
    beta = O.beta_schedule("linear", sweeps, O.beta_max(D, F))
    ref = O.anneal(D, F, beta, sweeps, seed, 0, R, threads=6)
    target = int(ref["cost"] * 1.03)
    r = O.anneal(D, F, beta, sweeps, seed, 0, R, threads=6, target=target)
    want = int(r["reach_sweep"].min())
    dbeta = torch.from_numpy(beta).cuda()
    dt = torch.tensor([target], dtype=torch.int64, device="cuda")
    with P.Qap(D, F) as q:
        single = P.anneal_device(q, R, dbeta, sweeps, seed, target=dt)
        b = P.Batch([dict(qap=q, replicas=R, sweeps=sweeps, beta=dbeta, seed=seed, target=dt)])
        b.run()
        torch.cuda.synchronize()
        assert int(single["reach_sweep"].item()) == want
        assert int(b.out[0]["reach_sweep"].item()) == want
        assert int(single["reach_ns"].item()) > 0
        b.close()


def test_stop_at_target_stops_early_and_reports(P):
    D, F = G.named("n30")
    sweeps, R, seed = 400, 32, 5
    beta = O.beta_schedule("linear", sweeps, O.beta_max(D, F))
    dbeta = torch.from_numpy(beta).cuda()
    with P.Qap(D, F) as q:
        full = P.anneal_device(q, R, dbeta, sweeps, seed, per_replica=True)
        torch.cuda.synchronize()
        target = int(full["best_cost"].item() * 1.05)
        dt = torch.tensor([target], dtype=torch.int64, device="cuda")
        early = P.anneal_device(q, R, dbeta, sweeps, seed, target=dt, stop_at_target=True,
                                per_replica=True)
        b = P.Batch([dict(qap=q, replicas=R, sweeps=sweeps, beta=dbeta, seed=seed, target=dt)],
                    stop_at_target=True)
        b.run()
        torch.cuda.synchronize()
        for res in (early, b.out[0]):
            assert int(res["best_cost"].item()) <= target
            assert 0 <= int(res["reach_sweep"].item()) < sweeps
        # stopped replicas did less work than the full schedule
        assert int(early["replica_accepted"].sum().item()) < int(full["replica_accepted"].sum().item())
        b.close()
