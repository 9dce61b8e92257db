"""Serving with continuous batching: requests submitted while others run,
admitted by device-memory footprint, sliced into resumable chunks; each
result must equal the single-instance call with instance_id = request id."""

import threading
import time

import numpy as np
import pytest

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


def _alone(P, rid, replicas, sweeps, seed):
    D, F = G.request_instance(rid)
    with P.Qap(D, F) as q:
        beta = P.pdit_beta_schedule("linear", sweeps, P.pdit_beta_max(q))
        out = P.anneal_device(q, replicas, torch.from_numpy(beta).cuda(), sweeps, seed, instance_id=rid)
        torch.cuda.synchronize()
        return out["best_perm"].cpu().numpy(), int(out["best_cost"].item())


@pytest.mark.parametrize("budget,slice_sweeps", [(8 << 30, 40), (1024, 25)])
def test_results_equal_alone_and_in_the_mix(P, budget, slice_sweeps):
    rids = [3, 10, 11, 24, 37, 58]
    replicas, sweeps, seed = 48, 120, 9
    srv = P.Server(device_budget_bytes=budget, slice_sweeps=slice_sweeps, max_active=4)
    tickets = {}

    def producer():
        for k, rid in enumerate(rids):
            D, F = G.request_instance(rid)
            tickets[rid] = srv.submit(D, F, replicas, sweeps, seed, rid)
            time.sleep(0.01 * (k % 3))

    th = threading.Thread(target=producer)
    th.start()
    max_active = 0
    while True:
        a, q = srv.tick()
        max_active = max(max_active, a)
        if not th.is_alive() and a == 0 and q == 0 and len(tickets) == len(rids):
            break
    th.join()
    if budget > (1 << 24):
        assert max_active >= 2  # requests overlapped on the device
    else:
        # a budget below every request's footprint admits one request at a time
        # (an oversize request is admitted only when nothing else is resident)
        assert max_active == 1
    for rid in rids:
        st, perm, cost, lat = srv.result(tickets[rid])
        assert st == 2 and lat > 0
        aperm, acost = _alone(P, rid, replicas, sweeps, seed)
        assert cost == acost
        assert np.array_equal(perm, aperm)
    srv.close()
