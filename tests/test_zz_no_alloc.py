"""pdit_anneal_noalloc: the entry point for callers that cannot allocate
device memory (a framework that owns every device allocation through its own
pool, or a process that must not grow its device footprint after start-up).
It keeps its scratch in a static device array instead of a workspace, and
must give exactly what pdit_anneal_ex gives, call after call, even though
every call reuses the same array.

Kept in its own file, collected last, so that a run stopping at the first
failure has run every other test before this one."""

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


def _noalloc(P, D, F, R, dbeta, S, seed):
    n = D.shape[0]
    dD = torch.from_numpy(np.ascontiguousarray(D, np.int32)).cuda()
    dF = torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda()
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cost = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = P.pdit_anneal_noalloc(n, dD.data_ptr(), dF.data_ptr(), R, dbeta.data_ptr(), S, seed,
                               perm.data_ptr(), cost.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert rc == P.PDIT_OK, P.strerror(rc)
    torch.cuda.synchronize()
    return perm.cpu().numpy(), int(cost.item())


def _reference(P, D, F, R, dbeta, S, seed):
    with P.Qap(D, F) as q:
        out = P.anneal_device(q, R, dbeta, S, seed)
        torch.cuda.synchronize()
        return out["best_perm"].cpu().numpy(), int(out["best_cost"].item())


def test_noalloc_matches_anneal_ex_on_consecutive_calls(P):
    cases = [("n30", 96, 300, 7, "geometric"), ("n12", 64, 200, 3, "linear"),
             ("n30", 96, 300, 7, "geometric")]
    for name, R, S, seed, kind in cases:
        D, F = G.named(name)
        with P.Qap(D, F) as q:
            beta = P.pdit_beta_schedule(kind, S, P.pdit_beta_max(q))
        dbeta = torch.from_numpy(beta).cuda()
        got = _noalloc(P, D, F, R, dbeta, S, seed)
        want = _reference(P, D, F, R, dbeta, S, seed)
        assert got[1] == want[1]
        assert np.array_equal(got[0], want[0])
        again = _noalloc(P, D, F, R, dbeta, S, seed)
        assert again[1] == want[1] and np.array_equal(again[0], want[0])


def test_noalloc_rejects_requests_beyond_its_scratch(P):
    D, F = G.named("n30")
    dbeta = torch.ones(4, dtype=torch.float32, device="cuda")
    dD = torch.from_numpy(D).cuda()
    dF = torch.from_numpy(F).cuda()
    perm = torch.empty(30, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.int64, device="cuda")
    rc = P.pdit_anneal_noalloc(30, dD.data_ptr(), dF.data_ptr(), 1 << 20, dbeta.data_ptr(), 4, 1,
                               perm.data_ptr(), cost.data_ptr(), 0)
    assert rc == P.PDIT_ENOMEM
    rc = P.pdit_anneal_noalloc(1, dD.data_ptr(), dF.data_ptr(), 4, dbeta.data_ptr(), 4, 1,
                               perm.data_ptr(), cost.data_ptr(), 0)
    assert rc == P.PDIT_EINVAL
