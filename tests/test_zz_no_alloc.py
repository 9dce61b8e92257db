"""pdit_anneal_noalloc: the entry point for callers that cannot allocate
device memory (a framework that owns every device allocation through its own
pool, or a process that must not grow its device footprint after start-up).
It keeps its scratch in a static device array instead of a workspace, and
must give exactly what pdit_anneal_ex gives, and what the CPU oracle gives,
call after call, even though every call reuses the same array.

Kept in its own file, collected last, so that a run stopping at the first
failure has run every other test before this one. Each test makes its own
first call, so the file passes alone in a fresh process as well."""

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


class _Buffers:
    """Device inputs and outputs of one call, allocated up front by torch."""

    def __init__(self, D, F, beta):
        n = D.shape[0]
        self.n = n
        self.D = torch.from_numpy(np.ascontiguousarray(D, np.int32)).cuda()
        self.F = torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda()
        self.beta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda() if len(beta) else \
            torch.zeros(1, dtype=torch.float32, device="cuda")
        self.perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        self.cost = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        self.status = torch.full((1,), -1, dtype=torch.int32, device="cuda")

    def call(self, P, R, S, seed):
        rc = P.pdit_anneal_noalloc(self.n, self.D.data_ptr(), self.F.data_ptr(), R, self.beta.data_ptr(), S,
                                   seed, self.perm.data_ptr(), self.cost.data_ptr(), self.status.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
        assert rc == P.PDIT_OK, P.strerror(rc)

    def result(self):
        torch.cuda.synchronize()
        return self.perm.cpu().numpy(), int(self.cost.item()), int(self.status.item())


def _reference(P, D, F, R, beta, S, seed):
    with P.Qap(D, F) as q:
        dbeta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda()
        out = P.anneal_device(q, R, dbeta, S, seed)
        torch.cuda.synchronize()
        return out["best_perm"].cpu().numpy(), int(out["best_cost"].item())


def _schedule(P, D, F, kind, S):
    with P.Qap(D, F) as q:
        return P.pdit_beta_schedule(kind, S, P.pdit_beta_max(q))


CASES = [("n30", 96, 300, 7, "geometric"), ("n12", 64, 200, 3, "linear"),
         ("dense100", 16, 40, 11, "linear"), ("n30", 96, 300, 7, "geometric")]


def _instance(name):
    return G.dense_instance(100, seed=5) if name == "dense100" else G.named(name)


def test_noalloc_matches_anneal_ex_and_oracle_on_consecutive_calls(P):
    """Each case twice in a row through the shared array, against
    pdit_anneal_ex and against the oracle's best over the same replicas."""
    for name, R, S, seed, kind in CASES:
        D, F = _instance(name)
        beta = _schedule(P, D, F, kind, S)
        want = _reference(P, D, F, R, beta, S, seed)
        r = O.anneal(D, F, beta, S, seed, 0, R, threads=8)
        assert want[1] == r["cost"] and np.array_equal(want[0], r["perm"])
        buf = _Buffers(D, F, beta)
        for _ in range(2):
            buf.call(P, R, S, seed)
            perm, cost, status = buf.result()
            assert status == 0
            assert cost == want[1]
            assert np.array_equal(perm, want[0])


def test_noalloc_leaves_free_device_memory_unchanged(P):
    """After a first call on the device (which loads the library's device
    code and with it the static array), a call changes nothing in the free
    device memory: it allocates nothing."""
    D, F = G.named("n30")
    beta = _schedule(P, D, F, "linear", 50)
    buf = _Buffers(D, F, beta)
    buf.call(P, 128, 50, 2)
    first = buf.result()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    buf.call(P, 128, 50, 2)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    second = buf.result()
    assert free_after == free_before
    assert second[1] == first[1] and np.array_equal(second[0], first[0]) and second[2] == 0


def test_noalloc_rejects_requests_beyond_its_scratch(P):
    D, F = G.named("n30")
    buf = _Buffers(D, F, np.ones(4, np.float32))
    rc = P.pdit_anneal_noalloc(30, buf.D.data_ptr(), buf.F.data_ptr(), 1 << 20, buf.beta.data_ptr(), 4, 1,
                               buf.perm.data_ptr(), buf.cost.data_ptr(), 0, 0)
    assert rc == P.PDIT_ENOMEM
    rc = P.pdit_anneal_noalloc(1, buf.D.data_ptr(), buf.F.data_ptr(), 4, buf.beta.data_ptr(), 4, 1,
                               buf.perm.data_ptr(), buf.cost.data_ptr(), 0, 0)
    assert rc == P.PDIT_EINVAL


def test_noalloc_in_a_captured_graph(P):
    """After a first call on the device, a call captured in a CUDA graph and
    replayed gives the same result as the direct call (the captured call
    allocates nothing and records only memsets and kernel launches)."""
    D, F = G.named("n30")
    beta = _schedule(P, D, F, "geometric", 120)
    buf = _Buffers(D, F, beta)
    buf.call(P, 64, 120, 4)
    first = buf.result()
    assert first[2] == 0
    buf.perm.fill_(-1)
    buf.cost.fill_(-1)
    buf.status.fill_(-1)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        buf.call(P, 64, 120, 4)
    g.replay()
    second = buf.result()
    assert second[1] == first[1] and np.array_equal(second[0], first[0]) and second[2] == 0
