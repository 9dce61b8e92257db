"""The two-level-flow structure (Methods section, tai256c paragraph) that the
flow-class kernel relies on, pinned on the CPU against the plain definition
of Eq. 1 and the oracle's Eq. 3: with D symmetric (zero diagonal) and
F[c][d] = f0 + f x_c x_d off the diagonal, a swap within a class has dE = 0,
a swap moving class 1 from location u to w has dE = 2 f (G_w - G_u - D_uw)
with G_m = sum over class-1 locations j of D_mj, and
E = f0 sum_{i != j} D_ij + f sum over class-1 locations u of G_u."""

import itertools

import numpy as np
import pytest

import oracle as O
from paper_2605_24408_gb300 import instances as G


@pytest.mark.parametrize("n,k,f0,f,fdiag", [(6, 3, 0, 1, 0), (9, 4, 2, 5, 7), (12, 11, -3, 4, 0),
                                            (10, 2, 1, -2, 3), (8, 0, 4, 1, 0), (7, 7, 0, 3, 1)])
def test_class_energy_and_swap_formulas(n, k, f0, f, fdiag):
    D, F = G.flow_class_instance(n, k, seed=n + k, lo=0, hi=40, f0=f0, f=f, fdiag=fdiag)
    # class 1: the facilities with an in-class flow f0 + f to some other facility
    x = np.array([k > 1 and any(F[c, d] == f0 + f for d in range(n) if d != c) for c in range(n)])
    for rep in range(3):
        p = O.init_perm(n, 5, 0, rep)
        inS = x[p]
        Gv = D[:, inS].sum(axis=1).astype(np.int64)
        e = O.cost(D, F, p)
        assert e == f0 * int(D.sum()) + f * int(Gv[inS].sum())
        I = O.influence(D, F, p)
        for u, w in itertools.product(range(n), range(n)):
            q = p.copy()
            q[u], q[w] = q[w], q[u]
            brute = O.cost(D, F, q) - e
            assert O.delta_e(D, F, p, I, u, w) == brute
            if inS[u] == inS[w]:
                assert brute == 0
            elif inS[u]:
                assert brute == 2 * f * (Gv[w] - Gv[u] - D[u, w])
            else:
                assert brute == 2 * f * (Gv[u] - Gv[w] - D[u, w])


def test_c256_workload_shape():
    D, F = G.named("c256")
    n = 256
    assert D.shape == (n, n) and np.array_equal(D, D.T) and not D.diagonal().any()
    inK = F.sum(axis=1) > 0
    assert inK.sum() == 92
    assert not inK[:92].all()  # a hashed subset, not the first 92 facilities
    assert set(np.unique(F)) == {0, 1}
    assert np.array_equal(F, np.outer(inK, inK).astype(np.int32) - np.diag(inK.astype(np.int32)))
