"""The identities behind the dot-product kernel's two-location lookahead,
checked against direct recomputation on random states (no GPU).

With the flow permuted to location order, Q[x][y] = F[p(x)][p(y)], the
influence entries of the one-term table (Eq. 2) are I[i][p(j)] = D[i] . Q[j]
and I[j][p(i)] = D[j] . Q[i]. The kernel forms both for locations i and
i' = i + 1 from one pass over the rows; when the update of i swaps i and s
(tau = the transposition (i s)), the entries of i' under the new permutation
follow from the old ones:
  D[i'] . Q'[j] = D[i'] . Q[tau j] + (D[i'][s] - D[i'][i]) (Q[tau j][i] - Q[tau j][s])
  D[j] . Q'[i'] = D[j] . Q[tau i'] + (D[j][s] - D[j][i]) (Q[tau i'][i] - Q[tau i'][s])
(Q' = Q with rows and columns i, s exchanged)."""

import numpy as np


def test_next_location_entries_after_a_swap():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        n = int(rng.integers(3, 9))
        D = rng.integers(-9, 10, (n, n))
        D = D + D.T
        F = rng.integers(-9, 10, (n, n))
        F = F + F.T
        p = rng.permutation(n)
        i = int(rng.integers(0, n - 1))
        ip = i + 1
        s = int(rng.integers(0, n))
        if s == i:
            continue
        tau = np.arange(n)
        tau[i], tau[s] = s, i
        Q = F[np.ix_(p, p)]
        q = p[tau]  # the swap: locations i and s trade facilities
        Q2 = F[np.ix_(q, q)]
        assert np.array_equal(Q2, Q[np.ix_(tau, tau)])  # rows and columns i, s exchanged
        row_b, col_b, col_a = Q @ D[ip], D @ Q[ip], D @ Q[i]
        delta = D[ip][s] - D[ip][i]
        want_row, want_col = Q2 @ D[ip], D @ Q2[ip]
        for j in range(n):
            assert want_row[j] == row_b[tau[j]] + delta * (Q[tau[j]][i] - Q[tau[j]][s])
            base = col_b[j] if s != ip else col_a[j]  # tau i' = i' unless s = i'
            assert want_col[j] == base + (D[j][s] - D[j][i]) * (Q[tau[ip]][i] - Q[tau[ip]][s])
