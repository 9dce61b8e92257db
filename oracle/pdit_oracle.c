/*
 * CPU ORACLE for the annealed p-dit sweep on the QAP (symmetric, and the
 * general form with asymmetric D, F or nonzero diagonals).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only tests/, __graft_entry__.smoke()
 * and the CPU-baseline / reference arm of bench.py load this library. It
 * shares no code, header, table or constant with the CUDA path; both sides
 * only receive the same seeded inputs (D, F, beta values, seed).
 *
 * Plain and slow on purpose: one replica at a time, every step in the order
 * the paper gives it, 64-bit integers for the influence table and the costs.
 * Source: arXiv 2605.24408, "P-dit Probabilistic Ising Machine for Solving
 * the Quadratic Assignment Problem".
 *
 *   oracle_cost           Eq. 1 (QAP objective), written out.
 *   oracle_influence      Eq. 2, stored in the unsigned one-term form
 *                         I[m][c] = sum_j D[m][j] F[c][p(j)]; for symmetric D, F
 *                         the paper's I equals -2 times this (reading R1).
 *   oracle_delta_e        Eq. 3 restated in those units (reading R2: Eq. 3,
 *                         not the Eq. 4 shortcut, which drops a term).
 *   oracle_delta_e_eq3    the general form: Eq. 2 taken literally (both
 *                         terms, the paper's sign) and Eq. 3 taken literally;
 *                         used when D or F is not symmetric (reading R13).
 *   oracle_update         Eq. 5 over the N outcomes of one p-dit update
 *                         (swap with each other location, or stay), sampled
 *                         with the fp32 weights of reading R4.
 *   oracle_anneal         Implementation section: swap-only moves from a
 *                         valid permutation, each sweep every p-dit
 *                         initiates one update (order R3); incremental
 *                         influence update after each swap (Methods,
 *                         GPU-CUPIM Algorithm: the sequential PIM keeps I
 *                         up to date incrementally);
 *                         best-so-far as first logged (Hardware and Data
 *                         Reporting Details, reading R6); parallel
 *                         tempering (Implementation + CPU-PIM Algorithm,
 *                         reading R7).
 *   oracle_philox4x32_10  Salmon, Moraes, Dror, Shaw, "Parallel random
 *                         numbers: as easy as 1, 2, 3", SC'11 (reading R5).
 *   cupim_iteration       the concurrent-update variant (GPU-CUPIM Algorithm
 *                         section; reading R12).
 *   oracle_brute_force    min over all N! permutations of Eq. 1.
 *
 * Pins (tests/test_oracle_*.py): Eq. 1 on a hand-worked 3-facility case and
 * closed forms; Eq. 3 against cost(swap(p)) - cost(p) by brute recomputation;
 * incremental tables and costs against full recomputation; Philox against
 * cuRAND's host Philox4_32_10 and the published known-answer vectors; the
 * fp32 exponential against double exp; sampler probabilities against exact
 * double Eq. 5, beta = 0 (uniform) and beta -> infinity (argmin) closed
 * forms, and a chi-square test of the one-step law; anneal results against
 * brute-force optima for N <= 9; parallel-tempering exchange on hand-made
 * energy sequences. General form (tests/test_oracle_general.py): Eq. 1 on a
 * hand-worked asymmetric case, Eq. 3 as printed against brute recomputation
 * with any diagonal, sum_m Ip[m][p(m)] = -2 E, and the exact reduction of a
 * one-sided asymmetric instance to the symmetric form at half the beta.
 *
 * Floating point: compile with -ffp-contract=off; every float operation below
 * is one correctly rounded IEEE binary32 operation (fmaf is a fused one).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the Philox S-box with  */
/* multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,   */
/* 0xBB67AE85, as published.                                                */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Reading R5: the random words of replica `rep` of instance `inst`.
 * Key = (seed low word, seed high word).
 * Initial permutation, Fisher-Yates step k: counter (inst, rep, 0xFFFFFFFF, k/4), word k%4.
 * Update of location i in sweep s: counter (inst, rep, s, i), r = word0 | word1 << 32. */
static void key_of(uint64_t seed, uint32_t key[2]) {
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
}

uint64_t oracle_update_draw(uint64_t seed, uint32_t inst, uint32_t rep, uint32_t sweep,
                            uint32_t loc) {
    uint32_t key[2], ctr[4] = {inst, rep, sweep, loc}, out[4];
    key_of(seed, key);
    oracle_philox4x32_10(ctr, key, out);
    return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

/* Reading R5: uniform random initial permutation (every p-dit starts in a
 * distinct dimension, Implementation section). Fisher-Yates from the
 * last position down; the index for step k is the high word of u * (k + 1). */
void oracle_init_perm(int n, uint64_t seed, uint32_t inst, uint32_t rep, int32_t *p) {
    uint32_t key[2];
    key_of(seed, key);
    for (int m = 0; m < n; ++m) p[m] = m;
    for (int k = n - 1; k >= 1; --k) {
        uint32_t ctr[4] = {inst, rep, 0xFFFFFFFFu, (uint32_t)k / 4u}, out[4];
        oracle_philox4x32_10(ctr, key, out);
        uint32_t u = out[k % 4];
        int j = (int)(((uint64_t)u * (uint64_t)(k + 1)) >> 32);
        int32_t t = p[k];
        p[k] = p[j];
        p[j] = t;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1, Eq. 2, Eq. 3                                                       */
/* ------------------------------------------------------------------------ */
int64_t oracle_cost(int n, const int32_t *D, const int32_t *F, const int32_t *p) {
    int64_t e = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            e += (int64_t)D[(size_t)i * n + j] * F[(size_t)p[i] * n + p[j]];
    return e;
}

/* Unsigned one-term influence (reading R1): I[m][c] = sum_j D[m][j] F[c][p(j)]. */
void oracle_influence(int n, const int32_t *D, const int32_t *F, const int32_t *p,
                      int64_t *I) {
    for (int m = 0; m < n; ++m)
        for (int c = 0; c < n; ++c) {
            int64_t s = 0;
            for (int j = 0; j < n; ++j)
                s += (int64_t)D[(size_t)m * n + j] * F[(size_t)c * n + p[j]];
            I[(size_t)m * n + c] = s;
        }
}

/* The paper's Eq. 2 taken literally (both terms, minus sign), for checking
 * reading R1 against it. */
void oracle_influence_eq2(int n, const int32_t *D, const int32_t *F, const int32_t *p,
                          int64_t *Ip) {
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < n; ++a) {
            int64_t s = 0;
            for (int j = 0; j < n; ++j)
                s += (int64_t)D[(size_t)i * n + j] * F[(size_t)a * n + p[j]] +
                     (int64_t)D[(size_t)j * n + i] * F[(size_t)p[j] * n + a];
            Ip[(size_t)i * n + a] = -s;
        }
}

/* Eq. 3 in the units of reading R1. With Ip = -2 I (symmetric D, F):
 *   dE = -[Ip_ib - Ip_ia + Ip_ja - Ip_jb - (D_ii + D_jj - D_ij - D_ji)(F_aa + F_bb - F_ab - F_ba)]
 *      = 2 (I_ib - I_ia + I_ja - I_jb) + (D_ii + D_jj - D_ij - D_ji)(F_aa + F_bb - F_ab - F_ba)
 * with a = p(i), b = p(j). Staying (j == i) changes nothing: dE = 0. */
int64_t oracle_delta_e(int n, const int32_t *D, const int32_t *F, const int32_t *p,
                       const int64_t *I, int i, int j) {
    if (i == j) return 0;
    int a = p[i], b = p[j];
    int64_t t = I[(size_t)i * n + b] - I[(size_t)i * n + a] + I[(size_t)j * n + a] -
                I[(size_t)j * n + b];
    int64_t dd = (int64_t)D[(size_t)i * n + i] + D[(size_t)j * n + j] - D[(size_t)i * n + j] -
                 D[(size_t)j * n + i];
    int64_t ff = (int64_t)F[(size_t)a * n + a] + F[(size_t)b * n + b] - F[(size_t)a * n + b] -
                 F[(size_t)b * n + a];
    return 2 * t + dd * ff;
}

/* The incremental influence update after a swap at locations i, j (facility
 * a at i moves to j, b at j moves to i). It is two single-location moves of
 * Eq. 2's sum: location i goes a -> b and location j goes b -> a, so for all
 * m, c:  I[m][c] += D[m][i] (F[c][b] - F[c][a]) + D[m][j] (F[c][a] - F[c][b]). */
static void apply_swap_to_influence(int n, const int32_t *D, const int32_t *F, int64_t *I,
                                    int i, int j, int a, int b) {
    for (int m = 0; m < n; ++m)
        for (int c = 0; c < n; ++c) {
            int64_t move_i = (int64_t)D[(size_t)m * n + i] *
                             ((int64_t)F[(size_t)c * n + b] - F[(size_t)c * n + a]);
            int64_t move_j = (int64_t)D[(size_t)m * n + j] *
                             ((int64_t)F[(size_t)c * n + a] - F[(size_t)c * n + b]);
            I[(size_t)m * n + c] += move_i + move_j;
        }
}

/* General D and F (reading R13). Eq. 3 with the table Ip of Eq. 2 as printed:
 *   dE = -[Ip_ib - Ip_ia + Ip_ja - Ip_jb - (D_ii + D_jj - D_ij - D_ji)(F_aa + F_bb - F_ab - F_ba)]
 * with a = p(i), b = p(j); staying (j == i) changes nothing. */
int64_t oracle_delta_e_eq3(int n, const int32_t *D, const int32_t *F, const int32_t *p,
                           const int64_t *Ip, int i, int j) {
    if (i == j) return 0;
    int a = p[i], b = p[j];
    int64_t t = Ip[(size_t)i * n + b] - Ip[(size_t)i * n + a] + Ip[(size_t)j * n + a] -
                Ip[(size_t)j * n + b];
    int64_t dd = (int64_t)D[(size_t)i * n + i] + D[(size_t)j * n + j] - D[(size_t)i * n + j] -
                 D[(size_t)j * n + i];
    int64_t ff = (int64_t)F[(size_t)a * n + a] + F[(size_t)b * n + b] - F[(size_t)a * n + b] -
                 F[(size_t)b * n + a];
    return -(t - dd * ff);
}

/* Eq. 2's table after the swap (facility a at i moves to j, b at j moves to
 * i). Of the sum over j in Eq. 2 only the terms of locations i and j change:
 *   Ip[m][c] -= D[m][i] (F[c][b] - F[c][a]) + D[m][j] (F[c][a] - F[c][b])
 *             + D[i][m] (F[b][c] - F[a][c]) + D[j][m] (F[a][c] - F[b][c]). */
static void apply_swap_to_eq2(int n, const int32_t *D, const int32_t *F, int64_t *Ip, int i,
                              int j, int a, int b) {
    for (int m = 0; m < n; ++m)
        for (int c = 0; c < n; ++c) {
            int64_t out_i = (int64_t)D[(size_t)m * n + i] *
                            ((int64_t)F[(size_t)c * n + b] - F[(size_t)c * n + a]);
            int64_t out_j = (int64_t)D[(size_t)m * n + j] *
                            ((int64_t)F[(size_t)c * n + a] - F[(size_t)c * n + b]);
            int64_t in_i = (int64_t)D[(size_t)i * n + m] *
                           ((int64_t)F[(size_t)b * n + c] - F[(size_t)a * n + c]);
            int64_t in_j = (int64_t)D[(size_t)j * n + m] *
                           ((int64_t)F[(size_t)a * n + c] - F[(size_t)b * n + c]);
            Ip[(size_t)m * n + c] -= out_i + out_j + in_i + in_j;
        }
}

/* 1 if M equals its transpose. */
int oracle_is_symmetric(int n, const int32_t *M) {
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (M[(size_t)i * n + j] != M[(size_t)j * n + i]) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Reading R4: the Eq. 5 weights in binary32.                               */
/*   x = (float)(dE_j - dE_min) * beta                  (one rounded multiply)
 *   w = 0                               if x > 40
 *   w = trunc(expneg(x) * 2^53)         otherwise (a uint64; the scaling is exact)
 * expneg(x) = e^-x by Cody and Waite's two-constant argument reduction
 * (W. J. Cody and W. Waite, Software Manual for the Elementary Functions,
 * 1980): x = k ln2 + r with k the nearest integer to x log2(e), then the
 * degree-7 Taylor polynomial of e^-r in Horner form, then an exact scaling by
 * 2^-k. The constants are ln 2 split into a head with 15 significant bits and
 * its binary32 remainder, and the Taylor coefficients 1/k!.                 */
/* ------------------------------------------------------------------------ */
float oracle_expneg_f32(float x) {
    const float log2e = 1.44269502f;          /* nearest float to 1/ln 2 */
    const float ln2_head = 0.693145751953125f; /* 0x3F317200 */
    const float ln2_tail = 1.42860677e-06f;   /* nearest float to ln 2 - ln2_head */
    const float inv_fact[8] = {1.0f,           1.0f,           0.5f,
                               0.166666672f,   0.0416666679f,  0.00833333377f,
                               0.00138888892f, 0.000198412701f};
    float t = x * log2e;
    t = t + 0.5f;
    int k = (int)t; /* x >= 0: truncation of x log2(e) + 1/2 */
    float kf = (float)k;
    float r = fmaf(-kf, ln2_head, x);
    r = fmaf(-kf, ln2_tail, r);
    float y = -r;
    float q = inv_fact[7];
    for (int d = 6; d >= 0; --d) q = fmaf(q, y, inv_fact[d]);
    /* 2^-k as a binary32 bit pattern; k <= 58 here so it is a normal number */
    union { uint32_t u; float f; } s;
    s.u = (uint32_t)(127 - k) << 23;
    return q * s.f;
}

uint64_t oracle_weight(float x) {
    if (!(x <= 40.0f)) return 0;
    float e = oracle_expneg_f32(x);
    float scaled = e * 9007199254740992.0f; /* 2^53 */
    return (uint64_t)scaled;
}

/* ------------------------------------------------------------------------ */
/* One p-dit update (Eq. 5) at location i.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    const int32_t *D, *F;
    int32_t *p;
    int64_t *I;     /* symmetric form: I of reading R1; general form: Ip of Eq. 2 */
    int64_t E;
    int general;    /* 1: the general form (reading R13) */
} replica_t;

/* Exact double-precision Eq. 5 CDF boundaries, used only to count the draws
 * that fall within 1e-6 of a boundary (reading R4). */
static int near_exact_boundary(int n, const int64_t *dE, int64_t dmin, float beta,
                               uint64_t r) {
    double *pr = (double *)malloc(sizeof(double) * (size_t)n);
    double z = 0.0;
    for (int j = 0; j < n; ++j) {
        pr[j] = exp(-(double)beta * (double)(dE[j] - dmin));
        z += pr[j];
    }
    double u = (double)(r >> 11) * (1.0 / 9007199254740992.0); /* r / 2^64 */
    double c = 0.0;
    int near = 0;
    for (int j = 0; j + 1 < n; ++j) {
        c += pr[j] / z;
        if (fabs(u - c) < 1e-6) near = 1;
    }
    free(pr);
    return near;
}

/* Computes every candidate's dE and quantised weight, then picks the outcome
 * with the 64-bit draw r: t = floor(r * W / 2^64), W = sum of weights, and the
 * outcome is the smallest j whose inclusive prefix sum exceeds t. Returns j;
 * j == i means stay. Optional outputs: dE_out[n], w_out[n], near. */
int oracle_choose(const replica_t *R, int i, float beta, uint64_t r, int64_t *dE_out,
                  uint64_t *w_out, int *near) {
    int n = R->n;
    int64_t *dE = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    for (int j = 0; j < n; ++j)
        dE[j] = R->general ? oracle_delta_e_eq3(n, R->D, R->F, R->p, R->I, i, j)
                           : oracle_delta_e(n, R->D, R->F, R->p, R->I, i, j);
    int64_t dmin = dE[0];
    for (int j = 1; j < n; ++j)
        if (dE[j] < dmin) dmin = dE[j];
    uint64_t W = 0;
    for (int j = 0; j < n; ++j) {
        float x = (float)(dE[j] - dmin) * beta;
        w[j] = oracle_weight(x);
        W += w[j];
    }
    uint64_t t = (uint64_t)(((unsigned __int128)r * (unsigned __int128)W) >> 64);
    uint64_t prefix = 0;
    int chosen = n - 1;
    for (int j = 0; j < n; ++j) {
        prefix += w[j];
        if (prefix > t) {
            chosen = j;
            break;
        }
    }
    if (near) *near = near_exact_boundary(n, dE, dmin, beta, r);
    if (dE_out) memcpy(dE_out, dE, sizeof(int64_t) * (size_t)n);
    if (w_out) memcpy(w_out, w, sizeof(uint64_t) * (size_t)n);
    free(dE);
    free(w);
    return chosen;
}

/* Apply the chosen swap: influence table, permutation, energy. */
static void apply_choice(replica_t *R, int i, int j, int64_t dEj) {
    int a = R->p[i], b = R->p[j];
    if (R->general)
        apply_swap_to_eq2(R->n, R->D, R->F, R->I, i, j, a, b);
    else
        apply_swap_to_influence(R->n, R->D, R->F, R->I, i, j, a, b);
    R->p[i] = b;
    R->p[j] = a;
    R->E += dEj;
}

/* ------------------------------------------------------------------------ */
/* Parallel tempering exchange for one set (reading R7).                    */
/* rung_of_slot[k]: rung of the set's k-th replica; rung 0 = smallest beta. */
/* After every `period` sweeps: for rungs q = 0 .. L-2 in ascending order, if */
/* the replica at rung q+1 has an energy >= that at rung q, the two swap     */
/* rungs (their configurations trade temperatures). If the top rung took no  */
/* part in a swap for `timeout` consecutive exchange periods, the top and    */
/* bottom rungs swap and the count restarts.                                 */
/* ------------------------------------------------------------------------ */
void oracle_pt_exchange(int L, const int64_t *E_of_slot, int32_t *rung_of_slot,
                        int32_t *periods_since_top_swap, int timeout) {
    int32_t *slot_at = (int32_t *)malloc(sizeof(int32_t) * (size_t)L);
    for (int k = 0; k < L; ++k) slot_at[rung_of_slot[k]] = k;
    int top_swapped = 0;
    for (int q = 0; q + 1 < L; ++q) {
        int lo = slot_at[q], hi = slot_at[q + 1];
        if (E_of_slot[hi] >= E_of_slot[lo]) {
            slot_at[q] = hi;
            slot_at[q + 1] = lo;
            if (q + 1 == L - 1) top_swapped = 1;
        }
    }
    if (top_swapped)
        *periods_since_top_swap = 0;
    else
        *periods_since_top_swap += 1;
    if (timeout > 0 && *periods_since_top_swap >= timeout) {
        int t = slot_at[L - 1];
        slot_at[L - 1] = slot_at[0];
        slot_at[0] = t;
        *periods_since_top_swap = 0;
    }
    for (int q = 0; q < L; ++q) rung_of_slot[slot_at[q]] = q;
    free(slot_at);
}

/* ------------------------------------------------------------------------ */
/* Anneal (plain mode) and parallel tempering (PT mode).                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    const int32_t *D, *F;
    int rep_begin, rep_end;   /* replicas [rep_begin, rep_end) */
    int mode;                 /* 0: anneal beta[sweep]; 1: PT beta[rung]; 2: beta[replica]; 3: concurrent updates, beta[sweep] */
    int ladder_len, period, timeout;
    const float *beta;        /* anneal: [sweeps]; PT: [ladder_len] */
    int sweeps;
    uint64_t seed;
    uint32_t inst;
    /* outputs, indexed by replica - rep_begin */
    int32_t *final_p;     /* [R*n] */
    int64_t *final_E;     /* [R] */
    int32_t *best_p;      /* [R*n] */
    int64_t *best_E;      /* [R] */
    int32_t *best_sweep;  /* [R] */
    int64_t *accepted;    /* [R] */
    int64_t *near;        /* [R] or NULL */
    int64_t *final_I;     /* [R*n*n] or NULL */
    int32_t *final_rung;  /* [R] or NULL (PT) */
    int has_target;       /* record the first sweep at which best <= target */
    int64_t target;
    int32_t *reach;       /* [R] or NULL: that sweep (-1 = initial state), INT32_MAX if never */
    int general;          /* keep Eq. 2's table and use Eq. 3 as printed (reading R13) */
    int status;
} anneal_job_t;

/* ------------------------------------------------------------------------ */
/* Concurrent updates (GPU-CUPIM Algorithm section; reading R12). One        */
/* iteration: (1) every location i draws a proposal j_i from Eq. 5 over the   */
/* swap energies of the current state (a snapshot: nothing changes while the  */
/* proposals are drawn), with the draw of location i in that iteration;      */
/* (2) the proposals that move (j_i != i) are ranked by their snapshot energy */
/* change, ascending, ties to the lower initiating location, and accepted in */
/* that order when neither of their two locations is taken yet (a pair       */
/* proposed from both ends is accepted once); losers stay; (3) the accepted   */
/* swaps are applied in that order, each with its exact energy change on the  */
/* then-current table (Eq. 3) and the incremental influence update.          */
/* Returns the number of swaps applied.                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int i, j;
    int64_t dE;
} proposal_t;

static int proposal_before(const proposal_t *x, const proposal_t *y) {
    return x->dE < y->dE || (x->dE == y->dE && x->i < y->i);
}

static int cupim_iteration(replica_t *X, float beta, uint64_t seed, uint32_t inst, uint32_t rep,
                           uint32_t sweep) {
    const int n = X->n;
    proposal_t *prop = (proposal_t *)malloc(sizeof(proposal_t) * (size_t)n);
    int64_t *dE = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int np = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t r = oracle_update_draw(seed, inst, rep, sweep, (uint32_t)i);
        int j = oracle_choose(X, i, beta, r, dE, NULL, NULL);
        if (j != i) {
            prop[np].i = i;
            prop[np].j = j;
            prop[np].dE = dE[j];
            ++np;
        }
    }
    /* insertion sort by (dE, i) */
    for (int a = 1; a < np; ++a) {
        proposal_t key = prop[a];
        int b = a - 1;
        while (b >= 0 && proposal_before(&key, &prop[b])) {
            prop[b + 1] = prop[b];
            --b;
        }
        prop[b + 1] = key;
    }
    unsigned char *taken = (unsigned char *)calloc((size_t)n, 1);
    int applied = 0;
    for (int a = 0; a < np; ++a) {
        int i = prop[a].i, j = prop[a].j;
        if (taken[i] || taken[j]) continue;
        taken[i] = taken[j] = 1;
        int64_t d = X->general ? oracle_delta_e_eq3(n, X->D, X->F, X->p, X->I, i, j)
                               : oracle_delta_e(n, X->D, X->F, X->p, X->I, i, j);
        apply_choice(X, i, j, d);
        ++applied;
    }
    free(taken);
    free(prop);
    free(dE);
    return applied;
}

static void run_job(anneal_job_t *J) {
    const int n = J->n;
    const int R = J->rep_end - J->rep_begin;
    replica_t *reps = (replica_t *)calloc((size_t)R, sizeof(replica_t));
    int32_t *rung = (int32_t *)calloc((size_t)R, sizeof(int32_t));
    int nsets = J->mode == 1 ? R / J->ladder_len : 0;
    int32_t *since_top = (int32_t *)calloc((size_t)(nsets > 0 ? nsets : 1), sizeof(int32_t));
    for (int k = 0; k < R; ++k) {
        uint32_t rep = (uint32_t)(J->rep_begin + k);
        replica_t *X = &reps[k];
        X->n = n;
        X->D = J->D;
        X->F = J->F;
        X->p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        X->I = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * n);
        X->general = J->general;
        oracle_init_perm(n, J->seed, J->inst, rep, X->p);
        if (X->general)
            oracle_influence_eq2(n, J->D, J->F, X->p, X->I);
        else
            oracle_influence(n, J->D, J->F, X->p, X->I);
        X->E = oracle_cost(n, J->D, J->F, X->p);
        memcpy(J->best_p + (size_t)k * n, X->p, sizeof(int32_t) * (size_t)n);
        J->best_E[k] = X->E;
        J->best_sweep[k] = -1;
        J->accepted[k] = 0;
        if (J->reach) J->reach[k] = (J->has_target && X->E <= J->target) ? -1 : 0x7FFFFFFF;
        if (J->near) J->near[k] = 0;
        if (J->mode == 1) rung[k] = (int32_t)(rep % (uint32_t)J->ladder_len);
    }
    for (int s = 0; s < J->sweeps; ++s) {
        for (int k = 0; k < R; ++k) {
            replica_t *X = &reps[k];
            uint32_t rep = (uint32_t)(J->rep_begin + k);
            float beta = J->mode == 1 ? J->beta[rung[k]] : J->mode == 2 ? J->beta[k] : J->beta[s];
            if (J->mode == 3) {
                J->accepted[k] += cupim_iteration(X, beta, J->seed, J->inst, rep, (uint32_t)s);
                if (X->E < J->best_E[k]) {
                    J->best_E[k] = X->E;
                    J->best_sweep[k] = s;
                    memcpy(J->best_p + (size_t)k * n, X->p, sizeof(int32_t) * (size_t)n);
                    if (J->reach && J->has_target && J->reach[k] == 0x7FFFFFFF && X->E <= J->target)
                        J->reach[k] = s;
                }
                continue;
            }
            for (int i = 0; i < n; ++i) {
                uint64_t r = oracle_update_draw(J->seed, J->inst, rep, (uint32_t)s, (uint32_t)i);
                int64_t *dE = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
                int near = 0;
                int j = oracle_choose(X, i, beta, r, dE, NULL, J->near ? &near : NULL);
                if (J->near) J->near[k] += near;
                if (j != i) {
                    apply_choice(X, i, j, dE[j]);
                    J->accepted[k] += 1;
                    if (X->E < J->best_E[k]) {
                        J->best_E[k] = X->E;
                        J->best_sweep[k] = s;
                        memcpy(J->best_p + (size_t)k * n, X->p, sizeof(int32_t) * (size_t)n);
                        if (J->reach && J->has_target && J->reach[k] == 0x7FFFFFFF &&
                            X->E <= J->target)
                            J->reach[k] = s;
                    }
                }
                free(dE);
            }
        }
        if (J->mode == 1 && (s + 1) % J->period == 0) {
            int L = J->ladder_len;
            int64_t *Es = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
            for (int g = 0; g < nsets; ++g) {
                for (int q = 0; q < L; ++q) Es[q] = reps[g * L + q].E;
                oracle_pt_exchange(L, Es, rung + (size_t)g * L, &since_top[g], J->timeout);
            }
            free(Es);
        }
    }
    for (int k = 0; k < R; ++k) {
        replica_t *X = &reps[k];
        memcpy(J->final_p + (size_t)k * n, X->p, sizeof(int32_t) * (size_t)n);
        J->final_E[k] = X->E;
        if (J->final_I) memcpy(J->final_I + (size_t)k * n * n, X->I, sizeof(int64_t) * (size_t)n * n);
        if (J->final_rung) J->final_rung[k] = rung[k];
        free(X->p);
        free(X->I);
    }
    free(reps);
    free(rung);
    free(since_top);
    J->status = 0;
}

static void *job_thread(void *arg) {
    run_job((anneal_job_t *)arg);
    return NULL;
}

/* Runs replicas [rep_begin, rep_end) on `threads` POSIX threads, each a
 * contiguous block of whole replicas (whole PT sets in PT mode). Every
 * replica is an independent chain, so the split does not change results.
 * form: 0 = the symmetric form when D and F are both symmetric, else the
 * general form; 1 = the general form always. final_I receives the table of
 * the form used (I, or Eq. 2's Ip). Returns 0, or -1 on invalid arguments. */
int oracle_anneal(int n, const int32_t *D, const int32_t *F, int rep_begin, int rep_end,
                  int mode, int ladder_len, int period, int timeout, const float *beta,
                  int sweeps, uint64_t seed, uint32_t inst, int threads, int32_t *final_p,
                  int64_t *final_E, int32_t *best_p, int64_t *best_E, int32_t *best_sweep,
                  int64_t *accepted, int64_t *near, int64_t *final_I, int32_t *final_rung,
                  int has_target, int64_t target, int32_t *reach, int form) {
    if (n < 2 || rep_end <= rep_begin || sweeps < 0 || !D || !F || !beta) return -1;
    if (form != 0 && form != 1) return -1;
    const int general = form == 1 || !oracle_is_symmetric(n, D) || !oracle_is_symmetric(n, F);
    int R = rep_end - rep_begin;
    int unit = 1;
    if (mode == 1) {
        if (ladder_len < 2 || period < 1 || rep_begin % ladder_len || R % ladder_len) return -1;
        unit = ladder_len;
    }
    int units = R / unit;
    if (threads < 1) threads = 1;
    if (threads > units) threads = units;
    anneal_job_t *jobs = (anneal_job_t *)calloc((size_t)threads, sizeof(anneal_job_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    int u0 = 0;
    for (int t = 0; t < threads; ++t) {
        int cnt = units / threads + (t < units % threads ? 1 : 0);
        int k0 = u0 * unit, k1 = (u0 + cnt) * unit;
        u0 += cnt;
        anneal_job_t *J = &jobs[t];
        J->n = n;
        J->D = D;
        J->F = F;
        J->rep_begin = rep_begin + k0;
        J->rep_end = rep_begin + k1;
        J->mode = mode;
        J->ladder_len = ladder_len;
        J->period = period;
        J->timeout = timeout;
        J->beta = mode == 2 ? beta + k0 : beta;
        J->sweeps = sweeps;
        J->seed = seed;
        J->inst = inst;
        J->final_p = final_p + (size_t)k0 * n;
        J->final_E = final_E + k0;
        J->best_p = best_p + (size_t)k0 * n;
        J->best_E = best_E + k0;
        J->best_sweep = best_sweep + k0;
        J->accepted = accepted + k0;
        J->near = near ? near + k0 : NULL;
        J->final_I = final_I ? final_I + (size_t)k0 * n * n : NULL;
        J->final_rung = final_rung ? final_rung + k0 : NULL;
        J->has_target = has_target;
        J->target = target;
        J->reach = reach ? reach + k0 : NULL;
        J->general = general;
    }
    if (threads == 1) {
        run_job(&jobs[0]);
    } else {
        for (int t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, job_thread, &jobs[t]);
        for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    }
    free(jobs);
    free(tid);
    return 0;
}

/* Final answer over replicas: smallest best cost, ties to the lowest replica
 * index (reading R6). Returns the winning replica's position in the arrays. */
int oracle_argmin_best(int R, const int64_t *best_E) {
    int w = 0;
    for (int k = 1; k < R; ++k)
        if (best_E[k] < best_E[w]) w = k;
    return w;
}

/* ------------------------------------------------------------------------ */
/* Brute force: min of Eq. 1 over all n! permutations (Heap's algorithm).    */
/* Returns the optimum; writes one optimal permutation (the first found).    */
/* ------------------------------------------------------------------------ */
int64_t oracle_brute_force(int n, const int32_t *D, const int32_t *F, int32_t *best_perm,
                           int64_t *count_optimal) {
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int *c = (int *)calloc((size_t)n, sizeof(int));
    for (int k = 0; k < n; ++k) p[k] = k;
    int64_t best = oracle_cost(n, D, F, p);
    int64_t cnt = 1;
    memcpy(best_perm, p, sizeof(int32_t) * (size_t)n);
    int k = 1;
    while (k < n) {
        if (c[k] < k) {
            int a = (k % 2 == 0) ? 0 : c[k];
            int32_t t = p[a];
            p[a] = p[k];
            p[k] = t;
            int64_t e = oracle_cost(n, D, F, p);
            if (e < best) {
                best = e;
                cnt = 1;
                memcpy(best_perm, p, sizeof(int32_t) * (size_t)n);
            } else if (e == best) {
                cnt += 1;
            }
            c[k] += 1;
            k = 1;
        } else {
            c[k] = 0;
            k += 1;
        }
    }
    free(p);
    free(c);
    if (count_optimal) *count_optimal = cnt;
    return best;
}

/* ------------------------------------------------------------------------ */
/* Beta schedules (reading R8). beta_max convention: 10 / mean positive dE   */
/* over all n(n-1)/2 swaps from the identity permutation, Eq. 3 (the general */
/* form when D or F is not symmetric).                                      */
/* kind 0: linear 0 -> beta_max; kind 1: geometric beta_max/1000 -> beta_max */
/* ------------------------------------------------------------------------ */
double oracle_beta_max(int n, const int32_t *D, const int32_t *F) {
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *I = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * n);
    for (int k = 0; k < n; ++k) p[k] = k;
    const int general = !oracle_is_symmetric(n, D) || !oracle_is_symmetric(n, F);
    if (general)
        oracle_influence_eq2(n, D, F, p, I);
    else
        oracle_influence(n, D, F, p, I);
    double sum = 0.0;
    int64_t cnt = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            int64_t d = general ? oracle_delta_e_eq3(n, D, F, p, I, i, j)
                                : oracle_delta_e(n, D, F, p, I, i, j);
            if (d > 0) {
                sum += (double)d;
                cnt += 1;
            }
        }
    free(p);
    free(I);
    if (cnt == 0) return 1.0;
    return 10.0 / (sum / (double)cnt);
}

void oracle_beta_schedule(int kind, int sweeps, double beta_max, float *out) {
    for (int s = 0; s < sweeps; ++s) {
        double f = sweeps > 1 ? (double)s / (double)(sweeps - 1) : 1.0;
        double b;
        if (kind == 0)
            b = beta_max * f;
        else
            b = (beta_max / 1000.0) * pow(1000.0, f);
        out[s] = (float)b;
    }
}
