// Annealed p-dit sweep with the influence entries formed by 8-bit dot
// products (symmetric instances whose D and F entries fit a signed byte).
//
// Every swap energy of Eq. 3 needs, for the updating location i and each
// candidate j, two entries of the influence table of Eq. 2 (one-term form
// I[m][c] = sum_y D[m][y] F[c][p(y)]): I[i][p(j)] and I[j][p(i)]. With the
// flow matrix permuted to location order, Q[x][y] = F[p(x)][p(y)], both are
// dot products of length N of byte rows:
//   I[i][p(j)] = sum_y D[i][y] Q[j][y],   I[j][p(i)] = sum_y D[j][y] Q[i][y].
// So instead of the N x N int32 table (40 KB per replica at N = 100, updated
// by a rank-1 term after every accepted swap), a replica keeps Q (N x N
// bytes, 11 KB at N = 100), and an accepted swap i <-> s exchanges rows i, s
// and columns i, s of Q: O(N) bytes instead of O(N^2) table entries. The
// entries are the same exact integers as the table's, so every Eq. 5 draw and
// the whole trajectory are those of the table kernels and the CPU oracle;
// the p-diagonal h[x] = I[x][p(x)] is still maintained incrementally (the
// rank-1 update of Eq. 2 evaluated on the diagonal only).
//
// A group of 32 * WPR threads runs one replica; thread t owns the MAXK
// consecutive locations t*MAXK + k (outcome order = location order, so the
// swap energies go to the sampler in registers). Rows of D and Q are kept in
// slot order, row x at slot (x % MAXK) * TA + x / MAXK with TA = ceil(N /
// MAXK): the rows a thread reads at one step sit in consecutive slots across
// threads, and with a row stride of an odd number of 16-byte units the
// 128-bit loads of 8 consecutive threads hit 8 distinct bank groups.
#include "pdit_sweep.cuh"

namespace pdit {

// acc += the dot product of 16 signed bytes. The operands are taken by value
// so that each is one 128-bit shared-memory load (four 32-bit loads of a row
// at this stride would collide in the banks).
__device__ __forceinline__ void dot4(const int4 x, const int4 y, int &acc) {
    acc = __dp4a(x.x, y.x, acc);
    acc = __dp4a(x.y, y.y, acc);
    acc = __dp4a(x.z, y.z, acc);
    acc = __dp4a(x.w, y.w, acc);
}

// 128-bit load from a 32-bit shared-window address. Volatile, so it stays on
// its side of the group barriers (the rows it reads are rewritten between
// them).
__device__ __forceinline__ int4 lds128(uint32_t addr) {
    int4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

// Location held by slot `row` (inverse of the slot map).
template <int MAXK>
__device__ __forceinline__ int dot_loc(int row, int ta) {
    return (row % ta) * MAXK + row / ta;
}

template <int MAXK>
__device__ __forceinline__ int dot_slot(int x, int ta) {
    return (x % MAXK) * ta + x / MAXK;
}

// Part `part` of replica r's sweeps (see part_begin). The first part starts
// as the call says (a Fisher-Yates permutation when a.fresh, Q from the saved
// copy when a.table_in); later parts resume from the state the previous part
// left, Q included. The last part leaves Q as a.table_out says and runs the
// end-of-call Eq. 1 audit. NCH > 0: the row stride is 16 * NCH bytes, fixed
// at compile time, so the chunk loop of the products is unrolled with
// constant offsets; NCH = 0 reads the stride from the descriptor. The state
// a part resumes from is read through L2 (__ldcg): another SM may have
// written it in the same launch.
template <int MAXK, int WPR, int NCH = 0, bool PARTS = false>
__device__ __forceinline__ void run_dot_replica(const SweepArgs &a, int r, int t, int bar, const int8_t *sD,
                                                int8_t *sQ, int32_t *sp, int32_t *sh, GroupScratch *gs) {
    // PARTS: the part (gs->cnt, set by the caller before a group
    // synchronisation) and its last sweep stay in the group scratch, read
    // where needed, rather than in registers across the sweeps; otherwise
    // the whole call is one part
    const int part = PARTS ? *reinterpret_cast<volatile const int *>(&gs->cnt) : 0;
    const bool first_part = part == 0;
    const int seg_fresh = first_part ? a.fresh : 0;
    if (PARTS && t == 0) gs->part_end = part >= a.segments - 1 ? a.sweep_end : part_begin(a, part + 1);
    constexpr int G = 32 * WPR;
    const int lane = t & 31;
    const int wg = t >> 5;
    const int n = a.n;
    const int S8 = NCH > 0 ? 16 * NCH : a.stride;  // row stride of D and Q in bytes: 16 x odd >= n
    const int W4 = S8 >> 2;   // 32-bit words per row
    const int TA = (n + MAXK - 1) / MAXK;
    const int rows = TA * MAXK;
    const uint32_t grep = a.rep_base + (uint32_t)r;
    int32_t *gp = a.perm + (size_t)r * n;
    int32_t *gbp = a.best_perm + (size_t)r * n;
    const bool active = t < TA;  // threads t >= TA own no location

    // ---- permutation (sh serves as scratch for the Fisher-Yates draws)
    if (seg_fresh) {
        fisher_yates<WPR>(a, grep, n, t, sh, sp, bar);
    } else {
        for (int m = t; m < n; m += G) sp[m] = __ldcg(gp + m);
    }
    group_sync<WPR>(bar);

    // ---- Q[slot(x)][y] = F[p(x)][p(y)], zero outside n x n; or the copy
    // saved by the previous call on this replica (a.tables, rows x stride
    // bytes per replica)
    const size_t qbytes = (size_t)rows * S8;
    if (first_part ? a.table_in : 1) {
        const int4 *src = reinterpret_cast<const int4 *>(reinterpret_cast<const int8_t *>(a.tables) + (size_t)r * qbytes);
        for (int idx = t; idx < (int)(qbytes / 16); idx += G) reinterpret_cast<int4 *>(sQ)[idx] = __ldcg(src + idx);
    } else {
        for (int idx = t; idx < rows * W4; idx += G) {
            const int row = idx / W4, w = idx - row * W4;
            const int x = dot_loc<MAXK>(row, TA);
            uint32_t word = 0;
            if (x < n) {
                const int32_t *Fx = a.F + (size_t)sp[x] * n;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int y = 4 * w + b;
                    if (y < n) word |= (uint32_t)(uint8_t)(int8_t)Fx[sp[y]] << (8 * b);
                }
            }
            reinterpret_cast<uint32_t *>(sQ + (size_t)row * S8)[w] = word;
        }
    }
    group_sync<WPR>(bar);

    // ---- p-diagonal h[x] = I[x][p(x)] = D[x] . Q[x]; E = sum_x h[x] (Eq. 1 regrouped)
    int pc[MAXK], hc[MAXK];  // facility and p-diagonal of this thread's locations
    long long esum = 0;
#pragma unroll
    for (int k = 0; k < MAXK; ++k) {
        const int x = t * MAXK + k;
        pc[k] = 0;
        hc[k] = 0;
        if (active && x < n) {
            const int slot = k * TA + t;
            const int8_t *Dx = sD + (size_t)slot * S8, *Qx = sQ + (size_t)slot * S8;
            int acc = 0;
            for (int c = 0; c < S8; c += 16)
                dot4(*reinterpret_cast<const int4 *>(Dx + c), *reinterpret_cast<const int4 *>(Qx + c), acc);
            hc[k] = acc;
            pc[k] = sp[x];
            sh[x] = acc;
            esum += acc;
        }
    }
    esum = warp_sum(esum);
    if constexpr (WPR > 1) {
        if (lane == 0) gs->wtot[wg] = (unsigned long long)esum;
        group_sync<WPR>(bar);
        esum = 0;
#pragma unroll
        for (int w = 0; w < WPR; ++w) esum += (long long)gs->wtot[w];
    }
    long long E, bestE, acc_moves;
    int bsweep;
    bool reached = false;
    if (seg_fresh) {
        E = esum;
        bestE = esum;
        bsweep = -1;
        acc_moves = 0;
        for (int m = t; m < n; m += G) gbp[m] = sp[m];
        if (t == 0) note_target(a, bestE, -1, reached);
    } else {
        E = __ldcg(a.energy + r);
        bestE = __ldcg(a.best_energy + r);
        bsweep = __ldcg(a.best_sweep + r);
        acc_moves = __ldcg(a.accepted + r);
        if (E != esum && t == 0) atomicOr(a.status, 1);
    }
    group_sync<WPR>(bar);

    const int s_begin = part_begin(a, part);
    const float beta_fixed = a.sweep_end <= a.sweep_begin ? 0.0f
                           : a.mode == 1 ? a.beta[a.rung[r]] : a.mode == 2 ? a.beta[r] : 0.0f;
    const int zero_diag = a.zero_diag;
    // shared-window addresses of the rows of this thread's locations
    const uint32_t sD32 = (uint32_t)__cvta_generic_to_shared(sD);
    const uint32_t sQ32 = (uint32_t)__cvta_generic_to_shared(sQ);
    uint32_t rowD[MAXK], rowQ[MAXK];
#pragma unroll
    for (int k = 0; k < MAXK; ++k) {
        rowD[k] = sD32 + (uint32_t)((k * TA + t) * S8);
        rowQ[k] = sQ32 + (uint32_t)((k * TA + t) * S8);
    }

    for (int s = s_begin; s < (PARTS ? *reinterpret_cast<volatile const int *>(&gs->part_end) : a.sweep_end); ++s) {
        if (a.stop) {
            // group-uniform decision from one read of the instance's flag
            if (t == 0) gs->stop = *reinterpret_cast<volatile int *>(a.done);
            group_sync<WPR>(bar);
            const int stop_now = gs->stop;
            group_sync<WPR>(bar);
            if (stop_now) break;
        }
        const float beta_now = (a.mode == 1 || a.mode == 2) ? beta_fixed : a.beta[s];
        // One p-dit update of location i with the influence entries rowv[k] =
        // I[i][p(j)], colv[k] = I[j][p(i)] of this thread's locations j. With
        // `fix`, rowB and colB hold the entries of the next location i + 1
        // (computed from the same state) and are brought up to date when
        // the update swaps, before the rows of Q move.
        auto step = [&](const int i, const unsigned long long draw, const int (&rowv)[MAXK],
                        const int (&colv)[MAXK], const bool fix, int (&rowB)[MAXK], int (&colB)[MAXK]) {
            const int si = dot_slot<MAXK>(i, TA);
            const int hi = sh[i];
            const int8_t *Di = sD + (size_t)si * S8;
            const int8_t *Qi = sQ + (size_t)si * S8;

            // ---- swap energies (Eq. 3 in the one-term units)
            int dc[MAXK];
            int lmin = 0x7FFFFFFF;
#pragma unroll
            for (int k = 0; k < MAXK; ++k) {
                const int j = t * MAXK + k;
                dc[k] = 0;
                if (active && j < n) {
                    const int dij = Di[j];
                    const int fab = Qi[j];  // F[p(i)][p(j)]
                    int d = 2 * (rowv[k] - hi + colv[k] - hc[k]);
                    if (zero_diag) {
                        d += 4 * dij * fab;
                    } else {
                        const size_t sj = (size_t)(k * TA + t) * S8;
                        d += ((int)Di[i] + (int)sD[sj + j] - 2 * dij) * ((int)Qi[i] + (int)sQ[sj + j] - 2 * fab);
                    }
                    if (j == i) d = 0;
                    dc[k] = d;
                    lmin = min(lmin, d);
                }
            }
            auto fac = [&](int kk) {  // pc[kk] without indexing registers at run time
                int v = 0;
#pragma unroll
                for (int k = 0; k < MAXK; ++k)
                    if (k == kk) v = pc[k];
                return v;
            };
            const int3 sel = eq5_draw_regs<MAXK, WPR>(dc, fac, n, t, lmin, beta_now, draw, bar, gs);
            const int js = sel.x, dstar = sel.y, fb = sel.z;
            if (js == i) return;

            // ---- apply the swap i <-> js (facilities fa = p(i), fb = p(js))
            const int sj = dot_slot<MAXK>(js, TA);
            const int8_t *Dj = sD + (size_t)sj * S8;
            const int8_t *Qj = sQ + (size_t)sj * S8;
            const int fa = sp[i];
            const bool own_i = active && (unsigned)(i - t * MAXK) < (unsigned)MAXK;
            const bool own_j = active && (unsigned)(js - t * MAXK) < (unsigned)MAXK;
            // p-diagonal of the locations that keep their facility: h[m] +=
            // (D[i][m] - D[js][m]) (F[fb][p(m)] - F[fa][p(m)]), read from the
            // rows of Q before they move
#pragma unroll
            for (int k = 0; k < MAXK; ++k) {
                const int m = t * MAXK + k;
                if (active && m < n && m != i && m != js) {
                    hc[k] += ((int)Di[m] - (int)Dj[m]) * ((int)Qj[m] - (int)Qi[m]);
                    sh[m] = hc[k];
                }
            }
            // the two moved entries, by the owner of js (which holds
            // I[i][fb] = rowv and I[js][fa] = colv for it)
            if (own_j) {
                const int kk = js - t * MAXK;
                int rv = 0, cv = 0;
#pragma unroll
                for (int k = 0; k < MAXK; ++k)
                    if (k == kk) {
                        rv = rowv[k];
                        cv = colv[k];
                    }
                const int hi_new = rv + ((int)Di[i] - (int)Dj[i]) * ((int)Qj[js] - (int)Qi[js]);
                const int hj_new = cv + ((int)Di[js] - (int)Dj[js]) * ((int)Qj[i] - (int)Qi[i]);
                sh[i] = hi_new;
                sh[js] = hj_new;
#pragma unroll
                for (int k = 0; k < MAXK; ++k)
                    if (k == kk) {
                        hc[k] = hj_new;
                        pc[k] = fa;
                    }
            }
            // The next location's entries under the swap tau = (i js), from
            // the rows before they move (i' = i + 1):
            //   I'[i'][p'(j)] = D[i'] . Q[tau j] o tau
            //                 = rowB[tau j] + (D[i'][js] - D[i'][i]) (Q[tau j][i] - Q[tau j][js]),
            //   I'[j][p'(i')] = D[j] . Q[tau i'] o tau
            //                 = (colB[j], or colv[j] when js = i') + (D[j][js] - D[j][i]) (Q[tau i'][i] - Q[tau i'][js]).
            // rowB at i and at js trade through the group scratch.
            int fixI = 0, fixJ = 0;
            if (fix) {
                const int ip = i + 1;
                const int8_t *Dip = sD + (size_t)dot_slot<MAXK>(ip, TA) * S8;
                const int8_t *Qip = sQ + (size_t)dot_slot<MAXK>(ip, TA) * S8;
                const int delta = (int)Dip[js] - (int)Dip[i];
                const int qf = js != ip ? (int)Qip[i] - (int)Qip[js] : (int)Qi[i] - (int)Qi[js];
                fixI = delta * ((int)Qj[i] - (int)Qj[js]);
                fixJ = delta * ((int)Qi[i] - (int)Qi[js]);
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int j = t * MAXK + k;
                    if (active && j < n) {
                        const size_t sjk = (size_t)(k * TA + t) * S8;
                        const int dfac = (int)sD[sjk + js] - (int)sD[sjk + i];
                        colB[k] = (js != ip ? colB[k] : colv[k]) + dfac * qf;
                        if (j != i && j != js) rowB[k] += delta * ((int)sQ[sjk + i] - (int)sQ[sjk + js]);
                    }
                }
                if (own_j) {
                    int v = 0;
#pragma unroll
                    for (int k = 0; k < MAXK; ++k)
                        if (k == js - t * MAXK) v = rowB[k];
                    gs->aux0 = v;  // rowB at js before the swap
                }
                if (own_i) {
                    int v = 0;
#pragma unroll
                    for (int k = 0; k < MAXK; ++k)
                        if (k == i - t * MAXK) v = rowB[k];
                    gs->aux1 = v;  // rowB at i before the swap
                }
            }
            group_sync<WPR>(bar);  // every read of the old rows, sp[i], sh and the scratch writes done
            if (fix) {
                const int bj = gs->aux0, bi = gs->aux1;
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    if (own_i && k == i - t * MAXK) rowB[k] = bj + fixI;
                    if (own_j && k == js - t * MAXK) rowB[k] = bi + fixJ;
                }
            }
            // rows i and js of Q trade places
            for (int c = 16 * t; c < S8; c += 16 * G) {
                int4 *ri = reinterpret_cast<int4 *>(sQ + (size_t)si * S8 + c);
                int4 *rj = reinterpret_cast<int4 *>(sQ + (size_t)sj * S8 + c);
                const int4 x = *ri;
                *ri = *rj;
                *rj = x;
            }
            if (t == 0) {
                sp[i] = fb;
                sp[js] = fa;
            }
            group_sync<WPR>(bar);
            // then columns i and js, in every row
            for (int row = t; row < rows; row += G) {
                int8_t *q = sQ + (size_t)row * S8;
                const int8_t x = q[i];
                q[i] = q[js];
                q[js] = x;
            }
            if (own_i) {
                const int ki = i - t * MAXK;
                const int hnew = sh[i];
#pragma unroll
                for (int k = 0; k < MAXK; ++k)
                    if (k == ki) {
                        hc[k] = hnew;
                        pc[k] = fb;
                    }
            }
            E += dstar;
            acc_moves += 1;
            if (E < bestE) {
                bestE = E;
                bsweep = s;
                for (int m = t; m < n; m += G) gbp[m] = sp[m];
                if (t == 0) note_target(a, bestE, s, reached);
            }
            group_sync<WPR>(bar);  // Q complete before the next update's products
        };

        for (int i0 = 0; i0 < n; i0 += 32) {
            // Philox(inst, replica, sweep, location) for the next 32 locations
            const uint4 rw = philox4x32_10(a.inst, grep, (uint32_t)s, (uint32_t)(i0 + lane), a.key0, a.key1);
            const int cnt = min(32, n - i0);
            for (int ii = 0; ii < cnt; ii += 2) {
                // locations i and i + 1 (when it is in this batch) from one
                // pass over this thread's rows of D and Q
                const int i = i0 + ii;
                const bool two = ii + 1 < cnt;
                int rowA[MAXK], colA[MAXK], rowB[MAXK], colB[MAXK];
#pragma unroll
                for (int k = 0; k < MAXK; ++k) rowA[k] = colA[k] = rowB[k] = colB[k] = 0;
                if (active) {
                    const int si = dot_slot<MAXK>(i, TA);
                    const uint32_t aDi = sD32 + (uint32_t)(si * S8), aQi = sQ32 + (uint32_t)(si * S8);
                    if (two) {
                        const int si1 = dot_slot<MAXK>(i + 1, TA);
                        const uint32_t aDi1 = sD32 + (uint32_t)(si1 * S8), aQi1 = sQ32 + (uint32_t)(si1 * S8);
                        // one 16-byte chunk of every row at a time
                        auto chunk2 = [&](const uint32_t c) {
                            const int4 di = lds128(aDi + c), qi = lds128(aQi + c);
                            const int4 di1 = lds128(aDi1 + c), qi1 = lds128(aQi1 + c);
#pragma unroll
                            for (int k = 0; k < MAXK; ++k) {
                                const int4 qj = lds128(rowQ[k] + c), dj = lds128(rowD[k] + c);
                                dot4(di, qj, rowA[k]);
                                dot4(di1, qj, rowB[k]);
                                dot4(dj, qi, colA[k]);
                                dot4(dj, qi1, colB[k]);
                            }
                        };
                        if constexpr (NCH > 0) {
#pragma unroll
                            for (int ch = 0; ch < NCH; ++ch) chunk2(16u * ch);
                        } else {
#pragma unroll 1
                            for (int c = 0; c < S8; c += 16) chunk2((uint32_t)c);
                        }
                    } else {
                        auto chunk1 = [&](const uint32_t c) {
                            const int4 di = lds128(aDi + c), qi = lds128(aQi + c);
#pragma unroll
                            for (int k = 0; k < MAXK; ++k) {
                                dot4(di, lds128(rowQ[k] + c), rowA[k]);
                                dot4(lds128(rowD[k] + c), qi, colA[k]);
                            }
                        };
                        if constexpr (NCH > 0) {
#pragma unroll
                            for (int ch = 0; ch < NCH; ++ch) chunk1(16u * ch);
                        } else {
#pragma unroll 1
                            for (int c = 0; c < S8; c += 16) chunk1((uint32_t)c);
                        }
                    }
                }
                const unsigned long long drawA =
                    ((unsigned long long)__shfl_sync(kFull, rw.y, ii) << 32) |
                    (unsigned long long)__shfl_sync(kFull, rw.x, ii);
                step(i, drawA, rowA, colA, two, rowB, colB);
                if (two) {
                    const unsigned long long drawB =
                        ((unsigned long long)__shfl_sync(kFull, rw.y, ii + 1) << 32) |
                        (unsigned long long)__shfl_sync(kFull, rw.x, ii + 1);
                    step(i + 1, drawB, rowB, colB, false, rowB, colB);
                }
            }
        }
    }

    // ---- audit (the last unit of a call): Eq. 1 of the final permutation,
    // from D and the global F, equals the tracked energy
    const int part_now = PARTS ? *reinterpret_cast<volatile const int *>(&gs->cnt) : 0;
    const bool last_part = !PARTS || part_now >= a.segments - 1;
    if (last_part) {
        long long eq1 = 0;
        for (int x = t; x < n; x += G) {
            const int8_t *Dx = sD + (size_t)dot_slot<MAXK>(x, TA) * S8;
            const int32_t *Fx = a.F + (size_t)sp[x] * n;
            long long acc = 0;
            for (int y = 0; y < n; ++y) acc += (long long)Dx[y] * Fx[sp[y]];
            eq1 += acc;
        }
        eq1 = warp_sum(eq1);
        if constexpr (WPR > 1) {
            group_sync<WPR>(bar);
            if (lane == 0) gs->wtot[wg] = (unsigned long long)eq1;
            group_sync<WPR>(bar);
            eq1 = 0;
#pragma unroll
            for (int w = 0; w < WPR; ++w) eq1 += (long long)gs->wtot[w];
        }
        if (t == 0 && eq1 != E) atomicOr(a.status, 1);
    }

    // ---- write back
    for (int m = t; m < n; m += G) gp[m] = sp[m];
    if (t == 0) {
        a.energy[r] = E;
        a.best_energy[r] = bestE;
        a.best_sweep[r] = bsweep;
        a.accepted[r] = acc_moves;
    }
    if (last_part ? a.table_out : 1) {
        int4 *dst = reinterpret_cast<int4 *>(reinterpret_cast<int8_t *>(a.tables) + (size_t)r * qbytes);
        for (int idx = t; idx < (int)(qbytes / 16); idx += G) dst[idx] = reinterpret_cast<const int4 *>(sQ)[idx];
    }
    // A call split into parts: publish this part once every thread's writes
    // of the replica's state are visible device-wide.
    if (PARTS) __threadfence();
    group_sync<WPR>(bar);
    if (PARTS && t == 0) publish_part(a, r, part_now + 1);
}

// D of an n-location instance as int8 rows in slot order (rows x stride
// bytes), zero outside n x n.
template <int MAXK>
__device__ __forceinline__ void stage_dot_d(const int32_t *D, int n, int S8, int8_t *sD) {
    const int W4 = S8 >> 2;
    const int TA = (n + MAXK - 1) / MAXK;
    const int rows = TA * MAXK;
    for (int idx = threadIdx.x; idx < rows * W4; idx += blockDim.x) {
        const int row = idx / W4, w = idx - row * W4;
        const int x = dot_loc<MAXK>(row, TA);
        uint32_t word = 0;
        if (x < n) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int y = 4 * w + b;
                if (y < n) word |= (uint32_t)(uint8_t)(int8_t)D[(size_t)x * n + y] << (8 * b);
            }
        }
        reinterpret_cast<uint32_t *>(sD + (size_t)row * S8)[w] = word;
    }
}

// Persistent: each group of 32 * WPR threads pulls work units from a.queue.
// Shared memory: D as int8 in slot order (rows x stride bytes), then per
// group: scratch, Q (rows x stride bytes), p and h (npad int32 each).
template <int MAXK, int WPR, int NCH, bool PARTS>
__global__ void __launch_bounds__(dot_bound(MAXK, WPR)) dot_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int G = 32 * WPR;
    const int n = a.n;
    const int S8 = NCH > 0 ? 16 * NCH : a.stride;
    const int TA = (n + MAXK - 1) / MAXK;
    const int rows = TA * MAXK;
    const int npad = (n + 3) & ~3;
    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int bar = 1 + grp;  // named barrier of this group (WPR > 1); 0 is __syncthreads
    int8_t *sD = reinterpret_cast<int8_t *>(smem);
    stage_dot_d<MAXK>(a.D, n, S8, sD);
    __syncthreads();
    unsigned char *gb = smem + a.df_bytes + (size_t)grp * a.group_bytes;
    GroupScratch *gs = reinterpret_cast<GroupScratch *>(gb);
    int8_t *sQ = reinterpret_cast<int8_t *>(gb + kScratchBytes);
    int32_t *sp = reinterpret_cast<int32_t *>(gb + kScratchBytes + (size_t)rows * S8);
    int32_t *sh = sp + npad;
    if constexpr (!PARTS) {
        // one unit per replica: the whole call
        for (;;) {
            if (t == 0) gs->item = atomicAdd(a.queue, 1);
            group_sync<WPR>(bar);
            const int item = gs->item;
            if (item >= a.replicas) break;
            run_dot_replica<MAXK, WPR, NCH, false>(a, item, t, bar, sD, sQ, sp, sh, gs);
        }
        return;
    }
    // Work units in order (part k of every replica, then part k + 1): part k
    // of replica r starts once part k - 1 has been published. That part was
    // taken `replicas` units earlier by a group that is running, so the wait
    // ends (it is bounded all the same).
    const int K = a.segments > 1 ? a.segments : 1;
    const long long units = (long long)a.replicas * K;
    for (;;) {
        if (t == 0) {
            // thread 0 splits the unit into (part, replica) and waits for
            // the previous part; the group reads the replica, the part and
            // whether to go on from the scratch
            const int item = atomicAdd(a.queue, 1);
            int go = item < units ? 1 : 0, part = 0, r = item;
            if (go && K > 1) {
                part = item / a.replicas;
                r = item - part * a.replicas;
                if (part > 0) go = wait_part(a, r, part);
            }
            gs->item = r;
            gs->cnt = part;
            gs->stop = go;
        }
        group_sync<WPR>(bar);
        const int go = gs->stop, r = gs->item;
        if (!go) break;
        run_dot_replica<MAXK, WPR, NCH, true>(a, r, t, bar, sD, sQ, sp, sh, gs);
    }
}

// Persistent multi-instance kernel: CTAs take (instance, block of replicas)
// units from `queue` and restage D when they move to another instance.
// Every instance of a launch shares the compiled shape (MAXK, WPR).
template <int MAXK, int WPR>
__global__ void __launch_bounds__(dot_bound(MAXK, WPR))
    dot_batch_kernel(const SweepArgs *__restrict__ descs, const BatchUnit *__restrict__ units, int nunits,
                     int *queue) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepArgs sa;
    __shared__ int s_unit;
    constexpr int G = 32 * WPR;
    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int bar = 1 + grp;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(queue, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= nunits) break;
        const BatchUnit bu = units[u];
        if (bu.inst != cur) {
            // descriptor and D of the new instance
            const int *src = reinterpret_cast<const int *>(descs + bu.inst);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int w = threadIdx.x; w < (int)(sizeof(SweepArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
            stage_dot_d<MAXK>(descs[bu.inst].D, descs[bu.inst].n, descs[bu.inst].stride,
                              reinterpret_cast<int8_t *>(smem));
            cur = bu.inst;
        }
        __syncthreads();
        const int n = sa.n;
        const int r = bu.r0 + grp;
        if (grp < sa.groups && r < sa.replicas) {
            const int rows = ((n + MAXK - 1) / MAXK) * MAXK;
            const int npad = (n + 3) & ~3;
            unsigned char *gb = smem + sa.df_bytes + (size_t)grp * sa.group_bytes;
            GroupScratch *gs = reinterpret_cast<GroupScratch *>(gb);
            int8_t *sQ = reinterpret_cast<int8_t *>(gb + kScratchBytes);
            int32_t *sp = reinterpret_cast<int32_t *>(gb + kScratchBytes + (size_t)rows * sa.stride);
            int32_t *sh = sp + npad;
            run_dot_replica<MAXK, WPR>(sa, r, t, bar, reinterpret_cast<const int8_t *>(smem), sQ, sp, sh, gs);
        }
    }
}

#define PDIT_DOT_SHAPES(X) X(1, 1) X(2, 1) X(4, 1) X(8, 1) X(2, 2) X(1, 4) X(4, 2) X(2, 4) X(1, 8)

template <int MAXK, int WPR, int NCH = 0>
static int dot_one(const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t st, int *blocks,
                   bool query) {
    // calls split into parts run their own instantiation, so that whole
    // calls keep the registers of the plain loop
    auto fn = a.segments > 1 ? dot_kernel<MAXK, WPR, NCH, true> : dot_kernel<MAXK, WPR, NCH, false>;
    if (threads > dot_bound(MAXK, WPR)) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    if (query) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
    fn<<<grid, threads, smem, st>>>(a);
    return (int)cudaGetLastError();
}

static int dot_dispatch(int maxk, int wpr, const SweepArgs &a, int grid, int threads, size_t smem,
                        cudaStream_t st, int *blocks, bool query) {
    // rows of 7 chunks with four locations per thread and one warp per
    // replica (N = 97..112): the compile-time stride
    if (maxk == 4 && wpr == 1 && a.stride == 16 * 7) return dot_one<4, 1, 7>(a, grid, threads, smem, st, blocks, query);
#define PDIT_DOT_CASE(MK, W) \
    if (maxk == MK && wpr == W) return dot_one<MK, W>(a, grid, threads, smem, st, blocks, query);
    PDIT_DOT_SHAPES(PDIT_DOT_CASE)
#undef PDIT_DOT_CASE
    return (int)cudaErrorInvalidValue;
}

bool dot_shape_compiled(int maxk, int wpr) {
#define PDIT_DOT_HAS(MK, W) \
    if (maxk == MK && wpr == W) return true;
    PDIT_DOT_SHAPES(PDIT_DOT_HAS)
#undef PDIT_DOT_HAS
    return false;
}

template <int MAXK, int WPR>
static int dot_batch_one(const SweepArgs *d, const BatchUnit *u, int nu, int *q, int grid, int threads,
                         size_t smem, cudaStream_t st, int *blocks, bool query) {
    auto fn = dot_batch_kernel<MAXK, WPR>;
    if (threads > dot_bound(MAXK, WPR)) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    if (query) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
    fn<<<grid, threads, smem, st>>>(d, u, nu, q);
    return (int)cudaGetLastError();
}

static int dot_batch_dispatch(int maxk, int wpr, const SweepArgs *d, const BatchUnit *u, int nu, int *q, int grid,
                              int threads, size_t smem, cudaStream_t st, int *blocks, bool query) {
#define PDIT_DOT_BATCH_CASE(MK, W) \
    if (maxk == MK && wpr == W) return dot_batch_one<MK, W>(d, u, nu, q, grid, threads, smem, st, blocks, query);
    PDIT_DOT_SHAPES(PDIT_DOT_BATCH_CASE)
#undef PDIT_DOT_BATCH_CASE
    return (int)cudaErrorInvalidValue;
}

int dot_batch_blocks_per_sm(int maxk, int wpr, int threads, size_t smem, int *blocks) {
    return dot_batch_dispatch(maxk, wpr, nullptr, nullptr, 0, nullptr, 0, threads, smem, nullptr, blocks, true);
}

int dot_batch_launch(int maxk, int wpr, const SweepArgs *descs, const BatchUnit *units, int nunits, int *queue,
                     int grid, int threads, size_t smem, cudaStream_t stream) {
    return dot_batch_dispatch(maxk, wpr, descs, units, nunits, queue, grid, threads, smem, stream, nullptr, false);
}

int dot_blocks_per_sm(int maxk, int wpr, int stride, int threads, size_t smem, int *blocks) {
    SweepArgs dummy{};
    dummy.stride = stride;
    return dot_dispatch(maxk, wpr, dummy, 0, threads, smem, nullptr, blocks, true);
}

int dot_launch(int maxk, int wpr, const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t st) {
    return dot_dispatch(maxk, wpr, a, grid, threads, smem, st, nullptr, false);
}

}  // namespace pdit
