// Annealed p-dit sweep kernels for the QAP on sm_103a.
//
// A replica is owned by a group of G = 32 * WPR threads (WPR warps, 1..8).
// A CTA stages the instance's D and F once in shared memory (int8/int16/int32,
// whichever holds every value), and each group keeps its replica's influence
// table, permutation and scratch vectors in its own slice of shared memory
// (or, when the table does not fit, the table in global memory). Groups pull
// replicas from a global atomic counter until none are left.
//
// Per p-dit update (Eq. 5 over the N outcomes of location i):
//   gather   candidate j on thread j mod G: dE_j from Eq. 3 with the
//            influence table, dE_i = 0 (stay)
//   sample   group min of dE, binary32 weights (the arithmetic the CPU oracle
//            states), thread-contiguous 64-bit prefix sums, one 64-bit Philox
//            draw scaled by the total, first prefix above it
//   apply    if a swap j* was drawn: I[m][c] += (D[i][m]-D[j*][m]) (F[b][c]-F[a][c]),
//            either at once (int4 read-modify-writes on each thread's rows)
//            or deferred: the swap's factors are packed as bytes, every
//            query adds the pending terms with dp4a, and the table is
//            rewritten once 4 (16 for tables in global memory) terms are
//            pending; then p, the p-diagonal h and E
//   best     first occurrence of a new minimum of E (strict <)
// With one candidate per thread, thread t owns location t and keeps p(t),
// h(t) and its packed factors in registers. With tables in global memory the
// next update's row and column gathers are prefetched into registers.
// Sweeps visit locations 0..N-1 in order. Every integer is exact; the only
// floating point is the weight computation, made of single correctly rounded
// IEEE operations so the CPU oracle reproduces it bit for bit.
//
// General instances (ASYM: D or F not symmetric) keep Eq. 2's two-term table
// T[m][c] = sum_j D[m][j] F[c][p(j)] + D[j][m] F[p(j)][c] (the negated Eq. 2),
// take Eq. 3 as printed, and apply each swap as a rank-2 update:
//   T[m][c] += (D[m][i]-D[m][j*]) (F[c][b]-F[c][a]) + (D[i][m]-D[j*][m]) (F[b][c]-F[a][c]).
// D and F are then staged with an odd-word row stride so that their columns
// are read without bank conflicts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdit {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct SweepArgs {
    // instance (global, int32, row-major)
    const int32_t *D;
    const int32_t *F;
    int n;
    int stride;     // table row stride S: the smallest 4*odd >= n
    int dstride;    // row stride (elements) of the staged D and F; n for symmetric instances
    int zero_diag;  // D and F both have zero diagonals
    // run
    int replicas;
    int sweep_begin, sweep_end;
    uint32_t key0, key1;   // Philox key = seed
    uint32_t inst;         // Philox counter word 0
    uint32_t rep_base;     // global id of local replica 0 (counter word 1)
    int mode;              // 0 anneal (beta[s]), 1 parallel tempering (beta[rung]), 2 fixed (beta[r]),
                           // 3 concurrent updates (beta[s])
    int cupim_off;         // mode 3: offset (int32 entries) of the proposal arrays in the scratch vector
    int v2_off;            // general form, immediate updates: offset of the second column factor
    int rc_off;            // global tables: offset of the gathered table values (row, then column)
    // flow classes (pdit_class.cu): F[c][d] = f0 + f x_c x_d off the diagonal
    const uint8_t *cls_x;  // x_c of every facility
    int cls_f;             // f
    long long cls_e0;      // f0 * sum over i != j of D[i][j]
    const float *beta;
    int fresh;             // start from a Fisher-Yates permutation
    int table_in;          // take the influence table from `tables` instead of rebuilding it
    int table_out;         // leave the influence table in `tables` at the end
    // per-replica state, indexed by local replica id
    int32_t *perm;
    int32_t *best_perm;
    int64_t *energy;
    int64_t *best_energy;
    int32_t *best_sweep;
    int64_t *accepted;
    const int32_t *rung;
    int32_t *tables;       // [replicas][n][stride] when used
    int32_t *dump;         // optional [replicas][n][n]: final tables
    int *queue;            // work counter, zero at launch
    int *status;           // audit bits
    // dot kernel, anneal and fixed modes: each replica's sweep range split
    // into `segments` consecutive parts run as separate work units (1: one
    // unit per replica); seg_done[r] = parts of replica r finished, zero at
    // launch
    int segments;
    int *seg_done;
    // time-to-target bookkeeping (all optional, per instance)
    const int64_t *target;      // record the first time best <= *target
    unsigned long long *reach_ns;  // atomicMin of %globaltimer at that moment
    int *reach_sweep;           // atomicMin of the sweep index (-1 = initial state)
    int *done;                  // set once reached; replicas stop at their next sweep if stop
    int stop;                   // stop replicas of an instance whose target was reached
    // launch shape
    size_t df_bytes;       // bytes of staged D and F (16-byte multiple)
    size_t group_bytes;    // bytes of one group's slice
    int sv_len;            // int32 entries of the scratch vector (multiple of 4)
    int groups;            // replica groups per CTA (multi-instance launches)
};

// Per-group scratch for cross-warp reductions and broadcasts.
struct GroupScratch {
    unsigned long long wtot[8];
    int wmin[8];
    int sel_jf, sel_d;  // the drawn outcome: location | facility << 16, energy change
    int part_end;       // dot kernel: the last sweep (exclusive) of the part being run
    int item;
    int stop;
    int cnt;            // concurrent updates: accepted swaps; dot kernel: the part being run
    int aux0, aux1;
};
constexpr size_t kScratchBytes = sizeof(GroupScratch);  // 128

// Status bit: a wait for the previous part of a replica passed its bound
// (the value of PDIT_STATUS_SCHEDULE).
constexpr int kStatusSchedule = 2;

// ---------------------------------------------------------------------------
// Philox4x32-10, from its published definition (Salmon, Moraes, Dror and
// Shaw, SC'11): ten rounds of two 32x32->64 multiplies by 0xD2511F53 and
// 0xCD9E8D57, xor with the other words and the round key, key bumped by
// (0x9E3779B9, 0xBB67AE85) between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------
// Eq. 5 weight of one outcome, in binary32 with one rounding per operation:
//   x = (float)(dE - dE_min) * beta
//   w = 0 if x > 40, else trunc(e^-x * 2^53) as a uint64
// e^-x: Cody-Waite reduction x = k ln2 + r (k nearest to x log2 e, ln 2 as a
// 15-bit head plus its binary32 tail), Taylor polynomial q(r) of degree 7 for
// e^-r in Horner form with fused multiply-adds. Then e^-x * 2^53 = q 2^(53-k)
// exactly, so trunc() of it is q's 24-bit significand shifted by its binary
// exponent + 53 - k: integer operations only (a float -> uint64 conversion
// would run on the FP64 pipe).
// Evaluated without a branch, so that the weights of a thread's candidates
// proceed in parallel: an x beyond 40 (or not a number) is replaced by 0 for
// the arithmetic and its weight is zeroed at the end; every other x takes
// exactly the operations above.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long eq5_weight(int shifted_de, float beta) {
    const float x0 = __fmul_rn(__int2float_rn(shifted_de), beta);
    const bool live = x0 <= 40.0f;
    const float x = live ? x0 : 0.0f;
    const float t = __fadd_rn(__fmul_rn(x, 1.44269502f), 0.5f);
    const int k = __float2int_rz(t);
    const float kf = __int2float_rn(k);
    float r = __fmaf_rn(-kf, 0.693145751953125f, x);
    r = __fmaf_rn(-kf, 1.42860677e-06f, r);
    const float y = -r;
    float q = 1.98412701e-04f;             // 1/7!
    q = __fmaf_rn(q, y, 1.38888892e-03f);  // 1/6!
    q = __fmaf_rn(q, y, 8.33333377e-03f);  // 1/5!
    q = __fmaf_rn(q, y, 4.16666679e-02f);  // 1/4!
    q = __fmaf_rn(q, y, 1.66666672e-01f);  // 1/3!
    q = __fmaf_rn(q, y, 0.5f);
    q = __fmaf_rn(q, y, 1.0f);
    q = __fmaf_rn(q, y, 1.0f);
    // q in (0.7, 1.5): a normal float, q = mant * 2^(exp - 150) with exp 126
    // or 127, so w = trunc(q * 2^(53 - k)) = trunc(mant * 2^30 / 2^s) with
    // s = 127 - exp + k in [0, 59] (k <= 58 for x <= 40): one 64-bit right
    // shift of mant * 2^30 (< 2^54), exact for s <= 30 and the truncation
    // otherwise; s = 63 gives the 0 of x > 40.
    const uint32_t bits = __float_as_uint(q);
    const unsigned long long m30 = (unsigned long long)((bits & 0x7FFFFFu) | 0x800000u) << 30;
    const int s = live ? 127 - (int)(bits >> 23) + k : 63;
    return m30 >> s;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int K>
__device__ __forceinline__ void load_block(const int32_t *sv, int t, int (&d)[K]) {
    if constexpr (K == 1) {
        d[0] = sv[t];
    } else if constexpr (K == 2) {
        const int2 v = reinterpret_cast<const int2 *>(sv)[t];
        d[0] = v.x;
        d[1] = v.y;
    } else {
#pragma unroll
        for (int h = 0; h < K / 4; ++h) {
            const int4 v = reinterpret_cast<const int4 *>(sv)[t * (K / 4) + h];
            d[4 * h + 0] = v.x;
            d[4 * h + 1] = v.y;
            d[4 * h + 2] = v.z;
            d[4 * h + 3] = v.w;
        }
    }
}

template <int WPR>
__device__ __forceinline__ void group_sync(int bar) {
    if constexpr (WPR == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * WPR) : "memory");
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First time this replica's best reaches the instance target: record when.
__device__ __forceinline__ void note_target(const SweepArgs &a, long long bestE, int sweep, bool &reached) {
    if (reached || !a.target || bestE > *a.target) return;
    reached = true;
    if (a.reach_ns) atomicMin(a.reach_ns, global_ns());
    if (a.reach_sweep) atomicMin(a.reach_sweep, sweep);
    if (a.done) atomicExch(a.done, 1);
}

// Initial permutation of global replica `grep` into sp (reading R5):
// Fisher-Yates from the last position down; step k uses word k%4 of
// Philox(inst, replica, 0xFFFFFFFF, k/4) and index floor(u (k+1) / 2^32).
// sv receives the random words. No barrier at the end.
template <int WPR>
__device__ __forceinline__ void fisher_yates(const SweepArgs &a, uint32_t grep, int n, int t, int32_t *sv,
                                             int32_t *sp, int bar) {
    constexpr int G = 32 * WPR;
    for (int q = t; 4 * q < n; q += G) {
        const uint4 o = philox4x32_10(a.inst, grep, 0xFFFFFFFFu, (uint32_t)q, a.key0, a.key1);
        reinterpret_cast<uint4 *>(sv)[q] = o;
    }
    for (int m = t; m < n; m += G) sp[m] = m;
    group_sync<WPR>(bar);
    if (t == 0) {
        for (int k = n - 1; k >= 1; --k) {
            const int j = (int)__umulhi((uint32_t)sv[k], (uint32_t)(k + 1));
            const int x = sp[k];
            sp[k] = sp[j];
            sp[j] = x;
        }
    }
}

// ---------------------------------------------------------------------------
// Eq. 5 draw over n outcomes held thread-contiguously: thread t holds the
// swap energies of outcomes t*MAXK + k (k < MAXK; outcomes >= n are ignored),
// which `load(dc)` fills in once the group minimum is known (so energies that
// other threads wrote to shared memory are read after the synchronisation of
// the minimum), and `fac(k)` gives the facility at outcome t*MAXK + k (called
// on the owning thread only); lmin is the minimum over this thread's own
// outcomes. Group minimum, binary32 weights of the shifted energies, 64-bit
// prefix sums in outcome order, the 64-bit draw scaled by the total, and the
// first outcome whose inclusive prefix sum exceeds it. Returns (chosen
// location js, its energy change, the facility at js), the same on every
// thread of the group; the facility is read by the owning thread before the
// final synchronisation. Ends with the group synchronised.
// ---------------------------------------------------------------------------
template <int MAXK, int WPR, typename Load, typename Fac>
__device__ __forceinline__ int3 eq5_draw_core(Load load, Fac fac, int n, int t, int lmin, float beta,
                                              unsigned long long draw, int bar, GroupScratch *gs) {
    const int lane = t & 31;
    const int wg = t >> 5;
    int dmin = __reduce_min_sync(kFull, lmin);
    if constexpr (WPR > 1) {
        if (lane == 0) gs->wmin[wg] = dmin;
        group_sync<WPR>(bar);
        dmin = gs->wmin[0];
#pragma unroll
        for (int w = 1; w < WPR; ++w) dmin = min(dmin, gs->wmin[w]);
    } else {
        __syncwarp();
    }

    // ---- sample: thread-contiguous weights, 64-bit prefix sums
    int dc[MAXK];
    load(dc);
    unsigned long long pre[MAXK];
    unsigned long long lsum = 0;
#pragma unroll
    for (int k = 0; k < MAXK; ++k) {
        if (t * MAXK + k < n) lsum += eq5_weight(dc[k] - dmin, beta);
        pre[k] = lsum;
    }
    unsigned long long incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    unsigned long long total = __shfl_sync(kFull, incl, 31);
    if constexpr (WPR > 1) {
        if (lane == 31) gs->wtot[wg] = incl;
        group_sync<WPR>(bar);
        // every thread reads all warp totals (broadcast) and sums the
        // ones before its warp
        unsigned long long off = 0;
        total = 0;
#pragma unroll
        for (int w = 0; w < WPR; ++w) {
            const unsigned long long v = gs->wtot[w];
            off += w < wg ? v : 0ull;
            total += v;
        }
        incl += off;
    }
    const unsigned long long excl = incl - lsum;
    const unsigned long long tdraw = __umul64hi(draw, total);
    const bool own = (tdraw >= excl) && (tdraw < incl);
    int jloc = 0, dsel = 0, fsel = 0;
    if (own) {
        int kk = MAXK - 1;
#pragma unroll
        for (int k = MAXK - 1; k >= 0; --k)
            if (excl + pre[k] > tdraw) kk = k;
#pragma unroll
        for (int k = 0; k < MAXK; ++k)
            if (k == kk) dsel = dc[k];
        jloc = t * MAXK + kk;
        fsel = fac(kk);
    }
    int js, dstar, fb;
    if constexpr (WPR > 1) {
        // both below 2^16 (n <= 256): one 64-bit store and load
        if (own) *reinterpret_cast<int2 *>(&gs->sel_jf) = make_int2(jloc | (fsel << 16), dsel);
        group_sync<WPR>(bar);
        const int2 sel = *reinterpret_cast<const int2 *>(&gs->sel_jf);
        js = sel.x & 0xFFFF;
        fb = sel.x >> 16;
        dstar = sel.y;
    } else {
        const int src = __ffs(__ballot_sync(kFull, own)) - 1;
        js = __shfl_sync(kFull, jloc, src);
        dstar = __shfl_sync(kFull, dsel, src);
        fb = __shfl_sync(kFull, fsel, src);
        __syncwarp();
    }
    return make_int3(js, dstar, fb);
}

// The draw over energies that each thread holds in registers for its own
// outcomes t*MAXK + k.
template <int MAXK, int WPR, typename Fac>
__device__ __forceinline__ int3 eq5_draw_regs(const int (&dc)[MAXK], Fac fac, int n, int t, int lmin, float beta,
                                              unsigned long long draw, int bar, GroupScratch *gs) {
    auto load = [&](int (&o)[MAXK]) {
#pragma unroll
        for (int k = 0; k < MAXK; ++k) o[k] = dc[k];
    };
    return eq5_draw_core<MAXK, WPR>(load, fac, n, t, lmin, beta, draw, bar, gs);
}

// The draw over energies the group has written to sv[0..n) in location
// order (with one candidate per thread, MAXK = 1, each thread passes its own
// energy in dself and its location's facility in pself instead, and sv is
// not read). The facility of the drawn location is read from sp by its
// owner, so the caller may rewrite sp once every thread has returned.
template <int MAXK, int WPR>
__device__ __forceinline__ int3 eq5_draw(const int32_t *sv, const int32_t *sp, int n, int t, int lmin,
                                         int dself, int pself, float beta, unsigned long long draw,
                                         int bar, GroupScratch *gs) {
    auto load = [&](int (&o)[MAXK]) {
        if constexpr (MAXK == 1)
            o[0] = dself;
        else
            load_block<MAXK>(sv, t, o);
    };
    auto fac = [&](int kk) { return MAXK == 1 ? pself : sp[t * MAXK + kk]; };
    return eq5_draw_core<MAXK, WPR>(load, fac, n, t, lmin, beta, draw, bar, gs);
}

// Bytes of packed word w that hold one of the np pending terms (4 per word).
__device__ __forceinline__ uint32_t pending_mask(int np, int w) {
    const int v = np - 4 * w;
    return v >= 4 ? 0xFFFFFFFFu : (v <= 0 ? 0u : ((1u << (8 * v)) - 1u));
}

__device__ __forceinline__ void add_scaled(int4 &x, int u, const int4 &v) {
    x.x += u * v.x;
    x.y += u * v.y;
    x.z += u * v.z;
    x.w += u * v.w;
}

// ---------------------------------------------------------------------------
// Calls split into parts (more replicas than resident slots): each part of a
// replica's sweeps is a work unit; a part starts once the replica's previous
// part is published.
// ---------------------------------------------------------------------------
// Parts done of replica r, read with acquire semantics at GPU scope.
__device__ __forceinline__ int load_parts_done(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void publish_part(const SweepArgs &a, int r, int done) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.seg_done + r), "r"(done) : "memory");
}

// Thread 0 of a group: wait until `part` parts of replica r are published.
// Returns 1 when they are; 0 when another group gave up (the status word
// carries PDIT_STATUS_SCHEDULE) or this wait passes its bound, which then
// sets that bit so that every group stops taking work. The bound is 2^26
// polls about 1 us apart (roughly a minute, against parts of at most 1000
// sweeps that last well under a second); it counts polls rather than wall
// time, so a context that the GPU time-slices with others does not run out
// of it while nothing of its own runs.
__device__ __forceinline__ int wait_part(const SweepArgs &a, int r, int part) {
    for (unsigned it = 0;; ++it) {
        if (load_parts_done(a.seg_done + r) >= part) return 1;
        if (*reinterpret_cast<volatile int *>(a.status) & kStatusSchedule) return 0;
        if (it >= (1u << 26)) {
            atomicOr(a.status, kStatusSchedule);
            return 0;
        }
        __nanosleep(1000);
    }
}

// First sweep of part `part` when a launch's range [sweep_begin, sweep_end)
// is split into a.segments parts (one part: the whole range).
__device__ __forceinline__ int part_begin(const SweepArgs &a, int part) {
    const int k = a.segments > 1 ? a.segments : 1;
    return a.sweep_begin + (int)((long long)(a.sweep_end - a.sweep_begin) * part / k);
}

// ---------------------------------------------------------------------------
// One replica: initial state, table build, sweeps [sweep_begin, sweep_end),
// write-back. `T` is the replica's influence table (shared or global memory),
// row stride S; sp = permutation, sh = p-diagonal h[m] = I[m][p(m)],
// sv = scratch (swap energies in j order, then the rank-1 column factor).
// Thread t of the group owns candidates t + G k, k < MAXK, and weights
// t*MAXK .. t*MAXK + MAXK - 1; MAXK is a power of two >= n / G. In table
// updates lane l of each warp owns rows l + 32 k. PK = pending rank-1 terms
// held before the table is rewritten (1 = immediate updates); a swap is one
// term, or two in the general form (ASYM).
// ---------------------------------------------------------------------------
//
// `part`: which part of the launch's sweep range this unit runs when the
// range is split into a.segments parts (see part_begin; 0 with a.segments
// <= 1: the whole range). Later parts resume from the state the previous
// part left (the table included) and publish their own at the end. Tables
// in global memory (TG) are never split: their kernels keep the plain loop
// (the part bookkeeping slowed the N = 256 kernel by 4-6% even where it
// took no parts, for a 2% gain from parts).
template <typename DT, int MAXK, int WPR, int PK, bool TG = false, bool ASYM = false>
__device__ __forceinline__ void run_replica(const SweepArgs &a, int part_arg, int r, int t, int bar,
                                            const DT *sD, const DT *sF, int32_t *T, int32_t *sp,
                                            int32_t *sh, int32_t *sv, uint32_t *upk,
                                            uint32_t *vpk, GroupScratch *gs) {
    constexpr bool PARTS = !TG;
    const int part = PARTS ? part_arg : 0;
    constexpr int G = 32 * WPR;
    constexpr int ROWS = WPR * MAXK;       // table rows per lane in the rank-1 update (32-row slots)
    constexpr int QB = ROWS <= 4 ? 2 : 1;  // table quads per batch of the rank-1 update
    // Tables in global memory (TG): table updates run lanes along a row, so a
    // warp touches 512 contiguous bytes per access; each lane keeps the
    // column factors of its quads lane, lane + 32, ... in registers.
    constexpr int QL = (ROWS + 3) / 4;     // quads per lane along a row (cover / 128)
    constexpr int PW = PK > 1 ? PK / 4 : 1;  // packed words per entry (4 pending terms each)
    const int lane = t & 31;
    const int wg = t >> 5;
    const int n = a.n;
    const int S = a.stride;
    const int npad = (n + 3) & ~3;
    const int dn = ASYM ? a.dstride : n;  // row stride of sD, sF
    const uint32_t grep = a.rep_base + (uint32_t)r;
    int32_t *gp = a.perm + (size_t)r * n;
    int32_t *gbp = a.best_perm + (size_t)r * n;

    const int fresh = part == 0 ? a.fresh : 0;
    // ---- permutation (a resumed state is read through L2: another SM may
    // have written it in the same launch)
    if (fresh) {
        fisher_yates<WPR>(a, grep, n, t, sv, sp, bar);
    } else {
        for (int m = t; m < n; m += G) sp[m] = PARTS ? __ldcg(gp + m) : gp[m];
    }
    group_sync<WPR>(bar);

    // ---- influence table, Eq. 2 in the one-term form I[m][c] = sum_j D[m][j] F[c][p(j)]
    // (F symmetric, so row p(j) of F is read contiguously); general form:
    // both terms of Eq. 2, T[m][c] = sum_j D[m][j] F[c][p(j)] + D[j][m] F[p(j)][c].
    if (part == 0 ? a.table_in : 1) {
        const int32_t *src = a.tables + (size_t)r * n * S;
        if (src != T) {
            const int4 *s4 = reinterpret_cast<const int4 *>(src);
            int4 *d4 = reinterpret_cast<int4 *>(T);
            for (int idx = t; idx < n * S / 4; idx += G) d4[idx] = PARTS ? __ldcg(s4 + idx) : s4[idx];
        }
    } else {
        for (int m = 0; m < n; ++m) {
            const DT *Dm = sD + m * dn;
            for (int c0 = 0; c0 < npad; c0 += G) {
                const int c = c0 + t;
                int acc = 0;
                if (c < n) {
                    if constexpr (ASYM) {
                        for (int j = 0; j < n; ++j) {
                            const int pj = sp[j];
                            acc += (int)Dm[j] * (int)sF[c * dn + pj] + (int)sD[j * dn + m] * (int)sF[pj * dn + c];
                        }
                    } else {
                        for (int j = 0; j < n; ++j) acc += (int)Dm[j] * (int)sF[sp[j] * n + c];
                    }
                }
                if (c < npad) T[m * S + c] = acc;
            }
        }
    }
    group_sync<WPR>(bar);

    // ---- p-diagonal and energy: E = sum_m I[m][p(m)] (Eq. 1 regrouped);
    // general form: the sum is 2 E
    long long esum = 0;
    for (int m = t; m < n; m += G) {
        const int h = T[m * S + sp[m]];
        sh[m] = h;
        esum += h;
    }
    esum = warp_sum(esum);
    if constexpr (WPR > 1) {
        if (lane == 0) gs->wtot[wg] = (unsigned long long)esum;
        group_sync<WPR>(bar);
        esum = 0;
#pragma unroll
        for (int w = 0; w < WPR; ++w) esum += (long long)gs->wtot[w];
    }
    if constexpr (ASYM) esum >>= 1;
    long long E, bestE, acc_moves;
    int bsweep;
    bool reached = false;
    if (fresh) {
        E = esum;
        bestE = esum;
        bsweep = -1;
        acc_moves = 0;
        for (int m = t; m < n; m += G) gbp[m] = sp[m];
        if (t == 0) note_target(a, bestE, -1, reached);
    } else {
        if constexpr (PARTS) {
            E = __ldcg(a.energy + r);
            bestE = __ldcg(a.best_energy + r);
            bsweep = __ldcg(a.best_sweep + r);
            acc_moves = __ldcg(a.accepted + r);
        } else {
            E = a.energy[r];
            bestE = a.best_energy[r];
            bsweep = a.best_sweep[r];
            acc_moves = a.accepted[r];
        }
        if (E != esum && t == 0) atomicOr(a.status, 1);
    }
    group_sync<WPR>(bar);

    // the part's sweeps (its last sweep stays in the group scratch, read at
    // every sweep, rather than in a register across the sweeps)
    const int s_begin = PARTS ? part_begin(a, part) : a.sweep_begin;
    if constexpr (PARTS) {
        if (t == 0) gs->part_end = part >= a.segments - 1 ? a.sweep_end : part_begin(a, part + 1);
        group_sync<WPR>(bar);
    }
    const float beta_fixed = a.sweep_end <= a.sweep_begin ? 0.0f
                           : a.mode == 1 ? a.beta[a.rung[r]] : a.mode == 2 ? a.beta[r] : 0.0f;
    const int zero_diag = a.zero_diag;
    const int nq = npad / 4;

    // Deferred table updates (PK = 4): the influence table is
    //   I = T + sum_{q < np} u_q (x) v_q,  u_q[m] = D[i_q][m] - D[j_q][m],
    //   v_q[c] = F[b_q][c] - F[a_q][c]
    // for the np <= 4 accepted swaps (i_q <-> j_q, facilities a_q, b_q) since
    // the last rewrite of T (general form: two terms per swap, the column
    // term u[m] = D[m][i_q] - D[m][j_q], v[c] = F[c][b_q] - F[c][a_q] and the
    // row term above, so T is rewritten every two swaps). Word w of upk
    // (upk[w * Npad + m]) packs u_{4w}..u_{4w+3}[m] and word w of vpk packs
    // v_{4w}..v_{4w+3}[c] as signed bytes (exact: every |u|, |v| <= 127 for the
    // instances this path is chosen for), so one dp4a per word adds the
    // pending terms of an entry; bytes q >= np are masked off. PK = 4 (one
    // word) for tables in shared memory; PK = 16 (four words) for tables in
    // global memory, where every rewrite streams the whole table through L2.
    // Exact integers throughout.
    int np = 0;
    bool flushed = false;  // the last apply_swap rewrote the table
    if constexpr (PK > 1) {
        for (int c = t; c < PW * npad; c += G) {
            upk[c] = 0u;
            vpk[c] = 0u;
        }
    }

    // T += sum_{q < np} u_q (x) v_q on this thread's (rows, column quads).
    auto flush = [&]() {
        uint32_t mk[PW];
#pragma unroll
        for (int w = 0; w < PW; ++w) mk[w] = pending_mask(np, w);
        const int4 *v4 = reinterpret_cast<const int4 *>(vpk);
        if constexpr (TG) {
            // lanes along a row: a warp touches 512 contiguous bytes per access
            int4 vq[PW == 1 ? QL : 1];
            if constexpr (PW == 1) {
#pragma unroll
                for (int c2 = 0; c2 < QL; ++c2) {
                    const int cq = lane + 32 * c2;
                    vq[c2] = cq < nq ? v4[cq] : make_int4(0, 0, 0, 0);
                }
            }
#pragma unroll 4
            for (int m = wg; m < n; m += WPR) {
                int um[PW];
#pragma unroll
                for (int w = 0; w < PW; ++w) um[w] = (int)(upk[w * npad + m] & mk[w]);
                int4 *row = reinterpret_cast<int4 *>(T + m * S);
#pragma unroll
                for (int c2 = 0; c2 < QL; ++c2) {
                    const int cq = lane + 32 * c2;
                    if (cq < nq) {
                        int4 x = row[cq];
#pragma unroll
                        for (int w = 0; w < PW; ++w) {
                            int4 v;
                            if constexpr (PW == 1)
                                v = vq[c2];
                            else
                                v = v4[w * nq + cq];
                            x.x = __dp4a(um[w], v.x, x.x);
                            x.y = __dp4a(um[w], v.y, x.y);
                            x.z = __dp4a(um[w], v.z, x.z);
                            x.w = __dp4a(um[w], v.w, x.w);
                        }
                        row[cq] = x;
                    }
                }
            }
        } else {
            int uw[ROWS][PW];
#pragma unroll
            for (int k = 0; k < ROWS; ++k) {
                const int m = lane + 32 * k;
#pragma unroll
                for (int w = 0; w < PW; ++w) uw[k][w] = m < n ? (int)(upk[w * npad + m] & mk[w]) : 0;
            }
            for (int cq = wg; cq < nq; cq += WPR) {
                int4 vq[PW];
#pragma unroll
                for (int w = 0; w < PW; ++w) vq[w] = v4[w * nq + cq];
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    if (lane + 32 * k < n) {
                        int4 *row = reinterpret_cast<int4 *>(T + (lane + 32 * k) * S) + cq;
                        int4 x = *row;
#pragma unroll
                        for (int w = 0; w < PW; ++w) {
                            x.x = __dp4a(uw[k][w], vq[w].x, x.x);
                            x.y = __dp4a(uw[k][w], vq[w].y, x.y);
                            x.z = __dp4a(uw[k][w], vq[w].z, x.z);
                            x.w = __dp4a(uw[k][w], vq[w].w, x.w);
                        }
                        *row = x;
                    }
                }
            }
        }
    };

    // Apply the swap i <-> js (facilities fa, fb) to the table (immediately
    // or as a pending packed term), the p-diagonal and the permutation.
    // tib, tja: the current I[i][fb], I[js][fa] (thread 0's values are used).
    // Group-uniform; no barrier at the end.
    auto apply_swap = [&](int i, int js, int fa, int fb, int tib, int tja) {
        const DT *Di = sD + i * dn;
        const DT *Dj = sD + js * dn;
        const DT *Fa = sF + fa * dn;
        const DT *Fb = sF + fb * dn;
        if constexpr (PK == 1) {
            // Immediate rank-1 (general form: rank-2) update: lane l of every
            // warp owns rows l + 32 k; warp w owns column quads w, w + WPR, ...
            int32_t *sv2 = sv + a.v2_off;  // column factor of the general form
            for (int c = t; c < npad; c += G) {
                sv[c] = c < n ? (int)Fb[c] - (int)Fa[c] : 0;
                if constexpr (ASYM) sv2[c] = c < n ? (int)sF[c * dn + fb] - (int)sF[c * dn + fa] : 0;
            }
            if constexpr (TG) {
                group_sync<WPR>(bar);
                int4 vq[QL], wq[ASYM ? QL : 1];
#pragma unroll
                for (int c2 = 0; c2 < QL; ++c2) {
                    const int cq = lane + 32 * c2;
                    vq[c2] = cq < nq ? reinterpret_cast<const int4 *>(sv)[cq] : make_int4(0, 0, 0, 0);
                    if constexpr (ASYM)
                        wq[c2] = cq < nq ? reinterpret_cast<const int4 *>(sv2)[cq] : make_int4(0, 0, 0, 0);
                }
#pragma unroll 2
                for (int m = wg; m < n; m += WPR) {
                    const int um = (int)Di[m] - (int)Dj[m];
                    const int um2 = ASYM ? (int)sD[m * dn + i] - (int)sD[m * dn + js] : 0;
                    int4 *row = reinterpret_cast<int4 *>(T + m * S);
#pragma unroll
                    for (int c2 = 0; c2 < QL; ++c2) {
                        const int cq = lane + 32 * c2;
                        if (cq < nq) {
                            int4 x = row[cq];
                            add_scaled(x, um, vq[c2]);
                            if constexpr (ASYM) add_scaled(x, um2, wq[ASYM ? c2 : 0]);
                            row[cq] = x;
                        }
                    }
                }
            } else {
            int u[ROWS], u2[ASYM ? ROWS : 1];
#pragma unroll
            for (int k = 0; k < ROWS; ++k) {
                const int m = lane + 32 * k;
                u[k] = m < n ? (int)Di[m] - (int)Dj[m] : 0;
                if constexpr (ASYM) u2[k] = m < n ? (int)sD[m * dn + i] - (int)sD[m * dn + js] : 0;
            }
            group_sync<WPR>(bar);
            const int4 *v4 = reinterpret_cast<const int4 *>(sv);
            const int4 *w4 = reinterpret_cast<const int4 *>(sv2);
            int cq = wg;
            for (; cq + (QB - 1) * WPR < nq; cq += QB * WPR) {
                int4 vq[QB], wq[ASYM ? QB : 1];
#pragma unroll
                for (int b = 0; b < QB; ++b) {
                    vq[b] = v4[cq + b * WPR];
                    if constexpr (ASYM) wq[b] = w4[cq + b * WPR];
                }
                int4 x[ROWS][QB];
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    if (lane + 32 * k < n) {
                        const int4 *row = reinterpret_cast<const int4 *>(T + (lane + 32 * k) * S) + cq;
#pragma unroll
                        for (int b = 0; b < QB; ++b) x[k][b] = row[b * WPR];
                    }
                }
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    if (lane + 32 * k < n) {
                        int4 *row = reinterpret_cast<int4 *>(T + (lane + 32 * k) * S) + cq;
#pragma unroll
                        for (int b = 0; b < QB; ++b) {
                            add_scaled(x[k][b], u[k], vq[b]);
                            if constexpr (ASYM) add_scaled(x[k][b], u2[ASYM ? k : 0], wq[ASYM ? b : 0]);
                            row[b * WPR] = x[k][b];
                        }
                    }
                }
            }
            for (; cq < nq; cq += WPR) {
                const int4 vq = v4[cq];
                int4 wq = make_int4(0, 0, 0, 0);
                if constexpr (ASYM) wq = w4[cq];
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    if (lane + 32 * k < n) {
                        int4 *row = reinterpret_cast<int4 *>(T + (lane + 32 * k) * S) + cq;
                        int4 x = *row;
                        add_scaled(x, u[k], vq);
                        if constexpr (ASYM) add_scaled(x, u2[ASYM ? k : 0], wq);
                        *row = x;
                    }
                }
            }
            }
        } else {
            // Deferred: record u and v of this swap in slot np of upk, vpk
            // (general form: the column term in slot np, the row term in np + 1,
            // the same word since np is even then).
            int8_t *ub = reinterpret_cast<int8_t *>(upk + (np >> 2) * npad) + (np & 3);
            int8_t *vb = reinterpret_cast<int8_t *>(vpk + (np >> 2) * npad) + (np & 3);
            for (int c = t; c < npad; c += G) {
                if constexpr (ASYM) {
                    ub[4 * c] = (int8_t)(c < n ? (int)sD[c * dn + i] - (int)sD[c * dn + js] : 0);
                    vb[4 * c] = (int8_t)(c < n ? (int)sF[c * dn + fb] - (int)sF[c * dn + fa] : 0);
                    ub[4 * c + 1] = (int8_t)(c < n ? (int)Di[c] - (int)Dj[c] : 0);
                    vb[4 * c + 1] = (int8_t)(c < n ? (int)Fb[c] - (int)Fa[c] : 0);
                } else {
                    ub[4 * c] = (int8_t)(c < n ? (int)Di[c] - (int)Dj[c] : 0);
                    vb[4 * c] = (int8_t)(c < n ? (int)Fb[c] - (int)Fa[c] : 0);
                }
            }
        }
        // p-diagonal h[m] = I[m][p(m)] under the new influence and
        // permutation: h[m] += u_m v[p(m)] (general form: both terms) where
        // p(m) is unchanged; the two moved entries from the current I[i][fb],
        // I[js][fa]. Thread 0 writes sp[i], sp[js]; those two are not read here.
        for (int m = t; m < n; m += G)
            if (m != i && m != js) {
                const int pm = sp[m];
                int dh = ((int)Di[m] - (int)Dj[m]) * ((int)Fb[pm] - (int)Fa[pm]);
                if constexpr (ASYM)
                    dh += ((int)sD[m * dn + i] - (int)sD[m * dn + js]) *
                          ((int)sF[pm * dn + fb] - (int)sF[pm * dn + fa]);
                sh[m] += dh;
            }
        if (t == 0) {
            sp[i] = fb;
            sp[js] = fa;
            int hi_new = tib + ((int)Di[i] - (int)Dj[i]) * ((int)Fb[fb] - (int)Fa[fb]);
            int hj_new = tja + ((int)Di[js] - (int)Dj[js]) * ((int)Fb[fa] - (int)Fa[fa]);
            if constexpr (ASYM) {
                hi_new += ((int)Di[i] - (int)Di[js]) * ((int)sF[fb * dn + fb] - (int)sF[fb * dn + fa]);
                hj_new += ((int)Dj[i] - (int)Dj[js]) * ((int)sF[fa * dn + fb] - (int)sF[fa * dn + fa]);
            }
            sh[i] = hi_new;
            sh[js] = hj_new;
        }
        if constexpr (PK > 1) {
            np += ASYM ? 2 : 1;
            flushed = np == PK;
            if (np == PK) {
                group_sync<WPR>(bar);  // packed factors and thread 0's table reads complete
                flush();
                np = 0;
            }
        }
    };

    // Tables in global memory: the gathers of the next update (its row
    // T[l][p(j)] and column T[j][p(l)] for this thread's candidates) are
    // loaded one update ahead, so their latency overlaps the current update.
    // Between rewrites the global table does not change (pending terms are
    // added from shared memory when the values are used), so a prefetch
    // stays valid unless the table was rewritten or the swap changed p(l) or
    // a candidate's p(j); those cases are reloaded after the swap.
    int pre_row[TG ? MAXK : 1], pre_col[TG ? MAXK : 1];
    auto prefetch = [&](int l) {
        if constexpr (TG) {
            const int pl = sp[l];
#pragma unroll
            for (int k = 0; k < MAXK; ++k) {
                const int j = t + G * k;
                if (j < n) {
                    pre_row[k] = T[l * S + sp[j]];
                    pre_col[k] = T[j * S + pl];
                }
            }
        }
    };
    // One candidate per thread (MAXK = 1): thread t owns location t and keeps
    // p(t), h(t) and its packed u factors in registers for the gathers;
    // shared memory stays the copy that is written (and that other threads
    // read), and the owner refreshes its registers after every swap.
    constexpr bool OWN = MAXK == 1;
    int myp = 0, myh = 0;
    uint32_t myu[PW];
#pragma unroll
    for (int w = 0; w < PW; ++w) myu[w] = 0u;
    auto refresh_own = [&]() {
        if constexpr (OWN) {
            if (t < n) {
                myp = sp[t];
                myh = sh[t];
                if constexpr (PK > 1) {
#pragma unroll
                    for (int w = 0; w < PW; ++w) myu[w] = upk[w * npad + t];
                }
            }
        }
    };
    refresh_own();
    int32_t *srow = sv + a.rc_off;  // TG: gathered row values T[i][p(j)] by j, then the column values
    int32_t *scol = srow + npad;
    if constexpr (TG) {
        if (a.mode != 3 && a.sweep_begin < a.sweep_end) prefetch(0);
    }

    // (an if-constexpr function: a conditional expression with the volatile
    // read in its untaken arm changed the global-table kernels' register
    // allocation and cost them 4-9%)
    auto sweep_end_now = [&]() {
        if constexpr (PARTS)
            return *reinterpret_cast<volatile const int *>(&gs->part_end);
        else
            return a.sweep_end;
    };
    for (int s = s_begin; s < sweep_end_now(); ++s) {
        if (a.stop) {
            // group-uniform decision from one read of the instance's flag
            if (t == 0) gs->stop = *reinterpret_cast<volatile int *>(a.done);
            group_sync<WPR>(bar);
            const int stop_now = gs->stop;
            group_sync<WPR>(bar);
            if (stop_now) break;
        }
        const float beta = (a.mode == 1 || a.mode == 2) ? beta_fixed : a.beta[s];
        if (a.mode == 3) {
            // ---- concurrent updates (one iteration): proposals drawn from a
            // snapshot of the swap energies, ranked by energy change (ties to
            // the lower location), greedily accepted when both locations are
            // free, applied in that order with their exact energy changes.
            int32_t *pj = sv + a.cupim_off;  // proposal of each location
            int32_t *pd = pj + npad;          // its snapshot energy change; later: taken flags
            int32_t *ord = pd + npad;         // movers in priority order; then the accepted ones
            uint32_t pm[PW];
#pragma unroll
            for (int w = 0; w < PW; ++w) pm[w] = pending_mask(np, w);
            // A. warp wg draws the proposals of locations wg, wg + WPR, ...
            for (int ib = wg; ib < n; ib += 32 * WPR) {
                const int myrow = ib + WPR * lane;
                const uint4 rw = philox4x32_10(a.inst, grep, (uint32_t)s, (uint32_t)myrow, a.key0, a.key1);
                const int nrows = min(32, (n - ib + WPR - 1) / WPR);
                for (int q = 0; q < nrows; ++q) {
                    const int i = ib + WPR * q;
                    const unsigned long long draw =
                        ((unsigned long long)__shfl_sync(kFull, rw.y, q) << 32) |
                        (unsigned long long)__shfl_sync(kFull, rw.x, q);
                    const int fa = sp[i];
                    const int hi = sh[i];
                    const DT *Di = sD + i * dn;
                    const DT *Fa = sF + fa * dn;
                    int ui[PW], vfa[PW];
                    if constexpr (PK > 1) {
#pragma unroll
                        for (int w = 0; w < PW; ++w) {
                            ui[w] = (int)(upk[w * npad + i] & pm[w]);
                            vfa[w] = (int)vpk[w * npad + fa];
                        }
                    }
                    int dv[ROWS];
                    int lmin = 0x7FFFFFFF;
#pragma unroll
                    for (int k = 0; k < ROWS; ++k) {
                        const int j = lane + 32 * k;
                        int d = 0x7FFFFFFF;
                        if (j < n) {
                            const int b = sp[j];
                            const int dij = Di[j];
                            const int fab = Fa[b];
                            int row_ib = T[i * S + b];
                            int col_ja = T[j * S + fa];
                            if constexpr (PK > 1) {
#pragma unroll
                                for (int w = 0; w < PW; ++w) {
                                    row_ib = __dp4a(ui[w], (int)vpk[w * npad + b], row_ib);
                                    col_ja = __dp4a((int)(upk[w * npad + j] & pm[w]), vfa[w], col_ja);
                                }
                            }
                            if constexpr (ASYM) {
                                const int dji = sD[j * dn + i];
                                const int fba = sF[b * dn + fa];
                                d = row_ib - hi + col_ja - sh[j];
                                if (zero_diag)
                                    d += (dij + dji) * (fab + fba);
                                else
                                    d += ((int)Di[i] + (int)sD[j * dn + j] - dij - dji) *
                                         ((int)Fa[fa] + (int)sF[b * dn + b] - fab - fba);
                            } else {
                                d = 2 * (row_ib - hi + col_ja - sh[j]);
                                if (zero_diag)
                                    d += 4 * dij * fab;
                                else
                                    d += ((int)Di[i] + (int)sD[j * n + j] - 2 * dij) *
                                         ((int)Fa[fa] + (int)sF[b * n + b] - 2 * fab);
                            }
                            if (j == i) d = 0;
                            lmin = min(lmin, d);
                        }
                        dv[k] = d;
                    }
                    const int dmin = __reduce_min_sync(kFull, lmin);
                    unsigned long long incl[ROWS], tot[ROWS];
#pragma unroll
                    for (int k = 0; k < ROWS; ++k)
                        incl[k] = (lane + 32 * k < n) ? eq5_weight(dv[k] - dmin, beta) : 0ull;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                        for (int k = 0; k < ROWS; ++k) {
                            const unsigned long long y = __shfl_up_sync(kFull, incl[k], o);
                            if (lane >= o) incl[k] += y;
                        }
                    }
                    unsigned long long total = 0;
#pragma unroll
                    for (int k = 0; k < ROWS; ++k) {
                        tot[k] = __shfl_sync(kFull, incl[k], 31);
                        total += tot[k];
                    }
                    const unsigned long long tdraw = __umul64hi(draw, total);
                    int js = i, dsel = 0;
                    unsigned long long off = 0;
                    bool found = false;
#pragma unroll
                    for (int k = 0; k < ROWS; ++k) {
                        if (!found && tdraw < off + tot[k]) {  // uniform across the warp
                            const unsigned ball = __ballot_sync(kFull, off + incl[k] > tdraw);
                            const int src = __ffs(ball) - 1;
                            js = 32 * k + src;
                            dsel = __shfl_sync(kFull, dv[k], src);
                            found = true;
                        }
                        off += tot[k];
                    }
                    if (lane == 0) {
                        pj[i] = js;
                        pd[i] = dsel;
                    }
                }
            }
            group_sync<WPR>(bar);
            // B. priority rank of every mover
            for (int m = t; m < n; m += G) {
                const int jm = pj[m];
                if (jm != m) {
                    const int dm = pd[m];
                    int rank = 0;
                    for (int x = 0; x < n; ++x) {
                        const int jx = pj[x], dx = pd[x];
                        rank += (jx != x) && (dx < dm || (dx == dm && x < m));
                    }
                    ord[rank] = m;
                }
            }
            group_sync<WPR>(bar);
            // C. greedy matching in priority order (one thread)
            if (t == 0) {
                int movers = 0;
                for (int x = 0; x < n; ++x) movers += pj[x] != x;
                for (int x = 0; x < n; ++x) pd[x] = 0;
                int K = 0;
                for (int q = 0; q < movers; ++q) {
                    const int i = ord[q], j = pj[i];
                    if (!pd[i] && !pd[j]) {
                        pd[i] = 1;
                        pd[j] = 1;
                        ord[K++] = i;
                    }
                }
                gs->cnt = K;
            }
            group_sync<WPR>(bar);
            const int K = gs->cnt;
            // D. apply the accepted swaps in order, each with its exact energy change
            for (int q = 0; q < K; ++q) {
                const int i = ord[q];
                const int js = pj[i];
                const int fa = sp[i], fb = sp[js];
                if (t == 0) {
                    int rowv = T[i * S + fb];
                    int colv = T[js * S + fa];
                    if constexpr (PK > 1) {
#pragma unroll
                        for (int w = 0; w < PW; ++w) {
                            const uint32_t m4 = pending_mask(np, w);
                            rowv = __dp4a((int)(upk[w * npad + i] & m4), (int)vpk[w * npad + fb], rowv);
                            colv = __dp4a((int)(upk[w * npad + js] & m4), (int)vpk[w * npad + fa], colv);
                        }
                    }
                    const int dij = sD[i * dn + js];
                    const int fab = sF[fa * dn + fb];
                    int d;
                    if constexpr (ASYM) {
                        const int dji = sD[js * dn + i];
                        const int fba = sF[fb * dn + fa];
                        d = rowv - sh[i] + colv - sh[js];
                        if (zero_diag)
                            d += (dij + dji) * (fab + fba);
                        else
                            d += ((int)sD[i * dn + i] + (int)sD[js * dn + js] - dij - dji) *
                                 ((int)sF[fa * dn + fa] + (int)sF[fb * dn + fb] - fab - fba);
                    } else {
                        d = 2 * (rowv - sh[i] + colv - sh[js]);
                        if (zero_diag)
                            d += 4 * dij * fab;
                        else
                            d += ((int)sD[i * n + i] + (int)sD[js * n + js] - 2 * dij) *
                                 ((int)sF[fa * n + fa] + (int)sF[fb * n + fb] - 2 * fab);
                    }
                    gs->sel_d = d;
                    gs->aux0 = rowv;
                    gs->aux1 = colv;
                }
                group_sync<WPR>(bar);
                const int dstar = gs->sel_d;
                apply_swap(i, js, fa, fb, gs->aux0, gs->aux1);
                E += dstar;
                acc_moves += 1;
                group_sync<WPR>(bar);
            }
            // E. best-so-far after the iteration
            if (E < bestE) {
                bestE = E;
                bsweep = s;
                for (int m = t; m < n; m += G) gbp[m] = sp[m];
                if (t == 0) note_target(a, bestE, s, reached);
            }
            group_sync<WPR>(bar);
            continue;
        }
        for (int i0 = 0; i0 < n; i0 += 32) {
            // Philox(inst, replica, sweep, location) for the next 32 locations.
            const uint4 rw = philox4x32_10(a.inst, grep, (uint32_t)s, (uint32_t)(i0 + lane), a.key0, a.key1);
            const int cnt = min(32, n - i0);
            for (int ii = 0; ii < cnt; ++ii) {
                const int i = i0 + ii;
                const unsigned long long draw =
                    ((unsigned long long)__shfl_sync(kFull, rw.y, ii) << 32) |
                    (unsigned long long)__shfl_sync(kFull, rw.x, ii);
                const int fa = sp[i];
                const int hi = sh[i];
                const DT *Di = sD + i * dn;
                const DT *Fa = sF + fa * dn;
                // pending factors at this location: packed u_q[i] and v_q[fa]
                uint32_t pm[PW];
                int ui[PW], vfa[PW];
                if constexpr (PK > 1) {
#pragma unroll
                    for (int w = 0; w < PW; ++w) {
                        pm[w] = pending_mask(np, w);
                        ui[w] = (int)(upk[w * npad + i] & pm[w]);
                        vfa[w] = (int)vpk[w * npad + fa];
                    }
                }

                // ---- gather: Eq. 3 for every candidate j
                int lmin = 0x7FFFFFFF;
                int dself = 0;  // MAXK = 1: this thread's energy, handed to the draw in a register
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int j = t + G * k;
                    if (j < n) {
                        const int b = OWN ? myp : sp[j];
                        const int hj = OWN ? myh : sh[j];
                        const int dij = Di[j];
                        const int fab = Fa[b];
                        int row_ib, col_ja;
                        if constexpr (TG) {
                            row_ib = pre_row[k];
                            col_ja = pre_col[k];
                        } else {
                            row_ib = T[i * S + b];
                            col_ja = T[j * S + fa];
                        }
                        if constexpr (PK > 1) {
#pragma unroll
                            for (int w = 0; w < PW; ++w) {
                                const uint32_t uj = OWN ? myu[w] : upk[w * npad + j];
                                row_ib = __dp4a(ui[w], (int)vpk[w * npad + b], row_ib);
                                col_ja = __dp4a((int)(uj & pm[w]), vfa[w], col_ja);
                            }
                        }
                        if constexpr (TG) {
                            srow[j] = row_ib;
                            scol[j] = col_ja;
                        }
                        int d;
                        if constexpr (ASYM) {
                            const int dji = sD[j * dn + i];
                            const int fba = sF[b * dn + fa];
                            d = row_ib - hi + col_ja - hj;
                            if (zero_diag)
                                d += (dij + dji) * (fab + fba);
                            else
                                d += ((int)Di[i] + (int)sD[j * dn + j] - dij - dji) *
                                     ((int)Fa[fa] + (int)sF[b * dn + b] - fab - fba);
                        } else {
                            d = 2 * (row_ib - hi + col_ja - hj);
                            if (zero_diag)
                                d += 4 * dij * fab;
                            else
                                d += ((int)Di[i] + (int)sD[j * n + j] - 2 * dij) *
                                     ((int)Fa[fa] + (int)sF[b * n + b] - 2 * fab);
                        }
                        if (j == i) d = 0;
                        if constexpr (MAXK > 1)
                            sv[j] = d;
                        else
                            dself = d;
                        lmin = min(lmin, d);
                    }
                }
                const int nxt = i + 1 < n ? i + 1 : 0;  // the next update's location
                if constexpr (TG) prefetch(nxt);
                const int3 sel = eq5_draw<MAXK, WPR>(sv, sp, n, t, lmin, dself, myp, beta, draw, bar, gs);
                const int js = sel.x, dstar = sel.y;
                if (js == i) continue;

                // ---- apply the swap i <-> js
                const int fb = sel.z;  // sp[js], read before thread 0 rewrites it
                // current I[i][fb] and I[js][fa], for the two p-diagonal entries that move
                int tib = 0, tja = 0;
                if (t == 0) {
                    if constexpr (TG) {
                        tib = srow[js];  // gathered with the pending terms
                        tja = scol[js];
                    } else {
                        tib = T[i * S + fb];
                        tja = T[js * S + fa];
                        if constexpr (PK > 1) {
#pragma unroll
                            for (int w = 0; w < PW; ++w) {
                                tib = __dp4a(ui[w], (int)vpk[w * npad + fb], tib);
                                tja = __dp4a((int)(upk[w * npad + js] & pm[w]), vfa[w], tja);
                            }
                        }
                    }
                }
                apply_swap(i, js, fa, fb, tib, tja);
                E += dstar;
                acc_moves += 1;
                if (E < bestE) {
                    bestE = E;
                    bsweep = s;
                    for (int m = t; m < n; m += G) gbp[m] = m == i ? fb : (m == js ? fa : sp[m]);
                    if (t == 0) note_target(a, bestE, s, reached);
                }
                group_sync<WPR>(bar);
                refresh_own();
                if constexpr (TG) {
                    // the swap moved p(i) and p(js); a rewrite changed the table
                    if (PK == 1 || flushed || js == nxt) {
                        prefetch(nxt);
                    } else {
#pragma unroll
                        for (int k = 0; k < MAXK; ++k) {
                            const int j = t + G * k;
                            if (j == i || j == js) pre_row[k] = T[nxt * S + sp[j]];
                        }
                    }
                }
            }
        }
    }
    if constexpr (PK > 1) {
        if (np > 0) {
            flush();
            np = 0;
            group_sync<WPR>(bar);
        }
    }

    // ---- write back
    for (int m = t; m < n; m += G) gp[m] = sp[m];
    if (t == 0) {
        a.energy[r] = E;
        a.best_energy[r] = bestE;
        a.best_sweep[r] = bsweep;
        a.accepted[r] = acc_moves;
    }
    const bool last_part = !PARTS || part >= a.segments - 1;
    if (last_part ? a.table_out : 1) {
        int32_t *dst = a.tables + (size_t)r * n * S;
        if (dst != T) {
            const int4 *s4 = reinterpret_cast<const int4 *>(T);
            int4 *d4 = reinterpret_cast<int4 *>(dst);
            for (int idx = t; idx < n * S / 4; idx += G) d4[idx] = s4[idx];
        }
    }
    if (a.dump && last_part) {
        int32_t *dst = a.dump + (size_t)r * n * n;
        for (int idx = t; idx < n * n; idx += G) dst[idx] = T[(idx / n) * S + idx % n];
    }
    // a launch split into parts: publish this part once every thread's
    // writes of the replica's state are visible device-wide
    const bool publish = PARTS && a.segments > 1;
    if (publish) __threadfence();
    group_sync<WPR>(bar);
    if (publish && t == 0) publish_part(a, r, part + 1);
}

// Largest CTA each instantiation is compiled for; it caps the registers per
// thread at 65536 / bound, so it is set per shape from its register needs.
__host__ __device__ constexpr int sweep_bound(int maxk, int wpr) {
    return wpr == 1 ? (maxk == 1 ? 1024 : maxk == 2 ? 512 : maxk == 4 ? 384 : 128)
         : wpr == 2 ? (maxk == 1 ? 1024 : maxk == 2 ? 512 : 384)
         : wpr == 4 ? (maxk == 1 ? 640 : 512)
         : 512;
}

template <int MAXK, int WPR>
struct SweepBounds {
    static constexpr int threads = sweep_bound(MAXK, WPR);
};

// Stage D and F (global int32, n x n) as DT in shared memory with row stride
// ds (n, or the odd-word stride of the general form).
template <typename DT, bool ASYM>
__device__ __forceinline__ void stage_df(const int32_t *D, const int32_t *F, int n, int ds, DT *sD, DT *sF) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        int o = idx;
        if constexpr (ASYM) {
            const int m = idx / n;
            o = m * ds + (idx - m * n);
        }
        sD[o] = static_cast<DT>(D[idx]);
        sF[o] = static_cast<DT>(F[idx]);
    }
}

template <typename DT, int MAXK, int WPR, bool TSMEM, int PK, bool ASYM>
__global__ void __launch_bounds__(SweepBounds<MAXK, WPR>::threads) sweep_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int G = 32 * WPR;
    const int n = a.n;
    const int ds = ASYM ? a.dstride : n;
    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int bar = 1 + grp;  // named barrier of this group (WPR > 1); 0 is __syncthreads
    DT *sD = reinterpret_cast<DT *>(smem);
    DT *sF = sD + n * ds;
    stage_df<DT, ASYM>(a.D, a.F, n, ds, sD, sF);
    __syncthreads();
    unsigned char *gb = smem + a.df_bytes + (size_t)grp * a.group_bytes;
    const int npad = (n + 3) & ~3;
    GroupScratch *gs = reinterpret_cast<GroupScratch *>(gb);
    unsigned char *body = gb + kScratchBytes;
    int32_t *sT = reinterpret_cast<int32_t *>(body);
    int32_t *sp = reinterpret_cast<int32_t *>(body + (TSMEM ? (size_t)n * a.stride * 4 : 0));
    int32_t *sh = sp + npad;
    int32_t *sv = sh + npad;
    uint32_t *upk = reinterpret_cast<uint32_t *>(sv + a.sv_len);  // [PK / 4][npad], PK > 1 only
    uint32_t *vpk = upk + (PK / 4) * npad;
    if constexpr (!TSMEM) {
        // tables in global memory: one unit per replica, the whole call
        for (;;) {
            if (t == 0) gs->item = atomicAdd(a.queue, 1);
            group_sync<WPR>(bar);
            const int item = gs->item;
            if (item >= a.replicas) break;
            run_replica<DT, MAXK, WPR, PK, true, ASYM>(a, 0, item, t, bar, sD, sF,
                                                       a.tables + (size_t)item * n * a.stride, sp, sh, sv, upk,
                                                       vpk, gs);
        }
        return;
    }
    // Work units in order: part k of every replica, then part k + 1 (one
    // part: one unit per replica). Part k of replica r starts once part k - 1
    // is published; that part was taken `replicas` units earlier by a group
    // that is running, so the wait ends (it is bounded all the same).
    const int K = a.segments > 1 ? a.segments : 1;
    const long long units = (long long)a.replicas * K;
    for (;;) {
        if (t == 0) {
            const int item = atomicAdd(a.queue, 1);
            int go = item < units ? 1 : 0, part = 0, r = item;
            if (go && K > 1) {
                part = item / a.replicas;
                r = item - part * a.replicas;
                if (part > 0) go = wait_part(a, r, part);
            }
            gs->item = r;
            gs->sel_jf = part;
            gs->stop = go;
        }
        group_sync<WPR>(bar);
        const int go = gs->stop, r = gs->item, part = gs->sel_jf;
        group_sync<WPR>(bar);  // the scratch words are reused by the update
        if (!go) break;
        run_replica<DT, MAXK, WPR, PK, false, ASYM>(a, part, r, t, bar, sD, sF, sT, sp, sh, sv, upk, vpk, gs);
    }
}

// One unit of a multi-instance launch: replicas r0 .. r0 + groups - 1 of
// one instance, run by the groups of one CTA.
struct BatchUnit {
    int inst;
    int r0;
};

// Persistent multi-instance kernel: CTAs take units from `queue`; D and F are
// restaged when the CTA moves to another instance. Every instance of a launch
// shares the compiled shape (DT, MAXK, WPR, TSMEM, PK).
template <typename DT, int MAXK, int WPR, bool TSMEM, int PK, bool ASYM>
__global__ void __launch_bounds__(SweepBounds<MAXK, WPR>::threads)
    batch_kernel(const SweepArgs *__restrict__ descs, const BatchUnit *__restrict__ units, int nunits,
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
            // descriptor and matrices of the new instance
            const int *src = reinterpret_cast<const int *>(descs + bu.inst);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int w = threadIdx.x; w < (int)(sizeof(SweepArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
            const int n = descs[bu.inst].n;
            const int ds = ASYM ? descs[bu.inst].dstride : n;
            const int32_t *D = descs[bu.inst].D, *F = descs[bu.inst].F;
            DT *sD = reinterpret_cast<DT *>(smem);
            stage_df<DT, ASYM>(D, F, n, ds, sD, sD + n * ds);
            cur = bu.inst;
        }
        __syncthreads();
        const int n = sa.n;
        const int r = bu.r0 + grp;
        if (grp < sa.groups && r < sa.replicas) {
            const DT *sD = reinterpret_cast<const DT *>(smem);
            const DT *sF = sD + n * (ASYM ? sa.dstride : n);
            unsigned char *gb = smem + sa.df_bytes + (size_t)grp * sa.group_bytes;
            const int npad = (n + 3) & ~3;
            GroupScratch *gs = reinterpret_cast<GroupScratch *>(gb);
            unsigned char *body = gb + kScratchBytes;
            int32_t *sT = reinterpret_cast<int32_t *>(body);
            int32_t *sp = reinterpret_cast<int32_t *>(body + (TSMEM ? (size_t)n * sa.stride * 4 : 0));
            int32_t *sh = sp + npad;
            int32_t *sv = sh + npad;
            uint32_t *upk = reinterpret_cast<uint32_t *>(sv + sa.sv_len);
            uint32_t *vpk = upk + (PK / 4) * npad;
            int32_t *T = TSMEM ? sT : sa.tables + (size_t)r * n * sa.stride;
            run_replica<DT, MAXK, WPR, PK, !TSMEM, ASYM>(sa, 0, r, t, bar, sD, sF, T, sp, sh, sv, upk, vpk, gs);
        }
    }
}

// Host-side entry points, one per storage type of D and F and form
// (symmetric / general), defined in pdit_sweep_i8.cu, pdit_sweep_i16.cu,
// pdit_sweep_i32.cu and their pdit_sweep_gen_*.cu counterparts. Return a
// cudaError_t value; cudaErrorInvalidValue for a shape with no kernel.
template <typename DT, bool ASYM>
int sweep_blocks_per_sm(int maxk, int wpr, bool tsmem, int pk, int threads, size_t smem, int *blocks);
template <typename DT, bool ASYM>
int sweep_launch(int maxk, int wpr, bool tsmem, int pk, const SweepArgs &a, int grid, int threads,
                 size_t smem, cudaStream_t stream);
template <typename DT, bool ASYM>
int batch_blocks_per_sm(int maxk, int wpr, bool tsmem, int pk, int threads, size_t smem, int *blocks);
template <typename DT, bool ASYM>
int batch_launch(int maxk, int wpr, bool tsmem, int pk, const SweepArgs *descs, const BatchUnit *units,
                 int nunits, int *queue, int grid, int threads, size_t smem, cudaStream_t stream);

// Shapes with a compiled kernel: (MAXK, WPR) with 32 * WPR * MAXK in
// {32, 64, 128, 256}; the global-table variant only for 256; 16 pending
// terms only with global tables.
#define PDIT_SWEEP_SHAPES_COMMON(X)                                                              \
    X(1, 1, true, 1) X(2, 1, true, 1) X(1, 2, true, 1) X(4, 1, true, 1) X(2, 2, true, 1)         \
    X(1, 4, true, 1) X(8, 1, true, 1) X(4, 2, true, 1) X(2, 4, true, 1) X(1, 8, true, 1)         \
    X(8, 1, false, 1) X(4, 2, false, 1) X(2, 4, false, 1) X(1, 8, false, 1)
#define PDIT_SWEEP_SHAPES_DEFERRED(X)                                                            \
    X(1, 1, true, 4) X(2, 1, true, 4) X(1, 2, true, 4) X(4, 1, true, 4) X(2, 2, true, 4)         \
    X(1, 4, true, 4) X(8, 1, true, 4) X(4, 2, true, 4) X(2, 4, true, 4) X(1, 8, true, 4)         \
    X(8, 1, false, 4) X(4, 2, false, 4) X(2, 4, false, 4) X(1, 8, false, 4)                      \
    X(8, 1, false, 16) X(4, 2, false, 16) X(2, 4, false, 16) X(1, 8, false, 16)

#define PDIT_INSTANTIATE_SWEEP(DT, ASYM, SHAPES)                                                          \
    template <int MAXK, int WPR, bool TSMEM, int PK>                                                      \
    static int sweep_one(const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t st,         \
                         int *blocks, bool query) {                                                       \
        auto fn = sweep_kernel<DT, MAXK, WPR, TSMEM, PK, ASYM>;                                           \
        if (threads > SweepBounds<MAXK, WPR>::threads) return (int)cudaErrorInvalidValue;                 \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return (int)e;                                                              \
        if (query) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);  \
        fn<<<grid, threads, smem, st>>>(a);                                                               \
        return (int)cudaGetLastError();                                                                   \
    }                                                                                                     \
    static int sweep_dispatch(int maxk, int wpr, bool tsmem, int pk, const SweepArgs &a, int grid,        \
                              int threads, size_t smem, cudaStream_t st, int *blocks, bool query) {       \
        SHAPES(PDIT_CASE)                                                                                 \
        return (int)cudaErrorInvalidValue;                                                                \
    }                                                                                                     \
    template <>                                                                                           \
    int sweep_blocks_per_sm<DT, ASYM>(int maxk, int wpr, bool tsmem, int pk, int threads, size_t smem,    \
                                      int *blocks) {                                                      \
        SweepArgs dummy{};                                                                                \
        return sweep_dispatch(maxk, wpr, tsmem, pk, dummy, 0, threads, smem, nullptr, blocks, true);      \
    }                                                                                                     \
    template <>                                                                                           \
    int sweep_launch<DT, ASYM>(int maxk, int wpr, bool tsmem, int pk, const SweepArgs &a, int grid,       \
                               int threads, size_t smem, cudaStream_t st) {                               \
        return sweep_dispatch(maxk, wpr, tsmem, pk, a, grid, threads, smem, st, nullptr, false);          \
    }                                                                                                     \
    template <int MAXK, int WPR, bool TSMEM, int PK>                                                      \
    static int batch_one(const SweepArgs *d, const BatchUnit *u, int nu, int *q, int grid, int threads,   \
                         size_t smem, cudaStream_t st, int *blocks, bool query) {                         \
        auto fn = batch_kernel<DT, MAXK, WPR, TSMEM, PK, ASYM>;                                           \
        if (threads > SweepBounds<MAXK, WPR>::threads) return (int)cudaErrorInvalidValue;                 \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return (int)e;                                                              \
        if (query) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);  \
        fn<<<grid, threads, smem, st>>>(d, u, nu, q);                                                     \
        return (int)cudaGetLastError();                                                                   \
    }                                                                                                     \
    static int batch_dispatch(int maxk, int wpr, bool tsmem, int pk, const SweepArgs *d,                  \
                              const BatchUnit *u, int nu, int *q, int grid, int threads, size_t smem,     \
                              cudaStream_t st, int *blocks, bool query) {                                 \
        SHAPES(PDIT_BATCH_CASE)                                                                           \
        return (int)cudaErrorInvalidValue;                                                                \
    }                                                                                                     \
    template <>                                                                                           \
    int batch_blocks_per_sm<DT, ASYM>(int maxk, int wpr, bool tsmem, int pk, int threads, size_t smem,    \
                                      int *blocks) {                                                      \
        return batch_dispatch(maxk, wpr, tsmem, pk, nullptr, nullptr, 0, nullptr, 0, threads, smem,       \
                              nullptr, blocks, true);                                                     \
    }                                                                                                     \
    template <>                                                                                           \
    int batch_launch<DT, ASYM>(int maxk, int wpr, bool tsmem, int pk, const SweepArgs *d,                 \
                               const BatchUnit *u, int nu, int *q, int grid, int threads, size_t smem,    \
                               cudaStream_t st) {                                                         \
        return batch_dispatch(maxk, wpr, tsmem, pk, d, u, nu, q, grid, threads, smem, st, nullptr,        \
                              false);                                                                     \
    }

#define PDIT_CASE(MK, W, TS, K)                                                                  \
    if (maxk == MK && wpr == W && tsmem == TS && pk == K)                                        \
        return sweep_one<MK, W, TS, K>(a, grid, threads, smem, st, blocks, query);
#define PDIT_BATCH_CASE(MK, W, TS, K)                                                            \
    if (maxk == MK && wpr == W && tsmem == TS && pk == K)                                        \
        return batch_one<MK, W, TS, K>(d, u, nu, q, grid, threads, smem, st, blocks, query);

#define PDIT_SWEEP_SHAPES_ALL(X) PDIT_SWEEP_SHAPES_COMMON(X) PDIT_SWEEP_SHAPES_DEFERRED(X)

// Flow-class sweep kernels (pdit_class.cu): one per storage type of D and
// per (MAXK, WPR) with 32 * WPR * MAXK in {32, 64, 128, 256}. Return a
// cudaError_t value; cudaErrorInvalidValue for a shape with no kernel.
template <typename DT>
int class_blocks_per_sm(int maxk, int wpr, int threads, size_t smem, int *blocks);
template <typename DT>
int class_launch(int maxk, int wpr, const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t stream);
__host__ __device__ constexpr int class_bound(int maxk, int wpr) {
    return maxk >= 4 ? 512 : 1024;
}

// Dot-product sweep kernels (pdit_dot.cu): symmetric instances with every
// entry of D and F in a signed byte; no influence table, a permuted copy of F
// per replica (see that file). Shapes (MAXK, WPR) listed there. Return a
// cudaError_t value; cudaErrorInvalidValue for a shape with no kernel.
__host__ __device__ constexpr int dot_bound(int maxk, int wpr) {
    return maxk == 1 ? (wpr == 1 ? 768 : 512) : maxk <= 4 ? 512 : 384;
}
bool dot_shape_compiled(int maxk, int wpr);
int dot_blocks_per_sm(int maxk, int wpr, int stride, int threads, size_t smem, int *blocks);
int dot_launch(int maxk, int wpr, const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t stream);
int dot_batch_blocks_per_sm(int maxk, int wpr, int threads, size_t smem, int *blocks);
int dot_batch_launch(int maxk, int wpr, const SweepArgs *descs, const BatchUnit *units, int nunits, int *queue,
                     int grid, int threads, size_t smem, cudaStream_t stream);

}  // namespace pdit
