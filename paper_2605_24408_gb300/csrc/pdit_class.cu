// Flow-class sweep: the annealed p-dit sweep for instances whose flow takes
// two values in the pattern of the Methods section's tai256c paragraph.
//
// For D symmetric with a zero diagonal and F[c][d] = f0 + f x_c x_d off the
// diagonal (x_c in {0, 1}; F's diagonal meets only D's zero diagonal), the
// energy depends on the permutation only through the set S of locations whose
// facility has x = 1:
//   E = f0 sum_{i != j} D_ij + f sum_{u in S} G_u,   G_m = sum_{j in S} D_mj.
// Swapping two facilities of the same class leaves S, hence E, unchanged
// (dE = 0, the first symmetry the paper names). A swap that moves class 1 from
// location u to location w (u in S, w not in S) changes E by
//   dE = 2 f (G_w - G_u - D_uw),
// the same for every such pair of facilities (the second symmetry), and after
// it G_m += D_mw - D_mu. These are Eq. 3's exact values, so every Eq. 5 draw
// and the whole trajectory equal those of the table kernels; the N x N
// influence table becomes the vector G and an accepted swap costs O(N).
#include "pdit_sweep.cuh"

namespace pdit {

template <typename DT, int MAXK, int WPR>
__device__ __forceinline__ void run_class_replica(const SweepArgs &a, int r, int t, int bar, const DT *sD,
                                                  const uint8_t *sx, int32_t *sp, int32_t *sG, int32_t *sv,
                                                  GroupScratch *gs) {
    constexpr int G = 32 * WPR;
    const int lane = t & 31;
    const int wg = t >> 5;
    const int n = a.n;
    const int npad = (n + 3) & ~3;
    const uint32_t grep = a.rep_base + (uint32_t)r;
    int32_t *gp = a.perm + (size_t)r * n;
    int32_t *gbp = a.best_perm + (size_t)r * n;
    const int f2 = 2 * a.cls_f;

    if (a.fresh) {
        fisher_yates<WPR>(a, grep, n, t, sv, sp, bar);
    } else {
        for (int m = t; m < n; m += G) sp[m] = gp[m];
    }
    group_sync<WPR>(bar);

    // ---- G from the permutation, or the saved vector (parallel tempering segments)
    if (a.table_in) {
        for (int m = t; m < n; m += G) sG[m] = a.tables[(size_t)r * npad + m];
    } else {
        for (int m = t; m < n; m += G) {
            const DT *Dm = sD + m * n;
            int acc = 0;
            for (int j = 0; j < n; ++j) acc += sx[sp[j]] ? (int)Dm[j] : 0;
            sG[m] = acc;
        }
    }
    group_sync<WPR>(bar);

    // ---- energy: E = e0 + f sum_{m in S} G_m
    long long esum = 0;
    for (int m = t; m < n; m += G)
        if (sx[sp[m]]) esum += sG[m];
    esum = warp_sum(esum);
    if constexpr (WPR > 1) {
        if (lane == 0) gs->wtot[wg] = (unsigned long long)esum;
        group_sync<WPR>(bar);
        esum = 0;
#pragma unroll
        for (int w = 0; w < WPR; ++w) esum += (long long)gs->wtot[w];
    }
    esum = a.cls_e0 + (long long)a.cls_f * esum;
    long long E, bestE, acc_moves;
    int bsweep;
    bool reached = false;
    if (a.fresh) {
        E = esum;
        bestE = esum;
        bsweep = -1;
        acc_moves = 0;
        for (int m = t; m < n; m += G) gbp[m] = sp[m];
        if (t == 0) note_target(a, bestE, -1, reached);
    } else {
        E = a.energy[r];
        bestE = a.best_energy[r];
        bsweep = a.best_sweep[r];
        acc_moves = a.accepted[r];
        if (E != esum && t == 0) atomicOr(a.status, 1);
    }
    group_sync<WPR>(bar);

    const float beta_fixed = a.sweep_end <= a.sweep_begin ? 0.0f
                           : a.mode == 1 ? a.beta[a.rung[r]] : a.mode == 2 ? a.beta[r] : 0.0f;

    // Each thread keeps, for its candidates j = t + G k, the class bit of the
    // facility at j and G_j in registers; it also applies the G update for
    // exactly these j, so they stay equal to shared memory, which keeps the
    // copies other threads read (G_i at the start of every update).
    int cx[MAXK], cg[MAXK];
#pragma unroll
    for (int k = 0; k < MAXK; ++k) {
        const int j = t + G * k;
        cx[k] = j < n ? sx[sp[j]] : 0;
        cg[k] = j < n ? sG[j] : 0;
    }

    for (int s = a.sweep_begin; s < a.sweep_end; ++s) {
        if (a.stop) {
            if (t == 0) gs->stop = *reinterpret_cast<volatile int *>(a.done);
            group_sync<WPR>(bar);
            const int stop_now = gs->stop;
            group_sync<WPR>(bar);
            if (stop_now) break;
        }
        const float beta = (a.mode == 1 || a.mode == 2) ? beta_fixed : a.beta[s];
        for (int i0 = 0; i0 < n; i0 += 32) {
            const uint4 rw = philox4x32_10(a.inst, grep, (uint32_t)s, (uint32_t)(i0 + lane), a.key0, a.key1);
            const int cnt = min(32, n - i0);
            for (int ii = 0; ii < cnt; ++ii) {
                const int i = i0 + ii;
                const unsigned long long draw =
                    ((unsigned long long)__shfl_sync(kFull, rw.y, ii) << 32) |
                    (unsigned long long)__shfl_sync(kFull, rw.x, ii);
                const int xa = sx[sp[i]];
                const int gi = sG[i];
                const DT *Di = sD + i * n;
                // ---- swap energies: 0 within a class, 2 f (G_w - G_u - D_uw) across
                int lmin = 0x7FFFFFFF;
                int dself = 0;  // MAXK = 1: this thread's energy, handed to the draw in a register
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int j = t + G * k;
                    if (j < n) {
                        int d = 0;
                        if (cx[k] != xa) {
                            const int gd = cg[k] - gi;
                            d = f2 * ((xa ? gd : -gd) - (int)Di[j]);
                        }
                        if constexpr (MAXK > 1)
                            sv[j] = d;
                        else
                            dself = d;
                        lmin = min(lmin, d);
                    }
                }
                const int3 sel = eq5_draw<MAXK, WPR>(sv, sp, n, t, lmin, dself, MAXK == 1 && t < n ? sp[t] : 0, beta, draw, bar, gs);
                const int js = sel.x, dstar = sel.y, fb = sel.z;
                if (js == i) continue;
                const int fa = sp[i];
                const int xb = sx[fb];
                // ---- apply: G moves only when the classes differ
                if (xb != xa) {
                    const DT *Dj = sD + js * n;
#pragma unroll
                    for (int k = 0; k < MAXK; ++k) {
                        const int m = t + G * k;
                        if (m < n) {
                            const int dd = (int)Dj[m] - (int)Di[m];
                            const int v = xa ? dd : -dd;
                            sG[m] += v;
                            cg[k] += v;
                        }
                    }
                }
                // the facilities at i and js moved
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int j = t + G * k;
                    if (j == i) cx[k] = xb;
                    if (j == js) cx[k] = xa;
                }
                E += dstar;
                acc_moves += 1;
                if (E < bestE) {
                    bestE = E;
                    bsweep = s;
                    for (int m = t; m < n; m += G) gbp[m] = m == i ? fb : (m == js ? fa : sp[m]);
                    if (t == 0) note_target(a, bestE, s, reached);
                }
                group_sync<WPR>(bar);  // every read of sp[i] and sp[js] is done
                if (t == 0) {
                    sp[i] = fb;
                    sp[js] = fa;
                }
                group_sync<WPR>(bar);
            }
        }
    }

    // ---- audit: G recomputed from the final permutation equals the tracked one
    for (int m = t; m < n; m += G) {
        const DT *Dm = sD + m * n;
        int acc = 0;
        for (int j = 0; j < n; ++j) acc += sx[sp[j]] ? (int)Dm[j] : 0;
        if (acc != sG[m]) atomicOr(a.status, 1);
    }

    // ---- write back
    for (int m = t; m < n; m += G) gp[m] = sp[m];
    if (t == 0) {
        a.energy[r] = E;
        a.best_energy[r] = bestE;
        a.best_sweep[r] = bsweep;
        a.accepted[r] = acc_moves;
    }
    if (a.table_out)
        for (int m = t; m < n; m += G) a.tables[(size_t)r * npad + m] = sG[m];
    group_sync<WPR>(bar);
}

// Persistent: each group of 32 * WPR threads pulls replicas from a.queue.
// Shared memory: D as DT (n x n), x of every facility (bytes, padded to 16),
// then per group: scratch, p, G, and the scratch vector of swap energies.
template <typename DT, int MAXK, int WPR>
__global__ void __launch_bounds__(class_bound(MAXK, WPR)) class_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int G = 32 * WPR;
    const int n = a.n;
    const int npad = (n + 3) & ~3;
    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int bar = 1 + grp;
    DT *sD = reinterpret_cast<DT *>(smem);
    uint8_t *sx = smem + (((size_t)n * n * sizeof(DT) + 15) & ~(size_t)15);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) sD[idx] = static_cast<DT>(a.D[idx]);
    for (int c = threadIdx.x; c < n; c += blockDim.x) sx[c] = a.cls_x[c];
    __syncthreads();
    unsigned char *gb = smem + a.df_bytes + (size_t)grp * a.group_bytes;
    GroupScratch *gs = reinterpret_cast<GroupScratch *>(gb);
    int32_t *sp = reinterpret_cast<int32_t *>(gb + kScratchBytes);
    int32_t *sG = sp + npad;
    int32_t *sv = sG + npad;
    for (;;) {
        if (t == 0) gs->item = atomicAdd(a.queue, 1);
        group_sync<WPR>(bar);
        const int item = gs->item;
        if (item >= a.replicas) break;
        run_class_replica<DT, MAXK, WPR>(a, item, t, bar, sD, sx, sp, sG, sv, gs);
    }
}

#define PDIT_CLASS_SHAPES(X) \
    X(1, 1) X(2, 1) X(4, 1) X(8, 1) X(1, 2) X(2, 2) X(4, 2) X(1, 4) X(2, 4) X(1, 8)

template <typename DT, int MAXK, int WPR>
static int class_one(const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t st, int *blocks,
                     bool query) {
    auto fn = class_kernel<DT, MAXK, WPR>;
    if (threads > class_bound(MAXK, WPR)) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    if (query) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
    fn<<<grid, threads, smem, st>>>(a);
    return (int)cudaGetLastError();
}

template <typename DT>
static int class_dispatch(int maxk, int wpr, const SweepArgs &a, int grid, int threads, size_t smem,
                          cudaStream_t st, int *blocks, bool query) {
#define PDIT_CLASS_CASE(MK, W) \
    if (maxk == MK && wpr == W) return class_one<DT, MK, W>(a, grid, threads, smem, st, blocks, query);
    PDIT_CLASS_SHAPES(PDIT_CLASS_CASE)
#undef PDIT_CLASS_CASE
    return (int)cudaErrorInvalidValue;
}

template <typename DT>
int class_blocks_per_sm(int maxk, int wpr, int threads, size_t smem, int *blocks) {
    SweepArgs dummy{};
    return class_dispatch<DT>(maxk, wpr, dummy, 0, threads, smem, nullptr, blocks, true);
}

template <typename DT>
int class_launch(int maxk, int wpr, const SweepArgs &a, int grid, int threads, size_t smem, cudaStream_t st) {
    return class_dispatch<DT>(maxk, wpr, a, grid, threads, smem, st, nullptr, false);
}

template int class_blocks_per_sm<int8_t>(int, int, int, size_t, int *);
template int class_blocks_per_sm<int16_t>(int, int, int, size_t, int *);
template int class_blocks_per_sm<int32_t>(int, int, int, size_t, int *);
template int class_launch<int8_t>(int, int, const SweepArgs &, int, int, size_t, cudaStream_t);
template int class_launch<int16_t>(int, int, const SweepArgs &, int, int, size_t, cudaStream_t);
template int class_launch<int32_t>(int, int, const SweepArgs &, int, int, size_t, cudaStream_t);

}  // namespace pdit
