// Annealed p-dit sweep kernels for the symmetric QAP on sm_103a.
//
// One warp owns one replica at a time. A CTA stages the instance's D and F
// once in shared memory (int8/int16/int32, whichever holds every value), and
// each of its warps keeps its replica's influence table, permutation and
// scratch vectors in its own slice of shared memory (or, when the table does
// not fit, the table in global memory). Warps pull replicas from a global
// atomic counter until none are left.
//
// Per p-dit update (Eq. 5 over the N outcomes of location i):
//   gather   lane j-interleaved: dE_j from Eq. 3 with the influence table,
//            dE_i = 0 (stay)
//   sample   warp min of dE, binary32 weights (the same arithmetic the CPU
//            oracle states), lane-contiguous 64-bit prefix sums, one 64-bit
//            Philox draw scaled by the total, first prefix above it
//   apply    if a swap j* was drawn: I[m][c] += (D[i][m]-D[j*][m]) (F[b][c]-F[a][c])
//            as int4 read-modify-writes, then p, the p-diagonal h and E
//   best     first occurrence of a new minimum of E (strict <)
// Sweeps visit locations 0..N-1 in order. Every integer is exact; the only
// floating point is the weight computation, made of single correctly rounded
// IEEE operations so the CPU oracle reproduces it bit for bit.
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
    int zero_diag;  // D and F both have zero diagonals
    // run
    int replicas;
    int sweep_begin, sweep_end;
    uint32_t key0, key1;   // Philox key = seed
    uint32_t inst;         // Philox counter word 0
    uint32_t rep_base;     // global id of local replica 0 (counter word 1)
    int mode;              // 0 anneal (beta[s]), 1 parallel tempering (beta[rung])
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
    // launch shape
    size_t df_bytes;       // bytes of staged D and F (16-byte multiple)
    size_t warp_bytes;     // bytes of one warp's slice
};

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
// 15-bit head plus its binary32 tail), Taylor polynomial of degree 7 for
// e^-r in Horner form with fused multiply-adds, exact scaling by 2^-k.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float expneg_f32(float x) {
    const float t = __fadd_rn(__fmul_rn(x, 1.44269502f), 0.5f);
    const int k = __float2int_rz(t);
    const float kf = __int2float_rn(k);
    float r = __fmaf_rn(-kf, 0.693145751953125f, x);
    r = __fmaf_rn(-kf, 1.42860677e-06f, r);
    const float y = -r;
    float q = 1.98412701e-04f;      // 1/7!
    q = __fmaf_rn(q, y, 1.38888892e-03f);  // 1/6!
    q = __fmaf_rn(q, y, 8.33333377e-03f);  // 1/5!
    q = __fmaf_rn(q, y, 4.16666679e-02f);  // 1/4!
    q = __fmaf_rn(q, y, 1.66666672e-01f);  // 1/3!
    q = __fmaf_rn(q, y, 0.5f);
    q = __fmaf_rn(q, y, 1.0f);
    q = __fmaf_rn(q, y, 1.0f);
    return __fmul_rn(q, __int_as_float((127 - k) << 23));
}

__device__ __forceinline__ unsigned long long eq5_weight(int shifted_de, float beta) {
    const float x = __fmul_rn(__int2float_rn(shifted_de), beta);
    if (!(x <= 40.0f)) return 0ull;
    return __float2ull_rz(__fmul_rn(expneg_f32(x), 9007199254740992.0f));
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
__device__ __forceinline__ void load_lane_block(const int32_t *sv, int lane, int (&d)[K]) {
    if constexpr (K == 1) {
        d[0] = sv[lane];
    } else if constexpr (K == 2) {
        const int2 v = reinterpret_cast<const int2 *>(sv)[lane];
        d[0] = v.x;
        d[1] = v.y;
    } else {
#pragma unroll
        for (int h = 0; h < K / 4; ++h) {
            const int4 v = reinterpret_cast<const int4 *>(sv)[lane * (K / 4) + h];
            d[4 * h + 0] = v.x;
            d[4 * h + 1] = v.y;
            d[4 * h + 2] = v.z;
            d[4 * h + 3] = v.w;
        }
    }
}

// ---------------------------------------------------------------------------
// One replica: initial state, table build, sweeps [sweep_begin, sweep_end),
// write-back. `T` is the replica's influence table (shared or global memory),
// row stride S; sp = permutation, sh = p-diagonal h[m] = I[m][p(m)],
// sv = scratch (swap energies in j order, then the rank-1 column factor).
// MAXK = candidates (and table rows) per lane, a power of two >= n/32.
// ---------------------------------------------------------------------------
template <typename DT, int MAXK>
__device__ __forceinline__ void run_replica(const SweepArgs &a, int r, int lane, const DT *sD,
                                            const DT *sF, int32_t *T, int32_t *sp, int32_t *sh,
                                            int32_t *sv) {
    const int n = a.n;
    const int S = a.stride;
    const int npad = (n + 3) & ~3;
    const uint32_t grep = a.rep_base + (uint32_t)r;
    int32_t *gp = a.perm + (size_t)r * n;
    int32_t *gbp = a.best_perm + (size_t)r * n;

    // ---- permutation: Fisher-Yates from the last position down; step k uses
    // word k%4 of Philox(inst, replica, 0xFFFFFFFF, k/4) and index
    // floor(u (k+1) / 2^32).
    if (a.fresh) {
        for (int q = lane; 4 * q < n; q += 32) {
            const uint4 o = philox4x32_10(a.inst, grep, 0xFFFFFFFFu, (uint32_t)q, a.key0, a.key1);
            reinterpret_cast<uint4 *>(sv)[q] = o;
        }
        for (int m = lane; m < n; m += 32) sp[m] = m;
        __syncwarp();
        if (lane == 0) {
            for (int k = n - 1; k >= 1; --k) {
                const int j = (int)__umulhi((uint32_t)sv[k], (uint32_t)(k + 1));
                const int t = sp[k];
                sp[k] = sp[j];
                sp[j] = t;
            }
        }
    } else {
        for (int m = lane; m < n; m += 32) sp[m] = gp[m];
    }
    __syncwarp();

    // ---- influence table, Eq. 2 in the one-term form I[m][c] = sum_j D[m][j] F[c][p(j)]
    // (F symmetric, so row p(j) of F is read contiguously).
    if (a.table_in) {
        const int32_t *src = a.tables + (size_t)r * n * S;
        if (src != T) {
            const int4 *s4 = reinterpret_cast<const int4 *>(src);
            int4 *d4 = reinterpret_cast<int4 *>(T);
            for (int idx = lane; idx < n * S / 4; idx += 32) d4[idx] = s4[idx];
        }
    } else {
        for (int m = 0; m < n; ++m) {
            int acc[MAXK];
#pragma unroll
            for (int k = 0; k < MAXK; ++k) acc[k] = 0;
            const DT *Dm = sD + m * n;
            for (int j = 0; j < n; ++j) {
                const int d = Dm[j];
                const DT *Fr = sF + sp[j] * n;
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int c = lane + 32 * k;
                    if (c < n) acc[k] += d * (int)Fr[c];
                }
            }
#pragma unroll
            for (int k = 0; k < MAXK; ++k) {
                const int c = lane + 32 * k;
                if (c < npad) T[m * S + c] = c < n ? acc[k] : 0;
            }
        }
    }
    __syncwarp();

    // ---- p-diagonal and energy: E = sum_m I[m][p(m)] (Eq. 1 regrouped)
    long long esum = 0;
#pragma unroll
    for (int k = 0; k < MAXK; ++k) {
        const int m = lane + 32 * k;
        if (m < n) {
            const int h = T[m * S + sp[m]];
            sh[m] = h;
            esum += h;
        }
    }
    esum = warp_sum(esum);
    long long E, bestE, acc_moves;
    int bsweep;
    if (a.fresh) {
        E = esum;
        bestE = esum;
        bsweep = -1;
        acc_moves = 0;
        for (int m = lane; m < n; m += 32) gbp[m] = sp[m];
    } else {
        E = a.energy[r];
        bestE = a.best_energy[r];
        bsweep = a.best_sweep[r];
        acc_moves = a.accepted[r];
        if (E != esum && lane == 0) atomicOr(a.status, 1);
    }
    __syncwarp();

    const float beta_pt = (a.mode == 1 && a.sweep_end > a.sweep_begin) ? a.beta[a.rung[r]] : 0.0f;
    const int zero_diag = a.zero_diag;

    for (int s = a.sweep_begin; s < a.sweep_end; ++s) {
        const float beta = a.mode == 1 ? beta_pt : a.beta[s];
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
                const DT *Di = sD + i * n;
                const DT *Fa = sF + fa * n;
                const int dii = Di[i];
                const int faa = Fa[fa];

                // ---- gather: Eq. 3 for every candidate j (lane-interleaved)
                int lmin = 0x7FFFFFFF;
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int j = lane + 32 * k;
                    int d = 0x7FFFFFFF;
                    if (j < n) {
                        const int b = sp[j];
                        const int row_ib = T[i * S + b];
                        const int col_ja = T[j * S + fa];
                        const int dij = Di[j];
                        const int fab = Fa[b];
                        d = 2 * (row_ib - hi + col_ja - sh[j]);
                        if (zero_diag)
                            d += 4 * dij * fab;
                        else
                            d += (dii + (int)sD[j * n + j] - 2 * dij) * (faa + (int)sF[b * n + b] - 2 * fab);
                        if (j == i) d = 0;
                        sv[j] = d;
                    }
                    lmin = min(lmin, d);
                }
                const int dmin = warp_min(lmin);
                __syncwarp();

                // ---- sample: lane-contiguous weights, 64-bit prefix sums
                int dc[MAXK];
                load_lane_block<MAXK>(sv, lane, dc);
                unsigned long long pre[MAXK];
                unsigned long long lsum = 0;
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int j = lane * MAXK + k;
                    if (j < n) lsum += eq5_weight(dc[k] - dmin, beta);
                    pre[k] = lsum;
                }
                unsigned long long incl = lsum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned long long total = __shfl_sync(kFull, incl, 31);
                const unsigned long long excl = incl - lsum;
                const unsigned long long t = __umul64hi(draw, total);
                const bool own = (t >= excl) && (t < incl);
                const unsigned ball = __ballot_sync(kFull, own);
                const int src = __ffs(ball) - 1;
                int jloc = 0, dsel = 0;
                if (own) {
                    int kk = MAXK - 1;
#pragma unroll
                    for (int k = MAXK - 1; k >= 0; --k)
                        if (excl + pre[k] > t) kk = k;
#pragma unroll
                    for (int k = 0; k < MAXK; ++k)
                        if (k == kk) dsel = dc[k];
                    jloc = lane * MAXK + kk;
                }
                const int js = __shfl_sync(kFull, jloc, src);
                const int dstar = __shfl_sync(kFull, dsel, src);
                __syncwarp();
                if (js == i) continue;

                // ---- apply the swap i <-> js: rank-1 update of the table
                const int fb = sp[js];
                const DT *Fb = sF + fb * n;
                const DT *Dj = sD + js * n;
                for (int c = lane; c < npad; c += 32) sv[c] = c < n ? (int)Fb[c] - (int)Fa[c] : 0;
                int u[MAXK];
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int m = lane + 32 * k;
                    u[k] = m < n ? (int)Di[m] - (int)Dj[m] : 0;
                }
                __syncwarp();
                const int4 *v4 = reinterpret_cast<const int4 *>(sv);
#pragma unroll 2
                for (int cq = 0; cq < npad / 4; ++cq) {
                    const int4 vq = v4[cq];
#pragma unroll
                    for (int k = 0; k < MAXK; ++k) {
                        const int m = lane + 32 * k;
                        if (m < n) {
                            int4 *row = reinterpret_cast<int4 *>(T + m * S) + cq;
                            int4 x = *row;
                            x.x += u[k] * vq.x;
                            x.y += u[k] * vq.y;
                            x.z += u[k] * vq.z;
                            x.w += u[k] * vq.w;
                            *row = x;
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    sp[i] = fb;
                    sp[js] = fa;
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < MAXK; ++k) {
                    const int m = lane + 32 * k;
                    if (m < n) sh[m] = T[m * S + sp[m]];
                }
                E += dstar;
                acc_moves += 1;
                if (E < bestE) {
                    bestE = E;
                    bsweep = s;
                    for (int m = lane; m < n; m += 32) gbp[m] = sp[m];
                }
                __syncwarp();
            }
        }
    }

    // ---- write back
    for (int m = lane; m < n; m += 32) gp[m] = sp[m];
    if (lane == 0) {
        a.energy[r] = E;
        a.best_energy[r] = bestE;
        a.best_sweep[r] = bsweep;
        a.accepted[r] = acc_moves;
    }
    if (a.table_out) {
        int32_t *dst = a.tables + (size_t)r * n * S;
        if (dst != T) {
            const int4 *s4 = reinterpret_cast<const int4 *>(T);
            int4 *d4 = reinterpret_cast<int4 *>(dst);
            for (int idx = lane; idx < n * S / 4; idx += 32) d4[idx] = s4[idx];
        }
    }
    if (a.dump) {
        int32_t *dst = a.dump + (size_t)r * n * n;
        for (int idx = lane; idx < n * n; idx += 32) dst[idx] = T[(idx / n) * S + idx % n];
    }
    __syncwarp();
}

template <int MAXK>
struct SweepBounds {
    static constexpr int threads = MAXK == 1 ? 1024 : (MAXK == 2 ? 512 : (MAXK == 4 ? 384 : 128));
};

template <typename DT, int MAXK, bool TSMEM>
__global__ void __launch_bounds__(SweepBounds<MAXK>::threads) sweep_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    DT *sD = reinterpret_cast<DT *>(smem);
    DT *sF = sD + n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        sD[idx] = static_cast<DT>(a.D[idx]);
        sF[idx] = static_cast<DT>(a.F[idx]);
    }
    __syncthreads();
    unsigned char *wb = smem + a.df_bytes + (size_t)warp * a.warp_bytes;
    const int npad = (n + 3) & ~3;
    int32_t *sT = reinterpret_cast<int32_t *>(wb);
    int32_t *sp = reinterpret_cast<int32_t *>(wb + (TSMEM ? (size_t)n * a.stride * 4 : 0));
    int32_t *sh = sp + npad;
    int32_t *sv = sh + npad;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.queue, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.replicas) break;
        if constexpr (TSMEM) {
            run_replica<DT, MAXK>(a, item, lane, sD, sF, sT, sp, sh, sv);
        } else {
            run_replica<DT, MAXK>(a, item, lane, sD, sF, a.tables + (size_t)item * n * a.stride, sp,
                                  sh, sv);
        }
    }
}

// Host-side entry points, one per storage type of D and F (defined in
// pdit_sweep_i8.cu, pdit_sweep_i16.cu, pdit_sweep_i32.cu).
// maxk in {1, 2, 4, 8}. Return a cudaError_t value.
template <typename DT>
int sweep_blocks_per_sm(int maxk, bool tsmem, int threads, size_t smem, int *blocks);
template <typename DT>
int sweep_launch(int maxk, bool tsmem, const SweepArgs &a, int grid, int threads, size_t smem,
                 cudaStream_t stream);

#define PDIT_INSTANTIATE_SWEEP(DT)                                                               \
    template <int MAXK, bool TSMEM>                                                              \
    static int sweep_one(const SweepArgs &a, int grid, int threads, size_t smem,                \
                         cudaStream_t st, int *blocks, bool query) {                             \
        auto fn = sweep_kernel<DT, MAXK, TSMEM>;                                                 \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                             (int)smem);                                         \
        if (e != cudaSuccess) return (int)e;                                                     \
        if (query) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn,         \
                                                                              threads, smem);    \
        fn<<<grid, threads, smem, st>>>(a);                                                      \
        return (int)cudaGetLastError();                                                          \
    }                                                                                            \
    static int sweep_dispatch(int maxk, bool tsmem, const SweepArgs &a, int grid, int threads,   \
                              size_t smem, cudaStream_t st, int *blocks, bool query) {           \
        switch (maxk * 2 + (tsmem ? 1 : 0)) {                                                    \
        case 3: return sweep_one<1, true>(a, grid, threads, smem, st, blocks, query);            \
        case 5: return sweep_one<2, true>(a, grid, threads, smem, st, blocks, query);            \
        case 9: return sweep_one<4, true>(a, grid, threads, smem, st, blocks, query);            \
        case 17: return sweep_one<8, true>(a, grid, threads, smem, st, blocks, query);           \
        case 8: return sweep_one<4, false>(a, grid, threads, smem, st, blocks, query);           \
        case 16: return sweep_one<8, false>(a, grid, threads, smem, st, blocks, query);          \
        default: return (int)cudaErrorInvalidValue;                                              \
        }                                                                                        \
    }                                                                                            \
    template <>                                                                                  \
    int sweep_blocks_per_sm<DT>(int maxk, bool tsmem, int threads, size_t smem, int *blocks) {   \
        SweepArgs dummy{};                                                                       \
        return sweep_dispatch(maxk, tsmem, dummy, 0, threads, smem, nullptr, blocks, true);      \
    }                                                                                            \
    template <>                                                                                  \
    int sweep_launch<DT>(int maxk, bool tsmem, const SweepArgs &a, int grid, int threads,        \
                         size_t smem, cudaStream_t st) {                                         \
        return sweep_dispatch(maxk, tsmem, a, grid, threads, smem, st, nullptr, false);          \
    }

}  // namespace pdit
