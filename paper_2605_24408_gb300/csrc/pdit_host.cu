// C ABI of libpdit (include/pdit.h): instance upload, launch planning,
// parallel-tempering exchange, final reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pdit.h"
#include "pdit_sweep.cuh"

struct pdit_qap {
    int n = 0;
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    size_t l2_bytes = 0;
    int dt_bytes = 4;       // storage of D and F in shared memory: 1, 2 or 4 bytes
    int zero_diag = 0;
    int asym = 0;           // D or F not symmetric: the general form (two-term table)
    int cls = 0;            // two-level flow (pdit_class.cu): F = f0 + f x_c x_d off the diagonal
    int use_cls = 1;        // run such instances with the flow-class kernel
    int cls_f = 0;
    long long cls_e0 = 0;
    uint8_t *dx = nullptr;  // x_c on the device
    int packed_ok = 0;      // max-min of D and of F <= 127: swap factors fit int8
    std::vector<int32_t> hD, hF;
    std::vector<uint8_t> cls_x;  // class bit of every facility (two-level flows)
    int32_t *dD = nullptr, *dF = nullptr;
    // owned by the handle, grown on demand
    void *ws = nullptr;
    size_t ws_bytes = 0;
    float *dbeta = nullptr;
    size_t dbeta_cap = 0;
    int32_t *dperm = nullptr;
    int64_t *dcost = nullptr;
    int32_t *dstatus = nullptr;
    cudaStream_t stream = nullptr;
    int force_wpr = 0;      // warps per replica; 0 = chosen per launch
    int force_pk = 0;       // pending swaps before a table rewrite; 0 = chosen per launch
    int force_groups = 0;   // replicas per CTA; 0 = chosen per launch
    int force_place = 0;    // influence tables: 0 = shared memory when they fit, 1 = shared, 2 = global
    int force_infl = 0;     // influence entries: PDIT_INFLUENCE_AUTO, _TABLE or _PRODUCTS
};

namespace {

thread_local std::string g_last_error = "";

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return PDIT_ECUDA;
}

#define PDIT_CK(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Smallest 4*odd >= n: rows start 16-byte aligned and a quarter-warp's
// column-wise int4 accesses to 8 consecutive rows hit 8 disjoint bank groups.
int table_stride(int n) {
    int s = (n + 3) & ~3;
    if ((s / 4) % 2 == 0) s += 4;
    return s;
}

// Candidates covered by one group: 32 * WPR * MAXK, a power of two >= n.
int cover_for(int n) {
    int c = 32;
    while (c < n) c <<= 1;
    return c;
}

// Row stride (elements) of D and F as staged for the general form: rows of
// 4 x odd bytes, so that the 32 lanes of a warp reading one column hit 32
// distinct banks.
int stage_stride(int n, int dt) {
    const int per_word = 4 / dt;
    int words = (n + per_word - 1) / per_word;
    if (words % 2 == 0) words += 1;
    return words * per_word;
}

struct Plan {
    int maxk = 1, wpr = 1, pk = 1;
    bool tsmem = true, cls = false, dot = false;
    int stride = 0, sv_len = 0, cupim_off = 0, v2_off = 0, rc_off = 0, dstride = 0;
    size_t table_elems = 0;  // int32 entries of one replica's saved table (workspace)
    size_t df_bytes = 0, group_bytes = 0, smem = 0;
    int groups = 1, threads = 32, grid = 1;
};


template <bool ASYM>
int sweep_blocks_t(int dt, const Plan &p, int *blocks) {
    if (dt == 1) return pdit::sweep_blocks_per_sm<int8_t, ASYM>(p.maxk, p.wpr, p.tsmem, p.pk, p.threads, p.smem, blocks);
    if (dt == 2) return pdit::sweep_blocks_per_sm<int16_t, ASYM>(p.maxk, p.wpr, p.tsmem, p.pk, p.threads, p.smem, blocks);
    return pdit::sweep_blocks_per_sm<int32_t, ASYM>(p.maxk, p.wpr, p.tsmem, p.pk, p.threads, p.smem, blocks);
}

int sweep_blocks(int dt, bool asym, const Plan &p, int *blocks) {
    return asym ? sweep_blocks_t<true>(dt, p, blocks) : sweep_blocks_t<false>(dt, p, blocks);
}

template <bool ASYM>
int sweep_launch_t(int dt, const Plan &p, const pdit::SweepArgs &a, cudaStream_t st) {
    if (dt == 1) return pdit::sweep_launch<int8_t, ASYM>(p.maxk, p.wpr, p.tsmem, p.pk, a, p.grid, p.threads, p.smem, st);
    if (dt == 2) return pdit::sweep_launch<int16_t, ASYM>(p.maxk, p.wpr, p.tsmem, p.pk, a, p.grid, p.threads, p.smem, st);
    return pdit::sweep_launch<int32_t, ASYM>(p.maxk, p.wpr, p.tsmem, p.pk, a, p.grid, p.threads, p.smem, st);
}

int sweep_launch(int dt, bool asym, const Plan &p, const pdit::SweepArgs &a, cudaStream_t st) {
    return asym ? sweep_launch_t<true>(dt, p, a, st) : sweep_launch_t<false>(dt, p, a, st);
}

// Scratch-vector length (int32 entries) of a group: swap energies, the row
// factor of a table update, (general form) its column factor, (concurrent
// updates) the proposal arrays.
int sv_len_for(int stride, int cover) { return std::max(stride, cover); }

// Shared-memory slice of one replica group for a given shape: scratch
// struct, table (if in shared memory), p, h, the scratch vector, and the
// packed pending swap factors (int8 x 4 per word) when pk > 1.
size_t group_bytes_for(int n, int stride, int cover, bool tsmem, int pk, int extra_sv = 0) {
    const size_t npad = (size_t)((n + 3) & ~3);
    const size_t vec = 4 * (2 * npad + (size_t)sv_len_for(stride, cover) + (size_t)extra_sv);
    const size_t table = tsmem ? (size_t)4 * n * stride : 0;
    const size_t ring = pk > 1 ? (size_t)8 * npad * (pk / 4) : 0;  // packed u and v words
    return align_up(pdit::kScratchBytes + table + vec + ring, 16);
}

// Replicas a plan keeps resident at once.
int resident(const Plan &p, int replicas) { return std::min(replicas, p.grid * p.groups); }

// Launch shape for `replicas` chains of an n-location instance. `wpr` = warps
// per replica (0: choose).
int make_plan(const pdit_qap *h, int replicas, int wpr, int pk, Plan *p, size_t reserve = 0,
              bool cupim = false) {
    const int n = h->n;
    const int cover = cover_for(n);
    const int npad = (n + 3) & ~3;
    p->stride = table_stride(n);
    const int base = sv_len_for(p->stride, cover);
    // Extra scratch-vector entries for `k` pending terms: the column factor
    // of the general form's immediate rank-2 update, the gathered table
    // values (tables in global memory), and the proposal, energy-change and
    // order arrays of concurrent updates.
    auto extra_for = [&](int k) {
        return (h->asym && k == 1 ? npad : 0) + (p->tsmem ? 0 : 2 * npad) + (cupim ? 3 * npad : 0);
    };
    p->dstride = h->asym ? stage_stride(n, h->dt_bytes) : n;
    p->df_bytes = align_up((size_t)2 * n * p->dstride * h->dt_bytes, 16);
    const size_t budget = h->smem_optin - reserve;
    p->tsmem = true;
    const size_t g_smem = group_bytes_for(n, p->stride, cover, true, 1, extra_for(1));
    const bool fits = p->df_bytes + g_smem <= budget;
    const bool defer_ok = h->packed_ok != 0;
    if (h->force_place == PDIT_PLACE_SHARED && !fits) return PDIT_ENOTSUP;
    p->tsmem = h->force_place == PDIT_PLACE_GLOBAL ? false : fits;
    // Built-in choice: where shared memory holds a single replica per SM,
    // L2-resident tables (two or more replicas per SM, 16 pending terms) are
    // faster.
    if (h->force_place == PDIT_PLACE_AUTO && fits && defer_ok && cover == 256 &&
        (budget - p->df_bytes) / g_smem < 2)
        p->tsmem = false;
    if (!p->tsmem && cover < 256) return PDIT_ENOTSUP;  // global-table kernels: 32 * WPR * MAXK = 256
    if (pk != 0 && pk != 1 && pk != 4 && pk != 16) return PDIT_EINVAL;
    if (pk > 1 && !defer_ok) return PDIT_ENOTSUP;
    if (pk == 16 && p->tsmem) return PDIT_ENOTSUP;  // compiled for global tables only
    if (pk == 0) {
        // Defer table rewrites always for tables in global memory (16
        // pending terms: each rewrite streams the whole table through L2),
        // and for tables in shared memory (4 pending terms) unless the packed
        // factors would leave fewer replicas resident for this call.
        if (!defer_ok) {
            pk = 1;
        } else if (!p->tsmem) {
            pk = 16;
        } else {
            Plan p1, p4;
            const int r1 = make_plan(h, replicas, wpr, 1, &p1, reserve, cupim);
            const int r4 = make_plan(h, replicas, wpr, 4, &p4, reserve, cupim);
            if (r4 == PDIT_OK && (r1 != PDIT_OK || resident(p4, replicas) >= resident(p1, replicas))) {
                *p = p4;
                return PDIT_OK;
            }
            if (r1 != PDIT_OK) return r1;
            *p = p1;
            return PDIT_OK;
        }
    }
    p->pk = pk;
    p->table_elems = (size_t)n * p->stride;
    p->v2_off = base;
    p->rc_off = base + (h->asym && pk == 1 ? npad : 0);
    p->cupim_off = p->rc_off + (p->tsmem ? 0 : 2 * npad);
    p->sv_len = base + extra_for(pk);
    p->group_bytes = group_bytes_for(n, p->stride, cover, p->tsmem, pk, extra_for(pk));
    if (p->df_bytes + p->group_bytes > budget) return PDIT_ENOTSUP;
    int fit = (int)((budget - p->df_bytes) / p->group_bytes);  // replicas per CTA by memory
    int l2_cap = 1 << 30;  // resident replicas per SM whose tables fit three quarters of L2
    if (!p->tsmem && h->l2_bytes > 0 && h->num_sms > 0) {
        const size_t table = (size_t)4 * n * p->stride;
        l2_cap = (int)std::max<size_t>(1, (h->l2_bytes * 3 / 4) / (table * (size_t)h->num_sms));
        if (h->force_groups <= 0) fit = std::min(fit, l2_cap);
    }
    if (wpr <= 0) {
        // Aim for about 16 resident warps per SM to hide the latency of each
        // replica's sequential update chain; tables in global memory are
        // latency-bound on every access, so they take the most warps.
        wpr = 1;
        while (wpr < cover / 32 && (!p->tsmem || std::min(fit, 32 / wpr) * wpr < 16)) wpr <<= 1;
    }
    if (wpr < 1 || wpr > cover / 32 || (wpr & (wpr - 1))) return PDIT_EINVAL;
    p->wpr = wpr;
    p->maxk = cover / (32 * wpr);
    int g = std::min(fit, pdit::sweep_bound(p->maxk, wpr) / (32 * wpr));
    if (wpr > 1) g = std::min(g, 15);  // named barriers 1..15
    if (h->force_groups > 0) g = std::min(g, h->force_groups);
    const int per_sm = (replicas + h->num_sms - 1) / h->num_sms;
    g = std::max(1, std::min(g, per_sm));
    p->groups = g;
    p->threads = 32 * wpr * g;
    p->smem = p->df_bytes + (size_t)g * p->group_bytes;
    int bps = 0;
    int e = sweep_blocks(h->dt_bytes, h->asym != 0, *p, &bps);
    if (e != 0) return cuda_fail((cudaError_t)e, "occupancy query");
    if (bps < 1) bps = 1;
    if (!p->tsmem) bps = std::max(1, std::min(bps, l2_cap / g));  // CTAs per SM within the L2 cap
    const int need = (replicas + g - 1) / g;
    p->grid = std::max(1, std::min(need, h->num_sms * bps));
    return PDIT_OK;
}

// Launch shape of the flow-class kernel: D as DT and x in shared memory once
// per CTA, then per replica group: scratch, p, G and the swap energies.
int make_class_plan(const pdit_qap *h, int replicas, int wpr, Plan *p) {
    const int n = h->n;
    const int cover = cover_for(n);
    const int npad = (n + 3) & ~3;
    p->cls = true;
    p->tsmem = true;
    p->pk = 1;
    p->stride = npad;
    p->table_elems = (size_t)npad;  // G
    p->sv_len = cover;
    p->dstride = n;
    p->df_bytes = align_up((size_t)n * n * h->dt_bytes, 16) + align_up((size_t)npad, 16);
    p->group_bytes = align_up(pdit::kScratchBytes + (size_t)4 * (2 * npad + cover), 16);
    const size_t budget = h->smem_optin;
    if (p->df_bytes + p->group_bytes > budget) return PDIT_ENOTSUP;
    const int fit = (int)((budget - p->df_bytes) / p->group_bytes);
    if (wpr <= 0) wpr = 1;  // one warp per replica: many independent replicas per SM
    if (wpr < 1 || wpr > cover / 32 || (wpr & (wpr - 1))) return PDIT_EINVAL;
    p->wpr = wpr;
    p->maxk = cover / (32 * wpr);
    int g = std::min(fit, pdit::class_bound(p->maxk, wpr) / (32 * wpr));
    if (wpr > 1) g = std::min(g, 15);  // named barriers 1..15
    if (h->force_groups > 0) g = std::min(g, h->force_groups);
    const int per_sm = (replicas + h->num_sms - 1) / h->num_sms;
    g = std::max(1, std::min(g, per_sm));
    p->groups = g;
    p->threads = 32 * wpr * g;
    p->smem = p->df_bytes + (size_t)g * p->group_bytes;
    int bps = 0;
    int e = 0;
    if (h->dt_bytes == 1) e = pdit::class_blocks_per_sm<int8_t>(p->maxk, wpr, p->threads, p->smem, &bps);
    else if (h->dt_bytes == 2) e = pdit::class_blocks_per_sm<int16_t>(p->maxk, wpr, p->threads, p->smem, &bps);
    else e = pdit::class_blocks_per_sm<int32_t>(p->maxk, wpr, p->threads, p->smem, &bps);
    if (e != 0) return cuda_fail((cudaError_t)e, "occupancy query");
    if (bps < 1) bps = 1;
    const int need = (replicas + g - 1) / g;
    p->grid = std::max(1, std::min(need, h->num_sms * bps));
    return PDIT_OK;
}

int class_launch(int dt, const Plan &p, const pdit::SweepArgs &a, cudaStream_t st) {
    if (dt == 1) return pdit::class_launch<int8_t>(p.maxk, p.wpr, a, p.grid, p.threads, p.smem, st);
    if (dt == 2) return pdit::class_launch<int16_t>(p.maxk, p.wpr, a, p.grid, p.threads, p.smem, st);
    return pdit::class_launch<int32_t>(p.maxk, p.wpr, a, p.grid, p.threads, p.smem, st);
}

// Launch shape of the dot-product kernel (pdit_dot.cu): D as int8 in slot
// order once per CTA, then per replica group: scratch, the permuted flow
// matrix Q (rows x stride bytes), p and h. Row stride: 16 bytes x odd.
int make_dot_plan(const pdit_qap *h, int replicas, int wpr, Plan *p, size_t reserve = 0) {
    const int n = h->n;
    const int cover = cover_for(n);
    const int npad = (n + 3) & ~3;
    int s16 = (n + 15) / 16;
    if (s16 % 2 == 0) s16 += 1;
    p->dot = true;
    p->tsmem = true;
    p->pk = 1;
    p->stride = 16 * s16;
    p->dstride = n;
    p->sv_len = 0;
    const size_t budget = h->smem_optin - reserve;
    auto sizes = [&](int maxk, size_t *df, size_t *grp) {
        const size_t rows = (size_t)((n + maxk - 1) / maxk) * maxk;
        *df = rows * p->stride;
        *grp = align_up(pdit::kScratchBytes + rows * p->stride + (size_t)8 * npad, 16);
    };
    auto fit_for = [&](int w) {
        size_t df, grp;
        sizes(cover / (32 * w), &df, &grp);
        return df + grp > budget ? 0 : (int)((budget - df) / grp);
    };
    if (wpr <= 0) {
        // the fewest warps per replica that keep about 16 warps resident per
        // SM, among the compiled shapes; else the shape with the most
        int best = 0, best_warps = -1;
        for (int w = 1; w <= cover / 32; w <<= 1) {
            if (!pdit::dot_shape_compiled(cover / (32 * w), w)) continue;
            int g = std::min(fit_for(w), pdit::dot_bound(cover / (32 * w), w) / (32 * w));
            if (w > 1) g = std::min(g, 15);
            if (g * w >= 16) {
                best = w;
                break;
            }
            if (g * w > best_warps) {
                best = w;
                best_warps = g * w;
            }
        }
        if (!best) return PDIT_ENOTSUP;
        wpr = best;
    }
    if (wpr < 1 || wpr > cover / 32 || (wpr & (wpr - 1))) return PDIT_EINVAL;
    p->wpr = wpr;
    p->maxk = cover / (32 * wpr);
    if (!pdit::dot_shape_compiled(p->maxk, wpr)) return PDIT_ENOTSUP;
    sizes(p->maxk, &p->df_bytes, &p->group_bytes);
    // int32 words of one replica's saved permuted flow matrix (rows x stride bytes)
    p->table_elems = (size_t)((n + p->maxk - 1) / p->maxk) * p->maxk * p->stride / 4;
    if (p->df_bytes + p->group_bytes > budget) return PDIT_ENOTSUP;
    const int fit = (int)((budget - p->df_bytes) / p->group_bytes);
    int g = std::min(fit, pdit::dot_bound(p->maxk, wpr) / (32 * wpr));
    if (wpr > 1) g = std::min(g, 15);  // named barriers 1..15
    if (h->force_groups > 0) g = std::min(g, h->force_groups);
    const int per_sm = (replicas + h->num_sms - 1) / h->num_sms;
    g = std::max(1, std::min(g, per_sm));
    p->groups = g;
    p->threads = 32 * wpr * g;
    p->smem = p->df_bytes + (size_t)g * p->group_bytes;
    int bps = 0;
    const int e = pdit::dot_blocks_per_sm(p->maxk, wpr, p->stride, p->threads, p->smem, &bps);
    if (e != 0) return cuda_fail((cudaError_t)e, "occupancy query");
    if (bps < 1) bps = 1;
    const int need = (replicas + g - 1) / g;
    p->grid = std::max(1, std::min(need, h->num_sms * bps));
    return PDIT_OK;
}

// Whether an instance can run the dot-product kernel: symmetric, every entry
// of D and F in a signed byte (dp4a operands).
bool dot_eligible(const pdit_qap *h) { return !h->asym && h->dt_bytes == 1; }

// Whether a call runs the flow-class kernel: a two-level-flow instance with
// the path enabled, in a sequential mode, without a request for the N x N
// table dump (which only the table kernels keep).
bool use_class_path(const pdit_qap *h, const pdit_opts *o) {
    return h->cls && h->use_cls && o->mode != PDIT_MODE_CUPIM && !o->tables;
}

// The automatic choice of the dot kernel: it keeps an N x N byte matrix per
// replica, and where shared memory holds fewer than 3 replicas per SM (N
// above about 200) the table kernels are faster (measured: N = 190 2.38e8
// against 1.94e8 updates/s, N = 256 1.30e8 against 1.84e8). PDIT_ENOTSUP
// when it does not take the dot kernel.
int auto_dot_plan(const pdit_qap *h, int replicas, Plan *p, size_t reserve) {
    Plan full;
    int rc = make_dot_plan(h, 1 << 28, h->force_wpr, &full, reserve);
    if (rc != PDIT_OK) return rc;
    if (full.groups * std::max(1, full.grid / std::max(1, h->num_sms)) < 3) return PDIT_ENOTSUP;
    return make_dot_plan(h, replicas, h->force_wpr, p, reserve);
}

// Whether a call runs the dot-product kernel: an eligible instance in a
// sequential mode, without a request for the table dump or for table-kernel
// knobs (pending terms, table placement), unless the handle asks for it.
bool use_dot_path(const pdit_qap *h, const pdit_opts *o) {
    if (!dot_eligible(h) || o->mode == PDIT_MODE_CUPIM || o->tables) return false;
    return h->force_infl == PDIT_INFLUENCE_AUTO && h->force_pk == 0 && h->force_place == PDIT_PLACE_AUTO;
}

// Launch plan of a call: the flow-class kernel, the dot-product kernel or
// the table kernels.
int plan_for(const pdit_qap *h, const pdit_opts *o, Plan *p) {
    if (use_class_path(h, o)) return make_class_plan(h, o->replicas, h->force_wpr, p);
    if (h->force_infl == PDIT_INFLUENCE_PRODUCTS) {
        if (!dot_eligible(h) || o->mode == PDIT_MODE_CUPIM || o->tables) return PDIT_ENOTSUP;
        return make_dot_plan(h, o->replicas, h->force_wpr, p);
    }
    if (use_dot_path(h, o)) {
        const int rc = auto_dot_plan(h, o->replicas, p, 0);
        if (rc != PDIT_ENOTSUP) return rc;
        *p = Plan();  // no suitable dot shape: the table kernels
    }
    return make_plan(h, o->replicas, h->force_wpr, h->force_pk, p, 0, o->mode == PDIT_MODE_CUPIM);
}

// Plan of one instance in a multi-instance launch (batches, the server):
// the dot kernel where the automatic rule takes it, else the table kernels;
// the kernels keep their descriptor in `reserve` bytes of static shared
// memory.
int batch_plan(const pdit_qap *h, Plan *p, size_t reserve) {
    if (!h->cls || !h->use_cls) {
        if (h->force_infl == PDIT_INFLUENCE_PRODUCTS) {
            if (!dot_eligible(h)) return PDIT_ENOTSUP;
            return make_dot_plan(h, 1 << 28, h->force_wpr, p, reserve);
        }
        pdit_opts o;
        pdit_opts_init(&o);
        if (use_dot_path(h, &o)) {
            const int rc = auto_dot_plan(h, 1 << 28, p, reserve);
            if (rc != PDIT_ENOTSUP) return rc;
            *p = Plan();
        }
    }
    return make_plan(h, 1 << 28, h->force_wpr, h->force_pk, p, reserve);
}

struct Workspace {
    int32_t *perm, *best_perm, *best_sweep, *rung, *since_top, *queue, *status, *tables, *done, *seg_done;
    int64_t *energy, *best_energy, *accepted;
    size_t bytes;
};

// Parts a launch of `span` sweeps of the dot or table kernels splits every
// replica's sweeps into. With more replicas than resident slots, whole units
// leave the last round's idle slots idle until it ends (at n100, 4096
// replicas in 2432 slots ran at 0.85 of the full-round rate; the general
// form's table kernel, 4096 in 760 slots, at 0.94); parts run as separate
// work units of the one launch keep every slot busy to the end. Anneal,
// fixed and concurrent modes: up to 16 parts of at least 8 sweeps; PT
// launches (one exchange period each): up to 16 parts of one sweep. 1 when
// the replicas fill whole rounds, for the flow-class kernel and for tables
// in global memory.
// Whether launches of the plan may be split (the replicas exceed the slots
// and are not a whole number of rounds; dot kernel or tables in shared
// memory). It does not depend on the sweep range, so neither does the
// workspace: a resumed call over a longer range fits the workspace of the
// call before it.
bool may_split(const pdit_opts *o, const Plan &p) {
    if (p.cls || (!p.dot && !p.tsmem)) return false;  // global-table kernels take whole calls
    const long long slots = (long long)p.grid * p.groups;
    return o->replicas > slots && o->replicas % slots != 0;
}

int parts_of(const pdit_opts *o, const Plan &p, int span) {
    if (!may_split(o, p)) return 1;
    long long k = std::min(16, o->mode == PDIT_MODE_PT ? span : span / 8);
    // parts of at most 1000 sweeps, so that a part's wait for the one
    // before it stays far inside its bound however long the call
    k = std::max<long long>(k, (span + 999) / 1000);
    // the unit counter (int32, taken once more by every group at the end)
    // stays below 2^30
    k = std::min<long long>(k, (1ll << 30) / o->replicas);
    return (int)std::max<long long>(1, k);
}

// Whether the workspace holds every replica's table (the table kernels: PT
// segments and tables in global memory; `persist`: any kernel whose state is
// kept between calls by the server, the dot kernel's permuted flow matrix;
// either kernel's table between the parts of a launch).
bool needs_tables(const pdit_opts *o, const Plan &p, bool persist = false, bool whole = false) {
    return persist || o->mode == PDIT_MODE_PT || (!p.dot && !p.tsmem) || (!whole && may_split(o, p));
}

// `whole`: the caller runs every launch as whole calls (no parts), so no
// part counters or saved tables for them.
Workspace carve(const pdit_qap *h, const pdit_opts *o, const Plan &p, char *base, bool persist = false,
                bool whole = false) {
    const size_t R = (size_t)o->replicas, n = (size_t)h->n;
    size_t off = 0;
    Workspace w{};
    auto take = [&](size_t bytes) {
        char *ptr = base ? base + off : nullptr;
        off = align_up(off + bytes, kAlign);
        return ptr;
    };
    w.perm = (int32_t *)take(4 * R * n);
    w.best_perm = (int32_t *)take(4 * R * n);
    w.energy = (int64_t *)take(8 * R);
    w.best_energy = (int64_t *)take(8 * R);
    w.accepted = (int64_t *)take(8 * R);
    w.best_sweep = (int32_t *)take(4 * R);
    w.rung = (int32_t *)take(4 * R);
    const size_t nsets = o->mode == PDIT_MODE_PT && o->ladder_len > 0 ? R / (size_t)o->ladder_len : 1;
    w.since_top = (int32_t *)take(4 * nsets);
    w.queue = (int32_t *)take(4 * 64);
    w.status = (int32_t *)take(4);
    w.done = (int32_t *)take(4);
    w.seg_done = !whole && may_split(o, p) ? (int32_t *)take(4 * R) : nullptr;
    w.tables = needs_tables(o, p, persist, whole) ? (int32_t *)take(4 * R * p.table_elems) : nullptr;
    w.bytes = off;
    return w;
}

// The instance and launch-shape fields of a sweep descriptor.
void fill_shape(pdit::SweepArgs &a, const pdit_qap *h, const Plan &p) {
    a.D = h->dD;
    a.F = h->dF;
    a.n = h->n;
    a.stride = p.stride;
    a.dstride = p.dstride;
    a.zero_diag = h->zero_diag;
    a.df_bytes = p.df_bytes;
    a.group_bytes = p.group_bytes;
    a.sv_len = p.sv_len;
    a.cupim_off = p.cupim_off;
    a.v2_off = p.v2_off;
    a.rc_off = p.rc_off;
    a.groups = p.groups;
    a.cls_x = h->dx;
    a.cls_f = h->cls_f;
    a.cls_e0 = h->cls_e0;
}

// ---------------------------------------------------------------------------
// Device helpers: PT rung initialisation and exchange, final reduction.
// ---------------------------------------------------------------------------
// Reset the time-to-target outputs of one instance.
__global__ void init_target_kernel(unsigned long long *reach_ns, int *reach_sweep, int *done) {
    if (threadIdx.x == 0) {
        if (reach_ns) *reach_ns = ~0ull;
        if (reach_sweep) *reach_sweep = 0x7FFFFFFF;
        if (done) *done = 0;
    }
}

__global__ void init_pt_kernel(int replicas, int ladder, int32_t *rung, int32_t *since_top,
                               uint32_t rep_base) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < replicas) rung[r] = (int32_t)((rep_base + (uint32_t)r) % (uint32_t)ladder);
    if (r < replicas / ladder) since_top[r] = 0;
}

// One thread per set of `ladder` consecutive replicas. Rungs ascend in beta.
// For q = 0..L-2: if the replica at rung q+1 has energy >= that at rung q,
// they trade rungs. If the top rung took no part in a trade for `timeout`
// consecutive periods, top and bottom trade and the count restarts.
__global__ void pt_exchange_kernel(int nsets, int ladder, const int64_t *energy, int32_t *rung,
                                   int32_t *since_top, int timeout) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsets) return;
    int at[64];
    const int base = g * ladder;
    for (int k = 0; k < ladder; ++k) at[rung[base + k]] = k;
    bool top = false;
    for (int q = 0; q + 1 < ladder; ++q) {
        const int lo = at[q], hi = at[q + 1];
        if (energy[base + hi] >= energy[base + lo]) {
            at[q] = hi;
            at[q + 1] = lo;
            if (q + 1 == ladder - 1) top = true;
        }
    }
    int c = top ? 0 : since_top[g] + 1;
    if (timeout > 0 && c >= timeout) {
        const int t = at[ladder - 1];
        at[ladder - 1] = at[0];
        at[0] = t;
        c = 0;
    }
    since_top[g] = c;
    for (int q = 0; q < ladder; ++q) rung[base + at[q]] = q;
}

// Smallest best energy over replicas, ties to the lowest index; copies the
// winner's permutation. One block.
__global__ void finalize_kernel(int replicas, int n, const int64_t *best_energy,
                                const int32_t *best_perm, int32_t *out_perm, int64_t *out_cost,
                                const int32_t *status_in, int32_t *status_out) {
    __shared__ long long sval[32];
    __shared__ int sidx[32];
    __shared__ int winner;
    long long v = 0x7FFFFFFFFFFFFFFFll;
    int idx = 0x7FFFFFFF;
    for (int r = threadIdx.x; r < replicas; r += blockDim.x) {
        const long long e = best_energy[r];
        if (e < v || (e == v && r < idx)) {
            v = e;
            idx = r;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        const int oi = __shfl_xor_sync(0xFFFFFFFFu, idx, o);
        if (ov < v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sval[warp] = v;
        sidx[warp] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) / 32;
        long long bv = sval[0];
        int bi = sidx[0];
        for (int w = 1; w < nw; ++w)
            if (sval[w] < bv || (sval[w] == bv && sidx[w] < bi)) {
                bv = sval[w];
                bi = sidx[w];
            }
        winner = bi;
        *out_cost = bv;
        if (status_out) *status_out = *status_in;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < n; m += blockDim.x) out_perm[m] = best_perm[(size_t)winner * n + m];
}

// Two-level flow (the Methods section's tai256c structure): D symmetric with a
// zero diagonal and F[c][d] = f0 + f x_c x_d for every c != d with x_c in
// {0, 1}. Fills x, f0, f and returns true when (D, F) has this form.
bool detect_flow_classes(int n, const int32_t *D, const int32_t *F, std::vector<uint8_t> &x, int64_t &f0,
                         int64_t &f) {
    for (int i = 0; i < n; ++i) {
        if (D[(size_t)i * n + i] != 0) return false;
        for (int j = i + 1; j < n; ++j)
            if (D[(size_t)i * n + j] != D[(size_t)j * n + i]) return false;
    }
    int64_t v[2] = {0, 0};
    int nv = 0;
    for (int c = 0; c < n; ++c)
        for (int d = 0; d < n; ++d) {
            if (c == d) continue;
            const int64_t val = F[(size_t)c * n + d];
            if (nv > 0 && val == v[0]) continue;
            if (nv > 1 && val == v[1]) continue;
            if (nv == 2) return false;
            v[nv++] = val;
        }
    x.assign((size_t)n, 0);
    if (nv == 1) {
        f0 = v[0];
        f = 0;
        return true;
    }
    for (int pick = 0; pick < 2; ++pick) {
        const int64_t in = v[pick], out = v[1 - pick];
        for (int c = 0; c < n; ++c) {
            x[c] = 0;
            for (int d = 0; d < n; ++d)
                if (d != c && F[(size_t)c * n + d] == in) x[c] = 1;
        }
        bool ok = true;
        for (int c = 0; c < n && ok; ++c)
            for (int d = 0; d < n; ++d)
                if (d != c && F[(size_t)c * n + d] != ((x[c] && x[d]) ? in : out)) {
                    ok = false;
                    break;
                }
        if (ok) {
            f0 = out;
            f = in - out;
            return true;
        }
    }
    return false;
}

int validate_opts(const pdit_qap *h, const pdit_opts *o) {
    if (!h || !o) return PDIT_EINVAL;
    if (o->struct_size != sizeof(pdit_opts)) return PDIT_EINVAL;
    if (o->replicas < 1 || o->sweeps < 0) return PDIT_EINVAL;
    const int se = o->sweep_end < 0 ? o->sweeps : o->sweep_end;
    if (o->sweep_begin < 0 || se < o->sweep_begin || se > o->sweeps) return PDIT_EINVAL;
    if ((uint64_t)o->sweeps >= 0xFFFFFFFFull) return PDIT_EINVAL;
    if (!o->best_perm || !o->best_cost) return PDIT_EINVAL;
    if (se > o->sweep_begin && !o->beta) return PDIT_EINVAL;
    if (o->mode < PDIT_MODE_ANNEAL || o->mode > PDIT_MODE_CUPIM) return PDIT_EINVAL;
    if (o->mode == PDIT_MODE_PT) {
        if (o->ladder_len < 2 || o->ladder_len > 64 || o->replicas % o->ladder_len) return PDIT_EINVAL;
        if (o->exchange_period < 1 || o->timeout_periods < 0) return PDIT_EINVAL;
        if (o->replica_base % (uint32_t)o->ladder_len) return PDIT_EINVAL;
    }
    if (!(o->flags & PDIT_FLAG_RESUME) && o->sweep_begin != 0) return PDIT_EINVAL;
    return PDIT_OK;
}

}  // namespace

extern "C" {

const char *pdit_strerror(int code) {
    switch (code) {
    case PDIT_OK: return "success";
    case PDIT_EINVAL: return "invalid argument";
    case PDIT_ERANGE: return "instance values too large for exact int32 influence arithmetic";
    case PDIT_ENOMEM: return "out of memory or workspace too small";
    case PDIT_ECUDA: return "CUDA runtime error";
    case PDIT_EDEVICE: return "device consistency audit failed";
    case PDIT_ENOTSUP: return "not supported by the compiled kernels";
    case PDIT_EIO: return "file could not be opened, read or written";
    default: return "unknown error";
    }
}

const char *pdit_last_error(void) { return g_last_error.c_str(); }

void pdit_opts_init(pdit_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(pdit_opts);
    o->sweep_end = -1;
    o->mode = PDIT_MODE_ANNEAL;
    o->exchange_period = 4;
    o->timeout_periods = 100;
}

}  // extern "C"

// Host side of qap_create: validation, the instance form, the staging
// width and the device attributes; no device memory yet.
int qap_prepare(int n, const int32_t *D, const int32_t *F, pdit_qap **out) {
    if (!out) return PDIT_EINVAL;
    *out = nullptr;
    if (n < 2 || n > PDIT_N_MAX || !D || !F) return PDIT_EINVAL;
    int64_t maxd = 0, maxf = 0;
    int64_t dlo = D[0], dhi = D[0], flo = F[0], fhi = F[0];
    bool zd = true, asym = false;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const int32_t d = D[(size_t)i * n + j], f = F[(size_t)i * n + j];
            if (d != D[(size_t)j * n + i] || f != F[(size_t)j * n + i]) asym = true;
            dlo = std::min<int64_t>(dlo, d);
            dhi = std::max<int64_t>(dhi, d);
            flo = std::min<int64_t>(flo, f);
            fhi = std::max<int64_t>(fhi, f);
            maxd = std::max<int64_t>(maxd, std::llabs((long long)d));
            maxf = std::max<int64_t>(maxf, std::llabs((long long)f));
            if (i == j && (d != 0 || f != 0)) zd = false;
        }
    // |I| <= n maxD maxF (general form: |T| <= 2 n maxD maxF), |dE| <= 8 n
    // maxD maxF + 16 maxD maxF, and shifted energies span twice that: all of
    // it stays inside int32.
    if ((int64_t)16 * (n + 2) * maxd * maxf >= ((int64_t)1 << 31)) return PDIT_ERANGE;
    pdit_qap *h = new (std::nothrow) pdit_qap();
    if (!h) return PDIT_ENOMEM;
    h->n = n;
    h->zero_diag = zd ? 1 : 0;
    h->asym = asym ? 1 : 0;
    std::vector<uint8_t> cx;
    int64_t f0 = 0, fcls = 0;
    if (!asym && detect_flow_classes(n, D, F, cx, f0, fcls)) {
        int64_t dsum = 0;
        for (size_t k = 0; k < (size_t)n * n; ++k) dsum += D[k];
        h->cls = 1;
        h->cls_f = (int)fcls;
        h->cls_e0 = f0 * dsum;  // D's diagonal is zero
    }
    h->packed_ok = (dhi - dlo <= 127 && fhi - flo <= 127) ? 1 : 0;
    const int64_t mx = std::max(maxd, maxf);
    h->dt_bytes = mx <= 127 ? 1 : (mx <= 32767 ? 2 : 4);
    h->hD.assign(D, D + (size_t)n * n);
    h->hF.assign(F, F + (size_t)n * n);
    cudaError_t e = cudaGetDevice(&h->device);
    int v = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->smem_optin = (size_t)v;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, h->device);
    h->l2_bytes = (size_t)v;
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "qap_create");
        delete h;
        return rc;
    }
    h->cls_x.assign(cx.begin(), cx.end());
    *out = h;
    return PDIT_OK;
}

extern "C" {

int qap_create(int n, const int32_t *D, const int32_t *F, pdit_qap **out) {
    int rc = qap_prepare(n, D, F, out);
    if (rc) return rc;
    pdit_qap *h = *out;
    *out = nullptr;
    const size_t bytes = sizeof(int32_t) * (size_t)n * n;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->dD, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->dF, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(h->dD, D, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->dF, F, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h->cls) {
        e = cudaMalloc((void **)&h->dx, (size_t)n);
        if (e == cudaSuccess) e = cudaMemcpy(h->dx, h->cls_x.data(), (size_t)n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        const int rc = (e == cudaErrorMemoryAllocation) ? PDIT_ENOMEM : cuda_fail(e, "qap_create");
        qap_destroy(h);
        return rc;
    }
    *out = h;
    return PDIT_OK;
}

void qap_destroy(pdit_qap *h) {
    if (!h) return;
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    if (have && cur != h->device) cudaSetDevice(h->device);
    if (h->stream) cudaStreamDestroy(h->stream);
    cudaFree(h->dD);
    cudaFree(h->dF);
    cudaFree(h->dx);
    cudaFree(h->ws);
    cudaFree(h->dbeta);
    cudaFree(h->dperm);
    cudaFree(h->dcost);
    cudaFree(h->dstatus);
    if (have && cur != h->device) cudaSetDevice(cur);
    delete h;
}

int qap_n(const pdit_qap *h) { return h ? h->n : PDIT_EINVAL; }

int pdit_set_warps_per_replica(pdit_qap *h, int wpr) {
    if (!h || wpr < 0 || wpr > 8 || (wpr & (wpr - 1))) return PDIT_EINVAL;
    if (wpr > cover_for(h->n) / 32) return PDIT_EINVAL;
    h->force_wpr = wpr;
    return PDIT_OK;
}

int pdit_launch_shape(const pdit_qap *h, int replicas, int *shape) {
    if (!h || replicas < 1 || !shape) return PDIT_EINVAL;
    Plan p;
    pdit_opts o;
    pdit_opts_init(&o);
    o.replicas = replicas;
    const int rc = plan_for(h, &o, &p);
    if (rc) return rc;
    shape[0] = p.wpr;
    shape[1] = p.maxk;
    shape[2] = p.groups;
    shape[3] = p.grid;
    shape[4] = p.dot ? 2 : (p.tsmem ? 1 : 0);
    shape[5] = (int)p.smem;
    shape[6] = p.pk;
    return PDIT_OK;
}

int pdit_instance_form(const pdit_qap *h) {
    if (!h) return PDIT_EINVAL;
    if (h->cls) return PDIT_FORM_FLOW_CLASSES;
    return h->asym ? PDIT_FORM_GENERAL : PDIT_FORM_SYMMETRIC;
}

int pdit_set_class_update(pdit_qap *h, int enable) {
    if (!h || (enable != 0 && enable != 1)) return PDIT_EINVAL;
    h->use_cls = enable;
    return PDIT_OK;
}

int pdit_set_table_placement(pdit_qap *h, int place) {
    if (!h || place < PDIT_PLACE_AUTO || place > PDIT_PLACE_GLOBAL) return PDIT_EINVAL;
    h->force_place = place;
    return PDIT_OK;
}

int pdit_set_replicas_per_cta(pdit_qap *h, int g) {
    if (!h || g < 0) return PDIT_EINVAL;
    h->force_groups = g;
    return PDIT_OK;
}

int pdit_set_influence(pdit_qap *h, int mode) {
    if (!h || mode < PDIT_INFLUENCE_AUTO || mode > PDIT_INFLUENCE_PRODUCTS) return PDIT_EINVAL;
    h->force_infl = mode;
    return PDIT_OK;
}

int pdit_set_pending_swaps(pdit_qap *h, int k) {
    if (!h || (k != 0 && k != 1 && k != 4 && k != 16)) return PDIT_EINVAL;
    h->force_pk = k;
    return PDIT_OK;
}

size_t pdit_workspace_bytes(const pdit_qap *h, const pdit_opts *o) {
    if (!h || !o || o->replicas < 1) return 0;
    Plan p;
    if (plan_for(h, o, &p) != PDIT_OK) return 0;
    return carve(h, o, p, nullptr).bytes;
}

int pdit_anneal_ex(pdit_qap *h, const pdit_opts *o) {
    int rc = validate_opts(h, o);
    if (rc) return rc;
    Plan plan;
    rc = plan_for(h, o, &plan);
    if (rc) return rc;
    const size_t need = carve(h, o, plan, nullptr).bytes;
    char *base = (char *)o->workspace;
    if (base) {
        if (o->workspace_bytes < need) return PDIT_ENOMEM;
    } else {
        if (h->ws_bytes < need) {
            if (o->flags & PDIT_FLAG_RESUME) return PDIT_EINVAL;  // no state to resume from
            cudaFree(h->ws);
            h->ws = nullptr;
            h->ws_bytes = 0;
            cudaError_t e = cudaMalloc(&h->ws, need);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PDIT_ENOMEM : cuda_fail(e, "workspace");
            h->ws_bytes = need;
        }
        base = (char *)h->ws;
    }
    const Workspace w = carve(h, o, plan, base);
    cudaStream_t st = (cudaStream_t)o->stream;
    const bool resume = (o->flags & PDIT_FLAG_RESUME) != 0;
    const int sb = o->sweep_begin;
    const int se = o->sweep_end < 0 ? o->sweeps : o->sweep_end;
    const int R = o->replicas;
    const bool pt = o->mode == PDIT_MODE_PT;

    if (!resume) {
        PDIT_CK(cudaMemsetAsync(w.status, 0, sizeof(int32_t), st));
        if (o->target) {
            init_target_kernel<<<1, 32, 0, st>>>((unsigned long long *)o->reach_ns, o->reach_sweep, w.done);
            PDIT_CK(cudaGetLastError());
        }
        if (pt) {
            init_pt_kernel<<<(R + 255) / 256, 256, 0, st>>>(R, o->ladder_len, w.rung, w.since_top,
                                                            o->replica_base);
            PDIT_CK(cudaGetLastError());
        }
    }

    pdit::SweepArgs a{};
    fill_shape(a, h, plan);
    a.replicas = R;
    a.key0 = (uint32_t)o->seed;
    a.key1 = (uint32_t)(o->seed >> 32);
    a.inst = o->instance_id;
    a.rep_base = o->replica_base;
    a.mode = o->mode;
    a.beta = o->beta;
    a.perm = w.perm;
    a.best_perm = w.best_perm;
    a.energy = w.energy;
    a.best_energy = w.best_energy;
    a.best_sweep = w.best_sweep;
    a.accepted = w.accepted;
    a.rung = w.rung;
    a.tables = w.tables;
    a.queue = w.queue;
    a.status = w.status;
    a.target = o->target;
    a.reach_ns = (unsigned long long *)o->reach_ns;
    a.reach_sweep = o->reach_sweep;
    a.done = o->target ? w.done : nullptr;
    a.stop = (o->target && o->stop_at_target) ? 1 : 0;
    a.seg_done = w.seg_done;

    // Segments: the whole range in anneal mode; exchange periods in PT mode.
    bool first = true;
    int s = sb;
    do {
        int next = se;
        if (pt) next = std::min(se, (s / o->exchange_period + 1) * o->exchange_period);
        a.sweep_begin = s;
        a.sweep_end = next;
        a.fresh = (!resume && first) ? 1 : 0;
        // Tables (the dot kernel: permuted flow matrices) persist from one
        // PT segment to the next within a call. The first segment of every
        // call rebuilds them from the permutation (exact integers, so equal
        // to what was saved), so a resumed call does not depend on which
        // kernel or mode ran before it.
        a.table_in = (pt && !first) ? 1 : 0;
        a.table_out = (pt && next < se) ? 1 : 0;
        a.dump = (next == se) ? o->tables : nullptr;
        a.segments = parts_of(o, plan, next - s);
        if (!(first && resume && s == se)) {
            PDIT_CK(cudaMemsetAsync(w.queue, 0, sizeof(int32_t), st));
            if (a.segments > 1) PDIT_CK(cudaMemsetAsync(w.seg_done, 0, sizeof(int32_t) * R, st));
            const int e = plan.cls ? class_launch(h->dt_bytes, plan, a, st)
                        : plan.dot ? pdit::dot_launch(plan.maxk, plan.wpr, a, plan.grid, plan.threads, plan.smem, st)
                                   : sweep_launch(h->dt_bytes, h->asym != 0, plan, a, st);
            if (e != 0) return cuda_fail((cudaError_t)e, "sweep kernel launch");
        }
        if (pt && next < se + 1 && next % o->exchange_period == 0 && next > s) {
            const int nsets = R / o->ladder_len;
            pt_exchange_kernel<<<(nsets + 127) / 128, 128, 0, st>>>(nsets, o->ladder_len, w.energy, w.rung,
                                                                   w.since_top, o->timeout_periods);
            PDIT_CK(cudaGetLastError());
        }
        first = false;
        s = next;
    } while (s < se);

    finalize_kernel<<<1, 1024, 0, st>>>(R, h->n, w.best_energy, w.best_perm, o->best_perm, o->best_cost,
                                        w.status, o->status);
    PDIT_CK(cudaGetLastError());
    const size_t n = (size_t)h->n;
    if (o->replica_best_cost)
        PDIT_CK(cudaMemcpyAsync(o->replica_best_cost, w.best_energy, 8 * R, cudaMemcpyDeviceToDevice, st));
    if (o->replica_best_perm)
        PDIT_CK(cudaMemcpyAsync(o->replica_best_perm, w.best_perm, 4 * R * n, cudaMemcpyDeviceToDevice, st));
    if (o->replica_best_sweep)
        PDIT_CK(cudaMemcpyAsync(o->replica_best_sweep, w.best_sweep, 4 * R, cudaMemcpyDeviceToDevice, st));
    if (o->replica_final_perm)
        PDIT_CK(cudaMemcpyAsync(o->replica_final_perm, w.perm, 4 * R * n, cudaMemcpyDeviceToDevice, st));
    if (o->replica_final_cost)
        PDIT_CK(cudaMemcpyAsync(o->replica_final_cost, w.energy, 8 * R, cudaMemcpyDeviceToDevice, st));
    if (o->replica_accepted)
        PDIT_CK(cudaMemcpyAsync(o->replica_accepted, w.accepted, 8 * R, cudaMemcpyDeviceToDevice, st));
    if (o->replica_rung && pt)
        PDIT_CK(cudaMemcpyAsync(o->replica_rung, w.rung, 4 * R, cudaMemcpyDeviceToDevice, st));
    return PDIT_OK;
}

int pdit_anneal(pdit_qap *h, int replicas, const float *beta_schedule, int sweeps, uint64_t seed,
                int32_t *best_perm, int64_t *best_cost) {
    if (!h || replicas < 1 || sweeps < 0 || !best_perm || !best_cost) return PDIT_EINVAL;
    if (sweeps > 0 && !beta_schedule) return PDIT_EINVAL;
    for (int s = 0; s < sweeps; ++s)
        if (!(beta_schedule[s] >= 0.0f) || !std::isfinite(beta_schedule[s])) return PDIT_EINVAL;
    if (!h->stream) PDIT_CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    if (!h->dperm) PDIT_CK(cudaMalloc((void **)&h->dperm, sizeof(int32_t) * h->n));
    if (!h->dcost) PDIT_CK(cudaMalloc((void **)&h->dcost, sizeof(int64_t)));
    if (!h->dstatus) PDIT_CK(cudaMalloc((void **)&h->dstatus, sizeof(int32_t)));
    const size_t nb = (size_t)std::max(sweeps, 1);
    if (h->dbeta_cap < nb) {
        cudaFree(h->dbeta);
        h->dbeta = nullptr;
        h->dbeta_cap = 0;
        PDIT_CK(cudaMalloc((void **)&h->dbeta, sizeof(float) * nb));
        h->dbeta_cap = nb;
    }
    if (sweeps > 0)
        PDIT_CK(cudaMemcpyAsync(h->dbeta, beta_schedule, sizeof(float) * sweeps, cudaMemcpyHostToDevice,
                                h->stream));
    pdit_opts o;
    pdit_opts_init(&o);
    o.replicas = replicas;
    o.sweeps = sweeps;
    o.seed = seed;
    o.beta = h->dbeta;
    o.stream = h->stream;
    o.best_perm = h->dperm;
    o.best_cost = h->dcost;
    o.status = h->dstatus;
    int rc = pdit_anneal_ex(h, &o);
    if (rc) return rc;
    int32_t status = 0;
    PDIT_CK(cudaMemcpyAsync(best_perm, h->dperm, sizeof(int32_t) * h->n, cudaMemcpyDeviceToHost, h->stream));
    PDIT_CK(cudaMemcpyAsync(best_cost, h->dcost, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    PDIT_CK(cudaMemcpyAsync(&status, h->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    PDIT_CK(cudaStreamSynchronize(h->stream));
    return status ? PDIT_EDEVICE : PDIT_OK;
}

int pdit_beta_max(const pdit_qap *h, double *beta_max) {
    if (!h || !beta_max) return PDIT_EINVAL;
    const int n = h->n;
    const int32_t *D = h->hD.data(), *F = h->hF.data();
    // Identity permutation: T[m][c] = sum_j D[m][j] F[c][j] + D[j][m] F[j][c]
    // (the two-term table; 2 I for symmetric D and F).
    std::vector<int64_t> T((size_t)n * n, 0);
    for (int m = 0; m < n; ++m)
        for (int j = 0; j < n; ++j) {
            const int64_t d_out = D[(size_t)m * n + j], d_in = D[(size_t)j * n + m];
            if (!d_out && !d_in) continue;
            for (int c = 0; c < n; ++c)
                T[(size_t)m * n + c] += d_out * F[(size_t)c * n + j] + d_in * F[(size_t)j * n + c];
        }
    double sum = 0.0;
    long long cnt = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            // Eq. 3 with a = i, b = j (identity permutation).
            const int64_t t = T[(size_t)i * n + j] - T[(size_t)i * n + i] + T[(size_t)j * n + i] -
                              T[(size_t)j * n + j];
            const int64_t dd = (int64_t)D[(size_t)i * n + i] + D[(size_t)j * n + j] - D[(size_t)i * n + j] -
                               D[(size_t)j * n + i];
            const int64_t ff = (int64_t)F[(size_t)i * n + i] + F[(size_t)j * n + j] - F[(size_t)i * n + j] -
                               F[(size_t)j * n + i];
            const int64_t de = t + dd * ff;
            if (de > 0) {
                sum += (double)de;
                ++cnt;
            }
        }
    *beta_max = cnt ? 10.0 / (sum / (double)cnt) : 1.0;
    return PDIT_OK;
}

int pdit_autotune(pdit_qap *h, int replicas, const float *beta, int sweeps, int *shape) {
    if (!h || replicas < 1 || sweeps < 1 || !beta) return PDIT_EINVAL;
    if (!h->stream) PDIT_CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    struct Knobs {
        int place, wpr, pk, groups, infl;
    };
    const Knobs keep{h->force_place, h->force_wpr, h->force_pk, h->force_groups, h->force_infl};
    auto set = [h](const Knobs &k) {
        h->force_place = k.place;
        h->force_wpr = k.wpr;
        h->force_pk = k.pk;
        h->force_groups = k.groups;
        h->force_infl = k.infl;
    };
    const bool cls = h->cls && h->use_cls;
    auto plan_ok = [&](const Knobs &k, Plan *p) {
        set(k);
        if (cls) return make_class_plan(h, replicas, k.wpr, p) == PDIT_OK;
        if (k.infl == PDIT_INFLUENCE_PRODUCTS) return make_dot_plan(h, replicas, k.wpr, p) == PDIT_OK;
        return make_plan(h, replicas, k.wpr, k.pk, p) == PDIT_OK;
    };
    // Candidates: the table placement (a caller's choice, else the built-in
    // one and, where that keeps the tables in shared memory, global memory),
    // every warps-per-replica and pending-term count, and replicas per CTA =
    // the built-in choice plus 1..4 where the tables live in global memory
    // (there the built-in choice is an L2-capacity estimate). The flow-class
    // kernel keeps no table: only its warps per replica vary.
    // The dot-product kernel (eligible instances, unless the caller fixed the
    // table) adds its compiled warps-per-replica shapes.
    std::vector<Knobs> cand;
    const int cover = cover_for(h->n);
    const int tbl = cls ? keep.infl : (int)PDIT_INFLUENCE_TABLE;
    if (!cls && dot_eligible(h) && keep.infl != PDIT_INFLUENCE_TABLE)
        for (int wpr = 1; wpr <= cover / 32 && wpr <= 8; wpr <<= 1) {
            Plan p;
            if (plan_ok({0, wpr, 0, 0, (int)PDIT_INFLUENCE_PRODUCTS}, &p)) cand.push_back(
                {0, wpr, 0, 0, (int)PDIT_INFLUENCE_PRODUCTS});
        }
    for (int place : {keep.place, (int)PDIT_PLACE_GLOBAL}) {
        if (keep.infl == PDIT_INFLUENCE_PRODUCTS && !cls) break;
        if (place == PDIT_PLACE_GLOBAL && (keep.place != 0 || cls)) continue;
        for (int wpr = 1; wpr <= cover / 32 && wpr <= 8; wpr <<= 1)
            for (int pk : {1, 4, 16}) {
                if (cls && pk != 1) continue;
                Plan p;
                if (!plan_ok({place, wpr, pk, 0, tbl}, &p)) continue;
                if (place == PDIT_PLACE_GLOBAL) {
                    Plan q;
                    if (plan_ok({0, wpr, pk, 0, tbl}, &q) && !q.tsmem) continue;  // already the built-in choice
                }
                cand.push_back({place, wpr, pk, 0, tbl});
                if (!cls && !p.tsmem)
                    for (int g = 1; g <= 4; ++g)
                        if (g != p.groups) cand.push_back({place, wpr, pk, g, tbl});
            }
    }
    int32_t *dperm = nullptr;
    int64_t *dcost = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void **)&dperm, sizeof(int32_t) * h->n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dcost, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = PDIT_OK, best = -1;
    float best_ms = 0.0f;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess && rc == PDIT_OK; ++c) {
        set(cand[c]);
        pdit_opts o;
        pdit_opts_init(&o);
        o.replicas = replicas;
        o.sweeps = sweeps;
        o.seed = 0x5EED;
        o.beta = beta;
        o.stream = h->stream;
        o.best_perm = dperm;
        o.best_cost = dcost;
        rc = pdit_anneal_ex(h, &o);  // warm-up (and workspace)
        if (rc) break;
        e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess) rc = pdit_anneal_ex(h, &o);
        if (e == cudaSuccess && !rc) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess && !rc) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess && !rc) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && !rc && (best < 0 || ms < best_ms)) {
            best_ms = ms;
            best = (int)c;
        }
    }
    cudaFree(dperm);
    cudaFree(dcost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc || e != cudaSuccess || best < 0) {
        set(keep);
        if (rc) return rc;
        return e != cudaSuccess ? cuda_fail(e, "pdit_autotune") : PDIT_ENOTSUP;
    }
    set(cand[best]);
    if (shape) {
        shape[0] = cand[best].wpr;
        shape[1] = cand[best].infl == PDIT_INFLUENCE_PRODUCTS ? 1 : cand[best].pk;  // no pending terms
    }
    return PDIT_OK;
}

int pdit_beta_ladder(double beta_lo, double beta_hi, int len, float *out) {
    if (len < 1 || !out || !(beta_lo > 0.0) || !(beta_hi >= beta_lo) || !std::isfinite(beta_hi))
        return PDIT_EINVAL;
    for (int q = 0; q < len; ++q) {
        const double f = len > 1 ? (double)q / (double)(len - 1) : 0.0;
        out[q] = (float)(beta_lo * std::pow(beta_hi / beta_lo, f));
    }
    return PDIT_OK;
}

int pdit_beta_range(pdit_qap *h, int points, double beta_min, double beta_max, int replicas_per_point,
                    int sweeps, uint64_t seed, double *beta_lo, double *beta_hi, double *curve) {
    if (!h || points < 3 || replicas_per_point < 1 || sweeps < 1 || !beta_lo || !beta_hi) return PDIT_EINVAL;
    if ((int64_t)points * replicas_per_point > (1 << 24)) return PDIT_EINVAL;
    if (!(beta_min > 0.0) || !(beta_max > beta_min) || !std::isfinite(beta_max)) {
        double b = 0.0;
        const int rc = pdit_beta_max(h, &b);
        if (rc) return rc;
        beta_min = b / 1000.0;
        beta_max = b * 10.0;
    }
    std::vector<float> grid((size_t)points);
    for (int k = 0; k < points; ++k)
        grid[k] = (float)(beta_min * std::pow(beta_max / beta_min, (double)k / (double)(points - 1)));
    const int R = points * replicas_per_point;
    std::vector<float> rbeta((size_t)R);
    for (int r = 0; r < R; ++r) rbeta[r] = grid[r / replicas_per_point];
    if (!h->stream) PDIT_CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    // Temporary device buffers: betas, final costs, best permutation, best cost.
    float *dbeta = nullptr;
    int64_t *dfinal = nullptr, *dcost = nullptr;
    int32_t *dperm = nullptr;
    cudaError_t e = cudaMalloc((void **)&dbeta, sizeof(float) * R);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dfinal, sizeof(int64_t) * R);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dcost, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&dperm, sizeof(int32_t) * h->n);
    std::vector<int64_t> fin((size_t)R);
    int rc = PDIT_OK;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dbeta, rbeta.data(), sizeof(float) * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        pdit_opts o;
        pdit_opts_init(&o);
        o.replicas = R;
        o.sweeps = sweeps;
        o.seed = seed;
        o.mode = PDIT_MODE_FIXED;
        o.beta = dbeta;
        o.stream = h->stream;
        o.best_perm = dperm;
        o.best_cost = dcost;
        o.replica_final_cost = dfinal;
        rc = pdit_anneal_ex(h, &o);
        if (!rc) e = cudaMemcpyAsync(fin.data(), dfinal, sizeof(int64_t) * R, cudaMemcpyDeviceToHost, h->stream);
        if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    cudaFree(dbeta);
    cudaFree(dfinal);
    cudaFree(dcost);
    cudaFree(dperm);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "pdit_beta_range");
    // Mean ending energy per beta; lowest beta: the first point whose mean has
    // come down to 40% of the way from the smallest to the largest mean;
    // highest beta: two points past the smallest mean (clamped to the grid).
    std::vector<double> mean((size_t)points, 0.0);
    for (int r = 0; r < R; ++r) mean[r / replicas_per_point] += (double)fin[r];
    for (int k = 0; k < points; ++k) mean[k] /= (double)replicas_per_point;
    int kmin = 0, kmax = 0;
    for (int k = 1; k < points; ++k) {
        if (mean[k] < mean[kmin]) kmin = k;
        if (mean[k] > mean[kmax]) kmax = k;
    }
    const double thr = mean[kmin] + 0.4 * (mean[kmax] - mean[kmin]);
    int klo = kmin;
    for (int k = 0; k < points; ++k)
        if (mean[k] <= thr) {
            klo = k;
            break;
        }
    const int khi = std::min(kmin + 2, points - 1);
    *beta_lo = (double)grid[klo];
    *beta_hi = (double)grid[khi];
    if (curve)
        for (int k = 0; k < points; ++k) curve[k] = mean[k];
    return PDIT_OK;
}

int pdit_beta_schedule(int kind, int sweeps, double beta_max, float *out) {
    if (sweeps < 0 || (sweeps > 0 && !out) || (kind != 0 && kind != 1)) return PDIT_EINVAL;
    if (!(beta_max >= 0.0) || !std::isfinite(beta_max)) return PDIT_EINVAL;
    for (int s = 0; s < sweeps; ++s) {
        const double f = sweeps > 1 ? (double)s / (double)(sweeps - 1) : 1.0;
        const double b = kind == 0 ? beta_max * f : (beta_max / 1000.0) * std::pow(1000.0, f);
        out[s] = (float)b;
    }
    return PDIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point. Its scratch (the per-replica state that
// pdit_anneal_ex keeps in a workspace) is this file-scope device array, so
// the call never allocates device memory. In host code `g_noalloc_scratch`
// names a host-side stand-in, not a device address: the address is taken
// with cudaGetSymbolAddress on every call, with the caller's device current
// (a lookup once the module is loaded; taking it afresh keeps a context
// that was torn down and recreated from writing through a stale address).
// ---------------------------------------------------------------------------
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[PDIT_NOALLOC_SCRATCH_BYTES];

int noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = p;
    return PDIT_OK;
}

}  // namespace

extern "C" {

int pdit_anneal_noalloc(int n, const int32_t *D, const int32_t *F, int replicas, const float *beta,
                        int sweeps, uint64_t seed, int32_t *best_perm, int64_t *best_cost,
                        int32_t *status, void *stream) {
    if (n < 2 || n > PDIT_N_MAX || !D || !F || replicas < 1 || sweeps < 0) return PDIT_EINVAL;
    if (!best_perm || !best_cost || (sweeps > 0 && !beta)) return PDIT_EINVAL;
    if ((uint64_t)sweeps >= 0xFFFFFFFFull) return PDIT_EINVAL;
    // A stand-in instance description on the stack: D and F are read as
    // int32 with the general (any diagonal) swap energy and immediate table
    // updates, since their values are not inspected on the host here.
    pdit_qap q;
    q.n = n;
    q.dt_bytes = 4;
    q.zero_diag = 0;
    q.packed_ok = 0;
    q.dD = const_cast<int32_t *>(D);
    q.dF = const_cast<int32_t *>(F);
    int v = 0;
    PDIT_CK(cudaGetDevice(&q.device));
    PDIT_CK(cudaDeviceGetAttribute(&q.num_sms, cudaDevAttrMultiProcessorCount, q.device));
    PDIT_CK(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, q.device));
    q.smem_optin = (size_t)v;
    pdit_opts o;
    pdit_opts_init(&o);
    o.replicas = replicas;
    o.sweeps = sweeps;
    o.seed = seed;
    o.beta = beta;
    o.stream = stream;
    o.best_perm = best_perm;
    o.best_cost = best_cost;
    Plan plan;
    int rc = make_plan(&q, replicas, 0, 1, &plan);
    q.dD = q.dF = nullptr;  // not owned: nothing for ~pdit_qap to release
    if (rc) return rc;
    if (!plan.tsmem) return PDIT_ENOTSUP;
    const Workspace need = carve(&q, &o, plan, nullptr, false, true);  // whole calls only
    if (need.bytes > (size_t)PDIT_NOALLOC_SCRATCH_BYTES) return PDIT_ENOMEM;
    void *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    const Workspace w = carve(&q, &o, plan, (char *)scratch, false, true);
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: reset the status word
    // and the work counter; every replica's state is rewritten from scratch.
    PDIT_CK(cudaMemsetAsync(w.status, 0, sizeof(int32_t), st));
    PDIT_CK(cudaMemsetAsync(w.queue, 0, sizeof(int32_t), st));
    pdit::SweepArgs a{};
    a.D = D;
    a.F = F;
    a.n = n;
    a.stride = plan.stride;
    a.zero_diag = 0;
    a.replicas = replicas;
    a.sweep_begin = 0;
    a.sweep_end = sweeps;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.beta = beta;
    a.fresh = 1;
    a.perm = w.perm;
    a.best_perm = w.best_perm;
    a.energy = w.energy;
    a.best_energy = w.best_energy;
    a.best_sweep = w.best_sweep;
    a.accepted = w.accepted;
    a.rung = w.rung;
    a.queue = w.queue;
    a.status = w.status;
    a.df_bytes = plan.df_bytes;
    a.group_bytes = plan.group_bytes;
    a.sv_len = plan.sv_len;
    const int e = sweep_launch(4, false, plan, a, st);
    if (e != 0) return cuda_fail((cudaError_t)e, "sweep kernel launch");
    // the audit bits reach the caller through `status` when given
    finalize_kernel<<<1, 1024, 0, st>>>(replicas, n, w.best_energy, w.best_perm, best_perm, best_cost,
                                        w.status, status);
    PDIT_CK(cudaGetLastError());
    return PDIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Multi-instance batches.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kBatchStaticSmem = 512;
// the multi-instance kernel's static shared memory: its descriptor and a unit index
static_assert(sizeof(pdit::SweepArgs) + sizeof(int) + 16 <= kBatchStaticSmem,
              "batch kernel descriptor exceeds the static shared-memory reserve");

struct BatchOut {
    int32_t *perm;
    int64_t *cost;
    int n, replicas;
    const int64_t *best_energy;
    const int32_t *best_perm;
};

struct BatchClass {
    int dt = 1, maxk = 1, wpr = 1, pk = 1;
    bool tsmem = true, asym = false, dot = false;
    int threads = 32, grid = 1, nunits = 0;
    size_t smem = 0;
    std::vector<int> items;
    pdit::BatchUnit *d_units = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

template <bool ASYM>
int batch_blocks_t(const BatchClass &c, int *blocks) {
    if (c.dt == 1) return pdit::batch_blocks_per_sm<int8_t, ASYM>(c.maxk, c.wpr, c.tsmem, c.pk, c.threads, c.smem, blocks);
    if (c.dt == 2) return pdit::batch_blocks_per_sm<int16_t, ASYM>(c.maxk, c.wpr, c.tsmem, c.pk, c.threads, c.smem, blocks);
    return pdit::batch_blocks_per_sm<int32_t, ASYM>(c.maxk, c.wpr, c.tsmem, c.pk, c.threads, c.smem, blocks);
}

int batch_blocks(const BatchClass &c, int *blocks) {
    if (c.dot) return pdit::dot_batch_blocks_per_sm(c.maxk, c.wpr, c.threads, c.smem, blocks);
    return c.asym ? batch_blocks_t<true>(c, blocks) : batch_blocks_t<false>(c, blocks);
}

template <bool ASYM>
int batch_launch_t(const BatchClass &c, const pdit::SweepArgs *descs, int *queue) {
    if (c.dt == 1)
        return pdit::batch_launch<int8_t, ASYM>(c.maxk, c.wpr, c.tsmem, c.pk, descs, c.d_units, c.nunits, queue,
                                                c.grid, c.threads, c.smem, c.stream);
    if (c.dt == 2)
        return pdit::batch_launch<int16_t, ASYM>(c.maxk, c.wpr, c.tsmem, c.pk, descs, c.d_units, c.nunits, queue,
                                                 c.grid, c.threads, c.smem, c.stream);
    return pdit::batch_launch<int32_t, ASYM>(c.maxk, c.wpr, c.tsmem, c.pk, descs, c.d_units, c.nunits, queue,
                                             c.grid, c.threads, c.smem, c.stream);
}

int batch_launch(const BatchClass &c, const pdit::SweepArgs *descs, int *queue) {
    if (c.dot)
        return pdit::dot_batch_launch(c.maxk, c.wpr, descs, c.d_units, c.nunits, queue, c.grid, c.threads, c.smem,
                                      c.stream);
    return c.asym ? batch_launch_t<true>(c, descs, queue) : batch_launch_t<false>(c, descs, queue);
}

// Same compiled kernel shape.
bool same_class(const BatchClass &x, int dt, bool asym, const Plan &p) {
    if (x.dot || p.dot) return x.dot == p.dot && x.maxk == p.maxk && x.wpr == p.wpr;
    return x.dt == dt && x.asym == asym && x.maxk == p.maxk && x.wpr == p.wpr && x.pk == p.pk && x.tsmem == p.tsmem;
}

// A new shape class for plan p.
BatchClass class_for(int dt, bool asym, const Plan &p) {
    BatchClass x;
    x.dt = dt;
    x.asym = asym;
    x.dot = p.dot;
    x.maxk = p.maxk;
    x.wpr = p.wpr;
    x.pk = p.pk;
    x.tsmem = p.tsmem;
    return x;
}

// Per instance: reset its time-to-target outputs and stop flag.
__global__ void batch_init_kernel(int count, const pdit::SweepArgs *descs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const pdit::SweepArgs &a = descs[k];
    if (a.reach_ns) *a.reach_ns = ~0ull;
    if (a.reach_sweep) *a.reach_sweep = 0x7FFFFFFF;
    if (a.done) *a.done = 0;
}

// One block per instance: smallest best energy over its replicas (ties to the
// lowest replica) and that replica's permutation.
__global__ void batch_finalize_kernel(const BatchOut *outs) {
    const BatchOut o = outs[blockIdx.x];
    __shared__ long long sval[32];
    __shared__ int sidx[32];
    __shared__ int winner;
    long long v = 0x7FFFFFFFFFFFFFFFll;
    int idx = 0x7FFFFFFF;
    for (int r = threadIdx.x; r < o.replicas; r += blockDim.x) {
        const long long e = o.best_energy[r];
        if (e < v || (e == v && r < idx)) {
            v = e;
            idx = r;
        }
    }
    for (int off = 16; off; off >>= 1) {
        const long long ov = __shfl_xor_sync(0xFFFFFFFFu, v, off);
        const int oi = __shfl_xor_sync(0xFFFFFFFFu, idx, off);
        if (ov < v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sval[warp] = v;
        sidx[warp] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long bv = sval[0];
        int bi = sidx[0];
        for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w)
            if (sval[w] < bv || (sval[w] == bv && sidx[w] < bi)) {
                bv = sval[w];
                bi = sidx[w];
            }
        winner = bi;
        *o.cost = bv;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < o.n; m += blockDim.x) o.perm[m] = o.best_perm[(size_t)winner * o.n + m];
}

}  // namespace

struct pdit_batch {
    int device = 0;
    uint32_t flags = 0;
    std::vector<pdit_batch_item> items;
    std::vector<BatchClass> classes;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    pdit::SweepArgs *d_descs = nullptr;
    BatchOut *d_outs = nullptr;
    int *d_queues = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int batch_enqueue(pdit_batch *b, cudaStream_t st) {
    const int count = (int)b->items.size();
    PDIT_CK(cudaMemsetAsync(b->d_queues, 0, sizeof(int) * b->classes.size(), st));
    batch_init_kernel<<<(count + 127) / 128, 128, 0, st>>>(count, b->d_descs);
    PDIT_CK(cudaGetLastError());
    PDIT_CK(cudaEventRecord(b->fork, st));
    for (size_t c = 0; c < b->classes.size(); ++c) {
        BatchClass &k = b->classes[c];
        PDIT_CK(cudaStreamWaitEvent(k.stream, b->fork, 0));
        const int e = batch_launch(k, b->d_descs, b->d_queues + c);
        if (e != 0) return cuda_fail((cudaError_t)e, "batch kernel launch");
        PDIT_CK(cudaEventRecord(k.done, k.stream));
        PDIT_CK(cudaStreamWaitEvent(st, k.done, 0));
    }
    batch_finalize_kernel<<<count, 256, 0, st>>>(b->d_outs);
    PDIT_CK(cudaGetLastError());
    return PDIT_OK;
}

}  // namespace

extern "C" {

void pdit_batch_destroy(pdit_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (BatchClass &c : b->classes) {
        cudaFree(c.d_units);
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->ws);
    cudaFree(b->d_descs);
    cudaFree(b->d_outs);
    cudaFree(b->d_queues);
    delete b;
}

int pdit_batch_create(const pdit_batch_item *items, int count, uint32_t flags, pdit_batch **out) {
    if (!out) return PDIT_EINVAL;
    *out = nullptr;
    if (!items || count < 1 || (flags & ~(PDIT_BATCH_STOP_AT_TARGET | PDIT_BATCH_GRAPH))) return PDIT_EINVAL;
    int dev = 0;
    PDIT_CK(cudaGetDevice(&dev));
    for (int k = 0; k < count; ++k) {
        const pdit_batch_item &it = items[k];
        if (!it.qap || it.replicas < 1 || it.sweeps < 0 || (it.sweeps > 0 && !it.beta)) return PDIT_EINVAL;
        if (!it.best_perm || !it.best_cost || it.qap->device != dev) return PDIT_EINVAL;
        if ((uint64_t)it.sweeps >= 0xFFFFFFFFull) return PDIT_EINVAL;
    }
    pdit_batch *b = new (std::nothrow) pdit_batch();
    if (!b) return PDIT_ENOMEM;
    b->device = dev;
    b->flags = flags;
    b->items.assign(items, items + count);
    // Per instance: its shape with as many replica groups per CTA as fit.
    std::vector<Plan> plans((size_t)count);
    std::vector<size_t> ws_off((size_t)count);
    size_t ws_total = 0;
    for (int k = 0; k < count; ++k) {
        pdit_qap *h = items[k].qap;
        // the multi-instance kernels keep their instance descriptor in static shared memory
        int rc = batch_plan(h, &plans[k], kBatchStaticSmem);
        if (rc) {
            delete b;
            return rc;
        }
        pdit_opts o;
        pdit_opts_init(&o);
        o.replicas = items[k].replicas;
        ws_off[k] = ws_total;
        ws_total += align_up(carve(h, &o, plans[k], nullptr, false, true).bytes, kAlign);  // batches: whole calls
    }
    // Shape classes.
    for (int k = 0; k < count; ++k) {
        const Plan &p = plans[k];
        const int dt = items[k].qap->dt_bytes;
        const bool asym = items[k].qap->asym != 0;
        int found = -1;
        for (size_t c = 0; c < b->classes.size(); ++c)
            if (same_class(b->classes[c], dt, asym, p)) found = (int)c;
        if (found < 0) {
            b->classes.push_back(class_for(dt, asym, p));
            found = (int)b->classes.size() - 1;
        }
        BatchClass &x = b->classes[found];
        x.items.push_back(k);
        x.threads = std::max(x.threads, p.threads);
        x.smem = std::max(x.smem, p.smem);
    }
    int rc = PDIT_OK;
    cudaError_t e = cudaMalloc(&b->ws, std::max<size_t>(ws_total, 256));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_descs, sizeof(pdit::SweepArgs) * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_outs, sizeof(BatchOut) * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_queues, sizeof(int) * b->classes.size());
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? PDIT_ENOMEM : cuda_fail(e, "pdit_batch_create");
        pdit_batch_destroy(b);
        return rc;
    }
    b->ws_bytes = ws_total;
    // Descriptors.
    std::vector<pdit::SweepArgs> descs((size_t)count);
    std::vector<BatchOut> outs((size_t)count);
    for (int k = 0; k < count; ++k) {
        const pdit_batch_item &it = items[k];
        const Plan &p = plans[k];
        pdit_qap *h = it.qap;
        pdit_opts o;
        pdit_opts_init(&o);
        o.replicas = it.replicas;
        const Workspace w = carve(h, &o, p, (char *)b->ws + ws_off[k], false, true);
        pdit::SweepArgs &a = descs[k];
        a = pdit::SweepArgs{};
        fill_shape(a, h, p);
        a.replicas = it.replicas;
        a.sweep_begin = 0;
        a.sweep_end = it.sweeps;
        a.key0 = (uint32_t)it.seed;
        a.key1 = (uint32_t)(it.seed >> 32);
        a.inst = it.instance_id;
        a.mode = 0;
        a.beta = it.beta;
        a.fresh = 1;
        a.perm = w.perm;
        a.best_perm = w.best_perm;
        a.energy = w.energy;
        a.best_energy = w.best_energy;
        a.best_sweep = w.best_sweep;
        a.accepted = w.accepted;
        a.rung = w.rung;
        a.tables = w.tables;
        a.status = w.status;
        a.target = it.target;
        a.reach_ns = (unsigned long long *)it.reach_ns;
        a.reach_sweep = it.reach_sweep;
        a.done = w.done;
        a.stop = (it.target && (flags & PDIT_BATCH_STOP_AT_TARGET)) ? 1 : 0;
        outs[k] = BatchOut{it.best_perm, it.best_cost, h->n, it.replicas, w.best_energy, w.best_perm};
    }
    // Units, per class ordered by decreasing cost (sweeps x n^3 per unit).
    for (size_t c = 0; c < b->classes.size() && rc == PDIT_OK; ++c) {
        BatchClass &x = b->classes[c];
        std::vector<int> order = x.items;
        std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
            const double cu = (double)items[u].sweeps * std::pow((double)items[u].qap->n, 3.0);
            const double cv = (double)items[v].sweeps * std::pow((double)items[v].qap->n, 3.0);
            return cu > cv;
        });
        std::vector<pdit::BatchUnit> units;
        for (int k : order)
            for (int r0 = 0; r0 < items[k].replicas; r0 += plans[k].groups) units.push_back(pdit::BatchUnit{k, r0});
        x.nunits = (int)units.size();
        e = cudaMalloc((void **)&x.d_units, sizeof(pdit::BatchUnit) * units.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(x.d_units, units.data(), sizeof(pdit::BatchUnit) * units.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "pdit_batch_create");
            break;
        }
        int bps = 0;
        const int qe = batch_blocks(x, &bps);
        if (qe != 0) {
            rc = cuda_fail((cudaError_t)qe, "batch occupancy query");
            break;
        }
        if (bps < 1) bps = 1;
        if (!x.tsmem) bps = 1;
        const int sms = items[x.items[0]].qap->num_sms;
        x.grid = std::max(1, std::min(x.nunits, sms * bps));
    }
    if (rc == PDIT_OK) {
        e = cudaMemcpy(b->d_descs, descs.data(), sizeof(pdit::SweepArgs) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_outs, outs.data(), sizeof(BatchOut) * count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "pdit_batch_create");
    }
    if (rc) {
        pdit_batch_destroy(b);
        return rc;
    }
    *out = b;
    return PDIT_OK;
}

int pdit_batch_run(pdit_batch *b, void *stream) {
    if (!b) return PDIT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (!(b->flags & PDIT_BATCH_GRAPH)) return batch_enqueue(b, st);
    if (!st) return PDIT_EINVAL;  // the legacy default stream cannot be captured
    if (!b->exec) {
        PDIT_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const int rc = batch_enqueue(b, st);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(ie, "cudaGraphInstantiate");
        }
    }
    PDIT_CK(cudaGraphLaunch(b->exec, st));
    return PDIT_OK;
}

int pdit_batch_info(const pdit_batch *b, int *classes, size_t *workspace_bytes) {
    if (!b) return PDIT_EINVAL;
    if (classes) *classes = (int)b->classes.size();
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    return PDIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving loop with continuous batching.
// ---------------------------------------------------------------------------
namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerRequest {
    int64_t ticket = 0;
    uint32_t request_id = 0;
    int n = 0, replicas = 0, sweeps = 0;
    uint64_t seed = 0;
    std::vector<int32_t> D, F;
    std::vector<float> beta;  // host schedule until admission
    pdit_qap *qap = nullptr;
    void *ws = nullptr;
    float *dbeta = nullptr;
    int32_t *dperm = nullptr;
    int64_t *dcost = nullptr;
    Plan plan;
    Workspace w{};
    size_t footprint = 0;
    int done_sweeps = 0;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    double t_submit = 0, t_done = 0;
    std::vector<int32_t> perm;
    int64_t cost = 0;
};

}  // namespace

// Host-side staging of one tick. Two of them alternate, so that the host
// fills one while the copies of the other may still be pending on the GPU;
// a buffer is reused only after its event has completed.
struct TickBuf {
    pdit::SweepArgs *h_descs = nullptr;
    BatchOut *h_outs = nullptr;
    pdit::BatchUnit *h_units = nullptr;
    int32_t *h_perm = nullptr;  // results of the requests finishing with this tick: PDIT_N_MAX each
    int64_t *h_cost = nullptr;
    size_t cap_desc = 0, cap_units = 0, cap_res = 0;
    cudaEvent_t done = nullptr;  // recorded after the tick's result copies
    bool pending = false;
    std::vector<ServerRequest *> finishing;
};

struct pdit_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int slice = 100, max_active = 64;
    std::mutex mu;
    std::vector<ServerRequest *> all;   // by ticket
    std::vector<ServerRequest *> queue; // FIFO of queued tickets
    std::vector<ServerRequest *> active;
    // device arrays of a tick (stream-ordered on `main`, so one set serves
    // both host buffers), grown on demand
    pdit::SweepArgs *d_descs = nullptr;
    BatchOut *d_outs = nullptr;
    pdit::BatchUnit *d_units = nullptr;
    size_t cap_desc = 0, cap_units = 0;
    int *d_queues = nullptr;
    TickBuf buf[2];
    int cur = 0;
    std::vector<BatchClass> classes;  // streams and events reused
    cudaStream_t main = nullptr;
    cudaStream_t upload = nullptr;   // admissions: allocations and copies of new requests
    cudaEvent_t uploaded = nullptr;  // recorded after the last admission's copies
    bool new_uploads = false;
    cudaEvent_t fork = nullptr;
    int64_t completed = 0;
};

namespace {

// Stream-ordered release of a request's device memory, after the work
// queued on the main stream (which has joined every kernel that used it):
// no device-wide synchronisation, so the host keeps ahead of the GPU.
void release_request(pdit_server *s, ServerRequest *r) {
    void *bufs[] = {r->ws, r->dbeta, r->dperm, r->dcost, r->qap ? r->qap->dD : nullptr,
                    r->qap ? r->qap->dF : nullptr, r->qap ? r->qap->dx : nullptr};
    for (void *ptr : bufs)
        if (ptr) cudaFreeAsync(ptr, s->main);
    r->ws = nullptr;
    r->dbeta = nullptr;
    r->dperm = nullptr;
    r->dcost = nullptr;
    if (r->qap) {
        r->qap->dD = nullptr;
        r->qap->dF = nullptr;
        r->qap->dx = nullptr;
    }
    qap_destroy(r->qap);  // host state only now
    r->qap = nullptr;
    s->used -= std::min(s->used, r->footprint);
}

// Device memory a request holds while admitted: its workspace with every
// replica's state kept between slices (the table of the table kernels, the
// permuted flow matrix of the dot kernel), the matrices, the schedule and
// the result.
size_t request_footprint(const ServerRequest &r, const Plan &p) {
    pdit_opts o;
    pdit_opts_init(&o);
    o.replicas = r.replicas;
    return carve(r.qap, &o, p, nullptr, true, true).bytes + (size_t)8 * r.n * r.n + 4 * (size_t)r.sweeps + 4 * r.n + 8 +
           1024;
}

int admit(pdit_server *s, ServerRequest *r) {
    int rc = qap_prepare(r->n, r->D.data(), r->F.data(), &r->qap);
    if (rc) return rc;
    rc = batch_plan(r->qap, &r->plan, kBatchStaticSmem);
    if (rc) return rc;
    const size_t fp = request_footprint(*r, r->plan);
    // wait for memory; a request larger than the budget is admitted alone,
    // once nothing else holds device memory (finished requests release
    // theirs when their last tick has completed)
    if (s->used + fp > s->budget && s->used > 0) return 1;
    if (r->beta.empty()) {
        double bmax = 0.0;
        pdit_beta_max(r->qap, &bmax);
        r->beta.resize((size_t)std::max(r->sweeps, 1));
        pdit_beta_schedule(0, r->sweeps, bmax, r->beta.data());
    }
    pdit_opts o;
    pdit_opts_init(&o);
    o.replicas = r->replicas;
    const size_t wsb = carve(r->qap, &o, r->plan, nullptr, true, true).bytes;
    // stream-ordered allocations and copies on the upload stream (a copy from
    // pageable memory waits only for that stream's earlier work, none of
    // which is a kernel); the main stream waits for them before the next launch
    pdit_qap *h = r->qap;
    const size_t mb = sizeof(int32_t) * (size_t)r->n * r->n;
    cudaStream_t up = s->upload;
    cudaError_t e = cudaMallocAsync(&r->ws, wsb, up);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->dbeta, sizeof(float) * std::max(r->sweeps, 1), up);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->dperm, sizeof(int32_t) * r->n, up);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->dcost, sizeof(int64_t), up);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&h->dD, mb, up);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&h->dF, mb, up);
    if (e == cudaSuccess && h->cls) e = cudaMallocAsync((void **)&h->dx, (size_t)r->n, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dD, h->hD.data(), mb, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dF, h->hF.data(), mb, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess && h->cls)
        e = cudaMemcpyAsync(h->dx, h->cls_x.data(), (size_t)r->n, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess && r->sweeps > 0)
        e = cudaMemcpyAsync(r->dbeta, r->beta.data(), sizeof(float) * r->sweeps, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(s->uploaded, up);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PDIT_ENOMEM : cuda_fail(e, "server admit");
    s->new_uploads = true;
    r->w = carve(r->qap, &o, r->plan, (char *)r->ws, true, true);
    r->footprint = fp;
    s->used += fp;
    r->D.clear();
    r->D.shrink_to_fit();
    r->F.clear();
    r->F.shrink_to_fit();
    r->state = 1;
    return PDIT_OK;
}

// Capacity of the device arrays and of host buffer b for a tick of ndesc
// requests, nunits work units and nres finishing requests.
int grow(pdit_server *s, TickBuf &b, size_t ndesc, size_t nunits, size_t nres) {
    if (ndesc > s->cap_desc) {
        cudaFree(s->d_descs);
        cudaFree(s->d_outs);
        s->d_descs = nullptr;
        s->d_outs = nullptr;
        s->cap_desc = 0;
        const size_t c = std::max(ndesc, (size_t)64);
        PDIT_CK(cudaMalloc((void **)&s->d_descs, sizeof(pdit::SweepArgs) * c));
        PDIT_CK(cudaMalloc((void **)&s->d_outs, sizeof(BatchOut) * c));
        s->cap_desc = c;
    }
    if (nunits > s->cap_units) {
        cudaFree(s->d_units);
        s->d_units = nullptr;
        s->cap_units = 0;
        const size_t c = std::max(nunits * 2, (size_t)1024);
        PDIT_CK(cudaMalloc((void **)&s->d_units, sizeof(pdit::BatchUnit) * c));
        s->cap_units = c;
    }
    if (ndesc > b.cap_desc) {
        cudaFreeHost(b.h_descs);
        cudaFreeHost(b.h_outs);
        b.h_descs = nullptr;
        b.h_outs = nullptr;
        b.cap_desc = 0;
        const size_t c = std::max(ndesc, (size_t)64);
        PDIT_CK(cudaMallocHost((void **)&b.h_descs, sizeof(pdit::SweepArgs) * c));
        PDIT_CK(cudaMallocHost((void **)&b.h_outs, sizeof(BatchOut) * c));
        b.cap_desc = c;
    }
    if (nunits > b.cap_units) {
        cudaFreeHost(b.h_units);
        b.h_units = nullptr;
        b.cap_units = 0;
        const size_t c = std::max(nunits * 2, (size_t)1024);
        PDIT_CK(cudaMallocHost((void **)&b.h_units, sizeof(pdit::BatchUnit) * c));
        b.cap_units = c;
    }
    if (nres > b.cap_res) {
        cudaFreeHost(b.h_perm);
        cudaFreeHost(b.h_cost);
        b.h_perm = nullptr;
        b.h_cost = nullptr;
        b.cap_res = 0;
        const size_t c = std::max(nres, (size_t)64);
        PDIT_CK(cudaMallocHost((void **)&b.h_perm, sizeof(int32_t) * PDIT_N_MAX * c));
        PDIT_CK(cudaMallocHost((void **)&b.h_cost, sizeof(int64_t) * c));
        b.cap_res = c;
    }
    return PDIT_OK;
}

// The requests whose last slice ran in the tick of buffer b: its result
// copies have completed (the caller checked b.done); record the results and
// release the requests' device memory.
void retire(pdit_server *s, TickBuf &b) {
    const double t = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t k = 0; k < b.finishing.size(); ++k) {
        ServerRequest *r = b.finishing[k];
        r->perm.assign(b.h_perm + k * PDIT_N_MAX, b.h_perm + k * PDIT_N_MAX + r->n);
        r->cost = b.h_cost[k];
        r->t_done = t;
        r->state = 2;
        release_request(s, r);
        s->completed += 1;
    }
    b.finishing.clear();
    b.pending = false;
}

// Retire buffer b if its tick has completed (wait: block until it has).
int poll(pdit_server *s, TickBuf &b, bool wait) {
    if (!b.pending) return PDIT_OK;
    const cudaError_t e = wait ? cudaEventSynchronize(b.done) : cudaEventQuery(b.done);
    if (e == cudaErrorNotReady) return PDIT_OK;
    if (e != cudaSuccess) return cuda_fail(e, "server tick");
    retire(s, b);
    return PDIT_OK;
}

}  // namespace

extern "C" {

int pdit_server_create(size_t device_budget_bytes, int slice_sweeps, int max_active, pdit_server **out) {
    if (!out) return PDIT_EINVAL;
    *out = nullptr;
    if (device_budget_bytes == 0 || slice_sweeps < 1 || max_active < 1) return PDIT_EINVAL;
    pdit_server *s = new (std::nothrow) pdit_server();
    if (!s) return PDIT_ENOMEM;
    s->budget = device_budget_bytes;
    s->slice = slice_sweeps;
    s->max_active = max_active;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->main, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
    for (TickBuf &b : s->buf)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_queues, sizeof(int) * 64);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "pdit_server_create");
        pdit_server_destroy(s);
        return rc;
    }
    *out = s;
    return PDIT_OK;
}

void pdit_server_destroy(pdit_server *s) {
    if (!s) return;
    if (s->upload) cudaStreamSynchronize(s->upload);
    if (s->main) cudaStreamSynchronize(s->main);
    for (ServerRequest *r : s->all) {
        release_request(s, r);
        delete r;
    }
    if (s->main) cudaStreamSynchronize(s->main);  // the releases above are stream-ordered
    if (s->upload) cudaStreamDestroy(s->upload);
    if (s->uploaded) cudaEventDestroy(s->uploaded);
    for (BatchClass &c : s->classes) {
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    cudaFree(s->d_descs);
    cudaFree(s->d_outs);
    cudaFree(s->d_units);
    for (TickBuf &b : s->buf) {
        cudaFreeHost(b.h_descs);
        cudaFreeHost(b.h_outs);
        cudaFreeHost(b.h_units);
        cudaFreeHost(b.h_perm);
        cudaFreeHost(b.h_cost);
        if (b.done) cudaEventDestroy(b.done);
    }
    cudaFree(s->d_queues);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->main) cudaStreamDestroy(s->main);
    delete s;
}

int pdit_server_submit(pdit_server *s, int n, const int32_t *D, const int32_t *F, int replicas, int sweeps,
                       uint64_t seed, uint32_t request_id, const float *beta, int64_t *ticket) {
    // D and F are validated by qap_create when the request is admitted (a
    // rejected instance ends in the failed state)
    if (!s || !ticket || n < 2 || n > PDIT_N_MAX || !D || !F || replicas < 1 || sweeps < 0) return PDIT_EINVAL;
    ServerRequest *r = new (std::nothrow) ServerRequest();
    if (!r) return PDIT_ENOMEM;
    r->request_id = request_id;
    r->n = n;
    r->replicas = replicas;
    r->sweeps = sweeps;
    r->seed = seed;
    r->D.assign(D, D + (size_t)n * n);
    r->F.assign(F, F + (size_t)n * n);
    if (beta && sweeps > 0) r->beta.assign(beta, beta + sweeps);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    r->ticket = (int64_t)s->all.size();
    s->all.push_back(r);
    s->queue.push_back(r);
    *ticket = r->ticket;
    return PDIT_OK;
}

int pdit_server_tick(pdit_server *s, int *active, int *queued) {
    if (!s) return PDIT_EINVAL;
    // 0. results of earlier ticks whose work has completed
    for (TickBuf &b : s->buf) {
        const int rc = poll(s, b, false);
        if (rc) return rc;
    }
    // 1. admit queued requests (FIFO) while slots and device memory allow
    {
        std::lock_guard<std::mutex> lock(s->mu);
        while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
            ServerRequest *r = s->queue.front();
            const int rc = admit(s, r);
            if (rc == 1) {  // does not fit yet: release what admit created, retry later
                qap_destroy(r->qap);
                r->qap = nullptr;
                break;
            }
            s->queue.erase(s->queue.begin());
            if (rc) {
                r->state = 3;
                release_request(s, r);
                continue;
            }
            s->active.push_back(r);
        }
    }
    const int na = (int)s->active.size();
    if (na > 0) {
        // 2. one slice of sweeps for every active request, one launch per
        // kernel shape; each replica's state (permutation, energies, table
        // or permuted flow matrix) stays in the request's workspace between
        // slices
        TickBuf &b = s->buf[s->cur];
        int rc = poll(s, b, true);  // the buffer's previous copies are done
        if (rc) return rc;
        size_t nunits = 0, nres = 0;
        for (ServerRequest *r : s->active) {
            nunits += (size_t)(r->replicas + r->plan.groups - 1) / r->plan.groups;
            nres += r->done_sweeps + s->slice >= r->sweeps ? 1 : 0;
        }
        rc = grow(s, b, (size_t)na, nunits, nres);
        if (rc) return rc;
        std::vector<BatchClass> cls;
        std::vector<std::vector<int>> members;
        std::vector<ServerRequest *> finishing;
        int nout = 0;
        for (int k = 0; k < na; ++k) {
            ServerRequest *r = s->active[k];
            const Plan &p = r->plan;
            const int end = std::min(r->sweeps, r->done_sweeps + s->slice);
            pdit::SweepArgs &a = b.h_descs[k];
            a = pdit::SweepArgs{};
            fill_shape(a, r->qap, p);
            a.replicas = r->replicas;
            a.sweep_begin = r->done_sweeps;
            a.sweep_end = end;
            a.key0 = (uint32_t)r->seed;
            a.key1 = (uint32_t)(r->seed >> 32);
            a.inst = r->request_id;
            a.beta = r->dbeta;
            a.fresh = r->done_sweeps == 0 ? 1 : 0;
            a.table_in = a.fresh ? 0 : 1;       // resume from the saved state
            a.table_out = end < r->sweeps ? 1 : 0;  // save it for the next slice
            a.perm = r->w.perm;
            a.best_perm = r->w.best_perm;
            a.energy = r->w.energy;
            a.best_energy = r->w.best_energy;
            a.best_sweep = r->w.best_sweep;
            a.accepted = r->w.accepted;
            a.rung = r->w.rung;
            a.tables = r->w.tables;
            a.status = r->w.status;
            if (end >= r->sweeps) {
                b.h_outs[nout++] = BatchOut{r->dperm, r->dcost, r->n, r->replicas, r->w.best_energy, r->w.best_perm};
                finishing.push_back(r);
            }
            const int dt = r->qap->dt_bytes;
            const bool asym = r->qap->asym != 0;
            int found = -1;
            for (size_t c = 0; c < cls.size(); ++c)
                if (same_class(cls[c], dt, asym, p)) found = (int)c;
            if (found < 0) {
                cls.push_back(class_for(dt, asym, p));
                members.emplace_back();
                found = (int)cls.size() - 1;
            }
            cls[found].threads = std::max(cls[found].threads, p.threads);
            cls[found].smem = std::max(cls[found].smem, p.smem);
            members[found].push_back(k);
        }
        if (cls.size() > 64) return PDIT_ENOTSUP;
        while (s->classes.size() < cls.size()) {
            BatchClass c;
            PDIT_CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
            PDIT_CK(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
            s->classes.push_back(c);
        }
        size_t u = 0;
        for (size_t c = 0; c < cls.size(); ++c) {
            std::vector<int> order = members[c];
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                const ServerRequest *ra = s->active[x], *rb = s->active[y];
                return (double)ra->n * ra->n * ra->n > (double)rb->n * rb->n * rb->n;
            });
            cls[c].d_units = s->d_units + u;
            const size_t u0 = u;
            for (int k : order)
                for (int r0 = 0; r0 < s->active[k]->replicas; r0 += s->active[k]->plan.groups)
                    b.h_units[u++] = pdit::BatchUnit{k, r0};
            cls[c].nunits = (int)(u - u0);
            cls[c].stream = s->classes[c].stream;
            cls[c].done = s->classes[c].done;
            int bps = 0;
            const int qe = batch_blocks(cls[c], &bps);
            if (qe != 0) return cuda_fail((cudaError_t)qe, "server occupancy query");
            if (bps < 1 || !cls[c].tsmem) bps = 1;
            cls[c].grid = std::max(1, std::min(cls[c].nunits, s->active[members[c][0]]->qap->num_sms * bps));
        }
        // from pinned host buffers: asynchronous; the device arrays are read
        // in stream order, after the previous tick's kernels
        PDIT_CK(cudaMemcpyAsync(s->d_descs, b.h_descs, sizeof(pdit::SweepArgs) * na, cudaMemcpyHostToDevice, s->main));
        PDIT_CK(cudaMemcpyAsync(s->d_units, b.h_units, sizeof(pdit::BatchUnit) * u, cudaMemcpyHostToDevice, s->main));
        if (nout > 0)
            PDIT_CK(cudaMemcpyAsync(s->d_outs, b.h_outs, sizeof(BatchOut) * nout, cudaMemcpyHostToDevice, s->main));
        PDIT_CK(cudaMemsetAsync(s->d_queues, 0, sizeof(int) * cls.size(), s->main));
        if (s->new_uploads) {  // the matrices and schedules of newly admitted requests
            PDIT_CK(cudaStreamWaitEvent(s->main, s->uploaded, 0));
            s->new_uploads = false;
        }
        PDIT_CK(cudaEventRecord(s->fork, s->main));
        for (size_t c = 0; c < cls.size(); ++c) {
            PDIT_CK(cudaStreamWaitEvent(cls[c].stream, s->fork, 0));
            const int e = batch_launch(cls[c], s->d_descs, s->d_queues + c);
            if (e != 0) return cuda_fail((cudaError_t)e, "server batch launch");
            PDIT_CK(cudaEventRecord(cls[c].done, cls[c].stream));
            PDIT_CK(cudaStreamWaitEvent(s->main, cls[c].done, 0));
        }
        // 3. results of the requests whose schedule ends with this slice,
        // copied to pinned memory and picked up once the tick's event has
        // completed (at a later tick)
        if (nout > 0) {
            batch_finalize_kernel<<<nout, 256, 0, s->main>>>(s->d_outs);
            PDIT_CK(cudaGetLastError());
        }
        for (size_t k = 0; k < finishing.size(); ++k) {
            ServerRequest *r = finishing[k];
            PDIT_CK(cudaMemcpyAsync(b.h_perm + k * PDIT_N_MAX, r->dperm, sizeof(int32_t) * r->n,
                                    cudaMemcpyDeviceToHost, s->main));
            PDIT_CK(cudaMemcpyAsync(b.h_cost + k, r->dcost, sizeof(int64_t), cudaMemcpyDeviceToHost, s->main));
        }
        PDIT_CK(cudaEventRecord(b.done, s->main));
        b.pending = true;
        for (ServerRequest *r : s->active) r->done_sweeps = std::min(r->sweeps, r->done_sweeps + s->slice);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            for (ServerRequest *r : finishing) s->active.erase(std::find(s->active.begin(), s->active.end(), r));
        }
        b.finishing = std::move(finishing);
        s->cur ^= 1;
    } else {
        // nothing to launch: wait for the oldest outstanding tick
        for (int k = 1; k <= 2; ++k) {
            TickBuf &b = s->buf[(s->cur + k) % 2];
            if (b.pending) {
                const int rc = poll(s, b, true);
                if (rc) return rc;
                break;
            }
        }
    }
    std::lock_guard<std::mutex> lock(s->mu);
    int in_flight = 0;  // finished on the host side, results not yet picked up
    for (const TickBuf &b : s->buf) in_flight += b.pending ? (int)b.finishing.size() : 0;
    if (active) *active = (int)s->active.size() + in_flight;
    if (queued) *queued = (int)s->queue.size();
    return PDIT_OK;
}

int pdit_server_result(pdit_server *s, int64_t ticket, int *state, int32_t *best_perm, int64_t *best_cost,
                       double *latency_s) {
    if (!s || !state) return PDIT_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (ticket < 0 || ticket >= (int64_t)s->all.size()) return PDIT_EINVAL;
    const ServerRequest *r = s->all[(size_t)ticket];
    *state = r->state;
    if (r->state == 2) {
        if (best_perm) std::memcpy(best_perm, r->perm.data(), sizeof(int32_t) * r->n);
        if (best_cost) *best_cost = r->cost;
        if (latency_s) *latency_s = r->t_done - r->t_submit;
    }
    return PDIT_OK;
}

}  // extern "C"
