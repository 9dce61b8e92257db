/*
 * libpdit -- p-dit probabilistic Ising machine for the quadratic assignment
 * problem, on NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2605.24408, "P-dit Probabilistic Ising Machine for Solving
 * the Quadratic Assignment Problem". The QAP is min_p sum_ij D_ij F_{p(i)p(j)}
 * (Eq. 1). Each location holds a p-dit whose state is the facility assigned
 * to it. An update of location i chooses, with the Boltzmann law of Eq. 5,
 * between staying and swapping facilities with one of the other N-1
 * locations, using the exact swap energy of Eq. 3 computed from entries of
 * the influence table (Eq. 2): kept as a table updated incrementally after
 * every accepted swap, or formed by dot products from a permuted copy of F
 * (pdit_set_influence); the same integers either way. A sweep updates every
 * location once, in index order. Plain mode anneals the
 * inverse temperature beta along a per-sweep schedule; PT mode runs
 * parallel tempering (Implementation section; CPU-PIM Algorithm section).
 * Symmetric instances keep the one-term table I[m][c] = sum_j D[m][j]
 * F[c][p(j)] (for them Eq. 2 equals -2 I); instances with a non-symmetric
 * D or F keep Eq. 2's two-term table and use Eq. 3 as printed, which is
 * exact for any D and F.
 *
 * Conventions for every call:
 *  - Return 0 (PDIT_OK) on success, a negative PDIT_E* code on failure. No
 *    C++ exception crosses this interface.
 *  - Matrices are int32, row-major, N x N. Permutations are 0-based:
 *    perm[i] = facility at location i. Costs are int64 and exact.
 *  - Output buffers are owned by the caller. A handle is not thread-safe:
 *    use one handle per host thread.
 *  - Device work of pdit_anneal_ex is ordered on the caller's stream and is
 *    asynchronous; pdit_anneal is synchronous.
 *  - Results are a pure function of (D, F, beta values, seed, instance_id,
 *    global replica id): independent of the GPU, the launch shape and how
 *    replicas are split across calls.
 */
#ifndef PDIT_H
#define PDIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define PDIT_OK 0
#define PDIT_EINVAL (-1)  /* NULL pointer, size out of range, bad beta */
#define PDIT_ERANGE (-2)  /* 16 (N+2) max|D| max|F| >= 2^31: the int32 tables could overflow */
#define PDIT_ENOMEM (-3)  /* an allocation failed, or the caller's workspace is too small */
#define PDIT_ECUDA (-4)   /* a CUDA runtime call failed; see pdit_last_error() */
#define PDIT_EDEVICE (-5) /* a device-side consistency audit failed (see PDIT_STATUS_*) */
#define PDIT_ENOTSUP (-6) /* a valid request the compiled kernels cannot run */
#define PDIT_EIO (-7)     /* a file could not be opened, read or written */

/* Largest instance size. */
#define PDIT_N_MAX 256

/* Modes. */
#define PDIT_MODE_ANNEAL 0 /* beta[s] for sweep s, every replica */
#define PDIT_MODE_PT 1     /* parallel tempering over a beta ladder */
#define PDIT_MODE_FIXED 2  /* beta[r] for replica r, every sweep, no exchange (beta-range trials) */
#define PDIT_MODE_CUPIM 3  /* concurrent updates from a snapshot (GPU-CUPIM Algorithm section), beta[s] */

/* Flags. */
#define PDIT_FLAG_RESUME 1u /* continue from the replica state already in the workspace */

/* Device status bits (opts.status). */
#define PDIT_STATUS_ENERGY_AUDIT 1 /* tracked energy != energy recomputed (from the table or
                                      the flow-class vector at a resume or at the end; from
                                      Eq. 1 at the end of every dot-kernel call) */
#define PDIT_STATUS_SCHEDULE 2     /* a part of a replica's sweeps waited past its bound for the
                                      part before it (dot kernel, more replicas than resident
                                      slots); the call stopped early and its results are not valid */

typedef struct pdit_qap pdit_qap;

/*
 * qap_create -- upload one QAP instance (Eq. 1 inputs) to the current CUDA
 * device.
 *   n      : 2 <= n <= PDIT_N_MAX.
 *   D, F   : host pointers, n*n int32 each, row-major. Symmetric or not
 *            (Eq. 2 and Eq. 3 cover the general QAP; the paper's instances
 *            are symmetric), any diagonal, any sign. Copied; the caller
 *            keeps ownership.
 *   out    : receives the handle (owns device copies of D and F).
 * Errors: PDIT_EINVAL (n out of range, NULL), PDIT_ERANGE
 * (values too large for exact int32 table arithmetic), PDIT_ENOMEM,
 * PDIT_ECUDA. On error *out is set to NULL.
 */
int qap_create(int n, const int32_t *D, const int32_t *F, pdit_qap **out);

/* qap_destroy -- free the handle and its device memory. NULL-safe. */
void qap_destroy(pdit_qap *h);

/* qap_n -- the instance size of a handle, or PDIT_EINVAL for NULL. */
int qap_n(const pdit_qap *h);

/*
 * pdit_set_warps_per_replica -- thread mapping of later calls on this
 * handle: each replica is updated by `wpr` warps (1, 2, 4 or 8, at most
 * ceil(n/32) rounded up to a power of two); 0 restores the built-in choice.
 * Results do not depend on it (the paper parallelises each update across
 * threads, GPU Implementations section; the split is a performance knob).
 * Errors: PDIT_EINVAL.
 */
int pdit_set_warps_per_replica(pdit_qap *h, int wpr);

/*
 * pdit_autotune -- time every compiled thread mapping (warps per replica) of
 * the dot-product kernel (eligible instances; see pdit_set_influence) and of
 * the table kernels, with their table-update batching (1, 4 or 16 pending
 * terms), the table placement (shared or global memory, when both are
 * possible) and, where the tables live in global memory, replicas per CTA
 * (1..4 besides the built-in choice) valid for this instance on a short run
 * of `replicas` chains over the DEVICE schedule beta[sweeps] (CUDA events on
 * the handle's stream), keep the fastest for later calls on this handle and
 * write it to shape[0] (warps per replica) and shape[1] (pending terms; 1 for
 * the dot kernel) when shape is not NULL (pdit_launch_shape reports the
 * replicas per CTA and which kernel). Synchronous; allocates and frees
 * small temporary buffers. Results of later calls do not depend on the
 * choice. Errors: PDIT_EINVAL, PDIT_ENOTSUP, PDIT_ECUDA.
 */
int pdit_autotune(pdit_qap *h, int replicas, const float *beta, int sweeps, int *shape);

/* Influence-table placement (pdit_set_table_placement). */
#define PDIT_PLACE_AUTO 0   /* shared memory when a replica's table fits next to D and F, else global */
#define PDIT_PLACE_SHARED 1 /* shared memory (PDIT_ENOTSUP at the next call when it does not fit) */
#define PDIT_PLACE_GLOBAL 2 /* global memory, L2-resident (n > 128 only; PDIT_ENOTSUP otherwise) */

/*
 * pdit_set_table_placement -- where later calls on this handle keep the
 * replicas' influence tables. Global tables let more replicas share an SM
 * at the cost of L2 latency; the autotuner compares the two. Results do not
 * depend on it. Errors: PDIT_EINVAL.
 */
int pdit_set_table_placement(pdit_qap *h, int place);

/*
 * pdit_set_replicas_per_cta -- replica groups per CTA of later calls on this
 * handle: at most g (1 or more), within what shared memory, the compiled
 * thread bound and the named barriers allow; 0 restores the built-in choice
 * (as many as fit; with tables in global memory, as many as keep all
 * resident tables within three quarters of L2). Results do not depend on it.
 * Errors: PDIT_EINVAL.
 */
int pdit_set_replicas_per_cta(pdit_qap *h, int g);

/*
 * pdit_launch_shape -- the sweep-kernel launch a call with `replicas` chains
 * would use: shape[0] warps per replica, [1] candidates per thread, [2]
 * replicas per CTA, [3] CTAs, [4] 1 if the influence tables live in shared
 * memory (0: global memory; 2: no table, the dot-product kernel of
 * pdit_set_influence), [5] dynamic shared memory bytes per CTA.
 * [6] pending rank-1 terms held before the influence table is rewritten (1 =
 * after each swap; 4 or 16).
 * `shape` is a host array of 7 ints. Errors: PDIT_EINVAL, PDIT_ENOTSUP.
 */
int pdit_launch_shape(const pdit_qap *h, int replicas, int *shape);

/* Influence entries (pdit_set_influence). */
#define PDIT_INFLUENCE_AUTO 0     /* dot products where eligible and no table knob is set, else the table */
#define PDIT_INFLUENCE_TABLE 1    /* the influence table of Eq. 2, updated after every accepted swap */
#define PDIT_INFLUENCE_PRODUCTS 2 /* dot products of byte rows of D and of the permuted F (no table) */

/*
 * pdit_set_influence -- how later sequential-mode calls on this handle obtain
 * the two influence entries each swap energy needs (Eq. 3 in the one-term
 * units: I[i][p(j)] and I[j][p(i)], I[m][c] = sum_y D[m][y] F[c][p(y)]).
 *   PDIT_INFLUENCE_TABLE    : keep every replica's N x N int32 table and add
 *                             the rank-1 change of Eq. 2 after each accepted
 *                             swap (the paper's incremental scheme; the table
 *                             knobs above apply).
 *   PDIT_INFLUENCE_PRODUCTS : keep instead the flow matrix permuted to
 *                             location order, Q[x][y] = F[p(x)][p(y)] (N x N
 *                             bytes), and form both entries as 8-bit dot
 *                             products I[i][p(j)] = D[i] . Q[j], I[j][p(i)] =
 *                             D[j] . Q[i]; an accepted swap exchanges two rows
 *                             and two columns of Q and updates the p-diagonal
 *                             h[x] = I[x][p(x)] incrementally. Symmetric
 *                             instances whose D and F entries all lie in
 *                             -128..127, in the sequential modes, without
 *                             the table dump (PDIT_ENOTSUP otherwise, at the
 *                             next call). Two-level-flow instances keep the
 *                             flow-class kernel unless pdit_set_class_update
 *                             turns it off.
 *   PDIT_INFLUENCE_AUTO     : products where eligible and where shared
 *                             memory holds at least 3 replicas per SM (N up
 *                             to about 200), unless a table knob (pending
 *                             swaps, placement) is set; the table otherwise
 *                             (also for the concurrent-update mode and for
 *                             calls that dump the tables).
 * The entries are the same exact integers either way, so results do not
 * depend on the choice. Errors: PDIT_EINVAL.
 */
int pdit_set_influence(pdit_qap *h, int mode);

/* Instance forms (pdit_instance_form). */
#define PDIT_FORM_SYMMETRIC 0     /* D, F symmetric: one-term table I (Eq. 2 = -2 I) */
#define PDIT_FORM_GENERAL 1       /* D or F not symmetric: Eq. 2's two-term table, Eq. 3 as printed */
#define PDIT_FORM_FLOW_CLASSES 2  /* two-level flow (Methods, tai256c): an N-vector instead of the table */

/*
 * pdit_instance_form -- how the kernels treat this instance, decided at
 * qap_create: PDIT_FORM_FLOW_CLASSES when D is symmetric with a zero diagonal
 * and every off-diagonal flow is F[c][d] = f0 + f x_c x_d for some x in
 * {0,1}^n (the structure the Methods section exploits for tai256c: a swap
 * within a class leaves the energy unchanged, and every swap across the
 * classes has an energy change that depends only on the two locations); then
 * the influence table collapses to G[m] = sum over locations j holding a
 * class-1 facility of D[m][j], and an accepted swap costs O(n) instead of
 * O(n^2). Results are identical to the table path's (the swap energies are
 * the same exact integers). Concurrent-update mode and calls that request the
 * table dump run the table kernels. Returns the form or PDIT_EINVAL.
 */
int pdit_instance_form(const pdit_qap *h);

/*
 * pdit_set_class_update -- enable (1, the default) or disable (0) the
 * flow-class kernel for later calls on this handle; disabled, a
 * PDIT_FORM_FLOW_CLASSES instance runs the table kernels. Results do not
 * depend on it. Errors: PDIT_EINVAL.
 */
int pdit_set_class_update(pdit_qap *h, int enable);

/*
 * pdit_set_pending_swaps -- table-update batching of later calls on this
 * handle: k = 1 rewrites the influence table after every accepted swap
 * (the rank-1 update implied by Eq. 2); k = 4 keeps up to four pending
 * rank-1 terms (four accepted swaps; two in the general form) that every
 * query adds in, and rewrites the table once they are full (a rank-4
 * update); k = 16 does the same with sixteen terms and is available when
 * the tables live in global memory (n above about 190). 0 restores the
 * built-in choice (16 for global tables, else 4 when it costs no resident
 * replica, else 1). k > 1 needs max - min <= 127 over the entries of D and
 * of F (so every swap factor fits a signed byte); PDIT_ENOTSUP otherwise,
 * or for k = 16 with tables in shared memory, at the next call. Results do
 * not depend on k.
 * Errors: PDIT_EINVAL.
 */
int pdit_set_pending_swaps(pdit_qap *h, int k);

/*
 * pdit_anneal -- synchronous annealed p-dit sweep on HOST buffers.
 *   replicas      : >= 1 independent chains (replica ids 0..replicas-1).
 *   beta_schedule : host, `sweeps` floats, beta of sweep s (finite, >= 0).
 *   sweeps        : >= 0 (0 returns the best initial permutation).
 *   seed          : Philox key.
 *   best_perm     : host, n int32: the best permutation over all replicas
 *                   (smallest cost, ties to the lowest replica id).
 *   best_cost     : host, its Eq. 1 cost.
 * Copies beta to the device and the result back inside the call; uses a
 * stream and a workspace owned by the handle.
 * Errors: PDIT_EINVAL, PDIT_ENOMEM, PDIT_ECUDA, PDIT_EDEVICE.
 */
int pdit_anneal(pdit_qap *h, int replicas, const float *beta_schedule, int sweeps, uint64_t seed,
                int32_t *best_perm, int64_t *best_cost);

/*
 * Options of pdit_anneal_ex. Initialise with pdit_opts_init, then set
 * fields. Every pointer below is a DEVICE pointer on the handle's device.
 */
typedef struct pdit_opts {
    uint32_t struct_size;   /* sizeof(pdit_opts); set by pdit_opts_init */
    int replicas;           /* chains in this call, >= 1 */
    int sweeps;             /* schedule length S (anneal mode: length of beta) */
    int sweep_begin;        /* run sweeps [sweep_begin, sweep_end); default 0 */
    int sweep_end;          /* default -1 = sweeps */
    uint64_t seed;          /* Philox key */
    uint32_t instance_id;   /* Philox counter word 0; default 0 */
    uint32_t replica_base;  /* global id of this call's replica 0 (counter word 1); default 0 */
    int mode;               /* PDIT_MODE_ANNEAL (default), _PT, _FIXED or _CUPIM (one iteration per sweep) */
    const float *beta;      /* anneal: [sweeps]; PT: [ladder_len], rung 0 = smallest beta; fixed: [replicas] */
    int ladder_len;         /* PT: replicas per set (2..64); replicas % ladder_len == 0 */
    int exchange_period;    /* PT: sweeps between exchanges (paper: 4) */
    int timeout_periods;    /* PT: periods without a top-rung swap before top<->bottom (paper: 100); 0 = off */
    uint32_t flags;         /* PDIT_FLAG_* */
    void *stream;           /* cudaStream_t; NULL = the legacy default stream */
    void *workspace;        /* >= pdit_workspace_bytes(); NULL = owned by the handle (allocates) */
    size_t workspace_bytes;
    /* outputs; best_perm and best_cost are required, the rest optional (NULL) */
    int32_t *best_perm;          /* [n] */
    int64_t *best_cost;          /* [1] */
    int64_t *replica_best_cost;  /* [replicas] */
    int32_t *replica_best_perm;  /* [replicas * n] */
    int32_t *replica_best_sweep; /* [replicas]; -1 = the initial state */
    int32_t *replica_final_perm; /* [replicas * n] */
    int64_t *replica_final_cost; /* [replicas] */
    int64_t *replica_accepted;   /* [replicas]: accepted swaps in this call's sweeps (cumulative on resume) */
    int32_t *replica_rung;       /* [replicas]: PT rung of each replica at the end */
    int32_t *tables;             /* [replicas * n * n]: final influence tables I[m][c] */
    int32_t *status;             /* [1]: PDIT_STATUS_* bits, 0 if every audit passed */
    /* time to a target cost (optional) */
    const int64_t *target;       /* [1]: the cost to reach */
    uint64_t *reach_ns;          /* [1]: %globaltimer (ns) when some replica's best first got
                                    <= *target; UINT64_MAX if never */
    int32_t *reach_sweep;        /* [1]: the smallest sweep index at which a replica's best was
                                    <= *target (-1 = its initial state); INT32_MAX if never */
    int stop_at_target;          /* 1: once reached, every replica stops at its next sweep
                                    (results then depend on timing; reach_* stay exact only
                                    without stopping) */
} pdit_opts;

/* pdit_opts_init -- defaults (see the field comments). NULL-safe. */
void pdit_opts_init(pdit_opts *o);

/*
 * pdit_workspace_bytes -- device scratch needed by pdit_anneal_ex for the
 * given options (replicas, mode, ladder, and whether `tables` is requested,
 * which selects the table kernels): query it with the options of the call.
 * Returns 0 for invalid input.
 * The workspace holds every replica's state between calls (permutation,
 * energy, best-so-far, counters, and in PT mode the influence tables), so a
 * call with PDIT_FLAG_RESUME continues exactly where the previous one
 * stopped. With more replicas than the GPU holds at once (not a whole
 * number of rounds), the dot-product kernel and the table kernels with
 * tables in shared memory run each replica's sweeps as parts, separate work
 * units of one launch, in every mode. The parts are up to 16 of 8 to 1000
 * sweeps, or of one sweep per PT exchange period. The workspace then also
 * holds every replica's table (the dot kernel's permuted flow matrix, about
 * n * n bytes; an n x stride int32 influence table) and a 4-byte part
 * counter, whatever the sweep range, so a resumed call over a longer range
 * fits the workspace of the call before it. Results do not depend on the
 * parts.
 */
size_t pdit_workspace_bytes(const pdit_qap *h, const pdit_opts *o);

/*
 * pdit_anneal_ex -- asynchronous annealed p-dit sweep (or parallel
 * tempering) on DEVICE buffers, ordered on o->stream.
 * Without PDIT_FLAG_RESUME, replicas start from a Philox Fisher-Yates
 * permutation. Sweeps [sweep_begin, sweep_end) run; beta comes from
 * o->beta. The best over this call's replicas goes to best_perm/best_cost.
 * Errors (host-detected, nothing launched): PDIT_EINVAL, PDIT_ENOMEM,
 * PDIT_ECUDA. Device audits are reported through o->status.
 */
int pdit_anneal_ex(pdit_qap *h, const pdit_opts *o);

/*
 * pdit_beta_max -- the default largest beta for an instance: 10 / (mean
 * positive Eq. 3 swap energy over all n(n-1)/2 swaps from the identity
 * permutation). A convention of this library; the paper selects its beta
 * range by trial runs instead (Implementation section).
 */
int pdit_beta_max(const pdit_qap *h, double *beta_max);

/*
 * pdit_beta_schedule -- fill out[sweeps] on the host.
 *   kind 0: linear, beta_s = beta_max * s / (sweeps - 1) (0 -> beta_max);
 *   kind 1: geometric, beta_s = (beta_max/1000) * 1000^(s/(sweeps-1)).
 * A single sweep gets beta_max. Errors: PDIT_EINVAL.
 */
int pdit_beta_schedule(int kind, int sweeps, double beta_max, float *out);

/*
 * pdit_anneal_noalloc -- the annealed p-dit sweep of pdit_anneal_ex for
 * callers that cannot allocate device memory: code that runs where
 * cudaMalloc is not allowed or not wanted (inside a framework that owns every
 * device allocation through its own pool, or in a process that must not grow
 * its device footprint after start-up). It makes no cudaMalloc, cudaFree or
 * other allocating call. The paper has no counterpart; this is a packaging
 * of the same computation.
 *   n, D, F  : instance size and DEVICE pointers to the int32 row-major
 *              matrices, symmetric (the values stay on the device, so
 *              this entry point cannot detect the general form), 16 (n+2)
 *              max|D| max|F| < 2^31 (not checked here).
 *   replicas, beta (DEVICE, `sweeps` floats), sweeps, seed: as pdit_anneal.
 *   best_perm (DEVICE, n int32), best_cost (DEVICE, 1 int64): outputs.
 *   status   : DEVICE, 1 int32, or NULL: the PDIT_STATUS_* audit bits of
 *              the call (0 when every audit passed), as pdit_opts.status.
 *              With NULL the audit result is not reported.
 *   stream   : cudaStream_t (NULL = legacy default stream); asynchronous.
 * Replica ids are 0..replicas-1, instance id 0: the results equal those of
 * pdit_anneal / pdit_anneal_ex with the same arguments.
 * The per-replica state lives in one static device array of
 * PDIT_NOALLOC_SCRATCH_BYTES (8 MiB) that every GPU loading this library
 * keeps until exit. A call needs replicas * (8 n + 32) bytes of it plus at
 * most 3 KiB (each of its eleven arrays starts on a 256-byte boundary);
 * larger calls return PDIT_ENOMEM. The staged matrices must fit shared
 * memory with one replica table (n <= 150 or so): PDIT_ENOTSUP otherwise.
 * Every call shares the array and it keeps the last call's contents: calls
 * that overlap on the GPU (different streams, or host threads) race on it;
 * serialise them.
 * First call on each device: CUDA loads this library's device code lazily
 * (the default since CUDA 12.2), so the first call on a device is the one
 * that places the 8 MiB array there. A process that must not grow its
 * footprint later should make one call at start-up (or run with
 * CUDA_MODULE_LOADING=EAGER), and make that first call outside any stream
 * capture; later calls may be captured in a CUDA graph. Every call looks up
 * the array's device address afresh (with the caller's device current), so
 * calls after a cudaDeviceReset use the array of the new context.
 * Errors: PDIT_EINVAL, PDIT_ENOMEM, PDIT_ENOTSUP, PDIT_ECUDA.
 */
#define PDIT_NOALLOC_SCRATCH_BYTES (8u << 20)
int pdit_anneal_noalloc(int n, const int32_t *D, const int32_t *F, int replicas, const float *beta,
                        int sweeps, uint64_t seed, int32_t *best_perm, int64_t *best_cost,
                        int32_t *status, void *stream);

/*
 * pdit_beta_range -- the paper's beta-range selection (Implementation
 * section; CPU-PIM Algorithm section; Fig. 2b): short trials at fixed beta
 * without any exchange, whose ending energies (not best energies) are
 * averaged per beta.
 *   points              : >= 3 beta values, geometric from beta_min to beta_max
 *                         (both > 0; otherwise beta_max_conv/1000 .. 10 beta_max_conv
 *                         with beta_max_conv from pdit_beta_max).
 *   replicas_per_point  : trial replicas per beta value (ids point*rpp + k).
 *   sweeps              : trial length (the paper uses 400 iterations).
 *   seed                : Philox key of the trials.
 *   beta_lo, beta_hi    : outputs: beta_lo = the first (smallest) beta whose
 *                         mean ending energy has come down to within 40% of
 *                         the largest-minus-smallest mean above the smallest
 *                         mean; beta_hi = the beta two grid points past the one
 *                         with the smallest mean (clamped to the grid).
 *   curve               : optional host [points]: the mean ending energies.
 * Synchronous; allocates and frees temporary device buffers.
 * Errors: PDIT_EINVAL, PDIT_ENOMEM, PDIT_ECUDA.
 */
int pdit_beta_range(pdit_qap *h, int points, double beta_min, double beta_max, int replicas_per_point,
                    int sweeps, uint64_t seed, double *beta_lo, double *beta_hi, double *curve);

/*
 * pdit_beta_ladder -- fill out[len] with beta_lo (beta_hi/beta_lo)^(q/(len-1)),
 * the multiplicative ladder of the parallel-tempering replicas (CPU-PIM
 * Algorithm section: 10 replicas per set). Errors: PDIT_EINVAL.
 */
int pdit_beta_ladder(double beta_lo, double beta_hi, int len, float *out);

/*
 * Multi-instance batch: many instances of different sizes annealed by one
 * persistent launch per compiled kernel shape (instances of the same shape
 * share a launch; shapes run concurrently), all enqueued by one call and, on
 * request, captured once into a CUDA graph and replayed. Each instance's
 * results equal those of pdit_anneal_ex with the same arguments.
 */
typedef struct pdit_batch pdit_batch;

typedef struct pdit_batch_item {
    pdit_qap *qap;           /* the instance (not owned; must outlive the batch) */
    int replicas;            /* >= 1, replica ids 0..replicas-1 */
    int sweeps;              /* >= 0 */
    const float *beta;       /* DEVICE [sweeps] */
    uint64_t seed;
    uint32_t instance_id;    /* Philox counter word 0 */
    int32_t *best_perm;      /* DEVICE [n] output */
    int64_t *best_cost;      /* DEVICE [1] output */
    const int64_t *target;   /* DEVICE [1] or NULL: as pdit_opts.target */
    uint64_t *reach_ns;      /* DEVICE [1] or NULL */
    int32_t *reach_sweep;    /* DEVICE [1] or NULL */
} pdit_batch_item;

#define PDIT_BATCH_STOP_AT_TARGET 1u /* replicas of an instance stop once its target is reached */
#define PDIT_BATCH_GRAPH 2u          /* capture the launch sequence into a CUDA graph on the first run */

/*
 * pdit_batch_create -- plan a batch: per instance the launch shape of
 * pdit_launch_shape (its handle's settings apply), instances grouped by
 * shape, work units of one CTA's worth of replicas ordered by decreasing
 * cost, one device workspace. `items` is copied. Allocates device memory
 * and streams. Errors: PDIT_EINVAL, PDIT_ENOMEM, PDIT_ENOTSUP, PDIT_ECUDA.
 */
int pdit_batch_create(const pdit_batch_item *items, int count, uint32_t flags, pdit_batch **out);

/*
 * pdit_batch_run -- anneal every instance of the batch, asynchronously on
 * `stream` (cudaStream_t, NULL = legacy default stream). With
 * PDIT_BATCH_GRAPH the first call captures the sequence on `stream` (which
 * must not be the legacy default stream) and every call launches the graph.
 * Errors: PDIT_EINVAL, PDIT_ECUDA.
 */
int pdit_batch_run(pdit_batch *b, void *stream);

/* pdit_batch_info -- number of shape classes (launches) and workspace bytes. */
int pdit_batch_info(const pdit_batch *b, int *classes, size_t *workspace_bytes);

/* pdit_batch_destroy -- free the batch (not the instances). NULL-safe. */
void pdit_batch_destroy(pdit_batch *b);

/*
 * Serving with continuous batching. Requests (one QAP instance each) are
 * submitted from any host thread; pdit_server_tick, called in a loop by one
 * thread, admits queued requests in arrival order while active slots and the
 * device-memory budget allow (each request's footprint: its matrices,
 * replica state and schedule), runs the next `slice_sweeps` sweeps of every
 * active request in one batched launch per kernel shape, and retires the
 * requests whose schedule has ended. Every replica's whole state stays on
 * the device between slices (permutation, energies, best-so-far, and the
 * influence table of the table kernels or the permuted flow matrix of the
 * dot-product kernel), so a slice resumes exactly where the previous one
 * stopped without rebuilding anything. A request's result is the same as a
 * single pdit_anneal_ex call with instance_id = its request id: alone or in
 * any mix. Device memory of requests is allocated and released in stream
 * order (cudaMallocAsync / cudaFreeAsync on the device's default pool).
 */
typedef struct pdit_server pdit_server;

/*
 * pdit_server_create -- device_budget_bytes: device memory the admitted
 * requests may hold together (one oversize request is still admitted when
 * nothing else holds memory); slice_sweeps: sweeps per tick (>= 1);
 * max_active: requests resident at once. Errors: PDIT_EINVAL, PDIT_ECUDA.
 */
int pdit_server_create(size_t device_budget_bytes, int slice_sweeps, int max_active, pdit_server **out);

/*
 * pdit_server_submit -- queue one request: host D, F (n x n int32,
 * symmetric or not, copied), replicas, sweeps, seed, request_id (Philox counter
 * word 0), and beta (host [sweeps]; NULL = the linear schedule
 * 0 -> pdit_beta_max). Thread-safe. *ticket identifies the request. The
 * values of D and F are checked when the request is admitted (as by
 * qap_create); a request they would make fail ends in state 3.
 * Errors: PDIT_EINVAL, PDIT_ENOMEM.
 */
int pdit_server_submit(pdit_server *s, int n, const int32_t *D, const int32_t *F, int replicas, int sweeps,
                       uint64_t seed, uint32_t request_id, const float *beta, int64_t *ticket);

/*
 * pdit_server_tick -- one scheduling step: pick up the results of earlier
 * slices that have completed, admit, and enqueue one slice for every active
 * request on the server's streams. Asynchronous: the host prepares the next
 * tick while the GPU runs this one (two ticks in flight at most; the call
 * waits only for the tick before the previous one, or, when nothing is left
 * to enqueue, for the oldest outstanding tick). A request counts as active
 * until its result has been picked up. Reports how many requests are active
 * and queued afterwards.
 * Errors: PDIT_EINVAL, PDIT_ECUDA, PDIT_ENOTSUP.
 */
int pdit_server_tick(pdit_server *s, int *active, int *queued);

/*
 * pdit_server_result -- state of a request (0 queued, 1 running, 2 done,
 * 3 failed at admission); when done, its best permutation (host [n]), best
 * cost and latency (seconds from submit to the tick that picked up its
 * result, after its last slice completed).
 * Thread-safe. Errors: PDIT_EINVAL.
 */
int pdit_server_result(pdit_server *s, int64_t ticket, int *state, int32_t *best_perm, int64_t *best_cost,
                       double *latency_s);

/* pdit_server_destroy -- free the server and every request. NULL-safe. */
void pdit_server_destroy(pdit_server *s);

/* ---- QAPLIB text layout ------------------------------------------------- */

/*
 * pdit_read_qaplib -- read an instance in the QAPLIB text layout: the size n,
 * then the n x n matrix A, then the n x n matrix B, whitespace-separated
 * decimal integers (rows may wrap across lines). The objective of such a file
 * is sum_ij A_ij B_{p(i)p(j)}: Eq. 1 with D = A and F = B, so the result of
 * an anneal maps an index of A to an index of B.
 *   path    : file name.
 *   n       : receives n (2 <= n <= PDIT_N_MAX).
 *   D, F    : caller buffers of `capacity` int32 each, row-major; both NULL to
 *             read only n (the whole file is still validated).
 * Errors: PDIT_EINVAL (NULL path or n, one of D/F NULL, n out of range, a
 * token that is not a decimal integer, a value outside int32, too few or too
 * many values), PDIT_ENOMEM (capacity < n*n), PDIT_EIO (cannot open). On
 * error *n is 0 and D, F may be partly written.
 */
int pdit_read_qaplib(const char *path, int *n, int32_t *D, int32_t *F, size_t capacity);

/*
 * pdit_read_qaplib_solution -- read a solution in the QAPLIB layout: "n cost"
 * then the n entries of the permutation, 1-based. perm (caller buffer of
 * `capacity` int32, or NULL) receives it 0-based: perm[i] = the index of B
 * assigned to index i of A (facility at location i).
 * Errors: PDIT_EINVAL (malformed, not a permutation), PDIT_ENOMEM (capacity
 * < n), PDIT_EIO.
 */
int pdit_read_qaplib_solution(const char *path, int *n, int64_t *cost, int32_t *perm, int capacity);

/*
 * pdit_write_qaplib_solution -- write "n cost" and perm (0-based input,
 * written 1-based) in the QAPLIB layout. Errors: PDIT_EINVAL (perm is not a
 * permutation of 0..n-1, n out of range, NULL), PDIT_EIO.
 */
int pdit_write_qaplib_solution(const char *path, int n, int64_t cost, const int32_t *perm);

/*
 * pdit_probe_peaks -- measure, on the current device, the on-chip peaks that
 * bound the sweep kernels (the denominators of their rooflines; the paper
 * reports none): one CTA of 1024 threads per SM, timed with CUDA events and
 * with SM cycles (clock64).
 *   iters : loop trips of each probe (>= 1; 2000 takes a few milliseconds).
 *   out   : host array of 10 doubles:
 *           [0] shared-memory load bandwidth, bytes/s over all SMs
 *               (conflict-free 128-bit ld.shared, 512 contiguous bytes per warp);
 *           [1] the same in bytes per SM clock per SM;
 *           [2] dp4a.s32.s32 thread-operations/s over all SMs;  [3] per SM clock per SM;
 *           [4] mad.lo.s32 thread-operations/s over all SMs;    [5] per SM clock per SM;
 *           [6] mma.sync m16n8k16 f16 -> f32 multiply-adds/s;    [7] per SM clock per SM;
 *           [8] mma.sync m16n8k32 s8 -> s32 multiply-adds/s;     [9] per SM clock per SM.
 * Synchronous on a private stream; allocates and frees two small device
 * buffers. Errors: PDIT_EINVAL, PDIT_ENOMEM, PDIT_ECUDA.
 */
int pdit_probe_peaks(int iters, double *out);

/* pdit_strerror -- static text for an error code. */
const char *pdit_strerror(int code);

/* pdit_last_error -- text of the last CUDA failure on this host thread. */
const char *pdit_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PDIT_H */
