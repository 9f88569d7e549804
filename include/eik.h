/*
 * eik.h -- C ABI of libeik, a GB300 (sm_103a) implementation of the two-scale
 * domain-decomposition method for the static Eikonal boundary value problem
 *     |grad u| = r(x) in Omega,   u = g on Gamma
 * of Martin & Tsai, "A Multiscale Domain Decomposition Algorithm for Boundary
 * Value Problems for Eikonal Equations" (arXiv:1805.04198).
 *
 * Conventions shared by every entry point:
 *  - Every array argument is a DEVICE pointer unless a comment says "host".
 *    The caller allocates and owns all memory; the library never allocates
 *    device memory and never frees caller memory.
 *  - Nodes are indexed [z][y][x] with x fastest.  Node (x, y, z) of an array
 *    lives at element  x + y * stride[1] + z * stride[2]  (stride[0] must be 1).
 *  - Floating-point arrays hold eik_grid.dtype values (float or double).
 *    gamma is one byte per node (nonzero = node belongs to Gamma).
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = the
 *    legacy default stream).  Calls return as soon as the work is enqueued;
 *    results and device-side statistics are valid once the stream completes.
 *  - Validation errors return EIK_EINVAL before any CUDA work is enqueued;
 *    eik_last_error() then describes the problem (thread-local string).
 *  - Device-side bounded waits never trap: if one expires the kernel stops,
 *    and the `error` field of the device statistics is set to
 *    EIK_EDEVICE_TIMEOUT.
 *  - The discrete equation is the first-order Godunov upwind scheme of Sec. 1.1
 *    (eq. "godonuv"), with one-sided differences at the grid boundary.
 */
#ifndef EIK_H
#define EIK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { EIK_F32 = 0, EIK_F64 = 1 } eik_dtype;

typedef enum {
    EIK_OK = 0,
    EIK_EINVAL = -1,          /* invalid argument (nothing enqueued) */
    EIK_ENOMEM = -2,          /* workspace smaller than the size query returned */
    EIK_ECUDA = -3,           /* a CUDA call failed (see eik_last_error) */
    EIK_EDEVICE_TIMEOUT = -4, /* reported in the device stats: a bounded wait expired */
    EIK_EUNSUPPORTED = -5     /* valid request this build does not implement */
} eik_status;

/* Grid description.  ndim = 2 or 3 (1 for eik_dd_solve's one-dimensional
 * method only); n[a] = number of nodes along axis a (n[a] = 1 beyond ndim);
 * h = node spacing (same on every axis). */
typedef struct {
    int ndim;
    int dtype;          /* eik_dtype */
    int64_t n[3];
    int64_t stride[3];  /* element strides of the caller's arrays; stride[0] = 1 */
    double h;
} eik_grid;

/* ------------------------------------------------------------------------- */
/* Plain fast sweeping method (Sec. 1.1, "Initialization", "Sweeping          */
/* iterations", eq. "FSMupdate").                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t sweeps;     /* sweeps executed */
    int converged;      /* 1 if the last sweep changed no value */
    int error;          /* EIK_OK or EIK_EDEVICE_TIMEOUT */
    int64_t updates;    /* Godunov local solves executed */
    int64_t launches;   /* kernels enqueued by this call */
} eik_fsm_stats;

/* Workspace (bytes, device) needed by eik_fsm for this grid; 0 if invalid. */
size_t eik_fsm_workspace_size(const eik_grid *grid);

/*
 * eik_fsm: solve the Godunov system on the whole grid by Gauss-Seidel sweeps
 * in the 2^d orderings of Sec. 1.1 (the sign of x is the outermost loop,
 * -1 first), with the update u = min(u, u~).  Gamma nodes are fixed at g; all
 * other nodes start at +inf.  Stops after the first sweep that changes no value
 * (the discrete solution) or after max_sweeps sweeps.
 *   r      [in]  slowness, > 0 and finite at every non-Gamma node
 *   gamma  [in]  Gamma mask;  g [in] boundary values, read where gamma != 0
 *   u      [out] solution (unreached nodes are +inf)
 *   ws     [in]  scratch of at least eik_fsm_workspace_size(grid) bytes,
 *                256-byte aligned; its contents need no initialisation
 *   stats  [out] device pointer (may be NULL)
 * Returns EIK_OK, EIK_EINVAL, EIK_ENOMEM, EIK_ECUDA or EIK_EUNSUPPORTED.
 */
int eik_fsm(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, void *u,
            int64_t max_sweeps, void *ws, size_t ws_bytes, eik_fsm_stats *stats, void *stream);

/* Workspace for eik_fsm_many; 0 if invalid. */
size_t eik_fsm_many_workspace_size(const eik_grid *grid, int nprob);

/*
 * eik_fsm_many: nprob problems on one grid and one slowness r, differing in
 * their sources: problem p is eik_fsm(grid, r, gamma[p], g[p], u[p], ...).
 * Each problem's result and statistics are exactly those of its own eik_fsm
 * call; the problems run concurrently (one launch per stage for all of them).
 * A project addition for many-source workloads such as travel-time
 * tomography; the paper solves one source set at a time.
 *   nprob        1 .. 65535
 *   gamma, g, u  host arrays [nprob] of device pointers, each laid out as grid
 *   ws           scratch of eik_fsm_many_workspace_size() bytes, 256-byte aligned
 *   stats        device array [nprob] (may be NULL)
 */
int eik_fsm_many(const eik_grid *grid, int nprob, const void *r, const uint8_t *const *gamma,
                 const void *const *g, void *const *u, int64_t max_sweeps, void *ws, size_t ws_bytes,
                 eik_fsm_stats *stats, void *stream);

/* ------------------------------------------------------------------------- */
/* Two-scale domain decomposition (Sec. 3.2, Steps 1-4, Alg. 1-5).            */
/* ------------------------------------------------------------------------- */
typedef struct {
    int tiles[3];          /* subdomains per axis; (n[a]-1) % tiles[a] == 0 (host) */
    int coarse_ratio;      /* c: H = c h, (n[a]-1)/tiles[a] % c == 0; c equal to the
                              subdomain width is the paper's own construction */
    double theta;          /* weight of the theta-parareal correction (Alg. 5) */
    int max_iter;          /* parareal iteration cap (k of the last fine solve) */
    double tol;            /* stop once k >= 1 and max|U^k - U^{k-1}| < tol */
    int64_t max_fsm_sweeps;    /* cap per subdomain solve (Step 3) */
    int64_t max_coarse_sweeps; /* cap per coarse-grid solve (Steps 1 and 4) */
    /* Per-node weight (Sec. 4.2) instead of the constant theta when
     * theta_adaptive != 0 (2-D, 3-D and batched solves): the bound of Theorem 2
     * estimated by eq. secthetaest, (u^k - u^{k-1}) over the weighted mean of
     * the last (up to three) changes of C_H(nbrs U), damped by eq. thetaest
     * [s t + (1 - s) delta t]^+ with s = 1 / (1 + exp((t - x0) / gamma)), and
     * capped at theta_cap when theta_cap > 0.  theta is used where the
     * estimate is undefined (first update, zero or non-finite quotient). */
    int theta_adaptive;
    double omega[3];           /* weights of the last three coarse-solver changes */
    double sig_gamma, sig_delta, sig_x0, theta_cap;
} eik_dd_params;

typedef struct {
    int iters;             /* k of the last fine solve */
    int converged;         /* 1 if stopped by tol */
    int error;             /* EIK_OK or EIK_EDEVICE_TIMEOUT */
    int causal_rounds_max; /* rounds of the causal sweep (Alg. 2) until stable */
    int64_t fsm_sweeps_max, coarse_sweeps_max;
    int64_t fsm_cap_hits, coarse_cap_hits;
    double last_delta;     /* max|U^k - U^{k-1}| of the last coarse update */
    int64_t fine_updates;  /* Godunov local solves executed in the subdomains (Step 3) */
    int64_t coarse_updates;/* local solves executed on the coarse grids (Steps 1, 4) */
    int64_t launches;      /* kernels enqueued by this call */
    int64_t fine_solves_skipped; /* subdomain solves (Step 3) not repeated because the
                                    subdomain's Step 2 data equal those of its previous
                                    solve in this call (its results are kept: the same
                                    solve gives them bit for bit); 2-D solves */
} eik_dd_stats;

/* Workspace (bytes, device) needed by eik_dd_solve; 0 if the request is invalid. */
size_t eik_dd_workspace_size(const eik_grid *grid, const eik_dd_params *params);

/*
 * eik_dd_solve: the two-scale DD / theta-parareal iteration.
 *   Step 1  every shifted coarse grid (spacing H) solved by FSM with Alg. 1,
 *           then the causal sweep (Alg. 2)                        -> U^0, W^0
 *   repeat for k = 0, 1, ...
 *   Step 2  subdomain boundary starting values: U where W.n > 0 for an
 *           inward normal n (inflow), otherwise +inf; Gamma fixed at g
 *   Step 3  FSM in every subdomain (Alg. 3), boundary nodes included (one-
 *           sided differences; an inflow value can only decrease) -> u, w
 *   Alg. 4  u^k, w^k at every coarse-set node from the subdomain copies (the
 *           minimum, where taken, skips copies that kept their inflow U)
 *           stop if k == max_iter or (k >= 1 and max|U^k - U^{k-1}| < tol)
 *   Step 4  Alg. 5 weighted update U = u^k + theta (U~ - C_H(U^k)) swept on
 *           every shifted grid, W = w^k, then the causal sweep   -> U^{k+1}
 * u_out receives the fine solution patched from the last subdomain solves
 * (coarse-set nodes take the Alg. 4 value).  Hitting max_iter is not an error.
 * params is a host pointer; stats a device pointer (may be NULL).
 * ws: scratch of eik_dd_workspace_size() bytes, 256-byte aligned, no
 * initialisation needed.  Returns EIK_OK, EIK_EINVAL, EIK_ENOMEM, EIK_ECUDA or
 * EIK_EUNSUPPORTED.
 *
 * grid->ndim == 1: the one-dimensional method of Sec. 3.1 (eq. 1d, Steps 1-4)
 * on n[0] = N M + 1 nodes, N = tiles[0] subintervals (at most 2048) of M
 * cells; coarse_ratio must equal M (the coarse nodes are the subinterval
 * ends, H = M h).  C_H is eq. 1dgod; Step 1 is the coarse FSM with no causal
 * sweep; Step 3 chooses u^k_i between the two end copies by their fine winds;
 * Step 4 applies the weighted update where W^k = w^k = W~, u^k elsewhere,
 * then the causal sweep of Sec. 3.1 in both directions until stable.  The
 * per-node weight (theta_adaptive) is rejected.  The whole iteration runs in
 * one cooperative kernel launch (the subintervals spread over one CTA per SM,
 * the coarse state in CTA 0's shared memory, bounded grid barriers between
 * the phases); the workspace holds a few control words, U and W, and the
 * subintervals' end copies (a few kB).
 */
int eik_dd_solve(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                 const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes,
                 eik_dd_stats *stats, void *stream);

/*
 * eik_dd_coarse_state: the coarse state a 2-D DD workspace holds (same grid
 * and params as the call that filled it, after `stream` has run that call),
 * scattered to fine indexing: U at every coarse-set node into U_out (grid
 * dtype, strides of grid) and W into W_out (one byte per node: wind
 * components w_a = ((byte >> 2a) & 3) - 1, a = x, y).  After
 * eik_dd_shard_start (set-up, Step 1, causal sweep) that is U^0, W^0.  After
 * eik_dd_solve or eik_dd_shard_coarse stopped at iteration k it is U^k (u^k
 * with the constant weight 0, whose Step 4 result Alg. 4 writes in place) and
 * W = w^k (Alg. 4 sets W to the chosen fine winds).  Other nodes are left
 * untouched; either output may be NULL.  Returns EIK_OK, EIK_EINVAL,
 * EIK_ENOMEM, EIK_ECUDA or EIK_EUNSUPPORTED (3-D and 1-D).
 */
int eik_dd_coarse_state(const eik_grid *grid, const eik_dd_params *params, const void *ws, size_t ws_bytes,
                        void *U_out, uint8_t *W_out, void *stream);

/*
 * Sharded 2-D solve: the phases of eik_dd_solve for a caller that splits the
 * subdomain solves (Steps 2-3 of Sec. 3.2, which the paper runs "in parallel"
 * for every subdomain) over several processes, each owning a slab of
 * subdomain rows [row0, row1) along y, while every process keeps the whole
 * coarse state (Alg. 4, Step 4 and Alg. 2 run replicated on the same data, so
 * the update size that stops the iteration is the same everywhere and needs no
 * reduction).  Per iteration k = 0, 1, ...:
 *   eik_dd_shard_fine   Steps 2-3 on the slab's subdomains; each subdomain's
 *                       copies at its coarse-set nodes (the values Alg. 4
 *                       chooses from) go to its record of xbuf;
 *   the caller gathers every slab's records into its own xbuf (records of
 *                       subdomain t at offset t * record_bytes, t = ty * tx +
 *                       x-index, so a slab's records are one contiguous range:
 *                       one all-gather);
 *   eik_dd_shard_coarse the records into the copies, Alg. 4 and the stop test
 *                       of iteration k, then (k < max_iter) Step 4, the causal
 *                       sweep and the update size; statistics into stats
 *                       (device) as eik_dd_solve writes them, except that
 *                       fine_updates, fsm_sweeps_max, fsm_cap_hits and
 *                       fine_solves_skipped count this process's subdomains
 *                       (sum, max, sum and sum over the processes give
 *                       eik_dd_solve's).  The iteration stops
 *                       after k when stats.converged, stats.error or
 *                       k == max_iter.
 * eik_dd_shard_start (set-up, Step 1 and its causal sweep) runs once before.
 * Arguments are those of eik_dd_solve (workspace eik_dd_workspace_size, per
 * process); xbuf is a device buffer of eik_dd_shard_exchange_bytes bytes,
 * 16-byte aligned.  After the last iteration u_out holds, on every process,
 * all coarse-set nodes and the other nodes of its own slab's subdomains.  With
 * one slab covering every row the phases reproduce eik_dd_solve bitwise.
 * Validation failures return EIK_EINVAL (a 3-D grid: EIK_EUNSUPPORTED).
 */
size_t eik_dd_shard_exchange_bytes(const eik_grid *grid, const eik_dd_params *params, size_t *record_bytes);
int eik_dd_shard_start(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                       const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, void *stream);
int eik_dd_shard_fine(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                      const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, int row0, int row1,
                      void *xbuf, void *stream);
int eik_dd_shard_coarse(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                        const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, int k,
                        const void *xbuf, eik_dd_stats *stats, void *stream);

/* ------------------------------------------------------------------------- */
/* Gradient through the converged discrete system (a project addition: the    */
/* paper has no gradient).                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t sweeps;     /* adjoint sweeps executed */
    int converged;      /* 1 if the last sweep changed nothing */
    int error;          /* EIK_OK or EIK_EDEVICE_TIMEOUT */
    int64_t launches;   /* kernels enqueued by this call */
} eik_adjoint_stats;

/* Workspace (bytes, device) needed by eik_dd_adjoint; 0 if invalid (2-D only). */
size_t eik_dd_adjoint_workspace_size(const eik_grid *grid);

/*
 * eik_dd_adjoint: dJ/dr for a scalar J(u), at a converged solution u of the
 * Godunov system of Sec. 1.1 (as returned by eik_fsm, or by eik_dd_solve once
 * it has converged).  At every reached non-Gamma node j, u_j = F(a_j, r_j)
 * with a_j the neighbour minima of the branch Alg. 3 takes; the adjoint state
 * lambda = dJ/du + (dF/du)^T lambda is solved by Gauss-Seidel sweeps in the
 * 2^d orderings (the system is causal in reverse), and
 * dJ/dr_j = lambda_j dF_j/dr_j (0 at Gamma and at unreached nodes).  At a tie
 * (|a-b| = r h exactly, or equal neighbour values) the one-sided derivative of
 * the branch Alg. 3 selects is used.
 *   r, gamma, u  [in]  as for eik_fsm; u the forward solution
 *   dJdu         [in]  dJ/du at every node
 *   grad_r       [out] dJ/dr at every node
 *   max_sweeps   cap on the adjoint sweeps
 *   ws           scratch of eik_dd_adjoint_workspace_size() bytes, 256-byte aligned
 *   stats        [out] device pointer (may be NULL)
 */
int eik_dd_adjoint(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *u, const void *dJdu,
                   void *grad_r, int64_t max_sweeps, void *ws, size_t ws_bytes, eik_adjoint_stats *stats,
                   void *stream);

/* Workspace for eik_dd_adjoint_many; 0 if invalid. */
size_t eik_dd_adjoint_many_workspace_size(const eik_grid *grid, int nprob);

/*
 * eik_dd_adjoint_many: the adjoint of eik_dd_adjoint for nprob problems on
 * one grid and one slowness r (problem p: sources gamma[p], forward solution
 * u[p], dJ/du of that problem dJdu[p]).  grad_r[p] (when grad_r and grad_r[p]
 * are not NULL) receives exactly eik_dd_adjoint's result for problem p;
 * grad_sum (when not NULL) receives g_0 + g_1 + ... + g_{nprob-1} of those
 * gradients, added in problem order.  At least one of grad_r and grad_sum is
 * given.  A project addition (gradient of a sum of per-source misfits).
 *   gamma, u, dJdu, grad_r   host arrays [nprob] of device pointers
 *   ws     scratch of eik_dd_adjoint_many_workspace_size() bytes, 256-byte aligned
 *   stats  device array [nprob] (may be NULL)
 */
int eik_dd_adjoint_many(const eik_grid *grid, int nprob, const void *r, const uint8_t *const *gamma,
                        const void *const *u, const void *const *dJdu, void *const *grad_r, void *grad_sum,
                        int64_t max_sweeps, void *ws, size_t ws_bytes, eik_adjoint_stats *stats, void *stream);

/* ------------------------------------------------------------------------- */
/* Batched DD: many independent 2-D problems of mixed sizes, each solved by    */
/* the iteration of eik_dd_solve (Sec. 3.2).  A project addition: the paper     */
/* solves one problem at a time.                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int fine_queue;     /* Steps 2+3: 0 = one CTA per subdomain; 1 = the CTAs
                           that fit on the GPU draw subdomains from a queue */
    int coarse_queue;   /* the same for the shifted coarse grids (Steps 1, 4) */
    int ctas_per_sm;    /* queue forms: CTAs per SM (0 = as many as fit) */
    int largest_first;  /* hand out the boxes of the largest problems first */
} eik_dd_batch_config;

/* Workspace (bytes, device) for eik_dd_solve_batched; 0 if invalid.  The size
 * does not depend on the configuration. */
size_t eik_dd_batched_workspace_size(int nprob, const eik_grid *grids, const eik_dd_params *params);

/*
 * eik_dd_solve_batched: nprob independent problems, problem p being
 * eik_dd_solve(&grids[p], r[p], gamma[p], g[p], &params[p], u_out[p], ...).
 * Each problem produces exactly the u_out and statistics of its own
 * eik_dd_solve call (same arithmetic, same stopping rule on its own max_iter
 * and tol), except that causal_rounds_max counts the rounds of the batch-wide
 * causal sweep and `launches` the kernels of the whole batch.
 *   nprob            1 .. 65535 problems, all 2-D and of one dtype
 *   grids, params    host arrays [nprob]
 *   r, gamma, g,     host arrays [nprob] of device pointers, laid out as for
 *   u_out            eik_dd_solve
 *   config           host pointer, or NULL for {0, 0, 0, 1}; it changes only
 *                    the launch shapes, never a result
 *   ws               scratch of eik_dd_batched_workspace_size() bytes,
 *                    256-byte aligned, no initialisation needed
 *   stats            device array [nprob] (may be NULL)
 * The call only enqueues kernels on `stream` (no allocation, no host
 * synchronisation, no host<->device copy), so it may be captured into a CUDA
 * graph; the graph then replays the same problems with the same pointers.
 * Returns EIK_OK, EIK_EINVAL, EIK_ENOMEM, EIK_ECUDA or EIK_EUNSUPPORTED.
 */
int eik_dd_solve_batched(int nprob, const eik_grid *grids, const void *const *r, const uint8_t *const *gamma,
                         const void *const *g, const eik_dd_params *params, void *const *u_out,
                         const eik_dd_batch_config *config, void *ws, size_t ws_bytes, eik_dd_stats *stats,
                         void *stream);

/*
 * eik_dd_batched_autotune: times eik_dd_solve_batched on this batch under each
 * candidate configuration (queue or one-CTA-per-box forms of the two box
 * stages, CTAs per SM, item order), with every problem's max_iter lowered to
 * min(max_iter, tune_iters), and returns the fastest in *best (host) and its
 * time in *best_ms (host, may be NULL).  It overwrites u_out and synchronises
 * the stream after each candidate: call it before capturing a graph.
 */
int eik_dd_batched_autotune(int nprob, const eik_grid *grids, const void *const *r, const uint8_t *const *gamma,
                            const void *const *g, const eik_dd_params *params, void *const *u_out, int tune_iters,
                            void *ws, size_t ws_bytes, eik_dd_batch_config *best, double *best_ms, void *stream);

/*
 * eik_dd_solve_noalloc: eik_dd_solve for callers that cannot allocate device
 * memory (for example a host whose device allocator belongs to another runtime
 * that must not be bypassed, or a real-time loop that forbids allocation once
 * it runs).  It takes no workspace: the scratch is a static
 * device array of EIK_NOALLOC_SCRATCH_BYTES inside the library, which every
 * GPU that loads the library keeps until the process exits.  This entry point
 * has no counterpart in the paper; it only changes where the scratch lives.
 *  - Problems whose eik_dd_workspace_size exceeds the array are rejected with
 *    EIK_ENOMEM before any work is enqueued.
 *  - The first call on a device looks up the array's device address (a
 *    cudaGetSymbolAddress call, made once per device with that device
 *    current); make that first call before any stream capture.
 *  - It calls no cudaMalloc/cudaFree or other allocating routine.
 *  - All calls share the one array: calls whose work overlaps on the GPU
 *    (different streams, or different host threads) race and must be
 *    serialised by the caller.  The array keeps the last call's contents; the
 *    solve needs no cleared scratch.
 * Arguments and results are those of eik_dd_solve.
 */
#define EIK_NOALLOC_SCRATCH_BYTES (32u << 20)
int eik_dd_solve_noalloc(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                         const eik_dd_params *params, void *u_out, eik_dd_stats *stats, void *stream);

/* ------------------------------------------------------------------------- */
/* Optional per-kernel timing (a benchmarking aid, off by default).  While     */
/* enabled, every kernel the library launches is bracketed by two CUDA events  */
/* recorded on the launch's own stream.  Not thread-safe; enable it only when  */
/* one host thread drives the library.                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    const char *name;   /* static string owned by the library */
    int64_t launches;
    double total_ms;    /* sum of event-measured launch durations */
    double max_ms;
} eik_kernel_time;

/* Turns event bracketing on (on != 0) or off.  Returns the previous state. */
int eik_profile_enable(int on);

/* Waits for every recorded event, writes up to max_entries per-kernel totals
 * (host array) and clears the record.  Returns the number of kernels with at
 * least one timed launch (may exceed max_entries), or EIK_ECUDA. */
int eik_profile_collect(eik_kernel_time *out, int max_entries);

/*
 * eik_set_wait_limit: sets, on the current device, how many times a
 * device-side wait may poll before it gives up.  The waits are the hand-offs
 * between the warps and CTAs of a sweep and the grid barriers of the
 * cooperative kernels; an expired wait records EIK_EDEVICE_TIMEOUT in the
 * call's device statistics (eik_dd_stats.error, eik_fsm_stats.error, ...),
 * makes the rest of that call return early, and never traps, so the context
 * stays usable.  Each poll sleeps 32 ns to 1 us.  0 restores the default of
 * 2^22 polls (seconds).  A small limit makes ordinary waits expire: it exists
 * to test the timeout path.  It applies to work enqueued after it returns
 * (it is a cudaMemcpyToSymbol, ordered against the legacy default stream);
 * do not change it while a call is running.  No counterpart in the paper.
 * Returns EIK_OK, EIK_EINVAL (negative value) or EIK_ECUDA.
 */
int eik_set_wait_limit(int64_t iterations);

/* Thread-local description of the last non-OK status returned on this thread. */
const char *eik_last_error(void);

/* Library ABI version (major * 100 + minor). */
int eik_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EIK_H */
