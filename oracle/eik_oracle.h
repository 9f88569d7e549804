/*
 * eik_oracle.h -- serial FP64 CPU oracle for the two-scale domain-decomposition
 * Eikonal solver of Martin & Tsai, "A Multiscale Domain Decomposition Algorithm
 * for Boundary Value Problems for Eikonal Equations" (arXiv:1805.04198).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously-correct
 * statement of what the method computes.  Only the test suite, the smoke check
 * and the CPU-baseline leg of bench.py load it.  It shares no code with the CUDA
 * path (no headers, no helpers, no constants) and must never be called by it.
 *
 * Layout: nodes indexed [z][y][x], axis 0 (x) fastest, n[a] nodes per axis
 * (unused axes have n[a] = 1).  All arrays are caller-owned, FP64.
 * A wind is stored as d signed bytes per node (component a at [3*node + a]),
 * each in {-1, 0, +1}, +1 meaning travel toward +axis (upwind neighbour on the
 * minus side).
 */
#ifndef EIK_ORACLE_H
#define EIK_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* Godunov local solve, Sec. 1.1 eq. (godonuv) with Alg. 3's per-axis choice.
 * vm[a], vp[a]: neighbour values on the minus / plus side of axis a
 * (+inf where the neighbour does not exist: the one-sided rule of Sec. 1.1).
 * Returns u~; writes the wind of the branch taken into w[0..d-1]. */
double orc_local_solve(int d, const double *vm, const double *vp, double rh, signed char *w);

/* Plain fast sweeping method (Sec. 1.1) over a whole grid.
 * gamma[i] != 0 marks Gamma (u fixed at g[i]); every other node starts at +inf.
 * Sweeps cycle through the 2^d orderings of Sec. 1.1 until one sweep changes no
 * value or max_sweeps sweeps ran.  w (nullable) receives the wind of the local
 * solve at the final state.  Returns the number of sweeps; *converged set to 1
 * if the last sweep changed nothing. */
long orc_fsm(int d, const long *n, double h, const double *r, const unsigned char *gamma,
             const double *g, double *u, signed char *w, long max_sweeps, int *converged);

/* Dijkstra / fast-marching solve of the same discrete system (Sec. 1.1: the
 * scheme is causal, so accepting nodes in increasing order of value gives its
 * solution).  Used only to cross-check orc_fsm. */
void orc_fmm(int d, const long *n, double h, const double *r, const unsigned char *gamma,
             const double *g, double *u);

typedef struct {
    int d;
    long n[3];            /* nodes per axis */
    double h;             /* fine spacing */
    int tiles[3];         /* subdomains per axis, (n[a]-1) % tiles[a] == 0 */
    int c;                /* coarse ratio, H = c h; (n[a]-1)/tiles[a] % c == 0 */
    double theta;         /* weight of the theta-parareal correction (Sec. 2, Alg. 5) */
    int max_iter;         /* parareal iteration cap */
    double tol;           /* stop when max |U^k - U^{k-1}| < tol (k >= 1) */
    long max_fsm_sweeps;  /* per fine subdomain solve */
    long max_coarse_sweeps; /* per coarse grid solve (Step 1 and Step 4) */
    /* Per-node theta (Sec. 4.2, eq. secthetaest with the damping of eq.
     * thetaest) when theta_adaptive != 0; `theta` is then the value used
     * where the estimate is undefined (first update, non-finite quotient). */
    int theta_adaptive;
    double omega[3];      /* weights of the last three coarse-solver changes */
    double sig_gamma, sig_delta, sig_x0;  /* gamma, delta, x_0 of eq. thetaest */
    double theta_cap;     /* upper bound on the damped estimate (<= 0: none) */
} orc_dd_params;

typedef struct {
    int iters;            /* k of the last fine solve (number of coarse updates done) */
    int converged;        /* 1 if stopped by tol */
    double last_delta;    /* max |U^k - U^{k-1}| of the last update (inf if none) */
    long fsm_sweeps_max;  /* largest sweep count of any fine subdomain solve */
    long coarse_sweeps_max; /* largest sweep count of any coarse grid solve */
    long fsm_cap_hits;    /* fine solves stopped by max_fsm_sweeps */
    long coarse_cap_hits; /* coarse solves stopped by max_coarse_sweeps */
    long causal_rounds_max; /* rounds of 2^d causal passes until no change (>=1) */
    long long fine_updates;   /* local solves executed in subdomain sweeps */
    long long coarse_updates; /* local solves executed in coarse-grid sweeps */
} orc_dd_stats;

/* The two-scale DD / theta-parareal iteration of Sec. 3 (Steps 1-4, Alg. 1-5),
 * d = 2 or 3.  Outputs:
 *   u_out     fine solution patched from the last subdomain solves (coarse-set
 *             nodes take the Alg. 4 value);
 *   U_out     (nullable) coarse values U^k of the last iterate, +inf... only
 *             meaningful on the coarse set, NaN elsewhere;
 *   delta_log (nullable) max_iter+1 entries: delta_log[k] = max|U^k - U^{k-1}|
 *             (delta_log[0] = inf).
 * Returns 0 on success, -1 on invalid parameters. */
/* Per-node weight estimate of Sec. 4.2 (eq. secthetaest damped by eq.
 * thetaest, capped at p->theta_cap when positive): du = u^k - u^{k-1},
 * dC[s] = C_H(nbrs U^{k-s}) - C_H(nbrs U^{k-1-s}), s < n (n <= 3).  Returns
 * `fallback` when the quotient is undefined (no term, zero or non-finite). */
double orc_theta_estimate(const orc_dd_params *p, double du, const double *dC, int n, double fallback);

int orc_dd(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
           double *u_out, double *U_out, double *delta_log, orc_dd_stats *st);

/* Alg. 5 on one dense box (Step 4 of Sec. 3.2): C_H(nbrs U^k) from Uk into
 * Cold (nullable), then the weighted sweeps into U.  Per node: fixed (Gamma,
 * U = g), uk / wk (Alg. 4 output), Wk (W^k), axes (bit k: the node lies on a
 * coarse line of axis k; the agreement test runs on those axes), theta.
 * Winds are 3 bytes per node.  Returns sweeps; *capped = 1 if max_sweeps ran
 * without a sweep that changed nothing. */
long orc_step4_box(int d, const long *n, double H, const double *r, const unsigned char *fixed, const double *g,
                   const double *Uk, const double *uk, const signed char *wk, const signed char *Wk,
                   const int *axes, const double *theta, long max_sweeps, double *U, double *Cold, int *capped);

/* Alg. 4's choice among the ncopies subdomain copies of one coarse-set node
 * (enumerated axis 0 fastest, minus side first on each interface axis of B;
 * nc[k] copies along axis k).  Returns the index of the chosen copy. */
int orc_alg4_select(int d, int B, const int *nc, int ncopies, const double *u, const signed char *w,
                    const unsigned char *echo, const signed char *W);

/* Per-node weight of Sec. 4.2 from the history of one node: Ck = C^k,
 * C1..C3 = C^{k-1..k-3} (C^m = C_H(nbrs U^m); the first nhist are used),
 * uk = u^k, uprev = u^{k-1}; the constant p->theta when not adaptive or
 * nhist < 1. */
double orc_theta_node(const orc_dd_params *p, int nhist, double Ck, double C1, double C2, double C3, double uk,
                      double uprev);

/* orc_dd with a record of one node (fine index probe_node): probe_log[4k..4k+3]
 * = u^k, C^k = C_H(nbrs U^k) (from Step 4 of iteration k), the weight used
 * for U^{k+1}, and U^k; NaN where an iteration did not compute it. */
int orc_dd_probe(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
                 double *u_out, double *U_out, double *delta_log, orc_dd_stats *st, long probe_node,
                 double *probe_log);

/* orc_dd with hooks for tests that compare a lower-precision solve (every
 * pointer may be NULL).  W0_out [3 N] = W^0 (three components per node; 0 off
 * the coarse set) and margin_out [N] = at each coarse-set node the smallest
 * margin of the Alg. 1 decisions behind its wind (NaN elsewhere), both from
 * this solve's own Step 1.  U0_in [N] / W0_in [3 N] replace U^0 / W^0 at the
 * coarse-set nodes after Step 1 (the other solve's Step 1), so that Steps 2-3
 * and Alg. 4 take that solve's Step 2 decisions.  copies_out [4 N] = the
 * subdomain copies of iteration 0 at the coarse-set nodes (slot bit 0: the
 * node lies on the subdomain's x = 0 face on an interior x interface, bit 1 the
 * same for y; NaN where absent) and cmargin_out [N] = per coarse-set node the
 * smallest margin of the decisions behind Alg. 4's choice (Alg. 3 at each
 * copy, whether an inflow copy kept U).  Test
 * infrastructure: the method's arithmetic is orc_dd's. */
int orc_dd_margins(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
                   double *u_out, orc_dd_stats *st, signed char *W0_out, double *margin_out,
                   const double *U0_in, const signed char *W0_in, double *copies_out, double *cmargin_out);

/* The one-dimensional method of Sec. 3.1.  Fine grid of N*M+1 nodes, spacing
 * h; coarse nodes every M fine nodes (H = M h). */
typedef struct {
    long N, M;
    double h;
    double theta;
    int max_iter;
    double tol;
    long max_fsm_sweeps, max_coarse_sweeps;
} orc_dd1_params;

typedef struct {
    int iters, converged;
    double last_delta;
    long fsm_sweeps_max, coarse_sweeps_max, fsm_cap_hits, coarse_cap_hits, causal_rounds_max;
    long long fine_updates;
} orc_dd1_stats;

/* Steps 1-4 of Sec. 3.1 on r, gamma, g (fine grid).  u_out: patched fine
 * solution of the last iterate.  Logs (nullable, (max_iter+1) x (N+1) each):
 * U_log[k] = U^k, u_log[k] = u^k (Step 3's choice), W_log[k] = W^k,
 * Upre_log[k] = the Step 4 result of iteration k before the causal sweep. */
int orc_dd1(const orc_dd1_params *p, const double *r, const unsigned char *gamma, const double *g, double *u_out,
            double *U_log, double *u_log, double *Upre_log, signed char *W_log, orc_dd1_stats *st);

/* Discrete adjoint of the converged Godunov system at u (see oracle source):
 * given dJ/du at every node, returns dJ/dr at every node (0 on Gamma and on
 * unreached nodes). */
void orc_adjoint(int d, const long *n, double h, const double *r, const unsigned char *gamma,
                 const double *u, const double *dJdu, double *dJdr);

#ifdef __cplusplus
}
#endif
#endif
