/*
 * sdd.h - C ABI of the GB300 stochastic-deterministic domain decomposition
 * (SDD) mesh generator: Monte Carlo evaluation of the Feynman-Kac
 * representation of the linear Winslow generator at subdomain-interface nodes,
 * followed by independent Dirichlet solves on the subdomains.
 *
 * Method: Bihlo & Haynes, "Parallel stochastic methods for PDE based grid
 * generation" (arXiv 1310.3435).
 *   - generator  -div(c grad u) = 0 on the unit square, u = boundary map on the
 *     boundary (eq. WinslowTypeGridGenerator, §2.1); c = w or c = 1/w;
 *   - u(x) = E[boundary map at the first exit point of X]  (eq. ...StochasticSolutionA)
 *     for dX = grad(ln c) dt + sqrt(2) dW (eq. ...StochasticSolutionB, with the
 *     noise scale fixed by the expanded form, eq. ...Expanded);
 *   - Euler-Maruyama with time step dt, or exponential time stepping of mean
 *     step dt; an exit test at the end of each step, optionally with the
 *     Brownian-bridge crossing probability (§2.2); sample mean over N paths
 *     per node, error ~ N^-1/2 (§2.2);
 *   - interface values as Dirichlet data for independent subdomain solves,
 *     no iteration between subdomains (§2.1, Fig. 1; §3.5); conservative
 *     centred differences on a uniform grid (§3.2);
 *   - around that path: few-point interfaces (§3.6), the fully probabilistic
 *     mesh (§3.3), Perona-Malik smoothing of the whole mesh (§3.4) or of each
 *     subdomain (§3.5, §4), mesh quality (§3.1, §3.3),
 *     batches of meshes, runs split over calls with checkpoints.
 *
 * Conventions (all entry points):
 *   - Return SDD_OK (0) on success, a negative SDD_ERR_* code on failure;
 *     sdd_last_error() then gives a message (thread-local, valid until the
 *     next call on the same thread).
 *   - Grid: n x n nodes (s_i, t_j) = (i, j)/(n-1).  Mesh arrays are
 *     [n][n][2] doubles indexed [j][i][comp] (row j = t index), comp 0 = u1
 *     (the s-like coordinate), comp 1 = u2.
 *   - Interface nodes: the interior nodes (1 <= i, j <= n-2) on the interface
 *     lines i in I_x or j in I_y, I_k = round(k (n-1)/s) (halves up), each
 *     node once, ordered by j then i.  Per-node arrays are [n_nodes][2].
 *   - Output and input arrays are owned by the caller.  A pointer is device
 *     memory if cudaPointerGetAttributes reports a device or managed
 *     allocation, else host memory.  With device pointers a call is
 *     asynchronous and ordered on `stream` (a cudaStream_t, NULL = legacy
 *     default stream); with any host pointer among its outputs it copies and
 *     synchronises `stream` before returning.
 *   - A plan owns device buffers on the device that was current when it was
 *     created; calls must be made with that device current.  A plan is not
 *     thread-safe; concurrent calls on different plans are.
 */
#ifndef SDD_H
#define SDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SDD_OK                  0
#define SDD_ERR_INVALID_ARG   (-1)
#define SDD_ERR_OOM           (-2)
#define SDD_ERR_CUDA          (-3)
#define SDD_ERR_NOT_CONVERGED (-4)
#define SDD_ERR_NO_DEVICE     (-5)
/* There is no status code for a path stopped by the step cap: such paths are
 * scored at their nearest side and counted (sdd_mc_stats.non_exits).  Time
 * limits and cancellation belong to the caller's request loop (the Python
 * server cancels a request between launches), not to a call of this ABI. */

/* ---- density families (shapes of the paper's monitor functions) ---- */
/* BUMPS: params = [nb, (A, cs, ct, ks, kt) x nb], nb <= 6:
 *        w = 1 + sum A exp(-ks (s-cs)^2 - kt (t-ct)^2)   (eq. MonitorFunctionRunningExample)
 * RING : params = [A, cs, ct, k, r0]:
 *        w = 1 + A sech^2(k (|x - c| - r0))             (ring of eq. FiveRingMonitorFunction)
 * RIDGE: params = [A, k, t0, a, f]:
 *        w = 1 + A exp(-k (t - t0 - a sin(2 pi f s))^2)  (eq. MackenzieMonitorFunction)
 * TABLE: a density given as a table of ln w at the tn x tn nodes
 *        (a/(tn-1), b/(tn-1)), e.g. from a numerical solution: `table` (host,
 *        copied at plan creation) holds row b = 0 (t = 0) first, tn values per
 *        row; w = exp(L) with L the bilinear interpolant of the nodes, and the
 *        drift is sgn grad L, the interpolant's exact cellwise gradient.  The
 *        FP32 path kernel reads an FP32 copy through the read-only cache. */
#define SDD_FAMILY_BUMPS 0
#define SDD_FAMILY_RING  1
#define SDD_FAMILY_RIDGE 2
#define SDD_FAMILY_TABLE 3
#define SDD_MAX_TABLE    4097
#define SDD_MAX_BUMPS    6
#define SDD_MAX_PARAMS   32

/* coefficient of the generator: c = w (the paper's eq. as printed) or c = 1/w */
#define SDD_COEF_W     0
#define SDD_COEF_INV_W 1

/* boundary map u|boundary:
 *   IDENTITY : u = (s, t)
 *   PAPER_1D : u1 = 0 on s=0, 1 on s=1; u2 = 0 on t=0, 1 on t=1; u1 on t=0,1 and
 *              u2 on s=0,1 from the 1D generator -(c u')' = 0 discretised by
 *              the conservative three-point difference (§3.2)
 *   TABLE    : caller's tables edges[2 comps][4 edges][n] (host pointer), edge
 *              0 bottom (t=0, along s), 1 top (t=1), 2 left (s=0, along t),
 *              3 right (s=1).  Rows t=0 and t=1 take the bottom/top tables,
 *              corners included. */
#define SDD_BMAP_IDENTITY 0
#define SDD_BMAP_PAPER_1D 1
#define SDD_BMAP_TABLE    2

/* path precision: FP64 stepping, or FP32 stepping with FP64 exit-point
 * interpolation and compensated FP64 per-node sums */
#define SDD_FP64      0
#define SDD_FP32_STEP 1

/* exit test of a step (§2.2): at the end of the step only, or also the
 * Brownian-bridge test: a step x -> y that stayed inside crossed side s with
 * probability exp(-d_s(x) d_s(y) / dt) (d_s = distance to side s, noise
 * sqrt(2) dW), decided by the uniforms of Philox counter (k, path, node, 1) in
 * the side order s=0, s=1, t=0, t=1; skipped when every product is >= 23 dt
 * (probability below 2^-33, the smallest FP64 uniform), with FP32 stepping
 * >= 16.7 dt (below 2^-24, the smallest FP32 uniform), so the skip decides
 * nothing; exit point: the side, with the mean of the two
 * tangential coordinates.  Cuts the O(sqrt(dt)) exit bias to O(dt). */
#define SDD_EXIT_END_OF_STEP 0
#define SDD_EXIT_BRIDGE      1

/* time stepping of the paths (§2.2):
 *   EULER       : Euler-Maruyama with the constant step dt
 *   EXPONENTIAL : exponential time stepping (after Jansons and Lythe): step k
 *                 has the random length h = dt E, E = -ln U a unit-mean
 *                 exponential (density lambda exp(-lambda h), lambda = 1/dt),
 *                 U from word k mod 4 of Philox counter (k/4, path, node, 2);
 *                 the update is the Euler-Maruyama
 *                 one with step h, and the Brownian-bridge test (with
 *                 SDD_EXIT_BRIDGE) uses h in place of dt.  dt is the mean
 *                 step 1/lambda; the default step cap stays ceil(2/dt). */
#define SDD_STEP_EULER       0
#define SDD_STEP_EXPONENTIAL 1

/* few-point interface (§3.6): where the Monte Carlo estimate is computed; the
 * other interface nodes are interpolated linearly along their interface line
 * between the nearest Monte Carlo nodes or the line's boundary ends
 *   ALL        : every interface node (default)
 *   EQUISPACED : k equispaced points per interface line, positions
 *                round(r (n-1)/(k+1)), r = 1..k
 *   EXTREMA    : the nodes where the first or the second centred difference
 *                of the density w along the line has a local extremum
 * Crossings of two interface lines are always Monte Carlo nodes. */
#define SDD_PLACE_ALL        0
#define SDD_PLACE_EQUISPACED 1
#define SDD_PLACE_EXTREMA    2

/* subdomain solvers (each to the relative residual tol of the FP64 system)
 *   SOR                   : FP64 red-black SOR
 *   CG_FP32_REFINE        : FP64 iterative refinement around FP32 conjugate
 *                           gradients preconditioned by one geometric multigrid
 *                           V-cycle (bilinear transfers, Galerkin coarse
 *                           operators, Gauss-Seidel smoothing); tens of
 *                           iterations where diagonal preconditioning takes
 *                           hundreds to thousands
 *   CG_JACOBI_FP32_REFINE : the same refinement around diagonally
 *                           (Jacobi) preconditioned FP32 CG */
#define SDD_SOLVER_SOR                   0
#define SDD_SOLVER_CG_FP32_REFINE        1
#define SDD_SOLVER_CG_JACOBI_FP32_REFINE 2

typedef struct sdd_plan sdd_plan;

typedef struct {
    int32_t family;                    /* SDD_FAMILY_* */
    int32_t coef_mode;                 /* SDD_COEF_* */
    int32_t n_params;                  /* used entries of params (0 for TABLE) */
    int32_t tn;                        /* TABLE: nodes per side, 2..SDD_MAX_TABLE; else 0 */
    double params[SDD_MAX_PARAMS];
    const double* table;               /* TABLE: host [tn][tn] ln w; else NULL */
} sdd_density;

typedef struct {
    int32_t mode;                      /* SDD_BMAP_* */
    int32_t reserved;
    const double* edges;               /* host [2][4][n] for SDD_BMAP_TABLE, else NULL */
} sdd_bmap;

typedef struct {
    uint64_t paths_per_node;           /* N >= 2, < 2^32 */
    double dt;                         /* Euler-Maruyama step (mean step with
                                          SDD_STEP_EXPONENTIAL), > 0 */
    uint64_t seed;                     /* Philox4x32-10 key (lo, hi words) */
    int32_t precision;                 /* SDD_FP64 | SDD_FP32_STEP */
    int32_t chunk;                     /* paths per work item: 0 = automatic, else a
                                          multiple of 32, at most 8192 */
    uint64_t max_steps;                /* step cap per path, 0 = ceil(2/dt) */
    double tie_delta;                  /* <0: default (1e-11 FP64, 0 FP32) */
    int32_t exit_test;                 /* SDD_EXIT_END_OF_STEP | SDD_EXIT_BRIDGE */
    int32_t stepper;                   /* SDD_STEP_EULER | SDD_STEP_EXPONENTIAL */
    int32_t reserved;                  /* 0 */
    uint64_t path_begin;               /* 0: run every path.  > 0: continue the plan's
                                          previous run (see below) */
} sdd_mc_params;

/* Continuing a run (mc->path_begin > 0).  The estimator is a sum over paths,
 * so it is additive (§2.2; §6 notes the additivity of the expectation): a
 * short run made first, e.g. a pilot that measures the standard error to
 * choose N, need not be thrown away.  With path_begin = P the call takes
 * paths [0, P) of every node from the work items of the plan's previous
 * whole single-plan run (sdd_interface_mc, _sums or sdd_mesh_generate on this
 * plan, whose items stay in the plan's buffer) and runs only paths [P, N).
 * That run must have had paths_per_node = P and the same seed, dt,
 * precision, chunk, effective step cap, tie delta, exit test and stepper; P
 * must be a multiple of chunk, which must be given (not 0), and P <= N.  The
 * result (means, errors, sums, statistics) is bitwise that of one run of N
 * paths with the same chunk.  Batches accept it per plan (sdd_batch_create
 * checks it; the plan's previous run must stay its last single-plan run
 * until the batch has run).  Split runs (sdd_interface_mc_advance) and the
 * allocation-free entry point take path_begin = 0 only.  Errors:
 * INVALID_ARG when any condition above fails. */

typedef struct {
    uint64_t paths;                    /* paths run, all nodes */
    uint64_t path_steps;               /* Euler-Maruyama updates, counted exactly */
    uint64_t ties;                     /* paths flagged as exit-decision ties */
    uint64_t non_exits;                /* paths stopped by the step cap */
    double max_stderr;                 /* largest per-node standard error */
} sdd_mc_stats;

/* Per-node sums, d = F - X0 (score minus start point), all paths and the
 * paths not flagged as ties ("nt"). */
typedef struct {
    double sum[2];
    double sumsq[2];
    double sum_nt[2];
    double sumsq_nt[2];
    uint64_t paths;
    uint64_t ties;
    uint64_t non_exits;
    uint64_t steps;
} sdd_node_sums;

typedef struct {
    int32_t solver;                    /* SDD_SOLVER_* */
    int32_t max_iter;                  /* sweeps (SOR) or inner iterations (CG); 0 = default */
    double tol;                        /* relative residual ||b - A u||_2 / ||b||_2 per subdomain */
    double omega;                      /* SOR relaxation; 0 = per-subdomain estimate */
    int32_t block_threads;             /* threads per subdomain CTA: 256, 512, 1024; 0 = 1024
                                          (in a batch: the largest requested) */
    int32_t reserved;
} sdd_solve_params;

typedef struct {
    int32_t converged;                 /* subdomains that met tol */
    int32_t subdomains;
    int32_t max_iterations;            /* largest iteration count over subdomains */
    int32_t reserved;
    double max_rel_residual;           /* largest final relative residual */
    double node_iterations;            /* sum over subdomains of interior nodes x
                                          iterations (the solves' work) */
} sdd_solve_stats;

/* Builds a plan for an n x n grid split sx x sy (2 <= ... see below) with
 * density `dens` and boundary map `bmap`: enumerates the interface nodes,
 * builds the boundary tables and copies them to the current device.
 * Requires 3 <= n <= 16385, 1 <= sx, sy <= n-1.  *out receives the plan.
 * sx = sy = n-1 gives the fully probabilistic mesh (§3.3): every interior
 * grid line is an interface, so every interior node is a Monte Carlo node
 * ((n-2)^2 of them) and every subdomain is one empty cell.
 * Errors: INVALID_ARG (sizes, unknown family/mode, nb > SDD_MAX_BUMPS, NULL),
 * OOM, CUDA, NO_DEVICE.  Paper: §2.1, Fig. 1 (interfaces); §3.2 (boundary map). */
int sdd_mesh_plan(int n, int sx, int sy, const sdd_density* dens, const sdd_bmap* bmap,
                  sdd_plan** out);

/* Number of unique interface nodes of the plan. */
int sdd_plan_num_nodes(const sdd_plan* plan, int64_t* n_nodes);

/* Copies the interface nodes' (i, j) indices, host int32 [n_nodes][2]. */
int sdd_plan_nodes(const sdd_plan* plan, int32_t* ij);

/* Copies the plan's boundary tables, host double [2][4][n]. */
int sdd_plan_edges(const sdd_plan* plan, double* edges);

/* Monte Carlo estimate at every interface node (§2.2): N paths per node,
 * Euler-Maruyama steps, exit test at the end of each step, score by linear
 * interpolation of the boundary tables at the segment/side intersection,
 * sample mean and standard error.  Path p of node m draws its normals from
 * Philox4x32-10(key = seed, counter = (step/2, p, m, 0)), Box-Muller.
 * mean, stderr_: [n_nodes][2] (either may be NULL); stats: host or NULL.
 * Errors: INVALID_ARG (N < 2, N >= 2^32, dt <= 0, bad precision), OOM, CUDA. */
int sdd_interface_mc(sdd_plan* plan, const sdd_mc_params* mc, double* mean, double* stderr_,
                     sdd_mc_stats* stats, void* stream);

/* Same paths as sdd_interface_mc; returns the per-node sums instead
 * (host or device array of n_nodes sdd_node_sums). */
int sdd_interface_mc_sums(sdd_plan* plan, const sdd_mc_params* mc, sdd_node_sums* sums,
                          void* stream);

/* ---- one Monte Carlo run split over calls, and checkpoints of it ----
 * The estimator's sums are additive over the work items (a chunk of paths of
 * one node, §2.2; §6 notes the additivity of the expectation), so a run can
 * stop between items and go on later, on another plan built from the same
 * request, from a host copy of the items done.  The result is bitwise the
 * same as one sdd_interface_mc call with the same parameters (no counterpart
 * in the paper beyond that remark: preemption and recovery for serving).
 *
 * sdd_interface_mc_advance runs the next up to max_items work items of the
 * plan's run for `mc` (a call with other parameters, or after a whole
 * sdd_interface_mc call, starts a new run); *items_done and *items_total
 * (may be NULL) receive the progress.  Stream-ordered, asynchronous. */
int sdd_interface_mc_advance(sdd_plan* plan, const sdd_mc_params* mc, uint64_t max_items,
                             uint64_t* items_done, uint64_t* items_total, void* stream);

/* Reduces a finished split run (every item done) into the node means and
 * standard errors, like sdd_interface_mc.  Errors: INVALID_ARG when no run
 * with these parameters is in progress or items are left. */
int sdd_interface_mc_finish(sdd_plan* plan, const sdd_mc_params* mc, double* mean,
                            double* stderr_, sdd_mc_stats* stats, void* stream);

/* Size of a checkpoint of the plan's split run: a header (parameters,
 * progress, a hash of the plan's grid, density, boundary tables and Monte
 * Carlo nodes) and the sums of the items done. */
int sdd_mc_checkpoint_bytes(const sdd_plan* plan, uint64_t* bytes);

/* Writes the checkpoint into host memory `host` of `bytes` bytes (synchronises
 * `stream`).  Errors: INVALID_ARG (no run in progress, buffer too small). */
int sdd_mc_checkpoint_save(sdd_plan* plan, void* host, uint64_t bytes, void* stream);

/* Restores a checkpoint into a plan built from the same request, which then
 * continues with sdd_interface_mc_advance (same parameters) and finishes with
 * sdd_interface_mc_finish.  Errors: INVALID_ARG (not a checkpoint, another
 * plan, truncated). */
int sdd_mc_checkpoint_load(sdd_plan* plan, const void* host, uint64_t bytes, void* stream);

/* Statistics of the plan's last sdd_interface_mc / _sums / sdd_mesh_generate
 * call.  Waits for that call only (an event recorded after it), not for later
 * work on its stream.  After a batch run use sdd_batch_plan_stats. */
int sdd_plan_last_mc_stats(sdd_plan* plan, sdd_mc_stats* stats);

/* Subdomain solves (§2.1, §3.5): the interface values `iface` ([n_nodes][2],
 * host or device) and the boundary map are Dirichlet data; each subdomain's
 * conservative five-point system sum_nbr c_edge (u_nbr - u_ij) = 0, c at edge
 * midpoints (§3.2), is solved independently.  Writes the whole mesh
 * [n][n][2] (boundary, interfaces and interiors) to `mesh`.  stats: host or
 * NULL; when given, returns SDD_ERR_NOT_CONVERGED if a subdomain missed tol
 * (the mesh is still written).  Errors: INVALID_ARG, OOM, CUDA. */
int sdd_subdomain_solve(sdd_plan* plan, const double* iface, const sdd_solve_params* sp,
                        double* mesh, sdd_solve_stats* stats, void* stream);

/* The whole stochastic-deterministic decomposition (§2.1, Fig. 1): interface
 * Monte Carlo followed by the subdomain solves, once, with no iteration
 * between subdomains, all on `stream` with the interface values kept on the
 * device.  Outputs (each may be NULL except mesh): mesh [n][n][2],
 * iface_mean / iface_stderr [n_nodes][2].  Errors: those of
 * sdd_interface_mc and sdd_subdomain_solve. */
int sdd_mesh_generate(sdd_plan* plan, const sdd_mc_params* mc, const sdd_solve_params* sp,
                      double* mesh, double* iface_mean, double* iface_stderr,
                      sdd_mc_stats* mc_stats, sdd_solve_stats* solve_stats, void* stream);

/* Chooses the plan's Monte Carlo nodes (SDD_PLACE_*; k: points per line for
 * EQUISPACED).  The Monte Carlo then runs on those nodes only, each with its
 * Philox counter word of the full interface list (so its estimate equals the
 * full run's), and the other interface nodes are interpolated (their std-err
 * too).  Outputs keep the full [n_nodes] layout; node sums of interpolated
 * nodes are zero.  Paper: §3.6.  Errors: INVALID_ARG, OOM, CUDA. */
int sdd_plan_set_placement(sdd_plan* plan, int mode, int k);

/* The placement: mask [n_nodes] (1 = Monte Carlo node, host) and the count
 * of Monte Carlo nodes (either may be NULL). */
int sdd_plan_placement(const sdd_plan* plan, uint8_t* mask, int64_t* n_mc);

/* Mesh quality (§3.1 eq. Qmeasure, §3.3): per cell K of the computational
 * grid, Q(K) = 1/2 tr(J^T J) / sqrt(det(J^T J)) with J the Jacobian of
 * (s,t) -> u from the cell's edge differences (>= 1; a cell with det J <= 0
 * is folded and left out of max and mean).  With a reference mesh (e.g. the
 * single-domain mesh) also R_max = Q_max(ref)/Q_max, R_mean =
 * Q_mean(ref)/Q_mean and l_inf = max over nodes |w(u) - w(ref)|. */
typedef struct {
    double q_max, q_mean;
    int64_t folds;
    double ref_q_max, ref_q_mean;
    int64_t ref_folds;
    double r_max, r_mean, l_inf;
} sdd_quality;

/* mesh, ref: [n][n][2], host or device (ref may be NULL); out: host.
 * Synchronises `stream`. */
int sdd_mesh_quality(sdd_plan* plan, const double* mesh, const double* ref, sdd_quality* out,
                     void* stream);

/* Anisotropic (Perona-Malik) smoothing of a mesh (§3.4, eq.
 * PeronaMalikDiffusion): `steps` forward-Euler, centred-in-space (FTCS) steps
 * of length dt of u_t = div(g grad u) for each component, g =
 * exp(-|grad u|^2 / k^2).  Each of a node's four edges conducts with g of its
 * own difference over h = 1/(n-1) (Perona and Malik's discrete scheme):
 *   u <- u + dt/h^2 sum_{E,W,N,S} g(|u_nb - u| / h) (u_nb - u);
 * boundary values stay fixed.  mesh: [n][n][2] of the plan's grid, host or
 * device memory, smoothed in place (host: the call synchronises `stream`;
 * device: stream-ordered).  One kernel launch per step.  Errors: INVALID_ARG
 * (NULL, steps < 0, dt or k not positive and finite, dt/h^2 > 1/4, where the
 * FTCS step loses its maximum principle), OOM, CUDA. */
int sdd_mesh_smooth(sdd_plan* plan, double* mesh, int steps, double dt, double k, void* stream);

/* The same smoothing applied on each subdomain separately (§3.5, §4: local
 * smoothing, parallel over the subdomains): every node of an interface line
 * of the plan's split is held fixed like the boundary, so each subdomain is
 * smoothed with its ring as Dirichlet data.  shifted = 1 smooths over the
 * subdomains shifted by half a subdomain instead (the paper's second cycle,
 * which puts the original interfaces inside subdomains): the held lines are
 * the midlines floor((a + b) / 2) of the plan's blocks [a, b] between
 * consecutive lines of 0, the interface lines and n - 1, per axis.  Same
 * arguments, memory and stream rules and errors as sdd_mesh_smooth, plus
 * INVALID_ARG for shifted outside {0, 1}. */
int sdd_mesh_smooth_subdomains(sdd_plan* plan, double* mesh, int steps, double dt, double k,
                               int shifted, void* stream);

/* Copies the plan's last results: mesh [n][n][2] (after a solve), interface
 * means and standard errors [n_nodes][2] (after a Monte Carlo call or a batch
 * run).  Each pointer may be NULL, host or device memory. */
int sdd_plan_results(sdd_plan* plan, double* mesh, double* mean, double* stderr_, void* stream);

/* ---- batches: many meshes of uneven size generated together ----
 * The interface nodes of every plan of a batch run in one persistent path
 * kernel per (precision, density family) group, followed by one per-node
 * reduction per group, one Dirichlet-fill launch and one launch solving every
 * subdomain of every mesh (§2.1: the subdomains are independent, so meshes
 * batch the same way subdomains do).  Each plan keeps its own Philox key and
 * work-item size, so its results are bitwise the same as when it runs alone.
 * Results land in each plan's buffers (sdd_plan_results). */
typedef struct sdd_batch sdd_batch;

/* Builds a batch over n_plans distinct plans, with one sdd_mc_params and one
 * sdd_solve_params per plan (host arrays).  All device records are built and
 * copied here; the call synchronises the device.  Errors: INVALID_ARG, OOM,
 * CUDA. */
int sdd_batch_create(sdd_plan* const* plans, int n_plans, const sdd_mc_params* mc,
                     const sdd_solve_params* sp, sdd_batch** out);

/* Enqueues one run of the batch on `stream` (asynchronous).  use_graph != 0:
 * the first call captures the run into a CUDA graph, later calls replay it
 * (needs a non-default stream). */
int sdd_batch_run(sdd_batch* batch, int use_graph, void* stream);

/* Enqueues one phase of a run, without a graph: phases = 1 Monte Carlo only,
 * 2 fill + subdomain solves only (from the interface values already in the
 * plans), 3 both.  For timing the phases separately. */
int sdd_batch_run_phases(sdd_batch* batch, int phases, void* stream);

/* Statistics of plan `index` in the batch's last run (synchronises). */
int sdd_batch_plan_stats(sdd_batch* batch, int index, sdd_mc_stats* mc, sdd_solve_stats* solve);

/* Frees the batch (not its plans). */
void sdd_batch_destroy(sdd_batch* batch);

/* Allocation-free interface Monte Carlo, for callers that cannot allocate
 * device memory: code running under an allocator owned by someone else (a
 * framework's caching allocator, an embedded runtime with a fixed budget) or
 * at points where an allocation would synchronise or could fail.  The paper
 * has no counterpart: this is a deployment variant of sdd_interface_mc.
 * It needs no plan.  It runs the same path kernel and reduction as
 * sdd_interface_mc, and its only scratch (work counter, counters, per-work-item
 * sums) is one file-scope 8 MiB device array inside the library, which every
 * GPU that loads the library keeps until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating routine.
 * Inputs, all device memory of the current device owned by the caller: nodes
 * int32 [n_nodes][2] (i, j), in the order whose index is the node's Philox
 * counter word (the plans' order reproduces sdd_interface_mc); edges, the
 * boundary tables [2][4][n].  Host inputs: dens, mc (as sdd_interface_mc).
 * Outputs, device memory: mean [n_nodes][2] (required), stderr_
 * [n_nodes][2] (may be NULL).  Asynchronous on `stream`.
 * Before any launch each buffer is checked: device (or managed) memory of
 * the current device, 8-byte aligned, and an allocation that holds the
 * bytes above from the pointer on (cuMemGetAddressRange); INVALID_ARG with a
 * message otherwise.  Nodes must be interior, 0 < i, j < n-1: the kernel
 * does not check them, and the estimate of a node outside that range is
 * undefined (but reads and writes stay inside the buffers).
 * Limit: n_nodes * ceil(N / chunk) work items must fit the array (55185);
 * chunk = 0 picks the automatic size, raised up to 8192 until they fit;
 * larger requests fail with SDD_ERR_INVALID_ARG and a message.  The TABLE
 * density family is not accepted here (its table reaches the device through
 * a plan); INVALID_ARG.  mc->path_begin must be 0.
 * The first call on a device (and the first after that device's context was
 * replaced, e.g. by cudaDeviceReset) looks the array's address up
 * (cudaGetSymbolAddress) and should come before any stream capture.  All calls
 * share the array, which keeps the last call's contents (the parts that must
 * start at zero are cleared by each call): calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller. */
int sdd_interface_mc_static(int n, const int32_t* nodes, int64_t n_nodes, const double* edges,
                            const sdd_density* dens, const sdd_mc_params* mc, double* mean,
                            double* stderr_, void* stream);

/* Statistics (paths, path-steps, ties, capped paths, largest std-err) of the
 * last sdd_interface_mc_static call on the current device, read from the head
 * of its static array: synchronises `stream`, which must be the stream of
 * that call or one ordered after it.  Errors: INVALID_ARG (no call yet),
 * CUDA. */
int sdd_interface_mc_static_stats(sdd_mc_stats* stats, void* stream);

/* Frees the plan and its device buffers.  Memory is stream-ordered: the free
 * is queued on the plan's last stream after its work, and the call does not
 * synchronise.  A plan must outlive the batches that use it. */
void sdd_plan_destroy(sdd_plan* plan);

/* Message of the last failed call on this thread ("" if none). */
const char* sdd_last_error(void);

/* Number of kernels this library has launched in the process so far. */
int sdd_kernel_launches(uint64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* SDD_H */
