/*
 * hjbp.h -- C ABI of the GB300 patchy semi-Lagrangian solver for the
 * minimum-time Hamilton-Jacobi-Bellman equation
 *
 *     max_a { -f(x,a) . grad u(x) - 1 } = 0  on R^d \ Omega_0,   u = 0 on Omega_0
 *
 * (Cacace, Cristiani, Falcone, Picarelli, "A patchy dynamic programming scheme
 * for a class of HJB equations", Sec. 1, Eq. (HJB)), solved on a box Omega with
 * state constraints on its boundary.
 *
 * Conventions used by every entry point:
 *  - Every call returns an hjbp_status; nothing is thrown across the ABI.  On
 *    failure hjbp_last_error() returns a thread-local message.
 *  - Host arrays passed in are owned by the caller and copied before the call
 *    returns (create) or read during the call (set_initial).
 *  - Device memory belongs to the plan.  It comes from the allocator given at
 *    create (for example the PyTorch caching allocator) or, if none is given,
 *    from cudaMallocAsync on the plan's stream.  It is released by destroy.
 *  - Grids are node-centred: n[d] nodes per axis (n[d]-1 cells), equal
 *    spacing k on every axis, node index i = i1 + n1*(i2 + n2*i3) (x1 fastest).
 *  - All work of a plan runs on the CUDA stream given at create; calls that
 *    return data to the host synchronise that stream.
 */
#ifndef HJBP_H
#define HJBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HJBP_OK = 0,
    HJBP_EINVAL = 1,    /* invalid descriptor or argument */
    HJBP_ENOMEM = 2,    /* device or host allocation failed */
    HJBP_ENOCONV = 3,   /* sweep cap reached before the sup-norm test passed; results stay readable */
    HJBP_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    HJBP_ECUDA = 5,     /* a CUDA runtime call failed */
    HJBP_EBUSY = 6,     /* not admissible now (server), or the plan is still running */
    HJBP_ESTATE = 7     /* call not valid in the plan's current state */
} hjbp_status;

/* Speed fields c(x) of the dynamics f(x, a) = c(x) a, |a| = 1 (a fixed menu).
 *  HJBP_C_ONE        c = 1                                   (eikonal)
 *  HJBP_C_SINCOS2D   c = 1 + p0 sin(2 pi x1) cos(2 pi x2)
 *  HJBP_C_SIN3D      c = 1 + p0 sin(pi x1) sin(pi x2) sin(pi x3)
 *  HJBP_C_FOURIER2D  c = 1 + 0.5 g(x),  g = sum_{p,q=0..3} a_pq cos(pi p x1/2 + th_pq)
 *                                       cos(pi q x2/2 + ps_pq) / sum |a_pq|,
 *                    params = [a (16, row-major in p,q), th (16), ps (16)]
 *  HJBP_C_FAN        c = |p0 + p1 x1 + p2 x2 + p3 x3|   (Fan, Table 1: p = 0.1, 1, 1, 0);
 *                    a node where c <= 1e-12 cannot move and is treated like the
 *                    ghost ring (+inf, label -1) unless it is a target node        */
typedef enum {
    HJBP_C_ONE = 0,
    HJBP_C_SINCOS2D = 1,
    HJBP_C_SIN3D = 2,
    HJBP_C_FOURIER2D = 3,
    HJBP_C_FAN = 4
} hjbp_speed_kind;

/* Dynamics (Table 1).  HJBP_DYN_SPEED: f(x, a) = c(x) a with the speed field
 * above.  HJBP_DYN_DRIFT: f(x, a) = s a + w (Zermelo: s = 2.1, w = (2, 0)),
 * drift = {s, w_1, w_2, w_3}, speed must be HJBP_C_ONE, 2D only; every control
 * needs |s a + w| > 1e-15.  With |h f| = k (Sec. 2.1) the foot of control a is
 * x_i + k f/|f| and its time step k/|f|.                                    */
/* HJBP_DYN_BROCKETT (Sec. 7, 3D only, speed HJBP_C_ONE): Brockett's integrator
 * f(x, a) = (a_1, a_2, x_1 a_2 - x_2 a_1); control rows are (a_1, a_2, unused),
 * any finite values (the paper's set is {-5, 0, 5}^2); a = 0 cannot move and
 * is never evaluated.  The foot x_i + k f/|f| and the step k/|f| depend on the
 * node; the coarse boundary values of Step 1 divide the distance to the
 * target by the largest |f(x, a)| over the controls.                        */
typedef enum { HJBP_DYN_SPEED = 0, HJBP_DYN_DRIFT = 1, HJBP_DYN_BROCKETT = 2 } hjbp_dyn_kind;

/* Target Omega_0 and its parts Omega_0^j (one patch each, Sec. 3).
 * HJBP_TARGET_BALLS: every row of targets is a ball (centre, radius) and a part.
 * HJBP_TARGET_SECTORS: row 0 is one ball split into n_parts equal angular
 *   sectors, part j = floor(n_parts theta / (2 pi) + 1e-9) mod n_parts with
 *   theta the angle of (x_1 - c_1, x_2 - c_2) in [0, 2 pi) (in 3D: wedges
 *   around the x_3 axis through the centre).
 * HJBP_TARGET_SLAB (2D and 3D): row 0 = (v, unused.., r): the slab |x_1 - v| <= r
 *   (a line or plane target of half-width r) split into n_parts equal pieces
 *   along x_2 over the box, part j = floor(n_parts (x_2 - lo_2) / (hi_2 - lo_2)
 *   + 1e-9), clamped.
 * HJBP_TARGET_ORTHANTS: row 0 is one ball split into its 2^dim orthants
 *   (n_parts must be 2^dim): part j has bit d set iff x_{d+1} >= c_{d+1}.    */
typedef enum {
    HJBP_TARGET_BALLS = 0,
    HJBP_TARGET_SECTORS = 1,
    HJBP_TARGET_SLAB = 2,
    HJBP_TARGET_ORTHANTS = 3
} hjbp_target_kind;

/* Arithmetic of the fine-grid sweeps.  HJBP_FP64: every sweep in FP64.
 * HJBP_FP32_POLISH64: bulk sweeps in FP32, then FP64 polishing sweeps.      */
typedef enum { HJBP_FP64 = 0, HJBP_FP32_POLISH64 = 1 } hjbp_precision;

/* Problem descriptor (Sec. 2.1 and Sec. 3 of the paper):
 *   dim            2 or 3
 *   n[3]           nodes per side of the fine grid G (n[2] ignored in 2D)
 *   n_coarse[3]    nodes per side of the coarse grid G~; n_coarse[0] == 0 asks
 *                  for the plain global solve (no patches)
 *   lo[3], hi[3]   the box Omega; (hi-lo)/(n-1) must be equal on all axes
 *   speed, speed_params[64]   c(x), see hjbp_speed_kind
 *   n_controls, controls      discrete control set A: n_controls x dim unit
 *                  vectors (row-major), 1 <= n_controls <= HJBP_MAX_CONTROLS
 *                  (patchy solves: <= 255, the feedback a* being one byte)
 *                  (Brockett's integrator: rows (a_1, a_2, unused))
 *   n_targets, targets        Omega_0 = union of balls: n_targets x (dim+1)
 *                  rows (centre, radius); ball j is target part Omega_0^j and
 *                  seeds patch j (1 <= n_targets <= HJBP_MAX_TARGETS)
 *   tol            sup-norm stopping tolerance of the fine-grid iteration
 *                  (Sec. 2.2, Step 4)
 *   tol_coarse     same on the coarse grid (Step 1); <= 0 selects 1e-12
 *   tol_phi        same for the colour transport (Step 3.1); <= 0 selects 1e-10
 *   precision      hjbp_precision
 *   max_sweeps     cap on tile sweeps per phase (<= 0 selects 1e6)            */
#define HJBP_MAX_CONTROLS 256
#define HJBP_MAX_TARGETS 64
#define HJBP_MAX_OBSTACLES 16
typedef struct {
    int dim;
    int n[3];
    int n_coarse[3];
    double lo[3];
    double hi[3];
    int speed;
    double speed_params[64];
    int n_controls;
    const double *controls;
    int n_targets;
    const double *targets;
    double tol;
    double tol_coarse;
    double tol_phi;
    int precision;
    int max_sweeps;
    int flags;          /* HJBP_FLAG_* bits */
    int tune[8];        /* launch shape, 0 = default: [0] Gauss-Seidel rounds per tile
                           launch of the value sweep (2D: 4 where the halos are exchanged
                           (see [7]), else 2; 3D: 1),
                           [1] of the colour transport (2D: 4 where the halos are
                           exchanged, else 2; 3D: 2),
                           [2] passes per launch of the 3D reachability sweep (1; the 2D
                           one runs bit-set rounds to the tile's fixed point), [3] warps
                           per 32x32 tile of the 2D value sweep (1; 1, 2 or 4), [4] resident
                           warps per SM of the tile-queue sweep (occupancy limit), [5] the
                           fine-grid launches run the increasing or (alternately) the
                           decreasing pass of every axis: 3D default (0; 2 runs all six
                           passes), 2D only with 1 (measured slower there), [6] kernel
                           variants: 0 default, 1 the per-control FP64 polish (2D) instead
                           of the pair-form one, 2 the scalar FP32 update instead of the
                           packed FP32x2 one (2D and 3D; same results), [7] the FP32
                           monotone sweeps (value sweeps in 2D and 3D, the 2D colour-
                           transport bulk of up to four colours) publish their tile boundary
                           and re-read their
                           halo inside a launch: 0 after every pass (default), 2 after
                           every round (2D value sweep), 1 never (block-Jacobi launches,
                           results the same to the last bit from run to run; with the
                           exchange the iterates depend on timing, the fixed point does
                           not) */
    double reduce_r;    /* add-on AO3 (Sec. 6), patchy solves only: r > 1 restricts the
                           minimum of Step 3.2 at node i to the controls a with
                           a . a*_{k~}(x_i) >= cos(pi / r) - 1e-12 (a*_{k~}: the coarse
                           feedback of Step 2, Eq. feedbackcontrol); nodes without a
                           feedback keep every control.  0 keeps every control.  On the
                           2D path the control set must have at most 64 members; not
                           with HJBP_DYN_BROCKETT.                                     */
    int dyn;            /* hjbp_dyn_kind */
    double drift[4];    /* HJBP_DYN_DRIFT: s, w_1, w_2, w_3 */
    int target_kind;    /* hjbp_target_kind */
    int n_parts;        /* parts (patches) of HJBP_TARGET_SECTORS / SLAB, 1..64 */
    int n_obstacles;    /* obstacles (Sec. 4, "Patchy method with obstacles"), 0..HJBP_MAX_OBSTACLES */
    const double *obstacles;  /* n_obstacles x 7 rows, caller-owned, copied at create:
                           (0, c_1, c_2, c_3, r, -, -) the closed ball |x - c|^2 <= r^2, or
                           (1, l_1, l_2, l_3, u_1, u_2, u_3) the closed box l <= x <= u (the
                           third coordinate ignored in 2D).  A node inside an obstacle is a
                           state constraint like the ghost ring (+inf, label -1) unless it
                           is a target node; the coarse grid of Step 1 follows the same
                           rule.  NULL when n_obstacles is 0.                           */
} hjbp_problem_desc;

/* flags: HJBP_FLAG_TIME_SWEEPS records a CUDA event pair around every launch
 * of the fine-grid value-sweep kernel (on the plan's stream) and reports their
 * summed duration in hjbp_stats.ms_sweep_kernel.                              */
#define HJBP_FLAG_TIME_SWEEPS 1
/* HJBP_FLAG_DIRICHLET (patchy solves only): while patch j is solved in Step
 * 3.2, every node outside patch j and outside Omega_0^j holds the value
 * U_P^(0) of Step 2 (Eq. dbc, Sec. 5-6: 0 on every target part, +inf on the
 * ghost ring and where Step 2 finds no finite value) instead of +inf (the
 * state constraints of Sec. 3).  Patch nodes that can reach neither their
 * target part nor a finite boundary value stay +inf.
 * HJBP_FLAG_WARM_START (patchy solves only): add-on AO1 of Sec. 6, Step 3.2
 * starts from U_P^(0) where it is finite (the bound 1e6 elsewhere) and runs
 * the plain update u <- F(u); the fixed point is the same (it is unique on the
 * reachable set), only the iteration count changes.                         */
#define HJBP_FLAG_DIRICHLET 2
#define HJBP_FLAG_WARM_START 4
/* HJBP_FLAG_CAUSAL_SWEEPS (patchy solves only): add-on AO2 of Sec. 6 in the
 * form the tiled GPU iteration can use.  The paper orders the nodes of a
 * patch so that the update follows the characteristics; here each tile (32x32
 * in 2D, 8x8x8 in 3D) runs only the Gauss-Seidel directions along which the
 * coarse feedback
 * a*_{k~} of Step 2 carries information (a node depends on its foot
 * x_i + k a*, so the sweep moves against a*), in Step 3.1 and Step 3.2.  The
 * fixed point is the same; the solve stays deterministic.                    */
#define HJBP_FLAG_CAUSAL_SWEEPS 8
/* HJBP_FLAG_TILE_QUEUE (2D): the value iteration of Step 3.2 (or of the
 * global solve) runs as one persistent launch in which resident warps take
 * 32x32 tiles from a device work queue; a tile whose boundary changed queues
 * the neighbours that read it.  Values are updated in place, so the order of
 * the updates, and the last bits of the result, depend on timing (the fixed
 * point and the tolerance do not).  Ignored with HJBP_FLAG_WARM_START or
 * reduce_r (their updates are not monotone or not tiled the same way).      */
#define HJBP_FLAG_TILE_QUEUE 16

/* Device allocator hooks (optional).  alloc returns device memory of at least
 * `bytes` usable on `stream`, or NULL; release returns it.  ctx is passed back
 * unchanged.                                                                  */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*release)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} hjbp_allocator;

typedef struct hjbp_plan hjbp_plan;

/* Per-solve statistics.  Sweep counts are tile-sweep launches (each launch
 * runs every active tile through its in-tile Gauss-Seidel passes).           */
typedef struct {
    int n_patches;
    int sweeps_coarse;
    int sweeps_phi;
    int sweeps_reach;
    int sweeps_fine;
    int sweeps_polish;
    int sweeps_patch[HJBP_MAX_TARGETS];   /* launches in which patch j had an active tile */
    int64_t patch_nodes[HJBP_MAX_TARGETS];
    int64_t patch_tiles[HJBP_MAX_TARGETS];
    double residual_fine;                 /* last sup-norm change of the FP32/FP64 bulk */
    double residual_polish;               /* last FP64 polishing change */
    int64_t unreachable;                  /* free nodes with value +inf */
    int64_t uncovered_filled;             /* Remark 3.1 neighbour fills */
    int64_t node_updates;                 /* node updates executed on the fine grid */
    int64_t node_control_updates;         /* node_updates x controls */
    double ms_setup, ms_coarse, ms_feedback, ms_labels, ms_compact, ms_fine, ms_polish, ms_total;
    int64_t kernel_launches;              /* CUDA kernels launched by the solve */
    int64_t sweep_kernel_launches;        /* launches of the fine-grid value-sweep kernel */
    int64_t sweep_tile_visits;            /* active tiles summed over those launches */
    double ms_sweep_kernel;               /* their summed duration (HJBP_FLAG_TIME_SWEEPS), else 0 */
    int phi_refinements;                  /* FP64 residual evaluations of the colour transport */
    double ms_reach;                      /* S* computation on the fine grid (inside ms_fine) */
    double residual_patch[HJBP_MAX_TARGETS];  /* per patch: the largest FP64 sup-norm change of its
                                             tiles in the last launch each ran in (<= tol once the
                                             patch retired; patchy solves, 0 otherwise)   */
    int64_t phi_kernel_launches;          /* launches of the 2D colour-transport kernel that had work */
    int64_t phi_node_colour_updates;      /* node x colour updates they executed (2D) */
    double ms_phi_kernel;                 /* their summed duration (HJBP_FLAG_TIME_SWEEPS), else 0 */
} hjbp_stats;

/* Validate the descriptor, copy its arrays, allocate device memory.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * allocator: optional, see hjbp_allocator.  Errors: EINVAL, ENOMEM, ECUDA.  */
hjbp_status hjbp_create(const hjbp_problem_desc *desc, void *cuda_stream, const hjbp_allocator *allocator,
                        hjbp_plan **out);

/* Run the whole solve (global SL of Eq. (iterativeSLscheme), or the patchy
 * algorithm of Sec. 3, Steps 1-4) on the plan's stream.  Returns after the
 * work is complete.  Errors: ENOCONV (results readable), ECUDA, ETIMEOUT.   */
hjbp_status hjbp_solve(hjbp_plan *plan);

/* Copy the N = prod n[d] fine-grid values (FP64, +INFINITY where the target
 * cannot be reached) into host_out.                                          */
hjbp_status hjbp_get_values(hjbp_plan *plan, double *host_out);

/* Copy the N labels.  Patchy solve: j on patch j (Step 3.1; a node of patch j
 * that cannot reach its target inside the patch keeps label j and has value
 * +INFINITY) and on target part j, -1 on the ghost ring and where U_P^(0) is
 * unreachable.  Global solve: 0 on nodes that reach the target, the part index
 * on target nodes, -1 elsewhere.                                              */
hjbp_status hjbp_get_labels(hjbp_plan *plan, int8_t *host_out);

/* Intermediate arrays of the patchy algorithm (for verification):
 *  HJBP_OUT_UCOARSE  coarse values U~_P (FP64, N~)          Step 1
 *  HJBP_OUT_U0       U_P^(0) on G (FP64, N)                 Step 2
 *  HJBP_OUT_ASTAR    coarse feedback index a*_k~ (int32, N; -1 undefined)  Step 2
 *  HJBP_OUT_PHI      colour fields phi^j (FP64, R x N)      Step 3.1
 *  HJBP_OUT_U32      FP32 bulk values before polishing (float, N)
 * Errors: EINVAL (unknown id or not produced by this plan), ESTATE.          */
enum { HJBP_OUT_UCOARSE = 0, HJBP_OUT_U0 = 1, HJBP_OUT_ASTAR = 2, HJBP_OUT_PHI = 3, HJBP_OUT_U32 = 4 };
hjbp_status hjbp_get_intermediate(hjbp_plan *plan, int which, void *host_out, size_t bytes);

/* Waits for the plan's stream and returns the status of its last hjbp_solve
 * (HJBP_ESTATE if it was never solved).  hjbp_solve itself returns once its
 * stream work is done; hjbp_sync serves callers that hold only the plan.    */
hjbp_status hjbp_sync(hjbp_plan *plan);

/* Start values for the value iteration of the following solves (Step 3.2, or
 * the global solve): N doubles in node order (index i = i1 + n1 i2), each
 * >= 0 or +INFINITY.  On S* the iteration starts from them where they are
 * finite (from the bound 1e6 elsewhere) and runs the plain update
 * u <- F(u); the fixed point on S* is unique (Sec. 2.2 with R14), so the
 * result is the same as from the default start, only the work changes: a
 * resume from an earlier solution, or add-on AO1 of Sec. 6 with the caller's
 * own guess.  Copied into the plan; NULL clears them.  2D plans only
 * (HJBP_EINVAL otherwise).                                                 */
hjbp_status hjbp_set_initial(hjbp_plan *plan, const double *u_init);

/* Borrowed device pointers (valid until destroy): FP64 values and int8 labels. */
hjbp_status hjbp_get_device_views(hjbp_plan *plan, const double **u, const int8_t **labels);

hjbp_status hjbp_get_stats(hjbp_plan *plan, hjbp_stats *out);

/* Patch compaction of the last patchy solve (Sec. 3: the patches are
 * assembled from the labels of Step 3.1 before Step 3.2 solves each one), as
 * per-patch lists in CSR form.  The fine grid is cut into tiles of 32x32
 * interior nodes in 2D (8x8x8 in 3D) starting at node (1,1[,1]);
 * ntx = ceil((n[0]-2)/side), nty likewise, and tile t = tx + ntx (ty + nty tz).
 *   tile_offsets  R+1 int64: patch j owns entries tile_offsets[j] ..
 *                 tile_offsets[j+1]-1 of tile_ids and tile_nodes
 *   tile_ids      int32 per entry: a tile holding a free node of patch j, in
 *                 increasing order
 *   tile_nodes    int32 per entry: the free nodes of patch j in that tile
 *   node_offsets  R+1 int64: patch j owns node_ids[node_offsets[j] ..
 *                 node_offsets[j+1]-1]
 *   node_ids      int32 per free node of patch j: its node index, tile by tile
 *                 in the order of tile_ids, x fastest inside a tile
 * R = hjbp_stats.n_patches.  Free nodes are the nodes of label j that are
 * neither target nor ghost ring; the node lists are taken before S* pruning,
 * so node_offsets[j+1] - node_offsets[j] = hjbp_stats.patch_nodes[j].  Any
 * pointer may be NULL (call first with the offsets alone to size the others).
 * Host buffers, caller-owned.  Errors: ESTATE (no patchy solve yet), EINVAL. */
hjbp_status hjbp_get_patch_lists(hjbp_plan *plan, int64_t *tile_offsets, int32_t *tile_ids, int32_t *tile_nodes,
                                 int64_t *node_offsets, int32_t *node_ids);

/* Node count N and coarse count N~ of the plan.                              */
hjbp_status hjbp_get_sizes(hjbp_plan *plan, int64_t *n_nodes, int64_t *n_coarse_nodes);

void hjbp_destroy(hjbp_plan *plan);

const char *hjbp_last_error(void);

/* ---- batched and served solves (not in the paper: throughput patterns) ----
 *
 * hjbp_batch_solve: solve `count` plans at once.  `workers` host threads (<= 0
 * selects 8), each with its own non-blocking CUDA stream, take plans in order
 * and run their solves concurrently so that small problems overlap on the GPU.
 * Each plan's results are read as usual afterwards.  statuses (optional,
 * count entries) receives each plan's status; the return value is the worst
 * one (an error, else ENOCONV, else OK).                                     */
hjbp_status hjbp_batch_solve(hjbp_plan *const *plans, int count, int workers, hjbp_status *statuses);

/* hjbp_autotune: the launch shape (tune[0..3] of hjbp_problem_desc: Gauss-
 * Seidel rounds per launch of the value sweep and of the colour transport,
 * reach passes, warps per tile) for problems of the class of `desc`: its
 * dimension, log2 of its cells per side and of its control count, patchy or
 * not, its boundary and add-on options.  The first call for a class solves
 * `desc` (on `cuda_stream`) once per candidate shape after a warm-up solve
 * and keeps the fastest by GPU solve time; later calls for the class return
 * the kept shape (*from_cache = 1).  cache_path (optional) names a text file
 * read before the lookup and appended with each new class.  Errors: EINVAL for
 * a NULL argument, else the status of the failing solve.                    */
hjbp_status hjbp_autotune(const hjbp_problem_desc *desc, void *cuda_stream, const char *cache_path, int tune_out[4],
                          int *from_cache);

/* Serving.  A server owns a pool of `workers` threads (<= 0 selects 8) with
 * their own streams and a device-memory budget (0 selects half of the free
 * memory).  submit validates and copies a problem (EINVAL as hjbp_create),
 * estimates the device bytes its solve needs, and queues it; EBUSY if it can
 * never fit the budget.  A queued request holds no device memory.  It starts
 * as soon as a worker is idle and its bytes fit next to the requests in
 * flight (continuous batching); that worker creates the plan and solves it.
 * poll returns OK with *done = NULL while the request is queued or running;
 * once finished it hands over the plan (values and labels resident on the
 * device; the caller destroys it), returns that solve's status and the
 * latency from submit to completion in seconds.  A request whose plan could
 * not be created finishes with the create's status (ENOMEM, ECUDA) and
 * *done = NULL; hjbp_last_error then gives its message in the polling
 * thread.  destroy waits for running requests, drops queued ones and destroys
 * plans nobody collected.                                                    */
typedef struct hjbp_server hjbp_server;
hjbp_status hjbp_server_create(size_t device_budget_bytes, int workers, hjbp_server **out);
hjbp_status hjbp_server_submit(hjbp_server *server, const hjbp_problem_desc *desc, uint64_t *ticket);
hjbp_status hjbp_server_poll(hjbp_server *server, uint64_t ticket, hjbp_plan **done, double *latency_s);
hjbp_status hjbp_server_stats(hjbp_server *server, int *queued, int *running, size_t *bytes_in_use);
void hjbp_server_destroy(hjbp_server *server);

/* Plain global 2D solve in FP64 that allocates nothing.  The paper has no
 * counterpart: it serves callers that cannot allocate device memory at solve
 * time, such as real-time loops that forbid allocation after start-up (an
 * allocation may block or fail on a fragmented pool) or hosts whose memory
 * pool belongs to another component.
 *   desc        a 2D problem with n_coarse[0] == 0 (plain global solve), at
 *               most HJBP_NOALLOC_MAX_NODES nodes, f = c(x) a, ball targets,
 *               no patchy-only options (flags DIRICHLET / WARM_START /
 *               CAUSAL_SWEEPS, reduce_r); precision is ignored (FP64)
 *   cuda_stream the stream to run on (NULL = legacy default stream)
 *   u_out       device array of N doubles: the values (+INFINITY unreachable)
 *   labels_out  device array of N int8: 0 / target part / -1, as hjbp_get_labels
 * Runs the kernels hjbp_solve runs for the same descriptor with HJBP_FP64, in
 * the same order, so the results agree with hjbp_solve's.  Scratch comes from
 * one fixed device array inside the library (32 MiB, held by every GPU that
 * loads the library until the process exits); no cudaMalloc, cudaFree or
 * other allocator is called.  The first call on each device looks up that
 * array's device address and the SM count and caches them for the process
 * lifetime (one primary context per device; no cudaDeviceReset in between).
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  The call is synchronous: it reads counts back to
 * the host between launches and synchronises the stream before returning.
 * Errors: EINVAL (descriptor, too large, NULL outputs), ECUDA, ENOCONV
 * (max_sweeps reached; the outputs then hold the last iterate).              */
#define HJBP_NOALLOC_MAX_NODES (1 << 20)
hjbp_status hjbp_solve_global2d_noalloc(const hjbp_problem_desc *desc, void *cuda_stream, double *u_out,
                                        int8_t *labels_out);

/* Library version as major*10000 + minor*100 + patch.                        */
int hjbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HJBP_H */
