/*
 * hjbp_oracle.c -- plain, slow, FP64 CPU oracle for the patchy semi-Lagrangian
 * minimum-time scheme of Cacace, Cristiani, Falcone and Picarelli
 * ("A patchy dynamic programming scheme for a class of HJB equations").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header or
 * table with the CUDA library and never calls it.
 *
 * What it computes, in the paper's order and notation:
 *   - the SL operator F of Eq. (SLscheme): for interior non-target nodes
 *     [F(U)]_i = min_a { I[U](x_i + h_{i,a} f(x_i,a)) + h_{i,a} }, 0 on the
 *     target, +inf on the ghost ring dG (state constraints);
 *   - the fixed-point iteration U^{n+1} = F(U^n) of Eq. (iterativeSLscheme),
 *     started from 0 on the target and +inf elsewhere, stopped when the
 *     sup-norm change drops below tol (Sec. 2.2, Step 4), with Gauss-Seidel
 *     updates (Sec. 2.2);
 *   - the patchy algorithm of Sec. 3: Step 1 coarse solve, Step 2
 *     interpolation U_P^(0) and coarse feedback a*_{k~} (Eq. feedbackcontrol),
 *     Step 3.1 colour transport phi (Eq. HJBridotta_discreta) and projection
 *     (Eq. proiezionecolore, Remark 3.1), Step 3.2 per-patch solves with
 *     state constraints on the patch boundary, Step 4 merge.
 *
 * Readings of points the paper leaves open (each one is listed, with its
 * reason, in the design notes of the repository):
 *   R1  f(x,a) = c(x) a with |a| = 1, so |h f| = k gives h_i = k / c(x_i) and
 *       the foot x_i + h f = x_i + k a.  The foot is formed in grid-index
 *       coordinates, xi_d = i_d + a_d, so that axis controls land on nodes.
 *   R2  I is the tensor-product (bi/tri)linear interpolation on the grid cell
 *       containing the foot; cell index floor(xi) clamped to [0, n-2]; a foot
 *       outside the box is +inf.
 *   R3  I[U] is +inf iff some corner with positive weight is +inf; corners of
 *       weight exactly 0 are skipped.
 *   R4  Ghost ring = nodes with any index 0 or n-1; they stay +inf.  A node
 *       inside a target ball is a target node even on the ring.
 *   R5  Target part j = nodes with |x - c_j| <= r_j (lowest j on overlap).
 *   R6  The coarse grid cannot resolve a ball thinner than its spacing k~.
 *       Coarse nodes with |x - c_j| <= r_j + k~ sqrt(d)/2 are boundary nodes
 *       of Step 1 with the value max(0, |x - c_j| - r_j) / v(x) (the time to
 *       reach the ball moving straight at it; 0 inside it), lowest j first;
 *       v is the largest speed f allows towards the target: c(x) for
 *       f = c(x) a, and for the drift f = s a + w the largest v with
 *       |v e - w| = s, e the unit vector towards the target.
 *       With the value 0 on the whole enlarged set, U_P^(0) would vanish on
 *       a plateau around the ball where the feedback of Step 2 is all ties
 *       and its trajectories circle instead of reaching Omega_0^j.
 *   R7  U_P^(0) on fine nodes = Q1 of the coarse values, with a coarse value
 *       +inf (ghost ring, unreachable) entering as the finite bound
 *       M = 1e6, larger than any value of the solution; a fine node with
 *       U_P^(0) >= M (every corner +inf) is unreachable.  0 on fine target
 *       nodes, +inf on the fine ghost ring.  Read literally, U_P^(0) is +inf
 *       on the whole outer ring of coarse cells (every node there has a
 *       ghost corner), and renormalising over the finite corners makes it
 *       flat across that ring, where the feedback then circles.
 *   R8  Gauss-Seidel order: a single lexicographic order (order 0), the 2^d
 *       alternating orthant orders (order 1, fast-sweeping orders, Remark
 *       4.1), or plain Jacobi U^{n+1} = F(U^n) (order 2).  All reach the same
 *       fixed point.
 *   R9  |inf - inf| = 0 and |inf - finite| = inf in the sup-norm test.
 *   R10 argmin ties -> lowest control index; argmax ties -> lowest colour.
 *   R11 phi = 1 on Omega_0^j, 0 on the other targets, the ghost ring and
 *       unreachable nodes; Eq. (HJBridotta_discreta) holds elsewhere.
 *   R12 label = argmax_j phi^j when that maximum is positive (this is the 1/2
 *       projection wherever some colour reaches 1/2, and the "relaxed
 *       threshold" of Remark 3.1 elsewhere); nodes with all phi^j = 0 take
 *       the label of their first labelled axis neighbour in increasing node
 *       index, repeated (Jacobi rounds) until nothing changes.
 *   R13 The foot cell of x_i + k a always has x_i as a corner, with weight
 *       w_s(a) = prod_d (1 - |a_d|) > 0 unless the foot lands on a node.
 *       With R3, U = +inf off the target is therefore itself a fixed point
 *       of F whenever no control lands on a node, and fronts of other shapes
 *       stall the same way (a node needs a lateral neighbour that needs it).
 *       The start U^(0) = +inf of Eq. (iterativeSLscheme) cannot be taken
 *       literally; see R14.  (og_F_node mode 1, the scalar equation solved
 *       for u_i, is kept for the tests that check it has the same fixed
 *       points.)
 *   R14 The solution is the finite fixed point of F on S*, the nodes from
 *       which some admissible feedback reaches the target with probability
 *       one when the Q1 weights are read as transition probabilities (a
 *       control is admissible when no positive-weight corner is +inf); it is
 *       +inf off S*.  On S* this fixed point is unique (every other policy
 *       pays h > 0 forever), so the iteration may start from any finite
 *       value: it starts from M = 1e6, above every value of the solution,
 *       and decreases to it (a start from 0 also converges, but then the
 *       minimum over controls picks up values that are still too small and
 *       Gauss-Seidel needs O(n) sweeps).
 *   R16 Dirichlet patch boundary (Eq. dbc, Sec. 5): while patch j is solved,
 *       every node outside patch j and outside Omega_0^j holds the fixed
 *       value U_P^(0) = I[U~_P] of Step 2 read literally (R2, R3: +inf where a
 *       positive-weight coarse corner is +inf; the bound M of R7 serves the
 *       feedback only, its M-weighted values are no data), 0 on every target
 *       part, +inf on the ghost ring; nodes of patch j that are off S* stay
 *       +inf.  Nodes with a finite fixed value count as target for S* (R14).
 *   R17 AO1 (Sec. 6): the nodes of S* start from U_P^(0) where it is
 *       finite and from M elsewhere; the iteration is the plain U <- F(U)
 *       and reaches the same fixed point (R14: unique on S*).
 *   R18 AO2 (Sec. 6): Gauss-Seidel visits the nodes of a patch in
 *       increasing U_P^(0) (ties: increasing node index; +inf last), the
 *       same order every sweep.
 *   R19 AO3 (Sec. 6): at node i the minimum runs over
 *       A_r(i) = { a : a . a*_{k~}(x_i) >= cos(pi/r) }, with a*_{k~} from
 *       Step 2; the comparison has a slack of 1e-12 so that a control at
 *       exactly the angle pi/r is kept whatever the rounding of the dot
 *       product.  Nodes without a* keep the full set.  Labels (Step 3.1) do
 *       not change.
 *   R20 Dynamics other than c(x) a (Table 1): with |h f| = k (R1) the foot
 *       is x_i + k f/|f| and h_{i,a} = k/|f(x_i,a)|.  For the drift dynamics
 *       f = s a + w (Zermelo) both are fixed per control; components of f/|f|
 *       below 1e-15 are snapped to 0.  A control with |f| <= 1e-15 is not
 *       admissible.
 *   R21 A node where the speed c(x) is at most 1e-12 (the line where the Fan
 *       field vanishes) cannot move: it is treated like the ghost ring (+inf,
 *       colour 0, label -1) unless it is a target node.
 *   R22 Target split into R parts (Sec. 3, "the target is divided in R
 *       parts"; Table 1): one ball split into R equal angular sectors, part
 *       j = floor(R theta / (2 pi) + 1e-9) mod R with theta = atan2 of the
 *       offset from the centre in [0, 2 pi); or the slab |x_1 - v| <= r (a
 *       line target of half-width r) split into R equal pieces along x_2 over
 *       the box, part j = floor(R (x_2 - lo_2) / (hi_2 - lo_2) + 1e-9),
 *       clamped.  The 1e-9 puts nodes exactly on a sector boundary into the
 *       upper part whatever the last bit of atan2.  In 3D (Sec. 7, R = 8) a
 *       ball's sectors are the wedges of the azimuth theta of (x_1, x_2)
 *       around the x_3 axis through the centre, and the plane slab's pieces
 *       are strips along x_2, by the same formulas.  A ball may instead be
 *       split into its 2^d orthants: part j has bit d set iff x_d >= c_d.  On the coarse grid (R6) the
 *       ball or slab is widened by k~ sqrt(d)/2 with boundary value
 *       max(0, distance - r)/c(x).
 *   R24 Brockett's integrator (Sec. 7): f(x, a) = (a1, a2, x1 a2 - x2 a1)
 *       with a in {-5, 0, 5}^2 (rows (a1, a2, unused) of the control table,
 *       speed field c = 1).  As in R20 the foot is x_i + k f/|f| and h_{i,a} =
 *       k/|f|, now per node: x1 a2 - x2 a1 is formed at the node, |f| as
 *       sqrt(f1^2 + f2^2 + f3^2) summed in that order; a = 0 is not
 *       admissible.  The coarse boundary values of R6 use the largest |f(x, a)|
 *       over the controls as the speed (a lower bound on the time: the
 *       dynamics cannot head straight for the ball in general).
 *   R23 Obstacles (Sec. 4, "Patchy method with obstacles"): closed balls
 *       |x - c|^2 <= r^2 and closed boxes lo <= x <= hi (per axis) of the
 *       state space.  A node inside one is a state constraint like the ghost
 *       ring (+inf, never updated, colour 0, label -1) unless it is a target
 *       node; on the coarse grid of Step 1 the same rule holds for its nodes.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_FREE 0
#define OG_TARGET 1
#define OG_GHOST 2

typedef struct {
    int dim;                   /* 2 or 3 */
    int n[3];                  /* nodes per side; n[2] = 1 in 2D */
    double lo[3];              /* lower corner of the box Omega */
    double k;                  /* space step (equal on every axis) */
    int speed_kind;            /* 0 one, 1 sincos2d, 2 sin3d, 3 fourier2d */
    double speed_params[64];
    int n_controls;
    const double *controls;    /* n_controls x dim unit vectors */
    int n_targets;
    const double *targets;     /* n_targets x (dim + 1): centre, radius */
    int dyn_kind;              /* 0: f = c(x) a; 1: f = s a + w (R20);
                                  2: Brockett f = (a1, a2, x1 a2 - x2 a1) (R24) */
    double drift[4];           /* dyn_kind 1: s, w_1, w_2, w_3 */
    int target_kind;           /* 0: each row a ball and a part; 1: row 0 a ball in
                                  n_parts sectors; 2: row 0 = (v, ., r) the slab
                                  |x_1 - v| <= r in n_parts pieces; 3: row 0 a
                                  ball in its 2^dim orthants (R22) */
    int n_parts;               /* parts of target kinds 1 and 2 */
    int n_obstacles;           /* R23 */
    const double *obstacles;   /* n_obstacles x 7: kind (0 ball, 1 box), then a
                                  ball's centre (3) and radius, or a box's lower
                                  (3) and upper (3) corners */
} og_problem;

typedef struct {
    int sweeps_coarse;
    double residual_coarse;
    int sweeps_phi[64];
    double residual_phi[64];
    int sweeps_patch[64];
    double residual_patch[64];
    int64_t patch_nodes[64];
    int64_t unreachable;
    int64_t uncovered_filled;
    int64_t uncovered_left;
} og_patchy_stats;

/* Per-node control filter of AO3 (R19); a NULL filter keeps every control. */
typedef struct {
    const int *astar;   /* per node; -1 keeps the full set */
    double cos_r;       /* cos(pi / r) - 1e-12 */
} og_filter;

/* Options of the patchy solve beyond the basic algorithm of Sec. 3. */
typedef struct {
    int dirichlet;        /* R16: Eq. dbc instead of state constraints */
    int warm;             /* R17: AO1 */
    int causal;           /* R18: AO2 */
    double reduce_r;      /* R19: AO3 reduction factor r > 1; 0 = off */
    const double *data;   /* optional Dirichlet data replacing U_P^(0) (N) */
} og_addons;

static const double OG_PI = 3.14159265358979323846;

static int og_allowed(const og_problem *p, const og_filter *f, int64_t i, int m) {
    if (!f || !f->astar || f->astar[i] < 0) return 1;
    const double *a = p->controls + (size_t)m * p->dim;
    const double *b = p->controls + (size_t)f->astar[i] * p->dim;
    double dot = 0.0;
    for (int d = 0; d < p->dim; ++d) dot += a[d] * b[d];
    return dot >= f->cos_r;
}

/* ---------------------------------------------------------------- grid --- */

static int64_t og_count(const og_problem *p) {
    return (int64_t)p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1);
}

static void og_index3(const og_problem *p, int64_t i, int idx[3]) {
    idx[0] = (int)(i % p->n[0]);
    int64_t r = i / p->n[0];
    idx[1] = (int)(r % p->n[1]);
    idx[2] = (p->dim == 3) ? (int)(r / p->n[1]) : 0;
}

static int64_t og_linear(const og_problem *p, const int idx[3]) {
    return (int64_t)idx[0] + (int64_t)p->n[0] * ((int64_t)idx[1] + (int64_t)p->n[1] * idx[2]);
}

static void og_coords(const og_problem *p, const int idx[3], double x[3]) {
    for (int d = 0; d < 3; ++d) x[d] = (d < p->dim) ? p->lo[d] + idx[d] * p->k : 0.0;
}

/* Speed c(x) of the dynamics f(x,a) = c(x) a (fixed menu of fields). */
double og_speed(const og_problem *p, const double x[3]) {
    const double *q = p->speed_params;
    switch (p->speed_kind) {
    case 0:
        return 1.0;
    case 1:
        return 1.0 + q[0] * sin(2.0 * OG_PI * x[0]) * cos(2.0 * OG_PI * x[1]);
    case 2:
        return 1.0 + q[0] * sin(OG_PI * x[0]) * sin(OG_PI * x[1]) * sin(OG_PI * x[2]);
    case 4:
        /* Fan (Table 1): c(x) = |q0 + q1 x1 + q2 x2 + q3 x3| */
        return fabs(q[0] + q[1] * x[0] + q[2] * x[1] + q[3] * x[2]);
    case 3: {
        /* g(x) = sum_{p,q=0..3} a_pq cos(pi p x1/2 + th_pq) cos(pi q x2/2 + ps_pq) / sum |a_pq| */
        double g = 0.0, norm = 0.0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                int m = 4 * a + b;
                g += q[m] * cos(OG_PI * a * x[0] / 2.0 + q[16 + m]) * cos(OG_PI * b * x[1] / 2.0 + q[32 + m]);
                norm += fabs(q[m]);
            }
        return 1.0 + 0.5 * g / norm;
    }
    default:
        return NAN;
    }
}

/* Largest speed along the unit direction e that the dynamics allow at x
   (R6): c(x) for f = c(x) a; for f = s a + w the v >= 0 with |v e - w| = s
   (0 when e cannot be followed). */
static double og_approach_speed(const og_problem *p, const double x[3], const double e[3]) {
    if (p->dyn_kind == 2) {
        /* R24: the largest |f(x, a)| over the controls */
        double best = 0.0;
        for (int m = 0; m < p->n_controls; ++m) {
            const double *a = p->controls + (size_t)m * p->dim;
            const double f2 = x[0] * a[1] - x[1] * a[0];
            const double nf = sqrt(a[0] * a[0] + a[1] * a[1] + f2 * f2);
            if (nf > best) best = nf;
        }
        return best;
    }
    if (p->dyn_kind != 1) return og_speed(p, x);
    double ew = 0.0, ww = 0.0;
    for (int d = 0; d < p->dim; ++d) {
        ew += e[d] * p->drift[1 + d];
        ww += p->drift[1 + d] * p->drift[1 + d];
    }
    const double disc = ew * ew + p->drift[0] * p->drift[0] - ww;
    if (disc < 0.0) return 0.0;
    const double v = ew + sqrt(disc);
    return v > 0.0 ? v : 0.0;
}

/* Number of patches R: one per target row, or n_parts for a split target. */
int og_parts(const og_problem *p) {
    return p->target_kind == 0 ? p->n_targets : p->n_parts;
}

/* Target part of the point x (R5, R22), -1 outside the target; the balls or
   slab widened by extra (R6).  *gap gets the distance from x to the
   un-widened target (0 inside). */
static int og_target_part(const og_problem *p, const double x[3], double extra, double *gap, double e[3]) {
    const int R = og_parts(p);
    if (e) e[0] = e[1] = e[2] = 0.0;
    if (p->target_kind == 0) {
        for (int j = 0; j < p->n_targets; ++j) {
            const double *t = p->targets + (size_t)j * (p->dim + 1);
            double r2 = 0.0;
            for (int d = 0; d < p->dim; ++d) r2 += (x[d] - t[d]) * (x[d] - t[d]);
            const double dist = sqrt(r2);
            if (dist <= t[p->dim] + extra) {
                if (gap) *gap = dist > t[p->dim] ? dist - t[p->dim] : 0.0;
                if (e && dist > 0.0)
                    for (int d = 0; d < p->dim; ++d) e[d] = (t[d] - x[d]) / dist;
                return j;
            }
        }
        return -1;
    }
    const double *t = p->targets;
    if (p->target_kind == 1) {
        const double dx = x[0] - t[0], dy = x[1] - t[1];
        const double dz = p->dim == 3 ? x[2] - t[2] : 0.0;
        const double dist = sqrt(p->dim == 3 ? dx * dx + dy * dy + dz * dz : dx * dx + dy * dy);
        if (!(dist <= t[p->dim] + extra)) return -1;
        if (e && dist > 0.0) {
            e[0] = -dx / dist;
            e[1] = -dy / dist;
            e[2] = -dz / dist;
        }
        double th = atan2(dy, dx);
        if (th < 0.0) th += 2.0 * OG_PI;
        int j = (int)floor((double)R * th / (2.0 * OG_PI) + 1e-9);
        if (j >= R) j -= R;
        if (j < 0) j = 0;
        if (gap) *gap = dist > t[p->dim] ? dist - t[p->dim] : 0.0;
        return j;
    }
    if (p->target_kind == 3) {
        double r2 = 0.0;
        for (int d = 0; d < p->dim; ++d) r2 += (x[d] - t[d]) * (x[d] - t[d]);
        const double dist = sqrt(r2);
        if (!(dist <= t[p->dim] + extra)) return -1;
        int j = 0;
        for (int d = 0; d < p->dim; ++d) {
            if (x[d] >= t[d]) j |= 1 << d;
            if (e && dist > 0.0) e[d] = (t[d] - x[d]) / dist;
        }
        if (gap) *gap = dist > t[p->dim] ? dist - t[p->dim] : 0.0;
        return j;
    }
    /* slab |x_1 - v| <= r split along x_2 */
    const double dist = fabs(x[0] - t[0]);
    if (!(dist <= t[p->dim] + extra)) return -1;
    if (e && dist > 0.0) e[0] = x[0] < t[0] ? 1.0 : -1.0;
    const double lo1 = p->lo[1], hi1 = p->lo[1] + (double)(p->n[1] - 1) * p->k;
    int j = (int)floor((double)R * (x[1] - lo1) / (hi1 - lo1) + 1e-9);
    if (j >= R) j = R - 1;
    if (j < 0) j = 0;
    if (gap) *gap = dist > t[p->dim] ? dist - t[p->dim] : 0.0;
    return j;
}

/* Is x inside an obstacle (R23)? */
static int og_in_obstacle(const og_problem *p, const double x[3]) {
    for (int o = 0; o < p->n_obstacles; ++o) {
        const double *b = p->obstacles + (size_t)o * 7;
        if (b[0] == 0.0) {
            double r2 = 0.0;
            for (int d = 0; d < p->dim; ++d) r2 += (x[d] - b[1 + d]) * (x[d] - b[1 + d]);
            if (r2 <= b[4] * b[4]) return 1;
        } else {
            int in = 1;
            for (int d = 0; d < p->dim; ++d)
                if (!(x[d] >= b[1 + d] && x[d] <= b[4 + d])) in = 0;
            if (in) return 1;
        }
    }
    return 0;
}

/* Node kinds (R4, R5, R21, R22, R23): target part (>= 0) or -1; kind FREE /
   TARGET / GHOST.  h_i = k / c(x_i) on every node (R1); +inf where the node
   cannot move.  radius_extra widens the target (R6, on the coarse grid). */
int og_setup(const og_problem *p, double radius_extra, unsigned char *kind, int *part, double *h) {
    int64_t N = og_count(p);
    for (int64_t i = 0; i < N; ++i) {
        int idx[3];
        double x[3];
        og_index3(p, i, idx);
        og_coords(p, idx, x);
        int pj = og_target_part(p, x, radius_extra, NULL, NULL);
        int ring = 0;
        for (int d = 0; d < p->dim; ++d)
            if (idx[d] == 0 || idx[d] == p->n[d] - 1) ring = 1;
        const double c = og_speed(p, x);
        const int stopped = !(c > 1e-12);   /* R21 */
        part[i] = pj;
        const int blocked = og_in_obstacle(p, x);   /* R23 */
        kind[i] = (pj >= 0) ? OG_TARGET : ((ring || stopped || blocked) ? OG_GHOST : OG_FREE);
        h[i] = stopped ? INFINITY : p->k / c;
    }
    return 0;
}

/* Direction of the foot and time step of control m at node i (R1, R20):
   d = f/|f| and the return value h_{i,m} = k/|f| (+inf: not admissible).
   For f = c(x) a these are a and the node's h[i]. */
static double og_dir(const og_problem *p, const double *h, int64_t i, int m, double dv[3]) {
    const double *a = p->controls + (size_t)m * p->dim;
    dv[0] = dv[1] = dv[2] = 0.0;
    if (p->dyn_kind == 2) {
        /* Brockett (Sec. 7, R24): f = (a1, a2, x1 a2 - x2 a1) at the node */
        int idx[3];
        double x[3];
        og_index3(p, i, idx);
        og_coords(p, idx, x);
        const double f[3] = {a[0], a[1], x[0] * a[1] - x[1] * a[0]};
        const double nf = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        if (!(nf > 1e-15)) return INFINITY;
        for (int d = 0; d < 3; ++d) {
            const double v = f[d] / nf;
            dv[d] = fabs(v) < 1e-15 ? 0.0 : v;
        }
        return p->k / nf;
    }
    if (p->dyn_kind == 1) {
        double f[3] = {0.0, 0.0, 0.0}, n2 = 0.0;
        for (int d = 0; d < p->dim; ++d) {
            f[d] = p->drift[0] * a[d] + p->drift[1 + d];
            n2 += f[d] * f[d];
        }
        const double nf = sqrt(n2);
        if (!(nf > 1e-15)) return INFINITY;
        for (int d = 0; d < p->dim; ++d) {
            const double v = f[d] / nf;
            dv[d] = fabs(v) < 1e-15 ? 0.0 : v;
        }
        return p->k / nf;
    }
    for (int d = 0; d < p->dim; ++d) dv[d] = a[d];
    return h ? h[i] : p->k;
}

/* ------------------------------------------------------- interpolation --- */

/* I[U] at a point given in grid-index coordinates xi (R2, R3). */
double og_interp(const og_problem *p, const double *U, const double xi[3]) {
    int base[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < p->dim; ++d) {
        if (!(xi[d] >= 0.0 && xi[d] <= (double)(p->n[d] - 1))) return INFINITY;
        int b = (int)floor(xi[d]);
        if (b > p->n[d] - 2) b = p->n[d] - 2;
        if (b < 0) b = 0;
        base[d] = b;
        t[d] = xi[d] - b;
    }
    double sum = 0.0;
    int corners = 1 << p->dim;
    for (int c = 0; c < corners; ++c) {
        double w = 1.0;
        int idx[3] = {base[0], base[1], base[2]};
        for (int d = 0; d < p->dim; ++d) {
            if (c & (1 << d)) {
                w *= t[d];
                idx[d] += 1;
            } else {
                w *= 1.0 - t[d];
            }
        }
        if (w > 0.0) {
            double v = U[og_linear(p, idx)];
            if (isinf(v)) return INFINITY;
            sum += w * v;
        }
    }
    return sum;
}

#define OG_U0_BOUND 1.0e6

/* Q1 of the coarse values with +inf read as the bound M (R7). */
static double og_interp_bounded(const og_problem *p, const double *U, const double xi[3]) {
    int base[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < p->dim; ++d) {
        int b = (int)floor(xi[d]);
        if (b > p->n[d] - 2) b = p->n[d] - 2;
        if (b < 0) b = 0;
        base[d] = b;
        t[d] = xi[d] - b;
    }
    double sum = 0.0;
    int corners = 1 << p->dim;
    for (int c = 0; c < corners; ++c) {
        double w = 1.0;
        int idx[3] = {base[0], base[1], base[2]};
        for (int d = 0; d < p->dim; ++d) {
            if (c & (1 << d)) {
                w *= t[d];
                idx[d] += 1;
            } else {
                w *= 1.0 - t[d];
            }
        }
        if (w > 0.0) {
            double v = U[og_linear(p, idx)];
            sum += w * (isinf(v) ? OG_U0_BOUND : v);
        }
    }
    return sum;
}

int og_interp_points(const og_problem *p, const double *U, int64_t npts, const double *xi, double *out) {
    for (int64_t q = 0; q < npts; ++q) out[q] = og_interp(p, U, xi + 3 * q);
    return 0;
}

/* ----------------------------------------------------------- SL scheme --- */

/* One component at a free node i.
   mode 0: [F(U)]_i of Eq. (SLscheme) literally, min_a { I[U](x_i + k a) + h_i }.
   mode 1: the same scalar equation solved exactly for u_i (R13, tests): the foot
           cell of x_i + k a always has x_i itself as a corner, with weight
           w_s(a); u_i = min_a (sum_{c != i} w_c u_c + h_i) / (1 - w_s(a)).
   Returns the minimum; *arg gets the argmin (lowest index on ties, R10) and
   *gap the gap between the best and second-best values (both optional). */
static double og_F_node(const og_problem *p, const double *U, const double *h, int64_t i, int mode,
                        const og_filter *flt, int *arg, double *gap) {
    int idx[3];
    og_index3(p, i, idx);
    double best = INFINITY, second = INFINITY;
    int besta = -1;
    for (int m = 0; m < p->n_controls; ++m) {
        if (!og_allowed(p, flt, i, m)) continue;
        double a[3];
        const double hm = og_dir(p, h, i, m, a);
        if (isinf(hm)) continue;
        double xi[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < p->dim; ++d) xi[d] = (double)idx[d] + a[d];
        double v;
        if (mode == 0) {
            v = og_interp(p, U, xi) + hm;
        } else {
            int base[3] = {0, 0, 0};
            double t[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < p->dim; ++d) {
                int b = (int)floor(xi[d]);
                if (b > p->n[d] - 2) b = p->n[d] - 2;
                if (b < 0) b = 0;
                base[d] = b;
                t[d] = xi[d] - b;
            }
            double rest = 0.0, wself = 0.0;
            int corners = 1 << p->dim;
            for (int c = 0; c < corners && !isinf(rest); ++c) {
                double w = 1.0;
                int cidx[3] = {base[0], base[1], base[2]};
                for (int d = 0; d < p->dim; ++d) {
                    if (c & (1 << d)) {
                        w *= t[d];
                        cidx[d] += 1;
                    } else {
                        w *= 1.0 - t[d];
                    }
                }
                if (!(w > 0.0)) continue;
                int64_t ci = og_linear(p, cidx);
                if (ci == i) {
                    wself = w;
                } else if (isinf(U[ci])) {
                    rest = INFINITY;
                } else {
                    rest += w * U[ci];
                }
            }
            v = (wself < 1.0) ? (rest + hm) / (1.0 - wself) : INFINITY;
        }
        if (v < best) {
            second = best;
            best = v;
            besta = m;
        } else if (v < second) {
            second = v;
        }
    }
    if (arg) *arg = isinf(best) ? -1 : besta;
    if (gap) *gap = second - best;
    return best;
}

/* U_out = F(U_in) (Eq. SLscheme, mode 0) or its node-wise exact form (mode 1),
   one plain Jacobi application.  upd[i] selects the nodes where the
   min-formula applies; every other node keeps its value (0 on the target,
   +inf on dG as set by the caller). */
int og_sl_apply(const og_problem *p, const unsigned char *upd, const double *h, const double *Uin,
                double *Uout, int mode) {
    int64_t N = og_count(p);
    for (int64_t i = 0; i < N; ++i) Uout[i] = upd[i] ? og_F_node(p, Uin, h, i, mode, NULL, NULL, NULL) : Uin[i];
    return 0;
}

/* The same application with the nodes split over the host's threads (the
   paper's Method 1 of Sec. 3, "How to parallelize the algorithm": the nodes
   of a sweep divided among processors).  A Jacobi application reads only
   Uin, so the split changes no value.  Used to time the CPU baseline on all
   host cores; returns the thread count used. */
int og_sl_apply_par(const og_problem *p, const unsigned char *upd, const double *h, const double *Uin,
                    double *Uout, int mode) {
    int64_t N = og_count(p);
    int used = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) Uout[i] = upd[i] ? og_F_node(p, Uin, h, i, mode, NULL, NULL, NULL) : Uin[i];
    }
#else
    for (int64_t i = 0; i < N; ++i) Uout[i] = upd[i] ? og_F_node(p, Uin, h, i, mode, NULL, NULL, NULL) : Uin[i];
#endif
    return used;
}

static double og_change(double a, double b) {
    if (isinf(a) && isinf(b)) return 0.0;  /* R9 */
    return fabs(a - b);
}

/* Visit order of sweep s (R8).  Returns the node index of the q-th visit. */
static int64_t og_visit(const og_problem *p, int order, int s, int64_t q) {
    if (order != 1) return q;
    int idx[3];
    og_index3(p, q, idx);
    int dir = s % (1 << p->dim);
    for (int d = 0; d < p->dim; ++d)
        if (dir & (1 << d)) idx[d] = p->n[d] - 1 - idx[d];
    return og_linear(p, idx);
}

/* Corners of positive weight of the foot x_i + k a (grid coordinates),
   returned as node indices; the return value is their count. */
static int og_support(const og_problem *p, int64_t i, const double *a, int64_t *out) {
    int idx[3];
    og_index3(p, i, idx);
    int base[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < p->dim; ++d) {
        double xi = (double)idx[d] + a[d];
        if (!(xi >= 0.0 && xi <= (double)(p->n[d] - 1))) return -1;
        int b = (int)floor(xi);
        if (b > p->n[d] - 2) b = p->n[d] - 2;
        if (b < 0) b = 0;
        base[d] = b;
        t[d] = xi - b;
    }
    int cnt = 0;
    for (int c = 0; c < (1 << p->dim); ++c) {
        double w = 1.0;
        int cidx[3] = {base[0], base[1], base[2]};
        for (int d = 0; d < p->dim; ++d) {
            if (c & (1 << d)) { w *= t[d]; cidx[d] += 1; }
            else w *= 1.0 - t[d];
        }
        if (w > 0.0) out[cnt++] = og_linear(p, cidx);
    }
    return cnt;
}

/* The set S* of nodes (among upd[i] = 1) from which the target can be
   reached with probability one (R14).  A control is admissible at i when
   every positive-weight corner of its foot other than x_i lies in the
   current candidate set C or on the target (U finite and not updated); a
   node is kept when some admissible control puts positive weight on a node
   already known to reach the target.  C shrinks to the set reached, and the
   two steps repeat until C no longer changes (the classical fixed point for
   almost-sure reachability in Markov decision processes). */
static int og_reachable_f(const og_problem *p, const unsigned char *upd, const double *U, const og_filter *flt,
                          unsigned char *inS) {
    const int64_t N = og_count(p);
    unsigned char *C = (unsigned char *)malloc((size_t)N);
    if (!C) return -1;
    for (int64_t i = 0; i < N; ++i) C[i] = upd[i];
    int64_t sup[8];
    for (;;) {
        /* B = nodes of C reaching the target with positive probability */
        for (int64_t i = 0; i < N; ++i) inS[i] = 0;
        int grew = 1, pass = 0;
        while (grew) {
            grew = 0;
            for (int64_t q = 0; q < N; ++q) {
                int64_t i = og_visit(p, 1, pass, q);
                if (!C[i] || inS[i]) continue;
                for (int m = 0; m < p->n_controls && !inS[i]; ++m) {
                    if (!og_allowed(p, flt, i, m)) continue;
                    double dv[3];
                    if (isinf(og_dir(p, NULL, i, m, dv))) continue;
                    int cnt = og_support(p, i, dv, sup);
                    if (cnt < 0) continue;
                    int admissible = 1, hits = 0;
                    for (int c = 0; c < cnt; ++c) {
                        int64_t ci = sup[c];
                        if (ci == i) continue;
                        int target = !upd[ci] && !isinf(U[ci]);
                        if (!(C[ci] || target)) admissible = 0;
                        if (target || inS[ci]) hits = 1;
                    }
                    if (admissible && hits) { inS[i] = 1; grew = 1; }
                }
            }
            ++pass;
        }
        int64_t removed = 0;
        for (int64_t i = 0; i < N; ++i)
            if (C[i] && !inS[i]) { C[i] = 0; removed++; }
        if (!removed) break;
    }
    free(C);
    return 0;
}

int og_reachable(const og_problem *p, const unsigned char *upd, const double *U, unsigned char *inS) {
    return og_reachable_f(p, upd, U, NULL, inS);
}

/* Start value on S* (R14): any finite start converges to the unique fixed
   point on S*; a start above the solution converges fastest, because the
   minimum over controls ignores values that are still too large. */
#define OG_START 1.0e6

/* Fixed-point iteration of Eq. (iterativeSLscheme) on the nodes with upd[i]
   = 1 (R14): nodes outside S* are set to +inf, nodes of S* start from M (or
   from warm[i] where warm is given and finite, R17) and the iteration
   U <- F(U) runs in place (Gauss-Seidel: orders 0 and 1, or the fixed visit
   list perm of R18 when given) or as U^{n+1} = F(U^n) (order 2) until the
   sup-norm change of one sweep is below tol (Sec. 2.2, Step 4).  Values of
   nodes with upd[i] = 0 are read as given (0 on the target, +inf or fixed
   boundary data elsewhere).  flt restricts the controls (R19). */
static int og_iterate_ex(const og_problem *p, const unsigned char *upd, const double *h, double *U, double tol,
                         int max_sweeps, int order, const int64_t *perm, int64_t nperm, const double *warm,
                         const og_filter *flt, int *sweeps_out, double *res_out) {
    int64_t N = og_count(p);
    unsigned char *inS = (unsigned char *)malloc((size_t)N);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N);
    if (!inS || !tmp) {
        free(inS); free(tmp);
        return -1;
    }
    og_reachable_f(p, upd, U, flt, inS);
    for (int64_t i = 0; i < N; ++i)
        if (upd[i]) U[i] = inS[i] ? ((warm && isfinite(warm[i])) ? warm[i] : OG_START) : INFINITY;
    int s = 0;
    double res = INFINITY;
    while (s < max_sweeps) {
        res = 0.0;
        if (order == 2) {
            for (int64_t i = 0; i < N; ++i) tmp[i] = inS[i] ? og_F_node(p, U, h, i, 0, flt, NULL, NULL) : U[i];
            for (int64_t i = 0; i < N; ++i) {
                double c = og_change(tmp[i], U[i]);
                if (c > res) res = c;
                U[i] = tmp[i];
            }
        } else {
            const int64_t nv = perm ? nperm : N;
            for (int64_t q = 0; q < nv; ++q) {
                int64_t i = perm ? perm[q] : og_visit(p, order, s, q);
                if (!inS[i]) continue;
                double v = og_F_node(p, U, h, i, 0, flt, NULL, NULL);
                double c = og_change(v, U[i]);
                if (c > res) res = c;
                U[i] = v;
            }
        }
        ++s;
        if (res < tol) break;
    }
    free(tmp);
    free(inS);
    if (sweeps_out) *sweeps_out = s;
    if (res_out) *res_out = res;
    return res < tol ? 0 : 1;
}

int og_iterate(const og_problem *p, const unsigned char *upd, const double *h, double *U, double tol,
               int max_sweeps, int order, int *sweeps_out, double *res_out) {
    return og_iterate_ex(p, upd, h, U, tol, max_sweeps, order, NULL, 0, NULL, NULL, sweeps_out, res_out);
}

/* The same iteration with the AO3 control cones of R19 around a given
   per-node control index field astar (-1: full set) and factor r. */
int og_iterate_reduced(const og_problem *p, const unsigned char *upd, const double *h, double *U, double tol,
                       int max_sweeps, int order, const int *astar, double r, int *sweeps_out, double *res_out) {
    og_filter f = {astar, cos(OG_PI / r) - 1e-12};
    return og_iterate_ex(p, upd, h, U, tol, max_sweeps, order, NULL, 0, NULL, &f, sweeps_out, res_out);
}

/* Global SL solve (Eq. iterativeSLscheme on the whole grid): U^(0) = 0 on
   the target, +inf elsewhere; returns 0 when converged, 1 when the sweep cap
   was hit. */
int og_global_solve(const og_problem *p, double tol, int max_sweeps, int order, double *U,
                    int *sweeps_out, double *res_out) {
    int64_t N = og_count(p);
    unsigned char *kind = (unsigned char *)malloc((size_t)N);
    unsigned char *upd = (unsigned char *)malloc((size_t)N);
    int *part = (int *)malloc(sizeof(int) * (size_t)N);
    double *h = (double *)malloc(sizeof(double) * (size_t)N);
    if (!kind || !upd || !part || !h) {
        free(kind); free(upd); free(part); free(h);
        return -1;
    }
    og_setup(p, 0.0, kind, part, h);
    for (int64_t i = 0; i < N; ++i) {
        upd[i] = kind[i] == OG_FREE;
        U[i] = kind[i] == OG_TARGET ? 0.0 : INFINITY;
    }
    int rc = og_iterate(p, upd, h, U, tol, max_sweeps, order, sweeps_out, res_out);
    free(kind); free(upd); free(part); free(h);
    return rc;
}

/* ------------------------------------------------------- patchy method --- */

/* phi^j of Step 3.1 (Eq. HJBridotta_discreta) with the fixed coarse
   feedback astar: phi_i = I[phi](x_i + k a*_i) on nodes with upd[i] = 1,
   Gauss-Seidel in the given order until the sup-norm change is < tol. */
static int og_phi_iterate(const og_problem *p, const unsigned char *upd, const int *astar, double *phi,
                          double tol, int max_sweeps, int order, int *sweeps_out, double *res_out) {
    int64_t N = og_count(p);
    int s = 0;
    double res = INFINITY;
    while (s < max_sweeps) {
        res = 0.0;
        for (int64_t q = 0; q < N; ++q) {
            int64_t i = og_visit(p, order == 2 ? 0 : order, s, q);
            if (!upd[i]) continue;
            int idx[3];
            og_index3(p, i, idx);
            double a[3];
            og_dir(p, NULL, i, astar[i], a);
            double xi[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < p->dim; ++d) xi[d] = (double)idx[d] + a[d];
            double v = og_interp(p, phi, xi);
            double c = fabs(v - phi[i]);
            if (c > res) res = c;
            phi[i] = v;
        }
        ++s;
        if (res < tol) break;
    }
    if (sweeps_out) *sweeps_out = s;
    if (res_out) *res_out = res;
    return res < tol ? 0 : 1;
}

/* The patchy algorithm (Sec. 3).  Outputs: u (N), labels (N; -1 ghost or
   unreachable, j on patch j and on target part j).  Optional outputs (NULL to
   skip): Ucoarse (coarse N~), U0 = U_P^(0) (N), astar (N; -1 where
   undefined), gap (N; best-vs-second control gap of Step 2), phi (R x N). */
typedef struct {
    double key;
    int64_t i;
} og_keyed;

static int og_keyed_cmp(const void *a, const void *b) {
    const og_keyed *x = (const og_keyed *)a, *y = (const og_keyed *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->i > y->i) - (x->i < y->i);
}

int og_patchy_solve_ex(const og_problem *p, const int n_coarse[3], double tol, double tol_coarse,
                       double tol_phi, int max_sweeps, int order, const og_addons *ao, double *u,
                       signed char *labels, double *Ucoarse_out, double *U0_out, int *astar_out,
                       double *gap_out, double *phi_out, og_patchy_stats *st) {
    const int64_t N = og_count(p);
    const int R = og_parts(p);
    if (R < 1 || R > 64) return -2;
    og_patchy_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof(*st));

    /* ---- Step 1: coarse grid G~ on the same box, solved by the global SL
       scheme (the fixed point the paper's domain decomposition reaches). */
    og_problem pc = *p;
    for (int d = 0; d < 3; ++d) pc.n[d] = (d < p->dim) ? n_coarse[d] : 1;
    pc.k = p->k * (double)(p->n[0] - 1) / (double)(n_coarse[0] - 1);
    const int64_t Nc = og_count(&pc);
    unsigned char *ckind = (unsigned char *)malloc((size_t)Nc);
    unsigned char *cupd = (unsigned char *)malloc((size_t)Nc);
    int *cpart = (int *)malloc(sizeof(int) * (size_t)Nc);
    double *ch = (double *)malloc(sizeof(double) * (size_t)Nc);
    double *Uc = (double *)malloc(sizeof(double) * (size_t)Nc);
    unsigned char *kind = (unsigned char *)malloc((size_t)N);
    unsigned char *upd = (unsigned char *)malloc((size_t)N);
    int *part = (int *)malloc(sizeof(int) * (size_t)N);
    double *h = (double *)malloc(sizeof(double) * (size_t)N);
    double *U0 = (double *)malloc(sizeof(double) * (size_t)N);
    int *astar = (int *)malloc(sizeof(int) * (size_t)N);
    double *phi = (double *)malloc(sizeof(double) * (size_t)N);
    double *phimax = (double *)malloc(sizeof(double) * (size_t)N);
    signed char *lab2 = (signed char *)malloc((size_t)N);
    double *W = (double *)malloc(sizeof(double) * (size_t)N);
    double *Dlit = (double *)malloc(sizeof(double) * (size_t)N);   /* literal I[U~] (R16) */
    int rc = 0;
    if (!ckind || !cupd || !cpart || !ch || !Uc || !kind || !upd || !part || !h || !U0 || !astar || !phi ||
        !phimax || !lab2 || !W || !Dlit) {
        rc = -1;
        goto done;
    }
    og_setup(&pc, pc.k * sqrt((double)p->dim) / 2.0, ckind, cpart, ch);
    for (int64_t i = 0; i < Nc; ++i) {
        cupd[i] = ckind[i] == OG_FREE;
        Uc[i] = INFINITY;
        if (ckind[i] == OG_TARGET) {   /* R6: boundary value dist / c */
            int idx[3];
            double x[3], gap = 0.0, e[3];
            og_index3(&pc, i, idx);
            og_coords(&pc, idx, x);
            og_target_part(&pc, x, pc.k * sqrt((double)p->dim) / 2.0, &gap, e);
            Uc[i] = gap > 0.0 ? gap / og_approach_speed(&pc, x, e) : 0.0;
        }
    }
    if (og_iterate(&pc, cupd, ch, Uc, tol_coarse, max_sweeps, order, &st->sweeps_coarse, &st->residual_coarse))
        rc = 1;
    if (Ucoarse_out) memcpy(Ucoarse_out, Uc, sizeof(double) * (size_t)Nc);

    /* ---- Step 2: U_P^(0) = I[U~_P] on G (R7), then the coarse feedback
       a*_{k~}(x_i) of Eq. (feedbackcontrol) at every free fine node. */
    og_setup(p, 0.0, kind, part, h);
    for (int64_t i = 0; i < N; ++i) {
        if (kind[i] == OG_TARGET) { U0[i] = 0.0; Dlit[i] = 0.0; continue; }
        if (kind[i] == OG_GHOST) { U0[i] = INFINITY; Dlit[i] = INFINITY; continue; }
        int idx[3];
        og_index3(p, i, idx);
        double xi[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < p->dim; ++d)
            xi[d] = (double)idx[d] * (double)(n_coarse[d] - 1) / (double)(p->n[d] - 1);
        U0[i] = og_interp_bounded(&pc, Uc, xi);
        if (U0[i] >= OG_U0_BOUND) U0[i] = INFINITY;
        Dlit[i] = og_interp(&pc, Uc, xi);
    }
    st->unreachable = 0;
    for (int64_t i = 0; i < N; ++i) {
        astar[i] = -1;
        if (gap_out) gap_out[i] = INFINITY;
        if (kind[i] != OG_FREE || isinf(U0[i])) continue;
        int arg;
        double gap;
        og_F_node(p, U0, h, i, 0, NULL, &arg, &gap);
        astar[i] = arg;
        if (gap_out) gap_out[i] = gap;
    }
    for (int64_t i = 0; i < N; ++i)
        if (kind[i] == OG_FREE && astar[i] < 0) st->unreachable++;
    if (U0_out) memcpy(U0_out, U0, sizeof(double) * (size_t)N);
    if (astar_out) memcpy(astar_out, astar, sizeof(int) * (size_t)N);

    /* ---- Step 3.1: phi^j for every colour, then the projection (R11, R12). */
    for (int64_t i = 0; i < N; ++i) {
        upd[i] = kind[i] == OG_FREE && astar[i] >= 0;
        labels[i] = (signed char)(kind[i] == OG_TARGET ? part[i] : -1);
        phimax[i] = 0.0;
    }
    for (int j = 0; j < R; ++j) {
        for (int64_t i = 0; i < N; ++i) phi[i] = (kind[i] == OG_TARGET && part[i] == j) ? 1.0 : 0.0;
        if (og_phi_iterate(p, upd, astar, phi, tol_phi, max_sweeps, order, &st->sweeps_phi[j],
                           &st->residual_phi[j]))
            rc = 1;
        if (phi_out) memcpy(phi_out + (size_t)j * N, phi, sizeof(double) * (size_t)N);
        for (int64_t i = 0; i < N; ++i)
            if (upd[i] && phi[i] > phimax[i]) {  /* strict: ties keep the lower colour */
                phimax[i] = phi[i];
                labels[i] = (signed char)j;
            }
    }
    /* Uncovered reachable nodes (all phi^j = 0): label of the first labelled
       axis neighbour in increasing node index, Jacobi rounds. */
    for (;;) {
        int64_t changed = 0;
        memcpy(lab2, labels, (size_t)N);
        for (int64_t i = 0; i < N; ++i) {
            if (!upd[i] || labels[i] >= 0) continue;
            int idx[3];
            og_index3(p, i, idx);
            int64_t nb[6];
            int cnt = 0;
            for (int d = p->dim - 1; d >= 0; --d)
                if (idx[d] > 0) { int t[3] = {idx[0], idx[1], idx[2]}; t[d] -= 1; nb[cnt++] = og_linear(p, t); }
            for (int d = 0; d < p->dim; ++d)
                if (idx[d] < p->n[d] - 1) { int t[3] = {idx[0], idx[1], idx[2]}; t[d] += 1; nb[cnt++] = og_linear(p, t); }
            for (int c = 0; c < cnt; ++c)
                if (labels[nb[c]] >= 0) { lab2[i] = labels[nb[c]]; break; }
            if (lab2[i] >= 0) changed++;
        }
        memcpy(labels, lab2, (size_t)N);
        st->uncovered_filled += changed;
        if (!changed) break;
    }
    for (int64_t i = 0; i < N; ++i)
        if (upd[i] && labels[i] < 0) st->uncovered_left++;

    /* ---- Step 3.2: each patch solved on its own.  State constraints on its
       boundary (every node outside patch j and outside Omega_0^j is +inf),
       or the Dirichlet data of Eq. (dbc) there (R16); add-ons AO1-AO3 of
       Sec. 6 (R17-R19). */
    {
        const int dir = ao && ao->dirichlet;
        const double *D = (ao && ao->data) ? ao->data : Dlit;
        og_filter flt = {astar, 0.0};
        const og_filter *fp = NULL;
        if (ao && ao->reduce_r > 0.0) {
            flt.cos_r = cos(OG_PI / ao->reduce_r) - 1e-12;
            fp = &flt;
        }
        og_keyed *kv = NULL;
        int64_t *perm = NULL;
        if (ao && ao->causal) {
            kv = (og_keyed *)malloc(sizeof(og_keyed) * (size_t)N);
            perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
            if (!kv || !perm) {
                free(kv); free(perm);
                rc = -1;
                goto done;
            }
        }
        for (int64_t i = 0; i < N; ++i) u[i] = kind[i] == OG_TARGET ? 0.0 : INFINITY;
        for (int j = 0; j < R && rc >= 0; ++j) {
            int64_t cnt = 0;
            for (int64_t i = 0; i < N; ++i) {
                upd[i] = kind[i] == OG_FREE && labels[i] == j;
                if (upd[i] && kv) {
                    kv[cnt].key = U0[i];   /* +inf sorts last */
                    kv[cnt].i = i;
                }
                cnt += upd[i];
                if (kind[i] == OG_TARGET && part[i] == j) W[i] = 0.0;
                else W[i] = (dir && !upd[i]) ? D[i] : INFINITY;
            }
            st->patch_nodes[j] = cnt;
            if (kv) {
                qsort(kv, (size_t)cnt, sizeof(og_keyed), og_keyed_cmp);
                for (int64_t q = 0; q < cnt; ++q) perm[q] = kv[q].i;
            }
            int r2 = og_iterate_ex(p, upd, h, W, tol, max_sweeps, order, perm, cnt,
                                   (ao && ao->warm) ? U0 : NULL, fp, &st->sweeps_patch[j],
                                   &st->residual_patch[j]);
            if (r2 < 0) rc = -1;
            else if (r2 && rc == 0) rc = 1;
            /* ---- Step 4: merge. */
            for (int64_t i = 0; i < N; ++i)
                if (upd[i]) u[i] = W[i];
        }
        free(kv);
        free(perm);
    }

done:
    free(ckind); free(cupd); free(cpart); free(ch); free(Uc);
    free(kind); free(upd); free(part); free(h); free(U0); free(astar); free(phi); free(phimax);
    free(lab2); free(W); free(Dlit);
    return rc;
}

int og_patchy_solve(const og_problem *p, const int n_coarse[3], double tol, double tol_coarse,
                    double tol_phi, int max_sweeps, int order, double *u, signed char *labels,
                    double *Ucoarse_out, double *U0_out, int *astar_out, double *gap_out, double *phi_out,
                    og_patchy_stats *st) {
    return og_patchy_solve_ex(p, n_coarse, tol, tol_coarse, tol_phi, max_sweeps, order, NULL, u, labels,
                              Ucoarse_out, U0_out, astar_out, gap_out, phi_out, st);
}
