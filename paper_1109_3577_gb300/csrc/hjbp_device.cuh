// hjbp_device.cuh -- types and helpers shared by the CUDA kernels of libhjbp.
//
// Node codes (int8, one per node) drive every kernel:
//   -1          hard +inf node: ghost ring dG (state constraints, Sec. 2.1),
//               a node outside the set S* that reaches the target, or (in a
//               per-patch solve) nothing else needs it;
//   0 .. 63     free node belonging to patch j (the plain global solve uses 0);
//   64 + j      target node of part Omega_0^j (value fixed by the caller).
// A free node of patch j reads a neighbour as usable iff its code is j or
// 64 + j; every other neighbour is +inf for it (state constraints on the
// patch boundary, Sec. 3 "Details on boundary conditions").
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/hjbp.h"

namespace hjbp {

constexpr int kTile = 32;                 // 2D tile side (one warp per tile)
constexpr int kMaxControls = HJBP_MAX_CONTROLS;
constexpr int kMaxTargets = HJBP_MAX_TARGETS;
constexpr int8_t kHard = -1;
constexpr int8_t kTargetBase = 64;
constexpr uint8_t kNoControl = 255;

// +inf is carried as a finite sentinel so that a zero weight times "+inf"
// stays 0 (R3: corners of weight 0 are skipped); anything at or above the
// threshold is +inf.  The start value M of the fixed-point iteration on S*
// lies far below the threshold (R14).
template <typename T> struct Num;
template <> struct Num<float> {
    static __host__ __device__ constexpr float big() { return 1.0e30f; }
    static __host__ __device__ constexpr float thresh() { return 1.0e25f; }
    static __host__ __device__ constexpr double noise() { return 0x1p-21; }  // 4 units in the last place
};
template <> struct Num<double> {
    static __host__ __device__ constexpr double big() { return 1.0e300; }
    static __host__ __device__ constexpr double thresh() { return 1.0e290; }
    static __host__ __device__ constexpr double noise() { return 0x1p-50; }
};
constexpr double kStartValue = 1.0e6;     // M, above every solution value (R14)
constexpr double kU0Bound = 1.0e6;        // bound replacing +inf inside U_P^(0) (R7)

// Control table in the self-solved form (R13) grouped by quadrant.  For a
// control a with foot x_i + k a the cell corners other than x_i are
// (i+sx, j), (i, j+sy), (i+sx, j+sy), sx = sign(a_x), sy = sign(a_y) (a >= 0
// counts as +), with Q1 weights w10 = |a_x|(1-|a_y|), w01 = (1-|a_x|)|a_y|,
// w11 = |a_x||a_y| and self weight w00 = (1-|a_x|)(1-|a_y|).  kap = 1/(1-w00)
// and kw* = kap * w*; the update of node i under control a is
//   kap * (w10 u10 + w01 u01 + w11 u11 + h_i).
// Quadrant q = (sx > 0) + 2 (sy > 0); controls of quadrant q occupy
// [qbeg[q], qbeg[q+1]).
template <typename T> struct CtlTable2 {
    int nc;
    int qbeg[5];
    T kw10[kMaxControls];
    T kw01[kMaxControls];
    T kw11[kMaxControls];
    T kap[kMaxControls];
    // Symmetric form, used when the control set is invariant under the eight
    // symmetries of the square (d4 = 1).  Controls a and a' = (|a_y|, |a_x|)
    // in the same quadrant share kap and w11 and swap w10 <-> w01, so
    //   min(v_a, v_a') = kap h + kw11 u11 + s (u10 + u01) - t |u10 - u01|
    // with s = (kw10 + kw01)/2, t = |kw10 - kw01|/2 (t = 0 on the diagonal).
    // Each class stands for one such pair in every quadrant; the four axis
    // directions (kap = 1, one corner) are handled apart (axis = 1).
    int d4;
    int axis;
    int ncls;
    T cls_kap[kMaxControls / 4];
    T cls_s[kMaxControls / 4];
    T cls_t[kMaxControls / 4];
    T cls_kw11[kMaxControls / 4];
    float hfmax;   // max over controls of the time-step factor (kap holds kap * factor)
};

// Per-control self-solved weights in any order (one control per lane).
template <typename T> struct CtlSelf2 {
    int nc;
    int8_t sx[kMaxControls];
    int8_t sy[kMaxControls];
    T kw10[kMaxControls];
    T kw01[kMaxControls];
    T kw11[kMaxControls];
    T kap[kMaxControls];
};

// Literal Q1 weights in the caller's control order, for Eq. (feedbackcontrol),
// in FP64 and rounded to FP32 (the FP32 copy only filters candidates).
struct CtlLiteral2 {
    int nc;
    int8_t sx[kMaxControls];
    int8_t sy[kMaxControls];
    double w00[kMaxControls];
    double w10[kMaxControls];
    double w01[kMaxControls];
    double w11[kMaxControls];
    float f00[kMaxControls];
    float f10[kMaxControls];
    float f01[kMaxControls];
    float f11[kMaxControls];
    double hf[kMaxControls];   // time-step factor: h_{i,a} = hf[a] h_i (1 for f = c(x) a)
    float hff[kMaxControls];
    float hfmax;               // max over controls of hf
};

// Support masks for the almost-sure reachability sweep: bit 0 corner 10,
// bit 1 corner 01, bit 2 corner 11 (positive weight).  present[q] has bit m
// set when some control of quadrant q needs exactly mask m.
struct ReachTable2 {
    uint8_t present[4];
};

// Control cones of add-on AO3 (Sec. 6) for 2D sets of at most 64 controls:
// for a coarse feedback a* (entry nc: no feedback, every control), mask[a*]
// has bit q set when the control at position q of the quadrant-sorted table
// (CtlTable2 order) satisfies a . a* >= cos(pi / r) - 1e-12, and reach[a*]
// holds, per quadrant (8 bits each), the corner patterns of those controls in
// the encoding of ReachTable2.
struct Cone2 {
    unsigned long long mask[65];
    uint32_t reach[65];
    int nc;
    // the same cones in the symmetric pair form of the 8-class control set:
    // bit 16 q + 2 k + member for class k in quadrant q (member 0: the
    // control with |a_x| >= |a_y|, member 1 its mirror), and the axis
    // controls in amask (bit 0 +x, 1 -x, 2 +y, 3 -y); pairs = 0 when the
    // control set has no such form
    unsigned long long pmask[65];
    uint8_t amask[65];
    int pairs;
};

// Speed field c(x) (hjbp_speed_kind) and its parameters, passed by value.
struct SpeedParams {
    int kind;
    double p[64];
};

// Target balls: centres (c0, c1, c2) and radii, passed by value; kind and
// nparts select a split target (hjbp_target_kind), row 0 then describes it.
struct TargetSet {
    int n;
    int kind;
    int nparts;
    double c0[kMaxTargets], c1[kMaxTargets], c2[kMaxTargets], r[kMaxTargets];
};

// Obstacles (Sec. 4): closed balls and boxes whose nodes are state
// constraints like the ghost ring.
constexpr int kMaxObstacles = HJBP_MAX_OBSTACLES;
struct ObstacleSet {
    int n;
    int dim;
    int kind[kMaxObstacles];                // 0 ball, 1 box
    double a[kMaxObstacles][3];             // ball centre / box lower corner
    double b[kMaxObstacles][3];             // ball radius in b[.][0] / box upper corner
};

// Is the node x inside an obstacle?  |x - c|^2 is summed in axis order with
// each product and sum rounded, so membership is decided exactly.
__device__ inline bool in_obstacle(const ObstacleSet &os, double x0, double x1, double x2) {
    for (int o = 0; o < os.n; ++o) {
        if (os.kind[o] == 0) {
            const double d0 = __dsub_rn(x0, os.a[o][0]), d1 = __dsub_rn(x1, os.a[o][1]);
            double r2 = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
            if (os.dim == 3) {
                const double d2 = __dsub_rn(x2, os.a[o][2]);
                r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
            }
            if (r2 <= __dmul_rn(os.b[o][0], os.b[o][0])) return true;
        } else {
            bool in = x0 >= os.a[o][0] && x0 <= os.b[o][0] && x1 >= os.a[o][1] && x1 <= os.b[o][1];
            if (os.dim == 3) in = in && x2 >= os.a[o][2] && x2 <= os.b[o][2];
            if (in) return true;
        }
    }
    return false;
}

// Host side: the checks of the obstacle rows and their device form.
inline const char *check_obstacles(const hjbp_problem_desc *d) {
    if (d->n_obstacles < 0 || d->n_obstacles > HJBP_MAX_OBSTACLES) return "n_obstacles out of range";
    if (d->n_obstacles > 0 && !d->obstacles) return "obstacles is NULL";
    for (int o = 0; o < d->n_obstacles; ++o) {
        const double *r = d->obstacles + 7 * o;
        if (r[0] != 0.0 && r[0] != 1.0) return "obstacle kind must be 0 (ball) or 1 (box)";
        for (int c = 1; c < 7; ++c)
            if (!std::isfinite(r[c])) return "obstacle entry not finite";
        if (r[0] == 0.0 && !(r[4] >= 0.0)) return "obstacle radius must be >= 0";
    }
    return nullptr;
}

inline ObstacleSet make_obstacles(int dim, int n, const double *rows) {
    ObstacleSet os;
    std::memset(&os, 0, sizeof(os));
    os.n = n;
    os.dim = dim;
    for (int o = 0; o < n; ++o) {
        const double *r = rows + 7 * o;
        os.kind[o] = r[0] == 0.0 ? 0 : 1;
        for (int c = 0; c < 3; ++c) os.a[o][c] = r[1 + c];
        if (os.kind[o] == 0) os.b[o][0] = r[4];
        else
            for (int c = 0; c < 3; ++c) os.b[o][c] = r[4 + c];
    }
    return os;
}

// c(x) of f(x, a) = c(x) a (fixed menu, see hjbp_speed_kind).
__device__ inline double speed_at(const SpeedParams &sp, double x0, double x1, double x2) {
    const double pi = 3.14159265358979323846;
    switch (sp.kind) {
    case HJBP_C_ONE:
        return 1.0;
    case HJBP_C_SINCOS2D:
        return 1.0 + sp.p[0] * sin(2.0 * pi * x0) * cos(2.0 * pi * x1);
    case HJBP_C_SIN3D:
        return 1.0 + sp.p[0] * sin(pi * x0) * sin(pi * x1) * sin(pi * x2);
    case HJBP_C_FOURIER2D: {
        double g = 0.0, norm = 0.0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const int m = 4 * a + b;
                g += sp.p[m] * cos(pi * a * x0 / 2.0 + sp.p[16 + m]) * cos(pi * b * x1 / 2.0 + sp.p[32 + m]);
                norm += fabs(sp.p[m]);
            }
        return 1.0 + 0.5 * g / norm;
    }
    case HJBP_C_FAN:
        // |p0 + p1 x1 + p2 x2 + p3 x3|, rounded in this order (no contraction)
        return fabs(__dadd_rn(__dadd_rn(__dadd_rn(sp.p[0], __dmul_rn(sp.p[1], x0)), __dmul_rn(sp.p[2], x1)),
                              __dmul_rn(sp.p[3], x2)));
    default:
        return nan("");
    }
}

// Separable speeds (HJBP_C_SINCOS2D, HJBP_C_SIN3D, HJBP_C_FOURIER2D) are
// products of one factor per axis, so the set-up evaluates the trigonometric
// factors once per grid line (speed_factor, nt per line) and a node only
// multiplies them (speed_lines): the same FP64 operations on the same
// arguments as speed_at, without an FP64 sin or cos per node.
struct SpeedLines {
    const double *f[3];   // per axis: nt factors per grid line, line-major; NULL: evaluate per node
    int nt;
};

__host__ __device__ inline int speed_terms(int kind) {
    return kind == HJBP_C_SINCOS2D || kind == HJBP_C_SIN3D ? 1 : (kind == HJBP_C_FOURIER2D ? 16 : 0);
}

// Factor m of axis `axis` at the coordinate x (speed_terms(kind) > 0).
__device__ inline double speed_factor(const SpeedParams &sp, int axis, int m, double x) {
    const double pi = 3.14159265358979323846;
    switch (sp.kind) {
    case HJBP_C_SINCOS2D:
        return axis == 0 ? sin(2.0 * pi * x) : cos(2.0 * pi * x);
    case HJBP_C_SIN3D:
        return sin(pi * x);
    default: {   // HJBP_C_FOURIER2D: cos(pi a x0 / 2 + theta_ab) cos(pi b x1 / 2 + psi_ab), m = 4 a + b
        const int a = m / 4, b = m % 4;
        return axis == 0 ? cos(pi * a * x / 2.0 + sp.p[16 + m]) : cos(pi * b * x / 2.0 + sp.p[32 + m]);
    }
    }
}

// c at the node (i0, i1, i2) from its lines' factors.
__device__ inline double speed_lines(const SpeedParams &sp, const SpeedLines &L, int i0, int i1, int i2) {
    switch (sp.kind) {
    case HJBP_C_SINCOS2D:
        return 1.0 + sp.p[0] * L.f[0][i0] * L.f[1][i1];
    case HJBP_C_SIN3D:
        return 1.0 + sp.p[0] * L.f[0][i0] * L.f[1][i1] * L.f[2][i2];
    default: {   // HJBP_C_FOURIER2D
        double g = 0.0, norm = 0.0;
        for (int m = 0; m < 16; ++m) {
            g += sp.p[m] * L.f[0][16 * i0 + m] * L.f[1][16 * i1 + m];
            norm += fabs(sp.p[m]);
        }
        return 1.0 + 0.5 * g / norm;
    }
    }
}

// Factors of every grid line: thread e takes line e / nt of the axis whose
// range holds it, term e % nt; x = lo + i k rounded as the set-up rounds it.
static __global__ void k_speed_lines(SpeedParams sp, int nt, int n0, int n1, int n2, double lo0, double lo1,
                                     double lo2, double k, double *f0, double *f1, double *f2) {
    const int total = nt * (n0 + n1 + n2);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int line = e / nt;
        const int m = e % nt;
        int axis = 0;
        double lo = lo0;
        double *out = f0;
        if (line >= n0) {
            line -= n0;
            axis = 1;
            lo = lo1;
            out = f1;
            if (line >= n1) {
                line -= n1;
                axis = 2;
                lo = lo2;
                out = f2;
            }
        }
        const double x = __dadd_rn(lo, __dmul_rn((double)line, k));
        out[(int64_t)line * nt + m] = speed_factor(sp, axis, m, x);
    }
}

// Dynamics of the set-up (hjbp_dyn_kind): for HJBP_DYN_DRIFT, f = s a + w.
struct DynParams {
    int kind;
    double s, w[3];
};

// Largest speed the dynamics allow along the unit direction e at a node of
// speed c (the coarse boundary values): c for f = c(x) a; for f = s a + w the
// v >= 0 with |v e - w| = s (0 when e cannot be followed).
__device__ inline double approach_speed2(const DynParams &dp, double c, double e0, double e1) {
    if (dp.kind != HJBP_DYN_DRIFT) return c;
    const double ew = __dadd_rn(__dmul_rn(e0, dp.w[0]), __dmul_rn(e1, dp.w[1]));
    const double ww = __dadd_rn(__dmul_rn(dp.w[0], dp.w[0]), __dmul_rn(dp.w[1], dp.w[1]));
    const double disc = __dsub_rn(__dadd_rn(__dmul_rn(ew, ew), __dmul_rn(dp.s, dp.s)), ww);
    if (disc < 0.0) return 0.0;
    const double v = __dadd_rn(ew, __dsqrt_rn(disc));
    return v > 0.0 ? v : 0.0;
}

// A node whose speed is at most this cannot move (it is treated like the
// ghost ring unless it is a target node).
constexpr double kStoppedSpeed = 1e-12;

// Geometry of a 2D grid and its tiling of the interior nodes 1..n-2.
struct Grid2 {
    int n0, n1;        // nodes per side
    int ntx, nty;      // tiles per side
    double lo0, lo1, k;
};

// Target part of the 2D point (x0, x1), -1 outside the target; the target is
// widened by extra (the coarse grid's boundary band); *gap = distance to the
// un-widened target (0 inside).  Explicitly rounded operations, so that the
// decisions follow x = lo + i k and the definitions of hjbp_target_kind.
// *e (optional) gets the unit direction from the point towards the target.
// Target part of a 3D node (-1 outside), the target widened by extra; *gap
// the distance to the un-widened target (0 inside).  Balls; one ball in R
// wedges by the azimuth of (x_1, x_2) around the x_3 axis; the plane slab
// |x_1 - v| <= r in R strips along x_2 (Sec. 7).
__device__ inline int target_part3(const TargetSet &ts, double lo1, int n1, double k, double x0, double x1, double x2,
                                   double extra, double *gap) {
    const double pi = 3.14159265358979323846;
    *gap = 0.0;
    if (ts.kind == HJBP_TARGET_BALLS) {
        for (int j = 0; j < ts.n; ++j) {
            const double d0 = __dsub_rn(x0, ts.c0[j]), d1 = __dsub_rn(x1, ts.c1[j]), d2 = __dsub_rn(x2, ts.c2[j]);
            const double d =
                __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
            if (d <= __dadd_rn(ts.r[j], extra)) {
                *gap = d > ts.r[j] ? __dsub_rn(d, ts.r[j]) : 0.0;
                return j;
            }
        }
        return -1;
    }
    const int R = ts.nparts;
    if (ts.kind == HJBP_TARGET_ORTHANTS) {
        const double d0 = __dsub_rn(x0, ts.c0[0]), d1 = __dsub_rn(x1, ts.c1[0]), d2 = __dsub_rn(x2, ts.c2[0]);
        const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
        if (!(d <= __dadd_rn(ts.r[0], extra))) return -1;
        *gap = d > ts.r[0] ? __dsub_rn(d, ts.r[0]) : 0.0;
        return (x0 >= ts.c0[0] ? 1 : 0) | (x1 >= ts.c1[0] ? 2 : 0) | (x2 >= ts.c2[0] ? 4 : 0);
    }
    if (ts.kind == HJBP_TARGET_SECTORS) {
        const double d0 = __dsub_rn(x0, ts.c0[0]), d1 = __dsub_rn(x1, ts.c1[0]), d2 = __dsub_rn(x2, ts.c2[0]);
        const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
        if (!(d <= __dadd_rn(ts.r[0], extra))) return -1;
        double th = atan2(d1, d0);
        if (th < 0.0) th = __dadd_rn(th, 2.0 * pi);
        int j = (int)floor(__dadd_rn(__ddiv_rn(__dmul_rn((double)R, th), 2.0 * pi), 1e-9));
        if (j >= R) j -= R;
        if (j < 0) j = 0;
        *gap = d > ts.r[0] ? __dsub_rn(d, ts.r[0]) : 0.0;
        return j;
    }
    const double d = fabs(__dsub_rn(x0, ts.c0[0]));
    if (!(d <= __dadd_rn(ts.r[0], extra))) return -1;
    const double hi1 = __dadd_rn(lo1, __dmul_rn((double)(n1 - 1), k));
    int j = (int)floor(__dadd_rn(__ddiv_rn(__dmul_rn((double)R, __dsub_rn(x1, lo1)), __dsub_rn(hi1, lo1)), 1e-9));
    if (j >= R) j = R - 1;
    if (j < 0) j = 0;
    *gap = d > ts.r[0] ? __dsub_rn(d, ts.r[0]) : 0.0;
    return j;
}

__device__ inline int target_part2(const TargetSet &ts, const Grid2 &g, double x0, double x1, double extra,
                                   double *gap, double *e = nullptr) {
    const double pi = 3.14159265358979323846;
    if (e) e[0] = e[1] = 0.0;
    if (ts.kind == HJBP_TARGET_BALLS) {
        for (int j = 0; j < ts.n; ++j) {
            const double d0 = __dsub_rn(x0, ts.c0[j]), d1 = __dsub_rn(x1, ts.c1[j]);
            const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)));
            if (d <= __dadd_rn(ts.r[j], extra)) {
                *gap = d > ts.r[j] ? __dsub_rn(d, ts.r[j]) : 0.0;
                if (e && d > 0.0) {
                    e[0] = __ddiv_rn(__dsub_rn(ts.c0[j], x0), d);
                    e[1] = __ddiv_rn(__dsub_rn(ts.c1[j], x1), d);
                }
                return j;
            }
        }
        return -1;
    }
    const int R = ts.nparts;
    if (ts.kind == HJBP_TARGET_ORTHANTS) {
        const double d0 = __dsub_rn(x0, ts.c0[0]), d1 = __dsub_rn(x1, ts.c1[0]);
        const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)));
        if (!(d <= __dadd_rn(ts.r[0], extra))) return -1;
        if (e && d > 0.0) {
            e[0] = __ddiv_rn(-d0, d);
            e[1] = __ddiv_rn(-d1, d);
        }
        *gap = d > ts.r[0] ? __dsub_rn(d, ts.r[0]) : 0.0;
        return (x0 >= ts.c0[0] ? 1 : 0) | (x1 >= ts.c1[0] ? 2 : 0);
    }
    if (ts.kind == HJBP_TARGET_SECTORS) {
        const double d0 = __dsub_rn(x0, ts.c0[0]), d1 = __dsub_rn(x1, ts.c1[0]);
        const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)));
        if (!(d <= __dadd_rn(ts.r[0], extra))) return -1;
        if (e && d > 0.0) {
            e[0] = __ddiv_rn(-d0, d);
            e[1] = __ddiv_rn(-d1, d);
        }
        double th = atan2(d1, d0);
        if (th < 0.0) th = __dadd_rn(th, 2.0 * pi);
        int j = (int)floor(__dadd_rn(__ddiv_rn(__dmul_rn((double)R, th), 2.0 * pi), 1e-9));
        if (j >= R) j -= R;
        if (j < 0) j = 0;
        *gap = d > ts.r[0] ? __dsub_rn(d, ts.r[0]) : 0.0;
        return j;
    }
    const double d = fabs(__dsub_rn(x0, ts.c0[0]));
    if (!(d <= __dadd_rn(ts.r[0], extra))) return -1;
    if (e && d > 0.0) e[0] = x0 < ts.c0[0] ? 1.0 : -1.0;
    const double hi1 = __dadd_rn(g.lo1, __dmul_rn((double)(g.n1 - 1), g.k));
    int j = (int)floor(__dadd_rn(__ddiv_rn(__dmul_rn((double)R, __dsub_rn(x1, g.lo1)), __dsub_rn(hi1, g.lo1)), 1e-9));
    if (j >= R) j = R - 1;
    if (j < 0) j = 0;
    *gap = d > ts.r[0] ? __dsub_rn(d, ts.r[0]) : 0.0;
    return j;
}

// Device-side state of one tile-sweep phase (active list, parities, ...).
// Grid coordinates of node i of a row-major grid (n0 nodes per row, n1 rows
// per plane).  Node counts below 2^31 (every grid in practice) use 32-bit
// integer division, which runs on the integer and FP32 units; a 64-bit
// division is a long instruction sequence on the narrow FP64 pipe of GB300.
__device__ __forceinline__ void node_xy(int64_t i, int n0, int &x, int &y) {
    if (i <= 0x7fffffffll) {
        const unsigned j = (unsigned)i, q = j / (unsigned)n0;
        y = (int)q;
        x = (int)(j - q * (unsigned)n0);
    } else {
        const int64_t q = i / n0;
        y = (int)q;
        x = (int)(i - q * n0);
    }
}
__device__ __forceinline__ void node_xyz(int64_t i, int n0, int n1, int &x, int &y, int &z) {
    int r;
    if (i <= 0x7fffffffll) {
        const unsigned j = (unsigned)i, q = j / (unsigned)n0;
        x = (int)(j - q * (unsigned)n0);
        r = (int)q;
    } else {
        const int64_t q = i / n0;
        x = (int)(i - q * n0);
        r = (int)q;   // rows fit in 32 bits: n1 n2 < 2^31
    }
    const unsigned q2 = (unsigned)r / (unsigned)n1;
    z = (int)q2;
    y = (int)((unsigned)r - q2 * (unsigned)n1);
}

struct TileSched {
    int *list[2];         // active tile lists (double-buffered by launch parity)
    int *count;           // count[2]
    double *chg[2];       // per-tile max change of the last launch (FP64, double-buffered)
    uint8_t *latest;      // which value buffer holds each tile's current values
    uint8_t *processed;   // tile ran in the current launch
    uint64_t *tile_patch; // patch bitmask of each tile (for per-patch sweep counts)
    uint64_t *patch_hist; // per-launch mask of patches with an active tile
    double *res_hist;     // per-launch max change (FP64)
    int *count_hist;      // per-launch number of active tiles
    const uint8_t *dirs;  // per-tile Gauss-Seidel directions (bit d: run direction d); NULL: all
    int alt;              // 3D without dirs: launches alternate the increasing and the
                          // decreasing pass of each axis (half the passes per launch)
    double *last_chg;     // per-tile change of the last launch the tile ran in (NULL: not kept)
};

__device__ __forceinline__ int tile_of(const Grid2 &g, int x, int y) {
    if (x < 1 || y < 1 || x > g.n0 - 2 || y > g.n1 - 2) return -1;
    return ((y - 1) / kTile) * g.ntx + (x - 1) / kTile;
}

__device__ __forceinline__ float atomic_max_pos(float *addr, float v) {
    // non-negative floats order like their bit patterns
    return __int_as_float(atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v)));
}

__device__ __forceinline__ double atomic_max_pos(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    return __longlong_as_double(
        (long long)atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v)));
}

// |v - o| of two values in FP64 for the sup-norm stopping test: 0 when both
// are the +inf sentinel, a huge value when only one is.  (The tile sweeps use
// node_change below; this form serves the queue sweep and the coarse grid.)
template <typename T> __device__ __forceinline__ double change64(T v, T o, T thresh) {
    const bool vi = v >= thresh, oi = o >= thresh;
    return (vi && oi) ? 0.0 : ((vi || oi) ? 1e300 : fabs((double)v - (double)o));
}

// Per-node change of a tile sweep for the sup-norm stopping test.  FP32
// values: their difference rounded upward, an upper bound of the exact
// difference (which FP64 would hold) by at most one unit in the last place,
// formed without the FP64 pipe (a GB300 SM retires two FP64 operations per
// clock); the tile's maximum of these bounds is then widened to FP64 and the
// reduction over tiles and the comparison with tol run in FP64.  FP64
// values: the FP64 difference.  Both: 0 when v and o are the +inf sentinel, a
// huge value when only one is; with the plain update (clamp = 0) a move of a
// few units in the last place counts as no change.
__device__ __forceinline__ float node_change(float v, float o, int clamp) {
    const float th = Num<float>::thresh();
    const bool vi = v >= th, oi = o >= th;
    float d = (vi && oi) ? 0.f : ((vi || oi) ? 3.0e38f : __fsub_ru(fmaxf(v, o), fminf(v, o)));
    if (!clamp && d <= (float)Num<float>::noise() * fabsf(v)) d = 0.f;
    return d;
}

__device__ __forceinline__ double node_change(double v, double o, int clamp) {
    double d = change64(v, o, Num<double>::thresh());
    if (!clamp && d <= Num<double>::noise() * fabs(v)) d = 0.0;
    return d;
}

}  // namespace hjbp
