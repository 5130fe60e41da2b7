// kernels2d.cu -- CUDA kernels of the 2D path (sm_103a).
//
// Every hot step runs here: set-up of the node codes and time steps,
// the almost-sure reachability sweep (S*), the semi-Lagrangian value sweep of
// Eq. (SLscheme) (FP32 bulk / FP64), the colour transport of Eq.
// (HJBridotta_discreta) (FP64), the coarse feedback of Eq. (feedbackcontrol)
// (FP64), labels, patch compaction and the FP64 polishing pass.
//
// Tiled sweeps: the interior nodes 1..n-2 are cut into 32x32 tiles, one warp
// per tile.  A tile loads itself plus a one-node halo into shared memory
// (the foot x_i + k a of every control lies in the 3x3 neighbourhood, Sec.
// 2.1: |h f| = k), runs line Gauss-Seidel passes in the four axis directions
// (in each step the 32 lanes update one column or one row), and writes the
// tile back.  Across tiles the iteration is block-Jacobi: each launch reads the
// values of the previous launch (two value buffers, a per-tile parity bit says
// which one is current), so results do not depend on the order in which tiles
// run.  Only tiles whose 3x3 tile neighbourhood changed by more than the
// tolerance in the previous launch run again; the solve stops when none is
// left, which is the sup-norm test of Sec. 2.2 (Step 4) on launches.
#include <cmath>
#include <cstdint>

#include "hjbp_device.cuh"
#include "plan.h"

#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

namespace hjbp {

// ------------------------------------------------------------------ set-up --

// Node codes, h_i = k / c(x_i) (|h f| = k, Sec. 2.1) and the fixed values of
// target nodes; nodes in an obstacle (Sec. 4) are hard like the ghost ring.  Target part j: |x - c_j| <= r_j + extra (lowest j).  With
// boundary_values, a target node outside its ball gets the time
// (|x - c_j| - r_j) / c(x) to reach it (the coarse grid, Step 1); otherwise 0.
// Coordinates and distances use explicitly rounded operations so that target
// membership is decided exactly as x = lo + i k, r^2 = sum (x - c)^2 dictate.
__global__ void k_setup2d(Grid2 g, SpeedParams sp, TargetSet ts, double extra, int boundary_values,
                          int8_t *__restrict__ code, float *__restrict__ h32, double *__restrict__ h64,
                          double *__restrict__ fixed, DynParams dp, ObstacleSet os, SpeedLines sl) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy;
        node_xy(i, g.n0, ix, iy);
        const double x0 = __dadd_rn(g.lo0, __dmul_rn((double)ix, g.k));
        const double x1 = __dadd_rn(g.lo1, __dmul_rn((double)iy, g.k));
        double gap = 0.0, e[2];
        const int part = target_part2(ts, g, x0, x1, extra, &gap, e);
        const bool ring = ix == 0 || iy == 0 || ix == g.n0 - 1 || iy == g.n1 - 1;
        const double c = sl.f[0] ? speed_lines(sp, sl, ix, iy, 0) : speed_at(sp, x0, x1, 0.0);
        const bool stopped = !(c > kStoppedSpeed);   // cannot move: like the ghost ring
        const bool blocked = part < 0 && in_obstacle(os, x0, x1, 0.0);
        const double hh = stopped ? (double)INFINITY : __ddiv_rn(g.k, c);
        code[i] = part >= 0 ? (int8_t)(kTargetBase + part) : ((ring || stopped || blocked) ? kHard : (int8_t)0);
        if (h32) h32[i] = (float)hh;
        if (h64) h64[i] = hh;
        // coarse boundary value (R6): the gap over the speed towards the target
        if (fixed)
            fixed[i] = (part >= 0 && boundary_values && gap > 0.0) ? __ddiv_rn(gap, approach_speed2(dp, c, e[0], e[1]))
                                                                  : 0.0;
    }
}

// Start values of a value solve (R14): M on free nodes (or, with a warm
// start, the given value where it is finite: add-on AO1 of Sec. 6), the fixed
// value on targets, +inf on hard nodes; written to both buffers.
template <typename T>
__global__ void k_init_values2d(int64_t N, const int8_t *__restrict__ code, const double *__restrict__ fixed,
                                T start, T *__restrict__ b0, T *__restrict__ b1, const double *__restrict__ warm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        T v;
        if (c < 0) v = Num<T>::big();
        else if (c >= kTargetBase) v = fixed ? (T)fixed[i] : (T)0;
        else v = (warm && warm[i] < kU0Bound) ? (T)warm[i] : start;
        b0[i] = v;
        b1[i] = v;
    }
}

// ------------------------------------------------------------ scheduling --

// After each tile launch: flip the parity of the tiles that ran, activate every
// tile whose 3x3 tile neighbourhood changed by more than tol, record the max
// change and the patches that are still active, clear the other change buffer.
__global__ void k_schedule2d(Grid2 g, TileSched s, int par, double tol, int launch) {
    const int ntiles = g.ntx * g.nty;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    if (t == 0 && s.count_hist) s.count_hist[launch] = s.count[par];
    const bool ran = s.processed[t] != 0;
    if (ran) {
        s.latest[t] ^= 1;
        s.processed[t] = 0;
    }
    const int tx = t % g.ntx, ty = t / g.ntx;
    bool act = false;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int ux = tx + dx, uy = ty + dy;
            if (ux < 0 || uy < 0 || ux >= g.ntx || uy >= g.nty) continue;
            if ((par ? s.chg[1] : s.chg[0])[uy * g.ntx + ux] > tol) act = true;
        }
    if (act) {
        const int k = atomicAdd(&s.count[par ^ 1], 1);
        (par ? s.list[0] : s.list[1])[k] = t;
    }
    const double my = (par ? s.chg[1] : s.chg[0])[t];
    if (my > tol && s.tile_patch && s.patch_hist)
        atomicOr(reinterpret_cast<unsigned long long *>(&s.patch_hist[launch]),
                 (unsigned long long)s.tile_patch[t]);
    if (my > 0.0 && s.res_hist) atomic_max_pos(&s.res_hist[launch], my);
    if (ran && s.last_chg) s.last_chg[t] = my;
    (par ? s.chg[0] : s.chg[1])[t] = 0.0;
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Tile image for the value sweep: values and codes with the halo, plus h and
// a 9-bit usability mask per interior node (bit 3 dy + dx set when the
// neighbour (dx-1, dy-1) belongs to the node's patch or its target part;
// bit 15 set when the node itself is free).  Codes do not change during a
// solve, so the masks are formed once per launch.
template <typename T, bool kDir> struct TileSmemV {
    T u[kTile + 2][kTile + 3];
    int8_t c[kTile + 2][kTile + 4];
    T h[kTile][kTile + 1];
    uint16_t mk[kTile][kTile + 2];
    T d[kDir ? kTile + 2 : 1][kDir ? kTile + 3 : 1];  // Dirichlet data of the halo image (Eq. dbc)
};

// Self-solved SL update (R13) of node (c, r) of the tile:
//   min over controls of kap (w10 u10 + w01 u01 + w11 u11 + h_i),
// the neighbourhood masked by the node's precomputed usability mask: a
// neighbour outside the mask reads +inf (state constraints) or, with kDir,
// its fixed Dirichlet value (Eq. dbc).  Returns the +inf sentinel when no
// control has all its positive-weight corners finite.  Four independent
// minimum accumulators keep the FMA chains of different controls in flight
// together; NCLS > 0 fully unrolls the symmetric form for a table with
// exactly NCLS classes (every class then sits in the constant bank as
// immediates).
// kMasked = false: the tile's image holds no node of another patch and no
// other target part (every non-usable neighbour is then a node with a
// negative code, whose value is the +inf sentinel), so the mask can be
// skipped with the same result.
template <typename T, int NCLS, bool kDir, class S, bool kMasked = true>
__device__ __forceinline__ T sl_update_m(const S &sm, int c, int r, unsigned m, T hh, const CtlTable2<T> &ct) {
    T nb[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            if constexpr (!kMasked && !kDir)
                nb[dy][dx] = sm.u[r - 1 + dy][c - 1 + dx];
            else if constexpr (kDir)
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : sm.d[r - 1 + dy][c - 1 + dx];
            else
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : Num<T>::big();
        }
    T b0 = Num<T>::big(), b1 = Num<T>::big(), b2 = Num<T>::big(), b3 = Num<T>::big();
    if (NCLS > 0 || ct.d4) {
        T E[4], G[4], A[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
            const T a10 = nb[1][sx], a01 = nb[sy][1];
            E[q] = a10 + a01;
            G[q] = fabs(a10 - a01);
            A[q] = nb[sy][sx];
        }
        const int ncls = NCLS > 0 ? NCLS : ct.ncls;
#pragma unroll
        for (int k = 0; k < (NCLS > 0 ? NCLS : 1); ++k) {
            if (NCLS == 0) break;
            const T kh = ct.cls_kap[k] * hh;
            const T s = ct.cls_s[k], t = -ct.cls_t[k], w = ct.cls_kw11[k];
            const T v0 = fma(t, G[0], fma(s, E[0], fma(w, A[0], kh)));
            const T v1 = fma(t, G[1], fma(s, E[1], fma(w, A[1], kh)));
            const T v2 = fma(t, G[2], fma(s, E[2], fma(w, A[2], kh)));
            const T v3 = fma(t, G[3], fma(s, E[3], fma(w, A[3], kh)));
            b0 = v0 < b0 ? v0 : b0;
            b1 = v1 < b1 ? v1 : b1;
            b2 = v2 < b2 ? v2 : b2;
            b3 = v3 < b3 ? v3 : b3;
        }
        if (NCLS == 0) {
            for (int k = 0; k < ncls; ++k) {
                const T kh = ct.cls_kap[k] * hh;
                const T s = ct.cls_s[k], t = -ct.cls_t[k], w = ct.cls_kw11[k];
                const T v0 = fma(t, G[0], fma(s, E[0], fma(w, A[0], kh)));
                const T v1 = fma(t, G[1], fma(s, E[1], fma(w, A[1], kh)));
                const T v2 = fma(t, G[2], fma(s, E[2], fma(w, A[2], kh)));
                const T v3 = fma(t, G[3], fma(s, E[3], fma(w, A[3], kh)));
                b0 = v0 < b0 ? v0 : b0;
                b1 = v1 < b1 ? v1 : b1;
                b2 = v2 < b2 ? v2 : b2;
                b3 = v3 < b3 ? v3 : b3;
            }
        }
        if (ct.axis) {
            const T ax = fmin(fmin(nb[1][0], nb[1][2]), fmin(nb[0][1], nb[2][1])) + hh;
            b0 = ax < b0 ? ax : b0;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
            const T a10 = nb[1][sx], a01 = nb[sy][1], a11 = nb[sy][sx];
            int mm = ct.qbeg[q];
            const int me = ct.qbeg[q + 1];
            for (; mm + 3 < me; mm += 4) {
                const T v0 = fma(ct.kw11[mm], a11, fma(ct.kw01[mm], a01, fma(ct.kw10[mm], a10, ct.kap[mm] * hh)));
                const T v1 = fma(ct.kw11[mm + 1], a11,
                                 fma(ct.kw01[mm + 1], a01, fma(ct.kw10[mm + 1], a10, ct.kap[mm + 1] * hh)));
                const T v2 = fma(ct.kw11[mm + 2], a11,
                                 fma(ct.kw01[mm + 2], a01, fma(ct.kw10[mm + 2], a10, ct.kap[mm + 2] * hh)));
                const T v3 = fma(ct.kw11[mm + 3], a11,
                                 fma(ct.kw01[mm + 3], a01, fma(ct.kw10[mm + 3], a10, ct.kap[mm + 3] * hh)));
                b0 = v0 < b0 ? v0 : b0;
                b1 = v1 < b1 ? v1 : b1;
                b2 = v2 < b2 ? v2 : b2;
                b3 = v3 < b3 ? v3 : b3;
            }
            for (; mm < me; ++mm) {
                const T v = fma(ct.kw11[mm], a11, fma(ct.kw01[mm], a01, fma(ct.kw10[mm], a10, ct.kap[mm] * hh)));
                b0 = v < b0 ? v : b0;
            }
        }
    }
    const T b01 = b0 < b1 ? b0 : b1, b23 = b2 < b3 ? b2 : b3;
    return b01 < b23 ? b01 : b23;
}

// Packed FP32 pairs (two lanes of one 64-bit register, PTX .f32x2, sm_100
// and later): one instruction forms the same rounded FP32 operation on both
// halves, so pairing two quadrants halves the FMA count of the symmetric
// pair form with the same result to the last bit.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long f2_abs(unsigned long long a) { return a & 0x7FFFFFFF7FFFFFFFull; }

// sl_update_m for FP32 values and a compile-time NCLS-class symmetric table
// with the two quadrants of each row of the neighbourhood (sy = -1 and
// sy = +1) packed into one pair: per class one packed multiply, three packed
// FMAs for both rows instead of eight scalar FMAs and two multiplies.
template <int NCLS, bool kMasked, class S>
__device__ __forceinline__ float sl_update_x2(const S &sm, int c, int r, unsigned m, float hh,
                                              const CtlTable2<float> &ct) {
    float nb[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            if constexpr (kMasked)
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : Num<float>::big();
            else
                nb[dy][dx] = sm.u[r - 1 + dy][c - 1 + dx];
        }
    // row pair R (sy = -1: R = 0, +1: R = 1): halves = the quadrants sx = -1, +1
    unsigned long long E[2], G[2], A[2];
#pragma unroll
    for (int R = 0; R < 2; ++R) {
        const int sy = R ? 2 : 0;
        const unsigned long long a10 = f2_pack(nb[1][0], nb[1][2]);
        const unsigned long long a01 = f2_pack(nb[sy][1], nb[sy][1]);
        E[R] = f2_add(a10, a01);
        G[R] = f2_abs(f2_sub(a10, a01));
        A[R] = f2_pack(nb[sy][0], nb[sy][2]);
    }
    const unsigned long long hh2 = f2_pack(hh, hh);
    float b0 = Num<float>::big(), b1 = Num<float>::big(), b2 = Num<float>::big(), b3 = Num<float>::big();
#pragma unroll
    for (int k = 0; k < NCLS; ++k) {
        const unsigned long long kh = f2_mul(f2_pack(ct.cls_kap[k], ct.cls_kap[k]), hh2);
        const unsigned long long s2 = f2_pack(ct.cls_s[k], ct.cls_s[k]);
        const unsigned long long t2 = f2_pack(-ct.cls_t[k], -ct.cls_t[k]);
        const unsigned long long w2 = f2_pack(ct.cls_kw11[k], ct.cls_kw11[k]);
        const unsigned long long v0 = f2_fma(t2, G[0], f2_fma(s2, E[0], f2_fma(w2, A[0], kh)));
        const unsigned long long v1 = f2_fma(t2, G[1], f2_fma(s2, E[1], f2_fma(w2, A[1], kh)));
        float x0, x1, x2, x3;
        f2_unpack(v0, x0, x1);
        f2_unpack(v1, x2, x3);
        b0 = x0 < b0 ? x0 : b0;
        b1 = x1 < b1 ? x1 : b1;
        b2 = x2 < b2 ? x2 : b2;
        b3 = x3 < b3 ? x3 : b3;
    }
    if (ct.axis) {
        const float ax = fminf(fminf(nb[1][0], nb[1][2]), fminf(nb[0][1], nb[2][1])) + hh;
        b0 = ax < b0 ? ax : b0;
    }
    const float b01 = b0 < b1 ? b0 : b1, b23 = b2 < b3 ? b2 : b3;
    return b01 < b23 ? b01 : b23;
}

// The update over a per-node subset of the controls (AO3 cones).  mine: the
// node's mask over table positions; uni: the union of the masks of the warp's
// lanes (warp-uniform, so every lane walks the same positions); tab: kap-scaled
// weights per position.
template <typename T> struct Ctl4 {
    T kw10, kw01, kw11, kap;
};
// Quadrant ranges of the table, copied by value (taking the address of a
// kernel parameter would move the whole table to local memory).
struct QBeg {
    int v[5];
};

template <typename T, bool kDir, class S>
__device__ __forceinline__ T sl_update_cone(const S &sm, int c, int r, unsigned m, T hh, unsigned long long mine,
                                            unsigned long long uni, const QBeg qbeg, const Ctl4<T> *tab) {
    T nb[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            if constexpr (kDir)
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : sm.d[r - 1 + dy][c - 1 + dx];
            else
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : Num<T>::big();
        }
    T best = Num<T>::big();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
        const T a10 = nb[1][sx], a01 = nb[sy][1], a11 = nb[sy][sx];
        const int lo = qbeg.v[q], hi = qbeg.v[q + 1];
        const unsigned long long below_hi = hi >= 64 ? ~0ull : ((1ull << hi) - 1ull);
        unsigned long long uq = uni & below_hi & ~((1ull << lo) - 1ull);
        while (uq) {
            const int pos = __ffsll((long long)uq) - 1;
            uq &= uq - 1ull;
            const Ctl4<T> w = tab[pos];
            const T v = fma(w.kw11, a11, fma(w.kw01, a01, fma(w.kw10, a10, w.kap * hh)));
            if ((mine >> pos) & 1ull) best = v < best ? v : best;
        }
    }
    return best;
}

// AO3 in the symmetric pair form: class k of quadrant q holds the control
// a = (sx X, sy Y), X >= Y, and its mirror a' = (sx Y, sy X); with
// E = u10 + u01, D = u10 - u01 their values are base + t D and base - t D
// (base = kap h + kap w11 u11 + s E), so one pair costs the same three FMAs
// whichever members the node's cone keeps (both: base - t |D|).  Quadrants
// no lane of the warp uses (quni) are skipped warp-uniformly.
template <typename T, int NCLS, bool kDir, class S>
__device__ __forceinline__ T sl_update_pcone(const S &sm, int c, int r, unsigned m, T hh, const CtlTable2<T> &ct,
                                             unsigned long long pm, unsigned am, unsigned quni) {
    T nb[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            if constexpr (kDir)
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : sm.d[r - 1 + dy][c - 1 + dx];
            else
                nb[dy][dx] = ((m >> (3 * dy + dx)) & 1u) ? sm.u[r - 1 + dy][c - 1 + dx] : Num<T>::big();
        }
    T b[4] = {Num<T>::big(), Num<T>::big(), Num<T>::big(), Num<T>::big()};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!((quni >> q) & 1u)) continue;
        const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
        const T a10 = nb[1][sx], a01 = nb[sy][1], A = nb[sy][sx];
        const T E = a10 + a01, D = a10 - a01, G = fabs(D);
        const unsigned bits = (unsigned)(pm >> (16 * q));
#pragma unroll
        for (int k = 0; k < NCLS; ++k) {
            const unsigned cb = (bits >> (2 * k)) & 3u;
            const T base = fma(ct.cls_kw11[k], A, fma(ct.cls_s[k], E, ct.cls_kap[k] * hh));
            const T x = cb == 3u ? -G : (cb == 1u ? D : -D);
            const T v = cb ? fma(ct.cls_t[k], x, base) : Num<T>::big();
            b[q] = v < b[q] ? v : b[q];
        }
    }
    if (am) {
        // axis controls land on the neighbour: kap = 1
        if (am & 1u) b[0] = fmin(b[0], nb[1][2] + hh);
        if (am & 2u) b[1] = fmin(b[1], nb[1][0] + hh);
        if (am & 4u) b[2] = fmin(b[2], nb[2][1] + hh);
        if (am & 8u) b[3] = fmin(b[3], nb[0][1] + hh);
    }
    const T b01 = b[0] < b[1] ? b[0] : b[1], b23 = b[2] < b[3] ? b[2] : b[3];
    return b01 < b23 ? b01 : b23;
}

// Minimum of the self-solved update (R13) over the controls of quadrant q
// (corners a10 = (sx, 0), a01 = (0, sy), a11 = (sx, sy) relative to the node),
// in the symmetric pair form when the table has it.  Same operations as
// sl_update_m, so the result is the same to the last bit.
template <typename T, int NCLS>
__device__ __forceinline__ T quad_min(const CtlTable2<T> &ct, int q, T a10, T a01, T a11, T hh) {
    T b0 = Num<T>::big(), b1 = Num<T>::big();
    if (NCLS > 0 || ct.d4) {
        const T E = a10 + a01, G = fabs(a10 - a01);
        if constexpr (NCLS > 0) {
#pragma unroll
            for (int k = 0; k < NCLS; ++k) {
                const T kh = ct.cls_kap[k] * hh;
                const T v = fma(-ct.cls_t[k], G, fma(ct.cls_s[k], E, fma(ct.cls_kw11[k], a11, kh)));
                if (k & 1) b1 = v < b1 ? v : b1;
                else b0 = v < b0 ? v : b0;
            }
        } else {
            for (int k = 0; k < ct.ncls; ++k) {
                const T kh = ct.cls_kap[k] * hh;
                const T v = fma(-ct.cls_t[k], G, fma(ct.cls_s[k], E, fma(ct.cls_kw11[k], a11, kh)));
                b0 = v < b0 ? v : b0;
            }
        }
    } else {
        int mm = ct.qbeg[q];
        const int me = ct.qbeg[q + 1];
        for (; mm + 1 < me; mm += 2) {
            const T v0 = fma(ct.kw11[mm], a11, fma(ct.kw01[mm], a01, fma(ct.kw10[mm], a10, ct.kap[mm] * hh)));
            const T v1 = fma(ct.kw11[mm + 1], a11,
                             fma(ct.kw01[mm + 1], a01, fma(ct.kw10[mm + 1], a10, ct.kap[mm + 1] * hh)));
            b0 = v0 < b0 ? v0 : b0;
            b1 = v1 < b1 ? v1 : b1;
        }
        if (mm < me) {
            const T v = fma(ct.kw11[mm], a11, fma(ct.kw01[mm], a01, fma(ct.kw10[mm], a10, ct.kap[mm] * hh)));
            b0 = v < b0 ? v : b0;
        }
    }
    return b0 < b1 ? b0 : b1;
}

// Neighbour (c + dx, r + dy) of a node through its usability mask m: the
// value v if usable, else +inf (state constraint) or the Dirichlet data.
template <typename T, bool kDir, class S>
__device__ __forceinline__ T masked(const S &sm, unsigned m, T v, int c, int r, int dx, int dy) {
    const unsigned bit = 3u * (unsigned)(dy + 1) + (unsigned)(dx + 1);
    if constexpr (kDir) return ((m >> bit) & 1u) ? v : sm.d[r + dy][c + dx];
    else return ((m >> bit) & 1u) ? v : Num<T>::big();
}

// Parities of the 3x3 tile neighbourhood of tile (tx, ty) as a 9-bit mask
// (bit 3 (dy+1) + (dx+1)); tiles off the grid read 0 like the ghost ring.
__device__ __forceinline__ unsigned nbr_parities(const Grid2 &g, const TileSched &s, int tx, int ty) {
    unsigned m = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int ux = tx + dx, uy = ty + dy;
            if (ux >= 0 && uy >= 0 && ux < g.ntx && uy < g.nty && s.latest[uy * g.ntx + ux])
                m |= 1u << (3 * (dy + 1) + (dx + 1));
        }
    return m;
}

// One launch of the value iteration over the active tiles.  clamp != 0: the
// monotone update u <- min(u, F(u)) from the start value M; clamp == 0: the
// plain update u <- F(u) (warm start, add-on AO1).  kDir: nodes outside the
// node's patch read the Dirichlet data dval (Eq. dbc) instead of +inf.  A
// node's own patch includes its target part and its own pruned nodes (code
// -2 - patch, value +inf).
// kCone: the minimum runs over each node's AO3 cone (astar, cone).
template <typename T, int NCLS, bool kDir, bool kCone = false, bool kX = false>
__global__ void __launch_bounds__(32) k_value2d(Grid2 g, const int8_t *__restrict__ code,
                                                const T *__restrict__ h, T *__restrict__ b0, T *__restrict__ b1,
                                                TileSched s, int par, int rounds, unsigned long long *updates,
                                                const CtlTable2<T> ct, int clamp, const T *__restrict__ dval,
                                                const uint8_t *__restrict__ astar = nullptr,
                                                const Cone2 *__restrict__ cone = nullptr, int packed = 0,
                                                int xpass = 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int x0 = 1 + tx * kTile, y0 = 1 + ty * kTile;
    __shared__ TileSmemV<T, kDir> sm;
    __shared__ T u0[kTile][kTile + 1];
    __shared__ uint8_t sa[kCone ? kTile : 1][kCone ? kTile + 1 : 1];
    __shared__ unsigned long long cmask[kCone ? 65 : 1];
    __shared__ Ctl4<T> ctab[kCone && NCLS == 0 ? 64 : 1];
    __shared__ uint8_t camask[kCone && NCLS > 0 ? 65 : 1];
    const int lane = threadIdx.x;
    const QBeg qb{{ct.qbeg[0], ct.qbeg[1], ct.qbeg[2], ct.qbeg[3], ct.qbeg[4]}};
    if constexpr (kCone && NCLS > 0) {
        // the pair form: per feedback the pair and axis masks
        for (int q = lane; q <= cone->nc; q += 32) {
            cmask[q] = cone->pmask[q];
            camask[q] = cone->amask[q];
        }
    } else if constexpr (kCone) {
        for (int q = lane; q <= cone->nc; q += 32) cmask[q] = cone->mask[q];
        for (int q = lane; q < ct.nc; q += 32) ctab[q] = Ctl4<T>{ct.kw10[q], ct.kw01[q], ct.kw11[q], ct.kap[q]};
    }
    // load: the parity of every halo node follows from its position in the
    // 3x3 tile neighbourhood, so all loads are independent; the 34 x 34 halo
    // image is spread over the lanes cell by cell and fully unrolled so that
    // every load is in flight at once, then h (and a*) of the interior
    const unsigned pm = nbr_parities(g, s, tx, ty);
    unsigned long long ids = 0;   // patches and target parts present in the tile's image
    {
        constexpr int kH = kTile + 2, kCells = kH * kH, kPer = (kCells + 31) / 32;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int q = lane + 32 * k;
            if (q < kCells) {
                const int r = q / kH, c = q - r * kH;
                const int x = x0 - 1 + c, y = y0 - 1 + r;
                T v = Num<T>::big(), dv = Num<T>::big();
                int8_t cd = kHard;
                if (x < g.n0 && y < g.n1) {
                    const int64_t i = (int64_t)y * g.n0 + x;
                    cd = code[i];
                    const int px = (c == 0) ? 0 : (c == kH - 1 ? 2 : 1);
                    const int py = (r == 0) ? 0 : (r == kH - 1 ? 2 : 1);
                    const bool inner = x >= 1 && x <= g.n0 - 2 && y >= 1 && y <= g.n1 - 2;
                    const bool odd = inner && ((pm >> (3 * py + px)) & 1u);
                    if constexpr (kX) {
                        // the newer of the two buffers (values only decrease): a
                        // neighbour's boundary may already hold this launch's rounds
                        const T v0 = __ldcg(b0 + i), v1 = __ldcg(b1 + i);
                        v = v0 < v1 ? v0 : v1;
                    } else {
                        v = odd ? b1[i] : b0[i];
                    }
                    if constexpr (kDir) dv = dval[i];
                }
                sm.u[r][c] = v;
                sm.c[r][c] = cd;
                if (cd >= 0) ids |= 1ull << (cd >= kTargetBase ? cd - kTargetBase : cd);
                if constexpr (kDir) sm.d[r][c] = dv;
            }
        }
        const int x = x0 + lane;
#pragma unroll
        for (int r = 0; r < kTile; ++r) {
            const int y = y0 + r;
            const bool in = x < g.n0 && y < g.n1;
            sm.h[r][lane] = in ? h[(int64_t)y * g.n0 + x] : (T)0;
            if constexpr (kCone) sa[r][lane] = in ? astar[(int64_t)y * g.n0 + x] : (uint8_t)kNoControl;
        }
    }
    __syncwarp();
    int nfree = 0;
    {
        const int c = 1 + lane;
        for (int r = 1; r <= kTile; ++r) {
            const int8_t cd = sm.c[r][c];
            unsigned m = 0;
            if (cd >= 0 && cd < kTargetBase) {
                const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int8_t q = sm.c[r - 1 + dy][c - 1 + dx];
                        m |= (unsigned)(q == cd || q == tg || q == pr) << (3 * dy + dx);
                    }
                m |= 0x8000u;
                ++nfree;
            }
            sm.mk[r - 1][lane] = (uint16_t)m;
            if constexpr (kCone) {
                const int a = m ? sa[r - 1][lane] : kNoControl;
                sa[r - 1][lane] = (uint8_t)(a < cone->nc ? a : cone->nc);
            }
            u0[r - 1][lane] = sm.u[r][c];
        }
    }
    __syncwarp();
    const unsigned long long all_ids = ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(ids >> 32)) << 32) |
                                       __reduce_or_sync(0xffffffffu, (unsigned)ids);
    const bool uniform = !kDir && !kCone && __popcll(all_ids) <= 1;
    // AO2: the tile's sweep directions; or alternating halves (TileSched.alt)
    const unsigned tdirs = s.dirs ? s.dirs[t] : (s.alt ? (par ? 0xAu : 0x5u) : 0xFu);
    auto exchange = [&]() {
        // Halo exchange inside the launch (monotone update only): publish this
        // tile's boundary lines into the buffer the launch writes, then read
        // the halo again as the newer of the two buffers.  A neighbour that
        // has published its round shows it here, one that has not shows its
        // older value; both are values that node held, so the iteration keeps
        // decreasing to the same fixed point (R8), and a change can cross a tile
        // boundary at every exchange instead of once per launch.
        T *dsx = ((pm >> 4) & 1u) ? b0 : b1;
        const int xl = x0 + lane, yl = y0 + lane;
        if (xl <= g.n0 - 2) {
            if (y0 <= g.n1 - 2) dsx[(int64_t)y0 * g.n0 + xl] = sm.u[1][1 + lane];
            const int yb = min(y0 + kTile - 1, g.n1 - 2);
            if (yb >= y0) dsx[(int64_t)yb * g.n0 + xl] = sm.u[1 + yb - y0][1 + lane];
        }
        if (yl <= g.n1 - 2) {
            if (x0 <= g.n0 - 2) dsx[(int64_t)yl * g.n0 + x0] = sm.u[1 + lane][1];
            const int xb = min(x0 + kTile - 1, g.n0 - 2);
            if (xb >= x0) dsx[(int64_t)yl * g.n0 + xb] = sm.u[1 + lane][1 + xb - x0];
        }
        // the 132 halo cells: rows 0 and 33 (34 each), columns 0 and 33 (32 each)
        constexpr int kH = kTile + 2;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int q = lane + 32 * k;
            if (q < 4 * kH - 4) {
                int r, c;
                if (q < kH) { r = 0; c = q; }
                else if (q < 2 * kH) { r = kH - 1; c = q - kH; }
                else if (q < 3 * kH - 2) { r = q - 2 * kH + 1; c = 0; }
                else { r = q - (3 * kH - 2) + 1; c = kH - 1; }
                const int x = x0 - 1 + c, y = y0 - 1 + r;
                if (x >= 1 && x <= g.n0 - 2 && y >= 1 && y <= g.n1 - 2) {
                    const int64_t i = (int64_t)y * g.n0 + x;
                    const T v0 = __ldcg(b0 + i), v1 = __ldcg(b1 + i);
                    const T v = v0 < v1 ? v0 : v1;
                    if (v < sm.u[r][c]) sm.u[r][c] = v;
                }
            }
        }
        __syncwarp();
    };
    const int npass = __popc(tdirs);
    int pass = 0;
    for (int rd = 0; rd < rounds; ++rd) {
        for (int dir = 0; dir < 4; ++dir) {
            if (!((tdirs >> dir) & 1u)) continue;
            if constexpr (kX) {
                // between rounds (xpass = 0) or between passes (xpass = 1)
                if (pass > 0 && (xpass || pass % npass == 0)) exchange();
            }
            ++pass;
            for (int st = 0; st < kTile; ++st) {
                const int s1 = 1 + ((dir & 1) ? (kTile - 1 - st) : st);
                const int c = (dir < 2) ? s1 : 1 + lane;
                const int r = (dir < 2) ? 1 + lane : s1;
                const unsigned m = sm.mk[r - 1][c - 1];
                const bool active = (m & 0x8000u) != 0;
                T nw = sm.u[r][c];
                if constexpr (kCone && NCLS > 0) {
                    const int ai = sa[r - 1][c - 1];
                    const unsigned long long pm = active ? cmask[ai] : 0ull;
                    const unsigned am = active ? camask[ai] : 0u;
                    unsigned qb = am ? 16u : 0u;
#pragma unroll
                    for (int q = 0; q < 4; ++q) qb |= ((pm >> (16 * q)) & 0xffffull) ? (1u << q) : 0u;
                    const unsigned quni = __reduce_or_sync(0xffffffffu, qb);
                    if (active) {
                        const T best = sl_update_pcone<T, NCLS, kDir>(sm, c, r, m, sm.h[r - 1][c - 1], ct, pm, am, quni);
                        if (best < Num<T>::thresh()) nw = clamp ? (best < nw ? best : nw) : best;
                    }
                } else if constexpr (kCone) {
                    const unsigned long long mine = active ? cmask[sa[r - 1][c - 1]] : 0ull;
                    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)mine);
                    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(mine >> 32));
                    const unsigned long long uni = ((unsigned long long)hi << 32) | lo;
                    if (active) {
                        const T best = sl_update_cone<T, kDir>(sm, c, r, m, sm.h[r - 1][c - 1], mine, uni, qb, ctab);
                        if (best < Num<T>::thresh()) nw = clamp ? (best < nw ? best : nw) : best;
                    }
                } else if (active) {
                    T best;
                    if constexpr (std::is_same<T, float>::value && NCLS > 0 && !kDir) {
                        if (packed)
                            best = uniform ? sl_update_x2<NCLS, false>(sm, c, r, m, sm.h[r - 1][c - 1], ct)
                                           : sl_update_x2<NCLS, true>(sm, c, r, m, sm.h[r - 1][c - 1], ct);
                        else
                            best = uniform ? sl_update_m<T, NCLS, kDir, decltype(sm), false>(sm, c, r, m, sm.h[r - 1][c - 1], ct)
                                           : sl_update_m<T, NCLS, kDir>(sm, c, r, m, sm.h[r - 1][c - 1], ct);
                    } else {
                        best = uniform ? sl_update_m<T, NCLS, kDir, decltype(sm), false>(sm, c, r, m, sm.h[r - 1][c - 1], ct)
                                       : sl_update_m<T, NCLS, kDir>(sm, c, r, m, sm.h[r - 1][c - 1], ct);
                    }
                    if (best < Num<T>::thresh()) nw = clamp ? (best < nw ? best : nw) : best;
                }
                __syncwarp();
                if (active) sm.u[r][c] = nw;
                __syncwarp();
            }
        }
    }
    // store into the buffer that is not current; change against the start values
    T *dst = ((pm >> 4) & 1u) ? b0 : b1;
    T mc = 0;
    const int x = x0 + lane;
    for (int r = 1; r <= kTile; ++r) {
        const int y = y0 - 1 + r;
        if (y > g.n1 - 2) break;
        if (x > g.n0 - 2) continue;
        const T v = sm.u[r][1 + lane];
        const T o = u0[r - 1][lane];
        dst[(int64_t)y * g.n0 + x] = v;
        const T d = node_change(v, o, clamp);
        mc = d > mc ? d : mc;
    }
    mc = warp_max(mc);
    const int nf = warp_sum(nfree);
    if (lane == 0) {
        (par ? s.chg[1] : s.chg[0])[t] = (double)mc;
        s.processed[t] = 1;
        // node updates: one per pass actually run (AO2 may skip passes)
        if (updates) atomicAdd(updates, (unsigned long long)nf * (unsigned long long)__popc(tdirs) * (unsigned long long)rounds);
    }
}

// ------------------------------------------------- persistent tile queue --
//
// The wave launches above advance the front by one tile per launch and every
// launch lasts as long as its slowest tile.  The persistent sweep instead keeps
// one warp per resident block popping tiles from a device work queue: a tile
// whose boundary nodes changed queues the neighbours that read them, a tile
// that has not settled inside queues itself again, and the solve ends when no
// tile is queued or running.  Values live in one buffer updated in place;
// the update is monotone (u <- min(u, F(u))), so reading a neighbour's old or
// new value is both safe, and the chaotic relaxation reaches the same fixed
// point as the ordered one (R8).  Every wait is bounded: when one runs out the
// kernel records an error and returns.

struct TileQueue {
    int *slot;                    // ring of cap entries, -1 when empty
    unsigned *head, *tail;        // pop / push counters
    int *state;                   // per tile: kQIdle, kQQueued, kQRunning, kQDirty
    int *pending;                 // tiles queued or running
    int *err;                     // nonzero: a wait ran out (which one)
    unsigned long long *visits;   // tiles processed
    int cap;
};

constexpr int kQIdle = 0, kQQueued = 1, kQRunning = 2, kQDirty = 3;
constexpr long kSpinLimit = 1l << 22;

__device__ __forceinline__ void q_enqueue(const TileQueue &q, int t) {
    const unsigned pos = atomicAdd(q.tail, 1u) % (unsigned)q.cap;
    volatile int *sl = q.slot + pos;
    // the ring holds twice the tile count, so the slot is free unless its
    // previous occupant's consumer has not read it yet
    for (long it = 0; *sl != -1; ++it) {
        if (it > kSpinLimit) {
            atomicExch(q.err, 1);
            return;
        }
        __nanosleep(64);
    }
    *sl = t;
    __threadfence();
}

// Queue tile t unless it is queued already; a running tile is marked to run
// again when it finishes.
__device__ __forceinline__ void q_push(const TileQueue &q, int t) {
    for (int it = 0; it < 1024; ++it) {
        const int st = atomicAdd(q.state + t, 0);
        if (st == kQIdle) {
            if (atomicCAS(q.state + t, kQIdle, kQQueued) == kQIdle) {
                atomicAdd(q.pending, 1);
                q_enqueue(q, t);
                return;
            }
        } else if (st == kQRunning) {
            if (atomicCAS(q.state + t, kQRunning, kQDirty) == kQRunning) return;
        } else {
            return;
        }
    }
    atomicExch(q.err, 2);
}

// Next tile to run; -1 when no tile is queued or running, -2 after an error.
__device__ __forceinline__ int q_pop(const TileQueue &q) {
    volatile unsigned *vh = q.head, *vt = q.tail;
    volatile int *vp = q.pending, *ve = q.err;
    unsigned nap = 32;   // idle back-off (ns), doubled up to 4 us: idle warps must not crowd the queue words
    for (long it = 0; it < kSpinLimit; ++it) {
        const unsigned h = *vh;
        if (h < *vt) {
            if (atomicCAS(q.head, h, h + 1u) == h) {
                volatile int *sl = q.slot + (h % (unsigned)q.cap);
                int t = *sl;
                for (long w = 0; t == -1; ++w) {
                    if (w > kSpinLimit) {
                        atomicExch(q.err, 3);
                        return -2;
                    }
                    __nanosleep(32);
                    t = *sl;
                }
                *sl = -1;
                atomicExch(q.state + t, kQRunning);
                __threadfence();
                return t;
            }
            continue;
        }
        if (*vp == 0) return -1;
        if (*ve) return -2;
        __nanosleep(nap);
        nap = nap < 4096u ? 2u * nap : 4096u;
    }
    atomicExch(q.err, 4);
    return -2;
}

__device__ __forceinline__ void q_finish(const TileQueue &q, int t) {
    if (atomicCAS(q.state + t, kQRunning, kQIdle) == kQRunning) {
        atomicSub(q.pending, 1);
    } else {
        // changed by a neighbour while it ran: run it again (still pending)
        atomicExch(q.state + t, kQQueued);
        q_enqueue(q, t);
    }
}

template <typename T, int NCLS, bool kDir>
__global__ void __launch_bounds__(32) k_value2d_async(Grid2 g, const int8_t *__restrict__ code,
                                                      const T *__restrict__ h, T *u, TileQueue q, int rounds,
                                                      double tol, unsigned long long *updates, const CtlTable2<T> ct,
                                                      const T *__restrict__ dval) {
    __shared__ TileSmemV<T, kDir> sm;
    __shared__ T u0[kTile][kTile + 1];
    const int lane = threadIdx.x;
    for (;;) {
        int t = 0;
        if (lane == 0) t = q_pop(q);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t < 0) break;
        const int tx = t % g.ntx, ty = t / g.ntx;
        const int x0 = 1 + tx * kTile, y0 = 1 + ty * kTile;
        {
            constexpr int kH = kTile + 2, kCells = kH * kH, kPer = (kCells + 31) / 32;
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int qq = lane + 32 * k;
                if (qq < kCells) {
                    const int r = qq / kH, c = qq - r * kH;
                    const int x = x0 - 1 + c, y = y0 - 1 + r;
                    T v = Num<T>::big(), dv = Num<T>::big();
                    int8_t cd = kHard;
                    if (x < g.n0 && y < g.n1) {
                        const int64_t i = (int64_t)y * g.n0 + x;
                        cd = code[i];
                        v = __ldcg(u + i);   // other blocks write u: read through L2
                        if constexpr (kDir) dv = dval[i];
                    }
                    sm.u[r][c] = v;
                    sm.c[r][c] = cd;
                    if constexpr (kDir) sm.d[r][c] = dv;
                }
            }
            const int x = x0 + lane;
#pragma unroll
            for (int r = 0; r < kTile; ++r) {
                const int y = y0 + r;
                sm.h[r][lane] = (x < g.n0 && y < g.n1) ? h[(int64_t)y * g.n0 + x] : (T)0;
            }
        }
        __syncwarp();
        int nfree = 0;
        {
            const int c = 1 + lane;
            for (int r = 1; r <= kTile; ++r) {
                const int8_t cd = sm.c[r][c];
                unsigned m = 0;
                if (cd >= 0 && cd < kTargetBase) {
                    const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const int8_t qc = sm.c[r - 1 + dy][c - 1 + dx];
                            m |= (unsigned)(qc == cd || qc == tg || qc == pr) << (3 * dy + dx);
                        }
                    m |= 0x8000u;
                    ++nfree;
                }
                sm.mk[r - 1][lane] = (uint16_t)m;
                u0[r - 1][lane] = sm.u[r][c];
            }
        }
        __syncwarp();
        double last = 0.0;  // largest change in the last round (FP64)
        for (int rd = 0; rd < rounds; ++rd) {
            for (int dir = 0; dir < 4; ++dir) {
                for (int st = 0; st < kTile; ++st) {
                    const int s1 = 1 + ((dir & 1) ? (kTile - 1 - st) : st);
                    const int c = (dir < 2) ? s1 : 1 + lane;
                    const int r = (dir < 2) ? 1 + lane : s1;
                    const unsigned m = sm.mk[r - 1][c - 1];
                    const bool active = (m & 0x8000u) != 0;
                    const T old = sm.u[r][c];
                    T nw = old;
                    if (active) {
                        const T best = sl_update_m<T, NCLS, kDir>(sm, c, r, m, sm.h[r - 1][c - 1], ct);
                        if (best < nw) nw = best;
                        if (rd == rounds - 1 && nw < old)
                            last = fmax(last, old >= Num<T>::thresh() ? 1e300 : (double)old - (double)nw);
                    }
                    __syncwarp();
                    if (active) sm.u[r][c] = nw;
                    __syncwarp();
                }
            }
        }
        // store in place; change per side decides which neighbours run again
        const int x = x0 + lane;
        double colmax = 0.0, row1 = 0.0, rowL = 0.0;
        const int rlast = min(kTile, g.n1 - 2 - y0 + 1);
        for (int r = 1; r <= kTile; ++r) {
            const int y = y0 - 1 + r;
            if (y > g.n1 - 2) break;
            if (x > g.n0 - 2) continue;
            const T v = sm.u[r][1 + lane];
            const T o = u0[r - 1][lane];
            if (v != o) __stcg(u + (int64_t)y * g.n0 + x, v);
            const double d = change64(v, o, Num<T>::thresh());
            colmax = fmax(colmax, d);
            if (r == 1) row1 = d;
            if (r == rlast) rowL = d;
        }
        __threadfence();
        const unsigned bS = __ballot_sync(0xffffffffu, row1 > tol), bN = __ballot_sync(0xffffffffu, rowL > tol);
        const unsigned bC = __ballot_sync(0xffffffffu, colmax > tol);
        last = warp_max(last);
        const int nf = warp_sum(nfree);
        if (lane == 0) {
            atomicAdd(q.visits, 1ull);
            if (updates) atomicAdd(updates, (unsigned long long)nf * 4ull * (unsigned long long)rounds);
            const bool w = tx > 0, e = tx < g.ntx - 1, sth = ty > 0, nth = ty < g.nty - 1;
            if (w && (bC & 1u)) q_push(q, t - 1);
            if (e && (bC >> 31)) q_push(q, t + 1);
            if (sth && bS) q_push(q, t - g.ntx);
            if (nth && bN) q_push(q, t + g.ntx);
            if (w && sth && (bS & 1u)) q_push(q, t - g.ntx - 1);
            if (e && sth && (bS >> 31)) q_push(q, t - g.ntx + 1);
            if (w && nth && (bN & 1u)) q_push(q, t + g.ntx - 1);
            if (e && nth && (bN >> 31)) q_push(q, t + g.ntx + 1);
            if (last > tol) q_push(q, t);
            q_finish(q, t);
        }
        __syncwarp();
    }
}

// Every tile queued once, in index order.
__global__ void k_queue_init(TileQueue q, int ntiles) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.cap; i += gridDim.x * blockDim.x) {
        q.slot[i] = i < ntiles ? i : -1;
        if (i < ntiles) q.state[i] = kQQueued;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *q.head = 0u;
        *q.tail = (unsigned)ntiles;
        *q.pending = ntiles;
        *q.err = 0;
        *q.visits = 0ull;
    }
}

// One Gauss-Seidel pass (direction DIR: 0/1 columns left to right / right to
// left with lane = row, 2/3 rows bottom to top / top to bottom with lane =
// column) of a tile shared by W warps.  Warp w takes a share of the quadrants
// of every node (W = 2: the two with sy = -1 or the two with sy = +1; W = 4:
// quadrant w) and one or two of the axis controls; the partial minima meet in
// shared memory behind one barrier per step, and every warp forms the node's
// new value from them.  The line updated one step earlier is kept in the
// lanes' registers (every warp holds the same values) and read by shuffles;
// lines at or ahead of the step still hold their values from before the pass
// and are read from shared memory; only warp 0 writes the new values back.
// Same operations and the same minimum as the one-warp step loop.
template <typename T, int NCLS, bool kDir, int W, int DIR, class S, class P>
__device__ __forceinline__ void sweep_mw(S &sm, P &part, const CtlTable2<T> &ct, int clamp, int lane, int w) {
    constexpr bool kCols = DIR < 2;
    constexpr int sd = (DIR & 1) ? -1 : 1;
    constexpr unsigned kFull = 0xffffffffu;
    const int a = 1 + lane;
    const int p0 = sd > 0 ? 0 : kTile + 1;
    T prev = kCols ? sm.u[a][p0] : sm.u[p0][a];
    for (int st = 0; st < kTile; ++st) {
        const int pp = sd > 0 ? 1 + st : kTile - st, pb = pp - sd;
        const int c = kCols ? pp : a, r = kCols ? a : pp;
        const unsigned m = sm.mk[r - 1][c - 1];
        const T old = sm.u[r][c];
        // the line behind at across -1, 0, +1 (halo past the ends)
        T bm = __shfl_up_sync(kFull, prev, 1), bp = __shfl_down_sync(kFull, prev, 1);
        if (lane == 0) bm = kCols ? sm.u[0][pb] : sm.u[pb][0];
        if (lane == kTile - 1) bp = kCols ? sm.u[kTile + 1][pb] : sm.u[pb][kTile + 1];
        // neighbour (c + dx, r + dy) as the step reads it
        auto nbv = [&](int dx, int dy) -> T {
            const int along = kCols ? dx : dy, across = kCols ? dy : dx;
            T v;
            if (along == -sd) v = across < 0 ? bm : (across > 0 ? bp : prev);
            else v = sm.u[r + dy][c + dx];
            return masked<T, kDir>(sm, m, v, c, r, dx, dy);
        };
        T f = Num<T>::big();
        if (m & 0x8000u) {
            const T hh = sm.h[r - 1][c - 1];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool mine = W == 4 ? (q == w) : ((q >> 1) == w);
                if (!mine) continue;
                const int sx = (q & 1) ? 1 : -1, sy = (q & 2) ? 1 : -1;
                const T v = quad_min<T, NCLS>(ct, q, nbv(sx, 0), nbv(0, sy), nbv(sx, sy), hh);
                f = v < f ? v : f;
            }
            if (ct.axis) {
                // axis controls land on one neighbour (kap = 1); W = 2: warp 0 the
                // left and lower ones, warp 1 the right and upper ones
                T ax;
                if (W == 4) ax = w == 0 ? nbv(-1, 0) : (w == 1 ? nbv(1, 0) : (w == 2 ? nbv(0, -1) : nbv(0, 1)));
                else ax = w == 0 ? fmin(nbv(-1, 0), nbv(0, -1)) : fmin(nbv(1, 0), nbv(0, 1));
                const T av = ax + hh;
                f = av < f ? av : f;
            }
        }
        part[st & 1][w][lane] = f;
        __syncthreads();
        T b = part[st & 1][0][lane];
#pragma unroll
        for (int v = 1; v < W; ++v) b = part[st & 1][v][lane] < b ? part[st & 1][v][lane] : b;
        T nw = old;
        if ((m & 0x8000u) && b < Num<T>::thresh()) nw = clamp ? (b < old ? b : old) : b;
        if (w == 0 && (m & 0x8000u)) sm.u[r][c] = nw;
        prev = nw;
    }
    __syncthreads();
}

// The value sweep with W warps per tile (2 or 4, see sweep_mw): prologue,
// passes and epilogue of k_value2d with the work of a step spread over the
// warps.  Not for AO3 cones.
template <typename T, int NCLS, bool kDir, int W>
__global__ void __launch_bounds__(32 * W) k_value2d_mw(Grid2 g, const int8_t *__restrict__ code,
                                                       const T *__restrict__ h, T *__restrict__ b0,
                                                       T *__restrict__ b1, TileSched s, int par, int rounds,
                                                       unsigned long long *updates, const CtlTable2<T> ct, int clamp,
                                                       const T *__restrict__ dval) {
    constexpr int NT = 32 * W;
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int x0 = 1 + tx * kTile, y0 = 1 + ty * kTile;
    __shared__ TileSmemV<T, kDir> sm;
    __shared__ T u0[kTile][kTile + 1];
    __shared__ T part[2][W][kTile];
    __shared__ double red[W];
    __shared__ int nfr[W];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned pm = nbr_parities(g, s, tx, ty);
    {
        constexpr int kH = kTile + 2, kCells = kH * kH, kPer = (kCells + NT - 1) / NT;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int q = tid + NT * k;
            if (q < kCells) {
                const int r = q / kH, c = q - r * kH;
                const int x = x0 - 1 + c, y = y0 - 1 + r;
                T v = Num<T>::big(), dv = Num<T>::big();
                int8_t cd = kHard;
                if (x < g.n0 && y < g.n1) {
                    const int64_t i = (int64_t)y * g.n0 + x;
                    cd = code[i];
                    const int px = (c == 0) ? 0 : (c == kH - 1 ? 2 : 1);
                    const int py = (r == 0) ? 0 : (r == kH - 1 ? 2 : 1);
                    const bool inner = x >= 1 && x <= g.n0 - 2 && y >= 1 && y <= g.n1 - 2;
                    const bool odd = inner && ((pm >> (3 * py + px)) & 1u);
                    v = odd ? b1[i] : b0[i];
                    if constexpr (kDir) dv = dval[i];
                }
                sm.u[r][c] = v;
                sm.c[r][c] = cd;
                if constexpr (kDir) sm.d[r][c] = dv;
            }
        }
        const int x = x0 + lane;
#pragma unroll
        for (int rr = 0; rr < kTile / W; ++rr) {
            const int r = w + W * rr, y = y0 + r;
            sm.h[r][lane] = (x < g.n0 && y < g.n1) ? h[(int64_t)y * g.n0 + x] : (T)0;
        }
    }
    __syncthreads();
    int nfree = 0;
    {
        const int c = 1 + lane;
        for (int rr = 0; rr < kTile / W; ++rr) {
            const int r = 1 + w + W * rr;
            const int8_t cd = sm.c[r][c];
            unsigned m = 0;
            if (cd >= 0 && cd < kTargetBase) {
                const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int8_t q = sm.c[r - 1 + dy][c - 1 + dx];
                        m |= (unsigned)(q == cd || q == tg || q == pr) << (3 * dy + dx);
                    }
                m |= 0x8000u;
                ++nfree;
            }
            sm.mk[r - 1][lane] = (uint16_t)m;
            u0[r - 1][lane] = sm.u[r][c];
        }
    }
    __syncthreads();
    const unsigned tdirs = s.dirs ? s.dirs[t] : (s.alt ? (par ? 0xAu : 0x5u) : 0xFu);
    for (int rd = 0; rd < rounds; ++rd) {
        if (tdirs & 1u) sweep_mw<T, NCLS, kDir, W, 0>(sm, part, ct, clamp, lane, w);
        if (tdirs & 2u) sweep_mw<T, NCLS, kDir, W, 1>(sm, part, ct, clamp, lane, w);
        if (tdirs & 4u) sweep_mw<T, NCLS, kDir, W, 2>(sm, part, ct, clamp, lane, w);
        if (tdirs & 8u) sweep_mw<T, NCLS, kDir, W, 3>(sm, part, ct, clamp, lane, w);
    }
    // store into the buffer that is not current; change against the start values
    T *dst = ((pm >> 4) & 1u) ? b0 : b1;
    T mc = 0;
    const int x = x0 + lane;
    for (int rr = 0; rr < kTile / W; ++rr) {
        const int r = 1 + w + W * rr, y = y0 - 1 + r;
        if (y > g.n1 - 2 || x > g.n0 - 2) continue;
        const T v = sm.u[r][1 + lane];
        const T o = u0[r - 1][lane];
        dst[(int64_t)y * g.n0 + x] = v;
        const T d = node_change(v, o, clamp);
        mc = d > mc ? d : mc;
    }
    mc = warp_max(mc);
    const int nf = warp_sum(nfree);
    if (lane == 0) {
        red[w] = (double)mc;
        nfr[w] = nf;
    }
    __syncthreads();
    if (tid == 0) {
        double mm = red[0];
        int nt = nfr[0];
#pragma unroll
        for (int v = 1; v < W; ++v) {
            mm = fmax(mm, red[v]);
            nt += nfr[v];
        }
        (par ? s.chg[1] : s.chg[0])[t] = mm;
        s.processed[t] = 1;
        if (updates)
            atomicAdd(updates, (unsigned long long)nt * (unsigned long long)__popc(tdirs) * (unsigned long long)rounds);
    }
}

// ----------------------------------------- small grids: one warp per node --

// One Jacobi launch of the value iteration for grids too small to fill the
// GPU with 32x32 tiles (the coarse grid of Step 1): one warp per free node,
// lanes take the controls m = lane, lane + 32, ..., and a warp-shuffle
// minimum combines them.  Reads uin, writes uout (monotone clamp from M),
// max |change| of the launch into res[launch].
template <typename T>
__global__ void k_value_wide2d(Grid2 g, const int8_t *__restrict__ code, const T *__restrict__ h,
                               const T *__restrict__ uin, T *__restrict__ uout, double *__restrict__ res, int launch,
                               const CtlSelf2<T> ct) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double mc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += warps) {
        const int8_t cd = code[i];
        const T old = uin[i];
        T nw = old;
        if (cd >= 0 && cd < kTargetBase) {
            int ix, iy;
            node_xy(i, g.n0, ix, iy);
            const int8_t tg = (int8_t)(cd + kTargetBase);
            T nb[3][3];
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int64_t j = (int64_t)(iy - 1 + dy) * g.n0 + (ix - 1 + dx);
                    const int8_t q = code[j];
                    nb[dy][dx] = (q == cd || q == tg) ? uin[j] : Num<T>::big();
                }
            const T hh = h[i];
            T best = Num<T>::big();
            for (int m = lane; m < ct.nc; m += 32) {
                const int sx = ct.sx[m] > 0 ? 2 : 0, sy = ct.sy[m] > 0 ? 2 : 0;
                const T a10 = sx ? nb[1][2] : nb[1][0];
                const T a01 = sy ? nb[2][1] : nb[0][1];
                const T a11 = sy ? (sx ? nb[2][2] : nb[2][0]) : (sx ? nb[0][2] : nb[0][0]);
                const T v = fma(ct.kw11[m], a11, fma(ct.kw01[m], a01, fma(ct.kw10[m], a10, ct.kap[m] * hh)));
                best = v < best ? v : best;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T other = __shfl_xor_sync(0xffffffffu, best, o);
                best = other < best ? other : best;
            }
            if (best < Num<T>::thresh()) nw = best < old ? best : old;
        }
        if (lane == 0) {
            uout[i] = nw;
            mc = fmax(mc, change64(nw, old, Num<T>::thresh()));
        }
    }
    mc = warp_max(mc);
    if (lane == 0 && mc > 0.0) atomic_max_pos(&res[launch], mc);
}

// -------------------------------------------- almost-sure reachability (S*) --

// Positive-probability reachability within the candidate set: a free node
// becomes reached when some control whose positive-weight corners (other than
// the node) are all usable puts positive weight on a reached node or on a
// terminal node (R14).  Terminal: the node's own target part, and with
// Dirichlet data (dterm != NULL, Eq. dbc) every node outside the patch whose
// data is finite.  With AO3 cones (cone != NULL) a node uses only the controls
// of its cone.  In place; monotone, so the order does not matter.
// cache, cvalid (optional): the tile's row sets below depend on the codes
// only, which do not change during one reach run, so the first launch that
// visits a tile stores them (11 x 32 words per tile) and later ones load them.
__global__ void __launch_bounds__(32) k_reach2d(Grid2 g, const int8_t *__restrict__ code,
                                                uint8_t *__restrict__ rch, TileSched s, int par,
                                                ReachTable2 rt, int passes, const double *__restrict__ dterm,
                                                const uint8_t *__restrict__ astar, const Cone2 *__restrict__ cone,
                                                uint64_t *__restrict__ cache, uint8_t *__restrict__ cvalid) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int x0 = 1 + (t % g.ntx) * kTile, y0 = 1 + (t / g.ntx) * kTile;
    __shared__ uint8_t sr[kTile + 2][kTile + 4];
    __shared__ int8_t sc[kTile + 2][kTile + 4];
    __shared__ uint8_t sd[kTile + 2][kTile + 4];
    const int lane = threadIdx.x;
    const bool cached = cache && cvalid[t];
    for (int r = 0; r < kTile + 2; ++r) {
        const int y = y0 - 1 + r;
        for (int c = lane; c < kTile + 2; c += 32) {
            const int x = x0 - 1 + c;
            uint8_t v = 0, df = 0;
            int8_t cd = kHard;
            if (x < g.n0 && y < g.n1) {
                const int64_t i = (int64_t)y * g.n0 + x;
                v = rch[i];
                if (!cached) {
                    cd = code[i];
                    if (dterm) df = dterm[i] < kU0Bound;
                }
            }
            sr[r][c] = v;
            sc[r][c] = cd;
            sd[r][c] = df;
        }
    }
    __syncwarp();
    // per interior node: bits 0..8 candidate corners in the patch (3 dy + dx),
    // bit 9 a candidate is terminal, bit 31 node free; pres: the corner
    // patterns of the node's controls per quadrant
    uint64_t cand_b[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, term_b = 0, open_b = 0;
    uint64_t *cl = cache ? cache + (int64_t)t * 11 * 32 : nullptr;
    if (cached) {
#pragma unroll
        for (int b = 0; b < 9; ++b) cand_b[b] = cl[b * 32 + lane];
        term_b = cl[9 * 32 + lane];
        open_b = cl[10 * 32 + lane];
    } else {
        const int c = 1 + lane;
        const uint32_t all = (uint32_t)rt.present[0] | ((uint32_t)rt.present[1] << 8) |
                             ((uint32_t)rt.present[2] << 16) | ((uint32_t)rt.present[3] << 24);
        for (int r = 1; r <= kTile; ++r) {
            const int8_t cd = sc[r][c];
            uint32_t pw = all;
            if (cone) {
                const int x = x0 + lane, y = y0 - 1 + r;
                const int a = (cd >= 0 && cd < kTargetBase && x < g.n0 && y < g.n1) ? astar[(int64_t)y * g.n0 + x]
                                                                                     : kNoControl;
                pw = cone->reach[a < cone->nc ? a : cone->nc];
            }
            uint32_t m = 0;
            if (cd >= 0 && cd < kTargetBase) {
                const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
                uint32_t same = 0, term = 0;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int8_t q = sc[r - 1 + dy][c - 1 + dx];
                        const bool t = q == tg || (q != cd && q != pr && sd[r - 1 + dy][c - 1 + dx]);
                        same |= (uint32_t)(q == cd) << (3 * dy + dx);
                        term |= (uint32_t)t << (3 * dy + dx);
                    }
                // the corners that can reach the node: per quadrant the union of
                // its patterns whose corners are all usable (a pattern with all
                // corners usable and one terminal-or-reached corner exists iff
                // such a corner lies in that union)
                const uint32_t usable = same | term;
                uint32_t cand = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int sx = (q & 1) ? 1 : -1, sy = (q & 2) ? 1 : -1;
                    const int b10 = 3 * 1 + (1 + sx), b01 = 3 * (1 + sy) + 1, b11 = 3 * (1 + sy) + (1 + sx);
                    const unsigned us =
                        ((usable >> b10) & 1u) | (((usable >> b01) & 1u) << 1) | (((usable >> b11) & 1u) << 2);
                    const unsigned pres = (pw >> (8 * q)) & 0xffu;
                    unsigned u = 0;
#pragma unroll
                    for (unsigned k = 1; k < 8; ++k)
                        if (((pres >> k) & 1u) && (k & ~us) == 0) u |= k;
                    cand |= ((u & 1u) << b10) | (((u >> 1) & 1u) << b01) | (((u >> 2) & 1u) << b11);
                }
                // bits 0..8: candidate corners in the patch; bit 9: a candidate is terminal
                m = (cand & same) | ((uint32_t)((cand & term) != 0) << 9) | 0x80000000u;
            }
            // row r as bit sets over the columns (bit c = column c, 0..33): the
            // nodes with candidate corner b, with a terminal candidate, still open
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const uint64_t row = (uint64_t)__ballot_sync(0xffffffffu, (m >> b) & 1u) << 1;
                if (lane == r - 1) cand_b[b] = row;
            }
            const uint64_t trow = (uint64_t)__ballot_sync(0xffffffffu, (m >> 9) & 1u) << 1;
            const uint64_t orow = (uint64_t)__ballot_sync(0xffffffffu, (m >> 31) & 1u) << 1;
            if (lane == r - 1) {
                term_b = trow;
                open_b = orow;
            }
        }
        if (cl) {
#pragma unroll
            for (int b = 0; b < 9; ++b) cl[b * 32 + lane] = cand_b[b];
            cl[9 * 32 + lane] = term_b;
            cl[10 * 32 + lane] = open_b;
            if (lane == 0) cvalid[t] = 1;   // read by later launches only
        }
    }
    // Reached nodes as one 34-bit row per lane (lane = row 1..32, the halo rows
    // 0 and 33 kept apart): a node is reached when a terminal or a reached node
    // is among its candidate corners.  Jacobi rounds over the bit sets reach the
    // tile's least fixed point for the launch's halo, the one the step-by-step
    // Gauss-Seidel passes approach; a round costs a few dozen instructions for
    // all 1024 nodes of the tile.
    auto row_bits = [&](int r) -> uint64_t {
        const uint64_t lo = __ballot_sync(0xffffffffu, sr[r][lane] != 0);
        return lo | ((uint64_t)(sr[r][32] != 0) << 32) | ((uint64_t)(sr[r][33] != 0) << 33);
    };
    uint64_t R = 0;
    for (int r = 1; r <= kTile; ++r) {
        const uint64_t v = row_bits(r);
        if (lane == r - 1) R = v;
    }
    const uint64_t H0 = row_bits(0), H1 = row_bits(kTile + 1);
    const uint64_t R0 = R;
    for (int it = 0; it <= kTile * kTile; ++it) {
        const uint64_t up = __shfl_up_sync(0xffffffffu, R, 1), dn = __shfl_down_sync(0xffffffffu, R, 1);
        const uint64_t rows[3] = {lane == 0 ? H0 : up, R, lane == kTile - 1 ? H1 : dn};
        uint64_t hit = term_b;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const uint64_t src = rows[b / 3];
            const int dx = b % 3;
            hit |= cand_b[b] & (dx == 0 ? src << 1 : (dx == 2 ? src >> 1 : src));
        }
        const uint64_t nr = R | (hit & open_b);
        const bool moved = nr != R;
        R = nr;
        if (!__any_sync(0xffffffffu, moved)) break;
    }
    const int flips = __popcll(R) - __popcll(R0);
    // back to bytes, row by row (coalesced stores)
    const int x = x0 + lane;
    for (int r = 1; r <= kTile; ++r) {
        const uint64_t row = __shfl_sync(0xffffffffu, R, r - 1);
        const int y = y0 - 1 + r;
        if (y > g.n1 - 2) break;
        if (x > g.n0 - 2) continue;
        rch[(int64_t)y * g.n0 + x] = (uint8_t)((row >> (lane + 1)) & 1ull);
    }
    const int nf = warp_sum(flips);
    if (lane == 0) {
        (par ? s.chg[1] : s.chg[0])[t] = nf > 0 ? 1.0 : 0.0;
        s.processed[t] = 1;
    }
}

// Peel for S* (R14): a free node none of whose controls (its cone under
// AO3) has all its positive-weight corners in the patch or terminal cannot
// be in S*; it is pruned (code -2 - patch).  Gauss-Seidel passes inside the
// tile, the schedule carries removals across tiles; codes only move from free
// to pruned, so a stale halo value only delays a removal.
__global__ void __launch_bounds__(32) k_peel2d(Grid2 g, int8_t *__restrict__ code, TileSched s, int par,
                                               ReachTable2 rt, const double *__restrict__ dterm,
                                               const uint8_t *__restrict__ astar, const Cone2 *__restrict__ cone) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int x0 = 1 + (t % g.ntx) * kTile, y0 = 1 + (t / g.ntx) * kTile;
    __shared__ int8_t sc[kTile + 2][kTile + 4];
    __shared__ uint8_t sd[kTile + 2][kTile + 4];
    __shared__ uint32_t pws[kTile][kTile + 1];   // per node: its patterns per quadrant
    const int lane = threadIdx.x;
    for (int r = 0; r < kTile + 2; ++r) {
        const int y = y0 - 1 + r;
        for (int c = lane; c < kTile + 2; c += 32) {
            const int x = x0 - 1 + c;
            uint8_t df = 0;
            int8_t cd = kHard;
            if (x < g.n0 && y < g.n1) {
                const int64_t i = (int64_t)y * g.n0 + x;
                cd = code[i];
                if (dterm) df = dterm[i] < kU0Bound;
            }
            sc[r][c] = cd;
            sd[r][c] = df;
        }
    }
    {
        const uint32_t all = (uint32_t)rt.present[0] | ((uint32_t)rt.present[1] << 8) |
                             ((uint32_t)rt.present[2] << 16) | ((uint32_t)rt.present[3] << 24);
        for (int r = 1; r <= kTile; ++r) {
            const int8_t cd = sc[r][1 + lane];
            uint32_t pw = all;
            if (cone) {
                const int x = x0 + lane, y = y0 - 1 + r;
                const int a = (cd >= 0 && cd < kTargetBase && x < g.n0 && y < g.n1) ? astar[(int64_t)y * g.n0 + x]
                                                                                     : kNoControl;
                pw = cone->reach[a < cone->nc ? a : cone->nc];
            }
            pws[r - 1][lane] = pw;
        }
    }
    __syncwarp();
    int flips = 0;
    for (int dir = 0; dir < 4; ++dir)
        for (int st = 0; st < kTile; ++st) {
            const int s1 = 1 + ((dir & 1) ? (kTile - 1 - st) : st);
            const int c = (dir < 2) ? s1 : 1 + lane;
            const int r = (dir < 2) ? 1 + lane : s1;
            const int8_t cd = sc[r][c];
            bool kill = false;
            if (cd >= 0 && cd < kTargetBase && x0 + c - 1 <= g.n0 - 2 && y0 + r - 1 <= g.n1 - 2) {
                const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
                uint32_t usable = 0;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int8_t q = sc[r - 1 + dy][c - 1 + dx];
                        const bool u = q == cd || q == tg || (q != cd && q != pr && sd[r - 1 + dy][c - 1 + dx]);
                        usable |= (uint32_t)u << (3 * dy + dx);
                    }
                const uint32_t pw = pws[r - 1][c - 1];
                bool any = false;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int sx = (q & 1) ? 1 : -1, sy = (q & 2) ? 1 : -1;
                    const int b10 = 3 * 1 + (1 + sx), b01 = 3 * (1 + sy) + 1, b11 = 3 * (1 + sy) + (1 + sx);
                    const unsigned us =
                        ((usable >> b10) & 1u) | (((usable >> b01) & 1u) << 1) | (((usable >> b11) & 1u) << 2);
                    const unsigned pres = (pw >> (8 * q)) & 0xffu;
#pragma unroll
                    for (unsigned k = 1; k < 8; ++k)
                        if (((pres >> k) & 1u) && (k & ~us) == 0) any = true;
                }
                kill = !any;
            }
            __syncwarp();
            if (kill) {
                sc[r][c] = (int8_t)(-2 - cd);
                ++flips;
            }
            __syncwarp();
        }
    const int x = x0 + lane;
    for (int r = 1; r <= kTile; ++r) {
        const int y = y0 - 1 + r;
        if (y > g.n1 - 2) break;
        if (x > g.n0 - 2) continue;
        code[(int64_t)y * g.n0 + x] = sc[r][1 + lane];
    }
    const int nf = warp_sum(flips);
    if (lane == 0) {
        (par ? s.chg[1] : s.chg[0])[t] = nf > 0 ? 1.0 : 0.0;
        s.processed[t] = 1;
    }
}

// Free nodes not reached leave the candidate set: their code becomes
// -2 - patch (not free, value +inf, still known to belong to the patch, which
// the Dirichlet boundary needs); counts them.
__global__ void k_reach_prune(int64_t N, int8_t *__restrict__ code, const uint8_t *__restrict__ rch,
                              unsigned long long *removed) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c >= 0 && c < kTargetBase && !rch[i]) {
            code[i] = (int8_t)(-2 - c);
            ++cnt;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(removed, cnt);
}

// ------------------------------------------------------------- gathering --

template <typename T>
__global__ void k_gather2d(Grid2 g, const uint8_t *__restrict__ latest, const T *__restrict__ b0,
                           const T *__restrict__ b1, T *__restrict__ out_t, double *__restrict__ out64) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y;
        node_xy(i, g.n0, x, y);
        const int tt = tile_of(g, x, y);
        const T v = (tt >= 0 && latest[tt]) ? b1[i] : b0[i];
        if (out_t) out_t[i] = v;
        if (out64) out64[i] = v >= Num<T>::thresh() ? (double)INFINITY : (double)v;
    }
}

// ---------------------------------------------------- Step 2: U_P^(0), a* --

// U_P^(0)(x_i) = Q1 of the coarse values at the fine node (R7: a coarse +inf
// enters as the bound M; >= M means unreachable); 0 on fine targets, +inf on
// the fine ghost ring.
// dlit (optional): the literal interpolation, +inf where a positive-weight
// coarse corner is +inf (the Dirichlet data of Eq. dbc, R16).
__global__ void k_u0_2d(Grid2 g, Grid2 gc, const int8_t *__restrict__ code, const double *__restrict__ uc,
                        double *__restrict__ u0, double *__restrict__ dlit) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c >= kTargetBase) {
            u0[i] = 0.0;
            if (dlit) dlit[i] = 0.0;
            continue;
        }
        if (c < 0) {
            u0[i] = Num<double>::big();
            if (dlit) dlit[i] = Num<double>::big();
            continue;
        }
        int ix, iy;
        node_xy(i, g.n0, ix, iy);
        const double xi0 = (double)ix * (double)(gc.n0 - 1) / (double)(g.n0 - 1);
        const double xi1 = (double)iy * (double)(gc.n1 - 1) / (double)(g.n1 - 1);
        int b0 = (int)floor(xi0), b1 = (int)floor(xi1);
        b0 = min(max(b0, 0), gc.n0 - 2);
        b1 = min(max(b1, 0), gc.n1 - 2);
        const double t0 = xi0 - b0, t1 = xi1 - b1;
        double sum = 0.0;
        bool inf_corner = false;
        for (int cc = 0; cc < 4; ++cc) {
            const double w = ((cc & 1) ? t0 : 1.0 - t0) * ((cc & 2) ? t1 : 1.0 - t1);
            if (w > 0.0) {
                const double v = uc[(int64_t)(b1 + ((cc >> 1) & 1)) * gc.n0 + b0 + (cc & 1)];
                inf_corner |= v >= Num<double>::thresh();
                sum += w * (v >= Num<double>::thresh() ? kU0Bound : v);
            }
        }
        if (dlit) dlit[i] = inf_corner ? Num<double>::big() : sum;
        u0[i] = sum >= kU0Bound ? Num<double>::big() : sum;
    }
}

// a*_k~(x_i) = argmin_a { I[U_P^(0)](x_i + k a) + h_i } (Eq. feedbackcontrol),
// literal Q1 with the node itself as a corner, controls in the caller's order,
// lowest index on ties (R10); 255 where every control meets +inf.
__global__ void k_feedback2d(Grid2 g, const int8_t *__restrict__ code, const double *__restrict__ h,
                             const double *__restrict__ u0, uint8_t *__restrict__ astar, const CtlLiteral2 cl) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c < 0 || c >= kTargetBase || u0[i] >= Num<double>::thresh()) {
            astar[i] = kNoControl;
            continue;
        }
        int ix, iy;
        node_xy(i, g.n0, ix, iy);
        double nb[3][3];
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx) {
                const int x = ix - 1 + dx, y = iy - 1 + dy;
                nb[dy][dx] = (x >= 0 && y >= 0 && x < g.n0 && y < g.n1) ? u0[(int64_t)y * g.n0 + x]
                                                                         : Num<double>::big();
            }
        const double hh = h[i];
        // Pass 1 in FP32 finds the minimum up to its rounding; pass 2 evaluates
        // in FP64, in index order, only the controls whose FP32 value is within
        // a bound of that error of the FP32 minimum, so the FP64 argmin (lowest
        // index on ties, R10) is the one a full FP64 pass would find.  Values
        // are at most 1e6 (R7) and the weights sum to 1, so each FP32 value
        // is within 8 units in the last place of (h + max |U|) of its FP64
        // value; the margin 2^-18 (h + max |U|) is twice that bound.
        float nf[3][3];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const bool fin = nb[dy][dx] < Num<double>::thresh();
                nf[dy][dx] = fin ? (float)nb[dy][dx] : Num<float>::big();
            }
        const float hf = (float)hh;
        // the bound per quadrant (half the margin above, over the quadrant's
        // own corners), so that the bound M of U0 near the ghost ring (R7)
        // widens only the quadrants that touch it
        float eq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
            const float c4[4] = {nf[1][1], nf[1][sx], nf[sy][1], nf[sy][sx]};
            float am = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (c4[b] < Num<float>::thresh()) am = fmaxf(am, fabsf(c4[b]));
            eq[q] = ldexpf(hf * cl.hfmax + am, -19);
        }
        // corner values by quadrant, selected without indexing (registers)
        auto corners32 = [&](int m, float &a10, float &a01, float &a11) {
            const bool px = cl.sx[m] > 0, py = cl.sy[m] > 0;
            a10 = px ? nf[1][2] : nf[1][0];
            a01 = py ? nf[2][1] : nf[0][1];
            a11 = px ? (py ? nf[2][2] : nf[0][2]) : (py ? nf[2][0] : nf[0][0]);
        };
        float b32 = Num<float>::big(), eb = 0.f;
        for (int m = 0; m < cl.nc; ++m) {
            float a10, a01, a11;
            corners32(m, a10, a01, a11);
            const float v = cl.f00[m] * nf[1][1] + cl.f10[m] * a10 + cl.f01[m] * a01 + cl.f11[m] * a11 + hf * cl.hff[m];
            if (v < b32) {
                b32 = v;
                eb = eq[(cl.sx[m] > 0 ? 1 : 0) + (cl.sy[m] > 0 ? 2 : 0)];
            }
        }
        double best = Num<double>::big();
        int arg = kNoControl;
        if (b32 < Num<float>::thresh()) {
            // a control can be the FP64 minimum (or tie with it) only if its FP32
            // value minus its bound is at most b32 plus the bound of b32's control
            const float base = b32 + eb;
            for (int m = 0; m < cl.nc; ++m) {
                float a10, a01, a11;
                corners32(m, a10, a01, a11);
                const float v32 =
                    cl.f00[m] * nf[1][1] + cl.f10[m] * a10 + cl.f01[m] * a01 + cl.f11[m] * a11 + hf * cl.hff[m];
                if (v32 > base + eq[(cl.sx[m] > 0 ? 1 : 0) + (cl.sy[m] > 0 ? 2 : 0)]) continue;
                const bool px = cl.sx[m] > 0, py = cl.sy[m] > 0;
                const double d10 = px ? nb[1][2] : nb[1][0];
                const double d01 = py ? nb[2][1] : nb[0][1];
                const double d11 = px ? (py ? nb[2][2] : nb[0][2]) : (py ? nb[2][0] : nb[0][0]);
                const double v =
                    cl.w00[m] * nb[1][1] + cl.w10[m] * d10 + cl.w01[m] * d01 + cl.w11[m] * d11 + hh * cl.hf[m];
                if (v < best) {
                    best = v;
                    arg = m;
                }
            }
        }
        astar[i] = best < Num<double>::thresh() ? (uint8_t)arg : kNoControl;
    }
}

// Causal sweep directions per tile (AO2 on the tiled iteration).  A node
// depends on its foot x_i + k a*, so information travels against a*: where
// (at least a fraction frac of) the tile's feedback has a*_x < 0 the x sweep
// runs in increasing x only (direction 0), where it has a*_x > 0 in
// decreasing x only (direction 1), otherwise both; the same for y
// (directions 2, 3).  Tiles without feedback run all four.
struct DirCtl {
    int8_t sx[kMaxControls], sy[kMaxControls];
};

__global__ void __launch_bounds__(32) k_tile_dirs2d(Grid2 g, const int8_t *__restrict__ code,
                                                    const uint8_t *__restrict__ astar, const DirCtl dc, float frac,
                                                    uint8_t *__restrict__ dirs) {
    const int t = blockIdx.x;
    const int x0 = 1 + (t % g.ntx) * kTile, y0 = 1 + (t / g.ntx) * kTile;
    const int lane = threadIdx.x, x = x0 + lane;
    int xp = 0, xm = 0, yp = 0, ym = 0;
    if (x <= g.n0 - 2)
        for (int r = 0; r < kTile; ++r) {
            const int y = y0 + r;
            if (y > g.n1 - 2) break;
            const int64_t i = (int64_t)y * g.n0 + x;
            const int8_t c = code[i];
            const uint8_t a = astar[i];
            if (c < 0 || c >= kTargetBase || a == kNoControl) continue;
            xp += dc.sx[a] > 0;
            xm += dc.sx[a] < 0;
            yp += dc.sy[a] > 0;
            ym += dc.sy[a] < 0;
        }
    xp = warp_sum(xp);
    xm = warp_sum(xm);
    yp = warp_sum(yp);
    ym = warp_sum(ym);
    if (lane == 0) {
        unsigned m = 0;
        const int tx = xp + xm, ty = yp + ym;
        if (tx == 0) m |= 0x3u;
        else if ((float)xm >= frac * (float)tx) m |= 0x1u;
        else if ((float)xp >= frac * (float)tx) m |= 0x2u;
        else m |= 0x3u;
        if (ty == 0) m |= 0xCu;
        else if ((float)ym >= frac * (float)ty) m |= 0x4u;
        else if ((float)yp >= frac * (float)ty) m |= 0x8u;
        else m |= 0xCu;
        dirs[t] = (uint8_t)m;
    }
}

// --------------------------------------------------- Step 3.1: colours phi --

// Controls in the caller's order for the colour transport: literal Q1
// weights (FP64 residual) and the self-solved weights kw = kap w in FP32.
struct PhiCtl {
    int nc;
    int8_t sx[kMaxControls], sy[kMaxControls];
    double w00[kMaxControls], w10[kMaxControls], w01[kMaxControls], w11[kMaxControls];
    float kw10[kMaxControls], kw01[kMaxControls], kw11[kMaxControls], kap[kMaxControls];
};

// Colour transport of Step 3.1 in mixed precision.  Eq. (HJBridotta_discreta)
// is linear, so FP64 accuracy comes from iterative refinement: an FP32 tile
// solve gives phi, its residual is formed in FP64, the correction equation
// (same transport operator, the residual as source) is solved in FP32, and the
// correction is added in FP64; two or three rounds reach the FP64 tolerance
// while the many sweeps all run in FP32.

// phi planes at set-up for colours j0 .. j0+RG-1 (colour-major, N each):
// 1 on target part j, 0 elsewhere (with zero_all: 0 everywhere).
template <int RG>
__global__ void k_phi_init2d(int64_t N, const int8_t *__restrict__ code, int j0, int zero_all,
                             float *__restrict__ b0, float *__restrict__ b1) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const float v = (!zero_all && c == (int8_t)(kTargetBase + j0 + q)) ? 1.0f : 0.0f;
            b0[(int64_t)q * N + i] = v;
            b1[(int64_t)q * N + i] = v;
        }
    }
}

template <int RG, bool kSource> struct PhiSmem {
    float u[RG][kTile + 2][kTile + 3];
    float src[kSource ? RG : 1][kSource ? kTile : 1][kTile + 1];
    int8_t c[kTile + 2][kTile + 4];
    uint8_t a[kTile][kTile + 4];
    // the control table, so that per-node lookups hit shared memory
    float kw10[kMaxControls], kw01[kMaxControls], kw11[kMaxControls], kap[kMaxControls];
    int8_t sx[kMaxControls], sy[kMaxControls];
};

// One FP32 launch over the active tiles for RG colours, each node solved for
// itself (R13) with its fixed coarse feedback a*_i:
//   bulk (kSource = false):       phi_i <- max(phi_i, kap (w10 phi10 + w01 phi01 + w11 phi11))
//   correction (kSource = true):  d_i   <- kap (w10 d10 + w01 d01 + w11 d11 + r_i)
// The bulk rises monotonically from 0; the tile's change is the max over
// its colours.
//
// kX (bulk only: its values only rise): after every pass a colour's warp
// publishes the tile's boundary lines of its colour into the buffer the launch
// writes and re-reads its halo as the larger of the two buffers, so a
// neighbour's progress inside the launch reaches the tile (same fixed point,
// R8).
// Warps per tile of the colour transport: one per colour.
template <int RG> constexpr int phi_warps() { return RG; }

template <int RG, bool kSource, bool kX = false>
__global__ void __launch_bounds__(32 * phi_warps<RG>(), RG == 8 ? 4 : (kX ? 7 : 8))
    k_phi2d(Grid2 g, const int8_t *__restrict__ code,
                                              const uint8_t *__restrict__ astar, float *__restrict__ b0,
                                              float *__restrict__ b1, const float *__restrict__ src, TileSched s,
                                              int par, int rounds, const PhiCtl *__restrict__ pc,
                                              unsigned long long *updates = nullptr) {
    // one warp per colour: the colours are independent linear systems, so the
    // warps never wait on one another inside a pass
    constexpr int W = phi_warps<RG>();
    constexpr int NT = 32 * W;
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int x0 = 1 + tx * kTile, y0 = 1 + ty * kTile;
    const int64_t N = (int64_t)g.n0 * g.n1;
    // dynamic shared memory: the image of 8 colours with its source exceeds
    // the 48 KB of static shared memory
    extern __shared__ __align__(16) unsigned char phi_smem_raw[];
    PhiSmem<RG, kSource> &sm = *reinterpret_cast<PhiSmem<RG, kSource> *>(phi_smem_raw);
    __shared__ unsigned alive_w[W];
    __shared__ float red_w[W];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int ncu = pc->nc;
    for (int m = tid; m < ncu; m += NT) {
        sm.kw10[m] = pc->kw10[m];
        sm.kw01[m] = pc->kw01[m];
        sm.kw11[m] = pc->kw11[m];
        sm.kap[m] = pc->kap[m];
        sm.sx[m] = pc->sx[m];
        sm.sy[m] = pc->sy[m];
    }
    const unsigned pm = nbr_parities(g, s, tx, ty);
    unsigned alive = 0;   // colours with a nonzero value (or source) in the tile or its halo
    {
        // halo image cell by cell over the threads, fully unrolled so that the
        // loads are all in flight together; then a* (and the source) of the interior
        constexpr int kH = kTile + 2, kCells = kH * kH, kPer = (kCells + NT - 1) / NT;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int q0 = tid + NT * k;
            if (q0 < kCells) {
                const int r = q0 / kH, c = q0 - r * kH;
                const int x = x0 - 1 + c, y = y0 - 1 + r;
                const bool in = x < g.n0 && y < g.n1;
                const int64_t i = (int64_t)y * g.n0 + x;
                int8_t cd = kHard;
                if (in) {
                    cd = code[i];
                    const int px = (c == 0) ? 0 : (c == kH - 1 ? 2 : 1);
                    const int py = (r == 0) ? 0 : (r == kH - 1 ? 2 : 1);
                    const bool odd = x >= 1 && x <= g.n0 - 2 && y >= 1 && y <= g.n1 - 2 &&
                                     ((pm >> (3 * py + px)) & 1u);
                    const float *bs = odd ? b1 : b0;
#pragma unroll
                    for (int q = 0; q < RG; ++q) {
                        float v;
                        if constexpr (kX) v = fmaxf(__ldcg(b0 + (int64_t)q * N + i), __ldcg(b1 + (int64_t)q * N + i));
                        else v = bs[(int64_t)q * N + i];
                        sm.u[q][r][c] = v;
                        alive |= (unsigned)(v != 0.0f) << q;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < RG; ++q) sm.u[q][r][c] = 0.0f;
                }
                sm.c[r][c] = cd;
            }
        }
        const int x = x0 + lane;
#pragma unroll
        for (int rr = 0; rr < kTile / W; ++rr) {
            const int r = w + W * rr;
            const int y = y0 + r;
            const bool in = x < g.n0 && y < g.n1;
            const int64_t i = (int64_t)y * g.n0 + x;
            sm.a[r][lane] = in ? astar[i] : kNoControl;
            if (kSource) {
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    const float v = in ? src[(int64_t)q * N + i] : 0.0f;
                    sm.src[q][r][lane] = v;
                    alive |= (unsigned)(v != 0.0f) << q;
                }
            }
        }
    }
    alive = __reduce_or_sync(0xffffffffu, alive);
    if (lane == 0) alive_w[w] = alive;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < W; ++v) alive |= alive_w[v];
    const unsigned tdirs = s.dirs ? s.dirs[t] : 0xFu;
    if (updates && alive && w == 0) {
        // node-colour updates of this launch: transported nodes x live colours x passes
        int na = 0;
        for (int r = 1; r <= kTile; ++r) {
            const int8_t cd = sm.c[r][1 + lane];
            na += (cd >= 0 && cd < kTargetBase && sm.a[r - 1][lane] != kNoControl) ? 1 : 0;
        }
        na = __reduce_add_sync(0xffffffffu, na);
        if (lane == 0 && na)
            atomicAdd(updates, (unsigned long long)na * (unsigned long long)__popc(alive) *
                                   (unsigned long long)__popc(tdirs) * (unsigned long long)rounds);
    }
    // the passes of this warp's colours, one colour after the other.  What a
    // step needs besides the colour values (the node's code, a*, its weights
    // and the source) does not change inside the launch, so it is read one
    // step ahead and only the corner values stay on the step's dependent path.
    struct Rec {
        float k10, k01, k11, kp, sv;
        int sx, sy;
        bool active;
    };
    for (int q = w; q < RG; q += W) {
        if (!((alive >> q) & 1u)) continue;
        float(*u)[kTile + 3] = sm.u[q];
        auto node_at = [&](int dir, int st, int &r, int &c) {
            const int s1 = 1 + ((dir & 1) ? (kTile - 1 - st) : st);
            c = (dir < 2) ? s1 : 1 + lane;
            r = (dir < 2) ? 1 + lane : s1;
        };
        auto record = [&](int r, int c) {
            Rec e;
            const int8_t cd = sm.c[r][c];
            const uint8_t a = sm.a[r - 1][c - 1];
            e.active = cd >= 0 && cd < kTargetBase && a != kNoControl;
            const int ai = e.active ? a : 0;
            e.sx = sm.sx[ai];
            e.sy = sm.sy[ai];
            e.k10 = sm.kw10[ai];
            e.k01 = sm.kw01[ai];
            e.k11 = sm.kw11[ai];
            e.kp = kSource ? sm.kap[ai] : 0.0f;
            e.sv = kSource ? sm.src[kSource ? q : 0][r - 1][c - 1] : 0.0f;
            return e;
        };
        int pass = 0;
        for (int rd = 0; rd < rounds; ++rd) {
            for (int dir = 0; dir < 4; ++dir) {
                if (!((tdirs >> dir) & 1u)) continue;
                if constexpr (kX && !kSource) {
                    if (pass > 0) {
                        float *dq = (((pm >> 4) & 1u) ? b0 : b1) + (int64_t)q * N;
                        const int xl = x0 + lane, yl = y0 + lane;
                        if (xl <= g.n0 - 2) {
                            if (y0 <= g.n1 - 2) dq[(int64_t)y0 * g.n0 + xl] = u[1][1 + lane];
                            const int yb = min(y0 + kTile - 1, g.n1 - 2);
                            if (yb >= y0) dq[(int64_t)yb * g.n0 + xl] = u[1 + yb - y0][1 + lane];
                        }
                        if (yl <= g.n1 - 2) {
                            if (x0 <= g.n0 - 2) dq[(int64_t)yl * g.n0 + x0] = u[1 + lane][1];
                            const int xb = min(x0 + kTile - 1, g.n0 - 2);
                            if (xb >= x0) dq[(int64_t)yl * g.n0 + xb] = u[1 + lane][1 + xb - x0];
                        }
                        constexpr int kH = kTile + 2;
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const int qq = lane + 32 * k;
                            if (qq < 4 * kH - 4) {
                                int hr, hc;
                                if (qq < kH) { hr = 0; hc = qq; }
                                else if (qq < 2 * kH) { hr = kH - 1; hc = qq - kH; }
                                else if (qq < 3 * kH - 2) { hr = qq - 2 * kH + 1; hc = 0; }
                                else { hr = qq - (3 * kH - 2) + 1; hc = kH - 1; }
                                const int x = x0 - 1 + hc, y = y0 - 1 + hr;
                                if (x >= 1 && x <= g.n0 - 2 && y >= 1 && y <= g.n1 - 2) {
                                    const int64_t i = (int64_t)q * N + (int64_t)y * g.n0 + x;
                                    const float v = fmaxf(__ldcg(b0 + i), __ldcg(b1 + i));
                                    if (v > u[hr][hc]) u[hr][hc] = v;
                                }
                            }
                        }
                        __syncwarp();
                    }
                }
                ++pass;
                int r, c;
                node_at(dir, 0, r, c);
                Rec e = record(r, c);
                for (int st = 0; st < kTile; ++st) {
                    int rn, cn;
                    node_at(dir, st + 1 < kTile ? st + 1 : st, rn, cn);
                    const Rec en = record(rn, cn);
                    float nw = 0.0f;
                    if (e.active) {
                        float v = e.k10 * u[r][c + e.sx];
                        v = fmaf(e.k01, u[r + e.sy][c], v);
                        v = fmaf(e.k11, u[r + e.sy][c + e.sx], v);
                        if (kSource) {
                            nw = fmaf(e.kp, e.sv, v);
                        } else {
                            const float o = u[r][c];
                            nw = v > o ? v : o;
                        }
                    }
                    __syncwarp();
                    if (e.active) u[r][c] = nw;
                    __syncwarp();
                    e = en;
                    r = rn;
                    c = cn;
                }
            }
        }
    }
    __syncthreads();
    const int cur = (pm >> 4) & 1u;
    float *dst = cur ? b0 : b1;
    const float *old = cur ? b1 : b0;
    float mc = 0.f;
    const int x = x0 + lane;
    // predicated and unrolled so that the reads of the previous values are
    // all in flight together; warp w stores rows w, w + W, ...
#pragma unroll
    for (int q = 0; q < RG; ++q) {
        const bool live = (alive >> q) & 1u;
#pragma unroll 8
        for (int rr = 0; rr < kTile / W; ++rr) {
            const int r = 1 + w + W * rr;
            const int y = y0 - 1 + r;
            if (y <= g.n1 - 2 && x <= g.n0 - 2) {
                const int64_t i = (int64_t)q * N + (int64_t)y * g.n0 + x;
                const float v = sm.u[q][r][1 + lane];
                dst[i] = v;
                if (live) mc = fmaxf(mc, fabsf(v - old[i]));
            }
        }
    }
    mc = warp_max(mc);
    if (lane == 0) red_w[w] = mc;
    __syncthreads();
    if (tid == 0) {
        float m = red_w[0];
#pragma unroll
        for (int v = 1; v < W; ++v) m = fmaxf(m, red_w[v]);
        (par ? s.chg[1] : s.chg[0])[t] = m;
        s.processed[t] = 1;
    }
}

// Current FP32 planes (per-tile parity) -> FP64 planes: out = in (add = 0) or
// out += in (add = 1).
template <int RG>
__global__ void k_phi_collect2d(Grid2 g, const uint8_t *__restrict__ latest, const float *__restrict__ b0,
                                const float *__restrict__ b1, double *__restrict__ out, int add) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y;
        node_xy(i, g.n0, x, y);
        const int tt = tile_of(g, x, y);
        const float *src = (tt >= 0 && latest[tt]) ? b1 : b0;
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const double v = (double)src[(int64_t)q * N + i];
            if (add) out[(int64_t)q * N + i] += v;
            else out[(int64_t)q * N + i] = v;
        }
    }
}

// FP64 residual of Eq. (HJBridotta_discreta) with the literal Q1 weights:
//   r_i = w00 phi_i + w10 phi10 + w01 phi01 + w11 phi11 - phi_i
// at free nodes with a defined feedback (0 elsewhere), stored in FP32 as the
// source of the correction solve; max |r| into *rmax.
template <int RG>
__global__ void k_phi_residual2d(Grid2 g, const int8_t *__restrict__ code, const uint8_t *__restrict__ astar,
                                 const double *__restrict__ phi, float *__restrict__ r32, float *rmax,
                                 const PhiCtl *__restrict__ pc) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    float mc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        const uint8_t a = astar[i];
        const bool active = c >= 0 && c < kTargetBase && a != kNoControl;
        if (!active) {
#pragma unroll
            for (int q = 0; q < RG; ++q) r32[(int64_t)q * N + i] = 0.0f;
            continue;
        }
        const int64_t dx = pc->sx[a], dy = (int64_t)pc->sy[a] * g.n0;
        const double w00 = pc->w00[a], w10 = pc->w10[a], w01 = pc->w01[a], w11 = pc->w11[a];
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const double *f = phi + (int64_t)q * N;
            const double p0 = f[i];
            const double v = w00 * p0 + w10 * f[i + dx] + w01 * f[i + dy] + w11 * f[i + dx + dy];
            const double r = v - p0;
            r32[(int64_t)q * N + i] = (float)r;
            mc = fmaxf(mc, (float)fabs(r));
        }
    }
    mc = warp_max(mc);
    if ((threadIdx.x & 31) == 0 && mc > 0.f) atomic_max_pos(rmax, mc);
}

// label = argmax_j phi^j if positive (lowest j on ties, R12); targets keep
// their part; -1 on hard / unreachable nodes; -2 marks uncovered nodes.
__global__ void k_label2d(int64_t N, const int8_t *__restrict__ code, const uint8_t *__restrict__ astar,
                          const double *__restrict__ phi, int R, int8_t *__restrict__ label) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c >= kTargetBase) { label[i] = (int8_t)(c - kTargetBase); continue; }
        if (c < 0 || astar[i] == kNoControl) { label[i] = -1; continue; }
        double mx = 0.0;
        int arg = -2;
        for (int j = 0; j < R; ++j) {
            const double v = phi[(int64_t)j * N + i];
            if (v > mx) { mx = v; arg = j; }
        }
        label[i] = (int8_t)arg;
    }
}

// One Jacobi round of the neighbour fill of Remark 3.1 (R12): an uncovered
// node takes the label of its first labelled axis neighbour in increasing
// node index (-y, -x, +x, +y).
__global__ void k_fill2d(Grid2 g, const int8_t *__restrict__ lin, int8_t *__restrict__ lout,
                         unsigned long long *changed) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int8_t v = lin[i];
        if (v == -2) {
            int ix, iy;
            node_xy(i, g.n0, ix, iy);
            int8_t nv = -2;
            if (iy > 0 && lin[i - g.n0] >= 0) nv = lin[i - g.n0];
            else if (ix > 0 && lin[i - 1] >= 0) nv = lin[i - 1];
            else if (ix < g.n0 - 1 && lin[i + 1] >= 0) nv = lin[i + 1];
            else if (iy < g.n1 - 1 && lin[i + g.n0] >= 0) nv = lin[i + g.n0];
            if (nv >= 0) { v = nv; ++cnt; }
        }
        lout[i] = v;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(changed, cnt);
}

// Codes of the per-patch solves: free node of patch j -> j, target part j ->
// 64 + j, everything else hard.  Leftover uncovered nodes (-2) become -1.
__global__ void k_patch_codes(int64_t N, const int8_t *__restrict__ code0, int8_t *__restrict__ label,
                              int8_t *__restrict__ code) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c0 = code0[i];
        int8_t l = label[i];
        if (l == -2) { l = -1; label[i] = -1; }
        if (c0 >= kTargetBase) code[i] = c0;
        else if (c0 < 0 || l < 0) code[i] = kHard;
        else code[i] = l;
    }
}

// ------------------------------------------------------ patch compaction --

// Per tile: bitmask of the patches with a free node in it and the node count
// of each (tile_cnt[t R + j], zero-filled beforehand); per patch: its node and
// tile counts.  (Step 3.1 assembles the patches; the tile masks let every
// sweep launch report which patches are still active, and compact.cu turns
// masks and counts into the per-patch lists.)
__global__ void __launch_bounds__(32) k_compact2d(Grid2 g, const int8_t *__restrict__ code,
                                                  uint64_t *__restrict__ tile_patch,
                                                  unsigned long long *__restrict__ patch_nodes,
                                                  unsigned long long *__restrict__ patch_tiles,
                                                  int *__restrict__ tile_cnt, int R) {
    const int t = blockIdx.x;
    const int x0 = 1 + (t % g.ntx) * kTile, y0 = 1 + (t / g.ntx) * kTile;
    const int lane = threadIdx.x;
    uint64_t mask = 0;
    const int x = x0 + lane;
    for (int r = 0; r < kTile; ++r) {
        const int y = y0 + r;
        if (y > g.n1 - 2) break;
        int8_t c = kHard;
        if (x <= g.n0 - 2) c = code[(int64_t)y * g.n0 + x];
        if (c >= 0 && c < kTargetBase) mask |= 1ull << c;
    }
    for (int o = 16; o > 0; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    // per-patch node counts: one ballot per patch present in the tile
    uint64_t m = mask;
    while (m) {
        const int j = __ffsll((long long)m) - 1;
        m &= m - 1;
        int cnt = 0;
        for (int r = 0; r < kTile; ++r) {
            const int y = y0 + r;
            if (y > g.n1 - 2) break;
            const bool is = x <= g.n0 - 2 && code[(int64_t)y * g.n0 + x] == (int8_t)j;
            cnt += __popc(__ballot_sync(0xffffffffu, is));
        }
        if (lane == 0) {
            atomicAdd(&patch_nodes[j], (unsigned long long)cnt);
            atomicAdd(&patch_tiles[j], 1ull);
            if (j < R) tile_cnt[(int64_t)t * R + j] = cnt;
        }
    }
    if (lane == 0) tile_patch[t] = mask;
}

// ------------------------------------------------- FP64 polishing pass (a8) --

// u_out = F(u_in) in FP64 at every free node (self-solved form, no clamp),
// one Jacobi application; max |change| into *maxchg.
//
// FP32 filter: every control is first evaluated in FP32.  With inputs,
// weights and four operations rounded to FP32, |v32 - v64| <= 8 u (kap h +
// max |a|), u = 2^-24, and kap h + max|a| <= 2 (h + max|a|) here; so a
// control whose FP32 value exceeds the FP32 minimum by more than
// margin = 2^-18 (h + max|a|) cannot attain the FP64 minimum.  Only the
// remaining candidates are evaluated in FP64: the result is the FP64 minimum
// over all controls at close to FP32 cost.
__global__ void k_polish2d(Grid2 g, const int8_t *__restrict__ code, const double *__restrict__ h,
                           const double *__restrict__ uin, double *__restrict__ uout, double *maxchg,
                           const CtlTable2<float> c32, const CtlTable2<double> c64,
                           const double *__restrict__ dval, const uint8_t *__restrict__ astar,
                           const Cone2 *__restrict__ cone) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    double mc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t cd = code[i];
        double v = uin[i];
        if (cd >= 0 && cd < kTargetBase) {
            int ix, iy;
            node_xy(i, g.n0, ix, iy);
            const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
            double nb[3][3];
            float nf[3][3];
            float amax = 0.f;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int64_t j = (int64_t)(iy - 1 + dy) * g.n0 + (ix - 1 + dx);
                    const int8_t q = code[j];
                    // outside the patch: +inf, or the Dirichlet data (Eq. dbc)
                    const bool same = q == cd || q == tg || q == pr;
                    const double w = same ? uin[j] : (dval ? dval[j] : Num<double>::big());
                    const bool fin = w < Num<double>::thresh();
                    nb[dy][dx] = fin ? w : Num<double>::big();
                    nf[dy][dx] = fin ? (float)w : Num<float>::big();
                    if (fin) amax = fmaxf(amax, fabsf((float)w));
                }
            const double hh = h[i];
            const float hf = (float)hh;
            // AO3: the node's cone over table positions (every control without)
            unsigned long long allow = ~0ull;
            if (cone) {
                const int a = astar[i];
                allow = cone->mask[a < cone->nc ? a : cone->nc];
            }
            // pass 1: FP32 minimum
            float b32 = Num<float>::big();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
                const float a10 = nf[1][sx], a01 = nf[sy][1], a11 = nf[sy][sx];
                for (int m = c32.qbeg[q]; m < c32.qbeg[q + 1]; ++m) {
                    if (cone && !((allow >> m) & 1ull)) continue;
                    const float w = fmaf(c32.kw11[m], a11, fmaf(c32.kw01[m], a01, fmaf(c32.kw10[m], a10, c32.kap[m] * hf)));
                    b32 = w < b32 ? w : b32;
                }
            }
            if (b32 < Num<float>::thresh() && v < Num<double>::thresh()) {
                const float lim = b32 + ldexpf(hf * c32.hfmax + amax, -18);
                // pass 2: FP64 over the candidates
                double best = Num<double>::big();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
                    const float a10 = nf[1][sx], a01 = nf[sy][1], a11 = nf[sy][sx];
                    const double d10 = nb[1][sx], d01 = nb[sy][1], d11 = nb[sy][sx];
                    for (int m = c32.qbeg[q]; m < c32.qbeg[q + 1]; ++m) {
                        if (cone && !((allow >> m) & 1ull)) continue;
                        const float w =
                            fmaf(c32.kw11[m], a11, fmaf(c32.kw01[m], a01, fmaf(c32.kw10[m], a10, c32.kap[m] * hf)));
                        if (w <= lim) {
                            const double x =
                                fma(c64.kw11[m], d11, fma(c64.kw01[m], d01, fma(c64.kw10[m], d10, c64.kap[m] * hh)));
                            best = x < best ? x : best;
                        }
                    }
                }
                mc = fmax(mc, fabs(best - v));
                v = best;
            }
        }
        uout[i] = v;
    }
    mc = warp_max(mc);
    if ((threadIdx.x & 31) == 0 && mc > 0.0) atomic_max_pos(maxchg, mc);
}

// FP64 polish in the symmetric pair form (control sets with the eight
// symmetries of the square, NCLS classes).  Same FP32-filter argument as
// k_polish2d: pass 1 takes the FP32 minimum over the pairs (base - t |D|,
// the smaller of the two mirrored controls), pass 2 evaluates in FP64 only
// the pairs whose FP32 value lies within lim = b32 + 2^-18 (h hfmax + max|u|)
// of it; the FP32 error of a pair value (about six roundings of terms
// bounded by kap h and max|u|, kap <= sqrt 2) stays below half that margin,
// so the pair holding the FP64 minimum is always evaluated.  The neighbours
// come from an FP32 mirror of the values (written by the same pass), so the
// filter converts nothing on the FP64 pipe; the FP64 corners are read only
// for candidate pairs.
template <int NCLS>
__global__ void k_polish2d_pf(Grid2 g, const int8_t *__restrict__ code, const double *__restrict__ h,
                              const double *__restrict__ uin, const float *__restrict__ uin32,
                              double *__restrict__ uout, float *__restrict__ uout32, double *maxchg,
                              const CtlTable2<float> c32, const CtlTable2<double> c64,
                              const double *__restrict__ dval, const float *__restrict__ dval32) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    double mc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t cd = code[i];
        double v = uin[i];
        if (cd >= 0 && cd < kTargetBase && v < Num<double>::thresh()) {
            int ix, iy;
            node_xy(i, g.n0, ix, iy);
            const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
            float nf[3][3];
            unsigned same = 0;
            float amax = 0.f;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int64_t j = (int64_t)(iy - 1 + dy) * g.n0 + (ix - 1 + dx);
                    const int8_t q = code[j];
                    const bool s = q == cd || q == tg || q == pr;
                    same |= (unsigned)s << (3 * dy + dx);
                    // outside the patch: +inf, or the Dirichlet data (Eq. dbc)
                    const float w = s ? uin32[j] : (dval32 ? dval32[j] : Num<float>::big());
                    const bool fin = w < Num<float>::thresh();
                    nf[dy][dx] = fin ? w : Num<float>::big();
                    if (fin) amax = fmaxf(amax, fabsf(w));
                }
            const double hh = h[i];
            const float hf = (float)hh;
            float E[4], G[4], A[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
                E[q] = nf[1][sx] + nf[sy][1];
                G[q] = fabsf(nf[1][sx] - nf[sy][1]);
                A[q] = nf[sy][sx];
            }
            // pass 1: FP32 minimum over the pairs (and the axis controls)
            float b32 = Num<float>::big();
#pragma unroll
            for (int k = 0; k < NCLS; ++k) {
                const float kh = c32.cls_kap[k] * hf;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float w = fmaf(-c32.cls_t[k], G[q], fmaf(c32.cls_s[k], E[q], fmaf(c32.cls_kw11[k], A[q], kh)));
                    b32 = w < b32 ? w : b32;
                }
            }
            const float ax32 = fminf(fminf(nf[1][0], nf[1][2]), fminf(nf[0][1], nf[2][1])) + hf;
            if (c32.axis) b32 = ax32 < b32 ? ax32 : b32;
            if (b32 < Num<float>::thresh()) {
                const float lim = b32 + ldexpf(hf * c32.hfmax + amax, -18);
                auto d64 = [&](int dx, int dy) -> double {
                    const int64_t j = (int64_t)(iy - 1 + dy) * g.n0 + (ix - 1 + dx);
                    const double w = ((same >> (3 * dy + dx)) & 1u) ? uin[j] : (dval ? dval[j] : Num<double>::big());
                    return w < Num<double>::thresh() ? w : Num<double>::big();
                };
                // pass 2: FP64 over the candidate pairs
                double best = Num<double>::big();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int sx = (q & 1) ? 2 : 0, sy = (q & 2) ? 2 : 0;
                    bool loaded = false;
                    double e64 = 0.0, g64 = 0.0, a64 = 0.0;
#pragma unroll
                    for (int k = 0; k < NCLS; ++k) {
                        const float w = fmaf(-c32.cls_t[k], G[q],
                                             fmaf(c32.cls_s[k], E[q], fmaf(c32.cls_kw11[k], A[q], c32.cls_kap[k] * hf)));
                        if (w <= lim) {
                            if (!loaded) {
                                const double d10 = d64(sx, 1), d01 = d64(1, sy);
                                e64 = d10 + d01;
                                g64 = fabs(d10 - d01);
                                a64 = d64(sx, sy);
                                loaded = true;
                            }
                            const double x =
                                fma(-c64.cls_t[k], g64, fma(c64.cls_s[k], e64, fma(c64.cls_kw11[k], a64, c64.cls_kap[k] * hh)));
                            best = x < best ? x : best;
                        }
                    }
                }
                if (c32.axis && ax32 <= lim) {
                    const double ax = fmin(fmin(d64(0, 1), d64(2, 1)), fmin(d64(1, 0), d64(1, 2))) + hh;
                    best = ax < best ? ax : best;
                }
                if (best < Num<double>::thresh()) {
                    mc = fmax(mc, fabs(best - v));
                    v = best;
                }
            }
        }
        uout[i] = v;
        uout32[i] = v < Num<double>::thresh() ? (float)v : Num<float>::big();
    }
    mc = warp_max(mc);
    if ((threadIdx.x & 31) == 0 && mc > 0.0) atomic_max_pos(maxchg, mc);
}

// A global solve has one target (the union of all parts): every target node
// gets code 64 + 0 so that free nodes (code 0) read all of them.
__global__ void k_merge_targets(int64_t N, int8_t *__restrict__ code) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (code[i] >= kTargetBase) code[i] = kTargetBase;
}

// Output labels of the global solve: 0 on S*, the part on target nodes, -1
// on the ghost ring and on free nodes outside S* (label may be null: the
// patchy solve keeps its Step 3.1 labels); counts free nodes outside S*.
__global__ void k_final_labels(int64_t N, const int8_t *__restrict__ code0, const int8_t *__restrict__ code,
                               int8_t *__restrict__ label, unsigned long long *unreachable) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        const int8_t c0 = code0[i];
        if (label) label[i] = c0 >= kTargetBase ? (int8_t)(c0 - kTargetBase) : (c >= 0 && c < kTargetBase ? c : (int8_t)-1);
        if (c0 >= 0 && c0 < kTargetBase && c < 0) ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(unreachable, cnt);
}

// FP32 bulk -> FP64 (and +inf sentinels)
__global__ void k_widen(int64_t N, const float *__restrict__ in, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = in[i];
        out[i] = v >= Num<float>::thresh() ? Num<double>::big() : (double)v;
    }
}

__global__ void k_finalize(int64_t N, const double *__restrict__ in, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[i];
        out[i] = v >= Num<double>::thresh() ? (double)INFINITY : v;
    }
}

// Dirichlet data of Eq. (dbc) in the sweep's precision: U_P^(0), with the
// bound 1e6 and above (no finite value) mapped to the +inf sentinel.
template <typename T>
__global__ void k_dirichlet_data(int64_t N, const double *__restrict__ u0, T *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = u0[i] < kU0Bound ? (T)u0[i] : Num<T>::big();
}

// ---------------------------------------------------------- instantiation --

template __global__ void k_init_values2d<float>(int64_t, const int8_t *, const double *, float, float *, float *,
                                                 const double *);
template __global__ void k_init_values2d<double>(int64_t, const int8_t *, const double *, double, double *, double *,
                                                  const double *);
template __global__ void k_value_wide2d<double>(Grid2, const int8_t *, const double *, const double *, double *,
                                                double *, int, const CtlSelf2<double>);
template __global__ void k_gather2d<float>(Grid2, const uint8_t *, const float *, const float *, float *, double *);
template __global__ void k_gather2d<double>(Grid2, const uint8_t *, const double *, const double *, double *,
                                            double *);

// Host launchers of the FP64 template kernels for other translation units
// (the no-allocation entry point launches the same kernels as hjbp_solve).
void launch_init_values2d_f64(int blocks, cudaStream_t st, int64_t N, const int8_t *code, double start, double *b0,
                              double *b1) {
    k_init_values2d<double><<<blocks, 256, 0, st>>>(N, code, nullptr, start, b0, b1, nullptr);
}

void launch_value2d_f64(int ntiles, cudaStream_t st, Grid2 g, const int8_t *code, const double *h, double *b0,
                        double *b1, TileSched s, int par, int rounds, const CtlTable2<double> &ct) {
    k_value2d<double, 0, false><<<ntiles, 32, 0, st>>>(g, code, h, b0, b1, s, par, rounds, nullptr, ct, 1, nullptr);
}

void launch_gather2d_f64(int blocks, cudaStream_t st, Grid2 g, const uint8_t *latest, const double *b0,
                         const double *b1, double *out64) {
    k_gather2d<double><<<blocks, 256, 0, st>>>(g, latest, b0, b1, nullptr, out64);
}

}  // namespace hjbp

// =====================================================================
// Host driver of the 2D path
// =====================================================================
namespace hjbp {
namespace {

// The reachability sweep is monotone and settles after at most one launch per
// node of the longest path; its cap is independent of max_sweeps.
constexpr int kReachCap = 1 << 18;

inline int grid_for(int64_t n, int bs = 256) {
    int64_t b = (n + bs - 1) / bs;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

template <typename T> T *alloc_n(hjbp_plan &p, int64_t n) {
    return static_cast<T *>(p.dev_alloc(sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
}

struct Sched {
    TileSched d{};
    int ntiles = 0;
    int hist = 0;
    int *count_hist = nullptr;
    int *iota = nullptr;
};

__global__ void k_iota(int n, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

Sched make_sched(hjbp_plan &p, const Grid2 &g, int hist) {
    Sched s;
    s.ntiles = g.ntx * g.nty;
    s.hist = hist;
    const int nt = std::max(1, s.ntiles);
    s.d.list[0] = alloc_n<int>(p, nt);
    s.d.list[1] = alloc_n<int>(p, nt);
    s.d.count = alloc_n<int>(p, 2);
    s.d.chg[0] = alloc_n<double>(p, nt);
    s.d.chg[1] = alloc_n<double>(p, nt);
    s.d.latest = alloc_n<uint8_t>(p, nt);
    s.d.processed = alloc_n<uint8_t>(p, nt);
    s.d.tile_patch = nullptr;
    s.d.patch_hist = alloc_n<uint64_t>(p, hist);
    s.d.res_hist = alloc_n<double>(p, hist);
    s.count_hist = alloc_n<int>(p, hist);
    s.d.count_hist = s.count_hist;
    s.iota = alloc_n<int>(p, nt);
    k_iota<<<grid_for(nt), 256, 0, p.stream>>>(nt, s.iota);
    ++p.stats.kernel_launches;
    return s;
}

void reset_sched(hjbp_plan &p, Sched &s) {
    cudaStream_t st = p.stream;
    const int nt = std::max(1, s.ntiles);
    check_cuda(cudaMemcpyAsync(s.d.list[0], s.iota, sizeof(int) * nt, cudaMemcpyDeviceToDevice, st), "reset list");
    const int counts[2] = {s.ntiles, 0};
    check_cuda(cudaMemcpyAsync(s.d.count, counts, sizeof(counts), cudaMemcpyHostToDevice, st), "reset count");
    check_cuda(cudaMemsetAsync(s.d.chg[0], 0, sizeof(double) * nt, st), "reset chg");
    check_cuda(cudaMemsetAsync(s.d.chg[1], 0, sizeof(double) * nt, st), "reset chg");
    check_cuda(cudaMemsetAsync(s.d.latest, 0, nt, st), "reset latest");
    check_cuda(cudaMemsetAsync(s.d.processed, 0, nt, st), "reset processed");
    check_cuda(cudaMemsetAsync(s.d.patch_hist, 0, sizeof(uint64_t) * s.hist, st), "reset hist");
    check_cuda(cudaMemsetAsync(s.d.res_hist, 0, sizeof(double) * s.hist, st), "reset hist");
    check_cuda(cudaMemsetAsync(s.count_hist, 0, sizeof(int) * s.hist, st), "reset hist");
    // the counts copied from a host stack array must land before it goes away
    check_cuda(cudaStreamSynchronize(st), "reset sync");
}

struct RunResult {
    int64_t tile_visits = 0; // active tiles summed over launches
    int launches = 0;        // launches that had work
    bool converged = false;
    double last_res = 0.0;
};

// Launch sweep+schedule pairs until no tile is active or the cap is hit.
template <class Sweep>
RunResult run_tiles(hjbp_plan &p, const Grid2 &g, Sched &s, double tol, int cap, Sweep sweep) {
    RunResult rr;
    if (s.ntiles == 0) {
        rr.converged = true;
        return rr;
    }
    reset_sched(p, s);
    cap = std::min(cap, s.hist);
    int par = 0, L = 0;
    // one pinned word per plan, kept for its lifetime (allocating and freeing
    // pinned memory per loop costs more than a short sweep)
    if (!p.pinned_count) check_cuda(cudaMallocHost(&p.pinned_count, sizeof(int)), "pinned");
    int *pinned = p.pinned_count;
    int check_every = 4;
    while (L < cap) {
        sweep(par, L);
        check_cuda(cudaGetLastError(), "sweep launch");
        k_schedule2d<<<(s.ntiles + 255) / 256, 256, 0, p.stream>>>(g, s.d, par, tol, L);
        ++p.stats.kernel_launches;
        check_cuda(cudaGetLastError(), "schedule launch");
        par ^= 1;
        ++L;
        if (L % check_every == 0 || L == cap) {
            check_cuda(cudaMemcpyAsync(pinned, s.d.count + par, sizeof(int), cudaMemcpyDeviceToHost, p.stream),
                       "count readback");
            check_cuda(cudaStreamSynchronize(p.stream), "sweep sync");
            if (*pinned == 0) {
                rr.converged = true;
                break;
            }
            check_every = std::min(check_every * 2, 16);
        }
    }
    std::vector<int> ch(L);
    std::vector<double> rh(L);
    if (L) {
        check_cuda(cudaMemcpyAsync(ch.data(), s.count_hist, sizeof(int) * L, cudaMemcpyDeviceToHost, p.stream), "hist");
        check_cuda(cudaMemcpyAsync(rh.data(), s.d.res_hist, sizeof(double) * L, cudaMemcpyDeviceToHost, p.stream),
                   "hist");
        check_cuda(cudaStreamSynchronize(p.stream), "hist sync");
    }
    for (int l = 0; l < L; ++l)
        if (ch[l] > 0) {
            rr.launches = l + 1;
            rr.last_res = rh[l];
            rr.tile_visits += ch[l];
        }
    return rr;
}

// Fill the symmetric form of the table when the control set is invariant
// under the eight symmetries of the square (see CtlTable2).
template <typename T> void build_d4(const hjbp_plan &p, CtlTable2<T> &ct) {
    ct.d4 = 0;
    const int nc = p.desc.n_controls;
    for (int m = 0; m < nc; ++m)
        if (p.hfac[m] != 1.0) return;   // the pair form shares kap h between mirrored controls
    const double tol = 1e-12;
    auto has = [&](double x, double y) {
        for (int m = 0; m < nc; ++m)
            if (std::fabs(p.dirs[2 * m] - x) < tol && std::fabs(p.dirs[2 * m + 1] - y) < tol) return true;
        return false;
    };
    for (int m = 0; m < nc; ++m) {
        const double x = p.dirs[2 * m], y = p.dirs[2 * m + 1];
        const double img[8][2] = {{x, y}, {-x, y}, {x, -y}, {-x, -y}, {y, x}, {-y, x}, {y, -x}, {-y, -x}};
        for (auto &v : img)
            if (!has(v[0], v[1])) return;
    }
    int axis = 0, ncls = 0, count = 0;
    for (int m = 0; m < nc; ++m) {
        const double x = p.dirs[2 * m], y = p.dirs[2 * m + 1];
        if (x > 0.0 && y == 0.0) {
            axis = 1;
            count += 4;
        } else if (x > 0.0 && y > 0.0 && x >= y - tol) {
            if (ncls >= kMaxControls / 4) return;
            const double w00 = (1.0 - x) * (1.0 - y), w10 = x * (1.0 - y), w01 = (1.0 - x) * y, w11 = x * y;
            const double kap = 1.0 / (1.0 - w00);
            const bool diag = std::fabs(x - y) < tol;
            ct.cls_kap[ncls] = (T)kap;
            ct.cls_kw11[ncls] = (T)(kap * w11);
            ct.cls_s[ncls] = (T)(kap * (w10 + w01) / 2.0);
            ct.cls_t[ncls] = diag ? (T)0 : (T)(kap * std::fabs(w10 - w01) / 2.0);
            ++ncls;
            count += diag ? 4 : 8;
        }
    }
    if (count != nc) return;
    ct.d4 = 1;
    ct.axis = axis;
    ct.ncls = ncls;
}

template <typename T> CtlTable2<T> make_table(const hjbp_plan &p) {
    CtlTable2<T> ct;
    std::memset(&ct, 0, sizeof(ct));
    const int nc = p.desc.n_controls;
    ct.nc = nc;
    std::vector<int> order[4];
    for (int m = 0; m < nc; ++m) {
        const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
        order[(ax >= 0.0 ? 1 : 0) + (ay >= 0.0 ? 2 : 0)].push_back(m);
    }
    int pos = 0;
    for (int q = 0; q < 4; ++q) {
        ct.qbeg[q] = pos;
        for (int m : order[q]) {
            const double ax = std::fabs(p.dirs[2 * m]), ay = std::fabs(p.dirs[2 * m + 1]);
            const double w00 = (1.0 - ax) * (1.0 - ay), w10 = ax * (1.0 - ay), w01 = (1.0 - ax) * ay, w11 = ax * ay;
            const double kap = 1.0 / (1.0 - w00);
            ct.kw10[pos] = (T)(kap * w10);
            ct.kw01[pos] = (T)(kap * w01);
            ct.kw11[pos] = (T)(kap * w11);
            ct.kap[pos] = (T)(kap * p.hfac[m]);   // kap h_{i,a} = kap hfac[a] h_i
            ++pos;
        }
    }
    ct.qbeg[4] = pos;
    ct.hfmax = 0.f;
    for (int m = 0; m < nc; ++m) ct.hfmax = std::max(ct.hfmax, (float)p.hfac[m]);
    build_d4(p, ct);
    return ct;
}

template <typename T> CtlSelf2<T> make_self(const hjbp_plan &p) {
    CtlSelf2<T> cs;
    std::memset(&cs, 0, sizeof(cs));
    cs.nc = p.desc.n_controls;
    for (int m = 0; m < cs.nc; ++m) {
        const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
        const double bx = std::fabs(ax), by = std::fabs(ay);
        const double kap = 1.0 / (1.0 - (1.0 - bx) * (1.0 - by));
        cs.sx[m] = ax >= 0.0 ? 1 : -1;
        cs.sy[m] = ay >= 0.0 ? 1 : -1;
        cs.kw10[m] = (T)(kap * bx * (1.0 - by));
        cs.kw01[m] = (T)(kap * (1.0 - bx) * by);
        cs.kw11[m] = (T)(kap * bx * by);
        cs.kap[m] = (T)(kap * p.hfac[m]);
    }
    return cs;
}

CtlLiteral2 make_literal(const hjbp_plan &p) {
    CtlLiteral2 cl;
    std::memset(&cl, 0, sizeof(cl));
    cl.nc = p.desc.n_controls;
    for (int m = 0; m < cl.nc; ++m) {
        const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
        const double bx = std::fabs(ax), by = std::fabs(ay);
        cl.sx[m] = ax >= 0.0 ? 1 : -1;
        cl.sy[m] = ay >= 0.0 ? 1 : -1;
        cl.w00[m] = (1.0 - bx) * (1.0 - by);
        cl.w10[m] = bx * (1.0 - by);
        cl.w01[m] = (1.0 - bx) * by;
        cl.w11[m] = bx * by;
        cl.f00[m] = (float)cl.w00[m];
        cl.f10[m] = (float)cl.w10[m];
        cl.f01[m] = (float)cl.w01[m];
        cl.f11[m] = (float)cl.w11[m];
        cl.hf[m] = p.hfac[m];
        cl.hff[m] = (float)p.hfac[m];
        cl.hfmax = std::max(cl.hfmax, cl.hff[m]);
    }
    return cl;
}

ReachTable2 make_reach(const hjbp_plan &p) {
    ReachTable2 rt;
    std::memset(&rt, 0, sizeof(rt));
    for (int m = 0; m < p.desc.n_controls; ++m) {
        const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
        const double bx = std::fabs(ax), by = std::fabs(ay);
        const unsigned need = (unsigned)(bx * (1.0 - by) > 0.0) | ((unsigned)((1.0 - bx) * by > 0.0) << 1) |
                              ((unsigned)(bx * by > 0.0) << 2);
        if (need) rt.present[(ax >= 0.0 ? 1 : 0) + (ay >= 0.0 ? 2 : 0)] |= (uint8_t)(1u << need);
    }
    return rt;
}

// AO3 cones (Sec. 6) over the positions of the quadrant-sorted table of
// make_table; entry nc is the full set (nodes without a coarse feedback).
Cone2 make_cones(const hjbp_plan &p, double *mean_size) {
    Cone2 cn;
    std::memset(&cn, 0, sizeof(cn));
    const int nc = p.desc.n_controls;
    cn.nc = nc;
    std::vector<int> pos(nc);
    int at = 0;
    for (int q = 0; q < 4; ++q)
        for (int m = 0; m < nc; ++m) {
            const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
            if ((ax >= 0.0 ? 1 : 0) + (ay >= 0.0 ? 2 : 0) == q) pos[m] = at++;
        }
    const double cr = std::cos(3.14159265358979323846 / p.desc.reduce_r) - 1e-12;
    double total = 0.0;
    for (int a = 0; a <= nc; ++a) {
        unsigned long long mask = 0;
        uint32_t reach = 0;
        for (int m = 0; m < nc; ++m) {
            const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
            bool ok = true;
            if (a < nc) {
                // the cone is a set of controls a (Sec. 6), not of directions of f
                double dot = 0.0;
                dot += p.controls[2 * m] * p.controls[2 * a];
                dot += p.controls[2 * m + 1] * p.controls[2 * a + 1];
                ok = dot >= cr;
            }
            if (!ok) continue;
            mask |= 1ull << pos[m];
            const double bx = std::fabs(ax), by = std::fabs(ay);
            const unsigned need = (unsigned)(bx * (1.0 - by) > 0.0) | ((unsigned)((1.0 - bx) * by > 0.0) << 1) |
                                  ((unsigned)(bx * by > 0.0) << 2);
            if (need) reach |= (1u << need) << (8 * ((ax >= 0.0 ? 1 : 0) + (ay >= 0.0 ? 2 : 0)));
        }
        cn.mask[a] = mask;
        cn.reach[a] = reach;
        if (a < nc) total += (double)__builtin_popcountll(mask);
    }
    if (mean_size) *mean_size = total / nc;
    // the pair form: the classes of the 8-class symmetric set in the order the
    // pair table enumerates them (controls with x > 0, y > 0, x >= y)
    const CtlTable2<float> ct = make_table<float>(p);
    if (ct.d4 && ct.ncls == 8) {
        const double tol = 1e-12;
        std::vector<std::pair<double, double>> reps;
        for (int m = 0; m < nc; ++m) {
            const double x = p.dirs[2 * m], y = p.dirs[2 * m + 1];
            if (x > 0.0 && y > 0.0 && x >= y - tol) reps.emplace_back(x, y);
        }
        std::vector<int> bit(nc, -1), abit(nc, -1);
        bool ok = reps.size() == 8;
        for (int m = 0; m < nc && ok; ++m) {
            const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
            if (ay == 0.0 || ax == 0.0) {
                abit[m] = ay == 0.0 ? (ax > 0.0 ? 0 : 1) : (ay > 0.0 ? 2 : 3);
                continue;
            }
            const int q = (ax >= 0.0 ? 1 : 0) + (ay >= 0.0 ? 2 : 0);
            const double X = std::fabs(ax), Y = std::fabs(ay);
            const bool diag = std::fabs(X - Y) < tol;
            const int member = (X >= Y || diag) ? 0 : 1;
            const double rx = member ? Y : X, ry = member ? X : Y;
            int k = -1;
            for (int c = 0; c < 8; ++c)
                if (std::fabs(reps[c].first - rx) < tol && std::fabs(reps[c].second - ry) < tol) k = c;
            if (k < 0) ok = false;
            else bit[m] = 16 * q + 2 * k + member;
        }
        if (ok) {
            for (int a = 0; a <= nc; ++a) {
                unsigned long long pmk = 0;
                unsigned amk = 0;
                for (int m = 0; m < nc; ++m) {
                    if (!((cn.mask[a] >> pos[m]) & 1ull)) continue;
                    if (abit[m] >= 0) amk |= 1u << abit[m];
                    else pmk |= 1ull << bit[m];
                }
                cn.pmask[a] = pmk;
                cn.amask[a] = (uint8_t)amk;
            }
            cn.pairs = 1;
        }
    }
    return cn;
}

DynParams make_dyn(const hjbp_plan &p) {
    DynParams dp;
    dp.kind = p.desc.dyn;
    dp.s = p.desc.drift[0];
    for (int i = 0; i < 3; ++i) dp.w[i] = p.desc.drift[1 + i];
    return dp;
}

SpeedParams make_speed(const hjbp_plan &p) {
    SpeedParams sp;
    sp.kind = p.desc.speed;
    for (int i = 0; i < 64; ++i) sp.p[i] = p.desc.speed_params[i];
    return sp;
}

TargetSet make_targets(const hjbp_plan &p) {
    TargetSet ts;
    std::memset(&ts, 0, sizeof(ts));
    const int d = p.desc.dim;
    ts.n = p.desc.n_targets;
    ts.kind = p.desc.target_kind;
    ts.nparts = p.R;
    for (int j = 0; j < ts.n; ++j) {
        ts.c0[j] = p.targets[(d + 1) * j + 0];
        ts.c1[j] = p.targets[(d + 1) * j + 1];
        ts.c2[j] = d == 3 ? p.targets[(d + 1) * j + 2] : 0.0;
        ts.r[j] = p.targets[(d + 1) * j + d];
    }
    return ts;
}

Grid2 make_grid(int n0, int n1, double lo0, double lo1, double k) {
    Grid2 g;
    g.n0 = n0;
    g.n1 = n1;
    g.ntx = (n0 - 2 + kTile - 1) / kTile;
    g.nty = (n1 - 2 + kTile - 1) / kTile;
    g.lo0 = lo0;
    g.lo1 = lo1;
    g.k = k;
    return g;
}

struct Ev {
    cudaEvent_t e;
    explicit Ev(cudaStream_t s) {
        check_cuda(cudaEventCreate(&e), "event");
        check_cuda(cudaEventRecord(e, s), "event record");
    }
    ~Ev() { cudaEventDestroy(e); }
};

// CUDA event pairs around kernel launches on one stream; keep(n) retains the
// first n pairs of the last batch (launches after convergence did no work).
struct LaunchTimer {
    hjbp_plan &p;
    bool on;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> cur, kept;
    int64_t launches = 0;
    LaunchTimer(hjbp_plan &plan, bool enabled) : p(plan), on(enabled) {}
    void begin() {
        if (!on) return;
        cudaEvent_t a = p.pooled_event(), b = p.pooled_event();
        if (!a || !b) throw HjbpError{HJBP_ECUDA, "cudaEventCreate failed"};
        check_cuda(cudaEventRecord(a, p.stream), "event");
        cur.emplace_back(a, b);
    }
    void end() {
        if (on) check_cuda(cudaEventRecord(cur.back().second, p.stream), "event");
    }
    void keep(int n) {
        for (size_t l = 0; l < cur.size() && (int)l < n; ++l) kept.push_back(cur[l]);
        cur.clear();
        launches += n;
    }
    double total_ms() {
        double ms = 0.0;
        if (!on) return 0.0;
        if (!kept.empty()) check_cuda(cudaEventSynchronize(kept.back().second), "event sync");
        for (auto &e : kept) {
            float m = 0.f;
            cudaEventElapsedTime(&m, e.first, e.second);
            ms += m;
        }
        return ms;
    }
};

float ms_between(const Ev &a, const Ev &b) {
    float ms = 0.f;
    cudaEventSynchronize(b.e);
    cudaEventElapsedTime(&ms, a.e, b.e);
    return ms;
}

// S* on the current codes (R14): reach from the targets, prune, repeat.
int reach2d(hjbp_plan &p, const Grid2 &g, int8_t *code, uint8_t *rch, Sched &s, int cap, int64_t N,
            const double *dterm = nullptr, const Cone2 *cone = nullptr) {
    const int passes = p.desc.tune[2] > 0 ? p.desc.tune[2] : 1;
    const ReachTable2 rt = make_reach(p);
    unsigned long long *removed = alloc_n<unsigned long long>(p, 1);
    // per tile the candidate, terminal and free row sets of k_reach2d (11 x 32 words)
    uint64_t *rcache = alloc_n<uint64_t>(p, (int64_t)std::max(1, s.ntiles) * 11 * 32);
    uint8_t *rvalid = alloc_n<uint8_t>(p, std::max(1, s.ntiles));
    int total = 0;
    // each round prunes at least one node or ends the loop, so it ends after at
    // most N rounds
    for (int64_t round = 0;; ++round) {
        if (round > N) throw HjbpError{HJBP_ECUDA, "reachability pruning did not settle"};
        // peel the nodes left without any control first (they cannot be in S*)
        RunResult pe = run_tiles(p, g, s, 0.5f, cap, [&](int par, int) {
            k_peel2d<<<s.ntiles, 32, 0, p.stream>>>(g, code, s.d, par, rt, dterm, p.astar, cone);
            ++p.stats.kernel_launches;
        });
        total += pe.launches;
        if (!pe.converged) throw HjbpError{HJBP_ECUDA, "peeling did not settle"};
        check_cuda(cudaMemsetAsync(rch, 0, (size_t)N, p.stream), "reach reset");
        // the codes changed (peel, prune): the tiles' cached row sets are stale
        check_cuda(cudaMemsetAsync(rvalid, 0, (size_t)std::max(1, s.ntiles), p.stream), "reach cache reset");
        RunResult rr = run_tiles(p, g, s, 0.5f, cap, [&](int par, int) {
            k_reach2d<<<s.ntiles, 32, 0, p.stream>>>(g, code, rch, s.d, par, rt, passes, dterm, p.astar, cone,
                                                     rcache, rvalid);
            ++p.stats.kernel_launches;
        });
        total += rr.launches;
        if (!rr.converged) throw HjbpError{HJBP_ECUDA, "reachability sweep did not settle"};
        check_cuda(cudaMemsetAsync(removed, 0, sizeof(unsigned long long), p.stream), "memset");
        k_reach_prune<<<grid_for(N), 256, 0, p.stream>>>(N, code, rch, removed);
        ++p.stats.kernel_launches;
        unsigned long long h = 0;
        check_cuda(cudaMemcpyAsync(&h, removed, sizeof(h), cudaMemcpyDeviceToHost, p.stream), "removed");
        check_cuda(cudaStreamSynchronize(p.stream), "reach sync");
        if (h == 0) break;
    }
    return total;
}

template <typename T, int NCLS, int W>
void launch_mw(int ntiles, cudaStream_t st, const Grid2 &g, const int8_t *code, const T *h, T *b0, T *b1,
               const TileSched &s, int par, int rounds, unsigned long long *updates, const CtlTable2<T> &ct,
               int clamp, const T *dval) {
    if (dval)
        k_value2d_mw<T, NCLS, true, W><<<ntiles, 32 * W, 0, st>>>(g, code, h, b0, b1, s, par, rounds, updates, ct,
                                                                    clamp, dval);
    else
        k_value2d_mw<T, NCLS, false, W><<<ntiles, 32 * W, 0, st>>>(g, code, h, b0, b1, s, par, rounds, updates, ct,
                                                                     clamp, nullptr);
}

// Value iteration on S* (R14) to the sup-norm tolerance: monotone from M, or
// plain from the warm start (AO1); dval: Dirichlet data (Eq. dbc) or NULL.
template <typename T>
RunResult value2d(hjbp_plan &p, const Grid2 &g, const int8_t *code, const T *h, const double *fixed, T *b0, T *b1,
                  Sched &s, double tol, int cap, int rounds, T *out_t, double *out64, unsigned long long *updates,
                  bool fine, const T *dval = nullptr, const double *warm = nullptr, const Cone2 *cone = nullptr) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    k_init_values2d<T><<<grid_for(N), 256, 0, p.stream>>>(N, code, fixed, (T)kStartValue, b0, b1, warm);
    const int clamp = warm ? 0 : 1;
    ++p.stats.kernel_launches;
    const CtlTable2<T> ct = make_table<T>(p);
    const bool timed = fine && (p.desc.flags & HJBP_FLAG_TIME_SWEEPS);
    const int warps = p.desc.tune[3] > 0 ? p.desc.tune[3] : 1;
    const bool pairs = cone && ct.d4 && ct.ncls == 8 && p.cone_pairs;   // AO3 in the pair form
    // the packed FP32-pair update (sl_update_x2, same result to the last bit);
    // tune[6] = 2: the scalar form
    const int packed = p.desc.tune[6] == 2 ? 0 : 1;
    // FP32 monotone sweeps without cones exchange their halos inside the
    // launch, after every pass (tune[7] = 0) or every round (2); tune[7] = 1
    // keeps the deterministic block-Jacobi launches
    const int xmode = p.desc.tune[7];
    const bool xchg = std::is_same<T, float>::value && clamp && !cone && xmode != 1 && !(warps == 2 || warps == 4);
    const int xpass = xmode == 2 ? 0 : 1;
    LaunchTimer timer(p, timed);
    RunResult rr = run_tiles(p, g, s, tol, cap, [&](int par, int) {
        timer.begin();
        const bool mw = !cone && (warps == 2 || warps == 4);   // several warps per tile (no AO3 cones)
        if (cone && pairs && dval)
            k_value2d<T, 8, true, true><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates,
                                                                       ct, clamp, dval, p.astar, cone);
        else if (cone && pairs)
            k_value2d<T, 8, false, true><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates,
                                                                        ct, clamp, nullptr, p.astar, cone);
        else if (cone && dval)
            k_value2d<T, 0, true, true><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates,
                                                                       ct, clamp, dval, p.astar, cone);
        else if (cone)
            k_value2d<T, 0, false, true><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates,
                                                                        ct, clamp, nullptr, p.astar, cone);
        else if (mw && warps == 2 && ct.d4 && ct.ncls == 8)
            launch_mw<T, 8, 2>(s.ntiles, p.stream, g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (mw && warps == 2)
            launch_mw<T, 0, 2>(s.ntiles, p.stream, g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (mw && ct.d4 && ct.ncls == 8)
            launch_mw<T, 8, 4>(s.ntiles, p.stream, g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (mw)
            launch_mw<T, 0, 4>(s.ntiles, p.stream, g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (xchg && dval && ct.d4 && ct.ncls == 8)
            k_value2d<T, 8, true, false, true><<<s.ntiles, 32, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval, nullptr, nullptr, 0, xpass);
        else if (xchg && dval)
            k_value2d<T, 0, true, false, true><<<s.ntiles, 32, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval, nullptr, nullptr, 0, xpass);
        else if (xchg && ct.d4 && ct.ncls == 8)
            k_value2d<T, 8, false, false, true><<<s.ntiles, 32, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, nullptr, nullptr, nullptr, packed, xpass);
        else if (xchg)
            k_value2d<T, 0, false, false, true><<<s.ntiles, 32, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, nullptr, nullptr, nullptr, 0, xpass);
        else if (dval && ct.d4 && ct.ncls == 8)
            k_value2d<T, 8, true><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                 clamp, dval);
        else if (dval)
            k_value2d<T, 0, true><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                 clamp, dval);
        else if (ct.d4 && ct.ncls == 8)
            k_value2d<T, 8, false><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                  clamp, nullptr, nullptr, nullptr, packed);
        else if (ct.d4 && ct.ncls == 4 && std::is_same<T, float>::value)
            k_value2d<T, 4, false><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                  clamp, nullptr, nullptr, nullptr, packed);
        else
            k_value2d<T, 0, false><<<s.ntiles, 32, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                  clamp, nullptr);
        ++p.stats.kernel_launches;
        if (fine) ++p.stats.sweep_kernel_launches;
        timer.end();
    });
    if (fine) p.stats.sweep_tile_visits += rr.tile_visits;
    // launches after convergence found no active tile and did no work
    timer.keep(rr.launches);
    if (timed) p.stats.ms_sweep_kernel += timer.total_ms();
    k_gather2d<T><<<grid_for(N), 256, 0, p.stream>>>(g, s.d.latest, b0, b1, out_t, out64);
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "gather");
    return rr;
}

// The same solve with the persistent tile queue (monotone update from M; no
// warm start, no control cones).  Returns launches = 1.
template <typename T, int NCLS, bool kDir>
void launch_async(hjbp_plan &p, int ntiles, const Grid2 &g, const int8_t *code, const T *h, T *u,
                  const TileQueue &q, int rounds, double tol, unsigned long long *updates, const CtlTable2<T> &ct,
                  const T *dval) {
    int per_sm = 0, sms = 0, dev = 0;
    check_cuda(cudaGetDevice(&dev), "device");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_value2d_async<T, NCLS, kDir>, 32, 0),
               "occupancy");
    // resident warps: the occupancy limit, or tune[4] per SM
    const int want = p.desc.tune[4] > 0 ? std::min(p.desc.tune[4], std::max(1, per_sm)) : std::max(1, per_sm);
    const int grid = std::max(1, std::min(ntiles, want * sms));
    k_value2d_async<T, NCLS, kDir><<<grid, 32, 0, p.stream>>>(g, code, h, u, q, rounds, tol, updates, ct, dval);
}

template <typename T>
RunResult value2d_async(hjbp_plan &p, const Grid2 &g, const int8_t *code, const T *h, T *b0, T *b1, Sched &s,
                        double tol, int rounds, T *out_t, double *out64, unsigned long long *updates,
                        const T *dval) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    cudaStream_t st = p.stream;
    RunResult rr;
    k_init_values2d<T><<<grid_for(N), 256, 0, st>>>(N, code, nullptr, (T)kStartValue, b0, b1, nullptr);
    ++p.stats.kernel_launches;
    const int nt = s.ntiles;
    if (nt > 0) {
        TileQueue q;
        q.cap = 2 * nt;
        q.slot = alloc_n<int>(p, q.cap);
        q.head = alloc_n<unsigned>(p, 1);
        q.tail = alloc_n<unsigned>(p, 1);
        q.state = alloc_n<int>(p, nt);
        q.pending = alloc_n<int>(p, 1);
        q.err = alloc_n<int>(p, 1);
        q.visits = alloc_n<unsigned long long>(p, 1);
        k_queue_init<<<grid_for(q.cap), 256, 0, st>>>(q, nt);
        ++p.stats.kernel_launches;
        const CtlTable2<T> ct = make_table<T>(p);
        const bool timed = p.desc.flags & HJBP_FLAG_TIME_SWEEPS;
        cudaEvent_t a = nullptr, b = nullptr;
        if (timed) {
            check_cuda(cudaEventCreate(&a), "event");
            check_cuda(cudaEventCreate(&b), "event");
            check_cuda(cudaEventRecord(a, st), "event");
        }
        const double ftol = tol;
        if (dval && ct.d4 && ct.ncls == 8) launch_async<T, 8, true>(p, nt, g, code, h, b0, q, rounds, ftol, updates, ct, dval);
        else if (dval) launch_async<T, 0, true>(p, nt, g, code, h, b0, q, rounds, ftol, updates, ct, dval);
        else if (ct.d4 && ct.ncls == 8) launch_async<T, 8, false>(p, nt, g, code, h, b0, q, rounds, ftol, updates, ct, nullptr);
        else launch_async<T, 0, false>(p, nt, g, code, h, b0, q, rounds, ftol, updates, ct, nullptr);
        check_cuda(cudaGetLastError(), "queue sweep launch");
        ++p.stats.kernel_launches;
        ++p.stats.sweep_kernel_launches;
        if (timed) check_cuda(cudaEventRecord(b, st), "event");
        int herr = 0;
        unsigned long long hv = 0;
        check_cuda(cudaMemcpyAsync(&herr, q.err, sizeof(int), cudaMemcpyDeviceToHost, st), "queue err");
        check_cuda(cudaMemcpyAsync(&hv, q.visits, sizeof(hv), cudaMemcpyDeviceToHost, st), "queue visits");
        check_cuda(cudaStreamSynchronize(st), "queue sync");
        if (timed) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            p.stats.ms_sweep_kernel += ms;
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
        if (herr) throw HjbpError{HJBP_ECUDA, "persistent tile sweep: a bounded wait ran out"};
        rr.tile_visits = (int64_t)hv;
        p.stats.sweep_tile_visits += (int64_t)hv;
    }
    rr.launches = 1;
    rr.converged = true;
    check_cuda(cudaMemsetAsync(s.d.latest, 0, std::max(1, nt), st), "latest");
    k_gather2d<T><<<grid_for(N), 256, 0, st>>>(g, s.d.latest, b0, b1, out_t, out64);
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "gather");
    return rr;
}

// Jacobi value iteration of a small grid with one warp per node (FP64).
RunResult value_wide2d(hjbp_plan &p, const Grid2 &g, const int8_t *code, const double *h, const double *fixed,
                       double *b0, double *b1, double tol, int cap, double *out64) {
    const int64_t N = (int64_t)g.n0 * g.n1;
    cudaStream_t st = p.stream;
    k_init_values2d<double><<<grid_for(N), 256, 0, st>>>(N, code, fixed, kStartValue, b0, b1, nullptr);
    ++p.stats.kernel_launches;
    const CtlSelf2<double> cs = make_self<double>(p);
    const int chunk = 16;
    double *res = alloc_n<double>(p, chunk);
    std::vector<double> hres(chunk);
    RunResult rr;
    const int blocks = (int)std::min<int64_t>((N + 7) / 8, 152 * 16);
    int L = 0;
    while (L < cap) {
        check_cuda(cudaMemsetAsync(res, 0, sizeof(double) * chunk, st), "memset");
        int n = std::min(chunk, cap - L);
        for (int l = 0; l < n; ++l) {
            const double *in = ((L + l) & 1) ? b1 : b0;
            double *out = ((L + l) & 1) ? b0 : b1;
            k_value_wide2d<double><<<blocks, 256, 0, st>>>(g, code, h, in, out, res, l, cs);
            ++p.stats.kernel_launches;
        }
        check_cuda(cudaGetLastError(), "wide launch");
        check_cuda(cudaMemcpyAsync(hres.data(), res, sizeof(double) * chunk, cudaMemcpyDeviceToHost, st), "res");
        check_cuda(cudaStreamSynchronize(st), "wide sync");
        for (int l = 0; l < n; ++l) {
            rr.launches = L + l + 1;
            rr.last_res = hres[l];
            if (hres[l] <= tol) {
                rr.converged = true;
                break;
            }
        }
        L += n;
        if (rr.converged) break;
    }
    // the launch that met the test wrote into the buffer of its parity
    const double *fin = (rr.launches & 1) ? b1 : b0;
    k_finalize<<<grid_for(N), 256, 0, st>>>(N, fin, out64);
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "wide finalize");
    return rr;
}

}  // namespace

// The per-line factors of a separable speed on grid g (SpeedLines), in the
// plan's arena; no factors (per-node evaluation) for the other speeds.
SpeedLines speed_lines2(hjbp_plan &p, const Grid2 &g, const SpeedParams &sp) {
    SpeedLines sl{{nullptr, nullptr, nullptr}, speed_terms(sp.kind)};
    if (sl.nt == 0) return sl;
    double *f0 = alloc_n<double>(p, (int64_t)g.n0 * sl.nt), *f1 = alloc_n<double>(p, (int64_t)g.n1 * sl.nt);
    const int total = sl.nt * (g.n0 + g.n1);
    k_speed_lines<<<(total + 255) / 256, 256, 0, p.stream>>>(sp, sl.nt, g.n0, g.n1, 0, g.lo0, g.lo1, 0.0, g.k, f0, f1,
                                                           nullptr);
    ++p.stats.kernel_launches;
    sl.f[0] = f0;
    sl.f[1] = f1;
    return sl;
}

hjbp_status solve2d(hjbp_plan &p) {
    const hjbp_problem_desc &d = p.desc;
    cudaStream_t st = p.stream;
    const int64_t N = p.N;
    const Grid2 g = make_grid(d.n[0], d.n[1], d.lo[0], d.lo[1], p.k);
    const SpeedParams sp = make_speed(p);
    const TargetSet ts = make_targets(p);
    const ObstacleSet os = make_obstacles(2, d.n_obstacles, d.obstacles);
    const int cap = d.max_sweeps > 0 ? d.max_sweeps : 1000000;
    const int hist = std::max(std::min(cap, 1 << 20), kReachCap);
    const bool fp32 = d.precision == HJBP_FP32_POLISH64;
    const int R = p.R;
    // rounds per launch: 4 where the halos are exchanged after every pass (a
    // launch then carries a change across several tiles: the FP32 monotone
    // value sweep and the colour bulk), 2 for block-Jacobi launches
    const bool vx = fp32 && d.tune[7] != 1 && !(d.flags & (HJBP_FLAG_WARM_START | HJBP_FLAG_TILE_QUEUE)) &&
                    d.reduce_r == 0.0 && d.tune[3] != 2 && d.tune[3] != 4;
    const int vrounds = d.tune[0] > 0 ? d.tune[0] : (vx ? 4 : 2);
    hjbp_stats &S = p.stats;
    std::memset(&S, 0, sizeof(S));
    hjbp_status status = HJBP_OK;

    Ev e0(st);
    int8_t *code0 = alloc_n<int8_t>(p, N);
    int8_t *code = alloc_n<int8_t>(p, N);
    uint8_t *rch = alloc_n<uint8_t>(p, N);
    double *h64 = alloc_n<double>(p, N);
    float *h32 = fp32 ? alloc_n<float>(p, N) : nullptr;
    unsigned long long *updates = alloc_n<unsigned long long>(p, 1);
    check_cuda(cudaMemsetAsync(updates, 0, sizeof(unsigned long long), st), "memset");
    k_setup2d<<<grid_for(N), 256, 0, st>>>(g, sp, ts, 0.0, 0, code0, h32, h64, nullptr, make_dyn(p), os,
                                           speed_lines2(p, g, sp));
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "setup");
    Sched sched = make_sched(p, g, hist);
    sched.d.alt = d.tune[5] == 1 ? 1 : 0;   // 2D: alternating halves only on request
    Ev e1(st);

    double *dlit = nullptr;   // literal U_P^(0): the Dirichlet data (R16)
    if (p.patchy) {
        // ---- Step 1: coarse solve (FP64)
        const Grid2 gc = make_grid(d.n_coarse[0], d.n_coarse[1], d.lo[0], d.lo[1], p.kc);
        const int64_t Nc = p.Nc;
        int8_t *ccode = alloc_n<int8_t>(p, Nc);
        uint8_t *crch = alloc_n<uint8_t>(p, Nc);
        double *ch64 = alloc_n<double>(p, Nc);
        double *cfix = alloc_n<double>(p, Nc);
        double *cb0 = alloc_n<double>(p, Nc), *cb1 = alloc_n<double>(p, Nc);
        k_setup2d<<<grid_for(Nc), 256, 0, st>>>(gc, sp, ts, p.kc * std::sqrt(2.0) / 2.0, 1, ccode, nullptr, ch64,
                                                cfix, make_dyn(p), os, speed_lines2(p, gc, sp));
        ++p.stats.kernel_launches;
        k_merge_targets<<<grid_for(Nc), 256, 0, st>>>(Nc, ccode);
        ++p.stats.kernel_launches;
        Sched csched = make_sched(p, gc, hist);
        S.sweeps_reach += reach2d(p, gc, ccode, crch, csched, kReachCap, Nc);
        const double tolc = d.tol_coarse > 0 ? d.tol_coarse : 1e-12;
        RunResult rc = value_wide2d(p, gc, ccode, ch64, cfix, cb0, cb1, tolc, cap, p.u_coarse);
        S.sweeps_coarse = rc.launches;
        if (!rc.converged) status = HJBP_ENOCONV;
        Ev e2(st);
        // ---- Step 2: U_P^(0) and the coarse feedback a*
        if (d.flags & HJBP_FLAG_DIRICHLET) dlit = alloc_n<double>(p, N);
        k_u0_2d<<<grid_for(N), 256, 0, st>>>(g, gc, code0, p.u_coarse, p.u0, dlit);
        ++p.stats.kernel_launches;
        k_feedback2d<<<grid_for(N, 128), 128, 0, st>>>(g, code0, h64, p.u0, p.astar, make_literal(p));
        ++p.stats.kernel_launches;
        check_cuda(cudaGetLastError(), "feedback");
        // AO2: causal sweep directions per tile from the feedback (Step 3.1 and 3.2)
        if ((d.flags & HJBP_FLAG_CAUSAL_SWEEPS) && sched.ntiles) {
            DirCtl dc;
            for (int m = 0; m < d.n_controls; ++m) {
                const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
                dc.sx[m] = (int8_t)(ax > 1e-12 ? 1 : (ax < -1e-12 ? -1 : 0));
                dc.sy[m] = (int8_t)(ay > 1e-12 ? 1 : (ay < -1e-12 ? -1 : 0));
            }
            uint8_t *dirs = alloc_n<uint8_t>(p, sched.ntiles);
            k_tile_dirs2d<<<sched.ntiles, 32, 0, st>>>(g, code0, p.astar, dc, 0.9f, dirs);
            ++p.stats.kernel_launches;
            check_cuda(cudaGetLastError(), "tile directions");
            sched.d.dirs = dirs;
        }
        Ev e3(st);
        // ---- Step 3.1: colours phi^j, projection, Remark 3.1 fill
        {
            PhiCtl hpc;
            std::memset(&hpc, 0, sizeof(hpc));
            hpc.nc = d.n_controls;
            for (int m = 0; m < d.n_controls; ++m) {
                const double ax = p.dirs[2 * m], ay = p.dirs[2 * m + 1];
                const double bx = std::fabs(ax), by = std::fabs(ay);
                const double w00 = (1.0 - bx) * (1.0 - by), w10 = bx * (1.0 - by), w01 = (1.0 - bx) * by;
                const double w11 = bx * by, kap = 1.0 / (1.0 - w00);
                hpc.sx[m] = ax >= 0 ? 1 : -1;
                hpc.sy[m] = ay >= 0 ? 1 : -1;
                hpc.w00[m] = w00;
                hpc.w10[m] = w10;
                hpc.w01[m] = w01;
                hpc.w11[m] = w11;
                hpc.kw10[m] = (float)(kap * w10);
                hpc.kw01[m] = (float)(kap * w01);
                hpc.kw11[m] = (float)(kap * w11);
                hpc.kap[m] = (float)kap;
            }
            PhiCtl *dpc = static_cast<PhiCtl *>(p.dev_alloc(sizeof(PhiCtl)));
            check_cuda(cudaMemcpyAsync(dpc, &hpc, sizeof(PhiCtl), cudaMemcpyHostToDevice, st), "phi ctl");
            // colours per transport pass: up to 8 (one front propagation per group)
            const int RG = R > 4 ? 8 : (R >= 3 ? 4 : (R == 2 ? 2 : 1));
            // the bulk of up to four colours exchanges halos inside a launch unless
            // tune[7] = 1 (4 rounds per launch, else 2).  With eight colours the
            // exchange's registers halve the resident CTAs (256 threads each) and the
            // block-Jacobi launches measured faster (labels of 8 patches at 2049^2:
            // 12.6 against 15.2 ms)
            const bool phi_x = d.tune[7] != 1 && RG <= 4;
            const int prounds = d.tune[1] > 0 ? d.tune[1] : (phi_x ? 4 : 2);
            float *f0 = alloc_n<float>(p, N * RG), *f1 = alloc_n<float>(p, N * RG), *r32 = alloc_n<float>(p, N * RG);
            double *phig = alloc_n<double>(p, N * RG);
            float *rmax = alloc_n<float>(p, 1);
            const double tolp = d.tol_phi > 0 ? d.tol_phi : 1e-10;
            // per-launch CUDA events (HJBP_FLAG_TIME_SWEEPS) and the node-colour update count
            LaunchTimer ptimer(p, (d.flags & HJBP_FLAG_TIME_SWEEPS) != 0);
            unsigned long long *pupd = alloc_n<unsigned long long>(p, 1);
            check_cuda(cudaMemsetAsync(pupd, 0, sizeof(unsigned long long), st), "memset");
            for (int j0 = 0; j0 < R; j0 += RG) {
                const int rg = std::min(RG, R - j0);
                // colours past R in the last group see no target and stay 0
                const int rgl = rg > 4 ? 8 : (rg >= 3 ? 4 : rg);
                auto launch_group = [&](auto tag) {
                    constexpr int G = decltype(tag)::value;
                    check_cuda(cudaFuncSetAttribute(k_phi2d<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)sizeof(PhiSmem<G, false>)), "phi smem");
                    check_cuda(cudaFuncSetAttribute(k_phi2d<G, false, (G <= 4)>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)sizeof(PhiSmem<G, false>)), "phi smem");
                    check_cuda(cudaFuncSetAttribute(k_phi2d<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)sizeof(PhiSmem<G, true>)), "phi smem");
                    // FP32 bulk solve
                    k_phi_init2d<G><<<grid_for(N), 256, 0, st>>>(N, code0, j0, 0, f0, f1);
                    ++p.stats.kernel_launches;
                    RunResult rp = run_tiles(p, g, sched, std::max(tolp, 2e-7), cap, [&](int par, int) {
                        ptimer.begin();
                        if (G <= 4 && phi_x)
                            k_phi2d<G, false, (G <= 4)><<<sched.ntiles, 32 * phi_warps<G>(), sizeof(PhiSmem<G, false>),
                                                      st>>>(g, code0, p.astar, f0, f1, nullptr, sched.d, par, prounds,
                                                            dpc, pupd);
                        else
                            k_phi2d<G, false><<<sched.ntiles, 32 * phi_warps<G>(), sizeof(PhiSmem<G, false>), st>>>(
                                g, code0, p.astar, f0, f1, nullptr, sched.d, par, prounds, dpc, pupd);
                        ptimer.end();
                        ++p.stats.kernel_launches;
                    });
                    ptimer.keep(rp.launches);
                    S.sweeps_phi += rp.launches;
                    if (!rp.converged) status = HJBP_ENOCONV;
                    k_phi_collect2d<G><<<grid_for(N), 256, 0, st>>>(g, sched.d.latest, f0, f1, phig, 0);
                    ++p.stats.kernel_launches;
                    // FP64 refinement: residual in FP64, correction solved in FP32
                    for (int it = 0; it < 6; ++it) {
                        check_cuda(cudaMemsetAsync(rmax, 0, sizeof(float), st), "memset");
                        k_phi_residual2d<G><<<grid_for(N), 256, 0, st>>>(g, code0, p.astar, phig, r32, rmax, dpc);
                        ++p.stats.kernel_launches;
                        float hr = 0.f;
                        check_cuda(cudaMemcpyAsync(&hr, rmax, sizeof(float), cudaMemcpyDeviceToHost, st), "rmax");
                        check_cuda(cudaStreamSynchronize(st), "rmax sync");
                        S.phi_refinements++;
                        if (hr <= tolp) break;
                        k_phi_init2d<G><<<grid_for(N), 256, 0, st>>>(N, code0, j0, 1, f0, f1);
                        ++p.stats.kernel_launches;
                        const float told = std::max((float)(tolp * 0.1), 1e-3f * hr);
                        RunResult rc = run_tiles(p, g, sched, told, cap, [&](int par, int) {
                            ptimer.begin();
                            k_phi2d<G, true><<<sched.ntiles, 32 * phi_warps<G>(), sizeof(PhiSmem<G, true>), st>>>(
                                g, code0, p.astar, f0, f1, r32, sched.d, par, prounds, dpc, pupd);
                            ptimer.end();
                            ++p.stats.kernel_launches;
                        });
                        ptimer.keep(rc.launches);
                        S.sweeps_phi += rc.launches;
                        k_phi_collect2d<G><<<grid_for(N), 256, 0, st>>>(g, sched.d.latest, f0, f1, phig, 1);
                        ++p.stats.kernel_launches;
                    }
                    check_cuda(cudaMemcpyAsync(p.phi + (int64_t)j0 * N, phig, sizeof(double) * N * rg,
                                               cudaMemcpyDeviceToDevice, st), "phi copy");
                };
                if (rgl == 8) launch_group(std::integral_constant<int, 8>());
                else if (rgl == 4) launch_group(std::integral_constant<int, 4>());
                else if (rgl == 2) launch_group(std::integral_constant<int, 2>());
                else launch_group(std::integral_constant<int, 1>());
            }
            {
                unsigned long long hp = 0;
                check_cuda(cudaMemcpyAsync(&hp, pupd, sizeof(hp), cudaMemcpyDeviceToHost, st), "phi updates");
                check_cuda(cudaStreamSynchronize(st), "phi updates");
                S.phi_node_colour_updates = (int64_t)hp;
                S.phi_kernel_launches = ptimer.launches;
                S.ms_phi_kernel = ptimer.total_ms();
            }
            k_label2d<<<grid_for(N), 256, 0, st>>>(N, code0, p.astar, p.phi, R, p.label_out);
            ++p.stats.kernel_launches;
            int8_t *lab2 = reinterpret_cast<int8_t *>(rch);  // scratch (reach flags are reset before use)
            unsigned long long *chg = alloc_n<unsigned long long>(p, 1);
            // Jacobi rounds of Remark 3.1's fill, ping-ponged between the two label
            // buffers, in batches between host checks (4, 8, .. 64 rounds): a round
            // after the last change changes nothing, so the batches give the rounds'
            // result exactly
            int8_t *la = p.label_out, *lb = lab2;
            int batch = 4;
            for (int it = 0; it < 100000;) {
                check_cuda(cudaMemsetAsync(chg, 0, sizeof(unsigned long long), st), "memset");
                for (int k = 0; k < batch; ++k, ++it) {
                    k_fill2d<<<grid_for(N), 256, 0, st>>>(g, la, lb, chg);
                    ++p.stats.kernel_launches;
                    std::swap(la, lb);
                }
                unsigned long long hc = 0;
                check_cuda(cudaMemcpyAsync(&hc, chg, sizeof(hc), cudaMemcpyDeviceToHost, st), "fill count");
                check_cuda(cudaStreamSynchronize(st), "fill sync");
                S.uncovered_filled += (int64_t)hc;
                if (!hc) break;
                batch = std::min(2 * batch, 64);
            }
            if (la != p.label_out)
                check_cuda(cudaMemcpyAsync(p.label_out, la, (size_t)N, cudaMemcpyDeviceToDevice, st), "fill copy");
            k_patch_codes<<<grid_for(N), 256, 0, st>>>(N, code0, p.label_out, code);
            ++p.stats.kernel_launches;
        }
        Ev e4(st);
        // ---- patch compaction
        {
            uint64_t *tile_patch = alloc_n<uint64_t>(p, sched.ntiles);
            unsigned long long *pn = alloc_n<unsigned long long>(p, kMaxTargets);
            unsigned long long *pt = alloc_n<unsigned long long>(p, kMaxTargets);
            int *tcnt = alloc_n<int>(p, (int64_t)sched.ntiles * R);
            check_cuda(cudaMemsetAsync(pn, 0, sizeof(unsigned long long) * kMaxTargets, st), "memset");
            check_cuda(cudaMemsetAsync(pt, 0, sizeof(unsigned long long) * kMaxTargets, st), "memset");
            check_cuda(cudaMemsetAsync(tcnt, 0, sizeof(int) * std::max<int64_t>(1, (int64_t)sched.ntiles * R), st),
                       "memset");
            if (sched.ntiles) k_compact2d<<<sched.ntiles, 32, 0, st>>>(g, code, tile_patch, pn, pt, tcnt, R);
            ++p.stats.kernel_launches;
            sched.d.tile_patch = tile_patch;
            unsigned long long hn[kMaxTargets], ht[kMaxTargets];
            check_cuda(cudaMemcpyAsync(hn, pn, sizeof(hn), cudaMemcpyDeviceToHost, st), "compact");
            check_cuda(cudaMemcpyAsync(ht, pt, sizeof(ht), cudaMemcpyDeviceToHost, st), "compact");
            check_cuda(cudaStreamSynchronize(st), "compact sync");
            for (int j = 0; j < R; ++j) {
                S.patch_nodes[j] = (int64_t)hn[j];
                S.patch_tiles[j] = (int64_t)ht[j];
            }
            // per-patch tile and node lists (CSR)
            build_patch_lists(p, tile_geom(d), sched.ntiles, tile_patch, tcnt, S.patch_nodes, S.patch_tiles, code);
        }
        Ev e5(st);
        S.ms_coarse = ms_between(e1, e2);
        S.ms_feedback = ms_between(e2, e3);
        S.ms_labels = ms_between(e3, e4);
        S.ms_compact = ms_between(e4, e5);
    } else {
        check_cuda(cudaMemcpyAsync(code, code0, (size_t)N, cudaMemcpyDeviceToDevice, st), "code copy");
        k_merge_targets<<<grid_for(N), 256, 0, st>>>(N, code);
        ++p.stats.kernel_launches;
    }

    // ---- Step 3.2 (or the global solve): S*, then the value iteration.
    // Patch boundaries: state constraints, or U_P^(0) (Eq. dbc); start: M, or
    // U_P^(0) (AO1).
    const bool dirichlet = p.patchy && (d.flags & HJBP_FLAG_DIRICHLET);
    const double *warm = (p.patchy && (d.flags & HJBP_FLAG_WARM_START)) ? p.u0 : nullptr;
    if (!p.init.empty()) {
        // the caller's start values (hjbp_set_initial), +inf mapped above the bound
        double *iv = alloc_n<double>(p, N);
        check_cuda(cudaMemcpyAsync(iv, p.init.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "start values");
        warm = iv;
    }
    const double *d64 = dirichlet ? dlit : nullptr;
    // AO3: control cones around the coarse feedback
    Cone2 *cone = nullptr;
    double cone_size = d.n_controls;
    if (p.patchy && d.reduce_r > 0.0) {
        const Cone2 hc = make_cones(p, &cone_size);
        p.cone_pairs = hc.pairs != 0;
        cone = static_cast<Cone2 *>(p.dev_alloc(sizeof(Cone2)));
        check_cuda(cudaMemcpyAsync(cone, &hc, sizeof(Cone2), cudaMemcpyHostToDevice, st), "cones");
        // the host copy goes out of scope: let the copy land first
        check_cuda(cudaStreamSynchronize(st), "cones sync");
    }
    // persistent tile queue: monotone update only (no warm start, no cones)
    const bool queue_ok = (d.flags & HJBP_FLAG_TILE_QUEUE) && !warm && !cone;
    Ev f0(st);
    S.sweeps_reach += reach2d(p, g, code, rch, sched, kReachCap, N, d64, cone);
    Ev fr(st);
    RunResult rv;
    float *d32 = nullptr;   // Dirichlet data in FP32 (FP32 sweeps and the polish filter)
    // per-patch residual at retirement: the tiles' last changes (FP64)
    double *last_chg = nullptr;
    if (p.patchy && sched.ntiles && !queue_ok) {
        last_chg = alloc_n<double>(p, sched.ntiles);
        check_cuda(cudaMemsetAsync(last_chg, 0, sizeof(double) * sched.ntiles, st), "memset");
        sched.d.last_chg = last_chg;
    }
    if (fp32) {
        float *b0 = alloc_n<float>(p, N), *b1 = alloc_n<float>(p, N);
        if (dirichlet) {
            d32 = alloc_n<float>(p, N);
            k_dirichlet_data<float><<<grid_for(N), 256, 0, st>>>(N, dlit, d32);
            ++p.stats.kernel_launches;
        }
        if (queue_ok)
            rv = value2d_async<float>(p, g, code, h32, b0, b1, sched, d.tol, vrounds, p.u32, nullptr, updates, d32);
        else
            rv = value2d<float>(p, g, code, h32, nullptr, b0, b1, sched, d.tol, cap, vrounds, p.u32, nullptr, updates,
                                true, d32, warm, cone);
    } else {
        double *b0 = alloc_n<double>(p, N), *b1 = alloc_n<double>(p, N);
        if (queue_ok)
            rv = value2d_async<double>(p, g, code, h64, b0, b1, sched, d.tol, vrounds, nullptr, p.u_out, updates, d64);
        else
            rv = value2d<double>(p, g, code, h64, nullptr, b0, b1, sched, d.tol, cap, vrounds, nullptr, p.u_out,
                                 updates, true, d64, warm, cone);
    }
    S.sweeps_fine = rv.launches;
    S.residual_fine = rv.last_res;
    if (!rv.converged) status = HJBP_ENOCONV;
    if (last_chg) {
        patch_residuals(p, sched.ntiles, sched.d.tile_patch, last_chg);
        sched.d.last_chg = nullptr;
    }
    // per-patch launch counts
    if (rv.launches > 0) {
        std::vector<uint64_t> ph(rv.launches);
        check_cuda(cudaMemcpyAsync(ph.data(), sched.d.patch_hist, sizeof(uint64_t) * rv.launches,
                                   cudaMemcpyDeviceToHost, st), "patch hist");
        check_cuda(cudaStreamSynchronize(st), "patch hist sync");
        for (int l = 0; l < rv.launches; ++l)
            for (int j = 0; j < R && j < 64; ++j)
                if ((ph[l] >> j) & 1ull) S.sweeps_patch[j]++;
    }
    Ev f1(st);
    // ---- FP64 polishing
    if (fp32) {
        double *pa = alloc_n<double>(p, N), *pb = alloc_n<double>(p, N);
        double *mc = alloc_n<double>(p, 1);
        k_widen<<<grid_for(N), 256, 0, st>>>(N, p.u32, pa);
        ++p.stats.kernel_launches;
        const CtlTable2<double> ct = make_table<double>(p);
        CtlTable2<float> ctf = make_table<float>(p);
        // the pair form with FP32 mirrors for the 8-class symmetric sets (not
        // with AO3 cones, whose masks address single controls); tune[6] = 1 keeps
        // the per-control kernel
        const bool pf = !cone && ctf.d4 && ctf.ncls == 8 && ct.d4 && ct.ncls == 8 && d.tune[6] != 1;
        float *pa32 = nullptr, *pb32 = nullptr;
        if (pf) {
            pa32 = alloc_n<float>(p, N);
            pb32 = alloc_n<float>(p, N);
            check_cuda(cudaMemcpyAsync(pa32, p.u32, sizeof(float) * N, cudaMemcpyDeviceToDevice, st), "mirror");
        }
        ctf.d4 = pf ? 1 : 0;
        double last = 0.0;
        int it = 0;
        for (; it < 8; ++it) {
            check_cuda(cudaMemsetAsync(mc, 0, sizeof(double), st), "memset");
            if (pf)
                k_polish2d_pf<8><<<grid_for(N, 128), 128, 0, st>>>(g, code, h64, pa, pa32, pb, pb32, mc, ctf, ct, d64,
                                                                   d32);
            else
                k_polish2d<<<grid_for(N, 128), 128, 0, st>>>(g, code, h64, pa, pb, mc, ctf, ct, d64, p.astar, cone);
            ++p.stats.kernel_launches;
            check_cuda(cudaGetLastError(), "polish");
            std::swap(pa, pb);
            std::swap(pa32, pb32);
            double hm = 0.0;
            check_cuda(cudaMemcpyAsync(&hm, mc, sizeof(double), cudaMemcpyDeviceToHost, st), "polish res");
            check_cuda(cudaStreamSynchronize(st), "polish sync");
            last = hm;
            if (hm < d.tol) {
                ++it;
                break;
            }
        }
        S.sweeps_polish = it;
        S.residual_polish = last;
        k_finalize<<<grid_for(N), 256, 0, st>>>(N, pa, p.u_out);
        ++p.stats.kernel_launches;
    }
    unsigned long long *unreach = alloc_n<unsigned long long>(p, 1);
    check_cuda(cudaMemsetAsync(unreach, 0, sizeof(unsigned long long), st), "memset");
    k_final_labels<<<grid_for(N), 256, 0, st>>>(N, code0, code, p.patchy ? nullptr : p.label_out, unreach);
    ++p.stats.kernel_launches;
    Ev f2(st);
    unsigned long long hu = 0, hun = 0;
    check_cuda(cudaMemcpyAsync(&hu, updates, sizeof(hu), cudaMemcpyDeviceToHost, st), "updates");
    check_cuda(cudaMemcpyAsync(&hun, unreach, sizeof(hun), cudaMemcpyDeviceToHost, st), "unreachable");
    check_cuda(cudaStreamSynchronize(st), "final sync");
    S.unreachable = (int64_t)hun;
    S.node_updates = (int64_t)hu;
    // with AO3 a node evaluates its cone only (the mean cone size)
    S.node_control_updates = (int64_t)((double)hu * cone_size + 0.5);
    S.n_patches = p.patchy ? R : 1;
    S.ms_setup = ms_between(e0, e1);
    S.ms_fine = ms_between(f0, f1);
    S.ms_reach = ms_between(f0, fr);
    S.ms_polish = ms_between(f1, f2);
    S.ms_total = ms_between(e0, f2);
    return status;
}

}  // namespace hjbp
