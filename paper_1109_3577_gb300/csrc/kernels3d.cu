// kernels3d.cu -- CUDA kernels and host driver of the 3D path (sm_103a).
//
// Same method and structure as the 2D path (kernels2d.cu) with trilinear
// interpolation: the foot x_i + k a of every control lies in the 3x3x3
// neighbourhood (|h f| = k, Sec. 2.1).  Interior nodes are cut into 8x8x8
// tiles, one CTA of 64 threads per tile; a tile loads itself plus a one-node
// halo into shared memory and runs line Gauss-Seidel passes in the six axis
// directions (in each step the 64 threads update one 8x8 plane), then writes
// back.  Across tiles the iteration is block-Jacobi (two value buffers and a
// per-tile parity bit), and only tiles whose 3x3x3 tile neighbourhood changed
// by more than the tolerance run again.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "hjbp_device.cuh"
#include "plan.h"

namespace hjbp {

// Dimension-free kernels defined in kernels2d.cu.
__global__ void k_reach_prune(int64_t N, int8_t *code, const uint8_t *rch, unsigned long long *removed);
__global__ void k_label2d(int64_t N, const int8_t *code, const uint8_t *astar, const double *phi, int R,
                          int8_t *label);
__global__ void k_patch_codes(int64_t N, const int8_t *code0, int8_t *label, int8_t *code);
__global__ void k_merge_targets(int64_t N, int8_t *code);
__global__ void k_final_labels(int64_t N, const int8_t *code0, const int8_t *code, int8_t *label,
                               unsigned long long *unreachable);
__global__ void k_widen(int64_t N, const float *in, double *out);
__global__ void k_finalize(int64_t N, const double *in, double *out);

constexpr int kT3 = 8;          // tile side
constexpr int kT3n = kT3 * kT3; // threads per tile CTA (one 8x8 plane per step)

struct Grid3 {
    int n0, n1, n2;
    int ntx, nty, ntz;
    double lo0, lo1, lo2, k;
};

__device__ __forceinline__ int tile_of3(const Grid3 &g, int x, int y, int z) {
    if (x < 1 || y < 1 || z < 1 || x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) return -1;
    return (((z - 1) / kT3) * g.nty + (y - 1) / kT3) * g.ntx + (x - 1) / kT3;
}

// Self-solved trilinear controls grouped by octant o = (a_x>=0) + 2(a_y>=0) +
// 4(a_z>=0); controls of octant o occupy [obeg[o], obeg[o+1]).  Corner b =
// (bx, by, bz) != 0 of the cell is offset (bx sx, by sy, bz sz) from the
// node with weight prod_d (b_d ? |a_d| : 1-|a_d|); kw[b-1] = kap w_b,
// kap = 1/(1 - w_000).
template <typename T> struct CtlTable3 {
    int nc;
    int obeg[9];
    T kw[7][kMaxControls];
    T kap[kMaxControls];
};

// Per-control table in the caller's order: literal weights w[0..7] (corner
// b = bit0 x, bit1 y, bit2 z, b = 0 the node) for the feedback and the FP64
// residual of the colour transport, self-solved FP32 weights for the sweeps.
struct Ctl3 {
    int nc;
    int8_t sx[kMaxControls], sy[kMaxControls], sz[kMaxControls];
    double w[8][kMaxControls];
    float kw[8][kMaxControls];   // kw[0] = kap, kw[b] = kap w_b
};

// Literal weights in the octant order of CtlTable3 (FP64, and rounded to FP32
// for the filter pass), with each control's index in the caller's order.
struct CtlLit3 {
    int nc;
    int obeg[9];
    int16_t idx[kMaxControls];
    double w[8][kMaxControls];
    float f[8][kMaxControls];
};

// Masks of positive-weight corners (bits 0..6 for b = 1..7) present in each octant.
// uni[o][us]: the union of the corner masks (bits 0..6 for b = 1..7) of the
// octant-o patterns whose corners all lie in the usable set us.  A node is
// reached with positive probability iff some corner in the union over the
// octants is terminal or reached: a pattern with all corners usable and one
// such corner exists iff that corner lies in one of the unions.
struct ReachTable3 {
    uint32_t present[8][4];
    uint8_t uni[8][128];
};

// Add-on AO3 (Sec. 6, R19) in 3D: per coarse feedback a* (row nc: no
// feedback, every control) the controls a with a . a* >= cos(pi / r) - 1e-12
// as bits over the octant-sorted table positions, and the union tables of
// their corner patterns per octant (as ReachTable3.uni).
struct Cone3 {
    int nc;
    uint64_t mask[kMaxControls + 1][4];
    uint8_t uni[kMaxControls + 1][8][128];
};

// Controls (a1, a2) of Brockett's integrator (R24).
struct GenCtl {
    int nc;
    double a1[kMaxControls], a2[kMaxControls];
};

__device__ __forceinline__ float warp_max3(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max3(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Max over the 64 threads of the CTA (two warps).
template <typename V> __device__ __forceinline__ V block_max64(V v, V *scratch) {
    v = warp_max3(v);
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    const V r = scratch[0] > scratch[1] ? scratch[0] : scratch[1];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ set-up --

// gctl (Brockett, R24): the coarse boundary values divide by the largest
// |f(x, a)| over the controls instead of c(x).
__global__ void k_setup3d(Grid3 g, SpeedParams sp, TargetSet ts, double extra, int boundary_values,
                          int8_t *__restrict__ code, float *__restrict__ h32, double *__restrict__ h64,
                          double *__restrict__ fixed, ObstacleSet os, SpeedLines sl,
                          const GenCtl *__restrict__ gctl = nullptr) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(i, g.n0, g.n1, ix, iy, iz);
        const double x0 = __dadd_rn(g.lo0, __dmul_rn((double)ix, g.k));
        const double x1 = __dadd_rn(g.lo1, __dmul_rn((double)iy, g.k));
        const double x2 = __dadd_rn(g.lo2, __dmul_rn((double)iz, g.k));
        double dist = 0.0;
        const int part = target_part3(ts, g.lo1, g.n1, g.k, x0, x1, x2, extra, &dist);
        const bool ring = ix == 0 || iy == 0 || iz == 0 || ix == g.n0 - 1 || iy == g.n1 - 1 || iz == g.n2 - 1;
        const double c = sl.f[0] ? speed_lines(sp, sl, ix, iy, iz) : speed_at(sp, x0, x1, x2);
        const bool stopped = !(c > kStoppedSpeed);   // cannot move: like the ghost ring
        const bool blocked = part < 0 && in_obstacle(os, x0, x1, x2);   // obstacle (Sec. 4)
        const double hh = stopped ? (double)INFINITY : __ddiv_rn(g.k, c);
        code[i] = part >= 0 ? (int8_t)(kTargetBase + part) : ((ring || stopped || blocked) ? kHard : (int8_t)0);
        if (h32) h32[i] = (float)hh;
        if (h64) h64[i] = hh;
        double v = c;
        if (gctl && fixed) {
            v = 0.0;
            for (int m = 0; m < gctl->nc; ++m) {
                const double a1 = gctl->a1[m], a2 = gctl->a2[m];
                const double f2 = __dsub_rn(__dmul_rn(x0, a2), __dmul_rn(x1, a1));
                const double nf =
                    __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a1, a1), __dmul_rn(a2, a2)), __dmul_rn(f2, f2)));
                v = nf > v ? nf : v;
            }
        }
        if (fixed) fixed[i] = (part >= 0 && boundary_values && dist > 0.0) ? __ddiv_rn(dist, v) : 0.0;
    }
}

// Start values (R14): M on free nodes, or the warm start where it is finite
// (AO1); the fixed value on targets; +inf on hard nodes.
template <typename T>
__global__ void k_init3d(int64_t N, const int8_t *__restrict__ code, const double *__restrict__ fixed, T start,
                         T *__restrict__ b0, T *__restrict__ b1, const double *__restrict__ warm) {
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

// Target nodes get back their exact FP64 values (0, or the coarse boundary
// values of R6) after an FP32 solve.
__global__ void k_restore_fixed3(int64_t N, const int8_t *__restrict__ code, const double *__restrict__ fixed,
                                 double *__restrict__ u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (code[i] >= kTargetBase) u[i] = fixed ? fixed[i] : 0.0;
}

// Dirichlet data of Eq. (dbc) in FP32: U_P^(0), the bound 1e6 and above
// (no finite value) mapped to the +inf sentinel.
__global__ void k_narrow_data3(int64_t N, const double *__restrict__ u0, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = u0[i] < kU0Bound ? (float)u0[i] : Num<float>::big();
}

// ------------------------------------------------------------ scheduling --

__global__ void k_schedule3d(Grid3 g, TileSched s, int par, double tol, int launch) {
    const int ntiles = g.ntx * g.nty * g.ntz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    if (t == 0 && s.count_hist) s.count_hist[launch] = s.count[par];
    const bool ran = s.processed[t] != 0;
    if (ran) {
        s.latest[t] ^= 1;
        s.processed[t] = 0;
    }
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    bool act = false;
    for (int dz = -1; dz <= 1 && !act; ++dz)
        for (int dy = -1; dy <= 1 && !act; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int ux = tx + dx, uy = ty + dy, uz = tz + dz;
                if (ux < 0 || uy < 0 || uz < 0 || ux >= g.ntx || uy >= g.nty || uz >= g.ntz) continue;
                if ((par ? s.chg[1] : s.chg[0])[(uz * g.nty + uy) * g.ntx + ux] > tol) {
                    act = true;
                    break;
                }
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

// Tile image in shared memory: u[z][y][x] with a one-node halo.
template <typename T, bool kDir = false> struct Tile3 {
    T u[kT3 + 2][kT3 + 2][kT3 + 3];
    int8_t c[kT3 + 2][kT3 + 2][kT3 + 4];
    T d[kDir ? kT3 + 2 : 1][kDir ? kT3 + 2 : 1][kDir ? kT3 + 3 : 1];   // Dirichlet data (Eq. dbc)
    double red[2];
    T redt[2];          // per-warp maxima of the tile change (type of the values)
};

template <typename T, bool kDir>
__device__ __forceinline__ void load_tile3(const Grid3 &g, const TileSched &s, const int8_t *__restrict__ code,
                                           const T *__restrict__ b0, const T *__restrict__ b1, int x0, int y0, int z0,
                                           Tile3<T, kDir> &sm, const T *__restrict__ dval = nullptr) {
    constexpr int E = kT3 + 2;
    for (int e = threadIdx.x; e < E * E * E; e += blockDim.x) {
        const int lx = e % E, ly = (e / E) % E, lz = e / (E * E);
        const int x = x0 - 1 + lx, y = y0 - 1 + ly, z = z0 - 1 + lz;
        T v = Num<T>::big(), dv = Num<T>::big();
        int8_t cd = kHard;
        if (x < g.n0 && y < g.n1 && z < g.n2) {
            const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
            cd = code[i];
            const int tt = tile_of3(g, x, y, z);
            v = (tt >= 0 && s.latest[tt]) ? b1[i] : b0[i];
            if constexpr (kDir) dv = dval[i];
        }
        sm.u[lz][ly][lx] = v;
        sm.c[lz][ly][lx] = cd;
        if constexpr (kDir) sm.d[lz][ly][lx] = dv;
    }
    __syncthreads();
}

template <typename T, bool kDir>
__device__ __forceinline__ double store_tile3(const Grid3 &g, const TileSched &s, int t, T *__restrict__ b0,
                                             T *__restrict__ b1, int x0, int y0, int z0, Tile3<T, kDir> &sm,
                                             int clamp = 1) {
    const int cur = s.latest[t];
    T *dst = cur ? b0 : b1;
    const T *src = cur ? b1 : b0;
    T mc = 0;
    for (int e = threadIdx.x; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int lx = e % kT3, ly = (e / kT3) % kT3, lz = e / (kT3 * kT3);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
        const T v = sm.u[lz + 1][ly + 1][lx + 1];
        const T o = src[i];
        dst[i] = v;
        const T d = node_change(v, o, clamp);
        mc = d > mc ? d : mc;
    }
    // the tile's maximum in FP64 (an upper bound of the exact change, see node_change)
    return (double)block_max64(mc, sm.redt);
}

// Halo exchange inside a launch of the monotone value sweep: the tile's
// boundary nodes go to the buffer the launch writes, then the 488 halo cells
// are read again as the newer (smaller) of the two buffers.  A neighbour that
// has published shows its progress inside this launch, one that has not its
// older value; either is a value that node held, an upper bound of the fixed
// point, so the decreasing iteration keeps its fixed point (R8).  Ends with a
// block barrier.
template <typename T, bool kDir>
__device__ __forceinline__ void exchange3(const Grid3 &g, const TileSched &s, int t, T *b0, T *b1, int x0, int y0,
                                          int z0, Tile3<T, kDir> &sm) {
    T *dst = s.latest[t] ? b0 : b1;
    for (int e = threadIdx.x; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int lx = e % kT3, ly = (e / kT3) % kT3, lz = e / (kT3 * kT3);
        const bool edge = lx == 0 || lx == kT3 - 1 || ly == 0 || ly == kT3 - 1 || lz == 0 || lz == kT3 - 1;
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (!edge || x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        dst[((int64_t)z * g.n1 + y) * g.n0 + x] = sm.u[lz + 1][ly + 1][lx + 1];
    }
    constexpr int E = kT3 + 2;
    for (int e = threadIdx.x; e < E * E * E; e += blockDim.x) {
        const int lx = e % E, ly = (e / E) % E, lz = e / (E * E);
        const bool halo = lx == 0 || lx == E - 1 || ly == 0 || ly == E - 1 || lz == 0 || lz == E - 1;
        const int x = x0 - 1 + lx, y = y0 - 1 + ly, z = z0 - 1 + lz;
        if (!halo || x < 1 || y < 1 || z < 1 || x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
        const T v0 = __ldcg(b0 + i), v1 = __ldcg(b1 + i);
        const T v = v0 < v1 ? v0 : v1;
        if (v < sm.u[lz][ly][lx]) sm.u[lz][ly][lx] = v;
    }
    __syncthreads();
}

// Local coordinates (1..8) of the node thread `tid` updates at step `st` of
// pass `dir` (0/1: +-x, 2/3: +-y, 4/5: +-z).
__device__ __forceinline__ void plane_node(int dir, int st, int tid, int &lx, int &ly, int &lz) {
    const int s1 = 1 + ((dir & 1) ? (kT3 - 1 - st) : st);
    const int a = 1 + (tid % kT3), b = 1 + (tid / kT3);
    if (dir < 2) { lx = s1; ly = a; lz = b; }
    else if (dir < 4) { lx = a; ly = s1; lz = b; }
    else { lx = a; ly = b; lz = s1; }
}

// --------------------------------------------------------- value sweep 3D --

// One control's weights in shared memory, k[0..6] = kap w_b (b = 1..7) and
// k[7] = kap, aligned so that they load as two (FP32) or four (FP64)
// 16-byte vectors.
template <typename T> struct alignas(16) W3 {
    T k[8];
};

template <typename T> __device__ __forceinline__ void load_w3(const W3<T> &w, T out[8]) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = reinterpret_cast<const float4 *>(w.k)[0], b = reinterpret_cast<const float4 *>(w.k)[1];
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
        out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 a = reinterpret_cast<const double2 *>(w.k)[q];
            out[2 * q] = a.x;
            out[2 * q + 1] = a.y;
        }
    }
}

// Packed FP32 pairs (PTX .f32x2, sm_100 and later): one instruction forms the
// same rounded operation on both halves of a 64-bit register pair.
__device__ __forceinline__ unsigned long long p2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void p2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long p2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long p2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The update of node (lx, ly, lz); mask has bit 9 dz + 3 dy + dx set when the
// neighbour (dx-1, dy-1, dz-1) belongs to the node's patch or target part
// (formed once per launch), everything else reads +inf.  tab: the weights in
// shared memory, in the octant order of ct.
template <typename T, bool kDir, bool kCone = false>
__device__ __forceinline__ T sl_update3(const Tile3<T, kDir> &sm, int lx, int ly, int lz, uint32_t mask, T hh,
                                        const CtlTable3<T> &ct, const W3<T> *tab, const uint64_t *cm = nullptr) {
    T nb[3][3][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                T other;
                if constexpr (kDir) other = sm.d[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx];   // Eq. (dbc)
                else other = Num<T>::big();
                nb[dz][dy][dx] = ((mask >> (9 * dz + 3 * dy + dx)) & 1u) ? sm.u[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx]
                                                                        : other;
            }
    T b0 = Num<T>::big(), b1 = Num<T>::big();
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int sx = (o & 1) ? 2 : 0, sy = (o & 2) ? 2 : 0, sz = (o & 4) ? 2 : 0;
        T c[7];
#pragma unroll
        for (int b = 1; b < 8; ++b) c[b - 1] = nb[(b & 4) ? sz : 1][(b & 2) ? sy : 1][(b & 1) ? sx : 1];
        int m = ct.obeg[o];
        const int me = ct.obeg[o + 1];
        if constexpr (kCone) {
            // the node's cone (AO3): only the controls whose bit is set
            for (; m < me; ++m) {
                if (!((cm[m >> 6] >> (m & 63)) & 1ull)) continue;
                T w0[8];
                load_w3(tab[m], w0);
                T v0 = w0[7] * hh;
#pragma unroll
                for (int b = 0; b < 7; ++b) v0 = fma(w0[b], c[b], v0);
                b0 = v0 < b0 ? v0 : b0;
            }
            continue;
        }
        for (; m + 1 < me; m += 2) {
            T w0[8], w1[8];
            load_w3(tab[m], w0);
            load_w3(tab[m + 1], w1);
            T v0 = w0[7] * hh, v1 = w1[7] * hh;
#pragma unroll
            for (int b = 0; b < 7; ++b) {
                v0 = fma(w0[b], c[b], v0);
                v1 = fma(w1[b], c[b], v1);
            }
            b0 = v0 < b0 ? v0 : b0;
            b1 = v1 < b1 ? v1 : b1;
        }
        if (m < me) {
            T w0[8];
            load_w3(tab[m], w0);
            T v0 = w0[7] * hh;
#pragma unroll
            for (int b = 0; b < 7; ++b) v0 = fma(w0[b], c[b], v0);
            b0 = v0 < b0 ? v0 : b0;
        }
    }
    return b0 < b1 ? b0 : b1;
}

// The same minimum with the controls of an octant two at a time through the
// packed pairs (FP32, no cones), every operation rounded as in sl_update3.
// tab holds, per octant, each pair (m, m + 1) of controls in the slots m and
// m + 1 with their weights interleaved, slot m = (w_m[0], w_m+1[0], w_m[1],
// w_m+1[1]) (w_m[2], ..), slot m + 1 the same for w[4..7] (w[7] = kap), and
// an octant's last control, when its count is odd, plainly as in sl_update3.
template <bool kDir>
__device__ __forceinline__ float sl_update3p(const Tile3<float, kDir> &sm, int lx, int ly, int lz, uint32_t mask,
                                             float hh, const CtlTable3<float> &ct, const W3<float> *tab) {
    float nb[3][3][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                float other;
                if constexpr (kDir) other = sm.d[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx];   // Eq. (dbc)
                else other = Num<float>::big();
                nb[dz][dy][dx] = ((mask >> (9 * dz + 3 * dy + dx)) & 1u) ? sm.u[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx]
                                                                        : other;
            }
    const unsigned long long h2 = p2_pack(hh, hh);
    float b0 = Num<float>::big(), b1 = Num<float>::big();
    const float4 *t4 = reinterpret_cast<const float4 *>(tab);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int sx = (o & 1) ? 2 : 0, sy = (o & 2) ? 2 : 0, sz = (o & 4) ? 2 : 0;
        float c[7];
#pragma unroll
        for (int b = 1; b < 8; ++b) c[b - 1] = nb[(b & 4) ? sz : 1][(b & 2) ? sy : 1][(b & 1) ? sx : 1];
        int m = ct.obeg[o];
        const int me = ct.obeg[o + 1];
        for (; m + 1 < me; m += 2) {
            const float4 q0 = t4[2 * m], q1 = t4[2 * m + 1], q2 = t4[2 * m + 2], q3 = t4[2 * m + 3];
            unsigned long long v = p2_mul(p2_pack(q3.z, q3.w), h2);
            v = p2_fma(p2_pack(q0.x, q0.y), p2_pack(c[0], c[0]), v);
            v = p2_fma(p2_pack(q0.z, q0.w), p2_pack(c[1], c[1]), v);
            v = p2_fma(p2_pack(q1.x, q1.y), p2_pack(c[2], c[2]), v);
            v = p2_fma(p2_pack(q1.z, q1.w), p2_pack(c[3], c[3]), v);
            v = p2_fma(p2_pack(q2.x, q2.y), p2_pack(c[4], c[4]), v);
            v = p2_fma(p2_pack(q2.z, q2.w), p2_pack(c[5], c[5]), v);
            v = p2_fma(p2_pack(q3.x, q3.y), p2_pack(c[6], c[6]), v);
            float v0, v1;
            p2_unpack(v, v0, v1);
            b0 = v0 < b0 ? v0 : b0;
            b1 = v1 < b1 ? v1 : b1;
        }
        if (m < me) {
            float w0[8];
            load_w3(tab[m], w0);
            float v0 = w0[7] * hh;
#pragma unroll
            for (int b = 0; b < 7; ++b) v0 = fmaf(w0[b], c[b], v0);
            b0 = v0 < b0 ? v0 : b0;
        }
    }
    return b0 < b1 ? b0 : b1;
}

// ------------------------------------------- per-node dynamics (Brockett) --

// Brockett's integrator f(x, a) = (a1, a2, x1 a2 - x2 a1) (Sec. 7, R24): the
// foot x + k f/|f| and the step k/|f| depend on the node through (x1, x2)
// only, so the tables hold one row per grid column c = iy n0 + ix and
// control m, at index c nc + m.  Corner b (bits 0..2: a step along x, y, z)
// of the foot's cell lies at the node plus (b0 sx, b1 sy, b2 sz), s = +1 where
// the component of f/|f| is >= 0, and has weight w_b = prod_d (b_d ? t_d :
// 1 - t_d), t = |f|/|f| componentwise; w_0 belongs to the node itself.
struct Gen3 {
    int nc;
    const double4 *dh;       // f/|f| (x, y, z) and h = k/|f| (+inf: a = 0, not admissible)
    const W3<float> *v32;    // k[0..6] = kap w_b (b = 1..7), k[7] = kap h, kap = 1/(1 - w_0)
    const W3<double> *v64;   // the same in FP64
    const W3<float> *p32;    // k[0] = kap, k[b] = kap w_b (b = 1..7): the colour transport
    const uint8_t *oct;      // bit 0..2 set where sx, sy, sz = +1
    const uint32_t *cset;    // positive-weight corners other than the node (bit 9 dz + 3 dy + dx,
                             // offsets dz - 1 ..); 0 when a is not admissible
};

// Literal Q1 weights (w_0 .. w_7) and corner offsets of the foot of the per-node
// control row e (Brockett, R24), in FP64.
__device__ __forceinline__ void gen_weights(const Gen3 &gen, int64_t e, double w[8], int &sx, int &sy, int &sz) {
    const double4 q = gen.dh[e];
    const double t[3] = {fabs(q.x), fabs(q.y), fabs(q.z)};
    sx = q.x >= 0.0 ? 1 : -1;
    sy = q.y >= 0.0 ? 1 : -1;
    sz = q.z >= 0.0 ? 1 : -1;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        double v = 1.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) v *= ((b >> d) & 1) ? t[d] : 1.0 - t[d];
        w[b] = v;
    }
}

// The column tables, formed in FP64 with each operation rounded in the order
// x_d = lo_d + i_d k, f3 = x1 a2 - x2 a1, |f| = sqrt(a1^2 + a2^2 + f3^2).
__global__ void k_gen_table3(Grid3 g, GenCtl gc, double4 *__restrict__ dh, W3<float> *__restrict__ v32,
                             W3<double> *__restrict__ v64, W3<float> *__restrict__ p32, uint8_t *__restrict__ oct,
                             uint32_t *__restrict__ cset) {
    const int64_t total = (int64_t)g.n0 * g.n1 * gc.nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e % gc.nc);
        const int64_t col = e / gc.nc;
        const int ix = (int)(col % g.n0), iy = (int)(col / g.n0);
        const double x0 = __dadd_rn(g.lo0, __dmul_rn((double)ix, g.k));
        const double x1 = __dadd_rn(g.lo1, __dmul_rn((double)iy, g.k));
        const double a1 = gc.a1[m], a2 = gc.a2[m];
        const double f[3] = {a1, a2, __dsub_rn(__dmul_rn(x0, a2), __dmul_rn(x1, a1))};
        const double nf =
            __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(f[0], f[0]), __dmul_rn(f[1], f[1])), __dmul_rn(f[2], f[2])));
        W3<float> w32, q32;
        W3<double> w64;
        if (!(nf > 1e-15)) {
            dh[e] = make_double4(0.0, 0.0, 0.0, (double)INFINITY);
            for (int b = 0; b < 8; ++b) {
                w32.k[b] = 0.f;
                q32.k[b] = 0.f;
                w64.k[b] = 0.0;
            }
            v32[e] = w32;
            v64[e] = w64;
            p32[e] = q32;
            oct[e] = 0;
            cset[e] = 0;
            continue;
        }
        double dv[3], t[3];
        uint8_t o = 0;
        for (int d = 0; d < 3; ++d) {
            const double v = __ddiv_rn(f[d], nf);
            dv[d] = fabs(v) < 1e-15 ? 0.0 : v;
            t[d] = fabs(dv[d]);
            if (dv[d] >= 0.0) o |= (uint8_t)(1u << d);
        }
        const double h = __ddiv_rn(g.k, nf);
        dh[e] = make_double4(dv[0], dv[1], dv[2], h);
        double w[8];
        uint32_t cs = 0;
        for (int b = 0; b < 8; ++b) {
            w[b] = 1.0;
            for (int d = 0; d < 3; ++d) w[b] *= ((b >> d) & 1) ? t[d] : 1.0 - t[d];
            if (b > 0 && w[b] > 0.0) {
                const int dx = (b & 1) ? ((o & 1) ? 1 : -1) : 0, dy = (b & 2) ? ((o & 2) ? 1 : -1) : 0,
                          dz = (b & 4) ? ((o & 4) ? 1 : -1) : 0;
                cs |= 1u << (9 * (dz + 1) + 3 * (dy + 1) + (dx + 1));
            }
        }
        const double kap = 1.0 / (1.0 - w[0]);
        for (int b = 1; b < 8; ++b) {
            w64.k[b - 1] = kap * w[b];
            w32.k[b - 1] = (float)(kap * w[b]);
            q32.k[b] = (float)(kap * w[b]);
        }
        w64.k[7] = kap * h;
        w32.k[7] = (float)(kap * h);
        q32.k[0] = (float)kap;
        v32[e] = w32;
        v64[e] = w64;
        p32[e] = q32;
        oct[e] = o;
        cset[e] = cs;
    }
}

// The update of node (lx, ly, lz) with per-node feet: rows e0 .. e0 + nc - 1
// of the column tables (read through the L1 cache); mask as in sl_update3.
template <typename T, bool kDir>
__device__ __forceinline__ T sl_update3g(const Tile3<T, kDir> &sm, int lx, int ly, int lz, uint32_t mask,
                                         int64_t e0, const Gen3 &gen) {
    const W3<T> *tab;
    if constexpr (sizeof(T) == 4) tab = gen.v32;
    else tab = gen.v64;
    T best = Num<T>::big();
    for (int m = 0; m < gen.nc; ++m) {
        const uint32_t cs = __ldg(&gen.cset[e0 + m]);
        if (!cs) continue;
        if constexpr (!kDir) {
            if (cs & ~mask) continue;   // a positive-weight corner outside the patch: +inf
        }
        const unsigned of = __ldg(&gen.oct[e0 + m]);
        const int sx = (of & 1u) ? 1 : -1, sy = (of & 2u) ? 1 : -1, sz = (of & 4u) ? 1 : -1;
        T w[8];
        load_w3(tab[e0 + m], w);
        T v = w[7];
#pragma unroll
        for (int b = 1; b < 8; ++b) {
            const int dx = (b & 1) ? sx : 0, dy = (b & 2) ? sy : 0, dz = (b & 4) ? sz : 0;
            const int bit = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
            T c;
            if ((mask >> bit) & 1u) c = sm.u[lz + dz][ly + dy][lx + dx];
            else if constexpr (kDir) c = sm.d[lz + dz][ly + dy][lx + dx];   // Eq. (dbc)
            else c = Num<T>::big();
            v = fma(w[b - 1], c, v);
        }
        best = v < best ? v : best;
    }
    return best;
}

// clamp != 0: monotone update from M; clamp == 0: the plain update of the
// warm start (AO1).  kDir: neighbours outside the patch read the Dirichlet
// data dval (Eq. dbc); a node's own pruned nodes (code -2 - patch) read +inf.
// kGen: per-node feet from the column tables of gen (h is then unused).
// kCone: add-on AO3, the minimum over the node's cone (cone, astar).
// kPk (FP32, no kGen or kCone): the packed-pair update of sl_update3p, the
// same results as the scalar one.
// kX: exchange the halo after every pass (exchange3; monotone update only).
template <typename T, bool kDir = false, bool kGen = false, bool kCone = false, bool kPk = false, bool kX = false>
__global__ void __launch_bounds__(kT3n) k_value3d(Grid3 g, const int8_t *__restrict__ code,
                                                  const T *__restrict__ h, T *__restrict__ b0, T *__restrict__ b1,
                                                  TileSched s, int par, int rounds, unsigned long long *updates,
                                                  const CtlTable3<T> ct, int clamp = 1,
                                                  const T *__restrict__ dval = nullptr, const Gen3 gen = Gen3{},
                                                  const Cone3 *__restrict__ cone = nullptr,
                                                  const uint8_t *__restrict__ astar = nullptr) {
    static_assert(!kPk || (sizeof(T) == 4 && !kGen && !kCone), "packed pairs: FP32 control tables only");
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int x0 = 1 + (t % g.ntx) * kT3, y0 = 1 + ((t / g.ntx) % g.nty) * kT3, z0 = 1 + (t / (g.ntx * g.nty)) * kT3;
    __shared__ Tile3<T, kDir> sm;
    // per interior node: neighbour mask (bit 31: the node is free) and h
    __shared__ uint32_t mk[kT3][kT3][kT3];
    __shared__ T hs[kT3][kT3][kT3];
    __shared__ uint8_t as[kCone ? kT3 : 1][kCone ? kT3 : 1][kCone ? kT3 : 1];   // a* per node (AO3)
    __shared__ W3<T> tab[kGen ? 1 : kMaxControls];
    if constexpr (kPk) {
        // slot m: the first (or second) half of the pair (m, m + 1) (or (m - 1, m)),
        // or the octant's odd last control alone
        for (int m = threadIdx.x; m < ct.nc; m += blockDim.x) {
            int o = 0;
            while (ct.obeg[o + 1] <= m) ++o;
            const int r = m - ct.obeg[o];
            float *k = reinterpret_cast<float *>(tab[m].k);
            if ((r & 1) == 0 && m + 1 == ct.obeg[o + 1]) {
                for (int b = 0; b < 7; ++b) k[b] = ct.kw[b][m];
                k[7] = ct.kap[m];
            } else {
                const int m0 = m - (r & 1), half = r & 1;
                for (int q = 0; q < 4; ++q) {
                    const int b = 4 * half + q;
                    k[2 * q] = b < 7 ? ct.kw[b][m0] : ct.kap[m0];
                    k[2 * q + 1] = b < 7 ? ct.kw[b][m0 + 1] : ct.kap[m0 + 1];
                }
            }
        }
    } else if constexpr (!kGen)
        for (int m = threadIdx.x; m < ct.nc; m += blockDim.x) {
            for (int b = 0; b < 7; ++b) tab[m].k[b] = ct.kw[b][m];
            tab[m].k[7] = ct.kap[m];
        }
    load_tile3(g, s, code, b0, b1, x0, y0, z0, sm, dval);   // ends with a block barrier
    const int tid = threadIdx.x;
    int nfree = 0;
    for (int e = tid; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int lx = e % kT3, ly = (e / kT3) % kT3, lz = e / (kT3 * kT3);
        const int8_t cd = sm.c[lz + 1][ly + 1][lx + 1];
        uint32_t m = 0;
        T hv = (T)0;
        if (cd >= 0 && cd < kTargetBase) {
            const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int8_t q = sm.c[lz + dz][ly + dy][lx + dx];
                        m |= (uint32_t)(q == cd || q == tg || q == pr) << (9 * dz + 3 * dy + dx);
                    }
            m |= 0x80000000u;
            ++nfree;
            if constexpr (!kGen) hv = h[((int64_t)(z0 + lz) * g.n1 + (y0 + ly)) * g.n0 + (x0 + lx)];
        }
        if constexpr (kCone) {
            uint8_t a = kNoControl;
            if (m) a = astar[((int64_t)(z0 + lz) * g.n1 + (y0 + ly)) * g.n0 + (x0 + lx)];
            as[lz][ly][lx] = a < cone->nc ? a : (uint8_t)cone->nc;
        }
        mk[lz][ly][lx] = m;
        hs[lz][ly][lx] = hv;
    }
    __syncthreads();
    // AO2: the tile's sweep directions; or alternating halves
    const unsigned tdirs = s.dirs ? s.dirs[t] : (s.alt ? (par ? 0x2Au : 0x15u) : 0x3Fu);
    int pass = 0;
    for (int rd = 0; rd < rounds; ++rd)
        for (int dir = 0; dir < 6; ++dir) {
            if (!((tdirs >> dir) & 1u)) continue;
            if constexpr (kX) {
                if (pass > 0) exchange3(g, s, t, b0, b1, x0, y0, z0, sm);
            }
            ++pass;
            for (int st = 0; st < kT3; ++st) {
                int lx, ly, lz;
                plane_node(dir, st, tid, lx, ly, lz);
                const uint32_t m = mk[lz - 1][ly - 1][lx - 1];
                const bool active = (m & 0x80000000u) != 0;
                T nw = sm.u[lz][ly][lx];
                if (active) {
                    T best;
                    if constexpr (kGen)
                        best = sl_update3g<T, kDir>(sm, lx, ly, lz, m,
                                                    ((int64_t)(y0 + ly - 1) * g.n0 + (x0 + lx - 1)) * gen.nc, gen);
                    else if constexpr (kCone)
                        best = sl_update3<T, kDir, true>(sm, lx, ly, lz, m, hs[lz - 1][ly - 1][lx - 1], ct, tab,
                                                         cone->mask[as[lz - 1][ly - 1][lx - 1]]);
                    else if constexpr (kPk)
                        best = sl_update3p<kDir>(sm, lx, ly, lz, m, hs[lz - 1][ly - 1][lx - 1], ct, tab);
                    else
                        best = sl_update3<T, kDir>(sm, lx, ly, lz, m, hs[lz - 1][ly - 1][lx - 1], ct, tab);
                    if (best < Num<T>::thresh()) nw = clamp ? (best < nw ? best : nw) : best;
                }
                __syncthreads();
                if (active) sm.u[lz][ly][lx] = nw;
                __syncthreads();
            }
        }
    const double mc = store_tile3(g, s, t, b0, b1, x0, y0, z0, sm, clamp);
    nfree = __reduce_add_sync(0xffffffffu, nfree);
    if ((tid & 31) == 0 && updates && nfree)
        atomicAdd(updates, (unsigned long long)nfree * (unsigned long long)__popc(tdirs) * (unsigned long long)rounds);
    if (tid == 0) {
        (par ? s.chg[1] : s.chg[0])[t] = mc;
        s.processed[t] = 1;
    }
}

// ---------------------------------------------------------- reach (S*) 3D --

// dterm (optional): Dirichlet data (Eq. dbc); a node outside the patch with
// finite data is a terminal, like the patch's own target part.
// Union, over the controls whose positive-weight corners other than the node
// all lie in `usable` (27-bit over the 3x3x3 neighbourhood), of those
// corners; 0 when the node has no such control.  (lx, ly, lz): local
// coordinates 1..8 of a node of the tile whose first interior node is
// (x0, y0, .).
template <bool kGen>
__device__ __forceinline__ uint32_t usable_union3(uint32_t usable, int lx, int ly, int lz, int x0, int y0,
                                                  const Grid3 &g, const ReachTable3 &rt, const Gen3 &gen,
                                                  const uint8_t *cu = nullptr) {
    uint32_t c = 0;
    if constexpr (kGen) {
        const int64_t e0 = ((int64_t)(y0 + ly - 1) * g.n0 + (x0 + lx - 1)) * gen.nc;
        for (int m = 0; m < gen.nc; ++m) {
            const uint32_t need = __ldg(&gen.cset[e0 + m]);
            if (need && (need & ~usable) == 0) c |= need;
        }
    } else {
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int ox = (o & 1) ? 2 : 0, oy = (o & 2) ? 2 : 0, oz = (o & 4) ? 2 : 0;
            unsigned us = 0;
#pragma unroll
            for (int b = 1; b < 8; ++b) {
                const int bit = 9 * ((b & 4) ? oz : 1) + 3 * ((b & 2) ? oy : 1) + ((b & 1) ? ox : 1);
                us |= ((usable >> bit) & 1u) << (b - 1);
            }
            const unsigned u = cu ? cu[o * 128 + us] : rt.uni[o][us];
#pragma unroll
            for (int b = 1; b < 8; ++b) {
                const int bit = 9 * ((b & 4) ? oz : 1) + 3 * ((b & 2) ? oy : 1) + ((b & 1) ? ox : 1);
                c |= ((u >> (b - 1)) & 1u) << bit;
            }
        }
    }
    (void)lz;
    return c;
}

// kGen: the corner sets of the per-node feet from the column tables.
template <bool kGen>
// cache, cvalid (optional): the row sets below depend on the codes only, which
// do not change during one reach run, so the first launch that visits a tile
// stores them (29 words per thread) and later ones load them.
__global__ void __launch_bounds__(kT3n) k_reach3d(Grid3 g, const int8_t *__restrict__ code,
                                                  uint8_t *__restrict__ rch, TileSched s, int par, ReachTable3 rt,
                                                  const double *__restrict__ dterm, const Gen3 gen,
                                                  const Cone3 *__restrict__ cone, const uint8_t *__restrict__ astar,
                                                  uint32_t *__restrict__ cache, uint8_t *__restrict__ cvalid) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int x0 = 1 + (t % g.ntx) * kT3, y0 = 1 + ((t / g.ntx) % g.nty) * kT3, z0 = 1 + (t / (g.ntx * g.nty)) * kT3;
    constexpr int E = kT3 + 2;
    __shared__ uint8_t sr[E][E][E + 2];
    __shared__ int8_t sc[E][E][E + 2];
    __shared__ uint8_t sdf[E][E][E + 2];
    __shared__ int flips_s;
    const int tid = threadIdx.x;
    if (tid == 0) flips_s = 0;
    const bool cached = cache && cvalid[t];
    for (int e = tid; e < E * E * E; e += blockDim.x) {
        const int lx = e % E, ly = (e / E) % E, lz = e / (E * E);
        const int x = x0 - 1 + lx, y = y0 - 1 + ly, z = z0 - 1 + lz;
        uint8_t v = 0, df = 0;
        int8_t cd = kHard;
        if (x < g.n0 && y < g.n1 && z < g.n2) {
            const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
            v = rch[i];
            if (!cached) {
                cd = code[i];
                if (dterm) df = dterm[i] < kU0Bound;
            }
        }
        sr[lz][ly][lx] = v;
        sc[lz][ly][lx] = cd;
        sdf[lz][ly][lx] = df;
    }
    __syncthreads();
    // Thread (ly, lz) owns the x-row of the tile at (ly, lz) as a 10-bit set
    // (bit lx, the halo at 0 and 9).  Once per launch (codes do not change):
    // per node the corners that reach it (27 offsets over the 3x3x3
    // neighbourhood), whether one of them is terminal, whether the node is
    // free and unreached, gathered into one row set per offset.
    const int ly = 1 + tid % kT3, lz = 1 + tid / kT3;
    uint32_t cand_b[27];
#pragma unroll
    for (int b = 0; b < 27; ++b) cand_b[b] = 0u;
    uint32_t term_b = 0u, open_b = 0u;
    uint32_t *cl = cache ? cache + (int64_t)t * 29 * kT3n : nullptr;
    if (cached) {
#pragma unroll
        for (int b = 0; b < 27; ++b) cand_b[b] = cl[b * kT3n + tid];
        term_b = cl[27 * kT3n + tid];
        open_b = cl[28 * kT3n + tid];
    } else {
    for (int lx = 1; lx <= kT3; ++lx) {
        const int8_t cd = sc[lz][ly][lx];
        if (cd >= 0 && cd < kTargetBase) {
            const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
            uint32_t same = 0, term = 0;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int8_t q = sc[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx];
                        const int bit = 9 * dz + 3 * dy + dx;
                        same |= (uint32_t)(q == cd) << bit;
                        term |= (uint32_t)(q == tg || (q != cd && q != pr && sdf[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx]))
                                << bit;
                    }
            const uint8_t *cu = nullptr;
            if (cone) {
                const uint8_t a = astar[((int64_t)(z0 + lz - 1) * g.n1 + (y0 + ly - 1)) * g.n0 + (x0 + lx - 1)];
                cu = &cone->uni[a < cone->nc ? a : cone->nc][0][0];
            }
            const uint32_t c = usable_union3<kGen>(same | term, lx, ly, lz, x0, y0, g, rt, gen, cu);
            if (c & term) term_b |= 1u << lx;
            const uint32_t cs = c & same;
#pragma unroll
            for (int b = 0; b < 27; ++b) cand_b[b] |= ((cs >> b) & 1u) << lx;
            open_b |= 1u << lx;
        }
    }
    if (cl) {
#pragma unroll
        for (int b = 0; b < 27; ++b) cl[b * kT3n + tid] = cand_b[b];
        cl[27 * kT3n + tid] = term_b;
        cl[28 * kT3n + tid] = open_b;
        if (tid == 0) cvalid[t] = 1;   // read by later launches only
    }
    }
    // rows as bit sets, double-buffered: the halo rows (ly or lz 0 or 9) in both
    __shared__ uint32_t rows[2][E][E];
    for (int e = tid; e < E * E; e += blockDim.x) {
        const int y = e % E, z = e / E;
        uint32_t v = 0;
#pragma unroll
        for (int x = 0; x < E; ++x) v |= (uint32_t)(sr[z][y][x] != 0) << x;
        rows[0][z][y] = v;
        rows[1][z][y] = v;
    }
    __syncthreads();
    uint32_t R = rows[0][lz][ly];
    const uint32_t R0 = R;
    // Jacobi rounds to the tile's least fixed point for the launch's halo (the
    // one the plane-by-plane Gauss-Seidel passes approach), one barrier each
    int cur = 0;
    for (int it = 0; it <= kT3 * kT3 * kT3; ++it) {
        uint32_t hit = term_b;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const uint32_t src = (dz == 1 && dy == 1) ? R : rows[cur][lz - 1 + dz][ly - 1 + dy];
                const int b = 9 * dz + 3 * dy;
                hit |= cand_b[b] & (src << 1);
                hit |= cand_b[b + 1] & src;
                hit |= cand_b[b + 2] & (src >> 1);
            }
        const uint32_t nr = R | (hit & open_b);
        const int moved = nr != R;
        R = nr;
        rows[cur ^ 1][lz][ly] = R;
        if (!__syncthreads_or(moved)) break;
        cur ^= 1;
    }
    const int flips = __popc(R) - __popc(R0);
#pragma unroll
    for (int lx = 1; lx <= kT3; ++lx) sr[lz][ly][lx] = (uint8_t)((R >> lx) & 1u);
    __syncthreads();
    for (int e = tid; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int lx = e % kT3, ly = (e / kT3) % kT3, lz = e / (kT3 * kT3);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        rch[((int64_t)z * g.n1 + y) * g.n0 + x] = sr[lz + 1][ly + 1][lx + 1];
    }
    if (flips) atomicAdd(&flips_s, flips);
    __syncthreads();
    if (tid == 0) {
        (par ? s.chg[1] : s.chg[0])[t] = flips_s > 0 ? 1.0 : 0.0;
        s.processed[t] = 1;
    }
}

// Peel for S* (R14): a free node none of whose controls has all its
// positive-weight corners in the patch or terminal cannot be in S*; it is
// pruned (code -2 - patch), which may leave a neighbour without a control in
// turn, so the tile repeats Gauss-Seidel passes and the schedule carries the
// removals across tiles.  Codes only move from free to pruned, so a stale
// halo value only delays a removal.  dterm: Dirichlet data, as in k_reach3d.
template <bool kGen>
__global__ void __launch_bounds__(kT3n) k_peel3d(Grid3 g, int8_t *__restrict__ code, TileSched s, int par,
                                                 ReachTable3 rt, const double *__restrict__ dterm, const Gen3 gen,
                                                 const Cone3 *__restrict__ cone, const uint8_t *__restrict__ astar) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int x0 = 1 + (t % g.ntx) * kT3, y0 = 1 + ((t / g.ntx) % g.nty) * kT3, z0 = 1 + (t / (g.ntx * g.nty)) * kT3;
    constexpr int E = kT3 + 2;
    __shared__ int8_t sc[E][E][E + 2];
    __shared__ uint8_t sdf[E][E][E + 2];
    __shared__ int flips_s;
    const int tid = threadIdx.x;
    if (tid == 0) flips_s = 0;
    for (int e = tid; e < E * E * E; e += blockDim.x) {
        const int lx = e % E, ly = (e / E) % E, lz = e / (E * E);
        const int x = x0 - 1 + lx, y = y0 - 1 + ly, z = z0 - 1 + lz;
        uint8_t df = 0;
        int8_t cd = kHard;
        if (x < g.n0 && y < g.n1 && z < g.n2) {
            const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
            cd = code[i];
            if (dterm) df = dterm[i] < kU0Bound;
        }
        sc[lz][ly][lx] = cd;
        sdf[lz][ly][lx] = df;
    }
    __syncthreads();
    int flips = 0;
    for (int dir = 0; dir < 6; ++dir)
        for (int st = 0; st < kT3; ++st) {
            int lx, ly, lz;
            plane_node(dir, st, tid, lx, ly, lz);
            const int8_t cd = sc[lz][ly][lx];
            bool kill = false;
            if (cd >= 0 && cd < kTargetBase && x0 + lx - 1 <= g.n0 - 2 && y0 + ly - 1 <= g.n1 - 2 &&
                z0 + lz - 1 <= g.n2 - 2) {
                const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
                uint32_t usable = 0;
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const int8_t q = sc[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx];
                            const bool u = q == cd || q == tg ||
                                           (q != pr && q != cd && sdf[lz - 1 + dz][ly - 1 + dy][lx - 1 + dx]);
                            usable |= (uint32_t)u << (9 * dz + 3 * dy + dx);
                        }
                const uint8_t *cu = nullptr;
                if (cone) {
                    const uint8_t a = astar[((int64_t)(z0 + lz - 1) * g.n1 + (y0 + ly - 1)) * g.n0 + (x0 + lx - 1)];
                    cu = &cone->uni[a < cone->nc ? a : cone->nc][0][0];
                }
                kill = usable_union3<kGen>(usable, lx, ly, lz, x0, y0, g, rt, gen, cu) == 0;
            }
            __syncthreads();
            if (kill) {
                sc[lz][ly][lx] = (int8_t)(-2 - cd);
                ++flips;
            }
            __syncthreads();
        }
    for (int e = tid; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int lx = e % kT3, ly = (e / kT3) % kT3, lz = e / (kT3 * kT3);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        code[((int64_t)z * g.n1 + y) * g.n0 + x] = sc[lz + 1][ly + 1][lx + 1];
    }
    if (flips) atomicAdd(&flips_s, flips);
    __syncthreads();
    if (tid == 0) {
        (par ? s.chg[1] : s.chg[0])[t] = flips_s > 0 ? 1.0 : 0.0;
        s.processed[t] = 1;
    }
}

template <typename T>
__global__ void k_gather3d(Grid3 g, const uint8_t *__restrict__ latest, const T *__restrict__ b0,
                           const T *__restrict__ b1, T *__restrict__ out_t, double *__restrict__ out64) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(i, g.n0, g.n1, x, y, z);
        const int tt = tile_of3(g, x, y, z);
        const T v = (tt >= 0 && latest[tt]) ? b1[i] : b0[i];
        if (out_t) out_t[i] = v;
        if (out64) out64[i] = v >= Num<T>::thresh() ? (double)INFINITY : (double)v;
    }
}

// Causal sweep directions per tile (AO2 on the tiled iteration, as in 2D):
// information travels against a*, so where at least a fraction frac of the
// tile's feedback has a*_x < 0 the x sweep runs in increasing x only
// (direction 0), where it has a*_x > 0 in decreasing x only (direction 1),
// otherwise both; the same for y (2, 3) and z (4, 5).  With per-node feet
// (gen.nc > 0) the signs are those of the node's f/|f|.
struct DirCtl3 {
    int8_t s[3][kMaxControls];
};

__global__ void __launch_bounds__(kT3n) k_tile_dirs3d(Grid3 g, const int8_t *__restrict__ code,
                                                      const uint8_t *__restrict__ astar, const DirCtl3 dc,
                                                      const Gen3 gen, float frac, uint8_t *__restrict__ dirs) {
    const int t = blockIdx.x;
    const int x0 = 1 + (t % g.ntx) * kT3, y0 = 1 + ((t / g.ntx) % g.nty) * kT3, z0 = 1 + (t / (g.ntx * g.nty)) * kT3;
    __shared__ int cnt[6];
    if (threadIdx.x < 6) cnt[threadIdx.x] = 0;
    __syncthreads();
    int c[6] = {0, 0, 0, 0, 0, 0};   // per axis: count with the component < 0, > 0
    for (int e = threadIdx.x; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int x = x0 + e % kT3, y = y0 + (e / kT3) % kT3, z = z0 + e / (kT3 * kT3);
        if (x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
        const int8_t cd = code[i];
        const uint8_t a = astar[i];
        if (cd < 0 || cd >= kTargetBase || a == kNoControl) continue;
        int sg[3];
        if (gen.nc > 0) {
            const double4 q = gen.dh[((int64_t)y * g.n0 + x) * gen.nc + a];
            sg[0] = q.x > 1e-12 ? 1 : (q.x < -1e-12 ? -1 : 0);
            sg[1] = q.y > 1e-12 ? 1 : (q.y < -1e-12 ? -1 : 0);
            sg[2] = q.z > 1e-12 ? 1 : (q.z < -1e-12 ? -1 : 0);
        } else {
            sg[0] = dc.s[0][a];
            sg[1] = dc.s[1][a];
            sg[2] = dc.s[2][a];
        }
        for (int d = 0; d < 3; ++d) {
            c[2 * d] += sg[d] < 0;
            c[2 * d + 1] += sg[d] > 0;
        }
    }
    for (int k = 0; k < 6; ++k) {
        const int v = __reduce_add_sync(0xffffffffu, c[k]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cnt[k], v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned m = 0;
        for (int d = 0; d < 3; ++d) {
            const int neg = cnt[2 * d], pos = cnt[2 * d + 1], tot = neg + pos;
            if (tot == 0) m |= 3u << (2 * d);
            else if ((float)neg >= frac * (float)tot) m |= 1u << (2 * d);
            else if ((float)pos >= frac * (float)tot) m |= 2u << (2 * d);
            else m |= 3u << (2 * d);
        }
        dirs[t] = (uint8_t)m;
    }
}

// ---------------------------------------------------- Step 2: U_P^(0), a* --

// dlit (optional): the literal interpolation, +inf where a positive-weight
// coarse corner is +inf (the Dirichlet data of Eq. dbc, R16).
// u0f (optional): an FP32 copy of U0 (+inf as the FP32 sentinel) for the
// FP32 filter of the feedback, so that it converts nothing (conversions run
// on the FP64 pipe).
__global__ void k_u0_3d(Grid3 g, Grid3 gc, const int8_t *__restrict__ code, const double *__restrict__ uc,
                        double *__restrict__ u0, double *__restrict__ dlit, float *__restrict__ u0f = nullptr) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c >= kTargetBase) {
            u0[i] = 0.0;
            if (dlit) dlit[i] = 0.0;
            if (u0f) u0f[i] = 0.f;
            continue;
        }
        if (c < 0) {
            u0[i] = Num<double>::big();
            if (dlit) dlit[i] = Num<double>::big();
            if (u0f) u0f[i] = Num<float>::big();
            continue;
        }
        int ix, iy, iz;
        node_xyz(i, g.n0, g.n1, ix, iy, iz);
        const double xi[3] = {(double)ix * (double)(gc.n0 - 1) / (double)(g.n0 - 1),
                              (double)iy * (double)(gc.n1 - 1) / (double)(g.n1 - 1),
                              (double)iz * (double)(gc.n2 - 1) / (double)(g.n2 - 1)};
        const int nn[3] = {gc.n0, gc.n1, gc.n2};
        int bb[3];
        double tt[3];
        for (int d = 0; d < 3; ++d) {
            int b = (int)floor(xi[d]);
            b = min(max(b, 0), nn[d] - 2);
            bb[d] = b;
            tt[d] = xi[d] - b;
        }
        double sum = 0.0;
        bool inf_corner = false;
        for (int cc = 0; cc < 8; ++cc) {
            double w = 1.0;
            for (int d = 0; d < 3; ++d) w *= (cc >> d & 1) ? tt[d] : 1.0 - tt[d];
            if (w > 0.0) {
                const int64_t j = ((int64_t)(bb[2] + (cc >> 2 & 1)) * gc.n1 + (bb[1] + (cc >> 1 & 1))) * gc.n0 + bb[0] +
                                  (cc & 1);
                const double v = uc[j];
                inf_corner |= v >= Num<double>::thresh();
                sum += w * (v >= Num<double>::thresh() ? kU0Bound : v);
            }
        }
        if (dlit) dlit[i] = inf_corner ? Num<double>::big() : sum;
        u0[i] = sum >= kU0Bound ? Num<double>::big() : sum;
        if (u0f) u0f[i] = sum >= kU0Bound ? Num<float>::big() : (float)sum;
    }
}

// Eq. (feedbackcontrol) with literal trilinear weights, lowest index on ties.
// Pass 1 in FP32 over every control finds the minimum up to its rounding;
// pass 2 evaluates in FP64 only the controls whose FP32 value is within
// 2^-17 (h + max |U|) of it (more than twice the FP32 error bound of an
// 8-term convex combination plus h), so the FP64 argmin is the one a full
// FP64 pass finds; exact FP64 ties go to the lowest caller index.
__global__ void k_feedback3d(Grid3 g, const int8_t *__restrict__ code, const double *__restrict__ h,
                             const double *__restrict__ u0, uint8_t *__restrict__ astar,
                             const CtlLit3 *__restrict__ cl, const float *__restrict__ u0f) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    const int64_t sy = g.n0, sz = (int64_t)g.n0 * g.n1;
    // the weights in shared memory, loaded as 16-byte vectors
    __shared__ W3<float> wf[kMaxControls];
    __shared__ W3<double> wd[kMaxControls];
    __shared__ int16_t widx[kMaxControls];
    __shared__ int obeg[9];
    for (int m = threadIdx.x; m < cl->nc; m += blockDim.x) {
        for (int b = 0; b < 8; ++b) {
            wf[m].k[b] = cl->f[b][m];
            wd[m].k[b] = cl->w[b][m];
        }
        widx[m] = cl->idx[m];
    }
    if (threadIdx.x < 9) obeg[threadIdx.x] = cl->obeg[threadIdx.x];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c < 0 || c >= kTargetBase || u0f[i] >= Num<float>::thresh()) {
            astar[i] = kNoControl;
            continue;
        }
        // free nodes are interior, so the 3x3x3 neighbourhood lies in the grid.
        // Only FP32 copies stay live (one conversion each, the finiteness test
        // on the FP32 value: FP64 compares and conversions run at 1/64 rate);
        // the rare FP64 candidates re-read their corners.
        float nf[3][3][3];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float f = u0f[i + (dz - 1) * sz + (dy - 1) * sy + (dx - 1)];
                    nf[dz][dy][dx] = f < Num<float>::thresh() ? f : Num<float>::big();   // U0 is finite below 1e6
                }
        const double hh = h[i];
        const float hf = (float)hh;
        // FP32 evaluation error of a control of octant o: at most 2^-18 (h +
        // max |U0| over its corners); per octant, so that the bound M of U0
        // near the ghost ring (R7) widens only the octants that touch it
        float eo[8];
        float b32 = Num<float>::big(), eb = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int ox = (o & 1) ? 2 : 0, oy = (o & 2) ? 2 : 0, oz = (o & 4) ? 2 : 0;
            float c8[8];
            float am = 0.f;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                c8[b] = nf[(b & 4) ? oz : 1][(b & 2) ? oy : 1][(b & 1) ? ox : 1];
                if (c8[b] < Num<float>::thresh()) am = fmaxf(am, fabsf(c8[b]));
            }
            eo[o] = ldexpf(hf + am, -18);
            for (int m = obeg[o]; m < obeg[o + 1]; ++m) {
                float w[8];
                load_w3(wf[m], w);
                float v = hf;
#pragma unroll
                for (int b = 0; b < 8; ++b) v = fmaf(w[b], c8[b], v);
                if (v < b32) {
                    b32 = v;
                    eb = eo[o];
                }
            }
        }
        double best = Num<double>::big();
        int arg = kNoControl;
        if (b32 < Num<float>::thresh()) {
            // a control can be the FP64 minimum (or tie with it) only if its FP32
            // value minus its bound is at most b32 plus the bound of b32's control
            const float base = b32 + eb;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int ox = (o & 1) ? 2 : 0, oy = (o & 2) ? 2 : 0, oz = (o & 4) ? 2 : 0;
                float c8[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) c8[b] = nf[(b & 4) ? oz : 1][(b & 2) ? oy : 1][(b & 1) ? ox : 1];
                const float lim = base + eo[o];
                for (int m = obeg[o]; m < obeg[o + 1]; ++m) {
                    float w[8];
                    load_w3(wf[m], w);
                    float v32 = hf;
#pragma unroll
                    for (int b = 0; b < 8; ++b) v32 = fmaf(w[b], c8[b], v32);
                    if (v32 > lim) continue;
                    double wdv[8];
                    load_w3(wd[m], wdv);
                    double v = hh;
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int64_t j = i + (int64_t)(((b & 4) ? oz : 1) - 1) * sz +
                                          (int64_t)(((b & 2) ? oy : 1) - 1) * sy + (((b & 1) ? ox : 1) - 1);
                        v += wdv[b] * u0[j];
                    }
                    const int idx = widx[m];
                    if (v < best || (v == best && idx < arg)) {
                        best = v;
                        arg = idx;
                    }
                }
            }
        }
        astar[i] = best < Num<double>::thresh() ? (uint8_t)arg : kNoControl;
    }
}

// Eq. (feedbackcontrol) with per-node feet (Brockett, R24): a* = argmin_a
// { I[U0](x_i + k f/|f|) + k/|f| }, literal Q1 in FP64, lowest index on ties.
__global__ void k_feedback3g(Grid3 g, const int8_t *__restrict__ code, const double *__restrict__ u0,
                             uint8_t *__restrict__ astar, const Gen3 gen) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    const int64_t sy = g.n0, sz = (int64_t)g.n0 * g.n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        if (c < 0 || c >= kTargetBase || u0[i] >= Num<double>::thresh()) {
            astar[i] = kNoControl;
            continue;
        }
        const int64_t e0 = (i % sz) * gen.nc;
        double best = Num<double>::big();
        int arg = kNoControl;
        for (int m = 0; m < gen.nc; ++m) {
            if (!gen.cset[e0 + m]) continue;
            double w[8];
            int sx, sy1, sz1;
            gen_weights(gen, e0 + m, w, sx, sy1, sz1);
            double v = gen.dh[e0 + m].w;
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if (w[b] > 0.0)
                    v += w[b] * u0[i + ((b & 1) ? sx : 0) + ((b & 2) ? sy1 * sy : 0) + ((b & 4) ? sz1 * sz : 0)];
            if (v < best) {
                best = v;
                arg = m;
            }
        }
        astar[i] = best < Num<double>::thresh() ? (uint8_t)arg : kNoControl;
    }
}

// FP64 Jacobi sweep with per-node feet (the polish of Brockett's problem;
// eight controls need no FP32 filter).  Outside the patch: +inf, or the
// Dirichlet data (Eq. dbc).
__global__ void k_polish3g(Grid3 g, const int8_t *__restrict__ code, const double *__restrict__ uin,
                           double *__restrict__ uout, double *maxchg, const double *__restrict__ dval, const Gen3 gen) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    const int64_t sy = g.n0, sz = (int64_t)g.n0 * g.n1;
    double mc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t cd = code[i];
        double v = uin[i];
        if (cd >= 0 && cd < kTargetBase && v < Num<double>::thresh()) {
            const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
            const int64_t e0 = (i % sz) * gen.nc;
            double best = Num<double>::big();
            for (int m = 0; m < gen.nc; ++m) {
                if (!gen.cset[e0 + m]) continue;
                const unsigned of = gen.oct[e0 + m];
                const int64_t ox = (of & 1u) ? 1 : -1, oy = (of & 2u) ? sy : -sy, oz = (of & 4u) ? sz : -sz;
                const W3<double> wt = gen.v64[e0 + m];
                double x = wt.k[7];
#pragma unroll
                for (int b = 1; b < 8; ++b) {
                    const int64_t j = i + ((b & 1) ? ox : 0) + ((b & 2) ? oy : 0) + ((b & 4) ? oz : 0);
                    const int8_t q = code[j];
                    const double cv = (q == cd || q == tg || q == pr) ? uin[j] : (dval ? dval[j] : Num<double>::big());
                    x = fma(wt.k[b - 1], cv, x);
                }
                best = x < best ? x : best;
            }
            if (best < Num<double>::thresh()) {
                mc = fmax(mc, fabs(best - v));
                v = best;
            }
        }
        uout[i] = v;
    }
    mc = warp_max3(mc);
    if ((threadIdx.x & 31) == 0 && mc > 0.0) atomic_max_pos(maxchg, mc);
}

// --------------------------------------------------- Step 3.1: colours phi --

template <int RG>
__global__ void k_phi_init3d(int64_t N, const int8_t *__restrict__ code, int j0, int zero_all,
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

template <int RG, bool kS> struct Phi3Smem {
    float u[RG][kT3 + 2][kT3 + 2][kT3 + 3];
    float src[kS ? RG : 1][kS ? kT3 : 1][kS ? kT3 : 1][kS ? kT3 + 1 : 1];   // correction source only
    int8_t c[kT3 + 2][kT3 + 2][kT3 + 4];
    uint8_t a[kT3][kT3][kT3 + 4];
    // the control table: weights kw[0..7] (two 16-byte vectors) and corner
    // signs (bit 0..2: x, y, z positive) of every control
    float4 tw[kMaxControls][2];
    uint8_t toff[kMaxControls];
    float redf[8];   // per-warp maxima of the tile change
};

// FP32 colour transport (bulk: monotone max from 0; correction: with source).
// kGen: the weights of a node's a* from its column's row of gen.p32.
// The colours are independent linear systems: the block holds one group of
// kT3n threads per colour (up to four groups; eight colours give each group
// two), every group sweeps its own colours behind its own named barrier, so
// the groups never wait on one another inside a pass.
template <int RG> constexpr int phi3_groups() { return RG < 4 ? RG : 4; }

__device__ __forceinline__ void group_sync(int grp) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(kT3n) : "memory");
}

template <int RG, bool kSource, bool kGen = false>
__global__ void __launch_bounds__(kT3n * phi3_groups<RG>()) k_phi3d(Grid3 g, const int8_t *__restrict__ code,
                                                const uint8_t *__restrict__ astar, float *__restrict__ b0,
                                                float *__restrict__ b1, const float *__restrict__ src, TileSched s,
                                                int par, int rounds, const Ctl3 *__restrict__ pc,
                                                const Gen3 gen = Gen3{}) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.count[par ^ 1] = 0;
    if ((int)blockIdx.x >= s.count[par]) return;
    const int t = (par ? s.list[1] : s.list[0])[blockIdx.x];
    const int x0 = 1 + (t % g.ntx) * kT3, y0 = 1 + ((t / g.ntx) % g.nty) * kT3, z0 = 1 + (t / (g.ntx * g.nty)) * kT3;
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    // dynamic shared memory: eight colours with their source exceed the 48 KB
    // of static shared memory
    extern __shared__ __align__(16) unsigned char phi3_smem_raw[];
    Phi3Smem<RG, kSource> &sm = *reinterpret_cast<Phi3Smem<RG, kSource> *>(phi3_smem_raw);
    __shared__ unsigned salive;   // colours nonzero somewhere in the tile image or its source
    constexpr int E = kT3 + 2;
    const int tid = threadIdx.x;
    if (tid == 0) salive = 0u;
    __syncthreads();
    unsigned alive = 0;
    for (int e = tid; e < E * E * E; e += blockDim.x) {
        const int lx = e % E, ly = (e / E) % E, lz = e / (E * E);
        const int x = x0 - 1 + lx, y = y0 - 1 + ly, z = z0 - 1 + lz;
        const bool in = x < g.n0 && y < g.n1 && z < g.n2;
        const bool inner = lx >= 1 && lx <= kT3 && ly >= 1 && ly <= kT3 && lz >= 1 && lz <= kT3;
        const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
        int8_t cd = kHard;
        if (in) {
            cd = code[i];
            const int tt = tile_of3(g, x, y, z);
            const float *bs = (tt >= 0 && s.latest[tt]) ? b1 : b0;
#pragma unroll
            for (int q = 0; q < RG; ++q) {
                const float v = bs[(int64_t)q * N + i];
                sm.u[q][lz][ly][lx] = v;
                alive |= (unsigned)(v != 0.0f) << q;
            }
        } else {
#pragma unroll
            for (int q = 0; q < RG; ++q) sm.u[q][lz][ly][lx] = 0.0f;
        }
        if (inner) {
            sm.a[lz - 1][ly - 1][lx - 1] = in ? astar[i] : kNoControl;
            if (kSource) {
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    const float v = in ? src[(int64_t)q * N + i] : 0.0f;
                    sm.src[q][lz - 1][ly - 1][lx - 1] = v;
                    alive |= (unsigned)(v != 0.0f) << q;
                }
            }
        }
        sm.c[lz][ly][lx] = cd;
    }
    __syncthreads();
    if (alive) atomicOr(&salive, alive);
    if constexpr (!kGen)
        for (int m = tid; m < pc->nc; m += blockDim.x) {
            sm.toff[m] = (uint8_t)((pc->sx[m] > 0 ? 1u : 0u) | (pc->sy[m] > 0 ? 2u : 0u) | (pc->sz[m] > 0 ? 4u : 0u));
            sm.tw[m][0] = make_float4(pc->kw[0][m], pc->kw[1][m], pc->kw[2][m], pc->kw[3][m]);
            sm.tw[m][1] = make_float4(pc->kw[4][m], pc->kw[5][m], pc->kw[6][m], pc->kw[7][m]);
        }
    __syncthreads();
    // a colour that is zero over the whole image stays zero: skip it (uniform per tile)
    const unsigned live = salive;
    // AO2: the tile's sweep directions; or alternating halves
    const unsigned tdirs = s.dirs ? s.dirs[t] : (s.alt ? (par ? 0x2Au : 0x15u) : 0x3Fu);
    constexpr int NG = phi3_groups<RG>(), QPG = RG / NG;   // groups, colours per group
    const int grp = tid / kT3n, gt = tid % kT3n;
    unsigned mine = 0;   // this group's live colours
#pragma unroll
    for (int k = 0; k < QPG; ++k) mine |= live & (1u << (grp + NG * k));
    for (int rd = 0; rd < rounds && mine; ++rd)
        for (int dir = 0; dir < 6; ++dir) {
            if (!((tdirs >> dir) & 1u)) continue;
            for (int st = 0; st < kT3; ++st) {
                int lx, ly, lz;
                plane_node(dir, st, gt, lx, ly, lz);
                const int8_t cd = sm.c[lz][ly][lx];
                const uint8_t a = sm.a[lz - 1][ly - 1][lx - 1];
                const bool active = cd >= 0 && cd < kTargetBase && a != kNoControl;
                float nw[QPG];
                if (active) {
                    unsigned of;
                    float4 w0, w1;
                    if constexpr (kGen) {
                        const int64_t e = ((int64_t)(y0 + ly - 1) * g.n0 + (x0 + lx - 1)) * gen.nc + a;
                        of = __ldg(&gen.oct[e]);
                        const float4 *q = reinterpret_cast<const float4 *>(gen.p32[e].k);
                        w0 = __ldg(q);
                        w1 = __ldg(q + 1);
                    } else {
                        of = sm.toff[a];
                        w0 = sm.tw[a][0];
                        w1 = sm.tw[a][1];
                    }
                    const int sx = (of & 1u) ? 1 : -1, sy = (of & 2u) ? 1 : -1, sz = (of & 4u) ? 1 : -1;
                    const float kw[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int k = 0; k < QPG; ++k) {
                        const int q = grp + NG * k;
                        if (!((mine >> q) & 1u)) {
                            nw[k] = 0.0f;
                            continue;
                        }
                        float v = 0.0f;
#pragma unroll
                        for (int b = 1; b < 8; ++b)
                            v = fmaf(kw[b],
                                     sm.u[q][lz + ((b & 4) ? sz : 0)][ly + ((b & 2) ? sy : 0)][lx + ((b & 1) ? sx : 0)], v);
                        if (kSource) {
                            nw[k] = fmaf(kw[0], sm.src[q][lz - 1][ly - 1][lx - 1], v);
                        } else {
                            const float o = sm.u[q][lz][ly][lx];
                            nw[k] = v > o ? v : o;
                        }
                    }
                }
                group_sync(grp);
                if (active) {
#pragma unroll
                    for (int k = 0; k < QPG; ++k) {
                        const int q = grp + NG * k;
                        if ((mine >> q) & 1u) sm.u[q][lz][ly][lx] = nw[k];
                    }
                }
                group_sync(grp);
            }
        }
    __syncthreads();
    const int cur = s.latest[t];
    float *dst = cur ? b0 : b1;
    const float *old = cur ? b1 : b0;
    float mc = 0.f;
    // predicated and unrolled so that the reads of the previous values overlap;
    // differences rounded upward (an upper bound, no FP64 pipe per node)
#pragma unroll
    for (int k = 0; k < kT3 * kT3 * kT3 / (kT3n * NG); ++k) {
        const int e = tid + k * kT3n * NG;
        const int lx = e % kT3, ly = (e / kT3) % kT3, lz = e / (kT3 * kT3);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (x <= g.n0 - 2 && y <= g.n1 - 2 && z <= g.n2 - 2) {
            const int64_t i = ((int64_t)z * g.n1 + y) * g.n0 + x;
#pragma unroll
            for (int q = 0; q < RG; ++q) {
                const float v = sm.u[q][lz + 1][ly + 1][lx + 1];
                const float o = old[(int64_t)q * N + i];
                dst[(int64_t)q * N + i] = v;
                mc = fmaxf(mc, __fsub_ru(fmaxf(v, o), fminf(v, o)));
            }
        }
    }
    mc = warp_max3(mc);
    if ((tid & 31) == 0) sm.redf[tid >> 5] = mc;
    __syncthreads();
    if (tid == 0) {
        float m = sm.redf[0];
        for (int w = 1; w < kT3n * NG / 32; ++w) m = fmaxf(m, sm.redf[w]);
        (par ? s.chg[1] : s.chg[0])[t] = (double)m;
        s.processed[t] = 1;
    }
}

template <int RG>
__global__ void k_phi_collect3d(Grid3 g, const uint8_t *__restrict__ latest, const float *__restrict__ b0,
                                const float *__restrict__ b1, double *__restrict__ out, int add) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(i, g.n0, g.n1, x, y, z);
        const int tt = tile_of3(g, x, y, z);
        const float *src = (tt >= 0 && latest[tt]) ? b1 : b0;
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const double v = (double)src[(int64_t)q * N + i];
            if (add) out[(int64_t)q * N + i] += v;
            else out[(int64_t)q * N + i] = v;
        }
    }
}

template <int RG, bool kGen = false>
__global__ void k_phi_residual3d(Grid3 g, const int8_t *__restrict__ code, const uint8_t *__restrict__ astar,
                                 const double *__restrict__ phi, float *__restrict__ r32, float *rmax,
                                 const Ctl3 *__restrict__ pc, const Gen3 gen = Gen3{}) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    float mc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t c = code[i];
        const uint8_t a = astar[i];
        if (!(c >= 0 && c < kTargetBase && a != kNoControl)) {
#pragma unroll
            for (int q = 0; q < RG; ++q) r32[(int64_t)q * N + i] = 0.0f;
            continue;
        }
        double w[8];
        int64_t dx, dy, dz;
        if constexpr (kGen) {
            int sx, sy, sz;
            gen_weights(gen, (i % ((int64_t)g.n0 * g.n1)) * gen.nc + a, w, sx, sy, sz);
            dx = sx;
            dy = (int64_t)sy * g.n0;
            dz = (int64_t)sz * g.n0 * g.n1;
        } else {
            for (int b = 0; b < 8; ++b) w[b] = pc->w[b][a];
            dx = pc->sx[a];
            dy = (int64_t)pc->sy[a] * g.n0;
            dz = (int64_t)pc->sz[a] * g.n0 * g.n1;
        }
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const double *f = phi + (int64_t)q * N;
            double v = 0.0;
            for (int b = 0; b < 8; ++b)
                v += w[b] * f[i + ((b & 1) ? dx : 0) + ((b & 2) ? dy : 0) + ((b & 4) ? dz : 0)];
            const double r = v - f[i];
            r32[(int64_t)q * N + i] = (float)r;
            mc = fmaxf(mc, (float)fabs(r));
        }
    }
    mc = warp_max3(mc);
    if ((threadIdx.x & 31) == 0 && mc > 0.f) atomic_max_pos(rmax, mc);
}

// Remark 3.1 fill round (R12), axis neighbours in increasing node index.
__global__ void k_fill3d(Grid3 g, const int8_t *__restrict__ lin, int8_t *__restrict__ lout,
                         unsigned long long *changed) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    const int64_t sy = g.n0, sz = (int64_t)g.n0 * g.n1;
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int8_t v = lin[i];
        if (v == -2) {
            int ix, iy, iz;
            node_xyz(i, g.n0, g.n1, ix, iy, iz);
            int8_t nv = -2;
            if (iz > 0 && lin[i - sz] >= 0) nv = lin[i - sz];
            else if (iy > 0 && lin[i - sy] >= 0) nv = lin[i - sy];
            else if (ix > 0 && lin[i - 1] >= 0) nv = lin[i - 1];
            else if (ix < g.n0 - 1 && lin[i + 1] >= 0) nv = lin[i + 1];
            else if (iy < g.n1 - 1 && lin[i + sy] >= 0) nv = lin[i + sy];
            else if (iz < g.n2 - 1 && lin[i + sz] >= 0) nv = lin[i + sz];
            if (nv >= 0) { v = nv; ++cnt; }
        }
        lout[i] = v;
    }
    cnt = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(changed, cnt);
}

// Patch compaction: per-tile patch masks, per-patch node and tile counts.
__global__ void __launch_bounds__(kT3n) k_compact3d(Grid3 g, const int8_t *__restrict__ code,
                                                    uint64_t *__restrict__ tile_patch,
                                                    unsigned long long *__restrict__ patch_nodes,
                                                    unsigned long long *__restrict__ patch_tiles,
                                                    int *__restrict__ tile_cnt, int R) {
    const int t = blockIdx.x;
    const int x0 = 1 + (t % g.ntx) * kT3, y0 = 1 + ((t / g.ntx) % g.nty) * kT3, z0 = 1 + (t / (g.ntx * g.nty)) * kT3;
    __shared__ unsigned long long mask_s;
    __shared__ int cnt_s[kMaxTargets];
    if (threadIdx.x == 0) mask_s = 0;
    for (int j = threadIdx.x; j < kMaxTargets; j += blockDim.x) cnt_s[j] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < kT3 * kT3 * kT3; e += blockDim.x) {
        const int x = x0 + e % kT3, y = y0 + (e / kT3) % kT3, z = z0 + e / (kT3 * kT3);
        if (x > g.n0 - 2 || y > g.n1 - 2 || z > g.n2 - 2) continue;
        const int8_t c = code[((int64_t)z * g.n1 + y) * g.n0 + x];
        if (c >= 0 && c < kTargetBase) {
            atomicOr(&mask_s, 1ull << c);
            atomicAdd(&cnt_s[c], 1);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kMaxTargets; j += blockDim.x)
        if (cnt_s[j]) {
            atomicAdd(&patch_nodes[j], (unsigned long long)cnt_s[j]);
            atomicAdd(&patch_tiles[j], 1ull);
            if (j < R) tile_cnt[(int64_t)t * R + j] = cnt_s[j];
        }
    if (threadIdx.x == 0) tile_patch[t] = mask_s;
}

// FP64 polish with the FP32 filter (see k_polish2d): margin 2^-17 (h + max|a|)
// covers the eight-term trilinear sum.
// cone (AO3): the minimum over the node's cone of astar.
__global__ void k_polish3d(Grid3 g, const int8_t *__restrict__ code, const double *__restrict__ h,
                           const double *__restrict__ uin, double *__restrict__ uout, double *maxchg,
                           const CtlTable3<float> c32, const CtlTable3<double> c64,
                           const double *__restrict__ dval, const Cone3 *__restrict__ cone = nullptr,
                           const uint8_t *__restrict__ astar = nullptr) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    // the weights in shared memory (k[0..6] = kap w_b, k[7] = kap), 16-byte vectors
    __shared__ W3<float> t32[kMaxControls];
    __shared__ W3<double> t64[kMaxControls];
    for (int m = threadIdx.x; m < c32.nc; m += blockDim.x) {
        for (int b = 0; b < 7; ++b) {
            t32[m].k[b] = c32.kw[b][m];
            t64[m].k[b] = c64.kw[b][m];
        }
        t32[m].k[7] = c32.kap[m];
        t64[m].k[7] = c64.kap[m];
    }
    __syncthreads();
    double mc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int8_t cd = code[i];
        double v = uin[i];
        if (cd >= 0 && cd < kTargetBase) {
            int ix, iy, iz;
            node_xyz(i, g.n0, g.n1, ix, iy, iz);
            const int8_t tg = (int8_t)(cd + kTargetBase), pr = (int8_t)(-2 - cd);
            // only FP32 copies and masks stay live (FP64 compares and conversions
            // run at 1/64 rate); FP64 candidates re-read their corners.  Outside
            // the patch: +inf, or the Dirichlet data (Eq. dbc).
            float nf[3][3][3];
            uint32_t use = 0, fromd = 0;
            float amax = 0.f;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int64_t j = ((int64_t)(iz - 1 + dz) * g.n1 + (iy - 1 + dy)) * g.n0 + (ix - 1 + dx);
                        const int8_t q = code[j];
                        const bool same = q == cd || q == tg || q == pr;
                        const float f = same ? (float)uin[j] : (dval ? (float)dval[j] : Num<float>::big());
                        const bool fin = f < Num<float>::thresh();
                        nf[dz][dy][dx] = fin ? f : Num<float>::big();
                        use |= (uint32_t)fin << (9 * dz + 3 * dy + dx);
                        fromd |= (uint32_t)(!same) << (9 * dz + 3 * dy + dx);
                        if (fin) amax = fmaxf(amax, fabsf(f));
                    }
            const double hh = h[i];
            const float hf = (float)hh;
            const uint64_t *cm = nullptr;
            if (cone) {
                const uint8_t a = astar[i];
                cm = cone->mask[a < cone->nc ? a : cone->nc];
            }
            float b32 = Num<float>::big();
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int sx = (o & 1) ? 2 : 0, sy = (o & 2) ? 2 : 0, sz = (o & 4) ? 2 : 0;
                float c[7];
#pragma unroll
                for (int b = 1; b < 8; ++b) c[b - 1] = nf[(b & 4) ? sz : 1][(b & 2) ? sy : 1][(b & 1) ? sx : 1];
                for (int m = c32.obeg[o]; m < c32.obeg[o + 1]; ++m) {
                    if (cm && !((cm[m >> 6] >> (m & 63)) & 1ull)) continue;
                    float t[8];
                    load_w3(t32[m], t);
                    float w = t[7] * hf;
#pragma unroll
                    for (int b = 0; b < 7; ++b) w = fmaf(t[b], c[b], w);
                    b32 = w < b32 ? w : b32;
                }
            }
            if (b32 < Num<float>::thresh() && v < Num<double>::thresh()) {
                const float lim = b32 + ldexpf(hf + amax, -17);
                double best = Num<double>::big();
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const int sx = (o & 1) ? 2 : 0, sy = (o & 2) ? 2 : 0, sz = (o & 4) ? 2 : 0;
                    float c[7];
#pragma unroll
                    for (int b = 1; b < 8; ++b) c[b - 1] = nf[(b & 4) ? sz : 1][(b & 2) ? sy : 1][(b & 1) ? sx : 1];
                    for (int m = c32.obeg[o]; m < c32.obeg[o + 1]; ++m) {
                        if (cm && !((cm[m >> 6] >> (m & 63)) & 1ull)) continue;
                        float t[8];
                        load_w3(t32[m], t);
                        float w = t[7] * hf;
#pragma unroll
                        for (int b = 0; b < 7; ++b) w = fmaf(t[b], c[b], w);
                        if (w <= lim) {
                            double td[8];
                            load_w3(t64[m], td);
                            double x = td[7] * hh;
#pragma unroll
                            for (int b = 1; b < 8; ++b) {
                                const int ddz = (b & 4) ? sz : 1, ddy = (b & 2) ? sy : 1, ddx = (b & 1) ? sx : 1;
                                const int64_t j =
                                    ((int64_t)(iz - 1 + ddz) * g.n1 + (iy - 1 + ddy)) * g.n0 + (ix - 1 + ddx);
                                const int bit = 9 * ddz + 3 * ddy + ddx;
                                const double cv = ((use >> bit) & 1u) ? (((fromd >> bit) & 1u) ? dval[j] : uin[j])
                                                                      : Num<double>::big();
                                x = fma(td[b - 1], cv, x);
                            }
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
    mc = warp_max3(mc);
    if ((threadIdx.x & 31) == 0 && mc > 0.0) atomic_max_pos(maxchg, mc);
}

// ======================================================================
// Host driver of the 3D path
// ======================================================================
namespace {

constexpr int kReachCap3 = 1 << 18;

inline int grid_for3(int64_t n, int bs = 256) {
    int64_t b = (n + bs - 1) / bs;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

template <typename T> T *alloc3(hjbp_plan &p, int64_t n) {
    return static_cast<T *>(p.dev_alloc(sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
}

__global__ void k_iota3(int n, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

struct Sched3 {
    TileSched d{};
    int ntiles = 0;
    int hist = 0;
    int *iota = nullptr;
};

Sched3 make_sched3(hjbp_plan &p, const Grid3 &g, int hist) {
    Sched3 s;
    s.ntiles = g.ntx * g.nty * g.ntz;
    s.hist = hist;
    const int nt = std::max(1, s.ntiles);
    s.d.list[0] = alloc3<int>(p, nt);
    s.d.list[1] = alloc3<int>(p, nt);
    s.d.count = alloc3<int>(p, 2);
    s.d.chg[0] = alloc3<double>(p, nt);
    s.d.chg[1] = alloc3<double>(p, nt);
    s.d.latest = alloc3<uint8_t>(p, nt);
    s.d.processed = alloc3<uint8_t>(p, nt);
    s.d.tile_patch = nullptr;
    s.d.patch_hist = alloc3<uint64_t>(p, hist);
    s.d.res_hist = alloc3<double>(p, hist);
    s.d.count_hist = alloc3<int>(p, hist);
    s.iota = alloc3<int>(p, nt);
    k_iota3<<<grid_for3(nt), 256, 0, p.stream>>>(nt, s.iota);
    ++p.stats.kernel_launches;
    return s;
}

struct Run3 {
    int64_t tile_visits = 0;
    int launches = 0;
    bool converged = false;
    double last_res = 0.0;
};

template <class Sweep> Run3 run_tiles3(hjbp_plan &p, const Grid3 &g, Sched3 &s, double tol, int cap, Sweep sweep) {
    Run3 rr;
    if (s.ntiles == 0) {
        rr.converged = true;
        return rr;
    }
    cudaStream_t st = p.stream;
    const int nt = s.ntiles;
    check_cuda(cudaMemcpyAsync(s.d.list[0], s.iota, sizeof(int) * nt, cudaMemcpyDeviceToDevice, st), "reset");
    const int counts[2] = {nt, 0};
    check_cuda(cudaMemcpyAsync(s.d.count, counts, sizeof(counts), cudaMemcpyHostToDevice, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.chg[0], 0, sizeof(double) * nt, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.chg[1], 0, sizeof(double) * nt, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.latest, 0, nt, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.processed, 0, nt, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.patch_hist, 0, sizeof(uint64_t) * s.hist, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.res_hist, 0, sizeof(double) * s.hist, st), "reset");
    check_cuda(cudaMemsetAsync(s.d.count_hist, 0, sizeof(int) * s.hist, st), "reset");
    check_cuda(cudaStreamSynchronize(st), "reset sync");
    cap = std::min(cap, s.hist);
    int par = 0, L = 0, check_every = 4;
    while (L < cap) {
        sweep(par);
        check_cuda(cudaGetLastError(), "sweep3 launch");
        k_schedule3d<<<(nt + 255) / 256, 256, 0, st>>>(g, s.d, par, tol, L);
        ++p.stats.kernel_launches;
        par ^= 1;
        ++L;
        if (L % check_every == 0 || L == cap) {
            if (!p.pinned_count) check_cuda(cudaMallocHost(&p.pinned_count, sizeof(int)), "pinned");
            check_cuda(cudaMemcpyAsync(p.pinned_count, s.d.count + par, sizeof(int), cudaMemcpyDeviceToHost, st),
                       "count");
            check_cuda(cudaStreamSynchronize(st), "sweep3 sync");
            if (*p.pinned_count == 0) {
                rr.converged = true;
                break;
            }
            check_every = std::min(check_every * 2, 16);
        }
    }
    std::vector<int> ch(L);
    std::vector<double> rh(L);
    if (L) {
        check_cuda(cudaMemcpyAsync(ch.data(), s.d.count_hist, sizeof(int) * L, cudaMemcpyDeviceToHost, st), "hist");
        check_cuda(cudaMemcpyAsync(rh.data(), s.d.res_hist, sizeof(double) * L, cudaMemcpyDeviceToHost, st), "hist");
        check_cuda(cudaStreamSynchronize(st), "hist sync");
    }
    for (int l = 0; l < L; ++l)
        if (ch[l] > 0) {
            rr.launches = l + 1;
            rr.last_res = rh[l];
            rr.tile_visits += ch[l];
        }
    return rr;
}

template <typename T> CtlTable3<T> make_table3(const hjbp_plan &p) {
    CtlTable3<T> ct;
    std::memset(&ct, 0, sizeof(ct));
    const int nc = p.desc.n_controls;
    ct.nc = nc;
    int pos = 0;
    for (int o = 0; o < 8; ++o) {
        ct.obeg[o] = pos;
        for (int m = 0; m < nc; ++m) {
            const double *a = &p.controls[3 * m];
            const int oo = (a[0] >= 0.0 ? 1 : 0) + (a[1] >= 0.0 ? 2 : 0) + (a[2] >= 0.0 ? 4 : 0);
            if (oo != o) continue;
            const double b[3] = {std::fabs(a[0]), std::fabs(a[1]), std::fabs(a[2])};
            double w[8];
            for (int c = 0; c < 8; ++c) {
                w[c] = 1.0;
                for (int d = 0; d < 3; ++d) w[c] *= (c >> d & 1) ? b[d] : 1.0 - b[d];
            }
            const double kap = 1.0 / (1.0 - w[0]);
            for (int c = 1; c < 8; ++c) ct.kw[c - 1][pos] = (T)(kap * w[c]);
            ct.kap[pos] = (T)kap;
            ++pos;
        }
    }
    ct.obeg[8] = pos;
    return ct;
}

Ctl3 make_ctl3(const hjbp_plan &p) {
    Ctl3 c;
    std::memset(&c, 0, sizeof(c));
    c.nc = p.desc.n_controls;
    for (int m = 0; m < c.nc; ++m) {
        const double *a = &p.controls[3 * m];
        c.sx[m] = a[0] >= 0.0 ? 1 : -1;
        c.sy[m] = a[1] >= 0.0 ? 1 : -1;
        c.sz[m] = a[2] >= 0.0 ? 1 : -1;
        const double b[3] = {std::fabs(a[0]), std::fabs(a[1]), std::fabs(a[2])};
        double w[8];
        for (int cc = 0; cc < 8; ++cc) {
            w[cc] = 1.0;
            for (int d = 0; d < 3; ++d) w[cc] *= (cc >> d & 1) ? b[d] : 1.0 - b[d];
            c.w[cc][m] = w[cc];
        }
        const double kap = 1.0 / (1.0 - w[0]);
        c.kw[0][m] = (float)kap;
        for (int cc = 1; cc < 8; ++cc) c.kw[cc][m] = (float)(kap * w[cc]);
    }
    return c;
}

CtlLit3 make_lit3(const hjbp_plan &p) {
    CtlLit3 c;
    std::memset(&c, 0, sizeof(c));
    c.nc = p.desc.n_controls;
    int pos = 0;
    for (int o = 0; o < 8; ++o) {
        c.obeg[o] = pos;
        for (int m = 0; m < c.nc; ++m) {
            const double *a = &p.controls[3 * m];
            if ((a[0] >= 0.0 ? 1 : 0) + (a[1] >= 0.0 ? 2 : 0) + (a[2] >= 0.0 ? 4 : 0) != o) continue;
            const double b[3] = {std::fabs(a[0]), std::fabs(a[1]), std::fabs(a[2])};
            for (int cc = 0; cc < 8; ++cc) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) w *= (cc >> d & 1) ? b[d] : 1.0 - b[d];
                c.w[cc][pos] = w;
                c.f[cc][pos] = (float)w;
            }
            c.idx[pos] = (int16_t)m;
            ++pos;
        }
    }
    c.obeg[8] = pos;
    return c;
}

ReachTable3 make_reach3(const hjbp_plan &p) {
    ReachTable3 rt;
    std::memset(&rt, 0, sizeof(rt));
    for (int m = 0; m < p.desc.n_controls; ++m) {
        const double *a = &p.controls[3 * m];
        const int o = (a[0] >= 0.0 ? 1 : 0) + (a[1] >= 0.0 ? 2 : 0) + (a[2] >= 0.0 ? 4 : 0);
        const double b[3] = {std::fabs(a[0]), std::fabs(a[1]), std::fabs(a[2])};
        unsigned need = 0;
        for (int c = 1; c < 8; ++c) {
            double w = 1.0;
            for (int d = 0; d < 3; ++d) w *= (c >> d & 1) ? b[d] : 1.0 - b[d];
            if (w > 0.0) need |= 1u << (c - 1);
        }
        if (need) rt.present[o][need >> 5] |= 1u << (need & 31);
    }
    for (int o = 0; o < 8; ++o)
        for (unsigned us = 0; us < 128; ++us) {
            unsigned u = 0;
            for (unsigned m = 1; m < 128; ++m)
                if (((rt.present[o][m >> 5] >> (m & 31)) & 1u) && (m & ~us) == 0) u |= m;
            rt.uni[o][us] = (uint8_t)u;
        }
    return rt;
}

// The cones of AO3 (R19) over the octant-sorted control table; returns the
// mean cone size.
double make_cones3(const hjbp_plan &p, Cone3 &cn) {
    std::memset(&cn, 0, sizeof(cn));
    const int nc = p.desc.n_controls;
    cn.nc = nc;
    std::vector<int> pos(nc);
    std::vector<int> oct(nc);
    std::vector<unsigned> need(nc);
    int at = 0;
    for (int o = 0; o < 8; ++o)
        for (int m = 0; m < nc; ++m) {
            const double *a = &p.controls[3 * m];
            if ((a[0] >= 0.0 ? 1 : 0) + (a[1] >= 0.0 ? 2 : 0) + (a[2] >= 0.0 ? 4 : 0) != o) continue;
            pos[m] = at++;
            oct[m] = o;
            const double b[3] = {std::fabs(a[0]), std::fabs(a[1]), std::fabs(a[2])};
            unsigned nd = 0;
            for (int c = 1; c < 8; ++c) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) w *= (c >> d & 1) ? b[d] : 1.0 - b[d];
                if (w > 0.0) nd |= 1u << (c - 1);
            }
            need[m] = nd;
        }
    const double cr = std::cos(3.14159265358979323846 / p.desc.reduce_r) - 1e-12;
    double total = 0.0;
    for (int a = 0; a <= nc; ++a) {
        uint32_t present[8][4];
        std::memset(present, 0, sizeof(present));
        int cnt = 0;
        for (int m = 0; m < nc; ++m) {
            if (a < nc) {
                double dot = 0.0;
                for (int d = 0; d < 3; ++d) dot += p.controls[3 * m + d] * p.controls[3 * a + d];
                if (!(dot >= cr)) continue;
            }
            cn.mask[a][pos[m] >> 6] |= 1ull << (pos[m] & 63);
            ++cnt;
            if (need[m]) present[oct[m]][need[m] >> 5] |= 1u << (need[m] & 31);
        }
        for (int o = 0; o < 8; ++o)
            for (unsigned us = 0; us < 128; ++us) {
                unsigned u = 0;
                for (unsigned k = 1; k < 128; ++k)
                    if (((present[o][k >> 5] >> (k & 31)) & 1u) && (k & ~us) == 0) u |= k;
                cn.uni[a][o][us] = (uint8_t)u;
            }
        if (a < nc) total += cnt;
    }
    return total / nc;
}

Grid3 make_grid3(const int n[3], const double lo[3], double k) {
    Grid3 g;
    g.n0 = n[0];
    g.n1 = n[1];
    g.n2 = n[2];
    g.ntx = (n[0] - 2 + kT3 - 1) / kT3;
    g.nty = (n[1] - 2 + kT3 - 1) / kT3;
    g.ntz = (n[2] - 2 + kT3 - 1) / kT3;
    g.lo0 = lo[0];
    g.lo1 = lo[1];
    g.lo2 = lo[2];
    g.k = k;
    return g;
}

struct Ev3 {
    cudaEvent_t e;
    explicit Ev3(cudaStream_t s) {
        check_cuda(cudaEventCreate(&e), "event");
        check_cuda(cudaEventRecord(e, s), "event");
    }
    ~Ev3() { cudaEventDestroy(e); }
};

float ms3(const Ev3 &a, const Ev3 &b) {
    float ms = 0.f;
    cudaEventSynchronize(b.e);
    cudaEventElapsedTime(&ms, a.e, b.e);
    return ms;
}

int reach3(hjbp_plan &p, const Grid3 &g, int8_t *code, uint8_t *rch, Sched3 &s, int64_t N,
           const double *dterm = nullptr, const Gen3 *gen = nullptr, const Cone3 *cone = nullptr) {
    const ReachTable3 rt = make_reach3(p);
    unsigned long long *removed = alloc3<unsigned long long>(p, 1);
    // per tile the candidate, terminal and free row sets of k_reach3d (29 words per thread)
    uint32_t *rcache = alloc3<uint32_t>(p, (int64_t)std::max(1, s.ntiles) * 29 * kT3n);
    uint8_t *rvalid = alloc3<uint8_t>(p, std::max(1, s.ntiles));
    int total = 0;
    // each round prunes at least one node or ends the loop, so it ends after at
    // most N rounds
    for (int64_t round = 0;; ++round) {
        if (round > N) throw HjbpError{HJBP_ECUDA, "reachability pruning did not settle"};
        // peel the nodes left without any control first (they cannot be in S*)
        Run3 pe = run_tiles3(p, g, s, 0.5f, kReachCap3, [&](int par) {
            if (gen) k_peel3d<true><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, s.d, par, rt, dterm, *gen, cone, p.astar);
            else k_peel3d<false><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, s.d, par, rt, dterm, Gen3{}, cone, p.astar);
            ++p.stats.kernel_launches;
        });
        total += pe.launches;
        if (!pe.converged) throw HjbpError{HJBP_ECUDA, "peeling did not settle"};
        check_cuda(cudaMemsetAsync(rch, 0, (size_t)N, p.stream), "reach reset");
        // the codes changed (peel, prune): the tiles' cached row sets are stale
        check_cuda(cudaMemsetAsync(rvalid, 0, (size_t)std::max(1, s.ntiles), p.stream), "reach cache reset");
        Run3 rr = run_tiles3(p, g, s, 0.5f, kReachCap3, [&](int par) {
            if (gen)
                k_reach3d<true><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, rch, s.d, par, rt, dterm, *gen, cone, p.astar,
                                                                 rcache, rvalid);
            else
                k_reach3d<false><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, rch, s.d, par, rt, dterm, Gen3{}, cone,
                                                                  p.astar, rcache, rvalid);
            ++p.stats.kernel_launches;
        });
        total += rr.launches;
        if (!rr.converged) throw HjbpError{HJBP_ECUDA, "reachability sweep did not settle"};
        check_cuda(cudaMemsetAsync(removed, 0, sizeof(unsigned long long), p.stream), "memset");
        k_reach_prune<<<grid_for3(N), 256, 0, p.stream>>>(N, code, rch, removed);
        ++p.stats.kernel_launches;
        unsigned long long h = 0;
        check_cuda(cudaMemcpyAsync(&h, removed, sizeof(h), cudaMemcpyDeviceToHost, p.stream), "removed");
        check_cuda(cudaStreamSynchronize(p.stream), "reach sync");
        if (h == 0) break;
    }
    return total;
}

// dval: Dirichlet data (Eq. dbc) or NULL; warm: start values of AO1 or NULL
// (then the plain update instead of the monotone one).
template <typename T>
Run3 value3(hjbp_plan &p, const Grid3 &g, const int8_t *code, const T *h, T *b0, T *b1, Sched3 &s, double tol,
            int cap, int rounds, T *out_t, double *out64, unsigned long long *updates, const T *dval = nullptr,
            const double *warm = nullptr, const double *fixed = nullptr, const Gen3 *gen = nullptr,
            const Cone3 *cone = nullptr) {
    const int64_t N = (int64_t)g.n0 * g.n1 * g.n2;
    k_init3d<T><<<grid_for3(N), 256, 0, p.stream>>>(N, code, fixed, (T)kStartValue, b0, b1, warm);
    const int clamp = warm ? 0 : 1;
    ++p.stats.kernel_launches;
    const CtlTable3<T> ct = make_table3<T>(p);
    const bool timed = (p.desc.flags & HJBP_FLAG_TIME_SWEEPS) != 0;
    // FP32: controls two at a time as packed pairs (same results); tune[6] = 2: one at a time
    const bool packed = std::is_same<T, float>::value && p.desc.tune[6] != 2;
    // FP32 monotone sweeps exchange their halos after every pass (tune[7] = 1: block-Jacobi)
    const bool xchg = std::is_same<T, float>::value && clamp && p.desc.tune[7] != 1;
    constexpr bool kF = std::is_same<T, float>::value;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
    Run3 rr = run_tiles3(p, g, s, tol, cap, [&](int par) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (timed) {
            // events from the plan's pool (created once, reused by every solve)
            a = p.pooled_event();
            b = p.pooled_event();
            if (!a || !b) throw HjbpError{HJBP_ECUDA, "cudaEventCreate failed"};
            check_cuda(cudaEventRecord(a, p.stream), "event");
        }
        if (cone && dval)
            k_value3d<T, true, false, true><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval, Gen3{}, cone, p.astar);
        else if (cone)
            k_value3d<T, false, false, true><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, nullptr, Gen3{}, cone, p.astar);
        else if (gen && dval)
            k_value3d<T, true, true><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates,
                                                                       ct, clamp, dval, *gen);
        else if (gen)
            k_value3d<T, false, true><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates,
                                                                        ct, clamp, nullptr, *gen);
        else if (dval && packed && xchg)
            k_value3d<T, true, false, false, kF, kF><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (packed && xchg)
            k_value3d<T, false, false, false, kF, kF><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, nullptr);
        else if (dval && xchg)
            k_value3d<T, true, false, false, false, kF><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (xchg)
            k_value3d<T, false, false, false, false, kF><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, nullptr);
        else if (dval && packed)
            k_value3d<T, true, false, false, std::is_same<T, float>::value><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, dval);
        else if (dval)
            k_value3d<T, true><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                 clamp, dval);
        else if (packed)
            k_value3d<T, false, false, false, std::is_same<T, float>::value><<<s.ntiles, kT3n, 0, p.stream>>>(
                g, code, h, b0, b1, s.d, par, rounds, updates, ct, clamp, nullptr);
        else
            k_value3d<T, false><<<s.ntiles, kT3n, 0, p.stream>>>(g, code, h, b0, b1, s.d, par, rounds, updates, ct,
                                                                  clamp, nullptr);
        ++p.stats.kernel_launches;
        ++p.stats.sweep_kernel_launches;
        if (timed) {
            check_cuda(cudaEventRecord(b, p.stream), "event");
            evs.emplace_back(a, b);
        }
    });
    p.stats.sweep_tile_visits += rr.tile_visits;
    if (timed) {
        check_cuda(cudaStreamSynchronize(p.stream), "timing sync");
        double ms = 0.0;
        for (size_t l = 0; l < evs.size(); ++l) {
            float m = 0.f;
            if ((int)l < rr.launches) {
                cudaEventElapsedTime(&m, evs[l].first, evs[l].second);
                ms += m;
            }
        }
        p.stats.ms_sweep_kernel += ms;
    }
    k_gather3d<T><<<grid_for3(N), 256, 0, p.stream>>>(g, s.d.latest, b0, b1, out_t, out64);
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "gather3");
    return rr;
}

GenCtl make_genctl(const hjbp_plan &p) {
    GenCtl c;
    std::memset(&c, 0, sizeof(c));
    c.nc = p.desc.n_controls;
    for (int m = 0; m < c.nc; ++m) {
        c.a1[m] = p.controls[3 * m];
        c.a2[m] = p.controls[3 * m + 1];
    }
    return c;
}

// The column tables of the per-node feet on grid g (Brockett, R24).
Gen3 make_gen3(hjbp_plan &p, const Grid3 &g) {
    const GenCtl hc = make_genctl(p);
    const int64_t rows = (int64_t)g.n0 * g.n1 * hc.nc;
    double4 *dh = alloc3<double4>(p, rows);
    W3<float> *v32 = alloc3<W3<float>>(p, rows);
    W3<double> *v64 = alloc3<W3<double>>(p, rows);
    W3<float> *p32 = alloc3<W3<float>>(p, rows);
    uint8_t *oct = alloc3<uint8_t>(p, rows);
    uint32_t *cset = alloc3<uint32_t>(p, rows);
    k_gen_table3<<<grid_for3(rows), 256, 0, p.stream>>>(g, hc, dh, v32, v64, p32, oct, cset);
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "column tables");
    Gen3 r;
    r.nc = hc.nc;
    r.dh = dh;
    r.v32 = v32;
    r.v64 = v64;
    r.p32 = p32;
    r.oct = oct;
    r.cset = cset;
    return r;
}

// Step 1 on the coarse grid: FP32 Gauss-Seidel tiles to 1e-6 from M, then
// the FP32-filtered FP64 Jacobi sweep of the polish from that result (R17:
// the plain iteration reaches the same fixed point on S*) until the sup-norm
// change is below tol.  The fine-sweep statistics are left as they were.
Run3 coarse3(hjbp_plan &p, const Grid3 &gc, const int8_t *code, const float *h32, const double *h64,
             const double *fixed, Sched3 &s, double tol, int cap, double *out64, const Gen3 *gen = nullptr) {
    const int64_t Nc = (int64_t)gc.n0 * gc.n1 * gc.n2;
    cudaStream_t st = p.stream;
    hjbp_stats &S = p.stats;
    const int64_t launches = S.sweep_kernel_launches, visits = S.sweep_tile_visits;
    const double ms = S.ms_sweep_kernel;
    const int rounds = p.desc.tune[0] > 0 ? p.desc.tune[0] : 1;
    float *f0 = alloc3<float>(p, Nc), *f1 = alloc3<float>(p, Nc);
    double *pa = alloc3<double>(p, Nc), *pb = alloc3<double>(p, Nc);
    unsigned long long *cnt = alloc3<unsigned long long>(p, 1);
    check_cuda(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st), "memset");
    Run3 rr = value3<float>(p, gc, code, h32, f0, f1, s, std::max(tol, 1e-6), cap, rounds, nullptr, pa, cnt,
                            nullptr, nullptr, fixed, gen);
    S.sweep_kernel_launches = launches;
    S.sweep_tile_visits = visits;
    S.ms_sweep_kernel = ms;
    k_restore_fixed3<<<grid_for3(Nc), 256, 0, st>>>(Nc, code, fixed, pa);
    ++S.kernel_launches;
    const CtlTable3<double> c64 = make_table3<double>(p);
    const CtlTable3<float> c32 = make_table3<float>(p);
    constexpr int chunk = 8;
    double *res = alloc3<double>(p, chunk);
    double hres[chunk];
    // Jacobi moves information one cell per sweep; the cap covers many
    // crossings of the grid
    const int pcap = std::min(cap, 8 * (gc.n0 + gc.n1 + gc.n2) + 64);
    bool done = false;
    int L = 0;
    while (!done && L < pcap) {
        check_cuda(cudaMemsetAsync(res, 0, sizeof(res[0]) * chunk, st), "memset");
        for (int l = 0; l < chunk; ++l) {
            if (gen)
                k_polish3g<<<grid_for3(Nc, 128), 128, 0, st>>>(gc, code, (l & 1) ? pb : pa, (l & 1) ? pa : pb,
                                                               res + l, nullptr, *gen);
            else
                k_polish3d<<<grid_for3(Nc, 128), 128, 0, st>>>(gc, code, h64, (l & 1) ? pb : pa, (l & 1) ? pa : pb,
                                                               res + l, c32, c64, nullptr);
            ++S.kernel_launches;
        }
        check_cuda(cudaGetLastError(), "coarse polish");
        check_cuda(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, st), "coarse res");
        check_cuda(cudaStreamSynchronize(st), "coarse sync");
        for (int l = 0; l < chunk && !done; ++l) {
            ++L;
            rr.last_res = hres[l];
            if (hres[l] < tol) {
                done = true;
                // the sweeps after the converged one changed less: keep the last
            }
        }
    }
    rr.launches += L;
    rr.converged = rr.converged && done;
    k_finalize<<<grid_for3(Nc), 256, 0, st>>>(Nc, pa, out64);   // chunk is even: pa holds the last sweep
    ++S.kernel_launches;
    return rr;
}

}  // namespace

// The per-line factors of a separable speed on grid g (SpeedLines), in the
// plan's arena; no factors (per-node evaluation) for the other speeds.
SpeedLines speed_lines3(hjbp_plan &p, const Grid3 &g, const SpeedParams &sp) {
    SpeedLines sl{{nullptr, nullptr, nullptr}, speed_terms(sp.kind)};
    if (sl.nt == 0) return sl;
    double *f0 = alloc3<double>(p, (int64_t)g.n0 * sl.nt), *f1 = alloc3<double>(p, (int64_t)g.n1 * sl.nt);
    double *f2 = alloc3<double>(p, (int64_t)g.n2 * sl.nt);
    const int total = sl.nt * (g.n0 + g.n1 + g.n2);
    k_speed_lines<<<(total + 255) / 256, 256, 0, p.stream>>>(sp, sl.nt, g.n0, g.n1, g.n2, g.lo0, g.lo1, g.lo2, g.k, f0,
                                                           f1, f2);
    ++p.stats.kernel_launches;
    sl.f[0] = f0;
    sl.f[1] = f1;
    sl.f[2] = f2;
    return sl;
}

hjbp_status solve3d(hjbp_plan &p) {
    const hjbp_problem_desc &d = p.desc;
    cudaStream_t st = p.stream;
    const int64_t N = p.N;
    const Grid3 g = make_grid3(d.n, d.lo, p.k);
    SpeedParams sp;
    sp.kind = d.speed;
    for (int i = 0; i < 64; ++i) sp.p[i] = d.speed_params[i];
    TargetSet ts;
    std::memset(&ts, 0, sizeof(ts));
    ts.n = d.n_targets;
    ts.kind = d.target_kind;
    ts.nparts = p.R;
    for (int j = 0; j < ts.n; ++j) {
        ts.c0[j] = p.targets[4 * j];
        ts.c1[j] = p.targets[4 * j + 1];
        ts.c2[j] = p.targets[4 * j + 2];
        ts.r[j] = p.targets[4 * j + 3];
    }
    const int cap = d.max_sweeps > 0 ? d.max_sweeps : 1000000;
    const int hist = std::max(std::min(cap, 1 << 20), kReachCap3);
    const bool fp32 = d.precision == HJBP_FP32_POLISH64;
    const int R = p.R;
    const int vrounds = d.tune[0] > 0 ? d.tune[0] : 1;
    const int prounds = d.tune[1] > 0 ? d.tune[1] : 2;
    hjbp_stats &S = p.stats;
    std::memset(&S, 0, sizeof(S));
    hjbp_status status = HJBP_OK;

    Ctl3 hct = make_ctl3(p);
    Ctl3 *dct = static_cast<Ctl3 *>(p.dev_alloc(sizeof(Ctl3)));
    check_cuda(cudaMemcpyAsync(dct, &hct, sizeof(Ctl3), cudaMemcpyHostToDevice, st), "ctl3");
    // Brockett's integrator (R24): feet per node from column tables
    const bool per_node = d.dyn == HJBP_DYN_BROCKETT;
    GenCtl *dgc = nullptr;
    Gen3 gfine{};
    if (per_node) {
        const GenCtl hgc = make_genctl(p);
        dgc = static_cast<GenCtl *>(p.dev_alloc(sizeof(GenCtl)));
        check_cuda(cudaMemcpyAsync(dgc, &hgc, sizeof(GenCtl), cudaMemcpyHostToDevice, st), "controls");
        gfine = make_gen3(p, g);
    }
    const Gen3 *gf = per_node ? &gfine : nullptr;

    Ev3 e0(st);
    int8_t *code0 = alloc3<int8_t>(p, N);
    int8_t *code = alloc3<int8_t>(p, N);
    uint8_t *rch = alloc3<uint8_t>(p, N);
    double *h64 = alloc3<double>(p, N);
    float *h32 = fp32 ? alloc3<float>(p, N) : nullptr;
    unsigned long long *updates = alloc3<unsigned long long>(p, 1);
    check_cuda(cudaMemsetAsync(updates, 0, sizeof(unsigned long long), st), "memset");
    k_setup3d<<<grid_for3(N), 256, 0, st>>>(g, sp, ts, 0.0, 0, code0, h32, h64, nullptr,
                                            make_obstacles(3, d.n_obstacles, d.obstacles), speed_lines3(p, g, sp));
    ++S.kernel_launches;
    check_cuda(cudaGetLastError(), "setup3");
    Sched3 sched = make_sched3(p, g, hist);
    // fine-grid sweeps alternate the increasing and decreasing pass of each
    // axis from launch to launch (tune[5] = 2: all six passes every launch)
    sched.d.alt = d.tune[5] == 2 ? 0 : 1;
    Ev3 e1(st);

    double *dlit = nullptr;   // literal U_P^(0): the Dirichlet data (R16)
    if (p.patchy) {
        const Grid3 gc = make_grid3(d.n_coarse, d.lo, p.kc);
        const int64_t Nc = p.Nc;
        int8_t *ccode = alloc3<int8_t>(p, Nc);
        uint8_t *crch = alloc3<uint8_t>(p, Nc);
        double *ch64 = alloc3<double>(p, Nc);
        double *cfix = alloc3<double>(p, Nc);
        float *ch32 = alloc3<float>(p, Nc);
        k_setup3d<<<grid_for3(Nc), 256, 0, st>>>(gc, sp, ts, p.kc * std::sqrt(3.0) / 2.0, 1, ccode, ch32, ch64,
                                                 cfix, make_obstacles(3, d.n_obstacles, d.obstacles),
                                                 speed_lines3(p, gc, sp), dgc);
        k_merge_targets<<<grid_for3(Nc), 256, 0, st>>>(Nc, ccode);
        S.kernel_launches += 2;
        Gen3 gcoarse{};
        if (per_node) gcoarse = make_gen3(p, gc);
        const Gen3 *gcp = per_node ? &gcoarse : nullptr;
        Sched3 csched = make_sched3(p, gc, hist);
        S.sweeps_reach += reach3(p, gc, ccode, crch, csched, Nc, nullptr, gcp);
        const double tolc = d.tol_coarse > 0 ? d.tol_coarse : 1e-12;
        Run3 rc = coarse3(p, gc, ccode, ch32, ch64, cfix, csched, tolc, cap, p.u_coarse, gcp);
        S.sweeps_coarse = rc.launches;
        if (!rc.converged) status = HJBP_ENOCONV;
        Ev3 e2(st);
        if (d.flags & HJBP_FLAG_DIRICHLET) dlit = alloc3<double>(p, N);
        float *u0f = per_node ? nullptr : alloc3<float>(p, N);
        k_u0_3d<<<grid_for3(N), 256, 0, st>>>(g, gc, code0, p.u_coarse, p.u0, dlit, u0f);
        if (per_node) {
            k_feedback3g<<<grid_for3(N, 128), 128, 0, st>>>(g, code0, p.u0, p.astar, gfine);
        } else {
            const CtlLit3 hl = make_lit3(p);
            CtlLit3 *dl = static_cast<CtlLit3 *>(p.dev_alloc(sizeof(CtlLit3)));
            check_cuda(cudaMemcpyAsync(dl, &hl, sizeof(CtlLit3), cudaMemcpyHostToDevice, st), "feedback table");
            k_feedback3d<<<grid_for3(N, 128), 128, 0, st>>>(g, code0, h64, p.u0, p.astar, dl, u0f);
        }
        S.kernel_launches += 2;
        check_cuda(cudaGetLastError(), "feedback3");
        // AO2: causal sweep directions per tile from the feedback (Step 3.1 and 3.2)
        if ((d.flags & HJBP_FLAG_CAUSAL_SWEEPS) && sched.ntiles) {
            DirCtl3 dc;
            std::memset(&dc, 0, sizeof(dc));
            for (int m = 0; m < d.n_controls && !per_node; ++m)
                for (int c = 0; c < 3; ++c) {
                    const double v = p.controls[3 * m + c];
                    dc.s[c][m] = (int8_t)(v > 1e-12 ? 1 : (v < -1e-12 ? -1 : 0));
                }
            uint8_t *dirs = alloc3<uint8_t>(p, sched.ntiles);
            k_tile_dirs3d<<<sched.ntiles, kT3n, 0, st>>>(g, code0, p.astar, dc, gfine, 0.9f, dirs);
            ++S.kernel_launches;
            check_cuda(cudaGetLastError(), "tile directions");
            sched.d.dirs = dirs;
        }
        Ev3 e3(st);
        {
            // colours per transport pass: up to 8 on grids of at most 4096 tiles (one
            // front propagation for all colours; measured faster at 101^3), 4 on larger
            // grids, where the launches fill the GPU and a CTA of 8 colours (46 KB of
            // shared memory) halves the resident CTAs (257^3: labels 90 -> 100 ms)
            const int RG = (R > 4 && sched.ntiles <= 4096) ? 8 : (R >= 3 ? 4 : (R == 2 ? 2 : 1));
            float *f0 = alloc3<float>(p, N * RG), *f1 = alloc3<float>(p, N * RG), *r32 = alloc3<float>(p, N * RG);
            double *phig = alloc3<double>(p, N * RG);
            float *rmax = alloc3<float>(p, 1);
            const double tolp = d.tol_phi > 0 ? d.tol_phi : 1e-10;
            for (int j0 = 0; j0 < R; j0 += RG) {
                const int rg = std::min(RG, R - j0);
                // colours past R in the last group see no target and stay 0
                const int rgl = rg > 4 ? 8 : (rg >= 3 ? 4 : rg);
                auto launch_group = [&](auto tag) {
                    constexpr int G = decltype(tag)::value;
                    constexpr size_t kSb = sizeof(Phi3Smem<G, false>), kSs = sizeof(Phi3Smem<G, true>);
                    check_cuda(cudaFuncSetAttribute(k_phi3d<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)kSb), "phi smem");
                    check_cuda(cudaFuncSetAttribute(k_phi3d<G, false, true>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSb), "phi smem");
                    check_cuda(cudaFuncSetAttribute(k_phi3d<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)kSs), "phi smem");
                    check_cuda(cudaFuncSetAttribute(k_phi3d<G, true, true>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSs), "phi smem");
                    k_phi_init3d<G><<<grid_for3(N), 256, 0, st>>>(N, code0, j0, 0, f0, f1);
                    ++S.kernel_launches;
                    Run3 rp = run_tiles3(p, g, sched, std::max(tolp, 2e-7), cap, [&](int par) {
                        if (per_node)
                            k_phi3d<G, false, true><<<sched.ntiles, kT3n * phi3_groups<G>(), kSb, st>>>(
                                g, code0, p.astar, f0, f1, nullptr, sched.d, par, prounds, dct, gfine);
                        else
                            k_phi3d<G, false><<<sched.ntiles, kT3n * phi3_groups<G>(), kSb, st>>>(
                                g, code0, p.astar, f0, f1, nullptr, sched.d, par, prounds, dct);
                        ++S.kernel_launches;
                    });
                    S.sweeps_phi += rp.launches;
                    if (!rp.converged) status = HJBP_ENOCONV;
                    k_phi_collect3d<G><<<grid_for3(N), 256, 0, st>>>(g, sched.d.latest, f0, f1, phig, 0);
                    ++S.kernel_launches;
                    for (int it = 0; it < 6; ++it) {
                        check_cuda(cudaMemsetAsync(rmax, 0, sizeof(float), st), "memset");
                        if (per_node)
                            k_phi_residual3d<G, true><<<grid_for3(N), 256, 0, st>>>(g, code0, p.astar, phig, r32,
                                                                                     rmax, dct, gfine);
                        else
                            k_phi_residual3d<G><<<grid_for3(N), 256, 0, st>>>(g, code0, p.astar, phig, r32, rmax,
                                                                              dct);
                        ++S.kernel_launches;
                        float hr = 0.f;
                        check_cuda(cudaMemcpyAsync(&hr, rmax, sizeof(float), cudaMemcpyDeviceToHost, st), "rmax");
                        check_cuda(cudaStreamSynchronize(st), "rmax sync");
                        S.phi_refinements++;
                        if (hr <= tolp) break;
                        k_phi_init3d<G><<<grid_for3(N), 256, 0, st>>>(N, code0, j0, 1, f0, f1);
                        ++S.kernel_launches;
                        const float told = std::max((float)(tolp * 0.1), 1e-3f * hr);
                        Run3 rc2 = run_tiles3(p, g, sched, told, cap, [&](int par) {
                            if (per_node)
                                k_phi3d<G, true, true><<<sched.ntiles, kT3n * phi3_groups<G>(), kSs, st>>>(
                                    g, code0, p.astar, f0, f1, r32, sched.d, par, prounds, dct, gfine);
                            else
                                k_phi3d<G, true><<<sched.ntiles, kT3n * phi3_groups<G>(), kSs, st>>>(
                                    g, code0, p.astar, f0, f1, r32, sched.d, par, prounds, dct);
                            ++S.kernel_launches;
                        });
                        S.sweeps_phi += rc2.launches;
                        k_phi_collect3d<G><<<grid_for3(N), 256, 0, st>>>(g, sched.d.latest, f0, f1, phig, 1);
                        ++S.kernel_launches;
                    }
                    check_cuda(cudaMemcpyAsync(p.phi + (int64_t)j0 * N, phig, sizeof(double) * N * rg,
                                               cudaMemcpyDeviceToDevice, st), "phi copy");
                };
                if (rgl == 8) launch_group(std::integral_constant<int, 8>());
                else if (rgl == 4) launch_group(std::integral_constant<int, 4>());
                else if (rgl == 2) launch_group(std::integral_constant<int, 2>());
                else launch_group(std::integral_constant<int, 1>());
            }
            k_label2d<<<grid_for3(N), 256, 0, st>>>(N, code0, p.astar, p.phi, R, p.label_out);
            ++S.kernel_launches;
            int8_t *lab2 = reinterpret_cast<int8_t *>(rch);
            unsigned long long *chg = alloc3<unsigned long long>(p, 1);
            // Jacobi rounds of Remark 3.1's fill, ping-ponged between the two label
            // buffers, in batches between host checks (4, 8, .. 64 rounds): a round
            // after the last change changes nothing, so the batches give the rounds'
            // result exactly
            int8_t *la = p.label_out, *lb = lab2;
            int batch = 4;
            for (int it = 0; it < 100000;) {
                check_cuda(cudaMemsetAsync(chg, 0, sizeof(unsigned long long), st), "memset");
                for (int k = 0; k < batch; ++k, ++it) {
                    k_fill3d<<<grid_for3(N), 256, 0, st>>>(g, la, lb, chg);
                    ++S.kernel_launches;
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
            k_patch_codes<<<grid_for3(N), 256, 0, st>>>(N, code0, p.label_out, code);
            ++S.kernel_launches;
        }
        Ev3 e4(st);
        {
            uint64_t *tile_patch = alloc3<uint64_t>(p, sched.ntiles);
            unsigned long long *pn = alloc3<unsigned long long>(p, kMaxTargets);
            unsigned long long *pt = alloc3<unsigned long long>(p, kMaxTargets);
            int *tcnt = alloc3<int>(p, (int64_t)sched.ntiles * R);
            check_cuda(cudaMemsetAsync(pn, 0, sizeof(unsigned long long) * kMaxTargets, st), "memset");
            check_cuda(cudaMemsetAsync(pt, 0, sizeof(unsigned long long) * kMaxTargets, st), "memset");
            check_cuda(cudaMemsetAsync(tcnt, 0, sizeof(int) * std::max<int64_t>(1, (int64_t)sched.ntiles * R), st),
                       "memset");
            if (sched.ntiles) {
                k_compact3d<<<sched.ntiles, kT3n, 0, st>>>(g, code, tile_patch, pn, pt, tcnt, R);
                ++S.kernel_launches;
            }
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
        Ev3 e5(st);
        S.ms_coarse = ms3(e1, e2);
        S.ms_feedback = ms3(e2, e3);
        S.ms_labels = ms3(e3, e4);
        S.ms_compact = ms3(e4, e5);
    } else {
        check_cuda(cudaMemcpyAsync(code, code0, (size_t)N, cudaMemcpyDeviceToDevice, st), "code copy");
        k_merge_targets<<<grid_for3(N), 256, 0, st>>>(N, code);
        ++S.kernel_launches;
    }

    Ev3 f0(st);
    // patch boundary: state constraints, or U_P^(0) (Eq. dbc); start: M or U_P^(0) (AO1)
    const bool dirichlet = p.patchy && (d.flags & HJBP_FLAG_DIRICHLET);
    const double *warm = (p.patchy && (d.flags & HJBP_FLAG_WARM_START)) ? p.u0 : nullptr;
    const double *d64 = dirichlet ? dlit : nullptr;
    // AO3: the cones of the coarse feedback (Step 3.2 only; labels keep every control)
    Cone3 *cone = nullptr;
    double cone_size = 0.0;   // mean controls per node under AO3 (0: every control)
    if (p.patchy && d.reduce_r != 0.0) {
        std::unique_ptr<Cone3> hc(new Cone3);
        cone_size = make_cones3(p, *hc);
        cone = static_cast<Cone3 *>(p.dev_alloc(sizeof(Cone3)));
        check_cuda(cudaMemcpyAsync(cone, hc.get(), sizeof(Cone3), cudaMemcpyHostToDevice, st), "cones");
        check_cuda(cudaStreamSynchronize(st), "cones sync");   // the host copy is freed next
    }
    S.sweeps_reach += reach3(p, g, code, rch, sched, N, d64, gf, cone);
    Ev3 fr(st);
    Run3 rv;
    // per-patch residual at retirement: the tiles' last changes (FP64)
    double *last_chg = nullptr;
    if (p.patchy && sched.ntiles) {
        last_chg = alloc3<double>(p, sched.ntiles);
        check_cuda(cudaMemsetAsync(last_chg, 0, sizeof(double) * sched.ntiles, st), "memset");
        sched.d.last_chg = last_chg;
    }
    if (fp32) {
        float *b0 = alloc3<float>(p, N), *b1 = alloc3<float>(p, N);
        float *d32 = nullptr;
        if (dirichlet) {
            d32 = alloc3<float>(p, N);
            k_narrow_data3<<<grid_for3(N), 256, 0, st>>>(N, dlit, d32);
            ++S.kernel_launches;
        }
        rv = value3<float>(p, g, code, h32, b0, b1, sched, d.tol, cap, vrounds, p.u32, nullptr, updates, d32, warm,
                           nullptr, gf, cone);
    } else {
        double *b0 = alloc3<double>(p, N), *b1 = alloc3<double>(p, N);
        rv = value3<double>(p, g, code, h64, b0, b1, sched, d.tol, cap, vrounds, nullptr, p.u_out, updates, d64,
                            warm, nullptr, gf, cone);
    }
    S.sweeps_fine = rv.launches;
    S.residual_fine = rv.last_res;
    if (!rv.converged) status = HJBP_ENOCONV;
    if (last_chg) {
        patch_residuals(p, sched.ntiles, sched.d.tile_patch, last_chg);
        sched.d.last_chg = nullptr;
    }
    if (rv.launches > 0) {
        std::vector<uint64_t> ph(rv.launches);
        check_cuda(cudaMemcpyAsync(ph.data(), sched.d.patch_hist, sizeof(uint64_t) * rv.launches,
                                   cudaMemcpyDeviceToHost, st), "patch hist");
        check_cuda(cudaStreamSynchronize(st), "patch hist sync");
        for (int l = 0; l < rv.launches; ++l)
            for (int j = 0; j < R && j < 64; ++j)
                if ((ph[l] >> j) & 1ull) S.sweeps_patch[j]++;
    }
    Ev3 f1(st);
    if (fp32) {
        double *pa = alloc3<double>(p, N), *pb = alloc3<double>(p, N);
        double *mc = alloc3<double>(p, 1);
        k_widen<<<grid_for3(N), 256, 0, st>>>(N, p.u32, pa);
        ++S.kernel_launches;
        const CtlTable3<double> c64 = make_table3<double>(p);
        const CtlTable3<float> c32 = make_table3<float>(p);
        double last = 0.0;
        int it = 0;
        for (; it < 8; ++it) {
            check_cuda(cudaMemsetAsync(mc, 0, sizeof(double), st), "memset");
            if (per_node)
                k_polish3g<<<grid_for3(N, 128), 128, 0, st>>>(g, code, pa, pb, mc, d64, gfine);
            else
                k_polish3d<<<grid_for3(N, 128), 128, 0, st>>>(g, code, h64, pa, pb, mc, c32, c64, d64, cone,
                                                              p.astar);
            ++S.kernel_launches;
            check_cuda(cudaGetLastError(), "polish3");
            std::swap(pa, pb);
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
        k_finalize<<<grid_for3(N), 256, 0, st>>>(N, pa, p.u_out);
        ++S.kernel_launches;
    }
    unsigned long long *unreach = alloc3<unsigned long long>(p, 1);
    check_cuda(cudaMemsetAsync(unreach, 0, sizeof(unsigned long long), st), "memset");
    k_final_labels<<<grid_for3(N), 256, 0, st>>>(N, code0, code, p.patchy ? nullptr : p.label_out, unreach);
    ++S.kernel_launches;
    Ev3 f2(st);
    unsigned long long hu = 0, hun = 0;
    check_cuda(cudaMemcpyAsync(&hu, updates, sizeof(hu), cudaMemcpyDeviceToHost, st), "updates");
    check_cuda(cudaMemcpyAsync(&hun, unreach, sizeof(hun), cudaMemcpyDeviceToHost, st), "unreachable");
    check_cuda(cudaStreamSynchronize(st), "final sync");
    S.unreachable = (int64_t)hun;
    S.node_updates = (int64_t)hu;
    int admissible = d.n_controls;   // Brockett's a = 0 cannot move and is never evaluated
    if (per_node)
        for (int m = 0; m < d.n_controls; ++m)
            if (p.controls[3 * m] == 0.0 && p.controls[3 * m + 1] == 0.0) --admissible;
    S.node_control_updates = cone ? (int64_t)((double)hu * cone_size + 0.5) : (int64_t)hu * admissible;
    S.n_patches = p.patchy ? R : 1;
    S.ms_setup = ms3(e0, e1);
    S.ms_fine = ms3(f0, f1);
    S.ms_reach = ms3(f0, fr);
    S.ms_polish = ms3(f1, f2);
    S.ms_total = ms3(e0, f2);
    return status;
}

// ---------------------------------------------------------- instantiation --
template __global__ void k_init3d<float>(int64_t, const int8_t *, const double *, float, float *, float *,
                                          const double *);
template __global__ void k_init3d<double>(int64_t, const int8_t *, const double *, double, double *, double *,
                                           const double *);

}  // namespace hjbp
