// noalloc.cu -- hjbp_solve_global2d_noalloc: the plain global 2D solve (FP64)
// for callers that cannot allocate memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at solve time:
// real-time control loops that forbid allocation once they have started (an
// allocation can block for an unbounded time or fail when memory is
// fragmented), or hosts whose device memory pool is owned by someone else.
// This entry point runs the same kernels as hjbp_solve does for a global 2D
// FP64 problem, but takes every scratch array from one file-scope device array
// of fixed size (kScratchBytes) instead of allocating.  The caller passes the
// problem and the two output arrays.
//
// The call is synchronous: between launches it reads the active-tile and
// pruned-node counts back into host variables and waits for them, and it
// synchronises the stream before returning.
//
// The device array lives in every GPU that loads the library until the
// process exits.  In host code its name is only a host-side stand-in: the
// device address (and the SM count used to size grids) is looked up once per
// device index with cudaGetSymbolAddress and cached for the process lifetime,
// which assumes one primary context per device (no cudaDeviceReset between
// calls).  The first call on a device does that set-up.  Every call shares the
// array and it keeps the previous call's contents, so the solve clears what
// must start at zero; calls that overlap on the GPU (several streams or
// threads at once) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "hjbp_device.cuh"

namespace hjbp {

// Kernels defined in kernels2d.cu (the same ones hjbp_solve launches).
__global__ void k_setup2d(Grid2 g, SpeedParams sp, TargetSet ts, double extra, int boundary_values, int8_t *code,
                          float *h32, double *h64, double *fixed, DynParams dp, ObstacleSet os, SpeedLines sl);
__global__ void k_schedule2d(Grid2 g, TileSched s, int par, double tol, int launch);
__global__ void __launch_bounds__(32) k_reach2d(Grid2 g, const int8_t *code, uint8_t *rch, TileSched s, int par,
                                                ReachTable2 rt, int passes, const double *dterm,
                                                const uint8_t *astar, const Cone2 *cone, uint64_t *cache,
                                                uint8_t *cvalid);
__global__ void __launch_bounds__(32) k_peel2d(Grid2 g, int8_t *code, TileSched s, int par, ReachTable2 rt,
                                               const double *dterm, const uint8_t *astar, const Cone2 *cone);
__global__ void k_reach_prune(int64_t N, int8_t *code, const uint8_t *rch, unsigned long long *removed);
__global__ void k_merge_targets(int64_t N, int8_t *code);
__global__ void k_final_labels(int64_t N, const int8_t *code0, const int8_t *code, int8_t *label,
                               unsigned long long *unreachable);

void launch_init_values2d_f64(int blocks, cudaStream_t st, int64_t N, const int8_t *code, double start, double *b0,
                              double *b1);
void launch_value2d_f64(int ntiles, cudaStream_t st, Grid2 g, const int8_t *code, const double *h, double *b0,
                        double *b1, TileSched s, int par, int rounds, const CtlTable2<double> &ct);
void launch_gather2d_f64(int blocks, cudaStream_t st, Grid2 g, const uint8_t *latest, const double *b0,
                         const double *b1, double *out64);
void set_last_error_static(const char *msg);

}  // namespace hjbp

namespace {

using namespace hjbp;

// 32 MiB of scratch: up to HJBP_NOALLOC_MAX_NODES nodes (27 bytes per node for
// codes, reach flags, h and two FP64 value buffers, plus the tile lists).
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 128;
void *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of g_scratch and the SM count of the current device, looked
// up once per device index.
const char *scratch_address(void **out, int *sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return "cudaGetDevice failed";
    if (dev < 0 || dev >= kMaxDevices) return "device index out of range";
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return "cudaDeviceGetAttribute(MultiProcessorCount) failed";
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return "cudaGetSymbolAddress of the scratch array failed";
        g_sms[dev] = n;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return nullptr;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t code0, code, rch, h64, b0, b1, list0, list1, iota, count, chg0, chg1, latest, processed, counters, total;
};

Layout layout(int64_t N, int ntiles) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t nt = (size_t)(ntiles > 0 ? ntiles : 1);
    L.code0 = take((size_t)N);
    L.code = take((size_t)N);
    L.rch = take((size_t)N);
    L.h64 = take(sizeof(double) * N);
    L.b0 = take(sizeof(double) * N);
    L.b1 = take(sizeof(double) * N);
    L.list0 = take(sizeof(int) * nt);
    L.list1 = take(sizeof(int) * nt);
    L.iota = take(sizeof(int) * nt);
    L.count = take(2 * sizeof(int));
    L.chg0 = take(sizeof(double) * nt);
    L.chg1 = take(sizeof(double) * nt);
    L.latest = take(nt);
    L.processed = take(nt);
    L.counters = take(2 * sizeof(unsigned long long));
    L.total = o;
    return L;
}

__global__ void k_iota_noalloc(int n, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

// Grid of 256-thread blocks for n elements: at most 64 blocks per SM (the
// kernels stride over the rest).
int blocks_for(int64_t n, int sms) {
    const int64_t b = (n + 255) / 256, most = (int64_t)sms * 64;
    return (int)(b < 1 ? 1 : (b > most ? most : b));
}

// Host-side validation without allocating; returns a static message or null.
const char *check_desc(const hjbp_problem_desc *d) {
    if (!d) return "descriptor is NULL";
    if (d->dim != 2) return "the no-allocation entry point solves 2D problems only";
    if (d->n_coarse[0] != 0) return "the no-allocation entry point runs the plain global solve (n_coarse[0] must be 0)";
    if (d->n[0] < 3 || d->n[1] < 3) return "every axis needs at least 3 nodes";
    if (!(d->hi[0] > d->lo[0]) || !(d->hi[1] > d->lo[1])) return "hi must exceed lo on every axis";
    const double k0 = (d->hi[0] - d->lo[0]) / (d->n[0] - 1), k1 = (d->hi[1] - d->lo[1]) / (d->n[1] - 1);
    if (std::fabs(k1 - k0) > 1e-12 * k0) return "grid spacing must be equal on every axis";
    if ((int64_t)d->n[0] * d->n[1] > (int64_t)HJBP_NOALLOC_MAX_NODES) return "grid exceeds HJBP_NOALLOC_MAX_NODES";
    if (d->speed != HJBP_C_ONE && d->speed != HJBP_C_SINCOS2D && d->speed != HJBP_C_FOURIER2D &&
        d->speed != HJBP_C_FAN)
        return "speed field must be a 2D one";
    if (d->n_controls < 1 || d->n_controls > HJBP_MAX_CONTROLS || !d->controls) return "bad control set";
    for (int m = 0; m < d->n_controls; ++m) {
        const double ax = d->controls[2 * m], ay = d->controls[2 * m + 1];
        if (!std::isfinite(ax) || !std::isfinite(ay) || std::fabs(std::sqrt(ax * ax + ay * ay) - 1.0) > 1e-9)
            return "controls must be finite unit vectors";
    }
    if (d->n_targets < 1 || d->n_targets > HJBP_MAX_TARGETS || !d->targets) return "bad target set";
    for (int j = 0; j < 3 * d->n_targets; ++j)
        if (!std::isfinite(d->targets[j])) return "target entry not finite";
    if (!(d->tol > 0.0)) return "tol must be positive";
    if (const char *e = check_obstacles(d)) return e;
    if (d->dyn != HJBP_DYN_SPEED || d->target_kind != HJBP_TARGET_BALLS)
        return "the no-allocation entry point takes f = c(x) a and ball targets";
    // the options hjbp_create rejects for a plain global solve
    if (d->flags & (HJBP_FLAG_DIRICHLET | HJBP_FLAG_WARM_START | HJBP_FLAG_CAUSAL_SWEEPS))
        return "Dirichlet patch boundaries, the warm start and causal sweeps need a patchy solve (n_coarse)";
    if (d->reduce_r != 0.0) return "reduce_r needs a patchy solve (n_coarse)";
    if (d->speed == HJBP_C_FOURIER2D) {
        double norm = 0.0;
        for (int i = 0; i < 16; ++i) norm += std::fabs(d->speed_params[i]);
        if (!(norm > 0.0)) return "Fourier speed field needs a nonzero coefficient";
    }
    return nullptr;
}

hjbp_status fail_static(hjbp_status s, const char *msg) {
    set_last_error_static(msg);
    return s;
}

#define NA_CHECK(call)                                                                    \
    do {                                                                                  \
        const cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return fail_static(HJBP_ECUDA, cudaGetErrorString(e_));    \
    } while (0)

// Sweep + schedule launches until no tile is active (count read back every
// few launches into a stack variable) or the cap is hit.
template <class Sweep>
hjbp_status run(cudaStream_t st, const Grid2 &g, TileSched &s, int ntiles, int *iota_list, double tol, int cap,
                bool *converged, Sweep sweep) {
    *converged = false;
    if (ntiles == 0) {
        *converged = true;
        return HJBP_OK;
    }
    const int counts[2] = {ntiles, 0};
    NA_CHECK(cudaMemcpyAsync(s.list[0], iota_list, sizeof(int) * ntiles, cudaMemcpyDeviceToDevice, st));
    NA_CHECK(cudaMemcpyAsync(s.count, counts, sizeof(counts), cudaMemcpyHostToDevice, st));
    NA_CHECK(cudaMemsetAsync(s.chg[0], 0, sizeof(double) * ntiles, st));
    NA_CHECK(cudaMemsetAsync(s.chg[1], 0, sizeof(double) * ntiles, st));
    NA_CHECK(cudaMemsetAsync(s.latest, 0, ntiles, st));
    NA_CHECK(cudaMemsetAsync(s.processed, 0, ntiles, st));
    NA_CHECK(cudaStreamSynchronize(st));
    int par = 0;
    for (int L = 0; L < cap;) {
        sweep(par);
        k_schedule2d<<<(ntiles + 255) / 256, 256, 0, st>>>(g, s, par, tol, L);
        NA_CHECK(cudaGetLastError());
        par ^= 1;
        ++L;
        if (L % 4 == 0 || L == cap) {
            int left = 0;
            NA_CHECK(cudaMemcpyAsync(&left, s.count + par, sizeof(int), cudaMemcpyDeviceToHost, st));
            NA_CHECK(cudaStreamSynchronize(st));
            if (left == 0) {
                *converged = true;
                break;
            }
        }
    }
    return HJBP_OK;
}

}  // namespace

extern "C" hjbp_status hjbp_solve_global2d_noalloc(const hjbp_problem_desc *desc, void *cuda_stream,
                                                   double *u_out, int8_t *labels_out) {
    const char *bad = check_desc(desc);
    if (bad) return fail_static(HJBP_EINVAL, bad);
    if (!u_out || !labels_out) return fail_static(HJBP_EINVAL, "output pointers must be device arrays");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void *base = nullptr;
    int sms = 0;
    if (const char *e = scratch_address(&base, &sms)) return fail_static(HJBP_ECUDA, e);
    auto blocks_for = [sms](int64_t n) { return ::blocks_for(n, sms); };

    const int n0 = desc->n[0], n1 = desc->n[1];
    const int64_t N = (int64_t)n0 * n1;
    Grid2 g;
    g.n0 = n0;
    g.n1 = n1;
    g.ntx = (n0 - 2 + kTile - 1) / kTile;
    g.nty = (n1 - 2 + kTile - 1) / kTile;
    g.lo0 = desc->lo[0];
    g.lo1 = desc->lo[1];
    g.k = (desc->hi[0] - desc->lo[0]) / (n0 - 1);
    const int ntiles = g.ntx * g.nty;
    const Layout L = layout(N, ntiles);
    if (L.total > kScratchBytes) return fail_static(HJBP_EINVAL, "grid does not fit the scratch array");

    unsigned char *sc = static_cast<unsigned char *>(base);
    int8_t *code0 = reinterpret_cast<int8_t *>(sc + L.code0);
    int8_t *code = reinterpret_cast<int8_t *>(sc + L.code);
    uint8_t *rch = sc + L.rch;
    double *h64 = reinterpret_cast<double *>(sc + L.h64);
    double *b0 = reinterpret_cast<double *>(sc + L.b0);
    double *b1 = reinterpret_cast<double *>(sc + L.b1);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(sc + L.counters);
    TileSched s;
    std::memset(&s, 0, sizeof(s));
    s.list[0] = reinterpret_cast<int *>(sc + L.list0);
    s.list[1] = reinterpret_cast<int *>(sc + L.list1);
    s.count = reinterpret_cast<int *>(sc + L.count);
    s.chg[0] = reinterpret_cast<double *>(sc + L.chg0);
    s.chg[1] = reinterpret_cast<double *>(sc + L.chg1);
    s.latest = sc + L.latest;
    s.processed = sc + L.processed;
    // 0..ntiles-1, copied into list0 before each phase
    int *iota = reinterpret_cast<int *>(sc + L.iota);

    // Problem tables on the stack (kernel parameters).
    SpeedParams sp;
    sp.kind = desc->speed;
    for (int i = 0; i < 64; ++i) sp.p[i] = desc->speed_params[i];
    TargetSet ts;
    std::memset(&ts, 0, sizeof(ts));
    ts.n = desc->n_targets;
    for (int j = 0; j < ts.n; ++j) {
        ts.c0[j] = desc->targets[3 * j];
        ts.c1[j] = desc->targets[3 * j + 1];
        ts.r[j] = desc->targets[3 * j + 2];
    }
    CtlTable2<double> ct;
    std::memset(&ct, 0, sizeof(ct));
    ReachTable2 rt;
    std::memset(&rt, 0, sizeof(rt));
    ct.nc = desc->n_controls;
    int pos = 0;
    for (int q = 0; q < 4; ++q) {
        ct.qbeg[q] = pos;
        for (int m = 0; m < desc->n_controls; ++m) {
            const double ax = desc->controls[2 * m], ay = desc->controls[2 * m + 1];
            if ((ax >= 0.0 ? 1 : 0) + (ay >= 0.0 ? 2 : 0) != q) continue;
            const double bx = std::fabs(ax), by = std::fabs(ay);
            const double w00 = (1.0 - bx) * (1.0 - by), w10 = bx * (1.0 - by), w01 = (1.0 - bx) * by, w11 = bx * by;
            const double kap = 1.0 / (1.0 - w00);
            ct.kw10[pos] = kap * w10;
            ct.kw01[pos] = kap * w01;
            ct.kw11[pos] = kap * w11;
            ct.kap[pos] = kap;
            const unsigned need = (unsigned)(w10 > 0.0) | ((unsigned)(w01 > 0.0) << 1) | ((unsigned)(w11 > 0.0) << 2);
            if (need) rt.present[q] |= (uint8_t)(1u << need);
            ++pos;
        }
    }
    ct.qbeg[4] = pos;
    const int cap = desc->max_sweeps > 0 ? desc->max_sweeps : 1000000;

    // Set-up: node codes and h, all target parts merged (one global target).
    DynParams dp;
    std::memset(&dp, 0, sizeof(dp));   // f = c(x) a
    k_setup2d<<<blocks_for(N), 256, 0, st>>>(g, sp, ts, 0.0, 0, code0, nullptr, h64, nullptr, dp,
                                             make_obstacles(2, desc->n_obstacles, desc->obstacles),
                                             SpeedLines{{nullptr, nullptr, nullptr}, 0});   // c per node
    NA_CHECK(cudaGetLastError());
    NA_CHECK(cudaMemcpyAsync(code, code0, (size_t)N, cudaMemcpyDeviceToDevice, st));
    k_merge_targets<<<blocks_for(N), 256, 0, st>>>(N, code);
    if (ntiles) k_iota_noalloc<<<blocks_for(ntiles), 256, 0, st>>>(ntiles, iota);
    NA_CHECK(cudaGetLastError());

    // S*: reach from the target, prune, repeat until nothing is pruned.
    bool conv = false;
    // each round prunes at least one node or ends the loop (at most N rounds)
    for (int64_t round = 0;; ++round) {
        if (round > N) return fail_static(HJBP_ECUDA, "reachability pruning did not settle");
        // peel the nodes left without any usable control first: they cannot be
        // in S*, and removing them here saves one reach round per such node
        hjbp_status ps = run(st, g, s, ntiles, iota, 0.5, 1 << 18, &conv, [&](int par) {
            k_peel2d<<<ntiles, 32, 0, st>>>(g, code, s, par, rt, nullptr, nullptr, nullptr);
        });
        if (ps != HJBP_OK) return ps;
        if (!conv) return fail_static(HJBP_ECUDA, "peeling did not settle");
        NA_CHECK(cudaMemsetAsync(rch, 0, (size_t)N, st));
        hjbp_status rs = run(st, g, s, ntiles, iota, 0.5, 1 << 18, &conv, [&](int par) {
            k_reach2d<<<ntiles, 32, 0, st>>>(g, code, rch, s, par, rt, 2, nullptr, nullptr, nullptr, nullptr,
                                             nullptr);   // no row-set cache: nothing to allocate
        });
        if (rs != HJBP_OK) return rs;
        if (!conv) return fail_static(HJBP_ECUDA, "reachability sweep did not settle");
        NA_CHECK(cudaMemsetAsync(counters, 0, sizeof(unsigned long long), st));
        k_reach_prune<<<blocks_for(N), 256, 0, st>>>(N, code, rch, counters);
        NA_CHECK(cudaGetLastError());
        unsigned long long removed = 0;
        NA_CHECK(cudaMemcpyAsync(&removed, counters, sizeof(removed), cudaMemcpyDeviceToHost, st));
        NA_CHECK(cudaStreamSynchronize(st));
        if (!removed) break;
    }

    // Value iteration from M on S*, FP64, to the sup-norm tolerance.
    launch_init_values2d_f64(blocks_for(N), st, N, code, kStartValue, b0, b1);
    NA_CHECK(cudaGetLastError());
    hjbp_status vs = run(st, g, s, ntiles, iota, desc->tol, cap, &conv, [&](int par) {
        launch_value2d_f64(ntiles, st, g, code, h64, b0, b1, s, par, 2, ct);
    });
    if (vs != HJBP_OK) return vs;
    launch_gather2d_f64(blocks_for(N), st, g, s.latest, b0, b1, u_out);
    NA_CHECK(cudaMemsetAsync(counters + 1, 0, sizeof(unsigned long long), st));
    k_final_labels<<<blocks_for(N), 256, 0, st>>>(N, code0, code, labels_out, counters + 1);
    NA_CHECK(cudaGetLastError());
    NA_CHECK(cudaStreamSynchronize(st));
    if (!conv) return fail_static(HJBP_ENOCONV, "sweep cap reached before convergence");
    return HJBP_OK;
}
