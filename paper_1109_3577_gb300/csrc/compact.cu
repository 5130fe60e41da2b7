// compact.cu -- patch compaction (Sec. 3, the assembly of the patches before
// Step 3.2): per patch j, the tiles holding a free node of patch j and the
// nodes themselves, in CSR form.
//
//   tile_off[j] .. tile_off[j+1]   entries of patch j in tile_ids / tile_nodes
//   tile_ids[e]                    tile index (x fastest over the tile grid)
//   tile_nodes[e]                  free nodes of patch j in that tile
//   node_off[j] .. node_off[j+1]   entries of patch j in node_ids
//   node_ids[k]                    node index, tiles in increasing order and,
//                                  inside a tile, x fastest
//
// The compaction kernels of the 2D and 3D paths leave a patch bitmask per tile
// and a node count per (tile, patch); the two kernels here turn them into the
// lists with ordered scans, so the lists are deterministic.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hjbp_device.cuh"
#include "plan.h"

namespace hjbp {

namespace {

constexpr int kScanThreads = 1024;

// One block per patch j: the tiles whose mask holds bit j, in increasing tile
// order, with their node counts and the start of their nodes in node_ids.
__global__ void __launch_bounds__(kScanThreads) k_patch_tiles(int ntiles, int R, const uint64_t *__restrict__ tile_patch,
                                                              const int *__restrict__ tile_cnt,
                                                              const int64_t *__restrict__ tile_off,
                                                              const int64_t *__restrict__ node_off,
                                                              int *__restrict__ tile_ids, int *__restrict__ tile_nodes,
                                                              int64_t *__restrict__ entry_node0,
                                                              uint8_t *__restrict__ entry_patch) {
    const int j = blockIdx.x;
    const int tid = threadIdx.x;
    const int per = (ntiles + kScanThreads - 1) / kScanThreads;
    const int t0 = min(ntiles, tid * per), t1 = min(ntiles, t0 + per);
    int my_tiles = 0;
    long long my_nodes = 0;
    for (int t = t0; t < t1; ++t)
        if ((tile_patch[t] >> j) & 1ull) {
            ++my_tiles;
            my_nodes += tile_cnt[(int64_t)t * R + j];
        }
    // exclusive scan of (tiles, nodes) over the block: warp shuffles, then the
    // warp totals in shared memory
    __shared__ int wt[32];
    __shared__ long long wn[32];
    const int lane = tid & 31, w = tid >> 5;
    int it = my_tiles;
    long long in = my_nodes;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, it, o);
        const long long b = __shfl_up_sync(0xffffffffu, in, o);
        if (lane >= o) {
            it += a;
            in += b;
        }
    }
    if (lane == 31) {
        wt[w] = it;
        wn[w] = in;
    }
    __syncthreads();
    if (w == 0) {
        int a = wt[lane];
        long long b = wn[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int c = __shfl_up_sync(0xffffffffu, a, o);
            const long long d = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) {
                a += c;
                b += d;
            }
        }
        wt[lane] = a;
        wn[lane] = b;
    }
    __syncthreads();
    int pos = it - my_tiles + (w > 0 ? wt[w - 1] : 0);
    long long node = in - my_nodes + (w > 0 ? wn[w - 1] : 0);
    const int64_t tbase = tile_off[j];
    const int64_t nbase = node_off[j];
    for (int t = t0; t < t1; ++t)
        if ((tile_patch[t] >> j) & 1ull) {
            const int c = tile_cnt[(int64_t)t * R + j];
            const int64_t e = tbase + pos;
            tile_ids[e] = t;
            tile_nodes[e] = c;
            entry_node0[e] = nbase + node;
            entry_patch[e] = (uint8_t)j;
            ++pos;
            node += c;
        }
}

// One warp per list entry (patch j, tile t): the free nodes of patch j in
// tile t, x fastest, written from the entry's start in node_ids.
__global__ void __launch_bounds__(32) k_patch_nodes(TileGeom tg, const int8_t *__restrict__ code,
                                                    const int *__restrict__ tile_ids,
                                                    const int64_t *__restrict__ entry_node0,
                                                    const uint8_t *__restrict__ entry_patch,
                                                    int *__restrict__ node_ids) {
    const int64_t e = blockIdx.x;
    const int lane = threadIdx.x;
    const int t = tile_ids[e];
    const int8_t j = (int8_t)entry_patch[e];
    const int tx = t % tg.ntx, ty = (t / tg.ntx) % tg.nty, tz = t / (tg.ntx * tg.nty);
    const int x0 = 1 + tx * tg.side, y0 = 1 + ty * tg.side, z0 = tg.dim == 3 ? 1 + tz * tg.side : 0;
    const int cells = tg.dim == 3 ? tg.side * tg.side * tg.side : tg.side * tg.side;
    int64_t at = entry_node0[e];
    for (int b = 0; b < cells; b += 32) {
        const int q = b + lane;
        const int lx = q % tg.side, ly = (q / tg.side) % tg.side, lz = tg.dim == 3 ? q / (tg.side * tg.side) : 0;
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        bool is = false;
        int64_t i = 0;
        if (q < cells && x <= tg.n0 - 2 && y <= tg.n1 - 2 && (tg.dim == 2 || z <= tg.n2 - 2)) {
            i = ((int64_t)z * tg.n1 + y) * tg.n0 + x;
            is = code[i] == j;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, is);
        if (is) node_ids[at + __popc(bal & ((1u << lane) - 1u))] = (int)i;
        at += __popc(bal);
    }
}

}  // namespace

TileGeom tile_geom(const hjbp_problem_desc &d) {
    TileGeom tg{};
    tg.dim = d.dim;
    tg.side = d.dim == 3 ? 8 : kTile;
    tg.n0 = d.n[0];
    tg.n1 = d.n[1];
    tg.n2 = d.dim == 3 ? d.n[2] : 1;
    tg.ntx = (tg.n0 - 2 + tg.side - 1) / tg.side;
    tg.nty = (tg.n1 - 2 + tg.side - 1) / tg.side;
    tg.ntz = d.dim == 3 ? (tg.n2 - 2 + tg.side - 1) / tg.side : 1;
    return tg;
}

void build_patch_lists(hjbp_plan &p, const TileGeom &tg, int ntiles, const uint64_t *tile_patch, const int *tile_cnt,
                       const int64_t *patch_nodes, const int64_t *patch_tiles, const int8_t *code) {
    const int R = p.R;
    cudaStream_t st = p.stream;
    PatchLists &L = p.lists;
    L.built = false;
    L.geom = tg;
    L.R = R;
    L.tile_off.assign(R + 1, 0);
    L.node_off.assign(R + 1, 0);
    for (int j = 0; j < R; ++j) {
        L.tile_off[j + 1] = L.tile_off[j] + patch_tiles[j];
        L.node_off[j + 1] = L.node_off[j] + patch_nodes[j];
    }
    const int64_t ET = L.tile_off[R], EN = L.node_off[R];
    if (ET > L.cap_tiles || EN > L.cap_nodes || !L.d_tile_off)
        throw HjbpError{HJBP_ECUDA, "patch lists exceed their allocation"};
    int64_t *node0 = static_cast<int64_t *>(p.dev_alloc(sizeof(int64_t) * (size_t)(ET > 0 ? ET : 1)));
    uint8_t *epatch = static_cast<uint8_t *>(p.dev_alloc((size_t)(ET > 0 ? ET : 1)));
    // the host vectors outlive the copies (they belong to the plan)
    check_cuda(cudaMemcpyAsync(L.d_tile_off, L.tile_off.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, st),
               "list offsets");
    check_cuda(cudaMemcpyAsync(L.d_node_off, L.node_off.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, st),
               "list offsets");
    if (ET > 0 && ntiles > 0) {
        k_patch_tiles<<<R, kScanThreads, 0, st>>>(ntiles, R, tile_patch, tile_cnt, L.d_tile_off, L.d_node_off,
                                                  L.d_tile_ids, L.d_tile_nodes, node0, epatch);
        ++p.stats.kernel_launches;
        check_cuda(cudaGetLastError(), "patch tile lists");
        k_patch_nodes<<<(unsigned)ET, 32, 0, st>>>(tg, code, L.d_tile_ids, node0, epatch, L.d_node_ids);
        ++p.stats.kernel_launches;
        check_cuda(cudaGetLastError(), "patch node lists");
    }
    L.built = true;
}

// Per-patch sup-norm change at retirement: the largest last change of the
// patch's tiles (each tile stops once its neighbourhood changes by <= tol).
namespace {
__global__ void k_patch_residual(int ntiles, const uint64_t *__restrict__ tile_patch,
                                 const double *__restrict__ last_chg, double *__restrict__ res) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    uint64_t m = tile_patch[t];
    const double v = last_chg[t];
    if (!(v > 0.0)) return;
    while (m) {
        const int j = __ffsll((long long)m) - 1;
        m &= m - 1;
        atomic_max_pos(&res[j], v);
    }
}
}  // namespace

void patch_residuals(hjbp_plan &p, int ntiles, const uint64_t *tile_patch, const double *last_chg) {
    if (!p.patchy || ntiles == 0 || !tile_patch || !last_chg) return;
    cudaStream_t st = p.stream;
    double *res = static_cast<double *>(p.dev_alloc(sizeof(double) * kMaxTargets));
    check_cuda(cudaMemsetAsync(res, 0, sizeof(double) * kMaxTargets, st), "patch residual");
    k_patch_residual<<<(ntiles + 255) / 256, 256, 0, st>>>(ntiles, tile_patch, last_chg, res);
    ++p.stats.kernel_launches;
    check_cuda(cudaGetLastError(), "patch residual");
    check_cuda(cudaMemcpyAsync(p.stats.residual_patch, res, sizeof(double) * kMaxTargets, cudaMemcpyDeviceToHost, st),
               "patch residual");
    check_cuda(cudaStreamSynchronize(st), "patch residual");
}

}  // namespace hjbp
