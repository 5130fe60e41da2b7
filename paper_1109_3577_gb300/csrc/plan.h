// plan.h -- host-side state of one solve (internal to libhjbp).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hjbp.h"

// Tiling of the fine grid for the tile sweeps and the patch lists: tiles of
// side^dim interior nodes starting at node (1, 1[, 1]), ntx x nty [x ntz].
struct TileGeom {
    int dim, side, ntx, nty, ntz, n0, n1, n2;
};

// Patch compaction (Sec. 3): per patch j its tiles and nodes in CSR form
// (see compact.cu).  The device arrays are allocated at create with their
// largest sizes and filled by every patchy solve.
struct PatchLists {
    bool built = false;
    int R = 0;
    TileGeom geom{};
    std::vector<int64_t> tile_off, node_off;   // host copies of the offsets (R + 1 each)
    int64_t *d_tile_off = nullptr, *d_node_off = nullptr;
    int *d_tile_ids = nullptr, *d_tile_nodes = nullptr, *d_node_ids = nullptr;
    int64_t cap_tiles = 0, cap_nodes = 0;      // allocated entries
};

struct hjbp_plan {
    // --- descriptor (copied at create) ---
    hjbp_problem_desc desc;
    std::vector<double> controls;   // n_controls x dim
    std::vector<double> targets;    // n_targets x (dim + 1)
    std::vector<double> obstacles;  // n_obstacles x 7
    int R = 0;                      // patches (target parts)
    std::vector<double> dirs;       // per control: unit direction of f (dim each)
    std::vector<double> hfac;       // per control: h_{i,a} = hfac[a] h_i
    bool patchy = false;
    int64_t N = 0, Nc = 0;          // fine / coarse node counts
    double k = 0.0, kc = 0.0;       // fine / coarse spacing

    // --- execution ---
    cudaStream_t stream = nullptr;
    hjbp_allocator alloc{};
    bool has_alloc = false;
    bool solved = false;
    hjbp_status last_status = HJBP_ESTATE;
    hjbp_stats stats{};
    std::vector<double> init;       // caller's start values (hjbp_set_initial), empty: none
    bool cone_pairs = false;        // AO3 cones available in the symmetric pair form
    int *pinned_count = nullptr;    // pinned host word for the sweep loops' readbacks (lazy)
    // CUDA events for per-launch timing (HJBP_FLAG_TIME_SWEEPS), created once
    // and reused by every solve: creating and destroying events per launch
    // costs more host time than the launches
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    cudaEvent_t pooled_event() {
        if (events_used == events.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            events.push_back(e);
        }
        return events[events_used++];
    }
    ~hjbp_plan() {
        if (pinned_count) cudaFreeHost(pinned_count);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
    }

    // --- device arrays owned by the plan ---
    struct Block {
        void *ptr;
        size_t bytes;
    };
    std::vector<Block> blocks;

    double *u_out = nullptr;        // FP64 values (output)
    int8_t *label_out = nullptr;    // labels (output)
    double *u_coarse = nullptr;     // coarse values (Step 1)
    double *u0 = nullptr;           // U_P^(0) (Step 2)
    uint8_t *astar = nullptr;       // coarse feedback (Step 2)
    double *phi = nullptr;          // R x N colour fields (Step 3.1)
    float *u32 = nullptr;           // FP32 bulk values
    PatchLists lists;               // per-patch tile and node lists (patchy solves)

    void *dev_alloc(size_t bytes);  // throws std::bad_alloc on failure
    void release_all();
};

namespace hjbp {

struct HjbpError {
    hjbp_status status;
    std::string msg;
};

// Raise an HjbpError on a CUDA failure.
void check_cuda(cudaError_t e, const char *what);

void set_last_error(const std::string &msg);

// 2D and 3D drivers: run the whole solve on the plan's stream.
hjbp_status solve2d(hjbp_plan &p);
hjbp_status solve3d(hjbp_plan &p);

// Tiling of the plan's fine grid (32^2 tiles in 2D, 8^3 in 3D).
TileGeom tile_geom(const hjbp_problem_desc &d);

// Fill p.lists from the per-tile patch masks and per-(tile, patch) node
// counts left by the compaction kernels; counts are the per-patch totals.
void build_patch_lists(hjbp_plan &p, const TileGeom &tg, int ntiles, const uint64_t *tile_patch, const int *tile_cnt,
                       const int64_t *patch_nodes, const int64_t *patch_tiles, const int8_t *code);

// stats.residual_patch from the tiles' last changes (FP64).
void patch_residuals(hjbp_plan &p, int ntiles, const uint64_t *tile_patch, const double *last_chg);

}  // namespace hjbp
