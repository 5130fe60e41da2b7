// api.cu -- the C ABI of libhjbp (see include/hjbp.h): descriptor validation,
// device memory, dispatch to the 2D / 3D drivers, result copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "hjbp_device.cuh"
#include "plan.h"

namespace hjbp {

static thread_local std::string g_last_error;
static thread_local const char *g_last_static = nullptr;

void set_last_error(const std::string &msg) {
    g_last_error = msg;
    g_last_static = nullptr;
}

// Records a message with static storage without copying it (used by the
// entry point that must not allocate).
void set_last_error_static(const char *msg) { g_last_static = msg; }

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        throw HjbpError{HJBP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
    }
}

}  // namespace hjbp

using hjbp::HjbpError;

void *hjbp_plan::dev_alloc(size_t bytes) {
    void *ptr = nullptr;
    if (has_alloc) {
        ptr = alloc.alloc(bytes, stream, alloc.ctx);
        if (!ptr) throw HjbpError{HJBP_ENOMEM, "allocator returned NULL for " + std::to_string(bytes) + " bytes"};
    } else {
        cudaError_t e = cudaMallocAsync(&ptr, bytes, stream);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            throw HjbpError{HJBP_ENOMEM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed"};
        }
    }
    blocks.push_back({ptr, bytes});
    return ptr;
}

void hjbp_plan::release_all() {
    for (auto it = blocks.rbegin(); it != blocks.rend(); ++it) {
        if (has_alloc) alloc.release(it->ptr, it->bytes, stream, alloc.ctx);
        else cudaFreeAsync(it->ptr, stream);
    }
    blocks.clear();
    u_out = nullptr;
    label_out = nullptr;
    u_coarse = u0 = phi = nullptr;
    astar = nullptr;
    u32 = nullptr;
}

static hjbp_status fail(hjbp_status s, const std::string &msg) {
    hjbp::set_last_error(msg);
    return s;
}

// The descriptor checks of hjbp_create, host arithmetic only ("" when valid);
// the server runs them at submit, before it queues a request.
namespace hjbp {
std::string validate_desc(const hjbp_problem_desc *d) {
    if (!d) return "descriptor is NULL";
    if (d->dim != 2 && d->dim != 3) return "dim must be 2 or 3";
    for (int a = 0; a < d->dim; ++a) {
        if (d->n[a] < 3) return "every axis needs at least 3 nodes";
        if (!(d->hi[a] > d->lo[a])) return "hi must exceed lo on every axis";
    }
    const double k = (d->hi[0] - d->lo[0]) / (d->n[0] - 1);
    for (int a = 1; a < d->dim; ++a) {
        const double ka = (d->hi[a] - d->lo[a]) / (d->n[a] - 1);
        if (std::fabs(ka - k) > 1e-12 * k) return "grid spacing must be equal on every axis";
    }
    if (d->n_coarse[0] != 0) {
        for (int a = 0; a < d->dim; ++a) {
            if (d->n_coarse[a] < 3) return "every coarse axis needs at least 3 nodes";
            if (d->n_coarse[a] > d->n[a]) return "coarse grid finer than the fine grid";
        }
    }
    if (d->speed < HJBP_C_ONE || d->speed > HJBP_C_FAN) return "unknown speed field";
    if (d->speed == HJBP_C_SIN3D && d->dim != 3) return "SIN3D needs dim 3";
    if ((d->speed == HJBP_C_SINCOS2D || d->speed == HJBP_C_FOURIER2D) && d->dim != 2) return "2D speed field with dim 3";
    if (d->n_controls < 1 || d->n_controls > HJBP_MAX_CONTROLS) return "n_controls out of range";
    // the coarse feedback a* is one byte per node, 255 meaning "no feedback"
    if (d->n_coarse[0] != 0 && d->n_controls > 255) return "patchy solves take at most 255 controls";
    if (!d->controls) return "controls is NULL";
    bool moving = false;
    for (int m = 0; m < d->n_controls; ++m) {
        double s = 0.0;
        for (int a = 0; a < d->dim; ++a) {
            const double v = d->controls[m * d->dim + a];
            if (!std::isfinite(v)) return "control component not finite";
            s += v * v;
        }
        if (d->dyn == HJBP_DYN_BROCKETT) {
            // rows (a1, a2, unused); a = 0 is allowed but cannot move
            if (d->controls[m * d->dim] != 0.0 || d->controls[m * d->dim + 1] != 0.0) moving = true;
        } else if (std::fabs(std::sqrt(s) - 1.0) > 1e-9) {
            return "controls must be unit vectors";
        }
    }
    if (d->dyn == HJBP_DYN_BROCKETT && !moving) return "Brockett's controls are all zero";
    if (d->n_targets < 1 || d->n_targets > HJBP_MAX_TARGETS) return "n_targets out of range";
    if (d->target_kind < HJBP_TARGET_BALLS || d->target_kind > HJBP_TARGET_ORTHANTS) return "unknown target kind";
    if (d->target_kind == HJBP_TARGET_ORTHANTS && d->n_parts != (1 << d->dim)) return "orthant targets need n_parts = 2^dim";
    if (d->target_kind != HJBP_TARGET_BALLS) {
        if (d->n_parts < 1 || d->n_parts > HJBP_MAX_TARGETS) return "n_parts out of range";
    }
    if (d->dyn != HJBP_DYN_SPEED && d->dyn != HJBP_DYN_DRIFT && d->dyn != HJBP_DYN_BROCKETT)
        return "unknown dynamics";
    if (d->dyn == HJBP_DYN_BROCKETT) {
        if (d->dim != 3) return "Brockett's integrator is 3D";
        if (d->speed != HJBP_C_ONE) return "Brockett's integrator takes the speed field HJBP_C_ONE";
        if (d->flags & HJBP_FLAG_TILE_QUEUE) return "the tile queue runs the 2D path";
    }
    if (d->dyn == HJBP_DYN_DRIFT) {
        if (d->dim != 2) return "drift dynamics are 2D";
        if (d->speed != HJBP_C_ONE) return "drift dynamics take the speed field HJBP_C_ONE";
        for (int a = 0; a < 4; ++a)
            if (!std::isfinite(d->drift[a])) return "drift not finite";
        if (d->controls)
            for (int m = 0; m < d->n_controls; ++m) {
                double n2 = 0.0;
                for (int c = 0; c < d->dim; ++c) {
                    const double f = d->drift[0] * d->controls[m * d->dim + c] + d->drift[1 + c];
                    n2 += f * f;
                }
                if (!(std::sqrt(n2) > 1e-15)) return "a control has zero velocity under the drift";
            }
    }
    if (!d->targets) return "targets is NULL";
    for (int j = 0; j < d->n_targets; ++j)
        for (int a = 0; a <= d->dim; ++a)
            if (!std::isfinite(d->targets[j * (d->dim + 1) + a])) return "target entry not finite";
    if (const char *e = hjbp::check_obstacles(d)) return e;
    if (!(d->tol > 0.0)) return "tol must be positive";
    if (d->precision != HJBP_FP64 && d->precision != HJBP_FP32_POLISH64) return "unknown precision";
    if ((d->flags & (HJBP_FLAG_DIRICHLET | HJBP_FLAG_WARM_START | HJBP_FLAG_CAUSAL_SWEEPS)) && d->n_coarse[0] == 0)
        return "Dirichlet patch boundaries, the warm start and causal sweeps need a patchy solve (n_coarse)";
    if (!(d->reduce_r == 0.0 || d->reduce_r >= 1.0) || !std::isfinite(d->reduce_r))
        return "reduce_r must be 0 or at least 1";
    if (d->reduce_r != 0.0 && d->n_coarse[0] == 0) return "reduce_r needs a patchy solve (n_coarse)";
    if (d->reduce_r != 0.0 && d->dim == 2 && d->n_controls > 64) return "reduce_r on the 2D path needs <= 64 controls";
    if (d->reduce_r != 0.0 && d->dyn == HJBP_DYN_BROCKETT) return "control cones need f = c(x) a or the drift";
    if (d->speed == HJBP_C_FOURIER2D) {
        double norm = 0.0;
        for (int i = 0; i < 16; ++i) norm += std::fabs(d->speed_params[i]);
        if (!(norm > 0.0)) return "Fourier speed field needs a nonzero coefficient";
    }
    return "";
}
}  // namespace hjbp

extern "C" {

int hjbp_version(void) { return 100; }

const char *hjbp_last_error(void) {
    return hjbp::g_last_static ? hjbp::g_last_static : hjbp::g_last_error.c_str();
}

hjbp_status hjbp_create(const hjbp_problem_desc *desc, void *cuda_stream, const hjbp_allocator *allocator,
                        hjbp_plan **out) {
    if (!out) return fail(HJBP_EINVAL, "out is NULL");
    *out = nullptr;
    const std::string err = hjbp::validate_desc(desc);
    if (!err.empty()) return fail(HJBP_EINVAL, err);
    hjbp_plan *p = new (std::nothrow) hjbp_plan();
    if (!p) return fail(HJBP_ENOMEM, "host allocation failed");
    try {
        p->desc = *desc;
        p->controls.assign(desc->controls, desc->controls + (size_t)desc->n_controls * desc->dim);
        p->targets.assign(desc->targets, desc->targets + (size_t)desc->n_targets * (desc->dim + 1));
        p->desc.controls = p->controls.data();
        p->desc.targets = p->targets.data();
        if (desc->n_obstacles > 0)
            p->obstacles.assign(desc->obstacles, desc->obstacles + (size_t)desc->n_obstacles * 7);
        p->desc.obstacles = p->obstacles.empty() ? nullptr : p->obstacles.data();
        p->R = desc->target_kind == HJBP_TARGET_BALLS ? desc->n_targets : desc->n_parts;
        // per-control direction of f and time-step factor (|h f| = k, Sec. 2.1)
        p->dirs.assign((size_t)desc->n_controls * desc->dim, 0.0);
        p->hfac.assign((size_t)desc->n_controls, 1.0);
        for (int m = 0; m < desc->n_controls; ++m) {
            const double *a = desc->controls + (size_t)m * desc->dim;
            double *dv = p->dirs.data() + (size_t)m * desc->dim;
            if (desc->dyn == HJBP_DYN_DRIFT) {
                double f[3] = {0.0, 0.0, 0.0}, n2 = 0.0;
                for (int c = 0; c < desc->dim; ++c) {
                    f[c] = desc->drift[0] * a[c];
                    f[c] += desc->drift[1 + c];
                    n2 += f[c] * f[c];
                }
                const double nf = std::sqrt(n2);
                if (!(nf > 1e-15)) {
                    delete p;
                    return fail(HJBP_EINVAL, "a control has zero velocity under the drift");
                }
                for (int c = 0; c < desc->dim; ++c) {
                    const double v = f[c] / nf;
                    dv[c] = std::fabs(v) < 1e-15 ? 0.0 : v;
                }
                p->hfac[m] = 1.0 / nf;
            } else {
                for (int c = 0; c < desc->dim; ++c) dv[c] = a[c];
            }
        }
        p->stream = static_cast<cudaStream_t>(cuda_stream);
        if (allocator && allocator->alloc && allocator->release) {
            p->alloc = *allocator;
            p->has_alloc = true;
        }
        const int d = desc->dim;
        p->patchy = desc->n_coarse[0] != 0;
        p->N = 1;
        p->Nc = 1;
        for (int a = 0; a < d; ++a) {
            p->N *= desc->n[a];
            if (p->patchy) p->Nc *= desc->n_coarse[a];
        }
        if (!p->patchy) p->Nc = 0;
        p->k = (desc->hi[0] - desc->lo[0]) / (desc->n[0] - 1);
        // coarse spacing formed as k (n-1) / (n~-1)
        p->kc = p->patchy ? p->k * (double)(desc->n[0] - 1) / (double)(desc->n_coarse[0] - 1) : 0.0;
        p->u_out = static_cast<double *>(p->dev_alloc(sizeof(double) * p->N));
        p->label_out = static_cast<int8_t *>(p->dev_alloc(p->N));
        if (desc->precision == HJBP_FP32_POLISH64) p->u32 = static_cast<float *>(p->dev_alloc(sizeof(float) * p->N));
        if (p->patchy) {
            p->u_coarse = static_cast<double *>(p->dev_alloc(sizeof(double) * p->Nc));
            p->u0 = static_cast<double *>(p->dev_alloc(sizeof(double) * p->N));
            p->astar = static_cast<uint8_t *>(p->dev_alloc(p->N));
            p->phi = static_cast<double *>(p->dev_alloc(sizeof(double) * p->N * p->R));
            // the patch lists at their largest: every node, every (tile, patch) pair
            const TileGeom tg = hjbp::tile_geom(*desc);
            const int64_t nt = (int64_t)tg.ntx * tg.nty * tg.ntz;
            PatchLists &L = p->lists;
            L.cap_nodes = std::max<int64_t>(p->N, 1);
            L.cap_tiles = std::max<int64_t>(nt * p->R, 1);
            const size_t bytes = sizeof(int64_t) * 2 * (size_t)(p->R + 1) + sizeof(int) * (size_t)L.cap_nodes +
                                 2 * sizeof(int) * (size_t)L.cap_tiles;
            unsigned char *blk = static_cast<unsigned char *>(p->dev_alloc(bytes));
            L.d_tile_off = reinterpret_cast<int64_t *>(blk);
            L.d_node_off = L.d_tile_off + (p->R + 1);
            L.d_node_ids = reinterpret_cast<int *>(L.d_node_off + (p->R + 1));
            L.d_tile_ids = L.d_node_ids + L.cap_nodes;
            L.d_tile_nodes = L.d_tile_ids + L.cap_tiles;
        }
        hjbp::check_cuda(cudaStreamSynchronize(p->stream), "create");
    } catch (const HjbpError &e) {
        p->release_all();
        delete p;
        return fail(e.status, e.msg);
    } catch (const std::bad_alloc &) {
        p->release_all();
        delete p;
        return fail(HJBP_ENOMEM, "host allocation failed");
    }
    *out = p;
    return HJBP_OK;
}

hjbp_status hjbp_solve(hjbp_plan *p) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    // per-solve scratch lives after the fixed outputs; free it from earlier solves
    const size_t keep = (size_t)(p->patchy ? 7 : 2) + (p->u32 ? 1 : 0);
    try {
        while (p->blocks.size() > keep) {
            auto b = p->blocks.back();
            if (p->has_alloc) p->alloc.release(b.ptr, b.bytes, p->stream, p->alloc.ctx);
            else cudaFreeAsync(b.ptr, p->stream);
            p->blocks.pop_back();
        }
        p->events_used = 0;   // the timing events of the last solve are free again
        hjbp_status s = p->desc.dim == 2 ? hjbp::solve2d(*p) : hjbp::solve3d(*p);
        // release per-solve scratch
        while (p->blocks.size() > keep) {
            auto b = p->blocks.back();
            if (p->has_alloc) p->alloc.release(b.ptr, b.bytes, p->stream, p->alloc.ctx);
            else cudaFreeAsync(b.ptr, p->stream);
            p->blocks.pop_back();
        }
        hjbp::check_cuda(cudaStreamSynchronize(p->stream), "solve");
        p->solved = true;
        p->last_status = s;
        if (s == HJBP_ENOCONV) hjbp::set_last_error("sweep cap reached before convergence");
        return s;
    } catch (const HjbpError &e) {
        cudaStreamSynchronize(p->stream);
        cudaGetLastError();
        p->last_status = e.status;
        return fail(e.status, e.msg);
    } catch (const std::bad_alloc &) {
        p->last_status = HJBP_ENOMEM;
        return fail(HJBP_ENOMEM, "host allocation failed");
    }
}

hjbp_status hjbp_sync(hjbp_plan *p) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    const cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(HJBP_ECUDA, cudaGetErrorString(e));
    if (!p->solved && p->last_status == HJBP_ESTATE) return fail(HJBP_ESTATE, "plan has not been solved");
    return p->last_status;
}

hjbp_status hjbp_set_initial(hjbp_plan *p, const double *u_init) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    if (p->desc.dim != 2) return fail(HJBP_EINVAL, "start values are implemented for 2D plans");
    try {
        if (!u_init) {
            p->init.clear();
            return HJBP_OK;
        }
        for (int64_t i = 0; i < p->N; ++i)
            if (std::isnan(u_init[i]) || u_init[i] < 0.0) return fail(HJBP_EINVAL, "start values must be >= 0 or +inf");
        p->init.assign(u_init, u_init + p->N);
    } catch (const std::bad_alloc &) {
        return fail(HJBP_ENOMEM, "host allocation failed");
    }
    return HJBP_OK;
}

static hjbp_status copy_out(hjbp_plan *p, void *host, const void *dev, size_t bytes) {
    if (!p || !host) return fail(HJBP_EINVAL, "NULL argument");
    if (!p->solved) return fail(HJBP_ESTATE, "plan has not been solved");
    if (!dev) return fail(HJBP_EINVAL, "array not produced by this plan");
    cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(HJBP_ECUDA, cudaGetErrorString(e));
    return HJBP_OK;
}

hjbp_status hjbp_get_values(hjbp_plan *p, double *host_out) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    return copy_out(p, host_out, p->u_out, sizeof(double) * p->N);
}

hjbp_status hjbp_get_labels(hjbp_plan *p, int8_t *host_out) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    return copy_out(p, host_out, p->label_out, (size_t)p->N);
}

hjbp_status hjbp_get_intermediate(hjbp_plan *p, int which, void *host_out, size_t bytes) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
    case HJBP_OUT_UCOARSE: src = p->u_coarse; need = sizeof(double) * p->Nc; break;
    case HJBP_OUT_U0: src = p->u0; need = sizeof(double) * p->N; break;
    case HJBP_OUT_ASTAR: src = p->astar; need = (size_t)p->N; break;
    case HJBP_OUT_PHI: src = p->phi; need = sizeof(double) * p->N * p->R; break;
    case HJBP_OUT_U32: src = p->u32; need = sizeof(float) * p->N; break;
    default: return fail(HJBP_EINVAL, "unknown intermediate id");
    }
    if (!src) return fail(HJBP_EINVAL, "intermediate not produced by this plan");
    if (bytes < need) return fail(HJBP_EINVAL, "host buffer too small");
    if (which != HJBP_OUT_ASTAR) return copy_out(p, host_out, src, need);
    // a* is kept as uint8 (255 = undefined) and returned as int32 (-1 = undefined)
    std::string tmp(need, '\0');
    hjbp_status s = copy_out(p, &tmp[0], src, need);
    if (s != HJBP_OK) return s;
    int32_t *o = static_cast<int32_t *>(host_out);
    if (bytes < need * sizeof(int32_t)) return fail(HJBP_EINVAL, "host buffer too small (int32 per node)");
    for (size_t i = 0; i < need; ++i) {
        const uint8_t v = (uint8_t)tmp[i];
        o[i] = v == 255 ? -1 : (int32_t)v;
    }
    return HJBP_OK;
}

hjbp_status hjbp_get_device_views(hjbp_plan *p, const double **u, const int8_t **labels) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    if (u) *u = p->u_out;
    if (labels) *labels = p->label_out;
    return HJBP_OK;
}

hjbp_status hjbp_get_stats(hjbp_plan *p, hjbp_stats *out) {
    if (!p || !out) return fail(HJBP_EINVAL, "NULL argument");
    *out = p->stats;
    return HJBP_OK;
}

hjbp_status hjbp_get_patch_lists(hjbp_plan *p, int64_t *tile_offsets, int32_t *tile_ids, int32_t *tile_nodes,
                                 int64_t *node_offsets, int32_t *node_ids) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    if (!p->patchy || !p->lists.built) return fail(HJBP_ESTATE, "no patchy solve has built patch lists");
    const PatchLists &L = p->lists;
    const int R = L.R;
    if (tile_offsets) std::memcpy(tile_offsets, L.tile_off.data(), sizeof(int64_t) * (R + 1));
    if (node_offsets) std::memcpy(node_offsets, L.node_off.data(), sizeof(int64_t) * (R + 1));
    const int64_t ET = L.tile_off[R], EN = L.node_off[R];
    try {
        if (tile_ids && ET)
            hjbp::check_cuda(cudaMemcpyAsync(tile_ids, L.d_tile_ids, sizeof(int32_t) * ET, cudaMemcpyDeviceToHost,
                                             p->stream), "tile ids");
        if (tile_nodes && ET)
            hjbp::check_cuda(cudaMemcpyAsync(tile_nodes, L.d_tile_nodes, sizeof(int32_t) * ET, cudaMemcpyDeviceToHost,
                                             p->stream), "tile nodes");
        if (node_ids && EN)
            hjbp::check_cuda(cudaMemcpyAsync(node_ids, L.d_node_ids, sizeof(int32_t) * EN, cudaMemcpyDeviceToHost,
                                             p->stream), "node ids");
        hjbp::check_cuda(cudaStreamSynchronize(p->stream), "patch lists");
    } catch (const HjbpError &e) {
        return fail(e.status, e.msg);
    }
    return HJBP_OK;
}

hjbp_status hjbp_get_sizes(hjbp_plan *p, int64_t *n_nodes, int64_t *n_coarse_nodes) {
    if (!p) return fail(HJBP_EINVAL, "plan is NULL");
    if (n_nodes) *n_nodes = p->N;
    if (n_coarse_nodes) *n_coarse_nodes = p->Nc;
    return HJBP_OK;
}

void hjbp_destroy(hjbp_plan *p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    p->release_all();
    cudaStreamSynchronize(p->stream);
    delete p;
}

}  // extern "C"
