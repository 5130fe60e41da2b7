// autotune.cu -- choice of the launch shape (hjbp_problem_desc.tune) by timing.
//
// The tiled sweeps have a few launch-shape parameters whose best values depend
// on the problem class (dimension, control count, grid size): Gauss-Seidel
// rounds per launch of the value sweep and of the colour transport.  The tuner
// solves the given problem once per candidate shape (after one warm-up solve)
// and keeps the shape with the shortest GPU solve time (hjbp_stats.ms_total,
// CUDA events on the plan's stream).  Results are kept per problem class in
// the process and, optionally, in a text cache file, one line per class:
//   dim side_class control_class patchy options  t0 t1 t2 t3
// side_class = round(log2(n[0] - 1)), control_class = round(log2(n_controls)),
// options = the boundary/add-on flags and whether cones are on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hjbp.h"

namespace {

using Key = std::tuple<int, int, int, int, int>;

std::mutex g_mu;
std::map<Key, std::vector<int>> g_cache;

Key key_of(const hjbp_problem_desc *d) {
    const int side = (int)std::lround(std::log2((double)std::max(2, d->n[0] - 1)));
    const int ctl = (int)std::lround(std::log2((double)std::max(1, d->n_controls)));
    const int opts = (d->flags & (HJBP_FLAG_DIRICHLET | HJBP_FLAG_WARM_START | HJBP_FLAG_CAUSAL_SWEEPS)) |
                     (d->reduce_r != 0.0 ? 32 : 0) | (d->dyn << 6);
    return Key{d->dim, side, ctl, d->n_coarse[0] != 0 ? 1 : 0, opts};
}

void load_file(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int a, b, c, e, o, t0, t1, t2, t3;
    while (std::fscanf(f, "%d %d %d %d %d %d %d %d %d", &a, &b, &c, &e, &o, &t0, &t1, &t2, &t3) == 9)
        g_cache[Key{a, b, c, e, o}] = {t0, t1, t2, t3};
    std::fclose(f);
}

void append_file(const char *path, const Key &k, const std::vector<int> &t) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                 std::get<4>(k), t[0], t[1], t[2], t[3]);
    std::fclose(f);
}

// GPU time of one solve of d with the launch shape t (after a warm-up solve);
// a negative value when the shape fails.
double time_shape(const hjbp_problem_desc *d, void *stream, const std::vector<int> &t, hjbp_status *err) {
    hjbp_problem_desc q = *d;
    for (int i = 0; i < 4; ++i) q.tune[i] = t[i];
    hjbp_plan *plan = nullptr;
    hjbp_status s = hjbp_create(&q, stream, nullptr, &plan);
    if (s != HJBP_OK) {
        *err = s;
        return -1.0;
    }
    double best = -1.0;
    for (int rep = 0; rep < 2 && s == HJBP_OK; ++rep) {
        s = hjbp_solve(plan);
        if (s == HJBP_OK) s = hjbp_sync(plan);
        hjbp_stats st;
        if (s == HJBP_OK && hjbp_get_stats(plan, &st) == HJBP_OK && rep == 1) best = st.ms_total;
    }
    hjbp_destroy(plan);
    if (s != HJBP_OK) *err = s;
    return s == HJBP_OK ? best : -1.0;
}

}  // namespace

extern "C" hjbp_status hjbp_autotune(const hjbp_problem_desc *desc, void *cuda_stream, const char *cache_path,
                                     int tune_out[4], int *from_cache) {
    if (!desc || !tune_out) return HJBP_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cache_path) load_file(cache_path);
    const Key k = key_of(desc);
    auto it = g_cache.find(k);
    if (it != g_cache.end()) {
        for (int i = 0; i < 4; ++i) tune_out[i] = it->second[i];
        if (from_cache) *from_cache = 1;
        return HJBP_OK;
    }
    // candidates: value rounds x colour-transport rounds (one warp per tile,
    // one reach pass: the measured alternatives were slower everywhere)
    std::vector<int> vr = desc->dim == 2 ? std::vector<int>{2, 3, 4} : std::vector<int>{1, 2};
    std::vector<int> pr = desc->n_coarse[0] == 0 ? std::vector<int>{0}
                                                 : (desc->dim == 2 ? std::vector<int>{2, 3, 4} : std::vector<int>{1, 2, 3});
    std::vector<int> best_t;
    double best_ms = -1.0;
    hjbp_status err = HJBP_OK;
    for (int a : vr)
        for (int b : pr) {
            const std::vector<int> t{a, b, 0, 0};
            const double ms = time_shape(desc, cuda_stream, t, &err);
            if (ms >= 0.0 && (best_ms < 0.0 || ms < best_ms)) {
                best_ms = ms;
                best_t = t;
            }
        }
    if (best_ms < 0.0) return err != HJBP_OK ? err : HJBP_ECUDA;
    g_cache[k] = best_t;
    if (cache_path) append_file(cache_path, k, best_t);
    for (int i = 0; i < 4; ++i) tune_out[i] = best_t[i];
    if (from_cache) *from_cache = 0;
    return HJBP_OK;
}
