// serve.cu -- batched and served solves (host orchestration, C ABI).
//
// hjbp_batch_solve runs many plans at once: a pool of worker threads, each
// with its own non-blocking CUDA stream, takes plans from a shared counter and
// runs their solves concurrently, so that problems too small to fill the GPU
// (the batched family has sides of 65..513 nodes) overlap on the device.
//
// The server keeps requests in a queue as validated copies of their
// descriptors, holding no device memory, and admits them while the device
// memory they need fits in a budget (continuous batching: a request starts as
// soon as a worker and enough memory are free, while others are still
// running).  The admitting worker creates the plan, so its device arrays are
// allocated only then, solves it, and the finished plan (values and labels
// resident on the device) waits until the caller collects it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hjbp_device.cuh"
#include "plan.h"

namespace hjbp {
void set_last_error(const std::string &msg);
void set_last_error_static(const char *msg);
std::string validate_desc(const hjbp_problem_desc *d);
}

namespace {

hjbp_status worse(hjbp_status a, hjbp_status b) {
    auto rank = [](hjbp_status s) { return s == HJBP_OK ? 0 : (s == HJBP_ENOCONV ? 1 : 2); };
    return rank(b) > rank(a) ? b : a;
}

// Solve one plan on `stream` (the plan's own stream is restored afterwards).
hjbp_status solve_on(hjbp_plan *p, cudaStream_t stream) {
    cudaStream_t own = p->stream;
    // work queued on the plan's stream (creation) must be done before another stream uses its memory
    cudaStreamSynchronize(own);
    p->stream = stream;
    const hjbp_status s = hjbp_solve(p);
    cudaStreamSynchronize(stream);
    p->stream = own;
    return s;
}

}  // namespace

extern "C" hjbp_status hjbp_batch_solve(hjbp_plan *const *plans, int count, int workers, hjbp_status *statuses) {
    if (!plans || count < 0) {
        hjbp::set_last_error_static("plans is NULL or count negative");
        return HJBP_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (!plans[i]) {
            hjbp::set_last_error_static("NULL plan in the batch");
            return HJBP_EINVAL;
        }
    if (workers <= 0) workers = 8;
    workers = std::max(1, std::min(workers, count));
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> next(0);
    std::vector<hjbp_status> st(count, HJBP_OK);
    std::vector<std::thread> pool;
    std::atomic<int> stream_fail(0);
    for (int w = 0; w < workers; ++w) {
        pool.emplace_back([&, w]() {
            cudaSetDevice(dev);
            cudaStream_t s = nullptr;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                stream_fail = 1;
                return;
            }
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= count) break;
                st[i] = solve_on(plans[i], s);
            }
            cudaStreamDestroy(s);
        });
    }
    for (auto &t : pool) t.join();
    hjbp_status all = HJBP_OK;
    for (int i = 0; i < count; ++i) {
        if (statuses) statuses[i] = st[i];
        all = worse(all, st[i]);
    }
    if (stream_fail && next.load() < count) {
        hjbp::set_last_error_static("could not create worker streams");
        return HJBP_ECUDA;
    }
    return all;
}

// ------------------------------------------------------------------ server --

struct hjbp_server {
    size_t budget = 0;
    size_t in_use = 0;
    int workers = 0;
    int device = 0;
    bool stopping = false;
    uint64_t next_ticket = 1;
    struct Req {
        uint64_t ticket = 0;
        hjbp_problem_desc desc{};          // copy; its arrays point into the vectors below
        std::vector<double> controls, targets, obstacles;
        hjbp_plan *plan = nullptr;         // created by the admitting worker
        size_t bytes = 0;
        hjbp_status status = HJBP_EBUSY;
        std::string error;                 // message of a failed create or solve
        double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    };
    std::deque<uint64_t> queue;               // admitted order (FIFO)
    std::map<uint64_t, Req> reqs;             // every live request
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::thread> pool;
};

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

void worker_loop(hjbp_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        hjbp_server::Req *req = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // first queued request whose memory fits now (FIFO among those that fit)
            for (;;) {
                if (S->stopping) {
                    if (s) cudaStreamDestroy(s);
                    return;
                }
                for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
                    auto &r = S->reqs[*it];
                    if (S->in_use + r.bytes <= S->budget || S->in_use == 0) {
                        req = &r;
                        S->in_use += r.bytes;
                        r.t_start = now_s();
                        S->queue.erase(it);
                        break;
                    }
                }
                if (req) break;
                S->cv.wait(lk);
            }
        }
        // The request is running: nobody else touches it until t_done is set
        // (poll only takes finished requests, destroy waits for running ones).
        // Plans are created on the legacy stream and synchronised; the worker
        // runs the solve on its own stream.
        hjbp_plan *plan = nullptr;
        hjbp_status st = hjbp_create(&req->desc, nullptr, nullptr, &plan);
        if (st == HJBP_OK) st = solve_on(plan, s);
        const std::string err = st == HJBP_OK ? std::string() : std::string(hjbp_last_error());
        {
            std::lock_guard<std::mutex> lk(S->mu);
            req->plan = plan;
            req->status = st;
            req->error = err;
            req->t_done = now_s();
        }
        S->cv.notify_all();
    }
}

// Device bytes a plan needs while solving (outputs plus per-solve scratch).
size_t footprint(const hjbp_problem_desc *d) {
    int64_t N = 1, Nc = 0;
    for (int a = 0; a < d->dim; ++a) N *= d->n[a];
    if (d->n_coarse[0]) {
        Nc = 1;
        for (int a = 0; a < d->dim; ++a) Nc *= d->n_coarse[a];
    }
    const int R = d->target_kind == HJBP_TARGET_BALLS ? d->n_targets : d->n_parts;
    const int rg = R > 4 ? 8 : (R >= 4 ? 4 : R);
    // outputs + codes/h + value buffers + colour planes (FP32 x3, FP64 x2 per group) + phi (R planes)
    // + the reach's cached row sets (2D: 2.75 B per node, 3D: 14.5 B)
    size_t b = (size_t)N * (8 + 1 + 4 + 8 + 8 + 1 + 1 + 1 + 4 * 3 + 16 + (d->dim == 3 ? 15 : 3));
    // patchy: + U0, a*, colour planes, phi, the patch lists (node ids, tile entries)
    if (Nc) b += (size_t)N * (8 + 1 + (size_t)rg * (4 * 3 + 8) + 8 * (size_t)R + 4 + 8) + (size_t)Nc * 40;
    return b + (size_t(8) << 20);
}

}  // namespace

extern "C" hjbp_status hjbp_server_create(size_t device_budget_bytes, int workers, hjbp_server **out) {
    if (!out) {
        hjbp::set_last_error_static("out is NULL");
        return HJBP_EINVAL;
    }
    *out = nullptr;
    hjbp_server *S = new (std::nothrow) hjbp_server();
    if (!S) {
        hjbp::set_last_error_static("host allocation failed");
        return HJBP_ENOMEM;
    }
    if (device_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        device_budget_bytes = fr / 2;
    }
    S->budget = device_budget_bytes;
    S->workers = workers > 0 ? workers : 8;
    cudaGetDevice(&S->device);
    for (int w = 0; w < S->workers; ++w) S->pool.emplace_back(worker_loop, S);
    *out = S;
    return HJBP_OK;
}

extern "C" hjbp_status hjbp_server_submit(hjbp_server *S, const hjbp_problem_desc *desc, uint64_t *ticket) {
    if (!S || !desc || !ticket) {
        hjbp::set_last_error_static("NULL argument");
        return HJBP_EINVAL;
    }
    const std::string err = hjbp::validate_desc(desc);
    if (!err.empty()) {
        hjbp::set_last_error(err);
        return HJBP_EINVAL;
    }
    const size_t bytes = footprint(desc);
    if (bytes > S->budget) {
        hjbp::set_last_error_static("request needs more device memory than the server budget");
        return HJBP_EBUSY;
    }
    try {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const uint64_t t = S->next_ticket++;
            auto &r = S->reqs[t];
            r.ticket = t;
            r.desc = *desc;
            r.controls.assign(desc->controls, desc->controls + (size_t)desc->n_controls * desc->dim);
            r.targets.assign(desc->targets, desc->targets + (size_t)desc->n_targets * (desc->dim + 1));
            if (desc->n_obstacles > 0)
                r.obstacles.assign(desc->obstacles, desc->obstacles + (size_t)desc->n_obstacles * 7);
            r.desc.controls = r.controls.data();
            r.desc.targets = r.targets.data();
            r.desc.obstacles = r.obstacles.empty() ? nullptr : r.obstacles.data();
            r.bytes = bytes;
            r.t_submit = now_s();
            S->queue.push_back(t);
            *ticket = t;
        }
    } catch (const std::bad_alloc &) {
        hjbp::set_last_error_static("host allocation failed");
        return HJBP_ENOMEM;
    }
    S->cv.notify_all();
    return HJBP_OK;
}

extern "C" hjbp_status hjbp_server_poll(hjbp_server *S, uint64_t ticket, hjbp_plan **done, double *latency_s) {
    if (!S || !done) {
        hjbp::set_last_error_static("NULL argument");
        return HJBP_EINVAL;
    }
    *done = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        hjbp::set_last_error_static("unknown ticket");
        return HJBP_EINVAL;
    }
    auto &r = it->second;
    if (r.t_done == 0.0) return HJBP_OK;  // still queued or running
    *done = r.plan;  // NULL when the plan could not be created
    if (latency_s) *latency_s = r.t_done - r.t_submit;
    const hjbp_status st = r.status;
    if (st != HJBP_OK) hjbp::set_last_error(r.error);
    S->in_use -= r.bytes;
    S->reqs.erase(it);
    S->cv.notify_all();
    return st;
}

extern "C" hjbp_status hjbp_server_stats(hjbp_server *S, int *queued, int *running, size_t *bytes_in_use) {
    if (!S) {
        hjbp::set_last_error_static("server is NULL");
        return HJBP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    int run = 0;
    for (auto &kv : S->reqs)
        if (kv.second.t_start != 0.0 && kv.second.t_done == 0.0) ++run;
    if (queued) *queued = (int)S->queue.size();
    if (running) *running = run;
    if (bytes_in_use) *bytes_in_use = S->in_use;
    return HJBP_OK;
}

extern "C" void hjbp_server_destroy(hjbp_server *S) {
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // let running requests finish; queued ones are dropped
        S->queue.clear();
        S->cv.wait(lk, [&] {
            for (auto &kv : S->reqs)
                if (kv.second.t_start != 0.0 && kv.second.t_done == 0.0) return false;
            return true;
        });
        S->stopping = true;
    }
    S->cv.notify_all();
    for (auto &t : S->pool) t.join();
    for (auto &kv : S->reqs) hjbp_destroy(kv.second.plan);
    delete S;
}
