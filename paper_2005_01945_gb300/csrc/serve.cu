// serve.cu -- continuous-batching request loop over the bootstrapping kernels.
//
// Requests (one circuit instance each: a gate, an add, a mul, a matvec) are
// submitted from any host thread.  A worker thread owns one CUDA stream and
// a device ciphertext pool sized by an HBM budget; it admits queued requests
// in arrival order whenever their rows fit in the pool (first fit), copies
// their inputs in, and then runs iterations: one iteration is one batched
// blind-rotation launch plus one key-switch launch over the next level of
// every admitted request (oldest first, up to a gate cap).  A request's
// level k+1 is enqueued right behind level k on the same stream, so the
// worker keeps two iterations in flight and the device never waits for the
// host; requests admitted meanwhile join the next iteration.  When a
// request's last level has run, its outputs are gathered to the caller's
// buffer, and once that iteration's event has completed its pool rows are
// freed and its latency (submit to completion, host clock) is recorded.
//
// This is the paper's level-by-level batching (bit coalescing and compound
// gates, section V-A) generalised across requests that arrive over time.
// Every wait of the worker is bounded; a wait that runs out fails the
// in-flight requests with TFHE_ETIMEOUT instead of hanging.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "netlist.h"
#include "runtime.h"

namespace tgb {

static double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over pool rows.
struct RowAlloc {
    std::map<long, long> free_;  // start -> length
    long capacity = 0;
    void init(long cap)
    {
        capacity = cap;
        free_.clear();
        if (cap > 0)
            free_[0] = cap;
    }
    long alloc(long n)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                const long start = it->first, len = it->second;
                free_.erase(it);
                if (len > n)
                    free_[start + n] = len - n;
                return start;
            }
        return -1;
    }
    void release(long start, long n)
    {
        auto it = free_.emplace(start, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct SrvReq {
    uint64_t id = 0;
    tfhe_request r{};
    std::shared_ptr<const Netlist> nl;
    long rows0 = 0, rows1 = 0, inst_rows = 0, base = -1;
    int next_level = 1;
    int state = 0;                 // 0 queued, 1 admitted, 2 done, < 0 error code
    double t_submit = 0, t_done = 0;
    std::vector<long> level_start; // gates sorted by level: [level_start[l-1], level_start[l])
    std::vector<int32_t> order;    // gate indices sorted by level
};

struct Iter {                      // one in-flight iteration (pinned staging + device copy)
    uint8_t *h_ops = nullptr, *d_ops = nullptr;
    int32_t *h_idx = nullptr, *d_idx = nullptr;  // [4][cap]: a, b, c, out
    int32_t *h_out = nullptr, *d_out = nullptr;  // output rows of finishing requests
    long cap = 0, out_cap = 0;        // gates / output rows the buffers hold
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<SrvReq *> finishing;
    long gates = 0;
};

struct Server {
    tfhe_ctx *ctx = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stopping = false;
    cudaStream_t st = nullptr;
    int32_t *pool = nullptr;
    long pool_rows = 0;
    RowAlloc rows;
    int32_t *big = nullptr;
    long big_rows = 0, max_batch = 0;
    Iter it[2];
    uint64_t seq = 0, next_id = 1;
    std::deque<SrvReq *> queue;            // submitted, not admitted
    std::vector<SrvReq *> running;         // admitted, levels left
    std::unordered_map<uint64_t, SrvReq *> all;
    std::vector<double> latencies;
    tfhe_serve_info stats{};
    int fatal = TFHE_OK;
    double t_first_submit = -1, t_last_done = 0;
    int wait_limit_ms = 120000;
};

static int srv_fail_all(Server &S, int code)
{
    std::lock_guard<std::mutex> lock(S.mu);
    S.fatal = code;
    for (SrvReq *r : S.running)
        r->state = code, r->t_done = now_ms(), S.stats.failed++;
    for (SrvReq *r : S.queue)
        r->state = code, r->t_done = now_ms(), S.stats.failed++;
    S.running.clear();
    S.queue.clear();
    S.cv.notify_all();
    return code;
}

// Bounded wait for an iteration's event.
static int srv_wait(Server &S, Iter &I)
{
    if (!I.busy)
        return TFHE_OK;
    const double deadline = now_ms() + S.wait_limit_ms;
    for (;;) {
        cudaError_t e = cudaEventQuery(I.ev);
        if (e == cudaSuccess)
            break;
        if (e != cudaErrorNotReady) {
            (void)cudaGetLastError();
            return TFHE_ECUDA;
        }
        if (now_ms() > deadline)
            return TFHE_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    I.busy = false;
    const double t = now_ms();
    std::lock_guard<std::mutex> lock(S.mu);
    for (SrvReq *r : I.finishing) {
        r->state = 2;
        r->t_done = t;
        S.rows.release(r->base, r->inst_rows);
        S.latencies.push_back(r->t_done - r->t_submit);
        S.stats.completed++;
        S.t_last_done = t;
    }
    I.finishing.clear();
    S.cv.notify_all();
    return TFHE_OK;
}

// Grows an iteration's staging buffers (only between uses: the caller has
// waited for the iteration's event).
static bool iter_reserve(Iter &I, long gates, long outs)
{
    bool ok = true;
    if (I.cap < gates) {
        const long c = std::max(gates, 2 * I.cap);
        cudaFree(I.d_ops);
        cudaFreeHost(I.h_ops);
        cudaFree(I.d_idx);
        cudaFreeHost(I.h_idx);
        I.d_ops = I.h_ops = nullptr;
        I.d_idx = I.h_idx = nullptr;
        ok = cudaMalloc(&I.d_ops, c) == cudaSuccess &&
             cudaMallocHost(&I.h_ops, c) == cudaSuccess &&
             cudaMalloc(&I.d_idx, 4 * c * sizeof(int32_t)) == cudaSuccess &&
             cudaMallocHost(&I.h_idx, 4 * c * sizeof(int32_t)) == cudaSuccess;
        I.cap = ok ? c : 0;
    }
    if (ok && I.out_cap < outs) {
        const long c = std::max(outs, 2 * I.out_cap);
        cudaFree(I.d_out);
        cudaFreeHost(I.h_out);
        I.d_out = I.h_out = nullptr;
        ok = cudaMalloc(&I.d_out, c * sizeof(int32_t)) == cudaSuccess &&
             cudaMallocHost(&I.h_out, c * sizeof(int32_t)) == cudaSuccess;
        I.out_cap = ok ? c : 0;
    }
    if (!ok)
        (void)cudaGetLastError();
    return ok;
}

static void srv_loop(Server *Sp)
{
    Server &S = *Sp;
    tfhe_ctx *ctx = S.ctx;
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<SrvReq *> admitted;
        {
            std::unique_lock<std::mutex> lock(S.mu);
            if (S.running.empty() && !S.it[0].busy && !S.it[1].busy) {
                S.cv.wait_for(lock, std::chrono::milliseconds(20), [&] {
                    return S.stopping || !S.queue.empty();
                });
                if (S.stopping && S.queue.empty())
                    break;
            }
            // admission in arrival order while rows fit
            while (!S.queue.empty()) {
                SrvReq *r = S.queue.front();
                const long base = S.rows.alloc(r->inst_rows);
                if (base < 0)
                    break;
                r->base = base;
                r->state = 1;
                S.queue.pop_front();
                admitted.push_back(r);
                S.running.push_back(r);
            }
        }
        // inputs of newly admitted requests -> pool (stream ordered)
        for (SrvReq *r : admitted) {
            const size_t row = kLweStride * sizeof(int32_t);
            cudaError_t e = cudaMemcpyAsync(S.pool + r->base * kLweStride, r->r.in0, r->rows0 * row,
                                            cudaMemcpyDeviceToDevice, S.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(S.pool + (r->base + r->rows0) * kLweStride, r->r.in1,
                                    r->rows1 * row, cudaMemcpyDeviceToDevice, S.st);
            if (e != cudaSuccess) {
                srv_fail_all(S, TFHE_ECUDA);
                return;
            }
        }
        // build the iteration: next level of running requests, oldest first
        Iter &I = S.it[S.seq & 1];
        int rc = srv_wait(S, I);
        if (rc != TFHE_OK) {
            srv_fail_all(S, rc);
            return;
        }
        std::vector<SrvReq *> take, rest, finishing;
        long count = 0, nout = 0;
        {
            std::lock_guard<std::mutex> lock(S.mu);
            for (SrvReq *r : S.running) {
                const long w = r->level_start[r->next_level] - r->level_start[r->next_level - 1];
                if (!take.empty() && count + w > S.max_batch) {
                    rest.push_back(r);
                    continue;
                }
                take.push_back(r);
                count += w;
            }
        }
        if (take.empty()) {
            // nothing runnable: drain the other in-flight iteration, then retry
            Iter &O = S.it[(S.seq + 1) & 1];
            rc = srv_wait(S, O);
            if (rc != TFHE_OK) {
                srv_fail_all(S, rc);
                return;
            }
            continue;
        }
        for (SrvReq *r : take)
            if (r->next_level == r->nl->depth)
                nout += (long)r->nl->out.size();
        bool ok = iter_reserve(I, count, std::max(nout, 1L));
        if (ok && count > S.big_rows) {   // one request's level wider than the scratch
            cudaStreamSynchronize(S.st);
            cudaFree(S.big);
            S.big = nullptr;
            ok = cudaMalloc(&S.big, count * kBigStride * sizeof(int32_t)) == cudaSuccess;
            S.big_rows = ok ? count : 0;
        }
        if (!ok) {
            srv_fail_all(S, TFHE_ENOMEM);
            return;
        }
        const long icap = I.cap;
        long k = 0;
        for (SrvReq *r : take) {
            const Netlist &nl = *r->nl;
            const int l = r->next_level;
            for (long q = r->level_start[l - 1]; q < r->level_start[l]; ++q, ++k) {
                const int g = r->order[q];
                I.h_ops[k] = nl.op[g];
                I.h_idx[k] = (int32_t)(r->base + nl.a[g]);
                I.h_idx[icap + k] = (int32_t)(r->base + nl.b[g]);
                I.h_idx[2 * icap + k] = nl.c[g] >= 0 ? (int32_t)(r->base + nl.c[g]) : 0;
                I.h_idx[3 * icap + k] = (int32_t)(r->base + nl.n_in + g);
            }
            if (l == nl.depth)
                finishing.push_back(r);
        }
        long o = 0;
        for (SrvReq *r : finishing)
            for (int32_t w : r->nl->out)
                I.h_out[o++] = (int32_t)(r->base + w);
        cudaError_t e = cudaMemcpyAsync(I.d_ops, I.h_ops, count, cudaMemcpyHostToDevice, S.st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(I.d_idx, I.h_idx, 4 * icap * sizeof(int32_t),
                                cudaMemcpyHostToDevice, S.st);
        if (e == cudaSuccess && nout)
            e = cudaMemcpyAsync(I.d_out, I.h_out, nout * sizeof(int32_t), cudaMemcpyHostToDevice,
                                S.st);
        if (e == cudaSuccess)
            e = launch_blind_rotate(ctx->keys, I.d_ops, S.pool, I.d_idx, S.pool_rows, S.pool,
                                    I.d_idx + icap, S.pool_rows, S.big, count, kMu, ctx->status,
                                    ctx->br_grid, S.st, S.pool, I.d_idx + 2 * icap,
                                    S.pool_rows);
        if (e == cudaSuccess)
            e = launch_keyswitch(ctx->keys.ksk, S.big, S.pool, I.d_idx + 3 * icap, S.pool_rows,
                                 count, ctx->prm.n, ctx->num_sms, ctx->status, S.st,
                                 &ctx->keys);
        o = 0;
        for (SrvReq *r : finishing) {
            const long no = (long)r->nl->out.size();
            if (e == cudaSuccess)
                e = launch_gather_rows(r->r.out, S.pool, I.d_out + o, no, S.st);
            o += no;
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(I.ev, S.st);
        if (e != cudaSuccess) {
            srv_fail_all(S, TFHE_ECUDA);
            return;
        }
        I.busy = true;
        I.finishing = finishing;
        I.gates = count;
        {
            std::lock_guard<std::mutex> lock(S.mu);
            ctx->launches += 1 + keyswitch_kernels(count, ctx->num_sms, &ctx->keys) +
                             (long)finishing.size();
            S.stats.gates += count;
            S.stats.iterations++;
            for (SrvReq *r : take)
                r->next_level++;
            S.running.erase(std::remove_if(S.running.begin(), S.running.end(),
                                           [](SrvReq *r) { return r->next_level > r->nl->depth; }),
                            S.running.end());
        }
        S.seq++;
    }
    for (Iter &I : S.it)
        if (srv_wait(S, I) != TFHE_OK)
            srv_fail_all(S, TFHE_ETIMEOUT);
}

void release_serving(tfhe_ctx *ctx)
{
    if (!ctx->server)
        return;
    Server *S = ctx->server;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable())
        S->worker.join();
    for (Iter &I : S->it) {
        cudaFree(I.d_ops);
        cudaFreeHost(I.h_ops);
        cudaFree(I.d_idx);
        cudaFreeHost(I.h_idx);
        cudaFree(I.d_out);
        cudaFreeHost(I.h_out);
        if (I.ev)
            cudaEventDestroy(I.ev);
    }
    cudaFree(S->pool);
    cudaFree(S->big);
    if (S->st)
        cudaStreamDestroy(S->st);
    for (auto &kv : S->all)
        delete kv.second;
    delete S;
    ctx->server = nullptr;
}

}  // namespace tgb

using namespace tgb;

extern "C" {

int tfhe_serve_start(tfhe_ctx *ctx, size_t hbm_budget_bytes, size_t max_batch_gates)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (ctx->server)
        return fail(ctx, TFHE_EBUSY, "serving already started");
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "keys not set");
    const long rows = (long)(hbm_budget_bytes / (kLweStride * sizeof(int32_t)));
    if (rows < 64)
        return fail(ctx, TFHE_EINVAL, "HBM budget too small (%zu bytes)", hbm_budget_bytes);
    DeviceGuard dg(ctx->device);
    Server *S = new Server();
    S->ctx = ctx;
    S->pool_rows = std::min(rows, (long)(1L << 30));
    S->max_batch = max_batch_gates ? (long)max_batch_gates : 8L * ctx->br_grid;
    S->big_rows = S->max_batch;
    cudaError_t e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&S->pool, S->pool_rows * kLweStride * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&S->big, S->big_rows * kBigStride * sizeof(int32_t));
    for (Iter &I : S->it)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&I.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ctx->server = S;
        release_serving(ctx);
        return cuda_fail(ctx, e, "tfhe_serve_start");
    }
    S->rows.init(S->pool_rows);
    ctx->server = S;
    S->worker = std::thread(srv_loop, S);
    return TFHE_OK;
}

int tfhe_serve_submit(tfhe_ctx *ctx, const tfhe_request *req, uint64_t *id)
{
    if (!ctx || !req || !id)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    if (!S)
        return fail(ctx, TFHE_EINVAL, "serving not started");
    auto nl = get_netlist(req->kind, req->width, req->rows, req->cols);
    if (!nl || !req->in0 || !req->in1 || !req->out)
        return fail(ctx, TFHE_EINVAL, "tfhe_serve_submit: unsupported request or null pointer");
    SrvReq *r = new SrvReq();
    r->r = *req;
    r->nl = nl;
    input_groups(req->kind, req->width, req->rows, req->cols, r->rows0, r->rows1);
    r->inst_rows = nl->wires();
    // gates sorted by level
    r->level_start.assign(nl->depth + 1, 0);
    for (int l : nl->level)
        r->level_start[l]++;
    for (int l = 1; l <= nl->depth; ++l)
        r->level_start[l] += r->level_start[l - 1];
    std::vector<long> fill(r->level_start.begin(), r->level_start.end());
    r->order.resize(nl->op.size());
    for (size_t g = 0; g < nl->op.size(); ++g)
        r->order[fill[nl->level[g] - 1]++] = (int32_t)g;
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->fatal != TFHE_OK) {
        delete r;
        return fail(ctx, S->fatal, "serving stopped after an error");
    }
    if (r->inst_rows > S->pool_rows) {
        delete r;
        return fail(ctx, TFHE_ENOMEM, "request needs %ld rows, pool has %ld", (long)nl->wires(),
                    S->pool_rows);
    }
    r->id = S->next_id++;
    r->t_submit = now_ms();
    if (S->t_first_submit < 0)
        S->t_first_submit = r->t_submit;
    S->all[r->id] = r;
    S->queue.push_back(r);
    S->stats.submitted++;
    S->cv.notify_all();
    *id = r->id;
    return TFHE_OK;
}

int tfhe_serve_poll(tfhe_ctx *ctx, uint64_t id, int *state, double *latency_ms)
{
    if (!ctx || !state || !ctx->server)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end())
        return fail(ctx, TFHE_EINVAL, "unknown request %llu", (unsigned long long)id);
    const SrvReq *r = it->second;
    *state = r->state == 2 ? 1 : (r->state < 0 ? r->state : 0);
    if (latency_ms)
        *latency_ms = r->state == 2 ? r->t_done - r->t_submit : 0.0;
    return TFHE_OK;
}

int tfhe_serve_wait(tfhe_ctx *ctx, uint64_t id, int timeout_ms, double *latency_ms)
{
    if (!ctx || !ctx->server)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end())
        return fail(ctx, TFHE_EINVAL, "unknown request %llu", (unsigned long long)id);
    SrvReq *r = it->second;
    const bool done = S->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                     [&] { return r->state == 2 || r->state < 0; });
    if (!done)
        return TFHE_ETIMEOUT;
    if (r->state < 0)
        return r->state;
    if (latency_ms)
        *latency_ms = r->t_done - r->t_submit;
    return TFHE_OK;
}

int tfhe_serve_stats(tfhe_ctx *ctx, tfhe_serve_info *out)
{
    if (!ctx || !out || !ctx->server)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lock(S->mu);
    *out = S->stats;
    out->in_flight = (uint64_t)S->running.size();
    out->queued = (uint64_t)S->queue.size();
    out->wall_ms = S->t_first_submit < 0 ? 0.0 : S->t_last_done - S->t_first_submit;
    return TFHE_OK;
}

int tfhe_serve_latencies(tfhe_ctx *ctx, double *ms, size_t cap, size_t *count)
{
    if (!ctx || !count || !ctx->server)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lock(S->mu);
    *count = S->latencies.size();
    if (ms)
        std::memcpy(ms, S->latencies.data(), std::min(cap, S->latencies.size()) * sizeof(double));
    return TFHE_OK;
}

int tfhe_serve_stop(tfhe_ctx *ctx)
{
    if (!ctx)
        return TFHE_EINVAL;
    DeviceGuard dg(ctx->device);
    const int fatal = ctx->server ? ctx->server->fatal : TFHE_OK;
    release_serving(ctx);
    return fatal;
}

}  // extern "C"
