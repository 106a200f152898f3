// serve.cu -- continuous-batching request loop over the bootstrapping kernels.
//
// Requests (one circuit instance each: a gate, an add, a mul, a matvec) are
// submitted from any host thread.  A worker thread owns one CUDA stream and
// a device ciphertext pool; it admits queued requests in arrival order
// whenever their rows fit in the pool (first fit), growing the pool from
// the device's free HBM (under the caller's cap) when they do not, copies
// their inputs in, and then runs iterations: one iteration is one batched
// blind-rotation launch plus one key-switch launch over the next level of
// admitted requests, chosen by serve_select (deepest first, up to a gate
// cap, trimmed to the width that runs most gates per unit of time).  A request's
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
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda.h>

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
    // Rows the pool gained at its end become free (merged with a free tail).
    void grow(long cap)
    {
        if (cap > capacity) {
            const long old = capacity;
            capacity = cap;
            release(old, cap - old);
        }
    }
    // Free rows at the end of the pool.
    long tail() const
    {
        if (free_.empty())
            return 0;
        auto last = std::prev(free_.end());
        return last->first + last->second == capacity ? last->second : 0;
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

// The ciphertext pool: one reserved range of device virtual addresses (the
// caller's cap, or the device's memory) into which physical HBM is mapped
// in steps as admission needs it, through the driver's virtual memory
// management (entry points looked up through the runtime, no link against
// the driver).  The base address never moves, so every row index the
// kernels are given stays valid while the pool grows.  Without those entry
// points the pool is one cudaMalloc of the cap (or of the free memory minus
// the headroom), fixed for the whole session.
struct VmmApi {
    CUresult (*reserve)(CUdeviceptr *, size_t, size_t, CUdeviceptr, unsigned long long);
    CUresult (*addr_free)(CUdeviceptr, size_t);
    CUresult (*create)(CUmemGenericAllocationHandle *, size_t, const CUmemAllocationProp *,
                       unsigned long long);
    CUresult (*release)(CUmemGenericAllocationHandle);
    CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long);
    CUresult (*unmap)(CUdeviceptr, size_t);
    CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc *, size_t);
    CUresult (*granularity)(size_t *, const CUmemAllocationProp *,
                            CUmemAllocationGranularity_flags);
};

static const VmmApi *vmm_api()
{
    static std::once_flag once;
    static VmmApi api{};
    static bool ok = false;
    std::call_once(once, [] {
        struct {
            const char *name;
            void **slot;
        } fns[] = {{"cuMemAddressReserve", (void **)&api.reserve},
                   {"cuMemAddressFree", (void **)&api.addr_free},
                   {"cuMemCreate", (void **)&api.create},
                   {"cuMemRelease", (void **)&api.release},
                   {"cuMemMap", (void **)&api.map},
                   {"cuMemUnmap", (void **)&api.unmap},
                   {"cuMemSetAccess", (void **)&api.set_access},
                   {"cuMemGetAllocationGranularity", (void **)&api.granularity}};
        ok = true;
        for (auto &f : fns) {
            cudaDriverEntryPointQueryResult q{};
            if (cudaGetDriverEntryPointByVersion(f.name, f.slot, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !*f.slot)
                ok = false;
        }
        (void)cudaGetLastError();
    });
    return ok ? &api : nullptr;
}

// Free HBM that growing the pool always leaves to other allocations (the
// iteration buffers, the caller, other processes on the device).
constexpr size_t kPoolHeadroom = 1ull << 30;
constexpr size_t kRowBytes = kLweStride * sizeof(int32_t);

struct GrowPool {
    const VmmApi *api = nullptr;   // null: fixed cudaMalloc pool
    int device = 0;
    CUdeviceptr base = 0;
    size_t limit = 0;              // the cap in bytes (the device's memory if none)
    size_t reserved = 0, mapped = 0, gran = 0;
    std::vector<std::pair<CUmemGenericAllocationHandle, size_t>> chunks;
    int32_t *ptr() const { return reinterpret_cast<int32_t *>(base); }
    long rows() const { return (long)(std::min(mapped, limit) / kRowBytes); }
    long max_rows() const { return (long)(limit / kRowBytes); }

    CUmemAllocationProp prop() const
    {
        CUmemAllocationProp p{};
        p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
        p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
        p.location.id = device;
        return p;
    }

    // Maps `bytes` (a multiple of the granularity) more at the end.
    bool map_more(size_t bytes)
    {
        if (!api || bytes == 0 || mapped + bytes > reserved)
            return false;
        const CUmemAllocationProp pr = prop();
        CUmemGenericAllocationHandle h{};
        if (api->create(&h, bytes, &pr, 0) != CUDA_SUCCESS)
            return false;
        if (api->map(base + mapped, bytes, 0, h, 0) != CUDA_SUCCESS) {
            api->release(h);
            return false;
        }
        CUmemAccessDesc acc{};
        acc.location = pr.location;
        acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
        if (api->set_access(base + mapped, bytes, &acc, 1) != CUDA_SUCCESS) {
            api->unmap(base + mapped, bytes);
            api->release(h);
            return false;
        }
        chunks.push_back({h, bytes});
        mapped += bytes;
        return true;
    }

    // Reserves cap bytes of addresses (0: the device's memory) and maps the
    // first step; falls back to a fixed cudaMalloc pool.
    cudaError_t init(int dev, size_t cap, size_t free_bytes)
    {
        device = dev;
        size_t fr = 0, total = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &total);
        if (e != cudaSuccess)
            return e;
        api = vmm_api();
        const CUmemAllocationProp pr = prop();
        if (api && api->granularity(&gran, &pr, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) !=
                       CUDA_SUCCESS)
            api = nullptr;
        limit = cap ? cap : total;
        if (api) {
            reserved = (limit + gran - 1) / gran * gran;
            if (api->reserve(&base, reserved, gran, 0, 0) != CUDA_SUCCESS) {
                api = nullptr;
                base = 0;
            }
        }
        if (api) {
            // first step: 8 MB (or one granule when the device is short)
            size_t first = std::min(reserved, std::max<size_t>(gran, (8ull << 20) / gran * gran));
            if (free_bytes < first + kPoolHeadroom)
                first = gran;
            return map_more(first) ? cudaSuccess : cudaErrorMemoryAllocation;
        }
        // fixed pool: the cap, or half the free memory (at most 32 GB)
        size_t bytes = cap ? cap : std::min<size_t>(free_bytes / 2, 32ull << 30);
        bytes = std::max(bytes / kRowBytes, (size_t)64) * kRowBytes;
        void *p = nullptr;
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess)
            return e;
        base = reinterpret_cast<CUdeviceptr>(p);
        limit = reserved = mapped = bytes;
        return cudaSuccess;
    }

    // Grows so that `extra_rows` more rows exist at the end, if the device's
    // free memory (free_bytes) keeps the headroom and the cap allows.  Steps
    // double the mapping (at most 8 GB at a time), or are just what the
    // request needs when free memory is short.
    bool grow(long extra_rows, size_t free_bytes)
    {
        if (!api || extra_rows <= 0)
            return false;
        const size_t need = ((size_t)extra_rows * kRowBytes + gran - 1) / gran * gran;
        if (mapped + need > reserved || rows() + extra_rows > max_rows())
            return false;
        const size_t dbl = std::min<size_t>(std::max<size_t>(mapped, 64ull << 20), 8ull << 30);
        size_t bytes = std::min(std::max(need, (dbl + gran - 1) / gran * gran), reserved - mapped);
        if (free_bytes < bytes + kPoolHeadroom)
            bytes = need;   // only what this request needs
        if (free_bytes < bytes + kPoolHeadroom)
            return false;   // the device is short: wait for rows to free up
        return map_more(bytes);
    }

    void release()
    {
        if (api) {
            // each mapping is undone as it was made, chunk by chunk
            size_t off = 0;
            for (auto &c : chunks) {
                api->unmap(base + off, c.second);
                api->release(c.first);
                off += c.second;
            }
            if (base)
                api->addr_free(base, reserved);
        } else if (base) {
            cudaFree(reinterpret_cast<void *>(base));
        }
        chunks.clear();
        base = 0;
        mapped = reserved = 0;
    }
};

struct SrvReq {
    uint64_t id = 0;
    tfhe_request r{};
    std::shared_ptr<const Netlist> nl;
    long rows0 = 0, rows1 = 0, inst_rows = 0, base = -1;
    int next_level = 1;
    int waited = 0;                // iterations run since this request's last level ran
    int state = 0;                 // 0 queued, 1 admitted, 2 done, < 0 error code
                                   // (TFHE_ECANCELED: cancelled)
    bool last_taken = false;       // its last level is in an iteration: too late to cancel
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
    GrowPool gp;
    int32_t *pool = nullptr;       // gp's base
    long pool_rows = 0;            // rows mapped now (grows; worker thread only)
    long max_rows = 0;             // rows the pool may ever hold
    size_t test_free_hbm = 0;      // test hook: taken as the device's free memory
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

// Estimated device time (ms) of one serving iteration of n gates: the
// autotuner's measured level time of n's width bucket while n fits one wave
// of 4 bootstraps per SM, whole waves above.  Untuned (wave_ms 0) in units
// of one wave, with the ratios measured on GB300: a level of at most one
// bootstrap per SM takes 0.35 of a full wave, of at most two per SM 0.55.
static double iter_cost(long n, int num_sms, const float *level_ms, float wave_ms)
{
    const long w4 = 4L * num_sms;
    const double t4 = wave_ms > 0.f ? wave_ms : 1.0;
    if (n > w4)
        return (double)((n + w4 - 1) / w4) * t4;
    if (level_ms && wave_ms > 0.f && level_ms[tune_bucket(n)] > 0.f)
        return level_ms[tune_bucket(n)];
    return n <= num_sms ? 0.35 * t4 : (n <= 2L * num_sms ? 0.55 * t4 : t4);
}

// The requests one iteration takes, as indices into the running list
// (taken[0 .. return value)).  Requests are ranked by the levels they have
// left plus the iterations they have waited since their last level ran
// (the deepest ones bound when the work ends; waiting raises a shallow
// request's rank so that it is not starved), ties in admission order.  In
// rank order each request's next level is taken while the gate cap allows
// (a level that does not fit is passed over; the first is always taken).
// Of that list the prefix with the most gates per estimated unit of device
// time is kept (the longest on ties): an iteration that would spill a few
// gates into another wave, or past the width of a narrow level, leaves its
// lowest-ranked requests for the next one.  Host-only and deterministic.
long serve_select(long n, const long *width, const int *remaining, const int *waited, long cap,
                  int num_sms, const float *level_ms, float wave_ms, int32_t *taken)
{
    std::vector<int32_t> rank((size_t)n);
    std::iota(rank.begin(), rank.end(), 0);
    std::stable_sort(rank.begin(), rank.end(), [&](int32_t x, int32_t y) {
        return (long)remaining[x] + waited[x] > (long)remaining[y] + waited[y];
    });
    long k = 0, count = 0;
    for (int32_t i : rank) {
        if (k > 0 && count + width[i] > cap)
            continue;
        taken[k++] = i;
        count += width[i];
    }
    long keep = 0, c = 0;
    double best = -1.0;
    for (long j = 0; j < k; ++j) {
        c += width[taken[j]];
        const double rate = (double)c / iter_cost(c, num_sms, level_ms, wave_ms);
        if (rate >= best)
            best = rate, keep = j + 1;
    }
    return keep;
}

static int srv_fail_all(Server &S, int code)
{
    std::lock_guard<std::mutex> lock(S.mu);
    S.fatal = code;
    for (SrvReq *r : S.running)
        if (r->state >= 0)         // not cancelled
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
            // admission in arrival order while rows fit; the pool grows from
            // the device's free memory when they do not
            while (!S.queue.empty()) {
                SrvReq *r = S.queue.front();
                long base = S.rows.alloc(r->inst_rows);
                if (base < 0) {
                    size_t fr = 0, total = 0;
                    if (S.test_free_hbm)
                        fr = S.test_free_hbm;
                    else if (cudaMemGetInfo(&fr, &total) != cudaSuccess)
                        (void)cudaGetLastError();
                    if (S.gp.grow(r->inst_rows - S.rows.tail(), fr)) {
                        S.pool_rows = S.gp.rows();
                        S.rows.grow(S.pool_rows);
                        S.stats.pool_grows++;
                        S.stats.pool_bytes = S.gp.mapped;
                        base = S.rows.alloc(r->inst_rows);
                    }
                }
                if (base < 0)
                    break;
                r->base = base;
                r->state = 1;
                if (!S.running.empty() || S.it[0].busy || S.it[1].busy)
                    S.stats.admitted_busy++;
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
        // build the iteration: next levels of running requests (serve_select)
        Iter &I = S.it[S.seq & 1];
        int rc = srv_wait(S, I);
        if (rc != TFHE_OK) {
            srv_fail_all(S, rc);
            return;
        }
        std::vector<SrvReq *> take, finishing;
        long count = 0, nout = 0;
        {
            std::lock_guard<std::mutex> lock(S.mu);
            // requests cancelled since they were admitted: their rows go back
            // to the pool now.  Every device use of those rows (input copies,
            // levels of in-flight iterations) is already on S.st, ahead of
            // whatever reuses them, so nothing has to wait.
            S.running.erase(std::remove_if(S.running.begin(), S.running.end(),
                                           [&S](SrvReq *r) {
                                               if (r->state >= 0)
                                                   return false;
                                               S.rows.release(r->base, r->inst_rows);
                                               return true;
                                           }),
                            S.running.end());
            const long nr = (long)S.running.size();
            std::vector<long> wv((size_t)nr);
            std::vector<int> rem((size_t)nr), wt((size_t)nr);
            std::vector<int32_t> tk((size_t)nr);
            for (long i = 0; i < nr; ++i) {
                const SrvReq *r = S.running[i];
                wv[i] = r->level_start[r->next_level] - r->level_start[r->next_level - 1];
                rem[i] = r->nl->depth - r->next_level + 1;
                wt[i] = r->waited;
            }
            const long nt = serve_select(nr, wv.data(), rem.data(), wt.data(), S.max_batch,
                                         ctx->num_sms, ctx->keys.tune_ms, ctx->keys.wave_ms[0],
                                         tk.data());
            for (long j = 0; j < nt; ++j) {
                SrvReq *r = S.running[tk[j]];
                if (r->next_level == r->nl->depth)
                    r->last_taken = true;   // its output will be gathered
                take.push_back(r);
                count += wv[tk[j]];
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
        NvtxRange range("tfhe: serving iteration (one level of each selected request)");
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
                e = launch_gather_rows(r->r.out, S.pool, S.pool_rows, I.d_out + o, no,
                                       ctx->status, S.st);
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
            for (SrvReq *r : S.running)
                r->waited++;
            for (SrvReq *r : take) {
                r->next_level++;
                r->waited = 0;
            }
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
    if (S->st)
        cudaStreamSynchronize(S->st);
    S->gp.release();
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
    if (hbm_budget_bytes && hbm_budget_bytes / kRowBytes < 64)
        return fail(ctx, TFHE_EINVAL, "HBM budget too small (%zu bytes)", hbm_budget_bytes);
    // 0: no cap but the device's memory; row indices are 32-bit
    const size_t cap = hbm_budget_bytes ? std::min<size_t>(hbm_budget_bytes,
                                                           (size_t)(1L << 30) * kRowBytes)
                                        : 0;
    DeviceGuard dg(ctx->device);
    Server *S = new Server();
    S->ctx = ctx;
    S->test_free_hbm = ctx->test_free_hbm;
    S->max_batch = max_batch_gates ? (long)max_batch_gates : 8L * ctx->br_grid;
    S->big_rows = S->max_batch;
    size_t fr = 0, total = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &total);
    if (S->test_free_hbm)
        fr = S->test_free_hbm;
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = S->gp.init(ctx->device, cap, fr);
    if (e == cudaSuccess) {
        S->pool = S->gp.ptr();
        S->pool_rows = S->gp.rows();
        S->max_rows = S->gp.max_rows();
        S->stats.pool_bytes = S->gp.mapped;
        S->stats.pool_cap_bytes = S->gp.reserved;
    }
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
    if (r->inst_rows > S->max_rows) {
        delete r;
        return fail(ctx, TFHE_ENOMEM, "request needs %ld rows, the pool can hold %ld",
                    (long)nl->wires(), S->max_rows);
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

int tfhe_serve_cancel(tfhe_ctx *ctx, uint64_t id)
{
    if (!ctx || !ctx->server)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end())
        return fail(ctx, TFHE_EINVAL, "unknown request %llu", (unsigned long long)id);
    SrvReq *r = it->second;
    if (r->state == 2 || r->state < 0)
        return fail(ctx, TFHE_EINVAL, "request %llu has already finished",
                    (unsigned long long)id);
    if (r->last_taken)
        return fail(ctx, TFHE_EBUSY, "request %llu: its last level is already on the device",
                    (unsigned long long)id);
    if (r->state == 0) {
        auto q = std::find(S->queue.begin(), S->queue.end(), r);
        if (q != S->queue.end())
            S->queue.erase(q);
    }
    // an admitted request stays in the worker's running list until its next
    // iteration drops it and frees its rows
    r->state = TFHE_ECANCELED;
    r->t_done = now_ms();
    S->stats.cancelled++;
    S->cv.notify_all();
    return TFHE_OK;
}

int tfhe_serve_stats(tfhe_ctx *ctx, tfhe_serve_info *out)
{
    if (!ctx || !out || !ctx->server)
        return TFHE_EINVAL;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lock(S->mu);
    *out = S->stats;
    out->in_flight = (uint64_t)std::count_if(S->running.begin(), S->running.end(),
                                             [](const SrvReq *r) { return r->state >= 0; });
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

int tfhe_serve_select(const int64_t *width, const int32_t *remaining, const int32_t *waited,
                      size_t n, int64_t cap, int32_t num_sms, const float *level_ms,
                      float wave_ms, int32_t *taken, size_t *ntaken)
{
    if (!ntaken || num_sms <= 0 || cap <= 0 || (n && (!width || !remaining || !waited || !taken)))
        return TFHE_EINVAL;
    std::vector<long> w(n);
    std::vector<int> rem(n), wt(n);
    for (size_t i = 0; i < n; ++i) {
        if (width[i] <= 0 || remaining[i] <= 0 || waited[i] < 0)
            return TFHE_EINVAL;
        w[i] = (long)width[i];
        rem[i] = remaining[i];
        wt[i] = waited[i];
    }
    *ntaken = n ? (size_t)serve_select((long)n, w.data(), rem.data(), wt.data(), (long)cap,
                                       num_sms, level_ms, wave_ms, taken)
                : 0;
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
