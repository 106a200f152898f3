// circuits.cu -- boolean circuits over encrypted integers, compiled into a
// level schedule of batched bootstraps.
//
// Circuits (bit 0 least significant, all results mod 2^w):
//  * add: ripple-carry adder, r_i = a_i ^ b_i ^ c_(i-1) (Eq. "addres"),
//    c_i = a_i b_i | (a_i ^ b_i) c_(i-1) (Eq. "addcarry"); no carry in, no
//    carry out (sections III-A and V-B-1);
//  * mul: naive multiplication (section III-B-1): partial product i = A AND
//    b_i shifted left by i, truncated to w bits and accumulated one after
//    another with ripple-carry adders;
//  * matvec: y_r = sum_c M[r][c] v[c] (section IV-D) with the products of a
//    row reduced by tree-based accumulation (section V-B-2): neighbours
//    (0,1), (2,3), ... are added per level, an odd last term moves up.
//
// GB300 design: every gate gets its ASAP level (1 + the deeper input);
// gates of one level from all instances and all jobs of a batch form one
// blind-rotation launch and one key-switch launch that gather their inputs
// from, and scatter their outputs to, a device-resident ciphertext pool.
// The compiled schedule is cached per job signature and its level
// sequence is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "netlist.h"
#include "runtime.h"

namespace tgb {

// ---------------------------------------------------------------------
// Netlists
// ---------------------------------------------------------------------

// Ripple-carry adder on wire vectors x, y (w bits); returns sum wires.
static std::vector<int> build_add(Netlist &nl, const std::vector<int> &x, const std::vector<int> &y)
{
    const int w = (int)x.size();
    std::vector<int> r(w);
    int c = -1;
    for (int i = 0; i < w; ++i) {
        if (i == 0) {
            r[0] = nl.gate(TFHE_XOR, x[0], y[0]);
            if (w > 1)
                c = nl.gate(TFHE_AND, x[0], y[0]);
            continue;
        }
        const int p = nl.gate(TFHE_XOR, x[i], y[i]);   // propagate a_i ^ b_i
        r[i] = nl.gate(TFHE_XOR, p, c);                // sum bit
        if (i == w - 1)
            break;                                     // carry out is dropped
        const int g = nl.gate(TFHE_AND, x[i], y[i]);   // generate a_i b_i
        const int t = nl.gate(TFHE_AND, p, c);
        c = nl.gate(TFHE_OR, g, t);
    }
    return r;
}

// Truncated shift-and-add multiplier: w x w -> w bits.
static std::vector<int> build_mul(Netlist &nl, const std::vector<int> &x, const std::vector<int> &y)
{
    const int w = (int)x.size();
    std::vector<int> acc(w);
    for (int j = 0; j < w; ++j)
        acc[j] = nl.gate(TFHE_AND, x[j], y[0]);
    for (int i = 1; i < w; ++i) {
        const int m = w - i;
        std::vector<int> pp(m), hi(acc.begin() + i, acc.end());
        for (int j = 0; j < m; ++j)
            pp[j] = nl.gate(TFHE_AND, x[j], y[i]);     // a_j b_i has weight i + j
        std::vector<int> s = build_add(nl, hi, pp);
        std::copy(s.begin(), s.end(), acc.begin() + i);
    }
    return acc;
}

static std::vector<int> range_wires(int start, int count)
{
    std::vector<int> v(count);
    for (int k = 0; k < count; ++k)
        v[k] = start + k;
    return v;
}

// Input wires: ADD/MUL: A bits [0, w), B bits [w, 2w).  GATE: a = 0, b = 1.
// MATVEC: M[r][c] bits at (r*cols + c)*w + bit, then v[c] bits.
bool build_netlist(int kind, int w, int rows, int cols, Netlist &nl)
{
    switch (kind) {
    case TFHE_CIRCUIT_GATE:
        if (w < 0 || w > TFHE_XNOR)
            return false;
        nl.n_in = 2;
        nl.out = {nl.gate(w, 0, 1)};
        break;
    case TFHE_CIRCUIT_ADD:
    case TFHE_CIRCUIT_MUL:
        if (w < 1 || w > 64)
            return false;
        nl.n_in = 2 * w;
        nl.out = kind == TFHE_CIRCUIT_ADD ? build_add(nl, range_wires(0, w), range_wires(w, w))
                                          : build_mul(nl, range_wires(0, w), range_wires(w, w));
        break;
    case TFHE_CIRCUIT_MATVEC: {
        if (w < 1 || w > 64 || rows < 1 || cols < 1 || (long)rows * cols > 4096)
            return false;
        nl.n_in = (rows * cols + cols) * w;
        const int vbase = rows * cols * w;
        for (int r = 0; r < rows; ++r) {
            std::vector<std::vector<int>> terms;
            for (int c = 0; c < cols; ++c)
                terms.push_back(build_mul(nl, range_wires((r * cols + c) * w, w),
                                          range_wires(vbase + c * w, w)));
            while (terms.size() > 1) {
                std::vector<std::vector<int>> next;
                for (size_t i = 0; i + 1 < terms.size(); i += 2)
                    next.push_back(build_add(nl, terms[i], terms[i + 1]));
                if (terms.size() & 1)
                    next.push_back(terms.back());
                terms.swap(next);
            }
            nl.out.insert(nl.out.end(), terms[0].begin(), terms[0].end());
        }
        break;
    }
    default:
        return false;
    }
    nl.levelise();
    return true;
}

// Rows per instance of the two input groups.
void input_groups(int kind, int w, int rows, int cols, long &rows0, long &rows1)
{
    if (kind == TFHE_CIRCUIT_MATVEC) {
        rows0 = (long)rows * cols * w;
        rows1 = (long)cols * w;
    } else {
        rows0 = rows1 = kind == TFHE_CIRCUIT_GATE ? 1 : w;
    }
}

// ---------------------------------------------------------------------
// Compiled plans
// ---------------------------------------------------------------------

__global__ void k_gather_rows_impl(int32_t *dst, const int32_t *__restrict__ src,
                              const int32_t *__restrict__ rows, long count)
{
    const long r = blockIdx.x;
    if (r >= count)
        return;
    const int4 *s = reinterpret_cast<const int4 *>(src + (long)rows[r] * kLweStride);
    int4 *d = reinterpret_cast<int4 *>(dst + r * kLweStride);
    for (int k = threadIdx.x; k < kLweStride / 4; k += blockDim.x)
        d[k] = s[k];
}

cudaError_t launch_gather_rows(int32_t *dst, const int32_t *src, const int32_t *rows, long count,
                               cudaStream_t st)
{
    if (count <= 0)
        return cudaSuccess;
    k_gather_rows_impl<<<(unsigned)count, 128, 0, st>>>(dst, src, rows, count);
    return cudaGetLastError();
}

std::shared_ptr<const Netlist> get_netlist(int kind, int w, int rows, int cols)
{
    static std::mutex mu;
    static std::map<std::string, std::shared_ptr<const Netlist>> cache;
    char key[64];
    std::snprintf(key, sizeof(key), "%d:%d:%d:%d", kind, w, rows, cols);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end())
        return it->second;
    auto nl = std::make_shared<Netlist>();
    if (!build_netlist(kind, w, rows, cols, *nl))
        return nullptr;
    cache.emplace(key, nl);
    return nl;
}

struct JobLayout {
    int kind, w, rows, cols;
    long batch;
    long base;           // first pool row of instance 0
    long inst_rows;      // pool rows per instance
    long rows0, rows1;   // input rows per instance (group 0, group 1)
    long n_out;          // outputs per instance
    long out_off;        // offset of this job's output rows in d_out_rows
};

struct Plan {
    std::vector<JobLayout> jobs;
    long pool_rows = 0, gates = 0, max_width = 0;
    int depth = 0;
    std::vector<long> level_off;     // depth + 1 entries
    int32_t *pool = nullptr;
    int32_t *big = nullptr;
    uint8_t *d_ops = nullptr;
    int32_t *d_ia = nullptr, *d_ib = nullptr, *d_io = nullptr, *d_out_rows = nullptr;
    std::vector<uint8_t> h_ops;      // host copies for the per-gate schedule
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    bool graph_profiled = false;     // graph carries event-record nodes
    long kernels_per_run = 0;        // kernel launches of one level sequence
    std::vector<cudaEvent_t> ev;     // 3 per level: BR start, BR end / KS start, KS end

    ~Plan()
    {
        if (graph)
            cudaGraphExecDestroy(graph);
        for (cudaEvent_t e : ev)
            cudaEventDestroy(e);
        cudaFree(pool);
        cudaFree(big);
        cudaFree(d_ops);
        cudaFree(d_ia);
        cudaFree(d_ib);
        cudaFree(d_io);
        cudaFree(d_out_rows);
    }
};

struct CircuitCache {
    std::map<std::string, std::unique_ptr<Plan>> plans;
    std::vector<std::string> order;  // insertion order for eviction
    bool use_graphs = true;
    bool per_gate = false;
    bool profile = false;
    std::vector<Plan *> profiled;    // plans whose events hold the last run
    cudaStream_t capture_stream = nullptr;
    ~CircuitCache()
    {
        plans.clear();
        if (capture_stream)
            cudaStreamDestroy(capture_stream);
    }
};

static CircuitCache &cache_of(tfhe_ctx *ctx)
{
    if (!ctx->circuits)
        ctx->circuits = new CircuitCache();
    return *ctx->circuits;
}

void release_circuits(tfhe_ctx *ctx)
{
    delete ctx->circuits;
    ctx->circuits = nullptr;
}

static std::string signature(const tfhe_job *jobs, size_t njobs)
{
    std::string key;
    char buf[96];
    for (size_t j = 0; j < njobs; ++j) {
        std::snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%lld;", jobs[j].kind, jobs[j].width,
                      jobs[j].rows, jobs[j].cols, (long long)jobs[j].batch);
        key += buf;
    }
    return key;
}

static int compile_plan(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, Plan &P)
{
    std::vector<Netlist> nets(njobs);
    long pool = 0, nout = 0;
    int depth = 0;
    for (size_t j = 0; j < njobs; ++j) {
        const tfhe_job &J = jobs[j];
        if (J.batch < 0 || (J.batch > 0 && (!J.in0 || !J.in1 || !J.out)))
            return fail(ctx, TFHE_EINVAL, "job %zu: bad batch or null pointer", j);
        if (!build_netlist(J.kind, J.width, J.rows, J.cols, nets[j]))
            return fail(ctx, TFHE_EINVAL, "job %zu: unsupported circuit (kind %d width %d)", j,
                        J.kind, J.width);
        JobLayout L;
        L.kind = J.kind;
        L.w = J.width;
        L.rows = J.rows;
        L.cols = J.cols;
        L.batch = J.batch;
        L.base = pool;
        L.inst_rows = nets[j].wires();
        input_groups(J.kind, J.width, J.rows, J.cols, L.rows0, L.rows1);
        L.n_out = (long)nets[j].out.size();
        L.out_off = nout;
        pool += L.inst_rows * J.batch;
        nout += L.n_out * J.batch;
        if (J.batch > 0)
            depth = std::max(depth, nets[j].depth);
        P.jobs.push_back(L);
    }
    if (pool >= (1L << 31) / 2)
        return fail(ctx, TFHE_EINVAL, "batch too large for one schedule (%ld pool rows)", pool);
    // bucket gates by level
    std::vector<long> count(depth + 2, 0);
    for (size_t j = 0; j < njobs; ++j)
        for (int l : nets[j].level)
            count[l] += P.jobs[j].batch;
    P.level_off.assign(depth + 1, 0);
    for (int l = 1; l <= depth; ++l) {
        P.level_off[l] = P.level_off[l - 1] + count[l];
        P.max_width = std::max(P.max_width, count[l]);
    }
    // level l occupies [level_off[l-1], level_off[l])
    const long total = P.level_off[depth];
    std::vector<uint8_t> ops(total);
    std::vector<int32_t> ia(total), ib(total), io(total), outs(nout);
    std::vector<long> fill(P.level_off.begin(), P.level_off.end());
    for (size_t j = 0; j < njobs; ++j) {
        const Netlist &nl = nets[j];
        const JobLayout &L = P.jobs[j];
        for (long inst = 0; inst < L.batch; ++inst) {
            const long b = L.base + inst * L.inst_rows;
            for (size_t g = 0; g < nl.op.size(); ++g) {
                const long k = fill[nl.level[g] - 1]++;
                ops[k] = nl.op[g];
                ia[k] = (int32_t)(b + nl.a[g]);
                ib[k] = (int32_t)(b + nl.b[g]);
                io[k] = (int32_t)(b + nl.n_in + (long)g);
            }
            for (size_t o = 0; o < nl.out.size(); ++o)
                outs[L.out_off + inst * L.n_out + o] = (int32_t)(b + nl.out[o]);
        }
    }
    P.pool_rows = pool;
    P.gates = total;
    P.depth = depth;
    P.h_ops = ops;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess && bytes)
            e = cudaMalloc(p, bytes);
    };
    alloc((void **)&P.pool, (size_t)std::max(pool, 1L) * kLweStride * sizeof(int32_t));
    alloc((void **)&P.big, (size_t)std::max(P.max_width, 1L) * kBigStride * sizeof(int32_t));
    alloc((void **)&P.d_ops, std::max(total, 1L));
    alloc((void **)&P.d_ia, std::max(total, 1L) * sizeof(int32_t));
    alloc((void **)&P.d_ib, std::max(total, 1L) * sizeof(int32_t));
    alloc((void **)&P.d_io, std::max(total, 1L) * sizeof(int32_t));
    alloc((void **)&P.d_out_rows, std::max(nout, 1L) * sizeof(int32_t));
    if (e == cudaSuccess && total) {
        e = cudaMemcpy(P.d_ops, ops.data(), total, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_ia, ia.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_ib, ib.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_io, io.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && nout)
        e = cudaMemcpy(P.d_out_rows, outs.data(), nout * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "compile schedule");
    return TFHE_OK;
}

// Level sequence: one blind-rotation and one key-switch launch per level.
// With profile set, events are recorded around both launches (as external
// event-record nodes when the stream is being captured).
static cudaError_t enqueue_levels(tfhe_ctx *ctx, Plan &P, cudaStream_t st, bool profile,
                                  bool capturing)
{
    if (profile && P.ev.empty()) {
        P.ev.resize(3 * (size_t)P.depth, nullptr);
        for (cudaEvent_t &e : P.ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess)
                return r;
        }
    }
    auto mark = [&](int idx) -> cudaError_t {
        if (!profile)
            return cudaSuccess;
        return capturing ? cudaEventRecordWithFlags(P.ev[idx], st, cudaEventRecordExternal)
                         : cudaEventRecord(P.ev[idx], st);
    };
    long kernels = 0;
    for (int l = 1; l <= P.depth; ++l) {
        const long off = P.level_off[l - 1], cnt = P.level_off[l] - off;
        if (cnt == 0)
            continue;
        cudaError_t e = mark(3 * (l - 1));
        if (e == cudaSuccess)
            e = launch_blind_rotate(ctx->keys, P.d_ops + off, P.pool, P.d_ia + off, P.pool_rows,
                                    P.pool, P.d_ib + off, P.pool_rows, P.big, cnt, kMu,
                                    ctx->status, ctx->br_grid, st);
        if (e == cudaSuccess)
            e = mark(3 * (l - 1) + 1);
        if (e == cudaSuccess)
            e = launch_keyswitch(ctx->keys.ksk, P.big, P.pool, P.d_io + off, P.pool_rows, cnt,
                                 ctx->prm.n, ctx->num_sms, ctx->status, st);
        if (e == cudaSuccess)
            e = mark(3 * (l - 1) + 2);
        if (e != cudaSuccess)
            return e;
        kernels += 1 + keyswitch_kernels(cnt, ctx->num_sms);
    }
    P.kernels_per_run = kernels;
    return cudaSuccess;
}

// Baseline schedule: every gate on its own, one launch pair per gate.
static cudaError_t enqueue_per_gate(tfhe_ctx *ctx, Plan &P, cudaStream_t st)
{
    for (long k = 0; k < P.gates; ++k) {
        cudaError_t e = launch_blind_rotate(ctx->keys, P.d_ops + k, P.pool, P.d_ia + k, P.pool_rows,
                                            P.pool, P.d_ib + k, P.pool_rows, P.big, 1, kMu,
                                            ctx->status, ctx->br_grid, st);
        if (e != cudaSuccess)
            return e;
        e = launch_keyswitch(ctx->keys.ksk, P.big, P.pool, P.d_io + k, P.pool_rows, 1, ctx->prm.n,
                             ctx->num_sms, ctx->status, st);
        if (e != cudaSuccess)
            return e;
        ctx->launches += 1 + keyswitch_kernels(1, ctx->num_sms);
    }
    return cudaSuccess;
}

static int run_plan(tfhe_ctx *ctx, Plan &P, const tfhe_job *jobs, cudaStream_t st)
{
    CircuitCache &C = cache_of(ctx);
    cudaError_t e = cudaSuccess;
    // inputs -> pool (strided 2D copies, one per input group)
    for (size_t j = 0; j < P.jobs.size() && e == cudaSuccess; ++j) {
        const JobLayout &L = P.jobs[j];
        if (L.batch == 0)
            continue;
        const size_t row = kLweStride * sizeof(int32_t);
        e = cudaMemcpy2DAsync(P.pool + L.base * kLweStride, L.inst_rows * row, jobs[j].in0,
                              L.rows0 * row, L.rows0 * row, L.batch, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(P.pool + (L.base + L.rows0) * kLweStride, L.inst_rows * row,
                                  jobs[j].in1, L.rows1 * row, L.rows1 * row, L.batch,
                                  cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "copy inputs");
    if (C.per_gate) {
        e = enqueue_per_gate(ctx, P, st);
    } else if (C.use_graphs && !P.graph_failed) {
        if (P.graph && P.graph_profiled != C.profile) {   // recapture with/without events
            cudaGraphExecDestroy(P.graph);
            P.graph = nullptr;
        }
        if (!P.graph) {
            if (!C.capture_stream)
                e = cudaStreamCreateWithFlags(&C.capture_stream, cudaStreamNonBlocking);
            cudaGraph_t g = nullptr;
            if (e == cudaSuccess)
                e = cudaStreamBeginCapture(C.capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = enqueue_levels(ctx, P, C.capture_stream, C.profile, true);
                cudaError_t e2 = cudaStreamEndCapture(C.capture_stream, &g);
                e = e1 != cudaSuccess ? e1 : e2;
            }
            if (e == cudaSuccess)
                e = cudaGraphInstantiate(&P.graph, g, 0);
            if (g)
                cudaGraphDestroy(g);
            if (e != cudaSuccess) {  // fall back to direct launches for this plan
                (void)cudaGetLastError();
                P.graph = nullptr;
                P.graph_failed = true;
                e = cudaSuccess;
            }
            P.graph_profiled = C.profile;
        }
        if (P.graph) {
            e = cudaGraphLaunch(P.graph, st);
            ctx->launches += P.kernels_per_run;
        } else {
            e = enqueue_levels(ctx, P, st, C.profile, false);
            ctx->launches += P.kernels_per_run;
        }
    } else {
        e = enqueue_levels(ctx, P, st, C.profile, false);
        ctx->launches += P.kernels_per_run;
    }
    if (e == cudaSuccess && C.profile && !C.per_gate &&
        std::find(C.profiled.begin(), C.profiled.end(), &P) == C.profiled.end())
        C.profiled.push_back(&P);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "level launches");
    // pool -> outputs
    for (size_t j = 0; j < P.jobs.size() && e == cudaSuccess; ++j) {
        const JobLayout &L = P.jobs[j];
        const long cnt = L.n_out * L.batch;
        if (cnt == 0)
            continue;
        e = launch_gather_rows(jobs[j].out, P.pool, P.d_out_rows + L.out_off, cnt, st);
        ctx->launches += 1;
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "copy outputs");
    return TFHE_OK;
}

int run_jobs(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, cudaStream_t st)
{
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "keys not set");
    if (njobs == 0)
        return TFHE_OK;
    CircuitCache &C = cache_of(ctx);
    const std::string key = signature(jobs, njobs);
    auto it = C.plans.find(key);
    if (it == C.plans.end()) {
        std::unique_ptr<Plan> P(new Plan());
        int rc = compile_plan(ctx, jobs, njobs, *P);
        if (rc != TFHE_OK)
            return rc;
        if (C.order.size() >= 32) {   // keep device memory bounded
            Plan *victim = C.plans[C.order.front()].get();
            C.profiled.erase(std::remove(C.profiled.begin(), C.profiled.end(), victim),
                             C.profiled.end());
            C.plans.erase(C.order.front());
            C.order.erase(C.order.begin());
        }
        C.order.push_back(key);
        it = C.plans.emplace(key, std::move(P)).first;
    }
    return run_plan(ctx, *it->second, jobs, st);
}

}  // namespace tgb

using namespace tgb;

extern "C" {

int tfhe_run_jobs(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, void *stream)
{
    if (!ctx || (njobs && !jobs))
        return ctx ? fail(ctx, TFHE_EINVAL, "tfhe_run_jobs: null argument") : TFHE_EINVAL;
    DeviceGuard dg(ctx->device);
    return run_jobs(ctx, jobs, njobs, (cudaStream_t)stream);
}

static int one_job(tfhe_ctx *ctx, int kind, int width, int rows, int cols, const int32_t *a,
                   const int32_t *b, int32_t *out, size_t batch, void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (batch == 0)
        return TFHE_OK;
    tfhe_job J;
    J.kind = kind;
    J.width = width;
    J.rows = rows;
    J.cols = cols;
    J.batch = (int64_t)batch;
    J.in0 = a;
    J.in1 = b;
    J.out = out;
    return tfhe_run_jobs(ctx, &J, 1, stream);
}

int tfhe_add_n(tfhe_ctx *ctx, int width, const int32_t *A, const int32_t *B, int32_t *R,
               size_t batch, void *stream)
{
    return one_job(ctx, TFHE_CIRCUIT_ADD, width, 0, 0, A, B, R, batch, stream);
}

int tfhe_mul_n(tfhe_ctx *ctx, int width, const int32_t *A, const int32_t *B, int32_t *R,
               size_t batch, void *stream)
{
    return one_job(ctx, TFHE_CIRCUIT_MUL, width, 0, 0, A, B, R, batch, stream);
}

int tfhe_matvec(tfhe_ctx *ctx, int width, int rows, int cols, const int32_t *M, const int32_t *v,
                int32_t *y, void *stream)
{
    return one_job(ctx, TFHE_CIRCUIT_MATVEC, width, rows, cols, M, v, y, 1, stream);
}

int tfhe_circuit_info(int kind, int width, int rows, int cols, int64_t *gates, int32_t *depth)
{
    Netlist nl;
    if (!build_netlist(kind, width, rows, cols, nl))
        return TFHE_EINVAL;
    if (gates)
        *gates = (int64_t)nl.op.size();
    if (depth)
        *depth = nl.depth;
    return TFHE_OK;
}

int tfhe_ctx_set_option(tfhe_ctx *ctx, int option, int64_t value)
{
    if (!ctx)
        return TFHE_EINVAL;
    CircuitCache &C = cache_of(ctx);
    switch (option) {
    case TFHE_OPT_GRAPHS:
        C.use_graphs = value != 0;
        return TFHE_OK;
    case TFHE_OPT_PER_GATE:
        C.per_gate = value != 0;
        return TFHE_OK;
    case TFHE_OPT_PROFILE:
        C.profile = value != 0;
        return TFHE_OK;
    case TFHE_OPT_BR_GROUP:
        if (value != 0 && value != 1 && value != 2 && value != 4)
            return fail(ctx, TFHE_EINVAL, "TFHE_OPT_BR_GROUP must be 0, 1, 2 or 4");
        ctx->keys.br_group = (int)value;
        for (auto &kv : C.plans)   // captured graphs hold the old launch shape
            if (kv.second->graph) {
                cudaGraphExecDestroy(kv.second->graph);
                kv.second->graph = nullptr;
            }
        return TFHE_OK;
    default:
        return fail(ctx, TFHE_EINVAL, "unknown option %d", option);
    }
}

int tfhe_ctx_profile(tfhe_ctx *ctx, double *br_ms, int64_t *br_launches, int64_t *br_bootstraps,
                     double *ks_ms, int64_t *ks_launches)
{
    if (!ctx)
        return TFHE_EINVAL;
    DeviceGuard dg(ctx->device);
    CircuitCache &C = cache_of(ctx);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tfhe_ctx_profile");
    double bt = 0, kt = 0;
    int64_t bl = 0, kl = 0, bb = 0;
    for (Plan *P : C.profiled) {
        for (int l = 1; l <= P->depth; ++l) {
            const long cnt = P->level_off[l] - P->level_off[l - 1];
            if (cnt == 0)
                continue;
            float a = 0, b = 0;
            if (cudaEventElapsedTime(&a, P->ev[3 * (l - 1)], P->ev[3 * (l - 1) + 1]) != cudaSuccess ||
                cudaEventElapsedTime(&b, P->ev[3 * (l - 1) + 1], P->ev[3 * (l - 1) + 2]) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(ctx, TFHE_ECUDA, "profile events not recorded");
            }
            bt += a;
            kt += b;
            bl += 1;
            bb += cnt;
            kl += keyswitch_kernels(cnt, ctx->num_sms);
        }
    }
    C.profiled.clear();
    if (br_ms) *br_ms = bt;
    if (br_launches) *br_launches = bl;
    if (br_bootstraps) *br_bootstraps = bb;
    if (ks_ms) *ks_ms = kt;
    if (ks_launches) *ks_launches = kl;
    return TFHE_OK;
}

}  // extern "C"
