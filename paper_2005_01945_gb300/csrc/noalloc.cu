// noalloc.cu -- batched gate bootstrapping that allocates no device memory.
//
// tfhe_bootstrap_gates hands the extracted LWE_N samples from the
// blind-rotation kernel to the key-switch kernel through scratch rows that
// the context allocates with cudaMalloc (and grows) when a batch first needs
// them.  Some callers cannot let a library allocate on their call path:
// runtimes that pre-reserve all device memory and forbid any later
// allocation, real-time or serving loops that must not hit the allocator
// (cudaMalloc can synchronise the device and stall), and hosts that account
// for every byte a plugin may use.  tfhe_bootstrap_gates_noalloc gives them
// the same result with fixed scratch: an array placed in the library's own
// device image, which the CUDA runtime sets aside on every GPU that loads
// the library and keeps until the process exits.  The caller still passes
// (and owns) the inputs and outputs.
#include <mutex>

#include "runtime.h"

namespace tgb {

constexpr long kNoAllocMaxGates = TFHE_NOALLOC_MAX_GATES;

// The fixed scratch: kNoAllocMaxGates rows of kBigStride words
// (512 x 1056 x 4 B = 2,162,688 bytes per GPU).  Shared by every call on a
// device; no word of it needs to start at zero, because each call's
// blind-rotation kernel writes every word (rows < count, words 0..N) that
// the same call's key-switch kernel then reads.
static __device__ __align__(256) int32_t g_noalloc_big[kNoAllocMaxGates * kBigStride];

// In host code the name g_noalloc_big is only a host-side stand-in, not a
// device address.  The device address is looked up with the device current
// and cached per CUDA context: a device reset (or another context made
// current) loads the library's device image anew, where the array may sit
// elsewhere, so a cached address is used only for the context that gave it.
// The context handle comes from the driver's cuCtxGetCurrent, reached
// through the runtime's entry-point query (no link against the driver).
constexpr int kNoAllocMaxSlots = 64;
struct NoAllocSlot {
    void *cu_ctx;
    int32_t *ptr;
};
static NoAllocSlot g_noalloc_slots[kNoAllocMaxSlots];
static int g_noalloc_nslots = 0;
static std::mutex g_noalloc_mutex;

typedef int (*cu_ctx_get_current_fn)(void **);

static int current_cu_context(tfhe_ctx *ctx, void **cu_ctx)
{
    static cu_ctx_get_current_fn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f)
            return fail(ctx, TFHE_ECUDA, "tfhe_bootstrap_gates_noalloc: cuCtxGetCurrent "
                        "unavailable (%s)", cudaGetErrorString(e));
        fn = (cu_ctx_get_current_fn)f;
    }
    *cu_ctx = nullptr;
    if (fn(cu_ctx) != 0 || !*cu_ctx)
        return fail(ctx, TFHE_ECUDA, "tfhe_bootstrap_gates_noalloc: no current CUDA context");
    return TFHE_OK;
}

// Set-up, once per device (per CUDA context on it), with that device
// current: the caller holds a DeviceGuard for ctx->device.
static int noalloc_scratch(tfhe_ctx *ctx, int32_t **ptr)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    // cudaSetDevice (the caller's DeviceGuard) has made the device's primary
    // context current.
    void *cu_ctx = nullptr;
    int rc = current_cu_context(ctx, &cu_ctx);
    if (rc != TFHE_OK)
        return rc;
    for (int i = 0; i < g_noalloc_nslots; i++)
        if (g_noalloc_slots[i].cu_ctx == cu_ctx) {
            *ptr = g_noalloc_slots[i].ptr;
            return TFHE_OK;
        }
    int32_t *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_big);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
    // When the table is full, new entries overwrite the oldest from slot 0
    // (an entry of a context that no longer exists is only a lookup that
    // misses).
    if (g_noalloc_nslots == kNoAllocMaxSlots)
        g_noalloc_nslots = 0;
    g_noalloc_slots[g_noalloc_nslots++] = {cu_ctx, p};
    *ptr = p;
    return TFHE_OK;
}

}  // namespace tgb

using namespace tgb;

extern "C" int tfhe_bootstrap_gates_noalloc(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a,
                                            const int32_t *b, int32_t *out, size_t count,
                                            void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (count == 0)
        return TFHE_OK;
    if (count > (size_t)kNoAllocMaxGates)
        return fail(ctx, TFHE_EINVAL,
                    "tfhe_bootstrap_gates_noalloc: %zu gates exceed the fixed scratch of %ld "
                    "gates (TFHE_NOALLOC_MAX_GATES); split the batch",
                    count, kNoAllocMaxGates);
    if (!ops || !a || !b || !out)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap_gates_noalloc: null argument");
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap_gates_noalloc: keys not set");
    DeviceGuard dg(ctx->device);
    int32_t *big = nullptr;
    int rc = noalloc_scratch(ctx, &big);
    if (rc != TFHE_OK)
        return rc;
    const long n = (long)count;
    cudaStream_t st = (cudaStream_t)stream;
    NvtxRange range("tfhe: gate bootstrapping (fixed scratch)");
    cudaError_t e = launch_blind_rotate(ctx->keys, ops, a, nullptr, n, b, nullptr, n, big, n, kMu,
                                        ctx->status, ctx->br_grid, st);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "blind rotation launch");
    e = launch_keyswitch(ctx->keys.ksk, big, out, nullptr, n, n, ctx->prm.n, ctx->num_sms,
                         ctx->status, st, &ctx->keys);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "key switch launch");
    ctx->launches += 1 + keyswitch_kernels(n, ctx->num_sms, &ctx->keys);
    return TFHE_OK;
}
