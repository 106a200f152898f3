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
// device address: the device address is looked up once per device, with
// that device current, and cached here.
constexpr int kNoAllocMaxDevices = 64;
static int32_t *g_noalloc_dev_ptr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

static int noalloc_scratch(tfhe_ctx *ctx, int32_t **ptr)
{
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap_gates_noalloc: device %d out of range",
                    ctx->device);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_dev_ptr[ctx->device]) {
        int32_t *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_big);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_dev_ptr[ctx->device] = p;
    }
    *ptr = g_noalloc_dev_ptr[ctx->device];
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
    cudaError_t e = launch_blind_rotate(ctx->keys, ops, a, nullptr, n, b, nullptr, n, big, n, kMu,
                                        ctx->status, ctx->br_grid, st);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "blind rotation launch");
    e = launch_keyswitch(ctx->keys.ksk, big, out, nullptr, n, n, ctx->prm.n, ctx->num_sms,
                         ctx->status, st);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "key switch launch");
    ctx->launches += 1 + keyswitch_kernels(n, ctx->num_sms);
    return TFHE_OK;
}
