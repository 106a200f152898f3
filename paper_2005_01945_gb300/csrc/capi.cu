// capi.cu -- extern "C" entry points declared in include/tfhe_gb.h: context
// and key management, batched gate bootstrapping, its two stages, and the
// client-side helpers.  Circuit and serving entry points live in
// circuits.cu and serve.cu, the allocation-free gate call in noalloc.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "runtime.h"

namespace tgb {

cudaError_t upload_ntt_constants(uint2 *twb_dev, cudaStream_t stream);
cudaError_t launch_bk_to_ntt(const int32_t *bk_dev, uint32_t *bk_ntt, int n, const uint2 *twb,
                             cudaStream_t stream);
cudaError_t launch_keygen(int n, const int32_t *s, const int32_t *S, const uint32_t *bk_mask,
                          const int32_t *bk_noise, const uint32_t *ksk_mask,
                          const int32_t *ksk_noise, int32_t *bk_out, int32_t *ksk_out,
                          cudaStream_t stream);
cudaError_t launch_encrypt(int n, const int32_t *s, const uint32_t *mask, const int32_t *noise,
                           const uint8_t *bits, int32_t *cts, long count, cudaStream_t stream);
cudaError_t launch_phase(int n, const int32_t *s, const int32_t *cts, uint32_t *phase, long count,
                         cudaStream_t stream);
int br_blocks_per_sm();

int fail(tfhe_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> lock(ctx->err_mu);
        ctx->err = buf;
    }
    return code;
}

int cuda_fail(tfhe_ctx *ctx, cudaError_t e, const char *where)
{
    (void)cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? TFHE_ENOMEM : TFHE_ECUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

bool params_supported(const tfhe_params *p)
{
    return p && p->n >= 1 && p->n <= kMaxN && p->N == kN && p->k == 1 && p->l == kL &&
           p->bg_bit == kBgBit && p->ks_t == kKsT && p->ks_basebit == kKsBaseBit;
}

int ensure_big(tfhe_ctx *ctx, size_t rows)
{
    if (ctx->big_rows >= rows)
        return TFHE_OK;
    size_t want = ctx->big_rows ? ctx->big_rows : 1024;
    while (want < rows)
        want *= 2;
    if (ctx->big) {
        cudaError_t e = cudaFree(ctx->big);   // synchronising: safe w.r.t. in-flight use
        ctx->big = nullptr;
        ctx->big_rows = 0;
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "cudaFree(scratch)");
    }
    cudaError_t e = cudaMalloc(&ctx->big, want * kBigStride * sizeof(int32_t));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(scratch)");
    ctx->big_rows = want;
    return TFHE_OK;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int run_bootstrap(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a, const int32_t *idx_a,
                  long rows_a, const int32_t *b, const int32_t *idx_b, long rows_b, int32_t *out,
                  const int32_t *idx_out, long rows_out, long count, uint32_t mu,
                  cudaStream_t stream)
{
    int rc = ensure_big(ctx, (size_t)count);
    if (rc != TFHE_OK)
        return rc;
    cudaError_t e;
    {
        NvtxRange r("tfhe: gate combine + mod switch + blind rotation + extraction");
        e = launch_blind_rotate(ctx->keys, ops, a, idx_a, rows_a, b, idx_b, rows_b, ctx->big,
                                count, mu, ctx->status, ctx->br_grid, stream);
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "blind rotation launch");
    NvtxRange r("tfhe: key switch");
    e = launch_keyswitch(ctx->keys.ksk, ctx->big, out, idx_out, rows_out, count, ctx->prm.n,
                         ctx->num_sms, ctx->status, stream, &ctx->keys);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "key switch launch");
    ctx->launches += 1 + keyswitch_kernels(count, ctx->num_sms, &ctx->keys);
    return TFHE_OK;
}

}  // namespace tgb

using namespace tgb;

extern "C" {

int tfhe_ctx_create(const tfhe_params *params, int device, tfhe_ctx **out)
{
    if (!out)
        return TFHE_EINVAL;
    *out = nullptr;
    if (!params_supported(params))
        return TFHE_EINVAL;
    tfhe_ctx *ctx = new (std::nothrow) tfhe_ctx();
    if (!ctx)
        return TFHE_ENOMEM;
    ctx->prm = *params;
    ctx->device = device;
    DeviceGuard dg(device);
    if (!dg.ok) {
        delete ctx;
        return TFHE_ECUDA;
    }
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->twb, 2 * 2 * 32 * 32 * sizeof(uint2));
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->status, sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemset(ctx->status, 0, sizeof(uint32_t));
    if (e == cudaSuccess)
        e = upload_ntt_constants(ctx->twb, 0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        tfhe_ctx_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? TFHE_ENOMEM : TFHE_ECUDA;
    }
    ctx->br_grid = br_blocks_per_sm() * ctx->num_sms;
    ctx->keys.twb = ctx->twb;
    ctx->keys.n = params->n;
    *out = ctx;
    return TFHE_OK;
}

int tfhe_ctx_set_keys(tfhe_ctx *ctx, const int32_t *bk, const int32_t *ksk, void *stream)
{
    if (!ctx || !bk || !ksk)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_set_keys: null argument");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = ctx->prm.n;
    const size_t bk_words = (size_t)n * kRows * 2 * kN;
    const size_t ksk_rows = (size_t)kN * kKsT * kKsDigits;
    int32_t *bk_tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!ctx->bk_ntt)
        e = cudaMalloc(&ctx->bk_ntt, (size_t)n * 2 * 2 * kN * kRows * sizeof(uint32_t));
    if (e == cudaSuccess && !ctx->ksk)
        e = cudaMalloc(&ctx->ksk, ksk_rows * kLweStride * sizeof(int32_t));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(keys)");
    const int32_t *bk_dev = bk;
    if (!is_device_ptr(bk)) {
        e = cudaMalloc(&bk_tmp, bk_words * sizeof(int32_t));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bk_tmp, bk, bk_words * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(bk_tmp);
            return cuda_fail(ctx, e, "upload(bk)");
        }
        bk_dev = bk_tmp;
    }
    e = launch_bk_to_ntt(bk_dev, ctx->bk_ntt, n, ctx->twb, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->ksk, 0, ksk_rows * kLweStride * sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(ctx->ksk, kLweStride * sizeof(int32_t), ksk,
                              (size_t)(n + 1) * sizeof(int32_t), (size_t)(n + 1) * sizeof(int32_t),
                              ksk_rows, cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(bk_tmp);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tfhe_ctx_set_keys");
    ctx->keys.bk_ntt = reinterpret_cast<const uint4 *>(ctx->bk_ntt);
    ctx->keys.ksk = ctx->ksk;
    ctx->keys_loaded = true;
    return TFHE_OK;
}

void tfhe_ctx_destroy(tfhe_ctx *ctx)
{
    if (!ctx)
        return;
    {
        DeviceGuard dg(ctx->device);
        release_circuits(ctx);
        release_serving(ctx);
        cudaFree(ctx->twb);
        cudaFree(ctx->status);
        cudaFree(ctx->bk_ntt);
        cudaFree(ctx->ksk);
        cudaFree(ctx->big);
        (void)cudaGetLastError();
    }
    delete ctx;
}

int tfhe_last_error(const tfhe_ctx *ctx, char *buf, size_t len)
{
    if (!ctx || !buf || len == 0)
        return TFHE_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->err_mu);
    std::snprintf(buf, len, "%s", ctx->err.c_str());
    return TFHE_OK;
}

int tfhe_ctx_status(tfhe_ctx *ctx, uint32_t *code)
{
    if (!ctx)
        return TFHE_EINVAL;
    DeviceGuard dg(ctx->device);
    uint32_t w = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(&w, ctx->status, sizeof(w), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemset(ctx->status, 0, sizeof(uint32_t));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tfhe_ctx_status");
    if (code)
        *code = w;
    if (w)
        return fail(ctx, TFHE_EDEVICE, "device status word 0x%x", w);
    return TFHE_OK;
}

int tfhe_bootstrap_gates(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a, const int32_t *b,
                         int32_t *out, size_t count, void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (count == 0)
        return TFHE_OK;
    if (!ops || !a || !b || !out)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap_gates: null argument");
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap_gates: keys not set");
    DeviceGuard dg(ctx->device);
    return run_bootstrap(ctx, ops, a, nullptr, (long)count, b, nullptr, (long)count, out, nullptr,
                         (long)count, (long)count, kMu, (cudaStream_t)stream);
}

int tfhe_bootstrap(tfhe_ctx *ctx, const int32_t *in, int32_t *out, size_t count, uint32_t mu,
                   void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (count == 0)
        return TFHE_OK;
    if (!in || !out)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap: null argument");
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "tfhe_bootstrap: keys not set");
    DeviceGuard dg(ctx->device);
    return run_bootstrap(ctx, nullptr, in, nullptr, (long)count, nullptr, nullptr, 0, out, nullptr,
                         (long)count, (long)count, mu, (cudaStream_t)stream);
}

int tfhe_blind_rotate_extract(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a,
                              const int32_t *b, int32_t *big, size_t count, void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (count == 0)
        return TFHE_OK;
    if (!a || !big || (ops && !b))
        return fail(ctx, TFHE_EINVAL, "tfhe_blind_rotate_extract: null argument");
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "tfhe_blind_rotate_extract: keys not set");
    DeviceGuard dg(ctx->device);
    cudaError_t e = launch_blind_rotate(ctx->keys, ops, a, nullptr, (long)count, b, nullptr,
                                        (long)count, big, (long)count, kMu, ctx->status,
                                        ctx->br_grid, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "blind rotation launch");
    ctx->launches += 1;
    return TFHE_OK;
}

int tfhe_keyswitch(tfhe_ctx *ctx, const int32_t *big, int32_t *out, size_t count, void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (count == 0)
        return TFHE_OK;
    if (!big || !out)
        return fail(ctx, TFHE_EINVAL, "tfhe_keyswitch: null argument");
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "tfhe_keyswitch: keys not set");
    DeviceGuard dg(ctx->device);
    cudaError_t e = launch_keyswitch(ctx->keys.ksk, big, out, nullptr, (long)count, (long)count,
                                     ctx->prm.n, ctx->num_sms, ctx->status, (cudaStream_t)stream,
                                     &ctx->keys);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "key switch launch");
    ctx->launches += keyswitch_kernels((long)count, ctx->num_sms, &ctx->keys);
    return TFHE_OK;
}

int tfhe_ctx_launches(const tfhe_ctx *ctx, uint64_t *launches)
{
    if (!ctx || !launches)
        return TFHE_EINVAL;
    *launches = ctx->launches;
    return TFHE_OK;
}

int tfhe_keygen(const tfhe_params *params, const int32_t *s, const int32_t *S,
                const uint32_t *bk_mask, const int32_t *bk_noise, const uint32_t *ksk_mask,
                const int32_t *ksk_noise, int32_t *bk_out, int32_t *ksk_out, void *stream)
{
    if (!params_supported(params) || !s || !S || !bk_mask || !bk_noise || !ksk_mask ||
        !ksk_noise || !bk_out || !ksk_out)
        return TFHE_EINVAL;
    cudaError_t e = launch_keygen(params->n, s, S, bk_mask, bk_noise, ksk_mask, ksk_noise, bk_out,
                                  ksk_out, (cudaStream_t)stream);
    return e == cudaSuccess ? TFHE_OK : TFHE_ECUDA;
}

int tfhe_encrypt_bits(const tfhe_params *params, const int32_t *s, const uint32_t *masks,
                      const int32_t *noise, const uint8_t *bits, int32_t *cts, size_t count,
                      void *stream)
{
    if (!params_supported(params) || (count && (!s || !masks || !noise || !bits || !cts)))
        return TFHE_EINVAL;
    cudaError_t e = launch_encrypt(params->n, s, masks, noise, bits, cts, (long)count,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? TFHE_OK : TFHE_ECUDA;
}

int tfhe_phase(const tfhe_params *params, const int32_t *s, const int32_t *cts, uint32_t *phase,
               size_t count, void *stream)
{
    if (!params_supported(params) || (count && (!s || !cts || !phase)))
        return TFHE_EINVAL;
    cudaError_t e = launch_phase(params->n, s, cts, phase, (long)count, (cudaStream_t)stream);
    return e == cudaSuccess ? TFHE_OK : TFHE_ECUDA;
}

}  // extern "C"
