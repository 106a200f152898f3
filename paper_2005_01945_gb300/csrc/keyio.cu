// keyio.cu -- saving and loading a context's device keys.
//
// A serving process that restarts, or a second process on the same GPU,
// can reuse keys without the client's key material and without redoing the
// bootstrapping key's transform: the file holds the keys exactly as the
// context keeps them in device memory (the bootstrapping key in the NTT
// domain of the library's two primes, the key-switching key in padded
// rows).  The format is tied to this library: a header records the
// parameters, the primes, the sizes and a 64-bit FNV-1a checksum of the
// payload, and loading rejects any mismatch.
#include <cstdio>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace tgb {

constexpr char kKeyMagic[8] = {'T', 'F', 'H', 'E', 'G', 'B', 'K', '1'};

struct KeyFileHeader {
    char magic[8];
    uint32_t abi_version, header_bytes;
    int32_t n, N, k, l, bg_bit, ks_t, ks_basebit, pad;
    uint32_t q0, q1;
    uint64_t bk_bytes, ksk_bytes, checksum;
};

static uint64_t fnv1a(uint64_t h, const uint8_t *p, size_t len)
{
    for (size_t i = 0; i < len; ++i) {
        h ^= p[i];
        h *= 0x100000001B3ull;
    }
    return h;
}

static size_t bk_ntt_bytes(const tfhe_ctx *ctx)
{
    return (size_t)ctx->prm.n * 2 * 2 * kN * kRows * sizeof(uint32_t);
}

static size_t ksk_bytes()
{
    return (size_t)kN * kKsT * kKsDigits * kLweStride * sizeof(int32_t);
}

static KeyFileHeader header_of(const tfhe_ctx *ctx)
{
    KeyFileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kKeyMagic, sizeof(kKeyMagic));
    h.abi_version = TFHE_GB_ABI_VERSION;
    h.header_bytes = sizeof(KeyFileHeader);
    h.n = ctx->prm.n;
    h.N = ctx->prm.N;
    h.k = ctx->prm.k;
    h.l = ctx->prm.l;
    h.bg_bit = ctx->prm.bg_bit;
    h.ks_t = ctx->prm.ks_t;
    h.ks_basebit = ctx->prm.ks_basebit;
    h.q0 = kQ0;
    h.q1 = kQ1;
    h.bk_bytes = bk_ntt_bytes(ctx);
    h.ksk_bytes = ksk_bytes();
    return h;
}

}  // namespace tgb

using namespace tgb;

extern "C" int tfhe_ctx_save_keys(tfhe_ctx *ctx, const char *path)
{
    if (!ctx || !path)
        return TFHE_EINVAL;
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_save_keys: keys not set");
    DeviceGuard dg(ctx->device);
    KeyFileHeader h = header_of(ctx);
    std::vector<uint8_t> payload(h.bk_bytes + h.ksk_bytes);
    cudaError_t e = cudaMemcpy(payload.data(), ctx->bk_ntt, h.bk_bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(payload.data() + h.bk_bytes, ctx->ksk, h.ksk_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tfhe_ctx_save_keys");
    h.checksum = fnv1a(0xCBF29CE484222325ull, payload.data(), payload.size());
    FILE *f = std::fopen(path, "wb");
    if (!f)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_save_keys: cannot open %s", path);
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                    std::fwrite(payload.data(), 1, payload.size(), f) == payload.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_save_keys: write to %s failed", path);
    return TFHE_OK;
}

extern "C" int tfhe_ctx_load_keys(tfhe_ctx *ctx, const char *path)
{
    if (!ctx || !path)
        return TFHE_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_load_keys: cannot open %s", path);
    KeyFileHeader h;
    const KeyFileHeader want = header_of(ctx);
    if (std::fread(&h, sizeof(h), 1, f) != 1) {
        std::fclose(f);
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_load_keys: %s is too short", path);
    }
    if (std::memcmp(h.magic, want.magic, sizeof(h.magic)) != 0 ||
        h.abi_version != want.abi_version || h.header_bytes != want.header_bytes) {
        std::fclose(f);
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_load_keys: %s is not a key file of this library",
                    path);
    }
    if (h.n != want.n || h.N != want.N || h.k != want.k || h.l != want.l ||
        h.bg_bit != want.bg_bit || h.ks_t != want.ks_t || h.ks_basebit != want.ks_basebit ||
        h.q0 != want.q0 || h.q1 != want.q1 || h.bk_bytes != want.bk_bytes ||
        h.ksk_bytes != want.ksk_bytes) {
        std::fclose(f);
        return fail(ctx, TFHE_EINVAL,
                    "tfhe_ctx_load_keys: %s holds keys for other parameters (n = %d, N = %d)",
                    path, h.n, h.N);
    }
    std::vector<uint8_t> payload(h.bk_bytes + h.ksk_bytes);
    const bool ok = std::fread(payload.data(), 1, payload.size(), f) == payload.size();
    std::fclose(f);
    if (!ok)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_load_keys: %s is truncated", path);
    if (fnv1a(0xCBF29CE484222325ull, payload.data(), payload.size()) != h.checksum)
        return fail(ctx, TFHE_EINVAL, "tfhe_ctx_load_keys: checksum mismatch in %s", path);
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaSuccess;
    if (!ctx->bk_ntt)
        e = cudaMalloc(&ctx->bk_ntt, h.bk_bytes);
    if (e == cudaSuccess && !ctx->ksk)
        e = cudaMalloc(&ctx->ksk, h.ksk_bytes);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->bk_ntt, payload.data(), h.bk_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->ksk, payload.data() + h.bk_bytes, h.ksk_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tfhe_ctx_load_keys");
    ctx->keys.bk_ntt = reinterpret_cast<const uint4 *>(ctx->bk_ntt);
    ctx->keys.ksk = ctx->ksk;
    ctx->keys_loaded = true;
    return TFHE_OK;
}
