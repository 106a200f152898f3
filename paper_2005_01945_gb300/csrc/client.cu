// client.cu -- client-side helpers on the device: key generation and LWE
// encryption from raw random draws, and phase computation for decryption.
//
// These are not on the bootstrapping path; they let a user (and the
// benchmark) create keys and ciphertexts without a CPU implementation.
// Definitions follow section II-A: an LWE sample is (A, B) with
// B = A.S + e; TLWE samples are the same over Z[X]/(X^N+1); a TGSW
// encryption of s_i adds s_i * h_j, h_j = 2^(32 - 10 (j+1)), to polynomial c
// of row c*l + j of a matrix of TLWE encryptions of zero.
#include "common.cuh"

namespace tgb {

// Warp sum of 32-bit words mod 2^32.
__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per TLWE row (i, r): b(X) = a(X) S(X) + e(X), S binary.
__global__ void __launch_bounds__(256) k_keygen_bk(const int32_t *__restrict__ s,
                                                   const int32_t *__restrict__ S,
                                                   const uint32_t *__restrict__ mask,
                                                   const int32_t *__restrict__ noise,
                                                   int32_t *__restrict__ bk)
{
    __shared__ uint32_t a[kN];
    __shared__ int32_t key[kN];
    const long row = blockIdx.x;  // i * kRows + r
    const int i = (int)(row / kRows), r = (int)(row % kRows);
    for (int k = threadIdx.x; k < kN; k += blockDim.x) {
        a[k] = mask[row * kN + k];
        key[k] = S[k];
    }
    __syncthreads();
    uint32_t acc[kN / 256];
#pragma unroll
    for (int u = 0; u < kN / 256; ++u)
        acc[u] = 0;
    for (int j = 0; j < kN; ++j) {
        if (key[j] == 0)
            continue;  // uniform
#pragma unroll
        for (int u = 0; u < kN / 256; ++u) {
            const int k = threadIdx.x + 256 * u;
            // coefficient k of S_j X^j a(X): a_(k-j), negated when k - j wraps
            acc[u] += k >= j ? a[k - j] : 0u - a[k - j + kN];
        }
    }
    const int c = r / kL, jl = r % kL;
    const uint32_t h = 1u << (32 - kBgBit * (jl + 1));
    int32_t *ra = bk + (row * 2 + 0) * kN;
    int32_t *rb = bk + (row * 2 + 1) * kN;
#pragma unroll
    for (int u = 0; u < kN / 256; ++u) {
        const int k = threadIdx.x + 256 * u;
        uint32_t av = a[k], bv = acc[u] + (uint32_t)noise[row * kN + k];
        if (k == 0) {
            if (c == 0)
                av += (uint32_t)s[i] * h;
            else
                bv += (uint32_t)s[i] * h;
        }
        ra[k] = (int32_t)av;
        rb[k] = (int32_t)bv;
    }
}

// One warp per KSK row (j, q, d): LWE_s encryption of d S_j / base^(q+1).
__global__ void k_keygen_ksk(const int32_t *__restrict__ s, const int32_t *__restrict__ S,
                             const uint32_t *__restrict__ mask, const int32_t *__restrict__ noise,
                             int32_t *__restrict__ ksk, int n, long rows)
{
    const long row = (long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows)
        return;
    const int d = (int)(row % kKsDigits) + 1;
    const int q = (int)((row / kKsDigits) % kKsT);
    const int j = (int)(row / (kKsDigits * kKsT));
    const uint32_t *m = mask + row * n;
    int32_t *o = ksk + row * (n + 1);
    uint32_t dot = 0;
    for (int k = lane; k < n; k += 32) {
        dot += m[k] * (uint32_t)s[k];
        o[k] = (int32_t)m[k];
    }
    dot = warp_sum(dot);
    if (lane == 0) {
        const uint32_t msg = (uint32_t)d * (uint32_t)S[j] * (1u << (32 - kKsBaseBit * (q + 1)));
        o[n] = (int32_t)(dot + (uint32_t)noise[row] + msg);
    }
}

// One warp per ciphertext.
__global__ void k_encrypt(const int32_t *__restrict__ s, const uint32_t *__restrict__ mask,
                          const int32_t *__restrict__ noise, const uint8_t *__restrict__ bits,
                          int32_t *__restrict__ cts, int n, long count)
{
    const long g = (long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= count)
        return;
    const uint32_t *m = mask + g * n;
    int32_t *o = cts + g * kLweStride;
    uint32_t dot = 0;
    for (int k = lane; k < kLweStride; k += 32) {
        if (k < n) {
            dot += m[k] * (uint32_t)s[k];
            o[k] = (int32_t)m[k];
        } else if (k > n) {
            o[k] = 0;
        }
    }
    dot = warp_sum(dot);
    if (lane == 0)
        o[n] = (int32_t)(dot + (uint32_t)noise[g] + (bits[g] ? kMu : 0u - kMu));
}

__global__ void k_phase(const int32_t *__restrict__ s, const int32_t *__restrict__ cts,
                        uint32_t *__restrict__ phase, int n, long count)
{
    const long g = (long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= count)
        return;
    const int32_t *c = cts + g * kLweStride;
    uint32_t dot = 0;
    for (int k = lane; k < n; k += 32)
        dot += (uint32_t)c[k] * (uint32_t)s[k];
    dot = warp_sum(dot);
    if (lane == 0)
        phase[g] = (uint32_t)c[n] - dot;
}

cudaError_t launch_keygen(int n, const int32_t *s, const int32_t *S, const uint32_t *bk_mask,
                          const int32_t *bk_noise, const uint32_t *ksk_mask,
                          const int32_t *ksk_noise, int32_t *bk_out, int32_t *ksk_out,
                          cudaStream_t stream)
{
    k_keygen_bk<<<(unsigned)(n * kRows), 256, 0, stream>>>(s, S, bk_mask, bk_noise, bk_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const long rows = (long)kN * kKsT * kKsDigits;
    k_keygen_ksk<<<(unsigned)((rows + 7) / 8), 256, 0, stream>>>(s, S, ksk_mask, ksk_noise,
                                                                 ksk_out, n, rows);
    return cudaGetLastError();
}

cudaError_t launch_encrypt(int n, const int32_t *s, const uint32_t *mask, const int32_t *noise,
                           const uint8_t *bits, int32_t *cts, long count, cudaStream_t stream)
{
    if (count <= 0)
        return cudaSuccess;
    k_encrypt<<<(unsigned)((count + 7) / 8), 256, 0, stream>>>(s, mask, noise, bits, cts, n, count);
    return cudaGetLastError();
}

cudaError_t launch_phase(int n, const int32_t *s, const int32_t *cts, uint32_t *phase, long count,
                         cudaStream_t stream)
{
    if (count <= 0)
        return cudaSuccess;
    k_phase<<<(unsigned)((count + 7) / 8), 256, 0, stream>>>(s, cts, phase, n, count);
    return cudaGetLastError();
}

}  // namespace tgb
