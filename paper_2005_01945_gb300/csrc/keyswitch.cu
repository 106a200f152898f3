// keyswitch.cu -- LWE_N -> LWE_n key switching of extracted samples.
//
// The method (the paper times it as "Key Switch", Table "differentialtime";
// its key is the "KS key" of Fig. "gpu_execution"): every a'_j is rounded
// to t * basebit = 16 bits, written as 8 base-4 digits d_(j,q) of weight
// 4^-(q+1), and out = (0, b') - sum_(j,q) KSK[j][q][d_(j,q)] with the digit-0
// sample identically zero.
//
// GB300 design: the key-switching key (50 MB padded) is the only large
// operand.  One CTA keeps 16 gates' accumulators in registers (thread t
// owns words 4t..4t+3 of the 512-word row, read as 16-byte vectors) and
// streams the key rows of its j-range once for all 16 gates, so the key is
// read ceil(count/16) times over L2 instead of once per gate.  For small
// batches the j-range is split across CTAs and the partial sums are added
// with 32-bit atomics (integer addition mod 2^32 is associative, so the
// result is bit-identical to a sequential sum).
#include "common.cuh"

namespace tgb {

constexpr int kKsGates = 16;
constexpr int kKsThreads = 128;

struct KsArgs {
    const uint4 *ksk;         // [N][t][3][kLweStride/4]
    const int32_t *big;       // [count][kBigStride]
    int32_t *out;             // output base, row stride kLweStride
    const int32_t *idx_out;   // optional scatter rows (nullptr: row g)
    long rows_out;
    long count;
    int n;
    int j_chunk;              // j values per CTA (blockIdx.y selects the chunk)
    int atomic;               // 1: add into pre-initialised rows
    uint32_t *status;
};

__device__ __forceinline__ long ks_dest(const KsArgs &A, long g)
{
    return A.idx_out ? (long)A.idx_out[g] : g;
}

// out[dest][c] = (c == n) ? b' : 0, for the atomic accumulation path.
__global__ void k_ks_init(const KsArgs A)
{
    const long g = blockIdx.x;
    if (g >= A.count)
        return;
    const long d = ks_dest(A, g);
    if (d < 0 || d >= A.rows_out) {
        if (threadIdx.x == 0)
            atomicOr(A.status, kErrScatter);
        return;
    }
    const int32_t bprime = A.big[g * kBigStride + kN];
    for (int c = threadIdx.x; c < kLweStride; c += blockDim.x)
        A.out[d * kLweStride + c] = c == A.n ? bprime : 0;
}

__global__ void __launch_bounds__(kKsThreads) k_keyswitch(const KsArgs A)
{
    __shared__ __align__(16) uint16_t wsh[kN][kKsGates];  // rounded a'_j, 16 gates per j
    const int t = threadIdx.x;
    const long g0 = (long)blockIdx.x * kKsGates;
    const int j0 = blockIdx.y * A.j_chunk;
    const int j1 = min(kN, j0 + A.j_chunk);
    const int ng = (int)min((long)kKsGates, A.count - g0);

    for (int e = t; e < (j1 - j0) * kKsGates; e += kKsThreads) {
        const int jj = e / kKsGates, gg = e % kKsGates;
        uint32_t w = 0;
        if (gg < ng) {
            const uint32_t a = (uint32_t)A.big[(g0 + gg) * kBigStride + j0 + jj];
            w = ((a + (1u << 15)) >> 16) & 0xFFFFu;    // round to 16 bits
        }
        wsh[jj][gg] = (uint16_t)w;
    }
    __syncthreads();

    uint4 acc[kKsGates];
#pragma unroll
    for (int gg = 0; gg < kKsGates; ++gg)
        acc[gg] = make_uint4(0u, 0u, 0u, 0u);

    for (int j = j0; j < j1; ++j) {
        const uint4 wa = *reinterpret_cast<const uint4 *>(&wsh[j - j0][0]);
        const uint4 wb = *reinterpret_cast<const uint4 *>(&wsh[j - j0][8]);
        const uint32_t wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
        const uint4 *rowq = A.ksk + (long)j * kKsT * kKsDigits * (kLweStride / 4) + t;
#pragma unroll 2
        for (int q = 0; q < kKsT; ++q) {
            const uint4 *row = rowq + q * kKsDigits * (kLweStride / 4);
            const uint4 r1 = __ldg(row);
            const uint4 r2 = __ldg(row + (kLweStride / 4));
            const uint4 r3 = __ldg(row + 2 * (kLweStride / 4));
            const int shift = 14 - 2 * q;
#pragma unroll
            for (int gg = 0; gg < kKsGates; ++gg) {
                const uint32_t w = (wv[gg >> 1] >> ((gg & 1) * 16)) & 0xFFFFu;
                const uint32_t d = (w >> shift) & 3u;
                if (d != 0u) {   // uniform across the CTA
                    const uint4 v = d == 1u ? r1 : (d == 2u ? r2 : r3);
                    acc[gg].x -= v.x;
                    acc[gg].y -= v.y;
                    acc[gg].z -= v.z;
                    acc[gg].w -= v.w;
                }
            }
        }
    }

#pragma unroll
    for (int gg = 0; gg < kKsGates; ++gg) {
        if (gg >= ng)
            break;
        const long g = g0 + gg;
        const long d = ks_dest(A, g);
        if (d < 0 || d >= A.rows_out) {
            if (t == 0 && !A.atomic)
                atomicOr(A.status, kErrScatter);
            continue;
        }
        uint32_t *o = reinterpret_cast<uint32_t *>(A.out + d * kLweStride) + 4 * t;
        if (A.atomic) {
            atomicAdd(o + 0, acc[gg].x);
            atomicAdd(o + 1, acc[gg].y);
            atomicAdd(o + 2, acc[gg].z);
            atomicAdd(o + 3, acc[gg].w);
        } else {
            const uint32_t bprime = (uint32_t)A.big[g * kBigStride + kN];
            uint4 v = acc[gg];
            if (4 * t + 0 == A.n) v.x += bprime;
            if (4 * t + 1 == A.n) v.y += bprime;
            if (4 * t + 2 == A.n) v.z += bprime;
            if (4 * t + 3 == A.n) v.w += bprime;
            *reinterpret_cast<uint4 *>(o) = v;
        }
    }
}

static int ks_forced_chunks = 0;   // set while the autotuner measures

// j-chunks: the tuned value for the width bucket, else enough CTAs for two
// per SM.
static int ks_chunks(long count, int num_sms, const int8_t *tuned)
{
    if (ks_forced_chunks)
        return ks_forced_chunks;
    if (tuned && tuned[tune_bucket(count)] > 0)
        return tuned[tune_bucket(count)];
    const long tiles = (count + kKsGates - 1) / kKsGates;
    int chunks = 1;
    while (chunks < 32 && tiles * chunks < 2L * num_sms)
        chunks *= 2;
    return chunks;
}

void keyswitch_force_chunks(int chunks) { ks_forced_chunks = chunks; }

// Kernels one launch_keyswitch call issues.
int keyswitch_kernels(long count, int num_sms, const int8_t *tuned)
{
    return count <= 0 ? 0 : (ks_chunks(count, num_sms, tuned) > 1 ? 2 : 1);
}

// Splits the j-range so that small batches still occupy the GPU.
cudaError_t launch_keyswitch(const uint4 *ksk, const int32_t *big, int32_t *out,
                             const int32_t *idx_out, long rows_out, long count, int n,
                             int num_sms, uint32_t *status, cudaStream_t stream,
                             const int8_t *tuned)
{
    if (count <= 0)
        return cudaSuccess;
    const long tiles = (count + kKsGates - 1) / kKsGates;
    const int chunks = ks_chunks(count, num_sms, tuned);
    KsArgs A;
    A.ksk = ksk;
    A.big = big;
    A.out = out;
    A.idx_out = idx_out;
    A.rows_out = rows_out;
    A.count = count;
    A.n = n;
    A.j_chunk = kN / chunks;
    A.atomic = chunks > 1;
    A.status = status;
    if (A.atomic) {
        k_ks_init<<<(unsigned)count, 128, 0, stream>>>(A);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    dim3 grid((unsigned)tiles, (unsigned)chunks);
    k_keyswitch<<<grid, kKsThreads, 0, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace tgb
