// cmux_tc.cu -- the CMux external product's negacyclic products on the
// tensor pipe (tcgen05), exactly, as the measured alternative to the NTT.
//
// One CMux step multiplies the 4 digit polynomials d_r of every bootstrap
// (r = c l + j: gadget digit j of TLWE polynomial c, digits in [-512, 511])
// by the 4 x 2 polynomials BK_i[r][p] of the step's TGSW key and sums over
// r, in Z[X]/(X^N + 1) mod 2^32 (the external product of paper section II-A,
// the construction the paper adopts from TFHE):
//     out[m][p][k] = sum_r sum_i d_r[m][i] T_rp[i][k],
//     T_rp[i][k] = +b_rp[k - i] (i <= k),  -b_rp[N + k - i] (i > k).
// For a batch of bootstraps that is one matrix product
//     out[M][2N] = D[M][4N] . T[4N][2N]
// whose right operand is fixed by the key.  bf16 operands with fp32
// accumulation make it exact by limb splitting:
//   * d = d_lo + 32 d_hi, d_lo in [-16, 15], d_hi in [-16, 16] (2 limbs x);
//   * b = sum_j beta_j 256^j mod 2^32, balanced bytes beta_j in [-128, 127]
//     (4 limbs j); the sign of T is folded into the limbs, so entries lie in
//     [-128, 128];
//   * every product is at most 16 x 128 = 2^11 in magnitude and a sum of
//     K = 4N = 4096 of them at most 2^23 < 2^24, so each fp32 accumulation
//     S_xj is the exact integer (all partial sums are integers below 2^24);
//   * out = sum_xj S_xj 2^(5x + 8j) mod 2^32 (all 8 limb pairs, since
//     5 + 24 < 32).
// (The 8-bit integer MMA would need 7 limb pairs, but ptxas refuses
// .kind::i8 for sm_103a.)
//
// Layout (all K-major, no swizzle, 8 x 8 bf16 core matrices of 128 bytes):
//   A_x  [M/128][K/32][16 row groups][4 K groups][8][8]: one 8 KB tile per
//        (128 bootstraps, 32 K values);
//   B_j  [2N/256][K/32][32 column groups][4 K groups][8][8]: one 16 KB tile
//        per (256 output coefficients, 32 K values), the transposed Toeplitz
//        operand, prepared once per key (64 MB per CMux step).
// Kernel: one CTA per 128 bootstraps x 256 output coefficients.  Warp 0
// streams A and B tiles into a 3-stage ring with bulk copies (cp.async.bulk,
// completion on mbarriers); one thread of warp 1 issues tcgen05.mma
// (M = 128, N = 256, K = 16, bf16 x bf16 -> fp32) into one of two 256-column
// TMEM accumulators per limb pair; warps 4-7 read a finished accumulator
// (tcgen05.ld), convert it to integers and shift-add it into a 32-bit
// result tile in shared memory while the next pair accumulates.  Every wait
// is bounded: a wait that runs out sets kErrTimeout, the roles stop, the
// copies and MMAs in flight are waited for (bounded) and TMEM is freed.
#include <cuda_bf16.h>

#include "runtime.h"

namespace tgb {

constexpr int kTcM = 128;                  // bootstraps per CTA tile
constexpr int kTcN = 256;                  // output coefficients per CTA tile
constexpr int kTcKb = 32;                  // K values per stage
constexpr int kTcK = kRows * kN;           // 4096
constexpr int kTcNkb = kTcK / kTcKb;       // 128 stages per limb pair
constexpr int kTcPairs = 8;                // (x, j): 2 digit limbs x 4 key bytes
constexpr int kTcStages = 3;
constexpr int kTcABytes = kTcM * kTcKb * 2;    // 8 KB
constexpr int kTcBBytes = kTcN * kTcKb * 2;    // 16 KB
constexpr int kTcAccStride = kTcN + 1;         // words; odd: conflict-free rows
constexpr int kTcThreads = 256;
constexpr long kTcSpin = 1L << 20;             // bounded waits (x ~1 us)

struct TcSmem {
    uint8_t a[kTcStages][kTcABytes];               // 1024-byte aligned stages
    uint8_t b[kTcStages][kTcBBytes];
    uint32_t acc[kTcM * kTcAccStride];             // exact 32-bit results
    unsigned long long full[kTcStages], empty[kTcStages];
    unsigned long long acc_full[2], acc_empty[2], drain;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint32_t tc_smem(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tc_bar_init(unsigned long long *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(b)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void tc_bar_arrive(unsigned long long *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(b)) : "memory");
}

__device__ __forceinline__ void tc_bar_expect(unsigned long long *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(b)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait for phase `parity`; false if it ran out.
__device__ __forceinline__ bool tc_bar_wait(unsigned long long *b, uint32_t parity)
{
    for (long i = 0; i < kTcSpin; ++i) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(tc_smem(b)), "r"(parity), "r"(1000u)
                     : "memory");
        if (ok)
            return true;
    }
    return false;
}

__device__ __forceinline__ void tc_bulk(void *dst, const void *src, uint32_t bytes,
                                        unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];" ::"r"(tc_smem(dst)),
                 "l"(src), "r"(bytes), "r"(tc_smem(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance
// of core matrices adjacent in K, sbo = of 8-row groups adjacent in M / N.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------
// Operand preparation
// ---------------------------------------------------------------------

// Element offset of (row, k) in a tile-ordered K-major operand whose tiles
// hold `rows` rows x kTcKb K values.
__device__ __forceinline__ long tc_offset(long row, int k, int rows)
{
    const long tile = row / rows, rr = row % rows;
    const int kb = k / kTcKb, kk = k % kTcKb;
    return (((((tile * kTcNkb + kb) * (rows / 8) + rr / 8) * 4 + kk / 8) * 8 + rr % 8) * 8) +
           kk % 8;
}

// Digits [M][4][N] (int32 in [-512, 511]) -> A_0 (d_lo) and A_1 (d_hi).
__global__ void k_tc_prep_digits(const int32_t *__restrict__ digits, __nv_bfloat16 *a0,
                                 __nv_bfloat16 *a1, long M, uint32_t *status)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * kTcK)
        return;
    const long m = e / kTcK;
    const int k = (int)(e % kTcK);
    const int d = digits[e];
    if (d < -512 || d > 511) {
        atomicOr(status, kErrGather);
        return;
    }
    const int hi = (d + 16) >> 5;   // floor((d + 16) / 32)
    const int lo = d - 32 * hi;
    const long o = tc_offset(m, k, kTcM);
    a0[o] = __int2bfloat16_rn(lo);
    a1[o] = __int2bfloat16_rn(hi);
}

// Key polynomials [4 rows][2 polys][N] (uint32) -> B_j, j < 4: element
// (n' = p N + k, K' = r N + i) = sign * beta_j(b_rp[(k - i) mod N]).
__global__ void k_tc_prep_key(const uint32_t *__restrict__ bk, __nv_bfloat16 *bt)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per = (long)2 * kN * kTcK;
    if (e >= 4 * per)
        return;
    const int j = (int)(e / per);
    const long rem = e % per;
    const long np = rem / kTcK;
    const int kp = (int)(rem % kTcK);
    const int p = (int)(np / kN), k = (int)(np % kN);
    const int r = kp / kN, i = kp % kN;
    const uint32_t b = bk[(r * 2 + p) * kN + ((k - i) & (kN - 1))];
    // balanced bytes: b = sum beta_j 256^j mod 2^32, beta_j in [-128, 127]
    int64_t u = b;
    int beta = 0;
    for (int t = 0; t <= j; ++t) {
        beta = (int)(((u + 128) & 255) - 128);
        u = (u - beta) >> 8;
    }
    const int v = k >= i ? beta : -beta;
    bt[(long)j * per + tc_offset(np, kp, kTcN)] = __int2bfloat16_rn(v);
}

// ---------------------------------------------------------------------
// Product kernel
// ---------------------------------------------------------------------

struct TcArgs {
    const __nv_bfloat16 *a[2];   // A_x
    const __nv_bfloat16 *b[4];   // B_j
    uint32_t *out;               // [M][2][N]
    uint32_t *status;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_cmux_products_tc(const TcArgs A)
{
    extern __shared__ __align__(1024) uint8_t tc_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long mtile = blockIdx.y;
    const int ntile = blockIdx.x;

    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            tc_bar_init(&S.full[s], 1);
            tc_bar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc_bar_init(&S.acc_full[b], 1);
            tc_bar_init(&S.acc_empty[b], 128);
        }
        tc_bar_init(&S.drain, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(&S.tmem)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    volatile int *abort = &S.abort;

    if (warp == 0) {
        // producer: stage (pair q, K block kb) <- A_x and B_j tiles
        if (lane == 0) {
            int it = 0;
            for (int q = 0; q < kTcPairs && !*abort; ++q) {
                const int x = q >> 2, j = q & 3;
                const __nv_bfloat16 *asrc = A.a[x] + (mtile * kTcNkb) * (kTcABytes / 2);
                const __nv_bfloat16 *bsrc = A.b[j] + ((long)ntile * kTcNkb) * (kTcBBytes / 2);
                for (int kb = 0; kb < kTcNkb; ++kb, ++it) {
                    const int s = it % kTcStages;
                    if (it >= kTcStages &&
                        !tc_bar_wait(&S.empty[s], ((it / kTcStages) - 1) & 1)) {
                        *abort = 1;
                        atomicOr(A.status, kErrTimeout);
                        break;
                    }
                    tc_bar_expect(&S.full[s], kTcABytes + kTcBBytes);
                    tc_bulk(S.a[s], asrc + (long)kb * (kTcABytes / 2), kTcABytes, &S.full[s]);
                    tc_bulk(S.b[s], bsrc + (long)kb * (kTcBBytes / 2), kTcBBytes, &S.full[s]);
                }
                if (*abort)
                    break;
            }
            // copies still in flight must land before the CTA exits: the last
            // use of each stage completes its barrier's phase (use & 1)
            if (*abort)
                for (int t = it > kTcStages ? it - kTcStages : 0; t < it; ++t)
                    (void)tc_bar_wait(&S.full[t % kTcStages], (t / kTcStages) & 1);
        }
    } else if (warp == 1) {
        // MMA issuer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int q = 0; q < kTcPairs && ok; ++q) {
                const int buf = q & 1;
                if (q >= 2 && !tc_bar_wait(&S.acc_empty[buf], ((q >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * kTcN);
                for (int kb = 0; kb < kTcNkb; ++kb, ++it) {
                    const int s = it % kTcStages;
                    if (*abort || !tc_bar_wait(&S.full[s], (it / kTcStages) & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ab = tc_smem(S.a[s]), bb = tc_smem(S.b[s]);
#pragma unroll
                    for (int kk = 0; kk < kTcKb / 16; ++kk)
                        tc_mma(d, tc_desc(ab + kk * 256, 128, 512),
                               tc_desc(bb + kk * 256, 128, 512), (kb | kk) != 0);
                    tc_commit(&S.empty[s]);   // the stage is free once these MMAs are done
                }
                if (ok)
                    tc_commit(&S.acc_full[buf]);
            }
            if (!ok) {
                *abort = 1;
                atomicOr(A.status, kErrTimeout);
            }
            // every MMA issued so far has completed before TMEM is freed
            tc_commit(&S.drain);
            (void)tc_bar_wait(&S.drain, 0);
        }
    } else if (warp >= 4) {
        // epilogue: TMEM lanes 32 (warp - 4) .. + 31 hold bootstraps of the tile
        const int m = (warp - 4) * 32 + lane;
        uint32_t *row = &S.acc[m * kTcAccStride];
        for (int q = 0; q < kTcPairs; ++q) {
            const int buf = q & 1, x = q >> 2, j = q & 3;
            // one lane waits and the warp follows it, so the warp stays
            // converged for the .sync.aligned TMEM loads
            int ok = 0;
            if (lane == 0) {
                ok = !*abort && tc_bar_wait(&S.acc_full[buf], (q >> 1) & 1);
                if (!ok) {
                    *abort = 1;
                    atomicOr(A.status, kErrTimeout);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok)
                break;
            __syncwarp();
            tc_fence_after();
            const int shift = 5 * x + 8 * j;
            const uint32_t base = tmem + ((uint32_t)((warp - 4) * 32) << 16) + (uint32_t)(buf * kTcN);
            for (int c0 = 0; c0 < kTcN; c0 += 32) {
                float v[32];
                tc_ld32(base + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const uint32_t t = (uint32_t)__float2int_rn(v[i]) << shift;
                    row[c0 + i] = q == 0 ? t : row[c0 + i] + t;
                }
            }
            tc_fence_before();
            tc_bar_arrive(&S.acc_empty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!*abort && warp >= 4) {
        // the warp writes its 32 rows, 256 consecutive words each (coalesced)
        const int p = (ntile * kTcN) / kN, k0 = (ntile * kTcN) % kN;
        for (int rr = 0; rr < 32; ++rr) {
            const int mm = (warp - 4) * 32 + rr;
            const long g = mtile * kTcM + mm;
            uint32_t *dst = A.out + (g * 2 + p) * kN + k0;
            const uint32_t *src = &S.acc[mm * kTcAccStride];
#pragma unroll
            for (int c = 0; c < kTcN; c += 32)
                dst[c + lane] = src[c + lane];
        }
    }
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                     : "memory");
}

}  // namespace tgb

using namespace tgb;

extern "C" {

size_t tfhe_tc_key_bytes(void) { return (size_t)4 * 2 * kN * kTcK * 2; }

size_t tfhe_tc_digit_bytes(size_t count) { return (size_t)2 * count * kTcK * 2; }

int tfhe_tc_prepare_key(tfhe_ctx *ctx, const uint32_t *bk_rows, void *key_ops, void *stream)
{
    if (!ctx || !bk_rows || !key_ops)
        return ctx ? fail(ctx, TFHE_EINVAL, "tfhe_tc_prepare_key: null argument") : TFHE_EINVAL;
    if ((uintptr_t)key_ops % 16)
        return fail(ctx, TFHE_EINVAL, "tfhe_tc_prepare_key: key_ops must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    const long total = 4L * 2 * kN * kTcK;
    k_tc_prep_key<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        bk_rows, (__nv_bfloat16 *)key_ops);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tc key preparation");
    ctx->launches += 1;
    return TFHE_OK;
}

int tfhe_cmux_products_tc(tfhe_ctx *ctx, const int32_t *digits, const void *key_ops,
                          void *digit_ops, uint32_t *out, size_t count, void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (count == 0)
        return TFHE_OK;
    if (!digits || !key_ops || !digit_ops || !out)
        return fail(ctx, TFHE_EINVAL, "tfhe_cmux_products_tc: null argument");
    if (count % kTcM)
        return fail(ctx, TFHE_EINVAL, "tfhe_cmux_products_tc: count %zu is not a multiple of %d",
                    count, kTcM);
    if (count / kTcM > 65535)
        return fail(ctx, TFHE_EINVAL, "tfhe_cmux_products_tc: count %zu too large", count);
    if ((uintptr_t)key_ops % 16 || (uintptr_t)digit_ops % 16)
        return fail(ctx, TFHE_EINVAL, "tfhe_cmux_products_tc: operands must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long M = (long)count;
    __nv_bfloat16 *a0 = (__nv_bfloat16 *)digit_ops, *a1 = a0 + M * kTcK;
    k_tc_prep_digits<<<(unsigned)((M * kTcK + 255) / 256), 256, 0, st>>>(digits, a0, a1, M,
                                                                         ctx->status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tc digit preparation");
    const int smem = (int)sizeof(TcSmem);
    e = cudaFuncSetAttribute(k_cmux_products_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tc kernel attribute");
    TcArgs A;
    A.a[0] = a0;
    A.a[1] = a1;
    const __nv_bfloat16 *bt = (const __nv_bfloat16 *)key_ops;
    for (int j = 0; j < 4; ++j)
        A.b[j] = bt + (long)j * 2 * kN * kTcK;
    A.out = out;
    A.status = ctx->status;
    dim3 grid(2 * kN / kTcN, (unsigned)(M / kTcM));
    k_cmux_products_tc<<<grid, kTcThreads, smem, st>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tc product launch");
    ctx->launches += 2;
    return TFHE_OK;
}

}  // extern "C"
