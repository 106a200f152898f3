// keyswitch.cu -- LWE_N -> LWE_n key switching of extracted samples.
//
// The method (the paper times it as "Key Switch", Table "differentialtime";
// its key is the "KS key" of Fig. "gpu_execution"): every a'_j is rounded
// to t * basebit = 16 bits, written as 8 base-4 digits d_(j,q) of weight
// 4^-(q+1), and out = (0, b') - sum_(j,q) KSK[j][q][d_(j,q)] with the digit-0
// sample identically zero.
//
// GB300 design: the key-switching key (50 MB padded) is the only large
// operand, and the work is 3/4 x 8192 row subtractions of 512 words per
// gate.  Two kernels, picked per level width by the autotuner:
//  * k_keyswitch_tiled (default): a CTA owns 64 gates x one 256-word half
//    row x a range of j.  Warp 0 streams the 24 key-row halves of each j
//    (8 digits x 3 non-zero values, 24 KB) into a 2-stage shared-memory
//    ring with bulk asynchronous copies (cp.async.bulk, mbarrier
//    completion); the CTA adds them into the 9 sums of each digit pair
//    (q, q + 1), and every warp keeps 8 gates x 8 words of accumulators in
//    registers and subtracts one row per digit pair, chosen through a
//    table by the pair's 4-bit value (no data-dependent branch).  One key
//    read from L2 serves 64 gates; shared-memory bandwidth bounds the
//    kernel.  Partial sums of a j-split are added into the output with
//    coalesced 32-bit reductions (addition mod 2^32 is associative: the
//    result is bit-identical to a sequential sum).
//  * k_keyswitch: 16 gates per CTA, key rows read straight through L1, the
//    j-range split up to 32 ways (the autotuner's other candidate).
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
    long spin;                // tiled kernel: tries of one bounded mbarrier wait
    int stall;                // tiled kernel, test hook: every stage's wait also waits
                              // on a barrier that nothing completes, so it runs out
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

// ---------------------------------------------------------------------
// Tiled key switch: key-row halves staged in shared memory by bulk copies
// ---------------------------------------------------------------------

constexpr int kKtWarps = 8;                          // warps per CTA
constexpr int kKtGpw = 8;                            // gates per warp
constexpr int kKtTile = kKtWarps * kKtGpw;           // 64 gates per CTA
constexpr int kKtCols = 256;                         // words of a row per CTA (one half)
constexpr int kKtVecs = kKtCols / 4;                 // uint4 per row half
constexpr int kKtRows = kKsT * kKsDigits;            // 24 key-row halves per j
constexpr int kKtPairs = kKsT / 2;                   // digit pairs (q, q + 1) per j
constexpr int kKtCombos = kKsDigits * kKsDigits;     // both digits non-zero: 9 sums per pair
constexpr int kKtStages = 2;                         // shared-memory ring depth
constexpr uint32_t kKtStageBytes = kKtRows * kKtCols * 4;   // 24 KB
constexpr int kKtWin = 128;                          // j values of rounded a'_j held at once
constexpr int kKtWStride = kKtTile + 8;              // uint16 per window row (padded)
constexpr int kKtMaxChunks = 128;
constexpr long kKtSpin = 1L << 20;                   // bounded mbarrier wait: tries of at
constexpr uint32_t kKtTryNs = 1000;                  // most ~1 us each (about a second)
constexpr long kKtStallSpin = 1L << 10;              // ... under the stall test hook

// raw, combo and zero are contiguous: row offsets below count uint4 from raw.
struct KtSmem {
    uint4 raw[kKtStages][kKtRows][kKtVecs];          // 48 KB ring: KSK[j][q][d] halves
    uint4 combo[kKtPairs][kKtCombos][kKtVecs];       // 36 KB: KSK[j][2p][d1] + KSK[j][2p+1][d2]
    uint4 zero[kKtVecs];                             // 1 KB of zeros (digit pair 00)
    uint16_t w[kKtWin][kKtWStride];                  // rounded a'_j [j][gate] (18 KB)
    unsigned long long full[kKtStages];              // mbarriers: stage landed
    unsigned long long never;                        // test hook: never completes
    int abort;                                       // a wait ran out: stop
    uint32_t abort_it;                               // ... at this stage
};
static_assert(sizeof(uint4) * (kKtStages * kKtRows + kKtPairs * kKtCombos) * kKtVecs >=
                  sizeof(uint32_t) * kKtTile * kKtCols,
              "partial sums must fit in the raw ring and the combination rows");

// Row (in uint4 from KtSmem::raw) that digit pair value 4 d1 + d2 of pair p
// selects in ring slot `slot`: zeros, KSK[2p][d1] (d2 = 0), KSK[2p+1][d2]
// (d1 = 0) or the built sum.  A fixed table in the constant bank: the
// warp-uniform lookups go through the constant cache, not shared memory.
struct KtOffsets {
    uint32_t v[kKtStages][kKtPairs][16];
};

constexpr KtOffsets make_kt_offsets()
{
    KtOffsets T{};
    for (int slot = 0; slot < kKtStages; ++slot)
        for (int p = 0; p < kKtPairs; ++p)
            for (int idx = 0; idx < 16; ++idx) {
                const int d1 = idx >> 2, d2 = idx & 3;
                int r = 0;
                if (idx == 0)
                    r = kKtStages * kKtRows + kKtPairs * kKtCombos;
                else if (d2 == 0)
                    r = slot * kKtRows + (2 * p) * kKsDigits + d1 - 1;
                else if (d1 == 0)
                    r = slot * kKtRows + (2 * p + 1) * kKsDigits + d2 - 1;
                else
                    r = kKtStages * kKtRows + p * kKtCombos + (d1 - 1) * kKsDigits + d2 - 1;
                T.v[slot][p][idx] = (uint32_t)(r * kKtVecs);
            }
    return T;
}

__constant__ KtOffsets c_kt_off = make_kt_offsets();

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bounded wait on phase `parity` of an mbarrier: the thread is
// suspended until the phase completes or about kKtTryNs pass.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity), "r"(kKtTryNs)
                 : "memory");
    return ok != 0;
}

// Waits for phase `parity`, giving up after `spin` suspended tries
// (kKtSpin: about a second, far beyond any copy's latency); returns whether
// the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity,
                                                  long spin)
{
    for (long i = 0; i < spin; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) completing on an mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void red_add(int32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void sub4(uint4 &a, const uint4 &b)
{
    a.x -= b.x;
    a.y -= b.y;
    a.z -= b.z;
    a.w -= b.w;
}

// Warp 0 queues the 24 key-row halves of j into ring slot `slot`: lane 0
// posts the byte count, then lanes 0..23 issue one 1 KB copy each.
__device__ __forceinline__ void kt_issue(const KsArgs &A, KtSmem &S, int slot, int j, int half,
                                         int lane)
{
    if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&S.full[slot], kKtStageBytes);
    }
    __syncwarp();
    if (lane < kKtRows) {
        const uint4 *src = A.ksk + ((long)j * kKtRows + lane) * (kLweStride / 4) + half * kKtVecs;
        bulk_g2s(&S.raw[slot][lane][0], src, kKtCols * 4, &S.full[slot]);
    }
}

// grid: (j-chunks, 2 row halves, tiles of 64 gates).  A.atomic: add the
// partial sums into rows that k_ks_init prepared (j-split), else write
// (0, b') - sum directly.
//
// Per j the 8 digits of a gate form 4 pairs (q, q + 1); pair value
// 4 d1 + d2 selects one row: zeros, a single key row (one digit zero) or one
// of the 9 sums built for the stage.  So a gate subtracts 4 rows per j
// instead of up to 8, with no data-dependent branch: the digit pair indexes
// a table of row offsets, and the same instructions run for every gate.
__global__ void __launch_bounds__(32 * kKtWarps, 2) k_keyswitch_tiled(const KsArgs A)
{
    extern __shared__ __align__(128) uint8_t kt_raw[];
    KtSmem &S = *reinterpret_cast<KtSmem *>(kt_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunks = gridDim.x, chunk = blockIdx.x, half = blockIdx.y;
    const int ja = (int)((long)chunk * kN / chunks), jb = (int)((long)(chunk + 1) * kN / chunks);
    const int nj = jb - ja;
    const long tiles = (A.count + kKtTile - 1) / kKtTile;
    const uint4 *rows = &S.raw[0][0][0];

    if (tid == 0) {
        for (int s = 0; s < kKtStages; ++s)
            mbar_init(&S.full[s], 1);
        mbar_init(&S.never, 1);   // no thread ever arrives on it
        S.abort = 0;
        S.abort_it = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < kKtVecs)
        S.zero[tid] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    uint32_t it = 0;       // stages consumed so far (slot = it % kKtStages)
    uint32_t issued = 0;   // stages issued (counted in warp 0)
    for (long tile = blockIdx.z; tile < tiles; tile += gridDim.z) {
        const long g0 = tile * kKtTile;
        if (warp == 0 && !S.abort)
            for (int k = 0; k < kKtStages && k < nj; ++k) {
                kt_issue(A, S, (it + k) % kKtStages, ja + k, half, lane);
                ++issued;
            }

        uint4 acc[kKtGpw][2];
#pragma unroll
        for (int gi = 0; gi < kKtGpw; ++gi)
            acc[gi][0] = acc[gi][1] = make_uint4(0u, 0u, 0u, 0u);

        for (int k = 0; k < nj; ++k) {
            const int kw = k % kKtWin;
            if (kw == 0) {
                // rounded a'_j of the next window: consecutive threads read
                // consecutive j of one gate (coalesced)
                const int nw = min(kKtWin, nj - k);
                for (int e = tid; e < nw * kKtTile; e += 32 * kKtWarps) {
                    const int gg = e / nw, jj = e % nw;
                    uint32_t w = 0;
                    if (g0 + gg < A.count) {
                        const uint32_t a = (uint32_t)A.big[(g0 + gg) * kBigStride + ja + k + jj];
                        w = ((a + (1u << 15)) >> 16) & 0xFFFFu;   // round to 16 bits
                    }
                    S.w[jj][gg] = (uint16_t)w;
                }
                __syncthreads();
            }
            const int slot = it % kKtStages;
            if (!S.abort && (!mbar_wait_bounded(&S.full[slot], (it / kKtStages) & 1u, A.spin) ||
                             (A.stall && !mbar_wait_bounded(&S.never, 0u, A.spin)))) {
                S.abort_it = it;   // the same value in every thread that gets here
                S.abort = 1;
                atomicOr(A.status, kErrTimeout);
            }
            // the 9 sums of each digit pair: thread (p, v) builds column v
            if (!S.abort) {
                const int p = tid / kKtVecs, v = tid % kKtVecs;
                const uint4 *ra = &S.raw[slot][(2 * p) * kKsDigits][0];
                const uint4 *rb = ra + kKsDigits * kKtVecs;
                const uint4 b1 = rb[v], b2 = rb[kKtVecs + v], b3 = rb[2 * kKtVecs + v];
#pragma unroll 1
                for (int x = 0; x < kKsDigits; ++x) {
                    const uint4 a = ra[x * kKtVecs + v];
                    uint4 *c = &S.combo[p][x * kKsDigits][v];
                    c[0] = make_uint4(a.x + b1.x, a.y + b1.y, a.z + b1.z, a.w + b1.w);
                    c[kKtVecs] = make_uint4(a.x + b2.x, a.y + b2.y, a.z + b2.z, a.w + b2.w);
                    c[2 * kKtVecs] = make_uint4(a.x + b3.x, a.y + b3.y, a.z + b3.z, a.w + b3.w);
                }
            }
            __syncthreads();
            if (!S.abort) {
                const uint4 wq = *reinterpret_cast<const uint4 *>(&S.w[kw][warp * kKtGpw]);
                const uint32_t wv[4] = {wq.x, wq.y, wq.z, wq.w};
                const uint32_t *off = &c_kt_off.v[slot][0][0];
#pragma unroll 1
                for (int p = 0; p < kKtPairs; ++p)
#pragma unroll
                    for (int gi = 0; gi < kKtGpw; ++gi) {
                        const uint32_t idx = (wv[gi >> 1] >> ((gi & 1) * 16 + 12 - 4 * p)) & 15u;
                        const uint4 *r = rows + off[p * 16 + idx];
                        sub4(acc[gi][0], r[lane]);
                        sub4(acc[gi][1], r[32 + lane]);
                    }
            }
            __syncthreads();   // every warp is done with the slot and the sums
            if (warp == 0 && k + kKtStages < nj && !S.abort) {
                kt_issue(A, S, slot, ja + k + kKtStages, half, lane);
                ++issued;
            }
            ++it;
        }

        // lane owns words 4 lane .. 4 lane + 3 and 128 + 4 lane .. of the half
        if (!A.atomic) {
#pragma unroll
            for (int gi = 0; gi < kKtGpw; ++gi) {
                const long g = g0 + warp * kKtGpw + gi;
                if (g >= A.count)
                    break;
                const long dst = ks_dest(A, g);
                if (dst < 0 || dst >= A.rows_out) {
                    if (lane == 0 && half == 0)
                        atomicOr(A.status, kErrScatter);
                    continue;
                }
                const uint32_t bprime = (uint32_t)A.big[g * kBigStride + kN];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = half * kKtCols + h * 128 + 4 * lane;
                    uint4 v = acc[gi][h];   // already minus the row sum
                    if (c0 + 0 == A.n) v.x += bprime;
                    if (c0 + 1 == A.n) v.y += bprime;
                    if (c0 + 2 == A.n) v.z += bprime;
                    if (c0 + 3 == A.n) v.w += bprime;
                    *reinterpret_cast<uint4 *>(A.out + dst * kLweStride + c0) = v;
                }
            }
        } else {
            // transpose through the (idle) ring so that each reduction
            // instruction of a warp covers 32 consecutive words
            uint32_t *P = reinterpret_cast<uint32_t *>(&S.raw[0][0][0]);
#pragma unroll
            for (int gi = 0; gi < kKtGpw; ++gi) {
                uint32_t *row = P + (warp * kKtGpw + gi) * kKtCols;
                *reinterpret_cast<uint4 *>(row + 4 * lane) = acc[gi][0];
                *reinterpret_cast<uint4 *>(row + 128 + 4 * lane) = acc[gi][1];
            }
            __syncwarp();
            for (int gi = 0; gi < kKtGpw; ++gi) {
                const long g = g0 + warp * kKtGpw + gi;
                if (g >= A.count)
                    break;
                const long dst = ks_dest(A, g);
                if (dst < 0 || dst >= A.rows_out)
                    continue;   // flagged by k_ks_init
                const uint32_t *row = P + (warp * kKtGpw + gi) * kKtCols;
                int32_t *o = A.out + dst * kLweStride + half * kKtCols;
#pragma unroll
                for (int c = 0; c < kKtCols / 32; ++c)
                    red_add(o + 32 * c + lane, row[32 * c + lane]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();   // the ring is free for the next tile's copies
    }
    // after a timed-out wait: give the stages issued but never waited for a
    // bounded time to land before the CTA's shared memory is released (their
    // barriers count only the real copies' bytes, so under the test hook
    // these waits end as soon as the copies have landed)
    if (warp == 0 && lane == 0 && S.abort)
        for (uint32_t p = S.abort_it; p < issued; ++p)
            (void)mbar_wait_bounded(&S.full[p % kKtStages], (p / kKtStages) & 1u, A.spin);
}

// ---------------------------------------------------------------------
// Launch
// ---------------------------------------------------------------------

// Set while the autotuner measures, for the launches of its own thread
// only (other threads' contexts keep their choices).
static thread_local int ks_forced_chunks = 0;

// Launch choice: kKsTiled selects the tiled kernel, 1..32 the j-chunks of
// k_keyswitch.  A forced choice (autotuner, TFHE_OPT_KS_KERNEL) wins, then
// the tuned value for the width bucket; untuned, the tiled kernel (on
// GB300 it is the faster one from 1 to 10^4 gates).
static int ks_chunks(long count, int num_sms, const DevKeys *choice)
{
    if (ks_forced_chunks)
        return ks_forced_chunks;
    if (choice && choice->ks_kernel > 0)
        return choice->ks_kernel;
    if (choice && choice->tune_ks[tune_bucket(count)] > 0)
        return choice->tune_ks[tune_bucket(count)];
    (void)count;
    (void)num_sms;
    return kKsTiled;
}

// j-chunks of the tiled kernel: enough CTAs for two per SM (16 warps).
static int kt_chunks(long count, int num_sms)
{
    const long tiles = (count + kKtTile - 1) / kKtTile;
    long c = 2L * num_sms / (2 * tiles);
    return (int)(c < 1 ? 1 : c > kKtMaxChunks ? kKtMaxChunks : c);
}

void keyswitch_force_chunks(int chunks) { ks_forced_chunks = chunks; }

// Kernels one launch_keyswitch call issues.
int keyswitch_kernels(long count, int num_sms, const DevKeys *choice)
{
    if (count <= 0)
        return 0;
    const int c = ks_chunks(count, num_sms, choice);
    if (c == kKsTiled)
        return kt_chunks(count, num_sms) > 1 ? 2 : 1;
    return c > 1 ? 2 : 1;
}

cudaError_t launch_keyswitch(const uint4 *ksk, const int32_t *big, int32_t *out,
                             const int32_t *idx_out, long rows_out, long count, int n,
                             int num_sms, uint32_t *status, cudaStream_t stream,
                             const DevKeys *choice)
{
    if (count <= 0)
        return cudaSuccess;
    const int pick = ks_chunks(count, num_sms, choice);
    const bool tiled = pick == kKsTiled;
    const int chunks = tiled ? kt_chunks(count, num_sms) : pick;
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
    const bool stall = tiled && choice && choice->ks_stall;
    A.spin = stall ? kKtStallSpin : kKtSpin;
    A.stall = stall ? 1 : 0;
    if (A.atomic) {
        k_ks_init<<<(unsigned)count, 128, 0, stream>>>(A);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    if (tiled) {
        static int prepared[64] = {0};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !prepared[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_keyswitch_tiled,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sizeof(KtSmem));
            if (e != cudaSuccess)
                return e;
            prepared[dev] = 1;
        }
        const long tiles = (count + kKtTile - 1) / kKtTile;
        dim3 grid((unsigned)chunks, 2u, (unsigned)(tiles < 65535 ? tiles : 65535));
        k_keyswitch_tiled<<<grid, 32 * kKtWarps, sizeof(KtSmem), stream>>>(A);
        return cudaGetLastError();
    }
    const long tiles = (count + kKsGates - 1) / kKsGates;
    dim3 grid((unsigned)tiles, (unsigned)chunks);
    k_keyswitch<<<grid, kKsThreads, 0, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace tgb
