// common.cuh -- shared definitions of the sm_103a TFHE kernels.
//
// Ring and gadget shape are compile-time: N = 1024, k = 1, l = 2,
// Bg = 2^10, key switch t = 8, base 4.  The LWE dimension n is a runtime
// value (n <= 511).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tfhe_gb.h"

namespace tgb {

constexpr int kN = 1024;                 // TLWE ring degree
constexpr int kL = 2;                    // gadget levels
constexpr int kRows = 2 * kL;            // rows of a TGSW sample (k = 1)
constexpr int kBgBit = 10;               // log2 Bg
constexpr int kKsT = 8;                  // key-switch levels
constexpr int kKsBaseBit = 2;            // log2 key-switch base
constexpr int kKsDigits = (1 << kKsBaseBit) - 1;
constexpr int kLweStride = TFHE_LWE_STRIDE;
constexpr int kBigStride = TFHE_BIG_STRIDE;
constexpr int kMaxN = kLweStride - 1;
constexpr uint32_t kMu = 1u << 29;       // 1/8

// Word offset that turns signed gadget digits into unsigned bit fields:
// 1/2 Bg per level plus the rounding half of the last level.
constexpr uint32_t kDecompOffset = (1u << 31) + (1u << 21) + (1u << 11);

// Two NTT primes below 2^27 with 2048 | q - 1.  Their product P ~ 2^54
// exceeds twice the largest magnitude of an exact external-product
// coefficient, 4 * N * 2^9 * 2^31 = 2^52, so the centred CRT lift is the
// exact integer.  q < 2^27 keeps every lazy value below 32 q < 2^32 and the
// 4-term pointwise sum of [0,8q) x [0,q) products below q * 2^32.
constexpr uint32_t kQ0 = 134215681u;     // 0x07FFF801
constexpr uint32_t kQ1 = 134203393u;     // 0x07FFC801
static_assert(32ull * kQ0 < (1ull << 32) && 32ull * kQ1 < (1ull << 32), "lazy bound");
static_assert((kQ0 - 1) % 2048 == 0 && (kQ1 - 1) % 2048 == 0, "2N-th roots of unity");
static_assert((unsigned __int128)kQ0 * kQ1 > ((unsigned __int128)1 << 53), "centred CRT lift");

// Status word bits (device-side errors).
constexpr uint32_t kErrGather = 1u;
constexpr uint32_t kErrScatter = 2u;
constexpr uint32_t kErrTimeout = 4u;
constexpr uint32_t kErrOpcode = 8u;

#if defined(__CUDACC__)
// x * w mod q in [0, 2q) for any 32-bit x, with wp = floor(w 2^32 / q)
// (Shoup's precomputed-quotient multiplication).
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t wp, uint32_t q)
{
    return x * w - __umulhi(x, wp) * q;
}

// x in [0, 2m) -> [0, m): subtract m when x >= m (unsigned min trick).
__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m)
{
    return min(x, x - m);
}

// Montgomery reduction of a 64-bit x = hi 2^32 + lo < q 2^32: with
// m = lo q^-1 mod 2^32, m q has low word lo, so x - m q = (hi - mulhi(m, q))
// 2^32 exactly; the result hi - mulhi(m, q) + q = x 2^-32 mod q lies in
// (0, 2q).  q_inv = q^-1 mod 2^32.
__device__ __forceinline__ uint32_t mont_reduce(uint64_t x, uint32_t q, uint32_t q_inv)
{
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return hi - __umulhi(lo * q_inv, q) + q;
}
#endif  // __CUDACC__

// Per-context device pointers and sizes shared by the kernels.
// Blind-rotation CTA shape codes: one bootstrap spread over 8 warps, and
// one bootstrap on a cluster of two CTAs (one prime each).  The other
// codes, 1, 2 and 4, count 4-warp bootstraps per CTA.
constexpr int kBrSplit = 8;
constexpr int kBrPair = 16;
// Two 4-warp bootstraps per CTA with the CMux step's key staged in shared
// memory by bulk copies (one CTA per SM), and, for measuring that choice,
// the same shape reading the key through L1 at the same occupancy.
constexpr int kBrStaged = 32;
constexpr int kBrStagedCtl = 33;
// One bootstrap on 8 warps with the key staged (the latency shape, whose
// single pointwise warp per sub-partition otherwise waits on L2 each step).
constexpr int kBrSplitStaged = 40;
// One bootstrap on a two-CTA cluster with each CTA's half of the key staged.
constexpr int kBrPairStaged = 48;
// One bootstrap per 4-warp CTA compiled for five CTAs per SM (96 registers,
// 20 warps): one wave is 5 bootstraps per SM, for schedules whose levels
// fill such waves.
constexpr int kBrFive = 5;
// Key-switch launch code for the tiled kernel (shared-memory key stages);
// the codes 1 .. 32 are j-chunks of the direct kernel.
constexpr int kKsTiled = 64;

struct DevKeys {
    const uint4 *bk_ntt;   // [n][2 poly][2 prime][32 reg][32 lane] x uint4(4 rows)
    const uint4 *ksk;      // [N][t][base-1][kLweStride/4] words
    const uint2 *twb;      // stage-B twiddles [2 prime][2 dir][32 reg][32 lane] (w, w')
    int n;
    int br_group;          // blind-rotation CTA shape: 1, 2, 4 bootstraps per CTA,
                           // kBrSplit = one bootstrap on 8 warps, kBrPair = one
                           // bootstrap on two CTAs, 0 = tuned or by batch size
    int ks_kernel;         // key-switch kernel: kKsTiled, j-chunks 1 .. 32 of the
                           // direct kernel, 0 = tuned or by batch size
    int ks_stall;          // test hook (TFHE_OPT_TEST_KS_STALL): the tiled key
                           // switch's copy waits run out
    // Autotuned launch shapes per level-width bucket (0 = not tuned): bucket b
    // covers widths up to kTuneEdge[b] (the last bucket is unbounded).
    int8_t tune_br[8];     // bootstraps per blind-rotation CTA
    int8_t tune_ks[8];     // key-switch kernel: kKsTiled, or j-chunks 1 .. 32
    // Autotuned time (ms) of one full blind-rotation wave: [0] 4 bootstraps
    // per SM (the tuned shape), [1] 5 per SM (kBrFive); 0 = not measured.
    float wave_ms[2];
    // Autotuned time (ms) of a level at each bucket's widest width with the
    // bucket's chosen shape; 0 = not measured.
    float tune_ms[8];
};

constexpr long kTuneEdge[8] = {152, 304, 608, 1216, 2432, 4864, 9728, 1L << 40};

inline int tune_bucket(long count)
{
    int b = 0;
    while (b < 7 && count > kTuneEdge[b])
        ++b;
    return b;
}

}  // namespace tgb
