// bootstrap.cu -- blind rotation (n CMux external products), fused with the
// gate combine, mod switch, test-vector rotation and sample extraction.
//
// The method: TFHE gate bootstrapping as adopted by the paper (section II-A;
// bootstrapping and key switching are timed separately in Table
// "differentialtime").  For every gate the accumulator starts as
// (0, X^-bbar v), v = mu (1 + X + ... + X^(N-1)), and for i < n becomes
// acc + BK_i [x] (X^abar_i acc - acc), where [x] decomposes the two
// polynomials of the TLWE sample into l = 2 signed base-2^10 digit
// polynomials each and sums digit_r * BK_i[r] in Z[X]/(X^N + 1) mod 2^32.
//
// GB300 design (not the paper's: it used cuFFT in floating point):
//  * the products are exact: a negacyclic NTT modulo two primes below 2^27
//    and a centred CRT lift back to Z/2^32;
//  * one group of 4 warps owns one bootstrap; a CTA runs B in {1, 2, 4}
//    bootstraps in lockstep (4B warps) and loops over gate groups
//    (persistent grid); the accumulators never leave shared memory.  For
//    narrow levels one bootstrap can instead take 8 warps, or a cluster of
//    two CTAs (one prime each), and the key of the next CMux step can be
//    staged in shared memory by bulk copies;
//  * warp (c, h) of a bootstrap works modulo prime h for the whole CMux:
//    it forms both digit polynomials of TLWE polynomial c (one rotation)
//    and transforms them; then, as warp (p, h), it does the pointwise
//    products with BK_i for output polynomial p, the inverse transform and
//    half of the CRT + accumulate;
//  * one 1024-point transform is one warp: 32 coefficients per lane,
//    a 32-point transform in registers, a twiddle, one shared-memory
//    transpose, and a second 32-point transform (four-step NTT);
//  * code size is the binding constraint on instruction fetch: each
//    transform exists once (the prime is a runtime value), and the warps of
//    a CTA execute the same phase at the same time;
//  * the bootstrapping key is pre-transformed, scaled by 2^32 N^-1 and
//    interleaved so that lane l reads its 4 rows for one register as one
//    16-byte load; the 33 MB key stays L2-resident across gates, and the B
//    bootstraps of a CTA read each key row once through L1.
#include <cstdio>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace tgb {

// Shared-memory slots of 33 x 32 words: a transpose written as
// slot[i * 33 + lane] and read as slot[lane * 33 + j] is conflict-free with
// register + immediate addresses (no per-element address arithmetic).
constexpr int kSlot = 33 * 32;

struct NttConst {
    uint32_t za[2][32][2];   // forward stage A: w64^brv5(k), Shoup companion
    uint32_t zd[2][32][2];   // forward stage D: cyclic size-32 twiddles
    uint32_t iza[2][32][2];  // inverse of stage A
    uint32_t izd[2][32][2];  // inverse of stage D
    uint32_t q_inv[2];       // q^-1 mod 2^32
    uint32_t crt_c, crt_cp;  // q0^-1 mod q1 and its Shoup companion mod q1
    uint32_t p_lo, pad;      // (q0 q1) mod 2^32
    uint64_t p_half;         // (q0 q1 + 1) / 2
    uint32_t bk_scale[2][2]; // 2^32 N^-1 mod q and companion
};

__constant__ NttConst c_ntt;

__host__ __device__ constexpr int brv5(int k)
{
    return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

// The transforms take the prime as a runtime value (one of two) so that a
// single copy of each transform serves both primes; twiddles are read from
// the constant bank with an offset on the prime.
struct Prime {
    uint32_t q, q2, P;
    __device__ __forceinline__ explicit Prime(uint32_t p)
        : q(p ? kQ1 : kQ0), q2(2 * (p ? kQ1 : kQ0)), P(p) {}
    // K q for K in {1, 2, 4, 8, 16, 32} (32 q < 2^32 for both primes)
    __device__ __forceinline__ uint32_t kq(int K) const
    {
        return K == 1 ? q : K == 2 ? q2 : K == 4 ? q2 << 1 : K == 8 ? q2 << 2
             : K == 16 ? q2 << 3 : q2 << 4;
    }
};

// ---------------------------------------------------------------------
// Lazy reductions.  Values are kept in [0, b q) with a per-element bound b
// known at compile time; a reduction csub(x, K q) (valid for b <= 2K)
// leaves [0, K q).  LazyPlan walks the 80 butterflies of a 32-point pass
// in the same order as the code and places the fewest reductions that keep
// every sum below thr q (<= kLazyMax q < 2^32), and the final outputs below
// fin q:
//  * CT butterfly (u, v) -> (u + t, u - t + K' q), t = v (trivial twiddle)
//    or Shoup(v) in [0, 2q), K' >= bound(t) the smallest power of two;
//  * GS butterfly (u, v) -> (u + v, d), d = u - v + K' q (K' >= bound(v)),
//    passed on as is (trivial twiddle) or as Shoup(d) in [0, 2q).
// The reduction is applied to the larger operand until the sum fits.
// ---------------------------------------------------------------------
struct LazyStep {
    uint8_t ru[4], nru;     // csub multiples K applied to u, in order
    uint8_t rv[4], nrv;     // ... to v (t of a trivial CT butterfly)
    uint8_t off;            // K' of the difference
};
struct LazyPlan {
    LazyStep st[5][16];     // [level][butterfly g * ln + jj]
    uint8_t fin[32][4], nfin[32];
    int reductions;
    bool ok;
};

constexpr int kLazyMax = 32;   // every lazy value stays below 32 q < 2^32

__host__ __device__ constexpr int lazy_off(int b)
{
    return b <= 1 ? 1 : b <= 2 ? 2 : b <= 4 ? 4 : b <= 8 ? 8 : b <= 16 ? 16 : 32;
}

// One reduction step of a value with bound b: the smallest K in
// {1, 2, 4, 8, 16} with 2K >= b; returns the new bound (or b if none
// applies).
__host__ __device__ constexpr int lazy_step(int b, int &K)
{
    K = b <= 2 ? 1 : b <= 4 ? 2 : b <= 8 ? 4 : b <= 16 ? 8 : b <= 32 ? 16 : 0;
    if (K == 0 || K >= b)
        return b;
    return K > b - K ? K : b - K;
}

__host__ __device__ constexpr LazyPlan make_lazy_plan(bool ct, bool trivial_first, int in_b, int thr, int fin)
{
    LazyPlan P{};
    P.ok = true;
    int b[32] = {};
    for (int i = 0; i < 32; ++i)
        b[i] = in_b;
    for (int it = 0; it < 5; ++it) {
        const int s = ct ? it : 4 - it;
        const int m = 1 << s, ln = 16 >> s;
        for (int g = 0; g < m; ++g) {
            const bool triv = trivial_first && g == 0;
            for (int jj = 0; jj < ln; ++jj) {
                const int j = 2 * g * ln + jj;
                LazyStep &L = P.st[s][g * ln + jj];
                int bu = b[j], bv = b[j + ln];
                for (int guard = 0; guard < 8; ++guard) {
                    const int bt = (ct && !triv) ? 2 : bv;
                    if (bu + bt <= thr && bu + lazy_off(bt) <= kLazyMax)
                        break;
                    int K = 0;
                    if ((!ct || triv) && bt >= bu) {
                        const int nb = lazy_step(bv, K);
                        if (nb == bv || L.nrv == 4) { P.ok = false; break; }
                        L.rv[L.nrv++] = (uint8_t)K;
                        bv = nb;
                    } else {
                        const int nb = lazy_step(bu, K);
                        if (nb == bu || L.nru == 4) { P.ok = false; break; }
                        L.ru[L.nru++] = (uint8_t)K;
                        bu = nb;
                    }
                }
                const int bt = (ct && !triv) ? 2 : bv;
                L.off = (uint8_t)lazy_off(bt);
                P.reductions += L.nru + L.nrv;
                if (ct) {
                    b[j] = bu + bt;
                    b[j + ln] = bu + L.off;
                } else {
                    b[j] = bu + bv;
                    b[j + ln] = triv ? bu + L.off : 2;
                }
                if (b[j] > kLazyMax || b[j + ln] > kLazyMax)
                    P.ok = false;
            }
        }
    }
    for (int i = 0; i < 32; ++i) {
        while (b[i] > fin) {
            int K = 0;
            const int nb = lazy_step(b[i], K);
            if (nb == b[i] || P.nfin[i] == 4) { P.ok = false; break; }
            P.fin[i][P.nfin[i]++] = (uint8_t)K;
            b[i] = nb;
        }
        P.reductions += P.nfin[i];
    }
    return P;
}

// Forward passes: stage A (negacyclic twiddles, inputs [0, 2q), outputs
// < 12q, no reduction needed) and stage D (cyclic, the first twiddle of
// every level is 1; inputs [0, 2q), outputs [0, 8q) for the pointwise
// products).  Inverse passes: stage D' (cyclic GS, inputs [0, 2q) from the
// pointwise Montgomery step, outputs < 32q into the Shoup twiddle) and
// stage A' (negacyclic GS, inputs [0, 2q), outputs [0, 2q)).  The
// thresholds are the ones that need the fewest reductions.
constexpr LazyPlan kPlanFwdA = make_lazy_plan(true, false, 2, 12, kLazyMax);
constexpr LazyPlan kPlanFwdD = make_lazy_plan(true, true, 2, 8, 8);
constexpr LazyPlan kPlanInvD = make_lazy_plan(false, true, 2, kLazyMax, kLazyMax);
constexpr LazyPlan kPlanInvA = make_lazy_plan(false, false, 2, kLazyMax, 2);
static_assert(kPlanFwdA.ok && kPlanFwdD.ok && kPlanInvD.ok && kPlanInvA.ok, "lazy plan");
static_assert(kPlanFwdA.reductions == 0 && kPlanFwdD.reductions == 33 &&
              kPlanInvD.reductions == 4 && kPlanInvA.reductions == 32, "lazy plan size");

__device__ __forceinline__ uint32_t lazy_reduce_n(uint32_t x, const uint8_t (&ks)[4], int n,
                                                  const Prime &pr)
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < n)
            x = csub(x, pr.kq(ks[k]));
    return x;
}

// 32-point Cooley-Tukey pass in registers (CYC false: stage A, negacyclic
// twiddles; CYC true: stage D, cyclic twiddles), reductions by plan.
template <bool CYC>
__device__ __forceinline__ void ct32(uint32_t (&x)[32], const Prime &pr)
{
    constexpr LazyPlan PL = CYC ? kPlanFwdD : kPlanFwdA;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int m = 1 << s, ln = 16 >> s;
#pragma unroll
        for (int g = 0; g < m; ++g) {
            const uint32_t(*tb)[32][2] = CYC ? c_ntt.zd : c_ntt.za;
            const uint32_t w = tb[pr.P][m + g][0];
            const uint32_t wp = tb[pr.P][m + g][1];
#pragma unroll
            for (int jj = 0; jj < ln; ++jj) {
                const int j = 2 * g * ln + jj;
                const LazyStep &L = PL.st[s][g * ln + jj];
                const uint32_t u = lazy_reduce_n(x[j], L.ru, L.nru, pr);
                const uint32_t t = (CYC && g == 0) ? lazy_reduce_n(x[j + ln], L.rv, L.nrv, pr)
                                                   : mul_shoup(x[j + ln], w, wp, pr.q);
                x[j] = u + t;
                x[j + ln] = u - t + pr.kq(L.off);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
        x[r] = lazy_reduce_n(x[r], PL.fin[r], PL.nfin[r], pr);
}

// Inverse (Gentleman-Sande) of ct32, reductions by plan; the result is 32
// times the inverse transform.
template <bool CYC>
__device__ __forceinline__ void gs32(uint32_t (&x)[32], const Prime &pr)
{
    constexpr LazyPlan PL = CYC ? kPlanInvD : kPlanInvA;
#pragma unroll
    for (int s = 4; s >= 0; --s) {
        const int m = 1 << s, ln = 16 >> s;
#pragma unroll
        for (int g = 0; g < m; ++g) {
            const uint32_t(*tb)[32][2] = CYC ? c_ntt.izd : c_ntt.iza;
            const uint32_t w = tb[pr.P][m + g][0];
            const uint32_t wp = tb[pr.P][m + g][1];
#pragma unroll
            for (int jj = 0; jj < ln; ++jj) {
                const int j = 2 * g * ln + jj;
                const LazyStep &L = PL.st[s][g * ln + jj];
                const uint32_t u = lazy_reduce_n(x[j], L.ru, L.nru, pr);
                const uint32_t v = lazy_reduce_n(x[j + ln], L.rv, L.nrv, pr);
                x[j] = u + v;
                const uint32_t d = u - v + pr.kq(L.off);
                x[j + ln] = (CYC && g == 0) ? d : mul_shoup(d, w, wp, pr.q);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
        x[r] = lazy_reduce_n(x[r], PL.fin[r], PL.nfin[r], pr);
}

// Forward negacyclic NTT of one polynomial held by one warp.
// In : lane l, register r holds coefficient l + 32 r, value in [0, 2q).
// Out: lane l, register r holds the evaluation at psi^(2 (l + 32 brv5(r)) + 1),
//      value in [0, 8q).  sbuf: kSlot words of this warp's shared memory.
__device__ __forceinline__ void fwd_ntt(uint32_t (&x)[32], uint32_t *sbuf, int lane,
                                        const uint2 *__restrict__ twb, const Prime &pr)
{
    ct32<false>(x, pr);
    const uint2 *tw = twb + (pr.P * 2 + 0) * 1024 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {   // any 32-bit input -> [0, 2q)
        const uint2 t = __ldg(tw + r * 32);
        x[r] = mul_shoup(x[r], t.x, t.y, pr.q);
    }
    uint32_t *wr = sbuf + lane, *rd = sbuf + lane * 33;
#pragma unroll
    for (int r = 0; r < 32; ++r)
        wr[brv5(r) * 33] = x[r];       // lane i1, k1 = brv5(r) -> slot[k1][i1]
    __syncwarp();
#pragma unroll
    for (int i1 = 0; i1 < 32; ++i1)
        x[i1] = rd[i1];                // lane k1 reads slot[k1][i1]
    __syncwarp();
    ct32<true>(x, pr);
}

// Inverse of fwd_ntt up to the factor N: input layout of fwd_ntt's output
// with values in [0, 2q); output lane l, register r = N * coefficient
// l + 32 r, in [0, 2q).
__device__ __forceinline__ void inv_ntt(uint32_t (&x)[32], uint32_t *sbuf, int lane, int lane_brv,
                                        const uint2 *__restrict__ twb, const Prime &pr)
{
    gs32<true>(x, pr);
    const uint2 *tw = twb + (pr.P * 2 + 1) * 1024 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint2 t = __ldg(tw + r * 32);
        x[r] = mul_shoup(x[r], t.x, t.y, pr.q);
    }
    uint32_t *wr = sbuf + lane_brv, *rd = sbuf + lane * 33;
#pragma unroll
    for (int r = 0; r < 32; ++r)
        wr[r * 33] = x[r];             // lane k1, i1 = r -> slot[i1][brv5(k1)]
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r)
        x[r] = rd[r];                  // lane i1 reads slot[i1][r]
    __syncwarp();
    gs32<false>(x, pr);
}

// The inverse transform shared by two warps of one sub-partition (the
// 8-warp shapes): warp K holds registers 16K .. 16K + 15 of every lane.  In
// each 32-point Gentleman-Sande pass the butterflies of distance 1 .. 8 stay
// inside a warp's registers; the last stage (distance 16) pairs register j
// with j + 16, so each warp publishes its reduced inputs of that stage in
// `ex` ([32 registers][32 lanes]) and reads its partner's after a barrier
// of the two warps (named barrier `bar`).  Every butterfly, twiddle and
// reduction is the one gs32 / inv_ntt performs, so the result is identical.
__device__ __forceinline__ void pair_sync(int bar)
{
    asm volatile("bar.sync %0, 64;" ::"r"(bar) : "memory");
}

template <bool CYC, int K>
__device__ __forceinline__ void gs32_half(uint32_t (&x)[32], const Prime &pr, uint32_t *ex,
                                          int lane, int bar)
{
    constexpr LazyPlan PL = CYC ? kPlanInvD : kPlanInvA;
    const uint32_t(*tb)[32][2] = CYC ? c_ntt.izd : c_ntt.iza;
#pragma unroll
    for (int s = 4; s >= 1; --s) {
        const int m = 1 << s, ln = 16 >> s;
#pragma unroll
        for (int g = 0; g < m; ++g) {
            const uint32_t w = tb[pr.P][m + g][0];
            const uint32_t wp = tb[pr.P][m + g][1];
#pragma unroll
            for (int jj = 0; jj < ln; ++jj) {
                const int j = 2 * g * ln + jj;
                if ((j >> 4) != K)
                    continue;
                const LazyStep &L = PL.st[s][g * ln + jj];
                const uint32_t u = lazy_reduce_n(x[j], L.ru, L.nru, pr);
                const uint32_t v = lazy_reduce_n(x[j + ln], L.rv, L.nrv, pr);
                x[j] = u + v;
                const uint32_t d = u - v + pr.kq(L.off);
                x[j + ln] = (CYC && g == 0) ? d : mul_shoup(d, w, wp, pr.q);
            }
        }
    }
    // distance 16: warp 0 holds the u, warp 1 the v of every butterfly
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
        const LazyStep &L = PL.st[0][jj];
        const int r = 16 * K + jj;
        x[r] = K == 0 ? lazy_reduce_n(x[r], L.ru, L.nru, pr) : lazy_reduce_n(x[r], L.rv, L.nrv, pr);
        ex[r * 32 + lane] = x[r];
    }
    pair_sync(bar);
    const uint32_t w = tb[pr.P][1][0], wp = tb[pr.P][1][1];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
        const LazyStep &L = PL.st[0][jj];
        const int r = 16 * K + jj;
        const uint32_t other = ex[(16 * (1 - K) + jj) * 32 + lane];
        if (K == 0) {
            x[r] = x[r] + other;
        } else {
            const uint32_t d = other - x[r] + pr.kq(L.off);
            x[r] = CYC ? d : mul_shoup(d, w, wp, pr.q);
        }
        x[r] = lazy_reduce_n(x[r], PL.fin[r], PL.nfin[r], pr);
    }
}

// inv_ntt on two warps (see gs32_half): same input layout restricted to
// registers 16K .. 16K + 15, same output layout and values.  sbuf: the
// pair's transpose scratch (kSlot words).
template <int K>
__device__ __forceinline__ void inv_ntt_half(uint32_t (&x)[32], uint32_t *sbuf, uint32_t *ex,
                                             int lane, int lane_brv,
                                             const uint2 *__restrict__ twb, const Prime &pr,
                                             int bar)
{
    gs32_half<true, K>(x, pr, ex, lane, bar);
    const uint2 *tw = twb + (pr.P * 2 + 1) * 1024 + lane;
#pragma unroll
    for (int r = 16 * K; r < 16 * K + 16; ++r) {
        const uint2 t = __ldg(tw + r * 32);
        x[r] = mul_shoup(x[r], t.x, t.y, pr.q);
    }
    uint32_t *wr = sbuf + lane_brv, *rd = sbuf + lane * 33;
#pragma unroll
    for (int r = 16 * K; r < 16 * K + 16; ++r)
        wr[r * 33] = x[r];             // lane k1, i1 = r -> slot[i1][brv5(k1)]
    pair_sync(bar);
#pragma unroll
    for (int r = 16 * K; r < 16 * K + 16; ++r)
        x[r] = rd[r];                  // lane i1 reads slot[i1][r]
    gs32_half<false, K>(x, pr, ex, lane, bar);
}

// ---------------------------------------------------------------------
// Bootstrapping key -> NTT domain
// ---------------------------------------------------------------------

// One warp per (i, row, poly, prime).  bk: int32 [n][4][2][N] coefficient
// form.  Output element (i, p, q, reg, lane) is a uint4 over the 4 rows.
__global__ void __launch_bounds__(128) k_bk_to_ntt(const int32_t *__restrict__ bk, uint32_t *out,
                                                   int n, const uint2 *__restrict__ twb)
{
    __shared__ uint32_t sbuf[4][kSlot];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long task = (long)blockIdx.x * 4 + warp;  // ((i * 4 + r) * 2 + p) * 2 + q
    if (task >= (long)n * kRows * 2 * 2)
        return;
    const int qsel = task & 1, p = (task >> 1) & 1, r = (task >> 2) & 3;
    const long i = task >> 4;
    const int32_t *src = bk + ((i * kRows + r) * 2 + p) * kN;
    uint32_t x[32];
    const uint32_t q = qsel == 0 ? kQ0 : kQ1;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        int64_t v = src[lane + 32 * k];               // centred representative
        int64_t m = v % (int64_t)q;
        x[k] = (uint32_t)(m < 0 ? m + q : m);
    }
    fwd_ntt(x, sbuf[warp], lane, twb, Prime((uint32_t)qsel));
    const uint32_t sc = c_ntt.bk_scale[qsel][0], scp = c_ntt.bk_scale[qsel][1];
    // element index in uint32 words: ((((i*2+p)*2+q)*32 + reg)*32 + lane)*4 + r
    uint32_t *dst = out + ((((i * 2 + p) * 2 + qsel) * 32) * 32 + lane) * 4 + r;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        uint32_t v = x[k] % q;                         // [0, 8q) -> [0, q)
        v = csub(mul_shoup(v, sc, scp, q), q);        // * 2^32 N^-1, in [0, q)
        dst[k * 32 * 4] = v;
    }
}

// ---------------------------------------------------------------------
// Blind rotation
// ---------------------------------------------------------------------

struct BrArgs {
    DevKeys keys;
    const int32_t *in_a, *in_b, *in_c;    // ciphertext bases (row stride kLweStride)
    const int32_t *idx_a, *idx_b, *idx_c; // optional gather rows (nullptr: row g)
    long rows_a, rows_b, rows_c;          // rows addressable through the bases
    const uint8_t *ops;              // gate opcodes (nullptr: bootstrap in_a as is)
    int32_t *big;                    // out: LWE_N samples [count][kBigStride]
    long count;
    uint32_t mu;                     // test-vector amplitude
    uint32_t *status;
};

struct BrSmem {                 // one bootstrap
    uint32_t acc[2][kN];        // TLWE accumulator (a(X), b(X))
    uint32_t fwd[4][2][kSlot];  // forward outputs [digit][prime][reg*32+lane]; transpose scratch
    uint16_t abar[kLweStride];  // mod-switched mask and body
};

// Bootstrapping key staged in shared memory (shape kBrStaged): the key of
// CMux step i + 1, 64 KB, is bulk-copied (the TMA engine's cp.async.bulk,
// completion counted on an mbarrier) into one buffer while step i reads the
// other; the pointwise phase then reads the key from shared memory instead
// of through L1.
struct BkStage {
    uint4 bk[2][4][kN];         // [buffer][poly p * 2 + prime h][reg*32+lane]
    unsigned long long full[2]; // buffer landed
    uint32_t issued[2];         // uses issued into each buffer
    volatile int abort;         // a wait ran out: read the key from global memory
};
constexpr uint32_t kBkStepBytes = 4 * kN * sizeof(uint4);   // 64 KB

// The 8-warp shape's own transpose scratch, exchange rows and residue rows
// for its inverse transforms (one bootstrap per CTA leaves the room), so
// that the warps go from their pointwise products straight into their
// inverse transform without waiting for the others to finish reading the
// digit transforms.  Warps w and w + 4 (one sub-partition) share the
// pointwise products and inverse transform of (p, h) = (w >> 1, w & 1).
struct SplitExtra {
    uint32_t scratch[4][kSlot];  // transpose scratch of the warps of (p, h)
    uint32_t xch[4][kN];         // residues [p * 2 + h][reg*32+lane], [0, q)
    uint32_t ex[4][kN];          // last-stage exchange of the two warps of (p, h)
};
constexpr long kBkSpin = 1L << 20;                           // x ~1 us per try

__device__ __forceinline__ uint32_t br_saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait for phase `parity` of a stage barrier; false if it ran out.
__device__ __forceinline__ bool bk_wait(unsigned long long *bar, uint32_t parity)
{
    for (long i = 0; i < kBkSpin; ++i) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(br_saddr(bar)), "r"(parity), "r"(1000u)
                     : "memory");
        if (ok)
            return true;
    }
    return false;
}

// One thread: queue the key of CMux step i into buffer `buf` (four 16 KB
// bulk copies of the step's contiguous 64 KB).
__device__ __forceinline__ void bk_issue(BkStage &G, const uint4 *bk_ntt, int i, int buf)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     br_saddr(&G.full[buf])),
                 "r"(kBkStepBytes)
                 : "memory");
    const uint4 *src = bk_ntt + (long)i * 4 * kN;
#pragma unroll
    for (int part = 0; part < 4; ++part)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                     "[%0], [%1], %2, [%3];" ::"r"(br_saddr(&G.bk[buf][part][0])),
                     "l"(src + part * kN), "r"((uint32_t)(kN * sizeof(uint4))),
                     "r"(br_saddr(&G.full[buf]))
                     : "memory");
    G.issued[buf]++;
}

// Phase 1: warp (c, h) forms both digit polynomials of TLWE polynomial c of
// X^a acc - acc (one rotation, two digit extractions) and transforms them
// modulo prime h; results go to S.fwd[2c + j][h].  One transform copy: the
// two digits are a rolled loop.
__device__ __forceinline__ void br_digits_fwd(uint32_t (&x)[32], BrSmem &S, int c, int a,
                                              int lane, const uint2 *__restrict__ twb,
                                              const Prime &pr)
{
    const uint32_t *ac = S.acc[c];
    uint32_t *s0 = S.fwd[2 * c][pr.P], *s1 = S.fwd[2 * c + 1][pr.P];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int k = lane + 32 * r;
        const int idx = (k - a) & (2 * kN - 1);
        uint32_t v = ac[idx & (kN - 1)];
        v = idx >= kN ? 0u - v : v;
        const uint32_t u = v - ac[k] + kDecompOffset;
        x[r] = ((u >> 22) & 1023u) + (pr.q - 512u);            // level-0 digit + q
        s1[r * 32 + lane] = ((u >> 12) & 1023u) + (pr.q - 512u);  // level-1 digit, parked
    }
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
        uint32_t *sj = j ? s1 : s0;
        if (j) {
#pragma unroll
            for (int r = 0; r < 32; ++r)
                x[r] = s1[r * 32 + lane];
            __syncwarp();
        }
        fwd_ntt(x, sj, lane, twb, pr);
#pragma unroll
        for (int r = 0; r < 32; ++r)
            sj[r * 32 + lane] = x[r];
    }
}

// Phase 1 with eight warps per bootstrap: warp (c, j, h) forms digit
// polynomial j of TLWE polynomial c of X^a acc - acc and transforms it
// modulo prime h into S.fwd[2c + j][h] (its own slot, also the transpose
// scratch).
__device__ __forceinline__ void digit_fwd(uint32_t (&x)[32], const uint32_t *ac, uint32_t *sj,
                                          int j, int a, int lane, const uint2 *__restrict__ twb,
                                          const Prime &pr)
{
    const int shift = j ? 12 : 22;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int k = lane + 32 * r;
        const int idx = (k - a) & (2 * kN - 1);
        uint32_t v = ac[idx & (kN - 1)];
        v = idx >= kN ? 0u - v : v;
        const uint32_t u = v - ac[k] + kDecompOffset;
        x[r] = ((u >> shift) & 1023u) + (pr.q - 512u);
    }
    fwd_ntt(x, sj, lane, twb, pr);
#pragma unroll
    for (int r = 0; r < 32; ++r)
        sj[r * 32 + lane] = x[r];
}

__device__ __forceinline__ void br_digit_fwd(uint32_t (&x)[32], BrSmem &S, int c, int j, int a,
                                             int lane, const uint2 *__restrict__ twb,
                                             const Prime &pr)
{
    digit_fwd(x, S.acc[c], S.fwd[2 * c + j][pr.P], j, a, lane, twb, pr);
}

// Phase 2: pointwise products for output polynomial p modulo prime h,
// summed over the 4 digit rows; result in [0, 2q).  Registers R0 .. R0 +
// NR - 1 (all 32 unless two warps share the polynomial).
template <int R0 = 0, int NR = 32>
__device__ __forceinline__ void br_pointwise(uint32_t (&x)[32], const BrSmem &S,
                                             const uint4 *__restrict__ bkp, int lane,
                                             const Prime &pr)
{
    const uint32_t qn = c_ntt.q_inv[pr.P];
    const uint32_t *f0 = S.fwd[0][pr.P], *f1 = S.fwd[1][pr.P], *f2 = S.fwd[2][pr.P],
                   *f3 = S.fwd[3][pr.P];
#pragma unroll
    for (int r = R0; r < R0 + NR; ++r) {
        const uint4 b = __ldg(bkp + r * 32 + lane);
        const int e = r * 32 + lane;
        uint64_t s = (uint64_t)f0[e] * b.x;
        s += (uint64_t)f1[e] * b.y;
        s += (uint64_t)f2[e] * b.z;
        s += (uint64_t)f3[e] * b.w;
        x[r] = mont_reduce(s, pr.q, qn);
    }
}

// Phase 2 with the key staged in shared memory (shapes kBrStaged,
// kBrSplitStaged).
template <int R0 = 0, int NR = 32>
__device__ __forceinline__ void br_pointwise_staged(uint32_t (&x)[32], const BrSmem &S,
                                                    const uint4 *bks, int lane, const Prime &pr)
{
    const uint32_t qn = c_ntt.q_inv[pr.P];
    const uint32_t *f0 = S.fwd[0][pr.P], *f1 = S.fwd[1][pr.P], *f2 = S.fwd[2][pr.P],
                   *f3 = S.fwd[3][pr.P];
    const uint32_t base = br_saddr(bks);
#pragma unroll
    for (int r = R0; r < R0 + NR; ++r) {
        const int e = r * 32 + lane;
        uint4 b;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                     : "r"(base + (uint32_t)e * 16u));
        uint64_t s = (uint64_t)f0[e] * b.x;
        s += (uint64_t)f1[e] * b.y;
        s += (uint64_t)f2[e] * b.z;
        s += (uint64_t)f3[e] * b.w;
        x[r] = mont_reduce(s, pr.q, qn);
    }
}

// Phase 3: inverse transform, reduce to [0, q), publish all residues for
// the CRT (this warp's exchange slot).
__device__ __forceinline__ void br_inverse(uint32_t (&x)[32], BrSmem &S, int w4, int lane,
                                           int lane_brv, const uint2 *__restrict__ twb,
                                           const Prime &pr)
{
    inv_ntt(x, S.fwd[w4][0], lane, lane_brv, twb, pr);
    uint32_t *xch = S.fwd[w4][1];
#pragma unroll
    for (int r = 0; r < 32; ++r)
        xch[r * 32 + lane] = csub(x[r], pr.q);
}

// Phases 2 and 3 of the 8-warp shapes: warp K of the pair (w4, w4 + 4)
// takes registers 16K .. 16K + 15 of the pointwise products of (p, h) and
// of its inverse transform (named barrier 1 + w4), and publishes them
// reduced to [0, q) in the pair's residue row.
template <int K>
__device__ __forceinline__ void split_pointwise_inverse(uint32_t (&x)[32], const BrSmem &S,
                                                        SplitExtra &X, int w4, bool staged,
                                                        const uint4 *bks,
                                                        const uint4 *__restrict__ bki, int lane,
                                                        int lane_brv,
                                                        const uint2 *__restrict__ twb,
                                                        const Prime &pr)
{
    if (staged)
        br_pointwise_staged<16 * K, 16>(x, S, bks, lane, pr);
    else
        br_pointwise<16 * K, 16>(x, S, bki, lane, pr);
    inv_ntt_half<K>(x, X.scratch[w4], X.ex[w4], lane, lane_brv, twb, pr, 1 + w4);
#pragma unroll
    for (int r = 16 * K; r < 16 * K + 16; ++r)
        X.xch[w4][r * 32 + lane] = csub(x[r], pr.q);
}

// Phase 4: CRT of (r0 mod q0, r1 mod q1) to the centred integer, mod 2^32,
// added into the accumulator.  Warp (p, h) does registers 16h .. 16h + 15.
// Garner: u = (r1 - r0) q0^-1 mod q1, v = r0 + q0 u in [0, q0 q1).  The
// exact coefficient S satisfies |S| <= 4 N 2^9 2^31 = 2^52, so for S >= 0
// u = floor(S / q0) <= 2^52 / q0 < 2^25 + 2^9, and for S < 0
// (v = S + q0 q1) u >= q1 - 2^25 - 2^9; both primes exceed 2^26 + 2^25, so
// the centring decision (v >= q0 q1 / 2) is exactly u > (q1 - 1) / 2.
// The calling warp lifts registers r0 .. r0 + NR - 1 of polynomial p.
template <int NR>
__device__ __forceinline__ void crt_rows(uint32_t *acc, const uint32_t *x0, const uint32_t *x1,
                                         int r0, int lane)
{
    const uint32_t c = c_ntt.crt_c, cp = c_ntt.crt_cp, plo = c_ntt.p_lo;
    constexpr uint32_t uh = (kQ1 - 1) / 2;
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
        const int e = (r0 + rr) * 32 + lane;
        const uint32_t v0 = x0[e], v1 = x1[e];
        const uint32_t u = csub(mul_shoup(v1 - v0 + 2 * kQ1, c, cp, kQ1), kQ1);
        acc[e] += v0 + kQ0 * u - (u > uh ? plo : 0u);
    }
}

template <int NR>
__device__ __forceinline__ void br_crt(BrSmem &S, int p, int r0, int lane)
{
    crt_rows<NR>(S.acc[p], S.fwd[p * 2 + 0][1], S.fwd[p * 2 + 1][1], r0, lane);
}

// Linear part of gate `op`: c = mu + aa ca + ab cb + ac cc.  Returns false
// for an unknown opcode.
__device__ __forceinline__ bool gate_consts(int op, uint32_t &mu, uint32_t &aa, uint32_t &ab,
                                            uint32_t &ac)
{
    ac = 0u;
    switch (op) {
    case TFHE_NAND:  mu = kMu;           aa = ab = 0u - 1u; return true;
    case TFHE_AND:   mu = 0u - kMu;      aa = ab = 1u;      return true;
    case TFHE_OR:    mu = kMu;           aa = ab = 1u;      return true;
    case TFHE_XOR:   mu = 2u * kMu;      aa = ab = 2u;      return true;
    case TFHE_NOR:   mu = 0u - kMu;      aa = ab = 0u - 1u; return true;
    case TFHE_XNOR:  mu = 0u - 2u * kMu; aa = ab = 0u - 2u; return true;
    case TFHE_MAJ:   mu = 0u;            aa = ab = ac = 1u; return true;
    case TFHE_ANDNY: mu = 0u - kMu;      aa = 0u - 1u; ab = 1u; return true;
    case TFHE_ANDYN: mu = 0u - kMu;      aa = 1u; ab = 0u - 1u; return true;
    case TFHE_ORNY:  mu = kMu;           aa = 0u - 1u; ab = 1u; return true;
    case TFHE_ORYN:  mu = kMu;           aa = 1u; ab = 0u - 1u; return true;
    default:         mu = 0u;            aa = ab = 0u;      return false;
    }
}

// Gate combine + mod switch (the fused prologue) of gate slot g into
// abar[0..n] by the T threads of one bootstrap.  An empty slot (g >= count)
// or a bad one runs with abar = 0; a bad slot (opcode without its inputs,
// gather index out of range) is flagged in the status word and, when
// `writer`, its output row is zeroed.  Returns whether the slot is active.
template <int T>
__device__ __forceinline__ bool br_prologue(const BrArgs &A, long g, int tb, uint16_t *abar,
                                            bool writer)
{
    const int n = A.keys.n;
    bool active = g < A.count;
    long ra = 0, rb = 0, rc = -1;
    uint32_t mu_g = 0, aa = 1, ab = 0, ac = 0;
    if (active) {
        uint32_t err = 0;
        if (A.ops && !gate_consts(A.ops[g], mu_g, aa, ab, ac))
            err = kErrOpcode;
        ra = A.idx_a ? (long)A.idx_a[g] : g;
        rb = A.ops ? (A.idx_b ? (long)A.idx_b[g] : g) : 0;
        if (ac) {
            if (!A.in_c)
                err |= kErrOpcode;
            else
                rc = A.idx_c ? (long)A.idx_c[g] : g;
        }
        if (!(ra >= 0 && ra < A.rows_a && (!A.ops || (rb >= 0 && rb < A.rows_b)) &&
              (!ac || !A.in_c || (rc >= 0 && rc < A.rows_c))))
            err |= kErrGather;
        if (err) {
            if (writer) {
                if (tb == 0)
                    atomicOr(A.status, err);
                int32_t *bg = A.big + g * kBigStride;
                for (int k = tb; k <= kN; k += T)
                    bg[k] = 0;
            }
            active = false;
        }
    }
    if (active) {
        const int32_t *ca = A.in_a + ra * kLweStride;
        const int32_t *cb = A.ops ? A.in_b + rb * kLweStride : nullptr;
        const int32_t *cc = ac ? A.in_c + rc * kLweStride : nullptr;
        for (int i = tb; i <= n; i += T) {
            uint32_t c = (uint32_t)ca[i];
            if (A.ops) {
                c = aa * c + ab * (uint32_t)cb[i];
                if (ac)
                    c += ac * (uint32_t)cc[i];
            }
            if (i == n)
                c += mu_g;
            abar[i] = (uint16_t)(((c + (1u << 20)) >> 21) & (2 * kN - 1));
        }
    } else {
        for (int i = tb; i <= n; i += T)
            abar[i] = 0;
    }
    return active;
}

// acc = (0, X^(-bbar) v), v = mu (1 + X + ... + X^(N-1)).
template <int T>
__device__ __forceinline__ void br_acc_init(const BrArgs &A, uint32_t (*acc)[kN], int bbar, int tb)
{
    const int m = (2 * kN - bbar) & (2 * kN - 1);
    for (int k = tb; k < kN; k += T) {
        bool pos = k >= (m & (kN - 1));
        if (m >= kN)
            pos = !pos;
        acc[0][k] = 0u;
        acc[1][k] = pos ? A.mu : 0u - A.mu;
    }
}

// Sample extraction of coefficient 0: a'_0 = a_0, a'_j = -a_(N-j), b' = b_0.
template <int T>
__device__ __forceinline__ void br_extract(const BrArgs &A, long g, const uint32_t (*acc)[kN],
                                           int tb)
{
    int32_t *bg = A.big + g * kBigStride;
    for (int k = tb; k < kN; k += T)
        bg[k] = (int32_t)(k == 0 ? acc[0][0] : 0u - acc[0][kN - k]);
    if (tb == 0)
        bg[kN] = (int32_t)acc[1][0];
}

// B bootstraps per CTA, W warps each (W = 4: B in {1, 2, 4} in lockstep;
// W = 8: B = 1, the phases spread over twice the warps for lower latency on
// narrow levels); 128 registers per thread, 16 warps/SM.
//   W = 4: warp (p, h) runs phase 1 as (c = p, both digits), phases 2-3 as
//          output polynomial p modulo prime h, phase 4 on half of p.
//   W = 8: warp (c, j, h) runs phase 1 for digit j of polynomial c; warps
//          0..3 run phases 2-3 as (p, h); every warp runs phase 4 on a
//          quarter of polynomial w >> 2.
template <int B, int W, int STAGE = 0, int MINB = 0>
__global__ void __launch_bounds__(32 * W * B,
                                  MINB ? MINB : ((W * B >= 16 || W == 8) ? 1 : 16 / (W * B)))
    k_blind_rotate(const BrArgs A)
{
    constexpr int T = 32 * W;      // threads per bootstrap
    extern __shared__ uint4 smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bi = warp / W, wr = warp % W, tb = tid % T;   // bootstrap slot, role
    BrSmem &S = reinterpret_cast<BrSmem *>(smem_raw)[bi];
    BkStage &G = *reinterpret_cast<BkStage *>(reinterpret_cast<BrSmem *>(smem_raw) + B);
    SplitExtra &X = *reinterpret_cast<SplitExtra *>(
        reinterpret_cast<uint8_t *>(reinterpret_cast<BrSmem *>(smem_raw) + B) +
        (STAGE ? sizeof(BkStage) : 0));
    const int lane_brv = brv5(lane);
    const int n = A.keys.n;
    const int w4 = wr & 3, p = w4 >> 1, h = wr & 1;
    const Prime pr((uint32_t)h);
    uint32_t uses = 0;   // staged steps so far (the same in every thread)

    if (STAGE) {
        if (tid == 0) {
            for (int b = 0; b < 2; ++b) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(br_saddr(&G.full[b]))
                             : "memory");
                G.issued[b] = 0;
            }
            G.abort = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }

    for (long grp = blockIdx.x; grp * B < A.count; grp += gridDim.x) {
        const long g = grp * B + bi;
        const bool active = br_prologue<T>(A, g, tb, S.abar, true);
        if (STAGE && tid == 0 && n > 0 && !G.abort)
            bk_issue(G, A.keys.bk_ntt, 0, uses & 1);
        __syncthreads();
        br_acc_init<T>(A, S.acc, S.abar[n], tb);
        __syncthreads();

        // ---- n CMux steps, all B bootstraps in lockstep
        const BrSmem *all = reinterpret_cast<const BrSmem *>(smem_raw);
        for (int i = 0; i < n; ++i) {
            const uint32_t u = uses;   // this step's use of buffer u & 1
            if (STAGE) {
                ++uses;
                // the other buffer was last read in step i - 1, before the
                // barrier that ended that step's pointwise phase
                if (tid == 0 && i + 1 < n && !G.abort)
                    bk_issue(G, A.keys.bk_ntt, i + 1, (u + 1) & 1);
            }
            int any = 0;
#pragma unroll
            for (int b = 0; b < B; ++b)
                any |= all[b].abar[i];
            if (any == 0) {
                // X^0 acc - acc = 0 for every slot: nothing changes; the
                // step's copy still has to land before its buffer is reused
                if (STAGE && tid == 0 && !G.abort && !bk_wait(&G.full[u & 1], (u >> 1) & 1)) {
                    G.abort = 1;
                    atomicOr(A.status, kErrTimeout);
                }
                continue;
            }
            const int a = S.abar[i];  // a = 0 here gives zero digits: acc unchanged
            uint32_t x[32];
            const uint4 *bki = A.keys.bk_ntt + (((long)i * 2 + p) * 2 + h) * 1024;
            if (W == 4) {
                br_digits_fwd(x, S, p, a, lane, A.keys.twb, pr);
                __syncthreads();
                bool staged = false;
                if (STAGE) {
                    staged = !G.abort && bk_wait(&G.full[u & 1], (u >> 1) & 1);
                    if (!staged && !G.abort) {
                        G.abort = 1;   // read this and later steps from global memory
                        atomicOr(A.status, kErrTimeout);
                    }
                }
                if (staged)
                    br_pointwise_staged(x, S, &G.bk[u & 1][p * 2 + h][0], lane, pr);
                else
                    br_pointwise(x, S, bki, lane, pr);
                __syncthreads();
                br_inverse(x, S, w4, lane, lane_brv, A.keys.twb, pr);
                __syncthreads();
                br_crt<16>(S, p, 16 * h, lane);
                __syncthreads();
            } else {
                br_digit_fwd(x, S, wr >> 2, (wr >> 1) & 1, a, lane, A.keys.twb, pr);
                __syncthreads();
                bool staged = false;
                if (STAGE) {
                    staged = !G.abort && bk_wait(&G.full[u & 1], (u >> 1) & 1);
                    if (!staged && !G.abort) {
                        G.abort = 1;   // read this and later steps from global memory
                        atomicOr(A.status, kErrTimeout);
                    }
                }
                // warps w and w + 4 each take half the registers of (p, h);
                // straight on: the inverse writes only the pair's own
                // scratch, exchange and residue rows
                if (wr < 4)
                    split_pointwise_inverse<0>(x, S, X, w4, staged,
                                               STAGE ? &G.bk[u & 1][p * 2 + h][0] : nullptr, bki,
                                               lane, lane_brv, A.keys.twb, pr);
                else
                    split_pointwise_inverse<1>(x, S, X, w4, staged,
                                               STAGE ? &G.bk[u & 1][p * 2 + h][0] : nullptr, bki,
                                               lane, lane_brv, A.keys.twb, pr);
                __syncthreads();
                crt_rows<8>(S.acc[wr >> 2], X.xch[(wr >> 2) * 2 + 0], X.xch[(wr >> 2) * 2 + 1],
                            8 * (wr & 3), lane);
                __syncthreads();
            }
        }

        if (active)
            br_extract<T>(A, g, S.acc, tb);
        __syncthreads();
    }
    // after a wait that ran out: copies still in flight land before the
    // CTA's shared memory is released (the last use of each buffer)
    if (STAGE && tid == 0 && G.abort)
        for (int b = 0; b < 2; ++b)
            if (G.issued[b])
                (void)bk_wait(&G.full[b], (G.issued[b] - 1) & 1);
}

// ---------------------------------------------------------------------
// One bootstrap on a cluster of two CTAs (two SMs): CTA h works modulo
// prime h for the whole CMux and the two exchange their inverse-transform
// residues through distributed shared memory for the CRT.  For levels
// narrower than the GPU, where the per-CMux critical path sets the time.
// ---------------------------------------------------------------------

struct PairSmem {
    uint32_t acc[2][kN];        // TLWE accumulator (the same in both CTAs)
    uint32_t fwd[4][kSlot];     // digit rows modulo this CTA's prime; transpose scratch
    uint32_t pw[2][kN];         // pointwise products [p][reg*32+lane], [0, 2q)
    uint32_t res[2][2][kN];     // published residues [buffer][p][reg*32+lane], [0, q)
    uint16_t abar[kLweStride];
};

// Key stage of the cluster shape (kBrPairStaged): this CTA's prime half of
// the next CMux step's key, 2 polynomials x 16 KB, bulk-copied while the
// current step runs (double buffer).
struct PairStage {
    uint4 bk[2][2][kN];         // [buffer][poly p][reg*32+lane]
    unsigned long long full[2];
    uint32_t issued[2];
    volatile int abort;         // a wait ran out: read the key from global memory
};

__device__ __forceinline__ void pair_issue(PairStage &G, const uint4 *bk_ntt, int i, int rank,
                                           int buf)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     br_saddr(&G.full[buf])),
                 "r"((uint32_t)(2 * kN * sizeof(uint4)))
                 : "memory");
#pragma unroll
    for (int p = 0; p < 2; ++p)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                     "[%0], [%1], %2, [%3];" ::"r"(br_saddr(&G.bk[buf][p][0])),
                     "l"(bk_ntt + (((long)i * 2 + p) * 2 + rank) * kN),
                     "r"((uint32_t)(kN * sizeof(uint4))), "r"(br_saddr(&G.full[buf]))
                     : "memory");
    G.issued[buf]++;
}

// Pointwise products of rows r0 .. r0 + 15 of output polynomial p.
// SH: bkp points into the shared-memory key stage (ld.shared), else to the
// key in global memory (through L1).
template <bool SH>
__device__ __forceinline__ void pair_pointwise(PairSmem &S, const uint4 *__restrict__ bkp, int p,
                                               int r0, int lane, const Prime &pr)
{
    const uint32_t qn = c_ntt.q_inv[pr.P];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
        const int e = (r0 + rr) * 32 + lane;
        uint4 b;
        if (SH)
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                         : "r"(br_saddr(bkp) + (uint32_t)e * 16u));
        else
            b = __ldg(bkp + e);
        uint64_t s = (uint64_t)S.fwd[0][e] * b.x;
        s += (uint64_t)S.fwd[1][e] * b.y;
        s += (uint64_t)S.fwd[2][e] * b.z;
        s += (uint64_t)S.fwd[3][e] * b.w;
        S.pw[p][e] = mont_reduce(s, pr.q, qn);
    }
}

// 8 warps per CTA.  Per CMux: warps (c, j) < 4 form and transform digit j
// of polynomial c; warps (p, half) < 4 the pointwise products of half of
// output polynomial p; warps p < 2 the inverse transform of p, published to
// a residue buffer; then, after a cluster barrier, all 8 warps lift a
// quarter of one polynomial each, reading the partner's residues remotely.
// Both CTAs hold and update the whole accumulator, so the only exchange is
// the residues.  The residue buffers alternate by executed CMux: a buffer
// is rewritten two CMux steps after the partner read it, with the partner's
// barrier arrival of the step between in between.  Control flow is the
// same in both CTAs of a cluster (same gate, same abar), so every cluster
// barrier is reached by both.
template <int STAGE>
__global__ void __launch_bounds__(256, 1) k_blind_rotate_pair(const BrArgs A)
{
    extern __shared__ uint4 smem_raw[];
    PairSmem &S = *reinterpret_cast<PairSmem *>(smem_raw);
    PairStage &G = *reinterpret_cast<PairStage *>(reinterpret_cast<PairSmem *>(smem_raw) + 1);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lane_brv = brv5(lane);
    const int n = A.keys.n;
    const Prime pr((uint32_t)rank);
    const long nclusters = gridDim.x / 2, cid = blockIdx.x / 2;
    int par = 0;
    uint32_t uses = 0;   // staged steps so far (the same in every thread)
    if (STAGE) {
        if (tid == 0) {
            for (int b = 0; b < 2; ++b) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(br_saddr(&G.full[b]))
                             : "memory");
                G.issued[b] = 0;
            }
            G.abort = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    for (long g = cid; g < A.count; g += nclusters) {
        const bool active = br_prologue<256>(A, g, tid, S.abar, rank == 0);
        if (STAGE && tid == 0 && n > 0 && !G.abort)
            pair_issue(G, A.keys.bk_ntt, 0, rank, uses & 1);
        __syncthreads();
        br_acc_init<256>(A, S.acc, S.abar[n], tid);
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const uint32_t u = uses;   // this step's use of buffer u & 1
            if (STAGE) {
                ++uses;
                // the other buffer was last read in step i - 1, before the
                // barrier that ended that step's pointwise phase
                if (tid == 0 && i + 1 < n && !G.abort)
                    pair_issue(G, A.keys.bk_ntt, i + 1, rank, (u + 1) & 1);
            }
            const int a = S.abar[i];
            if (a == 0) {
                // X^0 acc - acc = 0: nothing changes (in both CTAs); the
                // step's copy still has to land before its buffer is reused
                if (STAGE && tid == 0 && !G.abort && !bk_wait(&G.full[u & 1], (u >> 1) & 1)) {
                    G.abort = 1;
                    atomicOr(A.status, kErrTimeout);
                }
                continue;
            }
            uint32_t x[32];
            if (warp < 4)
                digit_fwd(x, S.acc[warp >> 1], S.fwd[warp], warp & 1, a, lane, A.keys.twb, pr);
            __syncthreads();
            if (warp < 4) {
                const int p = warp >> 1;
                bool staged = false;
                if (STAGE) {
                    staged = !G.abort && bk_wait(&G.full[u & 1], (u >> 1) & 1);
                    if (!staged && !G.abort) {
                        G.abort = 1;   // read this and later steps from global memory
                        atomicOr(A.status, kErrTimeout);
                    }
                }
                if (staged)
                    pair_pointwise<true>(S, &G.bk[u & 1][p][0], p, 16 * (warp & 1), lane, pr);
                else
                    pair_pointwise<false>(S, A.keys.bk_ntt + (((long)i * 2 + p) * 2 + rank) * 1024,
                                          p, 16 * (warp & 1), lane, pr);
            }
            __syncthreads();
            if (warp < 2) {
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    x[r] = S.pw[warp][r * 32 + lane];
                inv_ntt(x, S.fwd[warp], lane, lane_brv, A.keys.twb, pr);
                uint32_t *out = S.res[par][warp];
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    out[r * 32 + lane] = csub(x[r], pr.q);
            }
            cl.sync();
            {
                const int p = warp >> 2;
                const uint32_t *mine = S.res[par][p];
                const uint32_t *other = cl.map_shared_rank(mine, rank ^ 1);
                crt_rows<8>(S.acc[p], rank == 0 ? mine : other, rank == 0 ? other : mine,
                            8 * (warp & 3), lane);
            }
            par ^= 1;
            __syncthreads();
        }
        if (active && rank == 0)
            br_extract<256>(A, g, S.acc, tid);
        __syncthreads();
    }
    cl.sync();   // the partner may still read this CTA's residues
    // after a wait that ran out: copies still in flight land before the
    // CTA's shared memory is released (the last use of each buffer)
    if (STAGE && tid == 0 && G.abort)
        for (int b = 0; b < 2; ++b)
            if (G.issued[b])
                (void)bk_wait(&G.full[b], (G.issued[b] - 1) & 1);
}

// ---------------------------------------------------------------------
// Host side: constants and launchers
// ---------------------------------------------------------------------

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (a * b) % m; }

static uint64_t powmod(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1;
    b %= m;
    while (e) {
        if (e & 1)
            r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}

static uint32_t shoup_of(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

// A primitive 2N-th root of unity: psi^N = -1.
static uint32_t find_psi(uint32_t q)
{
    for (uint64_t x = 2; x < 100000; ++x) {
        uint64_t psi = powmod(x, (q - 1) / (2 * kN), q);
        if (powmod(psi, kN, q) == q - 1)
            return (uint32_t)psi;
    }
    return 0;
}

static int bitrev(int k, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b)
        if (k & (1 << b))
            r |= 1 << (bits - 1 - b);
    return r;
}

// Builds the NTT constants into c_ntt (current device) and the stage-B
// twiddle table into twb_dev ([2][2][32][32] uint2).
cudaError_t upload_ntt_constants(uint2 *twb_dev, cudaStream_t stream)
{
    NttConst C;
    std::memset(&C, 0, sizeof(C));
    std::vector<uint2> twb(2 * 2 * 32 * 32);
    const uint32_t qs[2] = {kQ0, kQ1};
    for (int P = 0; P < 2; ++P) {
        const uint32_t q = qs[P];
        const uint64_t psi = find_psi(q), ipsi = powmod(psi, q - 2, q);
        const uint64_t w64 = powmod(psi, 32, q), w32 = powmod(psi, 64, q);
        const uint64_t iw64 = powmod(w64, q - 2, q), iw32 = powmod(w32, q - 2, q);
        for (int k = 0; k < 32; ++k) {
            uint32_t a = (uint32_t)powmod(w64, brv5(k), q), ia = (uint32_t)powmod(iw64, brv5(k), q);
            C.za[P][k][0] = a;
            C.za[P][k][1] = shoup_of(a, q);
            C.iza[P][k][0] = ia;
            C.iza[P][k][1] = shoup_of(ia, q);
        }
        for (int m = 1; m <= 16; m <<= 1) {
            int lg = 0;
            while ((1 << lg) < m)
                ++lg;
            for (int g = 0; g < m; ++g) {
                const int e = bitrev(g, lg) * (16 / m);
                uint32_t d = (uint32_t)powmod(w32, e, q), id = (uint32_t)powmod(iw32, e, q);
                C.zd[P][m + g][0] = d;
                C.zd[P][m + g][1] = shoup_of(d, q);
                C.izd[P][m + g][0] = id;
                C.izd[P][m + g][1] = shoup_of(id, q);
            }
        }
        for (int r = 0; r < 32; ++r)
            for (int l = 0; l < 32; ++l) {
                // forward: lane i1 = l, register r carries k1 = brv5(r)
                uint32_t f = (uint32_t)powmod(psi, (uint64_t)(2 * brv5(r) + 1) * l, q);
                // inverse: lane k1 = l, register i1 = r
                uint32_t iv = (uint32_t)powmod(ipsi, (uint64_t)(2 * l + 1) * r, q);
                twb[((P * 2 + 0) * 32 + r) * 32 + l] = make_uint2(f, shoup_of(f, q));
                twb[((P * 2 + 1) * 32 + r) * 32 + l] = make_uint2(iv, shoup_of(iv, q));
            }
        // q^-1 mod 2^32 by Newton iteration
        uint32_t inv = q;
        for (int it = 0; it < 5; ++it)
            inv *= 2u - q * inv;
        C.q_inv[P] = inv;
        const uint64_t ninv = powmod(kN, q - 2, q);
        const uint32_t sc = (uint32_t)mulmod((((uint64_t)1 << 32) % q), ninv, q);
        C.bk_scale[P][0] = sc;
        C.bk_scale[P][1] = shoup_of(sc, q);
    }
    C.crt_c = (uint32_t)powmod(kQ0, kQ1 - 2, kQ1);
    C.crt_cp = shoup_of(C.crt_c, kQ1);
    const unsigned __int128 Pp = (unsigned __int128)kQ0 * kQ1;
    C.p_lo = (uint32_t)Pp;
    C.p_half = (uint64_t)((Pp + 1) / 2);
    cudaError_t e = cudaMemcpyToSymbolAsync(c_ntt, &C, sizeof(C), 0, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyAsync(twb_dev, twb.data(), twb.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                        stream);
    if (e != cudaSuccess)
        return e;
    return cudaStreamSynchronize(stream);
}

cudaError_t launch_bk_to_ntt(const int32_t *bk_dev, uint32_t *bk_ntt, int n, const uint2 *twb,
                             cudaStream_t stream)
{
    const long tasks = (long)n * kRows * 2 * 2;
    k_bk_to_ntt<<<(unsigned)((tasks + 3) / 4), 128, 0, stream>>>(bk_dev, bk_ntt, n, twb);
    return cudaGetLastError();
}

// Dynamic shared memory of a shape: B bootstraps, plus the key stages for
// the staged shape and its control (which reserves them unused, so both run
// one CTA per SM).
template <int B, int STAGE, int W = 4>
constexpr size_t br_smem(bool stage_room)
{
    return B * sizeof(BrSmem) + (STAGE || stage_room ? sizeof(BkStage) : 0) +
           (W == 8 ? sizeof(SplitExtra) : 0);
}

template <int B, int W, int STAGE = 0, int MINB = 0>
static void br_prepare(size_t smem)
{
    cudaFuncSetAttribute(k_blind_rotate<B, W, STAGE, MINB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_blind_rotate<B, W, STAGE, MINB>,
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    (void)cudaGetLastError();
}

template <int B, int W, int STAGE = 0, int MINB = 0>
static int br_blocks(int dev, bool stage_room = false)
{
    static int cached[2][64] = {{0}};
    if (dev < 0 || dev >= 64)
        return 1;
    const size_t smem = br_smem<B, STAGE, W>(stage_room);
    if (!cached[stage_room][dev]) {
        // the attribute covers the larger of the two requests of the shape
        br_prepare<B, W, STAGE, MINB>(br_smem<B, STAGE, W>(B == 2 && W == 4));
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blind_rotate<B, W, STAGE, MINB>,
                                                          32 * W * B, smem) != cudaSuccess) {
            (void)cudaGetLastError();
            nb = 0;
        }
        cached[stage_room][dev] = nb > 0 ? nb : 1;
    }
    return cached[stage_room][dev];
}

// Bootstraps in flight per SM for the variant (all variants: 16 warps).
int br_blocks_per_sm()
{
    int dev = 0;
    cudaGetDevice(&dev);
    br_blocks<2, 4>(dev);
    br_blocks<4, 4>(dev);
    br_blocks<1, 8>(dev);
    return br_blocks<1, 4>(dev);
}

// CTA shape: 1, 2 or 4 bootstraps per CTA in lockstep (4 warps each; groups
// share instruction fetch and key reads but leave SMs idle when a level is
// narrow), or kBrSplit: one bootstrap on 8 warps (shorter critical path
// per CMux, for levels narrower than the GPU).
static bool br_shape_ok(int v)
{
    return v == 1 || v == 2 || v == 4 || v == kBrSplit || v == kBrPair || v == kBrStaged ||
           v == kBrStagedCtl || v == kBrSplitStaged || v == kBrFive || v == kBrPairStaged;
}

static int br_group(long count, int num_sms, int forced, const int8_t *tuned)
{
    if (br_shape_ok(forced))
        return forced;
    const int t = tuned[tune_bucket(count)];
    if (br_shape_ok(t))
        return t;
    const long per_sm = (count + num_sms - 1) / num_sms;
    return per_sm >= 8 ? 4 : (per_sm >= 3 ? 2 : kBrSplit);
}

cudaError_t launch_blind_rotate(const DevKeys &keys, const uint8_t *ops, const int32_t *in_a,
                                const int32_t *idx_a, long rows_a, const int32_t *in_b,
                                const int32_t *idx_b, long rows_b, int32_t *big, long count,
                                uint32_t mu, uint32_t *status, int grid, cudaStream_t stream,
                                const int32_t *in_c, const int32_t *idx_c, long rows_c)
{
    if (count <= 0)
        return cudaSuccess;
    BrArgs A;
    A.keys = keys;
    A.in_a = in_a;
    A.in_b = in_b;
    A.in_c = in_c;
    A.idx_a = idx_a;
    A.idx_b = idx_b;
    A.idx_c = idx_c;
    A.rows_a = rows_a;
    A.rows_b = rows_b;
    A.rows_c = rows_c;
    A.ops = ops;
    A.big = big;
    A.count = count;
    A.mu = mu;
    A.status = status;
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int shape = br_group(count, sms > 0 ? sms : 1, keys.br_group, keys.tune_br);
    if (shape == kBrPair || shape == kBrPairStaged) {
        const bool staged = shape == kBrPairStaged;
        const size_t smem = sizeof(PairSmem) + (staged ? sizeof(PairStage) : 0);
        static int prepared[2][64] = {{0}};
        if (dev >= 0 && dev < 64 && !prepared[staged][dev]) {
            cudaFuncSetAttribute(staged ? k_blind_rotate_pair<1> : k_blind_rotate_pair<0>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            (void)cudaGetLastError();
            prepared[staged][dev] = 1;
        }
        const long pairs = sms >= 2 ? sms / 2 : 1;   // one CTA per SM
        const long clusters = count < pairs ? count : pairs;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * clusters));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return staged ? cudaLaunchKernelEx(&cfg, k_blind_rotate_pair<1>, A)
                      : cudaLaunchKernelEx(&cfg, k_blind_rotate_pair<0>, A);
    }
    const int B = (shape == kBrSplit || shape == kBrSplitStaged || shape == kBrFive) ? 1
                : (shape == kBrStaged || shape == kBrStagedCtl) ? 2 : shape;
    const long groups = (count + B - 1) / B;
    long blocks_per_sm = shape == 4 ? br_blocks<4, 4>(dev)
                       : shape == 2 ? br_blocks<2, 4>(dev)
                       : shape == kBrStaged ? br_blocks<2, 4, 1>(dev)
                       : shape == kBrStagedCtl ? br_blocks<2, 4>(dev, true)
                       : shape == kBrSplitStaged ? br_blocks<1, 8, 1>(dev)
                       : shape == kBrFive ? br_blocks<1, 4, 0, 5>(dev)
                       : shape == kBrSplit ? br_blocks<1, 8>(dev) : br_blocks<1, 4>(dev);
    const long cap = blocks_per_sm * (sms > 0 ? sms : 1);
    const unsigned blocks = (unsigned)(groups < cap ? groups : cap);
    (void)grid;
    switch (shape) {
    case 4: k_blind_rotate<4, 4><<<blocks, 512, 4 * sizeof(BrSmem), stream>>>(A); break;
    case 2: k_blind_rotate<2, 4><<<blocks, 256, 2 * sizeof(BrSmem), stream>>>(A); break;
    case kBrStaged:
        k_blind_rotate<2, 4, 1><<<blocks, 256, br_smem<2, 1>(false), stream>>>(A);
        break;
    case kBrStagedCtl:
        k_blind_rotate<2, 4><<<blocks, 256, br_smem<2, 0>(true), stream>>>(A);
        break;
    case kBrSplitStaged:
        k_blind_rotate<1, 8, 1><<<blocks, 256, br_smem<1, 1, 8>(false), stream>>>(A);
        break;
    case kBrFive: k_blind_rotate<1, 4, 0, 5><<<blocks, 128, sizeof(BrSmem), stream>>>(A); break;
    case kBrSplit:
        k_blind_rotate<1, 8><<<blocks, 256, br_smem<1, 0, 8>(false), stream>>>(A);
        break;
    default: k_blind_rotate<1, 4><<<blocks, 128, sizeof(BrSmem), stream>>>(A); break;
    }
    return cudaGetLastError();
}

}  // namespace tgb

