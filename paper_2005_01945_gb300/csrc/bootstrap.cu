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
//  * the products are exact: a negacyclic NTT modulo two primes below 2^28
//    and a centred CRT lift back to Z/2^32;
//  * one CTA of 4 warps owns one bootstrap at a time and loops over gates
//    (persistent grid); the accumulator never leaves shared memory;
//  * warp w = (c, j) forms digit polynomial (c, j) in registers and runs the
//    forward transforms for both primes; warp w = (p, q) then does the
//    pointwise products with BK_i for output polynomial p modulo prime q,
//    the inverse transform, and half of the CRT + accumulate;
//  * one 1024-point transform is one warp: 32 coefficients per lane,
//    a 32-point transform in registers, a twiddle, one shared-memory
//    transpose, and a second 32-point transform (four-step NTT);
//  * the bootstrapping key is pre-transformed, scaled by 2^32 N^-1 and
//    interleaved so that lane l reads its 4 rows for one register as one
//    16-byte load; the 33 MB key stays L2-resident across gates.
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace tgb {

struct NttConst {
    uint32_t za[2][32][2];   // forward stage A: w64^brv5(k), Shoup companion
    uint32_t zd[2][32][2];   // forward stage D: cyclic size-32 twiddles
    uint32_t iza[2][32][2];  // inverse of stage A
    uint32_t izd[2][32][2];  // inverse of stage D
    uint32_t qneg_inv[2];    // -q^-1 mod 2^32
    uint32_t crt_c, crt_cp;  // q0^-1 mod q1 and its Shoup companion mod q1
    uint32_t p_lo, pad;      // (q0 q1) mod 2^32
    uint64_t p_half;         // (q0 q1 + 1) / 2
    uint32_t bk_scale[2][2]; // 2^32 N^-1 mod q and companion
};

__constant__ NttConst c_ntt;

template <int P>
__device__ __forceinline__ constexpr uint32_t prime() { return P == 0 ? kQ0 : kQ1; }

__host__ __device__ constexpr int brv5(int k)
{
    return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

// 32-point Cooley-Tukey pass in registers, lazy in [0, 4q).
// TBL 0: negacyclic (stage A) twiddles; 1: cyclic (stage D), whose first
// twiddle of every level is 1.
template <int P, int TBL>
__device__ __forceinline__ void ct32(uint32_t (&x)[32])
{
    constexpr uint32_t q = prime<P>(), q2 = 2 * prime<P>();
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int m = 1 << s, ln = 16 >> s;
#pragma unroll
        for (int g = 0; g < m; ++g) {
            const uint32_t w = TBL == 0 ? c_ntt.za[P][m + g][0] : c_ntt.zd[P][m + g][0];
            const uint32_t wp = TBL == 0 ? c_ntt.za[P][m + g][1] : c_ntt.zd[P][m + g][1];
#pragma unroll
            for (int jj = 0; jj < ln; ++jj) {
                const int j = 2 * g * ln + jj;
                const uint32_t u = csub(x[j], q2);
                const uint32_t t = (TBL == 1 && g == 0) ? csub(x[j + ln], q2)
                                                        : mul_shoup(x[j + ln], w, wp, q);
                x[j] = u + t;
                x[j + ln] = u - t + q2;
            }
        }
    }
}

// Inverse (Gentleman-Sande) of ct32, inputs and outputs in [0, 2q); the
// result is 32 times the inverse transform.
template <int P, int TBL>
__device__ __forceinline__ void gs32(uint32_t (&x)[32])
{
    constexpr uint32_t q = prime<P>(), q2 = 2 * prime<P>();
#pragma unroll
    for (int s = 4; s >= 0; --s) {
        const int m = 1 << s, ln = 16 >> s;
#pragma unroll
        for (int g = 0; g < m; ++g) {
            const uint32_t w = TBL == 0 ? c_ntt.iza[P][m + g][0] : c_ntt.izd[P][m + g][0];
            const uint32_t wp = TBL == 0 ? c_ntt.iza[P][m + g][1] : c_ntt.izd[P][m + g][1];
#pragma unroll
            for (int jj = 0; jj < ln; ++jj) {
                const int j = 2 * g * ln + jj;
                const uint32_t u = x[j], v = x[j + ln];
                x[j] = csub(u + v, q2);
                const uint32_t d = u - v + q2;
                x[j + ln] = (TBL == 1 && g == 0) ? csub(d, q2) : mul_shoup(d, w, wp, q);
            }
        }
    }
}

// Forward negacyclic NTT of one polynomial held by one warp.
// In : lane l, register r holds coefficient l + 32 r, value in [0, 4q).
// Out: lane l, register r holds the evaluation at psi^(2 (l + 32 brv5(r)) + 1),
//      value in [0, 4q).  sbuf: 1024 words of this warp's shared memory.
template <int P>
__device__ __forceinline__ void fwd_ntt(uint32_t (&x)[32], uint32_t *sbuf, int lane,
                                        const uint2 *__restrict__ twb)
{
    constexpr uint32_t q = prime<P>();
    ct32<P, 0>(x);
    const uint2 *tw = twb + (P * 2 + 0) * 1024 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint2 t = __ldg(tw + r * 32);
        x[r] = mul_shoup(x[r], t.x, t.y, q);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int k1 = brv5(r);
        sbuf[k1 * 32 + (lane ^ k1)] = x[r];
    }
    __syncwarp();
#pragma unroll
    for (int i1 = 0; i1 < 32; ++i1)
        x[i1] = sbuf[lane * 32 + (i1 ^ lane)];
    __syncwarp();
    ct32<P, 1>(x);
}

// Inverse of fwd_ntt up to the factor N: input layout of fwd_ntt's output
// with values in [0, 2q); output lane l, register r = N * coefficient
// l + 32 r, in [0, 2q).
template <int P>
__device__ __forceinline__ void inv_ntt(uint32_t (&x)[32], uint32_t *sbuf, int lane, int lane_brv,
                                        const uint2 *__restrict__ twb)
{
    constexpr uint32_t q = prime<P>();
    gs32<P, 1>(x);
    const uint2 *tw = twb + (P * 2 + 1) * 1024 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint2 t = __ldg(tw + r * 32);
        x[r] = mul_shoup(x[r], t.x, t.y, q);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
        sbuf[r * 32 + (lane_brv ^ r)] = x[r];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r)
        x[r] = sbuf[lane * 32 + (r ^ lane)];
    __syncwarp();
    gs32<P, 0>(x);
}

// ---------------------------------------------------------------------
// Bootstrapping key -> NTT domain
// ---------------------------------------------------------------------

// One warp per (i, row, poly, prime).  bk: int32 [n][4][2][N] coefficient
// form.  Output element (i, p, q, reg, lane) is a uint4 over the 4 rows.
__global__ void __launch_bounds__(128) k_bk_to_ntt(const int32_t *__restrict__ bk, uint32_t *out,
                                                   int n, const uint2 *__restrict__ twb)
{
    __shared__ uint32_t sbuf[4][1024];
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
    if (qsel == 0)
        fwd_ntt<0>(x, sbuf[warp], lane, twb);
    else
        fwd_ntt<1>(x, sbuf[warp], lane, twb);
    const uint32_t sc = c_ntt.bk_scale[qsel][0], scp = c_ntt.bk_scale[qsel][1];
    // element index in uint32 words: ((((i*2+p)*2+q)*32 + reg)*32 + lane)*4 + r
    uint32_t *dst = out + ((((i * 2 + p) * 2 + qsel) * 32) * 32 + lane) * 4 + r;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        uint32_t v = x[k] % q;                         // [0, 4q) -> [0, q)
        v = csub(mul_shoup(v, sc, scp, q), q);        // * 2^32 N^-1, in [0, q)
        dst[k * 32 * 4] = v;
    }
}

// ---------------------------------------------------------------------
// Blind rotation
// ---------------------------------------------------------------------

struct BrArgs {
    DevKeys keys;
    const int32_t *in_a, *in_b;      // ciphertext bases (row stride kLweStride)
    const int32_t *idx_a, *idx_b;    // optional gather rows (nullptr: row g)
    long rows_a, rows_b;             // rows addressable through the bases
    const uint8_t *ops;              // gate opcodes (nullptr: bootstrap in_a as is)
    int32_t *big;                    // out: LWE_N samples [count][kBigStride]
    long count;
    uint32_t mu;                     // test-vector amplitude
    uint32_t *status;
};

struct BrSmem {
    uint32_t acc[2][kN];        // TLWE accumulator (a(X), b(X))
    uint32_t fwd[4][2][kN];     // forward outputs [digit][prime][reg*32+lane]
    uint16_t abar[kLweStride];  // mod-switched mask and body
};

constexpr int kBrThreads = 128;

// Phase 2: pointwise products for output polynomial p modulo prime P,
// summed over the 4 digit rows; result in [0, 2q).
template <int P>
__device__ __forceinline__ void br_pointwise(uint32_t (&x)[32], const BrSmem &S,
                                             const uint4 *__restrict__ bkp, int lane)
{
    constexpr uint32_t q = prime<P>();
    const uint32_t qn = c_ntt.qneg_inv[P];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint4 b = __ldg(bkp + r * 32 + lane);
        const int e = r * 32 + lane;
        uint64_t s = (uint64_t)S.fwd[0][P][e] * b.x;
        s += (uint64_t)S.fwd[1][P][e] * b.y;
        s += (uint64_t)S.fwd[2][P][e] * b.z;
        s += (uint64_t)S.fwd[3][P][e] * b.w;
        x[r] = mont_reduce(s, q, qn);
    }
}

// Phase 3: inverse transform, reduce to [0, q), publish the half of the
// residues the partner warp needs for the CRT.
template <int P>
__device__ __forceinline__ void br_inverse(uint32_t (&x)[32], BrSmem &S, int warp, int lane,
                                           int lane_brv, const uint2 *__restrict__ twb)
{
    constexpr uint32_t q = prime<P>();
    inv_ntt<P>(x, S.fwd[warp][0], lane, lane_brv, twb);
    uint32_t *xch = S.fwd[warp][1];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        x[r] = csub(x[r], q);
        if ((P == 0 && r >= 16) || (P == 1 && r < 16))
            xch[r * 32 + lane] = x[r];
    }
}

// Phase 4: CRT of (r0 mod q0, r1 mod q1) to the centred integer, mod 2^32,
// added into the accumulator.  Warp (p, 0) does registers 0..15,
// warp (p, 1) registers 16..31.
template <int P>
__device__ __forceinline__ void br_crt(const uint32_t (&x)[32], BrSmem &S, int p, int lane)
{
    const uint32_t *other = S.fwd[p * 2 + (1 - P)][1];
    const uint32_t c = c_ntt.crt_c, cp = c_ntt.crt_cp, plo = c_ntt.p_lo;
    const uint64_t phalf = c_ntt.p_half;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
        const int r = P == 0 ? rr : rr + 16;
        const uint32_t r0 = P == 0 ? x[r] : other[r * 32 + lane];
        const uint32_t r1 = P == 0 ? other[r * 32 + lane] : x[r];
        uint32_t u = mul_shoup(r1 - r0 + 2 * kQ1, c, cp, kQ1);
        u = csub(u, kQ1);
        const uint64_t v = (uint64_t)r0 + (uint64_t)kQ0 * u;
        const uint32_t res = (uint32_t)v - (v >= phalf ? plo : 0u);
        S.acc[p][lane + 32 * r] += res;
    }
}

__device__ __forceinline__ void gate_consts(int op, uint32_t &mu, uint32_t &alpha)
{
    switch (op) {
    case TFHE_NAND: mu = kMu;           alpha = 0u - 1u; break;
    case TFHE_AND:  mu = 0u - kMu;      alpha = 1u;      break;
    case TFHE_OR:   mu = kMu;           alpha = 1u;      break;
    case TFHE_XOR:  mu = 2u * kMu;      alpha = 2u;      break;
    case TFHE_NOR:  mu = 0u - kMu;      alpha = 0u - 1u; break;
    default:        mu = 0u - 2u * kMu; alpha = 0u - 2u; break;  // XNOR
    }
}

__global__ void __launch_bounds__(kBrThreads) k_blind_rotate(const BrArgs A)
{
    extern __shared__ uint4 smem_raw[];
    BrSmem &S = *reinterpret_cast<BrSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lane_brv = brv5(lane);
    const int n = A.keys.n;

    for (long g = blockIdx.x; g < A.count; g += gridDim.x) {
        // ---- gate combine + mod switch (fused prologue)
        const long ra = A.idx_a ? (long)A.idx_a[g] : g;
        const long rb = A.ops ? (A.idx_b ? (long)A.idx_b[g] : g) : 0;
        const bool ok = ra >= 0 && ra < A.rows_a && (!A.ops || (rb >= 0 && rb < A.rows_b));
        if (!ok) {
            if (tid == 0)
                atomicOr(A.status, kErrGather);
            int32_t *bg = A.big + g * kBigStride;
            for (int k = tid; k <= kN; k += kBrThreads)
                bg[k] = 0;
            continue;  // uniform across the CTA
        }
        const int32_t *ca = A.in_a + ra * kLweStride;
        const int32_t *cb = A.ops ? A.in_b + rb * kLweStride : nullptr;
        uint32_t mu_g = 0, alpha = 1;
        if (A.ops)
            gate_consts(A.ops[g], mu_g, alpha);
        for (int i = tid; i <= n; i += kBrThreads) {
            uint32_t c = A.ops ? alpha * ((uint32_t)ca[i] + (uint32_t)cb[i]) : (uint32_t)ca[i];
            if (i == n)
                c += mu_g;
            S.abar[i] = (uint16_t)(((c + (1u << 20)) >> 21) & (2 * kN - 1));
        }
        __syncthreads();

        // ---- acc = (0, X^(-bbar) v)
        {
            const int m = (2 * kN - (int)S.abar[n]) & (2 * kN - 1);
            for (int k = tid; k < kN; k += kBrThreads) {
                bool pos = k >= (m & (kN - 1));
                if (m >= kN)
                    pos = !pos;
                S.acc[0][k] = 0u;
                S.acc[1][k] = pos ? A.mu : 0u - A.mu;
            }
        }
        __syncthreads();

        // ---- n CMux steps
        for (int i = 0; i < n; ++i) {
            const int a = S.abar[i];
            if (a == 0)
                continue;  // X^0 acc - acc = 0: the step leaves acc unchanged
            uint32_t x[32];
            {   // phase 1: warp (c, j) builds digit polynomial c*l + j, both NTTs
                const int c = warp >> 1, shift = 22 - 10 * (warp & 1);
                const uint32_t *ac = S.acc[c];
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const int k = lane + 32 * r;
                    const int idx = (k - a) & (2 * kN - 1);
                    uint32_t v = ac[idx & (kN - 1)];
                    v = idx >= kN ? 0u - v : v;
                    const uint32_t u = v - ac[k] + kDecompOffset;
                    x[r] = (u >> shift) & 1023u;  // digit + 512
                }
                uint32_t *s0 = S.fwd[warp][0], *s1 = S.fwd[warp][1];
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    s1[r * 32 + lane] = x[r];
                    x[r] += kQ0 - 512u;
                }
                fwd_ntt<0>(x, s0, lane, A.keys.twb);
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    s0[r * 32 + lane] = x[r];
                    x[r] = s1[r * 32 + lane] + (kQ1 - 512u);
                }
                __syncwarp();
                fwd_ntt<1>(x, s1, lane, A.keys.twb);
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    s1[r * 32 + lane] = x[r];
            }
            __syncthreads();
            const int p = warp >> 1, qs = warp & 1;
            const uint4 *bkp = A.keys.bk_ntt + (((long)i * 2 + p) * 2 + qs) * 1024;
            if (qs == 0)
                br_pointwise<0>(x, S, bkp, lane);
            else
                br_pointwise<1>(x, S, bkp, lane);
            __syncthreads();
            if (qs == 0)
                br_inverse<0>(x, S, warp, lane, lane_brv, A.keys.twb);
            else
                br_inverse<1>(x, S, warp, lane, lane_brv, A.keys.twb);
            __syncthreads();
            if (qs == 0)
                br_crt<0>(x, S, p, lane);
            else
                br_crt<1>(x, S, p, lane);
            __syncthreads();
        }

        // ---- sample extraction of coefficient 0
        int32_t *bg = A.big + g * kBigStride;
        for (int k = tid; k < kN; k += kBrThreads)
            bg[k] = (int32_t)(k == 0 ? S.acc[0][0] : 0u - S.acc[0][kN - k]);
        if (tid == 0)
            bg[kN] = (int32_t)S.acc[1][0];
        __syncthreads();
    }
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
        // -q^-1 mod 2^32 by Newton iteration
        uint32_t inv = q;
        for (int it = 0; it < 5; ++it)
            inv *= 2u - q * inv;
        C.qneg_inv[P] = 0u - inv;
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

size_t br_smem_bytes() { return sizeof(BrSmem); }

cudaError_t launch_blind_rotate(const DevKeys &keys, const uint8_t *ops, const int32_t *in_a,
                                const int32_t *idx_a, long rows_a, const int32_t *in_b,
                                const int32_t *idx_b, long rows_b, int32_t *big, long count,
                                uint32_t mu, uint32_t *status, int grid, cudaStream_t stream)
{
    if (count <= 0)
        return cudaSuccess;
    BrArgs A;
    A.keys = keys;
    A.in_a = in_a;
    A.in_b = in_b;
    A.idx_a = idx_a;
    A.idx_b = idx_b;
    A.rows_a = rows_a;
    A.rows_b = rows_b;
    A.ops = ops;
    A.big = big;
    A.count = count;
    A.mu = mu;
    A.status = status;
    const unsigned blocks = (unsigned)(count < grid ? count : grid);
    k_blind_rotate<<<blocks, kBrThreads, sizeof(BrSmem), stream>>>(A);
    return cudaGetLastError();
}

}  // namespace tgb

namespace tgb {
int br_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blind_rotate, kBrThreads,
                                                      sizeof(BrSmem)) != cudaSuccess) {
        (void)cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}
}  // namespace tgb
