/*
 * tfhe_oracle.c -- plain, slow, obviously correct CPU oracle for TFHE gate
 * bootstrapping and the boolean circuits built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it is used by tests/, by __graft_entry__.smoke() as the
 * checker, and by the cpu_baseline / reference leg of bench.py.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes (the paper builds on TFHE, section II-A "Torus FHE"):
 *   - Torus32: a real number mod 1 stored as a 32-bit word x, value x / 2^32.
 *     All torus arithmetic is uint32 arithmetic (wraps mod 2^32), which is
 *     exact.
 *   - LWE sample (A, B) with B = A.S + e (section II-A).
 *   - Gate bootstrapping = "bootstrapping" then "key switching", the two
 *     phases the paper times separately (Table "differentialtime", section
 *     VI-A; Fig. "gpu_execution" names the BS and KS keys).  Their internals
 *     are those of the TFHE construction the paper adopts: blind rotation as
 *     n CMux external products of a TGSW key with a TLWE accumulator, sample
 *     extraction, then LWE-to-LWE key switching.
 *   - Boolean circuits: ripple-carry adder (Eq. "addres", Eq. "addcarry",
 *     sections III-A and V-B-1), naive shift-and-add multiplication (section
 *     III-B-1) and the matrix-vector product of section IV-D with the
 *     tree-based accumulation of section V-B-2; and the variants: the
 *     number-wise adder of section V-B-1, majority-carry adders, tree
 *     multiplication, full products naive and by Karatsuba (section III-B),
 *     and the low-depth parallel-prefix adder and Dadda multiplier.
 *
 * Every polynomial product here is the schoolbook definition of a product in
 * Z[X]/(X^N+1) evaluated with uint32 wraparound, i.e. exactly mod 2^32.
 * No randomness is drawn here: key bits, masks and noise are inputs.
 *
 * Threads (OpenMP) only run independent work side by side: independent
 * gates of a batch, and the gates of circuits as tasks ordered by the rows
 * they read and write, so every result equals that of a one-by-one
 * evaluation (see "Order of evaluation" below).
 *
 * Parity of the noise statistics against a closed form is pinned in the
 * tests (measured variance vs. derived variance); every other function is
 * pinned against an independent computation (Karatsuba products, library
 * convolutions, exact noiseless identities, truth tables, brute force).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n;          /* LWE dimension                                  */
    int32_t N;          /* TLWE ring degree (power of two)                */
    int32_t l;          /* gadget decomposition levels                    */
    int32_t bg_bit;     /* log2 of the gadget base Bg                     */
    int32_t ks_t;       /* key-switch decomposition levels                */
    int32_t ks_basebit; /* log2 of the key-switch base                    */
} orc_params;

/* Gate opcodes (the boolean gates the paper evaluates, section II-A, and
 * the negated-input and majority gates of TFHE's gate set). */
enum { ORC_NAND = 0, ORC_AND = 1, ORC_OR = 2, ORC_XOR = 3, ORC_NOR = 4, ORC_XNOR = 5,
       ORC_MAJ = 6, ORC_ANDNY = 7, ORC_ANDYN = 8, ORC_ORNY = 9, ORC_ORYN = 10 };

#define ORC_MU (UINT32_C(1) << 29) /* 1/8 on the torus */

/* ------------------------------------------------------------------ */
/* Polynomial arithmetic in T_N[X] = T[X]/(X^N + 1)                     */
/* ------------------------------------------------------------------ */

/* out = a * b in Z[X]/(X^N+1), coefficients mod 2^32.
 * Definition: the term a_i b_j X^(i+j) lands on X^(i+j) when i+j < N and,
 * because X^N = -1, on -X^(i+j-N) otherwise.  a is any integer polynomial
 * (digits, key bits), b a torus polynomial. */
void orc_negacyclic_mul(int32_t N, const int32_t *a, const uint32_t *b, uint32_t *out)
{
    for (int32_t k = 0; k < N; k++)
        out[k] = 0;
    for (int32_t i = 0; i < N; i++) {
        uint32_t ai = (uint32_t)a[i];
        for (int32_t j = 0; j < N - i; j++)      /* i + j <  N: +X^(i+j)   */
            out[i + j] += ai * b[j];
        for (int32_t j = N - i; j < N; j++)      /* i + j >= N: -X^(i+j-N) */
            out[i + j - N] -= ai * b[j];
    }
}

/* out = X^k * p for k in [0, 2N); X^N = -1 so X^(2N) = 1. */
void orc_mul_by_xk(int32_t N, const uint32_t *p, int32_t k, uint32_t *out)
{
    k %= 2 * N;
    if (k < 0)
        k += 2 * N;
    for (int32_t i = 0; i < N; i++) {
        int32_t e = i + k;               /* exponent of the moved term */
        uint32_t v = p[i];
        while (e >= N) {                 /* each wrap multiplies by -1 */
            e -= N;
            v = (uint32_t)0 - v;
        }
        out[e] = v;
    }
}

/* ------------------------------------------------------------------ */
/* Rounding and gadget decomposition                                    */
/* ------------------------------------------------------------------ */

/* Round a torus element to the nearest multiple of 1/2^bits (ties up) and
 * return that multiple as an integer mod 2^bits.  Written as the real-number
 * definition floor(x * 2^bits / 2^32 + 1/2) in 64-bit integers. */
static uint32_t orc_round_to_bits(uint32_t x, int32_t bits)
{
    uint64_t scaled = (uint64_t)x << bits;            /* x * 2^bits (exact)   */
    uint64_t r = (scaled + (UINT64_C(1) << 31)) >> 32; /* + 1/2, floor        */
    return (uint32_t)(r & ((UINT64_C(1) << bits) - 1));
}

/* Mod switch: abar = round(x * 2N) mod 2N, N a power of two. */
int32_t orc_modswitch(int32_t N, uint32_t x)
{
    int32_t bits = 0;
    while ((1 << bits) < 2 * N)
        bits++;
    return (int32_t)orc_round_to_bits(x, bits);
}

/* Signed gadget decomposition of one torus element: digits d_0..d_{l-1} in
 * [-Bg/2, Bg/2) with sum_j d_j / Bg^(j+1) the closest multiple of 1/Bg^l to
 * x (ties up), modulo 1.  Textbook balanced-digit extraction: round, then
 * peel base-Bg digits from the least significant end, moving any digit
 * >= Bg/2 down by Bg with a carry into the next digit (the carry out of the
 * top digit is a whole torus turn and vanishes). */
void orc_decompose(int32_t bg_bit, int32_t l, uint32_t x, int32_t *d)
{
    int64_t bg = (int64_t)1 << bg_bit;
    int64_t w = orc_round_to_bits(x, bg_bit * l);   /* integer in [0, Bg^l) */
    for (int32_t j = l - 1; j >= 0; j--) {
        int64_t r = w % bg;
        w /= bg;
        if (r >= bg / 2) {
            r -= bg;
            w += 1;
        }
        d[j] = (int32_t)r;
    }
}

/* Vector form for tests. */
void orc_decompose_many(int32_t bg_bit, int32_t l, const uint32_t *x, int64_t count, int32_t *d)
{
    for (int64_t i = 0; i < count; i++)
        orc_decompose(bg_bit, l, x[i], d + i * l);
}

void orc_modswitch_many(int32_t N, const uint32_t *x, int64_t count, int32_t *out)
{
    for (int64_t i = 0; i < count; i++)
        out[i] = orc_modswitch(N, x[i]);
}

/* ------------------------------------------------------------------ */
/* LWE / TLWE encryption (client side) -- section II-A                   */
/* ------------------------------------------------------------------ */

/* ct = (A, B), B = A.S + mu + e.  ct has n + 1 words, B last. */
void orc_lwe_encrypt(int32_t n, const int32_t *s, const uint32_t *mask, int32_t noise,
                     uint32_t mu, uint32_t *ct)
{
    uint32_t b = mu + (uint32_t)noise;
    for (int32_t i = 0; i < n; i++) {
        ct[i] = mask[i];
        b += mask[i] * (uint32_t)s[i];
    }
    ct[n] = b;
}

/* phase(A, B) = B - A.S (as a torus element). */
uint32_t orc_lwe_phase(int32_t n, const int32_t *s, const uint32_t *ct)
{
    uint32_t ph = ct[n];
    for (int32_t i = 0; i < n; i++)
        ph -= ct[i] * (uint32_t)s[i];
    return ph;
}

/* Batch forms.  cts is [count][n+1]. */
void orc_lwe_encrypt_bits(int32_t n, const int32_t *s, int64_t count, const uint32_t *masks,
                          const int32_t *noise, const uint8_t *bits, uint32_t *cts)
{
    for (int64_t g = 0; g < count; g++)
        orc_lwe_encrypt(n, s, masks + g * n, noise[g],
                        bits[g] ? ORC_MU : (uint32_t)0 - ORC_MU, cts + g * (n + 1));
}

void orc_lwe_phase_many(int32_t n, const int32_t *s, int64_t count, int64_t stride,
                        const uint32_t *cts, uint32_t *phase)
{
    for (int64_t g = 0; g < count; g++)
        phase[g] = orc_lwe_phase(n, s, cts + g * stride);
}

/* Bootstrapping key: BK[i][r][p][N], i < n, r = c*l + j over the 2l rows of a
 * TGSW sample (c = 0 mask part, c = 1 body part, j = gadget level), p = 0 for
 * the TLWE mask polynomial a(X), p = 1 for the body b(X).
 * Row r is a TLWE encryption of 0 under S(X) -- a(X) = mask, b(X) = a*S + e
 * -- to which s_i * h_j, h_j = 1/Bg^(j+1), is added on polynomial c
 * (a TGSW encryption of the constant polynomial s_i). */
void orc_keygen_bk(const orc_params *P, const int32_t *s, const int32_t *S,
                   const uint32_t *masks, const int32_t *noise, uint32_t *bk)
{
    const int32_t n = P->n, N = P->N, rows = 2 * P->l;
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; i++) {
        for (int32_t r = 0; r < rows; r++) {
            const uint32_t *a = masks + ((int64_t)i * rows + r) * N;
            const int32_t *e = noise + ((int64_t)i * rows + r) * N;
            uint32_t *ra = bk + (((int64_t)i * rows + r) * 2 + 0) * N;
            uint32_t *rb = bk + (((int64_t)i * rows + r) * 2 + 1) * N;
            orc_negacyclic_mul(N, S, a, rb);          /* b = S * a         */
            for (int32_t k = 0; k < N; k++) {
                rb[k] += (uint32_t)e[k];               /*   + e             */
                ra[k] = a[k];
            }
            int32_t c = r / P->l, j = r % P->l;
            uint32_t h = (uint32_t)1 << (32 - P->bg_bit * (j + 1));
            uint32_t *target = (c == 0) ? ra : rb;
            target[0] += (uint32_t)s[i] * h;           /* + s_i * h_j       */
        }
    }
}

/* Key-switching key: KSK[j][q][d-1][n+1] for j < N, q < t, d in 1..base-1:
 * an LWE encryption under s of d * S_j / base^(q+1).  Digit 0 would be the
 * encryption of 0 and is never read, so it is not stored. */
void orc_keygen_ksk(const orc_params *P, const int32_t *s, const int32_t *S,
                    const uint32_t *masks, const int32_t *noise, uint32_t *ksk)
{
    const int32_t n = P->n, N = P->N, t = P->ks_t, bb = P->ks_basebit;
    const int32_t nd = (1 << bb) - 1;
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < N; j++)
        for (int32_t q = 0; q < t; q++)
            for (int32_t d = 1; d <= nd; d++) {
                int64_t row = ((int64_t)j * t + q) * nd + (d - 1);
                uint32_t msg = (uint32_t)d * (uint32_t)S[j] * ((uint32_t)1 << (32 - bb * (q + 1)));
                orc_lwe_encrypt(n, s, masks + row * n, noise[row], msg, ksk + row * (n + 1));
            }
}

/* ------------------------------------------------------------------ */
/* Gate bootstrapping                                                   */
/* ------------------------------------------------------------------ */

/* Linear part of a bootstrapped gate under the encoding bit 1 -> +1/8,
 * bit 0 -> -1/8: c = (0, mu_g) + alpha_a ca + alpha_b cb (+ cc for MAJ).
 * The sign of the phase of c is the gate's truth value before the
 * bootstrap re-encrypts it: e.g. AND has phase -1/8 + a + b, positive only
 * for a = b = +1/8; a negated input enters with the opposite sign (NOT x
 * has phase -x); MAJ sums three +-1/8 phases, positive iff two or three
 * inputs are 1. */
static void gate_linear(int32_t op, uint32_t *mu, int32_t *alpha_a, int32_t *alpha_b)
{
    switch (op) {
    case ORC_NAND:  *mu = ORC_MU;                   *alpha_a = -1; *alpha_b = -1; break;
    case ORC_AND:   *mu = (uint32_t)0 - ORC_MU;     *alpha_a = 1;  *alpha_b = 1;  break;
    case ORC_OR:    *mu = ORC_MU;                   *alpha_a = 1;  *alpha_b = 1;  break;
    case ORC_XOR:   *mu = 2 * ORC_MU;               *alpha_a = 2;  *alpha_b = 2;  break;
    case ORC_NOR:   *mu = (uint32_t)0 - ORC_MU;     *alpha_a = -1; *alpha_b = -1; break;
    case ORC_XNOR:  *mu = (uint32_t)0 - 2 * ORC_MU; *alpha_a = -2; *alpha_b = -2; break;
    case ORC_MAJ:   *mu = 0;                        *alpha_a = 1;  *alpha_b = 1;  break;
    case ORC_ANDNY: *mu = (uint32_t)0 - ORC_MU;     *alpha_a = -1; *alpha_b = 1;  break;
    case ORC_ANDYN: *mu = (uint32_t)0 - ORC_MU;     *alpha_a = 1;  *alpha_b = -1; break;
    case ORC_ORNY:  *mu = ORC_MU;                   *alpha_a = -1; *alpha_b = 1;  break;
    default:        *mu = ORC_MU;                   *alpha_a = 1;  *alpha_b = -1; break; /* ORYN */
    }
}

void orc_gate_combine(int32_t n, int32_t op, const uint32_t *ca, const uint32_t *cb, uint32_t *out)
{
    uint32_t mu;
    int32_t aa, ab;
    gate_linear(op, &mu, &aa, &ab);
    for (int32_t i = 0; i <= n; i++)
        out[i] = (uint32_t)aa * ca[i] + (uint32_t)ab * cb[i];
    out[n] += mu;
}

/* Three-input combine: MAJ(a, b, c) has linear part ca + cb + cc. */
void orc_gate_combine3(int32_t n, int32_t op, const uint32_t *ca, const uint32_t *cb,
                       const uint32_t *cc, uint32_t *out)
{
    orc_gate_combine(n, op, ca, cb, out);
    for (int32_t i = 0; i <= n; i++)
        out[i] += cc[i];
}

/* Blind rotation.  abar[0..n-1] are the mod-switched mask words, abar[n] the
 * mod-switched body.  acc starts as the trivial TLWE sample
 * (0, X^(-bbar) * v), v = mu * (1 + X + ... + X^(N-1)); then for every i a
 * CMux with BK_i replaces acc by acc + BK_i [x] (X^(abar_i) * acc - acc),
 * where [x] is the external product: decompose both polynomials of the TLWE
 * sample into l signed digit polynomials each and sum digit(r) * BK_i[r].
 * acc is [2][N]: acc[0] = a(X), acc[1] = b(X). */
void orc_blind_rotate(const orc_params *P, const uint32_t *bk, const int32_t *abar,
                      uint32_t mu, uint32_t *acc)
{
    const int32_t n = P->n, N = P->N, l = P->l, rows = 2 * l;
    uint32_t *v = malloc(sizeof(uint32_t) * N);
    uint32_t *rot = malloc(sizeof(uint32_t) * N);
    uint32_t *diff = malloc(sizeof(uint32_t) * 2 * N);
    int32_t *dig = malloc(sizeof(int32_t) * rows * N);
    int32_t *tmpd = malloc(sizeof(int32_t) * l);
    uint32_t *prod = malloc(sizeof(uint32_t) * N);

    for (int32_t k = 0; k < N; k++) {
        v[k] = mu;
        acc[k] = 0;
    }
    orc_mul_by_xk(N, v, 2 * N - abar[n], acc + N);

    for (int32_t i = 0; i < n; i++) {
        /* diff = X^(abar_i) * acc - acc, both polynomials */
        for (int32_t c = 0; c < 2; c++) {
            orc_mul_by_xk(N, acc + c * N, abar[i], rot);
            for (int32_t k = 0; k < N; k++)
                diff[c * N + k] = rot[k] - acc[c * N + k];
        }
        /* digit polynomials: row r = c*l + j holds digit j of polynomial c */
        for (int32_t c = 0; c < 2; c++)
            for (int32_t k = 0; k < N; k++) {
                orc_decompose(P->bg_bit, l, diff[c * N + k], tmpd);
                for (int32_t j = 0; j < l; j++)
                    dig[(c * l + j) * N + k] = tmpd[j];
            }
        /* acc += sum_r digit_r * BK_i[r]  (both output polynomials) */
        for (int32_t p = 0; p < 2; p++)
            for (int32_t r = 0; r < rows; r++) {
                const uint32_t *row = bk + (((int64_t)i * rows + r) * 2 + p) * N;
                orc_negacyclic_mul(N, dig + r * N, row, prod);
                for (int32_t k = 0; k < N; k++)
                    acc[p * N + k] += prod[k];
            }
    }
    free(v); free(rot); free(diff); free(dig); free(tmpd); free(prod);
}

/* Sample extraction of coefficient 0: the TLWE sample (a, b) under S(X) has
 * phase_0 = b_0 - (a*S)_0 = b_0 - a_0 S_0 + sum_{j>=1} a_(N-j) S_j, so the LWE
 * sample under the coefficient vector of S is a'_0 = a_0, a'_j = -a_(N-j),
 * b' = b_0.  out has N + 1 words. */
void orc_sample_extract(int32_t N, const uint32_t *acc, uint32_t *out)
{
    out[0] = acc[0];
    for (int32_t j = 1; j < N; j++)
        out[j] = (uint32_t)0 - acc[N - j];
    out[N] = acc[N];
}

/* Key switching LWE_N -> LWE_n: round every a'_j to t*basebit bits, write it
 * in base 2^basebit with digit q of weight 1/base^(q+1), and subtract the
 * key-switching samples selected by the digits from the trivial (0, b'). */
void orc_keyswitch(const orc_params *P, const uint32_t *ksk, const uint32_t *in, uint32_t *out)
{
    const int32_t n = P->n, N = P->N, t = P->ks_t, bb = P->ks_basebit;
    const int32_t nd = (1 << bb) - 1;
    for (int32_t i = 0; i < n; i++)
        out[i] = 0;
    out[n] = in[N];
    for (int32_t j = 0; j < N; j++) {
        uint32_t w = orc_round_to_bits(in[j], t * bb);
        for (int32_t q = 0; q < t; q++) {
            int32_t d = (int32_t)((w >> (bb * (t - 1 - q))) & (uint32_t)nd);
            if (d == 0)
                continue;                       /* KSK of digit 0 is zero */
            const uint32_t *row = ksk + (((int64_t)j * t + q) * nd + (d - 1)) * (n + 1);
            for (int32_t i = 0; i <= n; i++)
                out[i] -= row[i];
        }
    }
}

/* Bootstrap of one LWE_n sample with output message +-mu: mod switch, blind
 * rotate, extract, key switch.  in and out have n + 1 words. */
void orc_bootstrap(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                   const uint32_t *in, uint32_t mu, uint32_t *out)
{
    const int32_t n = P->n, N = P->N;
    int32_t *abar = malloc(sizeof(int32_t) * (n + 1));
    uint32_t *acc = malloc(sizeof(uint32_t) * 2 * N);
    uint32_t *big = malloc(sizeof(uint32_t) * (N + 1));
    for (int32_t i = 0; i <= n; i++)
        abar[i] = orc_modswitch(N, in[i]);
    orc_blind_rotate(P, bk, abar, mu, acc);
    orc_sample_extract(N, acc, big);
    orc_keyswitch(P, ksk, big, out);
    free(abar); free(acc); free(big);
}

/* One bootstrapped gate. */
void orc_gate(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t op,
              const uint32_t *ca, const uint32_t *cb, uint32_t *out)
{
    uint32_t *c = malloc(sizeof(uint32_t) * (P->n + 1));
    orc_gate_combine(P->n, op, ca, cb, c);
    orc_bootstrap(P, bk, ksk, c, ORC_MU, out);
    free(c);
}

/* One bootstrapped 3-input gate (MAJ). */
void orc_gate3(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t op,
               const uint32_t *ca, const uint32_t *cb, const uint32_t *cc, uint32_t *out)
{
    uint32_t *c = malloc(sizeof(uint32_t) * (P->n + 1));
    orc_gate_combine3(P->n, op, ca, cb, cc, c);
    orc_bootstrap(P, bk, ksk, c, ORC_MU, out);
    free(c);
}

/* Independent gates; ca/cb/out are [count][n+1].  Threads over gates. */
void orc_gates(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int64_t count,
               const uint8_t *ops, const uint32_t *ca, const uint32_t *cb, uint32_t *out,
               int32_t nthreads)
{
    const int64_t w = P->n + 1;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t g = 0; g < count; g++)
        orc_gate(P, bk, ksk, ops[g], ca + g * w, cb + g * w, out + g * w);
}

/* Batch of bootstraps of given LWE_n samples (no gate combine). */
void orc_bootstrap_many(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int64_t count,
                        const uint32_t *in, uint32_t mu, uint32_t *out, int32_t nthreads)
{
    const int64_t w = P->n + 1;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t g = 0; g < count; g++)
        orc_bootstrap(P, bk, ksk, in + g * w, mu, out + g * w);
}

/* Stage-by-stage batch entry points, so each stage can be pinned alone. */
void orc_blind_rotate_many(const orc_params *P, const uint32_t *bk, int64_t count,
                           const int32_t *abar, uint32_t mu, uint32_t *acc, int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t g = 0; g < count; g++)
        orc_blind_rotate(P, bk, abar + g * (P->n + 1), mu, acc + g * 2 * P->N);
}

void orc_keyswitch_many(const orc_params *P, const uint32_t *ksk, int64_t count,
                        const uint32_t *in, uint32_t *out)
{
    for (int64_t g = 0; g < count; g++)
        orc_keyswitch(P, ksk, in + g * (P->N + 1), out + g * (P->n + 1));
}

/* ------------------------------------------------------------------ */
/* Boolean circuits over encrypted integers (bit 0 = least significant) */
/* ------------------------------------------------------------------ */

/* Ciphertext rows of one evaluation (gate outputs and temporaries, n + 1
 * words each).  A row is freed only when the whole evaluation -- every gate
 * task that may read or write it -- has finished. */
typedef struct {
    uint32_t **buf;
    int64_t n, cap, words;
} orc_arena;

/* `rows` consecutive rows in one block. */
static uint32_t *arena_rows(orc_arena *A, int64_t rows)
{
    if (A->n == A->cap) {
        A->cap = A->cap ? 2 * A->cap : 64;
        A->buf = realloc(A->buf, sizeof(uint32_t *) * A->cap);
    }
    return A->buf[A->n++] = malloc(sizeof(uint32_t) * A->words * rows);
}

static uint32_t *arena_new(orc_arena *A)
{
    return arena_rows(A, 1);
}

static void arena_free(orc_arena *A)
{
    for (int64_t i = 0; i < A->n; i++)
        free(A->buf[i]);
    free(A->buf);
}

typedef struct {
    const orc_params *P;
    const uint32_t *bk, *ksk;
    int64_t gates;      /* bootstraps performed, for accounting */
    orc_arena A;        /* every row the circuit allocates */
} orc_ev;

/* Order of evaluation.  Each gate (and each copy of a row) is an OpenMP task
 * that names the rows it reads in depend(in) and the row it writes in
 * depend(out), each row by its first word; rows never overlap partially.
 * OpenMP then runs a task only after every earlier-created task that writes
 * a row it reads, or reads or writes the row it writes, so the result is
 * that of evaluating the gates one by one in the order the circuit code
 * creates them (each ciphertext is a deterministic function of its gate's
 * inputs), while independent gates of a circuit run on different threads.
 * Without OpenMP the pragmas are ignored and the gates run in that order.
 * The circuit functions below only build the task graph; the batched entry
 * points at the end run it. */
static void ev_gate(orc_ev *E, int32_t op, const uint32_t *a, const uint32_t *b, uint32_t *out)
{
    const orc_params *P = E->P;
    const uint32_t *bk = E->bk, *ksk = E->ksk;
#pragma omp task default(none) firstprivate(P, bk, ksk, op, a, b, out) \
    depend(in : a[0], b[0]) depend(out : out[0])
    orc_gate(P, bk, ksk, op, a, b, out);
    E->gates++;
}

static void ev_gate3(orc_ev *E, int32_t op, const uint32_t *a, const uint32_t *b,
                     const uint32_t *c, uint32_t *out)
{
    const orc_params *P = E->P;
    const uint32_t *bk = E->bk, *ksk = E->ksk;
#pragma omp task default(none) firstprivate(P, bk, ksk, op, a, b, c, out) \
    depend(in : a[0], b[0], c[0]) depend(out : out[0])
    orc_gate3(P, bk, ksk, op, a, b, c, out);
    E->gates++;
}

/* Row out = row in. */
static void ev_copy(orc_ev *E, const uint32_t *in, uint32_t *out)
{
    const size_t bytes = sizeof(uint32_t) * (size_t)(E->P->n + 1);
#pragma omp task default(none) firstprivate(bytes, in, out) depend(in : in[0]) depend(out : out[0])
    memcpy(out, in, bytes);
}

/* Row out = the trivial sample (0, ..., 0, -1/8) of a constant-0 bit. */
static void ev_const0(orc_ev *E, uint32_t *out)
{
    const int32_t n = E->P->n;
#pragma omp task default(none) firstprivate(n, out) depend(out : out[0])
    {
        memset(out, 0, sizeof(uint32_t) * (size_t)(n + 1));
        out[n] = (uint32_t)0 - ORC_MU;
    }
}

static int32_t ev_threads(int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#endif
    return nthreads > 0 ? nthreads : 1;
}

static orc_ev *ev_new_many(const orc_params *P, const uint32_t *bk, const uint32_t *ksk,
                           int64_t count)
{
    orc_ev *E = calloc(count > 0 ? count : 1, sizeof(orc_ev));
    for (int64_t i = 0; i < count; i++) {
        E[i].P = P;
        E[i].bk = bk;
        E[i].ksk = ksk;
        E[i].A.words = P->n + 1;
    }
    return E;
}

/* After the tasks have finished: total gates, rows freed. */
static int64_t ev_free_many(orc_ev *E, int64_t count)
{
    int64_t total = 0;
    for (int64_t i = 0; i < count; i++) {
        total += E[i].gates;
        arena_free(&E[i].A);
    }
    free(E);
    return total;
}

/* w-bit ripple-carry addition mod 2^w (sections III-A, V-B-1):
 *   r_i = a_i XOR b_i XOR c_(i-1)                          (Eq. addres)
 *   c_i = (a_i AND b_i) OR ((a_i XOR b_i) AND c_(i-1))     (Eq. addcarry)
 * with no carry into bit 0 (so r_0 = a_0 XOR b_0, c_0 = a_0 AND b_0) and no
 * carry out of bit w-1 (the sum is truncated to w bits).  A, B, R are
 * [w][n+1]; R may alias neither input. */
static void ev_add(orc_ev *E, int32_t w, const uint32_t *A, const uint32_t *B, uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    uint32_t *x = arena_new(&E->A), *g = arena_new(&E->A);
    uint32_t *t = arena_new(&E->A), *c = arena_new(&E->A);
    for (int32_t i = 0; i < w; i++) {
        const uint32_t *ai = A + i * W, *bi = B + i * W;
        uint32_t *ri = R + i * W;
        if (i == 0) {
            ev_gate(E, ORC_XOR, ai, bi, ri);
            if (w > 1)
                ev_gate(E, ORC_AND, ai, bi, c);
            continue;
        }
        ev_gate(E, ORC_XOR, ai, bi, x);
        ev_gate(E, ORC_XOR, x, c, ri);
        if (i == w - 1)
            break;                                  /* carry out discarded */
        ev_gate(E, ORC_AND, ai, bi, g);
        ev_gate(E, ORC_AND, x, c, t);
        ev_gate(E, ORC_OR, g, t, c);
    }
}

/* w x w -> w truncated naive multiplication (section III-B-1): partial
 * product i is A AND b_i shifted left by i; the shifted partial products are
 * accumulated one after another with ripple-carry adders.  Only bits below w
 * are formed.  acc starts as partial product 0; partial product i is then
 * added into bits i..w-1 with a (w-i)-bit adder. */
static void ev_mul(orc_ev *E, int32_t w, const uint32_t *A, const uint32_t *B, uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    uint32_t *pp = arena_rows(&E->A, w);
    uint32_t *sum = arena_rows(&E->A, w);
    for (int32_t j = 0; j < w; j++)                 /* partial product 0 */
        ev_gate(E, ORC_AND, A + j * W, B, R + j * W);
    for (int32_t i = 1; i < w; i++) {
        int32_t m = w - i;
        for (int32_t j = 0; j < m; j++)             /* a_j AND b_i, weight i+j */
            ev_gate(E, ORC_AND, A + j * W, B + i * W, pp + j * W);
        ev_add(E, m, R + i * W, pp, sum);
        for (int32_t j = 0; j < m; j++)
            ev_copy(E, sum + j * W, R + (i + j) * W);
    }
}

/* Matrix-vector product y_r = sum_c M[r][c] * v[c] mod 2^w (section IV-D:
 * every product independent, each output an accumulation).  The products of
 * one row are reduced by the tree-based accumulation of section V-B-2: at
 * every level neighbours (0,1), (2,3), ... are added and an odd last element
 * moves up unchanged, until one number is left.  M is [rows][cols][w][n+1],
 * v is [cols][w][n+1], Y is [rows][w][n+1]. */
static void ev_matvec_row(orc_ev *E, int32_t w, int32_t cols, const uint32_t *Mrow,
                          const uint32_t *v, uint32_t *Y)
{
    const int64_t W = E->P->n + 1, num = W * w;
    uint32_t *terms = arena_rows(&E->A, (int64_t)cols * w);
    uint32_t *next = arena_rows(&E->A, (int64_t)cols * w);
    for (int32_t c = 0; c < cols; c++)
        ev_mul(E, w, Mrow + c * num, v + c * num, terms + c * num);
    int32_t cnt = cols;
    while (cnt > 1) {
        int32_t k = 0;
        for (int32_t i = 0; i + 1 < cnt; i += 2, k++)
            ev_add(E, w, terms + i * num, terms + (i + 1) * num, next + k * num);
        if (cnt & 1) {
            for (int32_t j = 0; j < w; j++)
                ev_copy(E, terms + (cnt - 1) * num + j * W, next + k * num + j * W);
            k++;
        }
        for (int64_t j = 0; j < (int64_t)k * w; j++)
            ev_copy(E, next + j * W, terms + j * W);
        cnt = k;
    }
    for (int32_t j = 0; j < w; j++)
        ev_copy(E, terms + j * W, Y + j * W);
}

/* In the circuits below a wire may be the constant 0 (NULL), and every gate
 * output gets a fresh row from the evaluation's arena. */

/* One adder position with operands x, y and incoming carry c, any of which
 * may be the constant 0 (NULL).  Only the live operands are combined: one
 * live operand is the sum itself; two give a half adder (sum XOR, carry
 * AND); three give a full adder -- sum (x XOR y) XOR c, and carry either
 * (x AND y) OR ((x XOR y) AND c) (Eq. "addcarry") or MAJ(x, y, c).  The
 * carry is formed only when need_carry is set. */
static void ev_cell(orc_ev *E, orc_arena *A, const uint32_t *x, const uint32_t *y,
                    const uint32_t *c, int need_carry, int maj, const uint32_t **sum,
                    const uint32_t **carry)
{
    const uint32_t *live[3];
    int k = 0;
    if (x) live[k++] = x;
    if (y) live[k++] = y;
    if (c) live[k++] = c;
    *sum = NULL;
    *carry = NULL;
    if (k == 1) {
        *sum = live[0];
    } else if (k == 2) {
        uint32_t *s = arena_new(A);
        ev_gate(E, ORC_XOR, live[0], live[1], s);
        *sum = s;
        if (need_carry) {
            uint32_t *co = arena_new(A);
            ev_gate(E, ORC_AND, live[0], live[1], co);
            *carry = co;
        }
    } else if (k == 3) {
        uint32_t *p = arena_new(A), *s = arena_new(A);
        ev_gate(E, ORC_XOR, x, y, p);
        ev_gate(E, ORC_XOR, p, c, s);
        *sum = s;
        if (need_carry) {
            uint32_t *co = arena_new(A);
            if (maj) {
                ev_gate3(E, ORC_MAJ, x, y, c, co);
            } else {
                uint32_t *g = arena_new(A), *t = arena_new(A);
                ev_gate(E, ORC_AND, x, y, g);
                ev_gate(E, ORC_AND, p, c, t);
                ev_gate(E, ORC_OR, g, t, co);
            }
            *carry = co;
        }
    }
}

/* w-bit sum mod 2^w of wire vectors with constant-zero entries. */
static void ev_add_cells(orc_ev *E, orc_arena *A, int32_t w, const uint32_t **x,
                         const uint32_t **y, int maj, const uint32_t **r)
{
    const uint32_t *c = NULL;
    for (int32_t i = 0; i < w; i++)
        ev_cell(E, A, x[i], y[i], c, i < w - 1, maj, &r[i], &c);
}

static void copy_out(orc_ev *E, int32_t w, const uint32_t **r, uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    for (int32_t i = 0; i < w; i++)
        ev_copy(E, r[i], R + i * W);
}

/* Ripple adder whose carries are single majority gates. */
static void ev_add_maj(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv, uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    orc_arena *A = &E->A;
    const uint32_t **x = malloc(sizeof(*x) * w), **y = malloc(sizeof(*y) * w),
                   **r = malloc(sizeof(*r) * w);
    for (int32_t i = 0; i < w; i++) {
        x[i] = Av + i * W;
        y[i] = Bv + i * W;
    }
    ev_add_cells(E, A, w, x, y, 1, r);
    copy_out(E, w, r, R);
    free(x); free(y); free(r);
}

/* The paper's number-wise addition GPU_n (section V-B-1): R = A; then w
 * times C = R AND B, R = R XOR B, B = C << 1, on every bit at once.  Bits of
 * B that are the constant 0 (shifted in) leave R unchanged and give no
 * carry; the carry out of the top bit is dropped. */
static void ev_add_nw(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv, uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    orc_arena *A = &E->A;
    const uint32_t **r = malloc(sizeof(*r) * w), **b = malloc(sizeof(*b) * w),
                   **nb = malloc(sizeof(*nb) * w);
    for (int32_t i = 0; i < w; i++) {
        r[i] = Av + i * W;
        b[i] = Bv + i * W;
    }
    for (int32_t k = 0; k < w; k++) {
        for (int32_t i = 0; i < w; i++)
            nb[i] = NULL;
        for (int32_t i = 0; i < w; i++) {
            if (!b[i])
                continue;
            uint32_t *nr = arena_new(A);
            if (i + 1 < w) {
                uint32_t *cy = arena_new(A);
                ev_gate(E, ORC_AND, r[i], b[i], cy);
                nb[i + 1] = cy;
            }
            ev_gate(E, ORC_XOR, r[i], b[i], nr);
            r[i] = nr;
        }
        for (int32_t i = 0; i < w; i++)
            b[i] = nb[i];
    }
    copy_out(E, w, r, R);
    free(r); free(b); free(nb);
}

/* Truncated multiplication with tree-based accumulation (section V-B-2):
 * partial product i is A AND b_i shifted left by i (its low i bits the
 * constant 0); the w partial products are added pairwise, (0,1), (2,3),
 * ..., an odd last one moving up unchanged, until one is left.  The adders
 * carry by Eq. "addcarry" (maj = 0) or by single majority gates (maj = 1). */
static void ev_mul_tree_with(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv,
                             uint32_t *R, int maj)
{
    const int64_t W = E->P->n + 1;
    orc_arena *A = &E->A;
    const uint32_t **terms = malloc(sizeof(*terms) * w * w), **next = malloc(sizeof(*next) * w * w);
    for (int32_t i = 0; i < w; i++)
        for (int32_t j = 0; j < w; j++) {
            uint32_t *pp = NULL;
            if (j >= i) {
                pp = arena_new(A);
                ev_gate(E, ORC_AND, Av + (j - i) * W, Bv + i * W, pp);
            }
            terms[i * w + j] = pp;
        }
    int32_t cnt = w;
    while (cnt > 1) {
        int32_t k = 0;
        for (int32_t i = 0; i + 1 < cnt; i += 2, k++)
            ev_add_cells(E, A, w, terms + i * w, terms + (i + 1) * w, maj, next + k * w);
        if (cnt & 1) {
            memcpy(next + k * w, terms + (cnt - 1) * w, sizeof(*terms) * w);
            k++;
        }
        memcpy(terms, next, sizeof(*terms) * w * k);
        cnt = k;
    }
    copy_out(E, w, terms, R);
    free(terms); free(next);
}

static void ev_mul_tree(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv, uint32_t *R)
{
    ev_mul_tree_with(E, w, Av, Bv, R, 0);
}

static void ev_mul_tree_maj(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv,
                            uint32_t *R)
{
    ev_mul_tree_with(E, w, Av, Bv, R, 1);
}

/* Sklansky parallel-prefix addition of wire vectors (NULL = constant 0),
 * w bits mod 2^w, with majority gates.  Per bit i: g_i = x_i AND y_i (bits
 * below w-1: there is no carry out), k_i = x_i OR y_i (bits 1 .. w-2: the
 * group holding bit 0 never needs K) and p_i = x_i XOR y_i; with one operand
 * the constant 0, g_i = 0 and k_i, p_i are the other operand.  For a group of bits, G says it produces a carry
 * and K says it produces or passes one (G implies K); putting a high group
 * on top of a low one gives G = MAJ(G_hi, K_hi, G_lo) and
 * K = MAJ(G_hi, K_hi, K_lo), since G_hi OR (K_hi AND L) is the majority of
 * the three when G_hi implies K_hi.  For span = 1, 2, 4, ... while
 * span < w - 1, every bit i <= w - 2 in the upper half of its block of
 * 2 span bits takes in the group ending at the lower half's top bit j; K is
 * updated only where the merged group does not reach bit 0 (i >= 2 span).
 * A merge with a constant-0 low signal or K_hi keeps G_hi; with G_hi the
 * constant 0 it is K_hi AND low.  Then s_0 = p_0 and s_i = p_i XOR G_(i-1),
 * without a gate when one side is the constant 0.  This is the gate list
 * the CUDA library's netlist builds (the circuit is defined gate for gate). */
static const uint32_t *ev_merge(orc_ev *E, orc_arena *A, const uint32_t *g_hi,
                                const uint32_t *k_hi, const uint32_t *lo)
{
    if (!lo || !k_hi)
        return g_hi;
    uint32_t *o = arena_new(A);
    if (!g_hi) {
        ev_gate(E, ORC_AND, k_hi, lo, o);
    } else {
        ev_gate3(E, ORC_MAJ, g_hi, k_hi, lo, o);
    }
    return o;
}

static void ev_prefix_cells(orc_ev *E, orc_arena *A, int32_t w, const uint32_t **x,
                            const uint32_t **y, const uint32_t **s)
{
    const uint32_t **g = calloc(w, sizeof(*g)), **kk = calloc(w, sizeof(*kk));
    const uint32_t **bitp = calloc(w, sizeof(*bitp));
    const uint32_t **ng = calloc(w, sizeof(*ng)), **nk = calloc(w, sizeof(*nk));
    for (int32_t i = 0; i < w; i++) {
        if (x[i] && y[i]) {
            if (i < w - 1) {
                uint32_t *o1 = arena_new(A);
                ev_gate(E, ORC_AND, x[i], y[i], o1);
                g[i] = o1;
            }
            if (i > 0 && i < w - 1) {
                uint32_t *o2 = arena_new(A);
                ev_gate(E, ORC_OR, x[i], y[i], o2);
                kk[i] = o2;
            }
            uint32_t *o = arena_new(A);
            ev_gate(E, ORC_XOR, x[i], y[i], o);
            bitp[i] = o;
        } else {
            bitp[i] = x[i] ? x[i] : y[i];
            if (i < w - 1)
                kk[i] = bitp[i];
        }
    }
    for (int32_t span = 1; span < w - 1; span *= 2) {
        memcpy(ng, g, sizeof(*g) * w);
        memcpy(nk, kk, sizeof(*kk) * w);
        for (int32_t i = 0; i <= w - 2; i++) {
            if ((i / span) % 2 == 0)
                continue;                               /* lower half: unchanged */
            const int32_t j = (i / (2 * span)) * (2 * span) + span - 1;
            ng[i] = ev_merge(E, A, g[i], kk[i], g[j]);
            if (i >= 2 * span)
                nk[i] = ev_merge(E, A, g[i], kk[i], kk[j]);
        }
        memcpy(g, ng, sizeof(*g) * w);
        memcpy(kk, nk, sizeof(*kk) * w);
    }
    for (int32_t i = 0; i < w; i++) {
        const uint32_t *c = i > 0 ? g[i - 1] : NULL;
        if (!c) {
            s[i] = bitp[i];
        } else if (!bitp[i]) {
            s[i] = c;
        } else {
            uint32_t *o = arena_new(A);
            ev_gate(E, ORC_XOR, bitp[i], c, o);
            s[i] = o;
        }
    }
    free(g); free(kk); free(bitp); free(ng); free(nk);
}

static void ev_add_prefix(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv,
                          uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    orc_arena *A = &E->A;
    const uint32_t **x = malloc(sizeof(*x) * w), **y = malloc(sizeof(*y) * w),
                   **r = malloc(sizeof(*r) * w);
    for (int32_t i = 0; i < w; i++) {
        x[i] = Av + i * W;
        y[i] = Bv + i * W;
    }
    ev_prefix_cells(E, A, w, x, y, r);
    copy_out(E, w, r, R);
    free(x); free(y); free(r);
}

/* Truncated w x w -> w multiplication by a Dadda tree.  Column c (weight
 * 2^c) begins with the partial products a_(c-i) AND b_i, i = 0 .. c, in that
 * order.  The stage targets are the numbers 2, 3, 4, 6, 9, 13, ... (each
 * the floor of 3/2 times the one before) below w, used from the largest
 * down.  A stage with target d walks the columns from c = 0 up; the height
 * of column c is its own wires plus the carries column c - 1 has already
 * sent it in this stage.  While the height exceeds d, the column's oldest
 * unused wires go into a half adder (sum u XOR v, carry u AND v) if the
 * height is d + 1, else into a full adder (sum (u XOR v) XOR z, carry
 * MAJ(u, v, z)); sums stay in column c, carries go to column c + 1 (none is
 * formed out of column w - 1).  The column's next contents are the carries
 * it received, its sums, then its unused wires, in that order.  The two
 * rows left are added by the parallel-prefix adder above.  Returns -1 if a
 * column runs out of wires (not the case for w <= 64). */
static int ev_mul_dadda_impl(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv,
                             uint32_t *R)
{
    const int64_t W = E->P->n + 1;
    const int32_t cap = 2 * w + 8;
    orc_arena *A = &E->A;
    const uint32_t **col = malloc(sizeof(*col) * w * cap), **nxt = malloc(sizeof(*nxt) * w * cap);
    int32_t *len = calloc(w, sizeof(int32_t)), *nlen = calloc(w, sizeof(int32_t));
    int32_t target[16], nt = 0, ok = 0;
    for (int32_t c = 0; c < w; c++)
        for (int32_t i = 0; i <= c; i++) {
            uint32_t *o = arena_new(A);
            ev_gate(E, ORC_AND, Av + (c - i) * W, Bv + i * W, o);
            col[c * cap + len[c]++] = o;
        }
    for (int32_t d = 2; d < w; d = d * 3 / 2)
        target[nt++] = d;
    for (int32_t t = nt - 1; t >= 0; t--) {
        const int32_t d = target[t];
        memset(nlen, 0, sizeof(int32_t) * w);
        for (int32_t c = 0; c < w; c++) {
            int32_t used = 0, h = len[c] + nlen[c];
            while (h > d) {
                const int32_t need = h == d + 1 ? 2 : 3;
                if (used + need > len[c])
                    goto done;
                const uint32_t *u = col[c * cap + used], *v = col[c * cap + used + 1];
                uint32_t *sum = arena_new(A);
                if (need == 2) {
                    ev_gate(E, ORC_XOR, u, v, sum);
                    if (c + 1 < w) {
                        uint32_t *cy = arena_new(A);
                        ev_gate(E, ORC_AND, u, v, cy);
                        nxt[(c + 1) * cap + nlen[c + 1]++] = cy;
                    }
                    h -= 1;
                } else {
                    const uint32_t *z = col[c * cap + used + 2];
                    uint32_t *uv = arena_new(A);
                    ev_gate(E, ORC_XOR, u, v, uv);
                    ev_gate(E, ORC_XOR, uv, z, sum);
                    if (c + 1 < w) {
                        uint32_t *cy = arena_new(A);
                        ev_gate3(E, ORC_MAJ, u, v, z, cy);
                        nxt[(c + 1) * cap + nlen[c + 1]++] = cy;
                    }
                    h -= 2;
                }
                nxt[c * cap + nlen[c]++] = sum;
                used += need;
            }
            for (; used < len[c]; used++)
                nxt[c * cap + nlen[c]++] = col[c * cap + used];
        }
        const uint32_t **tmp = col;
        col = nxt;
        nxt = tmp;
        int32_t *tl = len;
        len = nlen;
        nlen = tl;
    }
    {
        const uint32_t **x = calloc(w, sizeof(*x)), **y = calloc(w, sizeof(*y)),
                       **r = malloc(sizeof(*r) * w);
        int32_t fits = 1;
        for (int32_t c = 0; c < w; c++) {
            if (len[c] > 2)
                fits = 0;
            if (len[c] > 0)
                x[c] = col[c * cap];
            if (len[c] > 1)
                y[c] = col[c * cap + 1];
        }
        if (fits) {
            ev_prefix_cells(E, A, w, x, y, r);
            copy_out(E, w, r, R);
            ok = 1;
        }
        free(x); free(y); free(r);
    }
done:
    free(col); free(nxt); free(len); free(nlen);
    return ok ? 0 : -1;
}

static void ev_mul_dadda(orc_ev *E, int32_t w, const uint32_t *Av, const uint32_t *Bv,
                         uint32_t *R)
{
    /* (on failure no gate task reads or writes R, so it is cleared here) */
    if (ev_mul_dadda_impl(E, w, Av, Bv, R) != 0)
        memset(R, 0, sizeof(uint32_t) * (E->P->n + 1) * w);
}

/* Full product Z = X Y of n-bit X, Y as 2n bits (section III-B-1, "Naive
 * Approach", without truncation): partial product i is X AND y_i moved up by
 * i bits, so it covers weights i .. i+n-1 of the 2n; the n partial products
 * are then summed by the tree of section V-B-2 with 2n-bit adders. */
static void ev_full_product(orc_ev *E, orc_arena *A, int32_t n, const uint32_t **x,
                            const uint32_t **y, const uint32_t **z)
{
    const int32_t w = 2 * n;
    const uint32_t **terms = calloc((size_t)n * w, sizeof(*terms));
    const uint32_t **next = calloc((size_t)n * w, sizeof(*next));
    for (int32_t i = 0; i < n; i++)
        for (int32_t j = 0; j < n; j++) {
            uint32_t *pp = arena_new(A);
            ev_gate(E, ORC_AND, x[j], y[i], pp);
            terms[i * w + i + j] = pp;
        }
    int32_t cnt = n;
    while (cnt > 1) {
        int32_t k = 0;
        for (int32_t i = 0; i + 1 < cnt; i += 2, k++)
            ev_add_cells(E, A, w, terms + i * w, terms + (i + 1) * w, 0, next + k * w);
        if (cnt & 1) {
            memcpy(next + k * w, terms + (cnt - 1) * w, sizeof(*terms) * w);
            k++;
        }
        memcpy(terms, next, sizeof(*terms) * w * k);
        cnt = k;
    }
    memcpy(z, terms, sizeof(*terms) * w);
    free(terms); free(next);
}

/* D = S - T mod 2^L for L-bit S (every bit an encrypted wire) and m-bit T,
 * m <= L: the two's-complement form S + T' + 1 of the paper's last step of
 * the vector Karatsuba (section V-B, "Karatsuba Multiplication"), with the
 * +1 entering as the carry into bit 0 and the complement of T folded into
 * the gates, since negating a ciphertext is the free NOT of TFHE:
 *   bit 0, carry-in 1:      d = s XOR t,            carry = s OR NOT t
 *   bit i < m, carry c:     e = s XNOR t,  d = e XOR c,
 *                           carry = (s AND NOT t) OR (e AND c)
 *   bit i >= m (t' = 1):    d = s XNOR c,           carry = s OR c
 * The carry out of bit L-1 is not formed. */
static void ev_sub(orc_ev *E, orc_arena *A, int32_t L, const uint32_t **S, int32_t m,
                   const uint32_t **T, const uint32_t **D)
{
    const uint32_t *c = NULL;
    for (int32_t i = 0; i < L; i++) {
        const int carry = i < L - 1;
        uint32_t *d = arena_new(A);
        uint32_t *co = carry ? arena_new(A) : NULL;
        if (i == 0) {
            ev_gate(E, ORC_XOR, S[0], T[0], d);
            if (carry)
                ev_gate(E, ORC_ORYN, S[0], T[0], co);
        } else if (i < m) {
            uint32_t *e = arena_new(A);
            ev_gate(E, ORC_XNOR, S[i], T[i], e);
            ev_gate(E, ORC_XOR, e, c, d);
            if (carry) {
                uint32_t *g = arena_new(A), *t = arena_new(A);
                ev_gate(E, ORC_ANDYN, S[i], T[i], g);
                ev_gate(E, ORC_AND, e, c, t);
                ev_gate(E, ORC_OR, g, t, co);
            }
        } else {
            ev_gate(E, ORC_XNOR, S[i], c, d);
            if (carry)
                ev_gate(E, ORC_OR, S[i], c, co);
        }
        D[i] = d;
        c = co;
    }
}

/* Sum with carry out: R (max(lx, ly) + 1 bits) = X (lx bits) + Y (ly bits). */
static void ev_add_ext(orc_ev *E, orc_arena *A, int32_t lx, const uint32_t **X, int32_t ly,
                       const uint32_t **Y, const uint32_t **R)
{
    const int32_t L = (lx > ly ? lx : ly) + 1;
    const uint32_t **x = calloc(L, sizeof(*x)), **y = calloc(L, sizeof(*y));
    memcpy(x, X, sizeof(*x) * lx);
    memcpy(y, Y, sizeof(*y) * ly);
    ev_add_cells(E, A, L, x, y, 0, R);
    free(x); free(y);
}

/* Karatsuba multiplication (Algorithm "karatsuba", with the vector form of
 * section V-B): Z (2n bits) = X Y.  Below n0 = ORC_KARATSUBA_N0 bits the base
 * multiplication is the full product above.  Otherwise, with h = ceil(n/2):
 *   X0 = X mod 2^h, X1 = X / 2^h, Y0, Y1 likewise
 *   <Temp0, Temp1> = <X0, Y0> + <X1, Y1>            (h + 1 bits each)
 *   <Z0, Z1, Z2>   = <X0, X1, Temp0> . <Y0, Y1, Temp1>
 *   Temp1 = Z1 + Z0;  Z2 = Z2 - Temp1               (= X0 Y1 + X1 Y0)
 *   Z = Z0 + Z2 2^h + Z1 2^(2h)                    (mod 2^(2n))
 * The first and last terms do not overlap (Z0 has 2h bits), so they are
 * placed side by side and one 2n-bit addition adds the middle term. */
#define ORC_KARATSUBA_N0 8
static void ev_karatsuba(orc_ev *E, orc_arena *A, int32_t n, const uint32_t **X,
                         const uint32_t **Y, const uint32_t **Z)
{
    if (n < ORC_KARATSUBA_N0) {
        ev_full_product(E, A, n, X, Y, Z);
        return;
    }
    const int32_t h = (n + 1) / 2, m = n - h;
    const uint32_t **t0 = malloc(sizeof(*t0) * (h + 1)), **t1 = malloc(sizeof(*t1) * (h + 1));
    const uint32_t **z0 = malloc(sizeof(*z0) * 2 * h), **z1 = malloc(sizeof(*z1) * 2 * m);
    const uint32_t **z2 = malloc(sizeof(*z2) * (2 * h + 2)), **u = malloc(sizeof(*u) * (2 * h + 1));
    const uint32_t **d = malloc(sizeof(*d) * (2 * h + 2));
    const uint32_t **lo = calloc(2 * n, sizeof(*lo)), **mid = calloc(2 * n, sizeof(*mid));
    ev_add_ext(E, A, h, X, m, X + h, t0);
    ev_add_ext(E, A, h, Y, m, Y + h, t1);
    ev_karatsuba(E, A, h, X, Y, z0);
    ev_karatsuba(E, A, m, X + h, Y + h, z1);
    ev_karatsuba(E, A, h + 1, t0, t1, z2);
    ev_add_ext(E, A, 2 * h, z0, 2 * m, z1, u);
    ev_sub(E, A, 2 * h + 2, z2, 2 * h + 1, u, d);
    for (int32_t i = 0; i < 2 * h; i++)
        lo[i] = z0[i];
    for (int32_t i = 0; i < 2 * m; i++)
        lo[2 * h + i] = z1[i];
    for (int32_t i = 0; i < 2 * h + 2 && h + i < 2 * n; i++)
        mid[h + i] = d[i];
    ev_add_cells(E, A, 2 * n, lo, mid, 0, Z);
    free(t0); free(t1); free(z0); free(z1); free(z2); free(u); free(d); free(lo); free(mid);
}

typedef void (*orc_full_fn)(orc_ev *, orc_arena *, int32_t, const uint32_t **, const uint32_t **,
                            const uint32_t **);

/* Batched full products: A, B [batch][w][n+1] -> R [batch][2w][n+1].  One
 * thread builds every instance's gate tasks, the team runs them; they have
 * all finished when the parallel region ends. */
static int64_t run_full(orc_full_fn fn, const orc_params *P, const uint32_t *bk,
                        const uint32_t *ksk, int32_t w, int64_t batch, const uint32_t *Av,
                        const uint32_t *Bv, uint32_t *R, int32_t nthreads)
{
    const int64_t W = P->n + 1, num = W * w;
    orc_ev *E = ev_new_many(P, bk, ksk, batch);
    nthreads = ev_threads(nthreads);
#pragma omp parallel num_threads(nthreads)
#pragma omp single
    for (int64_t b = 0; b < batch; b++) {
        const uint32_t **x = malloc(sizeof(*x) * w), **y = malloc(sizeof(*y) * w),
                       **z = malloc(sizeof(*z) * 2 * w);
        for (int32_t i = 0; i < w; i++) {
            x[i] = Av + b * num + i * W;
            y[i] = Bv + b * num + i * W;
        }
        fn(&E[b], &E[b].A, w, x, y, z);
        for (int32_t i = 0; i < 2 * w; i++) {
            uint32_t *o = R + 2 * b * num + i * W;
            if (z[i])
                ev_copy(&E[b], z[i], o);
            else
                ev_const0(&E[b], o);   /* a constant-0 bit */
        }
        free(x); free(y); free(z);
    }
    return ev_free_many(E, batch);
}

int64_t orc_mul_full(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                     int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                     int32_t nthreads)
{
    return run_full(ev_full_product, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_mul_karatsuba(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                          int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                          int32_t nthreads)
{
    return run_full(ev_karatsuba, P, bk, ksk, w, batch, A, B, R, nthreads);
}

/* Batched circuit entry points: one thread builds the gate tasks of every
 * instance in program order and the team of nthreads threads runs them, so
 * independent gates -- of one instance or of different instances -- run in
 * parallel; they have all finished when the parallel region ends.  Return
 * the number of bootstrapped gates evaluated. */
typedef void (*orc_circuit_fn)(orc_ev *, int32_t, const uint32_t *, const uint32_t *, uint32_t *);

static int64_t run_batched(orc_circuit_fn fn, const orc_params *P, const uint32_t *bk,
                           const uint32_t *ksk, int32_t w, int64_t batch, const uint32_t *A,
                           const uint32_t *B, uint32_t *R, int32_t nthreads)
{
    const int64_t num = (int64_t)(P->n + 1) * w;
    orc_ev *E = ev_new_many(P, bk, ksk, batch);
    nthreads = ev_threads(nthreads);
#pragma omp parallel num_threads(nthreads)
#pragma omp single
    for (int64_t b = 0; b < batch; b++)
        fn(&E[b], w, A + b * num, B + b * num, R + b * num);
    return ev_free_many(E, batch);
}

int64_t orc_add(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R, int32_t nthreads)
{
    return run_batched(ev_add, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_mul(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R, int32_t nthreads)
{
    return run_batched(ev_mul, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_add_maj(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                    int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                    int32_t nthreads)
{
    return run_batched(ev_add_maj, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_add_nw(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                   int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                   int32_t nthreads)
{
    return run_batched(ev_add_nw, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_mul_tree(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                     int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                     int32_t nthreads)
{
    return run_batched(ev_mul_tree, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_mul_tree_maj(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                     int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                     int32_t nthreads)
{
    return run_batched(ev_mul_tree_maj, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_add_prefix(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                     int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                     int32_t nthreads)
{
    return run_batched(ev_add_prefix, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_mul_dadda(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                     int64_t batch, const uint32_t *A, const uint32_t *B, uint32_t *R,
                     int32_t nthreads)
{
    return run_batched(ev_mul_dadda, P, bk, ksk, w, batch, A, B, R, nthreads);
}

int64_t orc_matvec(const orc_params *P, const uint32_t *bk, const uint32_t *ksk, int32_t w,
                   int32_t rows, int32_t cols, const uint32_t *M, const uint32_t *v, uint32_t *Y,
                   int32_t nthreads)
{
    const int64_t num = (int64_t)(P->n + 1) * w;
    orc_ev *E = ev_new_many(P, bk, ksk, rows);
    nthreads = ev_threads(nthreads);
#pragma omp parallel num_threads(nthreads)
#pragma omp single
    for (int32_t r = 0; r < rows; r++)
        ev_matvec_row(&E[r], w, cols, M + (int64_t)r * cols * num, v, Y + r * num);
    return ev_free_many(E, rows);
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
