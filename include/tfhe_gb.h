/*
 * tfhe_gb.h -- C ABI of the GB300 (sm_103a) TFHE gate-bootstrapping library.
 *
 * The library evaluates TFHE boolean gates with one programmable bootstrap
 * each (the paper's section II-A and Table "differentialtime": bootstrapping
 * followed by key switching, with a bootstrapping key and a key-switching
 * key), and the boolean circuits the paper builds from them: ripple-carry
 * addition (Eq. "addres", Eq. "addcarry"; sections III-A and V-B-1),
 * shift-and-add multiplication (section III-B-1) and the matrix-vector
 * product with tree accumulation (sections IV-D and V-B-2), with variants
 * of lower depth (majority-carry, parallel-prefix and Dadda circuits).
 * Independent gates of a circuit level run together in one batched launch
 * (the paper's bit coalescing and compound gates, section V-A).
 *
 * Conventions used by every entry point:
 *   - Torus32: a torus element x/2^32 is stored as one 32-bit word.
 *   - LWE ciphertext array: int32 [count][TFHE_LWE_STRIDE]; words 0..n-1 are
 *     the mask a, word n the body b, words n+1..TFHE_LWE_STRIDE-1 are zero on
 *     output and ignored on input.  Integers are arrays of ciphertexts of
 *     their bits, least significant bit first: [batch][width][STRIDE].
 *   - Bit encoding: bit 1 <-> phase +1/8, bit 0 <-> phase -1/8.
 *   - Ciphertext pointers passed to the evaluation calls are DEVICE pointers
 *     on the context's device, owned by the caller; outputs must not alias
 *     inputs.  Key pointers may be host or device memory (detected).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL means the legacy default stream).  Argument errors are
 *     returned synchronously; errors raised by kernels (bad gather index,
 *     timeout of a bounded wait) are recorded in a device status word that
 *     tfhe_ctx_status() reads after the stream has been synchronised.
 *   - Every function returns a tfhe_status code; tfhe_last_error() gives the
 *     message of the last failure on that context.
 *   - A context is used by one host thread at a time (the serving API is the
 *     multi-request interface).
 */
#ifndef TFHE_GB_H
#define TFHE_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TFHE_GB_ABI_VERSION 1
#define TFHE_LWE_STRIDE 512   /* words per LWE ciphertext row (n <= 511)   */
#define TFHE_BIG_STRIDE 1056  /* words per extracted LWE_N row (N + 1 used) */

typedef struct tfhe_ctx tfhe_ctx; /* opaque, owned by the library */

/* Parameter set (section II-A names LWE dimension and key size; the values
 * are those of TFHE's gate bootstrapping): LWE dimension n, TLWE ring degree
 * N with k = 1, gadget base 2^bg_bit with l levels, key-switch base
 * 2^ks_basebit with ks_t levels.  The library supports n <= 511, N = 1024,
 * k = 1, bg_bit = 10, l = 2, ks_t = 8, ks_basebit = 2; anything else is
 * rejected with TFHE_EINVAL. */
typedef struct {
    int32_t n, N, k, l, bg_bit, ks_t, ks_basebit;
} tfhe_params;

typedef enum {
    TFHE_OK = 0,
    TFHE_EINVAL = -1,   /* bad argument                                  */
    TFHE_ENOMEM = -2,   /* device allocation failed                      */
    TFHE_ECUDA = -3,    /* CUDA runtime error                            */
    TFHE_ETIMEOUT = -4, /* a bounded device or host wait gave up         */
    TFHE_EBUSY = -5,    /* resource in use (e.g. serving already started) */
    TFHE_EDEVICE = -6,  /* a kernel reported an error in the status word */
    TFHE_ECANCELED = -7 /* a served request was cancelled (tfhe_serve_cancel) */
} tfhe_status;

/* Gate opcodes.  Gate g computes c = (0, mu_g) + alpha_a ca + alpha_b cb
 * (+ alpha_c cc) and bootstraps it; (mu, alpha_a, alpha_b, alpha_c):
 *   NAND (+1/8, -1, -1), AND (-1/8, +1, +1), OR (+1/8, +1, +1),
 *   XOR (+1/4, +2, +2), NOR (-1/8, -1, -1), XNOR (-1/4, -2, -2),
 *   ANDNY = AND(NOT a, b) (-1/8, -1, +1), ANDYN = AND(a, NOT b) (-1/8, +1, -1),
 *   ORNY = OR(NOT a, b) (+1/8, -1, +1), ORYN = OR(a, NOT b) (+1/8, +1, -1),
 *   MAJ = majority of three (0, +1, +1, +1): the only 3-input gate; it is
 *   available in circuits (a third input wire), not in tfhe_bootstrap_gates. */
typedef enum {
    TFHE_NAND = 0, TFHE_AND = 1, TFHE_OR = 2, TFHE_XOR = 3, TFHE_NOR = 4, TFHE_XNOR = 5,
    TFHE_MAJ = 6, TFHE_ANDNY = 7, TFHE_ANDYN = 8, TFHE_ORNY = 9, TFHE_ORYN = 10
} tfhe_gate;

/* ------------------------------------------------------------------ */
/* Context and keys                                                     */
/* ------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  Returns TFHE_EINVAL for an
 * unsupported parameter set.  *out is NULL on failure. */
int tfhe_ctx_create(const tfhe_params *params, int device, tfhe_ctx **out);

/* Upload keys (host or device pointers; copied, the caller keeps them):
 *   bk : int32 [n][2l][2][N]  bootstrapping key in coefficient form; row
 *        r = c*l + j of BK_i is a TLWE sample (a(X), b(X)) of a TGSW
 *        encryption of s_i (section II-A; Fig. "gpu_execution" "BS key").
 *        The context keeps it in the NTT domain of its two primes.
 *   ksk: int32 [N][ks_t][2^ks_basebit - 1][n + 1] key-switching key; entry
 *        [j][q][d-1] is an LWE_n encryption of d * S_j / base^(q+1)
 *        (Fig. "gpu_execution" "KS key").
 * Synchronous with respect to `stream` (returns after the upload). */
int tfhe_ctx_set_keys(tfhe_ctx *ctx, const int32_t *bk, const int32_t *ksk, void *stream);

void tfhe_ctx_destroy(tfhe_ctx *ctx);

/* Save the context's device keys to a file, and load them into a context of
 * the same parameters (no counterpart in the paper: checkpoint / resume of a
 * serving process).  The file holds the keys as the context keeps them (the
 * bootstrapping key already in the NTT domain of this library's primes) after
 * a header with the parameters, the primes, the sizes and a 64-bit checksum;
 * loading returns TFHE_EINVAL for another library's file, other parameters, a
 * short file or a checksum mismatch, and leaves the context's keys as they
 * were.  Both are synchronous (device <-> host copies on the legacy stream);
 * saving needs keys set. */
int tfhe_ctx_save_keys(tfhe_ctx *ctx, const char *path);
int tfhe_ctx_load_keys(tfhe_ctx *ctx, const char *path);

/* Last error message of the context (NUL-terminated, truncated to len). */
int tfhe_last_error(const tfhe_ctx *ctx, char *buf, size_t len);

/* Read and clear the device status word (synchronises the context's
 * device).  Returns TFHE_OK or TFHE_EDEVICE; *code (may be NULL) receives
 * the raw word: bit 0 gather index out of range, bit 1 scatter index out of
 * range, bit 2 bounded wait timed out, bit 3 opcode without its inputs
 * (MAJ given no third input, or an unknown opcode). */
int tfhe_ctx_status(tfhe_ctx *ctx, uint32_t *code);

/* ------------------------------------------------------------------ */
/* Gate bootstrapping                                                   */
/* ------------------------------------------------------------------ */

/* count independent bootstrapped gates: out[g] = ops[g](a[g], b[g]).
 * ops: uint8 [count] device; a, b, out: [count][TFHE_LWE_STRIDE] device.
 * The batch runs as one blind-rotation launch and one key switch (one
 * kernel, or two when the j-range is split and the output rows are
 * initialised first).  count == 0 is a no-op. */
int tfhe_bootstrap_gates(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a, const int32_t *b,
                         int32_t *out, size_t count, void *stream);

/* Bootstrap count ciphertexts as they are (no gate combine): the output
 * encrypts +mu if the input phase lies in [0, 1/2), else -mu. */
int tfhe_bootstrap(tfhe_ctx *ctx, const int32_t *in, int32_t *out, size_t count, uint32_t mu,
                   void *stream);

/* Stages of the bootstrap, exposed for testing and profiling:
 * blind rotation with fused gate combine, mod switch and sample extraction
 * (ops may be NULL: then b is ignored and a is bootstrapped as is with
 * mu = 1/8) writing LWE_N samples big: int32 [count][TFHE_BIG_STRIDE]
 * (a'_0..a'_(N-1), b' at word N); and key switching of those samples. */
int tfhe_blind_rotate_extract(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a,
                              const int32_t *b, int32_t *big, size_t count, void *stream);
int tfhe_keyswitch(tfhe_ctx *ctx, const int32_t *big, int32_t *out, size_t count, void *stream);

/* The external product's negacyclic products on the tensor pipe, exposed to
 * measure the alternative to the NTT (the product inside the CMux of the
 * TFHE blind rotation, paper section II-A): for `count` bootstraps at one
 * CMux step, out[m][p][k] = sum_r (d_r[m] * BK[r][p])[k] in
 * Z[X]/(X^1024 + 1) mod 2^32, r < 4, p < 2 -- the 8 products the NTT path
 * computes per CMux -- as tcgen05 matrix products of limb-split bf16
 * operands with exact fp32 sums (digits split in 2 limbs, key words in 4
 * balanced bytes).  The blind-rotation kernels do not use it: on GB300 the
 * 8 products take about 6 times as long as a whole NTT CMux step (160 ns
 * against 26 ns per bootstrap), and would still take 2.6 times as long at
 * the full bf16 tensor rate.
 *   tfhe_tc_prepare_key: bk_rows = device uint32 [4 rows][2 polys][1024]
 *     (one TGSW key sample in coefficient form, row r = c l + j) ->
 *     key_ops, a caller-owned device buffer of tfhe_tc_key_bytes() bytes
 *     (64 MB, 16-byte aligned): the transposed negacyclic Toeplitz operand,
 *     4 bytes x 2048 x 4096 bf16.
 *   tfhe_cmux_products_tc: digits = device int32 [count][4][1024], every
 *     digit in [-512, 511] (out-of-range digits set status bit 0 and give
 *     undefined outputs); digit_ops = caller-owned device scratch of
 *     tfhe_tc_digit_bytes(count) bytes (16-byte aligned); out = device
 *     uint32 [count][2][1024].  count must be a multiple of 128 (at most
 *     128 x 65535); TFHE_EINVAL otherwise.  Asynchronous on `stream`; a
 *     wait that runs out sets status bit 2. */
size_t tfhe_tc_key_bytes(void);
size_t tfhe_tc_digit_bytes(size_t count);
int tfhe_tc_prepare_key(tfhe_ctx *ctx, const uint32_t *bk_rows, void *key_ops, void *stream);
int tfhe_cmux_products_tc(tfhe_ctx *ctx, const int32_t *digits, const void *key_ops,
                          void *digit_ops, uint32_t *out, size_t count, void *stream);

/* Same computation and result as tfhe_bootstrap_gates, for callers that
 * cannot let the library allocate device memory while they call it
 * (runtimes that reserve all device memory up front, serving loops that
 * must not hit cudaMalloc and its implicit synchronisation, hosts that
 * account for every byte).  The paper has no counterpart; this is a
 * deployment interface.  It calls no cudaMalloc/cudaFree or any other
 * allocating routine: its scratch is a fixed array of
 * TFHE_NOALLOC_MAX_GATES rows (2,162,688 bytes) in the library's device
 * image, which every GPU that loads the library holds until the process
 * exits.  count > TFHE_NOALLOC_MAX_GATES is rejected with TFHE_EINVAL
 * (split the batch).  The first call on a device (and the first after a
 * device reset, which reloads the library's device image) looks up the
 * array's device address (cudaGetSymbolAddress) and caches it for that
 * CUDA context, so make that first call before any stream capture.  It
 * launches the same kernels as tfhe_bootstrap_gates, including the
 * context's key-switch kernel choice (TFHE_OPT_KS_KERNEL, autotuner).  All
 * calls on a device share the one array: calls that overlap on the GPU
 * (other streams, other contexts on the same device) race and must be
 * serialised by the caller.  Nothing in the array needs clearing between
 * calls. */
#define TFHE_NOALLOC_MAX_GATES 512
int tfhe_bootstrap_gates_noalloc(tfhe_ctx *ctx, const uint8_t *ops, const int32_t *a,
                                 const int32_t *b, int32_t *out, size_t count, void *stream);

/* ------------------------------------------------------------------ */
/* Circuits over encrypted integers (bit 0 first)                        */
/* ------------------------------------------------------------------ */

/* R = A + B mod 2^width, batch instances.  A, B, R: [batch][width][STRIDE]. */
int tfhe_add_n(tfhe_ctx *ctx, int width, const int32_t *A, const int32_t *B, int32_t *R,
               size_t batch, void *stream);

/* R = A * B mod 2^width (truncated shift-and-add), batch instances. */
int tfhe_mul_n(tfhe_ctx *ctx, int width, const int32_t *A, const int32_t *B, int32_t *R,
               size_t batch, void *stream);

/* y = M v mod 2^width: M [rows][cols][width][STRIDE], v [cols][width][STRIDE],
 * y [rows][width][STRIDE]; products accumulated by a balanced pairwise tree. */
int tfhe_matvec(tfhe_ctx *ctx, int width, int rows, int cols, const int32_t *M,
                const int32_t *v, int32_t *y, void *stream);

/* Mixed batches: several circuit jobs of different kinds, widths and
 * depths compiled into one level schedule, so that gates of every job that
 * are ready at the same depth share one blind-rotation launch (the paper's
 * compound gates and bit coalescing, section V-A, generalised across
 * circuits).  The schedule of a given list of (kind, width, rows, cols,
 * batch) is compiled once and cached; its level sequence is replayed as a
 * CUDA graph. */
typedef enum {
    TFHE_CIRCUIT_GATE = 0,     /* one 2-input gate, opcode in `width` (not MAJ)   */
    TFHE_CIRCUIT_ADD = 1,      /* tfhe_add_n: ripple carry, 5w - 6 gates, depth 2w-2 */
    TFHE_CIRCUIT_MUL = 2,      /* tfhe_mul_n: sequential shift-and-add           */
    TFHE_CIRCUIT_MATVEC = 3,   /* tfhe_matvec (rows x cols)                      */
    TFHE_CIRCUIT_ADD_MAJ = 4,  /* ripple adder with majority carries:            */
                               /*   3w - 2 gates, depth w (one MAJ per carry)     */
    TFHE_CIRCUIT_ADD_NW = 5,   /* the paper's number-wise adder GPU_n (section    */
                               /*   V-B-1): w rounds of (R AND B, R XOR B, B<<1),  */
                               /*   w^2 gates, depth w                            */
    TFHE_CIRCUIT_MUL_TREE = 6, /* multiplication with tree-based accumulation    */
                               /*   of the partial products (section V-B-2)       */
    TFHE_CIRCUIT_MUL_FULL = 7, /* full product, w x w -> 2w bits, 2 <= w <= 64:  */
                               /*   AND partial products at their weights summed  */
                               /*   by the tree of section V-B-2                  */
    TFHE_CIRCUIT_MUL_KARATSUBA = 8, /* full product by Karatsuba (Algorithm       */
                               /*   "karatsuba", vector form of section V-B),     */
                               /*   split at ceil(w/2), Z2 - (Z0 + Z1) by a       */
                               /*   two's-complement subtractor, the full product */
                               /*   above below 8 bits; 2w bits, 2 <= w <= 64     */
    TFHE_CIRCUIT_MUL_TREE_MAJ = 9, /* MUL_TREE whose adders carry with majority   */
                               /*   gates (one MAJ per carry): fewer gates and    */
                               /*   about half the depth, for latency             */
    TFHE_CIRCUIT_ADD_PREFIX = 10, /* parallel-prefix (Sklansky) adder on majority */
                               /*   gates, depth ceil(log2(w-1)) + 2, for latency */
    TFHE_CIRCUIT_MUL_DADDA = 11 /* truncated multiplication by a Dadda tree of    */
                               /*   full adders (XOR, XOR, MAJ) and half adders   */
                               /*   and a final ADD_PREFIX: lowest depth          */
} tfhe_circuit;

typedef struct {
    int32_t kind;           /* tfhe_circuit                                       */
    int32_t width;          /* bit width (ADD, MUL, MATVEC) or gate opcode (GATE) */
    int32_t rows, cols;     /* MATVEC shape; ignored otherwise                    */
    int64_t batch;          /* independent instances                              */
    const int32_t *in0;     /* A (GATE/ADD/MUL) or M (MATVEC), device, [batch]... */
    const int32_t *in1;     /* B or v, device                                     */
    int32_t *out;           /* R or y, device; [batch][w][512] except MUL_FULL    */
                            /* and MUL_KARATSUBA: [batch][2w][512]                */
} tfhe_job;

int tfhe_run_jobs(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, void *stream);

/* Level schedules of a job list (tfhe_run_jobs). */
typedef enum {
    TFHE_SCHED_ASAP = 0,     /* every gate at its earliest level              */
    TFHE_SCHED_BALANCED = 1  /* default: deadline-driven list scheduling that  */
                             /* fills each level up to a target width with the */
                             /* ready gates of the earliest latest-start level */
                             /* (same depth as ASAP; results identical)        */
} tfhe_schedule;

/* Host-only: the level widths of the schedule of `jobs` (pointers unused)
 * under `policy` with target width `target` (0: 608); widths[0..cap) get the
 * first cap levels.  Needs no context and no GPU. */
int tfhe_schedule_info(const tfhe_job *jobs, size_t njobs, int policy, int64_t target,
                       int32_t *widths, int32_t cap, int32_t *depth, int64_t *gates);

/* Bootstrapped-gate count and depth (levels) of one instance of a circuit;
 * needs no context and no GPU. */
int tfhe_circuit_info(int kind, int width, int rows, int cols, int64_t *gates, int32_t *depth);

/* Host-only: evaluate one instance of a circuit on plaintext bits, gate by
 * gate through the same netlist the GPU schedules run (no counterpart in
 * the paper; it lets a CPU check the circuit definitions).  in: n_in bits
 * (0/1), the input wires in the order of the circuit's inputs (A bits then
 * B bits, least significant first; MATVEC: M[r][c] bits then v[c] bits);
 * out: n_out bits in output order.  TFHE_EINVAL if the circuit is
 * unsupported or the counts do not match.  Needs no context and no GPU. */
int tfhe_circuit_eval_plain(int kind, int width, int rows, int cols, const uint8_t *in,
                            size_t n_in, uint8_t *out, size_t n_out);

/* Context options. */
typedef enum {
    TFHE_OPT_GRAPHS = 0,     /* 1 (default): replay level sequences as CUDA graphs  */
    TFHE_OPT_PER_GATE = 1,   /* 1: baseline schedule, one launch pair per gate      */
    TFHE_OPT_PROFILE = 2,    /* 1: record CUDA events around every blind-rotation   */
                             /*    and key-switch launch of circuit schedules (also */
                             /*    inside captured graphs)                          */
    TFHE_OPT_BR_GROUP = 3,   /* blind-rotation CTA shape: 1, 2 or 4 bootstraps per  */
                             /*    CTA (4 warps each), 5 = one per 4-warp CTA at 5  */
                             /*    CTAs per SM, 8 = one bootstrap on 8 warps,       */
                             /*    16 = one bootstrap on a cluster of two CTAs (two */
                             /*    SMs, one prime each; lowest latency), 32 = two   */
                             /*    bootstraps per CTA with each CMux step's key     */
                             /*    staged in shared memory by bulk copies (one CTA  */
                             /*    per SM), 33 = the same shape and occupancy with  */
                             /*    the key read through L1 (the staging's control), */
                             /*    40 = one bootstrap on 8 warps with the key       */
                             /*    staged, 48 = the two-CTA cluster with each CTA's */
                             /*    half of the key staged, or 0 (default):          */
                             /*    autotuned, else by batch size                    */
    TFHE_OPT_SCHEDULE = 4,   /* tfhe_schedule policy of circuit schedules           */
    TFHE_OPT_LEVEL_WIDTH = 5,/* target gates per level for BALANCED (0: one wave    */
                             /*    of 4 bootstraps per SM, or of 5 per SM (shape 5) */
                             /*    where the autotuner's wave times make that       */
                             /*    schedule cheaper)                                */
    TFHE_OPT_KS_KERNEL = 6,  /* key-switch kernel: 64 = tiled (64 gates per CTA, key */
                             /*    rows staged in shared memory by bulk copies),    */
                             /*    1, 2, 4, .. 32 = direct kernel with that j-split, */
                             /*    or 0 (default): autotuned, else by batch size    */
    TFHE_OPT_TEST_FREE_HBM = 8,/* test hook for serving admission, 0 (default) off: */
                             /*    a serving loop started afterwards takes this     */
                             /*    many bytes as the device's free memory           */
    TFHE_OPT_TEST_KS_STALL = 7 /* test hook for the timeout path, 0 (default) off:  */
                             /*    1 makes every stage of the tiled key switch also */
                             /*    wait on an mbarrier that nothing completes, so   */
                             /*    each bounded wait runs out after a short budget; */
                             /*    the kernel then lets the copies it issued land,  */
                             /*    the call sets status bit 2 (timeout), its outputs */
                             /*    are undefined, and the context stays usable     */
} tfhe_option;

int tfhe_ctx_set_option(tfhe_ctx *ctx, int option, int64_t value);

/* Autotune the launch shapes of the two bootstrapping kernels for this
 * context's device: for each level-width bucket (<= 152, 304, 608, 1216,
 * 2432, 4864, 9728 gates, and more) time the blind-rotation CTA shapes
 * (TFHE_OPT_BR_GROUP values) and the key-switch kernels (TFHE_OPT_KS_KERNEL
 * values) on synthetic ciphertexts, and keep the fastest; then time one
 * full wave of 4 bootstraps per SM and one of 5 per SM, from which each
 * circuit schedule picks its wave size (a few seconds; results never
 * change).  cache_path (may be NULL): a text file consulted
 * first and appended to after tuning, keyed by device name and SM count.
 * choices (may be NULL) receives 16 ints: the 8 blind-rotation shapes, then
 * the 8 key-switch choices.  Synchronous. */
int tfhe_ctx_autotune(tfhe_ctx *ctx, const char *cache_path, int32_t *choices);

/* Kernel launches the context has issued so far (kernels inside a replayed
 * graph count once per replay). */
int tfhe_ctx_launches(const tfhe_ctx *ctx, uint64_t *launches);

/* With TFHE_OPT_PROFILE on: device time of the blind-rotation and
 * key-switch launches of the most recent run of every circuit schedule run
 * since the previous call (synchronises the device, then resets). */
int tfhe_ctx_profile(tfhe_ctx *ctx, double *br_ms, int64_t *br_launches, int64_t *br_bootstraps,
                     double *ks_ms, int64_t *ks_launches);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of requests                              */
/* ------------------------------------------------------------------ */

/* One request: one instance of a circuit (kind/width/rows/cols as in
 * tfhe_job, batch 1).  in0/in1/out are device buffers owned by the caller
 * and must stay valid until the request completes. */
typedef struct {
    int32_t kind, width, rows, cols;
    const int32_t *in0, *in1;
    int32_t *out;
} tfhe_request;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t gates;          /* bootstraps run                               */
    uint64_t iterations;     /* batched launches (one level of many requests) */
    uint64_t in_flight;      /* admitted, not finished                       */
    uint64_t queued;         /* waiting for pool rows                        */
    double wall_ms;          /* first submit to last completion              */
    uint64_t pool_bytes;     /* device memory the ciphertext pool holds now  */
    uint64_t pool_cap_bytes; /* the most it may grow to (the caller's cap, or */
                             /* the device's memory)                         */
    uint64_t pool_grows;     /* times admission grew the pool                */
    uint64_t admitted_busy;  /* requests admitted while others were admitted  */
                             /* and unfinished (earlier in the same admission */
                             /* pass included) or an iteration was in flight */
    uint64_t cancelled;      /* requests cancelled before they completed      */
} tfhe_serve_info;

/* Start the request loop on the context's device: a worker thread with its
 * own stream and a ciphertext pool.  Requests are admitted in arrival order
 * when their rows (inputs and every gate output, 2 KB each) fit in the
 * pool; when they do not, the pool grows by mapping more device memory, as
 * long as the device's free HBM (cudaMemGetInfo) stays 1 GiB above the
 * growth and the pool stays within hbm_budget_bytes (0: no cap but the
 * device).  Otherwise the request waits until finished requests free rows.
 * The pool is one reserved range of device addresses mapped in steps
 * (driver virtual memory management); where that is unavailable it is one
 * fixed allocation of the cap (or of half the free memory, at most 32 GB).  Each iteration runs the
 * next level of admitted requests as one batched bootstrap, up to
 * max_batch_gates gates (0: a default of 8 waves of the GPU), chosen as
 * tfhe_serve_select describes with the autotuner's level times (call
 * tfhe_ctx_autotune first; untuned, a fixed model); requests that arrive
 * meanwhile join the next iteration.  While serving, the context
 * must not be used for other evaluation calls.  The paper's GPU framework
 * evaluates one circuit at a time; this is its level batching (section
 * V-A) extended across requests. */
int tfhe_serve_start(tfhe_ctx *ctx, size_t hbm_budget_bytes, size_t max_batch_gates);

/* Thread-safe.  *id identifies the request. */
int tfhe_serve_submit(tfhe_ctx *ctx, const tfhe_request *req, uint64_t *id);

/* *state: 1 done, 0 pending, < 0 failed with that tfhe_status.
 * *latency_ms (may be NULL): submit-to-completion host time when done. */
int tfhe_serve_poll(tfhe_ctx *ctx, uint64_t id, int *state, double *latency_ms);

/* Block up to timeout_ms for completion: TFHE_OK, TFHE_ETIMEOUT or the
 * request's failure status. */
int tfhe_serve_wait(tfhe_ctx *ctx, uint64_t id, int timeout_ms, double *latency_ms);

/* Thread-safe.  Cancel a request that has not completed (no counterpart in
 * the paper: a serving client that gives up on a request).  A queued
 * request leaves the queue; an admitted one runs no further level, and the
 * worker returns its pool rows at its next iteration (every device use of
 * them is already ordered on the worker's stream ahead of any reuse).  Its
 * output buffer is never written.  poll and wait then report
 * TFHE_ECANCELED.  Returns TFHE_OK when cancelled; TFHE_EBUSY when the
 * request's last level is already on the device (its result will arrive);
 * TFHE_EINVAL for an unknown id or a request that has completed or failed. */
int tfhe_serve_cancel(tfhe_ctx *ctx, uint64_t id);

int tfhe_serve_stats(tfhe_ctx *ctx, tfhe_serve_info *out);

/* Latencies (ms) of completed requests in completion order; *count gets the
 * total, at most cap are copied. */
int tfhe_serve_latencies(tfhe_ctx *ctx, double *ms, size_t cap, size_t *count);

/* Host-only: the choice each serving iteration makes (no counterpart in the
 * paper, which evaluates one circuit at a time; needs no context and no
 * GPU).  Inputs, one entry per admitted request in admission order:
 * width[i] > 0 the gates of its next level, remaining[i] > 0 its levels
 * left (that one included), waited[i] >= 0 the iterations run since its
 * last level ran.  Requests are ranked by remaining + waited, descending,
 * ties in admission order; in that order each next level is taken while
 * the running total stays within cap gates (a level that does not fit is
 * passed over; the first is always taken).  Of that list the prefix with
 * the most gates per estimated millisecond is kept, the longest on ties.
 * The estimate for g gates: while g <= 4 num_sms, level_ms[bucket of g]
 * (the autotuner's 8 level times for widths up to 152, 304, 608, 1216,
 * 2432, 4864, 9728 gates and more) when wave_ms > 0 and that entry is
 * > 0, else 0.35, 0.55 or 1 times wave_ms (1 when wave_ms is 0) for g up to
 * num_sms, 2 num_sms or 4 num_sms; above, ceil(g / (4 num_sms)) wave_ms.
 * level_ms may be NULL.  taken (n entries, caller-owned) receives the
 * indices of the requests kept, in rank order; *ntaken their number.
 * TFHE_EINVAL on a null pointer where n > 0, num_sms or cap <= 0, or an
 * entry out of range. */
int tfhe_serve_select(const int64_t *width, const int32_t *remaining, const int32_t *waited,
                      size_t n, int64_t cap, int32_t num_sms, const float *level_ms,
                      float wave_ms, int32_t *taken, size_t *ntaken);

/* Drain queued and in-flight requests, stop the worker, free the pool.
 * Returns TFHE_OK or the error that stopped serving. */
int tfhe_serve_stop(tfhe_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Client-side helpers (key generation and encryption on the device)     */
/* ------------------------------------------------------------------ */

/* Key generation from raw draws (all device pointers):
 *   s [n], S [N] key bits; bk_mask uint32 [n][2l][N], bk_noise int32
 *   [n][2l][N]; ksk_mask uint32 [N][ks_t][base-1][n], ksk_noise int32
 *   [N][ks_t][base-1].  Writes bk_out [n][2l][2][N] and ksk_out
 *   [N][ks_t][base-1][n+1] in the layouts tfhe_ctx_set_keys takes. */
int tfhe_keygen(const tfhe_params *params, const int32_t *s, const int32_t *S,
                const uint32_t *bk_mask, const int32_t *bk_noise, const uint32_t *ksk_mask,
                const int32_t *ksk_noise, int32_t *bk_out, int32_t *ksk_out, void *stream);

/* Encrypt count bits (device pointers): cts[g] = (mask[g], <mask[g], s> +
 * (bit ? +1/8 : -1/8) + noise[g]); masks uint32 [count][n]. */
int tfhe_encrypt_bits(const tfhe_params *params, const int32_t *s, const uint32_t *masks,
                      const int32_t *noise, const uint8_t *bits, int32_t *cts, size_t count,
                      void *stream);

/* phase[g] = b - <a, s> (device pointers); decrypt = phase > 0 as int32. */
int tfhe_phase(const tfhe_params *params, const int32_t *s, const int32_t *cts, uint32_t *phase,
               size_t count, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TFHE_GB_H */
