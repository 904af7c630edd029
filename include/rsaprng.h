/*
 * rsaprng.h -- C ABI of the GB300 bulk generator for the RSA-exponentiation
 * pseudorandom number generator of Datephanyawat & Beale (arXiv:1811.11629).
 *
 * What is computed (Sec. IV-V, Eq. algorithm1). An instance has fixed
 * parameters {p, q, n = p q, e, Q = 2^63 - 25, a} and a state {m, s}. Each
 * output k = 1, 2, ... advances the state and emits
 *     s_k = a s_{k-1} mod Q                 (Eq. congruentialgenerator1)
 *     m_k = (m_{k-1} + s_k) mod n           (Sec. IV message update)
 *     c_k = m_k^e mod n                     (Eq. encrypt2)
 *     r_k = RN(RN(c_k) / RN(n)), and 1 - 2^-53 in place of 1.0 (Sec. V)
 * where RN is IEEE-754 round-to-nearest-even to double. All integer steps
 * are exact; r_k is the C expression (double)c_k / (double)n.
 *
 * Parameters: p, q distinct primes in [2^31, 2^32) (Sec. V: 32-bit primes);
 * e odd, 3 <= e < 2^32, gcd(e, (p-1)(q-1)) = 1 (Sec. III); a one of the
 * restricted primitive roots mod Q listed below (Sec. V and its notes).
 *
 * Conventions for every call:
 *  - Return value: RSAPRNG_OK (0) or a negative RSAPRNG_ERR_* code.
 *    rsaprng_strerror() names it; rsaprng_last_error_detail() gives a
 *    thread-local sentence about the last failure.
 *  - Device pointers ("d_" prefix) are CUDA device addresses on the
 *    context's device, owned by the caller; the library never frees them.
 *    Host pointers ("h_" prefix or plain arrays) are read during the call
 *    only (unless a function says otherwise).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Generation is asynchronous on that stream; instance state
 *    advances in stream order, so calls for one instance must be ordered
 *    (one stream, or events). Calls on different streams that touch the same
 *    instance race.
 *  - A context is not thread-safe; one host thread drives it at a time
 *    (the server object has its own lock).
 */
#ifndef RSAPRNG_H
#define RSAPRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define RSAPRNG_OK 0
#define RSAPRNG_ERR_ARG (-1)         /* bad pointer, size or enum value */
#define RSAPRNG_ERR_NOT_PRIME (-2)   /* p or q failed Rabin-Miller (Sec. V) */
#define RSAPRNG_ERR_RANGE (-3)       /* p or q outside [2^31, 2^32) */
#define RSAPRNG_ERR_P_EQ_Q (-4)      /* p == q */
#define RSAPRNG_ERR_E (-5)           /* e even, < 3, or gcd(e,(p-1)(q-1)) != 1 */
#define RSAPRNG_ERR_ROOT (-6)        /* a is not an allowed multiplier (or a = 1 split) */
#define RSAPRNG_ERR_OOM (-7)         /* device or host allocation failed */
#define RSAPRNG_ERR_BUDGET (-8)      /* request larger than the server budget */
#define RSAPRNG_ERR_CUDA (-9)        /* a CUDA runtime call failed */
#define RSAPRNG_ERR_TIMEOUT (-10)    /* a host wait ran out of time */
#define RSAPRNG_ERR_DEVICE_FLAG (-11)/* a kernel raised its error flag */
#define RSAPRNG_ERR_CAPACITY (-12)   /* instance table full */
#define RSAPRNG_ERR_CANCELLED (-13)  /* server request was cancelled */
#define RSAPRNG_ERR_STATE (-14)      /* state (m, s) outside [0,n) x [1,Q-1] */
#define RSAPRNG_ERR_ID (-15)         /* unknown instance id / ticket */
#define RSAPRNG_ERR_BUSY (-16)       /* server queue full, try again */

/* Q = 2^63 - 25, the skip modulus (Sec. V). */
#define RSAPRNG_Q 0x7FFFFFFFFFFFFFE7ULL
/* Default skip multiplier: the primitive root recommended by L'Ecuyer,
 * Blouin & Couture (paper's reference note on that work). */
#define RSAPRNG_DEFAULT_ROOT 2307085864ULL

typedef struct rsaprng_ctx rsaprng_ctx;
typedef struct rsaprng_server rsaprng_server;
typedef struct rsaprng_plan rsaprng_plan;
typedef uint32_t rsaprng_id;

/* Encryption routes (both give bit-identical c_k). */
enum {
    RSAPRNG_MODEXP_AUTO = 0,
    RSAPRNG_MODEXP_CRT32 = 1,  /* CRT + Garner (Eq. CRTimplementation), two
                                  32-bit Montgomery exponentiations */
    RSAPRNG_MODEXP_MONT64 = 2  /* one 64-bit Montgomery exponentiation mod n */
};
/* Division routes for r_k (both give bit-identical r_k). */
enum {
    RSAPRNG_DIVIDE_AUTO = 0,
    RSAPRNG_DIVIDE_INT = 1,   /* integer rounding + division by the invariant
                                 significand of RN(n) (Moller & Granlund 2011) */
    RSAPRNG_DIVIDE_FP64 = 2,  /* IEEE double conversion and division */
    RSAPRNG_DIVIDE_HYBRID = 3,/* reciprocal route for three outputs in four, integer
                                 for the fourth: keeps FP64 and integer pipes busy */
    RSAPRNG_DIVIDE_RECIP = 4  /* FP64 multiply by the instance's correctly rounded
                                 reciprocal of RN(n) and one fused multiply-add
                                 correction (Markstein 1990); no division */
};
/* Exponent rules for rsaprng_params_from_seed. */
enum { RSAPRNG_E_SMALLEST = 0, RSAPRNG_E_UNIFORM = 1, RSAPRNG_E_AT_LEAST = 2 };

/* Reading of the division r = c / n (Eq. CodeFloatingPointStep). */
enum {
    RSAPRNG_ROUND_DEFAULT = 0, /* = RSAPRNG_ROUND_PAPER */
    RSAPRNG_ROUND_PAPER = 1,   /* RN(RN(c) / RN(n)): C's (double)c / (double)n */
    RSAPRNG_ROUND_EXACT = 2    /* RN(c / n) of the exact rational (the other reading) */
};

/* Tuning knobs; zero fields mean "use the tuned/default value". */
typedef struct {
    uint32_t struct_size;       /* sizeof(rsaprng_config) */
    int32_t modexp;             /* RSAPRNG_MODEXP_* */
    int32_t divide;             /* RSAPRNG_DIVIDE_* */
    int32_t threads_per_block;  /* 64, 128, 256 or 512 */
    int32_t numbers_per_thread; /* 2, 4, 8 or 16 (the 64-bit route uses 8 for 16; the
                                   interleaved call uses 8 for 16 on the CRT route in
                                   blocks of 128 threads, its tuned tile) */
    int32_t blocks_per_sm;      /* persistent-launch occupancy target */
    uint64_t chunk;             /* maximum numbers per chunk of a long stream
                                   (multiple of threads_per_block*numbers_per_thread);
                                   the planner also cuts streams whose work
                                   exceeds one resident block's share of the
                                   launch, in whole tiles */
    int32_t require_safe;       /* p, q must be safe primes (Sec. V) */
    int32_t rounding;           /* RSAPRNG_ROUND_*; with RSAPRNG_ROUND_EXACT the divide
                                   route is ignored (one integer route computes it) */
    int32_t lookback;           /* RSAPRNG_LOOKBACK_*: how the one-instance calls
                                   (rsaprng_generate_u64/f64/both) run */
    int32_t spin_limit;         /* empty poll rounds (64 ns apart) before a device-side
                                   wait gives up and raises the device error flag;
                                   0 = default (2^23, about a second), < 0 = none
                                   (give up at the first empty round; tests) */
    int32_t test_flags;         /* 0 in normal use. Bit 0: the first tile of a
                                   single-launch call publishes no prefix, so every
                                   later tile's wait runs out (tests of the device
                                   error path; no GPU fault is involved) */
    int32_t streams_per_block;  /* generation plans: 1 = one stream per block; 2, 4, 8
                                   or 16 = that many streams side by side in a block,
                                   threads_per_block / streams_per_block threads each
                                   (at least a warp), pieces grouped by length */
    int32_t unroll;             /* independent exponentiation chains a thread runs at
                                   once: 0 = all numbers_per_thread; a smaller power of
                                   two runs them in passes of that many (128 x 16 CRT
                                   tiles with 8, 8-per-thread CRT reciprocal tiles with
                                   4; other tilings run all at once) */
    int32_t pieces_per_block;   /* load balance of generation plans: streams whose work
                                   exceeds 1 / (resident blocks x this) of the launch are
                                   cut into pieces (each extra piece costs a skip-sum pass
                                   over the piece before it); 1 by default */
} rsaprng_config;

enum {
    RSAPRNG_LOOKBACK_AUTO = 0, /* one launch with a decoupled look-back: in the latency
                                  shape (512 threads x 16 per thread, CRT route, integer
                                  division) when the draw fits one wave of such blocks,
                                  else in the configured shape when the draw is at most
                                  4096 tiles and the tiling has such a kernel (16 per
                                  thread on the CRT route, 8 per thread on the CRT route
                                  with reciprocal division or on the 64-bit route with
                                  reciprocal or integer division); else the chunked path
                                  (skip-sum pre-pass, scan, generation) */
    RSAPRNG_LOOKBACK_OFF = 1,  /* always the chunked path */
    RSAPRNG_LOOKBACK_CONFIGURED = 2 /* as AUTO without the latency shape */
};

/* ------------------------------------------------------------- context */

/* Creates a context on CUDA device `device` with room for `max_instances`
 * instances (device table: 96 B parameters + 16 B state each). cfg may be
 * NULL. Makes `device` current on the calling thread. */
int rsaprng_ctx_create(rsaprng_ctx **out, int device, uint64_t max_instances,
                       const rsaprng_config *cfg);
void rsaprng_ctx_destroy(rsaprng_ctx *ctx);
/* Replaces the tuning knobs (validated; zero fields keep defaults). */
int rsaprng_ctx_configure(rsaprng_ctx *ctx, const rsaprng_config *cfg);
int rsaprng_ctx_get_config(const rsaprng_ctx *ctx, rsaprng_config *out);
uint64_t rsaprng_instance_count(const rsaprng_ctx *ctx);

/* ----------------------------------------------------------- instances */

/* One instance from {p, q, e} and a message seed (Sec. IV: "seeding is
 * simple"): a = RSAPRNG_DEFAULT_ROOT, m_0 = seed mod n, s_0 = 1, so the first
 * output uses m_1 = m_0 + a mod n. Validates p, q by trial division and
 * deterministic Rabin-Miller (Sec. V). Synchronous host->device write. */
int rsaprng_instance_create(rsaprng_ctx *ctx, uint64_t p, uint64_t q, uint64_t e, uint64_t seed,
                            rsaprng_id *out);
/* Explicit skip multiplier and start state: a must be an allowed multiplier
 * (rsaprng_root_allowed), m0 < n, 1 <= s0 < Q. a = 1 gives the unit skip
 * (s0 = 1: m_k = m_0 + k mod n, the block cipher in counter mode) or the
 * constant skip s_k = b = s0 of Sec. IV. */
int rsaprng_instance_create_ex(rsaprng_ctx *ctx, uint64_t p, uint64_t q, uint64_t e, uint64_t a,
                               uint64_t m0, uint64_t s0, rsaprng_id *out);
/* `count` instances from host arrays (same rules as rsaprng_instance_create);
 * ids are consecutive from *out_first. All or nothing: on error nothing is
 * added and the index of the first bad entry is in the error detail. */
int rsaprng_instances_create_bulk(rsaprng_ctx *ctx, uint64_t count, const uint64_t *p,
                                  const uint64_t *q, const uint64_t *e, const uint64_t *seed,
                                  rsaprng_id *out_first);
/* `count` instances from 64-bit seeds by rsaprng_params_from_seed; uses all
 * host cores. ids are consecutive from *out_first. */
int rsaprng_instances_create_seeded(rsaprng_ctx *ctx, uint64_t count, const uint64_t *seeds,
                                    int e_rule, uint64_t e_lo, uint64_t e_hi,
                                    rsaprng_id *out_first);

/* CRT exponents (the paper's note on large exponents, Sec. V): the p residue
 * is raised to e_p and the q residue to e_q, c = CRT(m_p^e_p mod p,
 * m_q^e_q mod q) by Garner's formula. e_p, e_q odd in [3, 2^32) with
 * gcd(e_p, p - 1) = gcd(e_q, q - 1) = 1. When e_p = e_q (mod gcd(p-1, q-1))
 * the output is m^e mod n for the large exponent e = e_p (mod p - 1),
 * e = e_q (mod q - 1); otherwise it is still a permutation of Z_n. Other
 * arguments as rsaprng_instance_create_ex. Such an instance runs on the CRT
 * route only: a launch with RSAPRNG_MODEXP_MONT64 that includes it fails
 * with RSAPRNG_ERR_ARG. Errors: RSAPRNG_ERR_RANGE, _P_EQ_Q, _NOT_PRIME, _E,
 * _ROOT, _STATE. */
int rsaprng_instance_create_crt(rsaprng_ctx *ctx, uint64_t p, uint64_t q, uint64_t e_p,
                                uint64_t e_q, uint64_t a, uint64_t m0, uint64_t s0,
                                rsaprng_id *out);
/* The exponents of the p and q residues (equal unless created by
 * rsaprng_instance_create_crt). */
int rsaprng_get_exponents(const rsaprng_ctx *ctx, rsaprng_id id, uint64_t *e_p, uint64_t *e_q);

/* Stream splitting (Sec. VI): Mv children of `parent`, child gamma with the
 * parent's parameters and current message, and skip
 *     s^(gamma) = s * a^(gamma floor((Q-1)/Mv)) mod Q.
 * Child 0 continues the parent's stream. The parent is unchanged. A constant
 * skip (a = 1) has no jump-ahead: RSAPRNG_ERR_ROOT. */
int rsaprng_split(rsaprng_ctx *ctx, rsaprng_id parent, uint32_t Mv, rsaprng_id *out_children);

/* Checkpoint / resume (Sec. IV: the state is {m, s}). Synchronous. */
int rsaprng_get_state(rsaprng_ctx *ctx, rsaprng_id id, uint64_t *m, uint64_t *s);
int rsaprng_set_state(rsaprng_ctx *ctx, rsaprng_id id, uint64_t m, uint64_t s);
/* Fixed parameters of an instance (any output pointer may be NULL). */
int rsaprng_get_params(rsaprng_ctx *ctx, rsaprng_id id, uint64_t *p, uint64_t *q, uint64_t *e,
                       uint64_t *a);

/* ---------------------------------------------------------- generation */

/* N outputs of one instance into caller device buffers (Eq. algorithm1):
 * d_c[k] = c_{k+1}, d_r[k] = r_{k+1}; advances the instance by N. A draw of
 * at most 4096 tiles runs as one launch: block b generates tile b and gets
 * the message before it (Sec. IV: m_0 plus the skips before it, mod n) by a
 * decoupled look-back over the earlier tiles' skip sums, every wait bounded
 * by cfg.spin_limit (see rsaprng_device_status). Longer draws are cut into
 * chunks whose start states come from an on-device skip-sum pass and scan.
 * Either way the whole GPU works on one instance. */
int rsaprng_generate_u64(rsaprng_ctx *ctx, rsaprng_id id, uint64_t N, uint64_t *d_c, void *stream);
int rsaprng_generate_f64(rsaprng_ctx *ctx, rsaprng_id id, uint64_t N, double *d_r, void *stream);
int rsaprng_generate_both(rsaprng_ctx *ctx, rsaprng_id id, uint64_t N, uint64_t *d_c, double *d_r,
                          void *stream);

/* The tile shape of the single launch above for a draw of N outputs on a GPU
 * with `sms` SMs, when the draw fits one wave of 512 x 16 tiles (the latency
 * mode; larger draws, and contexts configured with RSAPRNG_LOOKBACK_CONFIGURED,
 * use the configured tiling). Writes the threads per block (a multiple of 32,
 * 128 to 512) and the outputs per thread (12, 13, 14 or 16; 16 only when
 * rounding_exact is nonzero), with at most one tile per SM where such a shape
 * covers N. The paper has no counterpart: it is the launch geometry of this
 * implementation, a pure host function (no GPU, no context). Returns
 * RSAPRNG_ERR_ARG for a null output pointer or sms < 1. */
int rsaprng_latency_shape(uint64_t N, int sms, int rounding_exact, int *threads,
                          int *numbers_per_thread);

/* The same as rsaprng_generate_f64, for callers that cannot allocate device
 * memory when they draw numbers: latency-critical threads that forbid
 * allocator calls, or hosts that give all device memory to their own pool.
 * The paper has no counterpart; this is a deployment variant of the same
 * path. It allocates nothing: its scratch (chunk list, skip sums, work-queue
 * counter) is one fixed device array of about 330 KB inside the library,
 * which every GPU that loads the library keeps until the process exits.
 *  - Limit: N <= 2^36 outputs (at most 4096 chunks of at most 2^24 outputs);
 *    larger N returns RSAPRNG_ERR_ARG before anything is launched. Errors of
 *    this call return their code without setting rsaprng_last_error_detail.
 *  - Also RSAPRNG_ERR_ARG: a context on a device index of 64 or more, and an
 *    instance with CRT exponents when the context's route is
 *    RSAPRNG_MODEXP_MONT64. The chunk length is chosen here (the context's
 *    cfg.chunk is not used).
 *  - The first call on a device looks up the array's device address (one
 *    cudaGetSymbolAddress); make that first call before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents
 *    (the queue counter is cleared by every call). Calls whose kernels
 *    overlap on the GPU (different streams, or contexts on the same device)
 *    race on it: order them, e.g. on one stream.
 * Output and state advance are identical to rsaprng_generate_f64. */
int rsaprng_generate_f64_noalloc(rsaprng_ctx *ctx, rsaprng_id id, uint64_t N, double *d_r,
                                 void *stream);

/* Many requests in one launch sequence. Request i draws counts[i] outputs of
 * instance ids[i] into d_r/d_c at element offset out_offsets[i] (either
 * output may be NULL). ids, counts, out_offsets are HOST arrays. Requests of
 * the same instance are served in array order (each continues after the
 * previous one). Device arrays that start on a 16-byte boundary are written
 * by bulk tensor stores of whole tiles (faster; the bits are the same);
 * other arrays, and page-locked host memory mapped into the device, by
 * element stores. */
int rsaprng_generate_batch(rsaprng_ctx *ctx, uint64_t nreq, const rsaprng_id *ids,
                           const uint64_t *counts, const uint64_t *out_offsets, double *d_r,
                           uint64_t *d_c, void *stream);

/* The same with HOST output buffers (end to end); returns when h_r / h_c
 * hold the results. Either may be NULL. Page-locked (pinned) buffers are
 * written by the generation kernel itself over the CPU-GPU link; pageable
 * buffers are filled by device slices copied device->host, overlapped with
 * generation. */
int rsaprng_generate_batch_host(rsaprng_ctx *ctx, uint64_t nreq, const rsaprng_id *ids,
                                const uint64_t *counts, const uint64_t *out_offsets, double *h_r,
                                uint64_t *h_c, void *stream);

/* The vectorised call of Sec. VI (Eq. vectorize), for ngroups vectors at once
 * (one per process of the paper): group g is the Mv instances
 * ids[g Mv .. g Mv + Mv) (typically the substreams of one rsaprng_split);
 * they advance together by N outputs each, and the outputs are written
 * k-major, the order in which the vector update returns them:
 * d_r[g N Mv + k Mv + gamma] = r_{k+1} of instance ids[g Mv + gamma] (d_c
 * likewise; either may be NULL), for k < N. Every instance advances by N.
 * ids is a HOST array of ngroups Mv distinct ids; the outputs are DEVICE
 * arrays of ngroups N Mv elements. Asynchronous on stream. Errors:
 * RSAPRNG_ERR_ARG (Mv = 0, no output, repeated id), RSAPRNG_ERR_ID,
 * RSAPRNG_ERR_CUDA. */
int rsaprng_generate_interleaved(rsaprng_ctx *ctx, uint64_t ngroups, uint32_t Mv,
                                 const rsaprng_id *ids, uint64_t N, double *d_r, uint64_t *d_c,
                                 void *stream);

/* ------------------------------------------------ fused consumer (Sec. VII) */

/* Digit sources of rsaprng_histogram. */
enum {
    RSAPRNG_HIST_HIGH = 0, /* digit = floor(r d), exact, of the float output r */
    RSAPRNG_HIST_LOW = 1   /* digit = c mod d of the ciphertext c (d a power of two) */
};

/* The histogram of the paper's one-dimensional frequency test (D = 1) and
 * D-dimensional serial test (Sec. VII), accumulated while generating: the
 * next counts[i] outputs of instance ids[i] are generated (the instance
 * advances by counts[i], exactly as with rsaprng_generate_batch) and are not
 * stored; each request's outputs are cut into non-overlapping D-tuples of
 * consecutive outputs (x_{kD+1}, ..., x_{kD+D}), k = 0, 1, ..., and tuple k
 * adds one to d_hist[sum_{i=1..D} digit(x_{kD+i}) d^(i-1)]. Outputs after the
 * last whole tuple of a request are generated but not counted.
 *  - d_hist: DEVICE array of d^D uint64 counters, added to (not cleared);
 *    the caller keeps every counter below 2^64.
 *  - ids, counts: HOST arrays of nreq entries; an instance may appear in
 *    only one request of a call.
 *  - D in [1, 8], d >= 2, d^D <= 2^32; d a power of two for RSAPRNG_HIST_LOW.
 * Asynchronous on stream. Errors: RSAPRNG_ERR_ARG (bad D, d, source,
 * repeated id, NULL), RSAPRNG_ERR_ID, RSAPRNG_ERR_CUDA. */
int rsaprng_histogram(rsaprng_ctx *ctx, uint64_t nreq, const rsaprng_id *ids,
                      const uint64_t *counts, uint32_t D, uint32_t d, int source,
                      uint64_t *d_hist, void *stream);

/* chi^2 = sum_b (O_b - E)^2 / E of a HOST histogram of `bins` counts against
 * the uniform expectation E = total / bins (Sec. VII compares the histograms
 * with a uniform Poisson distribution; the p-value is the chi^2 survival
 * function with bins - 1 degrees of freedom). *total (optional) receives the
 * number of counted tuples. Errors: RSAPRNG_ERR_ARG (NULL, no bins, empty
 * histogram). */
int rsaprng_chi2_uniform(const uint64_t *h_hist, uint64_t bins, double *chi2, uint64_t *total);

/* ------------------------------------------------ plans and CUDA graphs */

/* A device-resident launch plan for a fixed set of requests (same meaning
 * as rsaprng_generate_batch). Launching it generates the next outputs of the
 * requests each time. rsaprng_plan_capture records the launches into a CUDA
 * graph bound to the given output buffers; rsaprng_plan_replay launches that
 * graph. */
int rsaprng_plan_create(rsaprng_ctx *ctx, uint64_t nreq, const rsaprng_id *ids,
                        const uint64_t *counts, const uint64_t *out_offsets, rsaprng_plan **out);
int rsaprng_plan_launch(rsaprng_plan *plan, double *d_r, uint64_t *d_c, void *stream);
/* rsaprng_plan_launch that also records the caller's CUDA events gen_start
 * and gen_end (cudaEvent_t, created by the caller, with timing) on the stream
 * right before and after the generation kernel, so that their elapsed time is
 * that kernel's alone; the skip-sum pre-pass and start-state scan, when the
 * plan has them, run before gen_start, and the generation kernel then starts
 * after the scan has completed instead of overlapping its end. Same outputs
 * and state advance as rsaprng_plan_launch. RSAPRNG_ERR_ARG for a null plan,
 * no output or a null event; RSAPRNG_ERR_CUDA when recording an event fails. */
int rsaprng_plan_launch_timed(rsaprng_plan *plan, double *d_r, uint64_t *d_c, void *stream,
                              void *gen_start, void *gen_end);
int rsaprng_plan_capture(rsaprng_plan *plan, double *d_r, uint64_t *d_c, void *stream);
int rsaprng_plan_replay(rsaprng_plan *plan, void *stream);
/* Kernel launches one rsaprng_plan_launch makes, and numbers it generates. */
int rsaprng_plan_info(const rsaprng_plan *plan, uint64_t *launches, uint64_t *numbers,
                      uint64_t *chunks);
/* Shape of the plan's most recent generation launch: grid blocks, threads
 * per block, resident blocks per SM, and whether blocks pull work items from
 * a queue (1) or take one each (0). Zeros before the first launch. */
int rsaprng_plan_shape(const rsaprng_plan *plan, int *grid, int *threads, int *blocks_per_sm,
                       int *persistent);
void rsaprng_plan_destroy(rsaprng_plan *plan);

/* --------------------------------------------------------------- tuning */

/* Times candidate configurations on a plan built from the given requests
 * (outputs go to scratch buffers the call allocates and frees; instance
 * states are restored after every trial) and stores the fastest in the
 * context's config and in the process's tuning cache. Stages, each starting
 * from the best so far: modexp and division routes; threads per block and
 * numbers per thread; unroll (chains in passes of half the numbers, where a
 * variant exists); streams per block (2, 4); resident blocks per SM (one or
 * two below the occupancy limit); the chunk cap of long streams. Every
 * candidate gives bit-identical outputs. `reps` timed launches per trial. */
int rsaprng_autotune(rsaprng_ctx *ctx, uint64_t nreq, const rsaprng_id *ids,
                     const uint64_t *counts, int reps, rsaprng_config *chosen);
/* As rsaprng_autotune, but first looks the workload up in the tuning cache,
 * keyed by device (compute capability, SM count), workload signature
 * (log2 buckets of the request count, the mean and the longest request; the
 * rounding reading) and exponent class (mean Montgomery products per
 * output, in steps of two). On a hit the cached knobs are applied at once
 * and *from_cache (may be NULL) is 1; otherwise it tunes. */
int rsaprng_autotune_cached(rsaprng_ctx *ctx, uint64_t nreq, const rsaprng_id *ids,
                            const uint64_t *counts, int reps, rsaprng_config *chosen,
                            int *from_cache);
/* The tuning cache: entries held, clear, and a text file of one line per
 * entry (key, then name=value knobs) to keep tuned choices across
 * processes. Load adds to (and overrides) the entries held; RSAPRNG_ERR_ARG
 * for an unreadable file or a malformed line (nothing is added then). */
uint64_t rsaprng_autotune_cache_size(void);
void rsaprng_autotune_cache_clear(void);
int rsaprng_autotune_cache_save(const char *path);
int rsaprng_autotune_cache_load(const char *path);

/* -------------------------------------------------------------- serving */

typedef struct {
    uint64_t submitted, admitted, completed, rejected, cancelled;
    uint64_t queued_now, inflight_now;
    uint64_t numbers_done;
    double p50_ms, p99_ms, mean_ms, max_ms; /* arrival -> completion latency */
    double busy_s, wall_s;                  /* device-busy and wall time */
    uint64_t iterations;                    /* batched launches issued */
    uint64_t max_inflight_iterations;       /* most iterations in flight at once
                                               (launched, not yet retired) */
    uint64_t overlapped_iterations;         /* iterations whose device interval (events
                                               on their stream before the plan upload and
                                               after the launch) overlapped the interval
                                               of another iteration */
} rsaprng_stats;

/* A continuous-batching request server over the context's instances. It owns
 * an output arena of `out_budget_bytes` device bytes: a request is admitted
 * when its 8 B/number fit in the arena, otherwise it waits in FIFO order.
 * Each server iteration gathers admitted work (large requests in chunks),
 * launches one batched pass on one of `nstreams` streams, and releases arena
 * space when the client calls rsaprng_server_release. */
int rsaprng_server_create(rsaprng_ctx *ctx, uint64_t out_budget_bytes, int nstreams,
                          rsaprng_server **out);
/* Queues `count` float64 outputs of instance `id`. The result is the
 * instance's next `count` outputs at the time of admission order. */
int rsaprng_server_submit(rsaprng_server *srv, rsaprng_id id, uint64_t count, uint64_t *ticket);
/* *done = 1 when the ticket's outputs are complete on the device. */
int rsaprng_server_poll(rsaprng_server *srv, uint64_t ticket, int *done);
/* Waits up to timeout_ns for the ticket (RSAPRNG_ERR_TIMEOUT otherwise). */
int rsaprng_server_wait(rsaprng_server *srv, uint64_t ticket, uint64_t timeout_ns);
/* Device address of a completed ticket's outputs (valid until released). */
int rsaprng_server_result(rsaprng_server *srv, uint64_t ticket, const double **d_r,
                          uint64_t *count);
/* Copies a completed ticket's outputs to d_dst (count doubles) on `stream`;
 * release the ticket only after that copy has completed. */
int rsaprng_server_copy(rsaprng_server *srv, uint64_t ticket, double *d_dst, void *stream);
int rsaprng_server_release(rsaprng_server *srv, uint64_t ticket);
/* Cancels a ticket that has not been admitted yet. */
int rsaprng_server_cancel(rsaprng_server *srv, uint64_t ticket);
int rsaprng_server_stats(rsaprng_server *srv, rsaprng_stats *out);
/* Open-loop trace replay for load measurements on an idle server: request i
 * (instance ids[i], counts[i] numbers) is submitted arrival_ns[i] ns after the
 * call starts, and its outputs are released as soon as they complete.
 * Returns when all n requests are done (RSAPRNG_ERR_TIMEOUT after timeout_ns).
 * Latencies in ms (arrival to completion) go to lat_ms_out[i] if not NULL, in
 * completion order; rsaprng_server_stats then reports this replay alone. */
int rsaprng_server_replay(rsaprng_server *srv, uint64_t n, const rsaprng_id *ids,
                          const uint64_t *counts, const uint64_t *arrival_ns,
                          uint64_t timeout_ns, double *lat_ms_out);
/* The same replay with every result kept: tickets_out[i] (a HOST array of n)
 * receives request i's ticket, whose outputs stay in the arena until the
 * caller reads them (rsaprng_server_result / _copy) and releases them, so the
 * budget must hold all n results. Used to check results of requests that
 * arrived while others were running. */
int rsaprng_server_replay_keep(rsaprng_server *srv, uint64_t n, const rsaprng_id *ids,
                               const uint64_t *counts, const uint64_t *arrival_ns,
                               uint64_t timeout_ns, uint64_t *tickets_out);
void rsaprng_server_destroy(rsaprng_server *srv);

/* ------------------------------------------------------- host utilities */

/* Deterministic primality of a 64-bit integer: trial division by small
 * primes, then Rabin-Miller with bases {2,3,5,7,11} below 2^32 and the
 * twelve smallest primes below 2^64 (Sec. V). Returns 1 or 0. */
int rsaprng_is_prime(uint64_t x);
/* Validates instance parameters without creating an instance: returns
 * RSAPRNG_OK or the code rsaprng_instance_create would return (RANGE,
 * P_EQ_Q, NOT_PRIME, E). require_safe adds the safe-prime rule of Sec. V. */
int rsaprng_validate_params(uint64_t p, uint64_t q, uint64_t e, int require_safe);
/* 1 if a is allowed as a skip multiplier: the recommended root, the eight
 * listed roots of Sezgin & Sezgin that are primitive (3163786287 is not: it
 * is a quadratic residue mod Q), one of the five smallest primitive roots
 * {3, 6, 7, 10, 11} used for the weakened-generator tests (Sec. VII), or 1
 * (the unit / constant skip of Sec. IV). */
int rsaprng_root_allowed(uint64_t a);

/* Instance parameters from one 64-bit seed (the rule the workloads use; it
 * is not from the paper). Draws x_1, x_2, ... come from SplitMix64 (Steele,
 * Lea & Flood 2014) started at `seed`. A prime candidate is (x >> 32) |
 * 0x80000001. p is the first prime candidate, q the next prime candidate
 * != p. e by rule: SMALLEST = smallest odd e >= 3 with gcd(e, phi) = 1;
 * AT_LEAST = smallest such odd e >= e_lo; UNIFORM = draws
 * e = e_lo + 2 (x mod ((e_hi - e_lo)/2 + 1)) until gcd(e, phi) = 1 (e_lo odd).
 * The message seed is the next draw. */
int rsaprng_params_from_seed(uint64_t seed, int e_rule, uint64_t e_lo, uint64_t e_hi,
                             uint64_t *p, uint64_t *q, uint64_t *e, uint64_t *msg_seed);

/* The output step alone (Eq. CodeFloatingPointStep with the Sec. V guard):
 * d_r[k] = RN(RN(d_c[k]) / RN(n_id)), 1 - 2^-53 in place of 1.0, for k < N,
 * using division route `divide` (RSAPRNG_DIVIDE_*; AUTO = the context's;
 * with RSAPRNG_DIVIDE_HYBRID element k takes the integer route when
 * k mod 4 = 3 and the reciprocal route otherwise, as output k of a thread's
 * run does in the generation kernels);
 * RN(d_c[k] / n_id) when the context's rounding is RSAPRNG_ROUND_EXACT.
 * d_c values must be < n of instance `id`. Asynchronous on `stream`. */
int rsaprng_unit_f64(rsaprng_ctx *ctx, rsaprng_id id, uint64_t N, const uint64_t *d_c,
                     double *d_r, int divide, void *stream);

/* Waits for `stream`, then reads and clears the context's device error word.
 * Returns RSAPRNG_ERR_DEVICE_FLAG if a device-side wait gave up since the last
 * call (a single-launch draw whose tile never received its predecessors'
 * prefix within spin_limit polls; that draw's outputs and the instance's
 * state are then undefined: restore it with rsaprng_set_state), else
 * RSAPRNG_OK. The paper has no counterpart (failure detection of this
 * library's own waits). */
int rsaprng_device_status(rsaprng_ctx *ctx, void *stream);

/* Kernel launches issued by this context so far (for launch accounting). */
uint64_t rsaprng_launch_count(const rsaprng_ctx *ctx);
/* Bytes the library itself has copied host->device (work lists) and
 * device->host (rsaprng_generate_batch_host results) on this context. */
int rsaprng_transfer_bytes(const rsaprng_ctx *ctx, uint64_t *h2d, uint64_t *d2h);

/* ----------------------------------------------------- microbenchmarks */

/* Device microbenchmarks for the roofline, timed with CUDA events on an
 * internal stream: kind 0 = 32-bit integer multiply-add issue rate
 * (result in G lane-ops/s), 1 = FP64 divide rate (G div/s), 2 = HBM write
 * bandwidth (GB/s) over `bytes` bytes, 3 = widening 32x32->64 multiply rate,
 * 4 = 32-bit high-half multiply rate, 5 = 32-bit Montgomery product rate,
 * 6 = FP64 fused multiply-add rate, 7 = unsigned 64-bit to double conversion
 * rate, 8 = rate of the whole reciprocal output step (conversion, product,
 * two FMAs, 1.0 guard) (3-8 in G per second, all lanes of the device). */
int rsaprng_microbench(rsaprng_ctx *ctx, int kind, uint64_t bytes, double *result);

const char *rsaprng_strerror(int code);
const char *rsaprng_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* RSAPRNG_H */
