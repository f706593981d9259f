/*
 * hmv.h -- exact multiprecision Hankel / Toeplitz / circulant matrix-vector
 * product on one NVIDIA GB300 GPU (sm_103a).
 *
 * Operation (Beliakov, arXiv:1402.5287, Sec. 1, matrices A_H, A_T, A_C and
 * the schoolbook product): for n x n structured A and vector x,
 *     Hankel     y_i = sum_{j<n} h_{i+j} x_j            h has 2n-1 entries
 *     Toeplitz   y_i = sum_{j<n} h_{n-1-i+j} x_j        h has 2n-1 entries
 *     Circulant  y_i = sum_{j<n} c_{(i-j) mod n} x_j     c has n entries
 * (0-based indices).  Toeplitz is computed as the row-reversed Hankel
 * product and circulant as a Toeplitz product with the wrapped sequence
 * h_k = c_{(n-1-k) mod n}, as Sec. 1 describes.
 *
 * Methods: the recursive half-size Hankel products of Sec. 3 (Algorithm 1)
 * down to a leaf size, with every leaf product done as an exact digit-plane
 * contraction on the tensor cores; or a plain schoolbook kernel on 32-bit
 * limbs (comparison).  Every intermediate is an exact integer, so all
 * methods return bit-identical results.
 *
 * Number format (block fixed point, one exponent per vector):
 *     value_k = (neg_k ? -1 : +1) * M_k * 2^(exponent - b),   0 <= M_k < 2^b
 * M_k is stored as ceil(b/32) little-endian uint32 limbs, entries one after
 * another (entry-major); neg_k is one uint8 per entry.  For nrhs > 1 the
 * right-hand sides are stored one after another (vector r holds entries
 * r*len .. r*len+len-1).
 *
 * Result rounding (the paper assumes MPFR-style numbers and states no rule):
 * the exact rows Z_i = sum_j (+-M_a)(+-M_x) are rounded to b bits, half to
 * even, with the least exponent E_y for which every rounded mantissa is
 * below 2^b.  E_y is chosen from the exact rows (no double rounding).  An
 * all-zero result has E_y = E_h + E_x; a zero entry has neg = 0.
 *
 * Errors: every call returns an hmv_status; nothing is thrown across this
 * interface.  A call that returns an error writes no output.
 * Concurrency: a plan is not re-entrant; distinct plans may be used from
 * different threads on different streams.
 */
#ifndef HMV_H_
#define HMV_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HMV_OK = 0,
    HMV_EINVAL = 1,        /* bad argument: sizes, b, kind, bits set at or above b, ... */
    HMV_ENOMEM = 2,        /* device or host allocation failed */
    HMV_ECUDA = 3,         /* a CUDA runtime/driver call failed */
    HMV_ETIMEOUT = 4,      /* a bounded device-side wait gave up (kernel returned early) */
    HMV_ENOTLOADED = 5,    /* hmv_matvec before hmv_load_matrix */
    HMV_EFFTBOUND = 6,     /* FFT path: error bound not below 1/2 (no result written) */
    HMV_EUNSUPPORTED = 7,  /* method or configuration the library does not support */
    HMV_EINTERNAL = 8      /* a device-side consistency check failed (a carry or an exact
                              division's remainder out of range): no result is written; this
                              indicates a defect in the library, not in the arguments */
} hmv_status;

typedef enum { HMV_HANKEL = 0, HMV_TOEPLITZ = 1, HMV_CIRCULANT = 2 } hmv_kind;

typedef enum {
    HMV_AUTO = 0,          /* Karatsuba recursion; with levels = -1 and no split flag the
                              cost model also picks the split of the mantissas (none,
                              Karatsuba one or two levels, Toom-4, Toom-6 or Toom-8) and
                              the leaf tile width */
    HMV_SCHOOLBOOK = 1,    /* plain schoolbook on 32-bit limbs, CUDA cores */
    HMV_KARATSUBA = 2,     /* Algorithm 1 to the given depth, tensor-core leaves */
    HMV_FFT64 = 3,         /* split-FP64 FFT with a proven rounding bound; when the bound
                              for the actual data is not below 1/2 the call computes the
                              product with the Karatsuba path instead (counted in
                              hmv_stats.fft_fallbacks) */
    HMV_NTT = 4            /* the same decomposition into 16-bit pieces and one cyclic
                              convolution (Secs. 1-2), done exactly with number-theoretic
                              transforms modulo two 31-bit primes: no error bound to check.
                              Needs (2n-1)(2 ceil(b/16) - 1) <= 2^26 (e.g. n <= 8079 at
                              b = 33220), else hmv_plan returns HMV_EUNSUPPORTED; levels
                              must be -1 or 0 and flags hold no split or tile flag */
} hmv_method;

/* flags for hmv_desc.flags */
#define HMV_FLAG_TIMING 1u     /* record CUDA-event times of each stage (hmv_get_stats) */
#define HMV_FLAG_SIMT_LEAF 2u  /* leaf products on CUDA cores instead of tensor cores */
/* Karatsuba splitting of the mantissas themselves (three products of half
 * the width per level), on top of the index recursion; HMV_AUTO/HMV_KARATSUBA */
#define HMV_FLAG_DIGIT_SPLIT1 4u  /* one level */
#define HMV_FLAG_DIGIT_SPLIT2 8u  /* two levels */
/* Leaf tile width in product digits.  Without either flag HMV_AUTO picks it
 * by its cost model (with the digit split) and the other methods take 256;
 * at most one of the two. */
#define HMV_FLAG_TILE128 16u      /* leaf tiles of 128 product digits */
#define HMV_FLAG_TILE256 128u     /* leaf tiles of 256 product digits */
/* Toom-Cook splitting of the mantissas instead: each mantissa cut into K
 * parts, 2K-1 products of about 1/K of the width, the exact rows recovered by
 * integer interpolation and an exact division (by 360 for K = 4, 1008000
 * for K = 6, 54486432000 for K = 8).  K = 4 evaluates at 0, 1, -1, 2, -2,
 * 1/2 and infinity; K = 6 adds -1/2, 3, -3 and 1/3; K = 8 adds -1/3, 3/2,
 * -3/2 and 2/3.  HMV_AUTO/HMV_KARATSUBA; at most one digit-split flag.
 * Without one, HMV_AUTO picks the digit split (none, Karatsuba one or two
 * levels, Toom-4, Toom-6, Toom-8) by its cost model.  Toom-8 returns
 * HMV_EUNSUPPORTED where its 64-bit interpolation sums could overflow (index
 * depths above 7, n beyond about 16000). */
#define HMV_FLAG_DIGIT_TOOM4 32u  /* needs b > 96 */
#define HMV_FLAG_DIGIT_TOOM6 64u  /* needs b > 160 */
#define HMV_FLAG_DIGIT_TOOM8 256u /* needs b > 224 */

typedef struct {
    int32_t n;        /* matrix order, n >= 1 */
    int32_t b;        /* mantissa bits, 1 <= b <= 1<<20 (HMV_SCHOOLBOOK: one row's operands,
                         8 ceil(b/32) bytes, must fit the device's opt-in shared memory per
                         block, else hmv_plan returns HMV_EINVAL) */
    int32_t nrhs;     /* right-hand sides per hmv_matvec, >= 1 */
    int32_t kind;     /* hmv_kind */
    int32_t method;   /* hmv_method */
    int32_t levels;   /* Karatsuba depth L (levels of Algorithm 1); -1 = cost model */
    uint32_t flags;   /* HMV_FLAG_* */
    int32_t piece_bits; /* HMV_FFT64 only: piece width w in bits (4..20), or 0 to take
                           the largest w whose worst-case error bound is below 1/2;
                           other methods: must be 0 */
} hmv_desc;

typedef struct {
    int32_t len;       /* entries per vector */
    int32_t nrhs;      /* vectors */
    int32_t b;         /* mantissa bits (must equal the plan's b) */
    int32_t exponent;  /* block exponent E (written by hmv_matvec for y) */
    uint32_t *limbs;   /* len*nrhs*ceil(b/32) limbs, caller-owned */
    uint8_t *neg;      /* len*nrhs sign flags, caller-owned */
    int32_t on_device; /* 1: limbs/neg are device pointers (stream-ordered on the
                          plan's stream), 0: host pointers (call is synchronous) */
    int32_t reserved;  /* must be 0 */
} hmv_vec;

typedef struct hmv_plan_s hmv_plan_t;

typedef struct {
    int32_t levels;          /* Karatsuba depth actually used */
    int32_t leaves;          /* 3^levels */
    int32_t leaf_rows_max;   /* largest leaf order */
    int32_t digits;          /* balanced radix-2^8 digits per operand in the tree */
    int64_t leaf_tiles;      /* 128 x leaf_tile_digits output tiles per matvec */
    double leaf_macs;        /* useful digit multiply-adds per matvec in the leaves */
    double leaf_macs_issued; /* digit multiply-adds issued to the tensor cores */
    int64_t device_bytes;    /* device memory held by the plan */
    /* with HMV_FLAG_TIMING: accumulated milliseconds and launch counts */
    double ms_prepass, ms_leaf, ms_post, ms_round, ms_total;
    int64_t launches_leaf, launches_total, matvecs;
    /* HMV_FFT64 and HMV_NTT plans */
    int32_t fft_piece_bits;  /* w (16 for HMV_NTT) */
    int32_t fft_log2_len;    /* K: cyclic convolution length 2^K */
    double fft_bound;        /* error bound of the last matvec (the result is exact when < 1/2) */
    double fft_max_dist;     /* largest |c - round(c)| seen in the last FFT matvec */
    int64_t fft_matvecs;     /* matvecs done by the FFT path */
    int64_t fft_fallbacks;   /* matvecs whose bound failed and that took the integer path */
    double ms_fft;           /* with HMV_FLAG_TIMING: time in the FFT path */
    int32_t leaf_tile_digits; /* product digits per leaf tile (256, or 128 with HMV_FLAG_TILE128
                                 or when HMV_AUTO's cost model prefers it); 0 without tiles */
    int32_t digit_products;  /* products the digit split runs (1; 3 or 9 Karatsuba; 7, 11 or 15
                                for Toom-4, Toom-6 or Toom-8) */
} hmv_stats;

/* Create a plan: checks the descriptor, chooses the recursion depth and
 * allocates device memory.  stream: a cudaStream_t (NULL = legacy default
 * stream).  *out is set only on HMV_OK; release it with hmv_free. */
hmv_status hmv_plan(const hmv_desc *desc, void *stream, hmv_plan_t **out);

/* Load the matrix sequence h (len 2n-1, or n for circulant; nrhs 1).  The
 * plan encodes it into resident device digit planes and runs the matrix
 * side of Algorithm 1, steps 4 and 6, for every level once; h may be freed
 * after the call returns (host) or after the stream reaches it (device). */
hmv_status hmv_load_matrix(hmv_plan_t *plan, const hmv_vec *h);

/* Y = A X for the loaded matrix and a block of nrhs right-hand sides (one
 * shared exponent, as every hmv_vec has).  x: len n, nrhs = plan nrhs.
 * y: len n, nrhs = plan nrhs, same b, limbs and neg allocated by the
 * caller; y->exponent is written: the least exponent over the whole block.
 * x and y must both be host or both be device pointers.  Device pointers:
 * the work is ordered on the plan's stream; the call returns once the
 * exponent has been read back (one stream synchronisation). */
hmv_status hmv_matvec(hmv_plan_t *plan, const hmv_vec *x, hmv_vec *y);

/* Release everything the plan holds.  NULL is ignored.  The plan's stream
 * must still exist; the call waits for the plan's work on it.  The device
 * memory goes back to the library's memory pool (kept for the next plan,
 * without a device-wide synchronisation); hmv_trim_memory returns it to the
 * device. */
void hmv_free(hmv_plan_t *plan);

/* Return the current device's unused pooled memory (freed plans' memory the
 * library keeps for reuse) to the device.  Synchronises the device first. */
hmv_status hmv_trim_memory(void);

/* Device memory hmv_plan would allocate for this descriptor, computed
 * without allocating (admission control by memory footprint). */
hmv_status hmv_plan_bytes(const hmv_desc *desc, uint64_t *bytes);

/* One product for each of `count` distinct loaded plans (Karatsuba
 * tensor-core path with tensor-core leaves, or the exact NTT path; nrhs = 1;
 * orders and precisions may differ): every leaf product of every Karatsuba
 * plan runs in ONE persistent tensor-core launch, the level kernels around
 * it, and every NTT plan runs its transforms, all on plans[0]'s stream.
 * This is the step of a continuous-batching server: the set of plans may
 * change from call to call.  xs[i], ys[i] as in hmv_matvec (all host or all
 * device pointers); every ys[i].exponent is written; the call returns when
 * all are done.  Results are bit-identical to separate hmv_matvec calls.
 * Other methods, external scratch or nrhs != 1: HMV_EUNSUPPORTED. */
hmv_status hmv_matvec_many(int32_t count, hmv_plan_t *const *plans, const hmv_vec *xs, hmv_vec *ys);

/* Plan facts and (with HMV_FLAG_TIMING) stage times. */
hmv_status hmv_get_stats(const hmv_plan_t *plan, hmv_stats *out);

/* Zero the timing counters of hmv_get_stats. */
hmv_status hmv_reset_stats(hmv_plan_t *plan);

/*
 * Batched products (block-Lanczos style workloads): `count` independent
 * Hankel/Toeplitz/circulant matrices, each with its own n, b, kind and
 * block of nrhs right-hand sides (descs[i]; method HMV_AUTO, HMV_KARATSUBA
 * or HMV_NTT, depth -1 for the cost model), advanced together.  Every
 * (matrix, right-hand side) pair is a leaf problem of Algorithm 1 (Sec. 3);
 * the leaf products of all pairs of a wave run in one persistent
 * tensor-core launch, and one hmv_batch_matvec call replays one captured
 * CUDA graph holding every wave and every level kernel.  wave_bytes bounds
 * the device memory of one wave's leaf operands and outputs (pairs are
 * grouped in order; a pair larger than the budget gets a wave of its own).
 * Matrices whose mantissas HMV_AUTO would split (or whose flags ask for a
 * digit split) keep the buffers of a single plan, outside wave_bytes, and
 * run in one round per right-hand side: every such matrix's vector side,
 * one persistent launch over all their digit products per tile width, then
 * their interpolation.  HMV_NTT matrices (the exact NTT path; their size
 * limit as for hmv_plan) keep their own buffers too and run their
 * transforms for each right-hand side in the same graph, on up to eight
 * parallel branches of it (the batch creates that many streams of its own
 * when it has HMV_NTT members, forked from and joined back to `stream`, and
 * destroys them in hmv_batch_free), so that different members' kernels
 * overlap on the device.
 * stream: as for hmv_plan; NULL makes the batch create its own stream
 * (the legacy default stream cannot be captured).  Results are bit-identical
 * to hmv_matvec on each matrix alone.
 */
typedef struct hmv_batch_s hmv_batch_t;
typedef struct {
    int32_t matrices;          /* count */
    int32_t pairs;             /* sum of nrhs */
    int32_t waves;             /* persistent leaf launches per call (waves plus split rounds) */
    int32_t reserved;
    int64_t leaf_tiles;        /* leaf tiles per call */
    double leaf_macs;          /* useful digit multiply-adds per call */
    int64_t device_bytes;      /* device memory held by the batch */
    int64_t graph_launches;    /* graph launches so far (one per hmv_batch_matvec) */
    int64_t kernels_per_graph; /* kernel launches captured in the graph */
} hmv_batch_info;

hmv_status hmv_batch_create(int32_t count, const hmv_desc *descs, void *stream, uint64_t wave_bytes,
                            hmv_batch_t **out);
/* Load matrix `index` (as hmv_load_matrix). */
hmv_status hmv_batch_load_matrix(hmv_batch_t *batch, int32_t index, const hmv_vec *h);
/* xs[i], ys[i]: the blocks of matrix i (all host or all device pointers);
 * every ys[i].exponent is written.  Synchronous: returns after the results
 * (and, for host buffers, their copies) are complete. */
hmv_status hmv_batch_matvec(hmv_batch_t *batch, const hmv_vec *xs, hmv_vec *ys);
hmv_status hmv_batch_get_info(const hmv_batch_t *batch, hmv_batch_info *out);
void hmv_batch_free(hmv_batch_t *batch);

/*
 * Scratch-free schoolbook product (no counterpart in the paper: it is an
 * interface for callers, not part of the method).
 *
 * For callers that cannot allocate device memory while they run: code that
 * must stay inside another runtime's memory budget, code on a path where a
 * cudaMalloc would synchronise the device or fail under a memory cap, and
 * callers with no allocator of their own.  hmv_schoolbook_noalloc computes
 * the same y = A x as hmv_matvec with HMV_SCHOOLBOOK (same rounding, bit for
 * bit) without a plan and without calling cudaMalloc, cudaFree or any
 * allocating routine.  Its only working memory is one scratch array of
 * HMV_NOALLOC_SCRATCH_BYTES compiled into the library as a device variable:
 * every GPU that loads the library holds it until the process exits.
 *
 * Arguments: n, b, kind as in hmv_desc; h_limbs/h_neg (2n-1 entries, or n
 * for circulant), x_limbs/x_neg (n entries) and y_limbs/y_neg (n entries)
 * are DEVICE pointers in the layout of hmv_vec, allocated by the caller;
 * the exponents of h and x are passed by value and E_y is written to the
 * host int *y_exponent.  stream: a cudaStream_t (NULL = legacy default).
 * The call orders its work on the stream and returns after one stream
 * synchronisation (to read E_y back).
 * Limit: with L = ceil(b/32), it needs at most
 *     n * (32 L + 8 L + 13) + 1536  bytes  <=  HMV_NOALLOC_SCRATCH_BYTES
 * (for example n <= 3200 at b = 1024, n <= 100 at b = 33220), and one row's
 * operands, 8 ceil(b/32) bytes, must fit the device's opt-in shared memory
 * per block (227 KB on GB300: b up to about 929,000); larger problems return
 * HMV_EINVAL and do nothing.  Bits at or above b in h or x also return
 * HMV_EINVAL and leave y unwritten.
 * Set-up: the first call on each device looks the scratch array's device
 * address up (cudaGetSymbolAddress) with that device current and keeps it
 * for the life of the process; after a cudaDeviceReset of that device the
 * kept address is no longer valid, so do not call this entry point on it
 * again in the same process.
 * Streams: the call copies E_y to host memory and synchronises the stream,
 * so it must never be made on a stream that is being captured into a CUDA
 * graph; on a capturing stream it returns HMV_EINVAL before queuing work.
 * Sharing: all calls on a device use the same scratch array, which keeps
 * the last call's contents (the call clears what must start at zero).
 * Calls whose work overlaps on the GPU (other streams, other threads) race
 * on it: order them on one stream or otherwise serialise them.
 */
#define HMV_NOALLOC_SCRATCH_BYTES (4u << 20)
hmv_status hmv_schoolbook_noalloc(int32_t n, int32_t b, int32_t kind,
                                  const uint32_t *h_limbs, const uint8_t *h_neg, int32_t h_exponent,
                                  const uint32_t *x_limbs, const uint8_t *x_neg, int32_t x_exponent,
                                  uint32_t *y_limbs, uint8_t *y_neg, int32_t *y_exponent, void *stream);

/* ---- Exact vector operations for Krylov drivers (Lanczos) --------------
 * The paper's introduction motivates fast multiprecision Hankel products by
 * Lanczos-type iterations on these matrices; the two calls below are the
 * vector operations such an iteration needs next to hmv_matvec, with the
 * same exactness contract: every result is the exact one before a single
 * rounding.  Both run on the plan's stream, take device vectors (on_device =
 * 1) of the plan's n and b with nrhs = 1, and return when the result is
 * ready.  The paper describes neither call; they serve the driver in
 * paper_1402_5287_gb300/lanczos.py. */

/* A b-bit scalar: value = (neg ? -1 : 1) * M * 2^exponent, M = sum_q limbs[q]
 * 2^(32 q) (host memory, 1 <= nlimbs <= ceil(b/32) + 1). */
typedef struct {
    const uint32_t *limbs;
    int32_t nlimbs;
    int32_t neg;
    int32_t exponent;
} hmv_scalar;

/* Exact inner product sum_i X_i Y_i of the signed mantissas of x and y (its
 * value is that integer times 2^(x.exponent + y.exponent - 2b)), written to
 * z (host, zl >= 2*ceil(b/32) + 2 limbs, little-endian magnitude) and
 * *z_neg.  HMV_EINVAL for mismatched vectors or a short z.  Large problems
 * (from about 2^26 limb products, b up to about 49,000) run the products as
 * GEMMs of 6-bit digit planes on the tensor cores (cuBLAS, every partial
 * sum exact); the result is the same exact integer either way. */
hmv_status hmv_dot(hmv_plan_t *plan, const hmv_vec *x, const hmv_vec *y, uint32_t *z, int32_t zl,
                   uint8_t *z_neg);

/* y = sum_{k<count} c[k] * xs[k] (count 1..3), exact, then rounded to b bits
 * with the least shared exponent and round-half-even (the same rule as
 * hmv_matvec); y->exponent is written.  y may be one of the xs[k]: every
 * term is read before y is written.  Terms with large scalars on large
 * problems run as GEMMs of digit planes on the tensor cores (as hmv_dot).
 * HMV_EUNSUPPORTED when two terms differ in scale by more than 128 ceil(b/32)
 * bits. */
hmv_status hmv_lincomb(hmv_plan_t *plan, int32_t count, const hmv_scalar *c, const hmv_vec *xs, hmv_vec *y);

/* ---- Test hook for the failure path --------------------------------------
 * Not part of the method and not for production use: it lets tests run the
 * tensor-core leaf kernel's failure path without faulting anything.  The
 * next `launches` leaf launches made directly on a stream (launches captured
 * into a batch's CUDA graph never take it) run with every wait limited to
 * wait_ns nanoseconds (1e6 .. 2e9; the normal limit is 2 s) and with one
 * epilogue warp holding back one release of an accumulator, so that an
 * MMA-issuing thread's wait for it runs out.  The kernel then records a
 * timeout, waits for its own MMAs and for the TMA loads it has in flight,
 * frees its tensor memory and returns; the call that launched it returns
 * HMV_ETIMEOUT and writes no output, and the plan stays usable.
 * launches = 0 disarms the hook.  HMV_EINVAL for arguments out of range. */
hmv_status hmv_test_leaf_stall(int32_t launches, int64_t wait_ns);

/* ---- Measurement --------------------------------------------------------
 * The rate of independent 32-bit Montgomery products (modulo the HMV_NTT
 * path's first prime) that this GPU sustains, from a short timed kernel on
 * `stream` (the best of three launches): the arithmetic that bounds the
 * NTT path's transform stages, used as that path's roofline.  Allocates
 * and frees a small buffer; synchronous. */
hmv_status hmv_measure_montgomery_rate(void *stream, double *products_per_s);

/* Static description of a status code. */
const char *hmv_status_string(hmv_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t hmv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HMV_H_ */
