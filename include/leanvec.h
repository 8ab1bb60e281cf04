/*
 * leanvec.h -- C ABI of the GB300 (sm_103a) LeanVec search library.
 *
 * LeanVec (Tepper et al., "LeanVec: Searching vectors faster by making them
 * fit", arXiv 2312.16335) approximates the inner product <q, x> by
 * <A q, quant(B x)> with A, B in R^{d x D}, d < D (Sec. 2, Eq. 1).  A graph is
 * traversed with the "primary" vectors quant(B x); the best candidates are then
 * rescored with the full-dimensional "secondary" vectors quant(x) and the top k
 * returned (Sec. 2, "Search").  quant() is LVQ, a per-vector scalar quantiser
 * around the dataset mean (cited in Sec. 2).
 *
 * Conventions for every function:
 *   - Returns 0 (LV_OK) or a negative lv_status.  leanvec_last_error() gives a
 *     message for the calling thread.  No C++ exception crosses this ABI.
 *   - Pointers named as "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  Work is enqueued asynchronously on the
 *     given stream (NULL = legacy default stream) unless stated otherwise.
 *   - Matrices are row-major float32: database X is n x D, queries Q are m x D,
 *     projections A and B are d x D (so the paper's X, a D x n column stack, is
 *     the transpose of the X here).
 *   - Ids are int32; n < 2^31.  Inner product is the similarity (higher is
 *     better); ties are broken by the smaller id.
 *   - Errors found while a kernel runs (a clamped capacity, an out-of-range id
 *     in a user graph) are recorded in a per-index device status word and are
 *     returned by leanvec_sync_status().
 */
#ifndef LEANVEC_H
#define LEANVEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lv_stream_t; /* same type as cudaStream_t */

typedef enum {
    LV_OK = 0,
    LV_ERR_ARG = -1,       /* invalid argument; nothing was launched */
    LV_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    LV_ERR_OOM = -3,       /* device allocation failed */
    LV_ERR_CAPACITY = -4,  /* a per-query size exceeded a compiled/allocated capacity */
    LV_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    LV_ERR_CANCELLED = -6, /* reserved for a cancellable call; no call of this version returns it */
    LV_ERR_CORRUPT = -7,   /* malformed input data (a graph id out of range, a damaged index file) */
    LV_ERR_STATE = -8      /* the index lacks what the call needs (no graph, no store) */
} lv_status;

/* Message for the last failing call on this thread ("" if none). */
const char *leanvec_last_error(void);

/* Scratch memory.  The temporaries of the offline calls (operand copies of the
 * tensor-core GEMMs, split-K partials, eigen-solver and fit buffers) come from one
 * stream-ordered memory pool per device owned by the library, which keeps freed
 * blocks for reuse instead of returning them to the driver.  This call returns the
 * unused blocks of `device`'s pool to the driver (blocks freed by work still in
 * flight are returned once a later call finds them idle; synchronise first to
 * release everything).  LV_ERR_ARG for a negative ordinal; LV_OK when the device
 * has no pool yet. */
int leanvec_trim_scratch(int device);

/* ------------------------------------------------------------------------ */
/* Record layout                                                            */
/* ------------------------------------------------------------------------ */
/*
 * An LVQ record of a dim-dimensional vector v (already minus the dataset mean
 * mu) with b in {4, 8} bits:
 *   bytes [0, cb)            codes, cb = dim (b = 8) or ceil(dim / 2) (b = 4);
 *                            for b = 4 code 2j is the low and 2j+1 the high nibble
 *                            of byte j; the code area is zero-padded to a multiple
 *                            of 16 bytes (padding codes decode to l and are never
 *                            multiplied by a non-zero query entry)
 *   bytes [co, co + 16)      float32 {delta, lower, G, H}, co = code area size
 *   stride                   co + 16 rounded up to 32 bytes
 * decode: x_j = mu_j + lower + delta * code_j.  With l = min v, u = max v:
 *   delta = (u - l) / (2^b - 1)   (IEEE float32 division, round to nearest)
 *   code  = floor((v_j - l) / delta + 0.5), clamped to [0, 2^b - 1]; 0 if delta = 0
 * G and H serve the graph build's exact pair score (leanvec_build_graph):
 *   mui_j = round(mu_j * 2^20) (int32),  M = sum_j mui_j code_j (int64),
 *   G = lower * float(sum_j mui_j) * 2^-20 + delta * float(M) * 2^-20,
 *   H = delta * float(sum_j code_j)        (float32, no fused multiply-add)
 * and are NaN when some |mu_j| >= 8.
 * A float32 record (bits = 32, the full-dimensional baseline) is the dim floats
 * zero-padded to a multiple of 32 bytes.
 * In an index with the L2 metric (leanvec_set_metric) an LVQ record has a second
 * 16-byte constants chunk at co + 16: float32 {N, ||x||^2, 0, 0}, N = <y, y> of the
 * decoded record by the build score below (P = sum_j code_j^2, the record paired
 * with itself) and ||x||^2 the squared norm of the original vector (squares and sum
 * in FP64, rounded to float32; N when the original vectors are not known; N is 0
 * in secondary records, which the build does not read); the stride is then co + 32
 * rounded up to 32 bytes.
 * Returns the stride in bytes (of an inner-product index), or a negative lv_status
 * for unsupported bits.
 */
int64_t leanvec_record_stride(int dim, int bits);

/* ------------------------------------------------------------------------ */
/* Stand-alone kernels on caller-owned device buffers                        */
/* ------------------------------------------------------------------------ */

/* Column mean of X (n x dim, device) rounded to float32 into mean (dim, device),
 * accumulated in a fixed order (so repeated calls agree bit for bit): per chunk of
 * 2048 rows in compensated float32 (each addition's rounding error carried in a
 * second float32, TwoSum: about 44 significant bits), the chunks in FP64.  The
 * dataset mean around which LVQ quantises (Sec. 2 cites LVQ for quant()). */
int leanvec_column_mean(const float *X, int64_t n, int dim, float *mean, lv_stream_t stream);

/* LVQ-encode the n rows of V (n x dim, device) around mean (dim, device) into
 * records (n x leanvec_record_stride(dim, bits) bytes, device), bits in {4, 8}.
 * Layout and arithmetic as documented above; the codes are bit-identical to an
 * IEEE float32 evaluation of the stated formula. */
int leanvec_lvq_encode(const float *V, int64_t n, int dim, const float *mean, int bits,
                       uint8_t *records, lv_stream_t stream);

/* Precision of a projection GEMM. */
typedef enum {
    LV_PREC_FP32 = 0,  /* float32 CUDA-core GEMM, float32 accumulate */
    LV_PREC_BF16 = 1,  /* bf16 operands on the tcgen05 tensor cores, float32 accumulate */
    LV_PREC_FP8 = 2,   /* e4m3 operands with per-row scales, float32 accumulate */
    LV_PREC_TF32X3 = 3 /* float32-accurate on the tensor cores: each operand split into tf32
                          hi + lo, three tf32 products (about 21 bits of every float32 product),
                          float32 accumulate; needs D % 4 == 0, 16-byte aligned rows, d <= 256 */
} lv_precision;

/* Y = X P^T: X is n x D, P is d x D, Y is n x ldy with ldy >= d (device); the
 * columns d..ldy-1 of Y are written with zeros.  This is the projection
 * x -> B x (encode) and q -> A q (search) of Eq. 1. */
int leanvec_project(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy,
                    int precision, lv_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Learning the projections (Sec. 2.1 - 2.4)                                 */
/* ------------------------------------------------------------------------ */

/* Second moment K = sum_i x_i x_i^T (D x D float32, device) of the n rows of X
 * (n x D, device): the uncentred K_X = X X^T / K_Q = Q Q^T of Sec. 2.2 "Efficiency"
 * (the caller passes a uniform subsample when n is large).  precision:
 * LV_PREC_FP32 (CUDA cores) or LV_PREC_BF16 (bf16 operands, tcgen05 tensor cores,
 * float32 accumulation). */
int leanvec_second_moment(const float *X, int64_t n, int D, float *K, int precision, lv_stream_t stream);

/* Eigen-decomposition of a symmetric D x D FP64 matrix K (device) by cyclic
 * Jacobi rotations in FP64: evals (D, device, may be NULL) in descending order,
 * evecs (D x D, device) with row r the eigenvector of evals[r], its
 * largest-magnitude entry positive (first index on ties).  Synchronises `stream`. */
int leanvec_eigh(const double *K, int D, double *evals, double *evecs, lv_stream_t stream);

/* The nout leading eigenpairs of a symmetric D x D FP64 matrix K (device; 8 <= D <= 4096,
 * 1 <= nout <= D), the part that LeanVec-ID (Sec. 2.1) and the eigenvector search (Algorithm 2)
 * use: Householder reduction to tridiagonal form (all SMs, one cooperative launch), bisection on
 * Sturm counts for the nout largest eigenvalues, inverse iteration for their tridiagonal
 * eigenvectors (Gram-Schmidt among eigenvalues closer than 1e-5 of the largest magnitude), and
 * the back-transformation; FP64 throughout.  evals (nout, device, nullable) descending, evecs
 * (nout x D, device) rows = unit eigenvectors with the largest-magnitude entry positive (first
 * index on ties), as leanvec_eigh.  Returns LV_ERR_TIMEOUT if a grid barrier of the reduction
 * gave up (seconds).  Synchronises `stream`.  leanvec_fit_id and leanvec_fit_ood use this path
 * whenever they need fewer than D eigenvectors. */
int leanvec_eigh_top(const double *K, int D, int nout, double *evals, double *evecs, lv_stream_t stream);

/* LeanVec-ID (Sec. 2.1, problem "pca"): A = B = M, the d leading eigenvectors of
 * K_X = sum x x^T over the n rows of X (the left singular vectors of the paper's
 * X), computed as second moment (`precision`) + FP64 eigh.  A_out, B_out: d x D
 * float32 (device; B_out may be NULL or equal A_out).  Synchronises `stream`. */
int leanvec_fit_id(const float *X, int64_t n, int D, int d, float *A_out, float *B_out, int precision,
                   lv_stream_t stream);

/* LeanVec-OOD optimisers. */
typedef enum {
    LV_FIT_FW = 0,    /* Frank-Wolfe BCD from A = B = 0 (Algorithm 1) */
    LV_FIT_ES = 1,    /* eigenvector search over beta (Algorithm 2), A = B = P */
    LV_FIT_ES_FW = 2  /* ES, then Frank-Wolfe BCD from A = B = P with the exact line search */
} lv_fit_method;

typedef struct {
    int32_t method;       /* lv_fit_method */
    float alpha;          /* FW step 1 / (t + 1)^alpha, alpha in (0, 1); 0 = 0.5 */
    float tol;            /* FW stop: |f(t+1) - f(t)| / f(t) <= tol; 0 = 1e-3 */
    int32_t max_iter;     /* FW iteration limit; 0 = 500 */
    int32_t line_search;  /* 1 = exact quadratic step (FP64 solve) instead of 1 / (t + 1)^alpha */
    int32_t precision;    /* second moments: LV_PREC_FP32 or LV_PREC_BF16 */
    double es_xatol;      /* ES Brent absolute tolerance on beta; 0 = 1e-5 */
} lv_fit_opts;

typedef struct {
    int32_t iterations;   /* FW iterations run */
    int32_t evaluations;  /* ES loss evaluations */
    double beta;          /* ES: the chosen beta */
    double loss0;         /* FW: loss at the starting point */
    double loss;          /* final loss f(A, B) (trace form, unnormalised K_Q, K_X) */
    double *loss_trace;   /* optional host array: loss after each FW iteration ([0] = start) */
    int32_t trace_capacity;
} lv_fit_report;

/* LeanVec-OOD (Sec. 2.2, problems "leanvec_orthonormal" / "leanvec"): learn A, B (d x D
 * float32, device) minimising f(A, B) = ||Q^T A^T B X - Q^T X||_F^2 through the second
 * moments K_X (n rows of X) and K_Q (m rows of Q, the caller's learning queries),
 * relaxed to the spectral-norm ball.  FW: block coordinate Frank-Wolfe, LMO = polar
 * factor of -grad (Sec. 2.3; FP64 eig of C C^T); ES: Brent over beta in [0, 1] of the
 * loss at P(beta) = the d leading eigenvectors of (1-beta)/m K_Q + beta/n K_X (Sec. 2.4;
 * FP64 eig).  At A = B = 0 the A-gradient vanishes; its LMO then returns the LeanVec-ID
 * solution.  rep (nullable) receives iterations / beta / losses.  Synchronises `stream`. */
int leanvec_fit_ood(const float *X, int64_t n, const float *Q, int64_t m, int D, int d, const lv_fit_opts *opts,
                    float *A_out, float *B_out, lv_fit_report *rep, lv_stream_t stream);

/* Differentiation form of the LeanVec-OOD loss over explicit sample pairs (problem
 * "leanvec_orthonormal" written per pair, Sec. 2.2):
 *   r_ij = q_j^T x_i - (A q_j)^T (B x_i),  L = sum_ij r_ij^2 / (n m)
 * over the m rows of Q (m x D) and the n rows of X (n x D), A, B d x D (all float32,
 * device; d <= 256).
 * fwd writes L to *loss (host; synchronises); the residuals are never stored.  With D a
 * multiple of 4 it computes
 * r_ij = qt_j^T x_i with qt_j = q_j - B^T (A q_j) (float32) on the tensor cores:
 * each operand split into tf32 hi + lo parts, three tf32 products per tile (about 21
 * bits of the float32 products), 128 x 256 tiles, squares summed in float32 per 16
 * residuals and in FP64 per CTA, the CTAs' partials in a fixed order; otherwise 64 x 64
 * float32 CUDA-core tiles with FP64 sums.
 * bwd writes scale * dL/dA and scale * dL/dB (d x D, device):
 *   dL/dA = -2/(nm) sum_ij r_ij (B x_i) q_j^T,  dL/dB = -2/(nm) sum_ij r_ij (A q_j) x_i^T
 * (equal to Eq. "leanvec_gradients" divided by n m).  With D a multiple of 4, on the
 * tensor cores in the same tf32x3 form: R = [r_ij] (m x chunk) is formed per chunk of
 * database rows and kept, as tf32 hi / lo pairs row-major and transposed, in at most
 * 4 GiB of library scratch; U = R X' (X' = X B^T) and V = R^T Q' (Q' = Q A^T) are split-K
 * contractions over it, U accumulated across chunks in chunk order; dL/dA = c U^T Q and
 * dL/dB = c V^T X likewise; every partial sum is combined in a fixed order (the result is
 * deterministic).  Otherwise float32 CUDA-core pair tiles, recomputed per use.  Returns
 * LV_ERR_OOM when the scratch cannot be had and LV_ERR_TIMEOUT when a tensor-core pipeline
 * wait gave up.  Synchronises `stream`. */
int leanvec_ood_loss_fwd(const float *A, const float *B, const float *Q, int64_t m, const float *X, int64_t n,
                         int D, int d, double *loss, lv_stream_t stream);
int leanvec_ood_loss_bwd(const float *A, const float *B, const float *Q, int64_t m, const float *X, int64_t n,
                         int D, int d, float scale, float *gA, float *gB, lv_stream_t stream);

/* Euclidean projection of A (d x D float32, device, in place) onto the spectral-norm
 * unit ball C = {A : ||A||_op <= 1} of Eq. "stiefel_convex_hull": singular values above 1
 * are clipped to 1 (FP64 eig of A A^T).  Keeps a gradient optimiser of the relaxed
 * problem "leanvec" feasible.  Synchronises `stream`. */
int leanvec_spectral_clip(float *A, int d, int D, lv_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Index                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct lv_index lv_index;

/* Create an empty index bound to CUDA device `device` (the library allocates its
 * stores there).  Free with leanvec_index_free. */
int leanvec_index_create(lv_index **out, int device);
int leanvec_index_free(lv_index *idx);

/* Similarity of an index (set before it holds a store; LV_ERR_STATE otherwise):
 *   LV_METRIC_IP  inner product <q, x> (the paper's setting; the default)
 *   LV_METRIC_L2  squared Euclidean distance, ranked by the score 2 <q, x> - ||x||^2
 *                 (= ||q||^2 - ||q - x||^2: the query's norm is a per-query constant).
 * With L2 the primary score is 2 <A q, decode(primary)> - ||x||^2, the rerank score
 * 2 <q, decode(secondary)> - ||x||^2 (||x||^2 of the original vector, stored per
 * record), the float32 baseline and FP16 secondaries use 2 <q, x> - ||x||^2 of their
 * own values, and the graph build scores -||y_a - y_b||^2 between decoded primaries
 * (leanvec_build_graph) with the entry point the primary nearest the mean. */
typedef enum { LV_METRIC_IP = 0, LV_METRIC_L2 = 1 } lv_metric;
int leanvec_set_metric(lv_index *idx, int metric);

typedef struct {
    int64_t n;              /* database size */
    int32_t D;              /* original dimensionality */
    int32_t d;              /* primary dimensionality (D for the float32 baseline) */
    int32_t primary_bits;   /* 4, 8, or 32 (float32 records) */
    int32_t secondary_bits; /* 8 (LVQ-8), 16 (FP16), or 0 when there is no secondary store */
    int64_t primary_stride;
    int64_t secondary_stride;
    int32_t R;              /* graph max out-degree, 0 when no graph */
    int32_t entry;          /* search entry point, -1 when no graph */
    float mu2;              /* build-score constant sum_j (mui_j 2^-20)^2 */
    int32_t last_search_kernels; /* kernels the last leanvec_search call launched (0 before any) */
} lv_index_info;

int leanvec_index_info(const lv_index *idx, lv_index_info *out);

/* Index files (the paper has no counterpart; they let a built index be searched again without
 * re-encoding or rebuilding).  One file holds the metric, the sizes, the primary store with its
 * mean, the secondary store with its mean (when present), the graph and its entry point.
 * Layout, little-endian, 96-byte header:
 *   0  char[8] "LEANVEC" (NUL-terminated)   8  u32 version = 1   12 u32 header bytes = 96
 *   16 i32 metric  20 i32 D  24 i32 d  28 i32 primary bits (4, 8, 32)  32 i32 secondary bits
 *      (0, 8, 16)  36 i32 R (0 = no graph)  40 i32 entry (-1 without a graph)  44 f32 mu2
 *   48 i64 n  56 i64 primary stride  64 i64 secondary stride (0 without secondaries)
 *   72 24 zero bytes
 *   96 primary records (n x primary stride bytes), primary mean (d float32; not for float32
 *      records), secondary records (n x secondary stride bytes), secondary mean (D float32; LVQ-8
 *      secondaries only), graph (n x R int32)
 *   then u64 checksum of every preceding byte: 64-bit FNV-1a (offset basis 0xcbf29ce484222325,
 *   prime 0x100000001b3) applied to the little-endian 64-bit words of the byte stream, the last
 *   word zero-padded.
 * leanvec_index_save synchronises `stream`, copies the stores to the host and writes `path`
 * (LV_ERR_STATE for an index without a store, LV_ERR_ARG when the file cannot be written).
 * leanvec_index_load reads and validates the whole file first -- magic and version, header
 * fields against each other, strides against the record geometry, the file size, the checksum,
 * every graph id in [-1, n) -- and returns LV_ERR_CORRUPT (index unchanged) on any mismatch;
 * then it replaces the index's stores (and metric) with the file's on the index's device and
 * synchronises `stream`.  Validation holds the whole file in host memory (about 11.6 GB for
 * 10^7 x 768 with LVQ-4 primaries and LVQ-8 secondaries); a device allocation or copy that fails
 * after it (LV_ERR_OOM / LV_ERR_CUDA) leaves the index without stores (load again or re-encode).
 * leanvec_index_file_check performs the same validation without a device and fills `out`
 * (nullable) from the header. */
int leanvec_index_save(const lv_index *idx, const char *path, lv_stream_t stream);
int leanvec_index_load(lv_index *idx, const char *path, lv_stream_t stream);
int leanvec_index_file_check(const char *path, lv_index_info *out);

/* Device pointers to the index's stores (read-only views, owned by the index;
 * valid until the index is freed or re-encoded). Any output may be NULL. */
int leanvec_index_buffers(const lv_index *idx, const uint8_t **primary, const float **primary_mean,
                          const uint8_t **secondary, const float **secondary_mean,
                          const int32_t **graph);

/* Encode the database (Sec. 2 "primary vectors" and "secondary vectors"):
 *   primary   = LVQ_{primary_bits}(B x - mu_B), mu_B = mean of B x over the database
 *   secondary = LVQ_8(x - mu), mu = mean of x       (secondary_bits = 8)
 *             = x rounded to IEEE half precision    (secondary_bits = 16, the FP16 secondaries of
 *               Sec. 3's experiments: D halves padded to 32 bytes, no constants; the rerank score
 *               is <q, fp16(x)> accumulated in float32)
 * X: n x D (device), B: d x D (device).  primary_bits in {4, 8};
 * secondary_bits in {8, 16, 0} (0: no secondary store, search cannot rerank).
 * projection_precision: lv_precision of the B x GEMM.  Replaces any previous
 * store and graph of the index. Synchronises `stream` before returning. */
int leanvec_encode(lv_index *idx, const float *X, int64_t n, int D, const float *B, int d,
                   int primary_bits, int secondary_bits, int projection_precision,
                   lv_stream_t stream);

/* Install the primary store from already reduced vectors: Y is n x d (device, e.g.
 * B x computed by the caller), mean (d, device) the vector to quantise around, or
 * NULL for the column mean of Y; bits in {4, 8}; D is the dimensionality of the
 * original vectors (the row length of the queries given to leanvec_search).  Drops
 * the graph, and the secondary store when n changes. Synchronises `stream`. */
int leanvec_set_primary(lv_index *idx, const float *Y, int64_t n, int d, const float *mean, int bits, int D,
                        lv_stream_t stream);

/* Install the LVQ-8 secondary store from the original vectors X (n x D, device)
 * around mean (D, device) or, when NULL, the column mean of X.  n and D must match
 * the primary store. Synchronises `stream`. */
int leanvec_set_secondary(lv_index *idx, const float *X, int64_t n, int D, const float *mean,
                          lv_stream_t stream);

/* Full-dimensional float32 baseline: the primary store holds x itself (D floats),
 * no projection, no secondary. Synchronises `stream` before returning. */
int leanvec_encode_fp32(lv_index *idx, const float *X, int64_t n, int D, lv_stream_t stream);

/* Install a graph: adj is n x R int32 (device), -1 marks an empty slot.  Repeated
 * ids within a row are removed (first kept).  entry < 0 selects the default entry
 * argmax_i <mu, decoded primary_i> (ties -> smaller id).  R <= 128. */
int leanvec_set_graph(lv_index *idx, const int32_t *adj, int R, int32_t entry, lv_stream_t stream);

/* Copy the graph (n x R int32) into adj (device) and the entry into *entry (host). */
int leanvec_get_graph(const lv_index *idx, int32_t *adj, int32_t *entry, lv_stream_t stream);

typedef enum { LV_PRUNE_SCALED = 0, LV_PRUNE_UNIT_L2 = 1 } lv_prune_rule;

/* Build the graph on the primaries (App. A: search + prune for every node; App. D:
 * Vamana with R, L, alpha).  Batch-synchronous Vamana:
 *   - initial graph: node v takes the first min(R, n-1) ids splitmix64(seed, v, j)
 *     mod n (j = 0, 1, ..) that are neither v nor repeated;
 *   - order: Fisher-Yates permutation with draws splitmix64(seed + 1, i, 0) mod (i+1);
 *   - pass t uses alpha_t = 1 for t < passes - 1 and alpha in the last pass;
 *   - each batch of `batch` nodes searches the graph as it was at the batch start
 *     (query = the node's primary, beam L_build, from the entry), prunes
 *     pool = beam u old out-list (minus itself) with RobustPrune -- drop p' when
 *       LV_PRUNE_SCALED:  alpha * s(p*, p') >= s(p, p')
 *       LV_PRUNE_UNIT_L2: alpha * s(p*, p') >= s(p, p') + alpha - 1
 *     (the second is Vamana's L2 rule alpha d(p*,p') <= d(p,p') with d = 2 - 2 s, i.e. for
 *     unit-norm vectors; the two coincide at alpha = 1) -- then adds the reverse edges by
 *     (target, source) ascending, pruning targets that exceed R;
 *   - pair scores are the exact build score described with the record layout,
 *     so the adjacency is reproducible bit for bit; with the L2 metric the pair score
 *     is -||y_a - y_b||^2 = 2 <y_a, y_b> - (N_a + N_b) (float32, the sum of the self
 *     scores first) and LV_PRUNE_SCALED with alpha > 1 is Vamana's rule on squared
 *     distances; the entry point is argmax 2 G_i - N_i (the primary nearest the mean)
 *     instead of argmax G_i.
 * splitmix64(s, a, b) is the SplitMix64 finaliser applied to
 * s + 0x9E3779B97F4A7C15 * (1 + a * 2^32 + b).  R <= 128, L_build <= 512.  If one
 * batch gives a target more new sources than its reverse-edge pool holds (about
 * 4 R + 256, shared-memory bound), the sources beyond are dropped (lowest ids kept)
 * and leanvec_sync_status reports LV_ERR_CAPACITY; smaller batches avoid it. */
int leanvec_build_graph(lv_index *idx, int R, int L_build, float alpha, int passes, int batch,
                        uint64_t seed, int prune_rule, lv_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Search (Sec. 2 "Search"; App. D "greedy traversal with backtracking")     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t k;         /* results per query (<= ldo) */
    int32_t L;         /* beam width (search window) */
    int32_t rerank;    /* candidates rescored with the secondary store; 0 = no rerank */
    int32_t max_hops;  /* expansion limit, 0 = none */
} lv_query_desc;

typedef struct {
    lv_query_desc uniform;   /* used for every query when desc == NULL */
    int32_t projection;      /* lv_precision of the q -> A q GEMM */
    int32_t hash_slots;      /* visited-cache slots per query (power of two; 0 = max(1024, 4 L) up to
                                8192 slots of 32-bit ids, or twice as many 16-bit tags, see
                                visited_bits) */
    int32_t warps_per_block; /* 0 = default */
    int32_t width;           /* search width: beam members expanded per round, 1..4 (0 = 1);
                                width * R <= 256.  1 is the classic best-first traversal */
    int32_t warps_per_query; /* warps that serve one query, 1, 2 or 4, dividing width (0 = 1):
                                each expands width / warps_per_query of a round's parents.
                                Results do not depend on it; with more warps per query each
                                query finishes sooner (shorter batch tail) */
    void *event_begin;       /* optional cudaEvent_t recorded on `stream` right before the */
    void *event_end;         /* beam-search kernel and right after the rerank kernel (or the
                                beam-search kernel without rerank) (profiling); may be NULL */
    int32_t queries_per_warp; /* 1: one query per warp (or per team of warps_per_query warps);
                                2: two queries per warp, one per 16 lanes, with a visited cache of
                                16-bit tags -- needs LVQ primaries, warps_per_query 1, width <= 2,
                                width * R <= 128 and n <= 65535 * hash_slots / 4 (the effective
                                slots: hash_slots is raised to 2 x L rounded up to 32, to a power
                                of two); 0 = 1.  Results do not depend on it: the same rounds,
                                beam and answers; the visited cache may forget different ids, so
                                lv_search_stats.scored may differ.  Both run the same number of
                                instructions per query; 2 holds 40 queries per SM instead of 24 and
                                is faster when the index's primaries and graph sit in L2 and the
                                batch spans several waves, 1 when they stream from DRAM */
    int32_t visited_bits;     /* slot width of the visited cache of one query per warp: 32 (whole
                                ids, buckets of 4 slots; 0 = 32) or 16 (tags, buckets of 8: id x is
                                kept as x >> b in bucket (x xor (x >> b)) mod 2^b of the 2^b =
                                slots / 8 buckets, which names x exactly; needs n <= 65535 * slots
                                / 8, else LV_ERR_ARG; with hash_slots 0 the default slot count is
                                doubled: the same bytes).  Results do not depend on it (the cache
                                may forget ids but never reports an unvisited one); 16 forgets
                                fewer ids, so fewer records are scored again
                                (lv_search_stats.scored), at a slightly longer lookup.  Ignored
                                with queries_per_warp 2 */
} lv_search_params;

/* Per-query counters (device, m entries) when stats != NULL. */
typedef struct {
    int32_t hops;    /* beam expansions */
    int32_t scored;  /* primary records scored (re-scores of evicted visited ids included) */
} lv_search_stats;

/* Search m queries Q (m x D, device).  A (d x D, device) projects the queries
 * (ignored for a float32 baseline index).  desc (device, m entries) gives per-query
 * {k, L, rerank, max_hops}; NULL uses params->uniform.  For each query the `width`
 * best unexpanded beam members are expanded per round until none is left (or
 * max_hops expansions); the top
 * min(rerank, |beam|) members are rescored with the secondary store against the
 * unreduced query and the best k written, sorted by score (ties -> smaller id), to
 * ids/scores (m x ldo, device); the rest of each row (fewer than k reachable
 * candidates, or k < ldo) is filled with -1 / -inf.  Reported scores are the
 * decoded inner products (secondary after rerank, primary otherwise).
 * Streams: the work is ordered after `stream`'s earlier work and `stream`'s later
 * work waits for all of it.  With rerank and m above one wave of the beam kernel's
 * resident query slots (and not a multiple of it), the queries past 90 % of the last
 * whole wave run as a second launch on a stream of the index's own, forked from and
 * joined back to `stream` by events (this also holds inside a CUDA-graph capture of
 * `stream`); results do not depend on it.  Calls on one index are not thread-safe. */
int leanvec_search(lv_index *idx, const float *Q, int64_t m, const float *A,
                   const lv_search_params *params, const lv_query_desc *desc,
                   int32_t *ids, float *scores, int ldo, lv_search_stats *stats,
                   lv_stream_t stream);

/* leanvec_search over queries and results in HOST memory (Sec. 2 "Search"; the staging is
 * this library's).  Q is m x D float32 and desc (nullable) m entries in host memory; ids /
 * scores (m x ldo) are host memory that receives the results.  The m queries are searched in
 * batches of `batch` rows (batch <= 0 or >= m: one batch); each batch is copied to a device
 * slot of the index, searched exactly as one leanvec_search call over those rows (same
 * results), and its results copied back.  Two slots alternate, and the copies run on two copy
 * streams of the index's own, so that batch i + 1's queries go in and batch i - 1's results
 * come out while batch i is searched; the searches themselves stay in order on `stream`.
 *   - Asynchronous like leanvec_search: the copies start after `stream`'s earlier work and
 *     `stream`'s later work waits for all of them; the host result buffers are complete once
 *     `stream` has completed (e.g. cudaStreamSynchronize), and Q / desc must stay unchanged
 *     until then.  Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister) for
 *     the copies to overlap; pageable memory works but its copies do not overlap.
 *   - The slots (2 x batch x (4 D + 8 ldo [+ 16]) bytes) are device workspace of the index,
 *     grown with cudaMalloc on first use at a batch size and kept until the index is freed.
 *   - params->event_begin / event_end are ignored.  Successive calls on one index must be
 *     ordered by the caller (the same `stream`, or events), as for leanvec_search.
 *   - Errors: as leanvec_search (arguments are checked per batch before its launches); a
 *     failure stops issuing batches, and `stream` still waits for the copies issued. */
int leanvec_search_host(lv_index *idx, const float *Q, int64_t m, const float *A,
                        const lv_search_params *params, const lv_query_desc *desc,
                        int32_t *ids, float *scores, int ldo, int64_t batch, lv_stream_t stream);

/* leanvec_search without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc while they serve
 * queries -- hosts whose device memory is owned by their own pool allocator and
 * that forbid libraries from allocating behind their back, or latency-bound
 * serving loops that cannot afford the implicit device synchronisation and the
 * possible failure of an allocation in the middle of a request.  leanvec_search
 * grows a workspace in the index with cudaMalloc on first use at a given batch
 * size; this variant instead uses one static 16 MiB device array compiled into
 * the library (held on every GPU that loads the library until the process exits)
 * and calls no cudaMalloc, cudaFree or allocating routine.
 *   - Same arguments, semantics and results as leanvec_search, except that for an LVQ
 *     index the projection must be LV_PREC_FP32, or LV_PREC_BF16 with 16-byte aligned
 *     query rows (D a multiple of 4: Q is converted inside the GEMM, so only the bf16
 *     copy of A needs scratch) -- a float32 index ignores the projection, as
 *     leanvec_search does -- and that the batch is one launch (no second stream).
 *   - Capacity: 256 + m * 4 * ldq [+ m * 4 * (Lc + 1) when the search reranks]
 *     [+ 2 d ldx with the bf16 projection, ldx = D rounded up to 8] bytes, each
 *     part rounded up to 256, must fit in 16 MiB, where ldq is the
 *     primary dimension rounded up to whole 16-byte code chunks (d for LVQ-8 with
 *     d a multiple of 16) and Lc is params->uniform.L rounded up to 32 (e.g.
 *     m <= 13,000 queries at d = 160, L = 160 with rerank; m <= 26,000 without);
 *     larger batches return LV_ERR_CAPACITY before anything is launched -- split
 *     them.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the same array and finds the previous call's
 *     contents in it (the work counter is cleared by each call): calls whose work
 *     overlaps on the GPU (different streams, or host threads issuing
 *     concurrently) race on it and must be serialised by the caller. */
int leanvec_search_noalloc(lv_index *idx, const float *Q, int64_t m, const float *A,
                           const lv_search_params *params, const lv_query_desc *desc,
                           int32_t *ids, float *scores, int ldo, lv_search_stats *stats,
                           lv_stream_t stream);

/* Synchronise `stream` and return (and clear) the index's device status word. */
int leanvec_sync_status(lv_index *idx, lv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LEANVEC_H */
