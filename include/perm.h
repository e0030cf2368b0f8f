/*
 * perm.h -- C ABI of the GB300 sparse-permanent library (libperm.so).
 *
 * What it computes (Elbek & Kaya, "Fully-Automated Code Generation for
 * Efficient Computation of Sparse Matrix Permanents on GPUs"):
 *
 *   perm(A) = sum over permutations s of prod_i a_{i,s(i)}                (Eq. 1)
 *
 * evaluated with the Nijenhuis-Wilf form of Ryser's formula (Eq. 2, Sec. II):
 * the 2^(n-1) subsets of the first n-1 columns are walked in Gray-code order
 * (Algorithm 1), each GPU thread owning an aligned chunk of the walk (Sec. II-A,
 * Lemma 1) and keeping its row-sum vector x in registers (Sec. III), with the
 * rows of x split between registers and global memory under the permanent
 * ordering and partitioning of Sec. V (Algorithms 3 and 4).
 *
 * Conventions shared by every entry point:
 *   - No C++ exception crosses this boundary.  Every call returns a
 *     perm_status_t; perm_last_error() gives a thread-local message for the
 *     last failing call on the calling thread.
 *   - Matrices are borrowed for the duration of the call: the library copies
 *     what it keeps (into plan- or server-owned host and device memory).
 *     Result structs are caller-allocated.  Handles are opaque.
 *   - Matrices are square, 1 <= n <= 64, given in CSR or CSC with 0-based
 *     int32 indices strictly increasing inside each row (CSR) or column (CSC).
 *     Out-of-range or repeated indices give PERM_ERR_PATTERN.  Explicit zero
 *     values are dropped on ingest.
 *   - Streams are cudaStream_t values passed as void*; NULL is the legacy
 *     default stream.  A call that takes a stream returns after the result has
 *     been copied back (it synchronises that stream).
 *   - FP64 results carry the permanent as an unevaluated pair f64 + f64_lo.
 *     Exact results (PERM_I64 inputs) are bit-exact; the plan refuses inputs
 *     whose a-priori bound does not fit the widest exact mode (PERM_ERR_OVERFLOW).
 *   - Every kernel the library launches is its own hand-written CUDA (or CUDA
 *     C++ it generates and compiles with NVRTC for sm_103a).  There is no CPU
 *     fallback: without a usable CUDA device every call that has a walk to do
 *     returns PERM_ERR_CUDA (a matrix without a perfect matching, or an empty
 *     sub-range, needs no walk and gives 0).
 */
#ifndef PERM_H
#define PERM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PERM_OK = 0,
    PERM_ERR_ARG = 1,        /* NULL pointer, bad enum, bad option value            */
    PERM_ERR_SIZE = 2,       /* n outside [1, 64], nnz inconsistent, count < 0      */
    PERM_ERR_PATTERN = 3,    /* index out of range / not strictly increasing        */
    PERM_ERR_OVERFLOW = 4,   /* exact path: |perm| bound too large for 2^191 mode;  */
                             /* or integer entries too large for int32 row sums     */
    PERM_ERR_CUDA = 5,       /* a CUDA runtime/driver call failed (see last error)  */
    PERM_ERR_NVRTC = 6,      /* generating/compiling a per-matrix kernel failed     */
    PERM_ERR_NOMEM = 7,      /* host or device allocation failed                    */
    PERM_ERR_TIMEOUT = 8,    /* timeout_ms passed: the device-side deadline of a    */
                             /* walk, or a server request that waited too long      */
    PERM_ERR_BUSY = 9,       /* server refused a submit (admission budget full)     */
    PERM_ERR_NOT_READY = 10, /* perm_poll: the ticket has not finished yet          */
    PERM_ERR_CANCELLED = 11, /* server shut down before the ticket finished         */
    PERM_ERR_INTERNAL = 12   /* a self-check failed (e.g. exact sum not divisible)  */
} perm_status_t;

/* The value type of a matrix selects the arithmetic path. */
typedef enum {
    PERM_F64 = 0,  /* double entries; FP64 walk, compensated reduction            */
    PERM_I64 = 1   /* int64 entries; exact walk modulo 2^(64w), w = 1..3          */
} perm_value_t;

typedef enum { PERM_CSR = 0, PERM_CSC = 1 } perm_layout_t;

/* A borrowed sparse matrix.  ptr has n+1 entries, idx and vals have nnz.
   vals points to double (PERM_F64) or int64_t (PERM_I64). */
typedef struct {
    int32_t n;
    int32_t nnz;
    perm_layout_t layout;
    const int32_t *ptr;
    const int32_t *idx;
    perm_value_t vtype;
    const void *vals;
} perm_matrix_t;

/* Column ordering (Sec. V and Sec. VI-B).  The last column of the order is the
   one the Nijenhuis-Wilf variant never flips. */
enum {
    PERM_ORDER_AUTO = 0,    /* the cheaper of DEGREE and PAPER under the step-cost model, */
                            /*   then SEARCH from it                                      */
    PERM_ORDER_NONE = 1,    /* columns as given                                          */
    PERM_ORDER_DEGREE = 2,  /* ascending nonzero count (Sec. VI-B, CPU-SparsePerman)    */
    PERM_ORDER_PAPER = 3,   /* PermanentOrdering, Algorithm 3                            */
    PERM_ORDER_SEARCH = 4   /* reported when AUTO's pairwise column swaps lowered the     */
                            /*   cost model of the scheme the walk runs (FP64: two-state */
                            /*   or paired chain; exact: one chain); as an option, same  */
                            /*   as AUTO                                                  */
};

/* Which kernel family runs the walk. */
enum {
    PERM_ENGINE_AUTO = 0,     /* codegen for single large matrices, generic otherwise     */
    PERM_ENGINE_GENERIC = 1,  /* precompiled kernels, matrix read from shared memory      */
    PERM_ENGINE_CODEGEN = 2,  /* per-matrix CUDA C++ generated and compiled with NVRTC    */
    PERM_ENGINE_XSHARED = 3   /* the GPU-SparsePerman baseline of Sec. VI-B (an ablation): */
                              /*   x in shared memory, columns read from a CSC image, zero */
                              /*   tracking, the product of all n rows at every step;      */
                              /*   FP64 inputs only                                         */
};

/* Arithmetic of the FP64 path (integer inputs are always exact).  The walk's
   sum alternates in sign (Sec. II), so its rounding error is about
   n 2^-53 sum_g |term_g|, which can be far above 2^-53 |perm| when the terms
   cancel.  Double-double arithmetic (every x_i, product and sum an unevaluated
   pair of doubles, FMA-based exact products) lowers that to a few 2^-104
   sum_g |term_g|, at several times the FP64 cost. */
enum {
    PERM_PREC_AUTO = 0,  /* FP64; a whole walk of n <= 32 whose estimate n 2^-53 sum|terms| / |perm|  */
                         /*   exceeds 1e-9 (or whose FP64 result is 0) is rerun in double-double       */
    PERM_PREC_F64 = 1,   /* FP64 only                                                                */
    PERM_PREC_DD = 2     /* double-double (generic kernels, n <= 48)                                  */
};

/* Option flags. */
enum {
    PERM_FLAG_NO_KERNEL_CACHE = 1,  /* codegen: compile even if this source was compiled before */
    PERM_FLAG_NO_GRAPH = 2,         /* perm_compute: never replay the plan as a CUDA graph     */
    PERM_FLAG_PAIRED_CHAIN = 4,     /* codegen FP64: the paired chain even where the two-state */
                                    /*   chains cost fewer operations per step                 */
    PERM_FLAG_PURE_REG = 8,         /* codegen: the paper's CodeGen-PureReg scheme (Sec. III-B,*/
                                    /*   Listings 2-3): every row of x in registers and the    */
                                    /*   product of all n rows at every step (no product      */
                                    /*   chain, no zero skip); an ablation baseline            */
    PERM_FLAG_ABS_SUM = 16          /* codegen FP64: accumulate abs_term_sum even where it is  */
                                    /*   not needed (it costs about a tenth of the speed of a  */
                                    /*   generated FP64 kernel; the generic kernels always     */
                                    /*   keep it)                                               */
};

/* Options; a zeroed struct (or NULL) means "choose automatically". */
typedef struct {
    int32_t ordering;      /* PERM_ORDER_*                                                 */
    int32_t engine;        /* PERM_ENGINE_*                                                */
    int32_t reg_rows;      /* codegen: rows of x kept in registers (k of Algorithm 4);     */
                           /*   0 = Algorithm 4 decides, n = all in registers              */
    int32_t chunk_log2;    /* K: each thread walks aligned chunks of 2^K Gray indices;     */
                           /*   0 = auto; a K below the kernel's unrolled block (2^5      */
                           /*   steps; 2^7 for generated FP64 kernels unless most terms   */
                           /*   of the walk are zero) is raised to it,                    */
                           /*   and a range must be aligned to the chunk (else           */
                           /*   PERM_ERR_ARG)                                              */
    int32_t threads;       /* resident threads of the persistent grid; 0 = auto            */
    int32_t exact_words;   /* exact path modulus 2^(64w): 0 = smallest w the bound allows, */
                           /*   and a whole walk then runs in the narrowest ring of 32-bit */
                           /*   limbs (2w-1 or 2w) that holds 2^(n-1) perm with its sign; */
                           /*   an explicit w walks modulo 2^(64w)                         */
    int32_t zero_skip;     /* 0 = on (skip 2^B-step blocks whose products are all zero),   */
                           /*   1 = off                                                    */
    int32_t flags;         /* PERM_FLAG_* bits                                             */
    double gr_ratio;       /* Algorithm 4 GRratio; 0 = the library's GB300 value           */
    uint64_t g_lo, g_hi;   /* Gray-index sub-range [g_lo, g_hi); both 0 = whole range.     */
                           /*   Both ends must be multiples of 32 (g_hi may also be       */
                           /*   2^(n-1)).  A sub-range result is the raw partial sum (see  */
                           /*   perm_result_t); an empty one [g, g), g > 0, gives 0 with   */
                           /*   steps = 0 and nothing launched.                            */
    int32_t timeout_ms;    /* device-side deadline for one compute: warps stop taking work */
                           /*   once the GPU clock passes it, and the call returns         */
                           /*   PERM_ERR_TIMEOUT (the context stays usable); 0 = none      */
    int32_t precision;     /* PERM_PREC_*: arithmetic of FP64 inputs (sub-ranges and       */
                           /*   checkpointed runs: AUTO means FP64)                         */
    int32_t shared_rows;   /* codegen: of the rows beyond reg_rows, this many live in      */
                           /*   shared memory (x[(slot - k) * 256 + thread] per block), the */
                           /*   rest in global memory -- the three-level placement of the  */
                           /*   Gray-frequency order (Sec. V, Sec. VIII); 0 = none         */
    int32_t reserved2;
} perm_opts_t;

/* Result of one permanent (or one Gray sub-range). */
typedef struct {
    perm_status_t status;
    perm_value_t vtype;
    /* PERM_F64: perm = f64 + f64_lo.  For a sub-range: the partial sum
       sum_{g in [g_lo,g_hi)} (-1)^g prod_i x_i(g) (no final factor). */
    double f64, f64_lo;
    /* PERM_I64: perm as a signed 128-bit integer (lo word, hi word).      */
    uint64_t i128_lo;
    int64_t i128_hi;
    /* PERM_I64 sub-range: sum_g (-1)^g prod_i 2x_i(g) modulo 2^(64 w),
       little-endian words, w = exact_words.                              */
    uint64_t partial[3];
    int32_t exact_words;
    int32_t engine;        /* PERM_ENGINE_GENERIC or PERM_ENGINE_CODEGEN that ran     */
    int32_t ordering;      /* PERM_ORDER_* that was used                              */
    int32_t reg_rows;      /* k: rows of x in registers                               */
    int32_t reg_cols;      /* c: columns that touch register rows only               */
    int32_t chunk_log2;    /* K                                                       */
    int32_t threads;       /* resident threads of the launch                          */
    int32_t regs_per_thread;
    uint64_t steps;        /* Gray indices walked                                     */
    double ms_plan;        /* host preprocessing                                      */
    double ms_compile;     /* NVRTC + module load (0 when cached or generic)          */
    double ms_kernel;      /* device time of the walk + reduction (CUDA events)       */
    double fp_ops_per_step;/* counted arithmetic ops per Gray step (cost model): FP64 */
                           /*   operations, or on the exact path integer multiply     */
                           /*   operations (perm_inspect_t.ring_ops_per_step)         */
    double zero_skip_frac; /* fraction of the walk skipped as all-zero: of the warp's */
                           /*   2^B-step blocks (32 chunks each, idle lanes of a      */
                           /*   range's last task included) for the block walks, of   */
                           /*   the threads' steps for PERM_ENGINE_XSHARED; 0 for the */
                           /*   direct kernel (n <= 8).  Sec. VI-E: repeated values   */
                           /*   leave zero entries in x; zero spans skip them.        */
    /* FP64 inputs: sum over the walk's Gray indices of |prod_i x_i(g)|, times 2 for
       a whole walk (the scale of the permanent), raw for a sub-range.  It is
       accumulated in FP32 on the GPU (relative accuracy about 1e-5); terms below
       2^-246 of the a-priori largest term are not counted.  abs_term_sum / |perm|
       is the cancellation of the alternating sum (Sec. II): an FP64 result is good
       to about n 2^-53 of it, a double-double one to about 2^-100 of it.  0 for
       integer inputs, and 0 (not computed) from a generated FP64 kernel of n > 32,
       a sub-range or precision F64 unless PERM_FLAG_ABS_SUM is set.          */
    double abs_term_sum;
    int32_t precision;     /* FP64 inputs: PERM_PREC_F64 or PERM_PREC_DD that produced */
                           /*   the value; 0 for integer inputs                         */
    int32_t shared_rows;   /* codegen: rows of x in shared memory                      */
} perm_result_t;

typedef struct perm_plan_s *perm_plan_t;

/* Validates A, orders and partitions it (Algorithms 3 and 4), picks the chunk
   plan, uploads what the kernels need and, for the codegen engine, generates
   and compiles the matrix-specific kernel (cached by structure and values).
   A matrix without a perfect matching (an empty row or column included) gets
   a plan whose compute returns 0 without launching.  Needs a CUDA device.
   Errors: ARG, SIZE, PATTERN, OVERFLOW, CUDA, NVRTC, NOMEM. */
perm_status_t perm_plan_create(const perm_matrix_t *A, const perm_opts_t *opts, perm_plan_t *out);

/* Runs the Gray-code walk of a plan on `stream` and fills *out.  The plan's
   device buffers are reused; two perm_compute calls on one plan must not
   overlap.  From the second call on, the plan's launches (workspace reset,
   walk, reduction, result copy) are captured once into a CUDA graph and
   replayed with one launch (unless PERM_FLAG_NO_GRAPH).
   Errors: ARG, CUDA, INTERNAL. */
perm_status_t perm_compute(perm_plan_t plan, void *stream, perm_result_t *out);

/* Frees a plan (NULL is allowed). */
void perm_plan_destroy(perm_plan_t plan);

/* Computes `count` permanents in one persistent launch per kernel family
   (NMAX bucket x arithmetic) fed by a device work queue (the matrices may
   differ in n and value type); the families' launches are captured as one
   CUDA graph (PERM_FLAG_NO_GRAPH launches them directly).  Precision AUTO
   reruns the ill-conditioned FP64 matrices in double-double as one more
   launch.  out has `count` entries; out[i].status reports each matrix on its
   own.  opts applies to every matrix (sub-ranges are not allowed here).
   Errors: ARG, SIZE, CUDA, NOMEM (per-matrix PATTERN/OVERFLOW go to out[i]). */
perm_status_t perm_batch(const perm_matrix_t *mats, int32_t count, const perm_opts_t *opts,
                         void *stream, perm_result_t *out);

/* One permanent without allocating anything, for callers that may not
   allocate device memory (a framework that owns the memory pool, a process
   that reserved all HBM up front, code that must not call cudaMalloc or
   cudaFree).  The paper has no counterpart: it is a packaging of the
   precompiled walk.  Its scratch memory is a file-scope device array of
   1 MiB that every GPU loading the library holds until exit; host
   temporaries live on the stack.  n <= 48 (PERM_ERR_SIZE beyond), generic
   kernels only (engine CODEGEN gives PERM_ERR_ARG).  The first call on a
   device looks up the array's device address with that device current, so
   make it before any stream capture.  All calls share the array: two calls
   whose GPU work overlaps race.  Results match perm_plan_create +
   perm_compute; ms_kernel is not measured (0).  The call synchronises
   `stream`. */
perm_status_t perm_compute_noalloc(const perm_matrix_t *A, const perm_opts_t *opts, void *stream,
                                   perm_result_t *out);

/* Same as perm_batch, but each matrix gets its own plan and its own launches
   (the plain one-launch-per-matrix form, for comparison). */
perm_status_t perm_batch_sequential(const perm_matrix_t *mats, int32_t count, const perm_opts_t *opts,
                                    void *stream, perm_result_t *out);

/* Resumable run (the sub-range form of Sec. II-A): walks A in aligned Gray
   slices of 2^slice_log2 indices and appends each finished slice's partial
   sum to the text file `path` (created if absent).  Slices already recorded
   are skipped, so a stopped run resumes where it left off.  At most
   max_slices new slices are computed per call (0 = all).  Returns OK with the
   permanent in *out once every slice is recorded (combined in slice order:
   the same bits however the run was split), or NOT_READY with out->steps =
   Gray indices recorded so far.  The file names the matrix (hash of values
   and order), the arithmetic and the slice size; a file written for another
   run gives ARG.  slice_log2 in [5, n-1]. */
perm_status_t perm_checkpoint_run(const perm_matrix_t *A, const perm_opts_t *opts, const char *path,
                                  int32_t slice_log2, int32_t max_slices, void *stream, perm_result_t *out);

/* ---------------------------------------------------------------- serving */

typedef struct perm_server_s *perm_server_t;

typedef struct {
    int32_t max_inflight;     /* device slots (matrices resident at once); 0 = 4096          */
    int32_t max_n;            /* largest n accepted; 0 = 40                                  */
    double step_budget;       /* admission: Gray steps in flight at most; 0 = auto          */
    int32_t device;           /* CUDA device ordinal                                        */
    int32_t timeout_ms;       /* a request unfinished after this long fails with TIMEOUT;  */
                              /*   0 = none                                                 */
    int32_t precision;        /* PERM_PREC_* for FP64 requests (AUTO: an ill-conditioned    */
                              /*   request is requeued once as a double-double request)    */
} perm_server_opts_t;

/* Starts a serving loop: a host thread that admits submitted matrices into
   device slots while earlier ones are still running, launches them in waves
   on its own stream, and publishes results for perm_poll. */
perm_status_t perm_server_create(const perm_server_opts_t *opts, perm_server_t *out);

/* Queues one matrix (copied).  Returns BUSY when the admission budget is full
   (the caller retries), SIZE for n > max_n.  *ticket identifies the request. */
perm_status_t perm_submit(perm_server_t s, const perm_matrix_t *A, uint64_t *ticket);

/* Waits up to timeout_ms (0 = just check, <0 = forever) for a ticket.  Returns
   OK with *out filled (out->status is the request's own status), NOT_READY,
   or ARG for an unknown ticket.  A ticket can be collected once. */
perm_status_t perm_poll(perm_server_t s, uint64_t ticket, int32_t timeout_ms, perm_result_t *out);

/* Server-side latency statistics in milliseconds (submit -> result ready). */
typedef struct {
    uint64_t completed, rejected, failed;
    double p50_ms, p99_ms, max_ms;
    double perms_per_s;
} perm_server_stats_t;

perm_status_t perm_server_stats(perm_server_t s, perm_server_stats_t *out);

/* Stops the loop, cancels unfinished tickets, frees everything (NULL is allowed). */
void perm_server_destroy(perm_server_t s);

/* ------------------------------------------------------------ inspection */
/* Host-only calls (no GPU needed): they expose the preprocessing so that it
   can be checked against the paper. */

typedef struct {
    int32_t n;
    int32_t structurally_zero;   /* 1 if there is no perfect matching                */
    int32_t ordering;            /* PERM_ORDER_* actually used                        */
    int32_t col_order[64];       /* col_order[p] = original column at position p     */
    int32_t row_order[64];       /* row_order[r] = original row at register slot r   */
    int32_t group_of_row[64];    /* by slot: first ordered column touching the row   */
    int32_t group_size[64];      /* |R_j|: rows whose first touching column is j     */
    int32_t col_nnz[64];         /* nonzeros of ordered column j                     */
    int32_t reg_rows, reg_cols;  /* k and c of Algorithm 4                           */
    int32_t exact_words;         /* w for the exact path (0 for FP64 inputs)         */
    double bound_log2;           /* log2 of the a-priori |perm| bound                */
    double ops_per_step;         /* cost model: arithmetic ops per step, this scheme */
    double ops_per_step_paper;   /* the same walk with a full product per step       */
    int32_t exact_limbs;         /* 32-bit limbs of the whole walk's ring: 2w-1 or 2w */
    int32_t reserved0;
    double ops_per_step_walk;    /* cost model of the scheme the walk runs (FP64:     */
                                 /*   two-state or paired chain; exact: one chain)    */
    double ring_ops_per_step;    /* exact inputs: integer multiply operations per step */
                                 /*   of the generated walk (its rows folded in 32 bits */
                                 /*   as the generator folds them), in the ring of     */
                                 /*   exact_limbs limbs; 0 for FP64 inputs             */
    /* A design study, not a scheme the kernels run: the FP64 operations per
       step of four-state chains (column 1 kept out of x like column 0, so
       every 4-step Gray quad flips only columns >= 2; a group of r rows costs
       r + 3 into the four chains, a row of column 0 or 1 five operations, a
       row of both seven; Lemma 2 weights as in the other models), on the
       plan's column order and on an order searched for it by pairwise swaps.
       0 for n < 3. */
    double ops_per_step_four_state;
    double ops_per_step_four_state_searched;
} perm_inspect_t;

perm_status_t perm_inspect(const perm_matrix_t *A, const perm_opts_t *opts, perm_inspect_t *out);

/* Signed changed-bit sequence SCBS(k) of a k-bit Gray code (Sec. IV): the
   2^k - 1 entries written to out as +(j+1) for inclusion of column j and
   -(j+1) for exclusion, computed by Theorem 1 (j = ctz(i); sign + iff
   floor(i / 2^(j+1)) is even).  k in [1, 24]. */
perm_status_t perm_scbs(int32_t k, int32_t *out);

/* GenerateLaunchParameters, Algorithm 2: for tau threads and dimension n,
   writes up to max_launches triples (start, delta, end) and their count. */
perm_status_t perm_alg2_launches(int64_t tau, int32_t n, int64_t *start, int64_t *delta, int64_t *end,
                                 int32_t max_launches, int32_t *count);

/* The CUDA C++ source that the codegen engine would compile for A (for
   inspection).  Writes at most cap bytes including the terminating NUL and
   sets *len to the full length.  A kernel whose register spills exceed 512
   bytes per thread is rebuilt from the same text with a 255-register budget
   (__launch_bounds__(256, 1) in place of (256, 2)). */
perm_status_t perm_codegen_source(const perm_matrix_t *A, const perm_opts_t *opts, char *buf, int64_t cap,
                                  int64_t *len);

/* The matrix image that the precompiled generic kernels read for A (for
   inspection).  Sec. III names the sparse A and x as the two data
   structures the walk touches; this is A as those kernels keep it in
   shared memory, with x's start values: column masks over row slots, group
   and S_m boundaries, the Nijenhuis-Wilf start values of Algorithm 1 by
   slot, then the values of the ordered columns 0..n-2.  Copies at most cap bytes to buf and sets
   *len to the image size, *nmax to its NMAX bucket (16, 32 or 48), *kind to
   its kernel family (0 FP64, 1 double-double, else 2 limbs + fold) and
   *abs_shift to the scale of its sum of |terms|.  Needs no GPU.  Errors:
   those of perm_plan_create's validation; SIZE for n > 48. */
perm_status_t perm_generic_image(const perm_matrix_t *A, const perm_opts_t *opts, void *buf, int64_t cap,
                                 int64_t *len, int32_t *nmax, int32_t *kind, int32_t *abs_shift);

/* Measures this GPU's FP64 (DFMA) and 32-bit IMAD issue rates in lane
   operations per second with two short probe kernels on `stream` (8
   independent chains per thread, 8 blocks of 256 threads per SM).  These are
   the ALU roofline denominators of the FP64 and exact walks. */
perm_status_t perm_issue_rates(void *stream, double *fp64_ops_per_s, double *imad_ops_per_s);

/* --------------------------------------------------- failure injection */
/* For tests of the failure paths, without any GPU fault: the next `count`
   calls the library makes at `site` are treated as failed (the call is not
   made; the library takes its error path exactly as for a real failure).
   count = 0 clears the site.  Sites: */
enum {
    PERM_SITE_WAVE_LAUNCH = 1,  /* serving: launch of a wave of the generic walk -> its      */
                                /*   requests fail with PERM_ERR_CUDA                        */
    PERM_SITE_NVRTC = 2,        /* codegen: NVRTC compile -> PERM_ERR_NVRTC                  */
    PERM_SITE_FINISH = 3,       /* serving: a final reduction -> its requests fail           */
    PERM_SITE_UPLOAD = 4,       /* serving: a request's matrix image upload -> it fails      */
    PERM_SITE_LAUNCH = 5        /* perm_compute: the walk launch -> PERM_ERR_CUDA            */
};
perm_status_t perm_debug_inject_failures(int32_t site, int32_t count);

/* ------------------------------------------------------------- misc */

const char *perm_status_string(perm_status_t s);
const char *perm_last_error(void);
/* 1 when a CUDA device is usable from this library, else 0 (never fails). */
int32_t perm_device_available(void);
/* Library version, "major.minor.patch" ("1.1.0": perm_inspect_t gained the
   four-state study fields and perm_generic_image was added). */
const char *perm_version(void);
/* sizeof of the ABI structs, so bindings can check their layout:
   0 perm_matrix_t, 1 perm_opts_t, 2 perm_result_t, 3 perm_inspect_t,
   4 perm_server_opts_t, 5 perm_server_stats_t; -1 for anything else. */
int64_t perm_sizeof(int32_t which);

#ifdef __cplusplus
}
#endif

#endif /* PERM_H */
