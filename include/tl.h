/*
 * tl.h -- C ABI of the fused metric-evolution kernels (sm_103a).
 *
 * At every point of an N-point grid the library evaluates, in one fused kernel, the chain of
 * Lewis & Pfeiffer, "Automatic generation of CUDA code performing tensor manipulations using C++
 * expression templates" (arXiv:1804.10120):
 *   1. g^ij, the inverse of the symmetric spatial metric g_ij (Sec. 1, after Eq. 6);
 *   2. the Christoffel symbols Gamma^i_jk = 1/2 g^il (d_k g_jl + d_j g_lk - d_l g_jk)   (Eq. 6);
 *   3. the covariant derivative of the shift nabla_j beta_i = d_j beta_i - Gamma^k_ij beta_k
 *      (footnote to Listing 1);
 *   4. d_t g_ij = -2 alpha K_ij + nabla_i beta_j + nabla_j beta_i   (Eq. 5);
 * its adjoint (reverse-mode derivative; the paper has none), and a batched form that runs many
 * multi-domain subgrids (Sec. 1: multi-domain methods evolve several spatial grids) in one launch.
 *
 * Data layout.  Structure of arrays: every tensor component is its own array of n elements (the
 * paper's Tensor<DataMesh>, Sec. 2.2), and a symmetric index pair is stored once (Sec. 2.2, lookup table).
 * Packed symmetric order p(i,j), i<=j:  (0,0)=0 (0,1)=1 (0,2)=2 (1,1)=3 (1,2)=4 (2,2)=5.
 *   inputs   g[p] = g_ij;  dg[3p+k] = d_k g_ij (derivative index innermost, as dg(i,j)(k) in
 *            Listing 3);  K[p] = K_ij;  alpha;  beta[i] = beta_i;  dbeta[3i+j] = d_j beta_i
 *   outputs  ginv[p] = g^ij;  gamma[6i + p(j,k)] = Gamma^i_jk;  dbcov[3i+j] = nabla_j beta_i;
 *            dtg[p] = d_t g_ij
 * Every table entry is a DEVICE pointer unless the function says otherwise.  Element type: double
 * for TL_F64 and TL_F64_FF, float for TL_F32.  Arrays need only element alignment (8 or 4 bytes).
 *
 * Ownership and ordering.  The caller owns every array.  tl_dtg_forward / tl_dtg_backward /
 * tl_dtg_batched allocate nothing, never synchronise, and only enqueue work on `stream` (NULL = the
 * legacy default stream); their results are ready when that stream reaches the enqueued work.
 * Outputs must not overlap inputs or each other (checked on the host: TL_ERR_INVALID_ARG).
 *
 * Errors.  Every function returns a status; no exception crosses the ABI.  Arguments are checked
 * before anything is enqueued, so a non-OK status means nothing was launched.  tl_last_error() returns
 * a thread-local message describing the last non-OK status of the calling thread.
 */
#ifndef TL_H
#define TL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TL_API __attribute__((visibility("default")))
#else
#define TL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t (CUDA's runtime defines cudaStream_t as struct CUstream_st *). */
typedef struct CUstream_st *tl_stream;

typedef enum {
    TL_OK = 0,
    TL_ERR_INVALID_ARG = 1,    /* NULL pointer, n < 0, overlapping outputs, bad dtype or size      */
    TL_ERR_ALIGNMENT = 2,      /* an array not aligned to its element size                         */
    TL_ERR_UNSUPPORTED = 3,    /* no sm_103a device / combination not provided                     */
    TL_ERR_CUDA = 4,           /* a CUDA runtime call or launch failed (message in tl_last_error) */
    TL_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up (batched status word)         */
    TL_ERR_PLAN_MISMATCH = 6   /* a batch plan used with another device or after destruction       */
} tl_status;

typedef enum {
    TL_F64 = 0,      /* binary64 storage; every arithmetic operation in IEEE binary64              */
    TL_F32 = 1,      /* binary32 storage and arithmetic; det(g) and the 3x3 inverse in binary64    */
    TL_F64_FF = 2    /* binary64 storage; inverse, Eq. 6 bracket and Eq. 5 in binary64; the two
                        contractions (raising Eq. 6 with g^il, and Gamma^k_ij beta_k) in float-float
                        arithmetic (pairs of binary32, >= 46 significant bits) on the FP32 pipes   */
} tl_dtype;

/* Component pointer tables (43 inputs, 39 outputs); layout as described above. */
typedef struct { const void *g[6], *dg[18], *K[6], *alpha, *beta[3], *dbeta[9]; } tl_dtg_in;
typedef struct { void *ginv[6], *gamma[18], *dbcov[9], *dtg[6]; } tl_dtg_out;
/* Upstream gradients, laid out like the outputs.  A NULL entry means that output does not enter the
 * functional (treated as an all-zero array, and never read). */
typedef struct { const void *ginv[6], *gamma[18], *dbcov[9], *dtg[6]; } tl_dtg_gout;
/* Input gradients, laid out like the inputs; all 43 required. */
typedef struct { void *g[6], *dg[18], *K[6], *alpha, *beta[3], *dbeta[9]; } tl_dtg_gin;

/*
 * Forward chain (steps 1-4 above) over n points: reads the 43 input arrays, writes the 39 output
 * arrays.  n == 0 returns TL_OK and launches nothing.  A point whose metric is singular yields
 * non-finite outputs (the definition divides by det g); no status reports it.
 */
TL_API tl_status tl_dtg_forward(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n, tl_dtype dtype,
                         tl_stream stream);

/*
 * Adjoint: with L = sum over points and outputs of gout * out, writes dL/d(input) for every stored
 * input element into gin.  A symmetric input stored once receives the sum over both index orders.
 * g^ij and Gamma are recomputed from the inputs, not read; d_j beta_i is never read (the gradient
 * does not depend on it).  TL_F64: binary64 throughout; TL_F64_FF: binary64 inverse, bracket and
 * the Eq. 5 terms, every contraction in float-float pairs; TL_F32: not provided
 * (TL_ERR_UNSUPPORTED).  Same rules as tl_dtg_forward; gin must not overlap in or gout.
 */
TL_API tl_status tl_dtg_backward(const tl_dtg_in *in, const tl_dtg_gout *gout, const tl_dtg_gin *gin, int64_t n,
                          tl_dtype dtype, tl_stream stream);

/*
 * Forward and adjoint in one pass, for a functional whose upstream gradients are known before the forward
 * runs (L = sum gout * out with gout given up front, e.g. a loss linear in the outputs): writes the 39
 * outputs exactly as tl_dtg_forward with the same dtype does (bit for bit) and the 43 input gradients
 * as tl_dtg_backward does (same definition; rounding may differ in the last bits), reading every input
 * once.  g^ij, the Eq. 6 bracket and Gamma are formed once and serve both.  TL_F64: binary64
 * throughout.  TL_F64_FF: the arithmetic of TL_F64_FF (contractions in float-float pairs, the rest in
 * binary64); a point whose inputs fall outside the pair format's range is evaluated in binary64, as the
 * float-float forward does, and one whose upstream gradients do gets its gradients from the binary64
 * adjoint (bit for bit those of tl_dtg_backward with TL_F64).  TL_F32: TL_ERR_UNSUPPORTED.
 * Same rules as tl_dtg_forward and tl_dtg_backward; out and gin must not overlap each other, in or gout.
 */
TL_API tl_status tl_dtg_forward_backward(const tl_dtg_in *in, const tl_dtg_out *out, const tl_dtg_gout *gout,
                                         const tl_dtg_gin *gin, int64_t n, tl_dtype dtype, tl_stream stream);

/*
 * Forward with HOST arrays (end-to-end form): copies the 43 input arrays host->device into `workspace`,
 * runs the forward kernel there and copies the 39 outputs device->host.  The work is cut into chunks of
 * 2^19 points that flow through three library-owned streams (host->device copies, kernel,
 * device->host copies) over three workspace slots, so both copy directions and the kernel overlap; the
 * streams fork from and join back into `stream`, so the host outputs are valid once `stream` reaches
 * the join.  When a table's arrays are equally spaced (one [43, n] or [39, n] host array) each chunk
 * moves with a single 2-D copy.  `in` and `out` hold HOST pointers (page-locked memory gives full
 * copy bandwidth; pageable memory works, but the copies then synchronise with the host).
 * `workspace` is a DEVICE buffer of at least tl_dtg_host_workspace_bytes(n, dtype) bytes
 * (at most 3 x 82 x 2^19 elements) owned by the caller.  The first call on a device creates the three
 * streams and their events, which live until exit; concurrent calls on one device are serialised on
 * the host while they enqueue.
 */
TL_API size_t tl_dtg_host_workspace_bytes(int64_t n, tl_dtype dtype);
TL_API tl_status tl_dtg_forward_host(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n, tl_dtype dtype,
                              void *workspace, size_t workspace_bytes, tl_stream stream);

/*
 * Batched forward over many grids (multi-domain subgrids of uneven size) in ONE persistent launch.
 *
 * tl_dtg_batched_prepare runs on the host, is not capturable, and may synchronise: it validates the G
 * grids' tables (in[d], out[d], n[d] for d < G; grids may have n[d] == 0; no written array may overlap
 * any other array of any grid), allocates and fills the plan's device-side data -- the G x 82 pointer
 * tables (uploaded once, cf. the paper's cached GPUPointers, Sec. 4), the tile prefix sums and a status
 * word -- and takes the launch configuration from the tuning cache when it holds an entry for this GPU,
 * dtype and batch shape (otherwise 256 threads and full occupancy).  The plan belongs to the device
 * current at prepare time; `in`, `out` and `n` are host arrays that the plan does not keep.
 *
 * tl_dtg_batched enqueues the single launch on `stream`; it allocates nothing, does not synchronise, and
 * may be captured in a CUDA graph.  A plan may be launched any number of times; the arrays it points to
 * must stay alive.  Calling it with another device current returns TL_ERR_PLAN_MISMATCH.
 *
 * tl_dtg_batched_tune times the candidate configurations (threads per block 128/256/512 x resident blocks
 * per SM x points per thread 1/2/4 x staging depth 0/2/3; a tile of a grid is threads x points-per-thread
 * points) by launching the plan on `stream` (so it writes the outputs), keeps the fastest in the plan and
 * records it in the tuning cache: the file named by TL_TUNE_CACHE, else $HOME/.cache/tl_dtg_tune.txt
 * (TL_TUNE_CACHE=off disables the cache).  It synchronises `stream`.  tl_batch_plan_config /
 * tl_batch_plan_set_config read and set threads and blocks per SM (TL_ERR_INVALID_ARG beyond the kernel's
 * occupancy); tl_batch_plan_points_per_thread / tl_batch_plan_set_points_per_thread the points per thread
 * (1, 2 or 4).  tl_batch_plan_staging / tl_batch_plan_set_staging read and set the staging depth: 0 loads
 * each point's inputs straight into registers; 2 or 3 brings the input rows of each tile into shared
 * memory by bulk copies that many tiles ahead of the arithmetic (TL_F64 and TL_F32 only, one point per
 * thread: setting a depth sets points per thread to 1 and caps blocks per SM at what the shared memory
 * allows; provided for binary64 128 x {2, 3} and 256 x 2 threads x depth, binary32 128 x {2, 3},
 * 256 x {2, 3} and 512 x 2; other pairs TL_ERR_INVALID_ARG, TL_F64_FF TL_ERR_UNSUPPORTED).  Rows that do
 * not start on a 16-byte boundary are read directly, whatever the depth.
 *
 * tl_batch_plan_check synchronises the plan's device and returns the status word recorded by its
 * launches (TL_OK, or TL_ERR_PLAN_MISMATCH if a launch found the plan inconsistent), then clears it.
 */
typedef struct tl_batch_plan tl_batch_plan;
TL_API tl_status tl_dtg_batched_prepare(const tl_dtg_in *in, const tl_dtg_out *out, const int64_t *n, int32_t G,
                                        tl_dtype dtype, tl_batch_plan **plan);
TL_API tl_status tl_dtg_batched(const tl_batch_plan *plan, tl_stream stream);
TL_API tl_status tl_dtg_batched_tune(tl_batch_plan *plan, tl_stream stream);
TL_API tl_status tl_batch_plan_config(const tl_batch_plan *plan, int32_t *threads, int32_t *blocks_per_sm);
TL_API tl_status tl_batch_plan_set_config(tl_batch_plan *plan, int32_t threads, int32_t blocks_per_sm);
TL_API tl_status tl_batch_plan_points_per_thread(const tl_batch_plan *plan, int32_t *points_per_thread);
TL_API tl_status tl_batch_plan_set_points_per_thread(tl_batch_plan *plan, int32_t points_per_thread);
TL_API tl_status tl_batch_plan_staging(const tl_batch_plan *plan, int32_t *stages);
TL_API tl_status tl_batch_plan_set_staging(tl_batch_plan *plan, int32_t stages);
TL_API tl_status tl_batch_plan_check(const tl_batch_plan *plan);
TL_API void tl_batch_plan_destroy(tl_batch_plan *plan);

/*
 * tl_dtg_batched_noalloc -- the batched forward for callers that cannot let a library allocate device
 * memory: code whose device memory is owned by a caching allocator or a fixed budget, loops that cannot
 * afford cudaMalloc's implicit device-wide synchronisation, or plug-ins handed only their buffers.  The
 * paper has no counterpart (it is an interface choice of this library).
 *
 * Same grids, layout, dtype and validation as tl_dtg_batched_prepare + tl_dtg_batched, but no plan: the
 * kernel's scratch (pointer tables, sizes, tile prefix sums, status word) lives in one fixed device
 * array inside the library, 688,392 bytes, which every GPU that loads the library holds until exit.
 * At most 1024 grids (G > 1024 returns TL_ERR_INVALID_ARG); 256 threads per block, no tuning.
 * Nothing is allocated by the library -- no cudaMalloc / cudaFree, no allocating library routine.
 * The first call on a device performs a one-time set-up on that device (it resolves the array's
 * device address), so make that first call before any stream capture.  Each call copies the tables
 * from a static host image into the array on `stream` (these copies come from pageable memory and
 * synchronise with the host), then launches.  Because the next call reuses that host image, a call
 * made while `stream` is being captured returns TL_ERR_UNSUPPORTED and enqueues nothing.  Every call
 * shares the one array and leaves its contents behind: calls whose work overlaps on the GPU
 * (different streams, or host threads racing) corrupt each other's tables -- order them on one
 * stream.  The tables are built by the call itself from the validated arguments, so there is no
 * plan-consistency status to report (no counterpart of tl_batch_plan_check).  Error behaviour as for
 * the other entry points.
 */
TL_API tl_status tl_dtg_batched_noalloc(const tl_dtg_in *in, const tl_dtg_out *out, const int64_t *n, int32_t G,
                                        tl_dtype dtype, tl_stream stream);

/*
 * The benchmark expressions of Sec. 5.1, Eqs. 9-21 (assignments, additions, outer products,
 * contractions, and K_ij = 2 alpha g_ij + beta_i beta_j), binary64, every index spatial.  Components are
 * arrays of n doubles, row-major over the indices as written (B_i^m -> B[3i+m], E_mjkl ->
 * E[27m+9j+3k+l]); Eq. 21's g_ij and K_ij are packed symmetric.  `in` lists the operands in the order
 * they appear in the equation as printed (Eq. 19: B, C, E; Eq. 20: B, C, D, E; Eq. 21: alpha, g,
 * beta), `out` the left-hand side; tl_expr_arity gives both counts.
 *   TL_EXPR_FUSED   one kernel for the whole expression (the paper's "Tensors")
 *   TL_EXPR_ARRAYS  explicit loops over left-hand-side components and contracted index values around
 *                   pointwise kernels, one launch each (the paper's "Arrays", Sec. 5.5)
 * Same argument rules as tl_dtg_forward (device arrays, element alignment, no aliasing of outputs).
 */
typedef enum { TL_EXPR_FUSED = 0, TL_EXPR_ARRAYS = 1 } tl_expr_mode;
TL_API tl_status tl_expr_arity(int32_t eq, int32_t *n_in, int32_t *n_out);
TL_API tl_status tl_expr_eval(int32_t eq, const double *const *in, double *const *out, int64_t n, tl_expr_mode mode,
                              tl_stream stream);

/*
 * Runtime generator (the GB300 counterpart of the paper's CodeWriter, Secs. 3-4): a program of tensor
 * index statements is parsed, checked against the paper's index rules, emitted as CUDA source for ONE
 * kernel with one thread per grid point, and compiled by NVRTC for sm_103a (libnvrtc is loaded at
 * first use).  Language, one item per ';':
 *   in NAME(d0, d1, ...) sym(a,b) ...;   out NAME(...);   temp NAME(...);   in NAME;  (scalar)
 *   index l(d) ...;  (a letter's range when it differs from its slot's dimension)
 *   NAME(idx, ...) = EXPR;   idx: letter, letter+k, letter-k, integer;  EXPR: numbers, NAME(idx...),
 *   + - * / (division by scalars only), unary -, parentheses, Sum(letter, EXPR)
 * `temp` tensors live in registers; only `out` tensors are stored.  Each stored component a left-hand
 * side reaches is evaluated once (a symmetric pair is one element).  The component tables list, for every `in` (then every
 * `out`) tensor in declaration order, its stored index tuples (symmetric pairs ascending) in row-major
 * order; tl_jit_info returns the counts, the generated source and one "in|out NAME i j ..." line per
 * table entry.  tl_jit_compile runs on the host without a device (TL_ERR_INVALID_ARG with the
 * parser's or NVRTC's message in `log` on failure); tl_jit_launch loads the module on the current
 * device at its first launch there (not capturable), then enqueues one launch on `stream`.
 */
typedef struct tl_jit_kernel tl_jit_kernel;
TL_API tl_status tl_jit_compile(const char *program, tl_jit_kernel **kernel, char *log, size_t log_size);
TL_API tl_status tl_jit_info(const tl_jit_kernel *kernel, int32_t *n_in, int32_t *n_out, const char **source,
                             const char **component_names);
/* reads[q] (q < n_in) = 1 when the generated kernel loads input table entry q, 0 for a component of an
 * `in` tensor that no statement references (its entry must still be a valid array: tl_jit_launch checks
 * every entry).  Lets a caller count the kernel's algorithmic traffic.  `reads` is caller-owned. */
TL_API tl_status tl_jit_reads(const tl_jit_kernel *kernel, uint8_t *reads);
TL_API tl_status tl_jit_launch(tl_jit_kernel *kernel, const double *const *in, double *const *out, int64_t n,
                               tl_stream stream);
TL_API void tl_jit_destroy(tl_jit_kernel *kernel);

/*
 * The forward chain with the spatial derivatives formed on the grid instead of read: d_k g_ij and
 * d_j beta_i by centred finite differences of order 2 or 4 on a periodic nx x ny x nz grid (x fastest:
 * point (ix, iy, iz) is element ix + nx (iy + ny iz) of every array), spacings hx, hy, hz.  The paper
 * takes the derivatives as inputs (Listing 3); here one launch reads 16 arrays -- g[6], K[6], alpha,
 * beta[3], layout as in tl_dtg_in -- and writes the 39 outputs of tl_dtg_forward, whose d_k g_ij and
 * d_j beta_i are these differences.  dtype TL_F64 or TL_F64_FF (TL_ERR_UNSUPPORTED otherwise); other
 * rules as for tl_dtg_forward.
 */
typedef struct { const void *g[6], *K[6], *alpha, *beta[3]; } tl_dtg_grid_in;
typedef struct { int64_t nx, ny, nz; double hx, hy, hz; int32_t order; } tl_grid3d;
TL_API tl_status tl_dtg_forward_fd(const tl_dtg_grid_in *in, const tl_dtg_out *out, const tl_grid3d *grid,
                                   tl_dtype dtype, tl_stream stream);

/*
 * Kernels that stage inputs through shared memory (the TL_F32 forward) wait on their own bulk copies
 * with a bounded number of polls; a wait that gives up makes its block stop early and counts here,
 * so a nonzero count means some outputs of an earlier call were not written.  *count = timeouts on
 * the current device since the library was loaded.  Synchronises with the device (host call only,
 * not capturable); TL_ERR_CUDA if the read fails.  Expected to stay 0.
 */
TL_API tl_status tl_wait_timeouts(uint32_t *count);

TL_API const char *tl_status_string(tl_status s);
TL_API const char *tl_last_error(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
TL_API int tl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TL_H */
