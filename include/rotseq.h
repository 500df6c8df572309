/*
 * rotseq.h -- C ABI of the GB300 (sm_103a) library that applies a sequence of
 * planar (Givens) rotations to the columns of a dense matrix.
 *
 * Method: Steel & Langou, "Communication efficient application of sequences
 * of planar rotations to a matrix".
 *
 * Problem (Algorithm 2, rot_sequence): A is m x n, C and S are (n-1) x k.
 * For p = 0..k-1 and j = 0..n-2, in that order, rotation (j,p) replaces
 * columns j and j+1 of A by (Algorithm 1, rot)
 *     A(:,j)   <-  c*A(:,j) + s*A(:,j+1)
 *     A(:,j+1) <- -s*A(:,j) + c*A(:,j+1)        with c = C(j,p), s = S(j,p),
 * i.e. A <- A * G(0,0) G(1,0) ... G(n-2,k-1) applied from the right.
 *
 * Layout: every matrix is column-major with a leading dimension:
 *     A(i,j) = A[i + j*lda],  C(j,p) = C[j + p*ldc],  S(j,p) = S[j + p*lds].
 * Pointers named A, C, S are DEVICE pointers unless the name says host.
 *
 * Ownership: the caller owns A, C and S.  A is updated in place.  C and S
 * must stay unmodified until the work queued on `stream` has finished.  The
 * library owns only its scratch memory, which it takes from the CUDA
 * stream-ordered allocator of the current device and returns on the same
 * stream.
 *
 * Execution: every rot_apply* call is asynchronous on `stream` (a
 * cudaStream_t passed as void*, NULL = legacy default stream) and uses the
 * current CUDA device.  A call returns once the work is queued.  Device-side
 * failures (a bounded wait that ran out) are recorded in a sticky status that
 * rot_device_status() returns.
 *
 * Errors: no entry point aborts or exits.  Quick return (ROT_OK, nothing
 * queued) when m == 0, n <= 1 or k == 0.
 *   ROT_EINVAL   a size < 0, lda < max(1,m), ldc or lds < max(1,n-1), a NULL
 *                pointer with work to do, or a size beyond the limits below.
 *   ROT_ENOMEM   scratch memory could not be obtained.
 *   ROT_ECUDA    a CUDA call or launch failed.
 * Limits: m, n, k and n+k must each be below 2^31.
 *
 * FMA placement: the FP64 and FP32 paths compute every rotation as
 *     x' = fma(c, x, RN(s*y)),   y' = fma(c, y, -RN(s*x)),
 * which makes the FP64 result bit-identical to a plain loop over Algorithm 2
 * with the same placement.
 */
#ifndef ROTSEQ_H
#define ROTSEQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ROT_OK = 0,
  ROT_EINVAL = 1,
  ROT_ECUDA = 2,
  ROT_ENOMEM = 3,
  ROT_ETIMEOUT = 4,
  ROT_EBUSY = 5,
  ROT_EUNSUPPORTED = 6
} rot_status;

/* Library version: major*10000 + minor*100 + patch. */
int rot_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char* rot_status_string(rot_status s);

/* Description of the last failure recorded on the calling host thread (for
 * ROT_ECUDA: the CUDA call and its error), or "" (never NULL). */
const char* rot_last_error(void);

/*
 * Algorithm 2 in FP64, computed in the wave order of Algorithm 3
 * (Section 1.1) by the row-parallel wavefront kernel.  Bit-identical to the
 * plain loop of Algorithm 2 with the FMA placement above.
 *   m, n, k   sizes (A is m x n; C, S are (n-1) x k)
 *   A, lda    device FP64, column-major, updated in place
 *   C, ldc    device FP64 cosines, column-major
 *   S, lds    device FP64 sines, column-major
 *   stream    cudaStream_t (as void*) the work is queued on
 */
rot_status rot_apply(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                     int64_t ldc, const double* S, int64_t lds, void* stream);

/*
 * Algorithm 2 in FP32 (FP32 data, FP32 rotations, FP32 fused multiply-add),
 * same kernel design and argument meaning as rot_apply.  Bit-identical to a
 * plain FP32 loop of Algorithm 2 with the FMA placement above; against the
 * FP64 result the per-row relative error stays below 8*k*2^-24.
 */
rot_status rot_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C,
                         int64_t ldc, const float* S, int64_t lds, void* stream);

/*
 * The rotations applied from the left, to rows: for p = 0..k-1 and
 * j = 0..m-2, rows j and j+1 of A (m x n, column-major) are replaced by
 *     A(j,:)   <-  c*A(j,:) + s*A(j+1,:)
 *     A(j+1,:) <- -s*A(j,:) + c*A(j+1,:)      with c = C(j,p), s = S(j,p),
 * i.e. Algorithm 2 on A^T (A <- (A^T G(0,0) ... G(m-2,k-1))^T).  C and S are
 * (m-1) x k with leading dimensions ldc, lds >= max(1, m-1).  Bit-identical
 * to a plain loop over rows with the same FMA placement.  Implemented as a
 * transpose into scratch, the column kernel and a transpose back; the scratch
 * (m*n doubles) comes from the stream-ordered allocator.  Quick return when
 * n == 0, m <= 1 or k == 0.
 */
rot_status rot_apply_left(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                          int64_t ldc, const double* S, int64_t lds, void* stream);

/*
 * 2x2 reflectors in place of rotations (Section 6): for p = 0..k-1 and
 * j = 0..n-2 in Algorithm 2's order, columns j and j+1 of A are multiplied
 * by the reflector H = I - tau*v*v^T with v = (1, nu), tau = T(j,p),
 * nu = V(j,p):
 *     x' = x - tau*(x + nu*y),   y' = y - nu*tau*(x + nu*y),
 * computed as t = fma(nu, y, x), w = RN(tau*t), x' = RN(x - w),
 * y' = fma(-nu, w, y) (bit-identical to a plain loop with that placement).
 * Same kernel, arguments and error behaviour as rot_apply with (T, V) in
 * place of (C, S); H is orthogonal when tau = 2/(1 + nu^2).
 */
rot_status rot_apply_reflectors(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* T,
                               int64_t ldt, const double* V, int64_t ldv, void* stream);

/*
 * Same computation as rot_apply on HOST buffers: copies A, C and S to the
 * current device, runs rot_apply on `stream`, copies A back into A_host and
 * synchronizes `stream` before returning.  Device memory comes from the
 * stream-ordered allocator and is released before return.  Pinned host
 * memory gives the fastest copies; pageable memory also works.
 */
rot_status rot_apply_host(int64_t m, int64_t n, int64_t k, double* A_host, int64_t lda,
                          const double* C_host, int64_t ldc, const double* S_host, int64_t lds,
                          void* stream);

/*
 * rot_apply without any allocation: the same FP64 computation, arguments,
 * result (bit-identical) and error codes as rot_apply, but its scratch memory
 * is a fixed 32 MiB static device array inside this library instead of
 * memory from the CUDA allocator.  The paper has no counterpart; this exists
 * for callers that cannot let a library allocate device memory -- programs
 * that reserve the GPU's memory for their own pool up front (or plugins
 * running inside one), where cudaMalloc would fail or fragment that pool and
 * its implicit device synchronization would stall their loop.
 *   Limit: the scratch needed is about 16*(n+k-2)*max(k rounded up to 4, 16)
 *   bytes for the repacked (c,s) rows plus 4*ceil(m/32)*ceil(k/16) bytes of
 *   counters (each part rounded up to 256 bytes, plus 256); a problem that
 *   needs more than 32 MiB is rejected with ROT_EINVAL and nothing is queued.
 *   (A 8192 x 8192, k = 192 problem needs 24.6 MiB.)
 *   The array exists on a device once the library's device code is loaded
 *   there.  Under the CUDA runtime's lazy module loading (the default) that
 *   happens at the first set-up on the device: rot_apply_noalloc_prepare()
 *   or the first rot_apply_noalloc.  That set-up is the one moment the 32 MiB
 *   come out of the device's free memory, so a caller that reserves the rest
 *   of the GPU for its own pool makes it before reserving the pool, and
 *   before any stream capture.  The array then stays until the process exits.
 *   The set-up (cudaGetSymbolAddress for the array's device address, and the
 *   kernel's shared-memory attribute) is done once per device and CUDA
 *   context; after a device reset the next call repeats it.
 *   All calls share the one array; the counters are cleared at the start of
 *   each call, the rest is overwritten.  Calls whose work overlaps on the GPU
 *   (different streams, or host threads racing on one device) race on it and
 *   give wrong results: order them on one stream or synchronize in between.
 *   Speed: this entry point always runs the wavefront kernel, with the
 *   p-block length rot_apply's wavefront kernel takes.  rot_apply picks
 *   faster kernels for few sequences (k <= 32), whose scratch is sized
 *   differently; at 8192 x 8192 with k = 8 this call takes about twice as
 *   long as rot_apply.  For k > 32 the two run the same kernel with the same
 *   tiling (unless the autotuner recorded one for rot_apply's shape).
 *   rot_last_error() names the failing CUDA call on ROT_ECUDA.
 */
rot_status rot_apply_noalloc(int64_t m, int64_t n, int64_t k, double* A, int64_t lda,
                             const double* C, int64_t ldc, const double* S, int64_t lds,
                             void* stream);

/* The set-up of rot_apply_noalloc on the current device, without queuing any
 * work: loads the library's device code there if needed (which creates the
 * 32 MiB array), looks up the array's address and sets the kernel's
 * shared-memory attribute.  Call it before reserving device memory for a pool
 * and before stream capture; repeated calls are cheap.  ROT_ECUDA if a CUDA
 * call fails (rot_last_error() names it).  The paper has no counterpart. */
rot_status rot_apply_noalloc_prepare(void);

/* ---- the packed resident layout (Section 4's pre-packed A, rs_kernel_v2) -- */

/*
 * Packed layout of an m x n matrix: ceil(m/32) strips of 32 rows, strip s a
 * 32 x n column-major panel (leading dimension 32) holding rows 32s..32s+31,
 * the strips one after the other:
 *     P[(i/32)*32*n + j*32 + i%32] = A(i,j),
 * rows past m in the last strip are zero.  A warp of the rotation kernels
 * owns 32 rows and walks the columns, so in this layout it reads and writes
 * one contiguous run of memory.  A matrix that stays on the device across
 * many applications is packed once.
 * rot_packed_elems: elements of the packed buffer, ceil(m/32)*32*n (-1 for
 * negative or too large sizes).
 */
int64_t rot_packed_elems(int64_t m, int64_t n);

/* Column-major A (lda >= max(1,m)) into packed P, and back (rot_unpack writes
 * rows < m only).  Device pointers, asynchronous on `stream`; P holds
 * rot_packed_elems(m, n) elements.  ROT_EINVAL for bad sizes or NULL
 * pointers with work to do. */
rot_status rot_pack(int64_t m, int64_t n, const double* A, int64_t lda, double* P, void* stream);
rot_status rot_unpack(int64_t m, int64_t n, const double* P, double* A, int64_t lda, void* stream);
rot_status rot_pack_f32(int64_t m, int64_t n, const float* A, int64_t lda, float* P, void* stream);
rot_status rot_unpack_f32(int64_t m, int64_t n, const float* P, float* A, int64_t lda, void* stream);

/*
 * rot_apply / rot_apply_f32 on a packed matrix P (m x n): the same result bit
 * for bit (rows are independent and each row sees the same operations).
 * Few sequences (k <= 16 in FP64, k <= 48 in FP32, with m, n >= 64 and P
 * 16-byte aligned) run the column stream over the strips; otherwise the
 * wavefront kernel.  What rot_apply uses on a column-major matrix beyond
 * that (the FP64 column stream split over warps, the lane pipelines for
 * 3 <= k <= 32 in FP64 and k > 55 in FP32, and the FP32 warp chain for
 * 16 <= k <= 55) is not used here, so those k run slower than on a
 * column-major matrix.  Same error codes as rot_apply.
 */
rot_status rot_apply_packed(int64_t m, int64_t n, int64_t k, double* P, const double* C, int64_t ldc,
                            const double* S, int64_t lds, void* stream);
rot_status rot_apply_packed_f32(int64_t m, int64_t n, int64_t k, float* P, const float* C, int64_t ldc,
                                const float* S, int64_t lds, void* stream);

/* ---- accumulated blocks applied by matrix products (rs_gemm, Section 8) -- */

typedef enum {
  ROT_GEMM_F64_DMMA = 0,    /* FP64 tensor MMA, FP64 accumulation */
  ROT_GEMM_SPLIT_BF16 = 1,  /* A, Q split into BF16 hi+lo; hi*hi+hi*lo+lo*hi, FP32 accumulation */
  ROT_GEMM_SPLIT_F16 = 2,   /* FP16 hi + 2^-11*lo; hi*hi and hi*lo+lo*hi in two FP32 accumulators */
  ROT_GEMM_SPLIT_BF16_Q32 = 3,  /* ROT_GEMM_SPLIT_BF16 with the blocks formed in FP32 (rot_form_blocks_f32) */
  ROT_GEMM_SPLIT_F16_Q32 = 4    /* ROT_GEMM_SPLIT_F16 with the blocks formed in FP32 */
} rot_gemm_mode;

/* Number of accumulated blocks for (n, k, nb, kb): for each group of kb
 * sequences (p-block), ceil(((n-2) + kb') / nb) blocks of nb waves, where
 * kb' = min(kb, k - p0).  0 when n < 2 or k < 1. */
int64_t rot_form_blocks_count(int64_t n, int64_t k, int nb, int kb);

/*
 * Form every accumulated block in FP64 (the paper's rs_gemm accumulates
 * blocks of rotations into orthogonal matrices).  Block b covers sequences
 * [p0, p0+kb) and waves w = j + (p - p0) in [w0, w0+nb) of that p-block; it
 * touches the L = nb + kb columns starting at c0 = w0 - kb + 1.  Q receives
 * rot_form_blocks_count() matrices of L x L, column-major, one after the
 * other (Q + b*L*L): block b's rotations applied, in Algorithm 2 order, to
 * the identity (columns outside [0, n) stay identity), so that
 * A(:, c0:c0+L) * Q_b equals applying the block to A.  Blocks are ordered
 * by p-block, then by w0.  Entries equal the same computation on the CPU with
 * this library's FMA placement; only the sign of zero entries may differ
 * (rotations on two zeros are skipped).  Requirements: nb, kb multiples of
 * 16, nb + kb <= 512; C, S, Q device memory.  Asynchronous on `stream`.
 */
rot_status rot_form_blocks(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S,
                           int64_t lds, int nb, int kb, double* Q, void* stream);

/*
 * rot_form_blocks in single precision: each (c,s) rounded to the nearest
 * FP32 value and the block's rotations applied to the FP32 identity with the
 * same FMA placement in FP32 (x' = fmaf(c,x,RN(s*y)), y' = fmaf(c,y,-RN(s*x))).
 * Entries equal that sequential FP32 computation exactly; only the sign of
 * zero entries may differ.  Q receives rot_form_blocks_count() matrices of
 * L x L floats (L = nb + kb), column-major, one after the other.  The
 * rotations are run as a pipeline over a warp's lanes, each lane holding up
 * to 4 sequences, so kb <= 128; otherwise the requirements of
 * rot_form_blocks, and Q 16-byte aligned.  Scratch (a per-block (c,s)
 * table) comes from the stream-ordered allocator.  ROT_EINVAL on bad
 * arguments.  Asynchronous on `stream`.
 */
rot_status rot_form_blocks_f32(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S,
                               int64_t lds, int nb, int kb, float* Q, void* stream);

/*
 * Algorithm 2's result computed the rs_gemm way: form the blocks
 * (rot_form_blocks, FP64), then update A block by block in the blocks' order,
 * A(:, c0:c0+L) <- A(:, c0:c0+L) * Q_b, with tensor-core matrix products of
 * the given mode.  The split modes run on tcgen05 (64-row tiles, FP32
 * accumulators in tensor memory) when nb + kb <= 320 (the FP16 split also
 * needs nb >= Lp/2, Lp = nb + kb rounded up to 32), otherwise on mma.sync
 * (32-row tiles); DMMA runs on mma.sync (m8n8k4 FP64).  A stays FP64 in
 * memory.  Accuracy against the FP64 result, per row, with P = ceil(k/kb)
 * p-blocks (bounds the tests hold the modes to; measured errors are 2x to 4x
 * below them): DMMA 32*sqrt(P)*2^-53; the split modes lose precision in the
 * products: FP16 split P*2^-20, BF16 split 1.5*P*2^-17.  The *_Q32 modes
 * form the blocks with rot_form_blocks_f32 instead (kb <= 128), which adds
 * FP32 rounding to the blocks (per-row error within the same bounds).  Same arguments as rot_apply plus nb, kb
 * (multiples of 16, nb + kb <= 512) and the mode.  Scratch (the blocks and their split copies)
 * comes from the stream-ordered allocator.
 */
rot_status rot_apply_gemm(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                          int64_t ldc, const double* S, int64_t lds, int nb, int kb, rot_gemm_mode mode,
                          void* stream);

/* Device bytes rot_apply_gemm_ws needs for these sizes (0 for a quick
 * return).  Host-only; ROT_EINVAL for the arguments rot_apply_gemm rejects. */
rot_status rot_apply_gemm_workspace_size(int64_t m, int64_t n, int64_t k, int nb, int kb, rot_gemm_mode mode,
                                         size_t* bytes);

/* rot_apply_gemm with caller-owned scratch: `workspace` is device memory of
 * at least rot_apply_gemm_workspace_size() bytes, 256-byte aligned, used by
 * the queued work until it completes on `stream`.  No allocation; the result
 * equals rot_apply_gemm's bit for bit.  ROT_EINVAL if the workspace is
 * missing, too small or misaligned. */
rot_status rot_apply_gemm_ws(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                             int64_t ldc, const double* S, int64_t lds, int nb, int kb, rot_gemm_mode mode,
                             void* workspace, size_t workspace_bytes, void* stream);

/* ---- batches of independent problems ------------------------------------ */

/* Tiling of the wavefront kernel; 0 in a field means "default" (or the
 * autotuner's cached choice when a batch plan is created without tuning). */
typedef struct {
  int K;             /* sequences fused per work item, 1..16 (default 16) */
  int NB;            /* waves per work item, rounded up to a multiple of 16 (default 32) */
  int ctas_per_sm;   /* resident CTAs of 8 warps per SM (default: occupancy limit) */
  int fp64_products; /* where the FP64 rotation's two products run: 0 default
                        (= 1), 1 FP64 pipe (as fma(s, x, -0), bit-identical to
                        DMUL and issued faster), 2 integer pipe (bit-identical
                        emulation, DMUL only for zero, subnormal, Inf/NaN or
                        out-of-range operands; slower on GB300); the FP32 path
                        ignores it */
} rot_tuning;

/* One FP64 problem of a batch: A (m x n), C and S ((n-1) x k), all device
 * pointers, column-major, same meaning as rot_apply's arguments. */
typedef struct {
  int64_t m, n, k;
  double* A;
  int64_t lda;
  const double* C;
  int64_t ldc;
  const double* S;
  int64_t lds;
} rot_problem;

typedef struct rot_batch_plan_s rot_batch_plan;

typedef struct {
  int problems;            /* problems with work (quick-return ones are dropped) */
  int64_t work_items;      /* (32-row chain, p-block, wave-block) items in the launch */
  int64_t rotation_rows;   /* sum of m*(n-1)*k */
  size_t workspace_bytes;  /* device memory the plan holds */
  rot_tuning tuning;       /* tiling in use */
} rot_batch_info;

/*
 * Plan one persistent launch over `count` independent problems (Algorithm 2
 * for each; rows of different problems never interact).  Every problem is
 * validated as rot_apply would; any invalid one fails the whole call with
 * ROT_EINVAL.  The plan allocates one device workspace on the current device
 * (descriptors, TMA descriptors, the wavefront-ordered work table, counters,
 * repacked (c,s) rows), uploads the descriptors and returns; it keeps the
 * problems' device pointers, which must stay valid while the plan is used.
 * `tuning` may be NULL: the autotuner's cached choice for this batch shape, or
 * the defaults, are used.  Limits: at most 65535 problems with work.
 */
rot_status rot_batch_plan_create(int count, const rot_problem* problems, const rot_tuning* tuning,
                                 rot_batch_plan** plan);

/* Queue the batch on `stream`: clear counters, repack C/S, one persistent
 * launch of the wavefront kernel over all problems, fold the status.  No
 * allocation and no host synchronization, so it can be captured in a CUDA
 * graph and replayed.  Executions of one plan must not overlap on the GPU. */
rot_status rot_batch_plan_execute(rot_batch_plan* plan, void* stream);

rot_status rot_batch_plan_info(const rot_batch_plan* plan, rot_batch_info* info);

/* Free the plan (synchronizes the device first: queued work may use it). */
rot_status rot_batch_plan_destroy(rot_batch_plan* plan);

/* rot_apply with an explicit tiling (NULL or zero fields: defaults); the
 * result is identical for every tiling.  ROT_EINVAL for out-of-range fields. */
rot_status rot_apply_tuned(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                           int64_t ldc, const double* S, int64_t lds, const rot_tuning* tuning, void* stream);

/* One-shot batch: create a plan, execute it on `stream`, wait, destroy. */
rot_status rot_apply_batched(int count, const rot_problem* problems, void* stream);

/* Device bytes rot_apply_batched_ws needs for this batch (0 when no problem
 * has work), with the tiling a plan would pick.  Host-only; ROT_EINVAL for an
 * invalid problem. */
rot_status rot_batched_workspace_size(int count, const rot_problem* problems, size_t* bytes);

/* One batch with caller-owned scratch: `workspace` is device memory of at
 * least rot_batched_workspace_size() bytes, 256-byte aligned.  The launch's
 * descriptors are copied from host memory before the call returns; the
 * kernels are queued on `stream` (no allocation, no wait).  The workspace must
 * stay untouched until they complete.  Same results as rot_apply_batched. */
rot_status rot_apply_batched_ws(int count, const rot_problem* problems, void* workspace, size_t workspace_bytes,
                                void* stream);

/*
 * Autotuner: times a small grid of tilings (K in {4,8,16}, NB in {32,64,128},
 * CTAs per SM in {1,2}) on scratch copies of the problems' A (so the caller's
 * data is not modified), stores the fastest in an in-process cache keyed by
 * the batch's shape signature and the device (and appends it to the file
 * named by the environment variable ROTSEQ_TUNE_CACHE, if set), and returns
 * it in *best (and its time in *best_ms, optional).  Synchronous; allocates
 * the scratch copies from the CUDA allocator.
 */
rot_status rot_batch_autotune(int count, const rot_problem* problems, void* stream,
                              rot_tuning* best, float* best_ms);
/* A batch of one problem tunes that shape for rot_apply too: when rot_apply
 * (or rot_apply_left, on the transpose) takes the wavefront kernel (k > 32,
 * or where the faster small-k kernels do not apply), it uses the tiling the
 * cache holds for its shape signature, else the defaults.  The result is the
 * same for every tiling. */

/* ---- serving: continuous batching of requests on resident matrices ------ */

typedef struct rot_server_s rot_server;

typedef struct {
  size_t hbm_budget_bytes;  /* device memory reserved up front for request
                               workspaces (C, S and the launch's working
                               buffers); at least 1 MiB */
  int max_inflight;         /* requests admitted and not yet complete */
  int streams;              /* launches that may run at the same time, 1..64 */
  int max_batch;            /* requests per launch */
  int max_fused_k;          /* most sequences of queued requests on one matrix
                               fused into one problem; 0 = no limit */
  int wide_rows;            /* matrices with at least this many rows are
                               "wide" (see rot_server_create); 0 = 2048,
                               negative = no matrix is wide */
} rot_server_config;

typedef struct {
  int64_t completed, rejected, pending, inflight, launches;
  double mean_batch;            /* requests per launch */
  double p50_ms, p99_ms, max_ms;/* submit-to-completion latency */
  int64_t rotation_rows;        /* of the completed requests */
  double busy_s;                /* first submit to last completion */
  double rotation_rows_per_s;   /* rotation_rows / busy_s */
  size_t arena_used_bytes;      /* workspace memory in use now */
} rot_server_stats_t;

/*
 * Start a server on the current device: reserves cfg->hbm_budget_bytes of
 * device memory as its workspace arena, creates cfg->streams streams and a
 * scheduler thread.  Each scheduling step admits pending requests in
 * submission order while a request slot (max_inflight) and arena memory are
 * free, puts everything admitted in that step (at most max_batch) into one
 * launch of the batched wavefront kernel, and issues it on a free stream;
 * launches on different streams overlap on the device.  A matrix is never in
 * two launches at once, so requests on one matrix apply in submission order;
 * consecutive pending requests on one matrix (up to cfg->max_fused_k
 * sequences together, or all of them when it is 0) go out as one problem whose sequences are theirs in submission order, which
 * is the same computation.  A launch's grid is sized to the work items it can
 * run at once, leaving SMs to the launches beside it, and a launch with few
 * items per key uses p-blocks of 8 or 4 sequences.  Matrices of
 * cfg->wide_rows rows or more (2048 by default) are "wide": a launch holds
 * only wide or only narrow matrices (a request completes with its launch, so
 * a small request never waits inside a long launch), at most one wide launch
 * runs at a time, and it runs one CTA per SM, which leaves the other resident
 * CTA slot of every SM to narrow launches that arrive meanwhile.  The paper has no serving
 * layer; every request computes Algorithm 2 on its matrix exactly as
 * rot_apply would (bit-identical results).
 */
rot_status rot_server_create(const rot_server_config* cfg, rot_server** server);

/* Register a resident device matrix A (m x n, lda), owned by the caller, which
 * must keep it alive and not touch it while requests on it are in flight. */
rot_status rot_server_register(rot_server* server, int64_t m, int64_t n, double* A, int64_t lda,
                               int* handle);

/*
 * Submit a request: apply the k sequences in host arrays C_host, S_host
 * ((n-1) x k, column-major, leading dimensions ldc, lds) to matrix `handle`.
 * C and S are copied before return.  Non-blocking; *ticket identifies the
 * request for rot_server_wait.  ROT_ENOMEM if the request could never fit in
 * the arena; ROT_EINVAL for bad arguments or after destroy began.
 */
rot_status rot_server_submit(rot_server* server, int handle, int64_t k, const double* C_host,
                             int64_t ldc, const double* S_host, int64_t lds, uint64_t* ticket);

/* Wait for a request (timeout_ms < 0: no limit).  Returns the request's
 * status (ROT_OK, or ROT_ETIMEOUT if its launch reported a device-side wait
 * that ran out), or ROT_ETIMEOUT if the wait itself ran out (the request is
 * still live and can be waited on again).  A ticket can be waited on until it
 * has returned its status once. */
rot_status rot_server_wait(rot_server* server, uint64_t ticket, int timeout_ms);

/* rot_server_wait that also reports the request's latency: on ROT_OK (or a
 * device-side ROT_ETIMEOUT) *latency_ms receives the time from its submission
 * to the completion of its launch (the same clock as the statistics).  It is
 * left alone when the wait itself runs out.  latency_ms may be NULL. */
rot_status rot_server_wait_latency(rot_server* server, uint64_t ticket, int timeout_ms, double* latency_ms);

/* Statistics since creation or the last reset (reset != 0 clears them). */
rot_status rot_server_stats(rot_server* server, rot_server_stats_t* stats, int reset);

/* Drain every submitted request, stop the scheduler and free the server. */
rot_status rot_server_destroy(rot_server* server);

/* ---- measurement ------------------------------------------------------- */

/* One traced kernel launch: its kind, device time and the rotation-row
 * updates (one rotation applied to one row) it performed.  For the block
 * formation kernels (ROT_KERNEL_FORM_BLOCKS) `work` counts what the kernel
 * executes: the FP64 formation skips the waves in which a chain's rows of
 * the block are still zero, and the FP32 pipeline runs every stage of every
 * step, (1,0) padding stages included. */
typedef struct {
  int kind;      /* ROT_KERNEL_* */
  float ms;      /* CUDA-event time on the launch stream, -1 if unavailable */
  int64_t work;  /* rotation-row updates done by the launch */
} rot_trace_record;

enum {
  ROT_KERNEL_WAVE_F64 = 1,
  ROT_KERNEL_WAVE_F32 = 2,
  ROT_KERNEL_WAVE_BATCHED = 3,
  ROT_KERNEL_FORM_BLOCKS = 4,
  ROT_KERNEL_GEMM_APPLY = 5,
  ROT_KERNEL_REFLECT_F64 = 6,
  ROT_KERNEL_PIPE_F32 = 7,    /* FP32 sequences pipelined across a warp's lanes */
  ROT_KERNEL_PIPE_F64 = 8     /* FP64 sequences pipelined across a warp's lanes */
};

/* Start recording a CUDA event pair around every main kernel the library
 * launches (discards earlier records). */
rot_status rot_trace_start(void);

/* Stop recording; waits for the recorded events, writes up to `capacity`
 * records to `out` and the number recorded to *count. */
rot_status rot_trace_stop(rot_trace_record* out, int capacity, int* count);

/* Number of kernels this library has launched in this process. */
int64_t rot_launch_count(void);

/* FP64 fused multiply-add throughput of the current device, measured by a
 * short microbenchmark (8 independent DFMA chains per thread, 2 CTAs of 1024
 * threads per SM): *gflops counts 2 flops per DFMA; *ms (optional) is the
 * time of one probe launch.  Synchronous. */
rot_status rot_measure_fp64_peak(double* gflops, double* ms);

/* FP64 issue rate of one instruction mix, registers only, as a ceiling for
 * the rotation kernels (the paper counts 6 flops per rotation-row; with the
 * placement above that is two rounded products and two FMAs, Section 1.1):
 *   kind 0  DFMA only      kind 1  DMUL only
 *   kind 2  the rotation's mix: per pair sy = RN(s*y), sx = RN(s*x),
 *           x' = fma(c,x,sy), y' = fma(c,y,-sx)
 *   kind 3  kind 2 with (c, s) read from shared memory per rotation
 *   kind 4  kind 3 with the products as fma(s, y, -0), fma(s, x, -0) (a
 *           freshly computed -0; bit-identical to the rounded products):
 *           the form the library's FP64 rotation kernels use
 *   kind 5  DFMA only, multiplier and addend read from shared memory
 * Every thread updates 4 independent pairs per iteration (kind 4 counts 4
 * FP64 instructions per pair and iteration, kind 5 two); the grid is
 * ctas_per_sm CTAs of warps_per_cta warps per SM (warps_per_cta 1..32,
 * ctas_per_sm 1..32, their product <= 64).  *lane_ops_per_s counts FP64
 * instructions times the lanes that executed them, per second (a rotation
 * applied to one row is 4 of them); *ms (optional) is one launch's time.
 * ROT_EINVAL for out-of-range arguments.  Synchronous. */
rot_status rot_measure_fp64_mix(int kind, int warps_per_cta, int ctas_per_sm, double* lane_ops_per_s,
                                double* ms);

/* Issue rate of the 5th-generation tensor cores for one product shape
 * (tcgen05.mma kind::f16, BF16 operands in shared memory, FP32 accumulator in
 * tensor memory, K = 16): one CTA per SM, one thread issues `mmas` products
 * from zeroed operands, cycling over `accumulators` independent accumulators
 * of n columns; *ns_per_mma is the mean time per product from the first issue
 * to the completion of the last.  m: 64 or 128; n: a multiple of 16 in
 * [16, 256]; accumulators * n <= 512; mmas in [1, 2^20]; ROT_EINVAL otherwise,
 * ROT_ETIMEOUT if a completion wait ran out (4 s).  A diagnostic for the block
 * apply's roofline (rot_apply_gemm issues M = 64, N = Lp/2 products over two
 * accumulators); synchronous. */
rot_status rot_measure_tc_issue(int m, int n, int accumulators, int mmas, double* ns_per_mma);

/*
 * Fault-detection self-test (the paper has no counterpart): runs the FP64
 * wavefront kernel on a small scratch problem whose ticket counter starts
 * past the first work item of every chain, so the items it hands out wait on
 * dependency counters that nothing advances.  Each wait gives up after
 * wait_ms (1..10000), records the timeout in the launch's status word and the
 * kernel returns normally; nothing faults, traps or hangs, and the context
 * stays usable.  Returns ROT_ETIMEOUT when the timeout was observed (the
 * expected outcome), ROT_ECUDA otherwise.  Synchronous.  Does not touch the
 * sticky status of rot_device_status.
 */
rot_status rot_selftest_wait_timeout(int wait_ms, void* stream);

/*
 * Synchronizes the current device, then returns and clears the sticky
 * device status: ROT_OK; ROT_ETIMEOUT if a kernel's bounded wait ran out
 * since the last call; ROT_ECUDA if the device reported an error (the
 * synchronization failed, or a kernel recorded an internal error such as a
 * work item decoded outside its problem).  rot_last_error() then names the
 * cause.
 */
rot_status rot_device_status(void);

/*
 * The rot_status a kernel's device status word stands for (host only, no
 * CUDA call), with rot_last_error() set to its description: 0 -> ROT_OK;
 * 1 (a dependency wait ran out) and 2 (a tile-copy wait ran out) ->
 * ROT_ETIMEOUT; 3 (a work item decoded outside the problem, an internal
 * error), 4 (cancelled) and any other code -> ROT_ECUDA.  The paper has no
 * counterpart.
 */
rot_status rot_device_code_status(int code);

#ifdef __cplusplus
}
#endif

#endif /* ROTSEQ_H */
