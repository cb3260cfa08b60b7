/*
 * bsm.h -- C ABI of libbsm: local block-sparse matrix-matrix multiply on one
 * GB300 (sm_103a), after the local multiplication of the DBCSR library
 * (Bethune, Gloess, Hutter, Lazzaro, Pabst, Reid 2017, "Porting of the DBCSR
 * library for Sparse Matrix-Matrix Multiplications to Intel Xeon Phi
 * systems", §2).
 *
 * Matrices are block-CSR (§2: "blocked compressed sparse row"): a vector of
 * block-row sizes, a vector of block-column sizes, int64 row pointers,
 * int32 column-block indices (strictly ascending inside each row), and one
 * int64 element offset per block.  Each block is a small dense matrix stored
 * row-major at its offset.  The product C = alpha*A.B + beta*C is a sum of
 * pairwise block products A_ik.B_kj (§2, C = C + A.B), and a block product is
 * skipped when the product of the two block norms does not exceed the
 * threshold (§2, on-the-fly filtering).
 *
 * Conventions shared by every entry point:
 *   - Every call returns a bsm_status; no call aborts, throws or traps.
 *     Argument errors are detected on the host before any launch.  After a
 *     non-OK status, bsm_last_error() gives a message (thread-local).
 *   - All device work is issued on the stream set by bsm_set_stream (default:
 *     the legacy default stream).  Calls that return sizes or counts
 *     synchronise that stream.
 *   - "host or device pointer" arguments are copied with cudaMemcpyDefault,
 *     so both work (pageable, pinned or device memory).
 *   - Handles are not thread-safe; distinct handles may be used from
 *     distinct threads only with distinct streams.
 *   - Device memory owned by the library is allocated stream-ordered on the
 *     library stream, from the device pool (cudaMallocAsync) or from the
 *     hooks installed with bsm_set_allocator, and freed the same way.
 */
#ifndef BSM_H
#define BSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsm_mat *bsm_t;

typedef enum {
    BSM_OK = 0,
    BSM_ERR_ARG = 1,          /* invalid argument, pattern or sizes          */
    BSM_ERR_BLOCKING = 2,     /* block sizes of the operands do not conform  */
    BSM_ERR_CAPACITY = 3,     /* a fixed capacity would be exceeded          */
    BSM_ERR_ALLOC = 4,        /* device or host allocation failed            */
    BSM_ERR_CUDA = 5,         /* a CUDA runtime call failed                  */
    BSM_ERR_TIMEOUT = 6,      /* a bounded device wait gave up               */
    BSM_ERR_UNSUPPORTED = 7   /* shape or size outside what the kernels take */
} bsm_status;

typedef enum { BSM_FP64 = 0, BSM_FP32 = 1 } bsm_dtype;

/* Arithmetic used for the block products (the filter, the norms and the
 * final alpha/beta combination are FP64 for every choice). */
typedef enum {
    BSM_P_FP64 = 0,       /* FP64 FMA (FP32 FMA for FP32 data), FP64 sum     */
    BSM_P_FP64_DMMA = 1,  /* FP64 tensor-core MMA (mma.sync m8n8k4, FP64 accumulate)
                             for output blocks of at least 8 x 8 elements, FP64 FMA
                             for smaller ones; FP64 data (FP32 data runs the FMA
                             path).  Same products and order of k as BSM_P_FP64. */
    BSM_P_TF32x3 = 2,     /* hi/lo TF32 split, 3 tensor-core products, FP32 accumulate, FP64 sum */
    BSM_P_BF16x3 = 3,     /* hi/lo BF16 split, 3 products                    */
    BSM_P_BF16x6 = 4,     /* hi/mid/lo BF16 split, 6 products                */
    BSM_P_OZAKI = 5,      /* error-free slicing after Ozaki et al. (2012): every
                             row of the left operand and every column of the
                             right one is put on its own power-of-two fixed-point
                             grid and cut into 6 BF16 slices of at most 9 bits;
                             the 21 slice products with slice levels p + q <= 5
                             run on the tensor cores, levels 0..3 summed exactly
                             in FP32 (the sum is flushed to FP64 before 64 terms
                             of k), levels 4..5 in one rounded FP32 sum.  Error
                             per term of k below 2^-44 of the product of the
                             row's and the column's largest |x|; FP64 data only
                             (BSM_ERR_UNSUPPORTED for FP32).  Non-finite inputs
                             give non-finite outputs in their rows / columns.  */
    BSM_P_TF32x3_PANEL = 6 /* TF32x3 (the split and piece products of
                             BSM_P_TF32x3) on the fifth-generation tensor cores
                             (tcgen05, accumulators in tensor memory), over dense
                             tiles of 5 x 5 output blocks: every k-step of a tile
                             is one 128 x 128 x 24 product; three k-steps are
                             summed in FP32 (at most 3 x 72 terms), and those
                             sums added into a compensated pair per element
                             (FP32 sum, BF16 compensation term).
                             Runs when the data is FP64, every block of A, B and
                             C has one size s <= 24 and the norm filter removed
                             no product; otherwise the multiply runs the
                             BSM_P_TF32x3 kernel (bsm_get_engine tells which).
                             The adjoint runs BSM_P_TF32x3.  Not with no_sync
                             (BSM_ERR_UNSUPPORTED).                             */
} bsm_prec;

typedef struct {
    int32_t prec;          /* bsm_prec                                              */
    int32_t post_filter;   /* 1: after the multiply drop C blocks with norm <= eps   */
    int32_t build_stacks;  /* 1: also bucket the products by (m,n,k) (bsm_get_stacks) */
    int32_t flush_every;   /* split paths: how the FP32 partial sums of the block
                              products are combined.  F > 0: FP64 running sum
                              refreshed every F block products; F < 0:
                              compensated FP32 pair (Kahan) refreshed every -F
                              products, converted to FP64 at the end; 0: as -1.
                              Range [-1024, 1024].  BSM_P_OZAKI ignores it (its
                              flushes follow from the exact-sum bound).            */
    int32_t no_sync;       /* 1: no host synchronisation (CUDA-graph capturable); see
                              bsm_multiply and bsm_add                               */
    int32_t reserved[3];   /* must be zero                                          */
} bsm_opts;

/* Timing phases recorded when profiling is on (milliseconds, CUDA events on
 * the library stream). */
enum {
    BSM_T_NORMS = 0, BSM_T_SYMBOLIC = 1, BSM_T_FILL = 2, BSM_T_STACKS = 3,
    BSM_T_NUMERIC = 4, BSM_T_POST = 5, BSM_T_TOTAL = 6, BSM_T_COUNT = 7
};

/* ---------------------------------------------------------------------- */
/* library state                                                            */
/* ---------------------------------------------------------------------- */

/* Message describing the last non-OK status on this thread ("" if none). */
const char *bsm_last_error(void);

/* All subsequent device work is issued on `stream` (a cudaStream_t; NULL
 * selects the legacy default stream). */
bsm_status bsm_set_stream(void *stream);

/*
 * Device-memory provider (a library service; the paper has no counterpart:
 * §2 only says that data is organised so that host-device transfers are
 * few).  By default the library allocates
 * from the device's stream-ordered pool (cudaMallocAsync / cudaFreeAsync on
 * the library stream).  A framework that owns device memory (PyTorch's
 * caching allocator, an arena) installs hooks instead:
 *   alloc(bytes, stream, ctx) returns device memory that may be used in
 *     stream order on `stream` (a cudaStream_t), or NULL on failure -- the
 *     call that needed it then returns BSM_ERR_ALLOC after releasing what it
 *     had taken;
 *   free_fn(ptr, bytes, stream, ctx) takes back a block from alloc; the
 *     library calls it after queueing the last work that touches ptr on
 *     `stream`, so the provider may reuse ptr for later work on that stream
 *     at once and for other streams only after synchronising with it (the
 *     rule of cudaFreeAsync and of stream-aware caching allocators).
 * Both hooks NULL restores the built-in pool; exactly one NULL is
 * BSM_ERR_ARG.  Process-wide; blocks keep going back to the hooks that made
 * them even after a change.  The hooks may be called from any library call
 * that allocates (never from bsm_count_products_static) and must not call
 * back into the library.
 */
typedef void *(*bsm_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*bsm_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
bsm_status bsm_set_allocator(bsm_alloc_fn alloc, bsm_free_fn free_fn, void *ctx);

/* Limit, in seconds within [0, 2], of the waits in the main loop of the
 * BSM_P_TF32x3_PANEL kernel (default 2).  A wait that runs out makes the
 * multiply return BSM_ERR_TIMEOUT after every CTA has waited (at most 2 s)
 * for its copies and tensor-core products in flight and freed its tensor
 * memory, so the context stays usable.  Exists so that tests can make a wait
 * run out on purpose (a limit of 0 gives up on the first wait that does not
 * complete at once); process-wide. */
bsm_status bsm_set_wait_limit(double seconds);

/* Most kept products one pass of bsm_multiply holds, in [1, 2^31 - 1]
 * (default 2^31 - 1, the limit of the 32-bit product indices; process-wide).
 * A multiply whose kept products exceed it runs its fill and numeric phases
 * row panel by row panel of C, each panel a run of whole C block rows with at
 * most this many products, so that the product list held at once stays
 * within the limit (the row-panel chunking of the local multiply, Section
 * 2).  The result is bit for bit that of one pass (every C block is computed
 * by the same kernel from the same products in the same order).  Such a C
 * keeps its pattern, data, counts and timings but no product list: no
 * stacks, no bsm_get_products list, no bsm_multiply_backward and no no_sync
 * replay; the tcgen05 row-panel engine does not take it (the mma.sync TF32x3
 * kernel runs instead).  A single C block row with more kept products than
 * the limit gives BSM_ERR_CAPACITY.  Exists for products beyond 2^31 and so
 * that tests can force the panels with a small limit. */
bsm_status bsm_set_product_limit(int64_t max_products);

/* Arithmetic units bsm_measure_peak can time. */
enum {
    BSM_U_FP64_FMA = 0,   /* FP64 fused multiply-add on the CUDA cores (DFMA)        */
    BSM_U_FP64_MMA = 1,   /* FP64 tensor-core mma.sync m8n8k4 (DMMA)                 */
    BSM_U_TF32_MMA = 2,   /* TF32 mma.sync m16n8k8, FP32 accumulate                  */
    BSM_U_BF16_MMA = 3,   /* BF16 mma.sync m16n8k16, FP32 accumulate                 */
    BSM_U_FP32_FMA = 4    /* FP32 fused multiply-add on the CUDA cores               */
};

/* Measured throughput of one arithmetic unit of the current GPU, the
 * denominator of the numeric kernels' roofline fractions (a library service;
 * the paper has no counterpart).  Runs a fixed-length loop of independent
 * instruction chains, 4 CTAs of 256 threads per SM, `reps` timed launches
 * (1..100) after one warm-up, CUDA events on the library stream; returns the
 * best rate in FLOP/s (a fused multiply-add counts 2, an MMA 2*M*N*K).
 * Synchronises the stream; allocates 16 bytes. */
bsm_status bsm_measure_peak(int32_t unit, int32_t reps, double *flop_per_s);

/* Number of blocks obtained from the installed hooks and not yet returned
 * (0 when every handle holding hook memory has been destroyed). */
bsm_status bsm_get_allocator_stats(int64_t *outstanding);

/* 1: record per-phase CUDA-event timings in every multiply (bsm_get_timings). */
bsm_status bsm_set_profiling(int32_t on);

/* Number of CUDA kernels the library has launched since it was loaded
 * (all handles, all streams). */
bsm_status bsm_get_launch_count(int64_t *count);

/* Numeric variant per precision and output block shape (m rows, n columns),
 * for tiny blocks (m*n <= 16, 5 x 5, and on the FP64 and Ozaki paths 6 x 6;
 * other shapes always use variant 0):
 * 0 = one warp per output block (FP64: lanes over its elements; split and
 * Ozaki paths: tensor-core MMA on packed fragments), 1 = one lane per output
 * block on CUDA cores (split paths: the same split pieces multiplied with FP32
 * FMA, exact piece products; Ozaki path: plain FP64 FMA).  -1 restores the
 * library default (1 for m*n <= 16, 0 for 5 x 5 and 6 x 6);
 * bsm_get_variant returns the variant in effect.
 * Process-wide; the autotuner (paper_1708_03604_gb300/autotune.py) sets it
 * from measurements.  Applies to multiplies issued afterwards (a no-sync
 * multiply keeps the choice of its eager call).  BSM_P_TF32x3_PANEL has no
 * variants (BSM_ERR_ARG); when it falls back to the BSM_P_TF32x3 kernel, that
 * kernel uses the BSM_P_TF32x3 table. */
bsm_status bsm_set_variant(int32_t prec, int32_t m, int32_t n, int32_t variant);
bsm_status bsm_get_variant(int32_t prec, int32_t m, int32_t n, int32_t *variant);

/*
 * Launch shape and pass shape of the numeric kernels, per precision (the
 * paper's GPU library finds kernel parameters per block shape by
 * auto-tuning, §2; paper_1708_03604_gb300/autotune.py measures these and
 * sets them).  value -1 restores the default.  Process-wide; applies to
 * multiplies and adjoints issued afterwards (a no-sync multiply keeps the
 * settings of its eager call only for sizes, not for these).
 *   BSM_TUNE_CTA_WARPS   warps per CTA of the persistent kernel: 2 or 4 for
 *                        BSM_P_TF32x3 / BF16x3 / BF16x6 / OZAKI (default 4);
 *                        4 only for the FP64 kernels
 *   BSM_TUNE_CTAS_PER_SM persistent CTAs per SM, 1..16, capped by what fits;
 *                        0 = as many as fit (default)
 *   BSM_TUNE_PASS_MT     fragment tiles along the output rows per pass over
 *                        a block's products: split paths 1..2 (16-row tiles;
 *                        default: output blocks of one tile row run in a
 *                        kernel instance compiled for 1-row passes -- fewer
 *                        registers, more warps per SM -- and the others in a
 *                        2-row instance, two launches; 1 or 2 runs every block
 *                        in that one instance), FP64_DMMA 1..3 (default 3,
 *                        8-row tiles)
 *   BSM_TUNE_PASS_NT     along the columns: split paths 1..3 (default 3,
 *                        8-column tiles), OZAKI 1..3 (default 3; 1 and 2 run
 *                        a kernel instance with a smaller staging ring and
 *                        fewer registers), FP64_DMMA 1..3 (default 3)
 *   BSM_TUNE_FP64_BUILD  BSM_P_FP64 only: FP64 FMA kernel build, 0 chosen by
 *                        the largest output block (default), 1 narrow (up to
 *                        9 elements per lane per pass), 2 wide (up to 24);
 *                        output blocks of at most 16 elements always run the
 *                        small build
 *   BSM_TUNE_SCHED_TILE  order of the output blocks inside a block-shape
 *                        class: 0 (default) by the breadth-first rank of
 *                        their block row; T in 8..4096 by 2-D tiles of T
 *                        ranked rows x T ranked columns (columns ranked the
 *                        same way through B's pattern), so that the blocks in
 *                        flight share both operands' blocks in L2.  A
 *                        permutation of independent work: results do not
 *                        depend on it.  Not for BSM_P_TF32x3_PANEL.
 *   BSM_TUNE_ENGINE      BSM_P_TF32x3 only: 0 (default) per-C-block mma.sync
 *                        kernel; 1 the tcgen05 row-panel engine of
 *                        BSM_P_TF32x3_PANEL wherever it applies (eager calls
 *                        with the compensated sum, flush_every <= 0), the
 *                        mma.sync kernel elsewhere -- for workloads where the
 *                        tuner measured the engine faster
 *   BSM_TUNE_PANEL_STEPS the tcgen05 row-panel engine (BSM_P_TF32x3_PANEL, and
 *                        BSM_P_TF32x3 with engine 1): k-steps (128 x 128 x 24
 *                        products) summed in one FP32 accumulator buffer of
 *                        tensor memory before the drain adds it into the
 *                        compensated pair, 1..8 (default 3).  Fewer drains per
 *                        k-step, at an error bound that grows with it: per
 *                        element (3 * 2^-22 + 3 * T * s * 2^-23 + 2^-22 +
 *                        steps * 2^-33) * sum_k |a_ik| |b_kj| for T k-steps per
 *                        buffer and blocks of s rows
 * Values outside these ranges are BSM_ERR_ARG.
 */
enum {
    BSM_TUNE_CTA_WARPS = 0, BSM_TUNE_CTAS_PER_SM = 1, BSM_TUNE_PASS_MT = 2, BSM_TUNE_PASS_NT = 3,
    BSM_TUNE_FP64_BUILD = 4, BSM_TUNE_SCHED_TILE = 5, BSM_TUNE_ENGINE = 6, BSM_TUNE_PANEL_STEPS = 7,
    BSM_TUNE_COUNT = 8
};
bsm_status bsm_set_tuning(int32_t prec, int32_t param, int32_t value);
bsm_status bsm_get_tuning(int32_t prec, int32_t param, int32_t *value);

/* Numeric kernels (bsm_get_launch_config). */
enum {
    BSM_K_NONE = -1, BSM_K_FP64_CORES = 0, BSM_K_FP64_MMA = 1, BSM_K_SPLIT_MMA = 2, BSM_K_OZAKI_MMA = 3,
    BSM_K_PANEL_TCGEN05 = 4
};
/* What the last numeric launch into C ran: cfg[0] kernel (BSM_K_*),
 * cfg[1] FP64 kernel build (0 small, 1 narrow, 2 wide; -1 for the others),
 * cfg[2] threads per CTA, cfg[3] CTAs, cfg[4] / cfg[5] fragment tiles per pass
 * along rows / columns (0 where the kernel has no passes; cfg[4] = 0 on the
 * split paths when one-tile-row blocks ran in their own instance, cfg[3] then
 * the CTAs of the 2-row instance). */
bsm_status bsm_get_launch_config(bsm_t C, int32_t *cfg);

/* Fills `opts` with the defaults (FP64, no post filter, stacks built). */
bsm_status bsm_opts_default(bsm_opts *opts);

/* ---------------------------------------------------------------------- */
/* matrices                                                                 */
/* ---------------------------------------------------------------------- */

/* Data modes of bsm_create. */
enum { BSM_DATA_COPY = 0, BSM_DATA_BORROW = 1 };

/*
 * Create a block-CSR matrix (§2, blocked CSR format).
 *   nbr, nbc        number of block rows / block columns (>= 0)
 *   row_bs, col_bs  block sizes, host arrays of nbr / nbc entries, each >= 1
 *                   and <= 256; copied.
 *   row_ptr         host, nbr+1 entries, row_ptr[0] == 0, non-decreasing;
 *                   nnzb = row_ptr[nbr].  Copied.
 *   col_idx         host, nnzb entries, strictly ascending inside a row, in
 *                   [0, nbc).  Copied.
 *   blk_off         host, nnzb element offsets; block b occupies
 *                   [blk_off[b], blk_off[b] + row_bs[i]*col_bs[j]) and must lie
 *                   inside [0, data_len); blocks must not overlap.  Copied.
 *   dtype           BSM_FP64 or BSM_FP32 element type.
 *   data, data_len  element storage (data_len elements).
 *                   BSM_DATA_COPY: host or device pointer, copied into
 *                   library-owned device memory.
 *                   BSM_DATA_BORROW: device pointer kept by the handle; the
 *                   caller keeps it alive and unchanged-in-size until the
 *                   handle is destroyed or its pattern is replaced.
 *   data may be NULL only when nnzb == 0.
 * Errors: BSM_ERR_ARG for any violated rule above (nothing is launched),
 * BSM_ERR_ALLOC / BSM_ERR_CUDA.
 */
bsm_status bsm_create(bsm_t *out, int32_t nbr, int32_t nbc, const int32_t *row_bs,
                      const int32_t *col_bs, const int64_t *row_ptr, const int32_t *col_idx,
                      const int64_t *blk_off, int32_t dtype, const void *data,
                      int64_t data_len, int32_t data_mode);

/* Create an empty matrix (no blocks) with the given blocking (§2 blocked CSR
 * format); the usual target of bsm_multiply / bsm_add. */
bsm_status bsm_create_empty(bsm_t *out, int32_t nbr, int32_t nbc, const int32_t *row_bs,
                            const int32_t *col_bs, int32_t dtype);

/* Create a matrix with X's blocking and pattern and zero-filled, library-
 * owned data (for gradients; a library service, the paper has no
 * counterpart). */
bsm_status bsm_create_like(bsm_t *out, bsm_t X);

/* Release the handle and the device memory it owns (stream-ordered). */
bsm_status bsm_destroy(bsm_t X);

/* Sizes of X: any output pointer may be NULL.  Synchronises the stream.
 * (Handle queries and copies below are library services; the paper has no
 * counterpart.) */
bsm_status bsm_get_info(bsm_t X, int32_t *nbr, int32_t *nbc, int64_t *nnzb,
                        int64_t *data_len, int32_t *dtype);

/* Copy X's pattern out (host or device destinations; NULL skips an array):
 * row_ptr nbr+1 entries, col_idx and blk_off nnzb entries. */
bsm_status bsm_copy_pattern(bsm_t X, int64_t *row_ptr, int32_t *col_idx, int64_t *blk_off);

/* Copy X's data_len elements to `dst` (host or device). */
bsm_status bsm_copy_data(bsm_t X, void *dst);

/* Overwrite X's data with data_len elements from `src` (host or device);
 * invalidates the cached block norms. */
bsm_status bsm_set_data(bsm_t X, const void *src);

/* Make X's element storage the caller's device buffer `dptr` (X's
 * data_len elements of X's dtype, caller-owned, kept alive while X uses it);
 * storage X owned is released (stream-ordered).  Lets a framework hold the
 * values of a product in its own tensor without a second handle. */
bsm_status bsm_borrow_data(bsm_t X, void *dptr);

/* Device pointer of X's element storage (owned or borrowed). */
bsm_status bsm_data_ptr(bsm_t X, void **dptr);

/* FP64 Frobenius norm of every block (§2 filtering criterion): fma chain
 * over the block's elements in row-major order from +0.0, then IEEE sqrt;
 * FP32 elements widened first.  `out`: nnzb doubles, host or device. */
bsm_status bsm_block_norms(bsm_t X, double *out);

/* ---------------------------------------------------------------------- */
/* multiply                                                                 */
/* ---------------------------------------------------------------------- */

/*
 * C = alpha * A.B + beta * C  (§2: local multiplication C = C + A.B as
 * pairwise products of small dense blocks, with on-the-fly filtering).
 *
 *   A: nbr x nbk blocks, B: nbk x nbc blocks; A's block-column sizes must
 *   equal B's block-row sizes, C's block-row sizes A's, C's block-column
 *   sizes B's (else BSM_ERR_BLOCKING).  A and B may be the same handle; C
 *   must differ from both.  A, B and C share one dtype.
 *   filter_eps: when > 0, the block product A_ik.B_kj is performed iff
 *   norm(A_ik) * norm(B_kj) > filter_eps (FP64 norms as bsm_block_norms);
 *   when <= 0 every product of present blocks is performed.
 *   beta == 0: the old C is not read and its pattern is dropped.
 *   beta != 0: C's new pattern is the union of the old pattern and the
 *   pattern of the kept products; old blocks are scaled by beta.
 *   C's pattern and data are always replaced by library-owned storage; C
 *   keeps the kept-product list (canonical order: C block row i, then C
 *   block column j, then k, all ascending) for bsm_multiply_backward and,
 *   with opts->build_stacks, the per-shape stacks for bsm_get_stacks.
 *   opts may be NULL (defaults).  The call synchronises the stream once,
 *   after the symbolic phase, to size C.
 *   opts->no_sync = 1: nothing synchronises the host, so the call can be
 *   captured in a CUDA graph.  It needs an earlier (eager) multiply of the same
 *   A and B handles into C with the same filter_eps and precision, beta == 0
 *   and no post filter; it recomputes the pattern and values on the device into
 *   C's present storage, whose sizes come from that eager call.  If the
 *   recomputed sizes differ, the device sets C's status word
 *   (bsm_get_status -> BSM_ERR_CAPACITY) and writes nothing into C.  Stacks
 *   are not rebuilt.
 */
bsm_status bsm_multiply(double alpha, bsm_t A, bsm_t B, double beta, bsm_t C,
                        double filter_eps, const bsm_opts *opts);

/*
 * Adjoint of the last bsm_multiply that wrote C (C = alpha*A.B + ...), at
 * that multiply's keep-decisions:
 *   dA_ik = alpha * sum_j dC_ij . B_kj^T   over the kept products (i,k,j)
 *   dB_kj = alpha * sum_i A_ik^T . dC_ij
 * dC_data: device pointer laid out with C's blk_off (C's data_len elements,
 * C's dtype).  dA_data / dB_data: device pointers laid out like A's / B's
 * data (overwritten, blocks without products set to zero); either may be
 * NULL.  A and B must be the handles (same pattern) used in that multiply.
 */
bsm_status bsm_multiply_backward(double alpha, bsm_t C, const void *dC_data, bsm_t A, bsm_t B,
                                 void *dA_data, void *dB_data, const bsm_opts *opts);

/* Counts of the last multiply into C (§2: the products kept by the
 * on-the-fly filter): kept products, filtered candidate products and useful
 * FLOPs (sum of 2*m*n*k over kept products). */
bsm_status bsm_get_counts(bsm_t C, int64_t *products, int64_t *filtered, double *useful_flop);

/* Numeric engine of the last multiply into C (a library service). */
typedef enum {
    BSM_E_NONE = -1,        /* no multiply (or no output block)                 */
    BSM_E_FP64_CORES = 0,   /* FP64 (or FP32) FMA on the CUDA cores             */
    BSM_E_SPLIT_MMA = 1,    /* split precision on mma.sync tensor-core tiles    */
    BSM_E_OZAKI_MMA = 2,    /* Ozaki slices on mma.sync tensor-core tiles       */
    BSM_E_PANEL_TCGEN05 = 3 /* BSM_P_TF32x3_PANEL: tcgen05 row-panel tiles      */
} bsm_engine;
bsm_status bsm_get_engine(bsm_t C, int32_t *engine);

/* Per-phase timings of the last multiply into C (BSM_T_COUNT doubles, ms),
 * valid when profiling was on (a library service).  Synchronises the stream. */
bsm_status bsm_get_timings(bsm_t C, double *ms);

/*
 * Kept products of the last multiply into C as block indices (canonical
 * order): a_idx into A's blocks, b_idx into B's, c_idx into C's.  Pass NULL
 * pointers to query *nprod only; otherwise each array holds *nprod entries
 * (host or device).
 */
bsm_status bsm_get_products(bsm_t C, int64_t *nprod, int32_t *a_idx, int32_t *b_idx,
                            int32_t *c_idx);

/*
 * Stacks of the last multiply into C (built with opts->build_stacks): the
 * kept products bucketed by block shape (m, n, k) -- the batches of §2.
 * Shapes appear in lexicographic (m, n, k) order; inside a shape, products
 * keep the canonical (i, j, k) order.  Pass NULL arrays to query
 * *nshapes / *nprod; then shapes holds 3*nshapes int32 (m, n, k),
 * stack_ptr nshapes+1 int64, triples 3*nprod int64 (a_off, b_off, c_off)
 * element offsets.  Host or device destinations.
 */
bsm_status bsm_get_stacks(bsm_t C, int32_t *nshapes, int64_t *nprod, int32_t *shapes,
                          int64_t *stack_ptr, int64_t *triples);

/*
 * Allocation-free sizing of C = A.B (the paper has no counterpart; this is
 * a library convenience).  For callers that must not allocate device memory
 * when they size a product -- code running inside another framework's
 * memory pool or arena, or a host thread that may not call cudaMalloc /
 * cudaFree because those calls synchronise the device -- it computes, per
 * block row i of C, the number of kept block products (prod_cnt[i]) and of
 * C blocks (cblk_cnt[i]) under the same filter rule as bsm_multiply, and
 * totals[0..2] = (kept products, filtered candidates, sum of m*n*k).
 * All three outputs are device pointers supplied by the caller (nbr, nbr and
 * 3 int64).  The call allocates nothing: the FP64 block norms it needs live
 * in one fixed 16 MiB device array inside the library, so with
 * filter_eps > 0 it accepts nnzb(A) + nnzb(B) <= 2,097,152 and returns
 * BSM_ERR_CAPACITY beyond that.  The first call on each device looks the
 * array up (cudaGetSymbolAddress) and should come before any stream
 * capture; the lookup is repeated when the device's CUDA context has
 * changed (for instance after cudaDeviceReset, which reloads the module).
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race on it.
 */
bsm_status bsm_count_products_static(bsm_t A, bsm_t B, double filter_eps, int64_t *prod_cnt,
                                     int64_t *cblk_cnt, int64_t *totals);

/* ---------------------------------------------------------------------- */
/* block add (the purification chain's Z = 3 X^2 - 2 X^3)                   */
/* ---------------------------------------------------------------------- */

/* Z = a*X + b*Y over the union of X's and Y's patterns; with
 * filter_eps > 0 a result block is kept iff its FP64 norm > filter_eps.
 * X, Y and Z share one blocking and dtype; Z differs from X and Y.  Z's
 * pattern and data are replaced.  opts may be NULL; opts->no_sync = 1 works as
 * for bsm_multiply (needs an earlier eager add of the same X, Y, a, b and
 * filter_eps into Z).  Each element is one rounded product per term and one
 * rounded sum (no fused multiply-add). */
bsm_status bsm_add(double a, bsm_t X, double b, bsm_t Y, bsm_t Z, double filter_eps, const bsm_opts *opts);

/* Device status word of the last call that wrote X (a library service): BSM_OK, or
 * BSM_ERR_CAPACITY when a no-sync call found sizes different from its eager
 * call (then *status has bit 1 set).  Synchronises the stream. */
bsm_status bsm_get_status(bsm_t X, int32_t *status);

/* Adjoint of the last bsm_add that wrote Z (the paper has no counterpart:
 * differentiation through the purification chain; Z = a*X + b*Y, blocks with norm
 * <= eps dropped), at that add's keep-decisions: dX = a*dZ on the X blocks
 * that reached Z, dY = b*dZ likewise, zero elsewhere.  dZ_data has Z's
 * layout; dX_data / dY_data have X's / Y's layout (overwritten; either may be
 * NULL).  X and Y must be the handles of that add. */
bsm_status bsm_add_backward(bsm_t Z, const void *dZ_data, bsm_t X, bsm_t Y, void *dX_data, void *dY_data);

#ifdef __cplusplus
}
#endif
#endif /* BSM_H */
