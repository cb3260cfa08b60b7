// Internal declarations of libbsm (not part of the C ABI).
//
// Device layout of a block-CSR matrix (the blocked CSR format of DBCSR,
// Bethune et al. 2017 §2):
//   row_bs[nbr], col_bs[nbc]      int32 block sizes
//   row_ptr[nbr+1]                int64
//   col_idx[nnzb]                 int32, ascending inside a row
//   blk_off[nnzb]                 int64 element offset of each block
//   blk_rc[nnzb]                  int32 packed (rows << 16) | cols of each block
//   data[data_len]                FP64 or FP32, row-major inside a block
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bsm.h"

namespace bsm {

constexpr int kMaxBlockDim = 256;

__host__ __device__ inline int rc_rows(int32_t rc) { return (int)((uint32_t)rc >> 16); }
__host__ __device__ inline int rc_cols(int32_t rc) { return (int)(rc & 0xffff); }

// Status bits written by kernels into a per-call device word.
enum : int32_t { DEV_OK = 0, DEV_ERR_CAPACITY = 1, DEV_ERR_RANGE = 2 };

// One stored operand view for the numeric kernels: element (r, t) of the
// logical R x T block is data[off + (trans ? t*R + r : r*T + t)], where the
// stored block is R x T (trans = 0) or T x R (trans = 1).
template <typename T>
struct OperandView {
    const T *data;
    const int64_t *blk_off;
    const int32_t *blk_rc;
    int trans;
};

}  // namespace bsm

// The handle behind bsm_t.
struct bsm_mat {
    int32_t nbr = 0, nbc = 0;
    int32_t dtype = BSM_FP64;
    int64_t nnzb = 0, data_len = 0;
    std::vector<int32_t> h_row_bs, h_col_bs;  // host copies of the blocking
    int32_t *row_bs = nullptr, *col_bs = nullptr;
    int64_t *row_ptr = nullptr;
    int32_t *col_idx = nullptr;
    int64_t *blk_off = nullptr;
    int32_t *blk_rc = nullptr;
    void *data = nullptr;
    bool own_data = false;
    double *norms = nullptr;
    bool norms_valid = false;
    int32_t max_bs_row = 0, max_bs_col = 0;

    // results of the last multiply that wrote this matrix
    int64_t nprod = 0, nfiltered = 0;
    double useful_flop = 0.0;
    int64_t *cptr = nullptr;  // [nnzb+1] product segment of every block
    int32_t *pa = nullptr, *pb = nullptr, *pc = nullptr;  // [nprod]
    int32_t nshapes = 0;
    std::vector<int32_t> h_shapes;  // 3*nshapes
    int64_t *stack_ptr = nullptr;   // [nshapes+1] device
    int64_t *triples = nullptr;     // [3*nprod] device
    bsm_t prod_A = nullptr, prod_B = nullptr;  // operands of that multiply
    int64_t prod_A_nnzb = -1, prod_B_nnzb = -1;
    double timings[BSM_T_COUNT] = {0};
    bool timings_valid = false;

    // device status word of the last call that wrote this matrix
    int32_t *status = nullptr;
    // sizes of the last eager call that wrote this matrix; a no-sync call
    // with the same operands reuses them and this matrix's storage
    struct Plan {
        int kind = 0;  // 0 none, 1 multiply, 2 add
        bsm_t A = nullptr, B = nullptr;
        int64_t A_nnzb = -1, B_nnzb = -1;
        double eps = 0.0;
        int32_t prec = 0;
        int32_t kprec = 0;  // precision the kernels ran (the Ozaki path with only lane items runs FP64)
        int64_t nprod = 0, nnzb = 0, len = 0, max_ccnt = 0, nfilt = 0, mnk = 0;
        int32_t nchunk = 1;
        int64_t packA = 0, packB = 0;
        bool uses_cores = false;  // some items run the CUDA-core split variant
        int64_t u_nnzb = 0, u_len = 0;  // add: union before the norm filter
    } plan;
    int32_t *item_order = nullptr;      // numeric processing order of the last eager multiply
    int64_t *n_marked = nullptr;        // device count of its second-variant items (or null)
    int64_t *item_groups = nullptr;     // device bounds of its tile-row groups (or null)
    // rank of every block row in a breadth-first order through shared block
    // columns (built on demand, dropped with the pattern); schedules numeric work
    int32_t *row_rank = nullptr;        // [nbr]
    // rank of every block column in a breadth-first order through shared block
    // rows (the same for columns; built on demand, dropped with the pattern)
    int32_t *col_rank = nullptr;        // [nbc]
    // first global row / column of every block row / column ([nbr+1], [nbc+1];
    // built on demand, kept until the handle is destroyed)
    int32_t *row_start = nullptr, *col_start = nullptr;
    // numeric engine of the last multiply into this matrix (bsm_engine) and
    // what its numeric launch ran (bsm_get_launch_config)
    int32_t engine = -1;
    int32_t launch_cfg[6] = {-1, -1, 0, 0, 0, 0};
    // row-panel tiling of this matrix as the left operand of a multiply with
    // panel_B (built on demand, dropped with the pattern): block rows in
    // ord_r order, the right operand's block columns in ord_c order (pos_c
    // is its inverse); only the tiles' locality depends on them
    bsm_t panel_B = nullptr;
    int64_t panel_B_nnzb = -1;
    int32_t panel_B_nbc = -1;
    int32_t *panel_ord_r = nullptr, *panel_ord_c = nullptr, *panel_pos_c = nullptr;
    // column-major copy of the pattern (built on demand, dropped with the pattern)
    int64_t *t_ptr = nullptr;           // [nbc+1]
    int32_t *t_row = nullptr, *t_blk = nullptr;  // [nnzb]

    // provenance of the last bsm_add that wrote this matrix (for its adjoint):
    // per block, the element offset of the matching X / Y block or -1
    int64_t *add_xsrc = nullptr, *add_ysrc = nullptr;
    bsm_t add_X = nullptr, add_Y = nullptr;
    int64_t add_X_nnzb = -1, add_Y_nnzb = -1;
    double add_a = 0.0, add_b = 0.0;
};

namespace bsm {

// ---------------------------------------------------------------- host glue
cudaStream_t stream();
bool profiling();
bsm_status set_error(bsm_status st, const std::string &msg);
bsm_status cuda_check(cudaError_t e, const char *what);
bsm_status dalloc(void **p, size_t bytes);
void dfree(void *p);
// Kernel launches issued by the library since it was loaded.
void count_launch(int n);
int64_t launch_count();
template <typename T>
inline bsm_status dalloc_t(T **p, size_t n) {
    return dalloc(reinterpret_cast<void **>(p), n * sizeof(T) + (n == 0 ? 16 : 0));
}

// ---------------------------------------------------------------- launchers
// (all asynchronous on `s`; they return cudaGetLastError())
cudaError_t launch_blk_rc(const bsm_mat *X, int32_t *out_rc, cudaStream_t s);
cudaError_t launch_block_norms(const bsm_mat *X, double *out, cudaStream_t s);

// Exclusive scan of n int64 values into out[0..n] (out[n] = total).
// `tmp` needs scan_tmp_elems(n) int64.
size_t scan_tmp_elems(int64_t n);
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);

struct SymbolicArgs {
    int32_t nbr, nbk, nbc;
    const int32_t *a_row_bs, *a_col_bs;  // m sizes, k sizes
    const int64_t *a_row_ptr;
    const int32_t *a_col_idx;
    const double *a_norm;
    const int64_t *b_row_ptr;
    const int32_t *b_col_idx;
    const int32_t *b_col_bs;             // n sizes
    const double *b_norm;
    const int64_t *o_row_ptr;            // old C (beta != 0) or nullptr
    const int32_t *o_col_idx;
    const int64_t *o_blk_off;
    double eps;
    int use_filter;
    int32_t nwords;                      // ceil(nbc / 32)
    const int32_t *status;               // nullable: kernels that read it do nothing when *status != 0
};

// Per block row: kept products, distinct C columns, C elements; bitmaps of
// the C columns (nbr * nwords words); totals[0] += filtered, totals[1] += sum m*n*k,
// totals[2] = max over rows of the distinct C columns.
cudaError_t launch_symbolic_count(const SymbolicArgs &a, int64_t *prod_cnt, int64_t *ccol_cnt,
                                  int64_t *celem_cnt, uint32_t *bitmaps,
                                  unsigned long long *totals, cudaStream_t s);

struct FillOut {
    const int64_t *prod_ptr, *crow_ptr, *celem_ptr;  // scans, [nbr+1]
    int32_t *c_col_idx;
    int64_t *c_blk_off;
    int32_t *c_blk_rc;
    int64_t *cptr;       // [nnzbC+1]
    int32_t *pa, *pb, *pc;
    int64_t *old_off;    // [nnzbC] or nullptr
    int32_t max_ccnt;
    int32_t nchunk;      // A-block chunks per row (1..8, one warp each)
    int32_t row0;        // first block row of this launch (row panels; 0 otherwise)
    int64_t prod_base;   // prod_ptr[row0]: product offsets are written relative to it
};
// Fill block rows [o.row0, o.row0 + nrows) (nrows < 0: all rows).
cudaError_t launch_symbolic_fill(const SymbolicArgs &a, const uint32_t *bitmaps, const FillOut &o,
                                 cudaStream_t s, int32_t nrows = -1);
int64_t symbolic_fill_smem_bytes(int32_t nwords, int32_t max_ccnt, int nchunk);
// Fill through B's columns (B transposed: bt_ptr[nbc+1], bt_k / bt_b = block row
// and block index of every B block, column-major, ascending k inside a column).
cudaError_t launch_symbolic_fill_cols(const SymbolicArgs &a, const uint32_t *bitmaps, const FillOut &o,
                                      const int64_t *bt_ptr, const int32_t *bt_k, const int32_t *bt_b,
                                      cudaStream_t s, int32_t nrows = -1);
int64_t symbolic_fill_cols_smem_bytes(int32_t nwords, int32_t max_ccnt, int32_t nbk);
cudaError_t launch_blk_rows(const bsm_mat *X, int32_t *rows, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits.
// Buffers: keys/vals in and out may not alias; `tmp` needs
// radix_tmp_elems(n) int64.  Result lands in (keys_out, vals_out).
size_t radix_tmp_elems(int64_t n);
cudaError_t launch_radix_sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, uint32_t *keys_alt,
                                    int32_t *vals_alt, uint32_t *keys_out, int32_t *vals_out,
                                    int64_t n, int key_bits, int64_t *tmp, cudaStream_t s);

// shape id of every product (for stacks): (mi * ns + ni) * ns + ki
cudaError_t launch_product_shape_ids(int64_t nprod, const int32_t *pa, const int32_t *pb,
                                     const int32_t *a_blk_rc, const int32_t *b_blk_rc,
                                     const int32_t *size_index /*[kMaxBlockDim+1]*/, int32_t ns,
                                     uint32_t *keys, int32_t *iota, cudaStream_t s);
// Stacks in two passes (per-tile shape histogram, then every triple written
// to its place) for at most stack_max_bins() shapes; counts[nbins] = products
// per shape.  `tmp` needs stack_tmp_elems(nprod, nbins) int64.
int stack_max_bins();
size_t stack_tmp_elems(int64_t nprod, int32_t nbins);
cudaError_t launch_stacks_direct(int64_t nprod, const int32_t *pa, const int32_t *pb, const int32_t *pc,
                                 const int32_t *a_rc, const int32_t *b_rc, const int32_t *size_index, int32_t ns,
                                 int32_t nbins, const int64_t *a_off, const int64_t *b_off, const int64_t *c_off,
                                 int64_t *triples, int64_t *counts, int64_t *tmp, cudaStream_t s);
cudaError_t launch_stack_triples(int64_t nprod, const int32_t *order, const int32_t *pa,
                                 const int32_t *pb, const int32_t *pc, const int64_t *a_off,
                                 const int64_t *b_off, const int64_t *c_off, int64_t *triples,
                                 cudaStream_t s);
cudaError_t launch_histogram_u32(int64_t n, const uint32_t *keys, int64_t nbins, int64_t *counts,
                                 cudaStream_t s);
cudaError_t launch_gather_i32(int64_t n, const int32_t *order, const int32_t *src, int32_t *dst,
                              cudaStream_t s);
cudaError_t launch_iota_keys(int64_t n, const int32_t *src, uint32_t *keys, int32_t *iota,
                             cudaStream_t s);
// Scheduling key of every block: class = table[size_index[rows] * ns +
// size_index[cols]], then row_rank[block row] (row_rank may be null: key =
// class only); with col_rank and tile > 0, the 2-D tile (row_rank / tile,
// col_rank[block column] / tile) instead of the row rank (nct = number of
// column tiles).
cudaError_t launch_class_keys(int64_t n, const int32_t *blk_rc, const int32_t *size_index, int32_t ns,
                              const int32_t *table, const int32_t *blk_row, const int32_t *row_rank, int32_t nbr,
                              const int32_t *blk_col, const int32_t *col_rank, int32_t tile, int32_t nct,
                              uint32_t *keys, int32_t *iota, cudaStream_t s);

// ---------------------------------------------------------------- numeric
struct NumericArgs {
    int64_t n_items;
    const int64_t *seg_ptr;     // [n_items+1] product range of each output block
    const int32_t *px, *py;     // operand block index of every product
    // output blocks: item q writes block q of the output matrix
    void *out_data;
    const int64_t *out_blk_off;
    const int32_t *out_blk_rc;
    // operands
    const void *x_data; const int64_t *x_blk_off; const int32_t *x_blk_rc; int x_trans;
    const void *y_data; const int64_t *y_blk_off; const int32_t *y_blk_rc; int y_trans;
    double alpha, beta;
    const void *old_data;       // beta != 0: old values at old_off[q] (or -1)
    const int64_t *old_off;
    int32_t dtype;
    int32_t prec;
    int32_t flush_every;
    // pre-split operand planes (tensor-core paths)
    const void *x_pack; const int64_t *x_pack_off;
    const void *y_pack; const int64_t *y_pack_off;
    // unpacked split pieces (CUDA-core variant of the split paths)
    const float *x_plain, *y_plain;
    int32_t max_out_rows, max_out_cols;
    const int32_t *item_order;  // nullable: processing order of the items (grouped by block shape);
                                // bit 31 marks the second variant of the item's shape
    const int64_t *n_lane_items;  // nullable (CUDA-core FP64 path): the last *n_lane_items items of
                                  // item_order are tiny blocks computed one per lane
    // nullable (split paths): item_order positions [0] end of the blocks of two
    // tile rows and more, [1] end of the blocks of one tile row (start of the
    // lane items); each group runs in its own kernel instance
    const int64_t *item_groups;
    int32_t group;              // set by the launcher: the group one launch covers
    const int32_t *status;      // nullable: the kernel does nothing when *status != 0
    unsigned long long *work_counter;  // 4 x 8 bytes of device memory, zeroed by the launcher
    // Ozaki path: biased FP64 exponent field of the largest |x| of every global
    // line (logical rows of X, logical columns of Y) and the first line of every block
    const int32_t *x_exp, *x_line0, *y_exp, *y_line0;
    // launch shape and pass caps (bsm_set_tuning; 0 = the kernel's default)
    int32_t pass_mt, pass_nt;   // fragment tiles per pass along M / N
    int32_t cta_warps;          // warps per CTA (4 or 8; mma.sync kernels)
    int32_t ctas_per_sm;        // persistent CTAs per SM (0: as many as fit)
    int32_t fp64_build;         // FP64 FMA kernel build: 0 by the largest block, 1 narrow, 2 wide
    // sizes the debug build's bounds checks test every item against
    int64_t n_prod;             // entries of px / py
    int64_t x_nnzb, y_nnzb;     // operand blocks
    int64_t x_len, y_len;       // operand elements
    int64_t out_len, old_len;   // output elements, old output elements (beta != 0)
    int64_t x_pack_words, y_pack_words;  // packed planes (0: none)
};
// Debug builds (BSM_DEBUG): bits of the bounds checks of the last numeric
// launch (read and cleared; 0 in release builds).
uint32_t numeric_debug_bits(cudaStream_t s);
// What a numeric launch ran (bsm_get_launch_config).
struct NumericLaunch {
    int32_t kernel;     // BSM_K_* of include/bsm.h
    int32_t build;      // FP64 FMA kernel build (0 small, 1 narrow, 2 wide) or -1
    int32_t cta_threads, grid, pass_mt, pass_nt;
};
cudaError_t launch_numeric(const NumericArgs &a, cudaStream_t s, NumericLaunch *info = nullptr);
// out[g] = number of keys below thr[g] in the ascending keys[0..n) (g < 2)
cudaError_t launch_group_bounds(const uint32_t *keys, int64_t n, uint32_t thr0, uint32_t thr1, int64_t *out,
                                cudaStream_t s);

// Ozaki path: line0[b] = first global line of block b, lines being the stored
// rows (by_rows) or the stored columns of M's blocks; exps[line] = max biased
// exponent field of |x| over the line (exps zeroed by the caller).
cudaError_t launch_oz_lines(const bsm_mat *M, int by_rows, int32_t *line0, int32_t *exps, cudaStream_t s);

// Tensor-core paths: packed fragment planes of a matrix in role X (A
// fragments, logical R x T) or Y (B fragments, logical T x S).
struct PackInfo {
    int64_t total_words;        // 32-bit words
};
cudaError_t launch_pack_sizes(const bsm_mat *M, int role_y, int trans, int prec, int64_t *pack_words,
                              cudaStream_t s);
// line0 / exps: the Ozaki path's line exponents of M in this role (else null)
cudaError_t launch_pack(const bsm_mat *M, int role_y, int trans, int prec, const int64_t *pack_off,
                        void *pack, const int32_t *status, cudaStream_t s, const int32_t *line0 = nullptr,
                        const int32_t *exps = nullptr);
// Unpacked split pieces of M's data (split_pieces(prec) floats per element).
int split_pieces(int prec);
cudaError_t launch_split_plain(const bsm_mat *M, int prec, float *out, cudaStream_t s);
// Mark the items of the classes that run the CUDA-core split variant (bit 31).
cudaError_t launch_mark_variant(int64_t n, int32_t *order, const int32_t *blk_rc, const int32_t *size_index, int32_t ns,
                                const int8_t *variant_of_class, unsigned long long *marked, cudaStream_t s);

// *status |= DEV_ERR_CAPACITY unless, for q < n (n <= 8), actual[q] == expected[q]
// (or actual[q] <= expected[q] where at_most[q] is set)
struct PlanCheck {
    const int64_t *actual[8];
    int64_t expected[8];
    int at_most[8];
    int n;
};
cudaError_t launch_check_plan(const PlanCheck &c, int32_t *status, cudaStream_t s);
// dst[0..n) = src[0..n) unless *status != 0
cudaError_t launch_copy_i64_if_ok(int64_t n, const int64_t *src, int64_t *dst, const int32_t *status, cudaStream_t s);

// ---------------------------------------------------------------- add
cudaError_t launch_add_count(const bsm_mat *X, const bsm_mat *Y, int64_t *ccnt, int64_t *celem,
                             cudaStream_t s);
struct AddFill {
    const int64_t *zrow_ptr, *zelem_ptr;
    int32_t *z_col_idx;
    int64_t *z_blk_off;
    int32_t *z_blk_rc;
    int64_t *x_src, *y_src;  // [nnzbZ] source block offsets or -1
};
cudaError_t launch_add_fill(const bsm_mat *X, const bsm_mat *Y, const AddFill &f, const int32_t *status,
                            cudaStream_t s);
cudaError_t launch_add_values(int64_t nnzb, const int64_t *z_blk_off, const int32_t *z_blk_rc,
                              const int64_t *x_src, const int64_t *y_src, double a, const void *x,
                              double b, const void *y, void *z, int32_t dtype, const int32_t *status,
                              cudaStream_t s);

// Post filter: keep flag per block (norm > eps), then compaction.
cudaError_t launch_keep_flags(int64_t nnzb, const double *norms, double eps, int64_t *keep,
                              cudaStream_t s);
cudaError_t launch_row_keep_counts(int32_t nbr, const int64_t *row_ptr, const int64_t *keep,
                                   const int32_t *blk_rc, int64_t *row_cnt, int64_t *row_elem,
                                   cudaStream_t s);
struct CompactArgs {
    int32_t nbr;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *blk_off;
    const int32_t *blk_rc;
    const int64_t *keep_scan;   // exclusive scan of keep flags [nnzb+1]
    const int64_t *nrow_ptr;    // new row pointers
    const int64_t *nelem_ptr;   // new per-row element starts
    const void *data;
    int32_t dtype;
    int32_t *n_col_idx;
    int64_t *n_blk_off;
    int32_t *n_blk_rc;
    void *n_data;
    const int32_t *status;      // nullable: nothing is written when *status != 0
};
cudaError_t launch_compact(const CompactArgs &c, cudaStream_t s);
// dst[kscan[b]] = src[b] for every kept block b (kscan: exclusive scan of keep flags)
cudaError_t launch_compact_i64(int64_t nnzb, const int64_t *kscan, const int64_t *src, int64_t *dst,
                               const int32_t *status, cudaStream_t s);
// adjoint of Z = a*X + b*Y: dX[xsrc+e] = a*dZ, dY[ysrc+e] = b*dZ (dX, dY zeroed by the caller)
cudaError_t launch_add_backward(int64_t nnzb, const int64_t *z_blk_off, const int32_t *z_blk_rc,
                                const int64_t *x_src, const int64_t *y_src, double a, double b, const void *dZ,
                                void *dX, void *dY, int32_t dtype, cudaStream_t s);

// ---------------------------------------------------------------------------
// Row-panel TF32x3 numeric kernel on tcgen05 tensor cores (k_panel.cu), for
// FP64 matrices whose blocks all have one size s <= 24 and multiplies whose
// norm filter removed no product.  Tiles of 5 x 5 output blocks: row group g
// holds block rows ord_r[5g .. 5g+4], column group h block columns
// ord_c[5h .. 5h+4]; cblk[t][5r + c] is the index of C block (row slot r,
// column slot c) of tile t, or -1.
struct PanelArgs {
    int32_t nbr, nbc, s;
    int32_t nbk;                          // inner block dimension (A's block columns)
    int64_t n_tiles;
    const int32_t *tile_order;            // [n_tiles] processing order
    const int32_t *tile_g, *tile_h;       // [n_tiles]
    const int32_t *cblk;                  // [n_tiles * 25]
    const int32_t *ord_r, *ord_c;         // block row / column of every position
    const int64_t *a_row_ptr; const int32_t *a_col_idx;              // A's pattern
    const int64_t *b_t_ptr; const int32_t *b_t_row, *b_t_blk;        // B's pattern by columns
    const uint8_t *a_pack, *b_pack;       // 4608 bytes per block (TF32 hi and lo planes)
    const uint8_t *zeros;                 // 4608 zero bytes
    // k-steps of every tile t: steps[step_ptr[t] .. step_ptr[t+1]), each 10
    // block indices (A's 5 row slots, then B's 5 column slots; -1: absent)
    const int64_t *step_ptr;
    int32_t *steps;
    double *c_data; const int64_t *c_blk_off;
    double alpha, beta;
    const void *old_data; const int64_t *old_off;  // beta != 0: old values (or null)
    int32_t *status;                      // set to BSM_ERR_TIMEOUT when a wait gives up
    unsigned long long *work_counter;     // zeroed by the caller
    unsigned long long wait_ns;           // limit of the main-loop waits (the drain of
                                          // work in flight always allows 2 s)
    int32_t pair;                         // k-steps summed in one accumulator buffer (>= 1)
};
// limit of the panel kernel's main-loop waits (bsm_set_wait_limit)
unsigned long long panel_wait_ns();
int64_t panel_pack_bytes(int64_t nblk);
int panel_slot();
int panel_pair();   // default k-steps per accumulator buffer
int panel_tile_rows();
int panel_tile_cols();
size_t panel_tile_smem(int32_t ngc);
size_t panel_smem_bytes();
// planes of every block of M (trans = 1: of its transposed blocks)
cudaError_t launch_panel_pack(const bsm_mat *M, int trans, void *out, cudaStream_t s);
cudaError_t launch_panel_tiles_count(int32_t nbr, const int32_t *ord_r, const int32_t *pos_c,
                                     const int64_t *c_row_ptr, const int32_t *c_col, int32_t ngc, int64_t *tile_cnt,
                                     cudaStream_t s);
cudaError_t launch_panel_tiles_fill(int32_t nbr, const int32_t *ord_r, const int32_t *pos_c,
                                    const int64_t *c_row_ptr, const int32_t *c_col, int32_t ngc,
                                    const int64_t *tile_ptr, int32_t *tile_g, int32_t *tile_h, int32_t *cblk,
                                    cudaStream_t s);
cudaError_t launch_panel_tile_keys(int64_t ntiles, const int32_t *tile_g, const int32_t *tile_h, int sg, int sh,
                                   int32_t ngc, uint32_t *keys, int32_t *iota, cudaStream_t s);
// k-steps of every tile: counts (fill = 0: step_cnt[t]) or records (fill = 1)
cudaError_t launch_panel_steps(const PanelArgs &a, int fill, int64_t *step_cnt, cudaStream_t s);
cudaError_t launch_panel_numeric(const PanelArgs &a, cudaStream_t s);

}  // namespace bsm
