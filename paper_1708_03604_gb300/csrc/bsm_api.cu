// C ABI of libbsm (declared in include/bsm.h): handle management, argument
// validation and the orchestration of the symbolic, stack and numeric
// kernels of the local block-sparse multiply (DBCSR, Bethune et al. 2017 §2).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "bsm_internal.cuh"

namespace bsm {

namespace {
thread_local std::string t_err;
cudaStream_t g_stream = nullptr;
bool g_prof = false;
bool g_pool_configured = false;
// limit of the panel kernel's main-loop waits (bsm_set_wait_limit)
std::atomic<unsigned long long> g_wait_ns{2000000000ull};
// kept products one pass of a multiply holds (bsm_set_product_limit)
std::atomic<int64_t> g_product_limit{INT32_MAX};
int64_t *g_host = nullptr;  // pinned host words for small device->host reads
// numeric variant per (precision, rows, cols) of the output block; -1 = the
// library default (see variant_of)
int8_t g_variant[6][kMaxBlockDim + 1][kMaxBlockDim + 1];
bool g_variant_init = false;

// shapes the lane-per-block variant takes: up to 16 elements, plus 5 x 5 (on
// the split paths the same pieces multiplied with FP32 FMA) and, on the paths
// whose lane variant is plain FP64 FMA, 6 x 6 (a 6 x 6 compensated pair would
// raise the split kernels' register count for every item)
bool lane_eligible(int prec, int m, int n) {
    const bool fp64 = prec == BSM_P_FP64 || prec == BSM_P_FP64_DMMA || prec == BSM_P_OZAKI;
    return m * n <= 16 || (m == 5 && n == 5) || (fp64 && m == 6 && n == 6);
}

int variant_of(int prec, int m, int n) {
    if (!g_variant_init) {
        std::memset(g_variant, -1, sizeof(g_variant));
        g_variant_init = true;
    }
    const int v = g_variant[prec][m][n];
    // variant 1: one lane per output block (CUDA cores), for blocks of up to 16
    // elements (default) and for 5 x 5 and 6 x 6 blocks (on request)
    if (!lane_eligible(prec, m, n)) return 0;
    if (v >= 0) return v;
    return m * n <= 16 ? 1 : 0;
}
// true when every output block shape (a row size of `rows` by a column size
// of `cols`) runs the lane-per-block variant for `prec`
bool all_lane(int prec, const std::vector<int32_t> &rows, const std::vector<int32_t> &cols) {
    bool rs[kMaxBlockDim + 1] = {}, cs[kMaxBlockDim + 1] = {};
    for (int32_t v : rows) rs[v] = true;
    for (int32_t v : cols) cs[v] = true;
    for (int m = 1; m <= kMaxBlockDim; ++m)
        if (rs[m])
            for (int n = 1; n <= kMaxBlockDim; ++n)
                if (cs[n] && variant_of(prec, m, n) != 1) return false;
    return true;
}
std::atomic<int64_t> g_launches{0};
// launch and pass shape per precision (bsm_set_tuning); -1 = the default
int32_t g_tune[7][BSM_TUNE_COUNT];
bool g_tune_init = false;
int32_t *tune_of(int prec) {
    if (!g_tune_init) {
        for (auto &row : g_tune)
            for (auto &v : row) v = -1;
        g_tune_init = true;
    }
    return g_tune[prec];
}
// allowed range of a tuning value for a precision: [lo, hi], lo > hi = none
void tune_range(int prec, int param, int *lo, int *hi) {
    const bool split = prec == BSM_P_TF32x3 || prec == BSM_P_BF16x3 || prec == BSM_P_BF16x6;
    *lo = 1;
    *hi = 0;
    switch (param) {
        case BSM_TUNE_CTA_WARPS:
            if (split || prec == BSM_P_OZAKI) { *lo = 2; *hi = 4; }
            else if (prec != BSM_P_TF32x3_PANEL) { *lo = 4; *hi = 4; }
            break;
        case BSM_TUNE_CTAS_PER_SM:
            if (prec != BSM_P_TF32x3_PANEL) { *lo = 0; *hi = 16; }
            break;
        case BSM_TUNE_PASS_MT:
            if (split) { *lo = 1; *hi = 2; }
            else if (prec == BSM_P_FP64_DMMA) { *lo = 1; *hi = 3; }
            break;
        case BSM_TUNE_PASS_NT:
            if (split || prec == BSM_P_FP64_DMMA || prec == BSM_P_OZAKI) { *lo = 1; *hi = 3; }
            break;
        case BSM_TUNE_FP64_BUILD:
            if (prec == BSM_P_FP64) { *lo = 0; *hi = 2; }
            break;
        case BSM_TUNE_SCHED_TILE:
            if (prec != BSM_P_TF32x3_PANEL) { *lo = 0; *hi = 4096; }
            break;
        case BSM_TUNE_ENGINE:
            if (prec == BSM_P_TF32x3) { *lo = 0; *hi = 1; }
            break;
        case BSM_TUNE_PANEL_STEPS:
            if (prec == BSM_P_TF32x3 || prec == BSM_P_TF32x3_PANEL) { *lo = 1; *hi = 8; }
            break;
    }
}
// the tuning of `prec` into the numeric launch arguments
void apply_tuning(int prec, NumericArgs &na) {
    const int32_t *t = tune_of(prec);
    na.cta_warps = t[BSM_TUNE_CTA_WARPS] > 0 ? t[BSM_TUNE_CTA_WARPS] : 4;
    na.ctas_per_sm = t[BSM_TUNE_CTAS_PER_SM] > 0 ? t[BSM_TUNE_CTAS_PER_SM] : 0;
    na.pass_mt = t[BSM_TUNE_PASS_MT] > 0 ? t[BSM_TUNE_PASS_MT] : 0;
    na.pass_nt = t[BSM_TUNE_PASS_NT] > 0 ? t[BSM_TUNE_PASS_NT] : 0;
    na.fp64_build = t[BSM_TUNE_FP64_BUILD] > 0 ? t[BSM_TUNE_FP64_BUILD] : 0;
}

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) dfree(p);
    }
    template <typename T>
    bsm_status get(T **p, size_t n) {
        bsm_status st = dalloc_t(p, n);
        if (st == BSM_OK) ptrs.push_back(*p);
        return st;
    }
    void release(void *p) {  // hand ownership of p to the caller
        ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end());
    }
};

bsm_status ensure_globals() {
    if (!g_pool_configured) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return set_error(BSM_ERR_CUDA, "cudaGetDevice failed");
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        g_pool_configured = true;
    }
    if (!g_host) {
        if (cudaMallocHost(&g_host, 64 * sizeof(int64_t)) != cudaSuccess) {
            g_host = nullptr;
            return set_error(BSM_ERR_ALLOC, "cudaMallocHost failed");
        }
    }
    return BSM_OK;
}

size_t esize(int32_t dtype) { return dtype == BSM_FP64 ? 8 : 4; }

bool same_vec(const std::vector<int32_t> &a, const std::vector<int32_t> &b) { return a == b; }

// Phase marks of a multiply: CUDA events on the library stream when
// profiling is on (bsm_get_timings), and NVTX ranges on the issuing host
// thread always (no-ops unless a profiler is attached).
struct Events {
    cudaEvent_t ev[BSM_T_COUNT + 1] = {};
    bool on = false;
    bool range_open = false;
    void start() {
        on = g_prof;
        if (!on) return;
        for (auto &e : ev) cudaEventCreate(&e);
    }
    void mark(int idx) {
        static const char *const names[BSM_T_COUNT + 1] = {"bsm norms",  "bsm symbolic count", "bsm fill",
                                                           "bsm stacks", "bsm pack and order", "bsm numeric",
                                                           "bsm post",   ""};
        if (on) cudaEventRecord(ev[idx], g_stream);
        if (range_open) nvtxRangePop();
        range_open = idx < BSM_T_COUNT;
        if (range_open) nvtxRangePushA(names[idx]);
    }
    ~Events() {
        if (range_open) nvtxRangePop();
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

void free_results(bsm_mat *C) {
    dfree(C->cptr); C->cptr = nullptr;
    dfree(C->pa); C->pa = nullptr;
    dfree(C->pb); C->pb = nullptr;
    dfree(C->pc); C->pc = nullptr;
    dfree(C->stack_ptr); C->stack_ptr = nullptr;
    dfree(C->triples); C->triples = nullptr;
    C->nprod = 0; C->nfiltered = 0; C->useful_flop = 0.0;
    C->nshapes = 0; C->h_shapes.clear();
    C->prod_A = C->prod_B = nullptr;
    C->prod_A_nnzb = C->prod_B_nnzb = -1;
    C->timings_valid = false;
    dfree(C->add_xsrc); C->add_xsrc = nullptr;
    dfree(C->add_ysrc); C->add_ysrc = nullptr;
    C->add_X = C->add_Y = nullptr;
    C->add_X_nnzb = C->add_Y_nnzb = -1;
    C->plan = bsm_mat::Plan{};
}

void free_pattern(bsm_mat *X) {
    dfree(X->row_ptr); X->row_ptr = nullptr;
    dfree(X->col_idx); X->col_idx = nullptr;
    dfree(X->blk_off); X->blk_off = nullptr;
    dfree(X->blk_rc); X->blk_rc = nullptr;
    if (X->own_data) dfree(X->data);
    X->data = nullptr;
    X->own_data = false;
    dfree(X->norms); X->norms = nullptr;
    X->norms_valid = false;
    dfree(X->item_order); X->item_order = nullptr;
    dfree(X->n_marked); X->n_marked = nullptr;
    dfree(X->item_groups); X->item_groups = nullptr;
    dfree(X->row_rank); X->row_rank = nullptr;
    dfree(X->col_rank); X->col_rank = nullptr;
    dfree(X->panel_ord_r); X->panel_ord_r = nullptr;
    dfree(X->panel_ord_c); X->panel_ord_c = nullptr;
    dfree(X->panel_pos_c); X->panel_pos_c = nullptr;
    X->panel_B = nullptr;
    dfree(X->t_ptr); X->t_ptr = nullptr;
    dfree(X->t_row); X->t_row = nullptr;
    dfree(X->t_blk); X->t_blk = nullptr;
    X->nnzb = 0;
    X->data_len = 0;
}

bsm_status check_opts(const bsm_opts *o, bsm_opts *out) {
    bsm_opts_default(out);
    if (!o) return BSM_OK;
    *out = *o;
    if (o->prec < BSM_P_FP64 || o->prec > BSM_P_TF32x3_PANEL) return set_error(BSM_ERR_ARG, "opts.prec out of range");
    if (o->flush_every < -1024 || o->flush_every > 1024) return set_error(BSM_ERR_ARG, "opts.flush_every outside [-1024, 1024]");
    if (o->no_sync != 0 && o->no_sync != 1) return set_error(BSM_ERR_ARG, "opts.no_sync must be 0 or 1");
    for (int q = 0; q < 3; ++q)
        if (o->reserved[q] != 0) return set_error(BSM_ERR_ARG, "opts.reserved must be zero");
    return BSM_OK;
}

bool is_tc(int prec) {
    return prec == BSM_P_TF32x3 || prec == BSM_P_BF16x3 || prec == BSM_P_BF16x6 || prec == BSM_P_OZAKI;
}
// split paths whose lane variant multiplies unpacked FP32 pieces
bool needs_plain(int prec) { return is_tc(prec) && prec != BSM_P_OZAKI; }

// first global row / column of every block row / column, on the device
bsm_status ensure_starts(bsm_mat *M) {
    if (M->row_start && M->col_start) return BSM_OK;
    std::vector<int32_t> rs((size_t)M->nbr + 1), cs((size_t)M->nbc + 1);
    int64_t t = 0;
    for (int32_t i = 0; i < M->nbr; ++i) {
        rs[i] = (int32_t)t;
        t += M->h_row_bs[i];
        if (t > INT32_MAX) return set_error(BSM_ERR_UNSUPPORTED, "more than 2^31 - 1 rows");
    }
    rs[M->nbr] = (int32_t)t;
    t = 0;
    for (int32_t j = 0; j < M->nbc; ++j) {
        cs[j] = (int32_t)t;
        t += M->h_col_bs[j];
        if (t > INT32_MAX) return set_error(BSM_ERR_UNSUPPORTED, "more than 2^31 - 1 columns");
    }
    cs[M->nbc] = (int32_t)t;
    bsm_status st;
    int32_t *r = nullptr, *c = nullptr;
    if ((st = dalloc_t(&r, rs.size()))) return st;
    if ((st = dalloc_t(&c, cs.size()))) {
        dfree(r);
        return st;
    }
    // pageable sources: the calls return once the host data has been taken
    cudaError_t e = cudaMemcpyAsync(r, rs.data(), sizeof(int32_t) * rs.size(), cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, cs.data(), sizeof(int32_t) * cs.size(), cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    if (e != cudaSuccess) {
        dfree(r);
        dfree(c);
        return cuda_check(e, "copy block starts");
    }
    M->row_start = r;
    M->col_start = c;
    return BSM_OK;
}

// Ozaki path: per-line exponents of M in a role (X lines = logical rows, Y
// lines = logical columns; stored rows when role_y == trans)
struct OzLines {
    int32_t *line0 = nullptr, *exps = nullptr;
};
bsm_status oz_lines(Scratch &sc, const bsm_mat *M, int role_y, int trans, OzLines &ol) {
    const int by_rows = role_y == trans ? 1 : 0;
    int64_t nlines = 0;
    for (int32_t v : (by_rows ? M->h_row_bs : M->h_col_bs)) nlines += v;
    bsm_status st;
    if ((st = sc.get(&ol.line0, (size_t)M->nnzb)) || (st = sc.get(&ol.exps, (size_t)nlines))) return st;
    cudaError_t e = cudaMemsetAsync(ol.exps, 0, sizeof(int32_t) * (size_t)nlines, g_stream);
    if (e == cudaSuccess) e = launch_oz_lines(M, by_rows, ol.line0, ol.exps, g_stream);
    return cuda_check(e, "line exponents");
}

// packed fragment planes of one operand (tensor-core paths)
struct Packed {
    int64_t *off = nullptr;  // [nnzb+1] word offsets
    uint32_t *words = nullptr;
};

// Launch pack-size computation and its scan; the total lands in off[nnzb].
bsm_status pack_prepare(Scratch &sc, const bsm_mat *M, int role_y, int trans, int prec, Packed &pk) {
    int64_t *w = nullptr, *tmp = nullptr;
    bsm_status st;
    if ((st = sc.get(&w, (size_t)M->nnzb)) != BSM_OK) return st;
    if ((st = sc.get(&pk.off, (size_t)M->nnzb + 1)) != BSM_OK) return st;
    if ((st = sc.get(&tmp, scan_tmp_elems(M->nnzb))) != BSM_OK) return st;
    cudaError_t e = launch_pack_sizes(M, role_y, trans, prec, w, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(w, pk.off, M->nnzb, tmp, g_stream);
    return cuda_check(e, "pack sizes");
}

bsm_status pack_fill(Scratch &sc, const bsm_mat *M, int role_y, int trans, int prec, Packed &pk,
                     int64_t total_words, OzLines *ol = nullptr) {
    bsm_status st;
    if ((st = sc.get(&pk.words, (size_t)total_words + 16)) != BSM_OK) return st;
    if (prec == BSM_P_OZAKI && (st = oz_lines(sc, M, role_y, trans, *ol))) return st;
    return cuda_check(launch_pack(M, role_y, trans, prec, pk.off, pk.words, nullptr, g_stream,
                                  ol ? ol->line0 : nullptr, ol ? ol->exps : nullptr),
                      "pack");
}

// Rank of every block row of X in a breadth-first order through shared block
// columns: rows that have block columns in common come out close together (a
// Cuthill-McKee-style ordering of the rows of X.X^T).  Only the numeric
// kernels' schedule uses it, so that warps running at the same time read the
// same operand blocks from L2.  Built on the host from X's pattern and kept
// on the handle.
// X's pattern on the host: rows (rp, ci) and columns (cp, cr)
struct HostPattern {
    std::vector<int64_t> rp, cp;
    std::vector<int32_t> ci, cr;
};
bsm_status host_pattern(const bsm_mat *X, HostPattern &h) {
    const int32_t nbr = X->nbr, nbc = X->nbc;
    h.rp.assign((size_t)nbr + 1, 0);
    h.ci.assign((size_t)X->nnzb, 0);
    cudaError_t e = cudaMemcpyAsync(h.rp.data(), X->row_ptr, sizeof(int64_t) * (nbr + 1), cudaMemcpyDeviceToHost,
                                    g_stream);
    if (e == cudaSuccess && X->nnzb)
        e = cudaMemcpyAsync(h.ci.data(), X->col_idx, sizeof(int32_t) * X->nnzb, cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    bsm_status st;
    if ((st = cuda_check(e, "read pattern"))) return st;
    h.cp.assign((size_t)nbc + 1, 0);
    for (int32_t c : h.ci) h.cp[(size_t)c + 1]++;
    for (int32_t c = 0; c < nbc; ++c) h.cp[c + 1] += h.cp[c];
    h.cr.assign((size_t)X->nnzb, 0);
    std::vector<int64_t> pos(h.cp.begin(), h.cp.end() - 1);
    for (int32_t r = 0; r < nbr; ++r)
        for (int64_t b = h.rp[r]; b < h.rp[r + 1]; ++b) h.cr[pos[h.ci[b]]++] = r;
    return BSM_OK;
}

// breadth-first rank of the rows of a pattern through shared columns
std::vector<int32_t> bfs_row_rank(const HostPattern &h, int32_t nbr, int32_t nbc) {
    const std::vector<int64_t> &rp = h.rp, &cp = h.cp;
    const std::vector<int32_t> &ci = h.ci, &cr = h.cr;
    std::vector<int32_t> seed((size_t)nbr);
    for (int32_t r = 0; r < nbr; ++r) seed[r] = r;
    std::stable_sort(seed.begin(), seed.end(), [&](int32_t x, int32_t y) { return rp[x + 1] - rp[x] < rp[y + 1] - rp[y]; });
    std::vector<char> vrow((size_t)nbr, 0), vcol((size_t)nbc, 0);
    std::vector<int32_t> rank((size_t)nbr), queue;
    queue.reserve(nbr);
    int32_t next = 0;
    for (int32_t s0 : seed) {
        if (vrow[s0]) continue;
        vrow[s0] = 1;
        size_t head = queue.size();
        queue.push_back(s0);
        while (head < queue.size()) {
            const int32_t r = queue[head++];
            rank[r] = next++;
            for (int64_t b = rp[r]; b < rp[r + 1]; ++b) {
                const int32_t c = ci[b];
                if (vcol[c]) continue;
                vcol[c] = 1;
                for (int64_t q = cp[c]; q < cp[c + 1]; ++q)
                    if (!vrow[cr[q]]) {
                        vrow[cr[q]] = 1;
                        queue.push_back(cr[q]);
                    }
            }
        }
    }
    return rank;
}

// breadth-first rank of the block columns of X through shared block rows
bsm_status ensure_col_rank(bsm_mat *X) {
    if (X->col_rank) return BSM_OK;
    HostPattern h;
    bsm_status st;
    if ((st = host_pattern(X, h))) return st;
    HostPattern t;  // the transposed pattern: columns become rows
    t.rp = h.cp; t.ci = h.cr; t.cp = h.rp; t.cr = h.ci;
    std::vector<int32_t> rank = bfs_row_rank(t, X->nbc, X->nbr);
    int32_t *d = nullptr;
    if ((st = dalloc_t(&d, X->nbc))) return st;
    cudaError_t e = cudaMemcpyAsync(d, rank.data(), sizeof(int32_t) * X->nbc, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    if ((st = cuda_check(e, "upload column order"))) {
        dfree(d);
        return st;
    }
    X->col_rank = d;
    return BSM_OK;
}

bsm_status ensure_row_rank(bsm_mat *X) {
    if (X->row_rank || X->nbr == 0) return BSM_OK;
    const int32_t nbr = X->nbr;
    HostPattern h;
    bsm_status st;
    if ((st = host_pattern(X, h))) return st;
    std::vector<int32_t> rank = bfs_row_rank(h, nbr, X->nbc);
    cudaError_t e;
    int32_t *d = nullptr;
    if ((st = dalloc_t(&d, nbr))) return st;
    e = cudaMemcpyAsync(d, rank.data(), sizeof(int32_t) * nbr, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    if ((st = cuda_check(e, "upload row order"))) {
        dfree(d);
        return st;
    }
    X->row_rank = d;
    return BSM_OK;
}

// Processing order of n output blocks for the numeric kernels: grouped by
// block shape, larger blocks first, so that neighbouring warps run the same
// code path and the heaviest items start early.
bsm_status shape_order(Scratch &sc, int64_t n, const int32_t *blk_rc, const std::vector<int32_t> &rsz,
                       const std::vector<int32_t> &csz, int32_t **order, const bsm_mat *rows_of = nullptr,
                       const int32_t *row_rank = nullptr, int prec = -1, bool *uses_cores = nullptr,
                       int64_t **n_marked = nullptr, const int32_t *blk_col = nullptr,
                       const int32_t *col_rank = nullptr, int32_t ncols = 0, int32_t tile = 0,
                       int64_t **groups = nullptr) {
    if (uses_cores) *uses_cores = false;
    *order = nullptr;
    if (n_marked) *n_marked = nullptr;
    if (groups) *groups = nullptr;
    if (n <= 1) return BSM_OK;
    std::vector<int32_t> sizes(rsz);
    sizes.insert(sizes.end(), csz.begin(), csz.end());
    std::sort(sizes.begin(), sizes.end());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    const int32_t ns = (int32_t)sizes.size();
    if ((int64_t)ns * ns > (1 << 16)) return BSM_OK;  // too many shapes: natural order
    std::vector<int32_t> sidx(kMaxBlockDim + 1, 0), table((size_t)ns * ns);
    for (int32_t q = 0; q < ns; ++q) sidx[sizes[q]] = q;
    // with groups, the blocks a smaller kernel instance takes come after the
    // others: split paths, one tile row (at most 16 rows); Ozaki path, one tile
    // column (at most 8 columns)
    const bool split = prec == BSM_P_TF32x3 || prec == BSM_P_BF16x3 || prec == BSM_P_BF16x6;
    const bool grouped = groups && (split || prec == BSM_P_OZAKI);
    auto group_of = [&](int32_t m, int32_t nn) -> int64_t {
        if (!grouped) return 0;
        return (split ? m <= 16 : nn <= 8) ? 1 : 0;
    };
    std::vector<std::pair<int64_t, int32_t>> cls;
    for (int32_t r = 0; r < ns; ++r)
        for (int32_t c = 0; c < ns; ++c)
            cls.emplace_back(group_of(sizes[r], sizes[c]) * (int64_t(1) << 40) - (int64_t)sizes[r] * sizes[c],
                             r * ns + c);
    std::sort(cls.begin(), cls.end());
    // per-class variant; second-variant classes sort after all others
    std::vector<int8_t> var((size_t)ns * ns, 0);
    bool any_var = false;
    if (prec >= 0) {
        for (int32_t r = 0; r < ns; ++r)
            for (int32_t c = 0; c < ns; ++c) {
                var[(size_t)r * ns + c] = (int8_t)variant_of(prec, sizes[r], sizes[c]);
                any_var = any_var || var[(size_t)r * ns + c];
            }
    }
    for (size_t q = 0; q < cls.size(); ++q)
        table[cls[q].second] = (int32_t)q + (var[cls[q].second] ? (int32_t)cls.size() : 0);
    const int32_t nbr = rows_of ? rows_of->nbr : 0;
    if (row_rank && 2 * (int64_t)table.size() * std::max(nbr, 1) >= (int64_t(1) << 31)) row_rank = nullptr;
    // 2-D schedule tiles when asked for and the keys fit in 31 bits
    const bool tiled = row_rank && blk_col && col_rank && tile > 0;
    const int64_t nrt = tiled ? (nbr + tile - 1) / tile : 0, nct = tiled ? (ncols + tile - 1) / tile : 0;
    const bool use_tiles = tiled && 2 * (int64_t)table.size() * nrt * nct < (int64_t(1) << 31);
    int bits = 1;
    while ((1ll << bits) < 2 * (int64_t)table.size() * (use_tiles ? nrt * nct : (row_rank ? nbr : 1))) ++bits;
    bsm_status st;
    int32_t *d_sidx, *d_table, *iota, *vals_alt, *out, *brow = nullptr;
    uint32_t *keys, *keys_alt, *keys_sorted;
    int64_t *rtmp;
    if ((st = sc.get(&d_sidx, sidx.size())) || (st = sc.get(&d_table, table.size())) || (st = sc.get(&iota, n)) ||
        (st = sc.get(&vals_alt, n)) || (st = sc.get(&out, n)) || (st = sc.get(&keys, n)) ||
        (st = sc.get(&keys_alt, n)) || (st = sc.get(&keys_sorted, n)) || (st = sc.get(&rtmp, radix_tmp_elems(n))))
        return st;
    if (row_rank && (st = sc.get(&brow, n))) return st;
    cudaError_t e = cudaMemcpyAsync(d_sidx, sidx.data(), sizeof(int32_t) * sidx.size(), cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_table, table.data(), sizeof(int32_t) * table.size(), cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess && row_rank) {
        bsm_mat view;  // rows of the output blocks
        view.nbr = rows_of->nbr; view.nnzb = n; view.row_ptr = rows_of->row_ptr;
        e = launch_blk_rows(&view, brow, g_stream);
    }
    if (e == cudaSuccess)
        e = launch_class_keys(n, blk_rc, d_sidx, ns, d_table, brow, row_rank, nbr, use_tiles ? blk_col : nullptr,
                              use_tiles ? col_rank : nullptr, use_tiles ? tile : 0, (int32_t)nct, keys, iota, g_stream);
    if (e == cudaSuccess)
        e = launch_radix_sort_pairs(keys, iota, keys_alt, vals_alt, keys_sorted, out, n, bits, rtmp, g_stream);
    if ((st = cuda_check(e, "shape order"))) return st;
    if (grouped) {
        // positions in the sorted order where group 1 and the lane items start
        const int64_t mult = use_tiles ? nrt * nct : (row_rank ? std::max(nbr, 1) : 1);
        const int32_t ncls = (int32_t)cls.size();
        int32_t q1 = 0;
        while (q1 < ncls && group_of(sizes[cls[q1].second / ns], sizes[cls[q1].second % ns]) == 0) ++q1;
        int64_t *gb;
        if ((st = sc.get(&gb, 2))) return st;
        if ((st = cuda_check(launch_group_bounds(keys_sorted, n, (uint32_t)(q1 * mult), (uint32_t)(ncls * mult), gb,
                                                 g_stream),
                             "tile-row groups")))
            return st;
        *groups = gb;
    }
    if (any_var) {
        int8_t *d_var;
        int64_t *cnt;
        if ((st = sc.get(&d_var, var.size())) || (st = sc.get(&cnt, 1))) return st;
        e = cudaMemcpyAsync(d_var, var.data(), var.size(), cudaMemcpyHostToDevice, g_stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int64_t), g_stream);
        if (e == cudaSuccess)
            e = launch_mark_variant(n, out, blk_rc, d_sidx, ns, d_var, reinterpret_cast<unsigned long long *>(cnt),
                                    g_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);  // var is pageable and local
        if ((st = cuda_check(e, "variant marks"))) return st;
        if (uses_cores) *uses_cores = true;
        if (n_marked) *n_marked = cnt;
    }
    *order = out;
    return BSM_OK;
}

// Column-major copy of X's pattern (kept on the handle until its pattern
// changes): t_ptr[nbc+1], and for every block in column order (ascending
// block row inside a column) its block row t_row and block index t_blk.
bsm_status ensure_transpose(bsm_mat *X) {
    if (X->t_ptr) return BSM_OK;
    Scratch sc;
    bsm_status st;
    const int64_t n = X->nnzb;
    int32_t *rows, *iota, *vals_alt;
    uint32_t *keys, *keys_alt, *keys_sorted;
    int64_t *rtmp, *counts, *stmp, *tptr;
    int32_t *trow, *tblk;
    if ((st = sc.get(&rows, n)) || (st = sc.get(&iota, n)) || (st = sc.get(&vals_alt, n)) || (st = sc.get(&keys, n)) ||
        (st = sc.get(&keys_alt, n)) || (st = sc.get(&keys_sorted, n)) || (st = sc.get(&rtmp, radix_tmp_elems(n))) ||
        (st = sc.get(&counts, X->nbc)) || (st = sc.get(&stmp, scan_tmp_elems(X->nbc))) ||
        (st = sc.get(&tptr, (size_t)X->nbc + 1)) || (st = sc.get(&trow, n)) || (st = sc.get(&tblk, n)))
        return st;
    int bits = 1;
    while ((1ll << bits) < (int64_t)X->nbc) ++bits;
    cudaError_t e = launch_blk_rows(X, rows, g_stream);
    if (e == cudaSuccess) e = launch_iota_keys(n, X->col_idx, keys, iota, g_stream);
    if (e == cudaSuccess)
        e = launch_radix_sort_pairs(keys, iota, keys_alt, vals_alt, keys_sorted, tblk, n, bits, rtmp, g_stream);
    if (e == cudaSuccess) e = launch_gather_i32(n, tblk, rows, trow, g_stream);
    if (e == cudaSuccess) e = launch_histogram_u32(n, keys, X->nbc, counts, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(counts, tptr, X->nbc, stmp, g_stream);
    if ((st = cuda_check(e, "transpose pattern"))) return st;
    X->t_ptr = tptr;
    X->t_row = trow;
    X->t_blk = tblk;
    sc.release(tptr);
    sc.release(trow);
    sc.release(tblk);
    return BSM_OK;
}

bsm_status read_words(const int64_t *const *src, int n) {
    for (int q = 0; q < n; ++q) {
        cudaError_t e = cudaMemcpyAsync(g_host + q, src[q], sizeof(int64_t), cudaMemcpyDeviceToHost, g_stream);
        if (e != cudaSuccess) return cuda_check(e, "reading sizes");
    }
    return cuda_check(cudaStreamSynchronize(g_stream), "stream synchronize");
}

// ---------------------------------------------------------------------------
// Row-panel engine (BSM_P_TF32x3_PANEL)

// the blocking of A, B (and so of C) is one size s <= the panel slot
bool panel_blocking(const bsm_mat *A, const bsm_mat *B, int32_t *s_out) {
    if (A->nbr == 0 || A->nbc == 0 || B->nbc == 0) return false;
    if (A->nnzb > INT32_MAX || B->nnzb > INT32_MAX) return false;
    const int32_t s = A->h_row_bs[0];
    if (s > panel_slot()) return false;
    for (const auto *v : {&A->h_row_bs, &A->h_col_bs, &B->h_col_bs})
        for (int32_t x : *v)
            if (x != s) return false;
    *s_out = s;
    return true;
}

// Positions of A's block rows and B's block columns along the band of the
// product: rows start at their breadth-first rank; a block index k of the
// inner dimension sits at the mean position of A's rows that hold it; a row
// is then placed at the mean position of its k, and a column of B at the
// mean position of its k.  Rows (columns) sorted by position form the
// groups of 5 of the tiles, so that a group's members share most of their k.
bsm_status panel_orders(bsm_mat *A, bsm_mat *B) {
    if (A->panel_ord_r && A->panel_B == B && A->panel_B_nnzb == B->nnzb && A->panel_B_nbc == B->nbc)
        return BSM_OK;
    dfree(A->panel_ord_r); A->panel_ord_r = nullptr;
    dfree(A->panel_ord_c); A->panel_ord_c = nullptr;
    dfree(A->panel_pos_c); A->panel_pos_c = nullptr;
    const int32_t nbr = A->nbr, nbk = A->nbc, nbc = B->nbc;
    HostPattern ha, hb;
    bsm_status st;
    if ((st = host_pattern(A, ha)) || (st = host_pattern(B, hb))) return st;
    const std::vector<int32_t> rank = bfs_row_rank(ha, nbr, nbk);
    std::vector<double> y((size_t)nbk, -1.0), x((size_t)nbr), z((size_t)nbc);
    for (int32_t k = 0; k < nbk; ++k) {
        const int64_t n = ha.cp[k + 1] - ha.cp[k];
        if (!n) continue;
        double acc = 0.0;
        for (int64_t q = ha.cp[k]; q < ha.cp[k + 1]; ++q) acc += rank[ha.cr[q]];
        y[k] = acc / (double)n;
    }
    for (int32_t i = 0; i < nbr; ++i) {
        double acc = 0.0;
        int64_t n = 0;
        for (int64_t b = ha.rp[i]; b < ha.rp[i + 1]; ++b) {
            acc += y[ha.ci[b]];
            ++n;
        }
        x[i] = n ? acc / (double)n : (double)rank[i];
    }
    for (int32_t j = 0; j < nbc; ++j) {
        double acc = 0.0;
        int64_t n = 0;
        for (int64_t q = hb.cp[j]; q < hb.cp[j + 1]; ++q) {
            const double v = y[hb.cr[q]];
            if (v < 0.0) continue;
            acc += v;
            ++n;
        }
        z[j] = n ? acc / (double)n : (double)nbr + j;
    }
    std::vector<int32_t> ord_r((size_t)nbr), ord_c((size_t)nbc), pos_c((size_t)nbc);
    for (int32_t i = 0; i < nbr; ++i) ord_r[i] = i;
    for (int32_t j = 0; j < nbc; ++j) ord_c[j] = j;
    std::stable_sort(ord_r.begin(), ord_r.end(), [&](int32_t p, int32_t q) { return x[p] < x[q]; });
    std::stable_sort(ord_c.begin(), ord_c.end(), [&](int32_t p, int32_t q) { return z[p] < z[q]; });
    for (int32_t p = 0; p < nbc; ++p) pos_c[ord_c[p]] = p;
    int32_t *dr = nullptr, *dc = nullptr, *dp = nullptr;
    if ((st = dalloc_t(&dr, nbr)) || (st = dalloc_t(&dc, nbc)) || (st = dalloc_t(&dp, nbc))) {
        dfree(dr);
        dfree(dc);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(dr, ord_r.data(), sizeof(int32_t) * nbr, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, ord_c.data(), sizeof(int32_t) * nbc, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, pos_c.data(), sizeof(int32_t) * nbc, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);  // the host vectors are pageable
    if ((st = cuda_check(e, "upload panel orders"))) {
        dfree(dr);
        dfree(dc);
        dfree(dp);
        return st;
    }
    A->panel_ord_r = dr;
    A->panel_ord_c = dc;
    A->panel_pos_c = dp;
    A->panel_B = B;
    A->panel_B_nnzb = B->nnzb;
    A->panel_B_nbc = nbc;
    return BSM_OK;
}

// super tiles of the panel schedule (row groups x column groups)
int g_panel_sg = 12, g_panel_sh = 12;

struct PanelOut {
    int64_t nnzbC;
    const int64_t *c_row_ptr;
    const int32_t *c_col;
    const int64_t *c_off;
    double *c_data;
    const int64_t *old_off;  // null unless beta != 0
    const void *old_data;
    double alpha, beta;
    int32_t *status;
};

bsm_status run_panel(Scratch &sc, bsm_mat *A, bsm_mat *B, int32_t s, const PanelOut &o, Events &ev, int tune_prec) {
    bsm_status st;
    if ((st = panel_orders(A, B)) || (st = ensure_transpose(B))) return st;
    const int32_t nbr = A->nbr, nbc = B->nbc;
    const int32_t ngr = (nbr + panel_tile_rows() - 1) / panel_tile_rows();
    const int32_t ngc = (nbc + panel_tile_cols() - 1) / panel_tile_cols();
    int64_t *tile_cnt, *tile_ptr, *stmp;
    if ((st = sc.get(&tile_cnt, ngr)) || (st = sc.get(&tile_ptr, (size_t)ngr + 1)) ||
        (st = sc.get(&stmp, scan_tmp_elems(ngr))))
        return st;
    cudaError_t e = launch_panel_tiles_count(nbr, A->panel_ord_r, A->panel_pos_c, o.c_row_ptr, o.c_col, ngc, tile_cnt,
                                             g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(tile_cnt, tile_ptr, ngr, stmp, g_stream);
    if ((st = cuda_check(e, "panel tiles"))) return st;
    const int64_t *src[1] = {tile_ptr + ngr};
    if ((st = read_words(src, 1))) return st;
    const int64_t ntiles = g_host[0];
    if (ntiles == 0) return BSM_OK;
    if (ntiles > INT32_MAX / 25) return set_error(BSM_ERR_UNSUPPORTED, "too many panel tiles");
    const int nt = panel_tile_rows() * panel_tile_cols();
    int32_t *tile_g, *tile_h, *cblk, *iota, *vals_alt, *order;
    uint32_t *keys, *keys_alt, *keys_sorted;
    int64_t *rtmp;
    if ((st = sc.get(&tile_g, ntiles)) || (st = sc.get(&tile_h, ntiles)) || (st = sc.get(&cblk, (size_t)ntiles * nt)) ||
        (st = sc.get(&iota, ntiles)) || (st = sc.get(&vals_alt, ntiles)) || (st = sc.get(&order, ntiles)) ||
        (st = sc.get(&keys, ntiles)) || (st = sc.get(&keys_alt, ntiles)) || (st = sc.get(&keys_sorted, ntiles)) ||
        (st = sc.get(&rtmp, radix_tmp_elems(ntiles))))
        return st;
    e = cudaMemsetAsync(cblk, 0xFF, sizeof(int32_t) * (size_t)ntiles * nt, g_stream);
    if (e == cudaSuccess)
        e = launch_panel_tiles_fill(nbr, A->panel_ord_r, A->panel_pos_c, o.c_row_ptr, o.c_col, ngc, tile_ptr, tile_g,
                                    tile_h, cblk, g_stream);
    const int sg = g_panel_sg, sh = g_panel_sh;
    const int64_t nkeys = (int64_t)((ngr + sg - 1) / sg) * ((ngc + sh - 1) / sh);
    int bits = 1;
    while ((1ll << bits) < nkeys) ++bits;
    if (e == cudaSuccess) e = launch_panel_tile_keys(ntiles, tile_g, tile_h, sg, sh, ngc, keys, iota, g_stream);
    if (e == cudaSuccess)
        e = launch_radix_sort_pairs(keys, iota, keys_alt, vals_alt, keys_sorted, order, ntiles, bits, rtmp, g_stream);
    if ((st = cuda_check(e, "panel tiles"))) return st;
    PanelArgs pa{};
    pa.nbr = nbr; pa.nbc = nbc; pa.s = s; pa.nbk = A->nbc;
    pa.n_tiles = ntiles;
    pa.tile_order = order; pa.tile_g = tile_g; pa.tile_h = tile_h; pa.cblk = cblk;
    pa.ord_r = A->panel_ord_r; pa.ord_c = A->panel_ord_c;
    pa.a_row_ptr = A->row_ptr; pa.a_col_idx = A->col_idx;
    pa.b_t_ptr = B->t_ptr; pa.b_t_row = B->t_row; pa.b_t_blk = B->t_blk;
    // the k-steps of every tile (a merge of its 10 block-index lists)
    int64_t *step_cnt, *step_ptr, *stmp2;
    if ((st = sc.get(&step_cnt, ntiles)) || (st = sc.get(&step_ptr, (size_t)ntiles + 1)) ||
        (st = sc.get(&stmp2, scan_tmp_elems(ntiles))))
        return st;
    e = launch_panel_steps(pa, 0, step_cnt, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(step_cnt, step_ptr, ntiles, stmp2, g_stream);
    if ((st = cuda_check(e, "panel steps"))) return st;
    const int64_t *ssrc[1] = {step_ptr + ntiles};
    if ((st = read_words(ssrc, 1))) return st;
    const int64_t nsteps = g_host[0];
    int32_t *steps;
    if ((st = sc.get(&steps, (size_t)nsteps * 2 * panel_tile_rows()))) return st;
    pa.step_ptr = step_ptr;
    pa.steps = steps;
    if ((st = cuda_check(launch_panel_steps(pa, 1, nullptr, g_stream), "panel steps"))) return st;
    // operand planes
    uint8_t *apk, *bpk, *zeros;
    unsigned long long *counter;
    if ((st = sc.get(&apk, (size_t)panel_pack_bytes(A->nnzb))) || (st = sc.get(&bpk, (size_t)panel_pack_bytes(B->nnzb))) ||
        (st = sc.get(&zeros, (size_t)panel_pack_bytes(1))) || (st = sc.get(&counter, 1)))
        return st;
    e = launch_panel_pack(A, 0, apk, g_stream);
    if (e == cudaSuccess) e = launch_panel_pack(B, 1, bpk, g_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(zeros, 0, (size_t)panel_pack_bytes(1), g_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), g_stream);
    if ((st = cuda_check(e, "panel operands"))) return st;
    pa.a_pack = apk; pa.b_pack = bpk; pa.zeros = zeros;
    pa.c_data = o.c_data; pa.c_blk_off = o.c_off;
    pa.alpha = o.alpha; pa.beta = o.beta;
    pa.old_data = o.old_data; pa.old_off = o.old_off;
    pa.status = o.status;
    pa.work_counter = counter;
    pa.wait_ns = panel_wait_ns();
    pa.pair = tune_of(tune_prec)[BSM_TUNE_PANEL_STEPS] > 0 ? tune_of(tune_prec)[BSM_TUNE_PANEL_STEPS] : panel_pair();
    ev.mark(5);
    if ((st = cuda_check(launch_panel_numeric(pa, g_stream), "panel numeric"))) return st;
    ev.mark(6);
    return BSM_OK;
}

}  // namespace

cudaStream_t stream() { return g_stream; }
unsigned long long panel_wait_ns() { return g_wait_ns.load(std::memory_order_relaxed); }
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
bool profiling() { return g_prof; }

bsm_status set_error(bsm_status st, const std::string &msg) {
    t_err = msg;
    return st;
}

bsm_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BSM_OK;
    return set_error(e == cudaErrorMemoryAllocation ? BSM_ERR_ALLOC : BSM_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

// Device memory provider: the built-in stream-ordered pool (cudaMallocAsync /
// cudaFreeAsync on the library stream) unless bsm_set_allocator installed
// hooks.  Every block obtained from hooks is remembered with its size and the
// hooks that made it, so it goes back to them even if the provider changes.
namespace {
struct Provider {
    bsm_alloc_fn alloc = nullptr;
    bsm_free_fn free = nullptr;
    void *ctx = nullptr;
};
struct HookBlock {
    size_t bytes;
    Provider prov;
};
std::mutex g_alloc_mu;
Provider g_provider;
std::unordered_map<void *, HookBlock> g_hook_blocks;
}  // namespace

bsm_status dalloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    Provider prov;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        prov = g_provider;
    }
    if (prov.alloc) {
        void *q = prov.alloc(bytes, static_cast<void *>(g_stream), prov.ctx);
        if (!q)
            return set_error(BSM_ERR_ALLOC, std::string("the installed allocator returned NULL for ") +
                                                std::to_string(bytes) + " bytes");
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        g_hook_blocks[q] = HookBlock{bytes, prov};
        *p = q;
        return BSM_OK;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, g_stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(BSM_ERR_ALLOC, std::string("device allocation of ") + std::to_string(bytes) +
                                            " bytes failed: " + cudaGetErrorString(e));
    }
    return BSM_OK;
}

void dfree(void *p) {
    if (!p) return;
    HookBlock hb{};
    bool hooked = false;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_hook_blocks.find(p);
        if (it != g_hook_blocks.end()) {
            hb = it->second;
            hooked = true;
            g_hook_blocks.erase(it);
        }
    }
    if (hooked) hb.prov.free(p, hb.bytes, static_cast<void *>(g_stream), hb.prov.ctx);
    else cudaFreeAsync(p, g_stream);
}

int64_t hook_blocks_outstanding() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return (int64_t)g_hook_blocks.size();
}

// --------------------------------------------------------------------------
// Drop blocks with norm <= eps from X, compacting.  Eager: sizes read back,
// new storage allocated and swapped in.  No-sync: the surviving blocks are
// written into X's present storage, whose sizes (nnz_out, len_out) must be
// what the filter leaves; the device checks that and flags `status`.
// The provenance arrays of an add are compacted alongside.
// --------------------------------------------------------------------------
bsm_status filter_compact(bsm_mat *X, double eps, bool no_sync, int32_t *status, int64_t nnz_out, int64_t len_out,
                          bsm_mat *dst) {
    Scratch sc;
    bsm_status st;
    const int64_t nb = X->nnzb;
    double *nrm = nullptr;
    int64_t *keep = nullptr, *kscan = nullptr, *tmp = nullptr, *rcnt = nullptr, *relem = nullptr,
            *nrow = nullptr, *nelem = nullptr;
    if ((st = sc.get(&nrm, nb)) || (st = sc.get(&keep, nb)) || (st = sc.get(&kscan, nb + 1)) ||
        (st = sc.get(&tmp, scan_tmp_elems(std::max<int64_t>(nb, X->nbr)))) || (st = sc.get(&rcnt, X->nbr)) ||
        (st = sc.get(&relem, X->nbr)) || (st = sc.get(&nrow, X->nbr + 1)) || (st = sc.get(&nelem, X->nbr + 1)))
        return st;
    cudaError_t e = launch_block_norms(X, nrm, g_stream);
    if (e == cudaSuccess) e = launch_keep_flags(nb, nrm, eps, keep, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(keep, kscan, nb, tmp, g_stream);
    if (e == cudaSuccess) e = launch_row_keep_counts(X->nbr, X->row_ptr, keep, X->blk_rc, rcnt, relem, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(rcnt, nrow, X->nbr, tmp, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(relem, nelem, X->nbr, tmp, g_stream);
    if ((st = cuda_check(e, "norm filter"))) return st;
    int64_t nnz2, len2;
    if (no_sync) {
        PlanCheck pc{};
        pc.actual[0] = nrow + X->nbr; pc.expected[0] = nnz_out;
        pc.actual[1] = nelem + X->nbr; pc.expected[1] = len_out;
        pc.n = 2;
        if ((st = cuda_check(launch_check_plan(pc, status, g_stream), "plan check"))) return st;
        nnz2 = nnz_out;
        len2 = len_out;
    } else {
        const int64_t *src[2] = {nrow + X->nbr, nelem + X->nbr};
        if ((st = read_words(src, 2))) return st;
        nnz2 = g_host[0];
        len2 = g_host[1];
    }
    // destination arrays
    int32_t *ncol, *nrc;
    int64_t *noff, *nxs = nullptr, *nys = nullptr, *nrowp;
    void *ndata;
    if (no_sync) {
        ncol = dst->col_idx; nrc = dst->blk_rc; noff = dst->blk_off; ndata = dst->data; nrowp = dst->row_ptr;
        nxs = dst->add_xsrc; nys = dst->add_ysrc;
    } else {
        if ((st = sc.get(&ncol, nnz2)) || (st = sc.get(&noff, nnz2)) || (st = sc.get(&nrc, nnz2))) return st;
        if ((st = dalloc(&ndata, (size_t)len2 * esize(X->dtype)))) return st;
        sc.ptrs.push_back(ndata);
        nrowp = nrow;
        if (X->add_xsrc && ((st = sc.get(&nxs, nnz2)) || (st = sc.get(&nys, nnz2)))) return st;
    }
    CompactArgs c{X->nbr, X->row_ptr, X->col_idx, X->blk_off, X->blk_rc, kscan, nrow, nelem,
                  X->data, X->dtype, ncol, noff, nrc, ndata, no_sync ? status : nullptr};
    e = launch_compact(c, g_stream);
    if (e == cudaSuccess && X->add_xsrc) {
        e = launch_compact_i64(nb, kscan, X->add_xsrc, nxs, no_sync ? status : nullptr, g_stream);
        if (e == cudaSuccess) e = launch_compact_i64(nb, kscan, X->add_ysrc, nys, no_sync ? status : nullptr, g_stream);
    }
    if (no_sync && e == cudaSuccess) e = launch_copy_i64_if_ok(X->nbr + 1, nrow, nrowp, status, g_stream);
    if ((st = cuda_check(e, "compact"))) return st;
    if (no_sync) return BSM_OK;
    // eager: swap the compacted storage into X
    dfree(X->row_ptr); dfree(X->col_idx); dfree(X->blk_off); dfree(X->blk_rc);
    if (X->own_data) dfree(X->data);
    dfree(X->norms);
    X->norms = nullptr;
    X->norms_valid = false;
    X->row_ptr = nrow; X->col_idx = ncol; X->blk_off = noff; X->blk_rc = nrc; X->data = ndata;
    X->own_data = true;
    X->nnzb = nnz2; X->data_len = len2;
    for (void *p : {(void *)nrow, (void *)ncol, (void *)noff, (void *)nrc, ndata}) sc.release(p);
    if (X->add_xsrc) {
        dfree(X->add_xsrc);
        dfree(X->add_ysrc);
        X->add_xsrc = nxs;
        X->add_ysrc = nys;
        sc.release(nxs);
        sc.release(nys);
    }
    return BSM_OK;
}

// status word of a handle, allocated on its first use
bsm_status ensure_status(bsm_mat *X) {
    if (X->status) return BSM_OK;
    return dalloc_t(&X->status, 1);
}

}  // namespace bsm

using namespace bsm;

// ==========================================================================
// ABI
// ==========================================================================
extern "C" {

const char *bsm_last_error(void) { return t_err.c_str(); }

bsm_status bsm_set_stream(void *s) {
    g_stream = static_cast<cudaStream_t>(s);
    return BSM_OK;
}

bsm_status bsm_get_launch_count(int64_t *count) {
    if (!count) return set_error(BSM_ERR_ARG, "count is NULL");
    *count = launch_count();
    return BSM_OK;
}

bsm_status bsm_set_allocator(bsm_alloc_fn alloc, bsm_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return set_error(BSM_ERR_ARG, "bsm_set_allocator needs both hooks or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_provider = Provider{alloc, free_fn, alloc ? ctx : nullptr};
    return BSM_OK;
}

bsm_status bsm_set_wait_limit(double seconds) {
    if (!(seconds >= 0.0 && seconds <= 2.0)) return set_error(BSM_ERR_ARG, "wait limit outside [0, 2] seconds");
    g_wait_ns.store((unsigned long long)(seconds * 1e9), std::memory_order_relaxed);
    return BSM_OK;
}

bsm_status bsm_set_product_limit(int64_t max_products) {
    if (max_products < 1 || max_products > INT32_MAX)
        return set_error(BSM_ERR_ARG, "product limit outside [1, 2^31-1]");
    g_product_limit.store(max_products, std::memory_order_relaxed);
    return BSM_OK;
}

bsm_status bsm_get_allocator_stats(int64_t *outstanding) {
    if (!outstanding) return set_error(BSM_ERR_ARG, "outstanding is NULL");
    *outstanding = hook_blocks_outstanding();
    return BSM_OK;
}

bsm_status bsm_set_profiling(int32_t on) {
    g_prof = on != 0;
    return BSM_OK;
}

bsm_status bsm_opts_default(bsm_opts *o) {
    if (!o) return set_error(BSM_ERR_ARG, "opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->prec = BSM_P_FP64;
    o->post_filter = 0;
    o->build_stacks = 1;
    o->flush_every = 0;
    return BSM_OK;
}

static bsm_status create_common(bsm_t *out, int32_t nbr, int32_t nbc, const int32_t *row_bs,
                                const int32_t *col_bs, int32_t dtype, bsm_mat **made) {
    if (!out) return set_error(BSM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nbr < 0 || nbc < 0) return set_error(BSM_ERR_ARG, "negative block count");
    if ((nbr > 0 && !row_bs) || (nbc > 0 && !col_bs)) return set_error(BSM_ERR_ARG, "block sizes are NULL");
    if (dtype != BSM_FP64 && dtype != BSM_FP32) return set_error(BSM_ERR_ARG, "dtype must be BSM_FP64 or BSM_FP32");
    for (int32_t i = 0; i < nbr; ++i)
        if (row_bs[i] < 1 || row_bs[i] > kMaxBlockDim) return set_error(BSM_ERR_ARG, "row block size outside [1, 256]");
    for (int32_t j = 0; j < nbc; ++j)
        if (col_bs[j] < 1 || col_bs[j] > kMaxBlockDim) return set_error(BSM_ERR_ARG, "column block size outside [1, 256]");
    bsm_status st = ensure_globals();
    if (st) return st;
    bsm_mat *X = new bsm_mat();
    X->nbr = nbr;
    X->nbc = nbc;
    X->dtype = dtype;
    X->h_row_bs.assign(row_bs, row_bs + nbr);
    X->h_col_bs.assign(col_bs, col_bs + nbc);
    for (int32_t v : X->h_row_bs) X->max_bs_row = std::max(X->max_bs_row, v);
    for (int32_t v : X->h_col_bs) X->max_bs_col = std::max(X->max_bs_col, v);
    if ((st = dalloc_t(&X->row_bs, nbr)) || (st = dalloc_t(&X->col_bs, nbc))) {
        dfree(X->row_bs);
        dfree(X->col_bs);
        delete X;
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(X->row_bs, row_bs, sizeof(int32_t) * nbr, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(X->col_bs, col_bs, sizeof(int32_t) * nbc, cudaMemcpyHostToDevice, g_stream);
    if (e != cudaSuccess) {
        dfree(X->row_bs); dfree(X->col_bs);
        delete X;
        return cuda_check(e, "copy block sizes");
    }
    *made = X;
    return BSM_OK;
}

bsm_status bsm_create(bsm_t *out, int32_t nbr, int32_t nbc, const int32_t *row_bs, const int32_t *col_bs,
                      const int64_t *row_ptr, const int32_t *col_idx, const int64_t *blk_off, int32_t dtype,
                      const void *data, int64_t data_len, int32_t data_mode) {
    if (!row_ptr) return set_error(BSM_ERR_ARG, "row_ptr is NULL");
    if (data_mode != BSM_DATA_COPY && data_mode != BSM_DATA_BORROW) return set_error(BSM_ERR_ARG, "bad data_mode");
    if (row_ptr[0] != 0) return set_error(BSM_ERR_ARG, "row_ptr[0] != 0");
    for (int32_t i = 0; i < nbr; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return set_error(BSM_ERR_ARG, "row_ptr decreases");
    const int64_t nnzb = nbr > 0 ? row_ptr[nbr] : 0;
    if (nnzb > INT32_MAX) return set_error(BSM_ERR_UNSUPPORTED, "more than 2^31-1 blocks");
    if (nnzb > 0 && (!col_idx || !blk_off || !data)) return set_error(BSM_ERR_ARG, "col_idx/blk_off/data NULL");
    if (data_len < 0) return set_error(BSM_ERR_ARG, "data_len < 0");
    // pattern checks (host, before any launch)
    if (nbr > 0 && !row_bs) return set_error(BSM_ERR_ARG, "row_bs is NULL");
    if (nbc > 0 && !col_bs) return set_error(BSM_ERR_ARG, "col_bs is NULL");
    // one pass; blocks laid out in CSR order with increasing offsets (the
    // usual layout) are proven disjoint on the way, anything else is sorted
    bool in_order = true;
    int64_t prev_end = 0;
    for (int32_t i = 0; i < nbr; ++i) {
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
            const int32_t j = col_idx[b];
            if (j < 0 || j >= nbc) return set_error(BSM_ERR_ARG, "col_idx out of range");
            if (b > row_ptr[i] && col_idx[b - 1] >= j) return set_error(BSM_ERR_ARG, "col_idx not strictly ascending in a row");
            if (row_bs[i] < 1 || row_bs[i] > kMaxBlockDim || col_bs[j] < 1 || col_bs[j] > kMaxBlockDim)
                return set_error(BSM_ERR_ARG, "block size outside [1, 256]");
            const int64_t len = (int64_t)row_bs[i] * col_bs[j];
            if (blk_off[b] < 0 || blk_off[b] + len > data_len) return set_error(BSM_ERR_ARG, "block outside data_len");
            if (blk_off[b] < prev_end) in_order = false;
            prev_end = blk_off[b] + len;
        }
    }
    if (!in_order) {
        std::vector<std::pair<int64_t, int64_t>> spans;
        spans.reserve((size_t)nnzb);
        for (int32_t i = 0; i < nbr; ++i)
            for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b)
                spans.emplace_back(blk_off[b], (int64_t)row_bs[i] * col_bs[col_idx[b]]);
        std::sort(spans.begin(), spans.end());
        for (size_t q = 1; q < spans.size(); ++q)
            if (spans[q - 1].first + spans[q - 1].second > spans[q].first) return set_error(BSM_ERR_ARG, "blocks overlap");
    }
    if (data_mode == BSM_DATA_BORROW && data) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, data) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return set_error(BSM_ERR_ARG, "BSM_DATA_BORROW needs a device pointer");
        }
    }
    bsm_mat *X = nullptr;
    bsm_status st = create_common(out, nbr, nbc, row_bs, col_bs, dtype, &X);
    if (st) return st;
    X->nnzb = nnzb;
    X->data_len = data_len;
    if ((st = dalloc_t(&X->row_ptr, (size_t)nbr + 1)) || (st = dalloc_t(&X->col_idx, nnzb)) ||
        (st = dalloc_t(&X->blk_off, nnzb)) || (st = dalloc_t(&X->blk_rc, nnzb))) {
        bsm_destroy(X);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(X->row_ptr, row_ptr, sizeof(int64_t) * (nbr + 1), cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess && nnzb)
        e = cudaMemcpyAsync(X->col_idx, col_idx, sizeof(int32_t) * nnzb, cudaMemcpyHostToDevice, g_stream);
    if (e == cudaSuccess && nnzb)
        e = cudaMemcpyAsync(X->blk_off, blk_off, sizeof(int64_t) * nnzb, cudaMemcpyHostToDevice, g_stream);
    if (e != cudaSuccess) {
        bsm_destroy(X);
        return cuda_check(e, "copy pattern");
    }
    if (data_mode == BSM_DATA_BORROW) {
        X->data = const_cast<void *>(data);
        X->own_data = false;
    } else {
        if ((st = dalloc(&X->data, (size_t)data_len * esize(dtype)))) {
            bsm_destroy(X);
            return st;
        }
        X->own_data = true;
        if (data_len > 0) {
            e = cudaMemcpyAsync(X->data, data, (size_t)data_len * esize(dtype), cudaMemcpyDefault, g_stream);
            if (e != cudaSuccess) {
                bsm_destroy(X);
                return cuda_check(e, "copy data");
            }
        }
    }
    if ((st = cuda_check(launch_blk_rc(X, X->blk_rc, g_stream), "block shapes"))) {
        bsm_destroy(X);
        return st;
    }
    // pageable host sources: make sure the copies have consumed them
    if ((st = cuda_check(cudaStreamSynchronize(g_stream), "stream synchronize"))) {
        bsm_destroy(X);
        return st;
    }
    *out = X;
    return BSM_OK;
}

bsm_status bsm_create_empty(bsm_t *out, int32_t nbr, int32_t nbc, const int32_t *row_bs, const int32_t *col_bs,
                            int32_t dtype) {
    bsm_mat *X = nullptr;
    bsm_status st = create_common(out, nbr, nbc, row_bs, col_bs, dtype, &X);
    if (st) return st;
    if ((st = dalloc_t(&X->row_ptr, (size_t)nbr + 1))) {
        bsm_destroy(X);
        return st;
    }
    cudaError_t e = cudaMemsetAsync(X->row_ptr, 0, sizeof(int64_t) * (nbr + 1), g_stream);
    if ((st = cuda_check(e, "memset"))) {
        bsm_destroy(X);
        return st;
    }
    if ((st = cuda_check(cudaStreamSynchronize(g_stream), "stream synchronize"))) {
        bsm_destroy(X);
        return st;
    }
    *out = X;
    return BSM_OK;
}

bsm_status bsm_create_like(bsm_t *out, bsm_t X) {
    if (!X) return set_error(BSM_ERR_ARG, "X is NULL");
    bsm_mat *Y = nullptr;
    bsm_status st = create_common(out, X->nbr, X->nbc, X->h_row_bs.data(), X->h_col_bs.data(), X->dtype, &Y);
    if (st) return st;
    Y->nnzb = X->nnzb;
    Y->data_len = X->data_len;
    if ((st = dalloc_t(&Y->row_ptr, (size_t)X->nbr + 1)) || (st = dalloc_t(&Y->col_idx, X->nnzb)) ||
        (st = dalloc_t(&Y->blk_off, X->nnzb)) || (st = dalloc_t(&Y->blk_rc, X->nnzb)) ||
        (st = dalloc(&Y->data, (size_t)X->data_len * esize(X->dtype)))) {
        bsm_destroy(Y);
        return st;
    }
    Y->own_data = true;
    cudaError_t e = cudaMemcpyAsync(Y->row_ptr, X->row_ptr, sizeof(int64_t) * (X->nbr + 1), cudaMemcpyDeviceToDevice, g_stream);
    if (e == cudaSuccess && X->nnzb) {
        e = cudaMemcpyAsync(Y->col_idx, X->col_idx, sizeof(int32_t) * X->nnzb, cudaMemcpyDeviceToDevice, g_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Y->blk_off, X->blk_off, sizeof(int64_t) * X->nnzb, cudaMemcpyDeviceToDevice, g_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Y->blk_rc, X->blk_rc, sizeof(int32_t) * X->nnzb, cudaMemcpyDeviceToDevice, g_stream);
    }
    if (e == cudaSuccess && X->data_len)
        e = cudaMemsetAsync(Y->data, 0, (size_t)X->data_len * esize(X->dtype), g_stream);
    if ((st = cuda_check(e, "create_like"))) {
        bsm_destroy(Y);
        return st;
    }
    *out = Y;
    return BSM_OK;
}

bsm_status bsm_destroy(bsm_t X) {
    if (!X) return BSM_OK;
    free_results(X);
    free_pattern(X);
    dfree(X->row_bs);
    dfree(X->col_bs);
    dfree(X->row_start);
    dfree(X->col_start);
    dfree(X->status);
    delete X;
    return BSM_OK;
}

bsm_status bsm_get_info(bsm_t X, int32_t *nbr, int32_t *nbc, int64_t *nnzb, int64_t *data_len, int32_t *dtype) {
    if (!X) return set_error(BSM_ERR_ARG, "X is NULL");
    if (nbr) *nbr = X->nbr;
    if (nbc) *nbc = X->nbc;
    if (nnzb) *nnzb = X->nnzb;
    if (data_len) *data_len = X->data_len;
    if (dtype) *dtype = X->dtype;
    return BSM_OK;
}

bsm_status bsm_copy_pattern(bsm_t X, int64_t *row_ptr, int32_t *col_idx, int64_t *blk_off) {
    if (!X) return set_error(BSM_ERR_ARG, "X is NULL");
    cudaError_t e = cudaSuccess;
    if (row_ptr) e = cudaMemcpyAsync(row_ptr, X->row_ptr, sizeof(int64_t) * (X->nbr + 1), cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess && col_idx && X->nnzb)
        e = cudaMemcpyAsync(col_idx, X->col_idx, sizeof(int32_t) * X->nnzb, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess && blk_off && X->nnzb)
        e = cudaMemcpyAsync(blk_off, X->blk_off, sizeof(int64_t) * X->nnzb, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    return cuda_check(e, "copy pattern");
}

bsm_status bsm_copy_data(bsm_t X, void *dst) {
    if (!X || (!dst && X->data_len)) return set_error(BSM_ERR_ARG, "NULL argument");
    if (X->data_len == 0) return BSM_OK;
    cudaError_t e = cudaMemcpyAsync(dst, X->data, (size_t)X->data_len * esize(X->dtype), cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    return cuda_check(e, "copy data");
}

bsm_status bsm_set_data(bsm_t X, const void *src) {
    if (!X || (!src && X->data_len)) return set_error(BSM_ERR_ARG, "NULL argument");
    X->norms_valid = false;
    if (X->data_len == 0) return BSM_OK;
    cudaError_t e = cudaMemcpyAsync(X->data, src, (size_t)X->data_len * esize(X->dtype), cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    return cuda_check(e, "set data");
}

bsm_status bsm_data_ptr(bsm_t X, void **dptr) {
    if (!X || !dptr) return set_error(BSM_ERR_ARG, "NULL argument");
    *dptr = X->data;
    return BSM_OK;
}

bsm_status bsm_block_norms(bsm_t X, double *out) {
    if (!X || (!out && X->nnzb)) return set_error(BSM_ERR_ARG, "NULL argument");
    if (X->nnzb == 0) return BSM_OK;
    Scratch sc;
    double *d = nullptr;
    bsm_status st = sc.get(&d, X->nnzb);
    if (st) return st;
    cudaError_t e = launch_block_norms(X, d, g_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * X->nnzb, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    return cuda_check(e, "block norms");
}

// --------------------------------------------------------------------------
// multiply
// --------------------------------------------------------------------------
bsm_status bsm_multiply(double alpha, bsm_t A, bsm_t B, double beta, bsm_t C, double filter_eps,
                        const bsm_opts *opts_in) {
    if (!A || !B || !C) return set_error(BSM_ERR_ARG, "NULL matrix");
    if (C == A || C == B) return set_error(BSM_ERR_ARG, "C must differ from A and B");
    bsm_opts opts;
    bsm_status st = check_opts(opts_in, &opts);
    if (st) return st;
    if (A->dtype != B->dtype || A->dtype != C->dtype) return set_error(BSM_ERR_ARG, "A, B and C must share a dtype");
    if (A->nbc != B->nbr || !same_vec(A->h_col_bs, B->h_row_bs))
        return set_error(BSM_ERR_BLOCKING, "A's block columns do not match B's block rows");
    if (C->nbr != A->nbr || !same_vec(C->h_row_bs, A->h_row_bs))
        return set_error(BSM_ERR_BLOCKING, "C's block rows do not match A's block rows");
    if (C->nbc != B->nbc || !same_vec(C->h_col_bs, B->h_col_bs))
        return set_error(BSM_ERR_BLOCKING, "C's block columns do not match B's block columns");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || std::isnan(filter_eps))
        return set_error(BSM_ERR_ARG, "alpha, beta and eps must be finite");
    const bool no_sync = opts.no_sync != 0;
    // BSM_P_TF32x3_PANEL: the tcgen05 row-panel engine where it applies, else
    // the mma.sync TF32x3 kernel (rprec: the precision of the mma.sync path)
    // BSM_P_TF32x3 with the tuned engine 1 (and the compensated sum) also takes
    // the row-panel engine where it applies
    const bool tuned_panel = opts.prec == BSM_P_TF32x3 && !no_sync && opts.flush_every <= 0 &&
                             tune_of(BSM_P_TF32x3)[BSM_TUNE_ENGINE] == 1;
    const bool want_panel = opts.prec == BSM_P_TF32x3_PANEL || tuned_panel;
    if (opts.prec == BSM_P_TF32x3_PANEL && no_sync)
        return set_error(BSM_ERR_UNSUPPORTED, "BSM_P_TF32x3_PANEL does not run with no_sync");
    const int rprec = want_panel ? BSM_P_TF32x3 : opts.prec;
    const auto &pl = C->plan;
    if (no_sync) {
        if (pl.kind != 1 || pl.A != A || pl.B != B || pl.A_nnzb != A->nnzb || pl.B_nnzb != B->nnzb ||
            pl.eps != filter_eps || pl.prec != opts.prec || !C->pa)
            return set_error(BSM_ERR_ARG, "no_sync needs an earlier eager multiply of the same A and B (same eps "
                                          "and precision) into C");
        if (beta != 0.0) return set_error(BSM_ERR_UNSUPPORTED, "no_sync needs beta == 0");
        if (opts.post_filter) return set_error(BSM_ERR_UNSUPPORTED, "no_sync excludes post_filter");
    } else if ((st = ensure_globals())) {
        return st;
    }
    // kernel precision: the Ozaki path whose output blocks all run one per lane
    // (plain FP64 FMA) needs no slices at all
    int kprec = rprec;
    if (opts.prec == BSM_P_OZAKI) {
        if (no_sync) kprec = pl.kprec;
        else if (all_lane(opts.prec, A->h_row_bs, B->h_col_bs)) kprec = BSM_P_FP64;
    }
    if (opts.prec == BSM_P_OZAKI) {
        if (A->dtype != BSM_FP64) return set_error(BSM_ERR_UNSUPPORTED, "BSM_P_OZAKI needs FP64 data");
        if (no_sync) {
            if (!A->row_start || !B->row_start) return set_error(BSM_ERR_ARG, "no_sync needs an earlier eager multiply");
        } else if ((st = ensure_starts(A)) || (st = ensure_starts(B))) {
            return st;
        }
    }
    if ((st = ensure_status(C))) return st;

    const int32_t nbr = A->nbr, nbk = A->nbc, nbc = B->nbc;
    const bool use_filter = filter_eps > 0.0;
    const bool use_old = beta != 0.0 && C->nnzb > 0;
    const int32_t nwords = (nbc + 31) / 32;
    Events ev;
    if (!no_sync) ev.start();
    ev.mark(0);
    Scratch sc;
    cudaError_t e = cudaMemsetAsync(C->status, 0, sizeof(int32_t), g_stream);
    if ((st = cuda_check(e, "status"))) return st;

    // ---- a1: block norms (FP64) of A and B
    double *nA = nullptr, *nB = nullptr;
    if (use_filter) {
        if ((st = sc.get(&nA, A->nnzb))) return st;
        if ((st = cuda_check(launch_block_norms(A, nA, g_stream), "norms A"))) return st;
        if (B == A) {
            nB = nA;
        } else {
            if ((st = sc.get(&nB, B->nnzb))) return st;
            if ((st = cuda_check(launch_block_norms(B, nB, g_stream), "norms B"))) return st;
        }
    }
    ev.mark(1);

    // ---- a2: symbolic count
    SymbolicArgs sa{};
    sa.nbr = nbr; sa.nbk = nbk; sa.nbc = nbc;
    sa.a_row_bs = A->row_bs; sa.a_col_bs = A->col_bs; sa.a_row_ptr = A->row_ptr; sa.a_col_idx = A->col_idx;
    sa.a_norm = nA;
    sa.b_row_ptr = B->row_ptr; sa.b_col_idx = B->col_idx; sa.b_col_bs = B->col_bs; sa.b_norm = nB;
    sa.o_row_ptr = use_old ? C->row_ptr : nullptr;
    sa.o_col_idx = use_old ? C->col_idx : nullptr;
    sa.o_blk_off = use_old ? C->blk_off : nullptr;
    sa.eps = filter_eps;
    sa.use_filter = use_filter ? 1 : 0;
    sa.nwords = nwords;
    sa.status = no_sync ? C->status : nullptr;
    if ((size_t)nwords * 4 > 200 * 1024) return set_error(BSM_ERR_UNSUPPORTED, "too many block columns for the symbolic phase");
    int64_t *prod_cnt, *ccol_cnt, *celem_cnt, *prod_ptr, *crow_ptr, *celem_ptr, *stmp;
    uint32_t *bitmaps;
    unsigned long long *totals;
    if ((st = sc.get(&prod_cnt, nbr)) || (st = sc.get(&ccol_cnt, nbr)) || (st = sc.get(&celem_cnt, nbr)) ||
        (st = sc.get(&prod_ptr, (size_t)nbr + 1)) || (st = sc.get(&crow_ptr, (size_t)nbr + 1)) ||
        (st = sc.get(&celem_ptr, (size_t)nbr + 1)) || (st = sc.get(&stmp, scan_tmp_elems(nbr))) ||
        (st = sc.get(&bitmaps, (size_t)nbr * nwords)) || (st = sc.get(&totals, 4)))
        return st;
    e = cudaMemsetAsync(totals, 0, 4 * sizeof(unsigned long long), g_stream);
    if (e == cudaSuccess) e = launch_symbolic_count(sa, prod_cnt, ccol_cnt, celem_cnt, bitmaps, totals, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(prod_cnt, prod_ptr, nbr, stmp, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(ccol_cnt, crow_ptr, nbr, stmp, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(celem_cnt, celem_ptr, nbr, stmp, g_stream);
    if ((st = cuda_check(e, "symbolic count"))) return st;
    // pack sizes of the tensor-core operands, known with the symbolic totals
    Packed pkA, pkB;
    const bool tc = is_tc(kprec);
    if (tc) {
        if ((st = pack_prepare(sc, A, 0, 0, kprec, pkA))) return st;
        if ((st = pack_prepare(sc, B, 1, 0, kprec, pkB))) return st;
    }
    int64_t nprod, nnzbC, lenC, nfilt, mnk, packA_words = 0, packB_words = 0, max_ccnt = 0;
    int nchunk = 8;
    // row panels of a multiply above the product limit (empty: one pass)
    std::vector<int32_t> panel_rows;
    std::vector<int64_t> h_pp, h_cp;
    int64_t panel_max = 0;
    if (no_sync) {
        // sizes of the eager call; the device checks that they hold
        nprod = pl.nprod; nnzbC = pl.nnzb; lenC = pl.len; nfilt = pl.nfilt; mnk = pl.mnk;
        packA_words = pl.packA; packB_words = pl.packB; max_ccnt = pl.max_ccnt; nchunk = pl.nchunk;
        PlanCheck pc{};
        pc.actual[0] = prod_ptr + nbr; pc.expected[0] = nprod;
        pc.actual[1] = crow_ptr + nbr; pc.expected[1] = nnzbC;
        pc.actual[2] = celem_ptr + nbr; pc.expected[2] = lenC;
        pc.actual[3] = (const int64_t *)(totals + 2); pc.expected[3] = max_ccnt; pc.at_most[3] = 1;
        pc.n = 4;
        if (tc) {
            pc.actual[4] = pkA.off + A->nnzb; pc.expected[4] = packA_words;
            pc.actual[5] = pkB.off + B->nnzb; pc.expected[5] = packB_words;
            pc.n = 6;
        }
        if ((st = cuda_check(launch_check_plan(pc, C->status, g_stream), "plan check"))) return st;
    } else {
        std::vector<int64_t> h_ccnt((size_t)nbr);
        const int64_t *src[7] = {prod_ptr + nbr, crow_ptr + nbr, celem_ptr + nbr, (const int64_t *)totals,
                                 (const int64_t *)(totals + 1), tc ? pkA.off + A->nnzb : nullptr,
                                 tc ? pkB.off + B->nnzb : nullptr};
        if (nbr > 0) {
            e = cudaMemcpyAsync(h_ccnt.data(), ccol_cnt, sizeof(int64_t) * nbr, cudaMemcpyDeviceToHost, g_stream);
            if ((st = cuda_check(e, "read counts"))) return st;
        }
        if ((st = read_words(src, tc ? 7 : 5))) return st;
        nprod = g_host[0]; nnzbC = g_host[1]; lenC = g_host[2]; nfilt = g_host[3]; mnk = g_host[4];
        if (tc) {
            packA_words = g_host[5];
            packB_words = g_host[6];
        }
        for (int64_t v : h_ccnt) max_ccnt = std::max(max_ccnt, v);
        if (nnzbC > INT32_MAX)
            return set_error(BSM_ERR_UNSUPPORTED, std::to_string(nnzbC) + " C blocks: more than 2^31-1 in one multiply");
        // more kept products than one pass holds: row panels of C, each within the limit
        const int64_t plimit = g_product_limit.load(std::memory_order_relaxed);
        if (nprod > plimit) {
            h_pp.resize((size_t)nbr + 1);
            h_cp.resize((size_t)nbr + 1);
            e = cudaMemcpyAsync(h_pp.data(), prod_ptr, sizeof(int64_t) * (nbr + 1), cudaMemcpyDeviceToHost, g_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_cp.data(), crow_ptr, sizeof(int64_t) * (nbr + 1), cudaMemcpyDeviceToHost, g_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
            if ((st = cuda_check(e, "read row pointers"))) return st;
            panel_rows.push_back(0);
            for (int32_t r = 0; r < nbr;) {
                if (h_pp[r + 1] - h_pp[r] > plimit)
                    return set_error(BSM_ERR_CAPACITY, "C block row " + std::to_string(r) + " has " +
                                                           std::to_string(h_pp[r + 1] - h_pp[r]) +
                                                           " kept products, above the product limit of one pass");
                int32_t r1 = r + 1;
                while (r1 < nbr && h_pp[r1 + 1] - h_pp[r] <= plimit) ++r1;
                panel_max = std::max(panel_max, h_pp[r1] - h_pp[r]);
                panel_rows.push_back(r1);
                r = r1;
            }
        }
        while (nchunk > 1 && symbolic_fill_smem_bytes(nwords, (int32_t)max_ccnt, nchunk) > 160 * 1024) nchunk >>= 1;
        if (symbolic_fill_smem_bytes(nwords, (int32_t)max_ccnt, nchunk) > 220 * 1024)
            return set_error(BSM_ERR_UNSUPPORTED, "a C block row has too many blocks for the fill phase");
    }
    const bool chunked = !panel_rows.empty();
    int32_t panel_s = 0;
    const bool use_panel = want_panel && !chunked && A->dtype == BSM_FP64 && nfilt == 0 && panel_blocking(A, B, &panel_s) &&
                           panel_tile_smem((B->nbc + panel_tile_cols() - 1) / panel_tile_cols()) <= 200 * 1024;
    ev.mark(2);

    // ---- a3: fill C's pattern and the product list
    int32_t *c_col = nullptr, *c_rc = nullptr, *pa = nullptr, *pb = nullptr, *pc = nullptr;
    int64_t *c_off = nullptr, *cptr = nullptr, *old_off = nullptr;
    void *c_data = nullptr;
    if (no_sync) {  // C's present storage has exactly these sizes
        c_col = C->col_idx; c_off = C->blk_off; c_rc = C->blk_rc; cptr = C->cptr;
        pa = C->pa; pb = C->pb; pc = C->pc; c_data = C->data;
    } else {
        const int64_t nprod_alloc = chunked ? panel_max : nprod;  // products held at once
        if ((st = sc.get(&c_col, nnzbC)) || (st = sc.get(&c_off, nnzbC)) || (st = sc.get(&c_rc, nnzbC)) ||
            (st = sc.get(&cptr, (size_t)nnzbC + 1)) || (st = sc.get(&pa, nprod_alloc)) ||
            (st = sc.get(&pb, nprod_alloc)) || (st = sc.get(&pc, nprod_alloc)))
            return st;
        if (use_old && (st = sc.get(&old_off, nnzbC))) return st;
        if ((st = dalloc(&c_data, (size_t)lenC * esize(C->dtype)))) return st;
        sc.ptrs.push_back(c_data);
    }
    FillOut fo{prod_ptr, crow_ptr, celem_ptr, c_col, c_off, c_rc, cptr, pa, pb, pc, old_off, (int32_t)max_ccnt, nchunk};
    // fill through B's columns when the k -> A block map fits in shared memory
    const bool by_cols = symbolic_fill_cols_smem_bytes(nwords, (int32_t)max_ccnt, nbk) <= 200 * 1024;
    if (by_cols) {
        if (no_sync && !B->t_ptr) return set_error(BSM_ERR_ARG, "no_sync: B's column copy is missing");
        if ((st = ensure_transpose(B))) return st;
    }
    // rows [r0, r1) of C's pattern and of the product list (offsets relative to prod_ptr[r0])
    auto fill_rows = [&](int32_t r0, int32_t r1, int64_t prod_base) -> cudaError_t {
        FillOut f = fo;
        f.row0 = r0;
        f.prod_base = prod_base;
        return by_cols ? launch_symbolic_fill_cols(sa, bitmaps, f, B->t_ptr, B->t_row, B->t_blk, g_stream, r1 - r0)
                       : launch_symbolic_fill(sa, bitmaps, f, g_stream, r1 - r0);
    };
    if (!chunked) {  // a chunked multiply fills each row panel right before its numeric pass
        e = fill_rows(0, nbr, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cptr + nnzbC, prod_ptr + nbr, sizeof(int64_t), cudaMemcpyDeviceToDevice, g_stream);
        if (e == cudaSuccess && no_sync) e = launch_copy_i64_if_ok(nbr + 1, crow_ptr, C->row_ptr, C->status, g_stream);
        if ((st = cuda_check(e, "symbolic fill"))) return st;
    }
    ev.mark(3);

    // ---- a4: stacks by shape (m, n, k)
    int32_t nshapes = 0;
    std::vector<int32_t> h_shapes;
    int64_t *stack_ptr = nullptr, *triples = nullptr;
    if (!no_sync && !chunked && opts.build_stacks && nprod > 0) {
        std::vector<int32_t> sizes;
        for (auto *v : {&A->h_row_bs, &A->h_col_bs, &B->h_col_bs}) sizes.insert(sizes.end(), v->begin(), v->end());
        std::sort(sizes.begin(), sizes.end());
        sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
        const int32_t ns = (int32_t)sizes.size();
        const int64_t nsh = (int64_t)ns * ns * ns;
        if (nsh > (1 << 24)) return set_error(BSM_ERR_UNSUPPORTED, "too many distinct block sizes for stacks");
        std::vector<int32_t> sidx(kMaxBlockDim + 1, 0);
        for (int32_t q = 0; q < ns; ++q) sidx[sizes[q]] = q;
        int32_t *d_sidx;
        int64_t *counts;
        if ((st = sc.get(&d_sidx, kMaxBlockDim + 1)) || (st = sc.get(&counts, nsh))) return st;
        if ((st = dalloc_t(&triples, (size_t)nprod * 3))) return st;
        sc.ptrs.push_back(triples);
        e = cudaMemcpyAsync(d_sidx, sidx.data(), sizeof(int32_t) * sidx.size(), cudaMemcpyHostToDevice, g_stream);
        if (nsh <= stack_max_bins()) {
            // few shapes: per-tile histogram, then every triple written to its place
            int64_t *stmp;
            if ((st = sc.get(&stmp, stack_tmp_elems(nprod, (int32_t)nsh)))) return st;
            if (e == cudaSuccess)
                e = launch_stacks_direct(nprod, pa, pb, pc, A->blk_rc, B->blk_rc, d_sidx, ns, (int32_t)nsh,
                                         A->blk_off, B->blk_off, c_off, triples, counts, stmp, g_stream);
        } else {
            // many shapes: stable radix sort of the shape ids, then the triples
            int32_t *iota, *order, *vals_alt;
            uint32_t *keys, *keys_sorted, *keys_alt;
            int64_t *rtmp;
            if ((st = sc.get(&iota, nprod)) || (st = sc.get(&order, nprod)) || (st = sc.get(&vals_alt, nprod)) ||
                (st = sc.get(&keys, nprod)) || (st = sc.get(&keys_sorted, nprod)) || (st = sc.get(&keys_alt, nprod)) ||
                (st = sc.get(&rtmp, radix_tmp_elems(nprod))))
                return st;
            int bits = 1;
            while ((1ll << bits) < nsh) ++bits;
            if (e == cudaSuccess)
                e = launch_product_shape_ids(nprod, pa, pb, A->blk_rc, B->blk_rc, d_sidx, ns, keys, iota, g_stream);
            if (e == cudaSuccess)
                e = launch_radix_sort_pairs(keys, iota, keys_alt, vals_alt, keys_sorted, order, nprod, bits, rtmp,
                                            g_stream);
            if (e == cudaSuccess) e = launch_histogram_u32(nprod, keys, nsh, counts, g_stream);
            if (e == cudaSuccess)
                e = launch_stack_triples(nprod, order, pa, pb, pc, A->blk_off, B->blk_off, c_off, triples, g_stream);
        }
        std::vector<int64_t> h_counts((size_t)nsh);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_counts.data(), counts, sizeof(int64_t) * nsh, cudaMemcpyDeviceToHost, g_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
        if ((st = cuda_check(e, "stacks"))) return st;
        std::vector<int64_t> h_ptr(1, 0);
        for (int64_t id = 0; id < nsh; ++id) {
            if (!h_counts[id]) continue;
            const int32_t mi = (int32_t)(id / ((int64_t)ns * ns)), ni = (int32_t)((id / ns) % ns), ki = (int32_t)(id % ns);
            h_shapes.push_back(sizes[mi]);
            h_shapes.push_back(sizes[ni]);
            h_shapes.push_back(sizes[ki]);
            h_ptr.push_back(h_ptr.back() + h_counts[id]);
        }
        nshapes = (int32_t)(h_ptr.size() - 1);
        if ((st = dalloc_t(&stack_ptr, h_ptr.size()))) return st;
        sc.ptrs.push_back(stack_ptr);
        e = cudaMemcpyAsync(stack_ptr, h_ptr.data(), sizeof(int64_t) * h_ptr.size(), cudaMemcpyHostToDevice, g_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);  // h_ptr is pageable
        if ((st = cuda_check(e, "stack pointers"))) return st;
    }
    ev.mark(4);

    // ---- a5/a6: numeric
    NumericLaunch nl{use_panel ? BSM_K_PANEL_TCGEN05 : BSM_K_NONE, -1, 0, 0, 0, 0};
    OzLines olA, olB;
    int32_t *order = nullptr;
    int64_t *n_marked = nullptr, *groups = nullptr;
    bool uses_cores = false;
    if (use_panel) {
        PanelOut po{nnzbC, crow_ptr, c_col, c_off, static_cast<double *>(c_data), old_off,
                    use_old ? C->data : nullptr, alpha, use_old ? beta : 0.0, C->status};
        if ((st = run_panel(sc, A, B, panel_s, po, ev, opts.prec))) return st;
        int32_t hs = 0;
        e = cudaMemcpyAsync(&hs, C->status, sizeof(int32_t), cudaMemcpyDeviceToHost, g_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
        if ((st = cuda_check(e, "panel status"))) return st;
        if (hs != 0) return set_error(BSM_ERR_TIMEOUT, "a wait of the row-panel kernel gave up");
    } else {
    if (tc) {
        if ((st = sc.get(&pkA.words, (size_t)packA_words + 16)) || (st = sc.get(&pkB.words, (size_t)packB_words + 16)))
            return st;
        if (kprec == BSM_P_OZAKI && ((st = oz_lines(sc, A, 0, 0, olA)) || (st = oz_lines(sc, B, 1, 0, olB))))
            return st;
        e = launch_pack(A, 0, 0, kprec, pkA.off, pkA.words, no_sync ? C->status : nullptr, g_stream, olA.line0,
                        olA.exps);
        if (e == cudaSuccess)
            e = launch_pack(B, 1, 0, kprec, pkB.off, pkB.words, no_sync ? C->status : nullptr, g_stream,
                            olB.line0, olB.exps);
        if ((st = cuda_check(e, "pack"))) return st;
    }
    // one numeric pass over the output blocks [cb0, cb0 + nitems) holding nprod_pass
    // products (the whole C, or one row panel of a chunked multiply)
    float *plain_x = nullptr, *plain_y = nullptr;
    // split paths: blocks of one tile row in their own kernel instance, unless
    // the tuning fixes the pass rows; Ozaki path: blocks of one tile column
    const bool want_groups = rprec == BSM_P_OZAKI || tune_of(rprec)[BSM_TUNE_PASS_MT] <= 0;
    auto numeric_pass = [&](int64_t cb0, int64_t nitems, int64_t nprod_pass, bool whole) -> bsm_status {
        NumericArgs na{};
        na.n_items = nitems;
        na.seg_ptr = cptr + cb0;
        na.px = pa;
        na.py = pb;
        na.out_data = c_data;
        na.out_blk_off = c_off + cb0;
        na.out_blk_rc = c_rc + cb0;
        na.x_data = A->data; na.x_blk_off = A->blk_off; na.x_blk_rc = A->blk_rc; na.x_trans = 0;
        na.y_data = B->data; na.y_blk_off = B->blk_off; na.y_blk_rc = B->blk_rc; na.y_trans = 0;
        na.alpha = alpha;
        na.beta = use_old ? beta : 0.0;
        na.old_data = use_old ? C->data : nullptr;
        na.old_off = old_off ? old_off + cb0 : nullptr;
        na.dtype = C->dtype;
        na.prec = kprec;
        na.flush_every = opts.flush_every;
        na.max_out_rows = A->max_bs_row; na.max_out_cols = B->max_bs_col;
        na.x_pack = pkA.words; na.x_pack_off = pkA.off;
        na.y_pack = pkB.words; na.y_pack_off = pkB.off;
        na.x_exp = olA.exps; na.x_line0 = olA.line0;
        na.y_exp = olB.exps; na.y_line0 = olB.line0;
        na.status = no_sync ? C->status : nullptr;
        bsm_status sst;
        if ((sst = sc.get(&na.work_counter, 4))) return sst;
        if (no_sync) {
            order = C->item_order;
            n_marked = C->n_marked;
            groups = C->item_groups;
            uses_cores = pl.uses_cores;
        } else if (whole) {
            if ((sst = ensure_row_rank(A))) return sst;
            const int32_t tile = tune_of(rprec)[BSM_TUNE_SCHED_TILE];
            if (tile > 0 && (sst = ensure_col_rank(B))) return sst;
            bsm_mat rows_view;
            rows_view.nbr = nbr;
            rows_view.row_ptr = crow_ptr;
            if ((sst = shape_order(sc, nitems, c_rc + cb0, A->h_row_bs, B->h_col_bs, &order, &rows_view, A->row_rank,
                                   rprec, &uses_cores, &n_marked, c_col + cb0, tile > 0 ? B->col_rank : nullptr, nbc,
                                   tile > 0 ? tile : 0, want_groups ? &groups : nullptr)))
                return sst;
        } else {  // a row panel: block-shape classes and variants only
            if ((sst = shape_order(sc, nitems, c_rc + cb0, A->h_row_bs, B->h_col_bs, &order, nullptr, nullptr, rprec,
                                   &uses_cores, &n_marked, nullptr, nullptr, 0, 0, want_groups ? &groups : nullptr)))
                return sst;
        }
        na.item_groups = groups;
        na.n_lane_items = n_marked;
        if (needs_plain(kprec) && uses_cores && !plain_x) {  // unpacked pieces for the CUDA-core split variant
            const int np = split_pieces(rprec);
            if ((sst = sc.get(&plain_x, (size_t)A->data_len * np))) return sst;
            cudaError_t pe = launch_split_plain(A, rprec, plain_x, g_stream);
            if (pe == cudaSuccess && B != A) {
                if ((sst = sc.get(&plain_y, (size_t)B->data_len * np))) return sst;
                pe = launch_split_plain(B, rprec, plain_y, g_stream);
            }
            if ((sst = cuda_check(pe, "split pieces"))) return sst;
        }
        na.x_plain = plain_x;
        na.y_plain = B == A ? plain_x : plain_y;
        na.item_order = order;
        apply_tuning(rprec, na);
        na.n_prod = nprod_pass;
        na.x_nnzb = A->nnzb; na.y_nnzb = B->nnzb;
        na.x_len = A->data_len; na.y_len = B->data_len;
        na.out_len = lenC; na.old_len = use_old ? C->data_len : 0;
        na.x_pack_words = packA_words; na.y_pack_words = packB_words;
        if (whole) ev.mark(5);
        if ((sst = cuda_check(launch_numeric(na, g_stream, &nl), "numeric"))) return sst;
#ifdef BSM_DEBUG
        if (!no_sync)
            if (const uint32_t bits = numeric_debug_bits(g_stream))
                return set_error(BSM_ERR_CUDA, "debug bounds check of the numeric kernel failed (bits " +
                                                   std::to_string(bits) + ")");
#endif
        return BSM_OK;
    };
    if (!chunked) {
        if ((st = numeric_pass(0, nnzbC, nprod, true))) return st;
    } else {
        ev.mark(5);  // the row panels' fill and numeric passes, timed together
        // row panels: fill the panel's pattern and products, then its numeric pass
        for (size_t q = 0; q + 1 < panel_rows.size(); ++q) {
            const int32_t r0 = panel_rows[q], r1 = panel_rows[q + 1];
            const int64_t cb0 = h_cp[r0], cb1 = h_cp[r1], np = h_pp[r1] - h_pp[r0];
            e = fill_rows(r0, r1, h_pp[r0]);
            // the panel's end of products (a pageable source: staged before the call returns)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(cptr + cb1, &np, sizeof(int64_t), cudaMemcpyHostToDevice, g_stream);
            if ((st = cuda_check(e, "symbolic fill of a row panel"))) return st;
            if (cb1 > cb0 && (st = numeric_pass(cb0, cb1 - cb0, np, false))) return st;
        }
        order = nullptr;  // the panels' orders are scratch
        n_marked = nullptr;
        groups = nullptr;
    }
    ev.mark(6);
    }
    if (no_sync) return BSM_OK;  // C's storage, counts and plan are unchanged

    // ---- swap C's pattern (old arrays are freed stream-ordered after the numeric kernel)
    free_results(C);
    free_pattern(C);
    C->item_order = order;
    C->n_marked = n_marked;
    C->item_groups = groups;
    C->row_ptr = crow_ptr;
    C->col_idx = c_col;
    C->blk_off = c_off;
    C->blk_rc = c_rc;
    C->data = c_data;
    C->own_data = true;
    C->nnzb = nnzbC;
    C->data_len = lenC;
    if (chunked) {  // no product list of the whole C is kept: it goes back with the scratch
        cptr = nullptr;
        pa = pb = pc = nullptr;
    }
    C->cptr = cptr;
    C->pa = pa; C->pb = pb; C->pc = pc;
    C->nprod = nprod;
    C->nfiltered = nfilt;
    C->useful_flop = 2.0 * (double)mnk;
    C->nshapes = nshapes;
    C->h_shapes = h_shapes;
    C->stack_ptr = stack_ptr;
    C->triples = triples;
    C->prod_A = chunked ? nullptr : A;
    C->prod_B = chunked ? nullptr : B;
    C->prod_A_nnzb = A->nnzb; C->prod_B_nnzb = B->nnzb;
    C->launch_cfg[0] = nl.kernel; C->launch_cfg[1] = nl.build; C->launch_cfg[2] = nl.cta_threads;
    C->launch_cfg[3] = nl.grid; C->launch_cfg[4] = nl.pass_mt; C->launch_cfg[5] = nl.pass_nt;
    C->engine = nnzbC == 0 ? BSM_E_NONE
                : use_panel ? BSM_E_PANEL_TCGEN05
                : kprec == BSM_P_OZAKI ? BSM_E_OZAKI_MMA
                : is_tc(kprec) ? BSM_E_SPLIT_MMA
                               : BSM_E_FP64_CORES;
    for (void *p : {(void *)crow_ptr, (void *)c_col, (void *)c_off, (void *)c_rc, c_data, (void *)cptr, (void *)pa,
                    (void *)pb, (void *)pc, (void *)stack_ptr, (void *)triples, (void *)order, (void *)n_marked,
                    (void *)groups})
        sc.release(p);
    C->plan = bsm_mat::Plan{};
    if (!use_old && !opts.post_filter && !chunked) {
        auto &P = C->plan;
        P.kind = 1; P.A = A; P.B = B; P.A_nnzb = A->nnzb; P.B_nnzb = B->nnzb; P.eps = filter_eps;
        P.prec = opts.prec; P.kprec = kprec; P.nprod = nprod; P.nnzb = nnzbC; P.len = lenC; P.max_ccnt = max_ccnt;
        P.uses_cores = uses_cores;
        P.nfilt = nfilt; P.mnk = mnk; P.nchunk = nchunk; P.packA = packA_words; P.packB = packB_words;
    }

    // ---- optional post filter (drops C blocks with norm <= eps)
    if (opts.post_filter && use_filter) {
        const int64_t before = C->nnzb;
        if ((st = filter_compact(C, filter_eps, false, nullptr, 0, 0, nullptr))) return st;
        if (C->nnzb != before) {
            // the product list no longer indexes C's blocks
            dfree(C->cptr); C->cptr = nullptr;
            dfree(C->pa); C->pa = nullptr;
            dfree(C->pb); C->pb = nullptr;
            dfree(C->pc); C->pc = nullptr;
            dfree(C->stack_ptr); C->stack_ptr = nullptr;
            dfree(C->triples); C->triples = nullptr;
            dfree(C->item_order); C->item_order = nullptr;
            dfree(C->n_marked); C->n_marked = nullptr;
            dfree(C->item_groups); C->item_groups = nullptr;
            C->nshapes = 0;
            C->h_shapes.clear();
            C->prod_A = C->prod_B = nullptr;
        }
    }
    ev.mark(7);
    if (ev.on) {
        cudaEventSynchronize(ev.ev[7]);
        float ms;
        const int pairs[BSM_T_COUNT][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {5, 6}, {6, 7}, {0, 7}};
        for (int q = 0; q < BSM_T_COUNT; ++q) {
            cudaEventElapsedTime(&ms, ev.ev[pairs[q][0]], ev.ev[pairs[q][1]]);
            C->timings[q] = ms;
        }
        C->timings_valid = true;
    }
    return BSM_OK;
}

// --------------------------------------------------------------------------
// adjoint
// --------------------------------------------------------------------------
static bsm_status group_products(Scratch &sc, int64_t nprod, const int32_t *key_src, int64_t nkeys,
                                 int32_t **order_out, int64_t **seg_out) {
    bsm_status st;
    int32_t *iota, *order, *vals_alt;
    uint32_t *keys, *keys_sorted, *keys_alt;
    int64_t *rtmp, *counts, *seg, *stmp;
    if ((st = sc.get(&iota, nprod)) || (st = sc.get(&order, nprod)) || (st = sc.get(&vals_alt, nprod)) ||
        (st = sc.get(&keys, nprod)) || (st = sc.get(&keys_sorted, nprod)) || (st = sc.get(&keys_alt, nprod)) ||
        (st = sc.get(&rtmp, radix_tmp_elems(nprod))) || (st = sc.get(&counts, nkeys)) ||
        (st = sc.get(&seg, (size_t)nkeys + 1)) || (st = sc.get(&stmp, scan_tmp_elems(nkeys))))
        return st;
    int bits = 1;
    while ((1ll << bits) < nkeys) ++bits;
    cudaError_t e = launch_iota_keys(nprod, key_src, keys, iota, g_stream);
    if (e == cudaSuccess)
        e = launch_radix_sort_pairs(keys, iota, keys_alt, vals_alt, keys_sorted, order, nprod, bits, rtmp, g_stream);
    if (e == cudaSuccess) e = launch_histogram_u32(nprod, keys, nkeys, counts, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(counts, seg, nkeys, stmp, g_stream);
    *order_out = order;
    *seg_out = seg;
    return cuda_check(e, "group products");
}

bsm_status bsm_multiply_backward(double alpha, bsm_t C, const void *dC_data, bsm_t A, bsm_t B, void *dA_data,
                                 void *dB_data, const bsm_opts *opts_in) {
    if (!C || !A || !B) return set_error(BSM_ERR_ARG, "NULL matrix");
    if (!dA_data && !dB_data) return BSM_OK;
    if (!dC_data && C->data_len) return set_error(BSM_ERR_ARG, "dC_data is NULL");
    bsm_opts opts;
    bsm_status st = check_opts(opts_in, &opts);
    if (st) return st;
    if (opts.prec == BSM_P_TF32x3_PANEL) opts.prec = BSM_P_TF32x3;  // the adjoint runs the mma.sync kernel
    if (C->prod_A != A || C->prod_B != B || C->prod_A_nnzb != A->nnzb || C->prod_B_nnzb != B->nnzb || !C->cptr)
        return set_error(BSM_ERR_ARG, "C does not hold the product list of a multiply of these A and B");
    if ((st = ensure_globals())) return st;
    if (opts.prec == BSM_P_OZAKI) {
        if (C->dtype != BSM_FP64) return set_error(BSM_ERR_UNSUPPORTED, "BSM_P_OZAKI needs FP64 data");
        if ((st = ensure_starts(A)) || (st = ensure_starts(B)) || (st = ensure_starts(C))) return st;
    }
    Scratch sc;
    // dC as a matrix with C's pattern (a view: owns nothing)
    bsm_mat dC;
    dC.nbr = C->nbr; dC.nbc = C->nbc; dC.dtype = C->dtype; dC.nnzb = C->nnzb; dC.data_len = C->data_len;
    dC.h_row_bs = C->h_row_bs; dC.h_col_bs = C->h_col_bs;
    dC.row_bs = C->row_bs; dC.col_bs = C->col_bs; dC.row_ptr = C->row_ptr; dC.col_idx = C->col_idx;
    dC.blk_off = C->blk_off; dC.blk_rc = C->blk_rc; dC.data = const_cast<void *>(dC_data);
    dC.row_start = C->row_start; dC.col_start = C->col_start;
    const int64_t nprod = C->nprod;
    for (int side = 0; side < 2; ++side) {
        void *out = side == 0 ? dA_data : dB_data;
        if (!out) continue;
        bsm_mat *OUT = side == 0 ? A : B;
        if (OUT->nnzb == 0) continue;
        int32_t *order = nullptr;
        int64_t *seg = nullptr;
        int32_t *px = nullptr, *py = nullptr;
        if (nprod > 0) {
            if ((st = group_products(sc, nprod, side == 0 ? C->pa : C->pb, OUT->nnzb, &order, &seg))) return st;
            if ((st = sc.get(&px, nprod)) || (st = sc.get(&py, nprod))) return st;
            cudaError_t e;
            if (side == 0) {  // dA = dC . B^T : X = dC (by C block), Y = B^T
                e = launch_gather_i32(nprod, order, C->pc, px, g_stream);
                if (e == cudaSuccess) e = launch_gather_i32(nprod, order, C->pb, py, g_stream);
            } else {          // dB = A^T . dC : X = A^T, Y = dC
                e = launch_gather_i32(nprod, order, C->pa, px, g_stream);
                if (e == cudaSuccess) e = launch_gather_i32(nprod, order, C->pc, py, g_stream);
            }
            if ((st = cuda_check(e, "gather products"))) return st;
        } else {
            if ((st = sc.get(&seg, (size_t)OUT->nnzb + 1))) return st;
            if ((st = cuda_check(cudaMemsetAsync(seg, 0, sizeof(int64_t) * (OUT->nnzb + 1), g_stream), "memset")))
                return st;
        }
        const bsm_mat *X = side == 0 ? &dC : A;
        const bsm_mat *Y = side == 0 ? B : &dC;
        int kprec = opts.prec;  // as in bsm_multiply
        if (opts.prec == BSM_P_OZAKI && all_lane(opts.prec, OUT->h_row_bs, OUT->h_col_bs)) kprec = BSM_P_FP64;
        const bool tc = is_tc(kprec);
        const int xt = side == 0 ? 0 : 1, yt = side == 0 ? 1 : 0;
        Packed pkX, pkY;
        OzLines olX, olY;
        int64_t wx_words = 0, wy_words = 0;
        if (tc && nprod > 0) {
            if ((st = pack_prepare(sc, X, 0, xt, kprec, pkX))) return st;
            if ((st = pack_prepare(sc, Y, 1, yt, kprec, pkY))) return st;
            const int64_t *src[2] = {pkX.off + X->nnzb, pkY.off + Y->nnzb};
            if ((st = read_words(src, 2))) return st;
            const int64_t wx = g_host[0], wy = g_host[1];
            wx_words = wx;
            wy_words = wy;
            if ((st = pack_fill(sc, X, 0, xt, kprec, pkX, wx, &olX))) return st;
            if ((st = pack_fill(sc, Y, 1, yt, kprec, pkY, wy, &olY))) return st;
        }
        NumericArgs na{};
        na.n_items = OUT->nnzb;
        na.seg_ptr = seg;
        na.px = px;
        na.py = py;
        na.out_data = out;
        na.out_blk_off = OUT->blk_off;
        na.out_blk_rc = OUT->blk_rc;
        na.x_data = X->data; na.x_blk_off = X->blk_off; na.x_blk_rc = X->blk_rc; na.x_trans = xt;
        na.y_data = Y->data; na.y_blk_off = Y->blk_off; na.y_blk_rc = Y->blk_rc; na.y_trans = yt;
        na.alpha = alpha;
        na.beta = 0.0;
        na.dtype = C->dtype;
        na.prec = kprec;
        na.max_out_rows = OUT->max_bs_row; na.max_out_cols = OUT->max_bs_col;
        na.flush_every = opts.flush_every;
        na.x_pack = pkX.words; na.x_pack_off = pkX.off;
        na.y_pack = pkY.words; na.y_pack_off = pkY.off;
        na.x_exp = olX.exps; na.x_line0 = olX.line0;
        na.y_exp = olY.exps; na.y_line0 = olY.line0;
        if ((st = sc.get(&na.work_counter, 4))) return st;
        int32_t *item_order = nullptr;
        int64_t *n_marked = nullptr;
        bool uses_cores = false;
        if ((st = shape_order(sc, OUT->nnzb, OUT->blk_rc, OUT->h_row_bs, OUT->h_col_bs, &item_order, nullptr, nullptr,
                              opts.prec, &uses_cores, &n_marked)))
            return st;
        na.n_lane_items = n_marked;
        if (needs_plain(kprec) && uses_cores && nprod > 0) {
            const int np = split_pieces(opts.prec);
            float *xp = nullptr, *yp = nullptr;
            cudaError_t e;
            if ((st = sc.get(&xp, (size_t)X->data_len * np)) || (st = sc.get(&yp, (size_t)Y->data_len * np))) return st;
            e = launch_split_plain(X, opts.prec, xp, g_stream);
            if (e == cudaSuccess) e = launch_split_plain(Y, opts.prec, yp, g_stream);
            if ((st = cuda_check(e, "split pieces"))) return st;
            na.x_plain = xp;
            na.y_plain = yp;
        }
        na.item_order = item_order;
        apply_tuning(opts.prec, na);
        na.n_prod = nprod;
        na.x_nnzb = X->nnzb; na.y_nnzb = Y->nnzb;
        na.x_len = X->data_len; na.y_len = Y->data_len;
        na.out_len = OUT->data_len; na.old_len = 0;
        na.x_pack_words = pkX.words ? wx_words : 0; na.y_pack_words = pkY.words ? wy_words : 0;
        if ((st = cuda_check(launch_numeric(na, g_stream), "adjoint numeric"))) return st;
#ifdef BSM_DEBUG
        if (const uint32_t bits = numeric_debug_bits(g_stream))
            return set_error(BSM_ERR_CUDA, "debug bounds check of the adjoint kernel failed (bits " +
                                               std::to_string(bits) + ")");
#endif
    }
    return BSM_OK;
}

bsm_status bsm_get_counts(bsm_t C, int64_t *products, int64_t *filtered, double *useful_flop) {
    if (!C) return set_error(BSM_ERR_ARG, "C is NULL");
    if (products) *products = C->nprod;
    if (filtered) *filtered = C->nfiltered;
    if (useful_flop) *useful_flop = C->useful_flop;
    return BSM_OK;
}

bsm_status bsm_get_engine(bsm_t C, int32_t *engine) {
    if (!C || !engine) return set_error(BSM_ERR_ARG, "NULL argument");
    *engine = C->engine;
    return BSM_OK;
}

bsm_status bsm_get_timings(bsm_t C, double *ms) {
    if (!C || !ms) return set_error(BSM_ERR_ARG, "NULL argument");
    if (!C->timings_valid) return set_error(BSM_ERR_ARG, "no timings recorded (profiling off?)");
    for (int q = 0; q < BSM_T_COUNT; ++q) ms[q] = C->timings[q];
    return BSM_OK;
}

bsm_status bsm_get_products(bsm_t C, int64_t *nprod, int32_t *a_idx, int32_t *b_idx, int32_t *c_idx) {
    if (!C || !nprod) return set_error(BSM_ERR_ARG, "NULL argument");
    *nprod = C->pa ? C->nprod : 0;
    if (!a_idx && !b_idx && !c_idx) return BSM_OK;
    if (!C->pa) return set_error(BSM_ERR_ARG, "C holds no product list");
    cudaError_t e = cudaSuccess;
    const size_t bytes = sizeof(int32_t) * (size_t)C->nprod;
    if (a_idx && bytes) e = cudaMemcpyAsync(a_idx, C->pa, bytes, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess && b_idx && bytes) e = cudaMemcpyAsync(b_idx, C->pb, bytes, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess && c_idx && bytes) e = cudaMemcpyAsync(c_idx, C->pc, bytes, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    return cuda_check(e, "copy products");
}

bsm_status bsm_get_stacks(bsm_t C, int32_t *nshapes, int64_t *nprod, int32_t *shapes, int64_t *stack_ptr,
                          int64_t *triples) {
    if (!C || !nshapes || !nprod) return set_error(BSM_ERR_ARG, "NULL argument");
    *nshapes = C->nshapes;
    *nprod = C->triples ? C->nprod : 0;
    if (!shapes && !stack_ptr && !triples) return BSM_OK;
    cudaError_t e = cudaSuccess;
    if (shapes && C->nshapes)
        e = cudaMemcpyAsync(shapes, C->h_shapes.data(), sizeof(int32_t) * 3 * C->nshapes, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess && stack_ptr && C->stack_ptr)
        e = cudaMemcpyAsync(stack_ptr, C->stack_ptr, sizeof(int64_t) * (C->nshapes + 1), cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess && triples && C->triples && C->nprod)
        e = cudaMemcpyAsync(triples, C->triples, sizeof(int64_t) * 3 * C->nprod, cudaMemcpyDefault, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    return cuda_check(e, "copy stacks");
}

// --------------------------------------------------------------------------
// add
// --------------------------------------------------------------------------
bsm_status bsm_add(double a, bsm_t X, double b, bsm_t Y, bsm_t Z, double filter_eps, const bsm_opts *opts_in) {
    if (!X || !Y || !Z) return set_error(BSM_ERR_ARG, "NULL matrix");
    if (Z == X || Z == Y) return set_error(BSM_ERR_ARG, "Z must differ from X and Y");
    bsm_opts opts;
    bsm_status st = check_opts(opts_in, &opts);
    if (st) return st;
    if (X->dtype != Y->dtype || X->dtype != Z->dtype) return set_error(BSM_ERR_ARG, "X, Y and Z must share a dtype");
    if (X->nbr != Y->nbr || X->nbc != Y->nbc || X->nbr != Z->nbr || X->nbc != Z->nbc ||
        !same_vec(X->h_row_bs, Y->h_row_bs) || !same_vec(X->h_col_bs, Y->h_col_bs) ||
        !same_vec(X->h_row_bs, Z->h_row_bs) || !same_vec(X->h_col_bs, Z->h_col_bs))
        return set_error(BSM_ERR_BLOCKING, "X, Y and Z must share one blocking");
    if (!std::isfinite(a) || !std::isfinite(b) || std::isnan(filter_eps))
        return set_error(BSM_ERR_ARG, "a, b and eps must be finite");
    const bool no_sync = opts.no_sync != 0;
    const auto &pl = Z->plan;
    if (no_sync) {
        if (pl.kind != 2 || pl.A != X || pl.B != Y || pl.A_nnzb != X->nnzb || pl.B_nnzb != Y->nnzb ||
            pl.eps != filter_eps || !Z->add_xsrc || Z->add_a != a || Z->add_b != b)
            return set_error(BSM_ERR_ARG, "no_sync needs an earlier eager add of the same X, Y, a, b and eps into Z");
    } else if ((st = ensure_globals())) {
        return st;
    }
    if ((st = ensure_status(Z))) return st;
    Scratch sc;
    const int32_t nbr = X->nbr;
    const bool filt = filter_eps > 0.0;
    int64_t *ccnt, *celem, *zrow, *zelem, *stmp;
    if ((st = sc.get(&ccnt, nbr)) || (st = sc.get(&celem, nbr)) || (st = sc.get(&zrow, (size_t)nbr + 1)) ||
        (st = sc.get(&zelem, (size_t)nbr + 1)) || (st = sc.get(&stmp, scan_tmp_elems(nbr))))
        return st;
    cudaError_t e = cudaMemsetAsync(Z->status, 0, sizeof(int32_t), g_stream);
    if (e == cudaSuccess) e = launch_add_count(X, Y, ccnt, celem, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(ccnt, zrow, nbr, stmp, g_stream);
    if (e == cudaSuccess) e = launch_scan_i64(celem, zelem, nbr, stmp, g_stream);
    if ((st = cuda_check(e, "add count"))) return st;
    int64_t nnz, len;
    if (no_sync) {
        nnz = pl.u_nnzb;
        len = pl.u_len;
        PlanCheck pc{};
        pc.actual[0] = zrow + nbr; pc.expected[0] = nnz;
        pc.actual[1] = zelem + nbr; pc.expected[1] = len;
        pc.n = 2;
        if ((st = cuda_check(launch_check_plan(pc, Z->status, g_stream), "plan check"))) return st;
    } else {
        const int64_t *src[2] = {zrow + nbr, zelem + nbr};
        if ((st = read_words(src, 2))) return st;
        nnz = g_host[0];
        len = g_host[1];
    }
    // the union: straight into Z's storage when no filter follows in no-sync mode
    const bool direct = no_sync && !filt;
    int32_t *zc, *zrc;
    int64_t *zo, *xs, *ys;
    void *zd;
    const int32_t *stat = no_sync ? Z->status : nullptr;
    if (direct) {
        zc = Z->col_idx; zrc = Z->blk_rc; zo = Z->blk_off; xs = Z->add_xsrc; ys = Z->add_ysrc; zd = Z->data;
    } else {
        if ((st = sc.get(&zc, nnz)) || (st = sc.get(&zo, nnz)) || (st = sc.get(&zrc, nnz)) || (st = sc.get(&xs, nnz)) ||
            (st = sc.get(&ys, nnz)))
            return st;
        if ((st = dalloc(&zd, (size_t)len * esize(X->dtype)))) return st;
        sc.ptrs.push_back(zd);
        if (no_sync) {  // read by unguarded kernels of the filter even when the fill is skipped
            e = cudaMemsetAsync(zo, 0, sizeof(int64_t) * nnz, g_stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(zrc, 0, sizeof(int32_t) * nnz, g_stream);
            if ((st = cuda_check(e, "memset"))) return st;
        }
    }
    AddFill f{zrow, zelem, zc, zo, zrc, xs, ys};
    e = launch_add_fill(X, Y, f, stat, g_stream);
    if (e == cudaSuccess) e = launch_add_values(nnz, zo, zrc, xs, ys, a, X->data, b, Y->data, zd, X->dtype, stat, g_stream);
    if (e == cudaSuccess && direct) e = launch_copy_i64_if_ok(nbr + 1, zrow, Z->row_ptr, Z->status, g_stream);
    if ((st = cuda_check(e, "add fill"))) return st;
    if (direct) return BSM_OK;
    if (no_sync) {
        // filter the union (scratch) into Z's storage; its row pointers are
        // all zero (empty rows) unless the device check passed
        int64_t *urow;
        if ((st = sc.get(&urow, (size_t)nbr + 1))) return st;
        e = cudaMemsetAsync(urow, 0, sizeof(int64_t) * (nbr + 1), g_stream);
        if (e == cudaSuccess) e = launch_copy_i64_if_ok(nbr + 1, zrow, urow, Z->status, g_stream);
        if ((st = cuda_check(e, "union rows"))) return st;
        bsm_mat U;
        U.nbr = nbr; U.nbc = X->nbc; U.dtype = X->dtype; U.nnzb = nnz; U.data_len = len;
        U.row_bs = X->row_bs; U.col_bs = X->col_bs;
        U.row_ptr = urow; U.col_idx = zc; U.blk_off = zo; U.blk_rc = zrc; U.data = zd;
        U.add_xsrc = xs; U.add_ysrc = ys;
        return filter_compact(&U, filter_eps, true, Z->status, pl.nnzb, pl.len, Z);
    }
    free_results(Z);
    free_pattern(Z);
    Z->row_ptr = zrow; Z->col_idx = zc; Z->blk_off = zo; Z->blk_rc = zrc; Z->data = zd; Z->own_data = true;
    Z->nnzb = nnz; Z->data_len = len;
    Z->add_xsrc = xs; Z->add_ysrc = ys;
    Z->add_X = X; Z->add_Y = Y;
    Z->add_X_nnzb = X->nnzb; Z->add_Y_nnzb = Y->nnzb;
    Z->add_a = a; Z->add_b = b;
    for (void *p : {(void *)zrow, (void *)zc, (void *)zo, (void *)zrc, zd, (void *)xs, (void *)ys}) sc.release(p);
    if (filt && (st = filter_compact(Z, filter_eps, false, nullptr, 0, 0, nullptr))) return st;
    auto &P = Z->plan;
    P.kind = 2; P.A = X; P.B = Y; P.A_nnzb = X->nnzb; P.B_nnzb = Y->nnzb; P.eps = filter_eps;
    P.u_nnzb = nnz; P.u_len = len; P.nnzb = Z->nnzb; P.len = Z->data_len;
    return BSM_OK;
}

bsm_status bsm_add_backward(bsm_t Z, const void *dZ_data, bsm_t X, bsm_t Y, void *dX_data, void *dY_data) {
    if (!Z || !X || !Y) return set_error(BSM_ERR_ARG, "NULL matrix");
    if (!dX_data && !dY_data) return BSM_OK;
    if (!dZ_data && Z->data_len) return set_error(BSM_ERR_ARG, "dZ_data is NULL");
    if (Z->add_X != X || Z->add_Y != Y || Z->add_X_nnzb != X->nnzb || Z->add_Y_nnzb != Y->nnzb || !Z->add_xsrc)
        return set_error(BSM_ERR_ARG, "Z does not hold the provenance of an add of these X and Y");
    const size_t es = esize(Z->dtype);
    cudaError_t e = cudaSuccess;
    if (dX_data && X->data_len) e = cudaMemsetAsync(dX_data, 0, (size_t)X->data_len * es, g_stream);
    if (e == cudaSuccess && dY_data && Y->data_len) e = cudaMemsetAsync(dY_data, 0, (size_t)Y->data_len * es, g_stream);
    if (e == cudaSuccess)
        e = launch_add_backward(Z->nnzb, Z->blk_off, Z->blk_rc, Z->add_xsrc, Z->add_ysrc, Z->add_a, Z->add_b, dZ_data,
                                dX_data, dY_data, Z->dtype, g_stream);
    return cuda_check(e, "add backward");
}

bsm_status bsm_set_tuning(int32_t prec, int32_t param, int32_t value) {
    if (prec < BSM_P_FP64 || prec > BSM_P_TF32x3_PANEL) return set_error(BSM_ERR_ARG, "prec out of range");
    if (param < 0 || param >= BSM_TUNE_COUNT) return set_error(BSM_ERR_ARG, "unknown tuning parameter");
    int lo, hi;
    tune_range(prec, param, &lo, &hi);
    if (lo > hi) return set_error(BSM_ERR_ARG, "this precision has no such tuning parameter");
    if (value != -1 && (value < lo || value > hi)) return set_error(BSM_ERR_ARG, "tuning value out of range");
    if (param == BSM_TUNE_CTA_WARPS && value == 3) return set_error(BSM_ERR_ARG, "warps per CTA must be 2 or 4");
    if (param == BSM_TUNE_SCHED_TILE && value > 0 && value < 8)
        return set_error(BSM_ERR_ARG, "schedule tile must be 0 or 8..4096");
    tune_of(prec)[param] = value;
    return BSM_OK;
}

bsm_status bsm_get_tuning(int32_t prec, int32_t param, int32_t *value) {
    if (!value) return set_error(BSM_ERR_ARG, "value is NULL");
    if (prec < BSM_P_FP64 || prec > BSM_P_TF32x3_PANEL) return set_error(BSM_ERR_ARG, "prec out of range");
    if (param < 0 || param >= BSM_TUNE_COUNT) return set_error(BSM_ERR_ARG, "unknown tuning parameter");
    *value = tune_of(prec)[param];
    return BSM_OK;
}

bsm_status bsm_get_launch_config(bsm_t C, int32_t *cfg) {
    if (!C || !cfg) return set_error(BSM_ERR_ARG, "NULL argument");
    for (int q = 0; q < 6; ++q) cfg[q] = C->launch_cfg[q];
    return BSM_OK;
}

bsm_status bsm_set_variant(int32_t prec, int32_t m, int32_t n, int32_t variant) {
    if (prec < BSM_P_FP64 || prec > BSM_P_OZAKI || m < 1 || m > kMaxBlockDim || n < 1 || n > kMaxBlockDim ||
        variant < -1 || variant > 1)
        return set_error(BSM_ERR_ARG, "bsm_set_variant: argument out of range");
    variant_of(prec, m, n);  // initialises the table
    g_variant[prec][m][n] = (int8_t)variant;
    return BSM_OK;
}

bsm_status bsm_get_variant(int32_t prec, int32_t m, int32_t n, int32_t *variant) {
    if (!variant || prec < BSM_P_FP64 || prec > BSM_P_OZAKI || m < 1 || m > kMaxBlockDim || n < 1 || n > kMaxBlockDim)
        return set_error(BSM_ERR_ARG, "bsm_get_variant: argument out of range");
    *variant = variant_of(prec, m, n);
    return BSM_OK;
}

bsm_status bsm_get_status(bsm_t X, int32_t *status) {
    if (!X || !status) return set_error(BSM_ERR_ARG, "NULL argument");
    *status = 0;
    if (!X->status) return BSM_OK;
    cudaError_t e = cudaMemcpyAsync(g_host, X->status, sizeof(int32_t), cudaMemcpyDeviceToHost, g_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_stream);
    if (e != cudaSuccess) return cuda_check(e, "read status");
    *status = *reinterpret_cast<int32_t *>(g_host);
    if (*status & DEV_ERR_CAPACITY)
        return set_error(BSM_ERR_CAPACITY, "the last no-sync call found sizes different from its eager call");
    return BSM_OK;
}

bsm_status bsm_borrow_data(bsm_t X, void *dptr) {
    if (!X) return set_error(BSM_ERR_ARG, "X is NULL");
    if (!dptr && X->data_len) return set_error(BSM_ERR_ARG, "dptr is NULL");
    if (dptr) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, dptr) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return set_error(BSM_ERR_ARG, "bsm_borrow_data needs a device pointer");
        }
    }
    if (X->own_data) dfree(X->data);
    X->data = dptr;
    X->own_data = false;
    X->norms_valid = false;
    return BSM_OK;
}

}  // extern "C"
