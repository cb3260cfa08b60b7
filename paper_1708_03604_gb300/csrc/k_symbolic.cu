// Symbolic phase of the block-sparse multiply: block norms, the filtered
// product count per C block row, the C pattern and the product list, and the
// stack (batch) bucketing by block shape.  All integer work is exact; the
// only floating point here is the FP64 block norm and the FP64 product of
// two norms compared with the filter threshold (on-the-fly filtering of
// DBCSR, Bethune et al. 2017 §2).
#include <cuda_runtime.h>

#include <algorithm>

#include "bsm_internal.cuh"

namespace bsm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive scan of a per-thread value across the CTA; returns the thread's
// exclusive prefix and writes the CTA total to *total.  `wtmp` holds 32
// entries of shared scratch.  All threads must call it.
template <typename T>
__device__ T block_exscan(T v, T *wtmp, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) wtmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? wtmp[lane] : T(0);
        w = warp_incl_scan(w);
        if (lane < nw) wtmp[lane] = w;
    }
    __syncthreads();
    T base = warp > 0 ? wtmp[warp - 1] : T(0);
    *total = wtmp[nw - 1];
    __syncthreads();
    return base + incl - v;
}

// In-place exclusive scan of arr[0..L) in shared memory; returns the total.
__device__ int32_t block_exscan_array(int32_t *arr, int L, int32_t *wtmp) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (L + nt - 1) / nt;
    const int beg = min(L, tid * per), end = min(L, beg + per);
    int32_t s = 0;
    for (int q = beg; q < end; ++q) s += arr[q];
    int32_t total;
    int32_t run = block_exscan<int32_t>(s, wtmp, &total);
    for (int q = beg; q < end; ++q) {
        int32_t v = arr[q];
        arr[q] = run;
        run += v;
    }
    __syncthreads();
    return total;
}

// ------------------------------------------------------------- block shapes
__global__ void k_blk_rc(int32_t nbr, const int32_t *row_bs, const int32_t *col_bs,
                         const int64_t *row_ptr, const int32_t *col_idx, int32_t *rc) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nbr; i += nwarp) {
        const int32_t m = row_bs[i];
        for (int64_t b = row_ptr[i] + lane; b < row_ptr[i + 1]; b += 32)
            rc[b] = (m << 16) | col_bs[col_idx[b]];
    }
}

// ------------------------------------------------------------- block norms
// One thread per block: the fma chain runs over the block's elements in
// row-major order from +0.0, then an IEEE square root, so the value is
// bit-identical to any other evaluation in that order.
template <typename T>
__global__ void k_block_norms(int64_t nnzb, const int64_t *blk_off, const int32_t *blk_rc,
                              const T *data, double *out) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnzb;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rc = blk_rc[b];
        const int64_t len = (int64_t)rc_rows(rc) * rc_cols(rc);
        const T *x = data + blk_off[b];
        double s = 0.0;
        for (int64_t e = 0; e < len; ++e) {
            const double v = (double)__ldg(x + e);
            s = __fma_rn(v, v, s);
        }
        out[b] = __dsqrt_rn(s);
    }
}

// ------------------------------------------------------------- scan (int64)
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__global__ void k_scan_tile_sums(const int64_t *in, int64_t n, int64_t *sums) {
    __shared__ int64_t wtmp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = base + (int64_t)q * kThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) wtmp[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += wtmp[w];
        sums[blockIdx.x] = t;
    }
}

// one CTA: exclusive scan of sums[0..nt) in place, sums[nt] = total
__global__ void k_scan_sums(int64_t *sums, int64_t nt) {
    __shared__ int64_t wtmp[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nt; base += kScanTile) {
        int64_t v[kScanItems];
        int64_t s = 0;
        for (int q = 0; q < kScanItems; ++q) {
            const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
            v[q] = idx < nt ? sums[idx] : 0;
            s += v[q];
        }
        int64_t total;
        int64_t run = block_exscan<int64_t>(s, wtmp, &total) + carry;
        for (int q = 0; q < kScanItems; ++q) {
            const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
            if (idx < nt) sums[idx] = run;
            run += v[q];
        }
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nt] = carry;
}

__global__ void k_scan_tiles(const int64_t *in, int64_t *out, int64_t n, const int64_t *sums,
                             int64_t nt) {
    __shared__ int64_t wtmp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
        v[q] = idx < n ? in[idx] : 0;
        s += v[q];
    }
    int64_t total;
    int64_t run = block_exscan<int64_t>(s, wtmp, &total) + sums[blockIdx.x];
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
        if (idx < n) out[idx] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[nt];
}

// ------------------------------------------------------------- symbolic count
__device__ __forceinline__ bool keep_product(const SymbolicArgs &a, double na, int64_t b) {
    return !a.use_filter || (__dmul_rn(na, a.b_norm[b]) > a.eps);
}

__global__ void __launch_bounds__(kThreads) k_sym_count(SymbolicArgs a, int64_t *prod_cnt,
                                                        int64_t *ccol_cnt, int64_t *celem_cnt,
                                                        uint32_t *bitmaps,
                                                        unsigned long long *totals) {
    extern __shared__ uint32_t bm[];
    __shared__ long long red[5][32];
    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nw = a.nwords;
    for (int w = tid; w < nw; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    long long cnt = 0, filt = 0, nk = 0;
    const int64_t a_end = a.a_row_ptr[i + 1];
    for (int64_t ai = a.a_row_ptr[i] + warp; ai < a_end; ai += nwarps) {
        const int32_t k = a.a_col_idx[ai];
        const int32_t kd = a.a_col_bs[k];
        const double na = a.use_filter ? a.a_norm[ai] : 0.0;
        const int64_t b_end = a.b_row_ptr[k + 1];
        for (int64_t b = a.b_row_ptr[k] + lane; b < b_end; b += 32) {
            const int32_t j = a.b_col_idx[b];
            if (keep_product(a, na, b)) {
                atomicOr(&bm[j >> 5], 1u << (j & 31));
                cnt++;
                nk += (long long)a.b_col_bs[j] * kd;
            } else {
                filt++;
            }
        }
    }
    if (a.o_row_ptr) {
        for (int64_t c = a.o_row_ptr[i] + tid; c < a.o_row_ptr[i + 1]; c += blockDim.x) {
            const int32_t j = a.o_col_idx[c];
            atomicOr(&bm[j >> 5], 1u << (j & 31));
        }
    }
    __syncthreads();
    long long ncol = 0, wsum = 0;
    for (int w = tid; w < nw; w += blockDim.x) {
        uint32_t bits = bm[w];
        bitmaps[(int64_t)i * nw + w] = bits;
        ncol += __popc(bits);
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            wsum += a.b_col_bs[w * 32 + bit];
        }
    }
    long long v[5] = {cnt, filt, nk, ncol, wsum};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        long long s = warp_sum(v[q]);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (tid == 0) {
        long long t[5] = {0, 0, 0, 0, 0};
        for (int q = 0; q < 5; ++q)
            for (int w = 0; w < nwarps; ++w) t[q] += red[q][w];
        const int64_t m = a.a_row_bs[i];
        prod_cnt[i] = t[0];
        ccol_cnt[i] = t[3];
        celem_cnt[i] = m * t[4];
        if (t[1]) atomicAdd(&totals[0], (unsigned long long)t[1]);
        if (t[2]) atomicAdd(&totals[1], (unsigned long long)(m * t[2]));
        atomicMax(&totals[2], (unsigned long long)t[3]);
    }
}

// ------------------------------------------------------------- symbolic fill
__device__ __forceinline__ int32_t col_rank(const uint32_t *bm, const int32_t *wpre, int32_t j) {
    const uint32_t w = bm[j >> 5];
    return wpre[j >> 5] + __popc(w & ((1u << (j & 31)) - 1u));
}

__global__ void __launch_bounds__(kThreads) k_sym_fill(SymbolicArgs a, const uint32_t *bitmaps,
                                                       FillOut o) {
    extern __shared__ uint32_t smem[];
    __shared__ int32_t wtmp[32];
    if (a.status && *a.status != 0) return;
    const int nw = a.nwords;
    uint32_t *bm = smem;
    int32_t *wpre = reinterpret_cast<int32_t *>(smem + nw);
    int32_t *cnt = wpre + nw;
    const int i = o.row0 + blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t crow = o.crow_ptr[i];
    const int32_t ccnt = (int32_t)(o.crow_ptr[i + 1] - crow);
    const int64_t prow = o.prod_ptr[i] - o.prod_base;
    const int32_t m = a.a_row_bs[i];

    for (int w = tid; w < nw; w += blockDim.x) {
        const uint32_t bits = bitmaps[(int64_t)i * nw + w];
        bm[w] = bits;
        wpre[w] = __popc(bits);
    }
    __syncthreads();
    block_exscan_array(wpre, nw, wtmp);

    // C columns in ascending order, and their widths for the element offsets
    for (int w = tid; w < nw; w += blockDim.x) {
        uint32_t bits = bm[w];
        int32_t r = wpre[w];
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            const int32_t j = w * 32 + bit;
            o.c_col_idx[crow + r] = j;
            cnt[r] = a.b_col_bs[j];
            r++;
        }
    }
    __syncthreads();
    block_exscan_array(cnt, ccnt, wtmp);
    const int64_t ebase = o.celem_ptr[i];
    for (int32_t r = tid; r < ccnt; r += blockDim.x) {
        const int32_t j = o.c_col_idx[crow + r];
        const int32_t n = a.b_col_bs[j];
        o.c_blk_off[crow + r] = ebase + (int64_t)m * cnt[r];
        o.c_blk_rc[crow + r] = (m << 16) | n;
        if (o.old_off) o.old_off[crow + r] = -1;
    }
    __syncthreads();
    if (o.old_off) {
        for (int64_t c = a.o_row_ptr[i] + tid; c < a.o_row_ptr[i + 1]; c += blockDim.x) {
            const int32_t j = a.o_col_idx[c];
            o.old_off[crow + col_rank(bm, wpre, j)] = a.o_blk_off[c];
        }
    }
    // Products per C block.  The row's A blocks are cut into o.nchunk
    // contiguous chunks, one per warp; wc[c][r] counts chunk c's products for
    // C column rank r.  Scanning over r (then over c) gives every chunk its own
    // cursor per C block, so each warp scatters its chunk in ascending k
    // without waiting for the others: chunk c's products of a C block all
    // precede chunk c+1's.
    int32_t *wc = cnt + o.max_ccnt;  // [nchunk][max_ccnt]
    const int nchunk = o.nchunk;
    for (int32_t r = tid; r < ccnt; r += blockDim.x)
        for (int c = 0; c < nchunk; ++c) wc[c * o.max_ccnt + r] = 0;
    __syncthreads();
    const int64_t a_beg = a.a_row_ptr[i], a_end = a.a_row_ptr[i + 1];
    const int64_t per = (a_end - a_beg + nchunk - 1) / nchunk;
    const int64_t c_beg = a_beg + (int64_t)warp * per, c_end = min(a_end, c_beg + per);
    int32_t *my = wc + warp * o.max_ccnt;
    if (warp < nchunk) {
        for (int64_t ai = c_beg; ai < c_end; ++ai) {
            const int32_t k = a.a_col_idx[ai];
            const double na = a.use_filter ? a.a_norm[ai] : 0.0;
            for (int64_t b = a.b_row_ptr[k] + lane; b < a.b_row_ptr[k + 1]; b += 32)
                if (keep_product(a, na, b)) my[col_rank(bm, wpre, a.b_col_idx[b])]++;
            __syncwarp();
        }
    }
    __syncthreads();
    // totals per C block, their scan, then the per-chunk cursors
    for (int32_t r = tid; r < ccnt; r += blockDim.x) {
        int32_t t = 0;
        for (int c = 0; c < nchunk; ++c) t += wc[c * o.max_ccnt + r];
        cnt[r] = t;
    }
    __syncthreads();
    block_exscan_array(cnt, ccnt, wtmp);
    for (int32_t r = tid; r < ccnt; r += blockDim.x) {
        o.cptr[crow + r] = prow + cnt[r];
        int32_t run = cnt[r];
        for (int c = 0; c < nchunk; ++c) {
            const int32_t v = wc[c * o.max_ccnt + r];
            wc[c * o.max_ccnt + r] = run;
            run += v;
        }
    }
    __syncthreads();
    // scatter: inside one A block the target columns j are distinct, so the
    // lanes' cursor increments do not collide
    if (warp < nchunk) {
        for (int64_t ai = c_beg; ai < c_end; ++ai) {
            const int32_t k = a.a_col_idx[ai];
            const double na = a.use_filter ? a.a_norm[ai] : 0.0;
            for (int64_t b = a.b_row_ptr[k] + lane; b < a.b_row_ptr[k + 1]; b += 32) {
                if (keep_product(a, na, b)) {
                    const int32_t r = col_rank(bm, wpre, a.b_col_idx[b]);
                    const int32_t pos = my[r]++;
                    o.pa[prow + pos] = (int32_t)ai;
                    o.pb[prow + pos] = (int32_t)b;
                    o.pc[prow + pos] = (int32_t)(crow + r);
                }
            }
            __syncwarp();
        }
    }
}

// Fill through B's columns.  Same outputs as k_sym_fill, but every C block
// (i, j) is built by walking B's column j (B transposed: ascending k) against
// a shared-memory map k -> A block of row i, so its products come out in
// ascending k already and are written contiguously (coalesced) instead of
// scattered across the row's C blocks.
__global__ void __launch_bounds__(kThreads) k_sym_fill_cols(SymbolicArgs a, const uint32_t *bitmaps, FillOut o,
                                                            const int64_t *bt_ptr, const int32_t *bt_k,
                                                            const int32_t *bt_b) {
    extern __shared__ uint32_t smem[];
    __shared__ int32_t wtmp[32];
    if (a.status && *a.status != 0) return;
    const int nw = a.nwords;
    uint32_t *bm = smem;
    int32_t *wpre = reinterpret_cast<int32_t *>(smem + nw);
    int32_t *cnt = wpre + nw;
    int32_t *amap = cnt + o.max_ccnt;  // [nbk]: A block of row i in column k, or -1
    const int i = o.row0 + blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int64_t crow = o.crow_ptr[i];
    const int32_t ccnt = (int32_t)(o.crow_ptr[i + 1] - crow);
    const int64_t prow = o.prod_ptr[i] - o.prod_base;
    const int32_t m = a.a_row_bs[i];

    for (int w = tid; w < nw; w += blockDim.x) {
        const uint32_t bits = bitmaps[(int64_t)i * nw + w];
        bm[w] = bits;
        wpre[w] = __popc(bits);
    }
    for (int32_t k = tid; k < a.nbk; k += blockDim.x) amap[k] = -1;
    __syncthreads();
    block_exscan_array(wpre, nw, wtmp);
    const int64_t a_beg = a.a_row_ptr[i], a_end = a.a_row_ptr[i + 1];
    for (int64_t ai = a_beg + tid; ai < a_end; ai += blockDim.x) amap[a.a_col_idx[ai]] = (int32_t)ai;
    // C columns in ascending order, and their widths for the element offsets
    for (int w = tid; w < nw; w += blockDim.x) {
        uint32_t bits = bm[w];
        int32_t r = wpre[w];
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            const int32_t j = w * 32 + bit;
            o.c_col_idx[crow + r] = j;
            cnt[r] = a.b_col_bs[j];
            r++;
        }
    }
    __syncthreads();
    block_exscan_array(cnt, ccnt, wtmp);
    const int64_t ebase = o.celem_ptr[i];
    for (int32_t r = tid; r < ccnt; r += blockDim.x) {
        const int32_t j = o.c_col_idx[crow + r];
        const int32_t n = a.b_col_bs[j];
        o.c_blk_off[crow + r] = ebase + (int64_t)m * cnt[r];
        o.c_blk_rc[crow + r] = (m << 16) | n;
        if (o.old_off) o.old_off[crow + r] = -1;
    }
    __syncthreads();
    if (o.old_off) {
        for (int64_t c = a.o_row_ptr[i] + tid; c < a.o_row_ptr[i + 1]; c += blockDim.x) {
            const int32_t j = a.o_col_idx[c];
            o.old_off[crow + col_rank(bm, wpre, j)] = a.o_blk_off[c];
        }
    }
    // pass 1: kept products per C block (one warp per C block)
    const unsigned lt = (1u << lane) - 1u;
    for (int32_t r = warp; r < ccnt; r += nwarps) {
        const int32_t j = o.c_col_idx[crow + r];
        const int64_t cb = bt_ptr[j], ce = bt_ptr[j + 1];
        int32_t total = 0;
        for (int64_t e0 = cb; e0 < ce; e0 += 32) {
            const int64_t e = e0 + lane;
            bool keep = false;
            if (e < ce) {
                const int32_t ai = amap[bt_k[e]];
                if (ai >= 0) keep = !a.use_filter || __dmul_rn(a.a_norm[ai], a.b_norm[bt_b[e]]) > a.eps;
            }
            total += __popc(__ballot_sync(0xffffffffu, keep));
        }
        if (lane == 0) cnt[r] = total;
    }
    __syncthreads();
    block_exscan_array(cnt, ccnt, wtmp);
    for (int32_t r = tid; r < ccnt; r += blockDim.x) o.cptr[crow + r] = prow + cnt[r];
    // pass 2: write each C block's products contiguously, ascending k
    for (int32_t r = warp; r < ccnt; r += nwarps) {
        const int32_t j = o.c_col_idx[crow + r];
        const int64_t cb = bt_ptr[j], ce = bt_ptr[j + 1];
        int64_t cur = prow + cnt[r];
        for (int64_t e0 = cb; e0 < ce; e0 += 32) {
            const int64_t e = e0 + lane;
            bool keep = false;
            int32_t ai = -1, bi = -1;
            if (e < ce) {
                ai = amap[bt_k[e]];
                if (ai >= 0) {
                    bi = bt_b[e];
                    keep = !a.use_filter || __dmul_rn(a.a_norm[ai], a.b_norm[bi]) > a.eps;
                }
            }
            const unsigned msk = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int64_t pos = cur + __popc(msk & lt);
                o.pa[pos] = ai;
                o.pb[pos] = bi;
                o.pc[pos] = (int32_t)(crow + r);
            }
            cur += __popc(msk);
        }
    }
}

// block row of every block
__global__ void k_blk_rows(int32_t nbr, const int64_t *row_ptr, int32_t *rows) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nbr; i += nwarp)
        for (int64_t b = row_ptr[i] + lane; b < row_ptr[i + 1]; b += 32) rows[b] = (int32_t)i;
}

// ------------------------------------------------------------- radix sort
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kThreads * kRadixRounds;

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t *keys, int64_t n, int shift,
                                                          int64_t ntiles, int64_t *hist) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int q = 0; q < kRadixRounds; ++q) {
        const int64_t idx = base + (int64_t)q * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint32_t *kin, const int32_t *vin,
                                                             uint32_t *kout, int32_t *vout, int64_t n,
                                                             int shift, int64_t ntiles,
                                                             const int64_t *offs) {
    __shared__ int64_t run[256];
    __shared__ int32_t wcnt[kThreads / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    run[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int q = 0; q < kRadixRounds; ++q) {
        for (int w = 0; w < kThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t idx = base + (int64_t)q * kThreads + tid;
        const bool valid = idx < n;
        const uint32_t key = valid ? kin[idx] : 0u;
        const int d = valid ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
        int32_t add = 0;
        for (int w = 0; w < kThreads / 32; ++w) add += wcnt[w][tid];
        run[tid] += add;
        __syncthreads();
    }
}

// ------------------------------------------------------------- stacks
__global__ void k_product_shape_ids(int64_t nprod, const int32_t *pa, const int32_t *pb,
                                    const int32_t *a_rc, const int32_t *b_rc,
                                    const int32_t *size_index, int32_t ns, uint32_t *keys,
                                    int32_t *iota) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nprod;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t ra = a_rc[pa[p]], rb = b_rc[pb[p]];
        const int32_t mi = size_index[rc_rows(ra)], ki = size_index[rc_cols(ra)],
                      ni = size_index[rc_cols(rb)];
        keys[p] = (uint32_t)((mi * ns + ni) * ns + ki);
        iota[p] = (int32_t)p;
    }
}

// Stacks in two passes when there are at most kStackBins shapes: per tile of
// kRadixTile products a shared-memory histogram of the shape ids (pass 1),
// then each product's triple is written straight to its place -- the shape's
// start, plus the earlier tiles' products of that shape, plus its rank inside
// the tile (warp by warp, lane by lane) -- so every stack keeps the canonical
// (i, j, k) order, as the stable sort did (pass 2).
constexpr int kStackBins = 256;
__device__ __forceinline__ uint32_t product_shape(int64_t p, const int32_t *pa, const int32_t *pb,
                                                  const int32_t *a_rc, const int32_t *b_rc,
                                                  const int32_t *size_index, int32_t ns) {
    const int32_t ra = a_rc[pa[p]], rb = b_rc[pb[p]];
    return (uint32_t)((size_index[rc_rows(ra)] * ns + size_index[rc_cols(rb)]) * ns + size_index[rc_cols(ra)]);
}

__global__ void __launch_bounds__(kThreads) k_stack_count(int64_t nprod, const int32_t *pa, const int32_t *pb,
                                                          const int32_t *a_rc, const int32_t *b_rc,
                                                          const int32_t *size_index, int32_t ns, int32_t nbins,
                                                          int64_t ntiles, int64_t *tile_hist,
                                                          unsigned long long *counts) {
    __shared__ int32_t h[kStackBins];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int q = 0; q < kRadixRounds; ++q) {
        const int64_t p = base + (int64_t)q * kThreads + threadIdx.x;
        const bool valid = p < nprod;
        const int d = valid ? (int)product_shape(p, pa, pb, a_rc, b_rc, size_index, ns) : kStackBins;
        // one shared-memory atomic per distinct shape of the warp (one shape
        // per warp is the common case: products of a C block share m and n)
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        tile_hist[(int64_t)b * ntiles + blockIdx.x] = h[b];
        if (h[b]) atomicAdd(&counts[b], (unsigned long long)h[b]);
    }
}

__global__ void __launch_bounds__(kThreads) k_stack_scatter(int64_t nprod, const int32_t *pa, const int32_t *pb,
                                                            const int32_t *pc, const int32_t *a_rc,
                                                            const int32_t *b_rc, const int32_t *size_index,
                                                            int32_t ns, int32_t nbins, int64_t ntiles,
                                                            const int64_t *offs, const int64_t *a_off,
                                                            const int64_t *b_off, const int64_t *c_off,
                                                            int64_t *triples) {
    __shared__ int64_t run[kStackBins];
    __shared__ int32_t wcnt[kThreads / 32][kStackBins];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int b = tid; b < nbins; b += blockDim.x) run[b] = offs[(int64_t)b * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int q = 0; q < kRadixRounds; ++q) {
        for (int w = 0; w < kThreads / 32; ++w)
            for (int b = tid; b < nbins; b += blockDim.x) wcnt[w][b] = 0;
        __syncthreads();
        const int64_t p = base + (int64_t)q * kThreads + tid;
        const bool valid = p < nprod;
        const int d = valid ? (int)product_shape(p, pa, pb, a_rc, b_rc, size_index, ns) : kStackBins;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            triples[3 * pos + 0] = a_off[pa[p]];
            triples[3 * pos + 1] = b_off[pb[p]];
            triples[3 * pos + 2] = c_off[pc[p]];
        }
        __syncthreads();
        for (int b = tid; b < nbins; b += blockDim.x) {
            int32_t add = 0;
            for (int w = 0; w < kThreads / 32; ++w) add += wcnt[w][b];
            run[b] += add;
        }
        __syncthreads();
    }
}

__global__ void k_stack_triples(int64_t nprod, const int32_t *order, const int32_t *pa,
                                const int32_t *pb, const int32_t *pc, const int64_t *a_off,
                                const int64_t *b_off, const int64_t *c_off, int64_t *triples) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nprod;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = order[q];
        triples[3 * q + 0] = a_off[pa[p]];
        triples[3 * q + 1] = b_off[pb[p]];
        triples[3 * q + 2] = c_off[pc[p]];
    }
}

// One block shape: the stack is the product list itself, in order.  Each
// thread writes the triples of two consecutive products as three 16-byte
// stores (48 contiguous bytes, 16-byte aligned).
__global__ void k_stack_single(int64_t nprod, const int32_t *pa, const int32_t *pb, const int32_t *pc,
                               const int64_t *a_off, const int64_t *b_off, const int64_t *c_off,
                               int64_t *triples, int64_t *counts) {
    const int64_t npair = (nprod + 1) / 2;
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[0] = nprod;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npair;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = 2 * t;
        const int64_t a0 = a_off[pa[p]], b0 = b_off[pb[p]], c0 = c_off[pc[p]];
        if (p + 1 < nprod) {
            const int64_t a1 = a_off[pa[p + 1]], b1 = b_off[pb[p + 1]], c1 = c_off[pc[p + 1]];
            longlong2 *dst = reinterpret_cast<longlong2 *>(triples + 3 * p);
            dst[0] = make_longlong2(a0, b0);
            dst[1] = make_longlong2(c0, a1);
            dst[2] = make_longlong2(b1, c1);
        } else {
            triples[3 * p + 0] = a0;
            triples[3 * p + 1] = b0;
            triples[3 * p + 2] = c0;
        }
    }
}

// Counts of keys < nbins.  Few bins (shape ids): a per-CTA shared-memory
// histogram merged with one global atomic per bin and CTA; many bins (block
// indices): global atomics, which then rarely collide.
constexpr int kSmemBins = 4096;
__global__ void k_histogram(int64_t n, const uint32_t *keys, int64_t nbins, int64_t *counts) {
    __shared__ unsigned int h[kSmemBins];
    const bool local = nbins <= kSmemBins;
    if (local) {
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0u;
        __syncthreads();
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[p];
        if ((int64_t)k < nbins) {
            if (local) atomicAdd(&h[k], 1u);
            else atomicAdd(reinterpret_cast<unsigned long long *>(counts + k), 1ull);
        }
    }
    if (local) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (h[b]) atomicAdd(reinterpret_cast<unsigned long long *>(counts + b), (unsigned long long)h[b]);
    }
}

__global__ void k_gather_i32(int64_t n, const int32_t *order, const int32_t *src, int32_t *dst) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = src[order[p]];
}

__global__ void k_iota_keys(int64_t n, const int32_t *src, uint32_t *keys, int32_t *iota) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        keys[p] = (uint32_t)src[p];
        iota[p] = (int32_t)p;
    }
}

__global__ void k_check_plan(PlanCheck c, int32_t *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int q = 0; q < c.n; ++q)
            if (c.at_most[q] ? (*c.actual[q] > c.expected[q]) : (*c.actual[q] != c.expected[q]))
                atomicOr(status, (int32_t)DEV_ERR_CAPACITY);
    }
}

__global__ void k_copy_i64_if_ok(int64_t n, const int64_t *src, int64_t *dst, const int32_t *status) {
    if (*status != 0) return;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = src[p];
}

__global__ void k_class_keys(int64_t n, const int32_t *blk_rc, const int32_t *size_index, int32_t ns,
                             const int32_t *table, const int32_t *blk_row, const int32_t *row_rank, int32_t nbr,
                             const int32_t *blk_col, const int32_t *col_rank, int32_t tile, int32_t nct,
                             uint32_t *keys, int32_t *iota) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rc = blk_rc[p];
        uint32_t k = (uint32_t)table[size_index[rc_rows(rc)] * ns + size_index[rc_cols(rc)]];
        if (row_rank && col_rank && tile > 0) {
            // 2-D tiles of (row rank, column rank), tiles row by row
            const uint32_t nrt = (uint32_t)((nbr + tile - 1) / tile);
            k = (k * nrt + (uint32_t)(row_rank[blk_row[p]] / tile)) * (uint32_t)nct +
                (uint32_t)(col_rank[blk_col[p]] / tile);
        } else if (row_rank) {
            k = k * (uint32_t)nbr + (uint32_t)row_rank[blk_row[p]];
        }
        keys[p] = k;
        iota[p] = (int32_t)p;
    }
}

// lower bounds of two thresholds in sorted keys (one thread each)
__global__ void k_group_bounds(const uint32_t *keys, int64_t n, uint32_t thr0, uint32_t thr1, int64_t *out) {
    const int g = threadIdx.x;
    if (g >= 2) return;
    const uint32_t thr = g == 0 ? thr0 : thr1;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < thr) lo = mid + 1;
        else hi = mid;
    }
    out[g] = lo;
}

inline int grid_for(int64_t n, int threads = kThreads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

}  // namespace

// =================================================================== launchers
cudaError_t launch_group_bounds(const uint32_t *keys, int64_t n, uint32_t thr0, uint32_t thr1, int64_t *out,
                                cudaStream_t s) {
    k_group_bounds<<<1, 32, 0, s>>>(keys, n, thr0, thr1, out);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_blk_rc(const bsm_mat *X, int32_t *out_rc, cudaStream_t s) {
    if (X->nnzb == 0) return cudaSuccess;
    const int64_t warps = X->nbr;
    k_blk_rc<<<grid_for(warps * 32), kThreads, 0, s>>>(X->nbr, X->row_bs, X->col_bs, X->row_ptr,
                                                       X->col_idx, out_rc);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_block_norms(const bsm_mat *X, double *out, cudaStream_t s) {
    if (X->nnzb == 0) return cudaSuccess;
    const int g = grid_for(X->nnzb, 128);
    if (X->dtype == BSM_FP64)
        k_block_norms<double><<<g, 128, 0, s>>>(X->nnzb, X->blk_off, X->blk_rc,
                                                 static_cast<const double *>(X->data), out);
    else
        k_block_norms<float><<<g, 128, 0, s>>>(X->nnzb, X->blk_off, X->blk_rc,
                                                static_cast<const float *>(X->data), out);
    count_launch(1);
    return cudaGetLastError();
}

size_t scan_tmp_elems(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 2; }

cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    k_scan_tile_sums<<<(unsigned)nt, kThreads, 0, s>>>(in, n, tmp);
    k_scan_sums<<<1, kThreads, 0, s>>>(tmp, nt);
    k_scan_tiles<<<(unsigned)nt, kThreads, 0, s>>>(in, out, n, tmp, nt);
    count_launch(3);
    return cudaGetLastError();
}

cudaError_t launch_symbolic_count(const SymbolicArgs &a, int64_t *prod_cnt, int64_t *ccol_cnt,
                                  int64_t *celem_cnt, uint32_t *bitmaps, unsigned long long *totals,
                                  cudaStream_t s) {
    if (a.nbr == 0) return cudaSuccess;
    const size_t smem = (size_t)a.nwords * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_sym_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_sym_count<<<a.nbr, kThreads, smem, s>>>(a, prod_cnt, ccol_cnt, celem_cnt, bitmaps, totals);
    count_launch(1);
    return cudaGetLastError();
}

int64_t symbolic_fill_smem_bytes(int32_t nwords, int32_t max_ccnt, int nchunk) {
    return (2 * (int64_t)nwords + (int64_t)(nchunk + 1) * max_ccnt + 1) * (int64_t)sizeof(int32_t);
}

int64_t symbolic_fill_cols_smem_bytes(int32_t nwords, int32_t max_ccnt, int32_t nbk) {
    return (2 * (int64_t)nwords + (int64_t)max_ccnt + nbk + 1) * (int64_t)sizeof(int32_t);
}

cudaError_t launch_symbolic_fill_cols(const SymbolicArgs &a, const uint32_t *bitmaps, const FillOut &o,
                                      const int64_t *bt_ptr, const int32_t *bt_k, const int32_t *bt_b,
                                      cudaStream_t s, int32_t nrows) {
    if (nrows < 0) nrows = a.nbr - o.row0;
    if (nrows <= 0) return cudaSuccess;
    const int smem = (int)symbolic_fill_cols_smem_bytes(a.nwords, o.max_ccnt, a.nbk);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_sym_fill_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k_sym_fill_cols<<<nrows, kThreads, smem, s>>>(a, bitmaps, o, bt_ptr, bt_k, bt_b);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_blk_rows(const bsm_mat *X, int32_t *rows, cudaStream_t s) {
    if (X->nnzb == 0) return cudaSuccess;
    k_blk_rows<<<grid_for((int64_t)X->nbr * 32), kThreads, 0, s>>>(X->nbr, X->row_ptr, rows);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_symbolic_fill(const SymbolicArgs &a, const uint32_t *bitmaps, const FillOut &o,
                                 cudaStream_t s, int32_t nrows) {
    if (nrows < 0) nrows = a.nbr - o.row0;
    if (nrows <= 0) return cudaSuccess;
    const int smem = (int)symbolic_fill_smem_bytes(a.nwords, o.max_ccnt, o.nchunk);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_sym_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k_sym_fill<<<nrows, kThreads, smem, s>>>(a, bitmaps, o);
    count_launch(1);
    return cudaGetLastError();
}

size_t radix_tmp_elems(int64_t n) {
    const int64_t nt = (n + kRadixTile - 1) / kRadixTile;
    const int64_t h = 256 * (nt > 0 ? nt : 1);
    return (size_t)(2 * h + 1 + scan_tmp_elems(h) + 2);
}

cudaError_t launch_radix_sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, uint32_t *keys_alt,
                                    int32_t *vals_alt, uint32_t *keys_out, int32_t *vals_out, int64_t n,
                                    int key_bits, int64_t *tmp, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int passes = (key_bits + 7) / 8;
    if (passes < 1) passes = 1;
    const int64_t nt = (n + kRadixTile - 1) / kRadixTile;
    const int64_t h = 256 * nt;
    int64_t *hist = tmp, *offs = tmp + h, *stmp = tmp + 2 * h + 1;  // offs holds h+1 entries
    // ping-pong so that the last pass writes (keys_out, vals_out)
    const uint32_t *ki = keys_in;
    const int32_t *vi = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool last = (p == passes - 1);
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *ko = to_out ? keys_out : keys_alt;
        int32_t *vo = to_out ? vals_out : vals_alt;
        (void)last;
        k_radix_hist<<<(unsigned)nt, kThreads, 0, s>>>(ki, n, 8 * p, nt, hist);
        cudaError_t e = launch_scan_i64(hist, offs, h, stmp, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<(unsigned)nt, kThreads, 0, s>>>(ki, vi, ko, vo, n, 8 * p, nt, offs);
        count_launch(2);
        ki = ko;
        vi = vo;
    }
    return cudaGetLastError();
}

cudaError_t launch_product_shape_ids(int64_t nprod, const int32_t *pa, const int32_t *pb,
                                     const int32_t *a_blk_rc, const int32_t *b_blk_rc,
                                     const int32_t *size_index, int32_t ns, uint32_t *keys,
                                     int32_t *iota, cudaStream_t s) {
    if (nprod == 0) return cudaSuccess;
    k_product_shape_ids<<<grid_for(nprod), kThreads, 0, s>>>(nprod, pa, pb, a_blk_rc, b_blk_rc,
                                                             size_index, ns, keys, iota);
    count_launch(1);
    return cudaGetLastError();
}

int stack_max_bins() { return kStackBins; }

size_t stack_tmp_elems(int64_t nprod, int32_t nbins) {
    const int64_t nt = (nprod + kRadixTile - 1) / kRadixTile;
    const int64_t h = (int64_t)nbins * (nt > 0 ? nt : 1);
    return (size_t)(2 * h + 1 + scan_tmp_elems(h));
}

cudaError_t launch_stacks_direct(int64_t nprod, const int32_t *pa, const int32_t *pb, const int32_t *pc,
                                 const int32_t *a_rc, const int32_t *b_rc, const int32_t *size_index, int32_t ns,
                                 int32_t nbins, const int64_t *a_off, const int64_t *b_off, const int64_t *c_off,
                                 int64_t *triples, int64_t *counts, int64_t *tmp, cudaStream_t s) {
    if (nprod == 0 || nbins > kStackBins) return nprod == 0 ? cudaSuccess : cudaErrorInvalidValue;
    if (nbins == 1) {  // every product has the one shape: no counting, no scatter
        k_stack_single<<<grid_for((nprod + 1) / 2), kThreads, 0, s>>>(nprod, pa, pb, pc, a_off, b_off, c_off, triples,
                                                                       counts);
        count_launch(1);
        return cudaGetLastError();
    }
    const int64_t nt = (nprod + kRadixTile - 1) / kRadixTile;
    const int64_t h = (int64_t)nbins * nt;
    int64_t *hist = tmp, *offs = tmp + h, *stmp = tmp + 2 * h + 1;  // offs holds h+1 entries
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * nbins, s);
    if (e != cudaSuccess) return e;
    k_stack_count<<<(unsigned)nt, kThreads, 0, s>>>(nprod, pa, pb, a_rc, b_rc, size_index, ns, nbins, nt, hist,
                                                    reinterpret_cast<unsigned long long *>(counts));
    e = launch_scan_i64(hist, offs, h, stmp, s);
    if (e != cudaSuccess) return e;
    k_stack_scatter<<<(unsigned)nt, kThreads, 0, s>>>(nprod, pa, pb, pc, a_rc, b_rc, size_index, ns, nbins, nt,
                                                      offs, a_off, b_off, c_off, triples);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_stack_triples(int64_t nprod, const int32_t *order, const int32_t *pa, const int32_t *pb,
                                 const int32_t *pc, const int64_t *a_off, const int64_t *b_off,
                                 const int64_t *c_off, int64_t *triples, cudaStream_t s) {
    if (nprod == 0) return cudaSuccess;
    k_stack_triples<<<grid_for(nprod), kThreads, 0, s>>>(nprod, order, pa, pb, pc, a_off, b_off, c_off,
                                                         triples);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_histogram_u32(int64_t n, const uint32_t *keys, int64_t nbins, int64_t *counts,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)nbins, s);
    if (e != cudaSuccess || n == 0) return e;
    const int g = nbins <= kSmemBins ? std::min(grid_for(n), 152 * 4) : grid_for(n);
    k_histogram<<<g, kThreads, 0, s>>>(n, keys, nbins, counts);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_i32(int64_t n, const int32_t *order, const int32_t *src, int32_t *dst,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_gather_i32<<<grid_for(n), kThreads, 0, s>>>(n, order, src, dst);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_iota_keys(int64_t n, const int32_t *src, uint32_t *keys, int32_t *iota, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_iota_keys<<<grid_for(n), kThreads, 0, s>>>(n, src, keys, iota);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_check_plan(const PlanCheck &c, int32_t *status, cudaStream_t s) {
    k_check_plan<<<1, 32, 0, s>>>(c, status);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_i64_if_ok(int64_t n, const int64_t *src, int64_t *dst, const int32_t *status,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_copy_i64_if_ok<<<grid_for(n), kThreads, 0, s>>>(n, src, dst, status);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_class_keys(int64_t n, const int32_t *blk_rc, const int32_t *size_index, int32_t ns,
                              const int32_t *table, const int32_t *blk_row, const int32_t *row_rank, int32_t nbr,
                              const int32_t *blk_col, const int32_t *col_rank, int32_t tile, int32_t nct,
                              uint32_t *keys, int32_t *iota, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_class_keys<<<grid_for(n), kThreads, 0, s>>>(n, blk_rc, size_index, ns, table, blk_row, row_rank, nbr, blk_col,
                                                  col_rank, tile, nct, keys, iota);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace bsm
