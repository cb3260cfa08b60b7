// Numeric phase: every output block accumulates its list of small dense
// block products (the "batches" of DBCSR, Bethune et al. 2017 §2) in a fixed
// order, owned by exactly one warp -- the GPU analogue of the paper's static
// assignment of an A row-block to one thread, so no atomics touch C.
//
// One generic contraction serves the forward product and both adjoints:
//   out_q = alpha * sum_{p in seg(q)} X_p . Y_p  (+ beta * old_q)
// with X_p a logical R x T block and Y_p a logical T x S block, either stored
// as is or transposed:
//   forward  C_ij  = sum_k A_ik . B_kj          X = A,      Y = B
//   adjoint  dA_ik = sum_j dC_ij . B_kj^T       X = dC,     Y = B^T
//   adjoint  dB_kj = sum_i A_ik^T . dC_ij       X = A^T,    Y = dC
//
// Two arithmetic paths:
//   * CUDA cores: FP64 FMA for FP64 data (FP32 FMA with an FP64 running sum
//     for FP32 data); one lane owns a fixed set of output elements.
//   * Tensor cores (mma.sync m16n8k8 TF32 / m16n8k16 BF16): operands were
//     split beforehand into 2 or 3 narrow pieces (hi, lo[, lo2]) and packed
//     in mma fragment order; the cross products of the pieces accumulate in
//     FP32 inside the tensor core and are added into an FP64 accumulator
//     every `flush_every` block products.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bsm_internal.cuh"

namespace bsm {

namespace {

// ---------------------------------------------------------------------
// Debug builds (-DBSM_DEBUG): before an item is computed, its output block
// and every product's operand blocks are checked against the arrays' sizes;
// a violation sets a bit in g_dbg_bits and the item is skipped (no access
// outside the arrays, no trap).  Bits: 1 item or product range, 2 operand
// block index, 4 operand block extent, 8 operand shapes that do not chain,
// 16 packed-plane extent, 32 output block extent.
// ---------------------------------------------------------------------
#ifdef BSM_DEBUG
__device__ unsigned int g_dbg_bits;

__device__ uint32_t dbg_product_bits(const NumericArgs &a, int64_t p, int R, int S) {
    const int32_t ix = a.px[p], iy = a.py[p];
    if (ix < 0 || ix >= a.x_nnzb || iy < 0 || iy >= a.y_nnzb) return 2u;
    const int32_t xrc = a.x_blk_rc[ix], yrc = a.y_blk_rc[iy];
    const int64_t xo = a.x_blk_off[ix], yo = a.y_blk_off[iy];
    uint32_t bits = 0;
    if (xo < 0 || xo + (int64_t)rc_rows(xrc) * rc_cols(xrc) > a.x_len || yo < 0 ||
        yo + (int64_t)rc_rows(yrc) * rc_cols(yrc) > a.y_len)
        bits |= 4u;
    const int xr = a.x_trans ? rc_cols(xrc) : rc_rows(xrc), xt = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
    const int yt = a.y_trans ? rc_cols(yrc) : rc_rows(yrc), ys = a.y_trans ? rc_rows(yrc) : rc_cols(yrc);
    if (xr != R || ys != S || xt != yt) bits |= 8u;
    if (a.x_pack && (a.x_pack_off[ix] < 0 || a.x_pack_off[ix + 1] > a.x_pack_words)) bits |= 16u;
    if (a.y_pack && (a.y_pack_off[iy] < 0 || a.y_pack_off[iy + 1] > a.y_pack_words)) bits |= 16u;
    return bits;
}

__device__ uint32_t dbg_item_bits(const NumericArgs &a, int64_t q) {
    if (q < 0 || q >= a.n_items) return 1u;
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    if (p0 < 0 || p1 < p0 || p1 > a.n_prod) return 1u;
    const int32_t orc = a.out_blk_rc[q];
    const int64_t rs = (int64_t)rc_rows(orc) * rc_cols(orc);
    uint32_t bits = 0;
    if (a.out_blk_off[q] < 0 || a.out_blk_off[q] + rs > a.out_len) bits |= 32u;
    if (a.beta != 0.0 && a.old_off && a.old_off[q] >= 0 && a.old_off[q] + rs > a.old_len) bits |= 32u;
    return bits;
}

// all lanes of the warp: true when item q may be computed
__device__ bool dbg_item_ok_warp(const NumericArgs &a, int64_t q, int lane) {
    uint32_t bits = dbg_item_bits(a, q);
    if (bits == 0) {
        const int32_t orc = a.out_blk_rc[q];
        for (int64_t p = a.seg_ptr[q] + lane; p < a.seg_ptr[q + 1]; p += 32)
            bits |= dbg_product_bits(a, p, rc_rows(orc), rc_cols(orc));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
    if (bits && lane == 0) atomicOr(&g_dbg_bits, bits);
    return bits == 0;
}

// one lane: true when item q may be computed
__device__ bool dbg_item_ok_lane(const NumericArgs &a, int64_t q) {
    uint32_t bits = dbg_item_bits(a, q);
    if (bits == 0) {
        const int32_t orc = a.out_blk_rc[q];
        for (int64_t p = a.seg_ptr[q]; p < a.seg_ptr[q + 1]; ++p) bits |= dbg_product_bits(a, p, rc_rows(orc), rc_cols(orc));
    }
    if (bits) atomicOr(&g_dbg_bits, bits);
    return bits == 0;
}
#define BSM_DBG_WARP_SKIP(a, q, lane) \
    if (!dbg_item_ok_warp(a, q, lane)) continue;
#define BSM_DBG_LANE_OK(a, q) dbg_item_ok_lane(a, q)
#else
#define BSM_DBG_WARP_SKIP(a, q, lane)
#define BSM_DBG_LANE_OK(a, q) true
#endif

constexpr int kWarpsPerCta = 4;             // default warps per CTA
constexpr int kThreadsNum = kWarpsPerCta * 32;

// =====================================================================
// CUDA-core path
// =====================================================================
template <typename T, int Q>
__device__ __forceinline__ void cc_item(const NumericArgs &a, int64_t q, int lane) {
    const T *__restrict__ X = static_cast<const T *>(a.x_data);
    const T *__restrict__ Y = static_cast<const T *>(a.y_data);
    T *__restrict__ O = static_cast<T *>(a.out_data);
    const int32_t orc = a.out_blk_rc[q];
    const int R = rc_rows(orc), S = rc_cols(orc);
    const int RS = R * S;
    const int64_t out_off = a.out_blk_off[q];
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
    const T *OLD = static_cast<const T *>(a.old_data);
    const int F = a.flush_every > 0 ? a.flush_every : 1;

    for (int e0 = 0; e0 < RS; e0 += 32 * Q) {
        int rr[Q], ss[Q];
        double acc[Q];
        T acc_n[Q];
#pragma unroll
        for (int u = 0; u < Q; ++u) {
            const int e = e0 + lane + 32 * u;
            const bool v = e < RS;
            rr[u] = v ? e / S : 0;
            ss[u] = v ? e % S : 0;
            acc[u] = 0.0;
            acc_n[u] = T(0);
        }
        int since = 0;
        for (int64_t p = p0; p < p1; ++p) {
            const int32_t ix = a.px[p], iy = a.py[p];
            const T *xb = X + a.x_blk_off[ix];
            const T *yb = Y + a.y_blk_off[iy];
            const int32_t xrc = a.x_blk_rc[ix];
            const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
            const int xs_r = a.x_trans ? 1 : Tn, xs_t = a.x_trans ? R : 1;
            const int ys_t = a.y_trans ? 1 : S, ys_s = a.y_trans ? Tn : 1;
            int xo[Q], yo[Q];
#pragma unroll
            for (int u = 0; u < Q; ++u) {
                xo[u] = rr[u] * xs_r;
                yo[u] = ss[u] * ys_s;
            }
            for (int t = 0; t < Tn; ++t) {
#pragma unroll
                for (int u = 0; u < Q; ++u) {
                    const T xv = __ldg(xb + xo[u] + t * xs_t);
                    const T yv = __ldg(yb + t * ys_t + yo[u]);
                    acc_n[u] = fma(xv, yv, acc_n[u]);
                }
            }
            if constexpr (sizeof(T) == 4) {
                if (++since == F) {
                    since = 0;
#pragma unroll
                    for (int u = 0; u < Q; ++u) {
                        acc[u] += (double)acc_n[u];
                        acc_n[u] = T(0);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < Q; ++u) {
            const int e = e0 + lane + 32 * u;
            if (e < RS) {
                double v = (sizeof(T) == 8) ? (double)acc_n[u] : acc[u] + (double)acc_n[u];
                v = a.alpha * v;
                if (old >= 0) v = fma(a.beta, (double)OLD[old + e], v);
                O[out_off + e] = (T)v;
            }
        }
    }
}

// Builds of the CUDA-core kernel (the widest element-per-lane template sets
// the register count, and with it how many warps an SM holds):
//   kCcSmall  every output block has at most 16 elements: one element per lane
//             at most (72 registers)
//   kCcNarrow up to 9 elements per lane per pass, more passes over the
//             products for larger blocks (128 registers)
//   kCcWide   up to 24 elements per lane per pass (253 registers)
constexpr int kCcSmall = 0, kCcNarrow = 1, kCcWide = 2;
template <typename T, int BUILD>
__device__ __forceinline__ void cc_dispatch(const NumericArgs &a, int64_t q, int lane) {
    if constexpr (BUILD == kCcSmall) {
        cc_item<T, 1>(a, q, lane);
        return;
    }
    const int32_t orc = a.out_blk_rc[q];
    const int RS = rc_rows(orc) * rc_cols(orc);
    const int need = (RS + 31) >> 5;
    if constexpr (BUILD == kCcNarrow) {
        if (need <= 1) cc_item<T, 1>(a, q, lane);
        else if (need <= 2) cc_item<T, 2>(a, q, lane);
        else if (need <= 3) cc_item<T, 3>(a, q, lane);
        else if (need <= 4) cc_item<T, 4>(a, q, lane);
        else if (need <= 6) cc_item<T, 6>(a, q, lane);
        else cc_item<T, 9>(a, q, lane);
        return;
    }
    if (need <= 1) cc_item<T, 1>(a, q, lane);
    else if (need <= 2) cc_item<T, 2>(a, q, lane);
    else if (need <= 3) cc_item<T, 3>(a, q, lane);
    else if (need <= 4) cc_item<T, 4>(a, q, lane);
    else if (need <= 6) cc_item<T, 6>(a, q, lane);
    else if (need <= 8) cc_item<T, 8>(a, q, lane);
    else if (need <= 10) cc_item<T, 10>(a, q, lane);
    else if (need <= 12) cc_item<T, 12>(a, q, lane);
    else if (need <= 14) cc_item<T, 14>(a, q, lane);
    else if (need <= 17) cc_item<T, 17>(a, q, lane);
    else if (need <= 20) cc_item<T, 20>(a, q, lane);
    else cc_item<T, 24>(a, q, lane);
}

// Tiny output blocks (at most 16 elements): one lane owns a whole block, so a
// warp advances 32 blocks at once instead of leaving most lanes idle.
template <typename T>
__device__ __forceinline__ void cc_lane_item(const NumericArgs &a, int64_t q) {
    constexpr int L = 16;
    const T *__restrict__ X = static_cast<const T *>(a.x_data);
    const T *__restrict__ Y = static_cast<const T *>(a.y_data);
    T *__restrict__ O = static_cast<T *>(a.out_data);
    const int32_t orc = a.out_blk_rc[q];
    const int R = rc_rows(orc), S = rc_cols(orc);
    const int RS = R * S;
    const int64_t out_off = a.out_blk_off[q];
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
    double acc[L];
    T acc_n[L];
#pragma unroll
    for (int e = 0; e < L; ++e) {
        acc[e] = 0.0;
        acc_n[e] = T(0);
    }
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t ix = a.px[p], iy = a.py[p];
        const T *xb = X + a.x_blk_off[ix];
        const T *yb = Y + a.y_blk_off[iy];
        const int32_t xrc = a.x_blk_rc[ix];
        const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
        const int xs_r = a.x_trans ? 1 : Tn, xs_t = a.x_trans ? R : 1;
        const int ys_t = a.y_trans ? 1 : S, ys_s = a.y_trans ? Tn : 1;
        for (int t = 0; t < Tn; ++t) {
#pragma unroll
            for (int e = 0; e < L; ++e) {
                if (e < RS) {
                    const int r = e / S, c = e - r * S;
                    acc_n[e] = fma(__ldg(xb + r * xs_r + t * xs_t), __ldg(yb + t * ys_t + c * ys_s), acc_n[e]);
                }
            }
        }
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int e = 0; e < L; ++e) {
                acc[e] += (double)acc_n[e];
                acc_n[e] = T(0);
            }
        }
    }
    const T *OLD = static_cast<const T *>(a.old_data);
#pragma unroll
    for (int e = 0; e < L; ++e) {
        if (e < RS) {
            double v = (sizeof(T) == 8) ? (double)acc_n[e] : acc[e];
            v = a.alpha * v;
            if (old >= 0) v = fma(a.beta, (double)OLD[old + e], v);
            O[out_off + e] = (T)v;
        }
    }
}

// Fixed shapes of the lane-per-block mode: column t of the X block and row t
// of the Y block are loaded once per k and applied as a rank-1 update.
template <typename T, int R, int S>
__device__ __forceinline__ void cc_lane_fixed(const NumericArgs &a, int64_t q) {
    const T *__restrict__ X = static_cast<const T *>(a.x_data);
    const T *__restrict__ Y = static_cast<const T *>(a.y_data);
    T *__restrict__ O = static_cast<T *>(a.out_data);
    const int64_t out_off = a.out_blk_off[q];
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
    double acc[R][S];
    T acc_n[R][S];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < S; ++c) {
            acc[r][c] = 0.0;
            acc_n[r][c] = T(0);
        }
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t ix = a.px[p], iy = a.py[p];
        const T *xb = X + a.x_blk_off[ix];
        const T *yb = Y + a.y_blk_off[iy];
        const int32_t xrc = a.x_blk_rc[ix];
        const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
        const int xs_r = a.x_trans ? 1 : Tn, xs_t = a.x_trans ? R : 1;
        const int ys_t = a.y_trans ? 1 : S, ys_s = a.y_trans ? Tn : 1;
        for (int t = 0; t < Tn; ++t) {
            T xv[R], yv[S];
#pragma unroll
            for (int r = 0; r < R; ++r) xv[r] = __ldg(xb + r * xs_r + t * xs_t);
#pragma unroll
            for (int c = 0; c < S; ++c) yv[c] = __ldg(yb + t * ys_t + c * ys_s);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < S; ++c) acc_n[r][c] = fma(xv[r], yv[c], acc_n[r][c]);
        }
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    acc[r][c] += (double)acc_n[r][c];
                    acc_n[r][c] = T(0);
                }
        }
    }
    const T *OLD = static_cast<const T *>(a.old_data);
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < S; ++c) {
            const int e = r * S + c;
            double v = (sizeof(T) == 8) ? (double)acc_n[r][c] : acc[r][c];
            v = a.alpha * v;
            if (old >= 0) v = fma(a.beta, (double)OLD[old + e], v);
            O[out_off + e] = (T)v;
        }
}

template <typename T, int BUILD = kCcWide>
__device__ __forceinline__ void cc_lane_dispatch(const NumericArgs &a, int64_t q) {
    const int32_t orc = a.out_blk_rc[q];
    if constexpr (BUILD == kCcSmall) {
        switch ((rc_rows(orc) << 8) | rc_cols(orc)) {
            case 0x101: cc_lane_fixed<T, 1, 1>(a, q); break;
            case 0x104: cc_lane_fixed<T, 1, 4>(a, q); break;
            case 0x401: cc_lane_fixed<T, 4, 1>(a, q); break;
            case 0x404: cc_lane_fixed<T, 4, 4>(a, q); break;
            case 0x202: cc_lane_fixed<T, 2, 2>(a, q); break;
            default: cc_lane_item<T>(a, q); break;
        }
        return;
    }
    switch ((rc_rows(orc) << 8) | rc_cols(orc)) {
        case 0x101: cc_lane_fixed<T, 1, 1>(a, q); break;
        case 0x102: cc_lane_fixed<T, 1, 2>(a, q); break;
        case 0x201: cc_lane_fixed<T, 2, 1>(a, q); break;
        case 0x202: cc_lane_fixed<T, 2, 2>(a, q); break;
        case 0x104: cc_lane_fixed<T, 1, 4>(a, q); break;
        case 0x401: cc_lane_fixed<T, 4, 1>(a, q); break;
        case 0x204: cc_lane_fixed<T, 2, 4>(a, q); break;
        case 0x402: cc_lane_fixed<T, 4, 2>(a, q); break;
        case 0x404: cc_lane_fixed<T, 4, 4>(a, q); break;
        case 0x505: cc_lane_fixed<T, 5, 5>(a, q); break;
        case 0x606: cc_lane_fixed<T, 6, 6>(a, q); break;
        default: cc_lane_item<T>(a, q); break;
    }
}

template <typename T, int BUILD>
__global__ void __launch_bounds__(kThreadsNum) k_numeric_cc(NumericArgs a) {
    const int lane = threadIdx.x & 31;
    if (a.status && *a.status != 0) return;
    unsigned long long *ctr = a.work_counter;
    // items [0, n0): a warp each; items [n0, n_items): marked tiny blocks, 32 per ticket
    const int64_t n_lane = a.n_lane_items ? *a.n_lane_items : 0;
    const int64_t n0 = a.n_items - n_lane;
    const int64_t tickets = n0 + (n_lane + 31) / 32;
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= tickets) break;
        if (t < n0) {
            int64_t q = t;
            if (a.item_order) q = (int64_t)((uint32_t)a.item_order[q] & 0x7fffffffu);
            BSM_DBG_WARP_SKIP(a, q, lane)
            cc_dispatch<T, BUILD>(a, q, lane);
        } else {
            const int64_t idx = n0 + (t - n0) * 32 + lane;
            if (idx < a.n_items) {
                const int64_t q = (int64_t)((uint32_t)a.item_order[idx] & 0x7fffffffu);
                if (BSM_DBG_LANE_OK(a, q)) cc_lane_dispatch<T, BUILD>(a, q);
            }
        }
    }
}

// =====================================================================
// FP64 tensor-core path (BSM_P_FP64_DMMA): mma.sync m8n8k4 with FP64
// operands and accumulators.  Fragment layout of m8n8k4 (lane = 4 g + t4):
// A (8 x 4, row) holds X(g, t4); B (4 x 8, col) holds Y(t4, g); the
// accumulator holds D(g, 2 t4) and D(g, 2 t4 + 1).  One warp per output
// block; blocks of at least 8 x 8 elements run here, in passes of up to
// 3 x 3 tiles of 8 x 8 (24 x 24 elements), every block product in ascending
// k steps of 4 with zero padding past the block edges.  Smaller output
// blocks run the FP64 FMA code.
// =====================================================================
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

template <int MTC, int NTC>
__device__ __forceinline__ void dmma_pass(const NumericArgs &a, int64_t q, int lane, int mt0, int nt0) {
    const double *__restrict__ X = static_cast<const double *>(a.x_data);
    const double *__restrict__ Y = static_cast<const double *>(a.y_data);
    const int32_t orc = a.out_blk_rc[q];
    const int R = rc_rows(orc), S = rc_cols(orc);
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const int g = lane >> 2, t4 = lane & 3;
    double acc[MTC][NTC][2];
#pragma unroll
    for (int i = 0; i < MTC; ++i)
#pragma unroll
        for (int j = 0; j < NTC; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    // rows of X and columns of Y this lane loads (clamped reads are masked)
    int xr[MTC], ys[NTC];
    bool xv[MTC], yv[NTC];
#pragma unroll
    for (int i = 0; i < MTC; ++i) {
        xr[i] = (mt0 + i) * 8 + g;
        xv[i] = xr[i] < R;
    }
#pragma unroll
    for (int j = 0; j < NTC; ++j) {
        ys[j] = (nt0 + j) * 8 + g;
        yv[j] = ys[j] < S;
    }
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t ix = a.px[p], iy = a.py[p];
        const double *xb = X + a.x_blk_off[ix];
        const double *yb = Y + a.y_blk_off[iy];
        const int32_t xrc = a.x_blk_rc[ix];
        const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
        const int xs_r = a.x_trans ? 1 : Tn, xs_t = a.x_trans ? R : 1;
        const int ys_t = a.y_trans ? 1 : S, ys_s = a.y_trans ? Tn : 1;
        for (int t0 = 0; t0 < Tn; t0 += 4) {
            const int t = t0 + t4;
            const bool tv = t < Tn;
            double fa[MTC], fb[NTC];
#pragma unroll
            for (int i = 0; i < MTC; ++i) fa[i] = (tv && xv[i]) ? __ldg(xb + xr[i] * xs_r + t * xs_t) : 0.0;
#pragma unroll
            for (int j = 0; j < NTC; ++j) fb[j] = (tv && yv[j]) ? __ldg(yb + t * ys_t + ys[j] * ys_s) : 0.0;
#pragma unroll
            for (int i = 0; i < MTC; ++i)
#pragma unroll
                for (int j = 0; j < NTC; ++j) dmma(acc[i][j], fa[i], fb[j]);
        }
    }
    double *O = static_cast<double *>(a.out_data);
    const double *OLD = static_cast<const double *>(a.old_data);
    const int64_t out_off = a.out_blk_off[q];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
#pragma unroll
    for (int i = 0; i < MTC; ++i)
#pragma unroll
        for (int j = 0; j < NTC; ++j)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int r = (mt0 + i) * 8 + g, c = (nt0 + j) * 8 + 2 * t4 + v;
                if (r < R && c < S) {
                    const int64_t e = (int64_t)r * S + c;
                    double val = a.alpha * acc[i][j][v];
                    if (old >= 0) val = fma(a.beta, OLD[old + e], val);
                    O[out_off + e] = val;
                }
            }
}

__device__ __forceinline__ void dmma_item(const NumericArgs &a, int64_t q, int lane) {
    const int32_t orc = a.out_blk_rc[q];
    const int MT = (rc_rows(orc) + 7) >> 3, NT = (rc_cols(orc) + 7) >> 3;
    const int pm = a.pass_mt > 0 ? a.pass_mt : 3, pn = a.pass_nt > 0 ? a.pass_nt : 3;
    for (int mt0 = 0; mt0 < MT; mt0 += pm) {
        const int mtc = min(pm, MT - mt0);
        for (int nt0 = 0; nt0 < NT; nt0 += pn) {
            const int ntc = min(pn, NT - nt0);
            switch (mtc * 4 + ntc) {
                case 5: dmma_pass<1, 1>(a, q, lane, mt0, nt0); break;
                case 6: dmma_pass<1, 2>(a, q, lane, mt0, nt0); break;
                case 7: dmma_pass<1, 3>(a, q, lane, mt0, nt0); break;
                case 9: dmma_pass<2, 1>(a, q, lane, mt0, nt0); break;
                case 10: dmma_pass<2, 2>(a, q, lane, mt0, nt0); break;
                case 11: dmma_pass<2, 3>(a, q, lane, mt0, nt0); break;
                case 13: dmma_pass<3, 1>(a, q, lane, mt0, nt0); break;
                case 14: dmma_pass<3, 2>(a, q, lane, mt0, nt0); break;
                default: dmma_pass<3, 3>(a, q, lane, mt0, nt0); break;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreadsNum) k_numeric_dmma(NumericArgs a) {
    const int lane = threadIdx.x & 31;
    if (a.status && *a.status != 0) return;
    unsigned long long *ctr = a.work_counter;
    const int64_t n_lane = a.n_lane_items ? *a.n_lane_items : 0;
    const int64_t n0 = a.n_items - n_lane;
    const int64_t tickets = n0 + (n_lane + 31) / 32;
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= tickets) break;
        if (t < n0) {
            int64_t q = t;
            if (a.item_order) q = (int64_t)((uint32_t)a.item_order[q] & 0x7fffffffu);
            BSM_DBG_WARP_SKIP(a, q, lane)
            const int32_t orc = a.out_blk_rc[q];
            if (rc_rows(orc) >= 8 && rc_cols(orc) >= 8) dmma_item(a, q, lane);
            else cc_dispatch<double, kCcNarrow>(a, q, lane);
        } else {
            const int64_t idx = n0 + (t - n0) * 32 + lane;
            if (idx < a.n_items) {
                const int64_t q = (int64_t)((uint32_t)a.item_order[idx] & 0x7fffffffu);
                if (BSM_DBG_LANE_OK(a, q)) cc_lane_dispatch<double, kCcNarrow>(a, q);
            }
        }
    }
}

// =====================================================================
// Tensor-core split path
// =====================================================================
// Packed fragment planes.  For a logical R x T operand in role X (mma "A"
// operand) the tiles are (kt, mt) with MT = ceil(R/16), kt over K steps;
// for a logical T x S operand in role Y ("B" operand) tiles are (kt, nt)
// with NT = ceil(S/8).  Words per lane per tile:
//   prec      K step   X words   Y words
//   TF32x3       8        8         4      (hi[4] lo[4] | hi[2] lo[2])
//   BF16x3      16        8         4      (hi[4] lo[4] | hi[2] lo[2])
//   BF16x6      16       12         8      (p0[4] p1[4] p2[4] | p0[2] p1[2] p2[2] pad[2])
// Inside a tile the words are chunk-major: 16-byte chunk c of lane L at word
// c * 128 + 4 * L (X chunk = one piece, Y chunk = two pieces), so a 16-byte
// copy of the warp reads 512 contiguous bytes.
template <int PREC> struct PrecTraits;
template <> struct PrecTraits<BSM_P_TF32x3> { static constexpr int K = 8, XW = 8, YW = 4, NP = 2; };
template <> struct PrecTraits<BSM_P_BF16x3> { static constexpr int K = 16, XW = 8, YW = 4, NP = 2; };
template <> struct PrecTraits<BSM_P_BF16x6> { static constexpr int K = 16, XW = 12, YW = 8, NP = 3; };

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int PREC>
__device__ __forceinline__ void mma_piece(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    if constexpr (PREC == BSM_P_TF32x3) mma_tf32(d, a, b);
    else mma_bf16(d, a, b);
}

// Per-lane staging ring: every lane copies its own fragment words of the
// next (product, k-step) steps from global memory into its private slots of
// shared memory with cp.async and reads back only those words, so the ring
// needs no warp barrier -- only each lane's own cp.async.wait_group.  A stage
// is chunk-major like the packs (chunk c of lane L at word c * 128 + 4 * L):
// every 16-byte copy and read of the warp covers 512 contiguous bytes.
// Stages, and words per lane of a stage for passes of at most PM x PN tiles.
// A kernel instance compiled for smaller passes holds fewer accumulators and
// a smaller ring, so more warps fit on an SM.
template <int PREC, int PM = 2, int PN = 3> struct RingTraits {
    static constexpr int STAGES = PREC == BSM_P_BF16x6 ? 3 : 4;
    static constexpr int SW = PM * PrecTraits<PREC>::XW + PN * PrecTraits<PREC>::YW;
};

template <int PREC, int PM = 2, int PN = 3>
__host__ __device__ constexpr int ring_words_per_warp() {
    return RingTraits<PREC, PM, PN>::STAGES * 32 * RingTraits<PREC, PM, PN>::SW;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 16-byte asynchronous copy global -> shared, cached in L2 only (the staged
// fragment words are read once per warp)
__device__ __forceinline__ void cp_async16_cg(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// Compensated (Kahan) addition of b into the pair (hi, lo), value hi + lo:
// the low part lost by each addition is fed into the next one (4 FP32 adds;
// error below about 2u of the sum of |b|, u = 2^-24).
__device__ __forceinline__ void kahan_acc(float &hi, float &lo, float b) {
    const float y = __fadd_rn(b, lo);
    const float t = __fadd_rn(hi, y);
    lo = __fsub_rn(y, __fsub_rn(t, hi));
    hi = t;
}

// FP32 -> FP64 (exact).  Widening by integer bit operations instead of the
// conversion instruction was measured no faster on GB300: the FP64 additions,
// not the conversions, are what the FP64 running sum pays for.
__device__ __forceinline__ double widen(float f) { return (double)f; }

// The value of a compensated pair (hi, lo) plus a last partial sum b, in
// FP64: b is first added into the pair in FP32 (one more compensated step),
// then the pair is widened and added once.
__device__ __forceinline__ double pair_total(float hi, float lo, float b) {
    kahan_acc(hi, lo, b);
    return widen(hi) + widen(lo);
}

// One pass over a super tile of MTC x NTC (at most 2 x 3) fragment tiles
// starting at (mt0, nt0) of output block q: at most 32 x 24 output elements.
// FF: cross-product sum as a compensated float pair (Kahan after every |F| block
// products); otherwise an FP64 sum refreshed every F products.
template <int PREC, int MTC, int NTC, bool FF, int PM, int PN, bool DUAL>
__device__ __forceinline__ void tc_pass(const NumericArgs &a, int64_t q, int lane, int mt0, int nt0,
                                        uint32_t *ring) {
    using PT = PrecTraits<PREC>;
    using RT = RingTraits<PREC, PM, PN>;
    constexpr int ST = RT::STAGES, SW = RT::SW;
    const int32_t orc = a.out_blk_rc[q];
    const int R = rc_rows(orc), S = rc_cols(orc);
    const int MT = (R + 15) >> 4, NT = (S + 7) >> 3;
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const uint32_t *XP = static_cast<const uint32_t *>(a.x_pack);
    const uint32_t *YP = static_cast<const uint32_t *>(a.y_pack);
    // FP64 mode: flush_every > 0 products per FP64 add; compensated mode:
    // |flush_every| products per compensated addition (0 means 1)
    const int F = a.flush_every > 0 ? a.flush_every : (a.flush_every < 0 ? -a.flush_every : 1);
    uint32_t *myring = ring + 4 * lane;  // chunk c of stage st at myring + st * 32 * SW + 128 * c
    const uint32_t ring_s = smem_addr(myring);
    constexpr int XC = PT::XW / 4, YC = PT::YW / 4;  // chunks per tile

    // DUAL (1-row instances summing more than one block product in the tensor
    // core, F > 1): the piece products of a k-step alternate between two
    // accumulators (term t into acc if t is even, acc2 if odd), so that the
    // tensor core's chain of dependent MMAs on one tile is about half as long;
    // the two are added (FP32, to nearest) where the single one was read
    float acc[MTC][NTC][4], acc2[DUAL ? MTC : 1][DUAL ? NTC : 1][4];
    float shi[FF ? MTC : 1][FF ? NTC : 1][4], slo[FF ? MTC : 1][FF ? NTC : 1][4];
    double s64[FF ? 1 : MTC][FF ? 1 : NTC][4];
#pragma unroll
    for (int i = 0; i < MTC; ++i)
#pragma unroll
        for (int j = 0; j < NTC; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                acc[i][j][v] = 0.f;
                if constexpr (DUAL) acc2[i][j][v] = 0.f;
                if constexpr (FF) {
                    shi[i][j][v] = 0.f;
                    slo[i][j][v] = 0.f;
                } else {
                    s64[i][j][v] = 0.0;
                }
            }
    int since = 0;
    for (int64_t pb = p0; pb < p1; pb += 32) {
        const int nb = (int)min((int64_t)32, p1 - pb);
        // metadata of up to 32 products, one per lane
        int64_t mxo = 0, myo = 0;
        int mkt = 0;
        if (lane < nb) {
            const int32_t ix = a.px[pb + lane], iy = a.py[pb + lane];
            const int32_t xrc = a.x_blk_rc[ix];
            const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
            mxo = a.x_pack_off[ix];
            myo = a.y_pack_off[iy];
            mkt = (Tn + PT::K - 1) / PT::K;
        }
        int nsteps = mkt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nsteps += __shfl_xor_sync(0xffffffffu, nsteps, o);
        // producer cursor over the (product, k-step) sequence
        int pu = 0, pk = 0;
        int64_t pxo = __shfl_sync(0xffffffffu, mxo, 0), pyo = __shfl_sync(0xffffffffu, myo, 0);
        int pkt = __shfl_sync(0xffffffffu, mkt, 0);
        auto produce = [&](int st) {
            const uint32_t dst = ring_s + (uint32_t)(st * 32 * SW) * 4u;
#pragma unroll
            for (int i = 0; i < MTC; ++i) {
                if (mt0 + i < MT) {
                    const uint32_t *src = XP + pxo + (int64_t)(pk * MT + mt0 + i) * (32 * PT::XW) + 4 * lane;
#pragma unroll
                    for (int c = 0; c < XC; ++c) cp_async16_cg(dst + 512u * (i * XC + c), src + 128 * c);
                }
            }
#pragma unroll
            for (int j = 0; j < NTC; ++j) {
                if (nt0 + j < NT) {
                    const uint32_t *src = YP + pyo + (int64_t)(pk * NT + nt0 + j) * (32 * PT::YW) + 4 * lane;
#pragma unroll
                    for (int c = 0; c < YC; ++c) cp_async16_cg(dst + 512u * (MTC * XC + j * YC + c), src + 128 * c);
                }
            }
            if (++pk == pkt) {
                pk = 0;
                ++pu;
                const int src_lane = pu < nb ? pu : 0;
                pxo = __shfl_sync(0xffffffffu, mxo, src_lane);
                pyo = __shfl_sync(0xffffffffu, myo, src_lane);
                pkt = __shfl_sync(0xffffffffu, mkt, src_lane);
            }
        };
#pragma unroll
        for (int st = 0; st < ST - 1; ++st) {
            if (st < nsteps) produce(st);
            cp_async_commit();
        }
        int cu = 0, ck = 0;
        int ckt = __shfl_sync(0xffffffffu, mkt, 0);
        for (int s = 0; s < nsteps; ++s) {
            if (s + ST - 1 < nsteps) produce((s + ST - 1) % ST);
            cp_async_commit();
            cp_async_wait<ST - 1>();
            const uint32_t *w = myring + (s % ST) * 32 * SW;
            uint32_t fa[MTC][PT::NP][4];
#pragma unroll
            for (int i = 0; i < MTC; ++i)
#pragma unroll
                for (int pc = 0; pc < PT::NP; ++pc) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(w + 128 * (i * XC + pc));
                    fa[i][pc][0] = v.x; fa[i][pc][1] = v.y; fa[i][pc][2] = v.z; fa[i][pc][3] = v.w;
                }
            uint32_t fb[NTC][PT::NP][2];
#pragma unroll
            for (int j = 0; j < NTC; ++j) {
                const uint32_t *wy = w + 128 * (MTC * XC + j * YC);
                const uint4 v = *reinterpret_cast<const uint4 *>(wy);
                fb[j][0][0] = v.x; fb[j][0][1] = v.y; fb[j][1][0] = v.z; fb[j][1][1] = v.w;
                if constexpr (PT::NP == 3) {
                    const uint2 u = *reinterpret_cast<const uint2 *>(wy + 128);
                    fb[j][2][0] = u.x; fb[j][2][1] = u.y;
                }
            }
            // piece products, smallest first; consecutive mma instructions go
            // to different tiles so their accumulator chains overlap
            constexpr int NTERM = PT::NP == 2 ? 3 : 6;
            constexpr int TA[6] = {1, 0, 0, 0, 0, 0}, TB[6] = {0, 1, 0, 0, 0, 0};
            constexpr int SA[6] = {2, 1, 0, 1, 0, 0}, SB[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
            for (int t = 0; t < NTERM; ++t) {
                const int ia = PT::NP == 2 ? TA[t] : SA[t];
                const int ib = PT::NP == 2 ? TB[t] : SB[t];
#pragma unroll
                for (int j = 0; j < NTC; ++j)
#pragma unroll
                    for (int i = 0; i < MTC; ++i)
                        if (mt0 + i < MT && nt0 + j < NT) {
                            if (DUAL && (t & 1)) mma_piece<PREC>(acc2[DUAL ? i : 0][DUAL ? j : 0], fa[i][ia], fb[j][ib]);
                            else mma_piece<PREC>(acc[i][j], fa[i][ia], fb[j][ib]);
                        }
            }
            if (++ck == ckt) {  // a block product is complete
                ck = 0;
                ++cu;
                ckt = __shfl_sync(0xffffffffu, mkt, cu < nb ? cu : 0);
                if (++since == F) {
                    since = 0;
#pragma unroll
                    for (int i = 0; i < MTC; ++i)
#pragma unroll
                        for (int j = 0; j < NTC; ++j)
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                float part = acc[i][j][v];
                                if constexpr (DUAL) {
                                    part = __fadd_rn(part, acc2[DUAL ? i : 0][DUAL ? j : 0][v]);
                                    acc2[DUAL ? i : 0][DUAL ? j : 0][v] = 0.f;
                                }
                                if constexpr (FF) kahan_acc(shi[i][j][v], slo[i][j][v], part);
                                else s64[i][j][v] += widen(part);
                                acc[i][j][v] = 0.f;
                            }
                }
            }
        }
        cp_async_wait<0>();
    }
    // epilogue: fragment element v of tile (i, j) sits at
    // row (mt0+i)*16 + g + 8*(v>=2), column (nt0+j)*8 + 2*t4 + (v&1)
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t out_off = a.out_blk_off[q];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
#pragma unroll
    for (int i = 0; i < MTC; ++i)
#pragma unroll
        for (int j = 0; j < NTC; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = (mt0 + i) * 16 + g + ((v >> 1) << 3);
                const int c = (nt0 + j) * 8 + 2 * t4 + (v & 1);
                if (r < R && c < S) {
                    double sum;
                    float part = acc[i][j][v];
                    if constexpr (DUAL) part = __fadd_rn(part, acc2[DUAL ? i : 0][DUAL ? j : 0][v]);
                    if constexpr (FF) sum = pair_total(shi[i][j][v], slo[i][j][v], part);
                    else sum = s64[i][j][v] + widen(part);
                    double val = a.alpha == 1.0 ? sum : a.alpha * sum;
                    const int64_t e = (int64_t)r * S + c;
                    if (a.dtype == BSM_FP64) {
                        if (old >= 0) val = fma(a.beta, static_cast<const double *>(a.old_data)[old + e], val);
                        static_cast<double *>(a.out_data)[out_off + e] = val;
                    } else {
                        if (old >= 0) val = fma(a.beta, (double)static_cast<const float *>(a.old_data)[old + e], val);
                        static_cast<float *>(a.out_data)[out_off + e] = (float)val;
                    }
                }
            }
}

template <int PREC, bool FF, int PM, int PN, bool DUAL>
__device__ __forceinline__ void tc_item(const NumericArgs &a, int64_t q, int lane, uint32_t *ring) {
    const int32_t orc = a.out_blk_rc[q];
    const int MT = (rc_rows(orc) + 15) >> 4, NT = (rc_cols(orc) + 7) >> 3;
    const int pm = min(PM, a.pass_mt > 0 ? a.pass_mt : PM), pn = min(PN, a.pass_nt > 0 ? a.pass_nt : PN);
    for (int mt0 = 0; mt0 < MT; mt0 += pm) {
        const int mtc = min(pm, MT - mt0);
        for (int nt0 = 0; nt0 < NT; nt0 += pn) {
            const int ntc = min(pn, NT - nt0);
            if (PM == 1 || mtc == 1) {
                if (PN == 1 || ntc == 1) tc_pass<PREC, 1, 1, FF, PM, PN, DUAL>(a, q, lane, mt0, nt0, ring);
                else if constexpr (PN >= 2) {
                    if (PN == 2 || ntc == 2) tc_pass<PREC, 1, 2, FF, PM, PN, DUAL>(a, q, lane, mt0, nt0, ring);
                    else if constexpr (PN >= 3) tc_pass<PREC, 1, 3, FF, PM, PN, DUAL>(a, q, lane, mt0, nt0, ring);
                }
            } else if constexpr (PM >= 2) {
                if (PN == 1 || ntc == 1) tc_pass<PREC, 2, 1, FF, PM, PN, DUAL>(a, q, lane, mt0, nt0, ring);
                else if constexpr (PN >= 2) {
                    if (PN == 2 || ntc == 2) tc_pass<PREC, 2, 2, FF, PM, PN, DUAL>(a, q, lane, mt0, nt0, ring);
                    else if constexpr (PN >= 3) tc_pass<PREC, 2, 3, FF, PM, PN, DUAL>(a, q, lane, mt0, nt0, ring);
                }
            }
        }
    }
}

// Tiny output blocks (at most 16 elements) on the split paths: one lane owns
// a whole block and multiplies the same narrow pieces with FP32 FMA on CUDA
// cores (a product of two TF32 or BF16 pieces is exact in FP32), FP32 sum
// inside a block product, the same compensated (or FP64) sum across products.
// A 16 x 8 MMA tile would be almost all padding for such blocks.
template <int PREC, bool FF>
__device__ __forceinline__ void cs_lane_item(const NumericArgs &a, int64_t q) {
    constexpr int NP = PrecTraits<PREC>::NP;
    constexpr int L = 16;
    const float *__restrict__ X = a.x_plain;
    const float *__restrict__ Y = a.y_plain;
    const int32_t orc = a.out_blk_rc[q];
    const int R = rc_rows(orc), S = rc_cols(orc);
    const int RS = R * S;
    const int64_t out_off = a.out_blk_off[q];
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
    const int F = a.flush_every > 0 ? a.flush_every : (a.flush_every < 0 ? -a.flush_every : 1);
    float acc[L], shi[FF ? L : 1], slo[FF ? L : 1];
    double s64[FF ? 1 : L];
#pragma unroll
    for (int e = 0; e < L; ++e) {
        acc[e] = 0.f;
        if constexpr (FF) {
            shi[e] = 0.f;
            slo[e] = 0.f;
        } else {
            s64[e] = 0.0;
        }
    }
    int since = 0;
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t ix = a.px[p], iy = a.py[p];
        const float *xb = X + a.x_blk_off[ix] * NP;
        const float *yb = Y + a.y_blk_off[iy] * NP;
        const int32_t xrc = a.x_blk_rc[ix];
        const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
        const int xs_r = a.x_trans ? 1 : Tn, xs_t = a.x_trans ? R : 1;
        const int ys_t = a.y_trans ? 1 : S, ys_s = a.y_trans ? Tn : 1;
        for (int t = 0; t < Tn; ++t) {
#pragma unroll
            for (int e = 0; e < L; ++e) {
                if (e < RS) {
                    const int r = e / S, c = e - r * S;
                    const float *xe = xb + (int64_t)(r * xs_r + t * xs_t) * NP;
                    const float *ye = yb + (int64_t)(t * ys_t + c * ys_s) * NP;
                    if constexpr (NP == 2) {
                        const float2 xv = __ldg(reinterpret_cast<const float2 *>(xe));
                        const float2 yv = __ldg(reinterpret_cast<const float2 *>(ye));
                        acc[e] = fmaf(xv.y, yv.x, acc[e]);
                        acc[e] = fmaf(xv.x, yv.y, acc[e]);
                        acc[e] = fmaf(xv.x, yv.x, acc[e]);
                    } else {
                        const float x0 = __ldg(xe), x1 = __ldg(xe + 1), x2 = __ldg(xe + 2);
                        const float y0 = __ldg(ye), y1 = __ldg(ye + 1), y2 = __ldg(ye + 2);
                        acc[e] = fmaf(x2, y0, acc[e]);
                        acc[e] = fmaf(x1, y1, acc[e]);
                        acc[e] = fmaf(x0, y2, acc[e]);
                        acc[e] = fmaf(x1, y0, acc[e]);
                        acc[e] = fmaf(x0, y1, acc[e]);
                        acc[e] = fmaf(x0, y0, acc[e]);
                    }
                }
            }
        }
        if (++since == F) {
            since = 0;
#pragma unroll
            for (int e = 0; e < L; ++e) {
                if constexpr (FF) kahan_acc(shi[e], slo[e], acc[e]);
                else s64[e] += widen(acc[e]);
                acc[e] = 0.f;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < L; ++e) {
        if (e < RS) {
            double sum;
            if constexpr (FF) sum = pair_total(shi[e], slo[e], acc[e]);
            else sum = s64[e] + widen(acc[e]);
            double val = a.alpha == 1.0 ? sum : a.alpha * sum;
            if (a.dtype == BSM_FP64) {
                if (old >= 0) val = fma(a.beta, static_cast<const double *>(a.old_data)[old + e], val);
                static_cast<double *>(a.out_data)[out_off + e] = val;
            } else {
                if (old >= 0) val = fma(a.beta, (double)static_cast<const float *>(a.old_data)[old + e], val);
                static_cast<float *>(a.out_data)[out_off + e] = (float)val;
            }
        }
    }
}

template <int PREC, bool FF, int R, int S>
__device__ __forceinline__ void cs_lane_fixed(const NumericArgs &a, int64_t q) {
    constexpr int NP = PrecTraits<PREC>::NP;
    const float *__restrict__ X = a.x_plain;
    const float *__restrict__ Y = a.y_plain;
    const int64_t out_off = a.out_blk_off[q];
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
    const int F = a.flush_every > 0 ? a.flush_every : (a.flush_every < 0 ? -a.flush_every : 1);
    float acc[R][S], shi[FF ? R : 1][FF ? S : 1], slo[FF ? R : 1][FF ? S : 1];
    double s64[FF ? 1 : R][FF ? 1 : S];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < S; ++c) {
            acc[r][c] = 0.f;
            if constexpr (FF) {
                shi[r][c] = 0.f;
                slo[r][c] = 0.f;
            } else {
                s64[r][c] = 0.0;
            }
        }
    int since = 0;
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t ix = a.px[p], iy = a.py[p];
        const float *xb = X + a.x_blk_off[ix] * NP;
        const float *yb = Y + a.y_blk_off[iy] * NP;
        const int32_t xrc = a.x_blk_rc[ix];
        const int Tn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
        const int xs_r = a.x_trans ? 1 : Tn, xs_t = a.x_trans ? R : 1;
        const int ys_t = a.y_trans ? 1 : S, ys_s = a.y_trans ? Tn : 1;
        for (int t = 0; t < Tn; ++t) {
            float xv[R][NP], yv[S][NP];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int pc = 0; pc < NP; ++pc) xv[r][pc] = __ldg(xb + (int64_t)(r * xs_r + t * xs_t) * NP + pc);
#pragma unroll
            for (int c = 0; c < S; ++c)
#pragma unroll
                for (int pc = 0; pc < NP; ++pc) yv[c][pc] = __ldg(yb + (int64_t)(t * ys_t + c * ys_s) * NP + pc);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    if constexpr (NP == 2) {
                        acc[r][c] = fmaf(xv[r][1], yv[c][0], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][0], yv[c][1], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][0], yv[c][0], acc[r][c]);
                    } else {
                        acc[r][c] = fmaf(xv[r][2], yv[c][0], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][1], yv[c][1], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][0], yv[c][2], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][1], yv[c][0], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][0], yv[c][1], acc[r][c]);
                        acc[r][c] = fmaf(xv[r][0], yv[c][0], acc[r][c]);
                    }
                }
        }
        if (++since == F) {
            since = 0;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    if constexpr (FF) kahan_acc(shi[r][c], slo[r][c], acc[r][c]);
                    else s64[r][c] += widen(acc[r][c]);
                    acc[r][c] = 0.f;
                }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < S; ++c) {
            const int e = r * S + c;
            double sum;
            if constexpr (FF) sum = pair_total(shi[r][c], slo[r][c], acc[r][c]);
            else sum = s64[r][c] + widen(acc[r][c]);
            double val = a.alpha == 1.0 ? sum : a.alpha * sum;
            if (a.dtype == BSM_FP64) {
                if (old >= 0) val = fma(a.beta, static_cast<const double *>(a.old_data)[old + e], val);
                static_cast<double *>(a.out_data)[out_off + e] = val;
            } else {
                if (old >= 0) val = fma(a.beta, (double)static_cast<const float *>(a.old_data)[old + e], val);
                static_cast<float *>(a.out_data)[out_off + e] = (float)val;
            }
        }
}

template <int PREC, bool FF>
__device__ __forceinline__ void cs_lane_dispatch(const NumericArgs &a, int64_t q) {
    const int32_t orc = a.out_blk_rc[q];
    switch ((rc_rows(orc) << 8) | rc_cols(orc)) {
        case 0x101: cs_lane_fixed<PREC, FF, 1, 1>(a, q); break;
        case 0x104: cs_lane_fixed<PREC, FF, 1, 4>(a, q); break;
        case 0x401: cs_lane_fixed<PREC, FF, 4, 1>(a, q); break;
        case 0x404: cs_lane_fixed<PREC, FF, 4, 4>(a, q); break;
        case 0x202: cs_lane_fixed<PREC, FF, 2, 2>(a, q); break;
        case 0x505: cs_lane_fixed<PREC, FF, 5, 5>(a, q); break;
        default: cs_lane_item<PREC, FF>(a, q); break;
    }
}

// PM x PN: the largest pass this instance runs.  Items [i0, i1) of the
// order, a warp each on the tensor cores: every item before the lane items
// (a.group < 0), or one group of a multiply whose blocks of one tile row run
// in a 1 x PN instance (group 1) and the rest in a 2 x PN instance (group 0).
template <int PREC, bool FF, int PM, int PN, bool DUAL>
__global__ void __launch_bounds__(kThreadsNum) k_numeric_tc(NumericArgs a) {
    extern __shared__ __align__(16) uint32_t tc_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *ring = tc_smem + warp * ring_words_per_warp<PREC, PM, PN>();
    if (a.status && *a.status != 0) return;
    const int64_t n_lane = a.n_lane_items ? *a.n_lane_items : 0;
    int64_t i0 = 0, i1 = a.n_items - n_lane;
    if (a.group == 0) i1 = a.item_groups[0];
    if (a.group == 1) i0 = a.item_groups[0];
    unsigned long long *ctr = a.work_counter + (a.group > 0 ? a.group : 0);
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0) + i0;
        if (t >= i1) break;
        int64_t q = t;
        if (a.item_order) q = (int64_t)((uint32_t)a.item_order[q] & 0x7fffffffu);
        BSM_DBG_WARP_SKIP(a, q, lane)
        tc_item<PREC, FF, PM, PN, DUAL>(a, q, lane, ring);
    }
}

// The last *n_lane_items items of the order: tiny blocks marked for the
// CUDA-core variant, 32 per ticket (a kernel of their own, so that the
// tensor-core instances do not carry its registers).
template <int PREC, bool FF>
__global__ void __launch_bounds__(kThreadsNum) k_numeric_tc_lane(NumericArgs a) {
    const int lane = threadIdx.x & 31;
    if (a.status && *a.status != 0) return;
    const int64_t n_lane = *a.n_lane_items;
    const int64_t lane0 = a.n_items - n_lane;
    unsigned long long *ctr = a.work_counter + 2;
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t * 32 >= n_lane) break;
        const int64_t idx = lane0 + t * 32 + lane;
        if (idx < a.n_items) {
            const int64_t q = (int64_t)((uint32_t)a.item_order[idx] & 0x7fffffffu);
            if (BSM_DBG_LANE_OK(a, q)) cs_lane_dispatch<PREC, FF>(a, q);
        }
    }
}

// =====================================================================
// Ozaki-style error-free slicing (BSM_P_OZAKI)
// =====================================================================
// Error-free transformation of a product into products of short-mantissa
// operands (Ozaki, Ogita, Oishi and Rump, 2012).  With 2^e the largest power
// of two not above max |x| over a line (a logical row of X, a logical column
// of Y), every x of the line is cut into integer digits
//   x * 2^(7-e) = d_0 + d_1 2^-9 + ... + d_5 2^-45 + rest,   |rest| <= 2^-46,
// d_0 = rint(x * 2^(7-e)) and each next digit the rounded remainder times 2^9,
// so |d_p| <= 256 and the slice d_p * 2^(-9p) is exact in BF16.  A slice
// product of level l = p + q lies on the grid 2^(-9l) (in units of the line
// pair's scale 2^(ex+ey-14)); products of one level summed in the tensor
// core's FP32 accumulator stay exact while the sum stays below 2^24 grid
// units: a level holding c slice pairs takes 2^24 / (c * 2^16) terms of k,
// 64 for level 3 (4 pairs).  Levels 0..3 have exact FP32 sums; before more
// than kOzWindow terms of k they are converted to integers and added into a
// 64-bit fixed-point sum with unit 2^-27 (exact; a window adds less than
// 2^49.01 units, so 8192 windows fit, after which the sum is moved into the
// output element).  Levels 4 and 5 (11 pairs, below 2^-33 of level 0) have
// a rounded FP32 sum each per window (the tensor core's FP32 additions round
// toward zero, so they are restarted every window; two sums rather than one
// keep every accumulator's chain of dependent MMAs at 6 per k-step or less),
// whose window values add up in an FP32 sum with round-to-nearest on the
// CUDA cores; levels >= 6 are dropped (below 2^-50 of level 0).  Per term of k the error is below 2^-44
// of 2^(ex+ey): the rounded sums plus the cut digits and levels.
constexpr int kOzSlices = 6;
constexpr int kOzLevels = 6;    // FP32 sums: levels 0, 1, 2, 3 exact, 4 and 5 rounded (one each,
                                // so that no accumulator takes more than 6 of a k-step's 21 MMAs)
constexpr int kOzWindow = 64;
constexpr int kOzSpillWindows = 8192;
constexpr int kOzStages = 3;
constexpr int kOzXW = 4 * kOzSlices;                 // X words per lane per tile
constexpr int kOzYW = 2 * kOzSlices;                 // Y words per lane per tile
// ring words per lane per stage for passes of at most MAXN tiles (1 x MAXN)
template <int MAXN>
__host__ __device__ constexpr int oz_sw() { return kOzXW + MAXN * kOzYW; }
template <int MAXN>
__host__ __device__ constexpr int oz_ring_words_per_warp() { return kOzStages * 32 * oz_sw<MAXN>(); }
// Packed tiles are chunk-major: chunk c (16 bytes) of lane L at word
// c * 128 + 4 * L, so one 16-byte cp.async per lane reads 512 contiguous
// bytes.  X tile: chunk p = plane p (registers v0..v3); Y tile: chunk c =
// planes 2c and 2c+1 (registers v0, v1 each; lanes with bit 3 set hold the two
// 8-byte halves swapped, so 8-byte reads of 16 lanes hit 16 distinct bank
// pairs).  A ring stage is chunk-major the same way (chunk c of lane L at
// word c * 128 + 4 * L): each 16-byte copy and read of the warp covers 512
// contiguous bytes of shared memory.

// One pass over a 1 x NTC super tile (16 x 8*NTC output elements) at (mt0, nt0),
// staged through a ring laid out for passes of at most MAXN tiles.
template <int NTC, int MAXN>
__device__ __forceinline__ void oz_pass(const NumericArgs &a, int64_t q, int lane, int mt0, int nt0,
                                        uint32_t *ring) {
    constexpr int ST = kOzStages, SW = oz_sw<MAXN>();
    const int32_t orc = a.out_blk_rc[q];
    const int R = rc_rows(orc), S = rc_cols(orc);
    const int MT = (R + 15) >> 4, NT = (S + 7) >> 3;
    const int64_t p0 = a.seg_ptr[q], p1 = a.seg_ptr[q + 1];
    const uint32_t *XP = static_cast<const uint32_t *>(a.x_pack);
    const uint32_t *YP = static_cast<const uint32_t *>(a.y_pack);
    double *O = static_cast<double *>(a.out_data);
    const int64_t out_off = a.out_blk_off[q];
    uint32_t *myring = ring + 4 * lane;  // chunk c of stage st at myring + st * 32 * SW + 128 * c
    const uint32_t ring_s = smem_addr(myring);
    const int hswz = (lane >> 3) & 1;  // 8-byte half order inside a Y chunk
    const int g = lane >> 2, t4 = lane & 3;
    // rows g + 8 of this tile exist (else fragment elements v = 2, 3 are padding)
    const bool hi_rows = R - mt0 * 16 > 8;

    float acc[kOzLevels][NTC][4];
    long long fx[NTC][4];  // exact sum of levels 0..3, unit 2^-27
    float low[NTC][4];     // sum of the windows' level 4..5 sums
#pragma unroll
    for (int j = 0; j < NTC; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            fx[j][v] = 0;
            low[j][v] = 0.f;
#pragma unroll
            for (int l = 0; l < kOzLevels; ++l) acc[l][j][v] = 0.f;
        }
    int kacc = 0;      // terms of k in the open exact window
    int nwin = 0;      // windows added into fx since it was last moved out
    bool spilled = false;
    // levels 0..3 -> fx (integers below 2^24 on their grids, so the conversions are exact)
    auto close_window = [&]() {
#pragma unroll
        for (int j = 0; j < NTC; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (v >= 2 && !hi_rows) continue;  // padding rows hold zeros
                long long t = (long long)__float2int_rn(acc[0][j][v]) << 27;
                t += (long long)__float2int_rn(acc[1][j][v] * 512.f) << 18;
                t += (long long)__float2int_rn(acc[2][j][v] * 262144.f) << 9;
                t += (long long)__float2int_rn(acc[3][j][v] * 134217728.f);
                fx[j][v] += t;
                low[j][v] = __fadd_rn(low[j][v], __fadd_rn(acc[4][j][v], acc[5][j][v]));
#pragma unroll
                for (int l = 0; l < kOzLevels; ++l) acc[l][j][v] = 0.f;
            }
        if (++nwin == kOzSpillWindows) {  // keep fx far from 2^63: move it into the output
            nwin = 0;
#pragma unroll
            for (int j = 0; j < NTC; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = mt0 * 16 + g + ((v >> 1) << 3);
                    const int c = (nt0 + j) * 8 + 2 * t4 + (v & 1);
                    if (r < R && c < S && nt0 + j < NT) {
                        const double part = (double)fx[j][v] * 0x1p-27;
                        const int64_t e = out_off + (int64_t)r * S + c;
                        O[e] = spilled ? O[e] + part : part;
                    }
                    fx[j][v] = 0;
                }
            spilled = true;
        }
    };
    for (int64_t pb = p0; pb < p1; pb += 32) {
        const int nb = (int)min((int64_t)32, p1 - pb);
        int64_t mxo = 0, myo = 0;
        int mkt = 0, mtn = 0;
        if (lane < nb) {
            const int32_t ix = a.px[pb + lane], iy = a.py[pb + lane];
            const int32_t xrc = a.x_blk_rc[ix];
            mtn = a.x_trans ? rc_rows(xrc) : rc_cols(xrc);
            mxo = a.x_pack_off[ix];
            myo = a.y_pack_off[iy];
            mkt = (mtn + 15) >> 4;
        }
        int nsteps = mkt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nsteps += __shfl_xor_sync(0xffffffffu, nsteps, o);
        int pu = 0, pk = 0;
        int64_t pxo = __shfl_sync(0xffffffffu, mxo, 0), pyo = __shfl_sync(0xffffffffu, myo, 0);
        int pkt = __shfl_sync(0xffffffffu, mkt, 0);
        auto produce = [&](int st) {
            const uint32_t dst = ring_s + (uint32_t)(st * 32 * SW) * 4u;
            const uint32_t *src = XP + pxo + (int64_t)(pk * MT + mt0) * (32 * kOzXW) + 4 * lane;
#pragma unroll
            for (int c = 0; c < kOzXW / 4; ++c) cp_async16_cg(dst + 512u * c, src + 128 * c);
#pragma unroll
            for (int j = 0; j < NTC; ++j) {
                if (nt0 + j < NT) {
                    const uint32_t *ys = YP + pyo + (int64_t)(pk * NT + nt0 + j) * (32 * kOzYW) + 4 * lane;
#pragma unroll
                    for (int c = 0; c < kOzYW / 4; ++c)
                        cp_async16_cg(dst + 512u * (kOzXW / 4 + j * (kOzYW / 4) + c), ys + 128 * c);
                }
            }
            if (++pk == pkt) {
                pk = 0;
                ++pu;
                const int src_lane = pu < nb ? pu : 0;
                pxo = __shfl_sync(0xffffffffu, mxo, src_lane);
                pyo = __shfl_sync(0xffffffffu, myo, src_lane);
                pkt = __shfl_sync(0xffffffffu, mkt, src_lane);
            }
        };
#pragma unroll
        for (int st = 0; st < ST - 1; ++st) {
            if (st < nsteps) produce(st);
            cp_async_commit();
        }
        int cu = 0, ck = 0;
        int ckt = __shfl_sync(0xffffffffu, mkt, 0), ctn = __shfl_sync(0xffffffffu, mtn, 0);
        for (int s = 0; s < nsteps; ++s) {
            if (s + ST - 1 < nsteps) produce((s + ST - 1) % ST);
            cp_async_commit();
            cp_async_wait<ST - 1>();
            const uint32_t *w = myring + (s % ST) * 32 * SW;
            uint32_t fa[kOzSlices][4];
#pragma unroll
            for (int p = 0; p < kOzSlices; ++p) {
                const uint4 v = *reinterpret_cast<const uint4 *>(w + 128 * p);
                fa[p][0] = v.x; fa[p][1] = v.y; fa[p][2] = v.z; fa[p][3] = v.w;
            }
            // close the exact window before it would pass kOzWindow terms of k
            const int kact = min(16, ctn - 16 * ck);
            if (kacc + kact > kOzWindow) {
                close_window();
                kacc = 0;
            }
            kacc += kact;
            // slice products: Y slice q (read from the ring when needed) with
            // every X slice p of level p + q <= 5
#pragma unroll
            for (int qq = kOzSlices - 1; qq >= 0; --qq) {
                uint32_t fb[NTC][2];
#pragma unroll
                for (int j = 0; j < NTC; ++j) {
                    const uint2 v = *reinterpret_cast<const uint2 *>(
                        w + 128 * (kOzXW / 4 + j * (kOzYW / 4) + (qq >> 1)) + 2 * ((qq & 1) ^ hswz));
                    fb[j][0] = v.x; fb[j][1] = v.y;
                }
#pragma unroll
                for (int p = kOzSlices - 1 - qq; p >= 0; --p)
#pragma unroll
                    for (int j = 0; j < NTC; ++j)
                        if (nt0 + j < NT) {
                            constexpr int top = kOzLevels - 1;
                            mma_bf16(acc[p + qq < top ? p + qq : top][j], fa[p], fb[j]);
                        }
            }
            if (++ck == ckt) {
                ck = 0;
                ++cu;
                const int src_lane = cu < nb ? cu : 0;
                ckt = __shfl_sync(0xffffffffu, mkt, src_lane);
                ctn = __shfl_sync(0xffffffffu, mtn, src_lane);
            }
        }
        cp_async_wait<0>();
    }
    close_window();
    // epilogue: scale by 2^(ex + ey - 14) of the element's row and column
    const int64_t old = (a.beta != 0.0 && a.old_off) ? a.old_off[q] : -1;
    const bool any = p1 > p0;
    const int32_t xl0 = any ? a.x_line0[a.px[p0]] : 0;
    const int32_t yl0 = any ? a.y_line0[a.py[p0]] : 0;
    int ex[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = mt0 * 16 + g + 8 * h;
        ex[h] = (any && r < R) ? a.x_exp[xl0 + r] - 1023 : 0;
    }
#pragma unroll
    for (int j = 0; j < NTC; ++j) {
        int ey[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = (nt0 + j) * 8 + 2 * t4 + h;
            ey[h] = (any && c < S) ? a.y_exp[yl0 + c] - 1023 : 0;
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = mt0 * 16 + g + ((v >> 1) << 3);
            const int c = (nt0 + j) * 8 + 2 * t4 + (v & 1);
            if (r < R && c < S && nt0 + j < NT) {
                const int64_t e = (int64_t)r * S + c;
                double sum = (double)fx[j][v] * 0x1p-27 + (double)low[j][v];
                if (spilled) sum += O[out_off + e];
                double val = a.alpha * ldexp(sum, ex[v >> 1] + ey[v & 1] - 14);
                if (old >= 0) val = fma(a.beta, static_cast<const double *>(a.old_data)[old + e], val);
                O[out_off + e] = val;
            }
        }
    }
}

template <int MAXN>
__device__ __forceinline__ void oz_item(const NumericArgs &a, int64_t q, int lane, uint32_t *ring) {
    const int32_t orc = a.out_blk_rc[q];
    const int MT = (rc_rows(orc) + 15) >> 4, NT = (rc_cols(orc) + 7) >> 3;
    const int pn = MAXN == 3 ? 3 : MAXN == 1 ? 1 : (a.pass_nt == 1 ? 1 : 2);
    for (int mt0 = 0; mt0 < MT; ++mt0)
        for (int nt0 = 0; nt0 < NT; nt0 += pn) {
            const int left = NT - nt0;
            if constexpr (MAXN == 3) {
                if (left >= 3) oz_pass<3, MAXN>(a, q, lane, mt0, nt0, ring);
                else if (left == 2) oz_pass<2, MAXN>(a, q, lane, mt0, nt0, ring);
                else oz_pass<1, MAXN>(a, q, lane, mt0, nt0, ring);
            } else if constexpr (MAXN == 2) {
                if (pn == 2 && left >= 2) oz_pass<2, MAXN>(a, q, lane, mt0, nt0, ring);
                else oz_pass<1, MAXN>(a, q, lane, mt0, nt0, ring);
            } else {
                oz_pass<1, MAXN>(a, q, lane, mt0, nt0, ring);
            }
        }
}

// Items [0, n0): a warp each on the tensor cores; items [n0, n_items): tiny
// blocks one per lane with plain FP64 FMA (exact enough, no slicing needed).
template <int MAXN>
__global__ void __launch_bounds__(kThreadsNum) k_numeric_oz(NumericArgs a) {
    extern __shared__ __align__(16) uint32_t oz_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *ring = oz_smem + warp * oz_ring_words_per_warp<MAXN>();
    if (a.status && *a.status != 0) return;
    // items [i0, i1): every item before the lane items (a.group < 0), or one
    // group: blocks of two tile columns and more (0), of one tile column (1)
    const int64_t n_lane = a.n_lane_items ? *a.n_lane_items : 0;
    int64_t i0 = 0, i1 = a.n_items - n_lane;
    if (a.group == 0) i1 = a.item_groups[0];
    if (a.group == 1) i0 = a.item_groups[0];
    unsigned long long *ctr = a.work_counter + (a.group > 0 ? a.group : 0);
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0) + i0;
        if (t >= i1) break;
        int64_t q = t;
        if (a.item_order) q = (int64_t)((uint32_t)a.item_order[q] & 0x7fffffffu);
        BSM_DBG_WARP_SKIP(a, q, lane)
        oz_item<MAXN>(a, q, lane, ring);
    }
}

// The lane items of the Ozaki path: plain FP64 FMA, one lane per block.
__global__ void __launch_bounds__(kThreadsNum) k_numeric_oz_lane(NumericArgs a) {
    const int lane = threadIdx.x & 31;
    if (a.status && *a.status != 0) return;
    const int64_t n_lane = *a.n_lane_items;
    const int64_t lane0 = a.n_items - n_lane;
    unsigned long long *ctr = a.work_counter + 2;
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t * 32 >= n_lane) break;
        const int64_t idx = lane0 + t * 32 + lane;
        if (idx < a.n_items) {
            const int64_t q = (int64_t)((uint32_t)a.item_order[idx] & 0x7fffffffu);
            if (BSM_DBG_LANE_OK(a, q)) cc_lane_dispatch<double>(a, q);
        }
    }
}

// =====================================================================
// Operand splitting and fragment packing
// =====================================================================
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Split x into `np` pieces of the precision's narrow type, most significant
// first; returns the bit patterns (TF32 in 32 bits, BF16 in the low 16).
template <int PREC>
__device__ __forceinline__ void split_value(double x, uint32_t (&out)[3]) {
    if constexpr (PREC == BSM_P_TF32x3) {
        const uint32_t hi = f32_to_tf32((float)x);
        const double r = x - (double)__uint_as_float(hi);
        out[0] = hi;
        out[1] = f32_to_tf32((float)r);
        out[2] = 0;
    } else {
        const __nv_bfloat16 h0 = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(h0);
        const __nv_bfloat16 h1 = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(h1);
        const __nv_bfloat16 h2 = __double2bfloat16(r2);
        out[0] = __bfloat16_as_ushort(h0);
        out[1] = __bfloat16_as_ushort(h1);
        out[2] = __bfloat16_as_ushort(h2);
    }
}

template <typename T>
__device__ __forceinline__ double elem(const T *b, int R, int Tn, int trans, int r, int t) {
    // logical R x Tn block, stored R x Tn (trans=0) or Tn x R (trans=1)
    if (r >= R || t >= Tn) return 0.0;
    return (double)(trans ? b[(int64_t)t * R + r] : b[(int64_t)r * Tn + t]);
}

// words of one block's packing
__device__ __forceinline__ int64_t pack_words(int R, int C, int role_y, int prec) {
    const int K = (prec == BSM_P_TF32x3) ? 8 : 16;
    if (!role_y) {
        const int XW = prec == BSM_P_OZAKI ? kOzXW : (prec == BSM_P_BF16x6) ? 12 : 8;
        return (int64_t)((R + 15) / 16) * ((C + K - 1) / K) * 32 * XW;
    }
    const int YW = prec == BSM_P_OZAKI ? kOzYW : (prec == BSM_P_BF16x6) ? 8 : 4;
    return (int64_t)((R + K - 1) / K) * ((C + 7) / 8) * 32 * YW;
}

// logical dims of block b for the role: X is R x T, Y is T x S
__device__ __forceinline__ void logical_dims(int32_t rc, int trans, int &rows, int &cols) {
    rows = trans ? rc_cols(rc) : rc_rows(rc);
    cols = trans ? rc_rows(rc) : rc_cols(rc);
}

__global__ void k_pack_sizes(int64_t nnzb, const int32_t *blk_rc, int role_y, int trans, int prec,
                             int64_t *words) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnzb;
         b += (int64_t)gridDim.x * blockDim.x) {
        int rows, cols;
        logical_dims(blk_rc[b], trans, rows, cols);
        words[b] = pack_words(rows, cols, role_y, prec);
    }
}

// one warp per block; lane L writes its fragment words of every tile
template <typename T, int PREC>
__global__ void k_pack(int64_t nnzb, const int64_t *blk_off, const int32_t *blk_rc, const T *data,
                       int role_y, int trans, const int64_t *pack_off, uint32_t *pack, const int32_t *status) {
    using PT = PrecTraits<PREC>;
    if (status && *status != 0) return;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = wid; b < nnzb; b += nwarp) {
        const T *src = data + blk_off[b];
        int rows, cols;
        logical_dims(blk_rc[b], trans, rows, cols);
        // element accessor of the logical rows x cols block
        auto at = [&](int r, int c) -> double {
            return elem<T>(src, rows, cols, trans, r, c);
        };
        uint32_t *dst = pack + pack_off[b];
        uint32_t sp[3];
        if (!role_y) {
            const int MT = (rows + 15) / 16, KT = (cols + PT::K - 1) / PT::K;
            for (int kt = 0; kt < KT; ++kt)
                for (int mt = 0; mt < MT; ++mt) {
                    // chunk pc (piece pc, registers v0..v3) of this lane at word 128 * pc
                    uint32_t *w = dst + (int64_t)(kt * MT + mt) * (32 * PT::XW) + 4 * lane;
                    const int r0 = mt * 16 + g, k0 = kt * PT::K;
                    if constexpr (PREC == BSM_P_TF32x3) {
                        const int rr[4] = {r0, r0 + 8, r0, r0 + 8};
                        const int kk[4] = {k0 + t4, k0 + t4, k0 + t4 + 4, k0 + t4 + 4};
                        for (int v = 0; v < 4; ++v) {
                            split_value<PREC>(at(rr[v], kk[v]), sp);
                            w[v] = sp[0];
                            w[128 + v] = sp[1];
                        }
                    } else {
                        // reg v holds (row, k) and (row, k+1)
                        const int rr[4] = {r0, r0 + 8, r0, r0 + 8};
                        const int kk[4] = {k0 + 2 * t4, k0 + 2 * t4, k0 + 2 * t4 + 8, k0 + 2 * t4 + 8};
                        for (int v = 0; v < 4; ++v) {
                            uint32_t lo[3], hi[3];
                            split_value<PREC>(at(rr[v], kk[v]), lo);
                            split_value<PREC>(at(rr[v], kk[v] + 1), hi);
                            for (int pc = 0; pc < PT::NP; ++pc) w[128 * pc + v] = lo[pc] | (hi[pc] << 16);
                        }
                    }
                }
        } else {
            const int KT = (rows + PT::K - 1) / PT::K, NT = (cols + 7) / 8;
            for (int kt = 0; kt < KT; ++kt)
                for (int nt = 0; nt < NT; ++nt) {
                    // piece pc, registers v0 v1 at word 128 * (pc >> 1) + 2 * (pc & 1)
                    uint32_t *w = dst + (int64_t)(kt * NT + nt) * (32 * PT::YW) + 4 * lane;
                    const int n0 = nt * 8 + g, k0 = kt * PT::K;
                    if constexpr (PREC == BSM_P_TF32x3) {
                        const int kk[2] = {k0 + t4, k0 + t4 + 4};
                        for (int v = 0; v < 2; ++v) {
                            split_value<PREC>(at(kk[v], n0), sp);
                            w[v] = sp[0];
                            w[2 + v] = sp[1];
                        }
                    } else {
                        const int kk[2] = {k0 + 2 * t4, k0 + 2 * t4 + 8};
                        for (int v = 0; v < 2; ++v) {
                            uint32_t lo[3], hi[3];
                            split_value<PREC>(at(kk[v], n0), lo);
                            split_value<PREC>(at(kk[v] + 1, n0), hi);
                            for (int pc = 0; pc < PT::NP; ++pc) w[128 * (pc >> 1) + 2 * (pc & 1) + v] = lo[pc] | (hi[pc] << 16);
                        }
                        if constexpr (PT::NP == 3) {  // padding words of the second chunk
                            w[128 + 2] = 0;
                            w[128 + 3] = 0;
                        }
                    }
                }
        }
    }
}

// Unpacked pieces: out[e*NP + p] = piece p of element e (as an FP32 value)
template <typename T, int PREC>
__global__ void k_split_plain(int64_t n, const T *data, float *out) {
    constexpr int NP = PrecTraits<PREC>::NP;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t sp[3];
        split_value<PREC>((double)data[e], sp);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float v;
            if constexpr (PREC == BSM_P_TF32x3) v = __uint_as_float(sp[p]);
            else v = __bfloat162float(__ushort_as_bfloat16((unsigned short)sp[p]));
            out[e * NP + p] = v;
        }
    }
}

// Digits of x on its line's grid (see the Ozaki section above): slice p is
// d_p * 2^(-9p) as BF16 bits, exact.  e = unbiased exponent of the line.
__device__ __forceinline__ void oz_slices(double x, int e, uint32_t (&out)[kOzSlices]) {
    // The recursion y_0 = x * 2^(7-e), d_p = rint(y_p), y_(p+1) = (y_p - d_p) * 512
    // is exact in FP64 (y_p - d_p is exact, |y_p - d_p| <= 1/2), so it is run on
    // the integers: r = |x| * 2^(62-e) truncated (below 2^63; `sticky` records
    // whether anything was cut), digit p = r / 2^(55-9p) rounded half to even
    // with the cut part counted, r minus the digit.  The same digits as the
    // FP64 recursion -- signs of zero digits included -- without the FP64 pipe.
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    if (mag == 0) {  // padding and exact zeros
#pragma unroll
        for (int p = 0; p < kOzSlices; ++p) out[p] = 0u;
        return;
    }
    const bool neg = (b >> 63) != 0;
    int ex = (int)(mag >> 52);
    unsigned long long m = mag & 0xfffffffffffffull;
    if (ex) m |= 1ull << 52;
    else ex = 1;
    // |x| * 2^(62-e) = m * 2^(ex - 1013 - e), ex - 1013 - e <= 11 and m < 2^53 (2^52 for ex = 1)
    const int sh = ex - 1013 - e;
    long long r;
    bool sticky;
    if (sh >= 0) {
        r = (long long)(m << sh);
        sticky = false;
    } else if (sh > -64) {
        r = (long long)(m >> -sh);
        sticky = (m & ((1ull << -sh) - 1ull)) != 0ull;
    } else {
        r = 0;
        sticky = true;
    }
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p) {
        const int k = 55 - 9 * p;
        const long long rp = r;
        long long q = r >> k;  // floor
        const long long rem = r - (long long)((unsigned long long)q << k);
        const long long half = 1ll << (k - 1);
        if (rem > half || (rem == half && (sticky || (q & 1)))) ++q;
        r = (long long)((unsigned long long)r - ((unsigned long long)q << k));
        // d_p * 2^(-9p) with |d_p| <= 256: exact in FP32 and in BF16; a zero digit
        // takes the sign of the remainder it rounded (rint keeps it)
        float v = (float)q * __int_as_float((127 - 9 * p) << 23);
        if (neg) v = -v;
        if (q == 0) v = (neg ? (rp > 0 || (rp == 0 && sticky)) : (rp < 0)) ? -0.0f : 0.0f;
        out[p] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
}

// Ozaki fragment planes of FP64 data: the tiles of k_pack's BF16 layout with
// kOzSlices planes, chunk-major inside a tile; X element (r, k) uses the
// exponent of line line0[b] + r, Y element (k, n) that of line line0[b] + n.
__global__ void k_pack_oz(int64_t nnzb, const int64_t *blk_off, const int32_t *blk_rc, const double *data,
                          int role_y, int trans, const int64_t *pack_off, uint32_t *pack, const int32_t *line0,
                          const int32_t *exps, const int32_t *status) {
    if (status && *status != 0) return;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = wid; b < nnzb; b += nwarp) {
        const double *src = data + blk_off[b];
        int rows, cols;
        logical_dims(blk_rc[b], trans, rows, cols);
        const int32_t l0 = line0[b];
        uint32_t *dst = pack + pack_off[b];
        uint32_t lo[kOzSlices], hi[kOzSlices];
        if (!role_y) {
            const int MT = (rows + 15) / 16, KT = (cols + 15) / 16;
            for (int kt = 0; kt < KT; ++kt)
                for (int mt = 0; mt < MT; ++mt) {
                    uint32_t *w = dst + (int64_t)(kt * MT + mt) * (32 * kOzXW) + 4 * lane;
                    const int r0 = mt * 16 + g, k0 = kt * 16;
                    const int rr[4] = {r0, r0 + 8, r0, r0 + 8};
                    const int kk[4] = {k0 + 2 * t4, k0 + 2 * t4, k0 + 2 * t4 + 8, k0 + 2 * t4 + 8};
                    for (int v = 0; v < 4; ++v) {
                        const int e = rr[v] < rows ? exps[l0 + rr[v]] - 1023 : 0;
                        oz_slices(elem<double>(src, rows, cols, trans, rr[v], kk[v]), e, lo);
                        oz_slices(elem<double>(src, rows, cols, trans, rr[v], kk[v] + 1), e, hi);
                        for (int p = 0; p < kOzSlices; ++p) w[128 * p + v] = lo[p] | (hi[p] << 16);
                    }
                }
        } else {
            const int KT = (rows + 15) / 16, NT = (cols + 7) / 8;
            for (int kt = 0; kt < KT; ++kt)
                for (int nt = 0; nt < NT; ++nt) {
                    uint32_t *w = dst + (int64_t)(kt * NT + nt) * (32 * kOzYW) + 4 * lane;
                    const int n0 = nt * 8 + g, k0 = kt * 16;
                    const int e = n0 < cols ? exps[l0 + n0] - 1023 : 0;
                    const int kk[2] = {k0 + 2 * t4, k0 + 2 * t4 + 8};
                    for (int v = 0; v < 2; ++v) {
                        oz_slices(elem<double>(src, rows, cols, trans, kk[v], n0), e, lo);
                        oz_slices(elem<double>(src, rows, cols, trans, kk[v] + 1, n0), e, hi);
                        for (int p = 0; p < kOzSlices; ++p)
                            w[128 * (p >> 1) + 2 * ((p & 1) ^ ((lane >> 3) & 1)) + v] = lo[p] | (hi[p] << 16);
                    }
                }
        }
    }
}

// line0[b] for every block: first global line of the block (one warp per block row)
__global__ void k_oz_line0(int32_t nbr, const int64_t *row_ptr, const int32_t *col_idx, const int32_t *row_start,
                           const int32_t *col_start, int by_rows, int32_t *line0) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nbr; i += nwarp)
        for (int64_t b = row_ptr[i] + lane; b < row_ptr[i + 1]; b += 32)
            line0[b] = by_rows ? row_start[i] : col_start[col_idx[b]];
}

// exps[line] = max over the line of the biased exponent field of |x| (one warp
// per block, a lane per line of the block)
__global__ void k_oz_line_exp(int64_t nnzb, const int64_t *blk_off, const int32_t *blk_rc, const double *data,
                              const int32_t *line0, int by_rows, int32_t *exps) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = wid; b < nnzb; b += nwarp) {
        const double *src = data + blk_off[b];
        const int R = rc_rows(blk_rc[b]), C = rc_cols(blk_rc[b]);
        const int nl = by_rows ? R : C, len = by_rows ? C : R;
        for (int l = lane; l < nl; l += 32) {
            int m = 0;
            for (int t = 0; t < len; ++t) {
                const double x = by_rows ? src[(int64_t)l * C + t] : src[(int64_t)t * C + l];
                m = max(m, (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
            }
            atomicMax(&exps[line0[b] + l], m);
        }
    }
}

// Set bit 31 of order[t] when the block order[t] is computed by the CUDA-core
// variant: variant_of_class[size_index[rows] * ns + size_index[cols]] != 0.
__global__ void k_mark_variant(int64_t n, int32_t *order, const int32_t *blk_rc, const int32_t *size_index,
                               int32_t ns, const int8_t *variant_of_class, unsigned long long *marked) {
    unsigned long long cnt = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = order[t] & 0x7fffffff;
        const int32_t rc = blk_rc[q];
        if (variant_of_class[size_index[rc_rows(rc)] * ns + size_index[rc_cols(rc)]]) {
            order[t] = (int32_t)((uint32_t)q | 0x80000000u);
            cnt++;
        }
    }
    if (marked && cnt) atomicAdd(marked, cnt);
}

int g_num_sms = 0;
int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

template <typename K>
int persistent_grid(K kernel, int64_t n_items, size_t smem = 0, int threads = kThreadsNum, int ctas_per_sm = 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t g = (int64_t)num_sms() * per_sm;
    const int warps = threads / 32;
    const int64_t need = (n_items + warps - 1) / warps;
    if (g > need) g = need;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T, int BUILD>
int launch_cc(const NumericArgs &a, cudaStream_t s) {
    const int g = persistent_grid(k_numeric_cc<T, BUILD>, a.n_items, 0, kThreadsNum, a.ctas_per_sm);
    k_numeric_cc<T, BUILD><<<g, kThreadsNum, 0, s>>>(a);
    return g;
}

template <int MAXN>
cudaError_t launch_oz(const NumericArgs &a, cudaStream_t s, int threads, int *grid) {
    const size_t smem = sizeof(uint32_t) * (size_t)oz_ring_words_per_warp<MAXN>() * (threads / 32);
    cudaError_t e = cudaFuncSetAttribute(k_numeric_oz<MAXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    *grid = persistent_grid(k_numeric_oz<MAXN>, a.n_items, smem, threads, a.ctas_per_sm);
    k_numeric_oz<MAXN><<<*grid, threads, smem, s>>>(a);
    count_launch(1);
    return cudaGetLastError();
}

template <int PREC, bool FF, int PM, int PN, bool DUAL>
cudaError_t launch_tc_inst(const NumericArgs &a, cudaStream_t s, int threads, int *grid) {
    const size_t smem = sizeof(uint32_t) * (size_t)ring_words_per_warp<PREC, PM, PN>() * (threads / 32);
    cudaError_t e = cudaFuncSetAttribute(k_numeric_tc<PREC, FF, PM, PN, DUAL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    *grid = persistent_grid(k_numeric_tc<PREC, FF, PM, PN, DUAL>, a.n_items, smem, threads, a.ctas_per_sm);
    k_numeric_tc<PREC, FF, PM, PN, DUAL><<<*grid, threads, smem, s>>>(a);
    count_launch(1);
    return cudaGetLastError();
}

// 1-row instances with two accumulators where F > 1 block products share the
// tensor core's sum
template <int PREC, bool FF, int PM, int PN>
cudaError_t launch_tc_pass(const NumericArgs &a, cudaStream_t s, int threads, int *grid) {
    const int F = a.flush_every > 0 ? a.flush_every : (a.flush_every < 0 ? -a.flush_every : 1);
    if constexpr (PM == 1) {
        if (F > 1) return launch_tc_inst<PREC, FF, PM, PN, true>(a, s, threads, grid);
    }
    return launch_tc_inst<PREC, FF, PM, PN, false>(a, s, threads, grid);
}

template <int PREC, bool FF, int PM>
cudaError_t launch_tc_pm(const NumericArgs &a, cudaStream_t s, int threads, int *grid, int pn) {
    if (pn >= 3) return launch_tc_pass<PREC, FF, PM, 3>(a, s, threads, grid);
    if (pn == 2) return launch_tc_pass<PREC, FF, PM, 2>(a, s, threads, grid);
    return launch_tc_pass<PREC, FF, PM, 1>(a, s, threads, grid);
}

// The instance by the largest pass asked for (pass_mt 1 or 2, pass_nt 1..3;
// default 2 x 3), or -- with item groups, the default -- the blocks of two
// tile rows and more in a 2 x PN instance and those of one tile row in a
// 1 x PN instance (fewer registers and a smaller ring: more warps per SM);
// then the lane items.
template <int PREC, bool FF>
cudaError_t launch_tc_ff(const NumericArgs &a, cudaStream_t s, int threads, int *grid) {
    const int pm = a.pass_mt > 0 ? a.pass_mt : 2, pn = a.pass_nt > 0 ? a.pass_nt : 3;
    cudaError_t e;
    if (a.item_groups) {
        NumericArgs b = a;
        b.group = 0;
        e = launch_tc_pm<PREC, FF, 2>(b, s, threads, grid, pn);
        if (e == cudaSuccess) {
            int g1 = 0;
            b.group = 1;
            e = launch_tc_pm<PREC, FF, 1>(b, s, threads, &g1, pn);
        }
    } else {
        NumericArgs b = a;
        b.group = -1;
        e = pm >= 2 ? launch_tc_pm<PREC, FF, 2>(b, s, threads, grid, pn)
                    : launch_tc_pm<PREC, FF, 1>(b, s, threads, grid, pn);
    }
    if (e == cudaSuccess && a.n_lane_items) {
        const int g = persistent_grid(k_numeric_tc_lane<PREC, FF>, a.n_items / 32 + 1, 0, kThreadsNum, a.ctas_per_sm);
        k_numeric_tc_lane<PREC, FF><<<g, kThreadsNum, 0, s>>>(a);
        count_launch(1);
        e = cudaGetLastError();
    }
    return e;
}

template <int PREC>
cudaError_t launch_tc(const NumericArgs &a, cudaStream_t s, int threads, int *grid) {
    return a.flush_every > 0 ? launch_tc_ff<PREC, false>(a, s, threads, grid)
                             : launch_tc_ff<PREC, true>(a, s, threads, grid);
}

}  // namespace

cudaError_t launch_numeric(const NumericArgs &a, cudaStream_t s, NumericLaunch *info) {
    NumericLaunch li{BSM_K_NONE, -1, 0, 0, 0, 0};
    if (info) *info = li;
    if (a.n_items == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.work_counter, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool tc = a.prec == BSM_P_TF32x3 || a.prec == BSM_P_BF16x3 || a.prec == BSM_P_BF16x6;
    // the mma.sync kernels run 2 or 4 warps per CTA (compiled for at most 4,
    // which keeps their register count at three CTAs per SM)
    const int tc_threads = (a.cta_warps == 2 ? 2 : 4) * 32;
    int grid = 0;
    if (a.prec == BSM_P_OZAKI) {
        // passes of up to 3 tiles (the default) take the instance with the
        // wider ring; with item groups the blocks of one tile column run in
        // the 1-tile instance
        const bool wide = a.pass_nt != 1 && a.pass_nt != 2;
        NumericArgs b = a;
        b.group = a.item_groups ? 0 : -1;
        e = wide ? launch_oz<3>(b, s, tc_threads, &grid) : launch_oz<2>(b, s, tc_threads, &grid);
        if (e == cudaSuccess && a.item_groups) {
            int g1 = 0;
            b.group = 1;
            e = launch_oz<1>(b, s, tc_threads, &g1);
        }
        if (e == cudaSuccess && a.n_lane_items) {
            const int g = persistent_grid(k_numeric_oz_lane, a.n_items / 32 + 1, 0, kThreadsNum, a.ctas_per_sm);
            k_numeric_oz_lane<<<g, kThreadsNum, 0, s>>>(a);
            count_launch(1);
            e = cudaGetLastError();
        }
        li = NumericLaunch{BSM_K_OZAKI_MMA, -1, tc_threads, grid, 1, wide ? 3 : (a.pass_nt == 1 ? 1 : 2)};
    } else if (a.prec == BSM_P_FP64_DMMA && a.dtype == BSM_FP64) {
        grid = persistent_grid(k_numeric_dmma, a.n_items, 0, kThreadsNum, a.ctas_per_sm);
        k_numeric_dmma<<<grid, kThreadsNum, 0, s>>>(a);
        li = NumericLaunch{BSM_K_FP64_MMA, -1, kThreadsNum, grid, a.pass_mt > 0 ? a.pass_mt : 3,
                           a.pass_nt > 0 ? a.pass_nt : 3};
    } else if (!tc) {
        // the build by the largest output block: all within one narrow pass
        // (<= 288 elements) or beyond the wide ladder's single pass (> 768)
        // run narrow -- measured faster there -- the rest wide; the tuner may
        // ask for narrow or wide instead (the small build only ever runs when
        // every output block has at most 16 elements)
        const int area = a.max_out_rows * a.max_out_cols;
        int build = (area > 0 && area <= 16) ? kCcSmall : (area <= 288 || area > 768) ? kCcNarrow : kCcWide;
        if (a.fp64_build == 1 && build != kCcSmall) build = kCcNarrow;
        if (a.fp64_build == 2 && build != kCcSmall) build = kCcWide;
        if (a.dtype == BSM_FP64) {
            if (build == kCcSmall) grid = launch_cc<double, kCcSmall>(a, s);
            else if (build == kCcNarrow) grid = launch_cc<double, kCcNarrow>(a, s);
            else grid = launch_cc<double, kCcWide>(a, s);
        } else {
            if (build == kCcSmall) grid = launch_cc<float, kCcSmall>(a, s);
            else if (build == kCcNarrow) grid = launch_cc<float, kCcNarrow>(a, s);
            else grid = launch_cc<float, kCcWide>(a, s);
        }
        li = NumericLaunch{BSM_K_FP64_CORES, build, kThreadsNum, grid, 0, 0};
    } else {
        if (a.prec == BSM_P_TF32x3) e = launch_tc<BSM_P_TF32x3>(a, s, tc_threads, &grid);
        else if (a.prec == BSM_P_BF16x3) e = launch_tc<BSM_P_BF16x3>(a, s, tc_threads, &grid);
        else e = launch_tc<BSM_P_BF16x6>(a, s, tc_threads, &grid);
        li = NumericLaunch{BSM_K_SPLIT_MMA, -1, tc_threads, grid,
                           a.item_groups ? 0 : (a.pass_mt > 0 ? a.pass_mt : 2), a.pass_nt > 0 ? a.pass_nt : 3};
    }
    if (e != cudaSuccess) return e;
    if (info) *info = li;
    if (!tc && a.prec != BSM_P_OZAKI) count_launch(1);  // the split and Ozaki paths count their own
    return cudaGetLastError();
}

uint32_t numeric_debug_bits(cudaStream_t s) {
#ifdef BSM_DEBUG
    uint32_t bits = 0;
    const uint32_t zero = 0;
    if (cudaMemcpyFromSymbolAsync(&bits, g_dbg_bits, sizeof(bits), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(g_dbg_bits, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return 0x80000000u;
    }
    return bits;
#else
    (void)s;
    return 0;
#endif
}

cudaError_t launch_split_plain(const bsm_mat *M, int prec, float *out, cudaStream_t s) {
    if (M->data_len == 0) return cudaSuccess;
    int64_t g = (M->data_len + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    const bool f64 = M->dtype == BSM_FP64;
    if (prec == BSM_P_TF32x3) {
        if (f64) k_split_plain<double, BSM_P_TF32x3><<<(unsigned)g, 256, 0, s>>>(M->data_len, static_cast<const double *>(M->data), out);
        else k_split_plain<float, BSM_P_TF32x3><<<(unsigned)g, 256, 0, s>>>(M->data_len, static_cast<const float *>(M->data), out);
    } else if (prec == BSM_P_BF16x3) {
        if (f64) k_split_plain<double, BSM_P_BF16x3><<<(unsigned)g, 256, 0, s>>>(M->data_len, static_cast<const double *>(M->data), out);
        else k_split_plain<float, BSM_P_BF16x3><<<(unsigned)g, 256, 0, s>>>(M->data_len, static_cast<const float *>(M->data), out);
    } else {
        if (f64) k_split_plain<double, BSM_P_BF16x6><<<(unsigned)g, 256, 0, s>>>(M->data_len, static_cast<const double *>(M->data), out);
        else k_split_plain<float, BSM_P_BF16x6><<<(unsigned)g, 256, 0, s>>>(M->data_len, static_cast<const float *>(M->data), out);
    }
    count_launch(1);
    return cudaGetLastError();
}

int split_pieces(int prec) { return prec == BSM_P_BF16x6 ? 3 : 2; }

cudaError_t launch_oz_lines(const bsm_mat *M, int by_rows, int32_t *line0, int32_t *exps, cudaStream_t s) {
    if (M->nnzb == 0) return cudaSuccess;
    if (M->dtype != BSM_FP64 || !M->row_start || !M->col_start) return cudaErrorInvalidValue;
    int64_t g = ((int64_t)M->nbr * 32 + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_oz_line0<<<(unsigned)g, 256, 0, s>>>(M->nbr, M->row_ptr, M->col_idx, M->row_start, M->col_start, by_rows,
                                           line0);
    g = (M->nnzb * 32 + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_oz_line_exp<<<(unsigned)g, 256, 0, s>>>(M->nnzb, M->blk_off, M->blk_rc, static_cast<const double *>(M->data),
                                              line0, by_rows, exps);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_mark_variant(int64_t n, int32_t *order, const int32_t *blk_rc, const int32_t *size_index, int32_t ns,
                                const int8_t *variant_of_class, unsigned long long *marked, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_mark_variant<<<(unsigned)g, 256, 0, s>>>(n, order, blk_rc, size_index, ns, variant_of_class, marked);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_sizes(const bsm_mat *M, int role_y, int trans, int prec, int64_t *pack_words,
                              cudaStream_t s) {
    if (M->nnzb == 0) return cudaSuccess;
    int64_t g = (M->nnzb + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_pack_sizes<<<(unsigned)g, 256, 0, s>>>(M->nnzb, M->blk_rc, role_y, trans, prec, pack_words);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pack(const bsm_mat *M, int role_y, int trans, int prec, const int64_t *pack_off,
                        void *pack, const int32_t *status, cudaStream_t s, const int32_t *line0,
                        const int32_t *exps) {
    if (M->nnzb == 0) return cudaSuccess;
    int64_t g = (M->nnzb * 32 + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    uint32_t *p = static_cast<uint32_t *>(pack);
    const bool f64 = M->dtype == BSM_FP64;
    if (prec == BSM_P_OZAKI) {
        if (!f64 || !line0 || !exps) return cudaErrorInvalidValue;
        k_pack_oz<<<(unsigned)g, 256, 0, s>>>(M->nnzb, M->blk_off, M->blk_rc, static_cast<const double *>(M->data),
                                              role_y, trans, pack_off, p, line0, exps, status);
        count_launch(1);
        return cudaGetLastError();
    }
#define BSM_PACK_CASE(PREC)                                                                           \
    if (f64)                                                                                          \
        k_pack<double, PREC><<<(unsigned)g, 256, 0, s>>>(M->nnzb, M->blk_off, M->blk_rc,              \
                                                         static_cast<const double *>(M->data), role_y, \
                                                         trans, pack_off, p, status);                         \
    else                                                                                              \
        k_pack<float, PREC><<<(unsigned)g, 256, 0, s>>>(M->nnzb, M->blk_off, M->blk_rc,               \
                                                        static_cast<const float *>(M->data), role_y,   \
                                                        trans, pack_off, p, status);
    if (prec == BSM_P_TF32x3) {
        BSM_PACK_CASE(BSM_P_TF32x3)
    } else if (prec == BSM_P_BF16x3) {
        BSM_PACK_CASE(BSM_P_BF16x3)
    } else {
        BSM_PACK_CASE(BSM_P_BF16x6)
    }
#undef BSM_PACK_CASE
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace bsm
