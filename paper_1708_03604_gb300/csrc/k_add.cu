// Block add Z = a*X + b*Y over the union of two block patterns, and the
// norm filter that drops blocks whose FP64 Frobenius norm does not exceed a
// threshold followed by the compaction of the survivors.  Both serve the
// purification chain X <- 3 X^2 - 2 X^3 and the optional post-filter of a
// product (filtering of DBCSR, Bethune et al. 2017 §2).
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "bsm_internal.cuh"

namespace bsm {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int threads = kThreads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

// number of entries of sorted v[0..n) that are < key
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *v, int64_t n, int32_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (v[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct Pat {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *blk_off;
    const int32_t *col_bs;
    const int32_t *row_bs;
};

inline Pat pat_of(const bsm_mat &m) {
    return Pat{m.row_ptr, m.col_idx, m.blk_off, m.col_bs, m.row_bs};
}

// per row: |union| and the union's element count
__global__ void k_add_count(int32_t nbr, Pat x, Pat y, int64_t *ccnt, int64_t *celem) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nbr; i += nwarp) {
        const int32_t *xc = x.col_idx + x.row_ptr[i];
        const int32_t *yc = y.col_idx + y.row_ptr[i];
        const int64_t nx = x.row_ptr[i + 1] - x.row_ptr[i], ny = y.row_ptr[i + 1] - y.row_ptr[i];
        long long c = 0, w = 0;
        for (int64_t q = lane; q < nx; q += 32) {
            c++;
            w += x.col_bs[xc[q]];
        }
        for (int64_t q = lane; q < ny; q += 32) {
            const int32_t j = yc[q];
            const int64_t pos = lower_bound_i32(xc, nx, j);
            if (pos == nx || xc[pos] != j) {
                c++;
                w += y.col_bs[j];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (lane == 0) {
            ccnt[i] = c;
            celem[i] = (int64_t)x.row_bs[i] * w;
        }
    }
}

// per row: the union in column order (one lane merges the two sorted lists),
// then element offsets by a warp scan
__global__ void k_add_fill(int32_t nbr, Pat x, Pat y, AddFill f, const int32_t *status) {
    const int lane = threadIdx.x & 31;
    if (status && *status != 0) return;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nbr; i += nwarp) {
        const int64_t xb = x.row_ptr[i], yb = y.row_ptr[i];
        const int32_t *xc = x.col_idx + xb;
        const int32_t *yc = y.col_idx + yb;
        const int64_t nx = x.row_ptr[i + 1] - xb, ny = y.row_ptr[i + 1] - yb;
        const int64_t z0 = f.zrow_ptr[i];
        const int64_t nz = f.zrow_ptr[i + 1] - z0;
        const int32_t m = x.row_bs[i];
        if (lane == 0) {
            // sequential merge of the two ascending column lists
            int64_t px = 0, py = 0, p = 0;
            while (px < nx || py < ny) {
                const int32_t jx = px < nx ? xc[px] : INT32_MAX;
                const int32_t jy = py < ny ? yc[py] : INT32_MAX;
                const int32_t j = jx < jy ? jx : jy;
                f.z_col_idx[z0 + p] = j;
                f.x_src[z0 + p] = (jx == j) ? x.blk_off[xb + px++] : -1;
                f.y_src[z0 + p] = (jy == j) ? y.blk_off[yb + py++] : -1;
                ++p;
            }
        }
        __syncwarp();
        int64_t run = f.zelem_ptr[i];
        for (int64_t base = 0; base < nz; base += 32) {
            const int64_t q = base + lane;
            const int32_t n = q < nz ? x.col_bs[f.z_col_idx[z0 + q]] : 0;
            int64_t v = (int64_t)m * n, incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (q < nz) {
                f.z_blk_off[z0 + q] = run + incl - v;
                f.z_blk_rc[z0 + q] = (m << 16) | n;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// z = a*x + b*y element by element, evaluated as one rounded product and
// one rounded sum (no fused multiply-add)
template <typename T>
__global__ void k_add_values(int64_t nnzb, const int64_t *z_off, const int32_t *z_rc, const int64_t *xs,
                             const int64_t *ys, double a, const T *x, double b, const T *y, T *z,
                             const int32_t *status) {
    const int lane = threadIdx.x & 31;
    if (status && *status != 0) return;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = wid; q < nnzb; q += nwarp) {
        const int32_t rc = z_rc[q];
        const int len = rc_rows(rc) * rc_cols(rc);
        const int64_t xo = xs[q], yo = ys[q], zo = z_off[q];
        for (int e = lane; e < len; e += 32) {
            double v;
            if (xo >= 0 && yo >= 0)
                v = __dadd_rn(__dmul_rn(a, (double)x[xo + e]), __dmul_rn(b, (double)y[yo + e]));
            else if (xo >= 0)
                v = __dmul_rn(a, (double)x[xo + e]);
            else
                v = __dmul_rn(b, (double)y[yo + e]);
            z[zo + e] = (T)v;
        }
    }
}

__global__ void k_keep_flags(int64_t nnzb, const double *norms, double eps, int64_t *keep) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnzb;
         b += (int64_t)gridDim.x * blockDim.x)
        keep[b] = (norms[b] > eps) ? 1 : 0;
}

__global__ void k_row_keep_counts(int32_t nbr, const int64_t *row_ptr, const int64_t *keep,
                                  const int32_t *blk_rc, int64_t *row_cnt, int64_t *row_elem) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nbr; i += nwarp) {
        long long c = 0, e = 0;
        for (int64_t b = row_ptr[i] + lane; b < row_ptr[i + 1]; b += 32)
            if (keep[b]) {
                c++;
                e += (long long)rc_rows(blk_rc[b]) * rc_cols(blk_rc[b]);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        if (lane == 0) {
            row_cnt[i] = c;
            row_elem[i] = e;
        }
    }
}

template <typename T>
__global__ void k_compact(CompactArgs c) {
    const int lane = threadIdx.x & 31;
    if (c.status && *c.status != 0) return;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const T *src = static_cast<const T *>(c.data);
    T *dst = static_cast<T *>(c.n_data);
    for (int64_t i = wid; i < c.nbr; i += nwarp) {
        int64_t run = c.nelem_ptr[i];
        const int64_t b0 = c.row_ptr[i], b1 = c.row_ptr[i + 1];
        for (int64_t base = b0; base < b1; base += 32) {
            const int64_t b = base + lane;
            const bool kept = b < b1 && (c.keep_scan[b + 1] - c.keep_scan[b]) != 0;
            const int32_t rc = kept ? c.blk_rc[b] : 0;
            const int64_t len = kept ? (int64_t)rc_rows(rc) * rc_cols(rc) : 0;
            int64_t incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (kept) {
                const int64_t nb = c.keep_scan[b];
                c.n_col_idx[nb] = c.col_idx[b];
                c.n_blk_off[nb] = run + incl - len;
                c.n_blk_rc[nb] = rc;
            }
            // copy the kept blocks of this group, one block at a time
            unsigned mask = __ballot_sync(0xffffffffu, kept);
            int64_t grp_off = run;
            while (mask) {
                const int src_lane = __ffs(mask) - 1;
                mask &= mask - 1;
                const int64_t sb = __shfl_sync(0xffffffffu, b, src_lane);
                const int64_t sl = __shfl_sync(0xffffffffu, len, src_lane);
                const int64_t so = __shfl_sync(0xffffffffu, incl - len, src_lane);
                const T *s = src + c.blk_off[sb];
                T *d = dst + grp_off + so;
                for (int64_t e = lane; e < sl; e += 32) d[e] = s[e];
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

__global__ void k_compact_i64(int64_t nnzb, const int64_t *kscan, const int64_t *src, int64_t *dst,
                              const int32_t *status) {
    if (status && *status != 0) return;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnzb;
         b += (int64_t)gridDim.x * blockDim.x)
        if (kscan[b + 1] != kscan[b]) dst[kscan[b]] = src[b];
}

template <typename T>
__global__ void k_add_backward(int64_t nnzb, const int64_t *z_off, const int32_t *z_rc, const int64_t *xs,
                               const int64_t *ys, double a, double b, const T *dz, T *dx, T *dy) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = wid; q < nnzb; q += nwarp) {
        const int32_t rc = z_rc[q];
        const int len = rc_rows(rc) * rc_cols(rc);
        const int64_t xo = xs[q], yo = ys[q], zo = z_off[q];
        for (int e = lane; e < len; e += 32) {
            const double g = (double)dz[zo + e];
            if (dx && xo >= 0) dx[xo + e] = (T)(a * g);
            if (dy && yo >= 0) dy[yo + e] = (T)(b * g);
        }
    }
}

}  // namespace

cudaError_t launch_compact_i64(int64_t nnzb, const int64_t *kscan, const int64_t *src, int64_t *dst,
                               const int32_t *status, cudaStream_t s) {
    if (nnzb == 0) return cudaSuccess;
    k_compact_i64<<<grid_for(nnzb), kThreads, 0, s>>>(nnzb, kscan, src, dst, status);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_add_backward(int64_t nnzb, const int64_t *z_blk_off, const int32_t *z_blk_rc,
                                const int64_t *x_src, const int64_t *y_src, double a, double b, const void *dZ,
                                void *dX, void *dY, int32_t dtype, cudaStream_t s) {
    if (nnzb == 0) return cudaSuccess;
    const int g = grid_for(nnzb * 32);
    if (dtype == BSM_FP64)
        k_add_backward<double><<<g, kThreads, 0, s>>>(nnzb, z_blk_off, z_blk_rc, x_src, y_src, a, b,
                                                       static_cast<const double *>(dZ), static_cast<double *>(dX),
                                                       static_cast<double *>(dY));
    else
        k_add_backward<float><<<g, kThreads, 0, s>>>(nnzb, z_blk_off, z_blk_rc, x_src, y_src, a, b,
                                                      static_cast<const float *>(dZ), static_cast<float *>(dX),
                                                      static_cast<float *>(dY));
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_add_count(const bsm_mat *X, const bsm_mat *Y, int64_t *ccnt, int64_t *celem,
                             cudaStream_t s) {
    if (X->nbr == 0) return cudaSuccess;
    k_add_count<<<grid_for((int64_t)X->nbr * 32), kThreads, 0, s>>>(X->nbr, pat_of(*X), pat_of(*Y), ccnt,
                                                                   celem);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_add_fill(const bsm_mat *X, const bsm_mat *Y, const AddFill &f, const int32_t *status,
                            cudaStream_t s) {
    if (X->nbr == 0) return cudaSuccess;
    k_add_fill<<<grid_for((int64_t)X->nbr * 32), kThreads, 0, s>>>(X->nbr, pat_of(*X), pat_of(*Y), f, status);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_add_values(int64_t nnzb, const int64_t *z_blk_off, const int32_t *z_blk_rc,
                              const int64_t *x_src, const int64_t *y_src, double a, const void *x, double b,
                              const void *y, void *z, int32_t dtype, const int32_t *status, cudaStream_t s) {
    if (nnzb == 0) return cudaSuccess;
    const int g = grid_for(nnzb * 32);
    if (dtype == BSM_FP64)
        k_add_values<double><<<g, kThreads, 0, s>>>(nnzb, z_blk_off, z_blk_rc, x_src, y_src, a,
                                                     static_cast<const double *>(x), b,
                                                     static_cast<const double *>(y), static_cast<double *>(z),
                                                     status);
    else
        k_add_values<float><<<g, kThreads, 0, s>>>(nnzb, z_blk_off, z_blk_rc, x_src, y_src, a,
                                                    static_cast<const float *>(x), b,
                                                    static_cast<const float *>(y), static_cast<float *>(z),
                                                    status);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_keep_flags(int64_t nnzb, const double *norms, double eps, int64_t *keep, cudaStream_t s) {
    if (nnzb == 0) return cudaSuccess;
    k_keep_flags<<<grid_for(nnzb), kThreads, 0, s>>>(nnzb, norms, eps, keep);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_row_keep_counts(int32_t nbr, const int64_t *row_ptr, const int64_t *keep,
                                   const int32_t *blk_rc, int64_t *row_cnt, int64_t *row_elem,
                                   cudaStream_t s) {
    if (nbr == 0) return cudaSuccess;
    k_row_keep_counts<<<grid_for((int64_t)nbr * 32), kThreads, 0, s>>>(nbr, row_ptr, keep, blk_rc, row_cnt,
                                                                      row_elem);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_compact(const CompactArgs &c, cudaStream_t s) {
    if (c.nbr == 0) return cudaSuccess;
    const int g = grid_for((int64_t)c.nbr * 32);
    if (c.dtype == BSM_FP64) k_compact<double><<<g, kThreads, 0, s>>>(c);
    else k_compact<float><<<g, kThreads, 0, s>>>(c);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace bsm
