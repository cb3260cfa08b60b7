// Allocation-free sizing entry point: bsm_count_products_static.
//
// Some callers cannot allocate device memory at the moment they need to
// size a product: code that runs inside another framework's memory pool or
// arena and must not grow it behind its back, or a host thread that may not
// call cudaMalloc / cudaFree because those calls synchronise the device.  For
// them this file offers the per-row count of the symbolic phase with all of
// its scratch (the FP64 block norms of A and B) in one fixed, file-scope
// device array instead of memory allocated per call.
//
// The array is 16 MiB (2^21 doubles): nnzb(A) + nnzb(B) may be at most
// 2,097,152 blocks when filter_eps > 0 (no scratch is needed otherwise).
// Every GPU that loads the library holds those 16 MiB until the process
// exits.  Every call uses the same array, so calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it; calls
// issued one after another on one stream are safe.
#include <cuda_runtime.h>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int64_t kStaticNormCapacity = int64_t(1) << 21;  // doubles (16 MiB)
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_static_norms[kStaticNormCapacity];

// Host copy of each device's address of g_static_norms, with the id of the
// CUDA context it was looked up in.  In host code the name g_static_norms is
// only a stand-in for the symbol, never a device address.  The address is
// looked up again when the current context is not the recorded one (after
// cudaDeviceReset the primary context is re-created and the module reloaded,
// so the array may move), and on every call when the context id cannot be
// read.
struct StaticAddr {
    double *addr = nullptr;
    unsigned long long ctx_id = 0;
};
StaticAddr g_static_norms_addr[kMaxDevices];

// Id of the current CUDA context (0 if there is none or it cannot be read),
// through the driver entry points the runtime exposes, so the library does
// not link the driver library itself.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
    }
    if (!get_cur || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != 0 || !ctx) return 0;
    if (get_id(ctx, &id) != 0) return 0;
    return id;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per C block row i: kept products, distinct C block columns, and the totals
// (kept products, filtered candidates, sum of m*n*k) added into totals[0..2].
// Same filter rule as the multiply: keep A_ik.B_kj iff eps <= 0 or
// norm(A_ik) * norm(B_kj) > eps (on-the-fly filtering, DBCSR §2).  The C
// column set lives in a shared-memory bitmap only.
__global__ void __launch_bounds__(kThreads)
    k_sym_count_static(SymbolicArgs a, int64_t *prod_cnt, int64_t *cblk_cnt, unsigned long long *totals) {
    extern __shared__ uint32_t bm[];
    __shared__ long long red[4][32];
    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int w = tid; w < a.nwords; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    long long cnt = 0, filt = 0, nk = 0;
    for (int64_t ai = a.a_row_ptr[i] + warp; ai < a.a_row_ptr[i + 1]; ai += nwarps) {
        const int32_t k = a.a_col_idx[ai];
        const int32_t kd = a.a_col_bs[k];
        const double na = a.use_filter ? a.a_norm[ai] : 0.0;
        for (int64_t b = a.b_row_ptr[k] + lane; b < a.b_row_ptr[k + 1]; b += 32) {
            const int32_t j = a.b_col_idx[b];
            if (!a.use_filter || __dmul_rn(na, a.b_norm[b]) > a.eps) {
                atomicOr(&bm[j >> 5], 1u << (j & 31));
                cnt++;
                nk += (long long)a.b_col_bs[j] * kd;
            } else {
                filt++;
            }
        }
    }
    __syncthreads();
    long long ncol = 0;
    for (int w = tid; w < a.nwords; w += blockDim.x) ncol += __popc(bm[w]);
    long long v[4] = {cnt, filt, nk, ncol};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long s = warp_sum(v[q]);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (tid == 0) {
        long long t[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
            for (int w = 0; w < nwarps; ++w) t[q] += red[q][w];
        prod_cnt[i] = t[0];
        cblk_cnt[i] = t[3];
        const long long m = a.a_row_bs[i];
        if (t[0]) atomicAdd(&totals[0], (unsigned long long)t[0]);
        if (t[1]) atomicAdd(&totals[1], (unsigned long long)t[1]);
        if (t[2]) atomicAdd(&totals[2], (unsigned long long)(m * t[2]));
    }
}

// Device address of the static scratch for the current device (and context).
bsm_status static_norms(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(BSM_ERR_UNSUPPORTED, "device index above 63");
    StaticAddr &sa = g_static_norms_addr[dev];
    const unsigned long long id = current_ctx_id();
    if (!sa.addr || id == 0 || id != sa.ctx_id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_norms);
        if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress of the static norm scratch");
        sa.addr = static_cast<double *>(p);
        sa.ctx_id = current_ctx_id();  // the lookup made the device's context current
    }
    *out = sa.addr;
    return BSM_OK;
}

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" bsm_status bsm_count_products_static(bsm_t A, bsm_t B, double filter_eps, int64_t *prod_cnt,
                                                int64_t *cblk_cnt, int64_t *totals) {
    if (!A || !B) return set_error(BSM_ERR_ARG, "NULL matrix");
    if (!totals || (A->nbr > 0 && (!prod_cnt || !cblk_cnt))) return set_error(BSM_ERR_ARG, "NULL output");
    if (A->dtype != B->dtype) return set_error(BSM_ERR_ARG, "A and B must share a dtype");
    if (A->nbc != B->nbr || A->h_col_bs != B->h_row_bs)
        return set_error(BSM_ERR_BLOCKING, "A's block columns do not match B's block rows");
    if (filter_eps != filter_eps) return set_error(BSM_ERR_ARG, "filter_eps is NaN");
    const bool use_filter = filter_eps > 0.0;
    const int64_t need = use_filter ? A->nnzb + (B == A ? 0 : B->nnzb) : 0;
    if (need > kStaticNormCapacity)
        return set_error(BSM_ERR_CAPACITY,
                         "nnzb(A) + nnzb(B) = " + std::to_string(need) +
                             " exceeds the static norm scratch of 2097152 blocks; use bsm_multiply");
    const int32_t nwords = (B->nbc + 31) / 32;
    const int smem = nwords * (int)sizeof(uint32_t);
    if (smem > 200 * 1024) return set_error(BSM_ERR_UNSUPPORTED, "too many block columns");
    cudaStream_t s = stream();
    double *scratch = nullptr;
    bsm_status st;
    if (use_filter && (st = static_norms(&scratch))) return st;
    cudaError_t e = cudaMemsetAsync(totals, 0, 3 * sizeof(int64_t), s);
    if (e == cudaSuccess && use_filter) {
        e = launch_block_norms(A, scratch, s);
        if (e == cudaSuccess && B != A) e = launch_block_norms(B, scratch + A->nnzb, s);
    }
    if (e != cudaSuccess) return cuda_check(e, "static count norms");
    if (A->nbr == 0) return BSM_OK;
    SymbolicArgs sa{};
    sa.nbr = A->nbr; sa.nbk = A->nbc; sa.nbc = B->nbc;
    sa.a_row_bs = A->row_bs; sa.a_col_bs = A->col_bs; sa.a_row_ptr = A->row_ptr; sa.a_col_idx = A->col_idx;
    sa.a_norm = scratch;
    sa.b_row_ptr = B->row_ptr; sa.b_col_idx = B->col_idx; sa.b_col_bs = B->col_bs;
    sa.b_norm = use_filter ? (B == A ? scratch : scratch + A->nnzb) : nullptr;
    sa.eps = filter_eps;
    sa.use_filter = use_filter ? 1 : 0;
    sa.nwords = nwords;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_sym_count_static, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute");
    }
    k_sym_count_static<<<A->nbr, kThreads, smem, s>>>(sa, prod_cnt, cblk_cnt,
                                                      reinterpret_cast<unsigned long long *>(totals));
    count_launch(1);
    return cuda_check(cudaGetLastError(), "static count");
}
