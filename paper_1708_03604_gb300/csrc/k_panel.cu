// Row-panel numeric kernel on the fifth-generation tensor cores (tcgen05,
// accumulators in tensor memory), TF32x3 split precision, for matrices whose
// blocks all have one size s <= 24.
//
// The local multiply (Bethune et al. 2017 §2: C = C + A.B as a sum of small
// dense block products) is regrouped into dense output tiles: 5 block rows of
// C by 5 block columns of C.  For every block index k for which some A_ik of
// the tile's rows and some B_kj of its columns are present, one k-step
// multiplies the 5 A blocks (absent ones read as zeros) stacked into a 120 x 24
// panel (rows padded to 128) by the 5 B blocks side by side (24 x 120, padded
// to 128 columns): a 128 x 128 x 24 product, three MMAs of K = 8 for each of
// the three TF32 piece products lo.hi, hi.lo and hi.hi (the split and the
// order of the mma.sync TF32x3 path).  Three consecutive k-steps of a tile
// accumulate in FP32 inside the tensor core (rounding toward zero, as
// measured: at most 3 x 72 terms per sum); each such sum is added on the CUDA
// cores into a compensated pair held in the drain threads' registers (Kahan
// summation as on the mma.sync path, the FP32 sum as there, the compensation
// term kept in BF16: at most 2^-33 of the sum lost per add), and converted to
// FP64 once per tile.  Products the tile computes for absent
// blocks are exact zeros.  A product removed by the norm filter would still
// be computed inside the dense tile, so the launcher uses this kernel only
// when the filter removed none.
//
// The k-steps of every tile (a merge of its five A rows' and five B columns'
// sorted block-index lists) are written beforehand by k_panel_steps, one warp
// per tile, as records of 10 block indices.  Roles in one persistent CTA per
// SM of the numeric kernel (12 warps):
//   warp 0      tickets: takes tiles from an atomic ticket and hands each,
//               with its range of k-step records, to the copy warps through a
//               shared ring;
//   warps 1, 2  copy: stage the 10 blocks of every k-step (warp 1 A's, warp 2
//               B's; the block indices of 32 k-steps per coalesced load), one
//               bulk copy of 4608 bytes per block pre-packed in the tensor
//               core's shared-memory layout (absent blocks from a zero block),
//               completion counted in bytes on the stage's "full" barrier
//               (4-stage ring);
//   warp 3      allocates tensor memory; one lane issues the MMAs of a k-step
//               into accumulator buffer b and commits them to the stage's
//               "empty" barrier and, every third k-step, to the buffer's
//               "full" barrier;
//   warps 4..11 drain: each owns one 32-lane quarter of tensor memory (32 rows
//               of the tile) and one half of its columns, reads the buffer
//               into registers, frees it, adds it into the compensated pair,
//               and on a tile's last k-step writes C.
// Every wait is bounded (2 s by default; the main-loop waits take
// PanelArgs::wait_ns, which tests shorten to make a wait run out); a wait that
// runs out sets the output's status word to BSM_ERR_TIMEOUT, every role then
// leaves its loop, waits (bounded by the full 2 s) for its own copies and MMAs
// in flight, and the tensor memory is freed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kSlot = 24;                 // rows (and k) of one block slot
constexpr int kRB = 5, kCB = 5;           // block rows / block columns of a tile
constexpr int kChunks = kSlot / 4;        // 16-byte chunks of one 24-term row
// In shared memory and in the packs the TF32 hi and lo planes of an operand
// alternate by row group: row group g (8 rows x 24 k) of the hi plane at byte
// g * 1536, of the lo plane at g * 1536 + 768, so that one block (3 row
// groups) is 4608 contiguous bytes.  Inside a row group the six 16-byte
// k-chunks are 8-row x 16-byte core matrices of 128 bytes.
constexpr int kGroup = kChunks * 128;     // bytes of one plane's row group: 768
constexpr int kGroupStride = 2 * kGroup;  // hi and lo row groups side by side: 1536
constexpr int kBlk = 3 * kGroupStride;    // bytes of one packed block (hi and lo): 4608
constexpr int kOperand = 16 * kGroupStride;  // one operand of a stage, 128 rows: 24576
constexpr int kStageBytes = 2 * kOperand;    // A, then B
constexpr int kStages = 4;
constexpr int kRing = 8;                  // tiles handed from the ticket warp to the copy warps
constexpr int kPre = 4;                   // list entries the merge loads ahead
constexpr int kPair = 3;                  // default k-steps summed in one accumulator buffer before a drain
constexpr int kCopyWarps = 2, kMmaWarp = 3, kDrainWarps = 8;
constexpr int kThreads = 32 * (2 + kCopyWarps + kDrainWarps);
constexpr unsigned long long kWaitNs = 2000000000ull;  // a wait gives up after 2 s
// instruction descriptor: D F32, A and B TF32, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr int kFirst = 1, kLast = 2, kDone = 4;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: 8-row x 16-byte core matrices,
// `lbo` bytes between core matrices along K, `sbo` bytes along M / N
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the fifth-generation tensor cores
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}
// bounded wait for the phase of the given parity; false when it gave up or
// when another role of the CTA has given up (*abort set)
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, const int32_t *abort,
                                          unsigned long long limit_ns = kWaitNs) {
    // each try_wait suspends the thread (no issue slots taken) until the
    // phase completes or the hinted time (20 us, less under a shorter limit)
    // passes
    const uint32_t hint = limit_ns < 20000ull ? (uint32_t)limit_ns : 20000u;
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity), "r"(hint)
            : "memory");
        if (ok) return true;
        if (*(volatile const int32_t *)abort) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// compensated add of b into (hi, lo) (the update of the mma.sync TF32x3
// path) with the compensation lo held as BF16: lo is below half an ulp of hi,
// so rounding it to 8 bits costs at most 2^-9 of it, 2^-33 of hi, per add
__device__ __forceinline__ void kahan_b2(float &hi0, float &hi1, __nv_bfloat162 &lo, float b0, float b1) {
    const float2 l = __bfloat1622float2(lo);
    const float y0 = __fadd_rn(b0, l.x), y1 = __fadd_rn(b1, l.y);
    const float t0 = __fadd_rn(hi0, y0), t1 = __fadd_rn(hi1, y1);
    lo = __floats2bfloat162_rn(__fsub_rn(y0, __fsub_rn(t0, hi0)), __fsub_rn(y1, __fsub_rn(t1, hi1)));
    hi0 = t0;
    hi1 = t1;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------
// Packing: every block of an operand as two planes (TF32 hi, lo) of a 24 x 24
// zero-padded tile in the tensor core's K-major no-swizzle layout: element
// (row, k) of plane p at byte (row / 8) * 1536 + p * 768 + (k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4.  For A the rows are the block's rows; for B
// (trans = 1) the rows are the block's columns and k runs down the block.
// One warp per block.
__global__ void __launch_bounds__(256) k_panel_pack(const double *data, const int64_t *blk_off, int64_t nblk, int s,
                                                    int trans, uint32_t *out) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nblk) return;
    const double *blk = data + blk_off[warp];
    uint32_t *o = out + warp * (kBlk / 4);
    // one word of the hi plane and the matching word of the lo plane per step
    for (int w = lane; w < kBlk / 8; w += 32) {
        const int g = w / (kGroup / 4), within = w % (kGroup / 4);
        const int row = g * 8 + ((within & 31) >> 2);
        const int k = (within >> 5) * 4 + (within & 3);
        uint32_t h = 0, l = 0;
        if (row < s && k < s) {
            const double x = trans ? blk[(int64_t)k * s + row] : blk[(int64_t)row * s + k];
            h = to_tf32((float)x);
            l = to_tf32((float)(x - (double)__uint_as_float(h)));
        }
        o[g * (kGroupStride / 4) + within] = h;
        o[g * (kGroupStride / 4) + kGroup / 4 + within] = l;
    }
}

// ---------------------------------------------------------------------------
// Tiles: row group g = block rows ord_r[5g .. 5g+4], column group h = block
// columns ord_c[5h .. 5h+4]; a tile (g, h) exists when C has a block in it.
// One CTA per row group; a shared bitmap over the column groups.
__global__ void __launch_bounds__(128) k_panel_tile_count(int32_t nbr, const int32_t *ord_r, const int32_t *pos_c,
                                                          const int64_t *c_row_ptr, const int32_t *c_col,
                                                          int32_t ngc, int64_t *tile_cnt) {
    extern __shared__ uint32_t bits[];
    const int g = blockIdx.x;
    const int nw = (ngc + 31) >> 5;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0;
    __syncthreads();
    for (int r = 0; r < kRB; ++r) {
        const int p = g * kRB + r;
        if (p >= nbr) break;
        const int i = ord_r[p];
        for (int64_t b = c_row_ptr[i] + threadIdx.x; b < c_row_ptr[i + 1]; b += blockDim.x) {
            const int h = pos_c[c_col[b]] / kCB;
            atomicOr(&bits[h >> 5], 1u << (h & 31));
        }
    }
    __syncthreads();
    int cnt = 0;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) cnt += __popc(bits[w]);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    __shared__ int part[4];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) tile_cnt[g] = part[0] + part[1] + part[2] + part[3];
}

// tile_gh[t] = (g, h) in ascending h inside a row group; cblk[t][5 r + c] =
// index of C block (ord_r[5g + r], ord_c[5h + c]) or -1 (cblk preset to -1)
__global__ void __launch_bounds__(128) k_panel_tile_fill(int32_t nbr, const int32_t *ord_r, const int32_t *pos_c,
                                                         const int64_t *c_row_ptr, const int32_t *c_col, int32_t ngc,
                                                         const int64_t *tile_ptr, int32_t *tile_g, int32_t *tile_h,
                                                         int32_t *cblk) {
    extern __shared__ uint32_t sm[];
    const int g = blockIdx.x;
    const int nw = (ngc + 31) >> 5;
    uint32_t *bits = sm;
    uint32_t *pre = sm + nw;  // set bits before word w
    for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0;
    __syncthreads();
    for (int r = 0; r < kRB; ++r) {
        const int p = g * kRB + r;
        if (p >= nbr) break;
        const int i = ord_r[p];
        for (int64_t b = c_row_ptr[i] + threadIdx.x; b < c_row_ptr[i + 1]; b += blockDim.x) {
            const int h = pos_c[c_col[b]] / kCB;
            atomicOr(&bits[h >> 5], 1u << (h & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < nw; ++w) {
            pre[w] = run;
            run += __popc(bits[w]);
        }
    }
    __syncthreads();
    const int64_t t0 = tile_ptr[g];
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t m = bits[w];
        int64_t t = t0 + pre[w];
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            tile_g[t] = g;
            tile_h[t] = w * 32 + bit;
            ++t;
        }
    }
    for (int r = 0; r < kRB; ++r) {
        const int p = g * kRB + r;
        if (p >= nbr) break;
        const int i = ord_r[p];
        for (int64_t b = c_row_ptr[i] + threadIdx.x; b < c_row_ptr[i + 1]; b += blockDim.x) {
            const int pc = pos_c[c_col[b]];
            const int h = pc / kCB;
            const int64_t t = t0 + pre[h >> 5] + __popc(bits[h >> 5] & ((1u << (h & 31)) - 1u));
            cblk[t * (kRB * kCB) + r * kCB + (pc - h * kCB)] = (int32_t)b;
        }
    }
}

// processing order of the tiles: super tiles of SG row groups x SH column
// groups, so that the operand blocks of the tiles in flight stay in L2
__global__ void k_panel_tile_keys(int64_t ntiles, const int32_t *tile_g, const int32_t *tile_h, int sg, int sh,
                                  int32_t ngc, uint32_t *keys, int32_t *iota) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t ncs = (uint32_t)(ngc + sh - 1) / sh;
    keys[t] = (uint32_t)(tile_g[t] / sg) * ncs + (uint32_t)(tile_h[t] / sh);
    iota[t] = (int32_t)t;
}

// ---------------------------------------------------------------------------
struct TileRec {
    int32_t tile;    // -1: no more tiles
    int64_t s0, s1;  // its k-steps
};

struct SmemCtl {
    uint64_t full[kStages], empty[kStages];
    uint64_t accf[2], acce[2];
    uint64_t rec_full[kRing], rec_empty[kRing];
    uint64_t fin;
    TileRec rec[kRing];
    int32_t smeta_t[kStages], smeta_f[kStages];
    int32_t ameta_t[2], ameta_f[2];
    uint32_t tmem;
    int32_t abort;
};

__device__ __forceinline__ void fail(SmemCtl &ctl, int32_t *status) {
    ctl.abort = 1;
    atomicExch(status, (int32_t)BSM_ERR_TIMEOUT);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The k-steps of tile t in ascending inner block index k: every k for which
// some A_ik of the tile's 5 block rows and some B_kj of its 5 block columns
// are present (a merge of the 10 sorted lists, lanes 0..4 walking A's rows,
// lanes 8..12 B's columns, the next kPre entries of every list loaded ahead).
// emit(blk) is called once per k-step by every lane, blk being the block of
// the lane's row / column slot there (or -1); a tile without any such k (only
// blocks kept from the old C) gets one step with all blocks absent.
template <class F>
__device__ __forceinline__ void panel_merge(const PanelArgs &a, int32_t t, int lane, F &&emit) {
    const int32_t g = a.tile_g[t], h = a.tile_h[t];
    // cursors: lanes 0..4 walk A's rows, lanes 8..12 B's columns; the
    // next kPre entries of every list are loaded ahead
    int64_t p = 0, pe = 0;
    const bool is_b = lane >= 8 && lane < 8 + kCB;
    const int32_t *list = is_b ? a.b_t_row : a.a_col_idx;
    if (lane < kRB) {
        const int pr = g * kRB + lane;
        if (pr < a.nbr) {
            const int i = a.ord_r[pr];
            p = a.a_row_ptr[i];
            pe = a.a_row_ptr[i + 1];
        }
    } else if (is_b) {
        const int pc = h * kCB + lane - 8;
        if (pc < a.nbc) {
            const int j = a.ord_c[pc];
            p = a.b_t_ptr[j];
            pe = a.b_t_ptr[j + 1];
        }
    }
    // q: block index k of the next entries; bq: their block (B: from
    // the column-major list; A: the CSR position itself)
    uint32_t q[kPre];
    int32_t bq[kPre];
#pragma unroll
    for (int d = 0; d < kPre; ++d) {
        q[d] = p + d < pe ? (uint32_t)list[p + d] : 0xFFFFFFFFu;
        bq[d] = p + d < pe ? (is_b ? a.b_t_blk[p + d] : (int32_t)(p + d)) : -1;
    }
    auto next_step = [&](int32_t &blk) -> bool {
        for (;;) {
            const uint32_t k = __reduce_min_sync(0xffffffffu, q[0]);
            if (k == 0xFFFFFFFFu) return false;
            const bool mine = q[0] == k;
            const uint32_t am = __ballot_sync(0xffffffffu, mine && lane < kRB);
            const uint32_t bm = __ballot_sync(0xffffffffu, mine && is_b);
            blk = mine ? bq[0] : -1;
            if (mine) {
                ++p;
#pragma unroll
                for (int d = 0; d + 1 < kPre; ++d) {
                    q[d] = q[d + 1];
                    bq[d] = bq[d + 1];
                }
                const int64_t n = p + kPre - 1;
                q[kPre - 1] = n < pe ? (uint32_t)list[n] : 0xFFFFFFFFu;
                bq[kPre - 1] = n < pe ? (is_b ? a.b_t_blk[n] : (int32_t)n) : -1;
            }
            if (am && bm) return true;
        }
    };
    int32_t cur = -1, nxt = -1;
    bool have = next_step(cur);
    if (!have) {
        emit(-1);
        return;
    }
    while (have) {
        const bool more = next_step(nxt);
        emit(cur);
        cur = nxt;
        have = more;
    }
}

// one warp per tile: fill = 0 counts the tile's k-steps into step_cnt[t],
// fill = 1 writes their records at step_ptr[t]
__global__ void __launch_bounds__(256) k_panel_steps(PanelArgs a, int fill, int64_t *step_cnt) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= a.n_tiles) return;
    int64_t n = 0;
    int32_t *rec = fill ? a.steps + a.step_ptr[t] * (kRB + kCB) : nullptr;
    panel_merge(a, (int32_t)t, lane, [&](int32_t blk) {
        if (fill) {
            if (lane < kRB) rec[n * (kRB + kCB) + lane] = blk;
            else if (lane >= 8 && lane < 8 + kCB) rec[n * (kRB + kCB) + kRB + lane - 8] = blk;
        }
        ++n;
    });
    if (!fill && lane == 0) step_cnt[t] = n;
}

// The same k-step records by bitmaps, one CTA of 128 threads per tile: each of
// the 10 block-index lists (A's 5 rows, B's 5 columns) becomes a bitmap over k
// in shared memory; the k-steps are the set bits of (OR of A's) AND (OR of
// B's), in ascending k; the block of a list at k is its entry of rank
// popcount(list bits below k) (A: the CSR position itself; B: b_t_blk of the
// column-major position).  A block index always comes from a bit of its own
// list, so it lies inside that list.  Used when the 22 bitmaps and prefix
// arrays of nw = ceil(nbk / 32) words fit in shared memory.
constexpr int kBmLists = kRB + kCB;
__global__ void __launch_bounds__(128) k_panel_steps_bm(PanelArgs a, int fill, int64_t *step_cnt) {
    extern __shared__ uint32_t bsm_[];
    __shared__ int64_t lbeg[kBmLists], lend[kBmLists];
    const int64_t t = blockIdx.x;
    const int tid = threadIdx.x;
    const int nw = (a.nbk + 31) >> 5;
    uint32_t *bm = bsm_;                                                  // [10][nw]
    int32_t *pre = reinterpret_cast<int32_t *>(bsm_ + kBmLists * nw);     // [10][nw] exclusive
    uint32_t *U = bsm_ + 2 * kBmLists * nw;                               // [nw]
    int32_t *upre = reinterpret_cast<int32_t *>(bsm_ + (2 * kBmLists + 1) * nw);  // [nw] exclusive
    if (tid < kBmLists) {
        int64_t p = 0, pe = 0;
        const int32_t g = a.tile_g[t], h = a.tile_h[t];
        if (tid < kRB) {
            const int pr = g * kRB + tid;
            if (pr < a.nbr) {
                const int i = a.ord_r[pr];
                p = a.a_row_ptr[i];
                pe = a.a_row_ptr[i + 1];
            }
        } else {
            const int pc = h * kCB + tid - kRB;
            if (pc < a.nbc) {
                const int j = a.ord_c[pc];
                p = a.b_t_ptr[j];
                pe = a.b_t_ptr[j + 1];
            }
        }
        lbeg[tid] = p;
        lend[tid] = pe;
    }
    for (int w = tid; w < kBmLists * nw; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    for (int l = 0; l < kBmLists; ++l) {
        const int32_t *list = l < kRB ? a.a_col_idx : a.b_t_row;
        for (int64_t e = lbeg[l] + tid; e < lend[l]; e += blockDim.x) {
            const uint32_t k = (uint32_t)list[e];
            atomicOr(&bm[l * nw + (k >> 5)], 1u << (k & 31));
        }
    }
    __syncthreads();
    for (int w = tid; w < nw; w += blockDim.x) {
        uint32_t ao = 0u, bo = 0u;
#pragma unroll
        for (int l = 0; l < kRB; ++l) ao |= bm[l * nw + w];
#pragma unroll
        for (int l = kRB; l < kBmLists; ++l) bo |= bm[l * nw + w];
        U[w] = ao & bo;
    }
    __syncthreads();
    // exclusive word prefixes of the popcounts: one thread per array
    if (tid <= kBmLists) {
        const uint32_t *src = tid < kBmLists ? bm + tid * nw : U;
        int32_t *dst = tid < kBmLists ? pre + tid * nw : upre;
        int32_t run = 0;
        for (int w = 0; w < nw; ++w) {
            dst[w] = run;
            run += __popc(src[w]);
        }
    }
    __syncthreads();
    const int32_t total = upre[nw - 1] + __popc(U[nw - 1]);
    if (!fill) {
        if (tid == 0) step_cnt[t] = total > 0 ? total : 1;  // a tile with only old blocks: one empty step
        return;
    }
    int32_t *rec = a.steps + a.step_ptr[t] * kBmLists;
    if (total == 0) {
        if (tid < kBmLists) rec[tid] = -1;
        return;
    }
    for (int w = tid; w < nw; w += blockDim.x) {
        uint32_t u = U[w];
        int32_t sidx = upre[w];
        while (u) {
            const int bit = __ffs(u) - 1;
            u &= u - 1u;
            const uint32_t below = (1u << bit) - 1u;
#pragma unroll
            for (int l = 0; l < kBmLists; ++l) {
                const uint32_t bits = bm[l * nw + w];
                int32_t blk = -1;
                if ((bits >> bit) & 1u) {
                    const int64_t pos = lbeg[l] + pre[l * nw + w] + __popc(bits & below);
                    blk = l < kRB ? (int32_t)pos : a.b_t_blk[pos];
                }
                rec[(int64_t)sidx * kBmLists + l] = blk;
            }
            ++sidx;
        }
    }
}

// Drain warp of tensor-memory lanes 32 quarter .. +31 (tile rows) and columns
// 64 HALF .. +63 of both accumulator buffers: its threads keep the compensated
// pair of their 64 elements in registers (sum FP32, compensation BF16), add
// every buffer into it, and on a tile's last k-step write the tile's C blocks.
template <int HALF>
__device__ __forceinline__ void drain(const PanelArgs &a, SmemCtl &ctl, uint32_t tmem, int quarter, int lane,
                                      bool dead) {
    const int row = quarter * 32 + lane;
    const int si = row / kSlot, ri = row - si * kSlot;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + HALF * 64;
    float sh[64];
    __nv_bfloat162 sl[32];  // compensation of elements 2i, 2i + 1
    uint32_t buf = 0, bph = 0;
    bool ok = !dead;
    while (ok) {
        if (!__all_sync(0xffffffffu, mbar_wait(saddr(&ctl.accf[buf]), bph, &ctl.abort, a.wait_ns))) {
            if (lane == 0) fail(ctl, a.status);
            break;
        }
        tc_fence_after();
        const int32_t t = ctl.ameta_t[buf], flags = ctl.ameta_f[buf];
        if (flags & kDone) break;
        const bool first = flags & kFirst, last = flags & kLast;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            uint32_t v[32];
            tmem_ld32(lane_base + buf * 128 + ch * 32, v);
            tmem_wait_ld();
            if (ch == 1) {  // the buffer is free as soon as it is in registers
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(saddr(&ctl.acce[buf]));
            }
#pragma unroll
            for (int e = 0; e < 32; e += 2) {
                if (first) {  // the compensated add of v into (0, 0)
                    sh[ch * 32 + e] = __uint_as_float(v[e]);
                    sh[ch * 32 + e + 1] = __uint_as_float(v[e + 1]);
                    sl[(ch * 32 + e) / 2] = __floats2bfloat162_rn(0.f, 0.f);
                } else {
                    kahan_b2(sh[ch * 32 + e], sh[ch * 32 + e + 1], sl[(ch * 32 + e) / 2], __uint_as_float(v[e]),
                             __uint_as_float(v[e + 1]));
                }
            }
        }
        buf ^= 1u;
        if (buf == 0) bph ^= 1u;
        if (last && si < kRB && ri < a.s) {
            const double *old = static_cast<const double *>(a.old_data);
            const int32_t *cb = a.cblk + (int64_t)t * (kRB * kCB) + si * kCB;
            // the column slots this half of the tile touches
            constexpr int c0 = (HALF * 64) / kSlot, c1 = (HALF * 64 + 63) / kSlot;
#pragma unroll
            for (int c = c0; c <= c1 && c < kCB; ++c) {
                const int32_t q = cb[c];
                if (q < 0) continue;
                const int64_t o = a.c_blk_off[q] + (int64_t)ri * a.s;
                const int64_t oo = (old && a.old_off) ? a.old_off[q] : -1;
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    const int col = HALF * 64 + e;
                    if (col / kSlot != c) continue;
                    const int cj = col - c * kSlot;
                    if (cj >= a.s) continue;
                    const float2 lo = __bfloat1622float2(sl[e / 2]);
                    double val = a.alpha * ((double)sh[e] + (double)((e & 1) ? lo.y : lo.x));
                    if (oo >= 0) val = fma(a.beta, old[oo + (int64_t)ri * a.s + cj], val);
                    a.c_data[o + cj] = val;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_panel_tf32x3(PanelArgs a) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t *stages = (uint8_t *)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    SmemCtl &ctl = *reinterpret_cast<SmemCtl *>(stages + kStages * kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // rows 120..127 (row group 15) of both operands stay zero (never copied)
    for (int st = 0; st < kStages; ++st)
        for (int p = 0; p < 2; ++p)
            for (int w = threadIdx.x; w < kGroupStride / 16; w += kThreads)
                reinterpret_cast<uint4 *>(stages + st * kStageBytes + p * kOperand + 15 * kGroupStride)[w] =
                    make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(saddr(&ctl.full[st]), kCopyWarps);
            mbar_init(saddr(&ctl.empty[st]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(saddr(&ctl.accf[b]), 2);
            mbar_init(saddr(&ctl.acce[b]), kDrainWarps);
        }
        for (int r = 0; r < kRing; ++r) {
            mbar_init(saddr(&ctl.rec_full[r]), 1);
            mbar_init(saddr(&ctl.rec_empty[r]), kCopyWarps);
        }
        mbar_init(saddr(&ctl.fin), 1);
        ctl.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(saddr(&ctl.tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem;
    const bool dead = *a.status != 0;
    const int32_t no_abort = 0;  // waits that must not be cut short by the abort flag

    if (warp == 0) {
        // ------------------------------------------------------------ tiles
        // hands the tiles of the atomic ticket, with their k-step ranges, to
        // the copy warps through the ring
        uint32_t rs = 0, rph = 0;
        bool ok = !dead;
        for (;;) {
            int64_t tk = 0;
            if (lane == 0) tk = (int64_t)atomicAdd(a.work_counter, 1ull);
            tk = __shfl_sync(0xffffffffu, tk, 0);
            const bool done = !ok || tk >= a.n_tiles || *(volatile int32_t *)&ctl.abort;
            if (!__all_sync(0xffffffffu, mbar_wait(saddr(&ctl.rec_empty[rs]), rph ^ 1u, &ctl.abort, a.wait_ns))) {
                if (lane == 0) fail(ctl, a.status);
                break;
            }
            if (lane == 0) {
                TileRec &r = ctl.rec[rs];
                if (done) {
                    r.tile = -1;
                } else {
                    const int32_t t = a.tile_order[tk];
                    r.tile = t;
                    r.s0 = a.step_ptr[t];
                    r.s1 = a.step_ptr[t + 1];
                }
                mbar_arrive(saddr(&ctl.rec_full[rs]));
            }
            if (++rs == kRing) {
                rs = 0;
                rph ^= 1u;
            }
            if (done) break;
        }
    } else if (warp <= kCopyWarps) {
        // ------------------------------------------------------------ copy
        // warp 1 stages A's 5 blocks of every k-step, warp 2 B's: one bulk
        // copy of 4608 bytes per block (absent blocks from a zero block),
        // completion counted in bytes on the stage's "full" barrier.  The
        // block indices of 32 k-steps come in with one load per lane.
        const int cw = warp - 1;
        const bool is_a = cw == 0;
        const uint8_t *pk = is_a ? a.a_pack : a.b_pack;
        uint32_t st = 0, ph = 0, rs = 0, rph = 0;
        int64_t issued = 0;
        bool ok = !dead;
        while (ok) {
            if (!__all_sync(0xffffffffu, mbar_wait(saddr(&ctl.rec_full[rs]), rph, &ctl.abort, a.wait_ns))) {
                if (lane == 0) fail(ctl, a.status);
                ok = false;
                break;
            }
            const TileRec r = ctl.rec[rs];
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&ctl.rec_empty[rs]));
            if (++rs == kRing) {
                rs = 0;
                rph ^= 1u;
            }
            if (r.tile < 0) {  // the end marker for the MMA lane
                if (!__all_sync(0xffffffffu, mbar_wait(saddr(&ctl.empty[st]), ph ^ 1u, &ctl.abort, a.wait_ns))) {
                    if (lane == 0) fail(ctl, a.status);
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    if (is_a) ctl.smeta_f[st] = kDone;
                    mbar_arrive(saddr(&ctl.full[st]));
                }
                break;
            }
            for (int64_t base = r.s0; base < r.s1 && ok; base += 32) {
                // lane l: the 5 block indices of this warp's operand for k-step base + l
                int32_t f[kRB];
                const int64_t sl = base + lane;
#pragma unroll
                for (int q = 0; q < kRB; ++q) f[q] = sl < r.s1 ? a.steps[sl * (kRB + kCB) + (is_a ? 0 : kRB) + q] : -1;
                const int n = (int)(r.s1 - base < 32 ? r.s1 - base : 32);
                for (int j = 0; j < n; ++j) {
                    int32_t blk = -1;
#pragma unroll
                    for (int q = 0; q < kRB; ++q) {
                        const int32_t x = __shfl_sync(0xffffffffu, f[q], j);
                        if (lane == q) blk = x;
                    }
                    if (!__all_sync(0xffffffffu, mbar_wait(saddr(&ctl.empty[st]), ph ^ 1u, &ctl.abort, a.wait_ns))) {
                        if (lane == 0) fail(ctl, a.status);
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        if (is_a) {
                            const int64_t sidx = base + j;
                            ctl.smeta_t[st] = r.tile;
                            ctl.smeta_f[st] = (sidx == r.s0 ? kFirst : 0) | (sidx + 1 == r.s1 ? kLast : 0);
                        }
                        mbar_arrive_tx(saddr(&ctl.full[st]), kRB * kBlk);
                    }
                    __syncwarp();
                    if (lane < kRB) {
                        const void *src = blk >= 0 ? (const void *)(pk + (int64_t)blk * kBlk) : (const void *)a.zeros;
                        bulk_copy(saddr(stages + st * kStageBytes + (is_a ? 0 : kOperand) + lane * kBlk), src, kBlk,
                                  saddr(&ctl.full[st]));
                    }
                    ++issued;
                    if (++st == kStages) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
        if (!ok) {
            // leaving after a failed wait: let the copies of stages not yet
            // consumed land (bounded) before the CTA can exit
            for (int64_t q = issued - kStages; q < issued; ++q) {
                if (q < 0) continue;
                mbar_wait(saddr(&ctl.full[q % kStages]), (uint32_t)((q / kStages) & 1), &no_abort);
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        // a.pair (default kPair) consecutive k-steps of a tile accumulate in
        // one buffer before the drain adds it into the compensated pair
        uint32_t st = 0, ph = 0, buf = 0, bph = 0;
        int in_group = 0, gflags = 0;
        if (lane == 0) {
            bool ok = !dead;
            while (ok) {
                if (!mbar_wait(saddr(&ctl.full[st]), ph, &ctl.abort, a.wait_ns)) {
                    fail(ctl, a.status);
                    break;
                }
                tc_fence_after();
                const int32_t tile = ctl.smeta_t[st], flags = ctl.smeta_f[st];
                if (in_group == 0 && !mbar_wait(saddr(&ctl.acce[buf]), bph ^ 1u, &ctl.abort, a.wait_ns)) {
                    fail(ctl, a.status);
                    break;
                }
                tc_fence_after();
                if (flags & kDone) {
                    ctl.ameta_t[buf] = 0;
                    ctl.ameta_f[buf] = kDone;
                    mma_commit(saddr(&ctl.accf[buf]));
                    mbar_arrive(saddr(&ctl.accf[buf]));
                    break;
                }
                const uint32_t base = saddr(stages + st * kStageBytes);
                const uint32_t acc = tmem + buf * 128;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    const uint64_t ahi = sdesc(base + kk * 256, 128, kGroupStride);
                    const uint64_t alo = sdesc(base + kGroup + kk * 256, 128, kGroupStride);
                    const uint64_t bhi = sdesc(base + kOperand + kk * 256, 128, kGroupStride);
                    const uint64_t blo = sdesc(base + kOperand + kGroup + kk * 256, 128, kGroupStride);
                    mma_tf32(acc, alo, bhi, in_group > 0 || kk > 0);
                    mma_tf32(acc, ahi, blo, 1);
                    mma_tf32(acc, ahi, bhi, 1);
                }
                mma_commit(saddr(&ctl.empty[st]));
                gflags |= flags & kFirst;
                if ((flags & kLast) || in_group + 1 == a.pair) {
                    ctl.ameta_t[buf] = tile;
                    ctl.ameta_f[buf] = gflags | (flags & kLast);
                    mma_commit(saddr(&ctl.accf[buf]));
                    mbar_arrive(saddr(&ctl.accf[buf]));
                    in_group = 0;
                    gflags = 0;
                    buf ^= 1u;
                    if (buf == 0) bph ^= 1u;
                } else {
                    ++in_group;
                }
                if (++st == kStages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            // every MMA issued has completed before the tensor memory is freed
            mma_commit(saddr(&ctl.fin));
            if (!mbar_wait(saddr(&ctl.fin), 0, &no_abort)) fail(ctl, a.status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ drain
        const int quarter = warp & 3;
        if ((warp - kMmaWarp - 1) / 4 == 0) drain<0>(a, ctl, tmem, quarter, lane, dead);
        else drain<1>(a, ctl, tmem, quarter, lane, dead);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

}  // namespace

int64_t panel_pack_bytes(int64_t nblk) { return nblk * kBlk; }
int panel_slot() { return kSlot; }
int panel_pair() { return kPair; }
int panel_tile_rows() { return kRB; }
int panel_tile_cols() { return kCB; }

cudaError_t launch_panel_pack(const bsm_mat *M, int trans, void *out, cudaStream_t s) {
    if (M->nnzb == 0) return cudaSuccess;
    const int64_t warps = M->nnzb;
    const int64_t blocks = (warps * 32 + 255) / 256;
    k_panel_pack<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double *>(M->data), M->blk_off, M->nnzb,
                                                  M->h_row_bs[0],
                                                  trans, static_cast<uint32_t *>(out));
    count_launch(1);
    return cudaGetLastError();
}

size_t panel_tile_smem(int32_t ngc) { return (size_t)((ngc + 31) / 32) * 2 * sizeof(uint32_t); }

cudaError_t launch_panel_tiles_count(int32_t nbr, const int32_t *ord_r, const int32_t *pos_c,
                                     const int64_t *c_row_ptr, const int32_t *c_col, int32_t ngc, int64_t *tile_cnt,
                                     cudaStream_t s) {
    const int32_t ngr = (nbr + kRB - 1) / kRB;
    if (ngr == 0) return cudaSuccess;
    const size_t smem = panel_tile_smem(ngc) / 2;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_panel_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_panel_tile_count<<<ngr, 128, smem, s>>>(nbr, ord_r, pos_c, c_row_ptr, c_col, ngc, tile_cnt);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_panel_tiles_fill(int32_t nbr, const int32_t *ord_r, const int32_t *pos_c,
                                    const int64_t *c_row_ptr, const int32_t *c_col, int32_t ngc,
                                    const int64_t *tile_ptr, int32_t *tile_g, int32_t *tile_h, int32_t *cblk,
                                    cudaStream_t s) {
    const int32_t ngr = (nbr + kRB - 1) / kRB;
    if (ngr == 0) return cudaSuccess;
    const size_t smem = panel_tile_smem(ngc);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_panel_tile_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_panel_tile_fill<<<ngr, 128, smem, s>>>(nbr, ord_r, pos_c, c_row_ptr, c_col, ngc, tile_ptr, tile_g, tile_h,
                                             cblk);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_panel_tile_keys(int64_t ntiles, const int32_t *tile_g, const int32_t *tile_h, int sg, int sh,
                                   int32_t ngc, uint32_t *keys, int32_t *iota, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    k_panel_tile_keys<<<(unsigned)((ntiles + 255) / 256), 256, 0, s>>>(ntiles, tile_g, tile_h, sg, sh, ngc, keys,
                                                                       iota);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_panel_steps(const PanelArgs &a, int fill, int64_t *step_cnt, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    const int nw = (a.nbk + 31) >> 5;
    const size_t smem = (size_t)(2 * kBmLists + 2) * nw * sizeof(uint32_t);
    if (nw > 0 && smem <= 48 * 1024 && a.n_tiles < (int64_t(1) << 31)) {
        k_panel_steps_bm<<<(unsigned)a.n_tiles, 128, smem, s>>>(a, fill, step_cnt);
    } else {  // the bitmaps do not fit: the warp-per-tile merge
        k_panel_steps<<<(unsigned)((a.n_tiles * 32 + 255) / 256), 256, 0, s>>>(a, fill, step_cnt);
    }
    count_launch(1);
    return cudaGetLastError();
}

size_t panel_smem_bytes() { return (size_t)kStages * kStageBytes + sizeof(SmemCtl) + 1024; }

cudaError_t launch_panel_numeric(const PanelArgs &a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = panel_smem_bytes();
    e = cudaFuncSetAttribute(k_panel_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(nsm, a.n_tiles);
    k_panel_tf32x3<<<(unsigned)grid, kThreads, smem, s>>>(a);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace bsm
