// Machinery shared by the persistent tensor-core kernels (op_tc.cu: FP16 hi+lo form with
// CUDA-core phases; op_tc_phase.cu: BF16 form with tensor-core phases): constants, operand
// packing, the CTA's barriers, work-item queue and bounded waits.  Everything has internal
// linkage; each translation unit instantiates what it uses.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "aexp_internal.cuh"
#include "tc_ptx.cuh"

namespace aexp {
namespace {

constexpr int kTcGen = 512;              // generator threads (16 warps)
constexpr int kProdWarp = kTcGen / 32;   // the first non-generator warp: MMA issue, owns TMEM
constexpr int kRows = 128;               // M
constexpr int kCols = 64;                // voxels (forward) or samples (adjoint) per stage
constexpr int kA_BYTES = kRows * kCols * 2 * 2;  // 128 rows x 128 bf16 = 32 KB
constexpr float kTwoPi = 6.283185307179586f;
constexpr int kSpin = 1 << 22;
constexpr int kNBMax = 6;  // deepest operand ring (slots with their own full / free barriers)
constexpr float kLoScale = 2048.f;           // 2^11: scale of the low parts
constexpr float kLoInv = 1.f / 2048.f;
constexpr int kPromote = 8;                  // FP16 hi+lo: stages per accumulator chunk

// TMEM columns of one accumulator (N = 2C columns rounded up to a power of two >= 32).
constexpr uint32_t tmem_acc_cols(int N) { return N <= 32 ? 32u : 64u; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// (a, b) -> FP16 pairs hi = (fp16 a, fp16 b) and lo = fp16(2^11 (a - hi.a)), fp16(2^11 (b - hi.b)).
// The differences are exact in FP32 (hi is the rounding of the same value).
__device__ __forceinline__ void split_f16(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn((a - hf.x) * kLoScale, (b - hf.y) * kLoScale);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// Power-of-two scale 2^e (or 2^-e when `inverse`) that maps a largest component with bit
// pattern `bits` into [2^top, 2^(top+1)) (top = 13 by default); zero (or subnormal) maxima give
// the largest scale, a non-finite one a small scale (the non-finite values then propagate).
__device__ __forceinline__ float hl_scale(unsigned bits, bool inverse, int top = 13) {
    const int ex = (int)((bits >> 23) & 0xffu);
    int se = 127 + top - max(ex, 1);  // top - (ex - 127)
    se = max(-126, min(126, se));
    return __int_as_float((127 + (inverse ? -se : se)) << 23);
}
// Operand packing of the contraction's B operand: BF16; FP16 hi | lo' (lo' = 2^11 (v - hi));
// FP16 hi2 | lo' with hi2 = 2^11 hi (the FP16 hi+lo form whose phases come from the tensor
// cores: one accumulator takes A_hi B_hi2 + A_hi B_lo' + A_lo B_hi2 = 2^11 A B, see op_tc_phase.cu).
enum PackMode { kPackBF16 = 0, kPackHL = 1, kPackHL2 = 2 };
constexpr int kHl2Top = 3;  // kPackHL2: the operand is scaled below 2^4, so that 2^11 hi < 2^15

// Bounded wait that also gives up as soon as another thread of the CTA has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, unsigned parity, volatile int *abort_flag,
                                              int *status) {
    for (int i = 0; i < kSpin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    set_status(status, AEXP_ERR_DEVICE_TIMEOUT);
    return false;
}

__device__ __forceinline__ uint32_t align1024(uint32_t a) { return (a + 1023u) & ~1023u; }

__device__ __forceinline__ int find_problem(const int *item_off, int nprob, int item) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Shared state of a persistent tensor-core CTA.
struct TcShared {
    uint64_t bfull[kNBMax], bfree[kNBMax], afull[2], afree[2], accfree[2];
    uint64_t phfull[4], phfree[4], apfull;  // tensor-core phases: tile ready / read, item operand loaded
    uint64_t pfull[kNBMax], pfree[kNBMax];  // tensor-core phases: ring of per-stage phase operands
    uint64_t drain;              // teardown: every MMA of the issuing thread has completed
    uint64_t accdone;            // tensor-core phases: an item's last contraction has completed
    uint32_t tmem_base;
    int abort_flag;
    int item[2], stop[2];
};

// afull_count: generator threads that fill one A stage (all of them, or one group of two
// that take alternate stages); phfree_count: generator warps that read one phase tile;
// pfree_count: arrivals that release one slot of the per-stage operand ring (the phase-GEMM
// issuer, or every generator thread when the generators read the slot themselves).
__device__ __forceinline__ void tc_setup(TcShared &sh, int tid, int warp, uint32_t ncols, unsigned acc_count,
                                         unsigned afull_count = kTcGen, unsigned phfree_count = kTcGen / 32,
                                         unsigned pfree_count = 1) {
    if (tid == 0) {
        for (int s = 0; s < kNBMax; ++s) {
            mbar_init(&sh.bfull[s], 1);
            mbar_init(&sh.bfree[s], 1);
            mbar_init(&sh.pfull[s], 1);
            mbar_init(&sh.pfree[s], pfree_count);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sh.afull[s], afull_count);
            mbar_init(&sh.afree[s], 1);
            mbar_init(&sh.accfree[s], acc_count);
        }
        for (int s = 0; s < 4; ++s) {
            mbar_init(&sh.phfull[s], 1);
            mbar_init(&sh.phfree[s], phfree_count);  // one arrival per generator warp
        }
        mbar_init(&sh.apfull, 1);
        mbar_init(&sh.accdone, 1);
        mbar_init(&sh.drain, 2);  // tensor-core-phase kernels: both MMA-issuing threads commit
        sh.abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kProdWarp) {
        tc::tmem_alloc(&sh.tmem_base, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Next work item, the same for every thread of the CTA (two slots: a thread still reading
// one slot never races the write of the other); false when the queue is empty or aborted.
__device__ __forceinline__ bool tc_next_item(TcShared &sh, int tid, int iter, int *counter, int total, int &item) {
    const int slot = iter & 1;
    if (tid == 0) {
        int it = atomicAdd(counter, 1);
        sh.item[slot] = it;
        sh.stop[slot] = (it >= total) || sh.abort_flag;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    item = sh.item[slot];
    return !sh.stop[slot];
}

// Ring loader, one item: stage g's slot (g mod depth) is refilled once the stage that used it
// last has released it; `load(it, slot)` issues the copies for the item's stage `it`.
template <class Load>
__device__ __forceinline__ void ring_load_item(uint64_t *free_bar, int depth, int gs, int n, volatile int *abort_flag,
                                               int *status, Load load) {
    for (int it = 0; it < n; ++it) {
        const int g = gs + it, s = g % depth;
        if (g >= depth && !wait_or_abort(&free_bar[s], ((g - depth) / depth) & 1, abort_flag, status)) return;
        load(it, s);
    }
}

__device__ __forceinline__ void tc_teardown(TcShared &sh, int warp, uint32_t ncols, int last_issued, int *status) {
    if (warp == kProdWarp && (threadIdx.x & 31) == 0 && last_issued >= 0)
        mbar_wait_bounded(&sh.afree[last_issued & 1], (last_issued >> 1) & 1, status);  // drain
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kProdWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(sh.tmem_base, ncols);
    }
}

// ---------------------------------------------------------------------------
// Packing of the B operands into the swizzled K-major smem image, one launch for all
// problems (grid.y = problem; blocks beyond a problem's extent return at once)
// ---------------------------------------------------------------------------

// Four (first, second) pairs -> one 16-byte chunk of the B image(s) at `dst` in mode MODE
// (FP16 forms: hi or hi2 at dst, lo' one image of `img_bytes` further).
template <int MODE>
__device__ __forceinline__ void store_b_chunk(unsigned char *dst, unsigned img_bytes, const float (&a)[4],
                                              const float (&b)[4]) {
    uint32_t w[4], wl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if constexpr (MODE == kPackBF16) {
            w[u] = pack_bf16(a[u], b[u]);
        } else {
            split_f16(a[u], b[u], w[u], wl[u]);
            if constexpr (MODE == kPackHL2) {  // hi2 = 2^11 hi: exact (a power of two, below 2^15)
                __half2 h = *reinterpret_cast<const __half2 *>(&w[u]);
                h = __hmul2(h, __float2half2_rn(kLoScale));
                w[u] = *reinterpret_cast<const uint32_t *>(&h);
            }
        }
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    if constexpr (MODE != kPackBF16)
        *reinterpret_cast<uint4 *>(dst + img_bytes) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

// Shared staging of one tile (64 voxels) or stage (64 samples) of C coil values, coil-major
// with the 64 positions stored as (position & 3) * 16 + position / 4: the packing loop reads
// positions 4 jj + u with jj across the lanes, which are then consecutive words (no bank
// conflicts); rows of 65 entries keep the coil-fastest fill conflict-free too.
constexpr int kStageRow = kCols + 1;
__device__ __forceinline__ int stage_slot(int c, int pos) { return c * kStageRow + (pos & 3) * 16 + (pos >> 2); }

// Blocks of a packing launch: one per tile (forward) or stage (adjoint) of the largest problem.
// The amax launches of the FP16 hi+lo form cover ntiles * 64 * CB / 2 (forward) and
// ntp * CB / 2 (adjoint) threads instead: fwd_pack_blocks / adj_pack_blocks count those, i.e.
// CB / 8 blocks per tile or stage.
inline int pack_grid(int amax_blocks, int CB) { return amax_blocks * 8 / CB; }

// The swizzled operand rows of one tile or stage from its staged values `sv` (stage_slot
// layout): rows n < C carry (Re, -Im), rows C + c carry (Im, Re) at K positions (2j, 2j+1),
// written as 16-byte chunks (a row's chunks across the lanes) at `dst` (the tile's or stage's
// operand image).  The block's threads share the work; the caller synchronises around it.
template <int CB, int MODE>
__device__ __forceinline__ void pack_staged_rows(const float2 *sv, unsigned char *dst) {
    constexpr int N = 2 * CB;
    for (int k = threadIdx.x; k < N * 16; k += blockDim.x) {  // (n, chunk of 4 positions)
        const int jj = k % 16, n = k / 16;
        const int c = n < CB ? n : n - CB;
        float a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float2 v = sv[c * kStageRow + u * 16 + jj];  // position 4 jj + u
            a[u] = n < CB ? v.x : v.y;
            b[u] = n < CB ? -v.y : v.x;
        }
        store_b_chunk<MODE>(dst + (jj >> 3) * (N * 128) + tc::swz128(n, jj & 7), N * 256, a, b);
    }
}

// Forward: coil-weighted image b_c(v) = S_c(v) x(v) of every 8x8 tile, rows n < C carry
// (Re b, -Im b), rows C + c carry (Im b, Re b) at K positions (2v, 2v+1).  The image is
// `x` when given (single problem) or the descriptor's vec[src].  FP16 hi+lo: b is scaled by
// the power of two fixed by the problem's amax[0].  One block per tile (grid-stride): the
// tile's coil maps are read coalesced (coils fastest) into shared memory, then every thread
// writes 16-byte chunks of the swizzled operand rows (a row's chunks across the lanes, so
// that the global writes are coalesced).
template <int CB, int MODE>
__global__ void __launch_bounds__(256) pack_b_fwd_kernel(const ProbDesc *__restrict__ pd, const float2 *__restrict__ x,
                                                         int src) {
    constexpr int N = 2 * CB;
    constexpr int NPK = MODE != kPackBF16 ? 2 : 1;
    __shared__ float2 sb[CB * kStageRow];
    const ProbDesc &P = pd[blockIdx.y];
    const float2 *img = x ? x : P.vec[src];
    const float sc = MODE != kPackBF16 ? hl_scale(P.hdr->amax[0], false, MODE == kPackHL2 ? kHl2Top : 13) : 1.f;
    for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
        const int tx = (tile % P.ntx) * kTileSide, ty = (tile / P.ntx) * kTileSide;
        for (int k = threadIdx.x; k < kTileVox * CB; k += blockDim.x) {
            const int v = k / CB, c = k % CB;
            const int ix = tx + v % kTileSide, iy = ty + v / kTileSide;
            float2 b = make_float2(0.f, 0.f);
            if (ix < P.nx && iy < P.ny) {
                const float2 s = P.Sp[(size_t)tile * kTileVox * CB + k];
                const float2 xv = img[(size_t)iy * P.nx + ix];
                b = make_float2((s.x * xv.x - s.y * xv.y) * sc, (s.x * xv.y + s.y * xv.x) * sc);
            }
            sb[stage_slot(c, v)] = b;
        }
        __syncthreads();
        pack_staged_rows<CB, MODE>(sb, P.bpk + (size_t)tile * (NPK * N * 256));
        __syncthreads();
    }
}

// Adjoint: k-space yt[t][c] (or the descriptor's vec[src], or rt when src < 0) per stage of
// 64 samples; rows n < C carry (Re y, -Im y), rows C + c carry (Im y, Re y) at K positions
// (2s, 2s+1).  FP16 hi+lo: y is scaled by the power of two fixed by amax[1].  One block per
// stage (grid-stride): the stage's 64 x C values are contiguous and read coalesced into shared
// memory, then written as 16-byte chunks of the swizzled operand rows.
template <int CB, int MODE>
__global__ void __launch_bounds__(256) pack_y_adj_kernel(const ProbDesc *__restrict__ pd, const float2 *__restrict__ yt,
                                                         int src) {
    constexpr int N = 2 * CB;
    constexpr int NPK = MODE != kPackBF16 ? 2 : 1;
    __shared__ float2 sy[CB * kStageRow];
    const ProbDesc &P = pd[blockIdx.y];
    const int nstages = P.ntp / kCols;
    const float2 *y = yt ? yt : (src >= 0 ? P.vec[src] : P.rt);
    const float sc = MODE != kPackBF16 ? hl_scale(P.hdr->amax[1], false, MODE == kPackHL2 ? kHl2Top : 13) : 1.f;
    for (int st = blockIdx.x; st < nstages; st += gridDim.x) {
        for (int k = threadIdx.x; k < kCols * CB; k += blockDim.x) {
            float2 v = y[(size_t)st * kCols * CB + k];
            v.x *= sc;
            v.y *= sc;
            sy[stage_slot(k % CB, k / CB)] = v;
        }
        __syncthreads();
        pack_staged_rows<CB, MODE>(sy, P.ypk + (size_t)st * (NPK * N * 256));
        __syncthreads();
    }
}

// BF16 form, the forward reduction, the residual and the adjoint's packing in one pass:
// r[t][c] = sum over splits (in split order) of the planar forward partials, minus the
// measured ymeas[t][c] when given (`ymeas`, or the descriptor's vec[ymeas_role] when
// ymeas_role >= 0), zero for padded samples and coils; r is packed as the adjoint's operand
// (the same values and rounding as the reduction kernel followed by pack_y_adj_kernel, without
// the FP32 residual round trip).  One block per stage (grid-stride), grid.y = problem; the
// partials are loaded kRedBatch splits at a time and added in split order.
constexpr int kReducePackThreads = 512;
constexpr int kRedBatch = 8;
template <int CB>
__global__ void __launch_bounds__(kReducePackThreads) reduce_pack_y_kernel(const ProbDesc *__restrict__ pd,
                                                            const float2 *__restrict__ ymeas, int ymeas_role) {
    constexpr int N = 2 * CB;
    __shared__ float2 sy[CB * kStageRow];
    const ProbDesc &P = pd[blockIdx.y];
    const int nstages = P.ntp / kCols;
    const float2 *ym = ymeas ? ymeas : (ymeas_role >= 0 ? P.vec[ymeas_role] : nullptr);
    for (int st = blockIdx.x; st < nstages; st += gridDim.x) {
        for (int k = threadIdx.x; k < kCols * CB; k += blockDim.x) {
            const int t = st * kCols + k / CB, c = k % CB;
            float2 s = make_float2(0.f, 0.f);
            if (t < P.nt && c < P.nc) {
                const float *col = P.fpart + (size_t)t * N + c;
                const size_t sstride = (size_t)P.ntp * N;
                for (int s0 = 0; s0 < P.fwd_splits; s0 += kRedBatch) {
                    float re[kRedBatch], im[kRedBatch];
#pragma unroll
                    for (int u = 0; u < kRedBatch; ++u) {
                        const bool in = s0 + u < P.fwd_splits;
                        re[u] = in ? col[(size_t)(s0 + u) * sstride] : 0.f;
                        im[u] = in ? col[(size_t)(s0 + u) * sstride + CB] : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < kRedBatch; ++u) {
                        if (s0 + u < P.fwd_splits) {
                            s.x += re[u];
                            s.y += im[u];
                        }
                    }
                }
                if (ym) {
                    const float2 m = ym[(size_t)st * kCols * CB + k];
                    s.x -= m.x;
                    s.y -= m.y;
                }
            }
            sy[stage_slot(c, k / CB)] = s;
        }
        __syncthreads();
        pack_staged_rows<CB, kPackBF16>(sy, P.ypk + (size_t)st * (N * 256));
        __syncthreads();
    }
}

// ---- FP16 hi+lo: largest component of the operand to be packed (atomic max on the bit
// pattern of a non-negative float, which orders like the value) ----
__global__ void amax_reset_kernel(const ProbDesc *__restrict__ pd, int nprob, int which) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nprob) pd[q].hdr->amax[which] = 0u;
}

__device__ __forceinline__ void amax_commit(float m, unsigned *slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(slot, __float_as_uint(m));
}

// max |Re|, |Im| of b_c(v) = S_c(v) x(v); thread = (voxel in tile order, pair of coils)
template <int CB>
__global__ void amax_b_kernel(const ProbDesc *__restrict__ pd, const float2 *__restrict__ x, int src) {
    const ProbDesc &P = pd[blockIdx.y];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < (size_t)P.ntiles * kTileVox * (CB / 2)) {
        const float2 *img = x ? x : P.vec[src];
        const int p = (int)(i / (CB / 2));
        const int tile = p / kTileVox, v = p % kTileVox;
        const int ix = (tile % P.ntx) * kTileSide + v % kTileSide, iy = (tile / P.ntx) * kTileSide + v / kTileSide;
        if (ix < P.nx && iy < P.ny) {
            const float4 s = reinterpret_cast<const float4 *>(P.Sp)[i];
            const float2 xv = img[(size_t)iy * P.nx + ix];
            m = fmaxf(fmaxf(fabsf(s.x * xv.x - s.y * xv.y), fabsf(s.x * xv.y + s.y * xv.x)),
                      fmaxf(fabsf(s.z * xv.x - s.w * xv.y), fabsf(s.z * xv.y + s.w * xv.x)));
        }
    }
    amax_commit(m, &P.hdr->amax[0]);
}

// max |Re|, |Im| of the sample-major k-space yt[t][CB] (or vec[src], or rt when src < 0)
template <int CB>
__global__ void amax_y_kernel(const ProbDesc *__restrict__ pd, const float2 *__restrict__ yt, int src) {
    const ProbDesc &P = pd[blockIdx.y];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < (size_t)P.ntp * (CB / 2)) {
        const float2 *y = yt ? yt : (src >= 0 ? P.vec[src] : P.rt);
        const float4 v = reinterpret_cast<const float4 *>(y)[i];
        m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
    }
    amax_commit(m, &P.hdr->amax[1]);
}

}  // namespace
}  // namespace aexp
