// A_exp and A_exp^H with the phase computed on the tensor cores as well: the BF16 form and the
// FP16 hi+lo form (FP32-class accuracy), one kernel template for both.
//
// Inside a work item the phase offsets of a stage are a small matrix product,
//   off(t, v) = sum_l khi(t, l) dh(v, l)        (t: 128 samples or 64 per stage, v: voxels,
//                                                l: field terms incl. B0, padded to 16 or 32)
// with khi = k / 2pi in turns and dh the basis offsets from the tile's reference voxel
// (the same quantities the CUDA-core generators sum with FMAs).  It runs as tcgen05.mma
// kind::f16 into a TMEM tile, each factor split x = x_hi + x_lo (x_hi rounded, x_lo = x - x_hi
// rounded again) and the products hi*hi + hi*lo + lo*hi accumulated in FP32.
//   BF16 form: BF16 parts, relative error ~2^-17 of sum_l |khi dh|, about 1e-4 rad for the
//     ~12 rad an 8x8 tile spans at the Nyquist edge of k-space, twenty times below the BF16
//     rounding of E (2^-9).
//   FP16 hi+lo form: FP16 parts (11 significant bits each, ~2^-22 together) after an exact
//     power-of-two rescaling per term (k_l 2^s_l, dh_l 2^-s_l, with s_l putting max_t |2 pi k_l|
//     into [1, 2): FP16's range then holds every product of the tile), ~1e-6 rad, the accuracy
//     of the FP32 phase sum it replaces.
// Each K step takes 16 terms, so up to 16 terms cost 3 MMAs per stage and up to 32 terms 6.
//
// Generators then read their row's phase offsets of the stage with one tcgen05.ld (in
// radians: the k operand carries the factor 2 pi), add 2 pi f0(tile, t) with the tile's
// tabulated reference phase f0 in [-1/2, 1/2) turn, take one MUFU sincos and write their row
// of the encoding tile E into TMEM with tcgen05.st (no shared-memory stores, no proxy fence);
// the contraction with the coil-weighted image (or the k-space data) is a tcgen05 kind::f16
// GEMM with A read from TMEM and B, the packed operand, from shared memory:
//   BF16 form: E in BF16, 8 MMAs per stage.
//   FP16 hi+lo form: E = E_hi + E_lo in FP16 (E_lo = E - E_hi unscaled: |E| <= 1, so the
//     absolute error of E_lo, subnormal or not, stays below 2^-25); B packed as hi2 = 2^11 B_hi
//     and lo' = 2^11 (B - B_hi) after scaling B by a power of two below 2^4 (hi2 < 2^15 fits
//     FP16); one accumulator takes A_hi B_hi2 + A_hi B_lo' + A_lo B_hi2 = 2^11 A B up to the
//     dropped lo x lo product (~2^-22): 24 MMAs per stage.  The tensor core's FP32 accumulation
//     loses about 2^-24 of the running sum per MMA, so the accumulator is promoted every
//     kChunk stages: two TMEM accumulator sets alternate by chunk of stages, the epilogue
//     warps add a finished set into FP32 partial sums (forward: the item's rows of the
//     partial-sum buffer; adjoint: the coil-combined value in registers) and release it.
// The two GEMMs are issued by two threads of their own: the contraction thread issues a
// stage's MMAs once the generators have stored A(g); the phase thread fills the TMEM phase
// tiles, each as soon as the generators have read it.  The generators form two groups of 8
// warps that take alternate stages, so that one group computes while the other waits for its
// next stage.  (A 128-row MMA with N <= 64 occupies the tensor pipe for ~40 cycles, so one
// thread issuing both GEMMs in turn would bound the stage rate.)
// The epilogue waits for the item's last contraction on a barrier of its own (accdone, one
// completion per item with stages, waited for by the same warps every item).  Waiting on the
// A-release barrier of the last stage instead was wrong for the generator group that did not
// produce that stage: it had not followed that barrier's phases, and when the contraction two
// stages back was still running the parity test passed one phase early, so that warp read
// partial accumulators (seen as run-to-run differences in one lane quadrant of one item).
//
// Phase operands, prepared once per problem (BF16 or FP16 images in the 128B-swizzled K-major
// layout, 64 K slots = 128 bytes per row: slots 0-31 hold the hi parts, 32-63 the lo parts):
//   kph   per block of 128 samples, rows = samples:  forward A_phase; adjoint B_phase
//         (the 64 rows of one stage are one half of a block)
//   dhph  per pair of tiles, rows = 128 voxels:      adjoint A_phase; forward B_phase
//         (the 64 rows of one tile are one half of a pair)
#include <algorithm>

#include "tc_common.cuh"

namespace aexp {
namespace {

constexpr unsigned kHalfImg = 64 * 128;         // the hi | lo image of 64 rows, 8 KB
constexpr unsigned kApBytes = kRows * 128;      // item operand: hi | lo image of 128 rows, 16 KB
constexpr uint32_t kLoBytes = 64;               // the lo parts start 32 slots (64 B) into a row
constexpr uint32_t kTmemCols = 512;

// The two forms (F = 0: BF16, F = 1: FP16 hi+lo) and their TMEM plans:
//   BF16:  accumulator 0..63 | 4 phase tiles 64..319 | 2 A buffers (E) 320..447
//   FP16:  2 accumulator sets 0..127 | 2 phase tiles 128..255 | 2 A buffers (E_hi | E_lo) 256..511
template <int F>
struct Form;
template <>
struct Form<0> {
    static constexpr int PH_BUFS = 4;
    static constexpr uint32_t PH_BASE = 64, A_BASE = 320, A_COLS = 64;
    static constexpr uint32_t AB = 1;  // BF16 operands
    static constexpr int NIMG = 1;     // B images per stage
};
template <>
struct Form<1> {
    static constexpr int PH_BUFS = 2;
    static constexpr uint32_t PH_BASE = 128, A_BASE = 256, A_COLS = 128;
    static constexpr uint32_t AB = 0;  // FP16 operands
    static constexpr int NIMG = 2;     // hi2 | lo'
};
static_assert(Form<0>::A_BASE + 2 * Form<0>::A_COLS <= kTmemCols && Form<1>::A_BASE + 2 * Form<1>::A_COLS <= kTmemCols,
              "TMEM plan");
// each generator group must own its phase tiles: with an odd count a tile would alternate
// between the groups, a group would skip every other phase of its barrier and its parity test
// could pass a phase early
static_assert(Form<0>::PH_BUFS % 2 == 0 && Form<1>::PH_BUFS % 2 == 0, "phase tiles per group");

template <int F>
__device__ __forceinline__ uint32_t phase_col(int g) {
    return Form<F>::PH_BASE + 64u * (uint32_t)(g % Form<F>::PH_BUFS);
}
template <int F>
__device__ __forceinline__ uint32_t a_col(int sa) {
    return Form<F>::A_BASE + Form<F>::A_COLS * (uint32_t)sa;
}

// ---- operand preparation ----

// Eight values -> 16-byte chunks of hi parts and of lo parts (lo = x - hi, rounded): BF16 (F = 0)
// or FP16 (F = 1).
template <int F>
__device__ __forceinline__ void split_8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if constexpr (F == 0) {
            const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
            const float2 hf = __bfloat1622float2(hb);
            const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * u] - hf.x, v[2 * u + 1] - hf.y);
            h[u] = *reinterpret_cast<const uint32_t *>(&hb);
            l[u] = *reinterpret_cast<const uint32_t *>(&lb);
        } else {
            const __half2 hh = __floats2half2_rn(v[2 * u], v[2 * u + 1]);
            const float2 hf = __half22float2(hh);
            const __half2 lh = __floats2half2_rn(v[2 * u] - hf.x, v[2 * u + 1] - hf.y);
            h[u] = *reinterpret_cast<const uint32_t *>(&hh);
            l[u] = *reinterpret_cast<const uint32_t *>(&lh);
        }
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// FP16 form: kscale[l] = 2^s_l with max_t |2 pi khi_t[t][l]| 2^s_l in [1, 2) (1 for a zero term).
// One block of 1024 threads, terms one after the other.
__global__ void __launch_bounds__(1024) term_scale_kernel(const float *__restrict__ khi_t, int ntp, int LP,
                                                          float *__restrict__ kscale) {
    __shared__ float s_m[32];
    for (int l = 0; l < LP; ++l) {
        float m = 0.f;
        for (int t = threadIdx.x; t < ntp; t += blockDim.x) m = fmaxf(m, fabsf(kTwoPi * khi_t[(size_t)t * LP + l]));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x < 32) {
            m = s_m[threadIdx.x];
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (threadIdx.x == 0) {
                const int ex = m > 0.f && isfinite(m) ? ilogbf(m) : 0;  // m in [2^ex, 2^(ex+1))
                kscale[l] = ldexpf(1.f, max(-100, min(100, -ex)));
            }
        }
        __syncthreads();
    }
}

// kph[block][row = sample % 128][hi slots 0-31 | lo slots 0-31] = 2 pi khi_t[sample][slot]
// (times kscale[slot] in the FP16 form; 0 beyond LP): the phase GEMM yields radians
template <int F>
__global__ void prep_kph_kernel(const float *__restrict__ khi_t, int ntp, int LP, const float *__restrict__ kscale,
                                unsigned char *__restrict__ kph) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (sample, chunk of 8 slots)
    if (i >= (size_t)ntp * 4) return;
    const int t = (int)(i / 4), c = (int)(i % 4);
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int l = 8 * c + u;
        v[u] = l < LP ? kTwoPi * khi_t[(size_t)t * LP + l] * (F == 1 ? kscale[l] : 1.f) : 0.f;
    }
    uint4 hi, lo;
    split_8<F>(v, hi, lo);
    unsigned char *blk = kph + (size_t)(t / kRows) * kPhaseBlockBytes;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(t % kRows, c)) = hi;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(t % kRows, c + 4)) = lo;
}

// dhph[pair][row = 64 (tile & 1) + voxel][hi slots | lo slots] = dh[tile][voxel][slot] (divided
// by kscale[slot] in the FP16 form; 0 beyond LP and for the missing second tile of an odd count)
template <int F>
__global__ void prep_dhph_kernel(const float *__restrict__ dh, int ntiles, int LP, const float *__restrict__ kscale,
                                 unsigned char *__restrict__ dhph) {
    const int npairs = (ntiles + 1) / 2;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (pair, row, chunk)
    if (i >= (size_t)npairs * kRows * 4) return;
    const int c = (int)(i % 4);
    const int r = (int)((i / 4) % kRows);
    const int pair = (int)(i / (4 * kRows));
    const int tile = 2 * pair + r / kTileVox, v = r % kTileVox;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int l = 8 * c + u;
        x[u] = (tile < ntiles && l < LP) ? dh[((size_t)tile * kTileVox + v) * LP + l] / (F == 1 ? kscale[l] : 1.f)
                                         : 0.f;
    }
    uint4 hi, lo;
    split_8<F>(x, hi, lo);
    unsigned char *blk = dhph + (size_t)pair * kPhaseBlockBytes;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(r, c)) = hi;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(r, c + 4)) = lo;
}

// ---- kernels ----

// Warp roles: 16 generator warps; warp 16 issues the contraction MMAs and owns TMEM (the whole
// warp runs its loop, lane 0 issues); warp 17 loads the contraction operands (+ reference
// phases); warp 18 issues the phase MMAs; warp 19 loads the phase operands (one lane each).
constexpr int kMmaWarp = kTcGen / 32;
constexpr int kLoadBWarp = kMmaWarp + 1;
constexpr int kPhaseWarp = kMmaWarp + 2;
constexpr int kLoadPWarp = kMmaWarp + 3;
constexpr int kTcpThreads = kTcGen + 128;
// Ring depths (template parameters NBB, NP of the kernels): per-stage contraction operands +
// reference phases (NBB) and per-stage phase operands (NP, hi | lo image of 8 KB).  BF16,
// tiling 0: 4 and 3; tiling 1 (aexp_recon_opts::tile_variant): 6 and 4.  FP16 hi+lo: 4 and 3.
// A generator group waits only on the stages of its parity, so each B slot must belong to one
// group (an even NBB).  (The MMA thread and the loaders wait on every stage; NP may be anything.)

// Shared-memory plan of both kernels (byte offsets from the 1024-aligned base; the generated
// encoding tiles live in TMEM):
//   AP item phase operand (hi | lo) | PH ring | B ring | FP16 hi+lo forward: the item's promoted
//   partial sums (128 rows x N floats, float4 c4 of row r at c4 * 128 + r: conflict-free)
template <int F, int N, int NBB, int NP>
struct TcpPlan {
    static_assert(NBB % 2 == 0, "each generator group must own its B slots");
    static_assert(NBB <= kNBMax && NP <= kNBMax, "ring deeper than the CTA's barriers");
    static constexpr unsigned B_BYTES = Form<F>::NIMG * N * 256;
    static constexpr unsigned F_BYTES = kRows * 4;  // forward: 128 f0; adjoint: 2 x 64 f0
    static constexpr unsigned BS = (B_BYTES + F_BYTES + 1023u) & ~1023u;  // B ring stride
    static constexpr unsigned PS = kHalfImg;                              // PH ring stride
    static constexpr unsigned OFF_AP = 0;
    static constexpr unsigned OFF_PH = OFF_AP + kApBytes;
    static constexpr unsigned OFF_B = OFF_PH + NP * PS;
    static constexpr unsigned OFF_ACC = OFF_B + NBB * BS;
    static constexpr unsigned ACC_BYTES = F == 1 ? kRows * N * 4 : 0;
    static constexpr unsigned BYTES = OFF_ACC + ACC_BYTES;
    static_assert(BYTES + 1024 <= 227 * 1024, "shared memory");
};

// Contraction of one stage into the accumulator at `acc`, A (the encoding tile) read from TMEM
// at `ta` (8 columns per K step of 16), B from shared memory at `db`: BF16, 8 MMAs; FP16
// hi+lo, 24 MMAs (A_hi B_hi2, A_hi B_lo', A_lo B_hi2; E_lo sits 64 columns after E_hi, lo' one
// image after hi2).
template <int F, int N>
__device__ __forceinline__ void contraction_mma(uint32_t acc, uint32_t ta, uint64_t db, bool first) {
    constexpr uint32_t ID = tc::idesc_f16(kRows, N, Form<F>::AB);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
        tc::mma_f16_ts(acc, ta + 8u * (uint32_t)kk, tc::sdesc_advance(db, kofb), ID, !(first && kk == 0));
    }
    if constexpr (F == 1) {
        const uint64_t dl = tc::sdesc_advance(db, N * 256);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
            tc::mma_f16_ts(acc, ta + 8u * (uint32_t)kk, tc::sdesc_advance(dl, kofb), ID, 1u);
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
            tc::mma_f16_ts(acc, ta + 64u + 8u * (uint32_t)kk, tc::sdesc_advance(db, kofb), ID, 1u);
        }
    }
}

// Phase GEMM of one stage into the tile at `d`: KS steps of 16 values, products
// hi*lo + lo*hi + hi*hi (the lo parts sit kLoBytes further along each row).  The small cross
// products go first, so that the FP32 accumulator rounds at the magnitude of the full phase
// only in the last KS MMAs.
template <int F, int KS>
__device__ __forceinline__ void phase_mma_ks(uint32_t d, uint64_t a, uint64_t b) {
    constexpr uint32_t ID = tc::idesc_f16(kRows, 64, Form<F>::AB);
#pragma unroll
    for (int k = 0; k < KS; ++k)
        tc::mma_f16(d, tc::sdesc_advance(a, 32 * k), tc::sdesc_advance(b, kLoBytes + 32 * k), ID, k > 0);
#pragma unroll
    for (int k = 0; k < KS; ++k)
        tc::mma_f16(d, tc::sdesc_advance(a, kLoBytes + 32 * k), tc::sdesc_advance(b, 32 * k), ID, 1u);
#pragma unroll
    for (int k = 0; k < KS; ++k) tc::mma_f16(d, tc::sdesc_advance(a, 32 * k), tc::sdesc_advance(b, 32 * k), ID, 1u);
}

template <int F>
__device__ __forceinline__ void phase_mma(int ks, uint32_t d, uint64_t a, uint64_t b) {
    if (ks <= 1) phase_mma_ks<F, 1>(d, a, b);
    else phase_mma_ks<F, 2>(d, a, b);
}

// FP16 hi+lo accumulator sets: chunk c (counted over the CTA's items) of kChunk stages
// accumulates in set c & 1 (TMEM columns 64 (c & 1)); the epilogue warps arrive on
// accfree[c & 1] once they have promoted it.
__device__ __forceinline__ uint32_t set_col(int c) { return 64u * (uint32_t)(c & 1); }
constexpr int kChunk = 4;  // 96 MMAs per chunk

// Contraction warp, one item: the whole warp runs the loop and waits, lane 0 (elected) issues the
// MMAs and commits.  FP16 hi+lo: `cbase` counts the CTA's chunks before this item; a set is
// reused for chunk c once the promotion of chunk c - 2 has released it.
template <int F, int N, int NBB, int NP>
__device__ __forceinline__ void tcp_contraction_item(TcShared &sh, uint32_t tmem, unsigned char *base, int gs, int n,
                                                     int cbase, int *status) {
    using PL = TcpPlan<F, N, NBB, NP>;
    const bool leader = tc::elect_lane0();
    for (int it = 0; it < n; ++it) {
        const int g = gs + it, sa = g & 1, sb = g % NBB;
        uint32_t acc = tmem;
        bool first = it == 0;
        bool ok = true;
        if constexpr (F == 1) {
            const int c = cbase + it / kChunk;
            first = it % kChunk == 0;
            if (first && c >= 2) ok = wait_or_abort(&sh.accfree[c & 1], ((c - 2) >> 1) & 1, &sh.abort_flag, status);
            acc = tmem + set_col(c);
        }
        if (ok) ok = wait_or_abort(&sh.afull[sa], (g >> 1) & 1, &sh.abort_flag, status);
        if (ok) ok = wait_or_abort(&sh.bfull[sb], (g / NBB) & 1, &sh.abort_flag, status);
        if (!__all_sync(0xffffffffu, ok)) return;
        tc::fence_after_sync();
        if (leader) {
            contraction_mma<F, N>(acc, tmem + a_col<F>(sa), tc::sdesc_k128(smem_u32(base + PL::OFF_B + sb * PL::BS)),
                                  first);
            tc::mma_commit(&sh.afree[sa]);
            tc::mma_commit(&sh.bfree[sb]);
        }
        __syncwarp();
    }
    if (n > 0 && leader) tc::mma_commit(&sh.accdone);  // the item's accumulators are final
}

// Phase role, one item: the phases of stage g go into tile g % PH_BUFS once the generators
// have read that tile for stage g - PH_BUFS and the stage's operand has landed.  WARP = false:
// lane 0 of the phase warp alone; WARP = true: the whole warp waits and lane 0 (elected) issues,
// which issues faster but lets the phases run up to PH_BUFS stages ahead of the contractions
// (measured: the BF16 adjoint 0.645 -> 0.600 ms, the BF16 forward and both FP16 hi+lo kernels
// slower).  The MMAs and their order are the same either way.
template <int F, int N, int NBB, int NP, bool WARP>
__device__ __forceinline__ void tcp_phase_item(TcShared &sh, uint32_t tmem, unsigned char *base, int gs, int n,
                                               int iter, int ks, int *status) {
    using PL = TcpPlan<F, N, NBB, NP>;
    constexpr int PB = Form<F>::PH_BUFS;
    const uint64_t ad = tc::sdesc_k128(smem_u32(base + PL::OFF_AP));
    const bool leader = WARP ? tc::elect_lane0() : true;
    bool ok = wait_or_abort(&sh.apfull, iter & 1, &sh.abort_flag, status);
    if (WARP) ok = __all_sync(0xffffffffu, ok);
    if (!ok) return;
    for (int it = 0; it < n; ++it) {
        const int g = gs + it, b = g % PB, sp = g % NP;
        ok = g < PB || wait_or_abort(&sh.phfree[b], ((g - PB) / PB) & 1, &sh.abort_flag, status);
        if (ok) ok = wait_or_abort(&sh.pfull[sp], (g / NP) & 1, &sh.abort_flag, status);
        if (WARP) ok = __all_sync(0xffffffffu, ok);
        if (!ok) return;
        tc::fence_after_sync();
        if (leader) {
            phase_mma<F>(ks, tmem + phase_col<F>(g), ad, tc::sdesc_k128(smem_u32(base + PL::OFF_PH + sp * PL::PS)));
            tc::mma_commit(&sh.phfull[b]);
            tc::mma_commit(&sh.pfree[sp]);
        }
        if (WARP) __syncwarp();
    }
}

// Teardown: both MMA threads commit to the drain barrier (count 2); the contraction thread
// waits (bounded) until every MMA has completed; then TMEM is released.
__device__ __forceinline__ void tcp_teardown(TcShared &sh, int tid, int warp, int *status) {
    if (tid == kPhaseWarp * 32) tc::mma_commit(&sh.drain);
    if (tid == kMmaWarp * 32) {
        tc::mma_commit(&sh.drain);
        mbar_wait_bounded(&sh.drain, 0, status);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(sh.tmem_base, kTmemCols);
    }
}

// One generator thread's part of a stage (generators work in two groups of 8 warps that take
// alternate stages; warp w of a group reads TMEM lanes 32 (w & 3) .. + 31 and owns the 32
// columns 32 (w >> 2) .. + 31): its row's 32 phase offsets (TMEM; the tile is released to the
// phase thread right after the read) plus the reference phases -> E (or conj E), one (re, im)
// pair per TMEM column of its row of the A tile at `ta`: BF16, or FP16 hi at `ta` and lo 64
// columns further.  Forward: one reference phase per row (fsrc[0]); adjoint: one per column
// (fsrc[0..31]).
template <int F, bool CONJ>
__device__ __forceinline__ bool generate_row(TcShared &sh, int g, uint32_t taddr, const float *fsrc, uint32_t ta,
                                             int *status) {
    float ph[32];
    tc::tmem_ld<32>(taddr, ph);
    tc::tmem_ld_wait();
    tc::tmem_regs_ready<32>(ph);
    tc::fence_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&sh.phfree[g % Form<F>::PH_BUFS]);
    uint32_t w[32], wl[F == 1 ? 32 : 1];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float f[4];
        if constexpr (CONJ) {
            const float4 fw = reinterpret_cast<const float4 *>(fsrc)[c];
            f[0] = fw.x;
            f[1] = fw.y;
            f[2] = fw.z;
            f[3] = fw.w;
        } else {
            f[0] = f[1] = f[2] = f[3] = fsrc[0];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // angle = 2 pi f0 + offset (radians); f0 lies in [-1/2, 1/2) turn and the offset spans
            // a few turns inside a tile, so the hardware sincos needs no further reduction (its
            // error grows like |angle| x 2^-24, ~1e-6 here)
            const float x = fmaf(f[u], kTwoPi, ph[4 * c + u]);
            float sn, cs;
            __sincosf(x, &sn, &cs);
            const float im = CONJ ? sn : -sn;  // E = cos - i sin, conj(E) = cos + i sin
            if constexpr (F == 0) {
                w[4 * c + u] = pack_bf16(cs, im);
            } else {
                const __half2 h = __floats2half2_rn(cs, im);
                const float2 hf = __half22float2(h);
                const __half2 l = __floats2half2_rn(cs - hf.x, im - hf.y);
                w[4 * c + u] = *reinterpret_cast<const uint32_t *>(&h);
                wl[4 * c + u] = *reinterpret_cast<const uint32_t *>(&l);
            }
        }
    }
    // The A buffer is claimed only now: the contraction of stage g - 2, which frees it,
    // overlaps the sincos work above.  This group waited on the barrier for stage g - 2's
    // previous use (stage g - 4), so the parity is unambiguous.
    bool ok = g < 2 || wait_or_abort(&sh.afree[g & 1], ((g - 2) >> 1) & 1, &sh.abort_flag, status);
    if (!__all_sync(0xffffffffu, ok)) return false;
    tc::fence_after_sync();
    tc::tmem_st32(ta, w);
    if constexpr (F == 1) tc::tmem_st32(ta + 64u, wl);
    tc::tmem_st_wait();
    return true;
}

// Generator waits of stage g before its TMEM read (warp-uniform result): reference phases
// landed, phase tile ready.  The A buffer is waited for inside generate_row.
template <int F, int NBB>
__device__ __forceinline__ bool gen_waits(TcShared &sh, int g, int *status) {
    constexpr int PB = Form<F>::PH_BUFS;
    bool ok = wait_or_abort(&sh.bfull[g % NBB], (g / NBB) & 1, &sh.abort_flag, status);
    if (ok) ok = wait_or_abort(&sh.phfull[g % PB], (g / PB) & 1, &sh.abort_flag, status);
    return __all_sync(0xffffffffu, ok);
}

// FP16 hi+lo promotion, forward: (accumulator set at `ta`) x inv for this thread's row x N/2
// columns, stored to (first chunk) or added into the item's partial sums in shared memory
// (`dst`, this thread's float4 chunks `kRows` apart).
template <int N>
__device__ __forceinline__ void fwd_promote1(uint32_t ta, float inv, float4 *dst, bool add) {
    constexpr int CH = N / 2 < 16 ? N / 2 : 16;
#pragma unroll
    for (int c0 = 0; c0 < N / 2; c0 += CH) {
        float v[CH];
        tc::tmem_ld<CH>(ta + (uint32_t)c0, v);
        tc::tmem_ld_wait();
        tc::tmem_regs_ready<CH>(v);
#pragma unroll
        for (int c = 0; c < CH / 4; ++c) {
            float4 *q = dst + (size_t)(c0 / 4 + c) * kRows;
            const float4 p = add ? *q : make_float4(0.f, 0.f, 0.f, 0.f);
            *q = make_float4(fmaf(v[4 * c], inv, p.x), fmaf(v[4 * c + 1], inv, p.y), fmaf(v[4 * c + 2], inv, p.z),
                             fmaf(v[4 * c + 3], inv, p.w));
        }
    }
}

// Adjoint accumulator read-out: xr + i xi += sum_c conj(S_c) u_c over the coils of one
// accumulator (set) at `ta` for this thread's voxel row, its coil maps as float4 pairs `stride`
// apart at `s4` (FP16 hi+lo: the scale is applied by the caller once the chunks are summed).
template <int CB>
__device__ __forceinline__ void adj_promote1(uint32_t ta, const float4 *s4, int stride, float &xr, float &xi) {
#pragma unroll 1
    for (int c0 = 0; c0 < CB; c0 += 8) {
        float ur[8], ui[8];
        tc::tmem_ld<8>(ta + (uint32_t)c0, ur);
        tc::tmem_ld<8>(ta + (uint32_t)(CB + c0), ui);
        tc::tmem_ld_wait();
        tc::tmem_regs_ready<8>(ur);
        tc::tmem_regs_ready<8>(ui);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            const float4 sv = s4[(size_t)(c0 / 2 + q4) * stride];
            xr = fmaf(sv.x, ur[2 * q4], xr);
            xr = fmaf(sv.y, ui[2 * q4], xr);
            xi = fmaf(sv.x, ui[2 * q4], xi);
            xi = fmaf(-sv.y, ur[2 * q4], xi);
            xr = fmaf(sv.z, ur[2 * q4 + 1], xr);
            xr = fmaf(sv.w, ui[2 * q4 + 1], xr);
            xi = fmaf(sv.z, ui[2 * q4 + 1], xi);
            xi = fmaf(-sv.w, ur[2 * q4 + 1], xi);
        }
    }
}

// The epilogue warps' release of a promoted accumulator set (one arrival per warp).
__device__ __forceinline__ void release_set(TcShared &sh, int c) {
    tc::fence_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&sh.accfree[c & 1]);
}

// Forward: item = (problem, block of 128 samples, run of voxel tiles).
template <int F, int CB, int NBB, int NP>
__global__ void __launch_bounds__(kTcpThreads, 1)
    fwd_tcp_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    using PL = TcpPlan<F, N, NBB, NP>;

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const int total = item_off[nprob];

    // two generator groups; FP16 hi+lo: the 8 epilogue warps release an accumulator set
    tc_setup(sh, tid, warp, kTmemCols, 8, kTcGen / 2, kTcGen / 64);
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;
    int nacc = 0;   // items with stages so far: the accdone phase this CTA waits for next
    int cbase = 0;  // FP16 hi+lo: accumulator chunks of the CTA's earlier items

    int item;
    for (int iter = 0; tc_next_item(sh, tid, iter, counter, total, item); ++iter) {
        const int q = find_problem(item_off, nprob, item);
        const ProbDesc &P = pd[q];
        int *status = &P.hdr->status;
        const int li = item - item_off[q];
        const int split = li % P.fwd_splits;
        const int tbase = (li / P.fwd_splits) * kRows;
        const int tile0 = split * P.fwd_tps;
        const int ntl = max(0, min(P.ntiles, tile0 + P.fwd_tps) - tile0);
        const int ntp = P.ntp;
        const int nch = (ntl + kChunk - 1) / kChunk;

        if (warp >= kMmaWarp) {
            const bool lead = (tid & 31) == 0;
            if (warp == kMmaWarp) {  // the whole warp (see tcp_contraction_item)
                tcp_contraction_item<F, N, NBB, NP>(sh, tmem, gbase, gs, ntl, cbase, status);
            } else if (warp == kPhaseWarp && lead) {
                tcp_phase_item<F, N, NBB, NP, false>(sh, tmem, gbase, gs, ntl, iter, (P.LP + 15) >> 4, status);
            } else if (warp == kLoadBWarp && lead) {
                ring_load_item(sh.bfree, NBB, gs, ntl, &sh.abort_flag, status, [&](int it, int sb) {
                    const int tile = tile0 + it;  // packed S x of the tile and its reference phases
                    unsigned char *dst = gbase + PL::OFF_B + sb * PL::BS;
                    mbar_arrive_expect_tx(&sh.bfull[sb], PL::B_BYTES + PL::F_BYTES);
                    bulk_g2s(dst, P.bpk + (size_t)tile * PL::B_BYTES, PL::B_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + PL::B_BYTES, P.f0 + (size_t)tile * ntp + tbase, PL::F_BYTES, &sh.bfull[sb]);
                });
            } else if (warp == kLoadPWarp && lead) {
                mbar_arrive_expect_tx(&sh.apfull, kApBytes);
                bulk_g2s(gbase + PL::OFF_AP, P.kph + (size_t)(tbase / kRows) * kPhaseBlockBytes, kApBytes, &sh.apfull);
                ring_load_item(sh.pfree, NP, gs, ntl, &sh.abort_flag, status, [&](int it, int sp) {
                    const int tile = tile0 + it;  // the tile's basis offsets, hi | lo
                    const unsigned char *dp =
                        P.dhph + (size_t)(tile >> 1) * kPhaseBlockBytes + (size_t)(tile & 1) * kHalfImg;
                    mbar_arrive_expect_tx(&sh.pfull[sp], kHalfImg);
                    bulk_g2s(gbase + PL::OFF_PH + sp * PL::PS, dp, kHalfImg, &sh.pfull[sp]);
                });
            }
        } else {
            // generator group warp >> 3 takes the stages of its parity; warp w reads TMEM lanes
            // 32 (w & 3) .. + 31 (its rows) and owns voxel columns 32 ((w >> 2) & 1) .. + 31
            const int row = 32 * (warp & 3) + (tid & 31);
            const int ch = (warp >> 2) & 1;
            const int grp = warp >> 3;
            const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
            // epilogue (warps 0-7 = group 0): 32 samples x N/2 columns of the planar partial sums
            float4 *dst = reinterpret_cast<float4 *>(P.fpart + ((size_t)split * ntp + tbase + row) * N + ch * (N / 2));
            // FP16 hi+lo: this thread's promoted partial sums in shared memory during the item
            float4 *sacc = reinterpret_cast<float4 *>(gbase + PL::OFF_ACC) + (size_t)ch * (N / 8) * kRows + row;
            float inv = 1.f;
            if constexpr (F == 1) inv = hl_scale(P.hdr->amax[0], true, kHl2Top) * kLoInv;
            int next_promo = 0;  // FP16 hi+lo: next chunk of this item to promote
            for (int it = 0; it < ntl; ++it) {
                const int g = gs + it, sa = g & 1, sb = g % NBB;
                if ((g & 1) != grp) continue;
                if (!gen_waits<F, NBB>(sh, g, status)) break;  // warp-uniform exit
                tc::fence_after_sync();
                if (!generate_row<F, false>(sh, g, tmem + lanes + phase_col<F>(g) + (uint32_t)(32 * ch),
                                       reinterpret_cast<const float *>(gbase + PL::OFF_B + sb * PL::BS + PL::B_BYTES) + row,
                                       tmem + lanes + a_col<F>(sa) + (uint32_t)(32 * ch), status))
                    break;  // warp-uniform exit
                tc::fence_before_sync();
                tc::mbar_arrive(&sh.afull[sa]);
                if constexpr (F == 1) {
                    // stages <= it - 2 are complete (this group waited for stage g - 2's MMAs):
                    // promote the finished chunks and release their sets
                    if (grp == 0) {
                        while (next_promo < (it - 1) / kChunk) {
                            tc::fence_after_sync();
                            fwd_promote1<N>(tmem + lanes + set_col(cbase + next_promo) + (uint32_t)(ch * (N / 2)), inv,
                                            sacc, next_promo > 0);
                            release_set(sh, cbase + next_promo);
                            ++next_promo;
                        }
                    }
                }
            }
            // epilogue (warps 0-7): the item's last MMAs done -> TMEM -> partials (planar re | im)
            if (warp < 8) {
                bool ok = !sh.abort_flag;
                if (ntl > 0 && ok) ok = wait_or_abort(&sh.accdone, nacc & 1, &sh.abort_flag, status);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
                tc::fence_after_sync();
                if constexpr (F == 0) {
                    float v[N / 2];
                    if (ntl > 0 && ok) {
                        tc::tmem_ld<N / 2>(tmem + lanes + (uint32_t)(ch * (N / 2)), v);
                        tc::tmem_ld_wait();
                        tc::tmem_regs_ready<N / 2>(v);
                    } else {
#pragma unroll
                        for (int c = 0; c < N / 2; ++c) v[c] = 0.f;
                    }
#pragma unroll
                    for (int c = 0; c < N / 8; ++c) dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                } else {
                    if (ntl > 0 && ok) {
                        for (int m = next_promo; m < nch; ++m) {
                            fwd_promote1<N>(tmem + lanes + set_col(cbase + m) + (uint32_t)(ch * (N / 2)), inv, sacc, m > 0);
                            release_set(sh, cbase + m);
                        }
#pragma unroll
                        for (int c = 0; c < N / 8; ++c) dst[c] = sacc[(size_t)c * kRows];
                    } else {
#pragma unroll
                        for (int c = 0; c < N / 8; ++c) dst[c] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        }
        gs += ntl;
        nacc += ntl > 0;
        cbase += nch;
    }
    tcp_teardown(sh, tid, warp, &pd[0].hdr->status);
}

// Adjoint: item = (problem, pair of voxel tiles, run of 64-sample stages).
template <int F, int CB, int NBB, int NP>
__global__ void __launch_bounds__(kTcpThreads, 1)
    adj_tcp_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    constexpr int TS = kCols;  // samples per stage
    using PL = TcpPlan<F, N, NBB, NP>;
    constexpr unsigned FT = TS * 4;  // reference phases of one tile for one stage

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const int total = item_off[nprob];

    // two generator groups; FP16 hi+lo: the 4 epilogue warps release an accumulator set
    tc_setup(sh, tid, warp, kTmemCols, 4, kTcGen / 2, kTcGen / 64);
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;
    int nacc = 0;   // items with stages so far: the accdone phase this CTA waits for next
    int cbase = 0;  // FP16 hi+lo: accumulator chunks of the CTA's earlier items

    int item;
    for (int iter = 0; tc_next_item(sh, tid, iter, counter, total, item); ++iter) {
        const int q = find_problem(item_off, nprob, item);
        const ProbDesc &P = pd[q];
        int *status = &P.hdr->status;
        const int li = item - item_off[q];
        const int vb = li / P.adj_splits, split = li % P.adj_splits;
        const int ntiles = P.ntiles, ntp = P.ntp;
        const int tileA = 2 * vb;
        const int tileB = min(tileA + 1, ntiles - 1);  // odd tile count: duplicate row, discarded
        const int t0 = split * P.adj_tps;
        const int nst = max(0, (min(ntp, t0 + P.adj_tps) - t0) / TS);
        const int nch = (nst + kChunk - 1) / kChunk;

        if (warp >= kMmaWarp) {
            const bool lead = (tid & 31) == 0;
            if (warp == kMmaWarp) {  // the whole warp (see tcp_contraction_item)
                tcp_contraction_item<F, N, NBB, NP>(sh, tmem, gbase, gs, nst, cbase, status);
            } else if (warp == kPhaseWarp && (F == 0 || lead)) {  // BF16: the converged warp
                tcp_phase_item<F, N, NBB, NP, F == 0>(sh, tmem, gbase, gs, nst, iter, (P.LP + 15) >> 4, status);
            } else if (warp == kLoadBWarp && lead) {
                ring_load_item(sh.bfree, NBB, gs, nst, &sh.abort_flag, status, [&](int it, int sb) {
                    const size_t ts = (size_t)t0 + (size_t)it * TS;  // packed y and both tiles' f0
                    unsigned char *dst = gbase + PL::OFF_B + sb * PL::BS;
                    mbar_arrive_expect_tx(&sh.bfull[sb], PL::B_BYTES + 2 * FT);
                    bulk_g2s(dst, P.ypk + (ts / TS) * PL::B_BYTES, PL::B_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + PL::B_BYTES, P.f0 + (size_t)tileA * ntp + ts, FT, &sh.bfull[sb]);
                    bulk_g2s(dst + PL::B_BYTES + FT, P.f0 + (size_t)tileB * ntp + ts, FT, &sh.bfull[sb]);
                });
            } else if (warp == kLoadPWarp && lead) {
                mbar_arrive_expect_tx(&sh.apfull, kApBytes);
                bulk_g2s(gbase + PL::OFF_AP, P.dhph + (size_t)vb * kPhaseBlockBytes, kApBytes, &sh.apfull);
                ring_load_item(sh.pfree, NP, gs, nst, &sh.abort_flag, status, [&](int it, int sp) {
                    const size_t ts = (size_t)t0 + (size_t)it * TS;  // the stage's k rows, hi | lo
                    const unsigned char *kp =
                        P.kph + (ts / kRows) * kPhaseBlockBytes + ((ts / TS) & 1) * (size_t)kHalfImg;
                    mbar_arrive_expect_tx(&sh.pfull[sp], kHalfImg);
                    bulk_g2s(gbase + PL::OFF_PH + sp * PL::PS, kp, kHalfImg, &sh.pfull[sp]);
                });
            }
        } else {
            // generator group warp >> 3 takes the stages of its parity; warp w reads TMEM lanes
            // 32 (w & 3) .. + 31 (voxel rows; rows 0-63 in tile A, 64-127 in tile B) and owns sample
            // columns 32 ((w >> 2) & 1) .. + 31
            const int row = 32 * (warp & 3) + (tid & 31);
            const int th = (warp & 3) >> 1;
            const int ch = (warp >> 2) & 1;
            const int grp = warp >> 3;
            const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
            // epilogue (warps 0-3, one voxel row per thread): conj(S) . u over coils
            const int p = vb * kRows + row;
            const bool inside = p < ntiles * kTileVox;
            const float4 *s4 = reinterpret_cast<const float4 *>(P.Sp + (size_t)(inside ? p : 0) * CB);
            // FP16 hi+lo: the promoting warps 0-3 keep their row's coil maps in shared memory for
            // the item (read once, not once per promotion)
            const float4 *sp4 = s4;
            int sstride = 1;
            if constexpr (F == 1) {
                if (warp < 4) {
                    float4 *ss = reinterpret_cast<float4 *>(gbase + PL::OFF_ACC) + row;
#pragma unroll
                    for (int q = 0; q < CB / 2; ++q) ss[(size_t)q * kRows] = s4[q];
                    sp4 = ss;
                    sstride = kRows;
                }
            }
            float xr = 0.f, xi = 0.f;  // coil-combined partial sum (FP16 hi+lo: promoted chunks)
            int next_promo = 0;
            for (int it = 0; it < nst; ++it) {
                const int g = gs + it, sa = g & 1, sb = g % NBB;
                if ((g & 1) != grp) continue;
                if (!gen_waits<F, NBB>(sh, g, status)) break;  // warp-uniform exit
                tc::fence_after_sync();
                if (!generate_row<F, true>(sh, g, tmem + lanes + phase_col<F>(g) + (uint32_t)(32 * ch),
                                      reinterpret_cast<const float *>(gbase + PL::OFF_B + sb * PL::BS + PL::B_BYTES + th * FT) +
                                          32 * ch,
                                      tmem + lanes + a_col<F>(sa) + (uint32_t)(32 * ch), status))
                    break;  // warp-uniform exit
                tc::fence_before_sync();
                tc::mbar_arrive(&sh.afull[sa]);
                if constexpr (F == 1) {
                    if (warp < 4) {  // stages <= it - 2 complete: promote finished chunks
                        while (next_promo < (it - 1) / kChunk) {
                            tc::fence_after_sync();
                            adj_promote1<CB>(tmem + lanes + set_col(cbase + next_promo), sp4, sstride, xr, xi);
                            release_set(sh, cbase + next_promo);
                            ++next_promo;
                        }
                    }
                }
            }
            if (warp < 4) {
                bool ok = !sh.abort_flag;
                if (nst > 0 && ok) ok = wait_or_abort(&sh.accdone, nacc & 1, &sh.abort_flag, status);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
                tc::fence_after_sync();
                const bool have = nst > 0 && ok;
                if constexpr (F == 0) {
                    if (have) adj_promote1<CB>(tmem + lanes, s4, 1, xr, xi);
                } else {
                    if (have) {
                        for (int m = next_promo; m < nch; ++m) {
                            adj_promote1<CB>(tmem + lanes + set_col(cbase + m), sp4, sstride, xr, xi);
                            release_set(sh, cbase + m);
                        }
                        const float inv = hl_scale(P.hdr->amax[1], true, kHl2Top) * kLoInv;
                        xr *= inv;
                        xi *= inv;
                    } else {
                        xr = xi = 0.f;
                    }
                }
                if (inside) P.apart[(size_t)split * (size_t)(ntiles * kTileVox) + p] = make_float2(xr, xi);
            }
        }
        gs += nst;
        nacc += nst > 0;
        cbase += nch;
    }
    tcp_teardown(sh, tid, warp, &pd[0].hdr->status);
}

// ---- launches ----
template <int F, int CB, int NBB, int NP>
size_t tcp_smem() {
    return 1024 + TcpPlan<F, 2 * CB, NBB, NP>::BYTES;
}

template <int F, int CB, int NBB, int NP>
cudaError_t launch_fwd_tcp(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x, int src,
                           const int *item_off, int total_items, int *counter, cudaStream_t st) {
    if constexpr (F == 1) {
        amax_reset_kernel<<<cdiv(nprob, 256), 256, 0, st>>>(pd, nprob, 0);
        amax_b_kernel<CB><<<dim3(max_pack_blocks, nprob), 256, 0, st>>>(pd, x, src);
    }
    pack_b_fwd_kernel<CB, F == 1 ? kPackHL2 : kPackBF16>
        <<<dim3(pack_grid(max_pack_blocks, CB), nprob), 256, 0, st>>>(pd, x, src);
    auto kern = fwd_tcp_kernel<F, CB, NBB, NP>;
    const size_t smem = tcp_smem<F, CB, NBB, NP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kTcpThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

// pack = 0: the adjoint operand is already packed (reduce_pack_y_kernel)
template <int F, int CB, int NBB, int NP>
cudaError_t launch_adj_tcp(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt, int src, int pack,
                           const int *item_off, int total_items, int *counter, cudaStream_t st) {
    if constexpr (F == 1) {
        amax_reset_kernel<<<cdiv(nprob, 256), 256, 0, st>>>(pd, nprob, 1);
        amax_y_kernel<CB><<<dim3(max_pack_blocks, nprob), 256, 0, st>>>(pd, yt, src);
    }
    if (pack || F == 1)
        pack_y_adj_kernel<CB, F == 1 ? kPackHL2 : kPackBF16>
            <<<dim3(pack_grid(max_pack_blocks, CB), nprob), 256, 0, st>>>(pd, yt, src);
    auto kern = adj_tcp_kernel<F, CB, NBB, NP>;
    const size_t smem = tcp_smem<F, CB, NBB, NP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kTcpThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

template <int CB>
cudaError_t launch_fwd_tcp_variant(int form, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                                   const float2 *x, int src, const int *item_off, int total_items, int *counter,
                                   cudaStream_t st) {
    if (form == 1)
        return launch_fwd_tcp<1, CB, 4, 3>(pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
    return variant == 1
               ? launch_fwd_tcp<0, CB, 6, 4>(pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st)
               : launch_fwd_tcp<0, CB, 4, 3>(pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
}

template <int CB>
cudaError_t launch_adj_tcp_variant(int form, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                                   const float2 *yt, int src, int pack, const int *item_off, int total_items,
                                   int *counter, cudaStream_t st) {
    if (form == 1)
        return launch_adj_tcp<1, CB, 4, 3>(pd, nprob, max_pack_blocks, yt, src, 1, item_off, total_items, counter, st);
    return variant == 1
               ? launch_adj_tcp<0, CB, 6, 4>(pd, nprob, max_pack_blocks, yt, src, pack, item_off, total_items, counter, st)
               : launch_adj_tcp<0, CB, 4, 3>(pd, nprob, max_pack_blocks, yt, src, pack, item_off, total_items, counter, st);
}

// BF16 form: forward reduction + residual + packing (one launch), then the adjoint kernel.
template <int CB>
cudaError_t launch_residual_adj_bf16(int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                                     const float2 *ymeas, int ymeas_role, const int *item_off, int total_items,
                                     int *counter, cudaStream_t st) {
    reduce_pack_y_kernel<CB>
        <<<dim3(pack_grid(max_pack_blocks, CB), nprob), kReducePackThreads, 0, st>>>(pd, ymeas, ymeas_role);
    return launch_adj_tcp_variant<CB>(0, variant, pd, nprob, max_pack_blocks, nullptr, -1, 0, item_off, total_items,
                                      counter, st);
}

}  // namespace

cudaError_t op_prepare_phase_operands(const OpLayout &L, char *ws, cudaStream_t st) {
    const int T = 256;
    const size_t nk = (size_t)L.ntp * 4;
    const size_t nd = (size_t)cdiv(L.ntiles, 2) * kRows * 4;
    const float *khi_t = (const float *)(ws + L.off_khi_t);
    const float *dh = (const float *)(ws + L.off_dh);
    unsigned char *kph = (unsigned char *)(ws + L.off_kph), *dhph = (unsigned char *)(ws + L.off_dhph);
    if (L.precision == AEXP_FP16X2_TC) {
        float *kscale = ((WsHeader *)(ws + L.off_hdr))->kscale;
        term_scale_kernel<<<1, 1024, 0, st>>>(khi_t, L.ntp, L.LP, kscale);
        prep_kph_kernel<1><<<(unsigned)((nk + T - 1) / T), T, 0, st>>>(khi_t, L.ntp, L.LP, kscale, kph);
        prep_dhph_kernel<1><<<(unsigned)((nd + T - 1) / T), T, 0, st>>>(dh, L.ntiles, L.LP, kscale, dhph);
    } else {
        prep_kph_kernel<0><<<(unsigned)((nk + T - 1) / T), T, 0, st>>>(khi_t, L.ntp, L.LP, nullptr, kph);
        prep_dhph_kernel<0><<<(unsigned)((nd + T - 1) / T), T, 0, st>>>(dh, L.ntiles, L.LP, nullptr, dhph);
    }
    return cudaGetLastError();
}

cudaError_t tcp_forward(int precision, int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                        const float2 *x, int src, const int *item_off, int total_items, int *counter, cudaStream_t st) {
    const int f = precision == AEXP_FP16X2_TC ? 1 : 0;
    switch (CB) {
        case 8: return launch_fwd_tcp_variant<8>(f, variant, pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
        case 16: return launch_fwd_tcp_variant<16>(f, variant, pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
        default: return launch_fwd_tcp_variant<32>(f, variant, pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
    }
}

cudaError_t tcp_adjoint(int precision, int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                        const float2 *yt, int src, const int *item_off, int total_items, int *counter, cudaStream_t st) {
    const int f = precision == AEXP_FP16X2_TC ? 1 : 0;
    switch (CB) {
        case 8: return launch_adj_tcp_variant<8>(f, variant, pd, nprob, max_pack_blocks, yt, src, 1, item_off, total_items, counter, st);
        case 16: return launch_adj_tcp_variant<16>(f, variant, pd, nprob, max_pack_blocks, yt, src, 1, item_off, total_items, counter, st);
        default: return launch_adj_tcp_variant<32>(f, variant, pd, nprob, max_pack_blocks, yt, src, 1, item_off, total_items, counter, st);
    }
}

cudaError_t tcp_residual_adjoint_bf16(int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                                      const float2 *ymeas, int ymeas_role, const int *item_off, int total_items,
                                      int *counter, cudaStream_t st) {
    switch (CB) {
        case 8: return launch_residual_adj_bf16<8>(variant, pd, nprob, max_pack_blocks, ymeas, ymeas_role, item_off, total_items, counter, st);
        case 16: return launch_residual_adj_bf16<16>(variant, pd, nprob, max_pack_blocks, ymeas, ymeas_role, item_off, total_items, counter, st);
        default: return launch_residual_adj_bf16<32>(variant, pd, nprob, max_pack_blocks, ymeas, ymeas_role, item_off, total_items, counter, st);
    }
}

}  // namespace aexp
