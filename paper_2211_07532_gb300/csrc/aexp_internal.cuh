// Internal declarations shared by the translation units of libaexp.
//
// Data layout in device memory (one workspace per problem, caller-owned):
//   - voxels are regrouped into 8x8 tiles ("tile order", p = tile*64 + (iy%8)*8 + ix%8);
//     partial tiles at the right/bottom edge are padded with inert voxels;
//   - field terms: the nl spherical-harmonic terms plus, when a B0 map is given,
//     one more term with coefficient t and basis omega(r) (phi = ... + omega(r) t);
//   - coefficients are kept in turns (k / 2pi) as an FP32 hi + lo pair;
//   - each tile has a reference voxel r0; its phase per sample,
//     f0(tile, t) = frac(sum_l k_l(t) h_l(r0) / 2pi), is tabulated accurately
//     once per preparation, and the kernels add the FP32 local offset
//     sum_l (k_l(t)/2pi) (h_l(r) - h_l(r0)), which stays small within a tile.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/aexp.h"

namespace aexp {

constexpr int kTileSide = 8;
constexpr int kTileVox = 64;
constexpr int kMaxTerms = 32;
constexpr int kMaxCoils = 32;
constexpr int kFwdThreads = 128;
constexpr int kAdjThreads = 128;
constexpr int kAdjStageT = 64;      // samples per adjoint smem stage
constexpr int kTPad = 512;          // nt is padded to a multiple of this
constexpr size_t kAlign = 256;

// Header at the start of every workspace (device memory).
struct WsHeader {
    int status;          // first device-side error, 0 = none
    int pad0;
    double lipschitz;    // L_f in use
    double mu;           // last Rayleigh quotient
    double nrm2;         // last squared norm
    int counter[2];      // work-item counters of the persistent kernels (forward, adjoint)
    int item_off[4];     // single problem: {0, forward items} and {0, adjoint items}
    double scratch[2];
    // FP16 hi+lo form: bit patterns of max |Re|, |Im| over the packed operand of the
    // current application (forward S x, adjoint y); they fix the power-of-two scales
    unsigned amax[2];
    int pad1[2];
    // FP64 norm reductions (dot_norm_f64): per-block partial sums (mu, nrm2) and the ticket
    // that elects the last block, which sums the partials in block order and resets it to 0
    unsigned red_ticket;
    int pad2;
    double red_part[2 * 128];
    // FP16 hi+lo form: per-term power-of-two scale of the phase-GEMM operands (k_l 2^s_l, dh_l 2^-s_l)
    float kscale[32];
};
constexpr int kRedMaxBlocks = 128;  // blocks of one dot_norm_f64 launch (WsHeader::red_part)

// Per-problem descriptor read by the persistent tensor-core kernels and by the batched
// solver kernels (device memory; one entry per problem).
struct ProbDesc {
    int nx, ny, nr, nt, nc, ntp, ntiles, ntx, nr_pad, CB, LP;
    int fwd_splits, fwd_tps, adj_splits, adj_tps, adj_vblocks;
    // operator workspace
    const float *khi_t, *f0, *dh;
    const float2 *Sp;
    unsigned char *bpk, *ypk;
    const unsigned char *kph, *dhph;  // BF16 form: phase-GEMM operands
    float *fpart;
    float2 *apart, *rt;
    WsHeader *hdr;
    // solver vectors: 0 xa, 1 xb, 2 z, 3 v, 4 w, 5 ymeas (sample-major)
    float2 *vec[6];
    char *wws;
    int npx, npy, levels, pad1;
    size_t off_pyr, off_approx[12];
    float lam;
    int pad2;
    const float2 *y_in;
    float2 *x_out;
    double *lip_out;
};

struct OpLayout {
    int nx, ny, nr, nt, nc, nl, has_b0;
    int nterms;      // nl + has_b0
    int LP;          // padded term count (template): 4, 8, 12, 20 or 32
    int CB;          // padded coil count (template): 4, 8, 16, 20, 32 (FP32) or 8, 16, 32 (TC)
    int ntx, nty, ntiles, nr_pad;
    int ntp;         // nt padded to kTPad
    int precision;
    int variant;     // kernel tiling (aexp_recon_opts::tile_variant)
    // forward split
    int fwd_mt, fwd_tblocks, fwd_splits, fwd_tiles_per_split;
    // adjoint split
    int adj_mr, adj_vblocks, adj_splits, adj_t_per_split;
    // byte offsets into the workspace
    size_t off_hdr, off_khi_l, off_klo_l, off_khi_t, off_h0, off_dh, off_f0, off_S, off_b,
        off_fpart, off_yt, off_apart, off_ypk, off_desc, off_hp;
    // BF16 form: BF16 hi | lo operands of the phase GEMM (k rows per 128 samples, basis
    // offsets per pair of tiles)
    size_t off_kph, off_dhph;
    int fwd_items, adj_items;  // persistent tensor-core work items
    size_t bytes;
};

struct WaveLayout {
    int nx, ny, levels, wavelet, npx, npy;
    size_t off_pyr;              // [npy][npx] complex
    size_t off_approx[16];       // level j approximation (j = 1..levels-1)
    size_t bytes;
};

struct RecLayout {
    OpLayout op;
    WaveLayout wv;               // offsets relative to off_wave (and off_wave2)
    size_t off_wave, off_ymeas, off_xa, off_xb, off_z, off_v, off_w;
    // differentiation buffers (with_grad only)
    size_t off_rk, off_xbar, off_vbar, off_wave2, off_zq, off_gq, off_gpart;
    // undecimated one-level wavelet: coefficients [4][nr] and the lambda-rule block
    size_t off_swt, off_swtaux;
    int grad_splits, grad_tiles_per_split;
    size_t bytes;
};

// Register blocking of the FP32 operator kernels: samples per thread in the forward,
// voxels per thread in the adjoint (each staged value is reused this many times).  At 32
// coils one per thread: 64 accumulator registers leave room for 4 blocks (16 warps) per SM,
// which hides the packed-FMA and sincos latencies better than 2 per thread at 2 blocks
// (200^2 / 32 coils: forward 5.03 -> 4.92 ms, adjoint 5.36 -> 5.17 ms).
#ifndef AEXP_FWD_MT32
#define AEXP_FWD_MT32 1
#endif
#ifndef AEXP_ADJ_MR32
#define AEXP_ADJ_MR32 1
#endif
constexpr int fwd_mt_for(int CB) { return CB >= 32 ? AEXP_FWD_MT32 : CB >= 16 ? 2 : 4; }
constexpr int adj_mr_for(int CB) { return CB >= 32 ? AEXP_ADJ_MR32 : CB >= 16 ? 2 : CB >= 8 ? 2 : 4; }
// tiling variant 1 of the FP32 form at 32 coils: two samples / voxels per thread, 2 blocks per SM
constexpr int kFp32AltBlocking = 2;
constexpr int kTileVariants = 2;

inline size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }
inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Host-side layout computation (layout.cu).
// target_items: blocks (FP32) or persistent work items (tensor cores) one launch aims for
// when the reduction dimensions are split; <= 0 selects the default, 152 SMs x
// default_items_per_sm(precision).  A batch passes its share of the target so that large
// batches use whole-problem items and few partial sums.
constexpr int kLayoutSMs = 152;
inline int default_items_per_sm(int precision) { return precision == AEXP_FP32 ? 16 : 8; }
inline int items_target(int precision, int items_per_sm) {
    return kLayoutSMs * (items_per_sm > 0 ? items_per_sm : default_items_per_sm(precision));
}
int op_layout(const aexp_problem *p, int precision, OpLayout *L, int target_items = -1, int variant = 0);
int wave_layout(int nx, int ny, int wavelet, int levels, WaveLayout *W);
// target_items < 0: taken from o->items_per_sm
int rec_layout(const aexp_problem *p, const aexp_recon_opts *o, RecLayout *R, int target_items = -1,
               int with_grad = 0);

// Launchers (all asynchronous on `st`; return cudaError_t of the launch).
cudaError_t op_prepare(const aexp_problem *p, const OpLayout &L, char *ws, cudaStream_t st);
// b = S * x into tile order; x in natural order [nr]
cudaError_t op_coil_weight(const OpLayout &L, const float2 *x, char *ws, cudaStream_t st);
// forward contraction on the prepared b -> partial sums
cudaError_t op_forward_core(const OpLayout &L, char *ws, cudaStream_t st);
// reduce forward partials: mode 0 -> y[c][t] public layout; mode 1 -> yt[t][CB] minus ymeas (residual)
cudaError_t op_forward_reduce_public(const OpLayout &L, char *ws, float2 *y, cudaStream_t st);
cudaError_t op_forward_reduce_residual(const OpLayout &L, char *ws, const float2 *ymeas_t, float2 *rt,
                                       cudaStream_t st);
// transpose public y[c][t] into yt[t][CB] (zero padded)
cudaError_t op_transpose_y(const OpLayout &L, const float2 *y, float2 *yt, cudaStream_t st);
// adjoint contraction of yt[t][CB] -> partials
cudaError_t op_adjoint_core(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st);
// reduce adjoint partials into natural order: out = sum (mode plain) or
// out = z - (2/L_f) * sum (gradient step, L_f read from the workspace header)
cudaError_t op_adjoint_reduce(const OpLayout &L, char *ws, float2 *out, cudaStream_t st);
cudaError_t op_adjoint_reduce_step(const OpLayout &L, char *ws, const float2 *z, float2 *out,
                                   cudaStream_t st);

// Descriptor of one problem's operator workspace (solver fields left empty).
ProbDesc make_op_desc(const OpLayout &L, char *ws);
cudaError_t write_desc(const ProbDesc &d, ProbDesc *dst, cudaStream_t st);
int num_sms();

// Tensor-core forms with the phase on the tensor cores (op_tc_phase.cu): operand preparation
// and the launches (same contract as batch_forward_tc / batch_adjoint_tc).  BF16: variant =
// tiling 0 (B ring 4, phase ring 3) or 1 (B ring 6, phase ring 4); FP16 hi+lo: tiling 0 (the
// FP16 hi+lo form with CUDA-core phases, op_tc.cu, is its tiling 1).
cudaError_t op_prepare_phase_operands(const OpLayout &L, char *ws, cudaStream_t st);
cudaError_t tcp_forward(int precision, int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x,
                        int src, const int *item_off, int total_items, int *counter, cudaStream_t st);
cudaError_t tcp_adjoint(int precision, int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt,
                        int src, const int *item_off, int total_items, int *counter, cudaStream_t st);
// BF16 form: A^H (A z - ymeas) from the forward partials of A z: the reduction, the residual and
// the packing in one launch, then the adjoint (ymeas as in reduce_pack_y_kernel).
cudaError_t tcp_residual_adjoint_bf16(int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks,
                                      const float2 *ymeas, int ymeas_role, const int *item_off, int total_items,
                                      int *counter, cudaStream_t st);
constexpr size_t kPhaseBlockBytes = 16384;  // 128 rows x 128 B: BF16 hi (32 K slots) | lo (32 K slots)

// Tensor-core forms (op_tc.cu): the forward packs S*x itself; the adjoint packs yt.
cudaError_t op_forward_tc(const OpLayout &L, const float2 *x, char *ws, cudaStream_t st);
cudaError_t op_adjoint_tc(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st);
// Batched tensor-core applications over nprob descriptors (uniform CB and LP): pack the
// image vec[src] (forward) or rt (adjoint), then one persistent launch over all work items.
// item_off: device prefix offsets [nprob + 1]; counter: device int reset by these calls.
// precision: AEXP_BF16_TC or AEXP_FP16X2_TC.
cudaError_t batch_forward_tc(int precision, int CB, int LP, int variant, const ProbDesc *pd, int nprob,
                             int max_pack_blocks, int src, const int *item_off, int total_items, int *counter,
                             cudaStream_t st);
cudaError_t batch_adjoint_tc(int precision, int CB, int LP, int variant, const ProbDesc *pd, int nprob,
                             int max_pack_blocks, int src, const int *item_off, int total_items, int *counter,
                             cudaStream_t st);
int fwd_pack_blocks(int ntiles, int CB);
int adj_pack_blocks(int ntp, int CB);
cudaError_t op_forward_reduce_planar_public(const OpLayout &L, char *ws, float2 *y, cudaStream_t st);
cudaError_t op_forward_reduce_planar_residual(const OpLayout &L, char *ws, const float2 *ymeas_t, float2 *rt,
                                              cudaStream_t st);

// Precision dispatch (op_dispatch.cu): one application = apply + reduce.
cudaError_t op_apply_forward(const OpLayout &L, const float2 *x, char *ws, cudaStream_t st);
cudaError_t op_reduce_forward_public(const OpLayout &L, char *ws, float2 *y, cudaStream_t st);
cudaError_t op_reduce_forward_residual(const OpLayout &L, char *ws, const float2 *ymeas_t, float2 *rt,
                                       cudaStream_t st);
cudaError_t op_apply_adjoint(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st);
// The adjoint applied to the residual of the last forward application, A^H (A z - ymeas_t)
// (ymeas_t == nullptr: A^H A z), into the adjoint partials; the FP32 residual in rt is written
// by every form but the BF16 one, which packs the residual directly.
cudaError_t op_residual_adjoint(const OpLayout &L, char *ws, const float2 *ymeas_t, cudaStream_t st);
cudaError_t op_residual_adjoint_tc(const OpLayout &L, char *ws, const float2 *ymeas_t, cudaStream_t st);

// Wavelet (wavelet.cu).  tau = lam / L_f with L_f from `lipschitz` (device), or
// lam itself when lipschitz == nullptr.  threshold == 0 disables shrinkage.
cudaError_t wave_forward(const WaveLayout &W, const float2 *img, char *wws, float lam,
                         const double *lipschitz, int threshold, cudaStream_t st);
// inverse into out (natural [ny][nx]); when momentum: x_new = result, z = x_new + beta (x_new - x_old)
cudaError_t wave_inverse(const WaveLayout &W, char *wws, float2 *out, int momentum, double beta,
                         const float2 *x_old, float2 *z_out, cudaStream_t st);

// Prox step crop(W^H soft(W pad img)) into out (natural [ny][nx]), with the momentum step when
// asked: level 1 each way plus one launch for levels 2..J when the level-1 approximation fits a
// CTA's shared memory (wave_mid_fits), else one launch per level.  Leaves the level-1 details in
// the pyramid; the coarser levels stay in shared memory.
bool wave_mid_fits(int npx, int npy, int levels);
cudaError_t wave_prox(const WaveLayout &W, const float2 *img, char *wws, float lam, const double *lipschitz,
                      float2 *out, int momentum, double beta, const float2 *x_old, float2 *z_out, cudaStream_t st);
cudaError_t batch_wave_prox(int wavelet, const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy,
                            int img_role, int out_role, int momentum, double beta, int xold_role, int z_role,
                            cudaStream_t st);

// Batched wavelet levels over a descriptor table (uniform wavelet and levels; grid sized
// for the largest padded image max_npy x max_npx).  Roles index ProbDesc::vec.
cudaError_t batch_wave_forward(int wavelet, const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy,
                               int img_role, int threshold, cudaStream_t st);
cudaError_t batch_wave_inverse(int wavelet, const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy,
                               int out_role, int momentum, double beta, int xold_role, int z_role, cudaStream_t st);

// Reductions and small vector kernels (recon.cu).
// mu = Re <v, w> (v may be null) and nrm2 = ||w||^2 in FP64; multi-block, fixed summation order;
// uses hdr->red_part and hdr->red_ticket as scratch.
cudaError_t dot_norm_f64(const float2 *v, const float2 *w, int n, double *mu, double *nrm2, WsHeader *hdr,
                         cudaStream_t st);
cudaError_t scale_inv_sqrt(const float2 *w, float2 *v, int n, const double *nrm2, cudaStream_t st);

// Solver pieces (recon.cu).
cudaError_t normal_apply(const OpLayout &L, char *ws, const float2 *v, float2 *w, cudaStream_t st);
cudaError_t power_iteration(const OpLayout &L, char *ws, const float2 *v0, float2 *v, float2 *w, int n_power,
                            double *out, cudaStream_t st);
cudaError_t set_lipschitz(const OpLayout &L, char *ws, double value, double *out, cudaStream_t st);
cudaError_t recon_issue(const aexp_problem *p, const RecLayout &R, const aexp_recon_opts *o, const float2 *y,
                        float lam, int iters, float2 *x_out, double *lip_out, char *ws, cudaStream_t st);

// The paper's undecimated one-level wavelet, tight frame W^H W = I, and lambda = sigma / 2
// (swt.cu).  Coefficients [4][ny][nx]; analysis thresholds the detail subbands with
// tau = *lam / *lip when lam is given, else with tau_host when >= 0; synthesis optionally
// applies the FISTA momentum.
size_t swt_aux_bytes();
double *swt_lambda_slot(char *aux);
cudaError_t swt_analysis(int wavelet, const float2 *v, float2 *c, int nx, int ny, float tau_host, const double *lam,
                         const double *lip, cudaStream_t st);
cudaError_t swt_synthesis(int wavelet, const float2 *c, float2 *out, int nx, int ny, int momentum, double beta,
                          const float2 *x_old, float2 *z, cudaStream_t st);
cudaError_t swt_rayleigh_lambda(const float2 *c, int nx, int ny, char *aux, double *lam_out, cudaStream_t st);
cudaError_t swt_set_lambda(char *aux, double lam, double *lam_out, cudaStream_t st);

// Coil compression by principal components of the data (coilcomp.cu): y [nc][nt], S [nc][nr]
// -> y_out [nv][nt], S_out [nv][nr]; ws of coil_compress_bytes(nc).
size_t coil_compress_bytes(int nc);
constexpr int kJacobiMaxSweeps = 40;
cudaError_t coil_compress(const float2 *y, const float2 *S, int nc, int nt, int nr, int nv, float2 *y_out,
                          float2 *S_out, double *eig_out, char *ws, cudaStream_t st,
                          int max_sweeps = kJacobiMaxSweeps);

// Least squares by CGLS (cgls.cu): operator workspace + image vectors x, p, s, k-space r, q,
// FP64 partial sums and scalars.
struct CglsLayout {
    OpLayout op;
    size_t off_x, off_p, off_s, off_r, off_q, off_part, off_scal;
    size_t bytes;
};
int cgls_layout(const aexp_problem *p, const aexp_recon_opts *o, CglsLayout *C);
cudaError_t cgls_issue(const aexp_problem *p, const CglsLayout &C, const float2 *y, int iters, float2 *x_out,
                       char *ws, cudaStream_t st);
// ||w||^2 in FP64, two-stage fixed-order reduction (partial: 256 doubles of scratch).
cudaError_t norm2_f64(const float2 *w, size_t n, double *partial, double *out, cudaStream_t st);

// Failure-detection probe (probe.cu): one block whose bounded waits on barriers that nothing
// completes must give up; result[0] / result[1] = 1 when the plain / the abort-aware wait gave up.
cudaError_t bounded_wait_probe(int polls, int *status, int *result, cudaStream_t st);

// Record a CUDA error for aexp_last_cuda_error() (capi.cu).
void aexp_set_last_cuda_error(int e);
// Drop the host-side record of what `ws` was prepared for (its contents were overwritten).
void forget_prepared(const void *ws);

// Differentiation through unrolled FISTA (grad.cu).
cudaError_t unroll_step(const RecLayout &R, const float2 *y, float lam, double lipschitz, const float2 *z,
                        const float2 *x_prev, double beta, float2 *x_out, float2 *z_out, char *ws, cudaStream_t st);
cudaError_t unroll_step_vjp(const RecLayout &R, const float2 *y, float lam, double lipschitz, const float2 *z,
                            double beta, double beta_next, const float2 *xbar_in, const float2 *zbar_next,
                            const float2 *zbar_next2, float2 *zbar_out, float *kbar, double *lambar, char *ws,
                            cudaStream_t st);

// Error flag writers used by the kernels.
__device__ __forceinline__ void set_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier + bulk (TMA) copies global -> shared.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (default ~2^22; each poll may suspend briefly),
// records AEXP_ERR_DEVICE_TIMEOUT and returns false.
constexpr int kWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int *status,
                                                  int limit = kWaitPolls) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    set_status(status, AEXP_ERR_DEVICE_TIMEOUT);
    return false;
}

// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// FP32 pair arithmetic (error-free transformations; Knuth two-sum, FMA two-product)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

}  // namespace aexp
