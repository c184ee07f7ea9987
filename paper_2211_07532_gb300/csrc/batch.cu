// Ragged batches: many independent slice problems (resolutions, diffusion volumes, slices,
// each with its own field coefficients) reconstructed together.  Every operator
// application of the whole batch is one persistent tensor-core launch (forward) plus one
// (adjoint) over a device table of per-problem descriptors; the small steps of the solver
// (reductions, norms, wavelet levels, momentum) are batched kernels whose grid carries
// the problem index; cs_recon_batched captures the whole solve in one CUDA graph.
#include <math.h>

#include <algorithm>
#include <vector>

#include "aexp_internal.cuh"
#include "batch_internal.h"
#include "reduce_f64.cuh"

namespace aexp {

namespace {

// prefix arrays of up to kMaxBatchProblems + 1 entries written through one kernel argument
struct OffsetsArg {
    int n;
    int v[kMaxBatchProblems + 1];
};

__global__ void set_offsets_kernel(int *dst, OffsetsArg a) {
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) dst[i] = a.v[i];
}

__device__ __forceinline__ int tile_index(const ProbDesc &P, int r) {
    const int ix = r % P.nx, iy = r / P.nx;
    return ((iy / kTileSide) * P.ntx + ix / kTileSide) * kTileVox + (iy % kTileSide) * kTileSide + ix % kTileSide;
}

// zero the per-problem header scalars, status and FP64-reduction ticket
__global__ void batch_reset_kernel(const ProbDesc *pd, int nprob) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    WsHeader *h = pd[q].hdr;
    h->status = 0;
    h->lipschitz = 0.0;
    h->mu = 0.0;
    h->nrm2 = 0.0;
    h->red_ticket = 0u;
}

// measured k-space y[c][t] -> sample-major vec[5][t][CB] (zero padded)
__global__ void batch_transpose_y_kernel(const ProbDesc *pd) {
    const ProbDesc &P = pd[blockIdx.y];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)P.ntp * P.CB) return;
    const int t = (int)(i / P.CB), c = (int)(i % P.CB);
    P.vec[5][i] = (t < P.nt && c < P.nc) ? P.y_in[(size_t)c * P.nt + t] : make_float2(0.f, 0.f);
}

// rt = sum of the planar forward partials (- ymeas when use_ymeas)
__global__ void batch_fwd_reduce_kernel(const ProbDesc *pd, int use_ymeas) {
    const ProbDesc &P = pd[blockIdx.y];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)P.ntp * P.CB) return;
    const int t = (int)(i / P.CB), c = (int)(i % P.CB);
    float2 s = make_float2(0.f, 0.f);
    if (t < P.nt && c < P.nc) {
        for (int k = 0; k < P.fwd_splits; ++k) {
            const float *row = P.fpart + ((size_t)k * P.ntp + t) * 2 * P.CB;
            s.x += row[c];
            s.y += row[P.CB + c];
        }
        if (use_ymeas) {
            s.x -= P.vec[5][i].x;
            s.y -= P.vec[5][i].y;
        }
    }
    P.rt[i] = s;
}

// out = sum of the adjoint partials (natural order), or the gradient step
// out = z - (2/L_f) * sum when z_role >= 0
__global__ void batch_adj_reduce_kernel(const ProbDesc *pd, int z_role, int out_role) {
    const ProbDesc &P = pd[blockIdx.y];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.nr) return;
    const int p = tile_index(P, r);
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < P.adj_splits; ++k) {
        float2 v = P.apart[(size_t)k * P.nr_pad + p];
        s.x += v.x;
        s.y += v.y;
    }
    if (z_role >= 0) {
        const float step = (float)(2.0 / P.hdr->lipschitz);
        const float2 zv = P.vec[z_role][r];
        s.x = zv.x - step * s.x;
        s.y = zv.y - step * s.y;
    }
    P.vec[out_role][r] = s;
}

// FP64 mu = Re <v, w> (when v_role >= 0) and nrm2 = ||w||^2 of every problem: blockIdx.y is
// the problem, its gridDim.x blocks form one deterministic grid reduction over its own
// partials and ticket (WsHeader of the problem)
__global__ void __launch_bounds__(kDotThreads) batch_dot_norm_kernel(const ProbDesc *pd, int v_role, int w_role) {
    const ProbDesc &P = pd[blockIdx.y];
    const float2 *w = P.vec[w_role];
    const float2 *v = v_role >= 0 ? P.vec[v_role] : nullptr;
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * kDotThreads + threadIdx.x; i < P.nr; i += gridDim.x * kDotThreads) {
        const float2 wv = w[i];
        if (v) {
            const float2 vv = v[i];
            a = fma((double)vv.x, (double)wv.x, a);
            a = fma((double)vv.y, (double)wv.y, a);
        }
        b = fma((double)wv.x, (double)wv.x, b);
        b = fma((double)wv.y, (double)wv.y, b);
    }
    if (grid_sum2(a, b, blockIdx.x, gridDim.x, P.hdr->red_part, &P.hdr->red_ticket)) {
        if (v) P.hdr->mu = a;
        P.hdr->nrm2 = b;
    }
}

__global__ void batch_scale_kernel(const ProbDesc *pd, int w_role, int v_role) {
    const ProbDesc &P = pd[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nr) return;
    const double nn = P.hdr->nrm2;
    const float s = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    const float2 a = P.vec[w_role][i];
    P.vec[v_role][i] = make_float2(a.x * s, a.y * s);
}

// L_f = 2 mu (or the given value when fixed > 0); records AEXP_ERR_NONFINITE per problem
__global__ void batch_finalize_kernel(const ProbDesc *pd, int nprob, double fixed) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    const ProbDesc &P = pd[q];
    double L = fixed > 0.0 ? fixed : 2.0 * P.hdr->mu;
    if (!(L > 0.0) || !isfinite(L)) {
        atomicCAS(&P.hdr->status, 0, AEXP_ERR_NONFINITE);
        L = 1.0;
    }
    P.hdr->lipschitz = L;
    if (P.lip_out) *P.lip_out = L;
}

__global__ void batch_zero_kernel(const ProbDesc *pd, int role) {
    const ProbDesc &P = pd[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.nr) P.vec[role][i] = make_float2(0.f, 0.f);
}

// first device-side error of any problem -> the batch header's status word
__global__ void batch_collect_status_kernel(const ProbDesc *pd, int nprob, WsHeader *bh) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    const int s = pd[q].hdr->status;
    if (s != 0) atomicCAS(&bh->status, 0, s);
}

__global__ void batch_copy_out_kernel(const ProbDesc *pd, int role) {
    const ProbDesc &P = pd[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.nr) P.x_out[i] = P.vec[role][i];
}

#define CK(x)                               \
    do {                                    \
        cudaError_t e__ = (x);              \
        if (e__ != cudaSuccess) return e__; \
    } while (0)

}  // namespace

int batch_layout(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts, BatchLayout *B) {
    BatchLayout b{};
    b.nprob = nprob;
    // whole-problem items once the batch alone fills the GPU several times over
    const int target = std::max(1, items_target(opts->precision, opts->items_per_sm) / nprob);
    b.R.resize(nprob);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    b.off_hdr = take(sizeof(WsHeader));
    b.off_desc = take(sizeof(ProbDesc) * (size_t)nprob);
    b.off_items_fwd = take(sizeof(int) * (size_t)(nprob + 1));
    b.off_items_adj = take(sizeof(int) * (size_t)(nprob + 1));
    b.items_fwd.assign(nprob + 1, 0);
    b.items_adj.assign(nprob + 1, 0);
    b.base.resize(nprob);
    for (int q = 0; q < nprob; ++q) {
        int rc = rec_layout(&probs[q], opts, &b.R[q], target);
        if (rc) return rc;
        const OpLayout &L = b.R[q].op;
        if (q == 0) {
            b.CB = L.CB;
            b.LP = L.LP;
        } else if (L.CB != b.CB || L.LP != b.LP) {
            return AEXP_ERR_UNSUPPORTED;  // one template instance per launch: uniform paddings
        }
        b.base[q] = take(b.R[q].bytes);
        b.items_fwd[q + 1] = b.items_fwd[q] + L.fwd_items;
        b.items_adj[q + 1] = b.items_adj[q] + L.adj_items;
        b.max_nr = std::max(b.max_nr, L.nr);
        b.max_ntpcb = std::max(b.max_ntpcb, L.ntp * L.CB);
        b.max_fwd_pack = std::max(b.max_fwd_pack, fwd_pack_blocks(L.ntiles, L.CB));
        b.max_adj_pack = std::max(b.max_adj_pack, adj_pack_blocks(L.ntp, L.CB));
        b.max_npx = std::max(b.max_npx, b.R[q].wv.npx);
        b.max_npy = std::max(b.max_npy, b.R[q].wv.npy);
    }
    b.bytes = off;
    *B = std::move(b);
    return AEXP_OK;
}

cudaError_t batch_setup(const aexp_problem *probs, const BatchLayout &B, const void *const *y, const float *lambda,
                        void *const *x_out, double *lip_out, char *ws, cudaStream_t st) {
    const int n = B.nprob;
    ProbDesc *pd = (ProbDesc *)(ws + B.off_desc);
    int *ifwd = (int *)(ws + B.off_items_fwd);
    int *iadj = (int *)(ws + B.off_items_adj);
    const int T = 256;

    // per-problem preparation and descriptors
    for (int q = 0; q < n; ++q) {
        const RecLayout &R = B.R[q];
        char *w = ws + B.base[q];
        CK(op_prepare(&probs[q], R.op, w, st));
        ProbDesc d = make_op_desc(R.op, w);
        d.vec[0] = (float2 *)(w + R.off_xa);
        d.vec[1] = (float2 *)(w + R.off_xb);
        d.vec[2] = (float2 *)(w + R.off_z);
        d.vec[3] = (float2 *)(w + R.off_v);
        d.vec[4] = (float2 *)(w + R.off_w);
        d.vec[5] = (float2 *)(w + R.off_ymeas);
        d.wws = w + R.off_wave;
        d.npx = R.wv.npx;
        d.npy = R.wv.npy;
        d.levels = R.wv.levels;
        d.off_pyr = R.wv.off_pyr;
        for (int j = 0; j < 12; ++j) d.off_approx[j] = R.wv.off_approx[j];
        d.lam = lambda ? lambda[q] : 0.f;
        d.y_in = y ? (const float2 *)y[q] : nullptr;
        d.x_out = x_out ? (float2 *)x_out[q] : nullptr;
        d.lip_out = lip_out ? lip_out + q : nullptr;
        CK(write_desc(d, pd + q, st));
    }
    {
        OffsetsArg a;
        a.n = n + 1;
        for (int q = 0; q <= n; ++q) a.v[q] = B.items_fwd[q];
        set_offsets_kernel<<<1, 256, 0, st>>>(ifwd, a);
        for (int q = 0; q <= n; ++q) a.v[q] = B.items_adj[q];
        set_offsets_kernel<<<1, 256, 0, st>>>(iadj, a);
    }
    batch_reset_kernel<<<cdiv(n, T), T, 0, st>>>(pd, n);
    return cudaGetLastError();
}

// One A^H A application of every problem of a set-up batch on a zero image (the
// autotuner's timing unit: the work does not depend on the values).
cudaError_t batch_normal_once(const BatchLayout &B, const aexp_recon_opts *o, char *ws, cudaStream_t st) {
    const int n = B.nprob;
    ProbDesc *pd = (ProbDesc *)(ws + B.off_desc);
    WsHeader *bh = (WsHeader *)(ws + B.off_hdr);
    const int *ifwd = (const int *)(ws + B.off_items_fwd);
    const int *iadj = (const int *)(ws + B.off_items_adj);
    const int T = 256;
    const dim3 g_nr(cdiv(B.max_nr, T), n), g_ntp(cdiv(B.max_ntpcb, T), n);
    enum { Z = 2, W = 4 };
    batch_zero_kernel<<<g_nr, T, 0, st>>>(pd, Z);
    CK(batch_forward_tc(o->precision, B.CB, B.LP, o->tile_variant, pd, n, B.max_fwd_pack, Z, ifwd, B.items_fwd[n], &bh->counter[0],
                        st));
    if (o->precision == AEXP_BF16_TC) {
        CK(tcp_residual_adjoint_bf16(B.CB, o->tile_variant, pd, n, B.max_adj_pack, nullptr, -1, iadj, B.items_adj[n],
                                     &bh->counter[1], st));
    } else {
        batch_fwd_reduce_kernel<<<g_ntp, T, 0, st>>>(pd, 0);
        CK(batch_adjoint_tc(o->precision, B.CB, B.LP, o->tile_variant, pd, n, B.max_adj_pack, -1, iadj, B.items_adj[n],
                            &bh->counter[1], st));
    }
    batch_adj_reduce_kernel<<<g_nr, T, 0, st>>>(pd, -1, W);
    return cudaGetLastError();
}

cudaError_t batch_recon_issue(const aexp_problem *probs, const BatchLayout &B, const aexp_recon_opts *o,
                              const void *const *y, const float *lambda, int iters, void *const *x_out,
                              double *lip_out, char *ws, cudaStream_t st) {
    const int n = B.nprob;
    ProbDesc *pd = (ProbDesc *)(ws + B.off_desc);
    WsHeader *bh = (WsHeader *)(ws + B.off_hdr);
    int *ifwd = (int *)(ws + B.off_items_fwd);
    int *iadj = (int *)(ws + B.off_items_adj);
    const int T = 256;

    CK(batch_setup(probs, B, y, lambda, x_out, lip_out, ws, st));
    batch_transpose_y_kernel<<<dim3(cdiv(B.max_ntpcb, T), n), T, 0, st>>>(pd);
    CK(cudaGetLastError());

    const int tot_f = B.items_fwd[n], tot_a = B.items_adj[n];
    const dim3 g_nr(cdiv(B.max_nr, T), n), g_ntp(cdiv(B.max_ntpcb, T), n);
    // FP64 norms: enough blocks per problem to spread the FP64 work, at most ~8 per SM in all
    const int g_red = std::max(1, std::min(std::min(kRedMaxBlocks, cdiv(B.max_nr, 2 * kDotThreads)), cdiv(8 * num_sms(), n)));
    // adjoint partials of A^H (A z - ymeas) (use_ymeas) or A^H A z, from the forward partials
    // of A z; the BF16 form packs the residual in the reduction's pass
    auto residual_adjoint = [&](int use_ymeas) -> cudaError_t {
        if (o->precision == AEXP_BF16_TC)
            return tcp_residual_adjoint_bf16(B.CB, o->tile_variant, pd, n, B.max_adj_pack, nullptr, use_ymeas ? 5 : -1,  // vec[5]: ymeas
                                            
                                             iadj, tot_a, &bh->counter[1], st);
        batch_fwd_reduce_kernel<<<g_ntp, T, 0, st>>>(pd, use_ymeas);
        return batch_adjoint_tc(o->precision, B.CB, B.LP, o->tile_variant, pd, n, B.max_adj_pack, -1, iadj, tot_a,
                                &bh->counter[1], st);
    };
    // w = A^H A v for every problem (v in role vr, w in role wr)
    auto normal = [&](int vr, int wr) -> cudaError_t {
        CK(batch_forward_tc(o->precision, B.CB, B.LP, o->tile_variant, pd, n, B.max_fwd_pack, vr, ifwd, tot_f, &bh->counter[0], st));
        CK(residual_adjoint(0));
        batch_adj_reduce_kernel<<<g_nr, T, 0, st>>>(pd, -1, wr);
        return cudaGetLastError();
    };

    enum { XA = 0, XB = 1, Z = 2, V = 3, W = 4, YM = 5 };
    if (o->lipschitz > 0.0) {
        batch_finalize_kernel<<<cdiv(n, T), T, 0, st>>>(pd, n, o->lipschitz);
    } else {
        // power iteration from A^H y
        CK(batch_adjoint_tc(o->precision, B.CB, B.LP, o->tile_variant, pd, n, B.max_adj_pack, YM, iadj, tot_a, &bh->counter[1], st));
        batch_adj_reduce_kernel<<<g_nr, T, 0, st>>>(pd, -1, W);
        batch_dot_norm_kernel<<<dim3(g_red, n), kDotThreads, 0, st>>>(pd, -1, W);
        batch_scale_kernel<<<g_nr, T, 0, st>>>(pd, W, V);
        for (int i = 0; i < o->n_power; ++i) {
            CK(normal(V, W));
            batch_dot_norm_kernel<<<dim3(g_red, n), kDotThreads, 0, st>>>(pd, V, W);
            batch_scale_kernel<<<g_nr, T, 0, st>>>(pd, W, V);
        }
        batch_finalize_kernel<<<cdiv(n, T), T, 0, st>>>(pd, n, 0.0);
    }
    CK(cudaGetLastError());

    // FISTA from zero for every problem
    batch_zero_kernel<<<g_nr, T, 0, st>>>(pd, XA);
    batch_zero_kernel<<<g_nr, T, 0, st>>>(pd, Z);
    int prev = XA, next = XB;
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        CK(batch_forward_tc(o->precision, B.CB, B.LP, o->tile_variant, pd, n, B.max_fwd_pack, Z, ifwd, tot_f, &bh->counter[0], st));
        CK(residual_adjoint(1));
        batch_adj_reduce_kernel<<<g_nr, T, 0, st>>>(pd, Z, V);
        const double t_next = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
        const double beta = (t - 1.0) / t_next;
        CK(batch_wave_prox(o->wavelet, pd, n, o->levels, B.max_npx, B.max_npy, V, next, 1, beta, prev, Z, st));
        t = t_next;
        std::swap(prev, next);
    }
    batch_copy_out_kernel<<<g_nr, T, 0, st>>>(pd, prev);
    batch_collect_status_kernel<<<cdiv(n, T), T, 0, st>>>(pd, n, bh);
    return cudaGetLastError();
}

}  // namespace aexp
