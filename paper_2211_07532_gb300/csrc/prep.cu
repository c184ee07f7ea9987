// Preparation kernels: derive the operator's internal layouts from a problem.
//
// The phase of Sec. 1 / Eq. 1's expanded model, phi(t,r) = sum_l k_l(t) h_l(r) + omega(r) t,
// reaches hundreds of radians at 1.1 mm resolution (k_max = pi/dx, |r| <= FOV/2), so a
// plain FP32 product-sum loses ~1e-5 rad.  The kernels therefore split it per 8x8 tile:
//   phi/2pi = f0(tile, t) + sum_l kt_l(t) (h_l(r) - h_l(r0(tile)))      (mod 1)
// with kt = k/2pi.  f0 is tabulated here from FP32 pairs (error-free products and sums)
// so that it is exact to ~1e-8 turns; the local sum only spans one tile.
#include "aexp_internal.cuh"

namespace aexp {

namespace {

constexpr double kInv2Pi = 0.15915494309189533576888376337251436;

__device__ __forceinline__ float term_coef(const float *k, const float *tt, int nl, int has_b0, int nt,
                                           int l, int t) {
    if (t >= nt) return 0.f;
    if (l < nl) return k[(size_t)l * nt + t];
    if (has_b0 && l == nl) return tt[t];
    return 0.f;
}

__device__ __forceinline__ float term_basis(const float *h, const float *om, int nl, int has_b0, int nr,
                                            int l, int r) {
    if (l < nl) return h[(size_t)l * nr + r];
    if (has_b0 && l == nl) return om[r];
    return 0.f;
}

// k_l(t) / 2pi as a hi + lo FP32 pair; l-major [LP][ntp] copies and a t-major hi copy.
__global__ void prep_coef_kernel(const float *k, const float *tt, int nl, int has_b0, int nt, int ntp, int LP,
                                 float *khi_l, float *klo_l, float *khi_t) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int l = blockIdx.y;
    if (t >= ntp) return;
    const float c_hi = (float)kInv2Pi;
    const float c_lo = (float)(kInv2Pi - (double)(float)kInv2Pi);
    float v = term_coef(k, tt, nl, has_b0, nt, l, t);
    float p = __fmul_rn(v, c_hi);
    float e = fmaf(v, c_hi, -p);
    e = fmaf(v, c_lo, e);
    float hi, lo;
    fast_two_sum(p, e, hi, lo);
    khi_l[(size_t)l * ntp + t] = hi;
    klo_l[(size_t)l * ntp + t] = lo;
    khi_t[(size_t)t * LP + l] = hi;
}

// Reference voxel of each tile (centre, clipped into the image), the FP32 basis offsets
// dh[p][l] = h_l(r) - h_l(r0) and the basis values hp[p][l] = h_l(r) in tile order, zero for
// padded voxels.  One thread per (p, l).
__global__ void prep_tile_kernel(const float *h, const float *om, int nl, int has_b0, int nx, int ny, int ntx,
                                 int ntiles, int LP, float *h0, float *dh, float *hp) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int l = blockIdx.y;
    if (p >= ntiles * kTileVox) return;
    int tile = p / kTileVox, v = p % kTileVox;
    int tx = tile % ntx, ty = tile / ntx;
    int ix = tx * kTileSide + v % kTileSide, iy = ty * kTileSide + v / kTileSide;
    int rx = min(tx * kTileSide + kTileSide / 2, nx - 1);
    int ry = min(ty * kTileSide + kTileSide / 2, ny - 1);
    int nr = nx * ny;
    float ref = term_basis(h, om, nl, has_b0, nr, l, ry * nx + rx);
    float d = 0.f, hv = 0.f;
    if (ix < nx && iy < ny) {
        hv = term_basis(h, om, nl, has_b0, nr, l, iy * nx + ix);
        d = __fsub_rn(hv, ref);
    }
    dh[(size_t)p * LP + l] = d;
    hp[(size_t)p * LP + l] = hv;  // basis values in tile order (gradient with respect to k)
    if (v == 0) h0[(size_t)tile * LP + l] = ref;
}

// f0(tile, t) = frac( sum_l (khi + klo)_l(t) * h0_l(tile) ), computed with exact products
// (FMA residual), exact fractional parts (x - rint(x) is exact in FP32) and two-sum
// accumulation.  Result in [-0.5, 0.5] turns.
__global__ void prep_f0_kernel(const float *khi_l, const float *klo_l, const float *h0, int nterms, int ntp,
                               int LP, float *f0) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int tile = blockIdx.y;
    if (t >= ntp) return;
    float s_hi = 0.f, s_lo = 0.f;
    for (int l = 0; l < nterms; ++l) {
        float hv = h0[(size_t)tile * LP + l];
        float kh = khi_l[(size_t)l * ntp + t];
        float kl = klo_l[(size_t)l * ntp + t];
        float p = __fmul_rn(kh, hv);
        float e = fmaf(kh, hv, -p);
        e = fmaf(kl, hv, e);
        p = __fsub_rn(p, rintf(p));
        float s, err;
        two_sum(s_hi, p, s, err);
        s_hi = __fsub_rn(s, rintf(s));
        s_lo = __fadd_rn(s_lo, __fadd_rn(err, e));
    }
    float f = __fadd_rn(s_hi, s_lo);
    f = __fsub_rn(f, rintf(f));
    f0[(size_t)tile * ntp + t] = f;
}

// Coil maps in tile order, voxel-major: Sp[p][c], zero for padded voxels / coils.
__global__ void prep_coil_kernel(const float2 *S, int nc, int nx, int ny, int ntx, int nr_pad, int CB, float2 *Sp) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nr_pad * CB) return;
    int p = (int)(i / CB), c = (int)(i % CB);
    int tile = p / kTileVox, v = p % kTileVox;
    int ix = (tile % ntx) * kTileSide + v % kTileSide, iy = (tile / ntx) * kTileSide + v / kTileSide;
    float2 s = make_float2(0.f, 0.f);
    if (c < nc && ix < nx && iy < ny) s = S[(size_t)c * nx * ny + (size_t)iy * nx + ix];
    Sp[i] = s;
}

// b[p][c] = S_c(r(p)) x(r(p)) in tile order (the coil-weighted images of the forward model).
// b[p][coil pair q] = (re c, re c+1, im c, im c+1), c = 2q: the FP32 forward's packed operands
__global__ void coil_weight_kernel(const float2 *Sp, const float2 *x, int nx, int ny, int ntx, int nr_pad, int CB,
                                   float *b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nr_pad * CB) return;
    int p = (int)(i / CB);
    int tile = p / kTileVox, v = p % kTileVox;
    int ix = (tile % ntx) * kTileSide + v % kTileSide, iy = (tile / ntx) * kTileSide + v / kTileSide;
    float2 out = make_float2(0.f, 0.f);
    if (ix < nx && iy < ny) {
        float2 s = Sp[i];
        float2 xv = x[(size_t)iy * nx + ix];
        out.x = s.x * xv.x - s.y * xv.y;
        out.y = s.x * xv.y + s.y * xv.x;
    }
    float *dst = b + (size_t)p * CB * 2 + ((i % CB) >> 1) * 4 + (i & 1);
    dst[0] = out.x;
    dst[2] = out.y;
}

__global__ void set_items_kernel(WsHeader *hdr, int fwd_items, int adj_items) {
    hdr->item_off[0] = 0;
    hdr->item_off[1] = fwd_items;
    hdr->item_off[2] = 0;
    hdr->item_off[3] = adj_items;
}

__global__ void transpose_y_kernel(const float2 *y, int nt, int nc, int ntp, int CB, float2 *yt) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)ntp * CB) return;
    int t = (int)(i / CB), c = (int)(i % CB);
    yt[i] = (t < nt && c < nc) ? y[(size_t)c * nt + t] : make_float2(0.f, 0.f);
}

}  // namespace

cudaError_t op_prepare(const aexp_problem *p, const OpLayout &L, char *ws, cudaStream_t st) {
    float *khi_l = (float *)(ws + L.off_khi_l);
    float *klo_l = (float *)(ws + L.off_klo_l);
    float *khi_t = (float *)(ws + L.off_khi_t);
    float *h0 = (float *)(ws + L.off_h0);
    float *dh = (float *)(ws + L.off_dh);
    float *f0 = (float *)(ws + L.off_f0);
    float2 *Sp = (float2 *)(ws + L.off_S);
    const int T = 256;
    prep_coef_kernel<<<dim3(cdiv(L.ntp, T), L.LP), T, 0, st>>>(p->k, p->t, L.nl, L.has_b0, L.nt, L.ntp, L.LP,
                                                              khi_l, klo_l, khi_t);
    prep_tile_kernel<<<dim3(cdiv(L.nr_pad, T), L.LP), T, 0, st>>>(p->h, p->omega, L.nl, L.has_b0, L.nx, L.ny,
                                                                 L.ntx, L.ntiles, L.LP, h0, dh,
                                                                 (float *)(ws + L.off_hp));
    prep_f0_kernel<<<dim3(cdiv(L.ntp, T), L.ntiles), T, 0, st>>>(khi_l, klo_l, h0, L.nterms, L.ntp, L.LP, f0);
    size_t n = (size_t)L.nr_pad * L.CB;
    prep_coil_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>((const float2 *)p->S, L.nc, L.nx, L.ny, L.ntx,
                                                               L.nr_pad, L.CB, Sp);
    if (L.precision != AEXP_FP32) {
        cudaError_t e = op_prepare_phase_operands(L, ws, st);
        if (e != cudaSuccess) return e;
    }
    if (L.precision != AEXP_FP32) {
        // descriptor and work items of the persistent tensor-core kernels
        cudaError_t e = write_desc(make_op_desc(L, ws), (ProbDesc *)(ws + L.off_desc), st);
        if (e != cudaSuccess) return e;
        set_items_kernel<<<1, 1, 0, st>>>((WsHeader *)(ws + L.off_hdr), L.fwd_items, L.adj_items);
    }
    return cudaGetLastError();
}

cudaError_t op_coil_weight(const OpLayout &L, const float2 *x, char *ws, cudaStream_t st) {
    size_t n = (size_t)L.nr_pad * L.CB;
    const int T = 256;
    coil_weight_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>((const float2 *)(ws + L.off_S), x, L.nx, L.ny,
                                                                 L.ntx, L.nr_pad, L.CB, (float *)(ws + L.off_b));
    return cudaGetLastError();
}

cudaError_t op_transpose_y(const OpLayout &L, const float2 *y, float2 *yt, cudaStream_t st) {
    size_t n = (size_t)L.ntp * L.CB;
    const int T = 256;
    transpose_y_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(y, L.nt, L.nc, L.ntp, L.CB, yt);
    return cudaGetLastError();
}

}  // namespace aexp
