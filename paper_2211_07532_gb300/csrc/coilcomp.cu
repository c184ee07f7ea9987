// Coil compression on the device (Sec. 2.2.1: 32 receive channels compressed to 20 virtual
// coils to speed the reconstruction up; Sec. 2.2.2 studies 8 / 16 / 32).  Principal components
// of the k-space data, applied to data and coil maps alike:
//   C = y y^H (FP64),  C = U diag(e) U^H (e descending),  every column u_k scaled so that its
//   largest component (lowest index on a tie) is real and positive,
//   y_v = U_v^H y ([nv][nt]),  S_v = U_v^H S ([nv][nr]),  U_v = the first nv columns.
// The encoding matrix does not depend on the coil, so the compressed problem keeps k, h,
// omega and t and takes nc = nv, S = S_v.
//
// Eigenvectors: cyclic Jacobi for Hermitian matrices in one block (nc <= 32), FP64, with the
// round-robin ordering (m / 2 disjoint pairs per round, m = nc rounded up to even) so that all
// rotations of a round are applied at once; at most 40 sweeps (a caller may cap them lower), stopping when the
// off-diagonal Frobenius norm falls below 1e-15 of the total.  Each rotation zeroes the (p, q)
// entry: with c = C_pq = |c| e^{i phi}, theta = atan2(2 |c|, C_pp - C_qq) / 2, the unitary acting
// on columns p, q is [[cos, -sin], [e^{-i phi} sin, e^{-i phi} cos]].
#include <math.h>

#include "aexp_internal.cuh"

namespace aexp {

namespace {

constexpr int kMaxC = 32;

struct cd {  // complex double in shared memory
    double x, y;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.x, -a.y}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd cscale(double s, cd a) { return {s * a.x, s * a.y}; }

// C[a][b] = sum_t y_a(t) conj(y_b(t)), one block per (a, b)
__global__ void covariance_kernel(const float2 *__restrict__ y, int nc, int nt, double2 *__restrict__ C) {
    const int a = blockIdx.x, b = blockIdx.y;
    __shared__ double sr[8], si[8];
    double re = 0.0, im = 0.0;
    const float2 *ya = y + (size_t)a * nt, *yb = y + (size_t)b * nt;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const float2 u = ya[t], v = yb[t];
        re += (double)u.x * v.x + (double)u.y * v.y;
        im += (double)u.y * v.x - (double)u.x * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sr[threadIdx.x >> 5] = re;
        si[threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r2 = 0.0, i2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            r2 += sr[w];
            i2 += si[w];
        }
        C[(size_t)a * nc + b] = make_double2(r2, i2);
    }
}

// One block of 256 threads: eigen-decomposition of the nc x nc Hermitian C, sorting, phase
// normalisation; writes the eigenvalues (descending) and U (column-major in [k][a]: U[k * nc + a]).
__global__ void __launch_bounds__(256) jacobi_kernel(const double2 *__restrict__ Cin, int nc, double2 *__restrict__ Uout,
                                                     double *__restrict__ eig, int max_sweeps, int *status) {
    __shared__ cd A[kMaxC][kMaxC + 1], V[kMaxC][kMaxC + 1];
    __shared__ double rc[kMaxC / 2], rs[kMaxC / 2];
    __shared__ cd rph[kMaxC / 2];
    __shared__ int rp[kMaxC / 2], rq[kMaxC / 2];
    __shared__ double s_off, s_tot;
    __shared__ int order[kMaxC];
    const int tid = threadIdx.x;
    const int m = nc + (nc & 1);
    for (int i = tid; i < nc * nc; i += blockDim.x) {
        const int r = i / nc, c = i % nc;
        const double2 v = Cin[i];
        A[r][c] = {v.x, v.y};
        V[r][c] = {r == c ? 1.0 : 0.0, 0.0};
    }
    __syncthreads();
    bool converged = false;
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        if (tid == 0) {
            double off = 0.0, tot = 0.0;
            for (int r = 0; r < nc; ++r)
                for (int c = 0; c < nc; ++c) {
                    const double v = A[r][c].x * A[r][c].x + A[r][c].y * A[r][c].y;
                    tot += v;
                    if (r != c) off += v;
                }
            s_off = off;
            s_tot = tot;
        }
        __syncthreads();
        converged = !(s_off > 1e-30 * s_tot);  // off-diagonal norm below 1e-15 of the total
        __syncthreads();
        if (converged) break;
        for (int rnd = 0; rnd < m - 1; ++rnd) {
            // rotations of this round (element m - 1 fixed, the rest rotate)
            if (tid < m / 2) {
                int p, q;
                if (tid == 0) {
                    p = m - 1;
                    q = rnd;
                } else {
                    p = (rnd + tid) % (m - 1);
                    q = (rnd - tid + (m - 1)) % (m - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                rp[tid] = p;
                rq[tid] = q;
                double cs = 1.0, sn = 0.0;
                cd ph = {1.0, 0.0};
                if (q < nc) {
                    const cd c = A[p][q];
                    const double r = sqrt(c.x * c.x + c.y * c.y);
                    if (r > 0.0) {
                        ph = {c.x / r, c.y / r};
                        const double th = 0.5 * atan2(2.0 * r, A[p][p].x - A[q][q].x);
                        cs = cos(th);
                        sn = sin(th);
                    }
                }
                rc[tid] = cs;
                rs[tid] = sn;
                rph[tid] = ph;
            }
            __syncthreads();
            // columns: A <- A U, V <- V U (U acts on columns p, q of each pair)
            for (int i = tid; i < (m / 2) * nc; i += blockDim.x) {
                const int k = i / nc, r = i % nc;
                const int p = rp[k], q = rq[k];
                if (q >= nc) continue;
                const double cs = rc[k], sn = rs[k];
                const cd e = cconj(rph[k]);  // e^{-i phi}
                const cd up = cscale(sn, e), uq = cscale(cs, e);
                cd ap = A[r][p], aq = A[r][q];
                A[r][p] = cadd(cscale(cs, ap), cmul(aq, up));
                A[r][q] = cadd(cscale(-sn, ap), cmul(aq, uq));
                cd vp = V[r][p], vq = V[r][q];
                V[r][p] = cadd(cscale(cs, vp), cmul(vq, up));
                V[r][q] = cadd(cscale(-sn, vp), cmul(vq, uq));
            }
            __syncthreads();
            // rows: A <- U^H A
            for (int i = tid; i < (m / 2) * nc; i += blockDim.x) {
                const int k = i / nc, c = i % nc;
                const int p = rp[k], q = rq[k];
                if (q >= nc) continue;
                const double cs = rc[k], sn = rs[k];
                const cd e = rph[k];  // conj of e^{-i phi}
                const cd ap = A[p][c], aq = A[q][c];
                A[p][c] = cadd(cscale(cs, ap), cmul(cscale(sn, e), aq));
                A[q][c] = cadd(cscale(-sn, ap), cmul(cscale(cs, e), aq));
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        if (!converged) atomicCAS(status, 0, AEXP_ERR_NONFINITE);
        // descending order of the eigenvalues (selection, ties by index)
        bool used[kMaxC] = {};
        for (int k = 0; k < nc; ++k) {
            int best = -1;
            for (int j = 0; j < nc; ++j)
                if (!used[j] && (best < 0 || A[j][j].x > A[best][best].x)) best = j;
            used[best] = true;
            order[k] = best;
            if (eig) eig[k] = A[best][best].x;
        }
    }
    __syncthreads();
    // phase normalisation and output: column k of U = column order[k] of V
    if (tid < nc) {
        const int j = order[tid];
        int a = 0;
        double best = -1.0;
        for (int r = 0; r < nc; ++r) {
            const double v = V[r][j].x * V[r][j].x + V[r][j].y * V[r][j].y;
            if (v > best) {
                best = v;
                a = r;
            }
        }
        const double mag = sqrt(best);
        const cd s = mag > 0.0 ? cd{V[a][j].x / mag, -V[a][j].y / mag} : cd{1.0, 0.0};
        for (int r = 0; r < nc; ++r) {
            const cd u = cmul(V[r][j], s);
            Uout[(size_t)tid * nc + r] = make_double2(u.x, u.y);
        }
    }
}

// out[k][i] = sum_a conj(U[k][a]) in[a][i] for k < nv (data: i = sample, maps: i = voxel)
__global__ void project_kernel(const float2 *__restrict__ in, int nc, size_t n, const double2 *__restrict__ U, int nv,
                               float2 *__restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= nv) return;
    double re = 0.0, im = 0.0;
    for (int a = 0; a < nc; ++a) {
        const double2 u = U[(size_t)k * nc + a];
        const float2 v = in[(size_t)a * n + i];
        re += u.x * v.x + u.y * v.y;   // conj(u) v
        im += u.x * v.y - u.y * v.x;
    }
    out[(size_t)k * n + i] = make_float2((float)re, (float)im);
}

}  // namespace

size_t coil_compress_bytes(int nc) {
    return align_up(sizeof(double2) * (size_t)nc * nc) * 2 + align_up(sizeof(double) * nc) + align_up(sizeof(int));
}

cudaError_t coil_compress(const float2 *y, const float2 *S, int nc, int nt, int nr, int nv, float2 *y_out,
                          float2 *S_out, double *eig_out, char *ws, cudaStream_t st, int max_sweeps) {
    double2 *C = (double2 *)ws;
    double2 *U = (double2 *)(ws + align_up(sizeof(double2) * (size_t)nc * nc));
    double *eig = (double *)(ws + 2 * align_up(sizeof(double2) * (size_t)nc * nc));
    int *status = (int *)(ws + 2 * align_up(sizeof(double2) * (size_t)nc * nc) + align_up(sizeof(double) * nc));
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    covariance_kernel<<<dim3(nc, nc), 256, 0, st>>>(y, nc, nt, C);
    jacobi_kernel<<<1, 256, 0, st>>>(C, nc, U, eig, max_sweeps, status);
    project_kernel<<<dim3(cdiv(nt, 256), nv), 256, 0, st>>>(y, nc, (size_t)nt, U, nv, y_out);
    project_kernel<<<dim3(cdiv(nr, 256), nv), 256, 0, st>>>(S, nc, (size_t)nr, U, nv, S_out);
    if (eig_out) e = cudaMemcpyAsync(eig_out, eig, sizeof(double) * nc, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace aexp
