/*
 * FP64 direct-sum oracle for the expanded encoding operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the timed CPU baseline of the bench use
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Model (Sec. 1 and Eq. 1: the encoding includes the B0 map and the
 * spherical-harmonic field terms monitored to 2nd/3rd order; Sec. 2.2.2 uses
 * y = A_exp x as the forward model):
 *
 *   phi(t, r)   = sum_l k_l(t) h_l(r) + omega(r) t
 *   E(t, r)     = exp(-i phi(t, r))
 *   (A x)_c(t)  = sum_r E(t, r) S_c(r) x(r)
 *   (A^H y)(r)  = sum_c conj(S_c(r)) sum_t conj(E(t, r)) y_c(t)
 *
 * The adjoint is the A^T of Sec. 2.1 (W A^T y) for complex data.
 *
 * Layouts: k[l*nt + t], h[l*nr + r], omega[r], tt[t], S[c*nr + r],
 * x[r], y[c*nt + t]; complex arrays are C99 double complex (re, im pairs).
 * Plain loops, no blocking, no reordering beyond the sums' definition.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>

static double phase(int nl, int nt, int nr, const double *k, const double *h,
                    const double *omega, const double *tt, int t, int r)
{
    double phi = 0.0;
    for (int l = 0; l < nl; ++l)
        phi += k[(size_t)l * nt + t] * h[(size_t)l * nr + r];
    if (omega)
        phi += omega[r] * tt[t];
    return phi;
}

/* y = A x.  Parallel over samples t; each y_c(t) is one plain sum over r. */
void oracle_forward(int nt, int nr, int nc, int nl, const double *k, const double *h,
                    const double *omega, const double *tt, const double complex *S,
                    const double complex *x, double complex *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t) {
        double complex acc[nc]; /* thread-local sums, stored once per sample */
        for (int c = 0; c < nc; ++c)
            acc[c] = 0.0;
        for (int r = 0; r < nr; ++r) {
            double phi = phase(nl, nt, nr, k, h, omega, tt, t, r);
            double complex e = cos(phi) - I * sin(phi);
            for (int c = 0; c < nc; ++c)
                acc[c] += e * S[(size_t)c * nr + r] * x[r];
        }
        for (int c = 0; c < nc; ++c)
            y[(size_t)c * nt + t] = acc[c];
    }
}

/* x = A^H y.  Parallel over voxels r. */
void oracle_adjoint(int nt, int nr, int nc, int nl, const double *k, const double *h,
                    const double *omega, const double *tt, const double complex *S,
                    const double complex *y, double complex *x)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < nr; ++r) {
        double complex acc = 0.0;
        for (int t = 0; t < nt; ++t) {
            double phi = phase(nl, nt, nr, k, h, omega, tt, t, r);
            double complex ec = cos(phi) + I * sin(phi); /* conj(E) */
            for (int c = 0; c < nc; ++c)
                acc += conj(S[(size_t)c * nr + r]) * ec * y[(size_t)c * nt + t];
        }
        x[r] = acc;
    }
}

/* Selected rows of A x: y_c(t) for the listed sample indices only
 * (used to check large problems one output at a time). y[c*ns + j]. */
void oracle_forward_rows(int nt, int nr, int nc, int nl, const double *k, const double *h,
                         const double *omega, const double *tt, const double complex *S,
                         const double complex *x, int ns, const int *ts, double complex *y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < ns; ++j) {
        int t = ts[j];
        double complex acc[nc];
        for (int c = 0; c < nc; ++c)
            acc[c] = 0.0;
        for (int r = 0; r < nr; ++r) {
            double phi = phase(nl, nt, nr, k, h, omega, tt, t, r);
            double complex e = cos(phi) - I * sin(phi);
            for (int c = 0; c < nc; ++c)
                acc[c] += e * S[(size_t)c * nr + r] * x[r];
        }
        for (int c = 0; c < nc; ++c)
            y[(size_t)c * ns + j] = acc[c];
    }
}

/* Selected entries of A^H y: x(r) for the listed voxels only. */
void oracle_adjoint_rows(int nt, int nr, int nc, int nl, const double *k, const double *h,
                         const double *omega, const double *tt, const double complex *S,
                         const double complex *y, int ns, const int *rs, double complex *x)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < ns; ++j) {
        int r = rs[j];
        double complex acc = 0.0;
        for (int t = 0; t < nt; ++t) {
            double phi = phase(nl, nt, nr, k, h, omega, tt, t, r);
            double complex ec = cos(phi) + I * sin(phi);
            for (int c = 0; c < nc; ++c)
                acc += conj(S[(size_t)c * nr + r]) * ec * y[(size_t)c * nt + t];
        }
        x[j] = acc;
    }
}

/*
 * Derivatives with respect to the field coefficients, for the gradient of
 * a real loss through y = A x and through x~ = A^H y.
 *
 * Forward:  d y_c(t) / d k_l(t) = sum_r (-i h_l(r)) E(t,r) S_c(r) x(r).
 * For a real loss with cotangent g = dLoss/dRe(y) + i dLoss/dIm(y), the
 * derivative with respect to a real parameter p is Re sum conj(g) dy/dp.
 * This returns G_l(t) = sum_c conj(g_c(t)) dy_c(t)/dk_l(t); the caller takes Re.
 */
void oracle_forward_dk(int nt, int nr, int nc, int nl, const double *k, const double *h,
                       const double *omega, const double *tt, const double complex *S,
                       const double complex *x, const double complex *g, double complex *G)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t) {
        double complex acc[nl > 0 ? nl : 1];
        for (int l = 0; l < nl; ++l)
            acc[l] = 0.0;
        for (int r = 0; r < nr; ++r) {
            double phi = phase(nl, nt, nr, k, h, omega, tt, t, r);
            double complex e = cos(phi) - I * sin(phi);
            double complex s = 0.0;
            for (int c = 0; c < nc; ++c)
                s += conj(g[(size_t)c * nt + t]) * S[(size_t)c * nr + r];
            double complex term = s * e * x[r] * (-I);
            for (int l = 0; l < nl; ++l)
                acc[l] += term * h[(size_t)l * nr + r];
        }
        for (int l = 0; l < nl; ++l)
            G[(size_t)l * nt + t] = acc[l];
    }
}

/* Adjoint:  d x~(r) / d k_l(t) = conj(S_c(r)) (+i h_l(r)) conj(E(t,r)) y_c(t) summed over c.
 * Returns G_l(t) = sum_r conj(g(r)) * d x~(r) / d k_l(t) for a cotangent g(r). */
void oracle_adjoint_dk(int nt, int nr, int nc, int nl, const double *k, const double *h,
                       const double *omega, const double *tt, const double complex *S,
                       const double complex *y, const double complex *g, double complex *G)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t) {
        double complex acc[nl > 0 ? nl : 1];
        for (int l = 0; l < nl; ++l)
            acc[l] = 0.0;
        for (int r = 0; r < nr; ++r) {
            double phi = phase(nl, nt, nr, k, h, omega, tt, t, r);
            double complex ec = cos(phi) + I * sin(phi);
            double complex s = 0.0;
            for (int c = 0; c < nc; ++c)
                s += conj(S[(size_t)c * nr + r]) * y[(size_t)c * nt + t];
            double complex term = conj(g[r]) * s * ec * I;
            for (int l = 0; l < nl; ++l)
                acc[l] += term * h[(size_t)l * nr + r];
        }
        for (int l = 0; l < nl; ++l)
            G[(size_t)l * nt + t] = acc[l];
    }
}
