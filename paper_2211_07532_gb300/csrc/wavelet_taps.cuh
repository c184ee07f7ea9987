// Wavelet filter taps shared by the decimated (wavelet.cu) and undecimated (swt.cu)
// transforms: internal linkage, each translation unit keeps its own constant copy.
#pragma once

namespace aexp {
namespace {

// Haar and Daubechies (4 vanishing moments) lowpass taps; the latter as tabulated by
// Daubechies (Comm. Pure Appl. Math. 41, 1988, Table 1, N = 4).  Each tap is carried as an
// FP32 pair hi + lo (hi the FP32 rounding, lo the rounding of the remainder), so that the
// filters the kernels apply are orthonormal to ~2^-48 instead of to the ~2^-25 of FP32 taps:
// with plain FP32 taps W^H W misses the identity by ~1e-7, a bias that a 100-iteration solve
// compounds to ~1e-5 of the image, while the FP32 rounding of the sums stays unbiased.
#define AEXP_TAP(v) (float)(v), (float)((v) - (double)(float)(v))
__constant__ float c_haar[2][2] = {{AEXP_TAP(0.70710678118654752440)}, {AEXP_TAP(0.70710678118654752440)}};
__constant__ float c_db4[8][2] = {{AEXP_TAP(0.23037781330889650086)},  {AEXP_TAP(0.71484657055291564709)},
                                  {AEXP_TAP(0.63088076792985890788)},  {AEXP_TAP(-0.02798376941685985421)},
                                  {AEXP_TAP(-0.18703481171909308408)}, {AEXP_TAP(0.03084138183556076363)},
                                  {AEXP_TAP(0.03288301166688519974)},  {AEXP_TAP(-0.01059740178506903210)}};
#undef AEXP_TAP

struct Tap {
    float hi, lo;
};

// lowpass h[m]; highpass g[m] = (-1)^m h[TAPS - 1 - m]
template <int TAPS>
__device__ __forceinline__ Tap tap_h(int m) {
    return TAPS == 2 ? Tap{c_haar[m][0], c_haar[m][1]} : Tap{c_db4[m][0], c_db4[m][1]};
}
template <int TAPS>
__device__ __forceinline__ Tap tap_g(int m) {
    Tap v = tap_h<TAPS>(TAPS - 1 - m);
    return (m & 1) ? Tap{-v.hi, -v.lo} : v;
}

// acc + t v with the tap's both parts (two FMAs; the small part first)
__device__ __forceinline__ float tfma(Tap t, float v, float acc) { return fmaf(t.hi, v, fmaf(t.lo, v, acc)); }
__device__ __forceinline__ float2 tmad(Tap t, float2 v, float2 acc) {
    return make_float2(tfma(t, v.x, acc.x), tfma(t, v.y, acc.y));
}

__device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

}  // namespace
}  // namespace aexp
