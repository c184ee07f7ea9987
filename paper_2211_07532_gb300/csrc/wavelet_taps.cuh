// Wavelet filter taps shared by the decimated (wavelet.cu) and undecimated (swt.cu)
// transforms: internal linkage, each translation unit keeps its own constant copy.
#pragma once

namespace aexp {
namespace {

// Haar and Daubechies (4 vanishing moments) lowpass taps; the latter as tabulated by
// Daubechies (Comm. Pure Appl. Math. 41, 1988, Table 1, N = 4).
__constant__ float c_haar[2] = {0.70710678118654752440f, 0.70710678118654752440f};
__constant__ float c_db4[8] = {0.23037781330889650086f,  0.71484657055291564709f,  0.63088076792985890788f,
                               -0.02798376941685985421f, -0.18703481171909308408f, 0.03084138183556076363f,
                               0.03288301166688519974f,  -0.01059740178506903210f};

// lowpass h[m]; highpass g[m] = (-1)^m h[TAPS - 1 - m]
template <int TAPS>
__device__ __forceinline__ float tap_h(int m) {
    return TAPS == 2 ? c_haar[m] : c_db4[m];
}
template <int TAPS>
__device__ __forceinline__ float tap_g(int m) {
    float v = tap_h<TAPS>(TAPS - 1 - m);
    return (m & 1) ? -v : v;
}

__device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

}  // namespace
}  // namespace aexp
