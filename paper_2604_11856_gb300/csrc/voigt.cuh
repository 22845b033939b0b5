// The exact Voigt line shape (the optional profile of Sec. 2.2.1's full
// broadening): phi(dlam) = 1e3 Re w(z) / (sigma sqrt(2 pi)) um^-1 with
// z = (dlam + i lamL) / (sigma sqrt 2), sigma = lamG / sqrt(2 ln 2), w the
// Faddeeva function.  Re w is evaluated by region so that its relative
// accuracy holds where Re w is a small part of |w| (the far wings of
// Doppler-dominated lines, Re w ~ y / (sqrt(pi) x^2) against |w| ~ 1 / x):
//   |z|^2 >= R2     asymptotic series w ~ (i / sqrt pi) (1/z) sum_n c_n z^{-2n}
//                   (fewer terms at larger |z|),
//                   c_n = (2n - 1)!! / 2^n (Abramowitz & Stegun 7.1.23); the
//                   imaginary parts of 1/z and 1/z^2 carry y explicitly, so
//                   Re w keeps its relative accuracy;
//   y >= YT         Weideman's rational expansion (J. A. C. Weideman, SIAM J.
//                   Numer. Anal. 31, 1994): w = 2 p(Z) / (L - iz)^2 +
//                   pi^{-1/2} / (L - iz), Z = (L + iz) / (L - iz), p a
//                   polynomial whose coefficients are the Fourier
//                   coefficients of L^2 sec^2(t/2) e^{-L^2 tan^2(t/2)};
//   y < YT          Taylor series in y about the real axis, with w(x) =
//                   e^{-x^2} + i Im w(x) (the rational form at y = 0) and the
//                   derivatives from w' = -2 z w + 2i / sqrt(pi) (A&S 7.1.20).
// FP64: R2 = 64, 40 coefficients, 18 series terms, YT = 0.01, 10 Taylor
// terms; FP32: R2 = 36, 24, 8, 0.07, 8.  Against an independent Faddeeva
// implementation over x in [0, 500], y in [1e-5, 300] the largest relative
// error of Re w is 5e-13 (FP64) and 1.1e-5 (FP32).
#pragma once

#define RAPRAL_VOIGT_NW64 40
#define RAPRAL_VOIGT_NW32 24

struct VoigtCoef {
    double a64[RAPRAL_VOIGT_NW64];
    double L64;
    float a32[RAPRAL_VOIGT_NW32];
    float L32;
};

template <typename T>
struct VoigtRegion;
template <>
struct VoigtRegion<double> {
    static constexpr int NW = RAPRAL_VOIGT_NW64, NA = 18, KT = 10;
    static constexpr double R2 = 64.0, YT = 0.01;
};
template <>
struct VoigtRegion<float> {
    static constexpr int NW = RAPRAL_VOIGT_NW32, NA = 8, KT = 8;
    static constexpr float R2 = 36.0f, YT = 0.07f;
};

__device__ __forceinline__ double vcoef(const VoigtCoef& v, int n, double) { return v.a64[n]; }
__device__ __forceinline__ float vcoef(const VoigtCoef& v, int n, float) { return v.a32[n]; }
__device__ __forceinline__ double vL(const VoigtCoef& v, double) { return v.L64; }
__device__ __forceinline__ float vL(const VoigtCoef& v, float) { return v.L32; }
__device__ __forceinline__ double vexp(double x) { return exp(x); }
__device__ __forceinline__ float vexp(float x) { return expf(x); }
__device__ __forceinline__ double vrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float vrcp(float x) { return 1.0f / x; }

// c_{NA-1} of the asymptotic series, (2n - 1)!! / 2^n at n = NA - 1
template <typename T>
__host__ __device__ constexpr T voigt_ctop(int na) {
    T c = T(1);
    for (int n = 1; n < na; ++n) c = c * T(2 * n - 1) / T(2);
    return c;
}

template <typename T, int NA>
__device__ __forceinline__ T voigt_asym(T x, T y) {
    const T ir = vrcp(x * x + y * y);
    const T zr = x * ir, zi = -y * ir;                     // 1/z
    const T ur = zr * zr - zi * zi, ui = T(2) * zr * zi;   // 1/z^2
    constexpr T ctop = voigt_ctop<T>(NA);
    T sr = ctop, si = T(0), cn = ctop;
#pragma unroll
    for (int n = NA - 1; n >= 1; --n) {
        cn = cn * T(2) / T(2 * n - 1);                     // c_{n-1}
        const T tr = sr * ur - si * ui + cn;
        si = sr * ui + si * ur;
        sr = tr;
    }
    // Re w = -Im((1/z) S) / sqrt(pi)
    return -(zr * si + zi * sr) * T(0.56418958354775628695);
}

// w(x + iy) by the rational expansion: (Re, Im)
template <typename T>
__device__ __forceinline__ void voigt_weid(const VoigtCoef& v, T x, T y, T& wr, T& wi) {
    constexpr int NW = VoigtRegion<T>::NW;
    const T L = vL(v, T());
    const T Ly = L + y;
    const T iD = vrcp(Ly * Ly + x * x);
    const T Zr = (L * L - x * x - y * y) * iD, Zi = T(2) * L * x * iD;
    T pr = vcoef(v, NW - 1, T()), pi = T(0);
#pragma unroll 4
    for (int n = NW - 2; n >= 0; --n) {
        const T tr = pr * Zr - pi * Zi + vcoef(v, n, T());
        pi = pr * Zi + pi * Zr;
        pr = tr;
    }
    const T qr = Ly * iD, qi = x * iD;                     // 1 / (L - iz)
    const T q2r = qr * qr - qi * qi, q2i = T(2) * qr * qi;
    const T s = T(0.56418958354775628695);
    wr = T(2) * (pr * q2r - pi * q2i) + qr * s;
    wi = T(2) * (pr * q2i + pi * q2r) + qi * s;
}

template <typename T>
__device__ __forceinline__ T voigt_taylor(const VoigtCoef& v, T x, T y) {
    constexpr int KT = VoigtRegion<T>::KT;
    T w0r, w0i;
    voigt_weid(v, x, T(0), w0r, w0i);
    w0r = vexp(-x * x);                                    // Re w on the real axis, exactly
    T ar = w0r, ai = w0i;                                  // w^(k-1)
    T br = T(-2) * x * w0r, bi = T(-2) * x * w0i + T(1.12837916709551257390);   // w^(k)
    T tot = w0r, f = T(1);
#pragma unroll
    for (int k = 1; k <= KT; ++k) {
        f = f * y / T(k);
        const T re = (k & 3) == 0 ? br : (k & 3) == 1 ? -bi : (k & 3) == 2 ? -br : bi;   // Re(i^k w^(k))
        tot = tot + re * f;
        const T nr = T(-2) * x * br - T(2 * k) * ar, ni = T(-2) * x * bi - T(2 * k) * ai;
        ar = br; ai = bi;
        br = nr; bi = ni;
    }
    return tot;
}

// Re w(x + iy), y >= 0.  The asymptotic series takes fewer terms farther
// out: its first omitted term, (2n + 1) c_n / |z|^{2n} relative to Re w, stays
// below 1e-15 (FP64) and 1e-7 (FP32) in every tier.
__device__ __forceinline__ double voigt_asym_tiers(double x, double y, double r2) {
    if (r2 >= 400.0) return voigt_asym<double, 8>(x, y);
    return voigt_asym<double, VoigtRegion<double>::NA>(x, y);
}
__device__ __forceinline__ float voigt_asym_tiers(float x, float y, float r2) {
    if (r2 >= 1000.0f) return voigt_asym<float, 3>(x, y);
    if (r2 >= 100.0f) return voigt_asym<float, 5>(x, y);
    return voigt_asym<float, VoigtRegion<float>::NA>(x, y);
}

// Re w(x + iy), y >= 0
template <typename T>
__device__ __forceinline__ T voigt_re(const VoigtCoef& v, T x, T y) {
    x = fabs(x);
    const T r2 = x * x + y * y;
    if (r2 >= VoigtRegion<T>::R2) return voigt_asym_tiers(x, y, r2);
    if (y >= VoigtRegion<T>::YT) {
        T wr, wi;
        voigt_weid(v, x, y, wr, wi);
        return wr;
    }
    return voigt_taylor(v, x, y);
}
