// Register-resident 64-point DFT, X[k] = sum_n x[n] exp(+2 pi i n k / 64),
// as 8 x 8 (two radix-8 stages with twiddles in between).  The twiddles are
// computed at compile time from their Taylor series and live in constant
// memory, so the compiler can use them as constant-bank operands.
#pragma once

#include "dft_small.cuh"

namespace epic {

struct Twiddle64 {
    float2 w[64];
};

// sin and cos on [0, pi/4] by their Taylor series (double precision)
constexpr double ce_sin_q(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 14; k++) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double ce_cos_q(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; k++) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// exp(+2 pi i j / 64) with exact octant reduction on the integer j
constexpr float2 ce_w64(int j)
{
    j &= 63;
    const int q = j / 16, r = j % 16;          // quadrant, index within it
    constexpr double step = 3.14159265358979323846 / 32.0;
    double c = 0, s = 0;
    if (r <= 8) {
        c = ce_cos_q(r * step);
        s = ce_sin_q(r * step);
    } else {
        c = ce_sin_q((16 - r) * step);
        s = ce_cos_q((16 - r) * step);
    }
    double re = c, im = s;                     // rotate by q quarter turns
    for (int i = 0; i < q; i++) {
        const double t = re;
        re = -im;
        im = t;
    }
    return float2{static_cast<float>(re), static_cast<float>(im)};
}

constexpr Twiddle64 make_twiddle64()
{
    Twiddle64 t{};
    for (int j = 0; j < 64; j++) t.w[j] = ce_w64(j);
    return t;
}

__constant__ const Twiddle64 c_tw64 = make_twiddle64();

// The same twiddles as lane pairs for the packed form: (re, re) and (-im, im).
struct Twiddle64p {
    float2 rr[64], ni[64];
};
constexpr Twiddle64p make_twiddle64p()
{
    Twiddle64p t{};
    for (int j = 0; j < 64; j++) {
        const float2 w = ce_w64(j);
        t.rr[j] = float2{w.x, w.x};
        t.ni[j] = float2{-w.y, w.y};
    }
    return t;
}
__constant__ const Twiddle64p c_tw64p = make_twiddle64p();

// Stage 1 in place: for each n2, DFT8 over x[n2 + 8 n1] and twiddle by w64^{n2 k1}.
__device__ __forceinline__ void fft64_stage1(float2 (&x)[64])
{
#pragma unroll
    for (int n2 = 0; n2 < 8; n2++) {
        float2 t[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; n1++) t[n1] = x[n2 + 8 * n1];
        dft8(t);
        x[n2] = t[0];
#pragma unroll
        for (int k1 = 1; k1 < 8; k1++) x[n2 + 8 * k1] = n2 == 0 ? t[k1] : cmul(t[k1], c_tw64.w[n2 * k1]);
    }
}

// Stage 2: for each k1, DFT8 over x[n2 + 8 k1]; X[k1 + 8 k2] is handed to sink(k, value).
template <class Sink>
__device__ __forceinline__ void fft64_stage2(float2 (&x)[64], Sink &&sink)
{
#pragma unroll
    for (int k1 = 0; k1 < 8; k1++) {
        float2 t[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; n2++) t[n2] = x[n2 + 8 * k1];
        dft8(t);
#pragma unroll
        for (int k2 = 0; k2 < 8; k2++) sink(k1 + 8 * k2, t[k2]);
    }
}

// The two stages in packed pairs (dft8p; twiddle a w = a.x (w.x, w.x) +
// (a.y, a.x) (-w.y, w.y), one multiply and one FMA per pair).
__device__ __forceinline__ void fft64p_stage1(float2 (&x)[64])
{
#pragma unroll
    for (int n2 = 0; n2 < 8; n2++) {
        float2 t[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; n1++) t[n1] = x[n2 + 8 * n1];
        dft8p(t);
        x[n2] = t[0];
#pragma unroll
        for (int k1 = 1; k1 < 8; k1++)
            x[n2 + 8 * k1] = n2 == 0 ? t[k1]
                                     : pfma(pswap(t[k1]), c_tw64p.ni[n2 * k1], pmul(t[k1], c_tw64p.rr[n2 * k1]));
    }
}

template <class Sink>
__device__ __forceinline__ void fft64p_stage2(float2 (&x)[64], Sink &&sink)
{
#pragma unroll
    for (int k1 = 0; k1 < 8; k1++) {
        float2 t[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; n2++) t[n2] = x[n2 + 8 * k1];
        dft8p(t);
#pragma unroll
        for (int k2 = 0; k2 < 8; k2++) sink(k1 + 8 * k2, t[k2]);
    }
}

}  // namespace epic
