// Register-resident 48-point DFT, X[k] = sum_n x[n] exp(+2 pi i n k / 48), as
// 8 x 6: with n = 6 n1 + n2 and k = k1 + 8 k2,
//   X[k1 + 8 k2] = sum_n2 w6^{n2 k2} [ w48^{n2 k1} sum_n1 x[6 n1 + n2] w8^{n1 k1} ],
// eight-point transforms over n1 (packed FP32 pairs), the w48 twiddles, then
// six-point transforms over n2.  The transform of the 48 x 48 folded grids of
// grid side 96 (two pixel classes per axis).
#pragma once

#include "fft64.cuh"

namespace epic {

// exp(+2 pi i j / 48) with exact reduction on the integer j: quadrant q = j / 12,
// r = j mod 12 steps of pi / 24 inside it, r <= 6 is at most pi / 4
constexpr float2 ce_w48(int j)
{
    j = ((j % 48) + 48) % 48;
    const int q = j / 12, r = j % 12;
    constexpr double step = 3.14159265358979323846 / 24.0;
    double c = 0, s = 0;
    if (r <= 6) {
        c = ce_cos_q(r * step);
        s = ce_sin_q(r * step);
    } else {
        c = ce_sin_q((12 - r) * step);
        s = ce_cos_q((12 - r) * step);
    }
    double re = c, im = s;
    for (int i = 0; i < q; i++) {
        const double t = re;
        re = -im;
        im = t;
    }
    return float2{static_cast<float>(re), static_cast<float>(im)};
}

// The twiddles as lane pairs for the packed form: (re, re) and (-im, im).
struct Twiddle48p {
    float2 rr[48], ni[48];
};
constexpr Twiddle48p make_twiddle48p()
{
    Twiddle48p t{};
    for (int j = 0; j < 48; j++) {
        const float2 w = ce_w48(j);
        t.rr[j] = float2{w.x, w.x};
        t.ni[j] = float2{-w.y, w.y};
    }
    return t;
}
__constant__ const Twiddle48p c_tw48p = make_twiddle48p();

// Three points on packed pairs: X0 = x0 + s, X1,2 = x0 - s/2 +- i sin60 (x1 - x2).
__device__ __forceinline__ void dft3p(float2 &x0, float2 &x1, float2 &x2)
{
    const float2 s = padd(x1, x2), d = pswap(psub(x1, x2));
    const float2 m = pfma(s, make_float2(-0.5f, -0.5f), x0);
    x0 = padd(x0, s);
    x1 = pfma(d, make_float2(-kSin60, kSin60), m);
    x2 = pfma(d, make_float2(kSin60, -kSin60), m);
}

// Six points as 2 x 3 with coprime factors (Good-Thomas index map: input n = 3 n1 + 2 n2
// mod 6, output k with k mod 2 = k1 and k mod 3 = k2), so no twiddles between the
// three-point and the two-point transforms.
__device__ __forceinline__ void dft6p(float2 *x)
{
    float2 a0 = x[0], a1 = x[2], a2 = x[4];   // n1 = 0: n2 = 0, 1, 2
    float2 b0 = x[3], b1 = x[5], b2 = x[1];   // n1 = 1
    dft3p(a0, a1, a2);
    dft3p(b0, b1, b2);
    x[0] = padd(a0, b0);   // (k1, k2) = (0, 0)
    x[3] = psub(a0, b0);   // (1, 0)
    x[4] = padd(a1, b1);   // (0, 1)
    x[1] = psub(a1, b1);   // (1, 1)
    x[2] = padd(a2, b2);   // (0, 2)
    x[5] = psub(a2, b2);   // (1, 2)
}

// Stage 1 in place: for each n2, DFT8 over x[n2 + 6 n1], then twiddle by w48^{n2 k1}
// (a w = a.x (w.x, w.x) + (a.y, a.x) (-w.y, w.y)); result k1 at x[n2 + 6 k1].
__device__ __forceinline__ void fft48p_stage1(float2 (&x)[48])
{
#pragma unroll
    for (int n2 = 0; n2 < 6; n2++) {
        float2 t[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; n1++) t[n1] = x[n2 + 6 * n1];
        dft8p(t);
        x[n2] = t[0];
#pragma unroll
        for (int k1 = 1; k1 < 8; k1++)
            x[n2 + 6 * k1] = n2 == 0 ? t[k1]
                                     : pfma(pswap(t[k1]), c_tw48p.ni[n2 * k1], pmul(t[k1], c_tw48p.rr[n2 * k1]));
    }
}

// Stage 2: for each k1, DFT6 over x[6 k1 + n2]; X[k1 + 8 k2] is handed to sink(k, value).
template <class Sink>
__device__ __forceinline__ void fft48p_stage2(float2 (&x)[48], Sink &&sink)
{
#pragma unroll
    for (int k1 = 0; k1 < 8; k1++) {
        float2 u[6];
#pragma unroll
        for (int n2 = 0; n2 < 6; n2++) u[n2] = x[6 * k1 + n2];
        dft6p(u);
#pragma unroll
        for (int k2 = 0; k2 < 6; k2++) sink(k1 + 8 * k2, u[k2]);
    }
}

}  // namespace epic
