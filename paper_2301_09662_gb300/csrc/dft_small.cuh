// Small in-register DFTs, X[k] = sum_n x[n] exp(+2 pi i n k / R), used as the
// radices of the shared-memory FFT passes (the +i sign of Eq. 4's FT^-1).
#pragma once

#include <cuda_runtime.h>

namespace epic {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * i
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }

// exp(+2 pi i f_c tau): the geometric-delay correction of one antenna at one
// channel (Sec. 2.2, delay-correction block).  d = (frac(f_ref tau), tau_hi,
// tau_lo) from the per-integration delay table (FP64 work done once per
// (t, antenna)); df = f_c - f_ref.  The turns are b + df tau with df tau_hi
// split exactly (two-product) so that whole turns drop out before rounding.
__device__ __forceinline__ float2 delay_phase(float4 d, float df)
{
    const float p = df * d.y;
    const float e = fmaf(df, d.y, -p);
    const float turns = (d.x + (p - rintf(p))) + fmaf(df, d.z, e);
    float s, c;
    sincospif(2.0f * turns, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

constexpr float kSqrtHalf = 0.70710678118654752440f;
constexpr float kSin60 = 0.86602540378443864676f;

__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2 *x)
{
    const float2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    const float2 s13 = cadd(x[1], x[3]), d13 = cmul_i(csub(x[1], x[3]));
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, d13);
    x[3] = csub(d02, d13);
}

__device__ __forceinline__ void dft8(float2 *x)
{
    float2 e[4] = {x[0], x[2], x[4], x[6]};
    float2 o[4] = {x[1], x[3], x[5], x[7]};
    dft4(e);
    dft4(o);
    // twiddles w8^k = exp(+2 pi i k / 8)
    const float2 o1 = make_float2(kSqrtHalf * (o[1].x - o[1].y), kSqrtHalf * (o[1].x + o[1].y));
    const float2 o2 = cmul_i(o[2]);
    const float2 o3 = make_float2(-kSqrtHalf * (o[3].x + o[3].y), kSqrtHalf * (o[3].x - o[3].y));
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);
    x[7] = csub(e[3], o3);
}

__device__ __forceinline__ void dft3(float2 *x)
{
    const float2 s = cadd(x[1], x[2]);
    const float2 d = cmul_i(cscale(csub(x[1], x[2]), kSin60));
    const float2 m = make_float2(x[0].x - 0.5f * s.x, x[0].y - 0.5f * s.y);
    x[0] = cadd(x[0], s);
    x[1] = cadd(m, d);
    x[2] = csub(m, d);
}

__device__ __forceinline__ void dft6(float2 *x)
{
    float2 e[3] = {x[0], x[2], x[4]};
    float2 o[3] = {x[1], x[3], x[5]};
    dft3(e);
    dft3(o);
    // w6 = exp(+i pi/3) = 1/2 + i sqrt(3)/2, w6^2 = -1/2 + i sqrt(3)/2
    const float2 o1 = cmul(o[1], make_float2(0.5f, kSin60));
    const float2 o2 = cmul(o[2], make_float2(-0.5f, kSin60));
    x[0] = cadd(e[0], o[0]);
    x[3] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[4] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[5] = csub(e[2], o2);
}

template <int R>
__device__ __forceinline__ void dft(float2 *x)
{
    if constexpr (R == 2) dft2(x[0], x[1]);
    else if constexpr (R == 3) dft3(x);
    else if constexpr (R == 4) dft4(x);
    else if constexpr (R == 6) dft6(x);
    else if constexpr (R == 8) dft8(x);
    else static_assert(R == 2, "unsupported radix");
}

}  // namespace epic
