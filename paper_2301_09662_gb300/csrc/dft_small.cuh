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

// Packed FP32 pairs: one instruction performs the operation on both lanes of a
// float2 (each an IEEE round-to-nearest operation, the same result as the
// scalar one).  The float2 halves already sit in a register pair, so packing
// costs no moves; pswap (a lane exchange) does.
__device__ __forceinline__ unsigned long long p_pack(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 p_unpack(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(p_pack(a)), "l"(p_pack(b)));
    return p_unpack(r);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(p_pack(a)), "l"(p_pack(b)));
    return p_unpack(r);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(p_pack(a)), "l"(p_pack(b)));
    return p_unpack(r);
}
// lane-wise a * b + c, one rounding per lane
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(p_pack(a)), "l"(p_pack(b)), "l"(p_pack(c)));
    return p_unpack(r);
}
__device__ __forceinline__ float2 pswap(float2 a) { return make_float2(a.y, a.x); }

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

// dft4 and dft8 in packed pairs.  Multiplying by +-i is a lane exchange and an
// FMA with a (-1, +1) or (+1, -1) pair, exact like the scalar add it replaces;
// the w8 twiddles fold sqrt(1/2) into the final FMA (one rounding fewer than
// the scalar form).
__device__ __forceinline__ void dft4p(float2 *x)
{
    const float2 NP = make_float2(-1.f, 1.f), PN = make_float2(1.f, -1.f);
    const float2 s02 = padd(x[0], x[2]), d02 = psub(x[0], x[2]);
    const float2 s13 = padd(x[1], x[3]), u = pswap(psub(x[1], x[3]));
    x[0] = padd(s02, s13);
    x[2] = psub(s02, s13);
    x[1] = pfma(u, NP, d02);          // d02 + i (x1 - x3)
    x[3] = pfma(u, PN, d02);          // d02 - i (x1 - x3)
}

__device__ __forceinline__ void dft8p(float2 *x)
{
    const float2 NP = make_float2(-1.f, 1.f), PN = make_float2(1.f, -1.f);
    const float2 H = make_float2(kSqrtHalf, kSqrtHalf), NH = make_float2(-kSqrtHalf, -kSqrtHalf);
    float2 e[4] = {x[0], x[2], x[4], x[6]};
    float2 o[4] = {x[1], x[3], x[5], x[7]};
    dft4p(e);
    dft4p(o);
    const float2 v1 = pfma(pswap(o[1]), NP, o[1]);   // (o.x - o.y, o.y + o.x) = w8 o / sqrt(1/2)
    const float2 u2 = pswap(o[2]);                   // i o = (-o.y, o.x) via NP
    const float2 v3 = pfma(pswap(o[3]), PN, o[3]);   // (o.x + o.y, o.y - o.x) = -w8^3 o / sqrt(1/2)
    x[0] = padd(e[0], o[0]);
    x[4] = psub(e[0], o[0]);
    x[1] = pfma(v1, H, e[1]);
    x[5] = pfma(v1, NH, e[1]);
    x[2] = pfma(u2, NP, e[2]);
    x[6] = pfma(u2, PN, e[2]);
    x[3] = pfma(v3, NH, e[3]);
    x[7] = pfma(v3, H, e[3]);
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
