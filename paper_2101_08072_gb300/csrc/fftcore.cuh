// Device helpers of the FP32 plane transforms (colfft.cu, planefft.cu): complex arithmetic on pairs of
// complex values held as float4 (two columns, or two rows, transformed together), register DFTs of radix
// 2, 4, 8 and 16, and the twiddles of the mixed-radix Stockham stages.  The formulation follows
// Govindaraju et al., "High performance discrete Fourier transforms on graphics processors" (SC 2008):
// stage s with radix R and Ns = product of the earlier radices takes, for butterfly j < N/R, the inputs
// x[j + r N/R] (r < R), multiplies input r by exp(-/+ 2 pi i r (j mod Ns) / (Ns R)), applies an R-point
// DFT and writes output r to y[(j div Ns) Ns R + (j mod Ns) + r Ns].  The R-point DFTs run in registers:
// 16 = 4 x 4 and 8 = 4 x 2 by the Cooley-Tukey split n = R2 n1 + n2, k = k1 + R1 k2 with the twiddles
// exp(-/+ 2 pi i n2 k1 / R) in between.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pfb {
namespace fft {

// Element types: float4 holds two complex values (two columns, or two rows, transformed together), float2
// one.  The arithmetic below is overloaded on both.
__device__ __forceinline__ float4 c_add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float4 c_sub(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float4 c_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float2 c_neg(float2 a) { return make_float2(-a.x, -a.y); }
// the complex value(s) of a times w
__device__ __forceinline__ float4 c_mul(float4 a, float2 w) {
    return make_float4(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x, a.z * w.x - a.w * w.y, a.z * w.y + a.w * w.x);
}
__device__ __forceinline__ float2 c_mul(float2 a, float2 w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// times -i (forward sign) or +i (inverse sign)
template <bool INV> __device__ __forceinline__ float4 c_rot(float4 a) {
    return INV ? make_float4(-a.y, a.x, -a.w, a.z) : make_float4(a.y, -a.x, a.w, -a.z);
}
template <bool INV> __device__ __forceinline__ float2 c_rot(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi e / 16), from cos(pi/8), sin(pi/8) and sqrt(1/2); sin(2 pi e / 16) = cos16(e - 4)
constexpr double kC8 = 0.92387953251128675613, kS8 = 0.38268343236508977173, kR2 = 0.70710678118654752440;
__host__ __device__ constexpr double cos16(int e) {
    return (e & 15) == 0 ? 1.0 : (e & 15) == 1 ? kC8 : (e & 15) == 2 ? kR2 : (e & 15) == 3 ? kS8
         : (e & 15) == 4 ? 0.0 : (e & 15) == 5 ? -kS8 : (e & 15) == 6 ? -kR2 : (e & 15) == 7 ? -kC8
         : (e & 15) == 8 ? -1.0 : (e & 15) == 9 ? -kC8 : (e & 15) == 10 ? -kR2 : (e & 15) == 11 ? -kS8
         : (e & 15) == 12 ? 0.0 : (e & 15) == 13 ? kS8 : (e & 15) == 14 ? kR2 : kC8;
}

// a times exp(-/+ 2 pi i e / R), R in {8, 16}; e is a compile-time constant once the loops unroll
template <int R, bool INV, typename E> __device__ __forceinline__ E c_tw(E a, int e) {
    const int f = (e * (16 / R)) & 15;
    if (f == 0) return a;
    if (f == 8) return c_neg(a);
    if (f == 4) return c_rot<INV>(a);
    if (f == 12) return c_rot<!INV>(a);
    const float c = (float)cos16(f), s = (float)cos16(f - 4);
    return c_mul(a, make_float2(c, INV ? s : -s));
}

template <bool INV, typename E> __device__ __forceinline__ void dft2(E &x0, E &x1) {
    const E a = c_add(x0, x1);
    x1 = c_sub(x0, x1);
    x0 = a;
}
template <bool INV, typename E> __device__ __forceinline__ void dft4(E &x0, E &x1, E &x2, E &x3) {
    const E a0 = c_add(x0, x2), a1 = c_sub(x0, x2), a2 = c_add(x1, x3), a3 = c_rot<INV>(c_sub(x1, x3));
    x0 = c_add(a0, a2);
    x1 = c_add(a1, a3);
    x2 = c_sub(a0, a2);
    x3 = c_sub(a1, a3);
}

// R-point DFT of x[0..R) in registers; output k ends up in x[operm<R>(k)]
template <int R> __device__ __forceinline__ constexpr int operm(int k) {
    return R == 16 ? 4 * (k & 3) + (k >> 2) : R == 8 ? 2 * (k & 3) + (k >> 2) : k;
}
template <int R, bool INV, typename E> __device__ __forceinline__ void dft_reg(E *x) {
    if constexpr (R == 2) {
        dft2<INV>(x[0], x[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(x[0], x[1], x[2], x[3]);
    } else if constexpr (R == 8) {   // n = 2 n1 + n2: DFT4 over n1, twiddle W8^(n2 k1), DFT2 over n2
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) dft4<INV>(x[n2], x[2 + n2], x[4 + n2], x[6 + n2]);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) x[2 * k1 + 1] = c_tw<8, INV>(x[2 * k1 + 1], k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft2<INV>(x[2 * k1], x[2 * k1 + 1]);
    } else {   // 16: n = 4 n1 + n2: DFT4 over n1, twiddle W16^(n2 k1), DFT4 over n2
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) x[4 * k1 + n2] = c_tw<16, INV>(x[4 * k1 + n2], n2 * k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    }
}

__host__ __device__ constexpr int spad(int i) { return i + (i >> 4); }

// twiddle exp(-/+ 2 pi i m / N) from the table of exp(-2 pi i m / N)
template <bool INV> __device__ __forceinline__ float2 twiddle(const float2 *__restrict__ W, int m) {
    float2 w = __ldg(W + m);
    if (INV) w.y = -w.y;
    return w;
}
__device__ __forceinline__ float2 c_mul1(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Inputs r = 1..R-1 of a butterfly times w^r, w = exp(-/+ 2 pi i k step / N).  w and (for R >= 8) w^4
// come from the table, the other powers from products of at most three of them (w^r = w^h w^(r-h),
// h the largest power of two below r): two gathered loads instead of R - 1, and a twiddle error of a
// few units in the last place, about the table's own rounding.
template <int R, bool INV, typename E>
__device__ __forceinline__ void apply_twiddles(E *v, const float2 *__restrict__ W, int k, int step) {
    float2 w[R];
    w[1] = twiddle<INV>(W, k * step);
    if (R >= 8) w[4 % R] = twiddle<INV>(W, 4 * k * step);
#pragma unroll
    for (int r = 2; r < R; ++r) {
        if (R >= 8 && r == 4) continue;
        const int h = r >= 8 ? 8 : r >= 4 ? 4 : 2;
        w[r] = h == r ? c_mul1(w[r / 2], w[r / 2]) : c_mul1(w[h], w[r - h]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], w[r]);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

}  // namespace fft
}  // namespace pfb
