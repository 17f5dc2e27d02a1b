// Internal declarations of libpfb (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "pfb.h"

namespace pfb {

constexpr int TILE = 32;                 // uv tile edge (cells) owned by one gridding CTA
constexpr double C_LIGHT = 299792458.0;  // m/s
constexpr int MAX_W = 16;                // largest ES support (taps per axis)
constexpr uint32_t VIS_MASK = 0x3fffffffu;  // item = vis index | du << 30 | dv << 31

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define PFB_CUDA(x)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess)                                                              \
            throw ::pfb::Error(PFB_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define PFB_CUFFT(x)                                                                        \
    do {                                                                                    \
        cufftResult r_ = (x);                                                               \
        if (r_ != CUFFT_SUCCESS)                                                            \
            throw ::pfb::Error(PFB_ERR_CUDA, std::string(#x) + ": cufft error " + std::to_string((int)r_)); \
    } while (0)

#define PFB_REQUIRE(cond, msg)                                   \
    do {                                                         \
        if (!(cond)) throw ::pfb::Error(PFB_ERR_ARG, (msg));     \
    } while (0)

inline void check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(PFB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

// ------------------------------------------------------------------ device math helpers
__device__ __forceinline__ void sincos_turns(float r, float *s, float *c) { sincospif(2.0f * r, s, c); }
__device__ __forceinline__ void sincos_turns(double r, double *s, double *c) { sincospi(2.0 * r, s, c); }

// Phase of w-plane k in turns, th0 + k * dth, for a pixel whose per-plane step
// dth = dth_hi + dth_lo (double-float) and offset th0 were reduced in FP64 once.
// FP32: the product k * dth_hi is split exactly (TwoProduct by FMA) and its integer
// part dropped before the small terms are added, so the result stays accurate to
// ~1e-9 turns for any plane count.
__device__ __forceinline__ float plane_turns(int k, float th0, float dth_hi, float dth_lo) {
    const float kf = (float)k;
    const float p = kf * dth_hi;
    const float e = fmaf(kf, dth_hi, -p);
    return (p - rintf(p)) + (e + fmaf(kf, dth_lo, th0));
}
__device__ __forceinline__ double plane_turns(int k, double th0, double dth_hi, double dth_lo) {
    return th0 + (double)k * (dth_hi + dth_lo);
}

// exp(i 2 pi phi) for a phase given in turns; the phase is range-reduced in FP64
// first, then evaluated in the working precision T.
template <typename T>
__device__ __forceinline__ void cis_turns(double phi, T *c, T *s) {
    double r = phi - rint(phi);
    sincos_turns((T)r, s, c);
}

// Exponential of semicircle kernel (Barnett, Magland & af Klinteberg 2019):
// phi(z) = exp(beta (sqrt(1 - (2z/W)^2) - 1)) for |z| < W/2, else 0.
__device__ __forceinline__ float es_kernel(float z, float inv_halfw, float beta) {
    float x = z * inv_halfw;
    float t = 1.0f - x * x;
    return t > 0.0f ? __expf(beta * (sqrtf(t) - 1.0f)) : 0.0f;
}
// Same kernel with sqrt(t) as t * rsqrt(t) (hardware approximation, relative error
// about 1e-7, i.e. about beta * 1e-7 in phi: far below the FP32 path's epsilon).
__device__ __forceinline__ float es_kernel_fast(float z, float inv_halfw, float beta) {
    float x = z * inv_halfw;
    float t = 1.0f - x * x;
    return t > 0.0f ? __expf(beta * (t * rsqrtf(t) - 1.0f)) : 0.0f;
}
// The same kernel from its scaled argument x = 2z/W and b2 = beta log2(e), for taps whose arguments step by
// a constant: exp(y) is evaluated as 2^(y log2 e) by the hardware approximation ex2.approx (relative error
// about 2^-22), sqrt(t) by sqrt.approx.  The taps of a visibility lie in -1 <= x < 1; t is clamped at 0, so
// at x = -1 exactly (a first tap at -W/2) the tap is exp(-beta), about 1e-6 of the peak, instead of 0.
__device__ __forceinline__ float es_kernel_x(float x, float b2) {
    const float t = fmaxf(fmaf(-x, x, 1.0f), 0.0f);
    float r, e;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fmaf(b2, r, -b2)));
    return e;
}
// beta log2(e) for es_kernel_x
__host__ __device__ inline float es_b2(double beta) { return (float)(beta * 1.4426950408889634); }
__device__ __forceinline__ double es_kernel(double z, double inv_halfw, double beta) {
    double x = z * inv_halfw;
    double t = 1.0 - x * x;
    return t > 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}

// Geometry of one band's w-stack as seen by the kernels (passed by value).
struct BandGeom {
    int Nu, Nv;          // oversampled grid
    int W;               // uv support (taps)
    int Ww;              // w support: W when w-stacking, 1 otherwise
    int ntu, ntv;        // tiles per axis
    int nkq, q;          // w buckets per key and planes per bucket
    int P;               // planes of this band
    int band;
    int nchan;
    double u2cell, v2cell;  // dl * Nu, dm * Nv: wavelengths -> grid cells
    double inv_dw, w0;      // w -> plane coordinate z_w = (w - w0) / dw
    double tc;              // centre of t = n - 1 - fa dl - fb dm over the image; removed per visibility
    // facet terms: u' = u + fa w, v' = v + fb w on the grid, and the phase u l0 + v m0 per visibility
    int facet;
    double fa, fb, l0, m0;
    int accumulate;         // degridding adds into the visibilities instead of writing them
    double beta;
    double inv_halfw;       // 2 / W
    // FP32 path: first-tap offsets O = W/2 (uv) and W/2 + w0/dw (w), split into
    // an integer and a fraction so that the cell arithmetic stays exact
    int uv_oi, w_oi;
    float uv_of, w_of, hw;
    float inv_Nu, inv_Nv;
    // FP32 path: w0 and the plane spacing dw as unevaluated float pairs (hi + lo) for the per-pixel
    // plane phases of the pre- and post-pass
    float w0_hi, w0_lo, dw_hi, dw_lo;
};

// frac(a t) in turns for a = a_hi + a_lo and t = t_hi + t_lo (unevaluated float pairs), as hi + lo.
// The leading product is split exactly by FMA (TwoProduct) and its integer part removed (exact for
// |a t| < 2^23); the cross terms a_hi t_lo + a_lo t_hi are added and the sum renormalised by TwoSum.
// The dropped a_lo t_lo and the rounding of the cross terms leave about 2^-46 |a t| of error, so the
// reduced phase is good to ~1e-12 turns for the phases of the w-stack (|a t| of a few hundred turns).
__device__ __forceinline__ void frac_prod_df(float a_hi, float a_lo, float t_hi, float t_lo, float *hi, float *lo) {
    const float p = a_hi * t_hi;
    const float e = fmaf(a_hi, t_hi, -p);
    const float q = p - rintf(p);
    const float s = e + fmaf(a_hi, t_lo, a_lo * t_hi);
    const float h = q + s;
    const float z = h - q;
    *hi = h;
    *lo = (q - (h - z)) + (s - z);
}

// x mod n in [0, n) for |x| < 2^24, by a float reciprocal and one correction
__device__ __forceinline__ int wrap_mod(int x, int n, float inv_n) {
    int q = (int)floorf((float)x * inv_n);
    int r = x - q * n;
    r += r < 0 ? n : 0;
    r -= r >= n ? n : 0;
    return r;
}

// Per-row / per-channel factors of the FP32 path, each FP64 value stored as an
// unevaluated sum hi + lo of two floats (double-float, Dekker 1971).
struct ChanDF {
    float su_hi, su_lo;   // f/c * dl * Nu  (metres -> u cells)
    float sv_hi, sv_lo;   // f/c * dm * Nv
    float sw_hi, sw_lo;   // f/c / dw       (metres -> w-plane coordinate)
    float sp_hi, sp_lo;   // f/c * t_c      (metres -> turns of exp(-2 pi i w t_c))
    // facets only
    float sa_hi, sa_lo;   // f/c * fa * dl * Nu  (metres of w -> u cells)
    float sb_hi, sb_lo;   // f/c * fb * dm * Nv  (metres of w -> v cells)
    float sl_hi, sl_lo;   // f/c * l0            (metres of u -> turns)
    float sm_hi, sm_lo;   // f/c * m0            (metres of v -> turns)
};

// Grid coordinates of one visibility.
template <typename T>
struct VisCoord {
    int gu0, gv0;   // first tap cell, wrapped into [0, Nu) / [0, Nv)
    int k0;         // first w-plane
    T ou, ov;       // first-tap offset from the visibility: gu0 - x_u, in (-W/2, -W/2 + 1]
    T ow;           // first-plane offset k0 - z_w
    T ph;           // w t_c in turns, reduced to [-1/2, 1/2]
    bool flip;      // the row was mapped (u,v,w) -> (-u,-v,-w) and V -> conj V
};

// ---- FP64 path
__device__ __forceinline__ VisCoord<double> vis_coord64(const double *__restrict__ uvw, int64_t row, double s,
                                                        const BandGeom &g) {
    VisCoord<double> c;
    double u = uvw[3 * row + 0] * s, v = uvw[3 * row + 1] * s, w = uvw[3 * row + 2] * s;
    c.flip = w < 0.0;
    if (c.flip) { u = -u; v = -v; w = -w; }
    const double hw = 0.5 * g.W;
    double xu = (g.facet ? u + g.fa * w : u) * g.u2cell, xv = (g.facet ? v + g.fb * w : v) * g.v2cell;
    xu -= g.Nu * floor(xu / g.Nu);            // periodic grid: wrap into [0, Nu)
    xv -= g.Nv * floor(xv / g.Nv);
    double fu = ceil(xu - hw), fv = ceil(xv - hw);
    c.ou = fu - xu;
    c.ov = fv - xv;
    int gu = (int)fu, gv = (int)fv;
    if (gu < 0) gu += g.Nu;
    if (gv < 0) gv += g.Nv;
    if (gu >= g.Nu) gu -= g.Nu;
    if (gv >= g.Nv) gv -= g.Nv;
    c.gu0 = gu;
    c.gv0 = gv;
    double ph = w * g.tc;
    ph -= rint(ph);
    if (g.facet) {
        double pu = u * g.l0, pv = v * g.m0;
        ph += (pu - rint(pu)) + (pv - rint(pv));
    }
    c.ph = ph - rint(ph);
    if (g.Ww > 1) {
        double zw = (w - g.w0) * g.inv_dw;
        double fk = ceil(zw - hw);
        int k0 = (int)fk;
        k0 = k0 < 0 ? 0 : (k0 > g.P - g.Ww ? g.P - g.Ww : k0);
        c.k0 = k0;
        c.ow = (double)k0 - zw;
    } else {
        c.k0 = 0;
        c.ow = 0.0;
    }
    return c;
}

// ---- FP32 path: double-float products, no FP64 instructions.
// a * s with a = a_hi + a_lo, s = s_hi + s_lo: p + e (TwoProduct by FMA; the
// a_lo * s_lo term is below the precision kept).
__device__ __forceinline__ void df_mul(float a_hi, float a_lo, float s_hi, float s_lo, float &p, float &e) {
    p = a_hi * s_hi;
    e = fmaf(a_hi, s_hi, -p) + fmaf(a_hi, s_lo, a_lo * s_hi);
}

// (p + e) += a * s in double-float: the new product by TwoProduct, the two high parts by TwoSum
// (Knuth), every rounding error gathered into e.
__device__ __forceinline__ void df_add_mul(float a_hi, float a_lo, float s_hi, float s_lo, float &p, float &e) {
    float q, f;
    df_mul(a_hi, a_lo, s_hi, s_lo, q, f);
    const float t = p + q;
    const float bb = t - p;
    const float err = (p - (t - bb)) + (q - bb);
    p = t;
    e = e + f + err;
}

// First tap g0 = ceil(x - O) and offset g0 - x for x = p + e, O = oi + of.
__device__ __forceinline__ void df_tap(float p, float e, int oi, float of, float hw, int &g0, float &off) {
    const float r = floorf(p);
    const float gf = ((p - r) + e) - of;    // p - r is exact
    const float c = ceilf(gf);
    g0 = (int)r - oi + (int)c;
    off = (c - gf) - hw;
}

__device__ __forceinline__ VisCoord<float> vis_coord32(const float2 *__restrict__ rowdf, int64_t row,
                                                       const ChanDF &cs, const BandGeom &g) {
    VisCoord<float> c;
    float2 u = rowdf[3 * row + 0], v = rowdf[3 * row + 1], w = rowdf[3 * row + 2];
    c.flip = w.x < 0.0f || (w.x == 0.0f && w.y < 0.0f);
    if (c.flip) {
        u.x = -u.x; u.y = -u.y; v.x = -v.x; v.y = -v.y; w.x = -w.x; w.y = -w.y;
    }
    float p, e;
    int g0;
    df_mul(u.x, u.y, cs.su_hi, cs.su_lo, p, e);
    if (g.facet) df_add_mul(w.x, w.y, cs.sa_hi, cs.sa_lo, p, e);
    df_tap(p, e, g.uv_oi, g.uv_of, g.hw, g0, c.ou);
    c.gu0 = wrap_mod(g0, g.Nu, g.inv_Nu);
    df_mul(v.x, v.y, cs.sv_hi, cs.sv_lo, p, e);
    if (g.facet) df_add_mul(w.x, w.y, cs.sb_hi, cs.sb_lo, p, e);
    df_tap(p, e, g.uv_oi, g.uv_of, g.hw, g0, c.ov);
    c.gv0 = wrap_mod(g0, g.Nv, g.inv_Nv);
    df_mul(w.x, w.y, cs.sp_hi, cs.sp_lo, p, e);
    c.ph = (p - rintf(p)) + e;
    if (g.facet) {
        df_mul(u.x, u.y, cs.sl_hi, cs.sl_lo, p, e);
        c.ph += (p - rintf(p)) + e;
        df_mul(v.x, v.y, cs.sm_hi, cs.sm_lo, p, e);
        c.ph += (p - rintf(p)) + e;
        c.ph -= rintf(c.ph);
    }
    if (g.Ww > 1) {
        df_mul(w.x, w.y, cs.sw_hi, cs.sw_lo, p, e);
        df_tap(p, e, g.w_oi, g.w_of, g.hw, g0, c.ow);
        c.k0 = g0 < 0 ? 0 : (g0 > g.P - g.Ww ? g.P - g.Ww : g0);
    } else {
        c.k0 = 0;
        c.ow = 0.0f;
    }
    return c;
}

// Per-visibility inputs of the coordinate computation, for either path.
struct CoordSrc {
    const double *uvw;      // FP64 path
    const double *scale;    // f / c per channel (FP64 path)
    const float2 *rowdf;    // FP32 path: uvw as double-float
    const ChanDF *chandf;   // FP32 path
};

template <typename T>
__device__ __forceinline__ VisCoord<T> vis_coord(const CoordSrc &s, int64_t row, int ch, const BandGeom &g);
template <>
__device__ __forceinline__ VisCoord<double> vis_coord<double>(const CoordSrc &s, int64_t row, int ch,
                                                              const BandGeom &g) {
    return vis_coord64(s.uvw, row, s.scale[ch], g);
}
template <>
__device__ __forceinline__ VisCoord<float> vis_coord<float>(const CoordSrc &s, int64_t row, int ch,
                                                            const BandGeom &g) {
    return vis_coord32(s.rowdf, row, s.chandf[ch], g);
}

// ES weights of the W taps starting at offset o (o, o+1, ..., o+W-1).
template <typename T>
__device__ __forceinline__ void es_taps(T o, int W, const BandGeom &g, T *out) {
    T o0 = o;
    T ihw = (T)g.inv_halfw, b = (T)g.beta;
#pragma unroll
    for (int t = 0; t < MAX_W; ++t)
        if (t < W) out[t] = es_kernel(o0 + (T)t, ihw, b);
}

// ------------------------------------------------------------------ host-side plan
struct Plan;
struct Ctx;

// Grow-only device buffer owned by the context.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace pfb
