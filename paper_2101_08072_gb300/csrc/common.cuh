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
    double tc;              // centre of (n - 1) over the image; removed per visibility
    double beta;
    double inv_halfw;       // 2 / W
};

// Grid coordinates of one visibility (FP64 arithmetic; fractional offsets of
// the first tap stay in FP64 until the kernel converts them).
struct VisCoord {
    int gu0, gv0;   // first tap cell, wrapped into [0, Nu) / [0, Nv)
    int k0;         // first w-plane
    double ou, ov;  // first-tap offset from the visibility: gu0 - x_u, in (-W/2, -W/2 + 1]
    double ow;      // first-plane offset k0 - z_w
    double wl;      // w in wavelengths after the Hermitian flip
    bool flip;      // the row was mapped (u,v,w) -> (-u,-v,-w) and V -> conj V
};

__device__ __forceinline__ VisCoord vis_coord(const double *__restrict__ uvw, int64_t row, double s,
                                              const BandGeom &g) {
    VisCoord c;
    double u = uvw[3 * row + 0] * s, v = uvw[3 * row + 1] * s, w = uvw[3 * row + 2] * s;
    c.flip = w < 0.0;
    if (c.flip) { u = -u; v = -v; w = -w; }
    const double hw = 0.5 * g.W;
    double xu = u * g.u2cell, xv = v * g.v2cell;
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
    c.wl = w;
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

// ES weights of the W taps starting at offset o (o, o+1, ..., o+W-1).
template <typename T>
__device__ __forceinline__ void es_taps(double o, int W, const BandGeom &g, T *out) {
    T o0 = (T)o;
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
