// Image-side operators of pfb-clean: the PSF convolution I^psf * x (Eq. 4), the
// preconditioner U = I^psf_sym * + sigma Id (Eq. 8), conjugate gradient for
// U delta = IR (Eq. 6), the Condat-Vu primal-dual solver for the backward step
// (Eq. 7) with r(x) = lambda ||Psi^dagger x||_{2,1} + iota_+(x) (Eq. 9), and the
// composed step.  All scalars of the iterations (CG alpha/beta, step sizes)
// stay on the device: a step launches a fixed sequence of kernels and reads
// results back only when the caller asks for host statistics.
#include "ctx.cuh"

#include <algorithm>
#include <complex>

namespace pfb {

template <typename T> struct RFft;
template <> struct RFft<float> {
    static constexpr cufftType r2c = CUFFT_R2C, c2r = CUFFT_C2R;
    static cufftResult fwd(cufftHandle h, float *in, float2 *out) {
        return cufftExecR2C(h, (cufftReal *)in, (cufftComplex *)out);
    }
    static cufftResult inv(cufftHandle h, float2 *in, float *out) {
        return cufftExecC2R(h, (cufftComplex *)in, (cufftReal *)out);
    }
};
template <> struct RFft<double> {
    static constexpr cufftType r2c = CUFFT_D2Z, c2r = CUFFT_Z2D;
    static cufftResult fwd(cufftHandle h, double *in, double2 *out) {
        return cufftExecD2Z(h, (cufftDoubleReal *)in, (cufftDoubleComplex *)out);
    }
    static cufftResult inv(cufftHandle h, double2 *in, double *out) {
        return cufftExecZ2D(h, (cufftDoubleComplex *)in, (cufftDoubleReal *)out);
    }
};

// ------------------------------------------------------------------ small kernels
// psf centre (nx, ny) moved to index (0, 0): s[i][j] = psf[(i + nx) mod 2nx][(j + ny) mod 2ny]
template <typename T>
__global__ void k_ifftshift(int nx, int ny, int nband, const T *__restrict__ psf, T *__restrict__ out) {
    const int64_t NX = 2 * nx, NY = 2 * ny;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nband * NX * NY) return;
    const int64_t b = e / (NX * NY), r = e - b * NX * NY;
    const int64_t i = r / NY, j = r - i * NY;
    int64_t si = i + nx, sj = j + ny;
    si -= si >= NX ? NX : 0;
    sj -= sj >= NY ? NY : 0;
    out[e] = psf[b * NX * NY + si * NY + sj];
}

// zero-padded copy of (a - b) (b may be null) into [nband][2nx][2ny]
// (blockIdx.y = band, blocks stride over the 2 nx padded rows)
template <typename T>
__global__ void k_pad(int nx, int ny, const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out) {
    const int bb = blockIdx.y;
    const int NX = 2 * nx, NY = 2 * ny;
    for (int i = blockIdx.x; i < NX; i += gridDim.x) {
        T *orow = out + ((int64_t)bb * NX + i) * NY;
        if (i < nx) {
            const int64_t s0 = ((int64_t)bb * nx + i) * ny;
#pragma unroll 4
            for (int j = threadIdx.x; j < ny; j += blockDim.x) orow[j] = b ? a[s0 + j] - b[s0 + j] : a[s0 + j];
            for (int j = ny + threadIdx.x; j < NY; j += blockDim.x) orow[j] = 0;
        } else {
            for (int j = threadIdx.x; j < NY; j += blockDim.x) orow[j] = 0;
        }
    }
}

// X *= S * scale (complex S)
template <typename T>
__global__ void k_spec_mul(int64_t n, const cx_t<T> *__restrict__ S, T scale, cx_t<T> *__restrict__ X) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const cx_t<T> s = S[e];
    cx_t<T> x = X[e];
    const T r = (x.x * s.x - x.y * s.y) * scale;
    const T i = (x.x * s.y + x.y * s.x) * scale;
    x.x = r;
    x.y = i;
    X[e] = x;
}

// X *= Re(S) * scale (the spectrum of the symmetrised PSF, Eq. 8)
template <typename T>
__global__ void k_spec_mul_re(int64_t n, const T *__restrict__ Sre, T scale, cx_t<T> *__restrict__ X) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const T s = Sre[e] * scale;
    cx_t<T> x = X[e];
    x.x *= s;
    x.y *= s;
    X[e] = x;
}

template <typename T>
__global__ void k_real_part(int64_t n, const cx_t<T> *__restrict__ S, T *__restrict__ re) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) re[e] = S[e].x;
}

// top-left [nx][ny] corner of each padded band (blockIdx.y = band, blocks stride over rows)
template <typename T>
__global__ void k_crop(int nx, int ny, const T *__restrict__ big, T *__restrict__ y) {
    const int b = blockIdx.y;
    for (int i = blockIdx.x; i < nx; i += gridDim.x) {
        const T *brow = big + ((int64_t)b * 2 * nx + i) * 2 * ny;
        T *yrow = y + ((int64_t)b * nx + i) * ny;
#pragma unroll 4
        for (int j = threadIdx.x; j < ny; j += blockDim.x) yrow[j] = brow[j];
    }
}

// max |v| over n values (bits of a non-negative double)
template <typename T>
__global__ void k_absmax(int64_t n, const T *__restrict__ v, unsigned long long *out) {
    T mt = 0;   // the maximum of the working-precision values is exact in that precision
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        mt = fmax(mt, fabs(v[e]));
    double m = (double)mt;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// block reduction of a double into *dst (atomic)
__device__ __forceinline__ void block_sum_atomic(double v, double *dst) {
    __shared__ double ws[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(dst, v);
    }
    __syncthreads();
}

// Sum of products per thread.  FP64 arithmetic runs at a small fraction of the FP32
// rate on this GPU, so FP32 work keeps its sums as an unevaluated float pair: each
// product split exactly into p + e (e by FMA) and each addition by Knuth's TwoSum,
// which keeps about 48 bits; the pair becomes a double once per thread.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float hi = 0, lo = 0;
    __device__ __forceinline__ void add(float v) {
        const float s = __fadd_rn(hi, v);
        const float vb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, vb)), __fsub_rn(v, vb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        add(p);
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Scalar slots of one step (device doubles)
enum {
    S_XHX = 0,      // x_k . H x_k
    S_XD,           // x_k . I^d
    S_UNORM,        // ||U|| (bits while reducing, then value)
    S_DX2,          // ||x_{k+1} - x_k||^2
    S_X2,           // ||x_{k+1}||^2
    S_L21,          // ||Psi^dagger x_k||_{2,1}
    S_TAU,          // primal step size of the Condat-Vu iteration
    S_COUNT
};
// per-band arrays follow: BB[nb] (||IR||^2), then RR[(iters+1)][nb], PAP[iters][nb]
#define S_UNORM_IDX S_UNORM

// IR = (I^d - H x) * inv_wbar; objective pieces (per band blocks, blockIdx.y = band):
// x . H x and x . I^d (both scaled by inv_wbar), ||IR||^2 per band
template <typename T>
__global__ void k_residual(int64_t npix, const T *__restrict__ dirty, const T *__restrict__ hx,
                           const T *__restrict__ x, double inv_wbar, T *__restrict__ ir, double *__restrict__ sc,
                           double *__restrict__ bb) {
    const int b = blockIdx.y;
    const T w = (T)inv_wbar;
    Acc<T> xhx, xd, rr;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = b * npix + p;
        const T d = dirty[e], h = hx[e], xv = x[e];
        const T r = (d - h) * w;
        ir[e] = r;
        xhx.add_prod(xv, h);
        xd.add_prod(xv, d);
        rr.add_prod(r, r);
    }
    block_sum_atomic(xhx.value() * inv_wbar, &sc[S_XHX]);
    block_sum_atomic(xd.value() * inv_wbar, &sc[S_XD]);
    block_sum_atomic(rr.value(), &bb[b]);
}

// CG start: delta = 0, r = p = IR, RR[0] = BB
template <typename T>
__global__ void k_cg_init(int64_t n, const T *__restrict__ ir, T *__restrict__ delta, T *__restrict__ r,
                          T *__restrict__ p) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const T v = ir[e];
    delta[e] = 0;
    r[e] = v;
    p[e] = v;
}

__device__ __forceinline__ bool cg_active(double rr, double bb, double tol2) { return rr > 0.0 && rr > tol2 * bb; }

// Ap = crop(conv) + sigma p, pap[b] += p . Ap   (blockIdx.y = band, blocks stride over rows)
template <typename T>
__global__ void k_cg_ap(int nx, int ny, const T *__restrict__ big, const T *__restrict__ p, T sigma,
                        T *__restrict__ ap, double *__restrict__ pap) {
    const int b = blockIdx.y;
    Acc<T> acc;
    for (int i = blockIdx.x; i < nx; i += gridDim.x) {
        const T *brow = big + ((int64_t)b * 2 * nx + i) * 2 * ny;
        const int64_t e0 = ((int64_t)b * nx + i) * ny;
#pragma unroll 4
        for (int j = threadIdx.x; j < ny; j += blockDim.x) {
            const T pv = p[e0 + j];
            const T v = brow[j] + sigma * pv;
            ap[e0 + j] = v;
            acc.add_prod(pv, v);
        }
    }
    block_sum_atomic(acc.value(), &pap[b]);
}

// delta += alpha p; r -= alpha Ap; rr_next[b] += r . r
template <typename T>
__global__ void k_cg_update(int64_t npix, const T *__restrict__ p, const T *__restrict__ ap,
                            const double *__restrict__ rr, const double *__restrict__ pap,
                            const double *__restrict__ bb, double tol2, T *__restrict__ delta, T *__restrict__ r,
                            double *__restrict__ rr_next) {
    const int b = blockIdx.y;
    __shared__ T s_alpha;
    if (threadIdx.x == 0) {
        const bool act = cg_active(rr[b], bb[b], tol2) && pap[b] > 0.0;
        s_alpha = act ? (T)(rr[b] / pap[b]) : (T)0;
    }
    __syncthreads();
    const T alpha = s_alpha;
    Acc<T> acc;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = b * npix + q;
        delta[e] += alpha * p[e];
        const T rv = r[e] - alpha * ap[e];
        r[e] = rv;
        acc.add_prod(rv, rv);
    }
    block_sum_atomic(acc.value(), &rr_next[b]);
}

// p = r + beta p, beta = rr_next / rr (0 once converged), written padded for the next U p
// (blockIdx.y = band, blocks stride over the 2 nx padded rows)
template <typename T>
__global__ void k_cg_dir(int nx, int ny, const T *__restrict__ r, const double *__restrict__ rr,
                         const double *__restrict__ rr_next, const double *__restrict__ bb, double tol2,
                         T *__restrict__ p, T *__restrict__ padded) {
    const int b = blockIdx.y;
    const int NX = 2 * nx, NY = 2 * ny;
    __shared__ T s_beta;
    if (threadIdx.x == 0) s_beta = cg_active(rr[b], bb[b], tol2) ? (T)(rr_next[b] / rr[b]) : (T)0;
    __syncthreads();
    const T beta = s_beta;
    for (int i = blockIdx.x; i < NX; i += gridDim.x) {
        T *prow = padded + ((int64_t)b * NX + i) * NY;
        if (i < nx) {
            const int64_t e0 = ((int64_t)b * nx + i) * ny;
#pragma unroll 4
            for (int j = threadIdx.x; j < ny; j += blockDim.x) {
                const T v = r[e0 + j] + beta * p[e0 + j];
                p[e0 + j] = v;
                prow[j] = v;
            }
            for (int j = ny + threadIdx.x; j < NY; j += blockDim.x) prow[j] = 0;
        } else {
            for (int j = threadIdx.x; j < NY; j += blockDim.x) prow[j] = 0;
        }
    }
}

template <typename T>
__global__ void k_axpy_clamp(int64_t n, const T *__restrict__ x, const T *__restrict__ d, T gamma,
                             T *__restrict__ xbar, T *__restrict__ xpd) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const T v = x[e] + gamma * d[e];
    xbar[e] = v;
    xpd[e] = v > 0 ? v : 0;
}

// Condat-Vu primal step size, once per step: tau = 0.98 / (||U|| / (2 gamma) + 1) with
// ||U|| = max |Re S| / wbar + sigma unless given (sc[S_UNORM] holds max |Re S|)
__global__ void k_pd_tau(double *__restrict__ sc, double inv_wbar, double sigma, double gamma,
                         double unorm_fixed) {
    const double unorm = unorm_fixed > 0 ? unorm_fixed : sc[S_UNORM] * inv_wbar + sigma;
    sc[S_TAU] = 0.98 / (0.5 * unorm / gamma + 1.0);
}

// One Condat-Vu iteration with Psi = Dirac (one thread per pixel, all bands; blocks stride over rows):
//   x~ = max(0, x - tau (grad + Psi v)),  grad = (conv + sigma (x - xbar)) / gamma
//   v~ = v + Psi^dagger (2 x~ - x);  v = v~ min(1, lam / ||v~||_bands);  x = x~
template <typename T>
__global__ void k_pd_dirac(int nx, int ny, int nband, const T *__restrict__ big, const T *__restrict__ xbar,
                           T sigma, T gamma, T lam, const double *__restrict__ sc, T *__restrict__ x,
                           T *__restrict__ v) {
    const int64_t npix = (int64_t)nx * ny;
    const T tau = (T)sc[S_TAU];
    for (int i = blockIdx.x; i < nx; i += gridDim.x) {
        for (int j = threadIdx.x; j < ny; j += blockDim.x) {
            const int64_t q = (int64_t)i * ny + j;
            T xt[32], vt[32];
            T nrm2 = 0;
            for (int b = 0; b < nband; ++b) {
                const int64_t e = b * npix + q;
                const T xv = x[e];
                const T grad = (big[((int64_t)b * 2 * nx + i) * 2 * ny + j] + sigma * (xv - xbar[e])) / gamma;
                T xn = xv - tau * (grad + v[e]);
                xn = xn > 0 ? xn : 0;
                xt[b] = xn;
                const T vn = v[e] + (2 * xn - xv);
                vt[b] = vn;
                nrm2 += vn * vn;
            }
            const T nrm = sqrt(nrm2);
            const T s = nrm > lam ? lam / nrm : (T)1;
            for (int b = 0; b < nband; ++b) {
                const int64_t e = b * npix + q;
                x[e] = xt[b];
                v[e] = vt[b] * s;
            }
        }
    }
}

// final statistics: ||x1 - x0||^2, ||x1||^2; copy x1 to the output (blockIdx.y = band)
template <typename T>
__global__ void k_finish(int64_t npix, const T *__restrict__ x1, T *__restrict__ x0_out, double *__restrict__ sc) {
    const int64_t off = (int64_t)blockIdx.y * npix;
    Acc<T> dx2, x2;
#pragma unroll 4
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
        const T a = x0_out[off + q], c = x1[off + q];
        dx2.add_prod(c - a, c - a);
        x2.add_prod(c, c);
        x0_out[off + q] = c;
    }
    block_sum_atomic(dx2.value(), &sc[S_DX2]);
    block_sum_atomic(x2.value(), &sc[S_X2]);
}

// ------------------------------------------------------------------ Daubechies dictionary (Eq. 9's Psi)
// Low-pass filter of db_N by spectral factorisation (Daubechies 1988): the roots
// y_k of P(y) = sum_{k<N} C(N-1+k, k) y^k (Durand-Kerner iteration), each mapped to
// the root inside the unit circle of z^2 - (2 - 4 y_k) z + 1; h holds the
// coefficients of (z + 1)^N prod (z - z_k), highest power first, scaled to sum sqrt(2).
static std::vector<double> daubechies_filter(int N) {
    typedef std::complex<double> C;
    if (N == 1) return {M_SQRT1_2, M_SQRT1_2};
    const int deg = N - 1;
    std::vector<double> c(N);   // increasing powers
    for (int k = 0; k < N; ++k) {
        double b = 1.0;   // C(N-1+k, k)
        for (int j = 1; j <= k; ++j) b = b * (N - 1 + j) / j;
        c[k] = b;
    }
    auto P = [&](C y) {
        C r = 0;
        for (int k = deg; k >= 0; --k) r = r * y + c[k];
        return r;
    };
    std::vector<C> ys(deg);
    for (int i = 0; i < deg; ++i) ys[i] = std::pow(C(0.4, 0.9), i);
    for (int it = 0; it < 500; ++it) {
        double move = 0;
        for (int i = 0; i < deg; ++i) {
            C den = c[deg];
            for (int j = 0; j < deg; ++j)
                if (j != i) den *= ys[i] - ys[j];
            const C d = P(ys[i]) / den;
            ys[i] -= d;
            move = std::max(move, std::abs(d));
        }
        if (move < 1e-15) break;
    }
    std::vector<C> poly(1, C(1));   // increasing powers
    auto mul = [&](C root) {       // poly *= (z - root)
        std::vector<C> np(poly.size() + 1, C(0));
        for (size_t k = 0; k < poly.size(); ++k) {
            np[k + 1] += poly[k];
            np[k] -= root * poly[k];
        }
        poly = np;
    };
    for (int k = 0; k < N; ++k) mul(C(-1));
    for (int i = 0; i < deg; ++i) {
        const C a = 1.0 - 2.0 * ys[i];
        const C sq = std::sqrt(a * a - 1.0);
        const C z1 = a + sq, z2 = a - sq;
        mul(std::abs(z1) < 1.0 ? z1 : z2);
    }
    std::vector<double> h(poly.size());
    double sum = 0;
    for (size_t k = 0; k < poly.size(); ++k) {
        h[k] = poly[poly.size() - 1 - k].real();   // highest power first
        sum += h[k];
    }
    for (auto &v : h) v *= M_SQRT2 / sum;
    return h;
}

constexpr int MAX_TAPS = 12;
struct WavFilt {
    int L;
    double h[MAX_TAPS], g[MAX_TAPS];   // low-pass and high-pass g_k = (-1)^k h_{L-1-k}
};
// taps in the working precision (passed to the kernels by value)
template <typename T>
struct WavTaps {
    int L;
    T h[MAX_TAPS], g[MAX_TAPS];
    explicit WavTaps(const WavFilt &f) : L(f.L) {
        for (int k = 0; k < MAX_TAPS; ++k) {
            h[k] = (T)(k < f.L ? f.h[k] : 0.0);
            g[k] = (T)(k < f.L ? f.g[k] : 0.0);
        }
    }
};

static WavFilt wav_filter(int N) {
    static std::map<int, WavFilt> cache;
    auto it = cache.find(N);
    if (it != cache.end()) return it->second;
    std::vector<double> h = daubechies_filter(N);
    WavFilt f;
    f.L = (int)h.size();
    for (int k = 0; k < f.L; ++k) {
        f.h[k] = h[k];
        f.g[k] = ((k & 1) ? -1.0 : 1.0) * h[f.L - 1 - k];
    }
    cache[N] = f;
    return f;
}

// ---- periodised 2-D DWT, one level per launch, both axes in shared memory
// One level maps an [n x m] block x to its four half-size subbands (Mallat layout):
//   along an axis of length N:  a[k] = sum_t h[t] x[(2k + t) mod N],  d[k] = sum_t g[t] x[(2k + t) mod N]
// applied along axis 0 (rows, i) and axis 1 (columns, j): (a,a) is the coarse band LL at (k, q),
// (a,d) sits at (k, q + m/2), (d,a) at (k + n/2, q) and (d,d) at (k + n/2, q + m/2).  Its transpose
// (= inverse, the filters being orthonormal) is, along an axis,
//   x[p] = sum_{t = p mod 2} h[t] a[((p - t) mod N) / 2] + g[t] d[((p - t) mod N) / 2].
// A CTA owns a tile: the forward kernel a 32 x 32 tile of every subband, whose (2*32 + L - 2)^2 input
// region (with the periodic halo) it stages once; the inverse kernel a 64 x 64 tile of x, staging the
// (32 + L/2 - 1)^2 coefficients of each subband it needs.  The coarse band goes to / comes from its own
// strided view, so a multi-level transform needs no copies (coarse bands ping-pong through scratch).
template <typename T> struct View2 {
    T *p;
    int64_t bs;   // band stride (elements)
    int rs;       // row stride (elements)
};
constexpr int DWT_TO = 32;   // forward: coefficients per tile edge, each subband
constexpr int DWT_TX = 64;   // inverse: pixels per tile edge
__host__ __device__ constexpr int dwt_edge(int L) { return 2 * DWT_TO + L - 2; }
__host__ __device__ constexpr int idwt_edge(int L) { return DWT_TX / 2 + L / 2 - 1; }
template <typename T> constexpr size_t dwt_smem(int L) {
    return sizeof(T) * ((size_t)dwt_edge(L) * dwt_edge(L) + 2 * (size_t)DWT_TO * dwt_edge(L));
}
template <typename T> constexpr size_t idwt_smem(int L) {
    return sizeof(T) * (4 * (size_t)idwt_edge(L) * idwt_edge(L) + 2 * (size_t)idwt_edge(L) * DWT_TX);
}

__device__ __forceinline__ int pmod(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

template <typename T, int L>
__global__ void __launch_bounds__(256) k_dwt2_tile(int n, int m, int tiles_q, View2<T> src, View2<T> ll,
                                                   View2<T> det, WavTaps<T> f) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int E = dwt_edge(L);
    T *xs = reinterpret_cast<T *>(sm_raw);   // [E][E] input region
    T *ts = xs + E * E;                      // [2 DWT_TO][E]: a and d along axis 0
    const int b = blockIdx.y;
    const int tk = blockIdx.x / tiles_q, tq = blockIdx.x - tk * tiles_q;
    const int K0 = tk * DWT_TO, Q0 = tq * DWT_TO;
    const int nh = n / 2, mh = m / 2;
    const T *sp = src.p + b * src.bs;
    if (2 * K0 + E <= n && 2 * Q0 + E <= m) {
        // interior tile: the region does not wrap
        const T *base = sp + (int64_t)(2 * K0) * src.rs + 2 * Q0;
        for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
            const int r = e / E, c = e - r * E;
            xs[e] = base[(int64_t)r * src.rs + c];
        }
    } else {
        for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
            const int r = e / E, c = e - r * E;
            xs[e] = sp[(int64_t)pmod(2 * K0 + r, n) * src.rs + pmod(2 * Q0 + c, m)];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < DWT_TO * E; e += blockDim.x) {
        const int kk = e / E, c = e - kk * E;
        const T *col = xs + 2 * kk * E + c;
        T lo = 0, hi = 0;
#pragma unroll
        for (int t = 0; t < L; ++t) {
            const T v = col[t * E];
            lo += f.h[t] * v;
            hi += f.g[t] * v;
        }
        ts[kk * E + c] = lo;
        ts[(DWT_TO + kk) * E + c] = hi;
    }
    __syncthreads();
    T *lp = ll.p + b * ll.bs;
    T *dp = det.p + b * det.bs;
    for (int e = threadIdx.x; e < DWT_TO * DWT_TO; e += blockDim.x) {
        const int kk = e / DWT_TO, qq = e - kk * DWT_TO;
        const int k = K0 + kk, q = Q0 + qq;
        if (k >= nh || q >= mh) continue;
        const T *lo = ts + kk * E + 2 * qq, *hi = ts + (DWT_TO + kk) * E + 2 * qq;
        T aa = 0, ad = 0, da = 0, dd = 0;
#pragma unroll
        for (int t = 0; t < L; ++t) {
            aa += f.h[t] * lo[t];
            ad += f.g[t] * lo[t];
            da += f.h[t] * hi[t];
            dd += f.g[t] * hi[t];
        }
        lp[(int64_t)k * ll.rs + q] = aa;
        dp[(int64_t)k * det.rs + q + mh] = ad;
        dp[(int64_t)(k + nh) * det.rs + q] = da;
        dp[(int64_t)(k + nh) * det.rs + q + mh] = dd;
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(256) k_idwt2_tile(int n, int m, int tiles_s, View2<T> ll, View2<T> det,
                                                    View2<T> dst, WavTaps<T> f, T alpha, int accumulate) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int C = idwt_edge(L);
    constexpr int H = L / 2 - 1;   // offset of coefficient k = p/2 in the staged region
    T *cs = reinterpret_cast<T *>(sm_raw);   // [4][C][C]: (a,a) (a,d) (d,a) (d,d)
    T *us = cs + 4 * C * C;                  // [2][C][DWT_TX]: axis-1 inverse of the a and d rows
    const int b = blockIdx.y;
    const int tp = blockIdx.x / tiles_s, tsi = blockIdx.x - tp * tiles_s;
    const int P0 = tp * DWT_TX, S0 = tsi * DWT_TX;
    const int nh = n / 2, mh = m / 2;
    const int kb0 = P0 / 2 - H, kb1 = S0 / 2 - H;
    const T *lp = ll.p + b * ll.bs;
    const T *dp = det.p + b * det.bs;
    const bool inner = kb0 >= 0 && kb1 >= 0 && kb0 + C <= nh && kb1 + C <= mh;   // no wrap
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
        const int r = e / C, c = e - r * C;
        const int k = inner ? kb0 + r : pmod(kb0 + r, nh), q = inner ? kb1 + c : pmod(kb1 + c, mh);
        cs[e] = lp[(int64_t)k * ll.rs + q];
        cs[C * C + e] = dp[(int64_t)k * det.rs + q + mh];
        cs[2 * C * C + e] = dp[(int64_t)(k + nh) * det.rs + q];
        cs[3 * C * C + e] = dp[(int64_t)(k + nh) * det.rs + q + mh];
    }
    __syncthreads();
    // axis 1: rows r of the a (resp. d) half of axis 0
    for (int e = threadIdx.x; e < 2 * C * DWT_TX; e += blockDim.x) {
        const int half = e / (C * DWT_TX), rem = e - half * C * DWT_TX;
        const int r = rem / DWT_TX, ss = rem - r * DWT_TX;
        const T *ra = cs + (2 * half) * C * C + r * C;   // a along axis 1
        const T *rd = ra + C * C;                         // d along axis 1
        const bool odd = ss & 1;
        const int base = (ss >> 1) + H;
        T acc = 0;
#pragma unroll
        for (int u = 0; u < L / 2; ++u) {   // taps t = 2u + (ss mod 2)
            const T hv = odd ? f.h[2 * u + 1] : f.h[2 * u], gv = odd ? f.g[2 * u + 1] : f.g[2 * u];
            acc += hv * ra[base - u] + gv * rd[base - u];
        }
        us[e] = acc;
    }
    __syncthreads();
    T *op = dst.p + b * dst.bs;
    for (int e = threadIdx.x; e < DWT_TX * DWT_TX; e += blockDim.x) {
        const int pp = e / DWT_TX, ss = e - pp * DWT_TX;
        const int p = P0 + pp, s2 = S0 + ss;
        if (p >= n || s2 >= m) continue;
        const bool odd = pp & 1;
        const int base = (pp >> 1) + H;
        T acc = 0;
#pragma unroll
        for (int u = 0; u < L / 2; ++u) {   // taps t = 2u + (pp mod 2)
            const T hv = odd ? f.h[2 * u + 1] : f.h[2 * u], gv = odd ? f.g[2 * u + 1] : f.g[2 * u];
            acc += hv * us[(base - u) * DWT_TX + ss] + gv * us[(C + base - u) * DWT_TX + ss];
        }
        T *o = op + (int64_t)p * dst.rs + s2;
        *o = accumulate ? *o + alpha * acc : alpha * acc;
    }
}

template <typename T, int L>
static void dwt_level_launch(int nband, int n, int m, View2<T> src, View2<T> ll, View2<T> det, const WavFilt &f,
                             cudaStream_t st) {
    const int tk = (n / 2 + DWT_TO - 1) / DWT_TO, tq = (m / 2 + DWT_TO - 1) / DWT_TO;
    const size_t sm = dwt_smem<T>(L);
    ensure_dynamic_smem(k_dwt2_tile<T, L>, (size_t)sm);
    k_dwt2_tile<T, L><<<dim3((unsigned)(tk * tq), (unsigned)nband), 256, sm, st>>>(n, m, tq, src, ll, det,
                                                                                  WavTaps<T>(f));
    check_launch("dwt");
}

template <typename T, int L>
static void idwt_level_launch(int nband, int n, int m, View2<T> ll, View2<T> det, View2<T> dst, const WavFilt &f,
                              T alpha, int accumulate, cudaStream_t st) {
    const int tp = (n + DWT_TX - 1) / DWT_TX, ts = (m + DWT_TX - 1) / DWT_TX;
    const size_t sm = idwt_smem<T>(L);
    ensure_dynamic_smem(k_idwt2_tile<T, L>, (size_t)sm);
    k_idwt2_tile<T, L><<<dim3((unsigned)(tp * ts), (unsigned)nband), 256, sm, st>>>(n, m, ts, ll, det, dst,
                                                                                   WavTaps<T>(f), alpha, accumulate);
    check_launch("idwt");
}

#define PFB_TAPS_SWITCH(LV, CALL)                                          \
    switch (LV) {                                                          \
        case 2: CALL(2); break;                                            \
        case 4: CALL(4); break;                                            \
        case 6: CALL(6); break;                                            \
        case 8: CALL(8); break;                                            \
        case 10: CALL(10); break;                                          \
        case 12: CALL(12); break;                                          \
        default: throw Error(PFB_ERR_ARG, "unsupported wavelet filter length"); \
    }

// coef = multi-level 2-D DWT of img (Mallat layout, [nband][nx][ny]).  tmp (>= nband nx ny / 2
// elements) holds the coarse bands between levels.
template <typename T>
static void dwt2(int nx, int ny, int nband, int nlevel, const WavFilt &f, const T *img, T *coef, T *tmp,
                 cudaStream_t st) {
    const int64_t full = (int64_t)nx * ny, quarter = (int64_t)(nx / 2) * (ny / 2);
    View2<T> src{const_cast<T *>(img), full, ny};
    const View2<T> det{coef, full, ny};
    for (int lv = 0; lv < nlevel; ++lv) {
        const int n = nx >> lv, m = ny >> lv;
        // the coarse band of an intermediate level: [nband][n/2][m/2], dense, read back by the next level
        const View2<T> ll = lv == nlevel - 1
                                ? det
                                : View2<T>{tmp + (lv & 1) * nband * quarter, (int64_t)(n / 2) * (m / 2), m / 2};
#define PFB_DWT_CALL(LV) dwt_level_launch<T, LV>(nband, n, m, src, ll, det, f, st)
        PFB_TAPS_SWITCH(f.L, PFB_DWT_CALL)
#undef PFB_DWT_CALL
        src = ll;
    }
}

// out = alpha * inverse multi-level DWT of coef (Mallat layout), or out += that with accumulate;
// tmp as for dwt2.
template <typename T>
static void idwt2(int nx, int ny, int nband, int nlevel, const WavFilt &f, const T *coef, T *out, T *tmp, T alpha,
                  bool accumulate, cudaStream_t st) {
    const int64_t full = (int64_t)nx * ny, quarter = (int64_t)(nx / 2) * (ny / 2);
    const View2<T> det{const_cast<T *>(coef), full, ny};
    View2<T> ll = det;
    for (int lv = nlevel - 1; lv >= 0; --lv) {
        const int n = nx >> lv, m = ny >> lv;
        const View2<T> dst = lv == 0 ? View2<T>{out, full, ny}
                                     : View2<T>{tmp + (lv & 1) * nband * quarter, (int64_t)n * m, m};
#define PFB_IDWT_CALL(LV) \
    idwt_level_launch<T, LV>(nband, n, m, ll, det, dst, f, lv == 0 ? alpha : (T)1, lv == 0 && accumulate, st)
        PFB_TAPS_SWITCH(f.L, PFB_IDWT_CALL)
#undef PFB_IDWT_CALL
        ll = dst;
    }
}

// primal update for a general dictionary: x~ = max(0, x - tau (grad + psiv)),
// u = 2 x~ - x (kept for the dual update), x = x~   (blockIdx.y = band, blocks stride over rows)
template <typename T>
__global__ void k_pd_primal(int nx, int ny, const T *__restrict__ big, const T *__restrict__ xbar,
                            const T *__restrict__ psiv, T sigma, T gamma, const double *__restrict__ sc,
                            T *__restrict__ x, T *__restrict__ u) {
    const int b = blockIdx.y;
    const T tau = (T)sc[S_TAU];
    for (int i = blockIdx.x; i < nx; i += gridDim.x) {
        const T *brow = big + ((int64_t)b * 2 * nx + i) * 2 * ny;
        const int64_t e0 = ((int64_t)b * nx + i) * ny;
#pragma unroll 4
        for (int j = threadIdx.x; j < ny; j += blockDim.x) {
            const int64_t e = e0 + j;
            const T xv = x[e];
            const T grad = (brow[j] + sigma * (xv - xbar[e])) / gamma;
            T xn = xv - tau * (grad + psiv[e]);
            xn = xn > 0 ? xn : 0;
            u[e] = 2 * xn - xv;
            x[e] = xn;
        }
    }
}

// dual update of one basis: v~ = v + c * s (s = 1/sqrt(K)), projected onto the l2
// ball of radius lam per group (the bands of one coefficient)
template <typename T>
__global__ void k_pd_dual(int64_t npix, int nband, const T *__restrict__ c, T s, T lam, T *__restrict__ v) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= npix) return;
    T vt[32];
    T n2 = 0;
    for (int b = 0; b < nband; ++b) {
        const T t = v[b * npix + q] + s * c[b * npix + q];
        vt[b] = t;
        n2 += t * t;
    }
    const T nrm = sqrt(n2);
    const T f = nrm > lam ? lam / nrm : (T)1;
    for (int b = 0; b < nband; ++b) v[b * npix + q] = vt[b] * f;
}

// y = a x, or y += a x with accumulate
template <typename T>
__global__ void k_axpy(int64_t n, T a, const T *__restrict__ x, int accumulate, T *__restrict__ y) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = accumulate ? y[e] + a * x[e] : a * x[e];
}

// sum_q ||coef[:, q]||_2 over bands (for the l2,1 term of the objective)
template <typename T>
__global__ void k_l21(int64_t npix, int nband, const T *__restrict__ c, double scale, double *__restrict__ out) {
    Acc<T> acc;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
        T g2 = 0;
        for (int b = 0; b < nband; ++b) {
            const T v = c[b * npix + q];
            g2 += v * v;
        }
        acc.add(sqrt(g2));
    }
    block_sum_atomic(acc.value() * scale, out);
}

// ------------------------------------------------------------------ spectrum cache
template <typename T>
static cx_t<T> *psf_spectrum(Ctx &ctx, int nx, int ny, int nband, const T *psf, cudaStream_t st) {
    const int prec = sizeof(T) == 8 ? PFB_F64 : PFB_F32;
    for (auto &s : ctx.spectra)
        if (s.psf == psf && s.nx == nx && s.ny == ny && s.nband == nband && s.prec == prec)
            return (cx_t<T> *)s.spec;
    const int64_t NX = 2 * nx, NY = 2 * ny, NH = NY / 2 + 1;
    PsfSpec s;
    s.psf = psf; s.nx = nx; s.ny = ny; s.nband = nband; s.prec = prec;
    // the complex spectrum, then its real part (the spectrum of the symmetrised PSF, which is
    // all that U and ||U|| read)
    const int64_t ns = nband * NX * NH;
    s.bytes = (size_t)ns * (sizeof(cx_t<T>) + sizeof(T));
    s.spec = ctx.dalloc(s.bytes);
    T *shifted = (T *)ctx.scratch("img_pad", (size_t)nband * NX * NY * sizeof(T));
    const int64_t n = nband * NX * NY;
    k_ifftshift<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nx, ny, nband, psf, shifted);
    check_launch("ifftshift");
    cufftHandle h = ctx.fft((int)NX, (int)NY, nband, RFft<T>::r2c);
    PFB_CUFFT(cufftSetStream(h, st));
    PFB_CUFFT(RFft<T>::fwd(h, shifted, (cx_t<T> *)s.spec));
    k_real_part<T><<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, (const cx_t<T> *)s.spec,
                                                                 (T *)((cx_t<T> *)s.spec + ns));
    check_launch("real_part");
    if (ctx.spectra.size() >= 4) {
        ctx.dfree(ctx.spectra.front().spec, ctx.spectra.front().bytes);
        ctx.spectra.erase(ctx.spectra.begin());
    }
    ctx.spectra.push_back(s);
    return (cx_t<T> *)s.spec;
}

// real part of the cached spectrum S of [nband][2nx][ny+1] values (stored right after S)
template <typename T> static const T *spec_re(const cx_t<T> *S, int nx, int ny, int nband) {
    return (const T *)(S + (int64_t)nband * 2 * nx * (ny + 1));
}

// padded real [nband][2nx][2ny] -> (conv with S, or with Re S when sym) -> padded real, in place
template <typename T>
static void conv_padded(Ctx &ctx, int nx, int ny, int nband, T *padded, const cx_t<T> *S, T scale, bool sym,
                        cudaStream_t st) {
    const int64_t NX = 2 * nx, NY = 2 * ny, NH = NY / 2 + 1;
    cx_t<T> *X = (cx_t<T> *)ctx.scratch("img_spec", (size_t)nband * NX * NH * sizeof(cx_t<T>));
    // algorithmic bytes: the padded image in and out, the half spectrum written and read twice, and the
    // cached PSF spectrum read (its real part alone when sym)
    KTimer tm(ctx, "img_conv", st,
              (double)nband * NX * (2.0 * NY * sizeof(T) + 3.0 * NH * sizeof(cx_t<T>) +
                                    NH * (sym ? sizeof(T) : sizeof(cx_t<T>))), 1);
    cufftHandle hf = ctx.fft((int)NX, (int)NY, nband, RFft<T>::r2c);
    PFB_CUFFT(cufftSetStream(hf, st));
    PFB_CUFFT(RFft<T>::fwd(hf, padded, X));
    const int64_t ns = nband * NX * NH;
    if (sym)
        k_spec_mul_re<T><<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, spec_re<T>(S, nx, ny, nband), scale, X);
    else
        k_spec_mul<T><<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, S, scale, X);
    check_launch("spec_mul");
    cufftHandle hi = ctx.fft((int)NX, (int)NY, nband, RFft<T>::c2r);
    PFB_CUFFT(cufftSetStream(hi, st));
    PFB_CUFFT(RFft<T>::inv(hi, X, padded));
}

// grid of the row kernels: blockIdx.y = band, about 8 CTAs per SM in all, each striding over rows
static dim3 row_grid(const Ctx &ctx, int rows, int nband) {
    const int per_band = std::max(1, (8 * ctx.num_sms + nband - 1) / nband);
    return dim3((unsigned)std::min(rows, per_band), (unsigned)nband);
}

template <typename T>
void op_psf_conv(Ctx &ctx, int nx, int ny, int nband, const T *psf, const T *x, T *y, cudaStream_t st) {
    const int64_t NX = 2 * nx, NY = 2 * ny;
    cx_t<T> *S = psf_spectrum<T>(ctx, nx, ny, nband, psf, st);
    T *padded = (T *)ctx.scratch("img_pad", (size_t)nband * NX * NY * sizeof(T));
    const int64_t nb = nband * NX * NY;
    k_pad<T><<<row_grid(ctx, 2 * nx, nband), 256, 0, st>>>(nx, ny, x, (const T *)nullptr, padded);
    check_launch("pad");
    conv_padded<T>(ctx, nx, ny, nband, padded, S, (T)(1.0 / (double)(NX * NY)), false, st);
    const int64_t n = (int64_t)nband * nx * ny;
    k_crop<T><<<row_grid(ctx, nx, nband), 256, 0, st>>>(nx, ny, padded, y);
    check_launch("crop");
}

static unsigned rblocks(int64_t n, int cap) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, cap)); }
// grid of the per-band reductions: blockIdx.y = band, about 8 CTAs of 256 threads per SM in all
static dim3 band_grid(const Ctx &ctx, int64_t npix, int nband) {
    return dim3(rblocks(npix, std::max(1, 8 * ctx.num_sms / nband)), (unsigned)nband);
}

template <typename T>
void op_step(Ctx &ctx, const Plan &p, const pfb_params &prm, const T *wgt, const T *dirty, const T *psf,
             const double *wsum_h, T *x, T *dual, double *stats_h, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, nb = p.nband;
    const int64_t npix = (int64_t)nx * ny, n = npix * nb;
    const int64_t NX = 2 * nx, NY = 2 * ny, nbig = nb * NX * NY;
    double wbar = 0;
    for (int b = 0; b < nb; ++b) wbar += wsum_h[b];
    wbar /= nb;
    PFB_REQUIRE(wbar > 0, "weight sums must be positive");
    const double inv_wbar = 1.0 / wbar;
    const int iters = std::max(0, prm.cg_iters);
    const double tol2 = prm.cg_tol > 0 ? prm.cg_tol * prm.cg_tol : 0.0;

    // scratch
    const size_t img = (size_t)n * sizeof(T);
    T *hx = (T *)ctx.scratch("st_hx", img);
    T *ir = (T *)ctx.scratch("st_ir", img);
    T *delta = (T *)ctx.scratch("st_delta", img);
    T *r = (T *)ctx.scratch("st_r", img);
    T *pp = (T *)ctx.scratch("st_p", img);
    T *ap = (T *)ctx.scratch("st_ap", img);
    T *xbar = (T *)ctx.scratch("st_xbar", img);
    T *xk1 = (T *)ctx.scratch("st_x1", img);
    const size_t nsc = S_COUNT + nb + (size_t)(iters + 1) * nb + (size_t)iters * nb;
    double *sc = (double *)ctx.scratch("st_scal", nsc * sizeof(double));
    double *bb = sc + S_COUNT, *RR = bb + nb, *PAP = RR + (size_t)(iters + 1) * nb;
    PFB_CUDA(cudaMemsetAsync(sc, 0, nsc * sizeof(double), st));

    // image-side buffers and FFT plans first: the Hessian's w-plane stack then takes
    // whatever the budget has left
    cx_t<T> *S = psf_spectrum<T>(ctx, nx, ny, nb, psf, st);
    T *padded = (T *)ctx.scratch("img_pad", (size_t)nbig * sizeof(T));
    ctx.scratch("img_spec", (size_t)nb * NX * (NY / 2 + 1) * sizeof(cx_t<T>));
    ctx.fft((int)NX, (int)NY, nb, RFft<T>::c2r);
    if (prm.basis_mask != 1u)
        for (const char *nm : {"st_wa", "st_wb", "st_psiv", "st_u"}) ctx.scratch(nm, img);
    // 1. one exact Hessian application: H x_k = R^dagger W R x_k (Eq. 3), or with
    //    PFB_STEP_APPROX_GRADIENT its stand-in of Eq. 4, I^psf * x_k (plain, not symmetrised)
    if (prm.flags & PFB_STEP_APPROX_GRADIENT) {
        k_pad<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, x, (const T *)nullptr, padded);
        check_launch("approx_pad");
        conv_padded<T>(ctx, nx, ny, nb, padded, S, (T)(1.0 / (double)(NX * NY)), false, st);
        k_crop<T><<<row_grid(ctx, nx, nb), 256, 0, st>>>(nx, ny, padded, hx);
        check_launch("approx_crop");
    } else {
        cx_t<T> *vis = (cx_t<T> *)ctx.scratch("st_vis", (size_t)p.nrow * p.nchan * sizeof(cx_t<T>));
        op_hessian<T>(ctx, p, x, wgt, vis, hx, st);
    }
    // 2. IR = (I^d - H x_k) / wbar
    {
        k_residual<T><<<band_grid(ctx, npix, nb), 256, 0, st>>>(npix, dirty, hx, x, inv_wbar, ir, sc, bb);
        check_launch("residual");
    }
    // objective's l2,1 term at x_k: ||Psi^dagger x_k||_{2,1} (Psi normalised by 1/sqrt(K))
    std::vector<int> bases;
    for (int k = 0; k < 7; ++k)
        if (prm.basis_mask >> k & 1u) bases.push_back(k);
    const int K = (int)bases.size();
    const double inv_sqrt_k = 1.0 / std::sqrt((double)K);
    // algorithmic bytes of one multi-level transform: every level reads its input band and writes it back
    double dwt_bytes = 0;
    for (int lv = 0; lv < std::max(0, prm.nlevel); ++lv)
        dwt_bytes += 2.0 * (double)(nx >> lv) * (double)(ny >> lv) * nb * sizeof(T);
    T *wa = nullptr, *wb = nullptr;
    if (prm.basis_mask != 1u) {
        wa = (T *)ctx.scratch("st_wa", img);
        wb = (T *)ctx.scratch("st_wb", img);
    }
    for (int k : bases) {
        const T *coef = x;
        if (k > 0) {
            KTimer tm(ctx, "dwt", st, dwt_bytes, prm.nlevel);
            dwt2<T>(nx, ny, nb, prm.nlevel, wav_filter(k), x, wa, wb, st);
            coef = wa;
        }
        k_l21<T><<<rblocks(npix, 8 * ctx.num_sms), 256, 0, st>>>(npix, nb, coef, inv_sqrt_k, &sc[S_L21]);
        check_launch("l21");
    }
    // 3. CG for U delta = IR (per band)
    const T conv_scale = (T)(inv_wbar / (double)(NX * NY));
    const T sigma = (T)prm.sigma;
    k_cg_init<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ir, delta, r, pp);
    check_launch("cg_init");
    PFB_CUDA(cudaMemcpyAsync(RR, bb, nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_pad<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, pp, (const T *)nullptr, padded);
    check_launch("cg_pad");
    for (int it = 0; it < iters; ++it) {
        double *rr = RR + (size_t)it * nb, *rrn = RR + (size_t)(it + 1) * nb, *pap = PAP + (size_t)it * nb;
        conv_padded<T>(ctx, nx, ny, nb, padded, S, conv_scale, true, st);
        k_cg_ap<T><<<row_grid(ctx, nx, nb), 256, 0, st>>>(nx, ny, padded, pp, sigma, ap, pap);
        check_launch("cg_ap");
        k_cg_update<T><<<band_grid(ctx, npix, nb), 256, 0, st>>>(npix, pp, ap, rr, pap, bb, tol2, delta, r, rrn);
        check_launch("cg_update");
        k_cg_dir<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, r, rr, rrn, bb, tol2, pp, padded);
        check_launch("cg_dir");
    }
    // 4. x_{k+1/2} = x_k + gamma delta; primal start max(x_{k+1/2}, 0)
    k_axpy_clamp<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, delta, (T)prm.gamma, xbar, xk1);
    check_launch("axpy");
    // 5. prox (Eq. 7) by Condat-Vu
    if (prm.unorm <= 0) {
        const int64_t ns = nb * NX * (NY / 2 + 1);
        k_absmax<T><<<rblocks(ns, 4 * ctx.num_sms), 256, 0, st>>>(ns, spec_re<T>(S, nx, ny, nb),
                                                                   (unsigned long long *)&sc[S_UNORM]);
        check_launch("absmax");
    }
    const double unorm_fixed = prm.unorm > 0 ? prm.unorm : -1.0;
    k_pd_tau<<<1, 1, 0, st>>>(sc, inv_wbar, (double)sigma, prm.gamma, unorm_fixed);
    check_launch("pd_tau");
    T *psiv = nullptr, *ubuf = nullptr;
    if (prm.basis_mask != 1u) {
        psiv = (T *)ctx.scratch("st_psiv", img);
        ubuf = (T *)ctx.scratch("st_u", img);
    }
    const unsigned gn = (unsigned)((n + 255) / 256);
    for (int it = 0; it < prm.pd_iters; ++it) {
        k_pad<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, xk1, xbar, padded);
        check_launch("pd_pad");
        conv_padded<T>(ctx, nx, ny, nb, padded, S, conv_scale, true, st);
        if (prm.basis_mask == 1u) {   // Dirac only: one fused kernel
            k_pd_dirac<T><<<row_grid(ctx, nx, 1), 256, 0, st>>>(nx, ny, nb, padded, xbar, sigma, (T)prm.gamma,
                                                                (T)prm.lambda, sc, xk1, dual);
            check_launch("pd_dirac");
            continue;
        }
        // Psi v = sum_k Psi_k v_k / sqrt(K): the first basis writes psiv, the others add to it
        for (int t = 0; t < K; ++t) {
            T *vk = dual + (size_t)t * n;
            if (bases[t] == 0) {
                k_axpy<T><<<gn, 256, 0, st>>>(n, (T)inv_sqrt_k, vk, t > 0 ? 1 : 0, psiv);
                check_launch("psi");
            } else {
                KTimer tm(ctx, "idwt", st, dwt_bytes + (t > 0 ? (double)img : 0.0), prm.nlevel);
                idwt2<T>(nx, ny, nb, prm.nlevel, wav_filter(bases[t]), vk, psiv, wa, (T)inv_sqrt_k, t > 0, st);
            }
        }
        k_pd_primal<T><<<row_grid(ctx, nx, nb), 256, 0, st>>>(nx, ny, padded, xbar, psiv, sigma, (T)prm.gamma, sc,
                                                              xk1, ubuf);
        check_launch("pd_primal");
        // v_k = proj(v_k + Psi_k^dagger (2 x~ - x) / sqrt(K))
        for (int t = 0; t < K; ++t) {
            const T *c = ubuf;
            if (bases[t] != 0) {
                KTimer tm(ctx, "dwt", st, dwt_bytes, prm.nlevel);
                dwt2<T>(nx, ny, nb, prm.nlevel, wav_filter(bases[t]), ubuf, wa, wb, st);
                c = wa;
            }
            k_pd_dual<T><<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(npix, nb, c, (T)inv_sqrt_k,
                                                                        (T)prm.lambda, dual + (size_t)t * n);
            check_launch("pd_dual");
        }
    }
    // 6. statistics and output
    k_finish<T><<<band_grid(ctx, npix, nb), 256, 0, st>>>(npix, xk1, x, sc);
    check_launch("finish");
    if (stats_h) {
        std::vector<double> h(nsc);
        PFB_CUDA(cudaMemcpyAsync(h.data(), sc, nsc * sizeof(double), cudaMemcpyDeviceToHost, st));
        PFB_CUDA(cudaStreamSynchronize(st));
        const double fx = 0.5 * h[S_XHX] - h[S_XD];
        stats_h[0] = fx + prm.lambda * h[S_L21];
        stats_h[1] = h[S_X2] > 0 ? std::sqrt(h[S_DX2] / h[S_X2]) : 0.0;
        double cgr = 0;
        for (int b = 0; b < nb; ++b) {
            const double rrl = h[S_COUNT + nb + (size_t)iters * nb + b];
            const double bbv = h[S_COUNT + b];
            cgr = std::max(cgr, bbv > 0 ? std::sqrt(rrl / bbv) : 0.0);
        }
        stats_h[2] = cgr;
    }
}

// ------------------------------------------------------------------ step-size bound
// 0.5 + u_e, u_e in [0, 1) from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) of the counter e + 1: the start
// vector of the step-size bound (a generic positive image)
template <typename T>
__global__ void k_bound_start(int64_t n, T *__restrict__ y) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    uint64_t z = ((uint64_t)e + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    y[e] = (T)(0.5 + (double)(z >> 11) * 0x1.0p-53);
}

template <typename T>
__global__ void k_sumsq(int64_t n, const T *__restrict__ x, double *__restrict__ out) {
    Acc<T> acc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        acc.add_prod(x[e], x[e]);
    block_sum_atomic(acc.value(), out);
}

// L_U = lambda_max(U^-1 H) in the step's normalised units (H, I^psf divided by wbar; U of Eq. 8), by
// power iteration: rho_k = z^T H z / z^T U z (a lower bound of L_U), z <- CG(U, H z) / ||.|| with
// cg_iters iterations per band, from z0 (0.5 + a SplitMix64 uniform per pixel when NULL).  Returns max_k rho_k.  Forward-backward in the
// metric U (Eqs. 6-7) converges for gamma < 2 / L_U.  The CG runs on -H z / wbar (the residual kernel
// with a zero dirty image), which flips the sign of z from one iteration to the next: rho is unchanged.
template <typename T>
double op_step_bound(Ctx &ctx, const Plan &p, const T *wgt, const T *psf, const double *wsum_h, double sigma_d,
                     int iters, int cg_iters, const T *z0, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, nb = p.nband;
    const int64_t npix = (int64_t)nx * ny, n = npix * nb;
    const int64_t NX = 2 * nx, NY = 2 * ny, nbig = nb * NX * NY;
    double wbar = 0;
    for (int b = 0; b < nb; ++b) wbar += wsum_h[b];
    wbar /= nb;
    PFB_REQUIRE(wbar > 0, "weight sums must be positive");
    const double inv_wbar = 1.0 / wbar;
    const size_t img = (size_t)n * sizeof(T);
    T *z = (T *)ctx.scratch("sb_z", img);
    T *hz = (T *)ctx.scratch("st_hx", img);
    T *zero = (T *)ctx.scratch("sb_zero", img);
    T *rhs = (T *)ctx.scratch("st_ir", img);
    T *delta = (T *)ctx.scratch("st_delta", img);
    T *r = (T *)ctx.scratch("st_r", img);
    T *pp = (T *)ctx.scratch("st_p", img);
    T *ap = (T *)ctx.scratch("st_ap", img);
    const int ci = std::max(0, cg_iters);
    const size_t nsc = S_COUNT + nb + (size_t)(ci + 1) * nb + (size_t)ci * nb + nb + 1;
    double *sc = (double *)ctx.scratch("sb_scal", nsc * sizeof(double));
    double *bb = sc + S_COUNT, *RR = bb + nb, *PAP = RR + (size_t)(ci + 1) * nb, *DEN = PAP + (size_t)ci * nb;
    double *NRM = DEN + nb;
    cx_t<T> *S = psf_spectrum<T>(ctx, nx, ny, nb, psf, st);
    T *padded = (T *)ctx.scratch("img_pad", (size_t)nbig * sizeof(T));
    ctx.scratch("img_spec", (size_t)nb * NX * (NY / 2 + 1) * sizeof(cx_t<T>));
    ctx.fft((int)NX, (int)NY, nb, RFft<T>::c2r);
    cx_t<T> *vis = (cx_t<T> *)ctx.scratch("st_vis", (size_t)p.nrow * p.nchan * sizeof(cx_t<T>));
    const unsigned gn = (unsigned)((n + 255) / 256);
    PFB_CUDA(cudaMemsetAsync(zero, 0, img, st));
    if (z0) {
        PFB_CUDA(cudaMemcpyAsync(z, z0, img, cudaMemcpyDeviceToDevice, st));
    } else {
        k_bound_start<T><<<gn, 256, 0, st>>>(n, z);
        check_launch("bound_start");
    }
    const T conv_scale = (T)(inv_wbar / (double)(NX * NY));
    const T sigma = (T)sigma_d;
    double best = 0;
    std::vector<double> h(nsc);
    for (int it = 0; it < iters; ++it) {
        PFB_CUDA(cudaMemsetAsync(sc, 0, nsc * sizeof(double), st));
        op_hessian<T>(ctx, p, z, wgt, vis, hz, st);
        // numerator z . H z / wbar (into S_XHX) and the CG right-hand side -H z / wbar with its norms
        k_residual<T><<<band_grid(ctx, npix, nb), 256, 0, st>>>(npix, zero, hz, z, inv_wbar, rhs, sc, bb);
        check_launch("sb_residual");
        // denominator z . U z
        k_pad<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, z, (const T *)nullptr, padded);
        check_launch("sb_pad");
        conv_padded<T>(ctx, nx, ny, nb, padded, S, conv_scale, true, st);
        k_cg_ap<T><<<row_grid(ctx, nx, nb), 256, 0, st>>>(nx, ny, padded, z, sigma, ap, DEN);
        check_launch("sb_uz");
        // CG for U delta = -H z / wbar
        k_cg_init<T><<<gn, 256, 0, st>>>(n, rhs, delta, r, pp);
        check_launch("sb_cg_init");
        PFB_CUDA(cudaMemcpyAsync(RR, bb, nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
        k_pad<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, pp, (const T *)nullptr, padded);
        check_launch("sb_cg_pad");
        for (int c = 0; c < ci; ++c) {
            double *rr = RR + (size_t)c * nb, *rrn = RR + (size_t)(c + 1) * nb, *pap = PAP + (size_t)c * nb;
            conv_padded<T>(ctx, nx, ny, nb, padded, S, conv_scale, true, st);
            k_cg_ap<T><<<row_grid(ctx, nx, nb), 256, 0, st>>>(nx, ny, padded, pp, sigma, ap, pap);
            check_launch("sb_cg_ap");
            k_cg_update<T><<<band_grid(ctx, npix, nb), 256, 0, st>>>(npix, pp, ap, rr, pap, bb, 0.0, delta, r, rrn);
            check_launch("sb_cg_update");
            k_cg_dir<T><<<row_grid(ctx, 2 * nx, nb), 256, 0, st>>>(nx, ny, r, rr, rrn, bb, 0.0, pp, padded);
            check_launch("sb_cg_dir");
        }
        k_sumsq<T><<<rblocks(n, 8 * ctx.num_sms), 256, 0, st>>>(n, delta, NRM);
        check_launch("sb_norm");
        PFB_CUDA(cudaMemcpyAsync(h.data(), sc, nsc * sizeof(double), cudaMemcpyDeviceToHost, st));
        PFB_CUDA(cudaStreamSynchronize(st));
        double den = 0;
        for (int b = 0; b < nb; ++b) den += h[S_COUNT + nb + (size_t)(ci + 1) * nb + (size_t)ci * nb + b];
        const double num = h[S_XHX], nrm2 = h[nsc - 1];
        if (den > 0) best = std::max(best, num / den);
        if (!(nrm2 > 0)) break;
        k_axpy<T><<<gn, 256, 0, st>>>(n, (T)(1.0 / std::sqrt(nrm2)), delta, 0, z);
        check_launch("sb_scale");
    }
    return best;
}

template void op_psf_conv<float>(Ctx &, int, int, int, const float *, const float *, float *, cudaStream_t);
template void op_psf_conv<double>(Ctx &, int, int, int, const double *, const double *, double *, cudaStream_t);
template void op_step<float>(Ctx &, const Plan &, const pfb_params &, const float *, const float *, const float *,
                             const double *, float *, float *, double *, cudaStream_t);
template void op_step<double>(Ctx &, const Plan &, const pfb_params &, const double *, const double *,
                              const double *, const double *, double *, double *, double *, cudaStream_t);

}  // namespace pfb

namespace pfb {
template double op_step_bound<float>(Ctx &, const Plan &, const float *, const float *, const double *, double, int,
                                     int, const float *, cudaStream_t);
template double op_step_bound<double>(Ctx &, const Plan &, const double *, const double *, const double *, double,
                                      int, int, const double *, cudaStream_t);
}  // namespace pfb
