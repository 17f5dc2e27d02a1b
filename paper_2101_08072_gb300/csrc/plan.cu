// Plan construction: kernel parameters from epsilon, w-stack geometry, the
// device sort of visibilities into (band, uv tile, w bucket) keys, pixel
// correction tables and the gridding work list.
//
// The operator is the wide-field measurement equation of Section 2 (Eq. 1),
// evaluated as a 2-D non-uniform FFT per imaging band with w-stacking (the
// "correction that accounts for wide field effects" of Section 2, following the
// w-stacking scheme of Arras et al. 2021, cited there).  With
//   x_u = u dl N_u,  x_v = v dm N_v   (grid cells),
//   t   = n - 1 - t_c                 (t_c: centre of n - 1 over the image),
//   w_k = w0 + k dw                   (w-planes),
// and the exponential-of-semicircle kernel phi with Fourier transform psihat,
// Poisson summation gives, for |p/N_u| <= 1/(2 sigma) and |dw t| <= 1/(2 sigma),
//   exp(-2 pi i x_u p / N_u) ~ psihat(p/N_u)^-1 sum_g phi(x_u - g) exp(-2 pi i g p / N_u)
//   exp(-2 pi i w t)         ~ psihat(dw t)^-1 sum_k phi((w - w_k)/dw) exp(-2 pi i w_k t)
// so that R x = exp(-2 pi i w t_c) sum_k phi_w sum_g phi_u phi_v G_k[g] with
// G_k = FFT2[x / (n psihat_u psihat_v psihat_w) exp(-2 pi i w_k t)] (zero padded).
#include "ctx.cuh"

#include <algorithm>
#include <numeric>

namespace pfb {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// psihat(xi) = int_{-W/2}^{W/2} phi(z) cos(2 pi xi z) dz, evaluated with the
// substitution z = (W/2) sin(theta), which removes the square-root edge of phi.
struct EsTransform {
    int W;
    double beta;
    std::vector<double> th, wt;
    EsTransform(int W_, double beta_, int nodes = 200) : W(W_), beta(beta_) {
        std::vector<double> x, w;
        gauss_legendre(nodes, x, w);
        th.resize(x.size());
        wt.resize(x.size());
        for (size_t i = 0; i < x.size(); ++i) {
            double t = 0.5 * M_PI * x[i];
            th[i] = t;
            wt[i] = 0.5 * M_PI * w[i] * 0.5 * W * std::cos(t) * std::exp(beta * (std::cos(t) - 1.0));
        }
    }
    double operator()(double xi) const {
        double s = 0;
        for (size_t i = 0; i < th.size(); ++i) s += wt[i] * std::cos(2.0 * M_PI * xi * 0.5 * W * std::sin(th[i]));
        return s;
    }
};

// ------------------------------------------------------------------ kernel parameters
// With oversampling 2 the correction psihat(xi)^-1 is applied for |xi| <= 1/4
// (uv: |p / N| <= nx / (2 N); w: |dw t| <= 1/4 by the choice of dw), and the
// Poisson-summation aliases psihat(xi + m), m != 0, are the approximation error.
// For each support W the shape parameter beta is chosen to minimise the
// worst-case aliasing ratio  max_{|xi| <= 1/4} sum_{m = +-1, +-2} |psihat(xi + m)| / psihat(xi),
// and W is the smallest support whose ratio is <= epsilon.
struct KernelChoice {
    int W;
    double beta, err;
};

static const std::vector<KernelChoice> &kernel_table() {
    static const std::vector<KernelChoice> tab = [] {
        std::vector<KernelChoice> t;
        for (int W = 4; W <= MAX_W; ++W) {
            KernelChoice best{W, 2.3 * W, 1e300};
            for (int k = 0; k <= 8; ++k) {
                const double beta = (2.0 + 0.05 * k) * W;
                EsTransform es(W, beta);
                double worst = 0;
                for (int i = 0; i <= 25; ++i) {
                    const double xi = 0.25 * i / 25.0;
                    double a = 0;
                    for (int m : {-2, -1, 1, 2}) a += std::fabs(es(xi + m));
                    worst = std::max(worst, a / es(xi));
                }
                if (worst < best.err) best = {W, beta, worst};
            }
            t.push_back(best);
        }
        return t;
    }();
    return tab;
}

int kernel_support(double eps) {
    for (const auto &k : kernel_table())
        if (k.err <= eps) return k.W;
    return MAX_W;
}

static double es_beta(int W) { return kernel_table()[W - 4].beta; }

// Smallest n >= lo that is a multiple of TILE and has no prime factor above 7.
static int good_size(int lo) {
    for (int n = ((lo + TILE - 1) / TILE) * TILE;; n += TILE) {
        int m = n;
        for (int f : {2, 3, 5, 7})
            while (m % f == 0) m /= f;
        if (m == 1) return n;
    }
}

// ------------------------------------------------------------------ device kernels
__global__ void k_w_range(const double *__restrict__ uvw, int64_t nrow, unsigned long long *out) {
    // out[0]: bits of max |w|, out[1]: bits of min |w|, out[2]: non-finite flag.
    // Non-negative doubles order like their bit patterns.
    double mx = 0.0, mn = INFINITY;
    unsigned long long nb = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow;
         r += (int64_t)gridDim.x * blockDim.x) {
        double u = uvw[3 * r], v = uvw[3 * r + 1], w = uvw[3 * r + 2];
        if (!isfinite(u) || !isfinite(v) || !isfinite(w)) { nb = 1; continue; }
        double a = fabs(w);
        mx = fmax(mx, a);
        mn = fmin(mn, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        nb |= __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(mx));
        atomicMin(&out[1], (unsigned long long)__double_as_longlong(mn));
        if (nb) atomicOr(&out[2], 1ull);
    }
}

// Count (SCATTER = false) or place (SCATTER = true) the gridding items of every
// visibility: its home tile (the tile of its first tap) and each neighbouring
// tile its W x W footprint spills into.  Lanes with equal keys are aggregated so
// that one atomic serves the whole group.
template <typename T, bool SCATTER>
__global__ void k_bucket(CoordSrc src, const int *__restrict__ band, int64_t nvis, int nchan,
                         const BandGeom *__restrict__ bgs, int halo, int *__restrict__ counts,
                         const int64_t *__restrict__ off, uint32_t *__restrict__ items) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nvis;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vis = base + threadIdx.x;
        long long keys[4] = {-1, -1, -1, -1};
        uint32_t code = 0;
        if (vis < nvis) {
            const int64_t row = vis / nchan;
            const int ch = (int)(vis - row * nchan);
            const BandGeom g = bgs[band[ch]];
            const VisCoord<T> c = vis_coord<T>(src, row, ch, g);
            const int tu = c.gu0 / TILE, tv = c.gv0 / TILE;
            // spill copies into the tiles the footprint crosses (none on halo plans)
            const bool su = !halo && c.gu0 - tu * TILE + g.W - 1 >= TILE;
            const bool sv = !halo && c.gv0 - tv * TILE + g.W - 1 >= TILE;
            const int tu1 = tu + 1 == g.ntu ? 0 : tu + 1, tv1 = tv + 1 == g.ntv ? 0 : tv + 1;
            const int kq = c.k0 / g.q;
            const long long bt = (long long)g.band * g.ntu * g.ntv;
            keys[0] = ((bt + (long long)tu * g.ntv + tv) * g.nkq + kq);
            if (su) keys[1] = ((bt + (long long)tu1 * g.ntv + tv) * g.nkq + kq);
            if (sv) keys[2] = ((bt + (long long)tu * g.ntv + tv1) * g.nkq + kq);
            if (su && sv) keys[3] = ((bt + (long long)tu1 * g.ntv + tv1) * g.nkq + kq);
            code = (uint32_t)vis;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long k = keys[e];
            const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)k);
            if (k >= 0) {
                const int leader = __ffs(peers) - 1;
                const int rank = __popc(peers & ((1u << lane) - 1u));
                int pos = 0;
                if (lane == leader) pos = atomicAdd(&counts[k], __popc(peers));
                pos = __shfl_sync(peers, pos, leader);
                if (SCATTER) {
                    const uint32_t du = (e == 1 || e == 3) ? 1u : 0u, dv = (e == 2 || e == 3) ? 1u : 0u;
                    items[off[k] + pos + rank] = code | (du << 30) | (dv << 31);
                }
            }
        }
    }
}

// ---- exclusive scan of int counts into int64 offsets (three passes, recursive on block sums)
constexpr int SCAN_T = 256, SCAN_E = 8, SCAN_CHUNK = SCAN_T * SCAN_E;

template <typename In>
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_sums[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < SCAN_T / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_T / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int64_t prefix = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[SCAN_T / 32 - 1];
    __syncthreads();
    return prefix + x - v;
}

template <typename In>
__global__ void k_scan_sums(const In *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_E;
    int64_t s = 0;
    for (int e = 0; e < SCAN_E; ++e)
        if (base + e < n) s += (int64_t)in[base + e];
    int64_t total;
    block_exclusive_scan<In>(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename In>
__global__ void k_scan_apply(const In *__restrict__ in, int64_t n, const int64_t *__restrict__ block_off,
                             int64_t *__restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_E;
    int64_t v[SCAN_E];
    int64_t s = 0;
    for (int e = 0; e < SCAN_E; ++e) {
        v[e] = base + e < n ? (int64_t)in[base + e] : 0;
        s += v[e];
    }
    int64_t total;
    int64_t run = block_exclusive_scan<In>(s, &total) + block_off[blockIdx.x];
    for (int e = 0; e < SCAN_E; ++e) {
        if (base + e < n) out[base + e] = run;
        run += v[e];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_T - 1) out[n] = run;
}

// out[0..n] = exclusive prefix sums of in[0..n-1] (out[n] = total).  tmp: scratch.
template <typename In>
static void exclusive_scan(Ctx &ctx, const In *in, int64_t n, int64_t *out, cudaStream_t st, int depth = 0) {
    int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nb == 0) {
        PFB_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return;
    }
    std::string nm = "scan" + std::to_string(depth);
    int64_t *sums = (int64_t *)ctx.scratch(nm + "a", (size_t)nb * sizeof(int64_t));
    int64_t *boff = (int64_t *)ctx.scratch(nm + "b", (size_t)(nb + 1) * sizeof(int64_t));
    k_scan_sums<In><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, sums);
    check_launch("scan_sums");
    if (nb == 1) {
        PFB_CUDA(cudaMemsetAsync(boff, 0, sizeof(int64_t), st));
    } else {
        exclusive_scan<int64_t>(ctx, sums, nb, boff, st, depth + 1);
    }
    k_scan_apply<In><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, boff, out);
    check_launch("scan_apply");
}

// Second-level sort of every (tile, w bucket) item list by the local first-tap
// cell (lu, lv) in [-TILE, TILE)^2 (spill copies have negative local indices).
// Items that start on the same cell then sit next to each other, so the gridding
// kernel's per-thread accumulators rarely change cell.  One CTA per (band, tile):
// a shared-memory histogram and scan per bucket, a scatter into tmp and a copy back.
// first-tap cell of the item relative to its tile (4 TILE^2 positions: home and spill copies), home
// items first, cells along a Hilbert curve (neighbouring cells stay close in the order, so the register
// runs of the gridding consumers break less often than in row order):
//   bin = spill * 4 TILE^2 + hilbert(lu + TILE, lv + TILE)
constexpr int FINE_BINS = 8 * TILE * TILE;

// position of (x, y) along the Hilbert curve that fills an n x n grid (n a power of two): at each scale
// s the quadrant contributes s^2 times its rank (0, 1, 2, 3 along the curve), and the remaining
// coordinates are reflected and transposed into that quadrant's orientation
__device__ __forceinline__ int hilbert_index(int n, int x, int y) {
    int d = 0;
    for (int s = n >> 1; s > 0; s >>= 1) {
        const int rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
        d += s * s * ((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            const int t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// bucket keys (band x tile x w bucket) a plan may use; beyond it w planes are grouped q to a bucket
#ifndef PFB_KEY_CAP_LOG2
#define PFB_KEY_CAP_LOG2 27
#endif

template <typename T>
__global__ void __launch_bounds__(256) k_fine_sort(CoordSrc src, const int64_t *__restrict__ off, int ntiles,
                                                   int nkq, const BandGeom *__restrict__ bgs, int nchan,
                                                   uint32_t *__restrict__ items, uint32_t *__restrict__ tmp) {
    __shared__ int hist[FINE_BINS];
    const int bt = blockIdx.x;                 // band * ntiles + tile
    const int band = bt / ntiles;
    const BandGeom g = bgs[band];
    auto key_of = [&](uint32_t code) {
        const uint32_t v = code & VIS_MASK;
        const int du = (code >> 30) & 1, dv = code >> 31;
        const uint32_t row = v / (uint32_t)nchan;
        const int ch = (int)(v - row * (uint32_t)nchan);
        const VisCoord<T> c = vis_coord<T>(src, row, ch, g);
        const int lu = (c.gu0 & (TILE - 1)) - du * TILE + TILE;
        const int lv = (c.gv0 & (TILE - 1)) - dv * TILE + TILE;
        return ((du | dv) ? 4 * TILE * TILE : 0) + hilbert_index(2 * TILE, lu, lv);
    };
    for (int kq = 0; kq < nkq; ++kq) {
        const int64_t s = off[(int64_t)bt * nkq + kq], e = off[(int64_t)bt * nkq + kq + 1];
        if (e - s < 2) continue;
        for (int i = threadIdx.x; i < FINE_BINS; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&hist[key_of(items[i])], 1);
        __syncthreads();
        // exclusive scan of hist (FINE_BINS / 256 per thread, then across threads)
        {
            constexpr int PER = FINE_BINS / 256;
            __shared__ int part[256];
            int loc[PER], sum = 0;
            for (int j = 0; j < PER; ++j) {
                loc[j] = hist[threadIdx.x * PER + j];
                sum += loc[j];
            }
            part[threadIdx.x] = sum;
            __syncthreads();
            if (threadIdx.x == 0) {
                int run = 0;
                for (int t = 0; t < 256; ++t) {
                    const int x = part[t];
                    part[t] = run;
                    run += x;
                }
            }
            __syncthreads();
            int run = part[threadIdx.x];
            for (int j = 0; j < PER; ++j) {
                hist[threadIdx.x * PER + j] = run;
                run += loc[j];
            }
        }
        __syncthreads();
        for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
            const uint32_t code = items[i];
            tmp[s + atomicAdd(&hist[key_of(code)], 1)] = code;
        }
        __syncthreads();
        for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) items[i] = tmp[i];
        __syncthreads();
    }
}

// uvw (FP64) -> double-float pairs (hi, lo) for the FP32 path
__global__ void k_split_uvw(const double *__restrict__ uvw, int64_t n, float2 *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = uvw[i];
    const float hi = (float)v;
    out[i] = make_float2(hi, (float)(v - (double)hi));
}

static void split_df(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__global__ void k_tile_begin(const int64_t *__restrict__ off, int64_t ntb, int nkq, int64_t *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i <= ntb) out[i] = off[i * nkq];
}

// Per-pixel tables: t = n - 1 - t_c (FP64) and the correction
// 1 / (n psihat_u psihat_v psihat_w(dw t)) in the working precision.
template <typename T>
__global__ void k_pixel_tables(int nx, int ny, double dl, double dm, double l0, double m0, double fa, double fb,
                               uint32_t flags, double tc, double dw,
                               int wstack, const double *__restrict__ psiu, const double *__restrict__ psiv,
                               const double *__restrict__ tab, int M, double xi0, double inv_h,
                               double *__restrict__ tp, T *__restrict__ corr) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= (int64_t)nx * ny) return;
    int i = (int)(p / ny), j = (int)(p - (int64_t)i * ny);
    const double dli = (i - nx / 2) * dl, dmj = (j - ny / 2) * dm;
    double l = l0 + dli, m = m0 + dmj;
    double r2 = l * l + m * m;
    double n = sqrt(1.0 - r2);
    double nm1 = (flags & PFB_NO_WTERM) ? 0.0 : -r2 / (1.0 + n) - fa * dli - fb * dmj;
    double t = nm1 - tc;
    double c = psiu[i] * psiv[j];
    if (!(flags & PFB_NO_DIVIDE_BY_N)) c *= n;
    if (wstack) {
        double s = (dw * t - xi0) * inv_h;
        int k = (int)floor(s);
        k = k < 1 ? 1 : (k > M - 3 ? M - 3 : k);
        double f = s - k;
        // cubic Lagrange through tab[k-1..k+2]
        double a0 = -f * (f - 1.0) * (f - 2.0) / 6.0;
        double a1 = (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0;
        double a2 = -(f + 1.0) * f * (f - 2.0) / 2.0;
        double a3 = (f + 1.0) * f * (f - 1.0) / 6.0;
        c *= a0 * tab[k - 1] + a1 * tab[k] + a2 * tab[k + 1] + a3 * tab[k + 2];
    }
    if constexpr (sizeof(T) == 4) {   // FP32 plans: t as an unevaluated float pair
        const float hi = (float)t;
        reinterpret_cast<float2 *>(tp)[p] = make_float2(hi, (float)(t - (double)hi));
    } else {
        tp[p] = t;
    }
    corr[p] = (T)(1.0 / c);
}

// ------------------------------------------------------------------ plan building
static void build_plan(Ctx &ctx, Plan &p, const double *uvw, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny;
    // ---- w range over rows (and a finiteness check)
    {
        unsigned long long *d = (unsigned long long *)ctx.scratch("wrange", 3 * sizeof(unsigned long long));
        const double zero_d = 0.0, inf_d = INFINITY;
        unsigned long long init[3] = {0ull, 0ull, 0ull};
        std::memcpy(&init[0], &zero_d, 8);
        std::memcpy(&init[1], &inf_d, 8);
        PFB_CUDA(cudaMemcpyAsync(d, init, sizeof(init), cudaMemcpyHostToDevice, st));
        int blocks = (int)std::min<int64_t>((p.nrow + 255) / 256, 4 * ctx.num_sms);
        k_w_range<<<std::max(blocks, 1), 256, 0, st>>>(uvw, p.nrow, d);
        check_launch("w_range");
        unsigned long long hb[3];
        PFB_CUDA(cudaMemcpyAsync(hb, d, sizeof(hb), cudaMemcpyDeviceToHost, st));
        PFB_CUDA(cudaStreamSynchronize(st));
        PFB_REQUIRE(hb[2] == 0, "uvw contains non-finite values");
        double h[2];
        std::memcpy(&h[0], &hb[0], 8);
        std::memcpy(&h[1], &hb[1], 8);
        double wmax = h[0], wmin = h[1];
        if (!(wmin <= wmax)) wmin = wmax = 0.0;
        // ---- geometry of the image: range of t = n - 1 - fa dl - fb dm over the pixels, where
        // (dl, dm) is the offset from the image centre (l0, m0) and (fa, fb) = grad n there.
        // t is concave with its maximum n0 - 1 at the centre, so its minimum is at a corner.
        const bool nowterm = p.flags & PFB_NO_WTERM;
        const double r20 = p.l0 * p.l0 + p.m0 * p.m0;
        PFB_REQUIRE(r20 < 1.0, "image centre beyond the horizon (l0^2 + m0^2 >= 1)");
        const double n0 = std::sqrt(1.0 - r20);
        p.fa = nowterm ? 0.0 : -p.l0 / n0;
        p.fb = nowterm ? 0.0 : -p.m0 / n0;
        auto t_at = [&](double dl_, double dm_) {
            const double l = p.l0 + dl_, m = p.m0 + dm_, r2 = l * l + m * m;
            PFB_REQUIRE(r2 < 1.0, "field of view reaches the horizon (l^2 + m^2 >= 1)");
            return -r2 / (1.0 + std::sqrt(1.0 - r2)) - p.fa * dl_ - p.fb * dm_;
        };
        const double tmax = -r20 / (1.0 + n0);
        double tmin = tmax;
        for (int ci : {-(nx / 2), nx - 1 - nx / 2})
            for (int cj : {-(ny / 2), ny - 1 - ny / 2}) tmin = std::min(tmin, t_at(ci * p.dl, cj * p.dm));
        p.tc = nowterm ? 0.0 : 0.5 * (tmin + tmax);
        p.Thalf = nowterm ? 0.0 : 0.5 * (tmax - tmin);
        p.wstack = !nowterm && p.Thalf > 0.0;
        p.Ww = p.wstack ? p.W : 1;
        p.dw = p.wstack ? 1.0 / (4.0 * p.Thalf) : 0.0;   // dw * max|t| = 1/(2 sigma), sigma = 2
        p.w0.assign(p.nband, 0.0);
        p.wlo.assign(p.nband, 0.0);
        p.whi.assign(p.nband, 0.0);
        p.P.assign(p.nband, 1);
        p.Pmax = 1;
        for (int b = 0; b < p.nband; ++b) {
            double fmin = INFINITY, fmax = 0;
            for (int c = 0; c < p.nchan; ++c)
                if (p.band_h[c] == b) {
                    fmin = std::min(fmin, p.scale[c]);
                    fmax = std::max(fmax, p.scale[c]);
                }
            if (!(fmin <= fmax)) fmin = fmax = 0.0;
            p.wlo[b] = wmin * fmin;
            p.whi[b] = wmax * fmax;
            if (p.wstack) {
                p.w0[b] = p.wlo[b] - 0.5 * p.W * p.dw;
                double zmax = (p.whi[b] - p.w0[b]) / p.dw;
                p.P[b] = (int)std::ceil(zmax - 0.5 * p.W) + p.W;
            }
            p.Pmax = std::max(p.Pmax, p.P[b]);
        }
    }
    // ---- grid and tiles
    p.ntu = p.Nu / TILE;
    p.ntv = p.Nv / TILE;
    const int64_t ntiles = (int64_t)p.ntu * p.ntv;
    const int64_t key_cap = int64_t(1) << PFB_KEY_CAP_LOG2;   // 1 GiB of bucket offsets at most
    p.q = 1;
    while ((int64_t)p.nband * ntiles * ((p.Pmax + p.q - 1) / p.q) > key_cap) ++p.q;
    p.nkq = (p.Pmax + p.q - 1) / p.q;
    p.nkeys = (int64_t)p.nband * ntiles * p.nkq;
    const size_t cxs = p.prec == PFB_F64 ? 16 : 8;
    PFB_REQUIRE((size_t)(p.Ww + p.q - 1) * TILE * TILE * cxs <= 227 * 1024,
                "w-plane ring of the gridding kernel exceeds shared memory (reduce epsilon demands or image size)");
    p.halo = halo_fits(p);

    // ---- device copies of per-channel data and band geometry
    p.d_scale = (double *)ctx.dalloc(p.nchan * sizeof(double));
    p.d_band = (int *)ctx.dalloc(p.nchan * sizeof(int));
    p.d_bg = (BandGeom *)ctx.dalloc(p.nband * sizeof(BandGeom));
    p.d_chandf = (ChanDF *)ctx.dalloc(p.nchan * sizeof(ChanDF));
    p.bytes += p.nchan * (sizeof(double) + sizeof(int) + sizeof(ChanDF)) + p.nband * sizeof(BandGeom);
    std::vector<BandGeom> bgs(p.nband);
    for (int b = 0; b < p.nband; ++b) bgs[b] = p.geom(b);
    std::vector<ChanDF> cdf(p.nchan);
    for (int c = 0; c < p.nchan; ++c) {
        split_df(p.scale[c] * p.dl * p.Nu, cdf[c].su_hi, cdf[c].su_lo);
        split_df(p.scale[c] * p.dm * p.Nv, cdf[c].sv_hi, cdf[c].sv_lo);
        split_df(p.wstack ? p.scale[c] / p.dw : 0.0, cdf[c].sw_hi, cdf[c].sw_lo);
        split_df(p.scale[c] * p.tc, cdf[c].sp_hi, cdf[c].sp_lo);
        split_df(p.scale[c] * p.fa * p.dl * p.Nu, cdf[c].sa_hi, cdf[c].sa_lo);
        split_df(p.scale[c] * p.fb * p.dm * p.Nv, cdf[c].sb_hi, cdf[c].sb_lo);
        split_df(p.scale[c] * p.l0, cdf[c].sl_hi, cdf[c].sl_lo);
        split_df(p.scale[c] * p.m0, cdf[c].sm_hi, cdf[c].sm_lo);
    }
    PFB_CUDA(cudaMemcpyAsync(p.d_scale, p.scale.data(), p.nchan * sizeof(double), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(p.d_band, p.band_h.data(), p.nchan * sizeof(int), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(p.d_bg, bgs.data(), p.nband * sizeof(BandGeom), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(p.d_chandf, cdf.data(), p.nchan * sizeof(ChanDF), cudaMemcpyHostToDevice, st));
    if (p.prec == PFB_F32) {
        p.d_rowdf = (float2 *)ctx.dalloc((size_t)p.nrow * 3 * sizeof(float2));
        p.bytes += (size_t)p.nrow * 3 * sizeof(float2);
        const int64_t n3 = p.nrow * 3;
        k_split_uvw<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(uvw, n3, p.d_rowdf);
        check_launch("split_uvw");
    }

    // ---- counting sort of gridding items by key
    const int64_t nvis = p.nrow * (int64_t)p.nchan;
    int *counts = (int *)ctx.scratch("counts", (size_t)p.nkeys * sizeof(int));
    PFB_CUDA(cudaMemsetAsync(counts, 0, (size_t)p.nkeys * sizeof(int), st));
    p.d_off = (int64_t *)ctx.dalloc((size_t)(p.nkeys + 1) * sizeof(int64_t));
    p.bytes += (size_t)(p.nkeys + 1) * sizeof(int64_t);
    const int bblocks = (int)std::max<int64_t>(1, std::min<int64_t>((nvis + 255) / 256, 32 * ctx.num_sms));
    if (p.prec == PFB_F64)
        k_bucket<double, false><<<bblocks, 256, 0, st>>>(p.coords(), p.d_band, nvis, p.nchan, p.d_bg, p.halo, counts,
                                                         nullptr, nullptr);
    else
        k_bucket<float, false><<<bblocks, 256, 0, st>>>(p.coords(), p.d_band, nvis, p.nchan, p.d_bg, p.halo, counts,
                                                        nullptr, nullptr);
    check_launch("bucket_count");
    exclusive_scan<int>(ctx, counts, p.nkeys, p.d_off, st);
    PFB_CUDA(cudaMemcpyAsync(&p.nitems, p.d_off + p.nkeys, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PFB_CUDA(cudaStreamSynchronize(st));
    p.d_items = (uint32_t *)ctx.dalloc((size_t)std::max<int64_t>(p.nitems, 1) * sizeof(uint32_t));
    p.bytes += (size_t)std::max<int64_t>(p.nitems, 1) * sizeof(uint32_t);
    PFB_CUDA(cudaMemsetAsync(counts, 0, (size_t)p.nkeys * sizeof(int), st));
    if (p.prec == PFB_F64)
        k_bucket<double, true><<<bblocks, 256, 0, st>>>(p.coords(), p.d_band, nvis, p.nchan, p.d_bg, p.halo, counts,
                                                        p.d_off, p.d_items);
    else
        k_bucket<float, true><<<bblocks, 256, 0, st>>>(p.coords(), p.d_band, nvis, p.nchan, p.d_bg, p.halo, counts,
                                                       p.d_off, p.d_items);
    check_launch("bucket_scatter");

    // ---- order each bucket by first-tap cell (FP32 path: feeds the register accumulators)
    if (p.prec == PFB_F32 && p.nitems > 0) {
        uint32_t *tmp = (uint32_t *)ctx.scratch("sort_tmp", (size_t)p.nitems * sizeof(uint32_t));
        k_fine_sort<float><<<(unsigned)(p.nband * ntiles), 256, 0, st>>>(p.coords(), p.d_off, (int)ntiles, p.nkq,
                                                                         p.d_bg, p.nchan, p.d_items, tmp);
        check_launch("fine_sort");
    }

    // ---- per-tile item ranges -> host -> work list
    const int64_t ntb = (int64_t)p.nband * ntiles;
    int64_t *d_tb = (int64_t *)ctx.scratch("tilebegin", (size_t)(ntb + 1) * sizeof(int64_t));
    k_tile_begin<<<(unsigned)((ntb + 1 + 255) / 256), 256, 0, st>>>(p.d_off, ntb, p.nkq, d_tb);
    check_launch("tile_begin");
    std::vector<int64_t> tb(ntb + 1);
    PFB_CUDA(cudaMemcpyAsync(tb.data(), d_tb, (ntb + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PFB_CUDA(cudaStreamSynchronize(st));
    std::vector<WorkItem> work, work_dg;
    std::vector<int> heavy;
    p.work_begin.assign(p.nband + 1, 0);
    p.work_dg_begin.assign(p.nband + 1, 0);
    p.work_heavy_end.assign(p.nband, 0);
    p.heavy_begin.assign(p.nband + 1, 0);
    p.empty_begin.assign(p.nband, 0);
    p.band_items_begin.assign(p.nband, 0);
    p.band_items_end.assign(p.nband, 0);
    for (int b = 0; b < p.nband; ++b) {
        const int64_t b0 = tb[b * ntiles], b1 = tb[(b + 1) * ntiles];
        p.band_items_begin[b] = b0;
        p.band_items_end[b] = b1;
        // tiles above `chunk` items are split into chunks of that many (heavy tiles); the gridding kernel of
        // halo plans balances best with finer chunks, the degridding kernel (which stages a tile's region per
        // chunk) with coarser ones (measured on the MeerKAT-like Hessian)
        auto chunk_of = [&](int64_t lo, int64_t per_sm) {
            return std::max<int64_t>(lo, (b1 - b0 + per_sm * ctx.num_sms - 1) / (per_sm * ctx.num_sms));
        };
        const int64_t chunk = p.halo ? chunk_of(2048, 64) : chunk_of(8192, 16);
        p.work_begin[b] = (int64_t)work.size();
        p.heavy_begin[b] = (int64_t)heavy.size();
        const int64_t *tbb = tb.data() + b * ntiles;
        auto has_items = [&](int tu, int tv) {
            const int64_t t = (int64_t)tu * p.ntv + tv;
            return tbb[t + 1] > tbb[t];
        };
        // on halo plans a tile's cells also receive the far edges of the regions of the tiles before it
        // (with wrap-around): every such tile is filled by reductions into zeroed cells
        auto reached = [&](int64_t t) {
            const int tu = (int)(t / p.ntv), tv = (int)(t - (int64_t)tu * p.ntv);
            const int pu = tu == 0 ? p.ntu - 1 : tu - 1, pv = tv == 0 ? p.ntv - 1 : tv - 1;
            return has_items(tu, tv) || has_items(pu, tv) || has_items(tu, pv) || has_items(pu, pv);
        };
        for (int64_t t = 0; t < ntiles; ++t) {
            const int64_t s = tbb[t], e = tbb[t + 1];
            if (e - s > chunk) {
                if (!p.halo) heavy.push_back((int)t);
                for (int64_t c = s; c < e; c += chunk) work.push_back({(int)t, 1, c, std::min(e, c + chunk)});
            }
        }
        p.work_heavy_end[b] = (int64_t)work.size();
        // tiles with items that one CTA takes whole, largest first (no long tile starts at the end of the
        // launch): they own their cells unless the plan is a halo plan.  Tiles that nothing writes follow
        // the reduction-filled ones in the list of tiles that a plain kernel zeroes.
        const size_t l0 = work.size();
        if (p.halo)
            for (int64_t t = 0; t < ntiles; ++t)
                if (reached(t)) heavy.push_back((int)t);
        p.empty_begin[b] = (int64_t)heavy.size();
        for (int64_t t = 0; t < ntiles; ++t) {
            const int64_t s = tbb[t], e = tbb[t + 1];
            if (p.halo ? !reached(t) : e == s) heavy.push_back((int)t);
            if (e > s && e - s <= chunk) work.push_back({(int)t, p.halo ? 1 : 0, s, e});
        }
        std::stable_sort(work.begin() + l0, work.end(), [](const WorkItem &x, const WorkItem &y) {
            return x.end - x.begin > y.end - y.begin;
        });
        // degridding's list on halo plans: heavy chunks, then whole tiles largest first
        p.work_dg_begin[b] = (int64_t)work_dg.size();
        if (p.halo) {
            const int64_t cdg = chunk_of(16384, 8);
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t s = tbb[t], e = tbb[t + 1];
                if (e - s > cdg)
                    for (int64_t c = s; c < e; c += cdg) work_dg.push_back({(int)t, 1, c, std::min(e, c + cdg)});
            }
            const size_t d0 = work_dg.size();
            for (int64_t t = 0; t < ntiles; ++t) {
                const int64_t s = tbb[t], e = tbb[t + 1];
                if (e > s && e - s <= cdg) work_dg.push_back({(int)t, 1, s, e});
            }
            std::stable_sort(work_dg.begin() + d0, work_dg.end(), [](const WorkItem &x, const WorkItem &y) {
                return x.end - x.begin > y.end - y.begin;
            });
        }
    }
    p.work_begin[p.nband] = (int64_t)work.size();
    p.work_dg_begin[p.nband] = (int64_t)work_dg.size();
    if (!work_dg.empty()) {
        p.d_work_dg = (WorkItem *)ctx.dalloc(work_dg.size() * sizeof(WorkItem));
        p.bytes += work_dg.size() * sizeof(WorkItem);
        PFB_CUDA(cudaMemcpyAsync(p.d_work_dg, work_dg.data(), work_dg.size() * sizeof(WorkItem),
                                 cudaMemcpyHostToDevice, st));
    }
    p.heavy_begin[p.nband] = (int64_t)heavy.size();
    p.d_work = (WorkItem *)ctx.dalloc(std::max<size_t>(work.size(), 1) * sizeof(WorkItem));
    p.bytes += work.size() * sizeof(WorkItem);
    if (!work.empty())
        PFB_CUDA(cudaMemcpyAsync(p.d_work, work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                 st));
    if (!heavy.empty()) {
        p.d_heavy = (int *)ctx.dalloc(heavy.size() * sizeof(int));
        p.bytes += heavy.size() * sizeof(int);
        PFB_CUDA(cudaMemcpyAsync(p.d_heavy, heavy.data(), heavy.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    }

    // ---- pixel correction tables
    EsTransform es(p.W, p.beta);
    std::vector<double> psiu(nx), psiv(ny);
    for (int i = 0; i < nx; ++i) psiu[i] = es((double)(i - nx / 2) / p.Nu);
    for (int j = 0; j < ny; ++j) psiv[j] = es((double)(j - ny / 2) / p.Nv);
    const int M = 4096;
    const double xi_max = 0.25 * 1.02;   // |dw t| <= 1/4 by the choice of dw
    std::vector<double> tab(M);
    const double h = 2.0 * xi_max / (M - 1);
    for (int k = 0; k < M; ++k) tab[k] = es(-xi_max + k * h);
    double *d_psiu = (double *)ctx.scratch("psiu", nx * sizeof(double));
    double *d_psiv = (double *)ctx.scratch("psiv", ny * sizeof(double));
    double *d_tab = (double *)ctx.scratch("psitab", M * sizeof(double));
    PFB_CUDA(cudaMemcpyAsync(d_psiu, psiu.data(), nx * sizeof(double), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(d_psiv, psiv.data(), ny * sizeof(double), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(d_tab, tab.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
    const int64_t npix = (int64_t)nx * ny;
    p.d_tp = (double *)ctx.dalloc(npix * sizeof(double));
    const size_t rs = p.prec == PFB_F64 ? 8 : 4;
    p.d_corr = ctx.dalloc(npix * rs);
    p.bytes += npix * (sizeof(double) + rs);
    const unsigned pb = (unsigned)((npix + 255) / 256);
    if (p.prec == PFB_F64)
        k_pixel_tables<double><<<pb, 256, 0, st>>>(nx, ny, p.dl, p.dm, p.l0, p.m0, p.fa, p.fb, p.flags, p.tc,
                                                   p.dw, p.wstack, d_psiu,
                                                   d_psiv, d_tab, M, -xi_max, 1.0 / h, p.d_tp,
                                                   (double *)p.d_corr);
    else
        k_pixel_tables<float><<<pb, 256, 0, st>>>(nx, ny, p.dl, p.dm, p.l0, p.m0, p.fa, p.fb, p.flags, p.tc,
                                                  p.dw, p.wstack, d_psiu,
                                                  d_psiv, d_tab, M, -xi_max, 1.0 / h, p.d_tp,
                                                  (float *)p.d_corr);
    check_launch("pixel_tables");
    build_item_records(ctx, p, st);
    build_pruned_tables(ctx, p, st);
    // the host vectors above die with this scope: wait for the copies
    PFB_CUDA(cudaStreamSynchronize(st));
    ctx.release("sort_tmp");
    ctx.release("counts");
}

Plan &get_plan(Ctx &ctx, const pfb_geom &g, int prec, int64_t nrow, int nchan, const double *uvw,
               const double *freq, const int32_t *band, bool psf_grid, cudaStream_t st) {
    const int nx = psf_grid ? 2 * g.nx : g.nx, ny = psf_grid ? 2 * g.ny : g.ny;
    const int W = kernel_support(g.epsilon);
    for (auto &pp : ctx.plans) {
        Plan &p = *pp;
        if (p.nx == nx && p.ny == ny && p.nband == g.nband && p.dl == g.dl && p.dm == g.dm && p.l0 == g.l0 &&
            p.m0 == g.m0 &&
            p.flags == (g.flags & ~PFB_ACCUMULATE) && p.prec == prec && p.W == W && p.nrow == nrow && p.nchan == nchan &&
            p.uvw == uvw && p.freq == freq && p.band == band) {
            p.last_use = ++ctx.clock;
            return p;
        }
    }
    // evict the least recently used plans beyond sixteen (a faceted image keeps one plan per facet), and
    // while the budget could not hold another plan of this size (items, records and tables)
    const size_t plan_need = (size_t)nrow * nchan * 48 + (size_t)nx * ny * 16 + (256u << 20);
    while (ctx.plans.size() >= 16 || (!ctx.plans.empty() && ctx.available() < plan_need)) {
        auto it = std::min_element(ctx.plans.begin(), ctx.plans.end(),
                                   [](const std::unique_ptr<Plan> &a, const std::unique_ptr<Plan> &b) {
                                       return a->last_use < b->last_use;
                                   });
        ctx.free_plan(**it);
        ctx.plans.erase(it);
    }
    auto pp = std::make_unique<Plan>();
    Plan &p = *pp;
    p.nx = nx; p.ny = ny; p.nband = g.nband; p.dl = g.dl; p.dm = g.dm; p.flags = g.flags & ~PFB_ACCUMULATE;
    p.prec = prec;
    p.l0 = g.l0; p.m0 = g.m0;
    p.W = W; p.beta = es_beta(W); p.nrow = nrow; p.nchan = nchan; p.uvw = uvw; p.freq = freq; p.band = band;
    PFB_REQUIRE(nrow * (int64_t)nchan < (int64_t)VIS_MASK, "more than 2^30 visibilities in one call");
    std::vector<double> fh(nchan);
    p.band_h.resize(nchan);
    PFB_CUDA(cudaMemcpyAsync(fh.data(), freq, nchan * sizeof(double), cudaMemcpyDeviceToHost, st));
    PFB_CUDA(cudaMemcpyAsync(p.band_h.data(), band, nchan * sizeof(int), cudaMemcpyDeviceToHost, st));
    PFB_CUDA(cudaStreamSynchronize(st));
    p.scale.resize(nchan);
    for (int c = 0; c < nchan; ++c) {
        PFB_REQUIRE(std::isfinite(fh[c]) && fh[c] > 0.0, "channel frequencies must be finite and positive");
        PFB_REQUIRE(p.band_h[c] >= 0 && p.band_h[c] < g.nband, "band_of_chan entry outside [0, nband)");
        p.scale[c] = fh[c] / C_LIGHT;
    }
    p.id = ++ctx.plan_serial;
    p.Nu = good_size(std::max(2 * nx, 2 * MAX_W));
    p.Nv = good_size(std::max(2 * ny, 2 * MAX_W));
    try {
        KTimer t(ctx, "plan", st, 0.0, 0);
        build_plan(ctx, p, uvw, st);
    } catch (...) {
        ctx.free_plan(p);
        throw;
    }
    p.last_use = ++ctx.clock;
    ctx.plans.push_back(std::move(pp));
    return *ctx.plans.back();
}

}  // namespace pfb
