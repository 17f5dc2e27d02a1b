// Pruned w-plane transforms of the FP32 path.
//
// R and R^dagger apply a 2-D DFT to every w-plane of a band (Section 2's w-stacking, Eqs. 1 and 3).  Two
// facts make most of that work avoidable:
//  - in image space only the image region carries data: the pixel (i, j) sits at
//    ((i - nx/2) mod Nu, (j - ny/2) mod Nv), so the forward transform's input is zero outside the image
//    rows and columns, and the inverse transform's output is needed only there;
//  - in uv space only the cells that some visibility's kernel footprint touches matter: the gridding
//    kernels leave every other cell zero, and degridding reads no other cell.  A w-plane of a wide-field
//    plan holds the visibilities of one narrow range of w, which lie along a band of the uv plane: in the
//    MeerKAT-like plan (4096^2 pixels of 1.5", 8192^2 planes) about 6% of the 32 x 32 tiles and 36% of the
//    tile-rows of a plane are touched.
// The plan records which tiles of each plane are touched (from the item counts per tile and w bucket:
// an item of bucket kq reaches planes kq q .. kq q + q + W_w - 2) and lists the (plane, tile-row) pairs
// that hold a touched tile.  Then
//   forward (degridding):
//     k_colfwd   per pair of adjacent image columns and every plane of the block: the pre-pass values
//                x corr exp(-2 pi i w_k t) at the image rows (zero at the other rows), an N-point DFT
//                along the column, and TMA stores of the occupied tile-rows only;
//     k_rowfft   per occupied row: a DFT along the row from its image columns (the rest is zero), stored
//                in the row's touched 32-cell segments only;
//   inverse (gridding):
//     k_rowfft   per occupied row: a DFT along the row from its touched segments (the rest is zero),
//                stored at the image columns only;
//     k_colinv   per image column pair and every plane: a DFT along the column from its occupied rows
//                (the other rows are zero) and the post-pass sum over planes of Re exp(+2 pi i w_k t) H_k
//                at the image rows, kept in shared memory and multiplied by the correction
//                1/(n psihat) at the end.
// The pre- and post-pass values never go through HBM, and no cell outside the touched tiles is computed
// or read.  The per-pixel inputs of the column kernels (x corr and t = n - 1 - t_c as a float pair) are
// first transposed into column-pair order, [q][i], so that the threads of a column read them coalesced;
// a column kernel re-reads its share from L2 for every plane.
//
// The DFTs are the mixed-radix Stockham stages of fftcore.cuh with N/16 threads per CTA, on pairs of complex
// values (two columns, or two rows, at once) for N <= 8192, and on single columns or rows for N = 16384,
// whose pairs would not fit in shared memory (those columns are stored per thread: a TMA box needs 16 bytes
// of inner extent).
#include "ctx.cuh"
#include "fftcore.cuh"

#include <algorithm>
#include <type_traits>

namespace pfb {
namespace {
using namespace fft;

// The Stockham stages of an N = 2^L point DFT (10 <= L <= 13) of float4 pairs held by T = N/16 threads.
// On entry v[r] = x[tid + r T].  On return thread tid holds output row d_b + r Ns in v[b RL + operm<RL>(r)]
// (b < BPT, r < RL), where j = tid + b T, d_b = (j / Ns) Ns RL + (j mod Ns) and Ns is the returned value.
// sm is the padded exchange buffer.  The function begins with a barrier (so the caller's earlier reads of
// sm are complete) and ends after its last read of sm, without a barrier.
template <int L>
struct Shape {
    static constexpr int N = 1 << L, T = N / 16;
    static constexpr int NST16 = L / 4, RL = (L % 4) ? (1 << (L % 4)) : 16, BPT = 16 / RL;
    static constexpr int NMID = NST16 - 1 - ((L % 4) ? 0 : 1);   // radix-16 stages between the first and last
};

// What one CTA transforms: E = float4, two adjacent columns (or rows) at once (transforms of up to 8192
// points); E = float2, one column (or row) (16384 points, whose pair would not fit in shared memory).
template <typename E> struct Lanes;
template <> struct Lanes<float4> {
    static constexpr int K = 2;
    using X = float2;   // x corr of the K pixels of an image row
    using Tt = float4;  // t of the K pixels (float pairs)
};
template <> struct Lanes<float2> {
    static constexpr int K = 1;
    using X = float;
    using Tt = float2;
};

template <int L, bool INV, typename E>
__device__ __forceinline__ int fft_stages(E *v, E *sm, const float2 *__restrict__ W, int tid) {
    using S = Shape<L>;
    constexpr int N = S::N, T = S::T, RL = S::RL, BPT = S::BPT;
    dft_reg<16, INV>(v);   // first stage: radix 16, Ns = 1, no twiddles
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[spad(tid * 16 + r)] = v[operm<16>(r)];
    __syncthreads();
    int Ns = 16;
#pragma unroll
    for (int s = 0; s < S::NMID; ++s) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = sm[spad(tid + r * T)];
        const int k = tid & (Ns - 1);
        apply_twiddles<16, INV>(v, W, k, N / (Ns * 16));
        dft_reg<16, INV>(v);
        __syncthreads();
        const int d = (tid / Ns) * Ns * 16 + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[spad(d + r * Ns)] = v[operm<16>(r)];
        __syncthreads();
        Ns *= 16;
    }
#pragma unroll
    for (int b = 0; b < BPT; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) v[b * RL + r] = sm[spad(tid + b * T + r * (N / RL))];
    const int step = N / (Ns * RL);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = tid + b * T, k = j & (Ns - 1);
        apply_twiddles<RL, INV>(v + b * RL, W, k, step);
        dft_reg<RL, INV>(v + b * RL);
    }
    return Ns;
}

// After fft_stages: write the outputs densely (row-major, no padding) into sm, then a barrier.
template <int L, typename E>
__device__ __forceinline__ void dense_to_smem(const E *v, E *sm, int tid, int Ns) {
    using S = Shape<L>;
    __syncthreads();   // every thread has read the exchange buffer
#pragma unroll
    for (int b = 0; b < S::BPT; ++b) {
        const int j = tid + b * S::T, k = j & (Ns - 1);
        const int d = (j / Ns) * Ns * S::RL + k;
#pragma unroll
        for (int r = 0; r < S::RL; ++r) sm[d + r * Ns] = v[b * S::RL + operm<S::RL>(r)];
    }
}

__device__ __forceinline__ bool bit_set(const uint32_t *__restrict__ words, int i) {
    return (__ldg(words + (i >> 5)) >> (i & 31)) & 1u;
}

// exp(-/+ 2 pi i w_k t) for t = (t_hi, t_lo) and w_k = (wk_hi, wk_lo): the phase frac(w_k t) in turns,
// reduced in float-float arithmetic (frac_prod_df) to [-1/2, 1/2], then evaluated by the hardware sine
// and cosine on [-pi, pi] (absolute error below 2^-21, far inside the FP32 path's epsilon).
__device__ __forceinline__ void screen(float2 wk, float t_hi, float t_lo, float *s, float *c) {
    float h, l;
    frac_prod_df(wk.x, wk.y, t_hi, t_lo, &h, &l);
    __sincosf(6.28318530717958647692f * (h + l), s, c);
}

// the pre-pass value x corr exp(-2 pi i w_k t) of the CTA's pixels of one image row
__device__ __forceinline__ float4 pre_value(float2 xc, float4 t, float2 w, int wstack) {
    if (!wstack) return make_float4(xc.x, 0.f, xc.y, 0.f);
    float s0, c0, s1, c1;
    screen(w, t.x, t.y, &s0, &c0);
    screen(w, t.z, t.w, &s1, &c1);
    return make_float4(xc.x * c0, -xc.x * s0, xc.y * c1, -xc.y * s1);
}
__device__ __forceinline__ float2 pre_value(float xc, float2 t, float2 w, int wstack) {
    if (!wstack) return make_float2(xc, 0.f);
    float s0, c0;
    screen(w, t.x, t.y, &s0, &c0);
    return make_float2(xc * c0, -xc * s0);
}
// the post-pass term Re exp(+2 pi i w_k t) h of the CTA's pixels of one image row, added to a
__device__ __forceinline__ void post_add(float2 &a, float4 h, float4 t, float2 w, int wstack) {
    if (!wstack) {
        a.x += h.x;
        a.y += h.z;
        return;
    }
    float s0, c0, s1, c1;
    screen(w, t.x, t.y, &s0, &c0);
    screen(w, t.z, t.w, &s1, &c1);
    a.x += h.x * c0 - h.y * s0;
    a.y += h.z * c1 - h.w * s1;
}
__device__ __forceinline__ void post_add(float &a, float2 h, float2 t, float2 w, int wstack) {
    if (!wstack) {
        a += h.x;
        return;
    }
    float s0, c0;
    screen(w, t.x, t.y, &s0, &c0);
    a += h.x * c0 - h.y * s0;
}
__device__ __forceinline__ float2 mul_corr(float2 a, float2 c) { return make_float2(a.x * c.x, a.y * c.y); }
__device__ __forceinline__ float mul_corr(float a, float c) { return a * c; }
__device__ __forceinline__ float2 add_prev(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float add_prev(float a, float b) { return a + b; }

// plane column and image column of the CTA's first lane: column groups q < ny / (2K) are the image columns
// right of the centre (plane columns from 0), the rest those left of it (plane columns from Nv - ny/2)
template <int K> __device__ __forceinline__ void column_of(int q, int Nv, int ny, int *c, int *j0) {
    const int hq = ny / (2 * K);
    *c = q < hq ? K * q : Nv - ny / 2 + K * (q - hq);
    *j0 = q < hq ? K * q + ny / 2 : K * (q - hq);
}

// ---------------------------------------------------------------- forward column pass (fused pre-pass)
// One CTA per group of K adjacent image columns; it takes them through the planes [k_lo, k_lo + nk) of
// band b.  xcT, tT: x corr and t of the group's pixels by image row; rowocc: the band's tile-row masks
// [Pmax][ntu / 32].  TMA (K = 2 only) stores boxes of 2 cells x TILE rows.
template <int L, bool TMA, typename E>
__global__ void __launch_bounds__((1 << L) / 16)
    k_colfwd(float2 *__restrict__ planes, int nk, int k_lo, int Nv, int64_t plane_sz, int nx, int ny,
             const typename Lanes<E>::X *__restrict__ xcT, const typename Lanes<E>::Tt *__restrict__ tT,
             const float2 *__restrict__ wk, int wstack, const uint32_t *__restrict__ rowocc,
             const float2 *__restrict__ W, const __grid_constant__ CUtensorMap tmap) {
    using S = Shape<L>;
    constexpr int N = S::N, T = S::T;
    extern __shared__ __align__(1024) unsigned char smraw[];
    E *sm = reinterpret_cast<E *>(smraw);
    const int tid = threadIdx.x;
    const int q = blockIdx.x;
    int c, j0;
    column_of<Lanes<E>::K>(q, Nv, ny, &c, &j0);
    const int rlo = nx / 2, rhi = N - nx / 2;
    const int ntu = N / TILE, nw = ntu / 32;
    const auto *xq = xcT + (int64_t)q * nx;
    const auto *tq = tT + (int64_t)q * nx;
    E v[16];

    for (int pl = 0; pl < nk; ++pl) {
        const int k = k_lo + pl;
        const float2 w = wk[k];
        const uint32_t *occ = rowocc + (int64_t)k * nw;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int row = tid + r * T;
            E e{};
            if (row < rlo || row >= rhi) {
                const int i = row < rlo ? row + nx / 2 : row - rhi;
                e = pre_value(xq[i], tq[i], w, wstack);
            }
            v[r] = e;
        }
        const int Ns = fft_stages<L, false>(v, sm, W, tid);
        if constexpr (TMA) {
            dense_to_smem<L>(v, sm, tid, Ns);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid < 32) {
                // the lanes of warp 0 store the occupied tile-rows: boxes of 2 cells x TILE rows
                for (int tu = tid; tu < ntu; tu += 32) {
                    if (!bit_set(occ, tu)) continue;
                    asm volatile(
                        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                            reinterpret_cast<uint64_t>(&tmap)),
                        "r"(c), "r"(tu * TILE), "r"(pl), "r"(smem_u32(sm + tu * TILE))
                        : "memory");
                }
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
        } else {
            float2 *base = planes + (int64_t)pl * plane_sz + c;
#pragma unroll
            for (int b = 0; b < S::BPT; ++b) {
                const int j = tid + b * T, kk = j & (Ns - 1);
                const int d = (j / Ns) * Ns * S::RL + kk;
#pragma unroll
                for (int r = 0; r < S::RL; ++r) {
                    const int row = d + r * Ns;
                    if (bit_set(occ, row / TILE))
                        *reinterpret_cast<E *>(base + (int64_t)row * Nv) = v[b * S::RL + operm<S::RL>(r)];
                }
            }
        }
    }
    if (TMA && tid < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------- inverse column pass (fused post-pass)
// One CTA per group of K image columns.  Shared memory: the exchange buffer, then the running post-pass
// sums of the group's image rows ([nx] X, one writer per row).  image [nx][ny] of the band; accumulate
// adds the result to it (a later plane block).
template <int L, typename E>
__global__ void __launch_bounds__((1 << L) / 16)
    k_colinv(const float2 *__restrict__ planes, int nk, int k_lo, int Nv, int64_t plane_sz, int nx, int ny,
             const typename Lanes<E>::Tt *__restrict__ tT, const float2 *__restrict__ wk, int wstack,
             const uint32_t *__restrict__ rowocc, const float *__restrict__ corr, int accumulate,
             float *__restrict__ image, const float2 *__restrict__ W) {
    using S = Shape<L>;
    using X = typename Lanes<E>::X;
    constexpr int N = S::N, T = S::T;
    extern __shared__ __align__(1024) unsigned char smraw[];
    E *sm = reinterpret_cast<E *>(smraw);
    X *acc = reinterpret_cast<X *>(sm + spad(N - 1) + 1);
    const int tid = threadIdx.x;
    const int q = blockIdx.x;
    int c, j0;
    column_of<Lanes<E>::K>(q, Nv, ny, &c, &j0);
    const int rlo = nx / 2, rhi = N - nx / 2;
    const int nw = (N / TILE) / 32;
    const auto *tq = tT + (int64_t)q * nx;
    for (int i = tid; i < nx; i += T) acc[i] = X{};
    E v[16];

    for (int pl = 0; pl < nk; ++pl) {
        const int k = k_lo + pl;
        const uint32_t *occ = rowocc + (int64_t)k * nw;
        const float2 *base = planes + (int64_t)pl * plane_sz + c;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int row = tid + r * T;
            v[r] = bit_set(occ, row / TILE) ? *reinterpret_cast<const E *>(base + (int64_t)row * Nv) : E{};
        }
        const int Ns = fft_stages<L, true>(v, sm, W, tid);
        const float2 w = wk[k];
#pragma unroll
        for (int b = 0; b < S::BPT; ++b) {
            const int j = tid + b * T, kk = j & (Ns - 1);
            const int d = (j / Ns) * Ns * S::RL + kk;
#pragma unroll
            for (int r = 0; r < S::RL; ++r) {
                const int row = d + r * Ns;
                if (row >= rlo && row < rhi) continue;
                const int i = row < rlo ? row + nx / 2 : row - rhi;
                X a = acc[i];
                post_add(a, v[b * S::RL + operm<S::RL>(r)], tq[i], w, wstack);
                acc[i] = a;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < nx; i += T) {
        const int64_t p = (int64_t)i * ny + j0;
        X o = mul_corr(acc[i], *reinterpret_cast<const X *>(corr + p));
        if (accumulate) o = add_prev(o, *reinterpret_cast<const X *>(image + p));
        *reinterpret_cast<X *>(image + p) = o;
    }
}

// ---------------------------------------------------------------- row pass
// One CTA per group of K rows of one occupied tile-row: list[e] = k << 16 | tu, and the CTA takes rows
// tu TILE + K p .. + K - 1, p = blockIdx.x mod (TILE / K).  occ: the band's tile masks [Pmax][ntu][ntv / 32].
//   INV: reads the touched segments (the rest is zero), writes the image columns;
//   forward: reads the image columns (the rest is zero), writes the touched segments.
template <typename E> __device__ __forceinline__ E load_rows(const float2 *r0, int64_t N, int m);
template <> __device__ __forceinline__ float4 load_rows<float4>(const float2 *r0, int64_t N, int m) {
    const float2 a = r0[m], b = r0[N + m];
    return make_float4(a.x, a.y, b.x, b.y);
}
template <> __device__ __forceinline__ float2 load_rows<float2>(const float2 *r0, int64_t N, int m) { return r0[m]; }
__device__ __forceinline__ void store_rows(float2 *r0, int64_t N, int m, float4 e) {
    r0[m] = make_float2(e.x, e.y);
    r0[N + m] = make_float2(e.z, e.w);
}
__device__ __forceinline__ void store_rows(float2 *r0, int64_t, int m, float2 e) { r0[m] = e; }

template <int L, bool INV, typename E>
__global__ void __launch_bounds__((1 << L) / 16)
    k_rowfft(float2 *__restrict__ planes, int k_lo, int ntu, int64_t plane_sz, int ny,
             const int *__restrict__ list, const uint32_t *__restrict__ occ, const float2 *__restrict__ W) {
    using S = Shape<L>;
    constexpr int N = S::N, T = S::T, K = Lanes<E>::K;
    constexpr int NW = N / TILE / 32;   // mask words per tile-row
    extern __shared__ __align__(1024) unsigned char smraw[];
    E *sm = reinterpret_cast<E *>(smraw);
    const int tid = threadIdx.x;
    const int ent = list[blockIdx.x / (TILE / K)];
    const int k = ent >> 16, tu = ent & 0xffff;
    const int u0 = tu * TILE + K * (int)(blockIdx.x % (TILE / K));
    float2 *row0 = planes + (int64_t)(k - k_lo) * plane_sz + (int64_t)u0 * N;
    const uint32_t *segs = occ + ((int64_t)k * ntu + tu) * NW;
    const int clo = ny / 2, chi = N - ny / 2;
    E v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int m = tid + r * T;
        const bool in = INV ? bit_set(segs, m / TILE) : (m < clo || m >= chi);
        v[r] = in ? load_rows<E>(row0, N, m) : E{};
    }
    const int Ns = fft_stages<L, INV>(v, sm, W, tid);
    dense_to_smem<L>(v, sm, tid, Ns);
    __syncthreads();
#pragma unroll 4
    for (int m = tid; m < N; m += T) {
        const bool out = INV ? (m < clo || m >= chi) : bit_set(segs, m / TILE);
        if (out) store_rows(row0, N, m, sm[m]);
    }
}

// ---------------------------------------------------------------- tables
// xcT[q][i] = (x corr)(i, j0(q) .. j0(q) + K - 1): the pre-pass inputs of column group q by image row
// (j0 as in column_of), by a 32 x 32 tile transpose.
template <int K>
__global__ void k_xc_transpose(const float *__restrict__ x, const float *__restrict__ corr, int nx, int ny,
                               typename Lanes<std::conditional_t<K == 2, float4, float2>>::X *__restrict__ xcT) {
    using X = typename Lanes<std::conditional_t<K == 2, float4, float2>>::X;
    __shared__ X tile[32][33];
    const int hq = ny / (2 * K), nq = ny / K;
    const int i0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
    for (int kk = threadIdx.y; kk < 32; kk += 8) {
        const int i = i0 + kk, q = q0 + threadIdx.x;
        X e{};
        if (i < nx && q < nq) {
            const int j0 = q < hq ? K * q + ny / 2 : K * (q - hq);
            const int64_t p = (int64_t)i * ny + j0;
            e = mul_corr(*reinterpret_cast<const X *>(x + p), *reinterpret_cast<const X *>(corr + p));
        }
        tile[kk][threadIdx.x] = e;
    }
    __syncthreads();
    for (int kk = threadIdx.y; kk < 32; kk += 8) {
        const int q = q0 + kk, i = i0 + threadIdx.x;
        if (q < nq && i < nx) xcT[(int64_t)q * nx + i] = tile[threadIdx.x][kk];
    }
}

// tT[q][i] = t(i, j0(q) .. j0(q) + K - 1) from the per-pixel float pairs of an FP32 plan
template <int K>
__global__ void k_t_transpose(const float2 *__restrict__ tp, int nx, int ny,
                              typename Lanes<std::conditional_t<K == 2, float4, float2>>::Tt *__restrict__ tT) {
    const int64_t n = (int64_t)nx * (ny / K);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / nx), i = (int)(e - (int64_t)q * nx);
        const int hq = ny / (2 * K);
        const int j0 = q < hq ? K * q + ny / 2 : K * (q - hq);
        const float2 a = tp[(int64_t)i * ny + j0];
        if constexpr (K == 2) {
            const float2 b = tp[(int64_t)i * ny + j0 + 1];
            tT[e] = make_float4(a.x, a.y, b.x, b.y);
        } else {
            tT[e] = a;
        }
    }
}

// Touched tiles: an item of bucket (b, tile, kq) reaches planes kq q .. kq q + q + W_w - 2 of tile, and on
// plans that list items in their home tile only (halo), of the tiles after it in u, v and both.
__global__ void k_occupancy(const int64_t *__restrict__ off, int64_t nkeys, int ntiles, int ntu, int ntv,
                            int nkq, int q, int Ww, int Pmax, int halo, const BandGeom *__restrict__ bgs,
                            uint32_t *__restrict__ occ) {
    for (int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; key < nkeys;
         key += (int64_t)gridDim.x * blockDim.x) {
        if (off[key + 1] <= off[key]) continue;
        const int kq = (int)(key % nkq);
        const int64_t bt = key / nkq;
        const int b = (int)(bt / ntiles), t = (int)(bt - (int64_t)b * ntiles);
        const int tu = t / ntv, tv = t - tu * ntv;
        const int P = bgs[b].P;
        const int tu1 = tu + 1 == ntu ? 0 : tu + 1, tv1 = tv + 1 == ntv ? 0 : tv + 1;
        for (int cc = 0; cc < q + Ww - 1; ++cc) {
            const int k = kq * q + cc;
            if (k >= P) break;
            uint32_t *o = occ + ((int64_t)b * Pmax + k) * ntu * (ntv / 32);
            atomicOr(&o[(int64_t)tu * (ntv / 32) + (tv >> 5)], 1u << (tv & 31));
            if (halo) {
                atomicOr(&o[(int64_t)tu1 * (ntv / 32) + (tv >> 5)], 1u << (tv & 31));
                atomicOr(&o[(int64_t)tu * (ntv / 32) + (tv1 >> 5)], 1u << (tv1 & 31));
                atomicOr(&o[(int64_t)tu1 * (ntv / 32) + (tv1 >> 5)], 1u << (tv1 & 31));
            }
        }
    }
}

int log2_exact(int n) {
    int L = 0;
    while ((1 << L) < n) ++L;
    return (1 << L) == n ? L : -1;
}

template <int L, typename E> constexpr size_t fft_smem() { return (size_t)(spad((1 << L) - 1) + 1) * sizeof(E); }
// column groups of K = 2 columns for transforms of up to 8192 points, single columns for 16384
template <int L> using ColE = std::conditional_t<(L <= 13), float4, float2>;

template <int L, bool TMA>
void launch_colfwd(cudaStream_t st, float2 *planes, int nk, int k_lo, int Nv, int64_t plane_sz, int nx, int ny,
                   const void *xcT, const void *tT, const float2 *wk, int wstack, const uint32_t *rowocc,
                   const float2 *W, const CUtensorMap &map) {
    using E = ColE<L>;
    const size_t smem = fft_smem<L, E>();
    const unsigned grid = (unsigned)(ny / Lanes<E>::K);
    ensure_dynamic_smem(k_colfwd<L, TMA, E>, (size_t)smem);
    k_colfwd<L, TMA, E><<<grid, (1 << L) / 16, smem, st>>>(
        planes, nk, k_lo, Nv, plane_sz, nx, ny, (const typename Lanes<E>::X *)xcT,
        (const typename Lanes<E>::Tt *)tT, wk, wstack, rowocc, W, map);
}

template <int L>
void launch_colinv(cudaStream_t st, const float2 *planes, int nk, int k_lo, int Nv, int64_t plane_sz, int nx, int ny,
                   const void *tT, const float2 *wk, int wstack, const uint32_t *rowocc, const float *corr,
                   int accumulate, float *image, const float2 *W) {
    using E = ColE<L>;
    const size_t smem = fft_smem<L, E>() + (size_t)nx * sizeof(typename Lanes<E>::X);
    const unsigned grid = (unsigned)(ny / Lanes<E>::K);
    ensure_dynamic_smem(k_colinv<L, E>, (size_t)smem);
    k_colinv<L, E><<<grid, (1 << L) / 16, smem, st>>>(planes, nk, k_lo, Nv, plane_sz, nx, ny,
                                                       (const typename Lanes<E>::Tt *)tT, wk, wstack, rowocc, corr,
                                                       accumulate, image, W);
}

template <int L, bool INV>
void launch_rowfft(int64_t entries, cudaStream_t st, float2 *planes, int k_lo, int ntu, int64_t plane_sz, int ny,
                   const int *list, const uint32_t *occ, const float2 *W) {
    using E = ColE<L>;
    const size_t smem = fft_smem<L, E>();
    const unsigned grid = (unsigned)(entries * (TILE / Lanes<E>::K));
    ensure_dynamic_smem(k_rowfft<L, INV, E>, (size_t)smem);
    k_rowfft<L, INV, E><<<grid, (1 << L) / 16, smem, st>>>(planes, k_lo, ntu, plane_sz, ny, list, occ, W);
}

#define PFB_L_SWITCH(Lv, CALL)                                              \
    switch (Lv) {                                                           \
        case 10: CALL(10); break;                                           \
        case 11: CALL(11); break;                                           \
        case 12: CALL(12); break;                                           \
        case 13: CALL(13); break;                                           \
        case 14: CALL(14); break;                                           \
        default: throw Error(PFB_ERR_ARG, "pruned plane transform: unsupported plane size"); \
    }

}  // namespace

// columns of the column kernels per CTA for planes of Nu rows: pairs up to 8192, single columns at 16384
static int col_group(int Nu) { return Nu <= 8192 ? 2 : 1; }

bool pruned_fits(const Plan &p) {
    const int Lu = log2_exact(p.Nu), Lv = log2_exact(p.Nv);
    return p.prec == PFB_F32 && Lu >= 10 && Lu <= 14 && Lv >= 10 && Lv <= 14 && p.nx % 2 == 0 && p.ny % 4 == 0 &&
           p.nx >= 2 && p.ny >= 4 && p.nx <= p.Nu && p.ny <= p.Nv && p.Pmax < (1 << 15) &&
           !(p.flags & PFB_NO_PRUNED_FFT);
}

void build_pruned_tables(Ctx &ctx, Plan &p, cudaStream_t st) {
    if (!pruned_fits(p)) return;
    const int nw = p.ntv / 32;
    const size_t occ_words = (size_t)p.nband * p.Pmax * p.ntu * nw;
    const size_t need = occ_words * 4 + (size_t)p.nx * p.ny * sizeof(float2) + (size_t)p.nband * p.Pmax * 8 +
                        (size_t)p.nband * p.Pmax * p.ntu * 4 + (16u << 20);
    if (ctx.available() < need) return;
    p.d_occ = (uint32_t *)ctx.dalloc(occ_words * 4);
    p.bytes += occ_words * 4;
    PFB_CUDA(cudaMemsetAsync(p.d_occ, 0, occ_words * 4, st));
    const int64_t ntiles = (int64_t)p.ntu * p.ntv;
    k_occupancy<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((p.nkeys + 255) / 256, 64LL * ctx.num_sms)), 256, 0,
                  st>>>(p.d_off, p.nkeys, (int)ntiles, p.ntu, p.ntv, p.nkq, p.q, p.Ww, p.Pmax, p.halo ? 1 : 0,
                        p.d_bg, p.d_occ);
    check_launch("occupancy");
    std::vector<uint32_t> occ(occ_words);
    PFB_CUDA(cudaMemcpyAsync(occ.data(), p.d_occ, occ_words * 4, cudaMemcpyDeviceToHost, st));
    PFB_CUDA(cudaStreamSynchronize(st));
    const int rw = p.ntu / 32;
    std::vector<uint32_t> rowocc((size_t)p.nband * p.Pmax * rw, 0u);
    std::vector<int> list;
    p.rowlist_off.assign((size_t)p.nband * (p.Pmax + 1), 0);
    for (int b = 0; b < p.nband; ++b) {
        for (int k = 0; k <= p.Pmax; ++k) {
            p.rowlist_off[(size_t)b * (p.Pmax + 1) + k] = (int64_t)list.size();
            if (k == p.Pmax || k >= p.P[b]) continue;
            for (int tu = 0; tu < p.ntu; ++tu) {
                const uint32_t *wd = occ.data() + (((size_t)b * p.Pmax + k) * p.ntu + tu) * nw;
                bool any = false;
                for (int w = 0; w < nw; ++w) any = any || wd[w] != 0u;
                if (!any) continue;
                list.push_back(k << 16 | tu);
                rowocc[((size_t)b * p.Pmax + k) * rw + tu / 32] |= 1u << (tu & 31);
            }
        }
    }
    std::vector<float2> wk((size_t)p.nband * p.Pmax, make_float2(0.f, 0.f));
    for (int b = 0; b < p.nband; ++b)
        for (int k = 0; k < p.P[b]; ++k) {
            const double w = p.w0[b] + (double)k * p.dw;
            const float hi = (float)w;
            wk[(size_t)b * p.Pmax + k] = make_float2(hi, (float)(w - (double)hi));
        }
    p.d_rowocc = (uint32_t *)ctx.dalloc(rowocc.size() * 4);
    p.d_rowlist = (int *)ctx.dalloc(std::max<size_t>(list.size(), 1) * sizeof(int));
    p.d_wk = (float2 *)ctx.dalloc(wk.size() * sizeof(float2));
    p.d_tT = (float4 *)ctx.dalloc((size_t)p.nx * p.ny * sizeof(float2));
    p.bytes += rowocc.size() * 4 + list.size() * sizeof(int) + wk.size() * sizeof(float2) +
               (size_t)p.nx * p.ny * sizeof(float2);
    PFB_CUDA(cudaMemcpyAsync(p.d_rowocc, rowocc.data(), rowocc.size() * 4, cudaMemcpyHostToDevice, st));
    if (!list.empty())
        PFB_CUDA(cudaMemcpyAsync(p.d_rowlist, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(p.d_wk, wk.data(), wk.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    const int K = col_group(p.Nu);
    const int64_t n = (int64_t)p.nx * (p.ny / K);
    const unsigned tb = (unsigned)std::min<int64_t>((n + 255) / 256, 32LL * ctx.num_sms);
    if (K == 2)
        k_t_transpose<2><<<tb, 256, 0, st>>>(reinterpret_cast<const float2 *>(p.d_tp), p.nx, p.ny, p.d_tT);
    else
        k_t_transpose<1><<<tb, 256, 0, st>>>(reinterpret_cast<const float2 *>(p.d_tp), p.nx, p.ny,
                                             reinterpret_cast<float2 *>(p.d_tT));
    check_launch("t_transpose");
    // the host vectors die with this scope
    PFB_CUDA(cudaStreamSynchronize(st));
    p.pruned = true;
}

// rows (tile-rows x TILE) and touched tiles of band b over planes [k_lo, k_hi), from the list
static void occupied_counts(const Plan &p, int b, int k_lo, int k_hi, double *rows) {
    const int64_t e0 = p.rowlist_off[(size_t)b * (p.Pmax + 1) + k_lo];
    const int64_t e1 = p.rowlist_off[(size_t)b * (p.Pmax + 1) + k_hi];
    *rows = (double)(e1 - e0) * TILE;
}

void plane_forward(Ctx &ctx, const Plan &p, int b, const float *x, int k_lo, int k_hi, float2 *planes,
                   cudaStream_t st) {
    const int nk = k_hi - k_lo;
    const int Lu = log2_exact(p.Nu), Lv = log2_exact(p.Nv);
    const int64_t npix = (int64_t)p.nx * p.ny;
    const int64_t plane_sz = (int64_t)p.Nu * p.Nv;
    const float2 *Wu = fft_twiddles(ctx, p.Nu, st);
    const float2 *Wv = p.Nv == p.Nu ? Wu : fft_twiddles(ctx, p.Nv, st);
    double rows = 0;
    occupied_counts(p, b, k_lo, k_hi, &rows);
    void *xcT = ctx.scratch("xcT", (size_t)npix * sizeof(float));
    const int K = col_group(p.Nu);
    // the w-planes of this block, as the bytes of one plane sweep (a count for the timing record, no kernel)
    { KTimer w(ctx, "w_planes", st, (double)nk * (double)plane_sz * sizeof(float2), 0); }
    {
        KTimer t(ctx, "xc_transpose", st, 12.0 * npix);
        const dim3 grid((unsigned)((p.nx + 31) / 32), (unsigned)((p.ny / K + 31) / 32));
        if (K == 2)
            k_xc_transpose<2><<<grid, dim3(32, 8), 0, st>>>(x, (const float *)p.d_corr, p.nx, p.ny, (float2 *)xcT);
        else
            k_xc_transpose<1><<<grid, dim3(32, 8), 0, st>>>(x, (const float *)p.d_corr, p.nx, p.ny, (float *)xcT);
        check_launch("xc_transpose");
    }
    const float2 *wk = p.d_wk + (size_t)b * p.Pmax;
    const uint32_t *rowocc = p.d_rowocc + (size_t)b * p.Pmax * (p.ntu / 32);
    {
        KTimer t(ctx, "col_fwd", st, 12.0 * npix + rows * p.ny * 8.0);
        CUtensorMap map;
        std::memset(&map, 0, sizeof(map));
        // TMA boxes of 2 cells x TILE rows for column pairs; single columns (8-byte rows) store per thread
        const bool tma = K == 2 && plane_tensor_map(&map, planes, p.Nu, p.Nv, nk, p.ny, TILE);
#define PFB_CF(LV)                                                                                          \
    (tma ? launch_colfwd<LV, (LV <= 13)>(st, planes, nk, k_lo, p.Nv, plane_sz, p.nx, p.ny, xcT, p.d_tT, wk,  \
                                         p.wstack ? 1 : 0, rowocc, Wu, map)                                   \
         : launch_colfwd<LV, false>(st, planes, nk, k_lo, p.Nv, plane_sz, p.nx, p.ny, xcT, p.d_tT, wk,        \
                                    p.wstack ? 1 : 0, rowocc, Wu, map))
        PFB_L_SWITCH(Lu, PFB_CF)
#undef PFB_CF
        check_launch("col_fwd");
    }
    const int64_t e0 = p.rowlist_off[(size_t)b * (p.Pmax + 1) + k_lo];
    const int64_t e1 = p.rowlist_off[(size_t)b * (p.Pmax + 1) + k_hi];
    if (e1 > e0) {
        KTimer t(ctx, "row_fwd", st, rows * (p.ny + p.Nv) * 8.0);
        const uint32_t *occ = p.d_occ + (size_t)b * p.Pmax * p.ntu * (p.ntv / 32);
#define PFB_RF(LV) launch_rowfft<LV, false>(e1 - e0, st, planes, k_lo, p.ntu, plane_sz, p.ny, p.d_rowlist + e0, occ, Wv)
        PFB_L_SWITCH(Lv, PFB_RF)
#undef PFB_RF
        check_launch("row_fwd");
    }
}

void plane_inverse(Ctx &ctx, const Plan &p, int b, int k_lo, int k_hi, float2 *planes, float *image,
                   cudaStream_t st) {
    const int nk = k_hi - k_lo;
    const int Lu = log2_exact(p.Nu), Lv = log2_exact(p.Nv);
    const int64_t npix = (int64_t)p.nx * p.ny;
    const int64_t plane_sz = (int64_t)p.Nu * p.Nv;
    const float2 *Wu = fft_twiddles(ctx, p.Nu, st);
    const float2 *Wv = p.Nv == p.Nu ? Wu : fft_twiddles(ctx, p.Nv, st);
    double rows = 0;
    occupied_counts(p, b, k_lo, k_hi, &rows);
    const int64_t e0 = p.rowlist_off[(size_t)b * (p.Pmax + 1) + k_lo];
    const int64_t e1 = p.rowlist_off[(size_t)b * (p.Pmax + 1) + k_hi];
    if (e1 > e0) {
        KTimer t(ctx, "row_inv", st, rows * (p.Nv + p.ny) * 8.0);
        const uint32_t *occ = p.d_occ + (size_t)b * p.Pmax * p.ntu * (p.ntv / 32);
#define PFB_RI(LV) launch_rowfft<LV, true>(e1 - e0, st, planes, k_lo, p.ntu, plane_sz, p.ny, p.d_rowlist + e0, occ, Wv)
        PFB_L_SWITCH(Lv, PFB_RI)
#undef PFB_RI
        check_launch("row_inv");
    }
    {
        KTimer t(ctx, "col_inv", st, rows * p.ny * 8.0 + npix * (8.0 + 4.0 + 4.0 + (k_lo > 0 ? 4.0 : 0.0)));
        const float2 *wk = p.d_wk + (size_t)b * p.Pmax;
        const uint32_t *rowocc = p.d_rowocc + (size_t)b * p.Pmax * (p.ntu / 32);
#define PFB_CI(LV)                                                                                              \
    launch_colinv<LV>(st, planes, nk, k_lo, p.Nv, plane_sz, p.nx, p.ny, p.d_tT, wk, p.wstack ? 1 : 0, rowocc,    \
                      (const float *)p.d_corr, k_lo > 0 ? 1 : 0, image, Wu)
        PFB_L_SWITCH(Lu, PFB_CI)
#undef PFB_CI
        check_launch("col_inv");
    }
}

}  // namespace pfb
