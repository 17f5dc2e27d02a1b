// Column pass of the FP32 w-plane transforms.  A 2-D DFT of a plane is a pass of 1-D DFTs along the
// rows and one along the columns.  cuFFT's 2-D plans take two passes over the plane for the columns;
// this kernel takes one, and it touches only the image region: the pre-pass puts pixel (i, j) at
// ((i - nx/2) mod Nu, (j - ny/2) mod Nv), so only the columns [0, ny/2) and [Nv - ny/2, Nv) and the rows
// [0, nx/2) and [Nu - nx/2, Nu) carry data into the forward transform, and the post-pass reads back
// only that region of the inverse transform.
//   forward (degridding): this pass first, reading the image rows of the image columns (the other rows
//            are zero) and writing whole columns; then the row pass (cuFFT, all rows);
//   inverse (gridding): the row pass first (cuFFT, all rows); then this pass, reading whole image
//            columns and writing back their image rows only.
// One CTA transforms two adjacent columns of one plane (a 16-byte element per row) of length N = 2^L,
// 10 <= L <= 13, with N/16 threads.  The algorithm is the mixed-radix Stockham autosort DFT (radix-16
// stages, the last of radix 2, 4 or 8 when L is not a multiple of 4) in the formulation of Govindaraju
// et al., "High performance discrete Fourier transforms on graphics processors" (SC 2008): stage s with
// radix R and Ns = product of the earlier radices takes, for butterfly j < N/R, the inputs
// x[j + r N/R] (r < R), multiplies input r by exp(-/+ 2 pi i r (j mod Ns) / (Ns R)), applies an R-point
// DFT and writes output r to y[(j div Ns) Ns R + (j mod Ns) + r Ns].  The first stage reads the plane,
// the last writes it; the stages between go through shared memory (one buffer, the reads of a stage
// finished before its writes, indexed i + i/16 so that the strided writes of the first stage do not
// conflict on banks).  The R-point DFTs run in registers: 16 = 4 x 4 and 8 = 4 x 2 by the Cooley-Tukey
// split n = R2 n1 + n2, k = k1 + R1 k2 with the twiddles exp(-/+ 2 pi i n2 k1 / R) in between.
#include "ctx.cuh"
#include "fftcore.cuh"

#include <cuda.h>

namespace pfb {
namespace {
using namespace fft;

// Forward: rows outside the image rows read as zero, all rows written; inverse: all rows read, the
// image rows written.  A CTA takes its column pair through all planes in turn, so the stores of one
// plane drain while the loads of the next are in flight.
// TMA: the last stage writes the transformed columns densely into shared memory and one thread stores
// them with tiled bulk copies (boxes of 2 cells x 256 rows), which keeps the 16-byte row stores off the
// load/store pipe.  Copies are issued by thread 0, which waits (a hardware wait) until they have read
// shared memory before the buffer is written again, and until they are complete before it exits.

template <int L, bool INV, bool TMA>
__global__ void __launch_bounds__((1 << L) / 16) k_colfft(float2 *__restrict__ data, int nplanes, int Nv,
                                                          int64_t plane_sz, int nx, int ny,
                                                          const float2 *__restrict__ W,
                                                          const __grid_constant__ CUtensorMap tmap) {
    constexpr int N = 1 << L, T = N / 16;
    constexpr int NST16 = L / 4, RL = (L % 4) ? (1 << (L % 4)) : 16, BPT = 16 / RL;
    constexpr int NMID = NST16 - 1 - ((L % 4) ? 0 : 1);   // radix-16 stages between the first and last
    extern __shared__ __align__(1024) float4 sm[];
    const int tid = threadIdx.x;
    const int q = blockIdx.x, hq = ny / 4;
    const int c = q < hq ? 2 * q : Nv - ny / 2 + 2 * (q - hq);
    const int rlo = nx / 2, rhi = N - nx / 2;
    float4 v[16];

    for (int pl = 0; pl < nplanes; ++pl) {
        float2 *base = data + (int64_t)pl * plane_sz + c;
        // first stage (radix 16, Ns = 1: no twiddles), from the plane
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int row = tid + r * T;
            v[r] = (!INV && row >= rlo && row < rhi) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                     : *reinterpret_cast<const float4 *>(base + (int64_t)row * Nv);
        }
        dft_reg<16, INV>(v);
        __syncthreads();   // the previous plane's last stage has read the buffer
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[spad(tid * 16 + r)] = v[operm<16>(r)];
        __syncthreads();

        int Ns = 16;
#pragma unroll
        for (int s = 0; s < NMID; ++s) {
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

        // last stage (radix RL, BPT butterflies per thread), to the plane
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
        if constexpr (TMA) {
            __syncthreads();   // every thread has read the buffer
#pragma unroll
            for (int b = 0; b < BPT; ++b) {
                const int j = tid + b * T, k = j & (Ns - 1);
                const int d = (j / Ns) * Ns * RL + k;
#pragma unroll
                for (int r = 0; r < RL; ++r) sm[d + r * Ns] = v[b * RL + operm<RL>(r)];   // row-major, dense
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                for (int r0 = 0; r0 < N; r0 += 256) {
                    if (INV && r0 >= rlo && r0 + 256 <= rhi) continue;   // no image row in this box
                    asm volatile(
                        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                            reinterpret_cast<uint64_t>(&tmap)),
                        "r"(c), "r"(r0), "r"(pl), "r"(smem_u32(sm + r0))
                        : "memory");
                }
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
        } else {
#pragma unroll
            for (int b = 0; b < BPT; ++b) {
                const int j = tid + b * T, k = j & (Ns - 1);
                const int d = (j / Ns) * Ns * RL + k;
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int row = d + r * Ns;
                    if (INV && row >= rlo && row < rhi) continue;
                    *reinterpret_cast<float4 *>(base + (int64_t)row * Nv) = v[b * RL + operm<RL>(r)];
                }
            }
        }
    }
    if (TMA && tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// W[m] = exp(-2 pi i m / n), rounded from double
__global__ void k_colfft_table(int n, float2 *W) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    W[m] = make_float2((float)c, (float)-s);
}

// Tensor map of a plane block for the TMA stores: [nplanes][Nu][Nv] cells of 8 bytes, box 2 x box_rows x 1.
// Returns false (plain stores) when the driver's encoder is not available or a layout rule of the copy
// is not met: 16-byte base and strides, a 16-byte inner box extent, and x coordinates (2 q or
// Nv - ny/2 + 2 q) that are even, i.e. 16-byte aligned.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

template <int L, bool INV>
void launch_colfft(float2 *data, int nplanes, int Nv, int64_t plane_sz, int nx, int ny, const float2 *W,
                   cudaStream_t st) {
    constexpr int N = 1 << L;
    const size_t smem = (size_t)(spad(N - 1) + 1) * sizeof(float4);
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (plane_tensor_map(&map, data, N, Nv, nplanes, ny, 256)) {
        ensure_dynamic_smem(k_colfft<L, INV, true>, (size_t)smem);
        k_colfft<L, INV, true><<<(unsigned)(ny / 2), N / 16, smem, st>>>(data, nplanes, Nv, plane_sz, nx, ny, W,
                                                                          map);
    } else {
        ensure_dynamic_smem(k_colfft<L, INV, false>, (size_t)smem);
        k_colfft<L, INV, false><<<(unsigned)(ny / 2), N / 16, smem, st>>>(data, nplanes, Nv, plane_sz, nx, ny, W,
                                                                           map);
    }
    check_launch("colfft");
}

}  // namespace

bool plane_tensor_map(CUtensorMap *map, float2 *data, int Nu, int Nv, int nplanes, int ny, int box_rows) {
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc || Nu < box_rows || Nu % box_rows || Nv % 2 || (Nv - ny / 2) % 2 || (ny / 2) % 2) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Nv, (cuuint64_t)Nu, (cuuint64_t)nplanes};
    const cuuint64_t strides[2] = {(cuuint64_t)Nv * 8, (cuuint64_t)Nu * Nv * 8};
    const cuuint32_t box[3] = {2, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (reinterpret_cast<uintptr_t>(data) % 16 || strides[0] % 16 || strides[1] % 16) return false;
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, data, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

const float2 *fft_twiddles(Ctx &ctx, int n, cudaStream_t st) {
    const std::string name = "colfft_w" + std::to_string(n);
    float2 *W = (float2 *)ctx.scratch(name, (size_t)n * sizeof(float2));
    auto tag = ctx.zero_tag.find(name);
    if (tag == ctx.zero_tag.end() || tag->second.first != (uint64_t)n) {
        k_colfft_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, W);
        check_launch("colfft_table");
        ctx.zero_tag[name] = {(uint64_t)n, 1};
    }
    return W;
}

bool colfft_fits(int Nu, int Nv, int nx, int ny) {
    int L = 0;
    while ((1 << L) < Nu) ++L;
    return (1 << L) == Nu && L >= 10 && L <= 13 && ny % 4 == 0 && nx % 2 == 0 && nx <= Nu && ny <= Nv &&
           Nv % 2 == 0;
}

void colfft_planes(Ctx &ctx, float2 *data, int nplanes, int Nu, int Nv, int nx, int ny, bool inverse,
                   cudaStream_t st) {
    PFB_REQUIRE(colfft_fits(Nu, Nv, nx, ny), "column transform: unsupported plane shape");
    const float2 *W = fft_twiddles(ctx, Nu, st);
    const int64_t plane_sz = (int64_t)Nu * Nv;
#define PFB_COLFFT(LV)                                                                                  \
    (inverse ? launch_colfft<LV, true>(data, nplanes, Nv, plane_sz, nx, ny, W, st)                      \
             : launch_colfft<LV, false>(data, nplanes, Nv, plane_sz, nx, ny, W, st))
    switch (Nu) {
        case 1024: PFB_COLFFT(10); break;
        case 2048: PFB_COLFFT(11); break;
        case 4096: PFB_COLFFT(12); break;
        default: PFB_COLFFT(13); break;
    }
#undef PFB_COLFFT
}

}  // namespace pfb
