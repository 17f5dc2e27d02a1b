// Allocation-free per-band weight sums (pfb_wsum_static).
//
// Some callers cannot allocate device memory at the point where they need the
// weight sums: an engine that hands out the whole HBM pool up front and forbids
// later allocations, or a caller on a latency-critical stream where cudaMalloc /
// cudaFree could synchronise the device and stall other streams.  This entry point
// computes the same per-band sums as the reduction behind pfb_dirty / pfb_psf's
// wsum_out, but its accumulators live in a fixed file-scope device array instead
// of context scratch, so it calls no allocator at all.
#include "ctx.cuh"

#include <mutex>

namespace pfb {

// Accumulators shared by every call of pfb_wsum_static on a device, held by every
// GPU that loads the library until the process exits.
constexpr int NOALLOC_MAX_BANDS = 32;
static __device__ __align__(256) double g_wsum_scratch[NOALLOC_MAX_BANDS];

template <typename T>
__global__ void k_wsum_static(const T *__restrict__ wgt, int64_t n, int nchan, int nband,
                              const int *__restrict__ band, double *__restrict__ acc) {
    __shared__ double sacc[NOALLOC_MAX_BANDS];
    for (int b = threadIdx.x; b < NOALLOC_MAX_BANDS; b += blockDim.x) sacc[b] = 0.0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = band[(int)(i % nchan)];
        if (b >= 0 && b < nband) atomicAdd(&sacc[b], wgt ? (double)wgt[i] : 1.0);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nband; b += blockDim.x)
        if (sacc[b] != 0.0) atomicAdd(&acc[b], sacc[b]);
}

__global__ void k_wsum_static_out(const double *__restrict__ acc, int nband, double *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nband) out[b] = acc[b];
}

// Device address of g_wsum_scratch, looked up once per device with that device
// current (host code only sees a stand-in for the symbol).
static double *scratch_address(int device) {
    static std::mutex mu;
    static std::map<int, double *> addr;
    std::lock_guard<std::mutex> lock(mu);
    auto it = addr.find(device);
    if (it != addr.end()) return it->second;
    double *p = nullptr;
    PFB_CUDA(cudaGetSymbolAddress((void **)&p, g_wsum_scratch));
    addr[device] = p;
    return p;
}

// message of the last failure of a context-free call on this thread
thread_local std::string g_free_error;

}  // namespace pfb

extern "C" int pfb_wsum_static(int device, pfb_prec prec, int64_t nrow, int32_t nchan, int32_t nband,
                               const int32_t *band_of_chan, const void *wgt, double *wsum_out, void *stream) {
    using namespace pfb;
    g_free_error.clear();
    if (nrow < 1 || nchan < 1 || nband < 1 || !band_of_chan || !wsum_out) {
        g_free_error = "pfb_wsum_static: nrow, nchan, nband must be >= 1 and band_of_chan, wsum_out non-NULL";
        return PFB_ERR_ARG;
    }
    if (nband > NOALLOC_MAX_BANDS) {
        g_free_error = "pfb_wsum_static: nband " + std::to_string(nband) + " exceeds the static maximum of " +
                       std::to_string(NOALLOC_MAX_BANDS) + " bands";
        return PFB_ERR_ARG;
    }
    if (prec != PFB_F32 && prec != PFB_F64) {
        g_free_error = "pfb_wsum_static: prec must be PFB_F32 or PFB_F64";
        return PFB_ERR_ARG;
    }
    try {
        PFB_CUDA(cudaSetDevice(device));
        double *acc = scratch_address(device);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        PFB_CUDA(cudaMemsetAsync(acc, 0, NOALLOC_MAX_BANDS * sizeof(double), st));
        const int64_t n = nrow * (int64_t)nchan;
        int sms = 0;
        PFB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8LL * sms));
        if (prec == PFB_F64)
            k_wsum_static<double><<<blocks, 256, 0, st>>>((const double *)wgt, n, nchan, nband, band_of_chan, acc);
        else
            k_wsum_static<float><<<blocks, 256, 0, st>>>((const float *)wgt, n, nchan, nband, band_of_chan, acc);
        check_launch("wsum_static");
        k_wsum_static_out<<<1, NOALLOC_MAX_BANDS, 0, st>>>(acc, nband, wsum_out);
        check_launch("wsum_static_out");
        return PFB_OK;
    } catch (const Error &e) {
        g_free_error = e.what();
        return e.code;
    }
}
