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
// (one more slot: the count of out-of-range band ids)
static __device__ __align__(256) double g_wsum_scratch[NOALLOC_MAX_BANDS + 1];

// Slot NOALLOC_MAX_BANDS counts the channels whose band id lies outside [0, nband).
template <typename T>
__global__ void k_wsum_static(const T *__restrict__ wgt, int64_t n, int nchan, int nband,
                              const int *__restrict__ band, double *__restrict__ acc) {
    __shared__ double sacc[NOALLOC_MAX_BANDS];
    for (int b = threadIdx.x; b < NOALLOC_MAX_BANDS; b += blockDim.x) sacc[b] = 0.0;
    __syncthreads();
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < nchan; c += blockDim.x)
            if (band[c] < 0 || band[c] >= nband) atomicAdd(&acc[NOALLOC_MAX_BANDS], 1.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = band[(int)(i % nchan)];
        if (b >= 0 && b < nband) atomicAdd(&sacc[b], wgt ? (double)wgt[i] : 1.0);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nband; b += blockDim.x)
        if (sacc[b] != 0.0) atomicAdd(&acc[b], sacc[b]);
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

// Restores the calling thread's current device when the call returns.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != device) PFB_CUDA(cudaSetDevice(device));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// True when the GPU can dereference p as device memory (device or managed allocations).
static bool device_pointer(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

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
        DeviceGuard dg(device);
        if (!device_pointer(band_of_chan) || (wgt && !device_pointer(wgt))) {
            g_free_error = "pfb_wsum_static: band_of_chan and wgt must be device (or managed) memory";
            return PFB_ERR_ARG;
        }
        double *acc = scratch_address(device);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        PFB_CUDA(cudaMemsetAsync(acc, 0, (NOALLOC_MAX_BANDS + 1) * sizeof(double), st));
        const int64_t n = nrow * (int64_t)nchan;
        int sms = 0;
        PFB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8LL * sms));
        if (prec == PFB_F64)
            k_wsum_static<double><<<blocks, 256, 0, st>>>((const double *)wgt, n, nchan, nband, band_of_chan, acc);
        else
            k_wsum_static<float><<<blocks, 256, 0, st>>>((const float *)wgt, n, nchan, nband, band_of_chan, acc);
        check_launch("wsum_static");
        // cudaMemcpyDefault takes a host or a device destination; the count of bad band ids
        // comes back to the stack, so the call returns after `stream` has done its work
        double bad = 0.0;
        PFB_CUDA(cudaMemcpyAsync(wsum_out, acc, (size_t)nband * sizeof(double), cudaMemcpyDefault, st));
        PFB_CUDA(cudaMemcpyAsync(&bad, acc + NOALLOC_MAX_BANDS, sizeof(double), cudaMemcpyDeviceToHost, st));
        PFB_CUDA(cudaStreamSynchronize(st));
        if (bad != 0.0) {
            g_free_error = "pfb_wsum_static: band_of_chan entry outside [0, nband)";
            return PFB_ERR_ARG;
        }
        return PFB_OK;
    } catch (const Error &e) {
        g_free_error = e.what();
        return e.code;
    }
}
