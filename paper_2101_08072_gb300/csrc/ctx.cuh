// Host-side context and plan structures of libpfb (internal).
#pragma once

#include "common.cuh"

#include <cuda.h>

#include <functional>
#include <mutex>
#include <utility>

namespace pfb {

// Raise a kernel's dynamic shared-memory limit on the current device only when a launch needs more than was set
// before: one driver call per kernel, device and size instead of one per launch.
template <typename K>
inline void ensure_dynamic_smem(K *kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    PFB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = set[{reinterpret_cast<const void *>(kernel), dev}];
    if (bytes <= have) return;
    PFB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
}

// One gridding work item: a uv tile of one band, either the tile's whole item
// list or one chunk of a heavy tile's list; atomic_mode says how its sums reach the
// planes (plain stores of cells the item owns, or reductions into zeroed cells).
struct WorkItem {
    int tile;
    int atomic_mode;
    long long begin, end;
};

struct Plan {
    // ---- key
    int nx = 0, ny = 0, nband = 0;
    double dl = 0, dm = 0;
    double l0 = 0, m0 = 0;    // image centre (facets)
    double fa = 0, fb = 0;    // dn/dl, dn/dm at the image centre (0 without w term)
    uint32_t flags = 0;
    int prec = 0;
    int W = 0;
    int64_t nrow = 0;
    int nchan = 0;
    const void *uvw = nullptr, *freq = nullptr, *band = nullptr;
    uint64_t last_use = 0;
    uint64_t id = 0;   // unique per context: tags buffers whose zero pattern belongs to this plan

    // ---- geometry
    int Nu = 0, Nv = 0, Ww = 1, ntu = 0, ntv = 0, q = 1, nkq = 1, Pmax = 1;
    double beta = 0, dw = 0, tc = 0, Thalf = 0;
    bool wstack = false;
    // FP32 tile kernels: every visibility is listed once, in the tile of its first-tap cell (no spill
    // copies into the tiles its footprint crosses); gridding adds each tile's (TILE + W - 1)^2 region
    bool halo = false;
    std::vector<double> w0, wlo, whi;
    std::vector<int> P;
    std::vector<double> scale;      // f / c per channel
    std::vector<int> band_h;
    std::vector<int64_t> band_items_begin, band_items_end;
    std::vector<int64_t> work_begin; // per band offset into d_work (size nband + 1)
    // halo plans: degridding's own work list, in coarser chunks (each chunk stages its tile's region again)
    std::vector<int64_t> work_dg_begin;
    std::vector<int64_t> work_heavy_end; // per band: end of the heavy-tile chunks (they come first)
    // per band offset into d_heavy (size nband + 1): the tiles that reductions fill (heavy tiles; on halo
    // plans every tile some footprint reaches), then, from empty_begin[b], the tiles nothing writes
    std::vector<int64_t> heavy_begin;
    std::vector<int64_t> empty_begin;

    // ---- device
    double *d_scale = nullptr;
    float2 *d_rowdf = nullptr;   // uvw as double-float (FP32 path)
    ChanDF *d_chandf = nullptr;  // per-channel double-float scales (FP32 path)
    int *d_band = nullptr;
    BandGeom *d_bg = nullptr;
    uint32_t *d_items = nullptr;
    int64_t nitems = 0;
    int64_t *d_off = nullptr;
    int64_t nkeys = 0;
    double *d_tp = nullptr;   // n - 1 - tc per pixel (FP32 plans: the same 8 bytes as a float pair hi, lo)
    void *d_corr = nullptr;   // 1 / (n psi_u psi_v psi_w) per pixel, working precision
    WorkItem *d_work = nullptr;
    WorkItem *d_work_dg = nullptr;
    int *d_heavy = nullptr;
    // FP32 tile kernels: per-item geometry records in item order (optional)
    float4 *d_rec = nullptr;
    float2 *d_rph = nullptr;
    // Pruned plane transforms (planefft.cu), FP32 plans with power-of-two planes of 1024..8192 cells:
    // which 32 x 32 tiles of each w-plane any visibility touches, the tile-rows holding at least one such
    // tile, and t per pixel transposed to the column-pair order of the column kernels.
    bool pruned = false;
    uint32_t *d_occ = nullptr;       // [nband][Pmax][ntu][ntv / 32] bit tv of tile (tu, tv) in plane k
    uint32_t *d_rowocc = nullptr;    // [nband][Pmax][ntu / 32] bit tu: tile-row tu holds a touched tile
    int *d_rowlist = nullptr;        // occupied (plane, tile-row) pairs as k << 16 | tu, by band, then k
    std::vector<int64_t> rowlist_off;  // [nband][Pmax + 1]: first list entry of (b, k)
    float4 *d_tT = nullptr;          // [ny / 2][nx]: t of the column pair q at image row i (two float pairs)
    float2 *d_wk = nullptr;          // [nband][Pmax]: w-plane k of band b, w0 + k dw, as a float pair
    size_t bytes = 0;

    BandGeom geom(int b) const {
        BandGeom g;
        g.Nu = Nu; g.Nv = Nv; g.W = W; g.Ww = Ww; g.ntu = ntu; g.ntv = ntv;
        g.nkq = nkq; g.q = q; g.P = P[b]; g.band = b; g.nchan = nchan;
        g.u2cell = dl * Nu; g.v2cell = dm * Nv;
        g.inv_dw = wstack ? 1.0 / dw : 0.0;
        g.w0 = w0[b];
        g.tc = tc; g.beta = beta; g.inv_halfw = 2.0 / W;
        g.facet = (l0 != 0.0 || m0 != 0.0) ? 1 : 0;
        g.fa = fa; g.fb = fb; g.l0 = l0; g.m0 = m0;
        g.accumulate = 0;
        const double hw = 0.5 * W;
        g.hw = (float)hw;
        g.uv_oi = (int)std::floor(hw);
        g.uv_of = (float)(hw - std::floor(hw));
        const double O = wstack ? hw + w0[b] / dw : hw;
        g.w_oi = (int)std::floor(O);
        g.w_of = (float)(O - std::floor(O));
        g.inv_Nu = 1.0f / (float)Nu;
        g.inv_Nv = 1.0f / (float)Nv;
        g.w0_hi = (float)w0[b];
        g.w0_lo = (float)(w0[b] - (double)g.w0_hi);
        const double dws = wstack ? dw : 0.0;
        g.dw_hi = (float)dws;
        g.dw_lo = (float)(dws - (double)g.dw_hi);
        return g;
    }
    CoordSrc coords() const { return CoordSrc{(const double *)uvw, d_scale, d_rowdf, d_chandf}; }
    int64_t key(int b, int tile, int kq) const { return ((int64_t)b * ntu * ntv + tile) * nkq + kq; }
};

struct PsfSpec {
    const void *psf = nullptr;
    int nx = 0, ny = 0, nband = 0, prec = 0;
    void *spec = nullptr;   // complex [nband][2nx][ny+1]
    size_t bytes = 0;
};

struct FftKey {
    int n0, n1, batch, type;
    bool operator<(const FftKey &o) const {
        if (n0 != o.n0) return n0 < o.n0;
        if (n1 != o.n1) return n1 < o.n1;
        if (batch != o.batch) return batch < o.batch;
        return type < o.type;
    }
};

// Per-kernel device timing: CUDA events recorded around each launch on the
// launch stream while enabled, resolved when read.
struct Timing {
    bool on = false;
    struct Rec {
        std::string name;
        cudaEvent_t a, b;
        double bytes;
    };
    struct Total {
        int64_t launches = 0;
        double ms = 0, bytes = 0;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    std::map<std::string, Total> totals;
    int64_t own_launches = 0;   // kernels of this library launched while enabled
    cudaEvent_t get();
    void resolve();
    void clear();
    ~Timing();
};

struct Ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    size_t used = 0;
    std::string err;
    uint64_t clock = 0;
    std::vector<std::unique_ptr<Plan>> plans;
    std::map<std::string, DevBuf> bufs;
    // named buffers whose contents are kept between calls: for kept zeros the plan id (and plane
    // count) they were cleared for, for a twiddle table its length; dropped whenever the buffer is
    // reallocated
    std::map<std::string, std::pair<uint64_t, int>> zero_tag;
    uint64_t plan_serial = 0;
    std::map<FftKey, cufftHandle> ffts;
    std::vector<PsfSpec> spectra;
    Timing timing;
    // pfb_hessian_host: a copy stream joined to the caller's stream by events, and the host
    // pointers whose contents the scratch copies (and the plans built on them) hold
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_events;
    const void *host_data[3] = {nullptr, nullptr, nullptr};
    int64_t host_nrow = -1;
    int host_nchan = -1;
    cudaStream_t copy_stream_get();
    cudaEvent_t copy_event(size_t i);
    // Stream-ordered memory: every buffer comes from the context's own pool, allocated and freed in the
    // order of the stream of the call that needs it (cur), so neither allocation nor release waits for the
    // device.  Each call records `done` on its stream when its work is queued; pfb_plan_reset and
    // pfb_destroy release the buffers on the context's own stream `own` after that event.
    cudaMemPool_t pool = nullptr;
    cudaStream_t own = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t cur = nullptr;
    bool in_call = false;
    double last_lmax = 0.0, last_gamma = 0.0;   // pfb_last_step_bound
    void init_memory();                    // pool, own stream and done event (at creation)
    void release_all_buffers();            // free plans, spectra and scratch on `own` after `done`

    ~Ctx();
    void *dalloc(size_t bytes);            // counted against the budget
    void dfree(void *p, size_t bytes);
    void *scratch(const std::string &name, size_t bytes);  // grow-only named buffer
    size_t scratch_bytes(const std::string &name) const;
    void release(const std::string &name);     // free a named scratch buffer
    size_t available() const { return budget > used ? budget - used : 0; }
    void free_plan(Plan &p);
    void reset();
    // cached cuFFT plan of `batch` contiguous n0 x n1 transforms (1-D of length n0 when n1 == 0),
    // bound to the shared work area
    cufftHandle fft(int n0, int n1, int batch, cufftType type);
};

// colfft.cu: the FP32 column pass of the w-plane transforms over the image region (see there)
bool colfft_fits(int Nu, int Nv, int nx, int ny);
void colfft_planes(Ctx &ctx, float2 *data, int nplanes, int Nu, int Nv, int nx, int ny, bool inverse,
                   cudaStream_t st);
// twiddle table exp(-2 pi i m / n), m < n, kept in the context
const float2 *fft_twiddles(Ctx &ctx, int n, cudaStream_t st);
// tensor map of a plane block [nplanes][Nu][Nv] (8-byte cells) for 2 x box_rows x 1 boxes; false when the
// driver's encoder or the layout rules of the copy do not allow one
bool plane_tensor_map(CUtensorMap *map, float2 *data, int Nu, int Nv, int nplanes, int ny, int box_rows);

// planefft.cu: pruned FP32 plane transforms (see there)
bool pruned_fits(const Plan &p);
void build_pruned_tables(Ctx &ctx, Plan &p, cudaStream_t st);
void plane_forward(Ctx &ctx, const Plan &p, int b, const float *x, int k_lo, int k_hi, float2 *planes,
                   cudaStream_t st);
void plane_inverse(Ctx &ctx, const Plan &p, int b, int k_lo, int k_hi, float2 *planes, float *image,
                   cudaStream_t st);

// Scoped timer: records events around the enclosed launches when timing is on.
// `bytes` is the algorithmic traffic of the enclosed work; `launches` the number
// of this library's kernels it launches (cuFFT calls pass 0).
struct KTimer {
    Ctx &c;
    const char *name;
    cudaStream_t st;
    double bytes;
    cudaEvent_t a = nullptr;
    KTimer(Ctx &c_, const char *n, cudaStream_t s, double b, int launches = 1) : c(c_), name(n), st(s), bytes(b) {
        if (!c.timing.on) return;
        c.timing.own_launches += launches;
        a = c.timing.get();
        cudaEventRecord(a, st);
    }
    ~KTimer() {
        if (!a) return;
        cudaEvent_t b = c.timing.get();
        cudaEventRecord(b, st);
        c.timing.pending.push_back({name, a, b, bytes});
        if (c.timing.pending.size() > 8192) c.timing.resolve();
    }
};

// noalloc.cu: message of the last failure of a context-free call on this thread
extern thread_local std::string g_free_error;

// plan.cu
Plan &get_plan(Ctx &ctx, const pfb_geom &g, int prec, int64_t nrow, int nchan, const double *uvw,
               const double *freq, const int32_t *band, bool psf_grid, cudaStream_t st);
int kernel_support(double eps);

// wstack.cu
bool halo_fits(const Plan &p);
void build_item_records(Ctx &ctx, Plan &p, cudaStream_t st);
template <typename T>
void op_degrid(Ctx &ctx, const Plan &p, const T *image, cx_t<T> *vis, cudaStream_t st, bool accumulate = false);
// band_done (may be empty) is called after the last launch that writes band b of image, on st
template <typename T>
void op_grid(Ctx &ctx, const Plan &p, const cx_t<T> *vis, const T *wgt, bool unit_vis, T *image,
             cudaStream_t st, const std::function<void(int)> &band_done = {});
// H x = R^dagger W R x (Eq. 3) into hx; vis is scratch of nrow x nchan complex values.  On plans that list
// every visibility once (halo plans) the intermediate R x stays in item order: degridding writes (R x)_v at
// each item's position and gridding reads it back in the same order, with the weight w_v gathered by the
// gridding producers.  wgt_ready (may be NULL): an event after which wgt may be read; R x does not wait.
template <typename T>
void op_hessian(Ctx &ctx, const Plan &p, const T *x, const T *wgt, cx_t<T> *vis, T *hx, cudaStream_t st,
                cudaEvent_t wgt_ready = nullptr, const std::function<void(int)> &band_done = {});
template <typename T>
void op_wsum(Ctx &ctx, const Plan &p, const T *wgt, double *d_wsum, cudaStream_t st);

// image.cu
template <typename T>
void op_psf_conv(Ctx &ctx, int nx, int ny, int nband, const T *psf, const T *x, T *y, cudaStream_t st);
template <typename T>
double op_step_bound(Ctx &ctx, const Plan &p, const T *wgt, const T *psf, const double *wsum_h, double sigma,
                     int iters, int cg_iters, const T *z0, cudaStream_t st);
template <typename T>
void op_step(Ctx &ctx, const Plan &p, const pfb_params &prm, const T *wgt, const T *dirty,
             const T *psf, const double *wsum_h, T *x, T *dual, double *stats_h, cudaStream_t st);

}  // namespace pfb
