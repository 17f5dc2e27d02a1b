// C ABI of libpfb: argument checking, the context (device buffers, plans,
// cuFFT handles, PSF spectra) and the entry points declared in include/pfb.h.
#include "ctx.cuh"

#include <algorithm>

struct pfb_ctx {
    pfb::Ctx impl;
};

namespace pfb {

Ctx::~Ctx() {
    cudaSetDevice(device);
    release_all_buffers();
    for (auto &kv : ffts) cufftDestroy(kv.second);
    ffts.clear();
    for (cudaEvent_t e : copy_events) cudaEventDestroy(e);
    copy_events.clear();
    // destroying a stream, event or pool with work or frees still queued returns at once; the resources
    // go when that work is done
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    if (pool) cudaMemPoolDestroy(pool);
    if (own) cudaStreamDestroy(own);
    if (done) cudaEventDestroy(done);
}

void Ctx::init_memory() {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    PFB_CUDA(cudaMemPoolCreate(&pool, &props));
    // keep released memory for the context's later plans instead of returning it at every synchronisation
    uint64_t keep = budget;
    PFB_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    PFB_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    PFB_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
}

void Ctx::release_all_buffers() {
    if (!own) return;
    // the frees follow the work queued so far: inside a call the work on its stream, otherwise the last call's
    if (in_call) cudaEventRecord(done, cur);
    cudaStreamWaitEvent(own, done, 0);
    const cudaStream_t saved = cur;
    cur = own;
    for (auto &pp : plans) free_plan(*pp);
    plans.clear();
    for (auto &sp : spectra) dfree(sp.spec, sp.bytes);
    spectra.clear();
    for (auto &b : bufs)
        if (b.second.ptr) dfree(b.second.ptr, b.second.bytes);
    bufs.clear();
    zero_tag.clear();
    cur = saved;
}

cudaStream_t Ctx::copy_stream_get() {
    if (!copy_stream) PFB_CUDA(cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking));
    return copy_stream;
}

cudaEvent_t Ctx::copy_event(size_t i) {
    while (copy_events.size() <= i) {
        cudaEvent_t e;
        PFB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        copy_events.push_back(e);
    }
    return copy_events[i];
}

void *Ctx::dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (used + bytes > budget)
        throw Error(PFB_ERR_OOM, "HBM budget exceeded: need " + std::to_string(bytes) + " more bytes, " +
                                     std::to_string(available()) + " left of " + std::to_string(budget));
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? PFB_ERR_OOM : PFB_ERR_CUDA,
                    std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
    }
    used += bytes;
    return p;
}

void Ctx::dfree(void *p, size_t bytes) {
    if (!p) return;
    cudaFreeAsync(p, cur);
    used -= std::min(used, bytes == 0 ? (size_t)16 : bytes);
}

void *Ctx::scratch(const std::string &name, size_t bytes) {
    DevBuf &b = bufs[name];
    if (b.bytes >= bytes && b.ptr) return b.ptr;
    zero_tag.erase(name);
    if (b.ptr) {
        dfree(b.ptr, b.bytes);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    b.ptr = dalloc(bytes);
    b.bytes = bytes == 0 ? 16 : bytes;
    return b.ptr;
}

void Ctx::release(const std::string &name) {
    zero_tag.erase(name);
    auto it = bufs.find(name);
    if (it == bufs.end()) return;
    dfree(it->second.ptr, it->second.bytes);
    bufs.erase(it);
}

size_t Ctx::scratch_bytes(const std::string &name) const {
    auto it = bufs.find(name);
    return it == bufs.end() ? 0 : it->second.bytes;
}

void Ctx::free_plan(Plan &p) {
    auto fr = [&](void *q, size_t n) {
        if (q) dfree(q, n);
    };
    fr(p.d_scale, p.nchan * sizeof(double));
    fr(p.d_rowdf, (size_t)p.nrow * 3 * sizeof(float2));
    fr(p.d_chandf, p.nchan * sizeof(ChanDF));
    fr(p.d_band, p.nchan * sizeof(int));
    fr(p.d_bg, p.nband * sizeof(BandGeom));
    fr(p.d_items, (size_t)std::max<int64_t>(p.nitems, 1) * sizeof(uint32_t));
    fr(p.d_off, (size_t)(p.nkeys + 1) * sizeof(int64_t));
    fr(p.d_tp, (size_t)p.nx * p.ny * sizeof(double));
    fr(p.d_corr, (size_t)p.nx * p.ny * (p.prec == PFB_F64 ? 8 : 4));
    if (p.d_work) fr(p.d_work, std::max<size_t>((size_t)p.work_begin.back(), 1) * sizeof(WorkItem));
    if (p.d_work_dg) fr(p.d_work_dg, (size_t)p.work_dg_begin.back() * sizeof(WorkItem));
    p.d_work_dg = nullptr;
    if (p.d_heavy) fr(p.d_heavy, (size_t)p.heavy_begin.back() * sizeof(int));
    fr(p.d_rec, (size_t)p.nitems * sizeof(float4));
    fr(p.d_rph, (size_t)p.nitems * sizeof(float2));
    p.d_rec = nullptr;
    p.d_rph = nullptr;
    fr(p.d_occ, (size_t)p.nband * p.Pmax * p.ntu * (p.ntv / 32) * sizeof(uint32_t));
    fr(p.d_rowocc, (size_t)p.nband * p.Pmax * (p.ntu / 32) * sizeof(uint32_t));
    if (p.d_rowlist) fr(p.d_rowlist, std::max<size_t>((size_t)p.rowlist_off.back(), 1) * sizeof(int));
    fr(p.d_tT, (size_t)p.nx * p.ny * sizeof(float2));
    fr(p.d_wk, (size_t)p.nband * p.Pmax * sizeof(float2));
    p.d_occ = nullptr;
    p.d_rowocc = nullptr;
    p.d_rowlist = nullptr;
    p.d_tT = nullptr;
    p.d_wk = nullptr;
    p.pruned = false;
    p.d_scale = nullptr; p.d_rowdf = nullptr; p.d_chandf = nullptr; p.d_band = nullptr; p.d_bg = nullptr; p.d_items = nullptr; p.d_off = nullptr;
    p.d_tp = nullptr; p.d_corr = nullptr; p.d_work = nullptr; p.d_heavy = nullptr;
}

void Ctx::reset() { release_all_buffers(); }

cufftHandle Ctx::fft(int n0, int n1, int batch, cufftType type) {
    FftKey k{n0, n1, batch, (int)type};
    auto it = ffts.find(k);
    cufftHandle h;
    size_t ws = 0;
    if (it == ffts.end()) {
        PFB_CUFFT(cufftCreate(&h));
        PFB_CUFFT(cufftSetAutoAllocation(h, 0));
        int n[2] = {n0, n1};
        cufftResult r = cufftMakePlanMany(h, n1 > 0 ? 2 : 1, n, nullptr, 1, 0, nullptr, 1, 0, type, batch, &ws);
        if (r != CUFFT_SUCCESS) {
            cufftDestroy(h);
            throw Error(PFB_ERR_CUDA, "cufftMakePlanMany failed: " + std::to_string((int)r));
        }
        ffts[k] = h;
    } else {
        h = it->second;
        PFB_CUFFT(cufftGetSize(h, &ws));
    }
    // every handle uses the shared work area; grow it if this plan needs more
    void *work = scratch("fftwork", std::max<size_t>(ws, 256));
    PFB_CUFFT(cufftSetWorkArea(h, work));
    return h;
}

cudaEvent_t Timing::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    PFB_CUDA(cudaEventCreate(&e));
    return e;
}

void Timing::resolve() {
    for (auto &r : pending) {
        cudaEventSynchronize(r.b);
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        Total &t = totals[r.name];
        t.launches += 1;
        t.ms += ms;
        t.bytes += r.bytes;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}

void Timing::clear() {
    resolve();
    totals.clear();
    own_launches = 0;
}

Timing::~Timing() {
    for (auto &r : pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace pfb

using namespace pfb;

namespace {

// Runs f on the context; a call that queues device work passes its stream, on which the context's
// allocations and frees are then ordered and `done` is recorded at the end.
template <typename F>
int guarded(pfb_ctx *ctx, void *stream, F &&f) {
    if (!ctx) return PFB_ERR_ARG;
    Ctx &c = ctx->impl;
    c.err.clear();
    struct Bind {
        Ctx &c;
        Bind(Ctx &c_, cudaStream_t s) : c(c_) {
            c.cur = s;
            c.in_call = true;
        }
        ~Bind() {
            cudaEventRecord(c.done, c.cur);
            c.in_call = false;
        }
    };
    try {
        PFB_CUDA(cudaSetDevice(c.device));
        Bind bind(c, reinterpret_cast<cudaStream_t>(stream));
        f(c);
        return PFB_OK;
    } catch (const Error &e) {
        c.err = e.what();
        return e.code;
    } catch (const std::bad_alloc &) {
        c.err = "host allocation failed";
        return PFB_ERR_OOM;
    } catch (const std::exception &e) {
        c.err = e.what();
        return PFB_ERR_CUDA;
    }
}
// calls without device work (timing, reset): the stream stays the last call's
template <typename F>
int guarded_host(pfb_ctx *ctx, F &&f) {
    if (!ctx) return PFB_ERR_ARG;
    Ctx &c = ctx->impl;
    c.err.clear();
    try {
        PFB_CUDA(cudaSetDevice(c.device));
        f(c);
        return PFB_OK;
    } catch (const Error &e) {
        c.err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        c.err = e.what();
        return PFB_ERR_CUDA;
    }
}

void check_geom(const pfb_geom *g, pfb_prec prec) {
    PFB_REQUIRE(g != nullptr, "geom is NULL");
    PFB_REQUIRE(prec == PFB_F32 || prec == PFB_F64, "prec must be PFB_F32 or PFB_F64");
    PFB_REQUIRE(g->nx >= 2 && g->ny >= 2 && g->nx % 2 == 0 && g->ny % 2 == 0, "nx, ny must be even and >= 2");
    PFB_REQUIRE(g->nx <= 65536 && g->ny <= 65536, "nx, ny must be <= 65536");
    PFB_REQUIRE(g->nband >= 1 && g->nband <= 32, "nband must be in [1, 32]");
    PFB_REQUIRE(std::isfinite(g->dl) && std::isfinite(g->dm) && g->dl > 0 && g->dm > 0, "dl, dm must be > 0");
    PFB_REQUIRE((g->flags & ~(PFB_NO_DIVIDE_BY_N | PFB_NO_WTERM | PFB_NO_ITEM_RECORDS | PFB_ACCUMULATE |
                                PFB_NO_PRUNED_FFT)) == 0,
                "unknown flag bits");
    PFB_REQUIRE(std::isfinite(g->l0) && std::isfinite(g->m0), "l0, m0 must be finite");
    if (g->fov_l != 0)
        PFB_REQUIRE(std::fabs(g->fov_l - g->nx * g->dl) <= 1e-9 * std::fabs(g->fov_l), "fov_l != nx * dl");
    if (g->fov_m != 0)
        PFB_REQUIRE(std::fabs(g->fov_m - g->ny * g->dm) <= 1e-9 * std::fabs(g->fov_m), "fov_m != ny * dm");
    if (!(g->epsilon > 0 && g->epsilon < 1)) throw Error(PFB_ERR_EPS, "epsilon must be in (0, 1)");
    if (prec == PFB_F32 && g->epsilon < 1e-6)
        throw Error(PFB_ERR_EPS, "epsilon below 1e-6 is not reachable in PFB_F32; use PFB_F64");
    if (prec == PFB_F64 && g->epsilon < 1e-12) throw Error(PFB_ERR_EPS, "epsilon below 1e-12 is not reachable");
}

void check_data(int64_t nrow, int32_t nchan, const double *uvw, const double *freq, const int32_t *band) {
    PFB_REQUIRE(nrow >= 1 && nchan >= 1, "nrow and nchan must be >= 1");
    PFB_REQUIRE(uvw && freq && band, "uvw, freq and band_of_chan must not be NULL");
}

cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

void check_params(const pfb_params *prm, const pfb_geom *g) {
    PFB_REQUIRE(prm, "params is NULL");
    PFB_REQUIRE(prm->gamma > 0 && prm->sigma > 0 && prm->lambda >= 0, "need gamma > 0, sigma > 0, lambda >= 0");
    PFB_REQUIRE(prm->cg_iters >= 0 && prm->pd_iters >= 0, "iteration counts must be >= 0");
    PFB_REQUIRE(prm->basis_mask >= 1u && prm->basis_mask < 128u, "basis_mask must select bits 0..6");
    PFB_REQUIRE((prm->flags & ~(PFB_STEP_APPROX_GRADIENT | PFB_STEP_SAFE_GAMMA)) == 0, "unknown params flag bits");
    if (prm->basis_mask != 1u) {
        PFB_REQUIRE(prm->nlevel >= 1 && prm->nlevel <= 12, "nlevel must be in [1, 12]");
        PFB_REQUIRE(g->nx % (1 << prm->nlevel) == 0 && g->ny % (1 << prm->nlevel) == 0,
                    "wavelet bases need nx, ny divisible by 2^nlevel (periodised transform)");
    }
}

void run_step(Ctx &c, const Plan &p, pfb_prec prec, const pfb_params &prm, const void *wgt, const void *dirty,
              const void *psf, const double *wsum, void *x, void *dual, double *stats, cudaStream_t st) {
    if (prec == PFB_F64)
        op_step<double>(c, p, prm, (const double *)wgt, (const double *)dirty, (const double *)psf, wsum,
                        (double *)x, (double *)dual, stats, st);
    else
        op_step<float>(c, p, prm, (const float *)wgt, (const float *)dirty, (const float *)psf, wsum, (float *)x,
                       (float *)dual, stats, st);
}

double run_step_bound(Ctx &c, const Plan &p, pfb_prec prec, const pfb_params &prm, const void *wgt, const void *psf,
                      const double *wsum, const void *z0, int iters, cudaStream_t st) {
    const double lm = prec == PFB_F64
                          ? op_step_bound<double>(c, p, (const double *)wgt, (const double *)psf, wsum, prm.sigma,
                                                  iters, prm.cg_iters, (const double *)z0, st)
                          : op_step_bound<float>(c, p, (const float *)wgt, (const float *)psf, wsum, prm.sigma, iters,
                                                 prm.cg_iters, (const float *)z0, st);
    c.last_lmax = lm;
    c.last_gamma = 0.0;
    return lm;
}

}  // namespace

namespace pfb {

// The Hessian from host buffers.  On the caller's stream: uvw, freq, band, x and the weights in, the
// plan, R x of every band, then R^dagger Sigma^-1 band by band.  On the copy stream: band b of the result
// as soon as its last post-pass has run, overlapping the later bands.  The caller's stream then waits for
// the copy stream, so work queued after this call (or a synchronisation of the stream) sees the result.
template <typename T>
static void hessian_host(Ctx &c, const pfb_geom *g, int prec, int64_t nrow, int32_t nchan, const double *uvw,
                         const double *freq, const int32_t *band, const T *wgt, const T *x, T *y, cudaStream_t st) {
    const int64_t npix = (int64_t)g->nx * g->ny, nimg = npix * g->nband;
    double *d_uvw = (double *)c.scratch("host_uvw", (size_t)nrow * 3 * sizeof(double));
    double *d_freq = (double *)c.scratch("host_freq", (size_t)nchan * sizeof(double));
    int32_t *d_band = (int32_t *)c.scratch("host_band", (size_t)nchan * sizeof(int32_t));
    // plans built on the scratch copies belong to the host pointers they were copied from
    const void *key[3] = {uvw, freq, band};
    if (std::memcmp(key, c.host_data, sizeof(key)) != 0 || c.host_nrow != nrow || c.host_nchan != nchan) {
        PFB_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < c.plans.size();) {
            if (c.plans[i]->uvw == d_uvw) {
                c.free_plan(*c.plans[i]);
                c.plans.erase(c.plans.begin() + i);
            } else {
                ++i;
            }
        }
        std::memcpy(c.host_data, key, sizeof(key));
        c.host_nrow = nrow;
        c.host_nchan = nchan;
    }
    T *d_x = (T *)c.scratch("host_x", (size_t)nimg * sizeof(T));
    T *d_y = (T *)c.scratch("host_y", (size_t)nimg * sizeof(T));
    T *d_w = wgt ? (T *)c.scratch("host_wgt", (size_t)nrow * nchan * sizeof(T)) : nullptr;
    cudaStream_t cs = c.copy_stream_get();
    PFB_CUDA(cudaMemcpyAsync(d_uvw, uvw, (size_t)nrow * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(d_freq, freq, (size_t)nchan * sizeof(double), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(d_band, band, (size_t)nchan * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PFB_CUDA(cudaMemcpyAsync(d_x, x, (size_t)nimg * sizeof(T), cudaMemcpyHostToDevice, st));
    // the weights go in on the copy stream while R x runs (only R^dagger Sigma^-1 reads them), after the
    // work already on the caller's stream, which may still read the previous call's weights
    cudaEvent_t e_w = nullptr;
    if (wgt) {
        cudaEvent_t e_in = c.copy_event(0);
        e_w = c.copy_event(1);
        PFB_CUDA(cudaEventRecord(e_in, st));
        PFB_CUDA(cudaStreamWaitEvent(cs, e_in, 0));
        PFB_CUDA(cudaMemcpyAsync(d_w, wgt, (size_t)nrow * nchan * sizeof(T), cudaMemcpyHostToDevice, cs));
        PFB_CUDA(cudaEventRecord(e_w, cs));
    }
    cudaEvent_t e_out = c.copy_event(2);
    Plan &p = get_plan(c, *g, prec, nrow, nchan, d_uvw, d_freq, d_band, false, st);
    cx_t<T> *vis = (cx_t<T> *)c.scratch("hess_vis", (size_t)nrow * nchan * sizeof(cx_t<T>));
    op_hessian<T>(c, p, d_x, d_w, vis, d_y, st, e_w, [&](int b) {
        cudaEvent_t e = c.copy_event(3 + (size_t)b);
        PFB_CUDA(cudaEventRecord(e, st));
        PFB_CUDA(cudaStreamWaitEvent(cs, e, 0));
        PFB_CUDA(cudaMemcpyAsync(y + b * npix, d_y + b * npix, (size_t)npix * sizeof(T), cudaMemcpyDeviceToHost,
                                 cs));
    });
    PFB_CUDA(cudaEventRecord(e_out, cs));
    PFB_CUDA(cudaStreamWaitEvent(st, e_out, 0));
}

}  // namespace pfb

extern "C" {

const char *pfb_version(void) { return "pfb-gb300 0.1 (sm_103a)"; }

int pfb_kernel_support(double epsilon, pfb_prec prec) {
    if (!(epsilon > 0.0) || !std::isfinite(epsilon) || (prec != PFB_F32 && prec != PFB_F64)) return PFB_ERR_ARG;
    if (epsilon < (prec == PFB_F32 ? 1e-6 : 1e-12)) return PFB_ERR_EPS;
    return kernel_support(epsilon);
}

int pfb_timing(pfb_ctx *ctx, int enable) {
    return guarded_host(ctx, [&](Ctx &c) {
        c.timing.clear();
        c.timing.on = enable != 0;
    });
}

int pfb_timing_read(pfb_ctx *ctx, const char *kernel, int64_t *launches, double *total_ms, double *bytes) {
    return guarded_host(ctx, [&](Ctx &c) {
        PFB_REQUIRE(kernel && launches && total_ms, "kernel, launches and total_ms must not be NULL");
        c.timing.resolve();
        if (std::string(kernel) == "*") {
            *launches = c.timing.own_launches;
            double ms = 0, by = 0;
            for (auto &kv : c.timing.totals) {
                ms += kv.second.ms;
                by += kv.second.bytes;
            }
            *total_ms = ms;
            if (bytes) *bytes = by;
            return;
        }
        auto it = c.timing.totals.find(kernel);
        *launches = it == c.timing.totals.end() ? 0 : it->second.launches;
        *total_ms = it == c.timing.totals.end() ? 0.0 : it->second.ms;
        if (bytes) *bytes = it == c.timing.totals.end() ? 0.0 : it->second.bytes;
    });
}

int pfb_timing_names(pfb_ctx *ctx, char *buf, size_t len) {
    return guarded_host(ctx, [&](Ctx &c) {
        PFB_REQUIRE(buf && len > 0, "buf must hold at least one byte");
        c.timing.resolve();
        std::string s;
        for (auto &kv : c.timing.totals) s += (s.empty() ? "" : ",") + kv.first;
        std::snprintf(buf, len, "%s", s.c_str());
    });
}

int pfb_create(pfb_ctx **out, int device, size_t budget) {
    if (!out) return PFB_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PFB_ERR_ARG;
    }
    pfb_ctx *c = new (std::nothrow) pfb_ctx;
    if (!c) return PFB_ERR_OOM;
    c->impl.device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return PFB_ERR_CUDA;
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cudaDeviceGetAttribute(&c->impl.num_sms, cudaDevAttrMultiProcessorCount, device);
    c->impl.budget = budget ? budget : (size_t)(0.85 * (double)fr);
    try {
        c->impl.init_memory();
    } catch (const Error &) {
        cudaGetLastError();
        delete c;
        return PFB_ERR_CUDA;
    }
    *out = c;
    return PFB_OK;
}

void pfb_destroy(pfb_ctx *ctx) { delete ctx; }

const char *pfb_last_error(const pfb_ctx *ctx) { return ctx ? ctx->impl.err.c_str() : pfb::g_free_error.c_str(); }

int pfb_plan_reset(pfb_ctx *ctx) {
    return guarded_host(ctx, [&](Ctx &c) { c.reset(); });
}

int pfb_degrid(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, int64_t nrow, int32_t nchan, const double *uvw,
               const double *freq, const int32_t *band, const void *image, void *vis_out, void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        PFB_REQUIRE(image && vis_out, "image and vis_out must not be NULL");
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, S(stream));
        const bool acc = g->flags & PFB_ACCUMULATE;
        if (prec == PFB_F64) op_degrid<double>(c, p, (const double *)image, (double2 *)vis_out, S(stream), acc);
        else op_degrid<float>(c, p, (const float *)image, (float2 *)vis_out, S(stream), acc);
    });
}

int pfb_grid(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, int64_t nrow, int32_t nchan, const double *uvw,
             const double *freq, const int32_t *band, const void *vis, const void *wgt, void *image_out,
             void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        PFB_REQUIRE(vis && image_out, "vis and image_out must not be NULL");
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, S(stream));
        if (prec == PFB_F64)
            op_grid<double>(c, p, (const double2 *)vis, (const double *)wgt, false, (double *)image_out, S(stream));
        else
            op_grid<float>(c, p, (const float2 *)vis, (const float *)wgt, false, (float *)image_out, S(stream));
    });
}

static void wsum_to_host(Ctx &c, const Plan &p, pfb_prec prec, const void *wgt, double *wsum_out, cudaStream_t st) {
    double *d = (double *)c.scratch("wsum", 32 * sizeof(double));
    if (prec == PFB_F64) op_wsum<double>(c, p, (const double *)wgt, d, st);
    else op_wsum<float>(c, p, (const float *)wgt, d, st);
    PFB_CUDA(cudaMemcpyAsync(wsum_out, d, p.nband * sizeof(double), cudaMemcpyDeviceToHost, st));
    PFB_CUDA(cudaStreamSynchronize(st));
}

int pfb_dirty(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, int64_t nrow, int32_t nchan, const double *uvw,
              const double *freq, const int32_t *band, const void *vis, const void *wgt, void *image_out,
              double *wsum_out, void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        PFB_REQUIRE(vis && image_out, "vis and image_out must not be NULL");
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, S(stream));
        if (prec == PFB_F64)
            op_grid<double>(c, p, (const double2 *)vis, (const double *)wgt, false, (double *)image_out, S(stream));
        else
            op_grid<float>(c, p, (const float2 *)vis, (const float *)wgt, false, (float *)image_out, S(stream));
        if (wsum_out) wsum_to_host(c, p, prec, wgt, wsum_out, S(stream));
    });
}

int pfb_psf(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, int64_t nrow, int32_t nchan, const double *uvw,
            const double *freq, const int32_t *band, const void *wgt, void *psf_out, double *wsum_out,
            void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        PFB_REQUIRE(psf_out, "psf_out must not be NULL");
        PFB_REQUIRE(2 * g->nx <= 65536 && 2 * g->ny <= 65536, "PSF grid too large");
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, true, S(stream));
        if (prec == PFB_F64)
            op_grid<double>(c, p, nullptr, (const double *)wgt, true, (double *)psf_out, S(stream));
        else
            op_grid<float>(c, p, nullptr, (const float *)wgt, true, (float *)psf_out, S(stream));
        if (wsum_out) wsum_to_host(c, p, prec, wgt, wsum_out, S(stream));
    });
}

int pfb_hessian(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, int64_t nrow, int32_t nchan, const double *uvw,
                const double *freq, const int32_t *band, const void *wgt, const void *x, void *y_out,
                void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        PFB_REQUIRE(x && y_out, "x and y_out must not be NULL");
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, S(stream));
        const size_t cxs = prec == PFB_F64 ? 16 : 8;
        void *vis = c.scratch("hess_vis", (size_t)nrow * nchan * cxs);
        if (prec == PFB_F64)
            op_hessian<double>(c, p, (const double *)x, (const double *)wgt, (double2 *)vis, (double *)y_out,
                               S(stream));
        else
            op_hessian<float>(c, p, (const float *)x, (const float *)wgt, (float2 *)vis, (float *)y_out, S(stream));
    });
}

int pfb_hessian_host(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, int64_t nrow, int32_t nchan, const double *uvw,
                     const double *freq, const int32_t *band, const void *wgt, const void *x, void *y_out,
                     void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        PFB_REQUIRE(x && y_out, "x and y_out must not be NULL");
        if (prec == PFB_F64)
            hessian_host<double>(c, g, prec, nrow, nchan, uvw, freq, band, (const double *)wgt, (const double *)x,
                                 (double *)y_out, S(stream));
        else
            hessian_host<float>(c, g, prec, nrow, nchan, uvw, freq, band, (const float *)wgt, (const float *)x,
                                (float *)y_out, S(stream));
    });
}

int pfb_psf_conv(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, const void *psf, const void *x, void *y_out,
                 void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        PFB_REQUIRE(g != nullptr, "geom is NULL");
        PFB_REQUIRE(prec == PFB_F32 || prec == PFB_F64, "prec must be PFB_F32 or PFB_F64");
        PFB_REQUIRE(g->nx >= 2 && g->ny >= 2 && g->nx % 2 == 0 && g->ny % 2 == 0, "nx, ny must be even");
        PFB_REQUIRE(g->nband >= 1 && g->nband <= 32, "nband must be in [1, 32]");
        PFB_REQUIRE(psf && x && y_out, "psf, x and y_out must not be NULL");
        if (prec == PFB_F64)
            op_psf_conv<double>(c, g->nx, g->ny, g->nband, (const double *)psf, (const double *)x, (double *)y_out,
                                S(stream));
        else
            op_psf_conv<float>(c, g->nx, g->ny, g->nband, (const float *)psf, (const float *)x, (float *)y_out,
                               S(stream));
    });
}

int pfb_step(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, const pfb_params *prm, int64_t nrow, int32_t nchan,
             const double *uvw, const double *freq, const int32_t *band, const void *wgt, const void *dirty,
             const void *psf, const double *wsum, void *x_inout, void *dual_inout, int64_t *n_hessian_out,
             double *stats_out, void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        check_params(prm, g);
        PFB_REQUIRE(dirty && psf && wsum && x_inout && dual_inout, "dirty, psf, wsum, x and dual must not be NULL");
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, S(stream));
        run_step(c, p, prec, *prm, wgt, dirty, psf, wsum, x_inout, dual_inout, stats_out, S(stream));
        // known on the host: no synchronisation
        if (n_hessian_out) *n_hessian_out = (prm->flags & PFB_STEP_APPROX_GRADIENT) ? 0 : 1;
    });
}

int pfb_step_bound(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, const pfb_params *prm, int64_t nrow,
                   int32_t nchan, const double *uvw, const double *freq, const int32_t *band, const void *wgt,
                   const void *psf, const double *wsum, const void *z0, int32_t iters, double *lmax_out,
                   void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        check_params(prm, g);
        PFB_REQUIRE(psf && wsum && lmax_out, "psf, wsum and lmax_out must not be NULL");
        PFB_REQUIRE(iters >= 1, "iters must be >= 1");
        const cudaStream_t st = S(stream);
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, st);
        *lmax_out = run_step_bound(c, p, prec, *prm, wgt, psf, wsum, z0, iters, st);
    });
}

int pfb_last_step_bound(pfb_ctx *ctx, double *lmax_out, double *gamma_out) {
    return guarded_host(ctx, [&](Ctx &c) {
        if (lmax_out) *lmax_out = c.last_lmax;
        if (gamma_out) *gamma_out = c.last_gamma;
    });
}

int pfb_clean(pfb_ctx *ctx, const pfb_geom *g, pfb_prec prec, const pfb_params *prm, int32_t max_outer, double tol,
              int64_t nrow, int32_t nchan, const double *uvw, const double *freq, const int32_t *band,
              const void *vis, const void *wgt, void *dirty_out, void *psf_out, double *wsum_out, void *x_inout,
              void *dual_inout, int32_t *n_outer_out, int64_t *n_hessian_out, double *history_out, void *stream) {
    return guarded(ctx, stream, [&](Ctx &c) {
        check_geom(g, prec);
        check_data(nrow, nchan, uvw, freq, band);
        check_params(prm, g);
        PFB_REQUIRE(max_outer >= 0, "max_outer must be >= 0");
        PFB_REQUIRE(std::isfinite(tol), "tol must be finite");
        PFB_REQUIRE(vis && dirty_out && psf_out && wsum_out && x_inout && dual_inout && n_outer_out && n_hessian_out,
                    "vis, dirty_out, psf_out, wsum_out, x, dual, n_outer_out and n_hessian_out must not be NULL");
        PFB_REQUIRE(2 * g->nx <= 65536 && 2 * g->ny <= 65536, "PSF grid too large");
        const cudaStream_t st = S(stream);
        // 1. I^psf on the 2x field and the weight sums
        {
            Plan &pp = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, true, st);
            if (prec == PFB_F64) op_grid<double>(c, pp, nullptr, (const double *)wgt, true, (double *)psf_out, st);
            else op_grid<float>(c, pp, nullptr, (const float *)wgt, true, (float *)psf_out, st);
            wsum_to_host(c, pp, prec, wgt, wsum_out, st);
        }
        // 2. the 2x-field plan and its plane stack give their memory back; then I^d
        c.reset();
        Plan &p = get_plan(c, *g, prec, nrow, nchan, uvw, freq, band, false, st);
        if (prec == PFB_F64)
            op_grid<double>(c, p, (const double2 *)vis, (const double *)wgt, false, (double *)dirty_out, st);
        else
            op_grid<float>(c, p, (const float2 *)vis, (const float *)wgt, false, (float *)dirty_out, st);
        // 3. outer steps until the relative update reaches tol
        const bool exact = !(prm->flags & PFB_STEP_APPROX_GRADIENT);
        int32_t k = 0;
        int64_t nh = 1;   // I^d and I^psf: one half each
        pfb_params ps = *prm;
        if ((prm->flags & PFB_STEP_SAFE_GAMMA) && exact) {
            const double lm = run_step_bound(c, p, prec, *prm, wgt, psf_out, wsum_out, nullptr, PFB_SAFE_GAMMA_ITERS, st);
            nh += PFB_SAFE_GAMMA_ITERS;
            if (lm > 0) ps.gamma = std::min(prm->gamma, 1.9 / lm);
            c.last_gamma = ps.gamma;
        }
        while (k < max_outer) {
            double stats[3];
            run_step(c, p, prec, ps, wgt, dirty_out, psf_out, wsum_out, x_inout, dual_inout, stats, st);
            if (history_out) std::copy(stats, stats + 3, history_out + 3 * (size_t)k);
            ++k;
            nh += exact ? 1 : 0;
            if (tol > 0 && stats[1] <= tol) break;
        }
        *n_outer_out = k;
        *n_hessian_out = nh;
    });
}

}  // extern "C"
