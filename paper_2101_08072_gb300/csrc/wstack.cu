// R (degridding) and R^dagger Sigma^-1 (gridding) by w-stacking (Section 2,
// Eqs. 1 and 3).  See plan.cu for the factorisation that these kernels apply:
//
//   R x       = exp(-2 pi i w t_c) sum_k phi_w sum_{g} phi_u phi_v FFT2[E_k x][g]
//   R^dagger y = Re corr . sum_k exp(+2 pi i w_k t) IFFT2[S_k y]   (cropped)
//
// with E_k x = x corr exp(-2 pi i w_k t) zero padded to N_u x N_v, corr =
// 1/(n psihat_u psihat_v psihat_w), S_k the adjoint of the kernel gather on
// plane k, and rows with w < 0 mapped to (-u,-v,-w) with V -> conj V (exact for
// a real image).  Planes are processed in blocks that fit the HBM budget; with
// GB300's memory a whole band's stack is usually one block.
#include "ctx.cuh"

#include <algorithm>

namespace pfb {

// ------------------------------------------------------------------ pre-pass (R)
// Writes x corr exp(-2 pi i w_k t) for planes [k_lo, k_hi) at the pixel's grid
// position (i - nx/2 mod N_u, j - ny/2 mod N_v); the rest of each plane was zeroed.
// Per-pixel base of the plane phases: th0 = frac(w0 t) and dth = frac(dw t) = dth_hi + dth_lo.  FP64
// plans reduce in FP64 (t a double); FP32 plans hold t as a float pair and reduce in float-float
// arithmetic, since FP64 runs at a small fraction of the FP32 rate on this GPU.
__device__ __forceinline__ void plane_phase_base(const double *__restrict__ tp, int64_t p, const BandGeom &g,
                                                 double dw, double *th0, double *dth_hi, double *dth_lo) {
    const double t = tp[p];
    const double a0 = g.w0 * t, a1 = dw * t;
    const double d1 = a1 - rint(a1);
    *th0 = a0 - rint(a0);
    *dth_hi = d1;
    *dth_lo = 0.0;
}
__device__ __forceinline__ void plane_phase_base(const double *__restrict__ tp, int64_t p, const BandGeom &g,
                                                 double dw, float *th0, float *dth_hi, float *dth_lo) {
    (void)dw;
    const float2 t = reinterpret_cast<const float2 *>(tp)[p];
    float h, l;
    frac_prod_df(g.w0_hi, g.w0_lo, t.x, t.y, &h, &l);
    *th0 = h + l;
    frac_prod_df(g.dw_hi, g.dw_lo, t.x, t.y, dth_hi, dth_lo);
}

template <typename T>
__global__ void k_prepass(int nx, int ny, const T *__restrict__ x, const T *__restrict__ corr,
                          const double *__restrict__ tp, BandGeom g, int k_lo, int k_hi, double dw,
                          cx_t<T> *__restrict__ planes) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= (int64_t)nx * ny) return;
    const int i = (int)(p / ny), j = (int)(p - (int64_t)i * ny);
    const T c = x[p] * corr[p];
    int gu = i - nx / 2, gv = j - ny / 2;
    gu += gu < 0 ? g.Nu : 0;
    gv += gv < 0 ? g.Nv : 0;
    const int64_t pos = (int64_t)gu * g.Nv + gv;
    const int64_t plane_sz = (int64_t)g.Nu * g.Nv;
    // phase of plane k in turns: (w0 + k dw) t = th0 + k dth, both reduced mod 1 once per
    // pixel; the per-plane sum is formed in the working precision
    T th0, dth_hi, dth_lo;
    plane_phase_base(tp, p, g, dw, &th0, &dth_hi, &dth_lo);
    for (int k = k_lo; k < k_hi; ++k) {
        T cs = 1, sn = 0;
        if (g.Ww > 1) sincos_turns(plane_turns(k, th0, dth_hi, dth_lo), &sn, &cs);
        cx_t<T> v;
        v.x = c * cs;
        v.y = -c * sn;
        planes[(int64_t)(k - k_lo) * plane_sz + pos] = v;
    }
}

// ------------------------------------------------------------------ gather (R)
// One thread per home item of band g.band: interpolate the W_w planes x W x W taps
// of the visibility, apply exp(-2 pi i w t_c) and the Hermitian flip.  Items whose
// first plane lies below k_lo add to the partial sum of an earlier block.
template <typename T>
__global__ void __launch_bounds__(256) k_gather(const uint32_t *__restrict__ items, int64_t n_items,
                                                CoordSrc src, BandGeom g, int k_lo, int k_hi,
                                                const cx_t<T> *__restrict__ planes, cx_t<T> *__restrict__ vis) {
    const int64_t plane_sz = (int64_t)g.Nu * g.Nv;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < n_items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t code = items[it];
        if (code >> 30) continue;   // spill copy of a visibility homed elsewhere
        const int64_t v = code;
        const int64_t row = v / g.nchan;
        const int ch = (int)(v - row * g.nchan);
        const VisCoord<T> c = vis_coord<T>(src, row, ch, g);
        if (c.k0 >= k_hi || c.k0 + g.Ww <= k_lo) continue;
        T ku[MAX_W], kv[MAX_W], kw[MAX_W];
        es_taps<T>(c.ou, g.W, g, ku);
        es_taps<T>(c.ov, g.W, g, kv);
        if (g.Ww > 1) es_taps<T>(c.ow, g.Ww, g, kw);
        else kw[0] = 1;
        T ar = 0, ai = 0;
        for (int cw = 0; cw < g.Ww; ++cw) {
            const int k = c.k0 + cw;
            if (k < k_lo || k >= k_hi) continue;
            const cx_t<T> *pl = planes + (int64_t)(k - k_lo) * plane_sz;
            T pr = 0, pi = 0;
            for (int a = 0; a < g.W; ++a) {
                int gu = c.gu0 + a;
                gu -= gu >= g.Nu ? g.Nu : 0;
                const cx_t<T> *prow = pl + (int64_t)gu * g.Nv;
                T rr = 0, ri = 0;
                if (c.gv0 + g.W <= g.Nv) {
                    for (int b = 0; b < g.W; ++b) {
                        const cx_t<T> gv = prow[c.gv0 + b];
                        rr += kv[b] * gv.x;
                        ri += kv[b] * gv.y;
                    }
                } else {
                    for (int b = 0; b < g.W; ++b) {
                        int gvi = c.gv0 + b;
                        gvi -= gvi >= g.Nv ? g.Nv : 0;
                        const cx_t<T> gv = prow[gvi];
                        rr += kv[b] * gv.x;
                        ri += kv[b] * gv.y;
                    }
                }
                pr += ku[a] * rr;
                pi += ku[a] * ri;
            }
            ar += kw[cw] * pr;
            ai += kw[cw] * pi;
        }
        // exp(-2 pi i w t_c)
        T cs = 1, sn = 0;
        if (g.tc != 0.0 || g.facet) sincos_turns(c.ph, &sn, &cs);
        T vr = ar * cs + ai * sn;
        T vi = ai * cs - ar * sn;
        if (c.flip) vi = -vi;
        cx_t<T> out;
        if (g.accumulate || c.k0 < k_lo) {
            out = vis[v];
            out.x += vr;
            out.y += vi;
        } else {
            out.x = vr;
            out.y = vi;
        }
        vis[v] = out;
    }
}

// ------------------------------------------------------------------ gridding (R^dagger)
template <typename T>
__device__ __forceinline__ void smem_add(cx_t<T> *cell, T re, T im) {
    atomicAdd(&cell->x, re);
    atomicAdd(&cell->y, im);
}

template <typename T>
__device__ __forceinline__ void global_add(cx_t<T> *cell, cx_t<T> v);
template <>
__device__ __forceinline__ void global_add<float>(float2 *cell, float2 v) {
    atomicAdd(cell, v);   // vector reduction (sm_90+)
}
template <>
__device__ __forceinline__ void global_add<double>(double2 *cell, double2 v) {
    atomicAdd(&cell->x, v.x);
    atomicAdd(&cell->y, v.y);
}

// One CTA per work item (a tile of TILE x TILE cells of band g.band, or a chunk
// of a heavy tile's items).  The CTA owns its tile's cells: it scatters every item
// listed for the tile (home items and spill copies of neighbours' items) into a
// ring of W_w + q - 1 shared-memory planes, sweeping the w buckets in order; after
// bucket kq the planes [kq q, kq q + q) are complete and are flushed to HBM with
// coalesced stores (plain mode) or vector reductions (heavy-tile chunks).
template <typename T>
__global__ void __launch_bounds__(256) k_grid_tiles(const WorkItem *__restrict__ work,
                                                    const uint32_t *__restrict__ items,
                                                    const int64_t *__restrict__ off, CoordSrc src,
                                                    const cx_t<T> *__restrict__ vis, const T *__restrict__ wgt,
                                                    int unit_vis, BandGeom g, int k_lo, int k_hi,
                                                    cx_t<T> *__restrict__ planes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx_t<T> *ring = reinterpret_cast<cx_t<T> *>(smem_raw);
    const int R = g.Ww + g.q - 1;
    const int cells = TILE * TILE;
    const WorkItem wi = work[blockIdx.x];
    const int tu = wi.tile / g.ntv, tv = wi.tile - tu * g.ntv;
    const int64_t plane_sz = (int64_t)g.Nu * g.Nv;
    for (int e = threadIdx.x; e < R * cells; e += blockDim.x) ring[e] = cx_t<T>{0, 0};

    const int64_t kbase = ((int64_t)g.band * g.ntu * g.ntv + wi.tile) * g.nkq;
    int kq_first, kq_last;
    if (!wi.atomic_mode) {
        kq_first = max(0, (k_lo - g.Ww + 1) / g.q);
        kq_last = (k_hi - 1) / g.q;
    } else {
        if (wi.end <= wi.begin) return;
        // buckets holding the first and last item of the chunk
        int lo = 0, hi = g.nkq - 1;
        while (lo < hi) {   // last bucket whose start <= begin
            int mid = (lo + hi + 1) >> 1;
            if (off[kbase + mid] <= wi.begin) lo = mid; else hi = mid - 1;
        }
        kq_first = lo;
        lo = kq_first; hi = g.nkq - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[kbase + mid] <= wi.end - 1) lo = mid; else hi = mid - 1;
        }
        kq_last = lo + (g.Ww - 1 + g.q - 1) / g.q;   // trailing planes of the last bucket
        kq_first = max(kq_first, max(0, (k_lo - g.Ww + 1) / g.q));
        kq_last = min(kq_last, (k_hi - 1) / g.q);
    }
    __syncthreads();
    for (int kq = kq_first; kq <= kq_last; ++kq) {
        int64_t s = kq < g.nkq ? off[kbase + kq] : wi.end;
        int64_t e = kq < g.nkq ? off[kbase + kq + 1] : wi.end;
        s = max(s, (int64_t)wi.begin);
        e = min(e, (int64_t)wi.end);
        // each thread takes a contiguous run of the bucket's items, so that the 32
        // lanes of a warp work on items far apart (different rows): consecutive
        // items are consecutive channels of one row and hit the same cells
        const int64_t n = e - s;
        const int64_t per = (n + blockDim.x - 1) / blockDim.x;
        const int64_t i_beg = s + per * threadIdx.x, i_end = min(e, i_beg + per);
        for (int64_t it = i_beg; it < i_end; ++it) {
            const uint32_t code = items[it];
            const int64_t v = code & VIS_MASK;
            const int du = (code >> 30) & 1, dv = code >> 31;
            const int64_t row = v / g.nchan;
            const int ch = (int)(v - row * g.nchan);
            const VisCoord<T> c = vis_coord<T>(src, row, ch, g);
            if (c.k0 >= k_hi || c.k0 + g.Ww <= k_lo) continue;
            T yr, yi;
            if (unit_vis) { yr = 1; yi = 0; }
            else { const cx_t<T> y = vis[v]; yr = y.x; yi = y.y; }
            if (wgt) { const T w = wgt[v]; yr *= w; yi *= w; }
            if (c.flip) yi = -yi;
            // multiply by exp(+2 pi i w t_c) (adjoint of the degridding phase)
            if (g.tc != 0.0 || g.facet) {
                T cs, sn;
                sincos_turns(c.ph, &sn, &cs);
                const T r0 = yr * cs - yi * sn;
                yi = yr * sn + yi * cs;
                yr = r0;
            }
            T ku[MAX_W], kv[MAX_W], kw[MAX_W];
            es_taps<T>(c.ou, g.W, g, ku);
            es_taps<T>(c.ov, g.W, g, kv);
            if (g.Ww > 1) es_taps<T>(c.ow, g.Ww, g, kw);
            else kw[0] = 1;
            const int lu = c.gu0 - (c.gu0 / TILE) * TILE - du * TILE;
            const int lv = c.gv0 - (c.gv0 / TILE) * TILE - dv * TILE;
            const int a0 = max(0, -lu), a1 = min(g.W, TILE - lu);
            const int b0 = max(0, -lv), b1 = min(g.W, TILE - lv);
            for (int cw = 0; cw < g.Ww; ++cw) {
                const int k = c.k0 + cw;
                if (k < k_lo || k >= k_hi) continue;
                cx_t<T> *slot = ring + (k % R) * cells;
                const T fr = kw[cw] * yr, fi = kw[cw] * yi;
                for (int a = a0; a < a1; ++a) {
                    const T gr = ku[a] * fr, gi = ku[a] * fi;
                    cx_t<T> *srow = slot + (lu + a) * TILE + lv;
                    for (int b = b0; b < b1; ++b) smem_add<T>(srow + b, kv[b] * gr, kv[b] * gi);
                }
            }
        }
        __syncthreads();
        // planes [kq q, kq q + q) are complete
        const int p0 = max(kq * g.q, k_lo), p1 = min(kq * g.q + g.q, k_hi);
        for (int k = p0; k < p1; ++k) {
            cx_t<T> *slot = ring + (k % R) * cells;
            cx_t<T> *dst = planes + (int64_t)(k - k_lo) * plane_sz + (int64_t)(tu * TILE) * g.Nv + tv * TILE;
            for (int e2 = threadIdx.x; e2 < cells; e2 += blockDim.x) {
                const int r = e2 / TILE, cc = e2 - r * TILE;
                const cx_t<T> val = slot[e2];
                if (wi.atomic_mode) {
                    if (val.x != 0 || val.y != 0) global_add<T>(dst + (int64_t)r * g.Nv + cc, val);
                } else {
                    dst[(int64_t)r * g.Nv + cc] = val;
                }
                slot[e2] = cx_t<T>{0, 0};
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ FP32 gridding by residue classes
// One CTA per work item: the items of one uv tile, or a chunk of a heavy tile's
// items.  The plan lists every visibility once, in the tile of its first-tap cell;
// its footprint reaches the W - 1 cells past the tile's far edges, which belong to the
// neighbouring tiles.  Sums go straight to the planes in HBM by global vector
// reductions (one instruction per plane and cell) into cells zeroed before the
// launch: the tiles a CTA works on stay in L2 meanwhile, and no shared-memory copy of
// the region is kept (floating-point adds to shared memory would be compare-and-swap
// loops).  Items are processed in chunks of at most res_ch(W) records of one w bucket.
//
// The CTA is warp-specialised.  Three producer warps stage chunk i+1 (one record per
// thread: coordinates, ES taps, weighted and phase-rotated value) into one of two
// shared buffers while nine consumer warps scatter chunk i from the other; named
// barriers hand each buffer back and forth (FULL: producers -> consumers, EMPTY:
// consumers -> producers).  The producers keep their global loads two chunks ahead:
// item codes of chunk i+2 and raw inputs (record, visibility, weight) of chunk i+1 are
// in flight while chunk i is staged.  With 56 registers per thread three CTAs share
// an SM.
//
// The consumers form groups of W * W threads: thread (a, b) of a group owns the
// footprint cell whose local indices are congruent to (a, b) mod W (exactly one per
// visibility), keeps the W_w plane sums of that cell in registers, and adds them to
// the planes only when its cell changes.  The plan sorts every bucket by first-tap
// cell, so in the dense tiles a thread stays on one cell for long runs of
// visibilities.  Staging does the per-visibility index work once: for every residue
// class j it stores the ES tap that lands on that class together with a packed cell
// key (u cell in the u entry, v cell in the v entry), so a scatter step is two
// 8-byte loads, an OR and a compare, one multiply and 2 W_w FMAs.  All items of a
// bucket start on the same w plane, so the planes of a run are set once per bucket,
// for all threads alike.
//
// cells a CTA's items reach, per axis: the tile and the W - 1 cells past its far edge
__host__ __device__ constexpr int res_edge(int W) { return TILE + W - 1; }
constexpr int GRID_NP = 96;         // producer threads (3 warps)
constexpr int GRID_NC = 288;        // consumer threads (9 warps: 8 groups of 36 at W = 6)
constexpr int GRID_NT = GRID_NP + GRID_NC;
// named barriers (0 is __syncthreads)
constexpr int BAR_FULL = 1, BAR_EMPTY = 3;
// packed cell key: (u + 64) << 25 | (v + 64) << 18 (the low bits are zero; plans of this path keep
// their plane count below 2^18)
constexpr int KEY_PLANE_BITS = 18;
constexpr uint32_t KEY_NONE = 0xffffffffu;   // decodes to u = 63, outside every reach

// records per chunk: one per producer thread
__host__ __device__ constexpr int res_ch(int W) { return GRID_NP; }
// w-tap row stride in float2: even, so a record's row starts on 16 bytes
__host__ __device__ constexpr int res_ws(int Ww) { return (Ww + 1) & ~1; }

struct ResSmem {
    int ru[2], rv[2], wy[2], meta, total;
};

__host__ __device__ inline ResSmem res_layout(int W, int Ww) {
    ResSmem L;
    const int ch = res_ch(W);
    int o = 0;
    for (int s = 0; s < 2; ++s) {
        L.ru[s] = o; o += ch * W * (int)sizeof(float2);
        L.rv[s] = o; o += ch * W * (int)sizeof(float2);
        L.wy[s] = o; o += ch * res_ws(Ww) * (int)sizeof(float2);
    }
    L.meta = o; o += 4 * (int)sizeof(int4);
    L.total = o;
    return L;
}

// barrier ids are immediates, so that only the barriers used are reserved
template <int ID, int N>
__device__ __forceinline__ void named_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory");
}
template <int ID, int N>
__device__ __forceinline__ void named_arrive() {
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(N) : "memory");
}
// buffer sb of a FULL / EMPTY pair
template <int ID>
__device__ __forceinline__ void pair_sync(int sb) {
    if (sb) named_sync<ID + 1, GRID_NT>(); else named_sync<ID, GRID_NT>();
}
template <int ID>
__device__ __forceinline__ void pair_arrive(int sb) {
    if (sb) named_arrive<ID + 1, GRID_NT>(); else named_arrive<ID, GRID_NT>();
}

// raw inputs of one record, held in registers between prefetch and staging
struct RawRec {
    uint32_t code;
    float2 u, v, w;   // uvw of the row as double-float (coordinates computed here)
    float4 rec;       // precomputed item record (see k_item_records)
    float2 ph;        // precomputed phase rotor
    float2 y;
    float wt;
};

// ---- precomputed item records
// The geometry of an item (its first-tap cell relative to its tile, first plane,
// Hermitian flip, fractional tap offsets and the rotor exp(2 pi i w t_c)) depends
// only on uvw, the frequencies and the plan, so a plan that has the room keeps it
// for every item, in item order: 16 + 8 bytes streamed per item instead of a
// gathered uvw row and the double-float coordinate arithmetic on every call.
//   rec = (ou, ov, ow, bits): bits = (lu + 32) | (lv + 32) << 6 | flip << 12 | k0 << 13
//   rph = (cos, sin) of 2 pi w t_c
__device__ __forceinline__ uint32_t rec_bits(int lu, int lv, bool flip, int k0) {
    return (uint32_t)(lu + 32) | ((uint32_t)(lv + 32) << 6) | (flip ? 1u << 12 : 0u) | ((uint32_t)k0 << 13);
}

__global__ void k_item_records(const uint32_t *__restrict__ items, int64_t i0, int64_t n, CoordSrc src, BandGeom g,
                               float4 *__restrict__ rec, float2 *__restrict__ rph) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + e;
        const uint32_t code = items[i];
        const uint32_t v = code & VIS_MASK;
        const int du = (code >> 30) & 1, dv = code >> 31;
        const uint32_t row = v / (uint32_t)g.nchan;
        const int ch = (int)(v - row * (uint32_t)g.nchan);
        const VisCoord<float> c = vis_coord32(src.rowdf, row, src.chandf[ch], g);
        const int lu = (c.gu0 & (TILE - 1)) - du * TILE;
        const int lv = (c.gv0 & (TILE - 1)) - dv * TILE;
        rec[i] = make_float4(c.ou, c.ov, c.ow, __uint_as_float(rec_bits(lu, lv, c.flip, c.k0)));
        float cs = 1.f, sn = 0.f;
        if (g.tc != 0.0 || g.facet) sincos_turns(c.ph, &sn, &cs);
        rph[i] = make_float2(cs, sn);
    }
}

template <int W, int Ww, bool REC>
__global__ void __launch_bounds__(GRID_NT, 3)
k_grid_res(const WorkItem *__restrict__ work, const uint32_t *__restrict__ items, const int64_t *__restrict__ off,
           CoordSrc src, const float4 *__restrict__ recs, const float2 *__restrict__ rph,
           const float2 *__restrict__ vis, const float *__restrict__ wgt, int unit_vis, int item_order, BandGeom g,
           int k_lo, int k_hi, float2 *__restrict__ planes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int E = res_edge(W);
    constexpr int WS = res_ws(Ww);
    constexpr int CH = res_ch(W);
    constexpr int G = W * W;         // consumer threads of a group (one per residue class)
    constexpr int NG = GRID_NC / G;  // consumer groups
    constexpr int RPG = CH / NG;     // records of one group in a chunk
    const ResSmem L = res_layout(W, Ww);
    int4 *meta = reinterpret_cast<int4 *>(smem_raw + L.meta);
    const WorkItem wi = work[blockIdx.x];
    if (wi.end <= wi.begin) return;
    const int tu = wi.tile / g.ntv, tv = wi.tile - tu * g.ntv;
    const int64_t plane_sz = (int64_t)g.Nu * g.Nv;

    if (threadIdx.x < GRID_NP) {
        // ================================================================ producers
        const int pt = threadIdx.x;
        const int64_t kbase = ((int64_t)g.band * g.ntu * g.ntv + wi.tile) * g.nkq;
        auto bucket_of = [&](int64_t pos) {
            int lo = 0, hi = g.nkq - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off[kbase + mid] <= pos) lo = mid; else hi = mid - 1;
            }
            return lo;
        };
        // A bucket's items (its part of this work item) are split into NG contiguous parts, one per
        // consumer group; chunk c of the bucket holds records [c RPG, c RPG + RPG) of every part, so
        // a group walks its part in order and its register runs break only where the cell changes.
        struct CPos {
            int kq, P, c, nch;   // bucket, part length, chunk within the bucket, chunks of the bucket
            int64_t s, e;        // the bucket's item range within this work item
            bool end;
        };
        auto init_bucket = [&](CPos &q) {
            q.s = max(off[kbase + q.kq], (int64_t)wi.begin);
            q.e = min(off[kbase + q.kq + 1], (int64_t)wi.end);
            q.P = (int)((q.e - q.s + NG - 1) / NG);
            q.nch = (q.P + RPG - 1) / RPG;
            q.c = 0;
        };
        auto advance = [&](CPos &q) {
            if (q.end) return;
            if (++q.c < q.nch) return;
            do {
                ++q.kq;
                if (q.kq >= g.nkq || off[kbase + q.kq] >= wi.end) {
                    q.end = true;
                    return;
                }
                init_bucket(q);
            } while (q.e <= q.s);
        };
        // this producer thread's item in chunk q (record slot pt), or -1
        auto item_of = [&](const CPos &q) -> int64_t {
            if (q.end || pt >= NG * RPG) return -1;
            const int gq = pt / RPG, j = pt - gq * RPG;
            const int64_t idx = q.s + (int64_t)gq * q.P + (int64_t)q.c * RPG + j;
            return idx < min(q.s + (int64_t)(gq + 1) * q.P, q.e) ? idx : -1;
        };
        auto load_raw = [&](RawRec &q, int64_t idx) {
            const uint32_t v = q.code & VIS_MASK;
            if constexpr (REC) {
                q.rec = recs[idx];
                q.ph = rph[idx];
            } else {
                const uint32_t row = v / (uint32_t)g.nchan;
                q.u = src.rowdf[3 * row + 0];
                q.v = src.rowdf[3 * row + 1];
                q.w = src.rowdf[3 * row + 2];
            }
            q.y = unit_vis ? make_float2(1.f, 0.f) : vis[item_order ? idx : (int64_t)v];
            q.wt = wgt ? wgt[v] : 1.f;
        };
        // kernel constants in FP32, converted once (FP64 arithmetic is slow on this GPU)
        const float ihw = (float)g.inv_halfw, b2 = es_b2(g.beta);
        // record t of buffer sb: per residue class the tap and the packed cell key
        auto stage = [&](const RawRec &q, int t, int sb) {
            float2 *ru = reinterpret_cast<float2 *>(smem_raw + L.ru[sb]);
            float2 *rv = reinterpret_cast<float2 *>(smem_raw + L.rv[sb]);
            float2 *rwy = reinterpret_cast<float2 *>(smem_raw + L.wy[sb]);
            VisCoord<float> c;
            int lu, lv;
            float cs2 = 1.f, sn = 0.f;
            if constexpr (REC) {
                const uint32_t bits = __float_as_uint(q.rec.w);
                c.ou = q.rec.x;
                c.ov = q.rec.y;
                c.ow = q.rec.z;
                lu = (int)(bits & 63u) - 32;
                lv = (int)((bits >> 6) & 63u) - 32;
                c.flip = (bits >> 12) & 1u;
                c.k0 = (int)(bits >> 13);
                cs2 = q.ph.x;
                sn = q.ph.y;
            } else {
                const uint32_t v = q.code & VIS_MASK;
                const int du = (q.code >> 30) & 1, dv = q.code >> 31;
                const uint32_t row = v / (uint32_t)g.nchan;
                const int ch = (int)(v - row * (uint32_t)g.nchan);
                const ChanDF cs = src.chandf[ch];
                float2 u = q.u, vv = q.v, w = q.w;
                c.flip = w.x < 0.0f || (w.x == 0.0f && w.y < 0.0f);
                if (c.flip) {
                    u.x = -u.x; u.y = -u.y; vv.x = -vv.x; vv.y = -vv.y; w.x = -w.x; w.y = -w.y;
                }
                float p, e;
                int g0;
                df_mul(u.x, u.y, cs.su_hi, cs.su_lo, p, e);
                df_tap(p, e, g.uv_oi, g.uv_of, g.hw, g0, c.ou);
                c.gu0 = wrap_mod(g0, g.Nu, g.inv_Nu);
                df_mul(vv.x, vv.y, cs.sv_hi, cs.sv_lo, p, e);
                df_tap(p, e, g.uv_oi, g.uv_of, g.hw, g0, c.ov);
                c.gv0 = wrap_mod(g0, g.Nv, g.inv_Nv);
                df_mul(w.x, w.y, cs.sp_hi, cs.sp_lo, p, e);
                c.ph = (p - rintf(p)) + e;
                if (Ww > 1) {
                    df_mul(w.x, w.y, cs.sw_hi, cs.sw_lo, p, e);
                    df_tap(p, e, g.w_oi, g.w_of, g.hw, g0, c.ow);
                    c.k0 = g0 < 0 ? 0 : (g0 > g.P - Ww ? g.P - Ww : g0);
                } else {
                    c.k0 = 0;
                    c.ow = 0.0f;
                }
                lu = (c.gu0 & (TILE - 1)) - du * TILE;
                lv = (c.gv0 & (TILE - 1)) - dv * TILE;
                if (g.tc != 0.0 || g.facet) sincos_turns(c.ph, &sn, &cs2);
            }
            float yr = q.y.x * q.wt, yi = q.y.y * q.wt;
            if (c.k0 >= k_hi || c.k0 + Ww <= k_lo) {
                yr = yi = 0.f;   // none of its planes is in this block: scattered with zero weight
            } else {
                if (c.flip) yi = -yi;
                const float r0 = yr * cs2 - yi * sn;
                yi = yr * sn + yi * cs2;
                yr = r0;
            }
            const int mu = (lu + 2 * TILE) % W, mv = (lv + 2 * TILE) % W;
            // tap i (cell lu + i) lands on residue class (mu + i) mod W; taps in natural order keep the
            // offsets compile-time constants, and the cell keys step by one cell per tap
            const uint32_t ku0 = (uint32_t)(lu + 64) << 25, kv0 = (uint32_t)(lv + 64) << KEY_PLANE_BITS;
            const float xu = c.ou * ihw, xv = c.ov * ihw;
            float2 *rut = ru + t * W, *rvt = rv + t * W;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int ju = mu + i - (mu + i >= W ? W : 0), jv = mv + i - (mv + i >= W ? W : 0);
                rut[ju] = make_float2(es_kernel_x(fmaf((float)i, ihw, xu), b2),
                                      __uint_as_float(ku0 + ((uint32_t)i << 25)));
                rvt[jv] = make_float2(es_kernel_x(fmaf((float)i, ihw, xv), b2),
                                      __uint_as_float(kv0 + ((uint32_t)i << KEY_PLANE_BITS)));
            }
            if (Ww > 1) {
                const float xw = c.ow * ihw;
                float kw[Ww];
#pragma unroll
                for (int i = 0; i < Ww; ++i) kw[i] = es_kernel_x(fmaf((float)i, ihw, xw), b2);
                // the row starts on 16 bytes (WS even): pairs of taps as 16-byte stores
                float4 *w4 = reinterpret_cast<float4 *>(rwy + t * WS);
#pragma unroll
                for (int i = 0; i + 1 < Ww; i += 2)
                    w4[i / 2] = make_float4(kw[i] * yr, kw[i] * yi, kw[i + 1] * yr, kw[i + 1] * yi);
                if (Ww & 1) rwy[t * WS + Ww - 1] = make_float2(kw[Ww - 1] * yr, kw[Ww - 1] * yi);
            } else {
                rwy[t * WS] = make_float2(yr, yi);
            }
        };

        // chunk i at cp, i+1 at np_, i+2 at mp: raw inputs of i+1 and item codes of i+2 are in flight
        // while chunk i is staged
        CPos cp;
        cp.kq = bucket_of(wi.begin);
        cp.end = false;
        init_bucket(cp);
        RawRec raw;
        int64_t ic = item_of(cp);
        raw.code = ic >= 0 ? items[ic] : 0u;
        if (ic >= 0) load_raw(raw, ic);
        CPos np_ = cp;
        advance(np_);
        int64_t in_ = item_of(np_);
        RawRec nxt;
        nxt.code = in_ >= 0 ? items[in_] : 0u;
        int i = 0;
        while (!cp.end) {
            const int sb = i & 1;
            if (in_ >= 0) load_raw(nxt, in_);
            CPos mp = np_;
            advance(mp);
            const int64_t im = item_of(mp);
            const uint32_t code2 = im >= 0 ? items[im] : 0u;
            if (i >= 2) pair_sync<BAR_EMPTY>(sb);   // buffer sb released (chunk i-2)
            if (ic >= 0) stage(raw, pt, sb);
            if (pt == 0) {
                meta[2 * sb] = make_int4(cp.kq, np_.end ? 1 : 0, np_.end ? -1 : np_.kq, 0);
                meta[2 * sb + 1] = make_int4(cp.P, (int)(cp.e - cp.s), cp.c, 0);
            }
            __threadfence_block();
            pair_arrive<BAR_FULL>(sb);
            raw = nxt;
            ic = in_;
            cp = np_;
            np_ = mp;
            in_ = im;
            nxt.code = code2;
            ++i;
        }
        // wait until the consumers have released the last buffers
        for (int j = i >= 2 ? i - 2 : 0; j < i; ++j) pair_sync<BAR_EMPTY>(j & 1);
    } else {
        // ================================================================ consumers
        const int ct = threadIdx.x - GRID_NP;
        const int grp = ct / G, lid = ct - grp * G;
        const int ta = lid / W, tb = lid - ta * W;
        const bool in_group = grp < NG;
        // a run starts by assignment (set), so the sums need no clearing
        float2 acc[Ww];
        uint32_t ckey = KEY_NONE;   // cell the accumulators belong to
        // per bucket (uniform): offset of the bucket's first plane in the plane block (negative when the
        // block starts later), and which of its W_w planes lie in the block (all items of a bucket share
        // their first plane: one w plane per bucket on this path)
        int64_t poff = 0;
        uint32_t vmask = 0u;
        auto flush_acc = [&]() {
            const int cu = (int)(ckey >> 25) - 64, cv = (int)((ckey >> KEY_PLANE_BITS) & 127u) - 64;
            if ((unsigned)cu < (unsigned)E && (unsigned)cv < (unsigned)E) {
                int gu = tu * TILE + cu, gv = tv * TILE + cv;
                gu -= gu >= g.Nu ? g.Nu : 0;
                gv -= gv >= g.Nv ? g.Nv : 0;
                const int64_t cell = poff + (int64_t)gu * g.Nv + gv;
#pragma unroll
                for (int c = 0; c < Ww; ++c)
                    if ((vmask >> c) & 1u) atomicAdd(planes + cell + c * plane_sz, acc[c]);
            }
        };
        int prev_kq = -1;
        for (int i = 0;; ++i) {
            const int sb = i & 1;
            pair_sync<BAR_FULL>(sb);
            const int4 m = meta[2 * sb];        // bucket, last chunk, bucket of the next chunk
            const int4 mc = meta[2 * sb + 1];   // part length, items of the bucket, chunk in the bucket
            if (m.x != prev_kq) {
                prev_kq = m.x;
                const int ck = m.x * g.q;
                poff = (int64_t)(ck - k_lo) * plane_sz;
                vmask = 0u;
#pragma unroll
                for (int c = 0; c < Ww; ++c) vmask |= (ck + c >= k_lo && ck + c < k_hi) ? 1u << c : 0u;
            }
            if (in_group) {
                const float2 *ru = reinterpret_cast<const float2 *>(smem_raw + L.ru[sb]);
                const float2 *rv = reinterpret_cast<const float2 *>(smem_raw + L.rv[sb]);
                const float2 *rwy = reinterpret_cast<const float2 *>(smem_raw + L.wy[sb]);
                // this group's records of the chunk: the next ones of its contiguous part
                const int part = min(mc.x, max(0, mc.y - grp * mc.x));
                const int cnt = min(RPG, max(0, part - mc.z * RPG));
                constexpr int NQ = WS / 2;   // float4 per w-tap row (odd W_w: the last half is padding)
                const float2 *pa = ru + grp * RPG * W + ta, *pb = rv + grp * RPG * W + tb;
                const float4 *pw = reinterpret_cast<const float4 *>(rwy + grp * RPG * WS);
                auto add = [&](float wuv, const float4 *q) {
#pragma unroll
                    for (int c = 0; c < Ww; ++c) {
                        const float4 v = q[c >> 1];
                        acc[c].x = fmaf(wuv, (c & 1) ? v.z : v.x, acc[c].x);
                        acc[c].y = fmaf(wuv, (c & 1) ? v.w : v.y, acc[c].y);
                    }
                };
                auto set = [&](float wuv, const float4 *q) {
#pragma unroll
                    for (int c = 0; c < Ww; ++c) {
                        const float4 v = q[c >> 1];
                        acc[c].x = wuv * ((c & 1) ? v.z : v.x);
                        acc[c].y = wuv * ((c & 1) ? v.w : v.y);
                    }
                };
                // one record per step: with 56 registers per thread three CTAs fit an SM, which hides the
                // loads' latency better than two records per step at two CTAs; unrolled by two, which
                // halves the pointer and loop arithmetic
                int n = cnt;
#pragma unroll 2
                for (; n > 0; --n, pa += W, pb += W, pw += NQ) {
                    const float2 a0 = pa[0], b0 = pb[0];
                    float4 q0[NQ];
#pragma unroll
                    for (int c2 = 0; c2 < NQ; ++c2) q0[c2] = pw[c2];
                    const uint32_t k0 = __float_as_uint(a0.y) | __float_as_uint(b0.y);
                    if (k0 != ckey) {
                        flush_acc();
                        ckey = k0;
                        set(a0.x * b0.x, q0);
                    } else {
                        add(a0.x * b0.x, q0);
                    }
                }
                // the sums stay in registers while the next chunk continues this bucket
                if (m.y || m.z != m.x) {
                    flush_acc();
                    ckey = KEY_NONE;
                }
            }
            __threadfence_block();
            pair_arrive<BAR_EMPTY>(sb);
            if (m.y) break;
        }
    }
}

// ------------------------------------------------------------------ FP32 degridding from staged tiles
// One CTA per work item (home items of a tile, or a chunk of a heavy tile).  For each
// w bucket the tile's footprint region of (TILE + W - 1)^2 cells is staged in shared
// memory for the bucket's W_w planes, with coalesced 8-byte loads, cell-major: a
// cell's planes lie side by side, so one 16-byte load brings two of them.  Then one
// thread per home item interpolates from shared memory, summing each cell over its
// planes before the u and v taps.
// threads per CTA: three CTAs (each with its staged region) share an SM at 56 registers per thread
constexpr int DEGRID_NT = 384;

template <int W, int Ww, bool REC>
__global__ void __launch_bounds__(DEGRID_NT, 3) k_degrid_tiles(const WorkItem *__restrict__ work,
                                                      const uint32_t *__restrict__ items,
                                                      const int64_t *__restrict__ off, CoordSrc src,
                                                      const float4 *__restrict__ recs, const float2 *__restrict__ rph,
                                                      BandGeom g, int k_lo, int k_hi, const float2 *__restrict__ planes,
                                                      const float *__restrict__ wgt, int item_order,
                                                      float2 *__restrict__ vis) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *reg = reinterpret_cast<float2 *>(smem_raw);
    // the region of the current bucket's W_w planes, cell-major: cell (r, c) holds its planes k0 .. k0 + W_w - 1
    // (padded to an even count) side by side, so that one 16-byte load brings two planes of a cell
    constexpr int RP = (Ww + 1) & ~1;
    constexpr int E = TILE + W - 1;      // region edge
    const WorkItem wi = work[blockIdx.x];
    if (wi.end <= wi.begin) return;
    const int tu = wi.tile / g.ntv, tv = wi.tile - tu * g.ntv;
    const int64_t plane_sz = (int64_t)g.Nu * g.Nv;
    const int64_t kbase = ((int64_t)g.band * g.ntu * g.ntv + wi.tile) * g.nkq;
    int lo = 0, hi = g.nkq - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[kbase + mid] <= wi.begin) lo = mid; else hi = mid - 1;
    }
    const int kq_first = lo;
    lo = kq_first; hi = g.nkq - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[kbase + mid] <= wi.end - 1) lo = mid; else hi = mid - 1;
    }
    const int kq_last = lo;
    // kernel constants in FP32, converted once (FP64 arithmetic is slow on this GPU)
    const float ihw = (float)g.inv_halfw, b2 = es_b2(g.beta);
    __syncthreads();
    for (int kq = kq_first; kq <= kq_last; ++kq) {
        const int64_t s = max(off[kbase + kq], (int64_t)wi.begin), e = min(off[kbase + kq + 1], (int64_t)wi.end);
        if (e <= s) continue;
        // planes this bucket needs, clipped to the block
        const int pa = max(kq * g.q, k_lo), pb = min(kq * g.q + g.q + Ww - 1, k_hi);
        if (pa >= pb) continue;
        // stage the bucket's planes k0 .. k0 + W_w - 1 (zero outside the block [pa, pb)); the previous bucket's
        // readers finished at the barrier that ends its item loop
        const int k0 = kq * g.q;
        for (int i = threadIdx.x; i < RP * E * E; i += blockDim.x) {
            const int p = i / (E * E), rc = i - p * (E * E);
            const int r = rc / E, c = rc - r * E;
            const int k = k0 + p;
            float2 val = make_float2(0.f, 0.f);
            if (p < Ww && k >= pa && k < pb) {
                int gu = tu * TILE + r, gv = tv * TILE + c;
                gu -= gu >= g.Nu ? g.Nu : 0;
                gv -= gv >= g.Nv ? g.Nv : 0;
                val = planes[(int64_t)(k - k_lo) * plane_sz + (int64_t)gu * g.Nv + gv];
            }
            reg[rc * RP + p] = val;
        }
        __syncthreads();
        // the bucket lists its home items first (the plan's fine sort), then spill copies of
        // neighbours' items, which this tile does not degrid: find the end of the home items
        int64_t he = s;
        {
            int64_t lo = s, hi = e;   // first index in [s, e) with spill bits, or e
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (items[mid] >> 30) hi = mid; else lo = mid + 1;
            }
            he = lo;
        }
        // each thread's next item is loaded while the current one is interpolated
        int64_t it = s + threadIdx.x;
        uint32_t code_n = 0;
        float4 rec_n = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 ph_n = make_float2(1.f, 0.f);
        if (it < he) {
            code_n = items[it];
            if constexpr (REC) {
                rec_n = recs[it];
                ph_n = rph[it];
            }
        }
        for (; it < he; it += blockDim.x) {
            const uint32_t code = code_n;
            const float4 r4 = rec_n;
            const float2 ph = ph_n;
            const int64_t nx_it = it + blockDim.x;
            if (nx_it < he) {
                code_n = items[nx_it];
                if constexpr (REC) {
                    rec_n = recs[nx_it];
                    ph_n = rph[nx_it];
                }
            }
            const uint32_t v = code;
            VisCoord<float> c;
            int lu, lv;
            float cs = 1.f, sn = 0.f;
            if constexpr (REC) {
                const uint32_t bits = __float_as_uint(r4.w);
                c.ou = r4.x;
                c.ov = r4.y;
                c.ow = r4.z;
                lu = (int)(bits & 63u) - 32;
                lv = (int)((bits >> 6) & 63u) - 32;
                c.flip = (bits >> 12) & 1u;
                c.k0 = (int)(bits >> 13);
                cs = ph.x;
                sn = ph.y;
            } else {
                const uint32_t row = v / (uint32_t)g.nchan;
                const int ch = (int)(v - row * (uint32_t)g.nchan);
                c = vis_coord<float>(src, row, ch, g);
                lu = c.gu0 - tu * TILE;
                lv = c.gv0 - tv * TILE;
                if (g.tc != 0.0 || g.facet) sincos_turns(c.ph, &sn, &cs);
            }
            if (c.k0 >= k_hi || c.k0 + Ww <= k_lo) continue;
            const float xu = c.ou * ihw, xv = c.ov * ihw, xw = c.ow * ihw;
            float ku[W], kv[W], kw[Ww];
#pragma unroll
            for (int i = 0; i < W; ++i) {
                ku[i] = es_kernel_x(fmaf((float)i, ihw, xu), b2);
                kv[i] = es_kernel_x(fmaf((float)i, ihw, xv), b2);
            }
            if (Ww > 1) {
#pragma unroll
                for (int i = 0; i < Ww; ++i) kw[i] = es_kernel_x(fmaf((float)i, ihw, xw), b2);
            } else {
                kw[0] = 1.f;
            }
            // per cell the sum over its planes first (planes outside the block are staged as zeros), then the
            // u and v taps; the item's planes are the bucket's (one w plane per bucket on this path)
            float kp[RP];
#pragma unroll
            for (int p = 0; p < RP; ++p) kp[p] = p < Ww ? kw[p < Ww ? p : 0] : 0.f;
            float ar = 0.f, ai = 0.f;
            const float4 *pl = reinterpret_cast<const float4 *>(reg + (lu * E + lv) * RP);
#pragma unroll
            for (int a = 0; a < W; ++a) {
                float rr = 0.f, ri = 0.f;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float4 *q = pl + (a * E + b) * (RP / 2);
                    float sr = 0.f, si = 0.f;
#pragma unroll
                    for (int h = 0; h < RP / 2; ++h) {
                        const float4 t = q[h];
                        sr = fmaf(kp[2 * h], t.x, sr);
                        si = fmaf(kp[2 * h], t.y, si);
                        sr = fmaf(kp[2 * h + 1], t.z, sr);
                        si = fmaf(kp[2 * h + 1], t.w, si);
                    }
                    rr = fmaf(kv[b], sr, rr);
                    ri = fmaf(kv[b], si, ri);
                }
                ar = fmaf(ku[a], rr, ar);
                ai = fmaf(ku[a], ri, ai);
            }
            float vr = ar * cs + ai * sn;
            float vi = ai * cs - ar * sn;
            if (c.flip) vi = -vi;
            // item order: the weighted value w_v (R x)_v at the item's position
            const int64_t o = item_order ? it : (int64_t)v;
            if (item_order && wgt) {
                const float wv = wgt[v];
                vr *= wv;
                vi *= wv;
            }
            float2 out;
            if (g.accumulate || c.k0 < k_lo) {
                out = vis[o];
                out.x += vr;
                out.y += vi;
            } else {
                out = make_float2(vr, vi);
            }
            vis[o] = out;
        }
        __syncthreads();
    }
}

// Zero the cells of heavy tiles (filled by reductions) in planes [0, nplanes).
template <typename T>
__global__ void k_zero_tiles(const int *__restrict__ tiles, int ntiles, int ntv, int Nv, int64_t plane_sz,
                             int nplanes, cx_t<T> *__restrict__ planes) {
    const int t = tiles[blockIdx.x % ntiles];
    const int k = blockIdx.x / ntiles;
    if (k >= nplanes) return;
    const int tu = t / ntv, tv = t - tu * ntv;
    cx_t<T> *dst = planes + (int64_t)k * plane_sz + (int64_t)(tu * TILE) * Nv + tv * TILE;
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        const int r = e / TILE, c = e - r * TILE;
        dst[(int64_t)r * Nv + c] = cx_t<T>{0, 0};
    }
}

// ------------------------------------------------------------------ post-pass (R^dagger)
// image[p] (+)= corr[p] Re sum_{k in block} exp(+2 pi i w_k t_p) H_k[pos(p)].
template <typename T>
__global__ void k_postpass(int nx, int ny, const T *__restrict__ corr, const double *__restrict__ tp, BandGeom g,
                           int k_lo, int k_hi, double dw, const cx_t<T> *__restrict__ planes, int accumulate,
                           T *__restrict__ image) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= (int64_t)nx * ny) return;
    const int i = (int)(p / ny), j = (int)(p - (int64_t)i * ny);
    int gu = i - nx / 2, gv = j - ny / 2;
    gu += gu < 0 ? g.Nu : 0;
    gv += gv < 0 ? g.Nv : 0;
    const int64_t pos = (int64_t)gu * g.Nv + gv;
    const int64_t plane_sz = (int64_t)g.Nu * g.Nv;
    T th0, dth_hi, dth_lo;
    plane_phase_base(tp, p, g, dw, &th0, &dth_hi, &dth_lo);
    T acc = 0;
    for (int k = k_lo; k < k_hi; ++k) {
        const cx_t<T> h = planes[(int64_t)(k - k_lo) * plane_sz + pos];
        if (g.Ww > 1) {
            T cs, sn;
            sincos_turns(plane_turns(k, th0, dth_hi, dth_lo), &sn, &cs);
            acc += h.x * cs - h.y * sn;
        } else {
            acc += h.x;
        }
    }
    acc *= corr[p];
    image[p] = accumulate ? image[p] + acc : acc;
}

// ------------------------------------------------------------------ weight sums
template <typename T>
__global__ void k_wsum(const T *__restrict__ wgt, int64_t nrow, int nchan, const int *__restrict__ band,
                       double *__restrict__ out) {
    // one thread per (row, chan); block-level reduction per band via shared atomics
    extern __shared__ double sacc[];
    const int nb = blockDim.y;   // number of bands (<= 32), passed through blockDim.y == 1 trick avoided
    (void)nb;
    for (int b = threadIdx.x; b < 32; b += blockDim.x) sacc[b] = 0.0;
    __syncthreads();
    const int64_t n = nrow * nchan;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % nchan);
        atomicAdd(&sacc[band[ch]], wgt ? (double)wgt[i] : 1.0);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 32; b += blockDim.x)
        if (sacc[b] != 0.0) atomicAdd(&out[b], sacc[b]);
}

// ------------------------------------------------------------------ cuFFT helpers
template <typename T> struct FftT;
template <> struct FftT<float> {
    static constexpr cufftType c2c = CUFFT_C2C;
    static cufftResult exec(cufftHandle h, float2 *in, float2 *out, int dir) {
        return cufftExecC2C(h, (cufftComplex *)in, (cufftComplex *)out, dir);
    }
};
template <> struct FftT<double> {
    static constexpr cufftType c2c = CUFFT_Z2Z;
    static cufftResult exec(cufftHandle h, double2 *in, double2 *out, int dir) {
        return cufftExecZ2Z(h, (cufftDoubleComplex *)in, (cufftDoubleComplex *)out, dir);
    }
};

// cuFFT work area of a batched 2-D C2C plan, without creating it
template <typename T>
static size_t fft_work_estimate(int Nu, int Nv, int batch) {
    int n[2] = {Nu, Nv};
    size_t ws = 0;
    if (cufftEstimateMany(2, n, nullptr, 1, 0, nullptr, 1, 0, FftT<T>::c2c, batch, &ws) != CUFFT_SUCCESS)
        ws = (size_t)Nu * Nv * sizeof(cx_t<T>) * batch;
    return ws;
}

// FFT of nplanes planes in batches of up to 8, smaller when the work area would not
// fit the context's HBM budget
template <typename T>
static void fft_planes(Ctx &ctx, cx_t<T> *data, int nplanes, int Nu, int Nv, int dir, cudaStream_t st,
                       cx_t<T> *out = nullptr) {
    int maxb = 8;
    const size_t room = ctx.available() + ctx.scratch_bytes("fftwork");
    const size_t plane_bytes = (size_t)Nu * Nv * sizeof(cx_t<T>);
    // the (host-side) estimate only when memory is tight: a batch needs at most a few planes of work area
    if (room < 4 * (size_t)maxb * plane_bytes)
        while (maxb > 1 && fft_work_estimate<T>(Nu, Nv, std::min(maxb, nplanes)) > room) maxb /= 2;
    const int64_t plane_sz = (int64_t)Nu * Nv;
    for (int k = 0; k < nplanes; k += maxb) {
        const int b = std::min(maxb, nplanes - k);
        cufftHandle h = ctx.fft(Nu, Nv, b, FftT<T>::c2c);
        PFB_CUFFT(cufftSetStream(h, st));
        PFB_CUFFT(FftT<T>::exec(h, data + k * plane_sz, (out ? out : data) + k * plane_sz, dir));
    }
}

// Row pass of a plane block: 1-D DFTs of length Nv along all nplanes * Nu rows (in -> out, or in place)
template <typename T>
static void fft_rows(Ctx &ctx, cx_t<T> *in, cx_t<T> *out, int nplanes, int Nu, int Nv, int dir, cudaStream_t st) {
    cufftHandle h = ctx.fft(Nv, 0, nplanes * Nu, FftT<T>::c2c);
    PFB_CUFFT(cufftSetStream(h, st));
    PFB_CUFFT(FftT<T>::exec(h, in, out, dir));
}

// FP32 planes whose column pass colfft.cu takes: power-of-two Nu up to 8192, image region aligned
template <typename T> static bool split_fft(const Plan &p) {
    return sizeof(T) == 4 && colfft_fits(p.Nu, p.Nv, p.nx, p.ny);
}

static int plane_block(Ctx &ctx, const Plan &p, size_t cxs, size_t reserve_unused) {
    // keep room for the cuFFT work area of a single-plane transform
    (void)reserve_unused;
    // leave room for the other buffers a call sequence needs after the stack exists:
    // a visibility-sized scratch (Hessian) and a dozen image-sized buffers (step)
    const size_t rs = cxs / 2;
    const size_t others = (size_t)p.nrow * p.nchan * cxs + 16 * (size_t)p.nband * p.nx * p.ny * rs;
    const size_t reserve = (cxs == 16 ? fft_work_estimate<double>(p.Nu, p.Nv, 1)
                                      : fft_work_estimate<float>(p.Nu, p.Nv, 1)) + others + (64u << 20);
    const size_t plane_bytes = (size_t)p.Nu * p.Nv * cxs;
    const size_t have = ctx.scratch_bytes("planes");
    const size_t avail = ctx.available() + have;
    size_t room = avail > reserve ? avail - reserve : 0;
    int blk = (int)std::min<size_t>((size_t)p.Pmax, room / plane_bytes);
    if (blk < 1) throw Error(PFB_ERR_OOM, "HBM budget too small for one w-plane of " +
                                              std::to_string(p.Nu) + "x" + std::to_string(p.Nv));
    return blk;
}

// Kept zero padding.  The zeros of a plane block (the padding around the image in degridding, the tiles
// without visibilities in gridding) are the same in every call with a plan, so when every band fits one
// block and the budget has room, the transform input gets buffers of its own that only the pre-pass or
// the tile kernels write, cleared once per plan, and the FFT writes the shared block out of place.
// Degridding keeps one input buffer, gridding one per band (each band has its own empty tiles).
static bool keep_zeros_fits(Ctx &ctx, const Plan &p, size_t cxs, int blk, int nbuf, const char *prefix) {
    if (blk < p.Pmax) return false;
    const size_t need = (size_t)nbuf * blk * p.Nu * p.Nv * cxs;
    size_t have = 0;
    for (int i = 0; i < nbuf; ++i) have += ctx.scratch_bytes(std::string(prefix) + std::to_string(i));
    const size_t others = (size_t)p.nrow * p.nchan * cxs + 16 * (size_t)p.nband * p.nx * p.ny * (cxs / 2) +
                          (256u << 20);
    return ctx.available() + have >= need + others;
}

// A kept-zero input buffer: cleared on `st` unless it already holds this plan's zeros.
template <typename T>
static cx_t<T> *kept_zero_buffer(Ctx &ctx, const Plan &p, const std::string &name, int blk, cudaStream_t st) {
    const size_t bytes = (size_t)blk * p.Nu * p.Nv * sizeof(cx_t<T>);
    cx_t<T> *buf = (cx_t<T> *)ctx.scratch(name, bytes);
    auto it = ctx.zero_tag.find(name);
    if (it == ctx.zero_tag.end() || it->second != std::make_pair(p.id, blk)) {
        KTimer t(ctx, "memset_planes", st, (double)bytes, 0);
        PFB_CUDA(cudaMemsetAsync(buf, 0, bytes, st));
        ctx.zero_tag[name] = std::make_pair(p.id, blk);
    }
    return buf;
}

static unsigned grid_blocks(int64_t n, int threads, int cap) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// ------------------------------------------------------------------ FP32 kernel dispatch on W
static bool fast_path_f32(const Plan &p) {
    return p.prec == PFB_F32 && p.W >= 4 && p.W <= 8 && p.q == 1 && p.Pmax < (1 << KEY_PLANE_BITS);
}
// Item records for the FP32 tile kernels, when the budget leaves room for them next to
// a plane block and a visibility-sized scratch; otherwise the kernels compute the
// geometry on the fly.
void build_item_records(Ctx &ctx, Plan &p, cudaStream_t st) {
    if (!fast_path_f32(p) || p.nitems <= 0 || (p.flags & PFB_NO_ITEM_RECORDS)) return;
    const size_t need = (size_t)p.nitems * (sizeof(float4) + sizeof(float2));
    const size_t keep = 2 * (size_t)p.Ww * p.Nu * p.Nv * sizeof(float2) + (size_t)p.nrow * p.nchan * sizeof(float2) +
                        16 * (size_t)p.nband * p.nx * p.ny * sizeof(float) + (256u << 20);
    if (ctx.available() < need + keep) return;
    p.d_rec = (float4 *)ctx.dalloc((size_t)p.nitems * sizeof(float4));
    p.d_rph = (float2 *)ctx.dalloc((size_t)p.nitems * sizeof(float2));
    p.bytes += need;
    for (int b = 0; b < p.nband; ++b) {
        const int64_t i0 = p.band_items_begin[b], n = p.band_items_end[b] - i0;
        if (n <= 0) continue;
        k_item_records<<<grid_blocks(n, 256, 32 * ctx.num_sms), 256, 0, st>>>(p.d_items, i0, n, p.coords(), p.geom(b),
                                                                             p.d_rec, p.d_rph);
        check_launch("item_records");
    }
}

static bool degrid_tiles_fit(const Plan &p) {
    const int RP = (p.Ww + 1) & ~1, E = TILE + p.W - 1;
    return fast_path_f32(p) && (size_t)RP * E * E * sizeof(float2) <= 227 * 1024;
}
// FP32 plans whose tile kernels fit: the plan lists each visibility once, in its home tile, and the
// gridding kernel adds the tile's region with the footprints' far edges (k_grid_res)
bool halo_fits(const Plan &p) {
    return fast_path_f32(p) && degrid_tiles_fit(p) && (size_t)res_layout(p.W, p.Ww).total <= 227 * 1024;
}
static bool grid_res_fit(const Plan &p) { return p.halo; }

template <int W, int Ww>
static void launch_grid_res_t(unsigned nblk, cudaStream_t st, const WorkItem *work, const Plan &p,
                              const float2 *vis, const float *wgt, int unit, int item_order, const BandGeom &g,
                              int k_lo, int k_hi, float2 *planes) {
    const size_t smem = (size_t)res_layout(W, Ww).total;
    if (p.d_rec) {
        ensure_dynamic_smem(k_grid_res<W, Ww, true>, (size_t)smem);
        k_grid_res<W, Ww, true><<<nblk, GRID_NT, smem, st>>>(work, p.d_items, p.d_off, p.coords(), p.d_rec,
                                                             p.d_rph, vis, wgt, unit, item_order, g, k_lo, k_hi, planes);
    } else {
        ensure_dynamic_smem(k_grid_res<W, Ww, false>, (size_t)smem);
        k_grid_res<W, Ww, false><<<nblk, GRID_NT, smem, st>>>(work, p.d_items, p.d_off, p.coords(), nullptr,
                                                              nullptr, vis, wgt, unit, item_order, g, k_lo, k_hi, planes);
    }
}

template <int W, int Ww>
static void launch_degrid_t(unsigned nblk, int R, cudaStream_t st, const WorkItem *work, const Plan &p,
                            const BandGeom &g, int k_lo, int k_hi, const float2 *planes, const float *wgt,
                            int item_order, float2 *vis) {
    (void)R;
    const int E = TILE + W - 1;
    const size_t smem = (size_t)((Ww + 1) & ~1) * E * E * sizeof(float2);
    if (p.d_rec) {
        ensure_dynamic_smem(k_degrid_tiles<W, Ww, true>, (size_t)smem);
        k_degrid_tiles<W, Ww, true><<<nblk, DEGRID_NT, smem, st>>>(work, p.d_items, p.d_off, p.coords(), p.d_rec, p.d_rph,
                                                             g, k_lo, k_hi, planes, wgt, item_order, vis);
    } else {
        ensure_dynamic_smem(k_degrid_tiles<W, Ww, false>, (size_t)smem);
        k_degrid_tiles<W, Ww, false><<<nblk, DEGRID_NT, smem, st>>>(work, p.d_items, p.d_off, p.coords(), nullptr, nullptr,
                                                              g, k_lo, k_hi, planes, wgt, item_order, vis);
    }
}

#define PFB_W_SWITCH(W, WS, CALL)                                                     \
    switch (W) {                                                                    \
        case 4: if (WS) CALL(4, 4); else CALL(4, 1); break;                          \
        case 5: if (WS) CALL(5, 5); else CALL(5, 1); break;                          \
        case 6: if (WS) CALL(6, 6); else CALL(6, 1); break;                          \
        case 7: if (WS) CALL(7, 7); else CALL(7, 1); break;                          \
        case 8: if (WS) CALL(8, 8); else CALL(8, 1); break;                          \
        default: throw Error(PFB_ERR_ARG, "no FP32 kernel for this support");        \
    }

// ------------------------------------------------------------------ operators
// visibilities of band b (rows x channels mapped to b)
static int64_t band_nvis(const Plan &p, int b) {
    int64_t nc = 0;
    for (int c = 0; c < p.nchan; ++c) nc += p.band_h[c] == b;
    return nc * p.nrow;
}

// item_order: vis is in item order and receives w_v (R x)_v, w = item_wgt (halo plans, FP32 tile kernels)
template <typename T>
static void degrid_impl(Ctx &ctx, const Plan &p, const T *image, cx_t<T> *vis, cudaStream_t st, bool accumulate,
                        bool item_order, const T *item_wgt) {
    const size_t cxs = sizeof(cx_t<T>);
    // room for cuFFT work areas is taken from the same budget
    const int blk = plane_block(ctx, p, cxs, (size_t)p.Nu * p.Nv * cxs * 2);
    cx_t<T> *planes = (cx_t<T> *)ctx.scratch("planes", (size_t)blk * p.Nu * p.Nv * cxs);
    // pruned transforms: one buffer, no kept zeros (cells outside the touched tiles are never read)
    const bool pruned = sizeof(T) == 4 && p.pruned;
    const bool keep = !pruned && keep_zeros_fits(ctx, p, cxs, blk, 1, "dg_in");
    cx_t<T> *in = keep ? kept_zero_buffer<T>(ctx, p, "dg_in0", blk, st) : planes;
    const int64_t npix = (int64_t)p.nx * p.ny;
    const double plane_bytes = (double)p.Nu * p.Nv * cxs;
    for (int b = 0; b < p.nband; ++b) {
        BandGeom g = p.geom(b);
        g.accumulate = accumulate ? 1 : 0;
        const int64_t i0 = p.band_items_begin[b], i1 = p.band_items_end[b];
        const double nvb = (double)band_nvis(p, b);
        for (int k_lo = 0; k_lo < g.P; k_lo += blk) {
            const int k_hi = std::min(g.P, k_lo + blk);
            const int nk = k_hi - k_lo;
            if (pruned) {
                plane_forward(ctx, p, b, (const float *)(image + b * npix), k_lo, k_hi, (float2 *)planes, st);
            } else {
            if (!keep) {
                KTimer t(ctx, "memset_planes", st, nk * plane_bytes, 0);
                PFB_CUDA(cudaMemsetAsync(planes, 0, (size_t)nk * p.Nu * p.Nv * cxs, st));
            }
            {
                KTimer t(ctx, "prepass", st, npix * (2.0 * sizeof(T) + 8.0 + nk * (double)cxs));
                k_prepass<T><<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(
                    p.nx, p.ny, image + b * npix, (const T *)p.d_corr, p.d_tp, g, k_lo, k_hi, p.dw, in);
                check_launch("prepass");
            }
            {
                KTimer t(ctx, "fft_fwd", st, 2.0 * nk * plane_bytes, split_fft<T>(p) ? 1 : 0);
                if (split_fft<T>(p)) {   // columns of the image region (in place), then all rows
                    colfft_planes(ctx, (float2 *)in, nk, p.Nu, p.Nv, p.nx, p.ny, false, st);
                    fft_rows<T>(ctx, in, planes, nk, p.Nu, p.Nv, CUFFT_FORWARD, st);
                } else {
                    fft_planes<T>(ctx, in, nk, p.Nu, p.Nv, CUFFT_FORWARD, st, keep ? planes : nullptr);
                }
            }
            }
            if (i1 > i0 && sizeof(T) == 4 && degrid_tiles_fit(p)) {
                // algorithmic bytes: halo plans read the reached tiles of the block's planes once, and per
                // item its code, record and rotor (when kept), output value and (item order) weight; other
                // plans count the whole planes
                const double nit = (double)(i1 - i0);
                const double dg_bytes =
                    p.halo ? (double)(p.empty_begin[b] - p.heavy_begin[b]) * nk * TILE * TILE * cxs +
                                 nit * (4.0 + (p.d_rec ? 24.0 : 0.0) + cxs + (item_order && item_wgt ? 4.0 : 0.0))
                           : nk * plane_bytes + 4.0 * nit + nvb * cxs;
                KTimer t(ctx, "degrid_tiles", st, dg_bytes);
                const WorkItem *wl = p.d_work_dg ? p.d_work_dg : p.d_work;
                const std::vector<int64_t> &wb = p.d_work_dg ? p.work_dg_begin : p.work_begin;
                const int64_t w0 = wb[b], w1 = wb[b + 1];
                const int R = p.Ww;
#define PFB_DEGRID_CALL(WV, WWV)                                                                          \
    launch_degrid_t<WV, WWV>((unsigned)(w1 - w0), R, st, wl + w0, p, g, k_lo, k_hi, (const float2 *)planes,   \
                             (const float *)item_wgt, item_order ? 1 : 0, (float2 *)vis)
                PFB_W_SWITCH(p.W, p.wstack, PFB_DEGRID_CALL)
#undef PFB_DEGRID_CALL
                check_launch("degrid_tiles");
            } else if (i1 > i0) {
                PFB_REQUIRE(!item_order, "item-order visibilities need the FP32 tile kernels");
                KTimer t(ctx, "gather", st, nk * plane_bytes + 4.0 * (i1 - i0) + nvb * cxs);
                k_gather<T><<<grid_blocks(i1 - i0, 256, 64 * ctx.num_sms), 256, 0, st>>>(
                    p.d_items + i0, i1 - i0, p.coords(), g, k_lo, k_hi, planes, vis);
                check_launch("gather");
            }
        }
    }
}

template <typename T>
void op_degrid(Ctx &ctx, const Plan &p, const T *image, cx_t<T> *vis, cudaStream_t st, bool accumulate) {
    degrid_impl<T>(ctx, p, image, vis, st, accumulate, false, nullptr);
}

// item_order: vis is in item order (halo plans); wgt, when given, stays in row order and is gathered per item
template <typename T>
static void grid_impl(Ctx &ctx, const Plan &p, const cx_t<T> *vis, const T *wgt, bool unit_vis, bool item_order,
                      T *image, cudaStream_t st, const std::function<void(int)> &band_done) {
    const size_t cxs = sizeof(cx_t<T>);
    const int blk = plane_block(ctx, p, cxs, (size_t)p.Nu * p.Nv * cxs * 2);
    cx_t<T> *planes = (cx_t<T> *)ctx.scratch("planes", (size_t)blk * p.Nu * p.Nv * cxs);
    // pruned transforms: one buffer; the tiles without items are never read, so they need no zeros
    const bool pruned = sizeof(T) == 4 && p.pruned;
    const bool keep = !pruned && keep_zeros_fits(ctx, p, cxs, blk, p.nband, "gr_in");
    const int64_t npix = (int64_t)p.nx * p.ny;
    const int R = p.Ww + p.q - 1;
    const size_t smem = (size_t)R * TILE * TILE * cxs;
    ensure_dynamic_smem(k_grid_tiles<T>, (size_t)smem);
    const double plane_bytes = (double)p.Nu * p.Nv * cxs;
    for (int b = 0; b < p.nband; ++b) {
        const BandGeom g = p.geom(b);
        const int64_t w0 = p.work_begin[b], w1 = p.work_begin[b + 1];
        // tiles zeroed per call: those that reductions fill (heavy tiles; on plans of home items, every
        // tile that some footprint reaches), and the rest unless kept or never read
        const int64_t h0 = p.heavy_begin[b], h1 = (keep || pruned) ? p.empty_begin[b] : p.heavy_begin[b + 1];
        const double nvb = (double)band_nvis(p, b);
        const double nit = (double)(p.band_items_end[b] - p.band_items_begin[b]);
        cx_t<T> *const out = planes;
        cx_t<T> *const in = keep ? kept_zero_buffer<T>(ctx, p, "gr_in" + std::to_string(b), blk, st) : planes;
        for (int k_lo = 0; k_lo < g.P; k_lo += blk) {
            const int k_hi = std::min(g.P, k_lo + blk);
            const int nk = k_hi - k_lo;
            if (h1 > h0) {
                KTimer t(ctx, "zero_tiles", st, (double)(h1 - h0) * nk * TILE * TILE * cxs);
                k_zero_tiles<T><<<(unsigned)((h1 - h0) * nk), 256, 0, st>>>(
                    p.d_heavy + h0, (int)(h1 - h0), p.ntv, p.Nv, (int64_t)p.Nu * p.Nv, nk, in);
                check_launch("zero_tiles");
            }
            {
                const double vb = unit_vis ? 0.0 : (double)cxs;
                const double wb = wgt ? (double)sizeof(T) : 0.0;
                // algorithmic bytes: halo plans write the reached tiles of the block's planes once, and read
                // per item its code, record and rotor (when kept) and value (item order: weighted, no
                // weight); other plans count the whole planes and a gathered value and weight per visibility
                const double g_bytes =
                    p.halo ? (double)(p.empty_begin[b] - p.heavy_begin[b]) * nk * TILE * TILE * cxs +
                                 nit * (4.0 + (p.d_rec ? 24.0 : 0.0) + vb + wb)
                           : 4.0 * nit + nvb * (vb + wb) + nk * plane_bytes;
                KTimer t(ctx, "grid_tiles", st, g_bytes);
                if (sizeof(T) == 4 && grid_res_fit(p)) {
                    // dense (chunked) tiles first, then the owned light tiles, as two timed launches
                    const int64_t wh = p.work_heavy_end[b];
                    for (int part = 0; part < 2; ++part) {
                        const int64_t a0 = part == 0 ? w0 : wh, a1 = part == 0 ? wh : w1;
                        if (a1 <= a0) continue;
                        KTimer tp(ctx, part == 0 ? "grid_dense" : "grid_light", st, 0.0, 0);
#define PFB_GRID_CALL(WV, WWV)                                                                            \
    launch_grid_res_t<WV, WWV>((unsigned)(a1 - a0), st, p.d_work + a0, p, (const float2 *)vis,             \
                               (const float *)wgt, unit_vis ? 1 : 0, item_order ? 1 : 0, g, k_lo, k_hi,     \
                               (float2 *)in)
                        PFB_W_SWITCH(p.W, p.wstack, PFB_GRID_CALL)
#undef PFB_GRID_CALL
                    }
                } else if (w1 > w0) {
                    PFB_REQUIRE(!item_order, "item-order visibilities need the FP32 tile kernels");
                    k_grid_tiles<T><<<(unsigned)(w1 - w0), 256, smem, st>>>(p.d_work + w0, p.d_items, p.d_off,
                                                                             p.coords(), vis, wgt,
                                                                             unit_vis ? 1 : 0, g, k_lo, k_hi, in);
                }
                check_launch("grid_tiles");
            }
            if (pruned) {
                plane_inverse(ctx, p, b, k_lo, k_hi, (float2 *)out, (float *)(image + b * npix), st);
                continue;
            }
            {
                KTimer t(ctx, "fft_inv", st, 2.0 * nk * plane_bytes, split_fft<T>(p) ? 1 : 0);
                if (split_fft<T>(p)) {   // all rows, then the image columns of the image rows (in place)
                    fft_rows<T>(ctx, in, out, nk, p.Nu, p.Nv, CUFFT_INVERSE, st);
                    colfft_planes(ctx, (float2 *)out, nk, p.Nu, p.Nv, p.nx, p.ny, true, st);
                } else {
                    fft_planes<T>(ctx, in, nk, p.Nu, p.Nv, CUFFT_INVERSE, st, keep ? out : nullptr);
                }
            }
            {
                KTimer t(ctx, "postpass", st, npix * (nk * (double)cxs + 2.0 * sizeof(T) + 8.0));
                k_postpass<T><<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(
                    p.nx, p.ny, (const T *)p.d_corr, p.d_tp, g, k_lo, k_hi, p.dw, out, k_lo > 0 ? 1 : 0,
                    image + b * npix);
                check_launch("postpass");
            }
        }
        if (band_done) band_done(b);
    }
}

template <typename T>
void op_grid(Ctx &ctx, const Plan &p, const cx_t<T> *vis, const T *wgt, bool unit_vis, T *image,
             cudaStream_t st, const std::function<void(int)> &band_done) {
    grid_impl<T>(ctx, p, vis, wgt, unit_vis, false, image, st, band_done);
}

template <typename T>
void op_hessian(Ctx &ctx, const Plan &p, const T *x, const T *wgt, cx_t<T> *vis, T *hx, cudaStream_t st,
                cudaEvent_t wgt_ready, const std::function<void(int)> &band_done) {
    // R x needs no weights: they are read (from wgt_ready on) by R^dagger Sigma^-1 alone
    const bool items = sizeof(T) == 4 && p.halo && p.nitems == p.nrow * (int64_t)p.nchan;
    degrid_impl<T>(ctx, p, x, vis, st, false, items, nullptr);
    if (wgt_ready) PFB_CUDA(cudaStreamWaitEvent(st, wgt_ready, 0));
    grid_impl<T>(ctx, p, vis, wgt, false, items, hx, st, band_done);
}

template <typename T>
void op_wsum(Ctx &ctx, const Plan &p, const T *wgt, double *d_wsum, cudaStream_t st) {
    PFB_CUDA(cudaMemsetAsync(d_wsum, 0, 32 * sizeof(double), st));
    const int64_t n = p.nrow * p.nchan;
    k_wsum<T><<<grid_blocks(n, 256, 8 * ctx.num_sms), 256, 32 * sizeof(double), st>>>(wgt, p.nrow, p.nchan,
                                                                                       p.d_band, d_wsum);
    check_launch("wsum");
}

template void op_degrid<float>(Ctx &, const Plan &, const float *, float2 *, cudaStream_t, bool);
template void op_degrid<double>(Ctx &, const Plan &, const double *, double2 *, cudaStream_t, bool);
template void op_grid<float>(Ctx &, const Plan &, const float2 *, const float *, bool, float *, cudaStream_t,
                             const std::function<void(int)> &);
template void op_grid<double>(Ctx &, const Plan &, const double2 *, const double *, bool, double *, cudaStream_t,
                              const std::function<void(int)> &);
template void op_hessian<float>(Ctx &, const Plan &, const float *, const float *, float2 *, float *, cudaStream_t,
                                cudaEvent_t, const std::function<void(int)> &);
template void op_hessian<double>(Ctx &, const Plan &, const double *, const double *, double2 *, double *,
                                 cudaStream_t, cudaEvent_t, const std::function<void(int)> &);
template void op_wsum<float>(Ctx &, const Plan &, const float *, double *, cudaStream_t);
template void op_wsum<double>(Ctx &, const Plan &, const double *, double *, cudaStream_t);

}  // namespace pfb
