// spl_raster.cu -- rasterisation (Sec. 2 "Processing and Rasterization",
// Sec. 4 one-thread-per-particle) and binning of particles into tile lists
// (the data organisation of Sec. 4, built with counts, a scan and a scatter
// instead of a radix sort by tile index).
#include "spl_geom.cuh"

namespace spl {

// ---------------------------------------------------------------------------
// double-float ("df") arithmetic in FP32: a value is hi + lo with |lo| <=
// ulp(hi)/2.  Error-free transforms: Knuth's two-sum, Dekker's fast two-sum
// (|a| >= |b|), and the FMA-based exact product.  The projection needs
// ~1e-9 relative accuracy (1e-6 px at a 1000 px offset); FP32 alone gives
// ~1e-4 px, which would cost ~1e-3 relative error on a 1 px Gaussian's tail.
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul_f(df a, float b) {
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a / b given rb ~ 1 / b.hi (a few ulp suffice): the first quotient's
// residual a - b q1 is formed in df and divided again, so the result keeps
// df accuracy (relative error ~ eps(rb) * 2^-24 + 2^-44).
__device__ __forceinline__ df df_div(df a, df b, float rb) {
    float q1 = a.hi * rb;
    df r = df_add(a, df_neg(df_mul_f(b, q1)));
    float q2 = r.hi * rb;
    return fast_two_sum(q1, q2);
}

// Split x_s = xi + xf with xi integral (int16 range) and xf in [0, 1).
__device__ __forceinline__ void split_pos(df v, int &xi, float &xf) {
    const float lim = 30000.f;
    if (v.hi < -lim || v.hi > lim) {       // far off screen: only a huge splat can reach
        float c = fminf(fmaxf(v.hi, -lim), lim);
        xi = (int)c;
        xf = (v.hi - c) + v.lo;
        return;
    }
    float fl = floorf(v.hi);
    xi = (int)fl;
    xf = (v.hi - fl) + v.lo;
    if (xf >= 1.f) { xf -= 1.f; xi += 1; }
    if (xf < 0.f) { xf += 1.f; xi -= 1; }
}

template <bool HALF>
__device__ __forceinline__ float load_attr(const void *p, int64_t i) {
    if (HALF) return __half2float(static_cast<const __half *>(p)[i]);
    return static_cast<const float *>(p)[i];
}

// Smoothing length of particle i: FP32 (ATTR 0, 2), binary16 (ATTR 1), or a
// 16-bit logarithmic code k with h = 2^(h_log2_min + k / 4096) (ATTR 3).
template <int ATTR>
__device__ __forceinline__ float load_h(const void *p, int64_t i, float h_log2_min) {
    if (ATTR == 3)
        return exp2f(fmaf((float)static_cast<const unsigned short *>(p)[i], 1.f / 4096.f, h_log2_min));
    return load_attr<ATTR == 1>(p, i);
}

// Rasterise one particle into its record; returns its class.  q2 receives
// (absorption coefficient A, depth key) for the absorption mode: A =
// absorption * brightness * I, the key z_c rounded to float (the double-float
// value's leading part).
__device__ __forceinline__ int raster_one(const FrameConst &fc, const float *spal, float x, float y,
                                          float z, float h, float inten, float s, const float *crgb,
                                          float4 &r0, float4 &r1, float2 &q2) {
    // roto-translation x_c = R x - R eye, in df
    df c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        df a = df_mul_f({fc.Rhi[3 * k + 0], fc.Rlo[3 * k + 0]}, x);
        a = df_add(a, df_mul_f({fc.Rhi[3 * k + 1], fc.Rlo[3 * k + 1]}, y));
        a = df_add(a, df_mul_f({fc.Rhi[3 * k + 2], fc.Rlo[3 * k + 2]}, z));
        c[k] = df_add(a, {-fc.Ehi[k], -fc.Elo[k]});
    }
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    r1 = make_float4(-1.f, 0.f, 0.f, 0.f);
    q2 = make_float2(0.f, 0.f);
    // non-finite inputs or a negative smoothing length: inactive
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(h) || !isfinite(inten) ||
        !isfinite(s) || h < 0.f)
        return CLS_INACTIVE;
    if (crgb && (!isfinite(crgb[0]) || !isfinite(crgb[1]) || !isfinite(crgb[2]))) return CLS_INACTIVE;
    const float zc = c[2].hi;
    if (!(zc > fc.z_near)) return CLS_INACTIVE;
    // logarithms of processed quantities (Sec. 2)
    if (fc.log_flags & 1) {
        if (!(inten > 0.f)) return CLS_INACTIVE;
        inten = log10f(inten);
    }
    if (fc.log_flags & 2) {
        if (!(s > 0.f)) return CLS_INACTIVE;
        s = log10f(s);
    }
    // perspective projection
    const df f = {fc.fhi, fc.flo};
    const float rz = 1.f / zc;
    df xs = df_add({fc.half_w, 0.f}, df_mul(f, df_div(c[0], c[2], rz)));
    df ys = df_add({fc.half_h, 0.f}, df_neg(df_mul(f, df_div(c[1], c[2], rz))));
    int xi, yi;
    float xf, yf;
    split_pos(xs, xi, xf);
    split_pos(ys, yi, yf);
    // screen smoothing length and radius (Eq. 7)
    const float sig = fc.sig_fac * h * fc.fhi / zc;
    const float r = fc.chi * sig;
    // colour: normalise, palette look-up, scale by intensity (Sec. 2)
    float sn = fminf(fmaxf((s - fc.s_min) * fc.s_inv, 0.f), 1.f);
    float col[3];
    if (crgb) {
        col[0] = crgb[0]; col[1] = crgb[1]; col[2] = crgb[2];
    } else if (fc.npal == 1) {
        col[0] = spal[0]; col[1] = spal[1]; col[2] = spal[2];
    } else {
        float u = sn * (float)(fc.npal - 1);
        int k0 = min((int)floorf(u), fc.npal - 2);
        float t = u - (float)k0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float a = spal[3 * k0 + k], b = spal[3 * k0 + 3 + k];
            col[k] = a + t * (b - a);
        }
    }
    const float amp = fc.brightness * inten;
    // inactive when the disc's box misses the screen (Sec. 2, Fig. 4)
    const float xsf = (float)xi + xf, ysf = (float)yi + yf;
    if (xsf + r < 0.f || xsf - r >= (float)fc.width || ysf + r < 0.f || ysf - r >= (float)fc.height)
        return CLS_INACTIVE;
    r0 = make_float4(pack_xy(xi, yi), xf, yf, 1.4426950408889634f / (sig * sig));
    r1 = make_float4(r * r, amp * col[0], amp * col[1], amp * col[2]);
    q2 = make_float2(fc.absorption * amp, zc);
    return record_class(fc, r1.x);
}

// Tile footprint of one rasterised particle for the point / small / medium
// lists: a box of tiles [tx0, tx0 + bw) x [ty0, ty0 + nbox / bw) (nbox = 0:
// no entry); disc = 1 when a tile of the box must also be reached by the disc.
// Large particles are handled by large_tiles_kernel.  In the absorption mode
// points join the medium list, so that a tile's particles form one list that
// can be ordered by depth.
struct TileFoot { int list, tx0, ty0, bw, nbox, disc; float reach2; };

__device__ __forceinline__ TileFoot tile_footprint(const FrameConst &fc, int cls, float4 r0, float4 r1) {
    TileFoot f{-1, 0, 0, 1, 0, 0, 0.f};
    if (cls == CLS_POINT) {
        const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
        if (xi >= 0 && yi >= 0 && xi < fc.width && yi < fc.height) {
            f.list = fc.absorb ? L_MEDIUM : L_POINT;
            f.tx0 = xi >> fc.tile_shift; f.ty0 = yi >> fc.tile_shift; f.nbox = 1;
        }
        return f;
    }
    if (cls != CLS_SMALL && cls != CLS_MEDIUM) return f;
    PixBox b;
    if (!splat_box(fc, r0, r1.x, b)) return f;
    f.list = cls == CLS_SMALL ? L_SMALL : L_MEDIUM;
    f.disc = 1;
    f.reach2 = disc_reach2(r1.x);
    // the box is clamped to the image: non-negative pixel indices
    f.tx0 = b.i0 >> fc.tile_shift;
    f.ty0 = b.j0 >> fc.tile_shift;
    f.bw = (b.i1 >> fc.tile_shift) - f.tx0 + 1;
    f.nbox = f.bw * ((b.j1 >> fc.tile_shift) - f.ty0 + 1);
    return f;
}

// The (particle, box tile) pairs of a warp's 32 particles, taken 32 at a time
// across the lanes instead of one particle per lane: a lane with a wide
// footprint no longer holds the warp for as many rounds as it has tiles.
// incl is the inclusive prefix sum of the lanes' box sizes (foot.nbox).  Pair
// j belongs to the smallest lane o with incl_o > j (a binary search over the
// lanes' prefix sums); its tile is the (j - start_o)-th of o's box, row by row.
// Every lane of the warp must call this (warp shuffles); returns the slot
// (list * ntiles + tile) of pair j, or -1 when j is past the warp's pairs or the
// disc misses that tile, and the owner lane in *owner.
struct FootLane {
    int incl, nbox, list_disc, txy, bw;
    float rbw, reach2, x, y, z;
};

__device__ __forceinline__ FootLane foot_lane(const TileFoot &f, float4 r0, int lane) {
    FootLane l;
    int incl = f.nbox;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    l.incl = incl;
    l.nbox = f.nbox;
    l.list_disc = ((f.list + 1) << 1) | f.disc;
    l.txy = (f.tx0 & 0xFFFF) | (f.ty0 << 16);
    l.bw = f.bw;
    l.rbw = 1.f / (float)f.bw;
    l.reach2 = f.reach2;
    l.x = r0.x; l.y = r0.y; l.z = r0.z;
    return l;
}

__device__ __forceinline__ int foot_pair(const FrameConst &fc, const FootLane &l, int j, int total,
                                         int &owner) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, l.incl, lo + step - 1);
        if (v <= j) lo += step;
    }
    lo = lo < 31 ? lo : 31;
    owner = lo;
    const int o_incl = __shfl_sync(0xffffffffu, l.incl, lo);
    const int o_nbox = __shfl_sync(0xffffffffu, l.nbox, lo);
    const int o_ld = __shfl_sync(0xffffffffu, l.list_disc, lo);
    const int o_txy = __shfl_sync(0xffffffffu, l.txy, lo);
    const int o_bw = __shfl_sync(0xffffffffu, l.bw, lo);
    const float o_rbw = __shfl_sync(0xffffffffu, l.rbw, lo);
    const float o_reach2 = __shfl_sync(0xffffffffu, l.reach2, lo);
    const float4 o_r0 = make_float4(__shfl_sync(0xffffffffu, l.x, lo), __shfl_sync(0xffffffffu, l.y, lo),
                                    __shfl_sync(0xffffffffu, l.z, lo), 0.f);
    if (j >= total) return -1;
    // (t + 1/2) / bw is at least 1/(2 bw) away from an integer, far more than
    // the rounding of the product: the quotient is exact
    const int t = j - (o_incl - o_nbox);
    const int ky = (int)(((float)t + 0.5f) * o_rbw), kx = t - ky * o_bw;
    const int tx = (o_txy & 0xFFFF) + kx, ty = (o_txy >> 16) + ky;
    if ((o_ld & 1) && !disc_meets_tile(fc, o_r0, o_reach2, tx, ty)) return -1;
    return ((o_ld >> 1) - 1) * fc.ntiles + ty * fc.ntx + tx;
}

// ---------------------------------------------------------------------------
// Per-CTA aggregation of list slots.  A clustered particle set puts 1e5-1e6
// entries into single tiles; one global atomic per entry then serialises in
// L2.  Each CTA takes a contiguous chunk of particles and accumulates its
// entries in a small shared-memory hash table (open addressing, key = list *
// ntiles + tile), so that a hot slot receives one global atomic per CTA.  A key that finds no
// free place within kProbe probes falls back to global atomics; the table is
// never emptied while a CTA runs, so that choice is the same for every
// occurrence of the key within the CTA.
// ---------------------------------------------------------------------------
// kHashBits, kHash (slots) and kChunk (particles per CTA) are in spl_internal.cuh
constexpr int kProbe = 32;

__device__ __forceinline__ int hash_slot(const int *keys, int key, bool insert) {
    unsigned h = ((unsigned)key * 2654435761u) >> (32 - kHashBits);
    for (int probe = 0; probe < kProbe; ++probe) {
        const int slot = (int)((h + (unsigned)probe) & (kHash - 1));
        const int k = *(volatile const int *)&keys[slot];
        if (k == key) return slot;
        if (k == -1) {
            if (!insert) return -1;
            const int old = atomicCAS((int *)&keys[slot], -1, key);
            if (old == -1 || old == key) return slot;
        }
    }
    return -1;
}

// Count the slots of one round (one (particle, tile) pair per lane); a key
// with no room in the table is counted in ovf (placed through the cursors).
// Each lane adds its own pair: the counts need no return value, and combining
// the warp's equal keys first (a match mask) cost more than it saved
// (clustered 10M / 1024^2 raster 0.425 -> 0.388 ms, 30M / 2048^2 1.462 ->
// 1.244 ms).  The scatter, which needs each entry's rank, keeps the match.
__device__ __forceinline__ void count_round(int key, int *keys, int *vals, int *govf) {
    if (key >= 0) {
        const int slot = hash_slot(keys, key, true);
        if (slot >= 0)
            atomicAdd(&vals[slot], 1);
        else
            atomicAdd(&govf[key], 1);
    }
}

__device__ __forceinline__ void hash_clear(int *keys, int *vals) {
    for (int k = threadIdx.x; k < kHash; k += blockDim.x) {
        keys[k] = -1;
        vals[k] = 0;
    }
}

// Flush the CTA's hash table into the global slot counts, keep the table
// with every slot's offset inside its slot (tab: kHash entries) for the
// scatter, and clear it.
__device__ __forceinline__ void hash_flush(int *keys, int *vals, int *gcounts, int2 *tab) {
    __syncthreads();
    for (int k = threadIdx.x; k < kHash; k += blockDim.x) {
        const int key = keys[k];
        int off = 0;
        if (key >= 0) off = atomicAdd(&gcounts[key], vals[k]);
        tab[k] = make_int2(key, off);
        keys[k] = -1;
        vals[k] = 0;
    }
    __syncthreads();
}

// Load view v's constants into shared memory (the whole CTA waits).
__device__ __forceinline__ void load_view(const FrameConst *fcs, int v, FrameConst *sfc) {
    __syncthreads();
    const int words = (int)(sizeof(FrameConst) / sizeof(int));
    for (int k = threadIdx.x; k < words; k += blockDim.x)
        reinterpret_cast<int *>(sfc)[k] = reinterpret_cast<const int *>(fcs + v)[k];
    __syncthreads();
}

// One thread per particle and view: the particle's chunk is rasterised for
// every view of the batch (its inputs are read from HBM once and then hit in
// L2), records are written to rec[view * n + id], list entries are counted.
// ATTR: 0 = h, I, s in FP32; 1 = all three in binary16; 2 = h in FP32, I and s
// in binary16; 3 = h as a 16-bit logarithmic code, I and s in binary16.  RGB:
// per-particle colour components replace the palette.
template <int ATTR, bool RGB>
__global__ void __launch_bounds__(256, 4) raster_kernel(Views vs, RasterArgs a) {
    __shared__ float spal[3 * kMaxPalette];
    __shared__ int keys[kHash], vals[kHash];
    __shared__ unsigned long long bstat[5];
    __shared__ FrameConst sfc;
    hash_clear(keys, vals);
    if (threadIdx.x < 5) bstat[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31;
    unsigned n_act = 0, n_pt = 0, n_sm = 0, n_md = 0, n_lg = 0;
    const int64_t c0 = (int64_t)blockIdx.x * kChunk;
    const int64_t c1 = c0 + kChunk < a.n ? c0 + kChunk : a.n;
    for (int v = 0; v < vs.nviews; ++v) {
        load_view(vs.fcs, v, &sfc);
        const FrameConst &fc = sfc;
        for (int k = threadIdx.x; k < 3 * fc.npal; k += blockDim.x) spal[k] = a.pal[k];
        __syncthreads();
        // all lanes of a warp run the same number of iterations (warp collectives)
        for (int64_t base = c0; base < c1; base += blockDim.x) {
            const int64_t i = base + threadIdx.x;
            const bool valid = i < c1;
            int cls = CLS_INACTIVE;
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(-1.f, 0.f, 0.f, 0.f);
            const int64_t rec = fc.rec_base + i;
            if (valid) {
                float2 q2;
                float crgb[3] = {0.f, 0.f, 0.f};
                if (RGB) {
                    crgb[0] = a.cr[i]; crgb[1] = a.cg[i]; crgb[2] = a.cb[i];
                }
                cls = raster_one(fc, spal, a.x[i], a.y[i], a.z[i], load_h<ATTR>(a.h, i, a.h_log2_min),
                                 load_attr<ATTR != 0>(a.I, i), load_attr<ATTR != 0>(a.s, i),
                                 RGB ? crgb : nullptr, r0, r1, q2);
                a.recs[rec] = Rec{r0, r1};
                if (a.rec2) a.rec2[rec] = q2;
            }
            const TileFoot foot = valid ? tile_footprint(fc, cls, r0, r1) : TileFoot{-1, 0, 0, 1, 0, 0, 0.f};
            const FootLane fl = foot_lane(foot, r0, lane);
            const int total = __shfl_sync(0xffffffffu, fl.incl, 31);
            for (int base = 0; base < total; base += 32) {
                int owner;
                const int ls = foot_pair(fc, fl, base + lane, total, owner);
                count_round(ls >= 0 ? fc.slot_base + ls : -1, keys, vals, a.ovf);
            }
            n_act += cls != CLS_INACTIVE;
            n_pt += cls == CLS_POINT;
            n_sm += cls == CLS_SMALL;
            n_md += cls == CLS_MEDIUM;
            n_lg += cls == CLS_LARGE;
            // append large records to the large list (one atomic per warp)
            const unsigned big = __ballot_sync(0xffffffffu, cls == CLS_LARGE);
            if (big) {
                unsigned basek = 0;
                const int leader = __ffs(big) - 1;
                if (lane == leader) basek = atomicAdd(&a.st->n_large_ids, (unsigned)__popc(big));
                basek = __shfl_sync(0xffffffffu, basek, leader);
                if (cls == CLS_LARGE)
                    a.large_ids[basek + __popc(big & ((1u << lane) - 1u))] = (unsigned)rec;
            }
        }
        // one global atomic per distinct slot of this CTA and view
        hash_flush(keys, vals, a.counts, a.ctab + ((int64_t)blockIdx.x * vs.nviews + v) * kHash);
    }
    n_act = __reduce_add_sync(0xffffffffu, n_act);
    n_pt = __reduce_add_sync(0xffffffffu, n_pt);
    n_sm = __reduce_add_sync(0xffffffffu, n_sm);
    n_md = __reduce_add_sync(0xffffffffu, n_md);
    n_lg = __reduce_add_sync(0xffffffffu, n_lg);
    if (lane == 0) {
        atomicAdd(&bstat[0], (unsigned long long)n_act);
        atomicAdd(&bstat[1], (unsigned long long)n_pt);
        atomicAdd(&bstat[2], (unsigned long long)n_sm);
        atomicAdd(&bstat[3], (unsigned long long)n_md);
        atomicAdd(&bstat[4], (unsigned long long)n_lg);
    }
    __syncthreads();
    if (threadIdx.x < 5 && bstat[threadIdx.x]) {
        // n_active .. n_large are consecutive fields of DevStats
        atomicAdd(&a.st->n_active + threadIdx.x, bstat[threadIdx.x]);
    }
}

void launch_raster(const Views &vs, const RasterArgs &a, int attr, cudaStream_t s) {
    if (a.n <= 0 || vs.nviews <= 0) return;
    const int64_t blocks = (a.n + kChunk - 1) / kChunk;
    const bool rgb = a.cr != nullptr;
    if (attr == 1) {
        if (rgb) raster_kernel<1, true><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
        else raster_kernel<1, false><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
    } else if (attr == 2) {
        if (rgb) raster_kernel<2, true><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
        else raster_kernel<2, false><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
    } else if (attr == 3) {
        if (rgb) raster_kernel<3, true><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
        else raster_kernel<3, false><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
    } else {
        if (rgb) raster_kernel<0, true><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
        else raster_kernel<0, false><<<(unsigned)blocks, 256, 0, s>>>(vs, a);
    }
    ++g_launches;
}

// ---------------------------------------------------------------------------
// Large particles: one warp per large record walks its (possibly thousands
// of) tiles.  mode 0 counts entries, mode 1 scatters record indices through
// the cursors.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) large_tiles_kernel(Views vs, BinArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned nl = a.st->n_large_ids;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nl; w += warps) {
        const unsigned rec = a.large_ids[w];
        const FrameConst &fc = vs.fcs[(int)(rec / (unsigned long long)vs.n)];
        const Rec rc = a.recs[rec];
        const float4 r0 = rc.r0, r1 = rc.r1;
        PixBox b;
        if (!splat_box(fc, r0, r1.x, b)) continue;
        const int tx0 = b.i0 >> fc.tile_shift, ty0 = b.j0 >> fc.tile_shift;
        const int ntx = (b.i1 >> fc.tile_shift) - tx0 + 1;
        const int nt = ntx * ((b.j1 >> fc.tile_shift) - ty0 + 1);
        const float reach2 = disc_reach2(r1.x);
        for (int k = lane; k < nt; k += 32) {
            const int tx = tx0 + k % ntx, ty = ty0 + k / ntx;
            if (!disc_meets_tile(fc, r0, reach2, tx, ty)) continue;
            const int slot = fc.slot_base + L_LARGE * fc.ntiles + ty * fc.ntx + tx;
            if (MODE == 0) {
                atomicAdd(&a.ovf[slot], 1);
            } else {
                const long long pos =
                    (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&a.cursor[slot]), 1ULL);
                if (pos < a.entries_cap)
                    a.entries[pos] = rec;
                else
                    atomicOr(&a.st->err, ERR_LIST_OVERFLOW);
            }
        }
    }
}

void launch_count_large(const Views &vs, const BinArgs &a, int sms, cudaStream_t s) {
    if (vs.n <= 0) return;
    large_tiles_kernel<0><<<sms * 2, 256, 0, s>>>(vs, a);
    ++g_launches;
}

__global__ void slot_sum_kernel(int m, const int *counts, int *ovf) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        ovf[k] += counts[k];
}

__global__ void slot_cursor_kernel(int m, const int *counts, const long long *offsets,
                                   long long *cursor) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        cursor[k] = offsets[k] + counts[k];
}

// ---------------------------------------------------------------------------
// Exclusive scan: one CTA of 1024 threads, each owning a contiguous run.
// ---------------------------------------------------------------------------
template <typename OT>
__global__ void __launch_bounds__(1024) scan_kernel(int m, const int *in, OT *out, OT *cursor,
                                                    int nseg, OT *seg_totals) {
    __shared__ OT wsum[32];
    const int t = threadIdx.x, per = (m + 1023) / 1024;
    const int lo = min(t * per, m), hi = min(lo + per, m);
    OT sum = 0;
    for (int k = lo; k < hi; ++k) sum += (OT)in[k];
    const int lane = t & 31, warp = t >> 5;
    OT incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        OT v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        OT v = wsum[lane];
        OT w = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            OT u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w - v;
    }
    __syncthreads();
    OT run = wsum[warp] + incl - sum;
    for (int k = lo; k < hi; ++k) {
        out[k] = run;
        if (cursor) cursor[k] = run;
        run += (OT)in[k];
    }
    if (t == 1023) out[m] = run;
    __syncthreads();   // makes every thread's results visible to the block
    if (t < nseg) {
        const int seg = m / nseg;
        seg_totals[t] = out[(t + 1) * seg] - out[t * seg];
    }
}

void launch_scan(int m, const int *in, long long *out, long long *cursor, int nseg,
                 long long *seg_totals, cudaStream_t s) {
    scan_kernel<long long><<<1, 1024, 0, s>>>(m, in, out, cursor, nseg, seg_totals);
    ++g_launches;
}

void launch_scan(int m, const int *in, int *out, int *cursor, int nseg, int *seg_totals,
                 cudaStream_t s) {
    scan_kernel<int><<<1, 1024, 0, s>>>(m, in, out, cursor, nseg, seg_totals);
    ++g_launches;
}

void launch_slot_cursor(int m, const int *counts, const long long *offsets, long long *cursor,
                        cudaStream_t s) {
    const int grid = (m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024;
    if (grid <= 0) return;
    slot_cursor_kernel<<<grid, 256, 0, s>>>(m, counts, offsets, cursor);
    ++g_launches;
}

void launch_slot_offsets(int m, int *counts, int *ovf, long long *offsets, long long *cursor,
                         long long *total, cudaStream_t s) {
    const int grid = (m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024;
    if (grid > 0) {
        slot_sum_kernel<<<grid, 256, 0, s>>>(m, counts, ovf);
        ++g_launches;
    }
    scan_kernel<long long><<<1, 1024, 0, s>>>(m, ovf, offsets, nullptr, 1, total);
    ++g_launches;
    if (grid > 0) {
        slot_cursor_kernel<<<grid, 256, 0, s>>>(m, counts, offsets, cursor);
        ++g_launches;
    }
}

// ---------------------------------------------------------------------------
// Work items: a light tile is one item (all its lists, pixels stored); a
// crowded tile is cut into segments of at most kSeg* entries per list, each
// its own item (pixels added).  Large-list entries always form separate
// items of the large pass.  item_counts = [tile-pass items | large items].
// ---------------------------------------------------------------------------
__device__ __forceinline__ int div_up(int a, int b) { return (a + b - 1) / b; }

__global__ void item_count_kernel(Views vs, const long long *off, int *item_counts, DevStats *st) {
    __shared__ int lt[NLIST];
    if (threadIdx.x < NLIST) lt[threadIdx.x] = 0;
    __syncthreads();
    const int T = vs.total_tiles;
    int tot[NLIST] = {0, 0, 0, 0};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < T; g += gridDim.x * blockDim.x) {
        const FrameConst &fc = vs.fcs[view_of_tile(vs.fcs, vs.nviews, g)];
        const int t = g - fc.tile_base, nt = fc.ntiles, sb = fc.slot_base;
        const int cp = (int)(off[sb + L_POINT * nt + t + 1] - off[sb + L_POINT * nt + t]);
        const int cs = (int)(off[sb + L_SMALL * nt + t + 1] - off[sb + L_SMALL * nt + t]);
        const int cm = (int)(off[sb + L_MEDIUM * nt + t + 1] - off[sb + L_MEDIUM * nt + t]);
        const int cl = (int)(off[sb + L_LARGE * nt + t + 1] - off[sb + L_LARGE * nt + t]);
        tot[0] += cp; tot[1] += cs; tot[2] += cm; tot[3] += cl;
        int n = 0;
        if (cp + cs + cm > 0) {
            if (cp <= kSegPoint && cs <= kSegSmall && cm <= kSegMedium)
                n = 1;
            else
                n = div_up(cp, kSegPoint) + div_up(cs, kSegSmall) + div_up(cm, kSegMedium);
        }
        item_counts[g] = n;
        item_counts[T + g] = div_up(cl, kSegLarge);
    }
    for (int l = 0; l < NLIST; ++l) {
        const int v = __reduce_add_sync(0xffffffffu, tot[l]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&lt[l], v);
    }
    __syncthreads();
    if (threadIdx.x < NLIST && lt[threadIdx.x]) atomicAdd(&st->totals[threadIdx.x], lt[threadIdx.x]);
}

void launch_item_counts(const Views &vs, const long long *offsets, int *item_counts, DevStats *st,
                        cudaStream_t s) {
    const int blocks = (vs.total_tiles + 255) / 256;
    item_count_kernel<<<blocks, 256, 0, s>>>(vs, offsets, item_counts, st);
    ++g_launches;
}

__device__ __forceinline__ void put_item(WorkItem *items, int cap, int pos, WorkItem w, DevStats *st) {
    if (pos < cap)
        items[pos] = w;
    else
        atomicOr(&st->err, ERR_LIST_OVERFLOW);
}

// One warp per tile: the lanes write the tile's segments side by side (a
// crowded tile has hundreds), in the same order as one thread would.
__global__ void fill_items_kernel(Views vs, const long long *off, const int *ioff, WorkItem *items,
                                  int cap, DevStats *st) {
    const int T = vs.total_tiles;
    const int seg[NLIST] = {kSegPoint, kSegSmall, kSegMedium, kSegLarge};
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < T; g += warps) {
        const int v = view_of_tile(vs.fcs, vs.nviews, g);
        const FrameConst &fc = vs.fcs[v];
        const int t = g - fc.tile_base, nt = fc.ntiles, sb = fc.slot_base;
        int w = ioff[g];
        const int nw = ioff[g + 1] - w;
        if (nw == 1) {
            if (lane == 0) put_item(items, cap, w, {g, (v << 8) | kAllLists, 0, 0}, st);
        } else if (nw > 1) {
            for (int l = 0; l < L_LARGE; ++l) {
                const long long b = off[sb + l * nt + t], e = off[sb + l * nt + t + 1];
                const int ns = (int)((e - b + seg[l] - 1) / seg[l]);
                for (int k = lane; k < ns; k += 32) {
                    const long long kb = b + (long long)k * seg[l];
                    put_item(items, cap, w + k, {g, (v << 8) | l, kb, kb + seg[l] < e ? kb + seg[l] : e}, st);
                }
                w += ns;
            }
        }
        const int wl = ioff[T + g];
        const long long b = off[sb + L_LARGE * nt + t], e = off[sb + L_LARGE * nt + t + 1];
        const int ns = (int)((e - b + kSegLarge - 1) / kSegLarge);
        for (int k = lane; k < ns; k += 32) {
            const long long kb = b + (long long)k * kSegLarge;
            put_item(items, cap, wl + k,
                     {g, (v << 8) | L_LARGE, kb, kb + kSegLarge < e ? kb + kSegLarge : e}, st);
        }
    }
}

void launch_fill_items(const Views &vs, const long long *offsets, const int *item_offsets,
                       WorkItem *items, int items_cap, DevStats *st, cudaStream_t s) {
    const int blocks = (vs.total_tiles + 7) / 8;     // 8 warps of 256 threads, a warp per tile
    fill_items_kernel<<<blocks, 256, 0, s>>>(vs, offsets, item_offsets, items, items_cap, st);
    ++g_launches;
}

// ---------------------------------------------------------------------------
// Scatter particle ids of points, small and medium particles into their
// tiles' lists (order inside a tile follows the atomics, which is harmless:
// E_p = A_p makes the sum order-independent, Sec. 2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ TileFoot load_foot(const FrameConst &fc, const BinArgs &a, int64_t rec,
                                              bool valid, float4 &r0, float4 &r1) {
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    r1 = make_float4(-1.f, 0.f, 0.f, 0.f);
    if (!valid) return TileFoot{-1, 0, 0, 1, 0, 0, 0.f};
    const Rec rc = a.recs[rec];
    r1 = rc.r1;
    const int cls = record_class(fc, r1.x);
    if (cls == CLS_INACTIVE || cls == CLS_LARGE) return TileFoot{-1, 0, 0, 1, 0, 0, 0.f};
    r0 = rc.r0;
    return tile_footprint(fc, cls, r0, r1);
}

// Scatter record indices of points, small and medium particles into their
// tiles' lists in one pass: per CTA and view, the rasteriser's table gives
// every slot the CTA used its range base offsets[slot] + offset; each entry
// goes to base + its rank among the CTA's entries of that slot (shared-memory
// counters, lanes of a warp with the same slot combined by a match mask).
// Keys that had no room in the table go through the cursors.  Order inside a
// tile follows the atomics, which is harmless: E_p = A_p makes the sum
// order-independent (Sec. 2); the absorption mode sorts the lists afterwards.
__global__ void __launch_bounds__(256) scatter_kernel(Views vs, BinArgs a) {
    extern __shared__ long long scatter_smem[];
    long long *bases = scatter_smem;                         // kHash
    int *keys = reinterpret_cast<int *>(bases + kHash);      // kHash
    int *vals = keys + kHash;                                // kHash
    __shared__ FrameConst sfc;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t c0 = (int64_t)blockIdx.x * kChunk;
    const int64_t c1 = c0 + kChunk < vs.n ? c0 + kChunk : vs.n;
    for (int v = 0; v < vs.nviews; ++v) {
        load_view(vs.fcs, v, &sfc);     // (begins and ends with a barrier)
        const FrameConst &fc = sfc;
        const int2 *tab = a.ctab + ((int64_t)blockIdx.x * vs.nviews + v) * kHash;
        for (int k = threadIdx.x; k < kHash; k += blockDim.x) {
            const int2 t = tab[k];
            keys[k] = t.x;
            vals[k] = 0;
            bases[k] = t.x >= 0 ? a.offsets[t.x] + t.y : 0;
        }
        __syncthreads();
        for (int64_t base = c0; base < c1; base += blockDim.x) {
            const int64_t i = base + threadIdx.x;
            const int64_t rec = fc.rec_base + i;
            float4 r0, r1;
            const TileFoot f = load_foot(fc, a, rec, i < c1, r0, r1);
            const FootLane fl = foot_lane(f, r0, lane);
            const int total = __shfl_sync(0xffffffffu, fl.incl, 31);
            for (int pbase = 0; pbase < total; pbase += 32) {
                int owner;
                const int ls = foot_pair(fc, fl, pbase + lane, total, owner);
                const unsigned orec = __shfl_sync(0xffffffffu, (unsigned)rec, owner);
                const int key = ls >= 0 ? fc.slot_base + ls : -1;
                const unsigned m = __match_any_sync(0xffffffffu, key);
                const int leader = __ffs(m) - 1;
                long long pos = 0;
                if (key >= 0 && lane == leader) {
                    const int slot = hash_slot(keys, key, false);
                    if (slot >= 0)
                        pos = bases[slot] + atomicAdd(&vals[slot], __popc(m));
                    else
                        pos = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&a.cursor[key]),
                                                   (unsigned long long)__popc(m));
                }
                pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(m & lt);
                if (key >= 0) {
                    if (pos < a.entries_cap)
                        a.entries[pos] = orec;
                    else
                        atomicOr(&a.st->err, ERR_LIST_OVERFLOW);
                }
            }
        }
    }
}

void launch_scatter(const Views &vs, const BinArgs &a, int sms, cudaStream_t s) {
    if (vs.n <= 0 || vs.nviews <= 0) return;
    const int64_t blocks = (vs.n + kChunk - 1) / kChunk;
    const size_t smem = (size_t)kHash * (sizeof(long long) + 2 * sizeof(int));
    cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    scatter_kernel<<<(unsigned)blocks, 256, smem, s>>>(vs, a);
    ++g_launches;
    large_tiles_kernel<1><<<sms * 2, 256, 0, s>>>(vs, a);
    ++g_launches;
}

// ---------------------------------------------------------------------------
// Diagnostic: exact count of covered (particle, pixel) pairs per class, using
// the same FP32 clip test as the render passes.  Not part of a render.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) count_work_kernel(FrameConst fc, const Rec *recs, int64_t n,
                                                         unsigned long long *work) {
    unsigned long long acc[4] = {0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 r1 = recs[i].r1;
        const int cls = record_class(fc, r1.x);
        if (cls == CLS_INACTIVE) continue;
        const float4 r0 = recs[i].r0;
        const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
        if (cls == CLS_POINT) {
            acc[0] += (xi >= 0 && yi >= 0 && xi < fc.width && yi < fc.height);
            continue;
        }
        PixBox b;
        if (!splat_box(fc, r0, r1.x, b)) continue;
        unsigned long long cnt = 0;
        for (int j = b.j0; j <= b.j1; ++j) {
            const float dy = (float)(j - yi) + (0.5f - r0.z);
            const float rem = r1.x - dy * dy;
            if (rem < 0.f) continue;
            for (int i2 = b.i0; i2 <= b.i1; ++i2) {
                const float dx = (float)(i2 - xi) + (0.5f - r0.y);
                cnt += dx * dx <= rem;
            }
        }
        acc[cls] += cnt;
    }
    for (int k = 0; k < 4; ++k) {
        unsigned long long v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&work[k], v);
    }
}

void launch_count_work(const FrameConst &fc, const Rec *recs, int64_t n,
                       unsigned long long *work, int sms, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
    count_work_kernel<<<(unsigned)blocks, 256, 0, s>>>(fc, recs, n, work);
    ++g_launches;
}

}  // namespace spl
