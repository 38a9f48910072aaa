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
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = a.hi / b.hi;
    df r = df_add(a, df_neg(df_mul_f(b, q1)));
    float q2 = r.hi / b.hi;
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

template <bool F16>
__device__ __forceinline__ float load_attr(const void *p, int64_t i) {
    if (F16) return __half2float(static_cast<const __half *>(p)[i]);
    return static_cast<const float *>(p)[i];
}

// Rasterise one particle into its record; returns its class.
__device__ __forceinline__ int raster_one(const FrameConst &fc, const float *spal, float x, float y,
                                          float z, float h, float inten, float s, float4 &r0,
                                          float4 &r1) {
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
    const float zc = c[2].hi;
    if (!(zc > fc.z_near)) return CLS_INACTIVE;
    // perspective projection
    const df f = {fc.fhi, fc.flo};
    df xs = df_add({fc.half_w, 0.f}, df_mul(f, df_div(c[0], c[2])));
    df ys = df_add({fc.half_h, 0.f}, df_neg(df_mul(f, df_div(c[1], c[2]))));
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
    if (fc.npal == 1) {
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
    return record_class(fc, r1.x);
}

// Count the tile-list entries of one rasterised particle (points, small and
// medium; large particles are counted by count_large_kernel).
__device__ __forceinline__ void count_entries(const FrameConst &fc, int cls, float4 r0, float4 r1,
                                              int *counts) {
    if (cls == CLS_POINT) {
        const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
        if (xi >= 0 && yi >= 0 && xi < fc.width && yi < fc.height)
            atomicAdd(&counts[L_POINT * fc.ntiles + (yi / fc.tile) * fc.ntx + xi / fc.tile], 1);
        return;
    }
    if (cls != CLS_SMALL && cls != CLS_MEDIUM) return;
    PixBox b;
    if (!splat_box(fc, r0, r1.x, b)) return;
    const int list = cls == CLS_SMALL ? L_SMALL : L_MEDIUM;
    for (int ty = b.j0 / fc.tile; ty <= b.j1 / fc.tile; ++ty)
        for (int tx = b.i0 / fc.tile; tx <= b.i1 / fc.tile; ++tx)
            if (disc_meets_tile(fc, r0, r1.x, tx, ty))
                atomicAdd(&counts[list * fc.ntiles + ty * fc.ntx + tx], 1);
}

template <bool F16>
__global__ void __launch_bounds__(256) raster_kernel(FrameConst fc, RasterArgs a) {
    __shared__ float spal[3 * kMaxPalette];
    for (int k = threadIdx.x; k < 3 * fc.npal; k += blockDim.x) spal[k] = a.pal[k];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned n_act = 0, n_pt = 0, n_sm = 0, n_md = 0, n_lg = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // all lanes of a warp run the same number of iterations (warp collectives)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < a.n;
        int cls = CLS_INACTIVE;
        float4 r0, r1;
        if (valid) {
            cls = raster_one(fc, spal, a.x[i], a.y[i], a.z[i], load_attr<F16>(a.h, i),
                             load_attr<F16>(a.I, i), load_attr<F16>(a.s, i), r0, r1);
            a.rec0[i] = r0;
            a.rec1[i] = r1;
            count_entries(fc, cls, r0, r1, a.counts);
        }
        n_act += cls != CLS_INACTIVE;
        n_pt += cls == CLS_POINT;
        n_sm += cls == CLS_SMALL;
        n_md += cls == CLS_MEDIUM;
        n_lg += cls == CLS_LARGE;
        // append large particles to the large list (one atomic per warp)
        const unsigned big = __ballot_sync(0xffffffffu, cls == CLS_LARGE);
        if (big) {
            unsigned basek = 0;
            const int leader = __ffs(big) - 1;
            if (lane == leader) basek = atomicAdd(&a.st->n_large_ids, (unsigned)__popc(big));
            basek = __shfl_sync(0xffffffffu, basek, leader);
            if (cls == CLS_LARGE)
                a.large_ids[basek + __popc(big & ((1u << lane) - 1u))] = (unsigned)i;
        }
    }
    n_act = __reduce_add_sync(0xffffffffu, n_act);
    n_pt = __reduce_add_sync(0xffffffffu, n_pt);
    n_sm = __reduce_add_sync(0xffffffffu, n_sm);
    n_md = __reduce_add_sync(0xffffffffu, n_md);
    n_lg = __reduce_add_sync(0xffffffffu, n_lg);
    if (lane == 0) {
        if (n_act) atomicAdd(&a.st->n_active, (unsigned long long)n_act);
        if (n_pt) atomicAdd(&a.st->n_point, (unsigned long long)n_pt);
        if (n_sm) atomicAdd(&a.st->n_small, (unsigned long long)n_sm);
        if (n_md) atomicAdd(&a.st->n_medium, (unsigned long long)n_md);
        if (n_lg) atomicAdd(&a.st->n_large, (unsigned long long)n_lg);
    }
}

void launch_raster(const FrameConst &fc, const RasterArgs &a, bool f16, int sms, cudaStream_t s) {
    if (a.n <= 0) return;
    int64_t blocks = (a.n + 255) / 256;
    blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
    if (f16)
        raster_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(fc, a);
    else
        raster_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(fc, a);
}

// ---------------------------------------------------------------------------
// Large particles: one warp per particle walks its (possibly thousands of)
// tiles.  mode 0 counts entries, mode 1 scatters ids through the cursors.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) large_tiles_kernel(FrameConst fc, BinArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned nl = a.st->n_large_ids;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nl; w += warps) {
        const unsigned id = a.large_ids[w];
        const float4 r0 = a.rec0[id];
        const float4 r1 = a.rec1[id];
        PixBox b;
        if (!splat_box(fc, r0, r1.x, b)) continue;
        const int tx0 = b.i0 / fc.tile, ty0 = b.j0 / fc.tile;
        const int ntx = b.i1 / fc.tile - tx0 + 1;
        const int nt = ntx * (b.j1 / fc.tile - ty0 + 1);
        for (int k = lane; k < nt; k += 32) {
            const int tx = tx0 + k % ntx, ty = ty0 + k / ntx;
            if (!disc_meets_tile(fc, r0, r1.x, tx, ty)) continue;
            const int slot = L_LARGE * fc.ntiles + ty * fc.ntx + tx;
            if (MODE == 0) {
                atomicAdd(&a.counts[slot], 1);
            } else {
                const int pos = atomicAdd(&a.cursor[slot], 1);
                if (pos < a.entries_cap)
                    a.entries[pos] = id;
                else
                    atomicOr(&a.st->err, ERR_LIST_OVERFLOW);
            }
        }
    }
}

void launch_count_large(const FrameConst &fc, const BinArgs &a, int sms, cudaStream_t s) {
    if (a.n <= 0) return;
    large_tiles_kernel<0><<<sms * 2, 256, 0, s>>>(fc, a);
}

// ---------------------------------------------------------------------------
// Exclusive scan of the (list, tile) counts: one CTA of 1024 threads, each
// owning a contiguous run of slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) scan_kernel(int m, int ntiles, const int *counts,
                                                    int *offsets, int *cursor, DevStats *st) {
    __shared__ int wsum[32];
    const int t = threadIdx.x, per = (m + 1023) / 1024;
    const int lo = min(t * per, m), hi = min(lo + per, m);
    int sum = 0;
    for (int k = lo; k < hi; ++k) sum += counts[k];
    // block-wide exclusive scan of the per-thread sums
    const int lane = t & 31, warp = t >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        int w = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w - v;
    }
    __syncthreads();
    int run = wsum[warp] + incl - sum;
    for (int k = lo; k < hi; ++k) {
        offsets[k] = run;
        cursor[k] = run;
        run += counts[k];
    }
    if (t == 1023) offsets[m] = run;
    __syncthreads();   // makes every thread's offsets visible to the block
    if (t < NLIST) st->totals[t] = offsets[(t + 1) * ntiles] - offsets[t * ntiles];
}

void launch_scan(const FrameConst &fc, int *counts, int *offsets, int *cursor, DevStats *st,
                 cudaStream_t s) {
    scan_kernel<<<1, 1024, 0, s>>>(NLIST * fc.ntiles, fc.ntiles, counts, offsets, cursor, st);
}

// ---------------------------------------------------------------------------
// Scatter particle ids of points, small and medium particles into their
// tiles' lists (order inside a tile follows the atomics, which is harmless:
// E_p = A_p makes the sum order-independent, Sec. 2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) scatter_kernel(FrameConst fc, BinArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const float4 r1 = a.rec1[i];
        const int cls = record_class(fc, r1.x);
        if (cls == CLS_INACTIVE || cls == CLS_LARGE) continue;
        const float4 r0 = a.rec0[i];
        if (cls == CLS_POINT) {
            const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
            if (xi < 0 || yi < 0 || xi >= fc.width || yi >= fc.height) continue;
            const int pos = atomicAdd(
                &a.cursor[L_POINT * fc.ntiles + (yi / fc.tile) * fc.ntx + xi / fc.tile], 1);
            if (pos < a.entries_cap) a.entries[pos] = (unsigned)i;
            else atomicOr(&a.st->err, ERR_LIST_OVERFLOW);
            continue;
        }
        PixBox b;
        if (!splat_box(fc, r0, r1.x, b)) continue;
        const int list = cls == CLS_SMALL ? L_SMALL : L_MEDIUM;
        for (int ty = b.j0 / fc.tile; ty <= b.j1 / fc.tile; ++ty)
            for (int tx = b.i0 / fc.tile; tx <= b.i1 / fc.tile; ++tx) {
                if (!disc_meets_tile(fc, r0, r1.x, tx, ty)) continue;
                const int pos = atomicAdd(&a.cursor[list * fc.ntiles + ty * fc.ntx + tx], 1);
                if (pos < a.entries_cap) a.entries[pos] = (unsigned)i;
                else atomicOr(&a.st->err, ERR_LIST_OVERFLOW);
            }
    }
}

void launch_scatter(const FrameConst &fc, const BinArgs &a, int sms, cudaStream_t s) {
    if (a.n <= 0) return;
    int64_t blocks = (a.n + 255) / 256;
    blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
    scatter_kernel<<<(unsigned)blocks, 256, 0, s>>>(fc, a);
    large_tiles_kernel<1><<<sms * 2, 256, 0, s>>>(fc, a);
}

// ---------------------------------------------------------------------------
// Diagnostic: exact count of covered (particle, pixel) pairs per class, using
// the same FP32 clip test as the render passes.  Not part of a render.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) count_work_kernel(FrameConst fc, const float4 *rec0,
                                                         const float4 *rec1, int64_t n,
                                                         unsigned long long *work) {
    unsigned long long acc[4] = {0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 r1 = rec1[i];
        const int cls = record_class(fc, r1.x);
        if (cls == CLS_INACTIVE) continue;
        const float4 r0 = rec0[i];
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

void launch_count_work(const FrameConst &fc, const float4 *rec0, const float4 *rec1, int64_t n,
                       unsigned long long *work, int sms, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
    count_work_kernel<<<(unsigned)blocks, 256, 0, s>>>(fc, rec0, rec1, n, work);
}

}  // namespace spl
