// spl_sched.cu -- scheduling of the work items of the persistent passes.
//
// The paper notes (Sec. 4 Remarks, Sec. 5.1) that the number of particles per
// tile varies a lot and unbalances the blocks.  Here every work item gets a
// 32-value description of its work -- per radius bin (bin b holds r in
// [0.5 2^b, 0.5 2^(b+1)), bin 0 also everything below 1 px, bin 15 everything
// above) the number of its particles and the number of tile pixels inside
// their boxes, both log1p-scaled -- from which a cost is predicted either by
// the tile-cost network (spl_mlp.cu) or by the count heuristic
// a + b log1p(entries).  Items are then taken longest-first (LPT) by the
// persistent CTAs: a counting sort of the predicted costs into 256 buckets.
#include "spl_geom.cuh"

namespace spl {

__device__ __forceinline__ int radius_bin(float r2) {
    const float r = sqrtf(r2);
    if (r < 1.f) return 0;
    const int b = (int)floorf(log2f(r)) + 1;
    return b > 15 ? 15 : b;
}

// Pixel-centre box of a splat without the safety margin of the binning (the
// feature is the number of tile pixels with |i + 1/2 - x_s| <= r and
// |j + 1/2 - y_s| <= r), cut to the image.
__device__ __forceinline__ bool exact_box(const FrameConst &fc, float4 r0, float r2, PixBox &b) {
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    const float r = sqrtf(r2), lim = 70000.f;
    b.i0 = max(xi + (int)ceilf(fmaxf(r0.y - 0.5f - r, -lim)), 0);
    b.i1 = min(xi + (int)floorf(fminf(r0.y - 0.5f + r, lim)), fc.width - 1);
    b.j0 = max(yi + (int)ceilf(fmaxf(r0.z - 0.5f - r, -lim)), 0);
    b.j1 = min(yi + (int)floorf(fminf(r0.z - 0.5f + r, lim)), fc.height - 1);
    return b.i0 <= b.i1 && b.j0 <= b.j1;
}

// One warp per item: histogram of its entries in shared memory.  With
// max_sample > 0 at most about max_sample entries per list range are read
// (evenly spaced) and the histogram is scaled up by the sampling stride: an
// estimate that costs a bounded number of gathers per item.
__global__ void __launch_bounds__(256) item_features_kernel(Views vs, TileArgs a, float area_scale,
                                                           int max_sample, float *feat,
                                                           int *n_entries) {
    __shared__ float hist[8][kFeat];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_all = min(a.st->item_totals[0] + a.st->item_totals[1], a.items_cap);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + warp; it < n_all; it += nwarps) {
        hist[warp][lane] = 0.f;
        __syncwarp();
        const WorkItem w = a.items[it];
        const FrameConst &fc = vs.fcs[item_view(w)];
        const int list = item_list(w);
        const int tile = w.tile - fc.tile_base;
        const int x0 = (tile % fc.ntx) * fc.tile, y0 = (tile / fc.ntx) * fc.tile;
        int total = 0;
        for (int l = 0; l < 3; ++l) {
            long long b, e;
            if (list < 0) {
                b = a.offsets[fc.slot_base + l * fc.ntiles + tile];
                e = a.offsets[fc.slot_base + l * fc.ntiles + tile + 1];
            } else {
                if (l > 0) break;
                b = w.start;
                e = w.end;
            }
            total += (int)(e - b);
            long long stride = 1;
            if (max_sample > 0 && e - b > max_sample) stride = (e - b + max_sample - 1) / max_sample;
            const float wgt = (float)stride;
            for (long long k = b + lane * stride; k < e; k += 32 * stride) {
                const unsigned rec = a.entries[k];
                const Rec rc = a.recs[rec];
                const float4 r0 = rc.r0, r1 = rc.r1;
                const int bin = radius_bin(r1.x);
                float area = 1.f;
                if (record_class(fc, r1.x) != CLS_POINT) {
                    PixBox bx;
                    area = 0.f;
                    if (exact_box(fc, r0, r1.x, bx)) {
                        const int i0 = max(bx.i0, x0), i1 = min(bx.i1, x0 + fc.tile - 1);
                        const int j0 = max(bx.j0, y0), j1 = min(bx.j1, y0 + fc.tile - 1);
                        if (i0 <= i1 && j0 <= j1) area = (float)((i1 - i0 + 1) * (j1 - j0 + 1));
                    }
                }
                atomicAdd(&hist[warp][bin], wgt);
                atomicAdd(&hist[warp][16 + bin], wgt * area);
            }
        }
        __syncwarp();
        const float v = hist[warp][lane];
        feat[(size_t)it * kFeat + lane] = lane < 16 ? log1pf(v) : log1pf(v / area_scale);
        if (lane == 0) n_entries[it] = total;
        __syncwarp();
    }
}

void launch_item_features(const Views &vs, const TileArgs &a, float area_scale, int max_sample,
                          float *feat, int *n_entries, int sms, cudaStream_t s) {
    item_features_kernel<<<sms * 4, 256, 0, s>>>(vs, a, area_scale, max_sample, feat, n_entries);
    ++g_launches;
}

// Entries of every item only (what the count heuristic needs): a segment's
// length, or the sum of a whole tile's list lengths.
__global__ void item_entries_kernel(Views vs, TileArgs a, int *n_entries) {
    const int n_all = min(a.st->item_totals[0] + a.st->item_totals[1], a.items_cap);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_all; it += gridDim.x * blockDim.x) {
        const WorkItem w = a.items[it];
        long long cnt = w.end - w.start;
        if (item_list(w) < 0) {
            const FrameConst &fc = vs.fcs[item_view(w)];
            const int tile = w.tile - fc.tile_base;
            cnt = 0;
            for (int l = 0; l < 3; ++l)
                cnt += a.offsets[fc.slot_base + l * fc.ntiles + tile + 1] -
                       a.offsets[fc.slot_base + l * fc.ntiles + tile];
        }
        n_entries[it] = (int)cnt;
    }
}

void launch_item_entries(const Views &vs, const TileArgs &a, int *n_entries, int sms,
                         cudaStream_t s) {
    item_entries_kernel<<<sms * 4, 256, 0, s>>>(vs, a, n_entries);
    ++g_launches;
}

// Predicted log-cycles of every item: the network when theta is given, else
// the count heuristic heur[0] + heur[1] log1p(entries).
__global__ void __launch_bounds__(256) item_cost_kernel(const float *feat, const int *n_entries,
                                                        const float *theta, const float *heur,
                                                        int items_cap, const DevStats *st,
                                                        float *cost) {
    __shared__ float w[kNParam];
    const int n_all = min(st->item_totals[0] + st->item_totals[1], items_cap);
    if (theta) {
        for (int k = threadIdx.x; k < kNParam; k += blockDim.x) w[k] = theta[k];
        __syncthreads();
    }
    const float *W1 = w, *b1 = w + kHid * kFeat, *w2 = b1 + kHid, *b2 = w2 + kHid;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_all; it += gridDim.x * blockDim.x) {
        if (!theta) {
            cost[it] = heur[0] + heur[1] * log1pf((float)n_entries[it]);
            continue;
        }
        float x[kFeat];
#pragma unroll
        for (int i = 0; i < kFeat; ++i) x[i] = feat[(size_t)it * kFeat + i];
        float y = b2[0];
        for (int j = 0; j < kHid; ++j) {
            float z = b1[j];
#pragma unroll
            for (int i = 0; i < kFeat; ++i) z = fmaf(W1[j * kFeat + i], x[i], z);
            if (z > 0.f) y = fmaf(w2[j], z, y);
        }
        cost[it] = y;
    }
}

void launch_item_cost(const float *feat, const int *n_entries, const float *theta,
                      const float *heur, int items_cap, const DevStats *st, float *cost,
                      cudaStream_t s) {
    item_cost_kernel<<<256, 256, 0, s>>>(feat, n_entries, theta, heur, items_cap, st, cost);
    ++g_launches;
}

// Longest first: bucket b holds predicted log-cycles in (25 - (b+1)/12.8, 25 - b/12.8].
__device__ __forceinline__ int cost_bucket(float c) {
    const int b = (int)((25.f - c) * 12.8f);
    return b < 0 ? 0 : (b > 255 ? 255 : b);
}

// hist: 2 x 256 bucket counts (pass 0: tile pass, pass 1: large pass).
__global__ void order_count_kernel(const float *cost, int items_cap, const DevStats *st, int *hist) {
    const int n0 = st->item_totals[0];
    const int n_all = min(n0 + st->item_totals[1], items_cap);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_all; it += gridDim.x * blockDim.x)
        atomicAdd(&hist[(it >= n0 ? 256 : 0) + cost_bucket(cost[it])], 1);
}

__global__ void order_scan_kernel(int *hist) {
    // two independent exclusive scans of 256 buckets (one warp each)
    const int pass = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (pass > 1) return;
    int *h = hist + 256 * pass;
    int run = 0;
    for (int base = 0; base < 256; base += 32) {
        const int v = h[base + lane];
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        h[base + lane] = run + incl - v;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void order_place_kernel(const float *cost, int items_cap, const DevStats *st, int *hist,
                                   int *order) {
    const int n0 = st->item_totals[0];
    const int n_all = min(n0 + st->item_totals[1], items_cap);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_all; it += gridDim.x * blockDim.x) {
        const int pass = it >= n0;
        const int pos = atomicAdd(&hist[256 * pass + cost_bucket(cost[it])], 1);
        order[(pass ? n0 : 0) + pos] = it - (pass ? n0 : 0);
    }
}

void launch_order_items(const float *cost, int items_cap, DevStats *st, int *hist, int *order,
                        cudaStream_t s) {
    cudaMemsetAsync(hist, 0, sizeof(int) * 512, s);
    order_count_kernel<<<256, 256, 0, s>>>(cost, items_cap, st, hist);
    ++g_launches;
    order_scan_kernel<<<1, 64, 0, s>>>(hist);
    ++g_launches;
    order_place_kernel<<<256, 256, 0, s>>>(cost, items_cap, st, hist, order);
    ++g_launches;
}

__global__ void log_cycles_kernel(const long long *cycles, int64_t n, float *logc) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        logc[k] = logf((float)(cycles[k] > 1 ? cycles[k] : 1));
}

void launch_log_cycles(const long long *cycles, int64_t n, float *logc, cudaStream_t s) {
    if (n <= 0) return;
    log_cycles_kernel<<<256, 256, 0, s>>>(cycles, n, logc);
    ++g_launches;
}

}  // namespace spl
