// spl_internal.cuh -- shared declarations of the GB300 Splotch renderer.
//
// Data layout in HBM (one frame):
//   particles   SoA: x, y, z (FP32) and h, I, s (FP32 or binary16), owned by the
//               context, read once per frame by the rasteriser.
//   records     one 32-byte Rec per particle id (and view):
//                 r0 = { packed (xi, yi) as two int16, xf, yf, kq }
//                 r1 = { r^2 (negative when inactive), e_R, e_G, e_B }
//               where x_s = xi + xf with xf in [0, 1) (the integer part keeps
//               the sub-pixel position exact to ~1e-7 px in FP32) and
//               kq = log2(e) / sigma_s^2, so exp(-d^2/sigma^2) = 2^(-kq d^2).
//   counts      int32 [NLIST][n_tiles]: entries per (list, tile), then an
//               exclusive scan into offsets [NLIST * n_tiles + 1].
//   entries     uint32 particle ids, grouped by list, then by tile.
//   image       caller-owned H x W x 3 FP32.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace spl {

// Lists a particle can be binned into (Sec. 4 classes by screen radius).
enum : int { L_POINT = 0, L_SMALL = 1, L_MEDIUM = 2, L_LARGE = 3, NLIST = 4 };
enum : int { CLS_INACTIVE = -2, CLS_POINT = 0, CLS_SMALL = 1, CLS_MEDIUM = 2, CLS_LARGE = 3 };

// Device-side error bits (reported as SPL_EDEVICE).
enum : unsigned { ERR_LIST_OVERFLOW = 1u, ERR_INDEX = 2u };

constexpr int kMaxPalette = 1024;
constexpr int kTileThreads = 256;        // 8 warps per tile CTA

// Per-frame constants (camera in double-float: hi + lo pairs of FP32).
struct FrameConst {
    float Rhi[9], Rlo[9];      // rows right, up', fwd
    float Ehi[3], Elo[3];      // R * eye
    float fhi, flo;            // focal length
    float half_w, half_h;
    float z_near;
    float sig_fac;             // sigma_per_h / s_box
    float chi;
    float r_sml2, r_small2, r_large2;   // squared class radii
    float s_min, s_inv;        // colour-scalar normalisation
    float brightness;
    int npal;
    int width, height;
    int tile, ntx, nty, ntiles;
    int tile_shift;            // log2(tile)
    // place of this view in a batch of views
    int view;                  // index in the batch
    int tile_base;             // first global tile: global tile = tile_base + local tile
    int slot_base;             // first list slot: slot = slot_base + list * ntiles + tile
    int absorb;                // general absorption (Eq. 1, E != A): one depth-sorted list per tile
    float absorption;          // A = absorption * brightness * I
    int log_flags;             // 1: log10 of I, 2: log10 of s before normalisation
    long long rec_base;        // first record: record = rec_base + particle id
};

// Kernels launched by this host thread: every launch site adds one, and a
// render reports the difference across its own launches.
extern thread_local long long g_launches;

// A batch of views rendered together: one particle set, nviews cameras.
// Per-view constants live in device memory; the tile side is common.
constexpr int kMaxViews = 64;
struct Views {
    const FrameConst *fcs;     // device, nviews entries
    int nviews;
    int total_tiles;           // sum over views of ntiles
    int tile;                  // common tile side
    int64_t n;                 // particles
};

// Device status block (one per context).
// Everything before `err` is cleared at the start of every frame; `err`
// accumulates until the host reads and clears it.
struct DevStats {
    unsigned long long n_active, n_point, n_small, n_medium, n_large;
    unsigned int n_large_ids;  // large records appended this frame
    int totals[NLIST];         // entries per list, summed over views
    long long slot_total;      // all entries (written by the slot scan)
    int item_totals[2];        // work items of the tile pass and of the large pass
    int item_counter[2];       // dynamic work-item counters of the two passes
    unsigned int err;          // ERR_* bits
};

// A work item of the persistent tile / large passes: a tile (global index
// over the batch) and a range of one of its lists, or every list of a tile
// light enough to be done by one CTA, which then stores its pixels instead of
// adding them.  lv packs the view (high bits) and the list (low 8 bits, 0xFF
// for "every list").
struct WorkItem {
    int tile, lv;
    long long start, end;
};
constexpr int kAllLists = 0xFF;
__host__ __device__ inline int item_view(const WorkItem &w) { return w.lv >> 8; }
__host__ __device__ inline int item_list(const WorkItem &w) {
    return (w.lv & 0xFF) == kAllLists ? -1 : (w.lv & 0xFF);
}

// Largest list segment one work item takes (per list), so that a crowded
// tile (a halo core holding 1e5-1e6 particles) is spread over many CTAs.
constexpr int kSegPoint = 8192, kSegSmall = 2048, kSegMedium = 1024, kSegLarge = 512;

// Binning CTAs: each takes kChunk consecutive particles and aggregates their
// list slots in a shared-memory hash table of kHash slots, which the scatter
// reuses (one table per CTA and view).
constexpr int kHashBits = 11;
constexpr int kHash = 1 << kHashBits;
constexpr int kChunk = 2048;
__host__ __device__ constexpr int64_t ctab_entries(int64_t n, int nviews) {
    return ((n + kChunk - 1) / kChunk > 0 ? (n + kChunk - 1) / kChunk : 1) *
           (nviews > 0 ? nviews : 1) * kHash;
}

// One rasterised particle: r0 = (packed pixel xi, yi; sub-pixel xf, yf;
// 1 / (sigma^2 ln 2)), r1 = (r^2; e_R, e_G, e_B).  The two halves sit in one
// 32-byte record, so that a gather through a tile list reads one sector.
struct Rec {
    float4 r0, r1;
};
static_assert(sizeof(Rec) == 32, "32-byte records");

struct RasterArgs {
    int64_t n;
    const float *x, *y, *z;
    const void *h, *I, *s;
    const float *pal;          // npal * 3
    const float *cr, *cg, *cb; // optional per-particle colour components (replace the palette)
    float h_log2_min;          // ATTR 3: h = 2^(h_log2_min + code / 4096)
    Rec *recs;                 // nviews * n records
    float2 *rec2;              // absorption mode: (A, depth key) per record, else null
    int *counts;               // list slots of all views: entries counted through the CTA tables
    int *ovf;                  // list slots: entries placed through the cursors (see BinArgs)
    int2 *ctab;                // per (CTA, view): the CTA hash table, (slot, offset in the slot)
    unsigned *large_ids;       // record indices, capacity nviews * n
    DevStats *st;
};

// A list slot's range [offsets[k], offsets[k+1]) holds first the entries
// whose place the rasteriser's CTA tables fixed (counts[k] of them: CTA b's
// share starts at offsets[k] + its table's offset), then the entries placed
// one warp group at a time through cursor[k] = offsets[k] + counts[k]: those
// of keys that found no room in a CTA table, and the large list (ovf[k]).
struct BinArgs {
    const Rec *recs;
    const unsigned *large_ids;
    long long *cursor;         // list slots, starts at offsets + counts
    int *counts;
    int *ovf;
    const long long *offsets;
    const int2 *ctab;
    unsigned *entries;         // record indices
    int64_t entries_cap;
    DevStats *st;
};

struct TileArgs {
    const Rec *recs;
    const long long *offsets;  // list slots of all views, + 1 (64-bit list positions)
    const unsigned *entries;
    const WorkItem *items;
    int items_cap;
    float *const *images;      // device array: one image per view
    DevStats *st;
    const int *order;          // optional: processing order of each pass's items
    long long *item_cycles;    // optional: SM clock cycles spent on each item
    int accumulate;            // add into the images instead of storing (streamed chunks)
    const float2 *rec2;        // absorption mode: per record (A, depth key)
    float4 *partial;           // absorption mode: (C, T) per pixel of every split item
};

// Tile-cost network 32 -> 64 (ReLU) -> 1; parameter vector layout
// W1[64][32] row-major, b1[64], w2[64], b2.
constexpr int kFeat = 32, kHid = 64;
constexpr int kNParam = kHid * kFeat + 2 * kHid + 1;

// Launchers (stream-ordered, no synchronisation).  Every count the kernels
// need after binning (entries, work items) is read from device memory, so
// the whole sequence can be captured in a CUDA graph.
void launch_raster(const Views &v, const RasterArgs &a, int attr, cudaStream_t s);
void launch_count_large(const Views &v, const BinArgs &a, int sms, cudaStream_t s);
// Slot offsets and cursors from counts + ovf (ovf is overwritten with the sums).
void launch_slot_offsets(int m, int *counts, int *ovf, long long *offsets, long long *cursor,
                         long long *total, cudaStream_t s);

// Exclusive scan of in[0..m) into out[0..m] (out[m] = total); cursor (may be
// null) receives a copy of out[0..m); seg_totals[k] = total of the k-th of
// nseg equal segments.
void launch_scan(int m, const int *in, long long *out, long long *cursor, int nseg,
                 long long *seg_totals, cudaStream_t s);
void launch_scan(int m, const int *in, int *out, int *cursor, int nseg, int *seg_totals,
                 cudaStream_t s);
void launch_item_counts(const Views &v, const long long *offsets, int *item_counts, DevStats *st,
                        cudaStream_t s);
void launch_fill_items(const Views &v, const long long *offsets, const int *item_offsets,
                       WorkItem *items, int items_cap, DevStats *st, cudaStream_t s);
void launch_scatter(const Views &v, const BinArgs &a, int sms, cudaStream_t s);
void launch_tile_pass(const Views &v, const TileArgs &a, int sms, cudaStream_t s);
void launch_large_pass(const Views &v, const TileArgs &a, int sms, cudaStream_t s);
// Absorption mode: the depth-ordered pass and the composition of split tiles.
void launch_absorb_pass(const Views &v, const TileArgs &a, const int *item_offsets, int sms,
                        cudaStream_t s);
int radix_blocks(int64_t n);
int64_t radix_scratch_ints(int64_t n);
void launch_depth_order(const Rec *recs, const float2 *rec2, int64_t n, unsigned *entries,
                        const long long *off, int ntiles, long long total, unsigned long long *pkeys,
                        unsigned long long *ptmp, unsigned long long *ekeys,
                        unsigned long long *etmp, unsigned *rank, int *hist, int sms,
                        cudaStream_t s);
void launch_epilogue_ea(float *image, int64_t nvals, int sms, cudaStream_t s);
// FP32 attributes h, I, s into storage layout `store` (SPL_ATTR_* value).
void launch_encode_attrs(const float *h, const float *I, const float *s, int64_t n, int store,
                         float h_log2_min, void *ho, void *Io, void *so, int sms, cudaStream_t st);
// cursor[k] = offsets[k] + counts[k] for the m list slots (re-arms the scatter).
void launch_slot_cursor(int m, const int *counts, const long long *offsets, long long *cursor,
                        cudaStream_t s);
// Zero every view's image / apply the E=A map to every view's image (the
// image pointers are read from device memory, so a graph can replay them).
void launch_zero_images(const Views &v, float *const *images, int sms, cudaStream_t s);
void launch_epilogue_views(const Views &v, float *const *images, int sms, cudaStream_t s);
void launch_count_work(const FrameConst &fc, const Rec *recs, int64_t n,
                       unsigned long long *work, int sms, cudaStream_t s);

// Scheduling of the work items (spl_sched.cu): per-item features, predicted
// cost (network or count heuristic), and a longest-first order per pass.
void launch_item_entries(const Views &v, const TileArgs &a, int *n_entries, int sms,
                         cudaStream_t s);
void launch_item_features(const Views &v, const TileArgs &a, float area_scale, int max_sample,
                          float *feat, int *n_entries, int sms, cudaStream_t s);
void launch_item_cost(const float *feat, const int *n_entries, const float *theta,
                      const float *heur, int items_cap, const DevStats *st, float *cost,
                      cudaStream_t s);
void launch_order_items(const float *cost, int items_cap, DevStats *st, int *hist, int *order,
                        cudaStream_t s);

// Network kernels (spl_mlp.cu); B samples, features row-major [B][32].
void launch_mlp_forward(const float *theta, const float *x, int64_t B, float *y, cudaStream_t s);
void launch_mlp_loss_grad(const float *theta, const float *x, const float *t, int64_t B,
                          float *work, float *grad, float *loss, cudaStream_t s);
void launch_mlp_adam(float *theta, const float *grad, float *m, float *v, int64_t np, int64_t step,
                     float lr, float b1, float b2, float eps, cudaStream_t s);
size_t mlp_work_floats(int64_t B);
// logc[k] = log(cycles[k]) (cycles clamped to >= 1).
void launch_log_cycles(const long long *cycles, int64_t n, float *logc, cudaStream_t s);

// View of a global tile index (binary search over the views' tile bases).
__device__ __forceinline__ int view_of_tile(const FrameConst *fcs, int nviews, int g) {
    int lo = 0, hi = nviews - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fcs[mid].tile_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace spl
