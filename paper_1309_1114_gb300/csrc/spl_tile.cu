// spl_tile.cu -- the rendering passes (Sec. 4.1-4.3 and Eq. 2).
//
// Work is cut into items: a T x T tile of the image (the tiling of Eq. 8)
// together with its lists, or -- for a crowded tile, the load imbalance of
// the Remarks of Sec. 4 -- a bounded segment of one of its lists.  Persistent
// CTAs take items from a device counter.  A tile that is one item is written
// by exactly one CTA with plain stores; the segments of a crowded tile add
// their partial tiles into the (zeroed) image with one atomic add per pixel
// and channel, instead of one per contribution (the write races of
// Sec. 3.2.2 / Fig. 3).
//
// Inside an item every pixel of the tile has one owner thread: warp w owns a
// band of the tile (16 x 8 pixels for T = 32, 16 x 2 for T = 16, 64 x 8 for
// T = 64), each lane a few pixels of it (T = 32: two adjacent columns of one
// row pair; T = 16: one pixel; T = 64: two columns 32 apart, eight rows), and
// the thread keeps its pixels' three channels in registers.  Then:
//   - point particles (r <= r_sml, Sec. 4.1) add their emission to one pixel
//     of a shared-memory copy of the tile; lanes of a warp that hit the same
//     pixel are summed with warp shuffles first;
//   - small particles (r_sml < r <= r_small, a few pixels wide): one thread
//     per particle walks the particle's pixel box, into shared memory;
//   - medium and large particles are taken in batches (the chunks of n_p
//     particles of Sec. 4.2): the CTA first tabulates, per particle, the
//     column weights w_x(i) = exp(-dx^2/sigma^2) and the row terms
//     e * w_y(j) (Eq. 2 is separable: exp(-(dx^2+dy^2)/sigma^2) = w_x w_y),
//     then every warp whose row band the particle reaches adds
//     e * w_y * w_x into its registers: three FMAs per pixel, plus a clip
//     test folded into one saturating add on the FMA pipe (see below);
//     where a lane holds an even number of rows, two rows go through one
//     packed FP32x2 instruction (the row table is laid out in row pairs);
//   - finally each thread adds the shared-memory part to its registers and
//     writes its pixels once.
// The large pass (r > r_large, Sec. 4.3) runs after the tile pass with the
// same scheme over segments of the tiles' large lists and adds its partial
// tiles into the image.
//
// Clip (Eq. 2: zero beyond chi*sigma).  With B = 2^20 / r^2 the tables hold
// dx^2 * B per column and (r^2 - dy^2) * B + 1 per row; the clip factor is
// m = saturate((r^2 - dy^2) B + 1 - dx^2 B), which is exactly 1 inside the
// disc and exactly 0 outside it, except for pixels whose distance lies within
// r * (1 + 5e-7) -- inside the band where FP32 and FP64 may legitimately
// disagree on an inclusive clip test anyway.
#include "spl_tile.cuh"

namespace spl {

// The registers of one thread's pixels: RPL rows x CPL columns x RGB, held
// as row pairs when the rows are processed two at a time.
template <int T, bool PAIRED = Shape<T>::PAIRED>
struct Acc {
    using S = Shape<T>;
    float v[S::RPL][S::CPL][3];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < S::RPL; ++q)
#pragma unroll
            for (int k = 0; k < S::CPL; ++k) v[q][k][0] = v[q][k][1] = v[q][k][2] = 0.f;
    }
    __device__ __forceinline__ float get(int q, int k, int c) const { return v[q][k][c]; }
};
template <int T>
struct Acc<T, true> {
    using S = Shape<T>;
    f32x2 v[S::RPL / 2][S::CPL][3];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < S::RPL / 2; ++q)
#pragma unroll
            for (int k = 0; k < S::CPL; ++k) v[q][k][0] = v[q][k][1] = v[q][k][2] = 0ull;
    }
    __device__ __forceinline__ float get(int q, int k, int c) const {
        float lo, hi;
        unpack2(v[q >> 1][k][c], lo, hi);
        return (q & 1) ? hi : lo;
    }
};

// One small particle (a few pixels wide) into the shared tile, by one thread:
// the pixel box inside the tile, the clip test and the weight of Eq. 2 per
// pixel, and one shared-memory add per channel.  A tiny splat costs a few
// pixels of work here instead of a batch-table share and a band visit.
template <int T>
__device__ __forceinline__ void thread_small(const FrameConst &fc, float4 r0, float4 r1, int x0,
                                             int y0, float (*sacc)[T][T]) {
    PixBox b;
    if (!splat_box(fc, r0, r1.x, b)) return;
    const int i0 = max(b.i0, x0), i1 = min(b.i1, x0 + T - 1);
    const int j0 = max(b.j0, y0), j1 = min(b.j1, y0 + T - 1);
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    const float xh = 0.5f - r0.y, yh = 0.5f - r0.z;
    const float kq = r0.w, r2 = r1.x;
    for (int j = j0; j <= j1; ++j) {
        const float dy = (float)(j - yi) + yh;
        const float rem = r2 - dy * dy;
        for (int i = i0; i <= i1; ++i) {
            const float dx = (float)(i - xi) + xh;
            const float dx2 = dx * dx;
            if (dx2 <= rem) {
                const float w = ex2_neg(kq * (dx2 + dy * dy));
                atomicAdd(&sacc[0][j - y0][i - x0], r1.y * w);
                atomicAdd(&sacc[1][j - y0][i - x0], r1.z * w);
                atomicAdd(&sacc[2][j - y0][i - x0], r1.w * w);
            }
        }
    }
}

// Points of one warp's 32 staged records: lanes that hit the same pixel are
// summed inside the warp first (match + shuffles), then one lane adds.
template <int T>
__device__ __forceinline__ void warp_points(const TileArgs &a, const float4 *s0, const float4 *s1,
                                            int cnt, int x0, int y0, float (*sacc)[T][T], int lane) {
    int key = -1;
    float er = 0.f, eg = 0.f, eb = 0.f;
    int i = 0, j = 0;
    if (lane < cnt) {
        const float4 r0 = s0[lane];
        const float4 r1 = s1[lane];
        i = unpack_xi(r0.x) - x0;
        j = unpack_yi(r0.x) - y0;
        if ((unsigned)i < (unsigned)T && (unsigned)j < (unsigned)T) {
            key = j * T + i;
            er = r1.y; eg = r1.z; eb = r1.w;
        } else {
            atomicOr(&a.st->err, ERR_INDEX);
        }
    }
    const unsigned m = __match_any_sync(0xffffffffu, key);
    if (__any_sync(0xffffffffu, key >= 0 && __popc(m) > 1)) {
        float sr = 0.f, sg = 0.f, sb = 0.f;
        for (int q = 0; q < 32; ++q) {
            const float vr = __shfl_sync(0xffffffffu, er, q);
            const float vg = __shfl_sync(0xffffffffu, eg, q);
            const float vb = __shfl_sync(0xffffffffu, eb, q);
            if ((m >> q) & 1u) { sr += vr; sg += vg; sb += vb; }
        }
        er = sr; eg = sg; eb = sb;
    }
    if (key >= 0 && lane == __ffs(m) - 1) {
        atomicAdd(&sacc[0][j][i], er);
        atomicAdd(&sacc[1][j][i], eg);
        atomicAdd(&sacc[2][j][i], eb);
    }
}

// Tabulate the separable factors of a batch of cnt <= 32 staged particles:
// swx[p][c] = (w_x, dx^2 B) for tile column c; for tile row j the row terms
// e_R w_y, e_G w_y, e_B w_y and (r^2 - dy^2) B + 1.  Rows are stored one
// float4 per row, or -- when the rows go two at a time -- per row pair
// (2m, 2m+1) in two tables, srow[p][m] = (e_R w_y, same for row 2m+1, e_G w_y,
// e_G w_y') in the first half of the row space and (e_B w_y, e_B w_y', rem,
// rem') in the second, so that every packed operand is one aligned half of a
// 16-byte load and the eight threads of a particle store consecutive entries.  Thread (p, q) = (tid / 8,
// tid % 8) fills columns q, q + 8, q + 16, ... (and the same rows, or row
// pairs q, q + 8, ...) of particle p.  It also decides for row band q whether
// the disc reaches it (bit p of band_mask[q]).  B only needs to be the same
// on both sides of the clip test, so a fast reciprocal serves.
template <int T>
__device__ __forceinline__ void tabulate(const float4 *st0, const float4 *st1, int cnt, int x0,
                                         int y0, float2 (*swx)[Shape<T>::WXS], float4 (*srow)[T],
                                         unsigned *band_mask, int tid) {
    using S = Shape<T>;
    const int p = tid >> 3, q = tid & 7;
    // every lane runs to the end (the band bits are combined by a ballot); the
    // entries of particles p >= cnt are written but never read (no band bit)
    const bool valid = p < cnt;
    const float4 r0 = st0[valid ? p : 0], r1 = st1[valid ? p : 0];
    const float kq = r0.w, r2 = r1.x;
    const float B = __fdividef(1048576.f, r2);
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    const float xh = 0.5f - r0.y, yh = 0.5f - r0.z;
    // the disc's radius for the band test (conservative by 1e-3 px)
    const float r = r2 * rsqrtf(r2) + 1e-3f;   // approximate: far inside the margin
    // offsets of this thread's first column and row from the particle centre;
    // the others follow by adding small integers (exact in FP32)
    const float dxq = ((float)(x0 - xi) + xh) + (float)q;
#pragma unroll
    for (int u = 0; u < S::PER; ++u) {
        const int k = q + 8 * u;
        const float dx = dxq + (float)(8 * u);
        const float dx2 = dx * dx;
        swx[p][k] = make_float2(ex2_neg(kq * dx2), dx2 * B);
    }
    if constexpr (S::PAIRED) {
        const float dyq = ((float)(y0 - yi) + yh) + (float)(2 * q);
#pragma unroll
        for (int u = 0; u < S::PER / 2; ++u) {
            const int m = q + 8 * u;
            const float dya = dyq + (float)(16 * u), dyb = dya + 1.f;
            const float a2 = dya * dya, b2 = dyb * dyb;
            const float wa = ex2_neg(kq * a2), wb = ex2_neg(kq * b2);
            float4 *rowA = reinterpret_cast<float4 *>(srow), *rowB = rowA + S::P * (T / 2);
            rowA[p * (T / 2) + m] = make_float4(r1.y * wa, r1.y * wb, r1.z * wa, r1.z * wb);
            rowB[p * (T / 2) + m] =
                make_float4(r1.w * wa, r1.w * wb, fmaf(r2 - a2, B, 1.f), fmaf(r2 - b2, B, 1.f));
        }
    } else {
#pragma unroll
        for (int u = 0; u < S::PER; ++u) {
            const int k = q + 8 * u;
            const float dy = (float)(y0 + k - yi) + yh;
            const float dy2 = dy * dy;
            const float wy = ex2_neg(kq * dy2);
            srow[p][k] = make_float4(r1.y * wy, r1.z * wy, r1.w * wy, fmaf(r2 - dy2, B, 1.f));
        }
    }
    // row band q: columns [bx BW, bx BW + BW), rows [by BH, by BH + BH); the
    // disc (with a margin) must reach the rectangle of the band's pixel
    // centres.  A superset of the bands that hold a covered pixel: a band
    // visited in vain adds clipped zeros.
    const int bx0 = (q % S::NBX) * S::BW, by0 = (q / S::NBX) * S::BH;
    const float ax = (float)(x0 + bx0 - xi) + xh, ay = (float)(y0 + by0 - yi) + yh;
    const float nx = fmaxf(ax, fminf(0.f, ax + (float)(S::BW - 1)));
    const float ny = fmaxf(ay, fminf(0.f, ay + (float)(S::BH - 1)));
    const bool hit = valid && nx * nx + ny * ny <= r * r;
    // lane 8j + q holds particle 4w + j of warp w and band q: lane q < 8 gathers
    // its band's four bits and sets them with one atomic
    const unsigned hb = __ballot_sync(0xffffffffu, hit);
    const int lane = tid & 31;
    if (lane < 8) {
        const unsigned nib = ((hb >> lane) & 1u) | (((hb >> (lane + 8)) & 1u) << 1) |
                             (((hb >> (lane + 16)) & 1u) << 2) | (((hb >> (lane + 24)) & 1u) << 3);
        if (nib) atomicOr(&band_mask[lane], nib << (4 * (tid >> 5)));
    }
}

// Add tabulated particle p into the registers of this thread's pixels.  The
// clip factor is exactly 1 inside the disc and 0 outside (see the top).
template <int T>
__device__ __forceinline__ void band_splat(const float2 *wxp, const float4 *rowp, int col, int row0,
                                           Acc<T, false> &acc) {
    using S = Shape<T>;
    float wx[S::CPL], dxb[S::CPL];
#pragma unroll
    for (int k = 0; k < S::CPL; ++k) {
        const float2 v = wxp[col + S::CSTEP * k];
        wx[k] = v.x;
        dxb[k] = v.y;
    }
#pragma unroll
    for (int q = 0; q < S::RPL; ++q) {
        const float4 rv = rowp[row0 + q];
#pragma unroll
        for (int k = 0; k < S::CPL; ++k) {
            const float wk = wx[k] * __saturatef(rv.w - dxb[k]);
            acc.v[q][k][0] = fmaf(rv.x, wk, acc.v[q][k][0]);
            acc.v[q][k][1] = fmaf(rv.y, wk, acc.v[q][k][1]);
            acc.v[q][k][2] = fmaf(rv.z, wk, acc.v[q][k][2]);
        }
    }
}

// The same two rows at a time: per row pair two 16-byte loads, and per
// column two scalar clips, one packed multiply and three packed FMAs (R, G, B
// of both rows).
// rowp points at the particle's first-half row-pair table (see tabulate).
template <int T>
__device__ __forceinline__ void band_splat(const float2 *wxp, const float4 *rowp, int col, int row0,
                                           Acc<T, true> &acc) {
    using S = Shape<T>;
    float dxb[S::CPL];
    f32x2 ww[S::CPL];
    if constexpr (S::CSTEP == 1 && S::CPL == 2) {
        // two adjacent columns in one 16-byte load (col is even, rows of the
        // column table are 16-byte aligned)
        const float4 v = *reinterpret_cast<const float4 *>(wxp + col);
        ww[0] = pack2(v.x, v.x);
        dxb[0] = v.y;
        ww[1] = pack2(v.z, v.z);
        dxb[1] = v.w;
    } else {
#pragma unroll
        for (int k = 0; k < S::CPL; ++k) {
            const float2 v = wxp[col + S::CSTEP * k];
            ww[k] = pack2(v.x, v.x);
            dxb[k] = v.y;
        }
    }
    const ulonglong2 *ra_ = reinterpret_cast<const ulonglong2 *>(rowp) + row0 / 2;
    const ulonglong2 *rb_ = ra_ + S::P * (T / 2);
#pragma unroll
    for (int m = 0; m < S::RPL / 2; ++m) {
        const ulonglong2 a = ra_[m], b = rb_[m];
        float ra, rb;
        unpack2(b.y, ra, rb);
#pragma unroll
        for (int k = 0; k < S::CPL; ++k) {
            const f32x2 w = mul2(pack2(__saturatef(ra - dxb[k]), __saturatef(rb - dxb[k])), ww[k]);
            fma2(acc.v[m][k][0], a.x, w);
            fma2(acc.v[m][k][1], a.y, w);
            fma2(acc.v[m][k][2], b.x, w);
        }
    }
}

// Dynamic shared memory of one CTA (bytes): the batch tables srow and swx,
// then the staged records st0, st1.  The shared tile sacc of the point and
// small passes (3 T^2 floats) reuses the table space: those passes run after
// the medium list, when the tables are no longer read.
template <int T>
__host__ __device__ constexpr size_t table_bytes() {
    using S = Shape<T>;
    return sizeof(float4) * S::P * T + sizeof(float2) * S::P * S::WXS;
}
static_assert(Shape<32>::WXS * sizeof(float2) % 16 == 0, "16-byte column-table rows");
static_assert(table_bytes<16>() >= sizeof(float) * 3 * 16 * 16, "shared tile fits the tables");
static_assert(table_bytes<32>() >= sizeof(float) * 3 * 32 * 32, "shared tile fits the tables");
static_assert(table_bytes<64>() >= sizeof(float) * 3 * 64 * 64, "shared tile fits the tables");
template <int T>
__host__ __device__ constexpr size_t smem_bytes() { return table_bytes<T>() + sizeof(float4) * 2 * kTileThreads; }

template <int T>
constexpr int min_ctas() { return T >= 64 ? 2 : (T == 32 ? 5 : 4); }

// Persistent pass over the work items of every view of the batch: the tile
// pass takes items [0, item_totals[0]), the large pass the next
// item_totals[1] (both counts read from device memory).
template <int T, bool LARGE>
__global__ void __launch_bounds__(kTileThreads, min_ctas<T>()) item_kernel(Views vs, TileArgs a) {
    using S = Shape<T>;
    constexpr int NW = kTileThreads / 32;
    extern __shared__ float4 smem_raw[];
    float4 (*srow)[T] = reinterpret_cast<float4 (*)[T]>(smem_raw);
    float2 (*swx)[S::WXS] = reinterpret_cast<float2 (*)[S::WXS]>(smem_raw + S::P * T);
    float (*sacc)[T][T] = reinterpret_cast<float (*)[T][T]>(smem_raw);   // after the tables
    float4 *st0 = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem_raw) + table_bytes<T>());
    float4 *st1 = st0 + kTileThreads;
    __shared__ unsigned band_mask[2][NW];
    __shared__ int s_item;
    __shared__ FrameConst sfc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int *counter = &a.st->item_counter[LARGE ? 1 : 0];
    const int item0 = LARGE ? a.st->item_totals[0] : 0;
    const int n_items = min(a.st->item_totals[LARGE ? 1 : 0], a.items_cap - item0);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int idx = item0 + (a.order ? a.order[item0 + it] : it);
        const WorkItem w = a.items[idx];
        const int view = item_view(w), list = item_list(w);
        const long long t_start = clock64();
        {
            const int words = (int)(sizeof(FrameConst) / sizeof(int));
            if (tid < words)
                reinterpret_cast<int *>(&sfc)[tid] = reinterpret_cast<const int *>(vs.fcs + view)[tid];
        }
        __syncthreads();
        const FrameConst &fc = sfc;
        const int tile = w.tile - fc.tile_base;
        const int x0 = (tile % fc.ntx) * T, y0 = (tile / fc.ntx) * T;
        const int nt = fc.ntiles, sb = fc.slot_base;
        long long lb0 = 0, le0 = 0, lb1 = 0, le1 = 0, lb2 = 0, le2 = 0;
        if (list < 0) {
            lb0 = a.offsets[sb + L_POINT * nt + tile]; le0 = a.offsets[sb + L_POINT * nt + tile + 1];
            lb1 = a.offsets[sb + L_SMALL * nt + tile]; le1 = a.offsets[sb + L_SMALL * nt + tile + 1];
            lb2 = a.offsets[sb + L_MEDIUM * nt + tile]; le2 = a.offsets[sb + L_MEDIUM * nt + tile + 1];
        } else if (list == L_POINT) {
            lb0 = w.start; le0 = w.end;
        } else if (list == L_SMALL) {
            lb1 = w.start; le1 = w.end;
        } else {
            lb2 = w.start; le2 = w.end;      // medium (tile pass) or large (large pass)
        }
        const int col = (warp % S::NBX) * S::BW + (lane % S::LW) * S::CMUL;
        const int row0 = (warp / S::NBX) * S::BH + (lane / S::LW) * S::RPL;
        Acc<T> acc;
        acc.zero();

        // medium (or large) particles: tabulate a batch, then every row band
        // adds it.  Records are staged in two alternating buffers (with two
        // band-mask sets): the next batch is stored while the bands of this one
        // are added, and the batch after it is fetched into registers.
        float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
        if (lb2 < le2) {
            if (lb2 + tid < le2 && tid < S::P) {
                const unsigned id = a.entries[lb2 + tid];
                const Rec rc = a.recs[id];
                st0[tid] = rc.r0;
                st1[tid] = rc.r1;
            }
            if (tid < NW) band_mask[0][tid] = 0u;
            if (lb2 + S::P + tid < le2 && tid < S::P) {
                const unsigned id = a.entries[lb2 + S::P + tid];
                const Rec rc = a.recs[id];
                n0 = rc.r0;
                n1 = rc.r1;
            }
            __syncthreads();
        }
        int buf = 0;
#pragma unroll 1
        for (long long base = lb2; base < le2; base += S::P) {
            const int cnt = (int)(le2 - base < S::P ? le2 - base : S::P);
            tabulate<T>(st0 + buf * S::P, st1 + buf * S::P, cnt, x0, y0, swx, srow, band_mask[buf],
                        tid);
            __syncthreads();
            // stage the next batch (its buffer and masks were last used a batch ago)
            if (tid < S::P) {
                if (base + S::P + tid < le2) {
                    st0[(buf ^ 1) * S::P + tid] = n0;
                    st1[(buf ^ 1) * S::P + tid] = n1;
                }
                if (base + 2 * S::P + tid < le2) {
                    const unsigned id = a.entries[base + 2 * S::P + tid];
                    const Rec rc = a.recs[id];
                    n0 = rc.r0;
                    n1 = rc.r1;
                }
            }
            if (tid < NW) band_mask[buf ^ 1][tid] = 0u;
            // this warp's row band: only the particles that reach it
            unsigned mask = band_mask[buf][warp];
            while (mask) {
                const int p = __ffs(mask) - 1;
                mask &= mask - 1u;
                band_splat<T>(swx[p], S::PAIRED ? srow[0] + p * (T / 2) : srow[p], col, row0, acc);
            }
            __syncthreads();
            buf ^= 1;
        }

        // points and small particles go through the shared tile, which reuses
        // the table space (the tables are dead once every warp is past here)
        const bool shared_tile = le0 > lb0 || le1 > lb1;
        if (shared_tile) {
            __syncthreads();
            for (int k = tid; k < 3 * T * T; k += kTileThreads) (&sacc[0][0][0])[k] = 0.f;
            __syncthreads();
        }
        // points (Sec. 4.1): batches of 256 staged records, warp-aggregated
#pragma unroll 1
        for (long long base = lb0; base < le0; base += kTileThreads) {
            const int cnt = (int)(le0 - base < kTileThreads ? le0 - base : kTileThreads);
            if (tid < cnt) {
                const unsigned id = a.entries[base + tid];
                const Rec rc = a.recs[id];
                st0[tid] = rc.r0;
                st1[tid] = rc.r1;
            }
            __syncthreads();
            warp_points<T>(a, st0 + warp * 32, st1 + warp * 32, cnt - warp * 32, x0, y0, sacc, lane);
            __syncthreads();
        }
        // small particles: one thread each over its pixel box (no staging)
#pragma unroll 1
        for (long long k = lb1 + tid; k < le1; k += kTileThreads) {
            const unsigned id = a.entries[k];
            const Rec rc = a.recs[id];
            thread_small<T>(fc, rc.r0, rc.r1, x0, y0, sacc);
        }
        if (le1 > lb1) __syncthreads();
        // write: shared part + registers, stored (only item of its tile; added
        // to the previous chunks' sum when accumulating) or added atomically
        const bool store = !LARGE && list < 0;
        float *image = a.images[view];
#pragma unroll
        for (int q = 0; q < S::RPL; ++q) {
            const int row = row0 + q;
#pragma unroll
            for (int k = 0; k < S::CPL; ++k) {
                const int cx = col + S::CSTEP * k;
                if (y0 + row >= fc.height || x0 + cx >= fc.width) continue;
                float *dst = image + 3 * ((int64_t)(y0 + row) * fc.width + x0 + cx);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float v = (shared_tile ? sacc[c][row][cx] : 0.f) + acc.get(q, k, c);
                    if (store)
                        dst[c] = a.accumulate ? dst[c] + v : v;
                    else if (v != 0.f)
                        atomicAdd(dst + c, v);
                }
            }
        }
        if (a.item_cycles) {
            __syncthreads();
            if (tid == 0) a.item_cycles[idx] = clock64() - t_start;
        }
    }
}

template <int T, bool LARGE>
static void launch_items_t(const Views &vs, const TileArgs &a, int sms, cudaStream_t s) {
    constexpr size_t bytes = smem_bytes<T>();
    cudaFuncSetAttribute(item_kernel<T, LARGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
    item_kernel<T, LARGE><<<sms * min_ctas<T>(), kTileThreads, bytes, s>>>(vs, a);
    ++g_launches;
}

template <bool LARGE>
static void launch_items(const Views &vs, const TileArgs &a, int sms, cudaStream_t s) {
    if (vs.tile == 16)
        launch_items_t<16, LARGE>(vs, a, sms, s);
    else if (vs.tile == 64)
        launch_items_t<64, LARGE>(vs, a, sms, s);
    else
        launch_items_t<32, LARGE>(vs, a, sms, s);
}

void launch_tile_pass(const Views &vs, const TileArgs &a, int sms, cudaStream_t s) {
    launch_items<false>(vs, a, sms, s);
}

void launch_large_pass(const Views &vs, const TileArgs &a, int sms, cudaStream_t s) {
    launch_items<true>(vs, a, sms, s);
}

// E_p = A_p solution of Eq. 1 applied to the additive sum: I = 1 - exp(-S).
__global__ void epilogue_ea_kernel(float *img, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        img[i] = -expm1f(-img[i]);
}

void launch_epilogue_ea(float *image, int64_t nvals, int sms, cudaStream_t s) {
    if (nvals <= 0) return;
    int64_t blocks = (nvals + 255) / 256;
    blocks = blocks < (int64_t)sms * 4 ? blocks : (int64_t)sms * 4;
    epilogue_ea_kernel<<<(unsigned)blocks, 256, 0, s>>>(image, nvals);
    ++g_launches;
}

// Grid-stride over every pixel value of every view (blockIdx.y = view).
template <bool EA>
__global__ void views_pointwise_kernel(Views vs, float *const *images) {
    const int v = blockIdx.y;
    const FrameConst &fc = vs.fcs[v];
    float *img = images[v];
    const int64_t n = (int64_t)3 * fc.width * fc.height;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        img[i] = EA ? -expm1f(-img[i]) : 0.f;
}

void launch_zero_images(const Views &vs, float *const *images, int sms, cudaStream_t s) {
    views_pointwise_kernel<false><<<dim3(sms * 2, vs.nviews), 256, 0, s>>>(vs, images);
    ++g_launches;
}

void launch_epilogue_views(const Views &vs, float *const *images, int sms, cudaStream_t s) {
    views_pointwise_kernel<true><<<dim3(sms * 2, vs.nviews), 256, 0, s>>>(vs, images);
    ++g_launches;
}

}  // namespace spl
