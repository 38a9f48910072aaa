// spl_tile.cu -- the rendering passes (Sec. 4.1-4.3 and Eq. 2).
//
// One CTA owns one T x T tile of the image (the tiling of Eq. 8) and is the
// only writer of its pixels, so there are no races on the image and no global
// atomics (the problem of Sec. 3.2.2 / Fig. 3).  Inside the CTA:
//   - point particles (r <= r_sml, Sec. 4.1) add their emission to one pixel
//     of a shared-memory copy of the tile (shared-memory atomics);
//   - small particles (r_sml < r <= r_small): one thread per particle walks the
//     particle's pixel box inside the tile, also into shared memory;
//   - medium particles: one warp per particle; every warp keeps a private
//     copy of the whole tile in registers (lane = column), so a particle costs
//     one exp2 per lane for its column weight, one exp2 per row for the row
//     weight (staged in shared memory), and then 3 FMAs plus one compare per
//     covered pixel-slot: exp(-(dx^2+dy^2)/sigma^2) = w_x * w_y (Eq. 2 is
//     separable), and the clip test dx^2 <= r^2 - dy^2 keeps the disc exact;
//   - the warps' register tiles are then added into the shared tile one warp
//     at a time (a fixed order), and the tile is written once, coalesced.
// The large pass (r > r_large, Sec. 4.3) runs after the tile pass with the
// same warp-register scheme over the tiles that large particles reach, and
// adds its tile into the image (one CTA per tile, stream-ordered after the
// tile pass, so again no atomics).
#include "spl_geom.cuh"

namespace spl {

template <int T>
struct TileShape {
    static constexpr int RPL = T * T / 32;   // rows held by one lane
    static constexpr int GROUPS = 32 / T;    // lane groups (rows split between them)
    static constexpr int CHUNK = 4;          // rows per guarded chunk
    static constexpr int NCHUNK = RPL / CHUNK;
};

// One medium/large particle into a warp's register tile.
template <int T>
__device__ __forceinline__ void warp_splat(const FrameConst &fc, float4 r0, float4 r1, int x0,
                                           int y0, float4 *rowbuf, float *ar, float *ag, float *ab,
                                           int lane) {
    using S = TileShape<T>;
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    const float xh = 0.5f - r0.y, yh = 0.5f - r0.z;   // pixel-centre offsets
    const float kq = r0.w, r2 = r1.x;
    // column weight of this lane
    const int col = lane % T, grp = lane / T;
    const float dx = (float)(x0 + col - xi) + xh;
    const float dx2 = dx * dx;
    const float wx = ex2_neg(kq * dx2);
    // row weights: lane l < T computes row l of the tile
    __syncwarp();
    if (lane < T) {
        const float dy = (float)(y0 + lane - yi) + yh;
        const float dy2 = dy * dy;
        const float wy = ex2_neg(kq * dy2);
        rowbuf[lane] = make_float4(r1.y * wy, r1.z * wy, r1.w * wy, r2 - dy2);
    }
    __syncwarp();
    // rows the disc can reach (conservative; the exact test is dx2 <= rem)
    const float r = sqrtf(r2) + 1e-3f;
    const int jlo = yi - y0 + (int)ceilf(fmaxf(r0.z - 0.5f - r, -1e6f));
    const int jhi = yi - y0 + (int)floorf(fminf(r0.z - 0.5f + r, 1e6f));
    const int rbase = grp * S::RPL;
#pragma unroll
    for (int c = 0; c < S::NCHUNK; ++c) {
        const int ra = rbase + c * S::CHUNK;
        if (ra + S::CHUNK - 1 < jlo || ra > jhi) continue;
#pragma unroll
        for (int q = 0; q < S::CHUNK; ++q) {
            const int k = c * S::CHUNK + q;
            const float4 v = rowbuf[ra + q];
            if (dx2 <= v.w) {
                ar[k] = fmaf(v.x, wx, ar[k]);
                ag[k] = fmaf(v.y, wx, ag[k]);
                ab[k] = fmaf(v.z, wx, ab[k]);
            }
        }
    }
}

// One small particle (one thread) into the shared tile.
template <int T>
__device__ __forceinline__ void thread_splat(const FrameConst &fc, float4 r0, float4 r1, int x0,
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
        if (rem < 0.f) continue;
        const float wy = ex2_neg(kq * dy * dy);
        for (int i = i0; i <= i1; ++i) {
            const float dx = (float)(i - xi) + xh;
            const float dx2 = dx * dx;
            if (dx2 <= rem) {
                const float w = wy * ex2_neg(kq * dx2);
                atomicAdd(&sacc[0][j - y0][i - x0], r1.y * w);
                atomicAdd(&sacc[1][j - y0][i - x0], r1.z * w);
                atomicAdd(&sacc[2][j - y0][i - x0], r1.w * w);
            }
        }
    }
}

// LARGE = false: tile pass (points, small, medium; writes every tile).
// LARGE = true:  large pass (adds into tiles that have large entries).
template <int T, bool LARGE>
__global__ void __launch_bounds__(kTileThreads) tile_kernel(FrameConst fc, TileArgs a) {
    using S = TileShape<T>;
    __shared__ float sacc[3][T][T];
    __shared__ float4 rowbuf[kTileThreads / 32][T];
    const int tile = blockIdx.x;
    const int tx = tile % fc.ntx, ty = tile / fc.ntx;
    const int x0 = tx * fc.tile, y0 = ty * fc.tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int *off = a.offsets;
    const int nt = fc.ntiles;
    const int med_list = LARGE ? L_LARGE : L_MEDIUM;
    const int m0 = off[med_list * nt + tile], m1 = off[med_list * nt + tile + 1];
    if (LARGE && m0 == m1) return;

    for (int k = tid; k < 3 * T * T; k += kTileThreads) (&sacc[0][0][0])[k] = 0.f;
    __syncthreads();

    if (!LARGE) {
        // points (Sec. 4.1): one pixel each
        const int p0 = off[L_POINT * nt + tile], p1 = off[L_POINT * nt + tile + 1];
        for (int k = p0 + tid; k < p1; k += kTileThreads) {
            const unsigned id = a.entries[k];
            const float4 r0 = a.rec0[id];
            const float4 r1 = a.rec1[id];
            const int i = unpack_xi(r0.x) - x0, j = unpack_yi(r0.x) - y0;
            if ((unsigned)i < (unsigned)T && (unsigned)j < (unsigned)T) {
                atomicAdd(&sacc[0][j][i], r1.y);
                atomicAdd(&sacc[1][j][i], r1.z);
                atomicAdd(&sacc[2][j][i], r1.w);
            } else {
                atomicOr(&a.st->err, ERR_INDEX);
            }
        }
        // small particles: one thread each
        const int s0 = off[L_SMALL * nt + tile], s1 = off[L_SMALL * nt + tile + 1];
        for (int k = s0 + tid; k < s1; k += kTileThreads) {
            const unsigned id = a.entries[k];
            thread_splat<T>(fc, a.rec0[id], a.rec1[id], x0, y0, sacc);
        }
    }

    // medium (or large) particles: one warp each, private register tiles
    float ar[S::RPL], ag[S::RPL], ab[S::RPL];
#pragma unroll
    for (int k = 0; k < S::RPL; ++k) ar[k] = ag[k] = ab[k] = 0.f;
    const bool busy = m0 + warp < m1;
    for (int k = m0 + warp; k < m1; k += kTileThreads / 32) {
        const unsigned id = a.entries[k];
        warp_splat<T>(fc, a.rec0[id], a.rec1[id], x0, y0, rowbuf[warp], ar, ag, ab, lane);
    }
    // add the register tiles into the shared tile, one warp after another
    const int col = lane % T, rbase = (lane / T) * S::RPL;
    for (int w = 0; w < kTileThreads / 32; ++w) {
        __syncthreads();
        if (w == warp && busy) {
#pragma unroll
            for (int k = 0; k < S::RPL; ++k) {
                sacc[0][rbase + k][col] += ar[k];
                sacc[1][rbase + k][col] += ag[k];
                sacc[2][rbase + k][col] += ab[k];
            }
        }
    }
    __syncthreads();

    // write (tile pass) or add (large pass) the tile, row segments contiguous
    const int wv = min(T, fc.width - x0), hv = min(T, fc.height - y0);
    for (int q = tid; q < 3 * T * T; q += kTileThreads) {
        const int row = q / (3 * T), rem = q - row * 3 * T;
        const int c = rem % 3, colq = rem / 3;
        if (row >= hv || colq >= wv) continue;
        float *dst = a.image + 3 * ((int64_t)(y0 + row) * fc.width + x0 + colq) + c;
        const float v = sacc[c][row][colq];
        if (LARGE)
            *dst += v;
        else
            *dst = v;
    }
}

void launch_tile_pass(const FrameConst &fc, const TileArgs &a, cudaStream_t s) {
    if (fc.tile == 16)
        tile_kernel<16, false><<<fc.ntiles, kTileThreads, 0, s>>>(fc, a);
    else
        tile_kernel<32, false><<<fc.ntiles, kTileThreads, 0, s>>>(fc, a);
}

void launch_large_pass(const FrameConst &fc, const TileArgs &a, cudaStream_t s) {
    if (fc.tile == 16)
        tile_kernel<16, true><<<fc.ntiles, kTileThreads, 0, s>>>(fc, a);
    else
        tile_kernel<32, true><<<fc.ntiles, kTileThreads, 0, s>>>(fc, a);
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
}

}  // namespace spl
