// spl_absorb.cu -- the general absorption pass (Eq. 1 with E_p != A_p):
// front-to-back compositing over depth-sorted tile lists, and the composition
// of the partials of split tiles.
#include "spl_tile.cuh"

namespace spl {

// ---------------------------------------------------------------------------
// General absorption (Eq. 1 with E_p != A_p).  Across particle p a ray's
// intensity becomes I exp(-tau) + S (1 - exp(-tau)) with tau = A_p w_p and the
// source term S = E_p / A_p; for the particles of a pixel taken front to back
// this is the same as keeping the transmittance T of the particles in front
// and adding T S (1 - exp(-tau)), then T *= exp(-tau) (the ray starts with
// zero intensity behind the last particle).  Every tile's list holds all its
// particles (points included) sorted front to back by (depth, index); a work
// item runs its range in that order with (T, C) per pixel in registers.  A
// tile that is one item stores C; the segments of a crowded tile store their
// (C, T) partials, and absorb_combine_kernel composes them in segment order:
// C = C_1 + T_1 C_2 + T_1 T_2 C_3 ..., which is the same recurrence.
// ---------------------------------------------------------------------------

// Tables of one batch: swx[p][c] = (w_x, dx^2 B) as in the additive pass (for a
// point: 1 in its column, 0 elsewhere, and no clip); srow[p][j] = (A w_y,
// (r^2 - dy^2) B + 1) (a point: A in its row, 2 for the clip), or, where a
// lane's rows go two at a time, per row pair (A w_a, A w_b, clip_a, clip_b);
// ssrc[2p], ssrc[2p + 1] = (E / A) per channel, each value twice (0 when
// A = 0).  Thread (p, q) fills columns and rows (row pairs) q, q + 8, ... of
// particle p and tests row band q.
template <int T>
__device__ __forceinline__ void absorb_tabulate(const FrameConst &fc, const float4 *st0,
                                                const float4 *st1, const float2 *st2, int cnt,
                                                int x0, int y0, float2 (*swx)[Shape<T>::WXS],
                                                float2 (*srow)[Shape<T>::WXS], float4 *ssrc,
                                                unsigned *band_mask, int tid) {
    using S = Shape<T>;
    const int p = tid >> 3, q = tid & 7;
    // every lane runs to the end (band bits by ballot); entries of p >= cnt are
    // written but never read
    const bool valid = p < cnt;
    const float4 r0 = st0[valid ? p : 0], r1 = st1[valid ? p : 0];
    const float A = st2[valid ? p : 0].x, r2 = r1.x;
    const bool point = r2 <= fc.r_sml2;
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    if (q == 0) {
        // E / A per channel, each twice: the operand pairs of the packed FMAs
        const float inv = A > 0.f ? 1.f / A : 0.f;
        const float e0 = r1.y * inv, e1 = r1.z * inv, e2 = r1.w * inv;
        ssrc[2 * p] = make_float4(e0, e0, e1, e1);
        ssrc[2 * p + 1] = make_float4(e2, e2, 0.f, 0.f);
    }
    // row table: per row (A w_y, clip term), or per row pair (A w_a, A w_b,
    // clip_a, clip_b) when rows go two at a time
    float4 *srow4 = reinterpret_cast<float4 *>(&srow[0][0]);
    int ilo, ihi, jlo, jhi;
    float r = 0.f, xh = 0.f, yh = 0.f;
    if (point) {
        ilo = ihi = xi - x0;
        jlo = jhi = yi - y0;
#pragma unroll
        for (int u = 0; u < S::PER; ++u) {
            const int k = q + 8 * u;
            swx[p][k] = make_float2(x0 + k == xi ? 1.f : 0.f, 0.f);
            if constexpr (!S::PAIRED) srow[p][k] = make_float2(y0 + k == yi ? A : 0.f, 2.f);
        }
        if constexpr (S::PAIRED) {
#pragma unroll
            for (int u = 0; u < S::PER / 2; ++u) {
                const int m = q + 8 * u;
                srow4[p * (T / 2) + m] = make_float4(y0 + 2 * m == yi ? A : 0.f,
                                                     y0 + 2 * m + 1 == yi ? A : 0.f, 2.f, 2.f);
            }
        }
    } else {
        const float kq = r0.w, B = __fdividef(1048576.f, r2);
        xh = 0.5f - r0.y;
        yh = 0.5f - r0.z;
        r = r2 * rsqrtf(r2) + 1e-3f;   // approximate: far inside the margin
        ilo = xi - x0 + (int)ceilf(fmaxf(r0.y - 0.5f - r, -1e6f));
        ihi = xi - x0 + (int)floorf(fminf(r0.y - 0.5f + r, 1e6f));
        jlo = yi - y0 + (int)ceilf(fmaxf(r0.z - 0.5f - r, -1e6f));
        jhi = yi - y0 + (int)floorf(fminf(r0.z - 0.5f + r, 1e6f));
#pragma unroll
        for (int u = 0; u < S::PER; ++u) {
            const int k = q + 8 * u;
            const float dx = (float)(x0 + k - xi) + xh;
            const float dx2 = dx * dx;
            swx[p][k] = make_float2(ex2_neg(kq * dx2), dx2 * B);
            if constexpr (!S::PAIRED) {
                const float dy = (float)(y0 + k - yi) + yh;
                const float dy2 = dy * dy;
                srow[p][k] = make_float2(A * ex2_neg(kq * dy2), fmaf(r2 - dy2, B, 1.f));
            }
        }
        if constexpr (S::PAIRED) {
#pragma unroll
            for (int u = 0; u < S::PER / 2; ++u) {
                const int m = q + 8 * u;
                const float dya = (float)(y0 + 2 * m - yi) + yh, dyb = dya + 1.f;
                const float a2 = dya * dya, b2 = dyb * dyb;
                srow4[p * (T / 2) + m] =
                    make_float4(A * ex2_neg(kq * a2), A * ex2_neg(kq * b2), fmaf(r2 - a2, B, 1.f),
                                fmaf(r2 - b2, B, 1.f));
            }
        }
    }
    // band q: box overlap, and for a disc its reach to the band's nearest pixel
    // centre (as in the additive pass); a warp's four particles by one ballot
    const int bx0 = (q % S::NBX) * S::BW, by0 = (q / S::NBX) * S::BH;
    const int bx1 = bx0 + S::BW - 1, by1 = by0 + S::BH - 1;
    bool hit = valid && jhi >= by0 && jlo <= by1 && ihi >= bx0 && ilo <= bx1;
    if (!point) {
        const float ax = (float)(x0 + bx0 - xi) + xh, ay = (float)(y0 + by0 - yi) + yh;
        const float nx = fmaxf(ax, fminf(0.f, ax + (float)(S::BW - 1)));
        const float ny = fmaxf(ay, fminf(0.f, ay + (float)(S::BH - 1)));
        hit = hit && nx * nx + ny * ny <= r * r;
    }
    const unsigned hb = __ballot_sync(0xffffffffu, hit);
    const int lane = tid & 31;
    if (lane < 8) {
        const unsigned nib = ((hb >> lane) & 1u) | (((hb >> (lane + 8)) & 1u) << 1) |
                             (((hb >> (lane + 16)) & 1u) << 2) | (((hb >> (lane + 24)) & 1u) << 3);
        if (nib) atomicOr(&band_mask[lane], nib << (4 * (tid >> 5)));
    }
}

// 1 - exp(-tau) for tau >= 0 with small relative error everywhere: below
// 1/16 the Taylor series to tau^5 (truncation < tau^5/720 relative, < 2e-9),
// above it one minus the hardware exp2 (relative error there < 16 * 2^-22).
// Computing 1 - exp(-tau) directly would lose all digits of a small tau.
__device__ __forceinline__ float one_minus_exp_neg(float tau) {
    const float series =
        tau * fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, 1.f / 120.f, -1.f / 24.f), 1.f / 6.f), -0.5f), 1.f);
    return tau < 0.0625f ? series : 1.f - ex2_neg(1.4426950408889634f * tau);
}

// The same for two values at once: the series and one minus the hardware exp2
// as packed FP32x2 operations (each half rounded as the scalar instruction, so
// the results equal one_minus_exp_neg's bit for bit).
__device__ __forceinline__ f32x2 one_minus_exp_neg2(f32x2 tau) {
    const f32x2 c5 = pack2(1.f / 120.f, 1.f / 120.f), c4 = pack2(-1.f / 24.f, -1.f / 24.f);
    const f32x2 c3 = pack2(1.f / 6.f, 1.f / 6.f), c2 = pack2(-0.5f, -0.5f);
    const f32x2 one = pack2(1.f, 1.f), mone = pack2(-1.f, -1.f);
    const f32x2 nl2e = pack2(-1.4426950408889634f, -1.4426950408889634f);
    f32x2 sr = fma2v(tau, c5, c4);
    sr = fma2v(tau, sr, c3);
    sr = fma2v(tau, sr, c2);
    sr = fma2v(tau, sr, one);
    sr = mul2(tau, sr);
    float u0, u1, e0, e1;
    unpack2(mul2(tau, nl2e), u0, u1);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(u0));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(u1));
    const f32x2 ge = fma2v(pack2(e0, e1), mone, one);
    float t0, t1, s0, s1, g0, g1;
    unpack2(tau, t0, t1);
    unpack2(sr, s0, s1);
    unpack2(ge, g0, g1);
    return pack2(t0 < 0.0625f ? s0 : g0, t1 < 0.0625f ? s1 : g1);
}

template <int T>
__host__ __device__ constexpr size_t absorb_smem_bytes() {
    using S = Shape<T>;
    return (sizeof(float2) * 2 * S::WXS + 2 * sizeof(float4)) * S::P +   // swx, srow, ssrc
           (2 * sizeof(float4) + sizeof(float2)) * S::P;              // staged records
}

// CTAs per SM.  The pass is latency-bound (each pixel's transmittance is a
// chain across its list), so occupancy pays: at T = 32, 2 -> 4 -> 6 CTAs per
// SM (106 -> 62 -> 40 registers, 8 bytes spilled at 40) took the clustered
// 10M / 1024^2 pass from 15.2 to 11.3 to 10.7 ms.  At T = 64 a lane's 16
// pixels need the registers of 2 CTAs per SM; at T = 16, 5 fit without spills.
template <int T>
constexpr int absorb_ctas() { return T == 64 ? 2 : (T == 32 ? 6 : 5); }

template <int T>
__global__ void __launch_bounds__(kTileThreads, absorb_ctas<T>()) absorb_kernel(Views vs, TileArgs a) {
    using S = Shape<T>;
    extern __shared__ float4 smem_raw[];
    float2 (*swx)[S::WXS] = reinterpret_cast<float2 (*)[S::WXS]>(smem_raw);
    float2 (*srow)[S::WXS] = swx + S::P;
    float4 *ssrc = reinterpret_cast<float4 *>(srow + S::P);   // two per particle
    float4 *st0 = ssrc + 2 * S::P;
    float4 *st1 = st0 + S::P;
    float2 *st2 = reinterpret_cast<float2 *>(st1 + S::P);
    __shared__ unsigned band_mask[kTileThreads / 32];
    __shared__ int s_item;
    __shared__ FrameConst sfc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_items = min(a.st->item_totals[0], a.items_cap);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(&a.st->item_counter[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int idx = a.order ? a.order[it] : it;
        const WorkItem w = a.items[idx];
        const int view = item_view(w), list = item_list(w);
        {
            const int words = (int)(sizeof(FrameConst) / sizeof(int));
            if (tid < words)
                reinterpret_cast<int *>(&sfc)[tid] = reinterpret_cast<const int *>(vs.fcs + view)[tid];
        }
        __syncthreads();
        const FrameConst &fc = sfc;
        const int tile = w.tile - fc.tile_base;
        const int x0 = (tile % fc.ntx) * T, y0 = (tile / fc.ntx) * T;
        long long lb = w.start, le = w.end;
        if (list < 0) {
            lb = a.offsets[fc.slot_base + L_MEDIUM * fc.ntiles + tile];
            le = a.offsets[fc.slot_base + L_MEDIUM * fc.ntiles + tile + 1];
        }
        const int col = (warp % S::NBX) * S::BW + (lane % S::LW) * S::CMUL;
        const int row0 = (warp / S::NBX) * S::BH + (lane / S::LW) * S::RPL;
        // (T, C) per pixel in registers: scalar, or two rows per FP32x2 pair
        constexpr int RP = S::PAIRED ? S::RPL / 2 : 1;
        float Tr[S::RPL][S::CPL], C[S::RPL][S::CPL][3];
        f32x2 Tr2[RP][S::CPL], C2[RP][S::CPL][3];
        if constexpr (S::PAIRED) {
#pragma unroll
            for (int m = 0; m < RP; ++m)
#pragma unroll
                for (int k = 0; k < S::CPL; ++k) {
                    Tr2[m][k] = pack2(1.f, 1.f);
                    C2[m][k][0] = C2[m][k][1] = C2[m][k][2] = 0ull;
                }
        } else {
#pragma unroll
            for (int q = 0; q < S::RPL; ++q)
#pragma unroll
                for (int k = 0; k < S::CPL; ++k) {
                    Tr[q][k] = 1.f;
                    C[q][k][0] = C[q][k][1] = C[q][k][2] = 0.f;
                }
        }
#pragma unroll 1
        for (long long base = lb; base < le; base += S::P) {
            const int cnt = (int)(le - base < S::P ? le - base : S::P);
            if (tid < cnt) {
                const unsigned id = a.entries[base + tid];
                const Rec rc = a.recs[id];
                st0[tid] = rc.r0;
                st1[tid] = rc.r1;
                st2[tid] = a.rec2[id];
            }
            if (tid < kTileThreads / 32) band_mask[tid] = 0u;
            __syncthreads();
            absorb_tabulate<T>(fc, st0, st1, st2, cnt, x0, y0, swx, srow, ssrc, band_mask, tid);
            __syncthreads();
            // this warp's band, particles front to back (increasing list position)
            unsigned mask = band_mask[warp];
            while (mask) {
                const int p = __ffs(mask) - 1;
                mask &= mask - 1u;
                float wx[S::CPL], dxb[S::CPL];
                if constexpr (S::CSTEP == 1 && S::CPL == 2) {
                    // two adjacent columns in one 16-byte load (col is even)
                    const float4 v = *reinterpret_cast<const float4 *>(&swx[p][col]);
                    wx[0] = v.x; dxb[0] = v.y; wx[1] = v.z; dxb[1] = v.w;
                } else {
#pragma unroll
                    for (int k = 0; k < S::CPL; ++k) {
                        const float2 v = swx[p][col + S::CSTEP * k];
                        wx[k] = v.x;
                        dxb[k] = v.y;
                    }
                }
                if constexpr (S::PAIRED) {
                    // per row pair: (A w_a, A w_b) and the two clip terms; E / A
                    // per channel as duplicated pairs
                    const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(ssrc) + 2 * p;
                    const ulonglong2 s01 = sv[0], s2x = sv[1];
                    const ulonglong2 *rp =
                        reinterpret_cast<const ulonglong2 *>(&srow[0][0]) + p * (T / 2) + row0 / 2;
#pragma unroll
                    for (int m = 0; m < RP; ++m) {
                        const ulonglong2 rv = rp[m];
                        float ca, cb;
                        unpack2(rv.y, ca, cb);
#pragma unroll
                        for (int k = 0; k < S::CPL; ++k) {
                            const f32x2 clip =
                                pack2(__saturatef(ca - dxb[k]), __saturatef(cb - dxb[k]));
                            const f32x2 tau = mul2(mul2(pack2(wx[k], wx[k]), clip), rv.x);
                            const f32x2 f = mul2(Tr2[m][k], one_minus_exp_neg2(tau));
                            fma2(C2[m][k][0], f, s01.x);
                            fma2(C2[m][k][1], f, s01.y);
                            fma2(C2[m][k][2], f, s2x.x);
                            Tr2[m][k] = fma2v(f, pack2(-1.f, -1.f), Tr2[m][k]);
                        }
                    }
                } else {
                    const float4 src = ssrc[2 * p];
                    const float src2 = ssrc[2 * p + 1].x;
#pragma unroll
                    for (int q = 0; q < S::RPL; ++q) {
                        const float2 rv = srow[p][row0 + q];
#pragma unroll
                        for (int k = 0; k < S::CPL; ++k) {
                            const float tau = wx[k] * __saturatef(rv.y - dxb[k]) * rv.x;
                            const float g = one_minus_exp_neg(tau);
                            const float f = Tr[q][k] * g;                 // T (1 - e^-tau)
                            C[q][k][0] = fmaf(f, src.x, C[q][k][0]);
                            C[q][k][1] = fmaf(f, src.z, C[q][k][1]);
                            C[q][k][2] = fmaf(f, src2, C[q][k][2]);
                            Tr[q][k] -= f;                                // T e^-tau
                        }
                    }
                }
            }
            __syncthreads();
        }
        float *image = a.images[view];
#pragma unroll
        for (int q = 0; q < S::RPL; ++q) {
            const int row = row0 + q;
#pragma unroll
            for (int k = 0; k < S::CPL; ++k) {
                float c0, c1, c2, tr;
                if constexpr (S::PAIRED) {
                    float lo, hi;
                    unpack2(C2[q >> 1][k][0], lo, hi); c0 = (q & 1) ? hi : lo;
                    unpack2(C2[q >> 1][k][1], lo, hi); c1 = (q & 1) ? hi : lo;
                    unpack2(C2[q >> 1][k][2], lo, hi); c2 = (q & 1) ? hi : lo;
                    unpack2(Tr2[q >> 1][k], lo, hi); tr = (q & 1) ? hi : lo;
                } else {
                    c0 = C[q][k][0]; c1 = C[q][k][1]; c2 = C[q][k][2]; tr = Tr[q][k];
                }
                const int cx = col + S::CSTEP * k;
                if (y0 + row >= fc.height || x0 + cx >= fc.width) continue;
                if (list < 0) {
                    float *dst = image + 3 * ((int64_t)(y0 + row) * fc.width + x0 + cx);
                    dst[0] = c0;
                    dst[1] = c1;
                    dst[2] = c2;
                } else {
                    a.partial[(size_t)idx * (T * T) + row * T + cx] = make_float4(c0, c1, c2, tr);
                }
            }
        }
    }
}

// Tiles cut into several items: compose the items' partials in list order.
template <int T>
__global__ void __launch_bounds__(256) absorb_combine_kernel(Views vs, const int *item_offsets,
                                                             const float4 *partial,
                                                             float *const *images) {
    for (int g = blockIdx.x; g < vs.total_tiles; g += gridDim.x) {
        const int i0 = item_offsets[g], i1 = item_offsets[g + 1];
        if (i1 - i0 < 2) continue;
        const int view = view_of_tile(vs.fcs, vs.nviews, g);
        const FrameConst &fc = vs.fcs[view];
        const int tile = g - fc.tile_base;
        const int x0 = (tile % fc.ntx) * T, y0 = (tile / fc.ntx) * T;
        for (int px = threadIdx.x; px < T * T; px += blockDim.x) {
            const int row = px / T, cx = px % T;
            if (y0 + row >= fc.height || x0 + cx >= fc.width) continue;
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, tr = 1.f;
            for (int it = i0; it < i1; ++it) {
                const float4 v = partial[(size_t)it * (T * T) + px];
                c0 = fmaf(tr, v.x, c0);
                c1 = fmaf(tr, v.y, c1);
                c2 = fmaf(tr, v.z, c2);
                tr *= v.w;
            }
            float *dst = images[view] + 3 * ((int64_t)(y0 + row) * fc.width + x0 + cx);
            dst[0] = c0;
            dst[1] = c1;
            dst[2] = c2;
        }
    }
}

template <int T>
static void launch_absorb_t(const Views &vs, const TileArgs &a, const int *item_offsets, int sms,
                            cudaStream_t s) {
    constexpr size_t bytes = absorb_smem_bytes<T>();
    absorb_kernel<T><<<sms * absorb_ctas<T>(), kTileThreads, bytes, s>>>(vs, a);
    ++g_launches;
    const int grid = vs.total_tiles < sms * 8 ? vs.total_tiles : sms * 8;
    if (grid > 0) {
        absorb_combine_kernel<T><<<grid, 256, 0, s>>>(vs, item_offsets, a.partial, a.images);
        ++g_launches;
    }
}

void launch_absorb_pass(const Views &vs, const TileArgs &a, const int *item_offsets, int sms,
                        cudaStream_t s) {
    if (vs.tile == 16)
        launch_absorb_t<16>(vs, a, item_offsets, sms, s);
    else if (vs.tile == 64)
        launch_absorb_t<64>(vs, a, item_offsets, sms, s);
    else
        launch_absorb_t<32>(vs, a, item_offsets, sms, s);
}

}  // namespace spl
