// spl_geom.cuh -- device helpers shared by the rasteriser, the binning kernels
// and the tile passes: record decoding and the tile footprint of a particle.
#pragma once

#include "spl_internal.cuh"

namespace spl {

__device__ __forceinline__ int unpack_xi(float packed) {
    return (int)(short)(__float_as_uint(packed) & 0xFFFFu);
}
__device__ __forceinline__ int unpack_yi(float packed) {
    return ((int)__float_as_uint(packed)) >> 16;
}
__device__ __forceinline__ float pack_xy(int xi, int yi) {
    return __uint_as_float(((unsigned)xi & 0xFFFFu) | ((unsigned)yi << 16));
}

// Class of a record from its squared radius (r2 < 0: inactive).
__device__ __forceinline__ int record_class(const FrameConst &fc, float r2) {
    if (r2 < 0.f) return CLS_INACTIVE;
    if (r2 <= fc.r_sml2) return CLS_POINT;
    if (r2 <= fc.r_small2) return CLS_SMALL;
    if (r2 <= fc.r_large2) return CLS_MEDIUM;
    return CLS_LARGE;
}

// Pixel-centre bounding box of a splat, cut to the image: the pixels i with
// |i + 1/2 - x_s| <= r (plus a margin of 1e-3 px + 1e-6 r, so that rounding
// never drops a pixel that the exact clip test would keep).  Returns false
// when no pixel centre can be inside.
struct PixBox { int i0, i1, j0, j1; };

__device__ __forceinline__ bool splat_box(const FrameConst &fc, float4 r0, float r2, PixBox &b) {
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    const float r = sqrtf(r2);
    const float m = r + 1e-3f + 1e-6f * r;
    // x_s - 1/2 relative to xi: xf - 1/2
    const float lo_x = (r0.y - 0.5f) - m, hi_x = (r0.y - 0.5f) + m;
    const float lo_y = (r0.z - 0.5f) - m, hi_y = (r0.z - 0.5f) + m;
    // clamp in float before converting, so huge radii cannot overflow int
    const float lim = 70000.f;
    int i0 = xi + (int)ceilf(fmaxf(lo_x, -lim)), i1 = xi + (int)floorf(fminf(hi_x, lim));
    int j0 = yi + (int)ceilf(fmaxf(lo_y, -lim)), j1 = yi + (int)floorf(fminf(hi_y, lim));
    b.i0 = max(i0, 0); b.i1 = min(i1, fc.width - 1);
    b.j0 = max(j0, 0); b.j1 = min(j1, fc.height - 1);
    return b.i0 <= b.i1 && b.j0 <= b.j1;
}

// Squared reach of a disc in the tile tests: the radius with the margin of
// splat_box.
__device__ __forceinline__ float disc_reach2(float r2) {
    const float r = sqrtf(r2);
    const float m = r + 1e-3f + 1e-6f * r;
    return m * m;
}

// Does the disc (reach2 = disc_reach2(r^2)) reach any pixel centre of tile
// (tx, ty)?
__device__ __forceinline__ bool disc_meets_tile(const FrameConst &fc, float4 r0, float reach2, int tx,
                                                int ty) {
    const int xi = unpack_xi(r0.x), yi = unpack_yi(r0.x);
    // tile pixel-centre rectangle, relative to (xi, yi)
    const float ax = (float)(tx * fc.tile - xi) + 0.5f;
    const float bx = (float)(min((tx + 1) * fc.tile, fc.width) - 1 - xi) + 0.5f;
    const float ay = (float)(ty * fc.tile - yi) + 0.5f;
    const float by = (float)(min((ty + 1) * fc.tile, fc.height) - 1 - yi) + 0.5f;
    const float dx = fminf(fmaxf(r0.y, ax), bx) - r0.y;
    const float dy = fminf(fmaxf(r0.z, ay), by) - r0.z;
    return dx * dx + dy * dy <= reach2;
}

// exp(-d2/sigma^2) = 2^(-kq d2) with the hardware exp2 (PTX ex2.approx.ftz.f32,
// maximum relative error about 2^-22 over the range used here).
__device__ __forceinline__ float ex2_neg(float kq_d2) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-kq_d2));
    return y;
}

}  // namespace spl
