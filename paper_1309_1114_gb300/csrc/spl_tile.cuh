// spl_tile.cuh -- the band geometry of a tile CTA and the packed FP32x2
// helpers shared by the additive passes (spl_tile.cu) and the general
// absorption pass (spl_absorb.cu).
#pragma once
#include "spl_geom.cuh"

namespace spl {

template <int T>
struct Shape {
    // A tile is cut into 8 row bands, one per warp: BW columns x BH rows.
    static constexpr int BW = T == 64 ? 64 : 16;
    static constexpr int BH = T * T / (8 * BW);
    static constexpr int NBX = T / BW;             // bands across the tile
    // lanes along a band row: 8 for T = 32, so that a lane's two columns
    // share each row-pair load and the column table is read 16 bytes at a time
    static constexpr int LW = T == 32 ? 8 : (BW < 32 ? BW : 32);
    // a lane's columns: col + CSTEP k, k < CPL, col = band column + CMUL * (lane % LW)
    static constexpr int CSTEP = T == 32 ? 1 : 32;
    static constexpr int CMUL = T == 32 ? 2 : 1;
    static constexpr int G = 32 / LW;              // lane groups (rows split between them)
    static constexpr int CPL = BW / LW;            // columns per lane
    static constexpr int RPL = BH / G;             // rows per lane
    static constexpr int P = 32;                   // particles per tabulated batch
    static constexpr int PER = T / 8;              // table columns (and rows) per thread
    static constexpr bool PAIRED = RPL % 2 == 0;   // rows two at a time (FP32x2)
    // row stride of the column table: 8 entries of padding put the two
    // particles that a half-warp's 64-bit stores reach in different banks
    static constexpr int WXS = T + 8;
};

// Two FP32 values in one 64-bit register pair: the operand of the packed
// FP32x2 multiply and FMA (each half rounded as the scalar instruction).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ void fma2(f32x2 &acc, f32x2 a, f32x2 b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ f32x2 fma2v(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace spl
