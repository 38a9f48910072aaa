// spl_attrs.cu -- storage layouts of the per-particle attributes h, I, s.
//
// The memory-access model of Sec. 3.2 charges every particle its bytes once
// per frame; the smaller layouts store the same particles in fewer bytes.  The
// encoder converts FP32 attributes into any layout the rasteriser reads:
//   SPL_ATTR_F32      h, I, s FP32 (a copy)
//   SPL_ATTR_F16      h, I, s IEEE binary16, round to nearest even
//   SPL_ATTR_F16_IS   h FP32; I, s binary16
//   SPL_ATTR_LOGH16   I, s binary16; h as the 16-bit code
//                     k = round_half_even(4096 (log2 h - h_log2_min)) clamped to
//                     [0, 65535], formed in FP64 so that the code is the
//                     correctly rounded one except within ~1e-16 of a half
//                     step; the rasteriser decodes h = 2^(h_log2_min + k/4096).
// A smoothing length that no code can stand for (negative, NaN or infinite --
// a particle the FP32 layout renders inactive) keeps the particle inactive in
// the coded layout too: its I is stored as a binary16 NaN.
#include "spl_internal.cuh"

namespace spl {

__global__ void encode_attrs_kernel(const float *h, const float *I, const float *s, int64_t n,
                                    int store, float h_log2_min, void *ho, void *Io, void *so) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float hv = h[i], iv = I[i], sv = s[i];
        if (store == 0) {
            static_cast<float *>(ho)[i] = hv;
            static_cast<float *>(Io)[i] = iv;
            static_cast<float *>(so)[i] = sv;
            continue;
        }
        static_cast<__half *>(so)[i] = __float2half_rn(sv);
        if (store == 1) {
            static_cast<__half *>(ho)[i] = __float2half_rn(hv);
            static_cast<__half *>(Io)[i] = __float2half_rn(iv);
        } else if (store == 2) {
            static_cast<float *>(ho)[i] = hv;
            static_cast<__half *>(Io)[i] = __float2half_rn(iv);
        } else {
            const bool codable = isfinite(hv) && hv >= 0.f;
            unsigned short k = 0;
            if (codable && hv > 0.f) {
                const double t = rint((log2((double)hv) - (double)h_log2_min) * 4096.0);
                k = (unsigned short)(t < 0.0 ? 0.0 : (t > 65535.0 ? 65535.0 : t));
            }
            static_cast<unsigned short *>(ho)[i] = k;
            static_cast<__half *>(Io)[i] = codable ? __float2half_rn(iv) : __ushort_as_half(0x7E00);
        }
    }
}

void launch_encode_attrs(const float *h, const float *I, const float *s, int64_t n, int store,
                         float h_log2_min, void *ho, void *Io, void *so, int sms, cudaStream_t st) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
    encode_attrs_kernel<<<(unsigned)blocks, 256, 0, st>>>(h, I, s, n, store, h_log2_min, ho, Io, so);
    ++g_launches;
}

}  // namespace spl
