// Lookup-only comparator (Section 4: texture mapping and The Lit Sphere map
// every target pixel through its own guide value, without chunks): each
// target pixel copies the style at the table entry of its own guide,
// C_T[p] = C_S[LUT(G_T[p])].  One thread per pixel; rows of 256 pixels per
// CTA, so guide reads and output stores are coalesced and the table and style
// gathers hit L2 (both are small and resident).
#include "sb_internal.cuh"

namespace sb {

constexpr int kLookupThreads = 256;

template <int C, int B>
__global__ void __launch_bounds__(kLookupThreads)
    lookup_kernel(const uint8_t *__restrict__ tgt, int64_t tgt_stride, int W,
                  const uint32_t *__restrict__ lut, int key_bits, int key_channels,
                  const uint32_t *__restrict__ style, int64_t style_stride_px,
                  uint32_t *__restrict__ out) {
    using F = GuideFmt<C, B>;
    const int x = blockIdx.x * kLookupThreads + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const uint32_t u =
        __ldg(lut + F::key(F::load(tgt, tgt_stride, x, y), key_bits, key_channels));
    out[(int64_t)y * W + x] = __ldg(style + (int64_t)(u >> 16) * style_stride_px + (u & 0xFFFFu));
}

struct LookupLaunch {
    const sb_guide *tgt;
    const sb_lut *lut;
    const sb_rgba8 *style;
    uint32_t *out;
    cudaStream_t s;
    template <int C, int B>
    void operator()() {
        const dim3 grid((tgt->width + kLookupThreads - 1) / kLookupThreads, tgt->height);
        lookup_kernel<C, B><<<grid, kLookupThreads, 0, s>>>(
            static_cast<const uint8_t *>(tgt->data), tgt->row_stride, tgt->width, lut->entries,
            lut->key_bits, lut->key_channels, reinterpret_cast<const uint32_t *>(style->data), style->row_stride / 4,
            out);
    }
};

}  // namespace sb

using namespace sb;

extern "C" sb_status sb_lookup_only(const sb_guide *tgt_guide, const sb_guide *src_guide,
                                    const sb_rgba8 *src_style, const sb_lut *lut,
                                    uint8_t *rgba8_out, sb_stream stream) {
    sb_status st = check_guide(tgt_guide, "tgt_guide", false);
    if (st != SB_OK) return st;
    if ((st = check_guide(src_guide, "src_guide", true)) != SB_OK) return st;
    if ((st = check_style(src_style, "src_style")) != SB_OK) return st;
    if (tgt_guide->channels != src_guide->channels || tgt_guide->bits != src_guide->bits)
        return fail(SB_ERR_INVALID_ARG, "target and source guides differ in channels or bits");
    if (!lut) return fail(SB_ERR_INVALID_ARG, "lut: NULL");
    if (lut->channels != src_guide->channels || lut->bits != src_guide->bits ||
        lut->src_w != src_guide->width || lut->src_h != src_guide->height)
        return fail(SB_ERR_INVALID_ARG, "lut was built for a different source guide format/size");
    if (src_style->width != src_guide->width || src_style->height != src_guide->height)
        return fail(SB_ERR_INVALID_ARG, "src_style and src_guide differ in size");
    if ((int64_t)tgt_guide->width * tgt_guide->height == 0) return ok();
    if (!rgba8_out || ((uintptr_t)rgba8_out % 4))
        return fail(SB_ERR_INVALID_ARG, "rgba8_out: NULL or not 4-byte aligned");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != lut->device) return fail(SB_ERR_INVALID_ARG, "lut lives on another device");
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    LookupLaunch L{tgt_guide, lut, src_style, reinterpret_cast<uint32_t *>(rgba8_out),
                   static_cast<cudaStream_t>(stream)};
    dispatch_format(tgt_guide->channels, tgt_guide->bits, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sb_lookup_only");
    return ok();
}
