// Lookup-only comparator (Section 4: texture mapping and The Lit Sphere map
// every target pixel through its own guide value, without chunks): each
// target pixel copies the style at the table entry of its own guide,
// C_T[p] = C_S[LUT(G_T[p])].  Four neighbouring pixels per thread, 1024 per
// CTA along a row, so guide reads and output stores are coalesced vectors and
// the table and style gathers (small, L2-resident) overlap.
#include "sb_internal.cuh"

namespace sb {

constexpr int kLookupThreads = 256;
constexpr int kLookupPx = 4;  // pixels per thread (one vector load of guide, one store)

// The packed guide values of pixels x .. x+3 of a row whose start is aligned to
// the vector width (x a multiple of 4): one to three aligned loads.
template <int C, int B>
__device__ __forceinline__ void load4(const uint8_t *row, int x, uint32_t (&p)[4]) {
    if constexpr (B == 8 && C == 1) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(row + x));
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = (w >> (8 * k)) & 0xFFu;
    } else if constexpr ((B == 8 && C == 2) || (B == 16 && C == 1)) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(row + 8 * (x / 4)));
        p[0] = w.x & 0xFFFFu;
        p[1] = w.x >> 16;
        p[2] = w.y & 0xFFFFu;
        p[3] = w.y >> 16;
    } else if constexpr (B == 8 && C == 3) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(row + 3 * x);
        const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
        p[0] = w0 & 0xFFFFFFu;
        p[1] = __funnelshift_r(w0, w1, 24) & 0xFFFFFFu;
        p[2] = __funnelshift_r(w1, w2, 16) & 0xFFFFFFu;
        p[3] = w2 >> 8;
    } else {  // 16 bytes: 8-bit x 4 or 16-bit x 2
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(row + 16 * (x / 4)));
        p[0] = w.x;
        p[1] = w.y;
        p[2] = w.z;
        p[3] = w.w;
    }
}

// Alignment (bytes) of the guide rows that load4 needs.
__host__ inline int lookup_vec_align(int channels, int bits) {
    const int bytes4 = 4 * channels * bits / 8;  // four pixels
    return bytes4 == 12 ? 4 : bytes4;
}

// Four pixels per thread.  With vec (guide rows aligned for load4, output
// rows 16-byte aligned, W a multiple of 4) a thread reads its four guide
// values with one to three vector loads and writes one 16-byte store; the
// four table and style gathers of a thread are independent, so they overlap.
template <int C, int B>
__global__ void __launch_bounds__(kLookupThreads)
    lookup_kernel(const uint8_t *__restrict__ tgt, int64_t tgt_stride, int W,
                  const uint32_t *__restrict__ lut, int key_bits, int key_channels,
                  const uint32_t *__restrict__ style, int64_t style_stride_px,
                  uint32_t *__restrict__ out, bool vec) {
    using F = GuideFmt<C, B>;
    const int x = (blockIdx.x * kLookupThreads + threadIdx.x) * kLookupPx;
    const int y = blockIdx.y;
    if (x >= W) return;
    const uint8_t *row = tgt + (int64_t)y * tgt_stride;
    uint32_t *orow = out + (int64_t)y * W;
    uint32_t g[kLookupPx];
    const int n = min(kLookupPx, W - x);
    if (vec) {
        load4<C, B>(row, x, g);
    } else {
#pragma unroll
        for (int k = 0; k < kLookupPx; ++k) g[k] = k < n ? F::load(row, 0, x + k, 0) : 0u;
    }
    uint32_t u[kLookupPx], c[kLookupPx];
#pragma unroll
    for (int k = 0; k < kLookupPx; ++k)
        u[k] = k < n ? __ldg(lut + F::key(g[k], key_bits, key_channels)) : 0u;
#pragma unroll
    for (int k = 0; k < kLookupPx; ++k)
        c[k] = k < n ? __ldg(style + (int64_t)(u[k] >> 16) * style_stride_px + (u[k] & 0xFFFFu))
                     : 0u;
    if (vec) {
        *reinterpret_cast<uint4 *>(orow + x) = make_uint4(c[0], c[1], c[2], c[3]);
    } else {
#pragma unroll
        for (int k = 0; k < kLookupPx; ++k)
            if (k < n) orow[x + k] = c[k];
    }
}

struct LookupLaunch {
    const sb_guide *tgt;
    const sb_lut *lut;
    const sb_rgba8 *style;
    uint32_t *out;
    cudaStream_t s;
    template <int C, int B>
    void operator()() {
        const int al = lookup_vec_align(C, B);
        const bool vec = tgt->width % 4 == 0 && (uintptr_t)tgt->data % al == 0 &&
                         tgt->row_stride % al == 0 && (uintptr_t)out % 16 == 0;
        constexpr int kPxPerBlock = kLookupThreads * kLookupPx;
        const dim3 grid((tgt->width + kPxPerBlock - 1) / kPxPerBlock, tgt->height);
        lookup_kernel<C, B><<<grid, kLookupThreads, 0, s>>>(
            static_cast<const uint8_t *>(tgt->data), tgt->row_stride, tgt->width, lut->entries,
            lut->key_bits, lut->key_channels, reinterpret_cast<const uint32_t *>(style->data),
            style->row_stride / 4, out, vec);
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
