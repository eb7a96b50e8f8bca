// Lookup-only comparator (Section 4: texture mapping and The Lit Sphere map
// every target pixel through its own guide value, without chunks): each
// target pixel copies the style at the table entry of its own guide,
// C_T[p] = C_S[LUT(G_T[p])].  Four or eight neighbouring pixels per thread
// along a row, so guide reads and output stores are coalesced vectors and the
// table and style gathers (small, L2-resident) overlap.  sb_lookup_only_batch
// maps many frames in one launch.
#include <climits>
#include <cstdio>
#include <string>

#include "sb_internal.cuh"

namespace sb {

constexpr int kLookupThreads = 256;

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

// One frame of the lookup: its target guide, table, style and output.
struct LookupFrame {
    const uint8_t *tgt;
    int64_t tgt_stride;
    const uint32_t *lut;
    const uint32_t *style;
    uint32_t *out;
    int W, H, key_bits, key_channels, style_stride_px;
    int vec;  // guide rows aligned for load4, output 16-byte aligned, W % 4 == 0
};

// Q quads of four pixels per thread, pixels [x, x + 4Q) of row y with x = (bx *
// 256 + thread) * 4Q.  With vec a thread reads each quad's guide values with
// one to three vector loads and writes one 16-byte store per quad; all guide
// loads are issued first, then the table and style gathers of every pixel,
// which are independent, so they overlap.  Two quads per thread keep more bytes
// in flight on wide rows; rows narrower than 2048 pixels use one (a second quad
// would leave most of a row's only block idle).
template <int C, int B, int Q>
__device__ __forceinline__ void lookup_chunk(const LookupFrame &f, int bx, int y) {
    using F = GuideFmt<C, B>;
    constexpr int P = 4 * Q;
    const int x = (bx * kLookupThreads + (int)threadIdx.x) * P;
    if (x >= f.W) return;
    const uint8_t *row = f.tgt + (int64_t)y * f.tgt_stride;
    uint32_t *orow = f.out + (int64_t)y * f.W;
    const int n = min(P, f.W - x);
    uint32_t g[Q][4];
    if (f.vec) {
        // W % 4 == 0: every quad is whole or absent
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (4 * q < n) {
                load4<C, B>(row, x + 4 * q, g[q]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) g[q][k] = 0u;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < P; ++k) g[k / 4][k % 4] = k < n ? F::load(row, 0, x + k, 0) : 0u;
    }
    uint32_t u[P], c[P];
#pragma unroll
    for (int k = 0; k < P; ++k)
        u[k] = k < n ? __ldg(f.lut + F::key(g[k / 4][k % 4], f.key_bits, f.key_channels)) : 0u;
#pragma unroll
    for (int k = 0; k < P; ++k)
        c[k] = k < n ? __ldg(f.style + (int64_t)(u[k] >> 16) * f.style_stride_px +
                             (u[k] & 0xFFFFu))
                     : 0u;
    if (f.vec) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (4 * q < n)
                *reinterpret_cast<uint4 *>(orow + x + 4 * q) =
                    make_uint4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < P; ++k)
            if (k < n) orow[x + k] = c[k];
    }
}

template <int C, int B, int Q>
__global__ void __launch_bounds__(kLookupThreads) lookup_kernel(const LookupFrame f) {
    lookup_chunk<C, B, Q>(f, blockIdx.x, blockIdx.y);
}

// Quads per thread for rows of width w, and pixels per block.
__host__ inline int lookup_quads(int w) { return w >= 2048 ? 2 : 1; }
__host__ inline int lookup_px_per_block(int quads) { return kLookupThreads * 4 * quads; }

// Many frames in one launch: block (t, k) maps row chunk t of frame k (the
// grid is as wide as the largest frame's chunk count; blocks past a smaller
// frame's end return at once).  Small frames then fill the GPU together
// instead of one short launch each, and no block searches for its frame.
constexpr int kMaxLookupBatch = 128;
struct LookupBatch {
    int n;
    int blocks[kMaxLookupBatch];    // row chunks of frame k (0 without pixels)
    int blocks_x[kMaxLookupBatch];  // chunks per row
    LookupFrame f[kMaxLookupBatch];
};

template <int C, int B, int Q>
__global__ void __launch_bounds__(kLookupThreads)
    lookup_batch_kernel(const __grid_constant__ LookupBatch b) {
    const int k = blockIdx.y, t = blockIdx.x;
    if (t >= b.blocks[k]) return;
    lookup_chunk<C, B, Q>(b.f[k], t % b.blocks_x[k], t / b.blocks_x[k]);
}

// The launch descriptor of one frame (guide format C, B).
template <int C, int B>
LookupFrame lookup_frame(const sb_guide *tgt, const sb_lut *lut, const sb_rgba8 *style,
                         uint32_t *out) {
    const int al = lookup_vec_align(C, B);
    LookupFrame f;
    f.tgt = static_cast<const uint8_t *>(tgt->data);
    f.tgt_stride = tgt->row_stride;
    f.lut = lut->entries;
    f.style = reinterpret_cast<const uint32_t *>(style->data);
    f.out = out;
    f.W = tgt->width;
    f.H = tgt->height;
    f.key_bits = lut->key_bits;
    f.key_channels = lut->key_channels;
    f.style_stride_px = (int)(style->row_stride / 4);
    f.vec = tgt->width % 4 == 0 && (uintptr_t)tgt->data % al == 0 && tgt->row_stride % al == 0 &&
            (uintptr_t)out % 16 == 0;
    return f;
}

struct LookupLaunch {
    const sb_guide *tgt;
    const sb_lut *lut;
    const sb_rgba8 *style;
    uint32_t *out;
    cudaStream_t s;
    template <int C, int B>
    void operator()() {
        const int q = lookup_quads(tgt->width), px = lookup_px_per_block(q);
        const dim3 grid((tgt->width + px - 1) / px, tgt->height);
        const LookupFrame f = lookup_frame<C, B>(tgt, lut, style, out);
        if (q == 2) lookup_kernel<C, B, 2><<<grid, kLookupThreads, 0, s>>>(f);
        else lookup_kernel<C, B, 1><<<grid, kLookupThreads, 0, s>>>(f);
    }
};

struct LookupBatchLaunch {
    const sb_frame *frames;
    LookupBatch *b;
    int quads;
    cudaStream_t s;
    template <int C, int B>
    void operator()() {
        for (int k = 0; k < b->n; ++k)
            b->f[k] = lookup_frame<C, B>(&frames[k].tgt_guide, frames[k].lut,
                                         &frames[k].src_style,
                                         reinterpret_cast<uint32_t *>(frames[k].rgba8_out));
        int width = 0;
        for (int k = 0; k < b->n; ++k) width = max(width, b->blocks[k]);
        if (width == 0) return;
        if (quads == 2) lookup_batch_kernel<C, B, 2><<<dim3(width, b->n), kLookupThreads, 0, s>>>(*b);
        else lookup_batch_kernel<C, B, 1><<<dim3(width, b->n), kLookupThreads, 0, s>>>(*b);
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
    if (!lut->entries)
        return fail(SB_ERR_UNSUPPORTED, "sb_lookup_only needs a table (keys of at most 24 bits)");
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

extern "C" sb_status sb_lookup_only_batch(const sb_frame *frames, int32_t n_frames,
                                          sb_stream stream) {
    if (n_frames < 0 || n_frames > kMaxLookupBatch)
        return fail(SB_ERR_INVALID_ARG, "n_frames must be in [0, 128]");
    if (n_frames == 0) return ok();
    if (!frames) return fail(SB_ERR_INVALID_ARG, "frames: NULL");
    static thread_local LookupBatch b;  // ~9 KB: kept off the stack
    const int channels = frames[0].tgt_guide.channels, bits = frames[0].tgt_guide.bits;
    char name[64];
    b.n = n_frames;
    // two quads per thread only when every frame's rows are wide enough
    int quads = 2;
    for (int k = 0; k < n_frames; ++k)
        if ((int64_t)frames[k].tgt_guide.width * frames[k].tgt_guide.height > 0)
            quads = min(quads, lookup_quads(frames[k].tgt_guide.width));
    const int px_per_block = lookup_px_per_block(quads);
    for (int k = 0; k < n_frames; ++k) {
        const sb_frame &f = frames[k];
        std::snprintf(name, sizeof name, "frames[%d].tgt_guide", k);
        sb_status st = check_guide(&f.tgt_guide, name, false);
        if (st != SB_OK) return st;
        if (f.tgt_guide.channels != channels || f.tgt_guide.bits != bits)
            return fail(SB_ERR_UNSUPPORTED,
                        "sb_lookup_only_batch: frames must share one guide format");
        std::snprintf(name, sizeof name, "frames[%d]", k);
        if (!f.lut) return fail(SB_ERR_INVALID_ARG, std::string(name) + ": lut NULL");
        if (!f.lut->entries)
            return fail(SB_ERR_UNSUPPORTED,
                        std::string(name) + ": sb_lookup_only needs a table (keys of at most 24 bits)");
        if (f.lut->channels != channels || f.lut->bits != bits)
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": lut built for another format");
        std::snprintf(name, sizeof name, "frames[%d].src_style", k);
        if ((st = check_style(&f.src_style, name)) != SB_OK) return st;
        if (f.src_style.width != f.lut->src_w || f.src_style.height != f.lut->src_h)
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": size differs from the lut's guide");
        std::snprintf(name, sizeof name, "frames[%d]", k);
        const int64_t npx = (int64_t)f.tgt_guide.width * f.tgt_guide.height;
        if (npx > 0 && (!f.rgba8_out || ((uintptr_t)f.rgba8_out % 4)))
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": rgba8_out NULL or misaligned");
        const int64_t bx = ((int64_t)f.tgt_guide.width + px_per_block - 1) / px_per_block;
        const int64_t blocks = npx > 0 ? bx * f.tgt_guide.height : 0;
        if (blocks > INT_MAX) return fail(SB_ERR_INVALID_ARG, std::string(name) + ": too many blocks");
        b.blocks[k] = (int)blocks;
        b.blocks_x[k] = bx > 1 ? (int)bx : 1;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    for (int k = 0; k < n_frames; ++k)
        if (frames[k].lut->device != dev) return fail(SB_ERR_INVALID_ARG, "a lut lives on another device");
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    LookupBatchLaunch L{frames, &b, quads, static_cast<cudaStream_t>(stream)};
    if (!dispatch_format(channels, bits, L))
        return fail(SB_ERR_UNSUPPORTED, "unsupported guide format");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sb_lookup_only_batch");
    return ok();
}
