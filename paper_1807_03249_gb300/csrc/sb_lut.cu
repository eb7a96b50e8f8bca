// Guide look-up table of StyleBlit (Section 3.1: the local guide names a
// source position, so a look-up table returns, for a guide value, the source
// pixel with the nearest guide; Algorithm 2 calls this lookup for u*).
//
// The table is exact: bin k maps to argmin_u |rep(k) - G_S[u]|^2 with ties to
// the smallest linear index.  8-bit guides keyed on at most three channels go
// through a distance transform over the grid of guide values (edt_* below);
// the others through a pruned search of two kernels:
//   1. lut_tile_bounds: per 16x16 source tile, the per-channel min/max of the
//      guide (an axis-aligned box in guide space).
//   2. lut_search: one thread per bin, bins enumerated in Morton order so a
//      warp covers a compact box of guide space.  Each lane first scans the
//      tile whose box is nearest to its representative, then the warp walks
//      every tile and scans it only if some lane's box distance can still
//      beat (or tie with a smaller index) that lane's best.  A skipped tile
//      holds no pixel strictly closer than the best and no tie with a smaller
//      linear index, so the result equals the brute-force argmin.
#include <algorithm>
#include <cstdio>

#include "sb_nn.cuh"

namespace sb {

constexpr int kLutThreads = 256;

// One packed uint32 per source pixel (the layout GuideFmt::load returns), so
// later gathers of G_S are single aligned 32-bit loads.
template <int C, int B>
__global__ void __launch_bounds__(256) pack_guide_kernel(const uint8_t *__restrict__ src,
                                                         int64_t stride, int W, int H,
                                                         uint32_t *__restrict__ packed) {
    using F = GuideFmt<C, B>;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * H) return;
    const int y = (int)(i / W), x = (int)(i % W);
    packed[i] = F::load(src, stride, x, y);
}

template <int C, int B>
__global__ void __launch_bounds__(256) lut_tile_bounds_kernel(const uint8_t *__restrict__ src,
                                                              int64_t stride, int W, int H,
                                                              int tiles_x, int n_tiles,
                                                              uint4 *__restrict__ bounds) {
    using F = GuideFmt<C, B>;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n_tiles) return;  // whole warps exit together
    const int x0 = (warp % tiles_x) * kLutTile;
    const int y0 = (warp / tiles_x) * kLutTile;
    uint32_t mn[C], mx[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        mn[c] = 0xFFFFu;
        mx[c] = 0u;
    }
#pragma unroll
    for (int k = 0; k < kLutTile * kLutTile / 32; ++k) {
        const int i = lane + 32 * k;
        const int x = x0 + (i % kLutTile), y = y0 + (i / kLutTile);
        if (x < W && y < H) {
            const uint32_t v = F::load(src, stride, x, y);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                mn[c] = min(mn[c], F::chan(v, c));
                mx[c] = max(mx[c], F::chan(v, c));
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            mn[c] = min(mn[c], __shfl_xor_sync(0xFFFFFFFFu, mn[c], off));
            mx[c] = max(mx[c], __shfl_xor_sync(0xFFFFFFFFu, mx[c], off));
        }
    }
    if (lane == 0) {
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < C; ++c) w[c] = mn[c] | (mx[c] << 16);
        bounds[warp] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Boxes of super-tiles (kSuper x kSuper tiles): the union of their tiles'
// boxes, stored after the n_tiles tile boxes.

template <int C>
__global__ void __launch_bounds__(256) lut_super_bounds_kernel(uint4 *__restrict__ bounds,
                                                              int tiles_x, int tiles_y,
                                                              int n_tiles, int supers_x,
                                                              int n_supers) {
    const int st = blockIdx.x * 256 + threadIdx.x;
    if (st >= n_supers) return;
    const int tx0 = (st % supers_x) * kSuper, ty0 = (st / supers_x) * kSuper;
    uint32_t mn[4] = {0xFFFFu, 0xFFFFu, 0xFFFFu, 0xFFFFu}, mx[4] = {0, 0, 0, 0};
    for (int ty = ty0; ty < min(ty0 + kSuper, tiles_y); ++ty)
        for (int tx = tx0; tx < min(tx0 + kSuper, tiles_x); ++tx) {
            const uint4 b = bounds[ty * tiles_x + tx];
            const uint32_t w[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int c = 0; c < C; ++c) {
                mn[c] = min(mn[c], w[c] & 0xFFFFu);
                mx[c] = max(mx[c], w[c] >> 16);
            }
        }
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < C; ++c) w[c] = mn[c] | (mx[c] << 16);
    bounds[n_tiles + st] = make_uint4(w[0], w[1], w[2], w[3]);
}

// Source-guide readers for the search: the packed copy owned by an sb_lut,
// or the caller's guide itself (used by the allocation-free build).
struct PackedReader {
    const uint32_t *p;
    int W;
    __device__ __forceinline__ uint32_t operator()(int x, int y) const {
        return __ldg(p + (int64_t)y * W + x);
    }
};

template <int C, int B>
struct RawReader {
    const uint8_t *base;
    int64_t stride;
    __device__ __forceinline__ uint32_t operator()(int x, int y) const {
        return GuideFmt<C, B>::load(base, stride, x, y);
    }
};

template <int C, int B, typename Reader>
__device__ __forceinline__ void scan_tile(const Reader &rd, int W, int H, int tiles_x, int t,
                                          uint32_t rep_packed, int kc, uint64_t &bd,
                                          uint32_t &bl) {
    using F = GuideFmt<C, B>;
    const int x0 = (t % tiles_x) * kLutTile;
    const int y0 = (t / tiles_x) * kLutTile;
    const int x1 = min(x0 + kLutTile, W), y1 = min(y0 + kLutTile, H);
    for (int y = y0; y < y1; ++y) {
#pragma unroll 4
        for (int x = x0; x < x1; ++x) {
            const uint64_t d = F::dist(rep_packed, F::key_part(rd(x, y), kc));
            const uint32_t lin = (uint32_t)y * (uint32_t)W + (uint32_t)x;
            if (d < bd || (d == bd && lin < bl)) {
                bd = d;
                bl = lin;
            }
        }
    }
}

template <int C, int B, typename Reader>
__global__ void __launch_bounds__(kLutThreads)
    lut_search_kernel(const Reader rd, int W, int H, int tiles_x, int n_tiles, int supers_x,
                      int n_supers, const uint4 *__restrict__ bounds, int key_bits, int kc,
                      uint32_t n_bins, uint32_t *__restrict__ lut) {
    const uint32_t g = blockIdx.x * kLutThreads + threadIdx.x;
    const bool valid = g < n_bins;

    // Morton order over the kc key channels: bit b*kc + c of g is bit b of
    // channel c's key; channels from kc on are not keyed
    uint32_t key[C];
#pragma unroll
    for (int c = 0; c < C; ++c) key[c] = 0;
#pragma unroll
    for (int c = 0; c < C; ++c)
        if (c < kc)
            for (int b = 0; b < key_bits; ++b) key[c] |= ((g >> (b * kc + c)) & 1u) << b;
    const int z = B - key_bits;
    uint32_t rep[C];
    uint32_t rep_packed = 0, idx = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        rep[c] = c < kc ? (key[c] << z) + (((1u << z) - 1u) >> 1) : 0u;
        rep_packed |= rep[c] << (c * B);
        idx |= key[c] << (c * key_bits);
    }

    const int tiles_y = (n_tiles + tiles_x - 1) / tiles_x;
    const uint4 *sup = bounds + n_tiles;  // super-tile boxes
    // pass A: the super-tile whose box is nearest, then its nearest tile
    uint64_t best_lb = ~0ull;
    int best_s = 0;
    for (int st = 0; st < n_supers; ++st) {
        const uint64_t lb = box_distance<C, B>(rep, __ldg(&sup[st]), kc);
        if (lb < best_lb) {
            best_lb = lb;
            best_s = st;
        }
    }
    const int stx0 = (best_s % supers_x) * kSuper, sty0 = (best_s / supers_x) * kSuper;
    int best_t = sty0 * tiles_x + stx0;
    best_lb = ~0ull;
    for (int ty = sty0; ty < min(sty0 + kSuper, tiles_y); ++ty)
        for (int tx = stx0; tx < min(stx0 + kSuper, tiles_x); ++tx) {
            const uint64_t lb = box_distance<C, B>(rep, __ldg(&bounds[ty * tiles_x + tx]), kc);
            if (lb < best_lb) {
                best_lb = lb;
                best_t = ty * tiles_x + tx;
            }
        }
    // pass B: an initial best from that tile
    uint64_t bd = ~0ull;
    uint32_t bl = 0xFFFFFFFFu;
    scan_tile<C, B>(rd, W, H, tiles_x, best_t, rep_packed, kc, bd, bl);
    // pass C: every super-tile, then every tile of it, that could still hold a
    // better or tied-earlier pixel (a tile's box lies in its super-tile's box
    // and its first pixel comes no earlier than the super-tile's)
    for (int st = 0; st < n_supers; ++st) {
        const int tx0 = (st % supers_x) * kSuper, ty0 = (st / supers_x) * kSuper;
        const uint64_t lbs = box_distance<C, B>(rep, __ldg(&sup[st]), kc);
        const uint32_t first_s = (uint32_t)(ty0 * kLutTile) * (uint32_t)W + (uint32_t)(tx0 * kLutTile);
        if (!__any_sync(0xFFFFFFFFu, valid && (lbs < bd || (lbs == bd && first_s < bl))))
            continue;
        for (int ty = ty0; ty < min(ty0 + kSuper, tiles_y); ++ty)
            for (int tx = tx0; tx < min(tx0 + kSuper, tiles_x); ++tx) {
                const int t = ty * tiles_x + tx;
                const uint64_t lb = box_distance<C, B>(rep, __ldg(&bounds[t]), kc);
                const uint32_t first = (uint32_t)(ty * kLutTile) * (uint32_t)W +
                                       (uint32_t)(tx * kLutTile);
                const bool need = valid && (lb < bd || (lb == bd && first < bl));
                if (__any_sync(0xFFFFFFFFu, need))
                    scan_tile<C, B>(rd, W, H, tiles_x, t, rep_packed, kc, bd, bl);
            }
    }
    if (valid) lut[idx] = (bl % (uint32_t)W) | ((bl / (uint32_t)W) << 16);
}

// ---------------------------------------------------------------------------
// Distance-transform build for 8-bit guides keyed on at most three channels.
// Over the 256^kc grid of keyed guide values, every value some source pixel
// holds is a site carrying the smallest linear index of those pixels.  Three
// separable passes (one per dimension) give each grid point its nearest site:
// the squared distance and, on ties, the smallest index, in one 64-bit key
// (distance << 32 | index), so each pass is a plain min.  The table reads the
// grid at the bin representatives.  The separable decomposition of the
// squared Euclidean distance makes the nested minima equal the minimum over
// all sites, and every pass keeps the smallest index among equal distances,
// so the entries equal the brute-force argmin (ties to the smallest index).
// no site yet: above every real key; adding three passes' (255^2 << 32) stays below 2^63
constexpr uint64_t kEdtEmpty = (uint64_t)1 << 62;

__global__ void __launch_bounds__(256) edt_fill_kernel(uint64_t *__restrict__ grid, uint32_t n) {
    const uint32_t i = blockIdx.x * 256u + threadIdx.x;
    if (i < n) grid[i] = kEdtEmpty;
}

// Site of every source pixel: its keyed value (channels 0..kc-1, 8 bits each,
// as packed) -> the smallest index holding it (distance 0).
__global__ void __launch_bounds__(256) edt_sites_kernel(const uint32_t *__restrict__ packed,
                                                       int64_t n_px, uint32_t key_mask,
                                                       unsigned long long *__restrict__ grid) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i < n_px) atomicMin(&grid[__ldg(packed + i) & key_mask], (unsigned long long)i);
}

// One pass along the dimension of element stride `stride` (1, 256 or 65536):
// CTA `line` holds the 256 grid points of one line, out[i] = min over j of
// in[j] + ((i - j)^2 << 32).
__global__ void __launch_bounds__(256) edt_pass_kernel(const uint64_t *__restrict__ in,
                                                      uint64_t *__restrict__ out, int stride) {
    __shared__ uint64_t line[256];
    const int l = blockIdx.x;
    const size_t base = (size_t)(l % stride) + (size_t)(l / stride) * (size_t)stride * 256;
    const int i = threadIdx.x;
    line[i] = in[base + (size_t)i * stride];
    __syncthreads();
    uint64_t best = kEdtEmpty << 1;
#pragma unroll 8
    for (int j = 0; j < 256; ++j) {
        const uint32_t d = (uint32_t)(i - j) * (uint32_t)(i - j);
        best = min(best, line[j] + ((uint64_t)d << 32));
    }
    out[base + (size_t)i * stride] = best;
}

// Table entry of bin g: the grid point at its representative.
__global__ void __launch_bounds__(256) edt_extract_kernel(const uint64_t *__restrict__ grid,
                                                         int kc, int key_bits, uint32_t n_bins,
                                                         int W, uint32_t *__restrict__ lut) {
    const uint32_t g = blockIdx.x * 256u + threadIdx.x;
    if (g >= n_bins) return;
    const int z = 8 - key_bits;
    uint32_t voxel = 0;
    for (int c = 0; c < kc; ++c) {
        const uint32_t key = (g >> (c * key_bits)) & ((1u << key_bits) - 1u);
        voxel |= ((key << z) + (((1u << z) - 1u) >> 1)) << (8 * c);
    }
    const uint32_t id = (uint32_t)(__ldg(grid + voxel) & 0xFFFFFFFFu);
    lut[g] = (id % (uint32_t)W) | ((id / (uint32_t)W) << 16);
}

// Whether the distance-transform build applies (8-bit guides, at most three
// keyed channels) and its scratch: two grids of 256^kc keys.
__host__ inline bool edt_applies(int bits, int key_channels) { return bits == 8 && key_channels <= 3; }
__host__ inline size_t edt_grid_points(int key_channels) { return (size_t)1 << (8 * key_channels); }

struct LutLaunch {
    const sb_guide *src;
    int key_bits;
    int key_channels;
    uint32_t n_bins;
    uint4 *bounds;
    uint32_t *entries;
    uint32_t *packed;   // NULL: search the caller's guide directly
    cudaStream_t stream;
    uint64_t *edt = nullptr;  // two grids: the distance-transform build (needs packed)
    template <int C, int B>
    void operator()() {
        if (edt && packed) {
            const uint8_t *p = static_cast<const uint8_t *>(src->data);
            const int64_t n_px = (int64_t)src->width * src->height;
            const uint32_t n = (uint32_t)edt_grid_points(key_channels);
            uint64_t *g0 = edt, *g1 = edt + n;
            pack_guide_kernel<C, B><<<(unsigned)((n_px + 255) / 256), 256, 0, stream>>>(
                p, src->row_stride, src->width, src->height, packed);
            edt_fill_kernel<<<(n + 255) / 256, 256, 0, stream>>>(g0, n);
            edt_sites_kernel<<<(unsigned)((n_px + 255) / 256), 256, 0, stream>>>(
                packed, n_px, n - 1u, reinterpret_cast<unsigned long long *>(g0));
            for (int d = 0; d < key_channels; ++d) {
                edt_pass_kernel<<<n / 256, 256, 0, stream>>>(g0, g1, 1 << (8 * d));
                uint64_t *t = g0;
                g0 = g1;
                g1 = t;
            }
            edt_extract_kernel<<<(n_bins + 255) / 256, 256, 0, stream>>>(
                g0, key_channels, key_bits, n_bins, src->width, entries);
            return;
        }
        const int tiles_x = (src->width + kLutTile - 1) / kLutTile;
        const int tiles_y = (src->height + kLutTile - 1) / kLutTile;
        const int n_tiles = tiles_x * tiles_y;
        const int supers_x = (tiles_x + kSuper - 1) / kSuper;
        const int n_supers = supers_x * ((tiles_y + kSuper - 1) / kSuper);
        const uint8_t *p = static_cast<const uint8_t *>(src->data);
        const int64_t n_px = (int64_t)src->width * src->height;
        const unsigned search_blocks = (n_bins + kLutThreads - 1) / kLutThreads;
        lut_tile_bounds_kernel<C, B><<<(n_tiles + 7) / 8, 256, 0, stream>>>(
            p, src->row_stride, src->width, src->height, tiles_x, n_tiles, bounds);
        lut_super_bounds_kernel<C><<<(n_supers + 255) / 256, 256, 0, stream>>>(
            bounds, tiles_x, tiles_y, n_tiles, supers_x, n_supers);
        if (packed) {
            pack_guide_kernel<C, B><<<(unsigned)((n_px + 255) / 256), 256, 0, stream>>>(
                p, src->row_stride, src->width, src->height, packed);
            lut_search_kernel<C, B><<<search_blocks, kLutThreads, 0, stream>>>(
                PackedReader{packed, src->width}, src->width, src->height, tiles_x, n_tiles,
                supers_x, n_supers, bounds, key_bits, key_channels, n_bins, entries);
        } else {
            lut_search_kernel<C, B><<<search_blocks, kLutThreads, 0, stream>>>(
                RawReader<C, B>{p, src->row_stride}, src->width, src->height, tiles_x, n_tiles,
                supers_x, n_supers, bounds, key_bits, key_channels, n_bins, entries);
        }
    }
};

// The search index of a source guide (keys wider than 24 bits): the packed
// guide and the tile and super-tile guide boxes.
struct IndexLaunch {
    const sb_guide *src;
    uint32_t *packed;
    uint4 *bounds;
    cudaStream_t stream;
    template <int C, int B>
    void operator()() {
        const NnGeometry g = NnGeometry::of(src->width, src->height);
        const uint8_t *p = static_cast<const uint8_t *>(src->data);
        const int64_t n_px = (int64_t)src->width * src->height;
        pack_guide_kernel<C, B><<<(unsigned)((n_px + 255) / 256), 256, 0, stream>>>(
            p, src->row_stride, src->width, src->height, packed);
        lut_tile_bounds_kernel<C, B><<<(g.n_tiles + 7) / 8, 256, 0, stream>>>(
            p, src->row_stride, src->width, src->height, g.tiles_x, g.n_tiles, bounds);
        lut_super_bounds_kernel<C><<<(g.n_supers + 255) / 256, 256, 0, stream>>>(
            bounds, g.tiles_x, g.tiles_y, g.n_tiles, g.supers_x, g.n_supers);
    }
};

// sb_build_lut_keyed for keys wider than 24 bits: no table; the frame
// kernels query the search index for every seed.
static sb_status build_search_index(const sb_guide *src, int32_t key_bits, int32_t key_channels,
                                    sb_lut **out, cudaStream_t s) {
    const NnGeometry g = NnGeometry::of(src->width, src->height);
    sb_lut *lut = new sb_lut;
    lut->key_channels = key_channels;
    lut->n_entries = 0;
    lut->channels = src->channels;
    lut->bits = src->bits;
    lut->key_bits = key_bits;
    lut->src_w = src->width;
    lut->src_h = src->height;
    cudaGetDevice(&lut->device);
    cudaError_t e;
    const size_t n_px = (size_t)src->width * src->height;
    if ((e = cudaMalloc(&lut->src_packed, sizeof(uint32_t) * n_px)) != cudaSuccess) {
        delete lut;
        return cuda_fail(e, "sb_build_lut: packed guide allocation");
    }
    if ((e = cudaMalloc(&lut->nn_bounds, sizeof(uint4) * (size_t)(g.n_tiles + g.n_supers))) !=
        cudaSuccess) {
        cudaFree(lut->src_packed);
        delete lut;
        return cuda_fail(e, "sb_build_lut: search index allocation");
    }
    IndexLaunch L{src, lut->src_packed, lut->nn_bounds, s};
    dispatch_format(src->channels, src->bits, L);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        cudaStreamSynchronize(s);
        cudaFree(lut->src_packed);
        cudaFree(lut->nn_bounds);
        delete lut;
        return cuda_fail(e, "sb_build_lut: launch");
    }
    *out = lut;
    return ok();
}

}  // namespace sb

using namespace sb;

extern "C" sb_status sb_build_lut_keyed(const sb_guide *src_guide, int32_t key_bits,
                                        int32_t key_channels, sb_lut **out, sb_stream stream) {
    sb_status st = check_guide(src_guide, "src_guide", true);
    if (st != SB_OK) return st;
    if (!out) return fail(SB_ERR_INVALID_ARG, "out: NULL");
    if (key_bits < 1 || key_bits > src_guide->bits)
        return fail(SB_ERR_INVALID_ARG, "key_bits must be in [1, bits]");
    if (key_channels < 1 || key_channels > src_guide->channels)
        return fail(SB_ERR_INVALID_ARG, "key_channels must be in [1, channels]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sb_build_lut: pending CUDA error");
    if (key_channels * key_bits > kMaxKeyBitsTotal)
        return build_search_index(src_guide, key_bits, key_channels, out, s);

    const uint32_t n_bins = 1u << (key_channels * key_bits);
    const int tiles_x = (src_guide->width + kLutTile - 1) / kLutTile;
    const int tiles_y = (src_guide->height + kLutTile - 1) / kLutTile;
    const size_t n_tiles = (size_t)tiles_x * tiles_y;

    sb_lut *lut = new sb_lut;
    lut->key_channels = key_channels;
    lut->n_entries = n_bins;
    lut->channels = src_guide->channels;
    lut->bits = src_guide->bits;
    lut->key_bits = key_bits;
    lut->src_w = src_guide->width;
    lut->src_h = src_guide->height;
    cudaGetDevice(&lut->device);
    if ((e = cudaMalloc(&lut->entries, sizeof(uint32_t) * n_bins)) != cudaSuccess) {
        delete lut;
        return cuda_fail(e, "sb_build_lut: table allocation");
    }
    const size_t n_px = (size_t)src_guide->width * src_guide->height;
    if ((e = cudaMalloc(&lut->src_packed, sizeof(uint32_t) * n_px)) != cudaSuccess) {
        cudaFree(lut->entries);
        delete lut;
        return cuda_fail(e, "sb_build_lut: packed guide allocation");
    }
    // scratch: tile bounds for the search, or two grids for the distance transform
    const bool edt = edt_applies(src_guide->bits, key_channels);
    void *scratch = nullptr;
    const size_t scratch_bytes =
        edt ? 2 * sizeof(uint64_t) * edt_grid_points(key_channels)
            : sizeof(uint4) * (n_tiles + (size_t)((tiles_x + kSuper - 1) / kSuper) *
                                             ((tiles_y + kSuper - 1) / kSuper));
    if ((e = cudaMallocAsync(&scratch, scratch_bytes, s)) != cudaSuccess) {
        cudaFree(lut->entries);
        cudaFree(lut->src_packed);
        delete lut;
        return cuda_fail(e, "sb_build_lut: scratch allocation");
    }
    LutLaunch L{src_guide, key_bits, key_channels, n_bins,
                edt ? nullptr : static_cast<uint4 *>(scratch), lut->entries, lut->src_packed, s,
                edt ? static_cast<uint64_t *>(scratch) : nullptr};
    dispatch_format(src_guide->channels, src_guide->bits, L);
    e = cudaGetLastError();
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        cudaFree(lut->entries);
        cudaFree(lut->src_packed);
        delete lut;
        return cuda_fail(e, "sb_build_lut: launch");
    }
    *out = lut;
    return ok();
}

extern "C" sb_status sb_build_lut(const sb_guide *src_guide, int32_t key_bits, sb_lut **out,
                                  sb_stream stream) {
    if (!src_guide) return fail(SB_ERR_INVALID_ARG, "src_guide: NULL guide descriptor");
    return sb_build_lut_keyed(src_guide, key_bits, src_guide->channels, out, stream);
}

extern "C" sb_status sb_lut_destroy(sb_lut *lut) {
    if (!lut) return ok();
    cudaError_t e = cudaFree(lut->entries);
    cudaError_t e2 = cudaFree(lut->src_packed);
    cudaError_t e3 = cudaFree(lut->nn_bounds);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = e3;
    delete lut;
    if (e != cudaSuccess) return cuda_fail(e, "sb_lut_destroy");
    return ok();
}

extern "C" sb_status sb_lut_info(const sb_lut *lut, const uint32_t **entries, int64_t *n_entries,
                                 int32_t *channels, int32_t *bits, int32_t *key_bits,
                                 int32_t *key_channels, int32_t *src_width,
                                 int32_t *src_height) {
    if (!lut) return fail(SB_ERR_INVALID_ARG, "lut: NULL");
    if (key_channels) *key_channels = lut->key_channels;
    if (entries) *entries = lut->entries;
    if (n_entries) *n_entries = lut->n_entries;
    if (channels) *channels = lut->channels;
    if (bits) *bits = lut->bits;
    if (key_bits) *key_bits = lut->key_bits;
    if (src_width) *src_width = lut->src_w;
    if (src_height) *src_height = lut->src_h;
    return ok();
}

// ---------------------------------------------------------------------------
// Allocation-free table build.
//
// Some callers cannot allocate device memory: a host application whose pool
// allocator already owns the device's memory, or a frame loop that must not
// call cudaMalloc (it can synchronise the device and fail under memory
// pressure).  sb_build_lut_noalloc builds the same table into a buffer the
// caller provides.  Its only scratch, the tile and super-tile guide boxes, lives in the
// fixed array below, which every GPU that loads this library holds until the
// process exits; the search reads the caller's guide directly instead of a
// packed copy.
// ---------------------------------------------------------------------------
namespace sb {

constexpr int kStaticBoundsTiles = 65536;  // 1 MiB: 16x16 tiles of a 4096 x 4096 source
constexpr int kStaticSupers = 5376;        // their super-tiles, any aspect (sides <= 32767)
static __device__ __align__(256) uint4 g_static_bounds[kStaticBoundsTiles + kStaticSupers];

// Device address of g_static_bounds on the current device (host code cannot
// use the symbol itself as a device pointer).  Looked up on every call, not
// cached: after a device reset the module is loaded again and the array may
// sit elsewhere.  cudaGetSymbolAddress allocates nothing.
static cudaError_t static_bounds_address(uint4 **out) {
    uint4 *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_static_bounds);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace sb

extern "C" sb_status sb_build_lut_noalloc(const sb_guide *src_guide, int32_t key_bits,
                                          uint32_t *table_out, sb_stream stream) {
    sb_status st = check_guide(src_guide, "src_guide", true);
    if (st != SB_OK) return st;
    if (key_bits < 1 || key_bits > src_guide->bits)
        return fail(SB_ERR_INVALID_ARG, "key_bits must be in [1, bits]");
    if (src_guide->channels * key_bits > kMaxKeyBitsTotal)
        return fail(SB_ERR_INVALID_ARG, "channels * key_bits must be <= 24");
    if (!table_out || ((uintptr_t)table_out % 4))
        return fail(SB_ERR_INVALID_ARG, "table_out: NULL or not 4-byte aligned");
    const int tiles_x = (src_guide->width + kLutTile - 1) / kLutTile;
    const int tiles_y = (src_guide->height + kLutTile - 1) / kLutTile;
    const int64_t n_supers = (int64_t)((tiles_x + kSuper - 1) / kSuper) * ((tiles_y + kSuper - 1) / kSuper);
    if ((int64_t)tiles_x * tiles_y > kStaticBoundsTiles || n_supers > kStaticSupers)
        return fail(SB_ERR_INVALID_ARG,
                    "sb_build_lut_noalloc: source guide too large for the fixed scratch "
                    "(at most 65536 tiles of 16x16 pixels, e.g. 4096 x 4096)");
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sb_build_lut_noalloc: pending CUDA error");
    uint4 *bounds = nullptr;
    if ((e = static_bounds_address(&bounds)) != cudaSuccess)
        return cuda_fail(e, "sb_build_lut_noalloc: scratch address");
    const uint32_t n_bins = 1u << (src_guide->channels * key_bits);
    LutLaunch L{src_guide, key_bits, src_guide->channels, n_bins, bounds, table_out, nullptr,
                static_cast<cudaStream_t>(stream)};
    dispatch_format(src_guide->channels, src_guide->bits, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sb_build_lut_noalloc: launch");
    return ok();
}
