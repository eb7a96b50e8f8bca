// Per-frame StyleBlit kernels: Algorithm 2 (ParallelStyleBlit) with the
// coordinate transfer and voting step of Section 3.2.  Templates only; the
// sb_frame_*.cu files instantiate them per guide format.
//
// One CTA owns a 64 x 32 output tile.  The fused kernel computes the
// assignment A of the tile plus a halo of R pixels (the vote window) in shared
// memory, so A never reaches device memory:
//
//   phase 0  target guide of the region -> smem (one packed uint32 per pixel),
//            read by vertical segments of 4 pixels (one region column per
//            lane); the seed cells of every level >= 3 are built at the same
//            time (levels 2 and 1 have many cells and are built only if a
//            pixel of the tile still needs them).  A cell is: jitter hash ->
//            seed q clamped into the target -> G_T[q] -> table entry u*(q).
//            Cells are stored column-major (x outer, y inner), each as
//            (-2q, |q|^2, u*) in region-centred coordinates, pre-scaled by
//            2^11 with the cell's column-major index in the low 11 bits.
//   levels   for l = L..1 while pixels are pending: a pixel p takes the
//            minimum over its 3 x 3 cells of |q|^2 - 2 q.p (which orders seeds
//            like |q - p|^2) packed with the cell index: one min gives the
//            nearest seed and, on ties, the first cell in x-outer, y-inner
//            order, as NearestSeed's strict < does.  The candidate
//            s = u* + (p - q) is accepted if it lies in the source and
//            |G_S[s] - G_T[p]|^2 <= t (level 1 always accepts, s clamped).
//            Work goes by the 4-pixel segments: a segment lies in one cell at
//            levels >= 2 and the pixels choosing a seed form a convex set, so
//            when its first and last pending pixels choose the same seed all
//            of them do and the search runs once.  Segments with rejected
//            pixels are compacted into the next level's list.
//   vote     ballot bitmasks mark, per row, where A steps by exactly one pixel
//            (horizontally and vertically); a window made of one translation
//            votes exactly C_S[A(p)], a plain copy.  Other pixels (chunk
//            boundaries, frame borders) are compacted and summed over the full
//            window with integer sums and round-half-up division.
//   store    uniform windows store from the copy pass (coalesced rows), the
//            others from the full-window passes.
#pragma once

#include <atomic>
#include <climits>

#include "sb_internal.cuh"

namespace sb {

constexpr int kTW = 64;
constexpr int kTH = 32;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kEagerMinLevel = 3;           // levels >= this get their cells in phase 0
constexpr int kKeyShift = 11;               // cell-index bits of the packed seed key
constexpr int kPackedMaxLevel = 8;          // levels whose packed keys fit 32 bits

enum Mode { kAssign = 0, kStylize = 1 };

struct FrameArgs {
    const uint8_t *tgt;
    int64_t tgt_stride;
    int W, H;
    const uint32_t *src_packed;  // G_S, one packed uint32 per pixel, row-major
    int Ws, Hs;
    const uint32_t *lut;
    int key_bits;
    int key_channels;
    const uint8_t *style;
    int style_stride_px;         // style row stride in pixels (height * stride < 2^31)
    int levels;
    uint64_t threshold;
    uint32_t seed;
    int radius;
    const uint32_t *assign_in;   // sb_blend
    uint32_t *assign_out;        // sb_assign_chunks
    uint8_t *level_out;          // sb_assign_chunks (nullable)
    uint32_t *rgba_out;          // RGBA8 as one uint32 per pixel
    float4 *f32_out;             // sb_blend float variant
};

// upper bound of the cells of level l touching a region of RW x RH pixels
__host__ __device__ constexpr int cells_bound(int RW, int RH, int l) {
    return (((RW - 1) >> l) + 4) * (((RH - 1) >> l) + 4);
}

struct SmemLayout {
    int RW, RH, NR, NC;
    size_t off_cells, off_gt, off_A, off_list0, off_list1, off_bytes, off_masks, off_cnt, total;
};

__host__ __device__ inline SmemLayout smem_layout(int r, int levels) {
    SmemLayout s;
    s.RW = kTW + 2 * r;
    s.RH = kTH + 2 * r;
    s.NR = s.RW * s.RH;
    s.NC = 0;
    for (int l = 1; l <= levels; ++l) s.NC += cells_bound(s.RW, s.RH, l);
    size_t o = 0;
    s.off_cells = o;
    o += sizeof(int4) * (size_t)s.NC;
    s.off_gt = o;
    o += sizeof(uint32_t) * (size_t)s.NR;
    s.off_A = o;
    o += sizeof(uint32_t) * (size_t)s.NR;
    s.off_masks = o;
    o += (2 * sizeof(uint64_t) + 4 * sizeof(uint32_t)) * (size_t)s.RH;
    s.off_list0 = o;
    o += sizeof(uint16_t) * (size_t)s.NR;
    s.off_list1 = o;
    o += sizeof(uint16_t) * (size_t)s.NR;
    s.off_bytes = o;
    o += (size_t)s.NR;
    o = (o + 15) & ~(size_t)15;
    s.off_cnt = o;
    o += 32;  // 3 level counters (rotating), slow and complex vote counters
    s.total = o;
    return s;
}

// Block-wide append to a shared list; every lane of the warp must call it.
__device__ __forceinline__ void list_push(bool pred, int val, uint16_t *list, int *counter) {
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = (uint16_t)val;
}

// Seed cells of level l for the clamped region [xa, xb] x [ya, yb].
struct LevelCells {
    int cx0, cy0, ncx, ncy;
};

__device__ __forceinline__ LevelCells level_cells(int l, int xa, int xb, int ya, int yb) {
    LevelCells g;
    g.cx0 = (xa >> l) - 1;
    g.ncx = (xb >> l) - (xa >> l) + 3;
    g.cy0 = (ya >> l) - 1;
    g.ncy = (yb >> l) - (ya >> l) + 3;
    return g;
}

// Number of cells of levels l_hi down to l_lo for the clamped region.
__device__ __forceinline__ int cell_count(int l_hi, int l_lo, int xa, int xb, int ya, int yb) {
    int total = 0;
    for (int l = l_hi; l >= l_lo; --l) {
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        total += g.ncx * g.ncy;
    }
    return total;
}

// Cell k of the levels stacked from l_hi downwards (each column-major): its
// level, column-major index within the level and seed q (clamped into the
// target).
struct CellTask {
    int l, ci, sx, sy;
};

__device__ __forceinline__ CellTask cell_task(const FrameArgs &a, int k, int l_hi, int xa, int xb,
                                              int ya, int yb) {
    CellTask t;
    int l = l_hi, off = 0;
    LevelCells g = level_cells(l, xa, xb, ya, yb);
    while (k >= off + g.ncx * g.ncy) {
        off += g.ncx * g.ncy;
        --l;
        g = level_cells(l, xa, xb, ya, yb);
    }
    const int ci = k - off;  // column-major: ci = lcx * ncy + lcy
    // ci / ncy through a float reciprocal: ci < 2^11 and ncy < 2^6 keep the
    // true quotient at least 0.5 / ncy from an integer, far above the
    // rounding error, so the truncation is exact
    const int lcx = (int)(((float)ci + 0.5f) * __frcp_rn((float)g.ncy));
    const int lcy = ci - lcx * g.ncy;
    const int h = 1 << l;
    const int bx = g.cx0 + lcx, by = g.cy0 + lcy;
    const uint32_t hsh = cell_hash(level_key(a.seed, l), bx, by);
    const int ox = (int)(((hsh & 0xFFFFu) * (uint32_t)h) >> 16);
    const int oy = (int)(((hsh >> 16) * (uint32_t)h) >> 16);
    t.l = l;
    t.ci = ci;
    t.sx = min(max(bx * h + ox, 0), a.W - 1);
    t.sy = min(max(by * h + oy, 0), a.H - 1);
    return t;
}

// The stored cell: (-2q, |q|^2, u*) in region-centred coordinates (q - (cxo,
// cyo)); levels with packed keys scale by 2^11 and add the cell index.
__device__ __forceinline__ int4 cell_value(const CellTask &t, uint32_t u, int cxo, int cyo) {
    const int qx = t.sx - cxo, qy = t.sy - cyo;
    if (t.l <= kPackedMaxLevel) {
        constexpr int S = 1 << kKeyShift;
        return make_int4(-2 * qx * S, -2 * qy * S, (qx * qx + qy * qy) * S + t.ci, (int)u);
    }
    return make_int4(-2 * qx, -2 * qy, qx * qx + qy * qy, (int)u);
}

// Builds cells k0, k0 + kThreads, ... of the levels l_hi down to l_lo into
// cells[base_hi + k].
template <int C, int B>
__device__ __forceinline__ void build_cells(const FrameArgs &a, int4 *cells, int l_hi, int l_lo,
                                            int base_hi, int xa, int xb, int ya, int yb,
                                            int cxo, int cyo, int k0 = 0, int total = -1) {
    using F = GuideFmt<C, B>;
    if (total < 0) total = cell_count(l_hi, l_lo, xa, xb, ya, yb);
#pragma unroll 1
    for (int k = k0 + (int)threadIdx.x; k < total; k += kThreads) {
        const CellTask t = cell_task(a, k, l_hi, xa, xb, ya, yb);
        const uint32_t u = __ldg(
            a.lut + F::key(F::load(a.tgt, a.tgt_stride, t.sx, t.sy), a.key_bits, a.key_channels));
        cells[base_hi + k] = cell_value(t, u, cxo, cyo);
    }
}

// Vertical segments of 4 pixels starting at target rows that are multiples of
// 4 cover the region (the tile plus its R halo): segment s takes region column
// s % RW, so the lanes of a warp hold neighbouring columns.  At every level
// >= 2 a segment lies inside one seed cell.
template <int R>
struct Segs {
    static constexpr int kPad = (R + 3) / 4 * 4;  // first segment row: kPad rows above the tile
    static constexpr int RW = kTW + 2 * R, RH = kTH + 2 * R;
    static constexpr int NSY = (kTH + 2 * kPad) / 4;
    static constexpr int NS = RW * NSY;
    __device__ __forceinline__ static int rx(int s) { return s % RW; }
    __device__ __forceinline__ static int ry(int s) { return 4 * (s / RW) - kPad + R; }
    // bit j: lo <= ry + j < hi
    __device__ __forceinline__ static uint32_t span(int ry, int lo, int hi) {
        const int a = min(max(lo - ry, 0), 4), b = min(max(hi - ry, 0), 4);
        return ((1u << b) - 1u) & ~((1u << a) - 1u);
    }
    // bit j: row ry + j lies in the region
    __device__ __forceinline__ static uint32_t rows(int ry) { return span(ry, 0, RH); }
};

// The region's columns [c_lo, c_hi) and rows [r_lo, r_hi) inside the target.
struct TileBounds {
    int c_lo, c_hi, r_lo, r_hi;
    template <int R>
    __device__ __forceinline__ static TileBounds of(int rx0, int ry0, int W, int H) {
        return TileBounds{max(0, -rx0), min(kTW + 2 * R, W - rx0), max(0, -ry0),
                          min(kTH + 2 * R, H - ry0)};
    }
    // bit j: pixel (rx, ry + j) of a segment lies in the region and the target
    template <int R>
    __device__ __forceinline__ uint32_t mask(int rx, int ry) const {
        return rx >= c_lo && rx < c_hi ? Segs<R>::span(ry, r_lo, r_hi) : 0u;
    }
};

// The source side of a candidate test.
struct SrcView {
    const uint32_t *src_packed;
    int Ws, Hs;
    uint64_t threshold;
};

// Candidate test of the pixels of one segment: pixel j sits at region index
// ibase + j * RW and its candidate source position is (sx[j], sy[j]).
// Accepted pixels get A (and the level); the bits of rejected pixels of m
// are returned.
template <int C, int B, int RW>
__device__ __forceinline__ uint32_t test_segment(const SrcView &a, const uint32_t *gt,
                                                 uint32_t *A, uint8_t *lev, int l, uint32_t t32,
                                                 uint32_t m, int ibase, const int (&sx)[4],
                                                 const int (&sy)[4]) {
    using F = GuideFmt<C, B>;
    uint32_t gsv[4];
    bool ok[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ok[j] = ((m >> j) & 1u) && (unsigned)sx[j] < (unsigned)a.Ws &&
                (unsigned)sy[j] < (unsigned)a.Hs;
        gsv[j] = ok[j] ? __ldg(a.src_packed + ((uint32_t)sy[j] * (uint32_t)a.Ws + (uint32_t)sx[j]))
                       : 0u;
    }
    uint32_t rej = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!((m >> j) & 1u)) continue;
        bool acc = false;
        if (ok[j]) {
            const uint64_t d = F::dist(gsv[j], gt[ibase + j * RW]);
            if constexpr (B == 8) acc = (uint32_t)d <= t32;
            else acc = d <= a.threshold;
        }
        if (acc) {
            A[ibase + j * RW] = (uint32_t)sx[j] + ((uint32_t)sy[j] << 16);
            if (lev) lev[ibase + j * RW] = (uint8_t)l;
        }
        rej |= (uint32_t)!acc << j;
    }
    return rej;
}

// Levels where every pixel searches its own seed: level 1 (a segment spans
// two cells) and the levels above kPackedMaxLevel (unscaled cells, 64-bit
// keys).  Both are rare, so pixels go one at a time with little live state
// (the common path keeps its registers).
template <int C, int B, int R>
__device__ __forceinline__ uint32_t segment_level_rare(const SrcView &a, const uint32_t *gt,
                                                       uint32_t *A, uint8_t *lev,
                                                       const int4 *cells, int base, int c0,
                                                       int ncy, int l, uint32_t t32, int rx,
                                                       int ry, uint32_t m) {
    using F = GuideFmt<C, B>;
    constexpr int RW = Segs<R>::RW, RH = Segs<R>::RH;
    constexpr int kMask = (1 << kKeyShift) - 1;
    const int prx = rx - RW / 2, pry = ry - RH / 2;
    const bool packed = l <= kPackedMaxLevel;
    uint32_t rej = 0;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        if (!((m >> j) & 1u)) continue;
        // level 1: rows 0-1 and 2-3 lie in consecutive cells of one column
        const int cj = c0 + (l == 1 ? (j >> 1) : 0);
        long long key = LLONG_MAX;
#pragma unroll 1
        for (int d = 0; d < 9; ++d) {
            const int c = cj + (d / 3 - 1) * ncy + (d % 3 - 1);
            const int4 cl = cells[c];
            const int e = cl.z + cl.x * prx + cl.y * (pry + j);
            // packed cells carry the index in their low bits already
            key = min(key, packed ? (long long)e : (((long long)e << kKeyShift) | (c - base)));
        }
        const int4 cl = cells[base + (int)(key & kMask)];
        const int sh = packed ? kKeyShift + 1 : 1;
        int sx = (int)((uint32_t)cl.w & 0xFFFFu) + prx + (cl.x >> sh);
        int sy = (int)((uint32_t)cl.w >> 16) + pry + j + (cl.y >> sh);
        const int i = (ry + j) * RW + rx;
        bool acc = true;
        if (l == 1) {
            sx = min(max(sx, 0), a.Ws - 1);
            sy = min(max(sy, 0), a.Hs - 1);
        } else {
            acc = (unsigned)sx < (unsigned)a.Ws && (unsigned)sy < (unsigned)a.Hs;
            if (acc) {
                const uint64_t d = F::dist(
                    __ldg(a.src_packed + ((uint32_t)sy * (uint32_t)a.Ws + (uint32_t)sx)), gt[i]);
                if constexpr (B == 8) acc = (uint32_t)d <= t32;
                else acc = d <= a.threshold;
            }
        }
        if (acc) {
            A[i] = (uint32_t)sx | ((uint32_t)sy << 16);
            if (lev) lev[i] = (uint8_t)l;
        } else {
            rej |= 1u << j;
        }
    }
    return rej;
}

// Level l (1 <= l <= kMaxLevels) of the pixels m of the segment at
// region (rx, ry): returns the rejected ones.  The packed keys of the nine
// candidates are affine in p, so the pixels that pick a given seed form a
// convex set: when the first and last pixel of m pick the same seed, every
// pixel between them does and the nine-way search runs once.  Otherwise each
// pixel searches (level 1 and the unscaled levels: segment_level_rare).
template <int C, int B, int R>
__device__ __forceinline__ uint32_t segment_level(const FrameArgs &a, const uint32_t *gt,
                                                  uint32_t *A, uint8_t *lev, const int4 *cells,
                                                  int base, const LevelCells &g, int l, int rx0,
                                                  int ry0, uint32_t t32, int rx, int ry,
                                                  uint32_t m) {
    using S = Segs<R>;
    constexpr int RW = S::RW, RH = S::RH;
    constexpr int kMask = (1 << kKeyShift) - 1;
    const int prx = rx - RW / 2, pry = ry - RH / 2;
    const int c0 = base + (((rx0 + rx) >> l) - g.cx0) * g.ncy + (((ry0 + ry) >> l) - g.cy0);
    const int ibase = ry * RW + rx;
    int sx[4], sy[4];
    auto candidate = [&](int j, int key) {
        const int4 cl = cells[base + (key & kMask)];
        sx[j] = (int)((uint32_t)cl.w & 0xFFFFu) + prx + (cl.x >> (kKeyShift + 1));
        sy[j] = (int)((uint32_t)cl.w >> 16) + pry + j + (cl.y >> (kKeyShift + 1));
    };
    const SrcView sv{a.src_packed, a.Ws, a.Hs, a.threshold};
    if (l == 1 || l > kPackedMaxLevel)
        return segment_level_rare<C, B, R>(sv, gt, A, lev, cells, base, c0, g.ncy, l, t32, rx, ry,
                                           m);
    const int jlo = __ffs(m) - 1, jhi = 31 - __clz(m);
    int klo = INT_MAX, khi = INT_MAX;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int4 cl = cells[c0 + dx * g.ncy + dy];
            const int e = cl.z + cl.x * prx + cl.y * (pry + jlo);
            klo = min(klo, e);
            khi = min(khi, e + (jhi - jlo) * cl.y);
        }
    }
    if (((klo ^ khi) & kMask) == 0) {
        candidate(0, klo);
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            sx[j] = sx[0];
            sy[j] = sy[0] + j;
        }
    } else {
        int k[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int4 cl = cells[c0 + dx * g.ncy + dy];
                const int e = cl.z + cl.x * prx + cl.y * pry;
#pragma unroll
                for (int j = 0; j < 4; ++j) k[j] = min(k[j], e + j * cl.y);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) candidate(j, k[j]);
    }
    return test_segment<C, B, RW>(sv, gt, A, lev, l, t32, m, ibase, sx, sy);
}

// One level over segments: the top level (top) visits every segment of the region
// (its in-target pixels), lower levels the list of segments with pending
// pixels (entries: segment index << 4 | pixel mask).  Segments with rejected
// pixels are appended to list_out.
template <int C, int B, int R>
__device__ __forceinline__ void level_segments(const FrameArgs &a, const uint32_t *gt,
                                               uint32_t *A, uint8_t *lev, const int4 *cells,
                                               int base, const LevelCells &g, int l, int rx0,
                                               int ry0, const TileBounds &tb, uint32_t t32,
                                               bool top, const uint16_t *list_in, int n_in,
                                               uint16_t *list_out, int *cnt_out) {
    using S = Segs<R>;
    const int n = top ? S::NS : n_in;
    for (int s0 = 0; s0 < n; s0 += kThreads) {
        const int jj = s0 + (int)threadIdx.x;
        int sg = 0;
        uint32_t m = 0;
        if (jj < n) {
            if (top) {
                sg = jj;
                m = tb.template mask<R>(S::rx(sg), S::ry(sg));
            } else {
                const uint32_t e = list_in[jj];
                sg = (int)(e >> 4);
                m = e & 15u;
            }
        }
        uint32_t rej = 0;
        if (m)
            rej = segment_level<C, B, R>(a, gt, A, lev, cells, base, g, l, rx0, ry0, t32,
                                         S::rx(sg), S::ry(sg), m);
        list_push(rej != 0, (sg << 4) | (int)rej, list_out, cnt_out);
    }
}

// ---------------------------------------------------------------------------
// assignment of the region held in shared memory (Algorithm 2)
// ---------------------------------------------------------------------------
template <int C, int B, int R>
__device__ __forceinline__ void assign_region(const FrameArgs &a, const SmemLayout &L, int rx0,
                                              int ry0, unsigned char *smem, uint8_t *lev) {
    using F = GuideFmt<C, B>;
    constexpr int RW = kTW + 2 * R, RH = kTH + 2 * R;
    int4 *cells = reinterpret_cast<int4 *>(smem + L.off_cells);
    uint32_t *gt = reinterpret_cast<uint32_t *>(smem + L.off_gt);
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.off_A);
    uint16_t *const list0 = reinterpret_cast<uint16_t *>(smem + L.off_list0);
    uint16_t *const list1 = reinterpret_cast<uint16_t *>(smem + L.off_list1);
    int *cnt = reinterpret_cast<int *>(smem + L.off_cnt);
    const int tid = threadIdx.x;

    const int xa = max(rx0, 0), xb = min(rx0 + RW, a.W) - 1;
    const int ya = max(ry0, 0), yb = min(ry0 + RH, a.H) - 1;
    const int cxo = rx0 + RW / 2, cyo = ry0 + RH / 2;
    const uint32_t t32 = a.threshold > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)a.threshold;
    const int L_top = a.levels;
    const int eager_lo = L_top <= kEagerMinLevel ? 1 : kEagerMinLevel;
    const TileBounds tb = TileBounds::of<R>(rx0, ry0, a.W, a.H);

    if (tid == 0) {
        cnt[0] = 0;
        cnt[1] = 0;
    }
    // phase 0: every global load (the guide at this thread's first seed, the
    // region's guide, then the seed's table entry) is issued before the
    // first store that waits on one
    const int n_eager = cell_count(L_top, eager_lo, xa, xb, ya, yb);
    const bool has_cell = tid < n_eager;
    CellTask ct{};
    uint32_t cg = 0;
    if (has_cell) {
        ct = cell_task(a, tid, L_top, xa, xb, ya, yb);
        cg = F::load(a.tgt, a.tgt_stride, ct.sx, ct.sy);
    }
    constexpr int kSegIters = (Segs<R>::NS + kThreads - 1) / kThreads;
    uint32_t gv[kSegIters][4], itq[kSegIters];
#pragma unroll
    for (int q = 0; q < kSegIters; ++q) {
        const int sg = q * kThreads + tid;
        const int rx = Segs<R>::rx(sg), ry = Segs<R>::ry(sg);
        const uint32_t it = sg < Segs<R>::NS ? tb.template mask<R>(rx, ry) : 0u;
        itq[q] = it;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            gv[q][j] = ((it >> j) & 1u) ? F::load(a.tgt, a.tgt_stride, rx0 + rx, ry0 + ry + j) : 0u;
    }
    uint32_t cu = 0;
    if (has_cell) cu = __ldg(a.lut + F::key(cg, a.key_bits, a.key_channels));
#pragma unroll
    for (int q = 0; q < kSegIters; ++q) {
        const int sg = q * kThreads + tid;
        if (sg >= Segs<R>::NS) continue;
        const int rx = Segs<R>::rx(sg), ry = Segs<R>::ry(sg);
        const uint32_t rl = Segs<R>::rows(ry);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!((rl >> j) & 1u)) continue;
            const int i = (ry + j) * RW + rx;
            if ((itq[q] >> j) & 1u) gt[i] = gv[q][j];
            else A[i] = kInvalid;
        }
    }
    if (has_cell) cells[tid] = cell_value(ct, cu, cxo, cyo);
    if (n_eager > kThreads)
        build_cells<C, B>(a, cells, L_top, eager_lo, 0, xa, xb, ya, yb, cxo, cyo, kThreads, n_eager);
    __syncthreads();

    // level step t (0 = top) appends to counter t % 3; the counter of step
    // t + 1 is cleared during step t (its last reader passed step t - 1's
    // barrier), so one barrier per level publishes both the list and the reset.
    // The top level visits every segment of the region; its cells start at 0.
    int n_pend = Segs<R>::NS, base = 0;
    const uint16_t *list_cur = list0;
    uint16_t *list_nxt = list1;
    for (int l = L_top, t = 0; l >= 1 && n_pend > 0; --l, ++t) {
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        if (l == kEagerMinLevel - 1 && eager_lo > 1) {
            // a pixel still needs the fine levels: build levels 2 and 1 now
            build_cells<C, B>(a, cells, l, 1, base, xa, xb, ya, yb, cxo, cyo);
            __syncthreads();
        }
        if (tid == 0) cnt[(t + 1) % 3] = 0;
        level_segments<C, B, R>(a, gt, A, lev, cells, base, g, l, rx0, ry0, tb, t32, t == 0,
                                list_cur, n_pend, list_nxt, &cnt[t % 3]);
        __syncthreads();
        n_pend = cnt[t % 3];
        base += g.ncx * g.ncy;
        const uint16_t *done = list_cur;
        list_cur = list_nxt;
        list_nxt = const_cast<uint16_t *>(done);
    }
}

// ---------------------------------------------------------------------------
// voting over the tile (Section 3.2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 rgba_f32(uint32_t col) {
    return make_float4(__fdiv_rn((float)(col & 0xFF), 255.f),
                       __fdiv_rn((float)((col >> 8) & 0xFF), 255.f),
                       __fdiv_rn((float)((col >> 16) & 0xFF), 255.f),
                       __fdiv_rn((float)(col >> 24), 255.f));
}

// Channel sums of a vote.  Windows of at most 15 x 15 taps keep two channels
// per 32-bit word (16-bit lanes: 225 * 255 < 2^16); larger ones one per word.
template <bool kPacked>
struct VoteAcc;

template <>
struct VoteAcc<true> {
    uint32_t lo = 0, hi = 0, n = 0;  // lo = c0 | c2 << 16, hi = c1 | c3 << 16
    __device__ __forceinline__ void add(uint32_t col, uint32_t cnt) {
        lo += (col & 0x00FF00FFu) * cnt;
        hi += ((col >> 8) & 0x00FF00FFu) * cnt;
        n += cnt;
    }
    __device__ __forceinline__ void sums(uint32_t &s0, uint32_t &s1, uint32_t &s2,
                                         uint32_t &s3) const {
        s0 = lo & 0xFFFFu;
        s2 = lo >> 16;
        s1 = hi & 0xFFFFu;
        s3 = hi >> 16;
    }
};

template <>
struct VoteAcc<false> {
    uint32_t s[4] = {0, 0, 0, 0}, n = 0;
    __device__ __forceinline__ void add(uint32_t col, uint32_t cnt) {
        s[0] += (col & 0xFFu) * cnt;
        s[1] += ((col >> 8) & 0xFFu) * cnt;
        s[2] += ((col >> 16) & 0xFFu) * cnt;
        s[3] += (col >> 24) * cnt;
        n += cnt;
    }
    __device__ __forceinline__ void sums(uint32_t &s0, uint32_t &s1, uint32_t &s2,
                                         uint32_t &s3) const {
        s0 = s[0];
        s1 = s[1];
        s2 = s[2];
        s3 = s[3];
    }
};

// Round-half-up quotient (s + n/2) / n for n >= 1 via a multiply-high:
// floor(y / n) == umulhi(y, floor((2^32 - 1) / n) + 1) for every n in
// [2, 961] and y <= 255 n + n / 2 (checked exhaustively); n == 1 is y.
__device__ __forceinline__ uint32_t div_round(uint32_t s, uint32_t n, uint32_t m) {
    const uint32_t y = s + (n >> 1);
    return n == 1 ? y : __umulhi(y, m);
}

template <bool F32, int R, typename Acc>
__device__ __forceinline__ void vote_store(const FrameArgs &a, const Acc &acc, int gx, int gy) {
    uint32_t s0, s1, s2, s3;
    acc.sums(s0, s1, s2, s3);
    const uint32_t n = acc.n;
    if constexpr (F32) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n) {
            const float dn = (float)(255u * n);
            o = make_float4(__fdiv_rn((float)s0, dn), __fdiv_rn((float)s1, dn),
                            __fdiv_rn((float)s2, dn), __fdiv_rn((float)s3, dn));
        }
        a.f32_out[(int64_t)gy * a.W + gx] = o;
    } else {
        uint32_t o = 0;
        if (n) {
            // a full window (the common case) divides by a constant
            constexpr uint32_t kFull = (2 * R + 1) * (2 * R + 1);
            const uint32_t m = n == kFull ? 0xFFFFFFFFu / kFull + 1u : 0xFFFFFFFFu / n + 1u;
            o = div_round(s0, n, m) | (div_round(s1, n, m) << 8) | (div_round(s2, n, m) << 16) |
                (div_round(s3, n, m) << 24);
        }
        a.rgba_out[(int64_t)gy * a.W + gx] = o;
    }
}

// Full-window vote of the listed pixels.  Along a window row, taps whose A
// steps by exactly one pixel form a run sharing one source position
// v = A(n) - o, so a run contributes len * C_S[v] with a single gather.  A
// row's run breaks come from the stored step bits E.  Pass 1 sums every
// listed pixel as if each window row had at most two runs (branch-free: two
// gathers per row) and compacts the pixels where some row has more breaks
// (junctions of chunks, frame borders) into a second list; pass 2 sums those
// tap by tap.  Every lane of a warp runs pass 1's loop the same number of
// times.  Pass 1 reads the calling warp's own list (no block barrier before
// it); pass 2 takes the block's complex pixels together (they are few).
template <int R, bool F32>
__device__ __forceinline__ void vote_slow_list(const FrameArgs &a, const uint32_t *A,
                                               const uint32_t *E, const uint16_t *slow,
                                               int n_slow, uint16_t *cplx, int *cplx_cnt,
                                               int x0, int y0) {
    constexpr int RW = kTW + 2 * R;
    constexpr bool kPacked = (2 * R + 1) * (2 * R + 1) * 255 < 65536;
    constexpr uint32_t kBreakMask = (2 * R >= 32) ? 0xFFFFFFFFu : ((1u << (2 * R)) - 1u);
    const uint32_t *style32 = reinterpret_cast<const uint32_t *>(a.style);
    const int sstride = a.style_stride_px;
    auto tap = [&](VoteAcc<kPacked> &acc, const uint32_t *row, int tx, int col, int oy,
                   uint32_t len) {
        const uint32_t c = row[col];
        const uint32_t v = c - (uint32_t)((col - tx - R) + (oy << 16));
        const uint32_t vx = v & 0xFFFFu, vy = v >> 16;
        // an out-of-target tap (kInvalid) lands out of the source here
        const bool ok = len != 0u && vx < (uint32_t)a.Ws && vy < (uint32_t)a.Hs;
        const uint32_t colr = ok ? __ldg(style32 + (vy * (uint32_t)sstride + vx)) : 0u;
        acc.add(colr, ok ? len : 0u);
    };
    const int lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < n_slow; j0 += 32) {
        const int j = j0 + lane;
        const bool act = j < n_slow;
        const int k = act ? slow[j] : 0;
        const int tx = k % kTW, ty = k / kTW;
        bool complex_row = false;
        if (act) {
            VoteAcc<kPacked> acc;
#pragma unroll
            for (int oy = -R; oy <= R; ++oy) {
                const int ry = ty + R + oy;
                const uint32_t *row = A + ry * RW;
                const uint32_t *e = E + ry * 4;
                const int b = tx + 1, w = b >> 5;
                const uint32_t m = ~__funnelshift_r(e[w], e[w + 1], b & 31) & kBreakMask;
                const int pc = __popc(m);
                complex_row |= pc > 1;
                const int j1 = pc ? __ffs(m) - 1 : 2 * R;
                tap(acc, row, tx, tx, oy, (uint32_t)(j1 + 1));
                tap(acc, row, tx, min(tx + j1 + 1, tx + 2 * R), oy,
                    pc == 1 ? (uint32_t)(2 * R - j1) : 0u);
            }
            if (!complex_row) vote_store<F32, R>(a, acc, x0 + tx, y0 + ty);
        }
        list_push(act && complex_row, k, cplx, cplx_cnt);
    }
    __syncthreads();
    const int n_cplx = *cplx_cnt;
    for (int j = threadIdx.x; j < n_cplx; j += kThreads) {
        const int k = cplx[j];
        const int tx = k % kTW, ty = k / kTW;
        VoteAcc<kPacked> acc;
        for (int oy = -R; oy <= R; ++oy) {
            const uint32_t *row = A + (ty + R + oy) * RW;
#pragma unroll
            for (int ox = 0; ox <= 2 * R; ++ox) tap(acc, row, tx, tx + ox, oy, 1u);
        }
        vote_store<F32, R>(a, acc, x0 + tx, y0 + ty);
    }
}

// bits [j, j + 64) of the 128-bit value hi:lo
__device__ __forceinline__ uint64_t shr128(uint64_t lo, uint64_t hi, int j) {
    return j == 0 ? lo : ((lo >> j) | (hi << (64 - j)));
}

template <int R, bool F32>
__device__ __forceinline__ void vote_tile(const FrameArgs &a, const SmemLayout &L, int x0,
                                          int y0, const uint32_t *A, unsigned char *smem) {
    constexpr int RW = kTW + 2 * R, RH = kTH + 2 * R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *hu_row = reinterpret_cast<uint64_t *>(smem + L.off_masks);
    uint64_t *v_row = hu_row + RH;
    uint32_t *E_row = reinterpret_cast<uint32_t *>(v_row + RH);  // 4 words per region row
    // each warp lists the pixels of its own output rows: 8 slots x 32 lanes
    constexpr int kWarpList = kTH / kWarps * 2 * 32;
    uint16_t *slow = reinterpret_cast<uint16_t *>(smem + L.off_list0) + warp * kWarpList;
    uint16_t *cplx = reinterpret_cast<uint16_t *>(smem + L.off_list1);
    int *cplx_cnt = reinterpret_cast<int *>(smem + L.off_cnt) + 3;
    const uint32_t *style32 = reinterpret_cast<const uint32_t *>(a.style);
    const int sstride = a.style_stride_px;

    if (threadIdx.x == 0) *cplx_cnt = 0;
    if constexpr (R > 0) {
        // per region row: E bit x <=> A[x] == A[x-1] + 1 (both valid);
        // hu bit tx <=> E bits tx+1 .. tx+2R all set (columns tx..tx+2R form
        // one horizontal translation); v bit tx <=> A[ry][tx+R] == A[ry-1][tx+R]
        // one row down (both valid)
        for (int ry = warp; ry < RH; ry += kWarps) {
            const uint32_t *row = A + ry * RW;
            uint32_t e[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int x = c * 32 + lane;
                bool bit = false;
                if (x >= 1 && x < RW) {
                    const uint32_t cur = row[x], prv = row[x - 1];
                    bit = cur == prv + 1u;  // never true next to kInvalid
                }
                e[c] = __ballot_sync(0xFFFFFFFFu, bit);
            }
            const uint64_t lo = (uint64_t)e[0] | ((uint64_t)e[1] << 32), hi = e[2];
            uint64_t hu = ~0ull;
#pragma unroll
            for (int j = 1; j <= 2 * R; ++j) hu &= shr128(lo, hi, j);
            uint32_t v[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int x = c * 32 + lane + R;
                bool bit = false;
                if (ry >= 1) {
                    const uint32_t cur = row[x], up = row[x - RW];
                    bit = cur == up + 0x10000u;
                }
                v[c] = __ballot_sync(0xFFFFFFFFu, bit);
            }
            if (lane == 0) {
                hu_row[ry] = hu;
                v_row[ry] = (uint64_t)v[0] | ((uint64_t)v[1] << 32);
                E_row[4 * ry + 0] = e[0];
                E_row[4 * ry + 1] = e[1];
                E_row[4 * ry + 2] = e[2];
                E_row[4 * ry + 3] = 0u;
            }
        }
    }
    __syncthreads();
    // output rows: warp w takes rows w, w + 8, ...; a uniform window copies
    constexpr int kRowsPerWarp = kTH / kWarps;
    uint32_t col[kRowsPerWarp][2];
    bool uni[kRowsPerWarp][2], need[kRowsPerWarp][2];
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
        const int ty = warp + q * kWarps;
        uint64_t U = ~0ull;
        if constexpr (R > 0) {
            // lane j < 2R + 1 brings window row ty + j; one AND-reduction per half
            uint64_t m = ~0ull;
            if (lane <= 2 * R) m = hu_row[ty + lane] & (lane > 0 ? v_row[ty + lane] : ~0ull);
            U = (uint64_t)__reduce_and_sync(0xFFFFFFFFu, (uint32_t)m) |
                ((uint64_t)__reduce_and_sync(0xFFFFFFFFu, (uint32_t)(m >> 32)) << 32);
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int tx = c * 32 + lane;
            const int gx = x0 + tx, gy = y0 + ty;
            uni[q][c] = need[q][c] = false;
            col[q][c] = 0;
            if (gx < a.W && gy < a.H) {
                const uint32_t cc = A[(ty + R) * RW + tx + R];
                const int cx = (int)(cc & 0xFFFFu), cy = (int)(cc >> 16);
                const bool ok = ((U >> tx) & 1ull) && cx < a.Ws && cy < a.Hs;
                uni[q][c] = ok;
                need[q][c] = !ok;
                if (ok) col[q][c] = __ldg(style32 + ((uint32_t)cy * (uint32_t)sstride + (uint32_t)cx));
            }
        }
    }
    const unsigned lt = (1u << lane) - 1u;
    int n_slow = 0;
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
        const int ty = warp + q * kWarps;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int tx = c * 32 + lane;
            const int k = ty * kTW + tx;
            if (uni[q][c]) {
                if constexpr (F32) {
                    a.f32_out[(int64_t)(y0 + ty) * a.W + x0 + tx] = rgba_f32(col[q][c]);
                } else {
                    a.rgba_out[(int64_t)(y0 + ty) * a.W + x0 + tx] = col[q][c];
                }
            }
            const unsigned nm = __ballot_sync(0xFFFFFFFFu, need[q][c]);
            if (need[q][c]) slow[n_slow + __popc(nm & lt)] = (uint16_t)k;
            n_slow += __popc(nm);
        }
    }
    __syncwarp();
    vote_slow_list<R, F32>(a, A, E_row, slow, n_slow, cplx, cplx_cnt, x0, y0);
}

// One 64 x 32 output tile (tile_x, tile_y) of one frame.
template <int C, int B, int MODE, int R>
__device__ __forceinline__ void frame_tile(const FrameArgs &a, const SmemLayout &L, int tile_x,
                                           int tile_y, unsigned char *smem) {
    const int x0 = tile_x * kTW, y0 = tile_y * kTH;
    uint8_t *bytes = smem + L.off_bytes;
    assign_region<C, B, R>(a, L, x0 - R, y0 - R, smem, MODE == kAssign ? bytes : nullptr);
    const uint32_t *A = reinterpret_cast<const uint32_t *>(smem + L.off_A);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (MODE == kAssign) {
        for (int ty = warp; ty < kTH; ty += kWarps) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int tx = c * 32 + lane;
                const int gx = x0 + tx, gy = y0 + ty;
                if (gx < a.W && gy < a.H) {
                    a.assign_out[(int64_t)gy * a.W + gx] = A[ty * kTW + tx];
                    if (a.level_out) a.level_out[(int64_t)gy * a.W + gx] = bytes[ty * kTW + tx];
                }
            }
        }
    } else {
        vote_tile<R, false>(a, L, x0, y0, A, smem);
    }
}

// CTAs per SM the kernels are compiled for: four (64 registers a thread) hide
// more of each tile's load latency than three with 80 registers; five (48)
// spill too much.
__host__ __device__ constexpr int min_ctas(int) { return 4; }

template <int C, int B, int MODE, int R>
__global__ void __launch_bounds__(kThreads, min_ctas(R))
    frame_kernel(const FrameArgs a, const SmemLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    frame_tile<C, B, MODE, R>(a, L, blockIdx.x, blockIdx.y, smem);
}

// Many frames in one launch: block b stylises tile b - tile_start[k] of the
// frame k with tile_start[k] <= b < tile_start[k + 1].  Frames may differ in
// size, exemplar, levels, threshold and seed; they share the guide format and
// the blend radius.  One launch lets the tiles of later frames fill the SMs
// while the last tiles of earlier frames finish.
constexpr int kMaxBatch = 128;

struct BatchArgs {
    int n;
    int tile_start[kMaxBatch + 1];
    int tiles_x[kMaxBatch];
    FrameArgs f[kMaxBatch];
};

// Tile t of a batch: the frame k with tile_start[k] <= t < tile_start[k + 1].
template <int C, int B, int R>
__device__ __forceinline__ void batch_tile(const BatchArgs &b, const SmemLayout &L, int t,
                                           unsigned char *smem) {
    int lo = 0, hi = b.n - 1;  // last frame whose first tile is <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.tile_start[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const FrameArgs a = b.f[lo];  // register copy: field reads become plain operands
    const int lt = t - b.tile_start[lo];
    frame_tile<C, B, kStylize, R>(a, L, lt % b.tiles_x[lo], lt / b.tiles_x[lo], smem);
}

template <int C, int B, int R>
__global__ void __launch_bounds__(kThreads, min_ctas(R))
    batch_kernel(const __grid_constant__ BatchArgs b, const SmemLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    batch_tile<C, B, R>(b, L, (int)blockIdx.x, smem);
}

// Work queues of persistent batch launches: CTAs take the next tile from
// `next` until the batch is exhausted; the last CTA to leave clears the queue
// for the next launch (CUDA graph replays included).  A launch uses slot
// `slot`; launches in flight at the same time need distinct slots.  No CTA
// waits on another.
struct TileQueue {
    unsigned int next, done;
};
constexpr int kQueueSlots = 64;
static __device__ TileQueue g_tile_queues[kQueueSlots];

template <int C, int B, int R>
__global__ void __launch_bounds__(kThreads, min_ctas(R))
    batch_kernel_persistent(const __grid_constant__ BatchArgs b, const SmemLayout L, int slot) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int tile;
    TileQueue &q = g_tile_queues[slot];
    const int n_tiles = b.tile_start[b.n];
    for (;;) {
        if (threadIdx.x == 0) tile = (int)atomicAdd(&q.next, 1u);
        __syncthreads();
        const int t = tile;
        __syncthreads();  // every thread has read `tile` before it is overwritten
        if (t >= n_tiles) break;
        batch_tile<C, B, R>(b, L, t, smem);
        __syncthreads();  // the tile's shared memory is free before the next tile writes it
    }
    if (threadIdx.x == 0) {
        // this CTA takes no more tiles; the last one out resets the queue
        if (atomicAdd(&q.done, 1u) == gridDim.x - 1) {
            atomicExch(&q.next, 0u);
            atomicExch(&q.done, 0u);
        }
    }
}

template <bool F32, int R>
__global__ void __launch_bounds__(kThreads) blend_kernel(const FrameArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int RW = kTW + 2 * R, NR = RW * (kTH + 2 * R);
    const SmemLayout L = smem_layout(R, 0);
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int rx0 = x0 - R, ry0 = y0 - R;
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.off_A);
#pragma unroll 4
    for (int i = threadIdx.x; i < NR; i += kThreads) {
        const int gx = rx0 + i % RW, gy = ry0 + i / RW;
        const bool inside = gx >= 0 && gy >= 0 && gx < a.W && gy < a.H;
        A[i] = inside ? __ldg(a.assign_in + (int64_t)gy * a.W + gx) : kInvalid;
    }
    __syncthreads();
    vote_tile<R, F32>(a, L, x0, y0, A, smem);
}

// Raises a kernel's dynamic shared-memory limit once per (kernel, device);
// later launches of no larger size skip the runtime call.  The cache is keyed
// by the kernel itself (one static per template instance).
template <auto Kernel>
cudaError_t ensure_smem(size_t smem) {
    constexpr int kMaxDev = 64;
    static std::atomic<uint32_t> done[kMaxDev] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t need = (uint32_t)smem;
    if (dev < kMaxDev && done[dev].load(std::memory_order_relaxed) >= need) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess && dev < kMaxDev) {
        uint32_t cur = done[dev].load();
        while (cur < need && !done[dev].compare_exchange_weak(cur, need)) {
        }
    }
    return e;
}

template <auto Kernel, typename... Args>
cudaError_t launch_tiles(size_t smem, int W, int H, cudaStream_t s, const Args &...args) {
    cudaError_t e = ensure_smem<Kernel>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
    Kernel<<<grid, kThreads, smem, s>>>(args...);
    return cudaGetLastError();
}

template <int C, int B, int R>
cudaError_t launch_stylize_r(const FrameArgs &a, cudaStream_t s) {
    const SmemLayout L = smem_layout(R, a.levels);
    return launch_tiles<frame_kernel<C, B, kStylize, R>>(L.total, a.W, a.H, s, a, L);
}

// CTAs of a persistent launch: as many as fit on the device at once (cached
// per kernel, device and shared-memory size), at most one per tile.
template <auto Kernel>
int persistent_grid(size_t smem, int n_tiles) {
    constexpr int kMaxDev = 64;
    static std::atomic<uint64_t> cache[kMaxDev] = {};  // smem << 32 | CTAs
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t c = dev < kMaxDev ? cache[dev].load(std::memory_order_relaxed) : 0;
    int ctas = 0;
    if (c && (c >> 32) == smem) {
        ctas = (int)(c & 0xFFFFFFFFu);
    } else {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, kThreads, smem);
        ctas = max(1, sms * max(per_sm, 1));
        if (dev < kMaxDev) cache[dev].store(((uint64_t)smem << 32) | (uint32_t)ctas);
    }
    return min(ctas, n_tiles);
}

template <int C, int B, int R>
cudaError_t launch_batch_r(const BatchArgs &b, int max_levels, bool persistent, cudaStream_t s) {
    // one layout (for the deepest frame) serves every tile of the launch
    const SmemLayout L = smem_layout(R, max_levels);
    const int n_tiles = b.tile_start[b.n];
    if (!persistent) {
        cudaError_t e = ensure_smem<batch_kernel<C, B, R>>(L.total);
        if (e != cudaSuccess) return e;
        batch_kernel<C, B, R><<<n_tiles, kThreads, L.total, s>>>(b, L);
        return cudaGetLastError();
    }
    cudaError_t e = ensure_smem<batch_kernel_persistent<C, B, R>>(L.total);
    if (e != cudaSuccess) return e;
    static std::atomic<unsigned> next_slot{0};
    const int slot = (int)(next_slot.fetch_add(1u) % kQueueSlots);
    const int grid = persistent_grid<batch_kernel_persistent<C, B, R>>(L.total, n_tiles);
    batch_kernel_persistent<C, B, R><<<grid, kThreads, L.total, s>>>(b, L, slot);
    return cudaGetLastError();
}

// Launches the batch kernel of guide format <C, B> for blend radius r.
template <int C, int B>
cudaError_t launch_batch(const BatchArgs &b, int r, int max_levels, bool persistent,
                         cudaStream_t s) {
    switch (r) {
        case 0: return launch_batch_r<C, B, 0>(b, max_levels, persistent, s);
        case 1: return launch_batch_r<C, B, 1>(b, max_levels, persistent, s);
        case 2: return launch_batch_r<C, B, 2>(b, max_levels, persistent, s);
        case 3: return launch_batch_r<C, B, 3>(b, max_levels, persistent, s);
        case 4: return launch_batch_r<C, B, 4>(b, max_levels, persistent, s);
        case 5: return launch_batch_r<C, B, 5>(b, max_levels, persistent, s);
        case 6: return launch_batch_r<C, B, 6>(b, max_levels, persistent, s);
        case 7: return launch_batch_r<C, B, 7>(b, max_levels, persistent, s);
    }
    return cudaErrorInvalidValue;
}

// Launches the frame kernel of guide format <C, B> in the given mode.
template <int C, int B>
cudaError_t launch_frame(int mode, const FrameArgs &a, cudaStream_t s) {
    if (mode == kAssign) {
        const SmemLayout L = smem_layout(0, a.levels);
        return launch_tiles<frame_kernel<C, B, kAssign, 0>>(L.total, a.W, a.H, s, a, L);
    }
    switch (a.radius) {
        case 0: return launch_stylize_r<C, B, 0>(a, s);
        case 1: return launch_stylize_r<C, B, 1>(a, s);
        case 2: return launch_stylize_r<C, B, 2>(a, s);
        case 3: return launch_stylize_r<C, B, 3>(a, s);
        case 4: return launch_stylize_r<C, B, 4>(a, s);
        case 5: return launch_stylize_r<C, B, 5>(a, s);
        case 6: return launch_stylize_r<C, B, 6>(a, s);
        case 7: return launch_stylize_r<C, B, 7>(a, s);
    }
    return cudaErrorInvalidValue;
}

// per-format launchers, one translation unit each (sb_frame_c<C>b<B>.cu)
// per-format batch launchers, defined next to the frame launchers
cudaError_t launch_batch_c1b8(const BatchArgs &b, int r, int max_levels, bool persistent,
                              cudaStream_t s);
cudaError_t launch_batch_c2b8(const BatchArgs &b, int r, int max_levels, bool persistent,
                              cudaStream_t s);
cudaError_t launch_batch_c3b8(const BatchArgs &b, int r, int max_levels, bool persistent,
                              cudaStream_t s);
cudaError_t launch_batch_c4b8(const BatchArgs &b, int r, int max_levels, bool persistent,
                              cudaStream_t s);
cudaError_t launch_batch_c1b16(const BatchArgs &b, int r, int max_levels, bool persistent,
                              cudaStream_t s);
cudaError_t launch_batch_c2b16(const BatchArgs &b, int r, int max_levels, bool persistent,
                              cudaStream_t s);
cudaError_t launch_frame_c1b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_c2b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_c3b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_c4b8(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_c1b16(int mode, const FrameArgs &a, cudaStream_t s);
cudaError_t launch_frame_c2b16(int mode, const FrameArgs &a, cudaStream_t s);

}  // namespace sb
