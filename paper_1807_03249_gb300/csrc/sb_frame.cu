// Per-frame StyleBlit kernels: Algorithm 2 (ParallelStyleBlit) with the
// coordinate transfer and voting step of Section 3.2.
//
// One CTA owns a 64 x 32 output tile.  For the fused path it computes the
// assignment A of the tile plus a halo of r pixels (the vote window) in shared
// memory, so A never touches device memory.  The work is arranged so every
// thread keeps several independent global loads in flight (the method is a
// chain of gathers: G_T[q] -> table -> G_S[s] -> C_S[...]):
//
//   phase 0  target guide of the region -> smem (one packed uint32 per
//            pixel), issued as independent loads; at the same time the seed
//            cells of all levels >= 3 are built (levels 2 and 1, which have
//            many cells, are built only if a pixel still needs them).  A cell
//            is: jitter hash -> seed q clamped into the target -> G_T[q] ->
//            table lookup u*(q); it keeps (-2 q, |q|^2, u*) in region-centred
//            coordinates.
//   levels   for l = L..1 while pixels are pending: every pending pixel takes
//            the nearest seed of its 3 x 3 cells (x outer, y inner, strict <)
//            by minimising |q|^2 - 2 q.p, which orders seeds exactly like
//            |q - p|^2; it forms s = u* + (p - q) and accepts it when s lies in
//            the source and |G_S[s] - G_T[p]|^2 <= t (level 1 always accepts,
//            s clamped into the source).  Pixels are processed in batches of
//            four per thread, gathers issued before any result is used;
//            rejected pixels are compacted into the next pending list.
//   vote     a window whose A values are all one translation of p (checked
//            separably: rows, then columns) votes C_S[A(p)] exactly, so it is
//            a plain copy; the other pixels (chunk boundaries, frame borders)
//            are compacted and summed over the full window (unrolled per
//            radius) with integer sums and round-half-up division.
//   store    the tile leaves shared memory with coalesced 32-bit stores.
#include <atomic>
#include <climits>
#include <cstdio>

#include "sb_internal.cuh"

namespace sb {

constexpr int kTW = 64;
constexpr int kTH = 32;
constexpr int kThreads = 256;
constexpr int kBatch = 4;                 // pixels per thread per batch
constexpr uint32_t kPending = 0xFFFFFFFEu;  // in-target pixel without an assignment yet
constexpr int kEagerMinLevel = 3;         // levels >= this get their cells in phase 0

enum Mode { kAssign = 0, kStylize = 1 };

struct FrameArgs {
    const uint8_t *tgt;
    int64_t tgt_stride;
    int W, H;
    const uint8_t *src;
    int64_t src_stride;
    int Ws, Hs;
    const uint32_t *lut;
    int key_bits;
    const uint8_t *style;
    int64_t style_stride;
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
__host__ __device__ inline int cells_bound(int RW, int RH, int l) {
    return (((RW - 1) >> l) + 4) * (((RH - 1) >> l) + 4);
}

struct SmemLayout {
    int RW, RH, NR, NC;
    size_t off_cells, off_gt, off_A, off_list0, off_list1, off_bytes, off_cnt, total;
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
    s.off_list0 = o;
    o += sizeof(uint16_t) * (size_t)s.NR;
    s.off_list1 = o;
    o += sizeof(uint16_t) * (size_t)s.NR;
    s.off_bytes = o;
    o += (size_t)s.NR;
    o = (o + 15) & ~(size_t)15;
    s.off_cnt = o;
    o += 16;
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

// Geometry of the seed cells of level l for the clamped region [xa, xb] x [ya, yb].
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

// Builds the cells of levels l_hi down to l_lo into cells[base_hi...]; the
// levels are stacked from l_hi downwards.
template <int C, int B>
__device__ __forceinline__ void build_cells(const FrameArgs &a, int4 *cells, int l_hi, int l_lo,
                                            int base_hi, int xa, int xb, int ya, int yb,
                                            int cxo, int cyo) {
    using F = GuideFmt<C, B>;
    int total = 0;
    for (int l = l_hi; l >= l_lo; --l) {
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        total += g.ncx * g.ncy;
    }
#pragma unroll 2
    for (int k = threadIdx.x; k < total; k += kThreads) {
        // locate the level of flat index k (few levels, short scan)
        int l = l_hi, off = 0;
        LevelCells g = level_cells(l, xa, xb, ya, yb);
        while (k >= off + g.ncx * g.ncy) {
            off += g.ncx * g.ncy;
            --l;
            g = level_cells(l, xa, xb, ya, yb);
        }
        const int ci = k - off;
        const int h = 1 << l;
        const int bx = g.cx0 + ci % g.ncx, by = g.cy0 + ci / g.ncx;
        const uint32_t hsh = cell_hash(level_key(a.seed, l), bx, by);
        const int ox = (int)(((hsh & 0xFFFFu) * (uint32_t)h) >> 16);
        const int oy = (int)(((hsh >> 16) * (uint32_t)h) >> 16);
        const int sx = min(max(bx * h + ox, 0), a.W - 1);
        const int sy = min(max(by * h + oy, 0), a.H - 1);
        const uint32_t u = __ldg(a.lut + F::key(F::load(a.tgt, a.tgt_stride, sx, sy), a.key_bits));
        const int qx = sx - cxo, qy = sy - cyo;
        cells[base_hi + k] = make_int4(-2 * qx, -2 * qy, qx * qx + qy * qy, (int)u);
    }
}

// ---------------------------------------------------------------------------
// assignment of the region held in shared memory (Algorithm 2)
// ---------------------------------------------------------------------------
template <int C, int B>
__device__ __forceinline__ void assign_region(const FrameArgs &a, const SmemLayout &L, int rx0,
                                              int ry0, unsigned char *smem, uint8_t *lev) {
    using F = GuideFmt<C, B>;
    int4 *cells = reinterpret_cast<int4 *>(smem + L.off_cells);
    uint32_t *gt = reinterpret_cast<uint32_t *>(smem + L.off_gt);
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.off_A);
    uint16_t *const list0 = reinterpret_cast<uint16_t *>(smem + L.off_list0);
    uint16_t *const list1 = reinterpret_cast<uint16_t *>(smem + L.off_list1);
    int *cnt = reinterpret_cast<int *>(smem + L.off_cnt);
    const int tid = threadIdx.x;

    // clamped region extent (every in-target region pixel lies inside it)
    const int xa = max(rx0, 0), xb = min(rx0 + L.RW, a.W) - 1;
    const int ya = max(ry0, 0), yb = min(ry0 + L.RH, a.H) - 1;
    const int cxo = rx0 + L.RW / 2, cyo = ry0 + L.RH / 2;
    const uint32_t t32 = a.threshold > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)a.threshold;
    const int L_top = a.levels;
    const int eager_lo = L_top <= kEagerMinLevel ? 1 : kEagerMinLevel;

    // phase 0: target guide of the region, cells of the coarse levels
    if (tid == 0) {
        cnt[0] = 0;
        cnt[1] = 0;
    }
#pragma unroll 4
    for (int i = tid; i < L.NR; i += kThreads) {
        const int gx = rx0 + i % L.RW, gy = ry0 + i / L.RW;
        const bool inside = gx >= 0 && gy >= 0 && gx < a.W && gy < a.H;
        gt[i] = inside ? F::load(a.tgt, a.tgt_stride, gx, gy) : 0u;
        A[i] = inside ? kPending : kInvalid;
    }
    build_cells<C, B>(a, cells, L_top, eager_lo, 0, xa, xb, ya, yb, cxo, cyo);
    __syncthreads();

    int cur = 0;
    int n_pend = L.NR;  // the top level scans the whole region
    int base = 0;       // first cell of the current level
    for (int l = L_top; l >= 1 && n_pend > 0; --l) {
        const LevelCells g = level_cells(l, xa, xb, ya, yb);
        if (l == kEagerMinLevel - 1 && eager_lo > 1) {
            // a pixel still needs the fine levels: build levels 2 and 1 now
            build_cells<C, B>(a, cells, l, 1, base, xa, xb, ya, yb, cxo, cyo);
            __syncthreads();
        }
        const int nxt = cur ^ 1;
        const uint16_t *list_cur = cur ? list1 : list0;
        uint16_t *list_nxt = cur ? list0 : list1;
        const bool top = l == L_top;
        for (int j0 = 0; j0 < n_pend; j0 += kThreads * kBatch) {
            int idx[kBatch];
            int sxv[kBatch], syv[kBatch];
            uint32_t gsv[kBatch];
            bool act[kBatch], inb[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int j = j0 + u * kThreads + tid;
                act[u] = j < n_pend;
                int i = 0;
                if (act[u]) {
                    i = top ? j : list_cur[j];
                    if (top) act[u] = A[i] == kPending;
                }
                idx[u] = i;
                inb[u] = false;
                gsv[u] = 0;
                sxv[u] = 0;
                syv[u] = 0;
                if (act[u]) {
                    const int rx = i % L.RW, ry = i / L.RW;
                    const int gx = rx0 + rx, gy = ry0 + ry;
                    const int prx = rx - L.RW / 2, pry = ry - L.RH / 2;
                    const int lcx = (gx >> l) - g.cx0, lcy = (gy >> l) - g.cy0;
                    int best_e = INT_MAX, best_c = 0;
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
#pragma unroll
                        for (int dy = -1; dy <= 1; ++dy) {
                            const int c = base + (lcy + dy) * g.ncx + (lcx + dx);
                            const int4 cl = cells[c];
                            const int e = cl.z + cl.x * prx + cl.y * pry;
                            if (e < best_e) {
                                best_e = e;
                                best_c = c;
                            }
                        }
                    }
                    const int4 cl = cells[best_c];
                    int sx = (int)((uint32_t)cl.w & 0xFFFFu) + prx + (cl.x >> 1);
                    int sy = (int)((uint32_t)cl.w >> 16) + pry + (cl.y >> 1);
                    if (l > 1) {
                        inb[u] = (unsigned)sx < (unsigned)a.Ws && (unsigned)sy < (unsigned)a.Hs;
                        if (inb[u]) gsv[u] = F::load(a.src, a.src_stride, sx, sy);
                    } else {
                        sx = min(max(sx, 0), a.Ws - 1);
                        sy = min(max(sy, 0), a.Hs - 1);
                    }
                    sxv[u] = sx;
                    syv[u] = sy;
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                bool acc = false;
                if (act[u]) {
                    if (l > 1) {
                        if (inb[u]) {
                            const uint64_t d = F::dist(gsv[u], gt[idx[u]]);
                            if constexpr (B == 8) acc = (uint32_t)d <= t32;
                            else acc = d <= a.threshold;
                        }
                    } else {
                        acc = true;
                    }
                    if (acc) {
                        A[idx[u]] = (uint32_t)sxv[u] | ((uint32_t)syv[u] << 16);
                        if (lev) lev[idx[u]] = (uint8_t)l;
                    }
                }
                list_push(act[u] && !acc, idx[u], list_nxt, &cnt[nxt]);
            }
        }
        __syncthreads();
        n_pend = cnt[nxt];
        // cnt[cur] was last read before the barrier above; it becomes the next
        // level's output counter, and the barrier below publishes the reset
        // before any thread appends to it
        if (tid == 0) cnt[cur] = 0;
        base += g.ncx * g.ncy;
        __syncthreads();
        cur = nxt;
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

template <bool F32>
__device__ __forceinline__ void vote_store(const FrameArgs &a, uint32_t s0, uint32_t s1,
                                           uint32_t s2, uint32_t s3, uint32_t n, int gx, int gy,
                                           int k, uint32_t *out_tile) {
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
            const uint32_t hn = n >> 1;
            o = ((s0 + hn) / n) | (((s1 + hn) / n) << 8) | (((s2 + hn) / n) << 16) |
                (((s3 + hn) / n) << 24);
        }
        out_tile[k] = o;
    }
}

// Full-window vote of the listed pixels; R > 0 is the radius known at compile
// time (loads unrolled), R < 0 means the runtime radius a.radius.
template <int R, bool F32>
__device__ __forceinline__ void vote_slow_list(const FrameArgs &a, const SmemLayout &L,
                                               const uint32_t *A, const uint16_t *slow,
                                               int n_slow, int x0, int y0, uint32_t *out_tile) {
    const uint32_t *style32 = reinterpret_cast<const uint32_t *>(a.style);
    const int64_t sstride = a.style_stride >> 2;
    const int r = R >= 0 ? R : a.radius;
    for (int j = threadIdx.x; j < n_slow; j += kThreads) {
        const int k = slow[j];
        const int tx = k % kTW, ty = k / kTW;
        const int i = (ty + r) * L.RW + tx + r;
        uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, n = 0;
        if constexpr (R >= 0) {
#pragma unroll
            for (int oy = -R; oy <= R; ++oy) {
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    const uint32_t c = A[i + oy * L.RW + ox];
                    const int vx = (int)(c & 0xFFFFu) - ox, vy = (int)(c >> 16) - oy;
                    const bool ok = c != kInvalid && (unsigned)vx < (unsigned)a.Ws &&
                                    (unsigned)vy < (unsigned)a.Hs;
                    const uint32_t col = ok ? __ldg(style32 + (int64_t)vy * sstride + vx) : 0u;
                    s0 += col & 0xFFu;
                    s1 += (col >> 8) & 0xFFu;
                    s2 += (col >> 16) & 0xFFu;
                    s3 += col >> 24;
                    n += ok ? 1u : 0u;
                }
            }
        } else {
            for (int oy = -r; oy <= r; ++oy) {
                for (int ox = -r; ox <= r; ++ox) {
                    const uint32_t c = A[i + oy * L.RW + ox];
                    if (c == kInvalid) continue;
                    const int vx = (int)(c & 0xFFFFu) - ox, vy = (int)(c >> 16) - oy;
                    if ((unsigned)vx >= (unsigned)a.Ws || (unsigned)vy >= (unsigned)a.Hs)
                        continue;
                    const uint32_t col = __ldg(style32 + (int64_t)vy * sstride + vx);
                    s0 += col & 0xFFu;
                    s1 += (col >> 8) & 0xFFu;
                    s2 += (col >> 16) & 0xFFu;
                    s3 += col >> 24;
                    n += 1;
                }
            }
        }
        vote_store<F32>(a, s0, s1, s2, s3, n, x0 + tx, y0 + ty, k, out_tile);
    }
}

template <bool F32>
__device__ __forceinline__ void vote_tile(const FrameArgs &a, const SmemLayout &L, int x0,
                                          int y0, const uint32_t *A, uint8_t *hu,
                                          uint16_t *slow, int *slow_cnt, uint32_t *out_tile) {
    const int r = a.radius;
    const int tid = threadIdx.x;
    const uint32_t *style32 = reinterpret_cast<const uint32_t *>(a.style);
    const int64_t sstride = a.style_stride >> 2;

    // rows: does A step by exactly +1 in x across the 2r+1 columns around n?
    for (int k = tid; k < kTW * L.RH; k += kThreads) {
        const int tx = k % kTW, ry = k / kTW;
        const int i = ry * L.RW + tx + r;
        const uint32_t c = A[i];
        bool ok = c != kInvalid;
        for (int o = -r; o <= r; ++o) ok = ok && (A[i + o] == c + (uint32_t)o);
        hu[k] = ok ? 1 : 0;
    }
    if (tid == 0) *slow_cnt = 0;
    __syncthreads();
    // columns: a uniform window votes the copy C_S[A(p)]
    for (int k0 = 0; k0 < kTW * kTH; k0 += kThreads * kBatch) {
        uint32_t col[kBatch];
        bool uni[kBatch], need[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = k0 + u * kThreads + tid;
            const int tx = k % kTW, ty = k / kTW;
            const int gx = x0 + tx, gy = y0 + ty;
            uni[u] = false;
            need[u] = false;
            col[u] = 0;
            if (k < kTW * kTH && gx < a.W && gy < a.H) {
                const int i = (ty + r) * L.RW + tx + r;
                const uint32_t c = A[i];
                const int cx = (int)(c & 0xFFFFu), cy = (int)(c >> 16);
                bool ok = cx < a.Ws && cy < a.Hs;
                for (int o = -r; o <= r && ok; ++o)
                    ok = hu[(ty + r + o) * kTW + tx] && A[i + o * L.RW] == c + ((uint32_t)o << 16);
                uni[u] = ok;
                need[u] = !ok;
                if (ok) col[u] = __ldg(style32 + (int64_t)cy * sstride + cx);
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = k0 + u * kThreads + tid;
            if (uni[u]) {
                if constexpr (F32) {
                    const int gx = x0 + k % kTW, gy = y0 + k / kTW;
                    a.f32_out[(int64_t)gy * a.W + gx] = rgba_f32(col[u]);
                } else {
                    out_tile[k] = col[u];
                }
            }
            list_push(need[u], k, slow, slow_cnt);
        }
    }
    __syncthreads();
    const int n_slow = *slow_cnt;
    switch (r) {
        case 0: vote_slow_list<0, F32>(a, L, A, slow, n_slow, x0, y0, out_tile); break;
        case 1: vote_slow_list<1, F32>(a, L, A, slow, n_slow, x0, y0, out_tile); break;
        case 2: vote_slow_list<2, F32>(a, L, A, slow, n_slow, x0, y0, out_tile); break;
        case 3: vote_slow_list<3, F32>(a, L, A, slow, n_slow, x0, y0, out_tile); break;
        default: vote_slow_list<-1, F32>(a, L, A, slow, n_slow, x0, y0, out_tile); break;
    }
}

template <int C, int B, int MODE>
__global__ void __launch_bounds__(kThreads) frame_kernel(const FrameArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int r = MODE == kStylize ? a.radius : 0;
    const SmemLayout L = smem_layout(r, a.levels);
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int rx0 = x0 - r, ry0 = y0 - r;
    uint8_t *bytes = smem + L.off_bytes;
    assign_region<C, B>(a, L, rx0, ry0, smem, MODE == kAssign ? bytes : nullptr);
    const uint32_t *A = reinterpret_cast<const uint32_t *>(smem + L.off_A);
    if constexpr (MODE == kAssign) {
        for (int k = threadIdx.x; k < kTW * kTH; k += kThreads) {
            const int gx = x0 + k % kTW, gy = y0 + k / kTW;
            if (gx < a.W && gy < a.H) {
                a.assign_out[(int64_t)gy * a.W + gx] = A[k];
                if (a.level_out) a.level_out[(int64_t)gy * a.W + gx] = bytes[k];
            }
        }
    } else {
        // the target guide is no longer needed: its slot holds the output tile
        uint32_t *out_tile = reinterpret_cast<uint32_t *>(smem + L.off_gt);
        uint16_t *slow = reinterpret_cast<uint16_t *>(smem + L.off_list0);
        int *cnt = reinterpret_cast<int *>(smem + L.off_cnt);
        vote_tile<false>(a, L, x0, y0, A, bytes, slow, &cnt[2], out_tile);
        __syncthreads();
        for (int k = threadIdx.x; k < kTW * kTH; k += kThreads) {
            const int gx = x0 + k % kTW, gy = y0 + k / kTW;
            if (gx < a.W && gy < a.H) a.rgba_out[(int64_t)gy * a.W + gx] = out_tile[k];
        }
    }
}

template <bool F32>
__global__ void __launch_bounds__(kThreads) blend_kernel(const FrameArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(a.radius, 0);
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int rx0 = x0 - a.radius, ry0 = y0 - a.radius;
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.off_A);
#pragma unroll 4
    for (int i = threadIdx.x; i < L.NR; i += kThreads) {
        const int gx = rx0 + i % L.RW, gy = ry0 + i / L.RW;
        const bool inside = gx >= 0 && gy >= 0 && gx < a.W && gy < a.H;
        A[i] = inside ? __ldg(a.assign_in + (int64_t)gy * a.W + gx) : kInvalid;
    }
    __syncthreads();
    uint32_t *out_tile = reinterpret_cast<uint32_t *>(smem + L.off_gt);
    uint16_t *slow = reinterpret_cast<uint16_t *>(smem + L.off_list0);
    int *cnt = reinterpret_cast<int *>(smem + L.off_cnt);
    vote_tile<F32>(a, L, x0, y0, A, smem + L.off_bytes, slow, &cnt[2], out_tile);
    if constexpr (!F32) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTW * kTH; k += kThreads) {
            const int gx = x0 + k % kTW, gy = y0 + k / kTW;
            if (gx < a.W && gy < a.H) a.rgba_out[(int64_t)gy * a.W + gx] = out_tile[k];
        }
    }
}

// Raises a kernel's dynamic shared-memory limit once per (kernel, device);
// later launches of no larger size skip the driver call.  The cache is keyed
// by the kernel itself (one static per template instance).
template <auto Kernel>
static cudaError_t ensure_smem(size_t smem) {
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

template <auto Kernel>
static cudaError_t launch_tiles(size_t smem, int W, int H, cudaStream_t s, const FrameArgs &a) {
    cudaError_t e = ensure_smem<Kernel>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH);
    Kernel<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
struct FrameLaunch {
    const FrameArgs *a;
    cudaStream_t s;
    cudaError_t err = cudaSuccess;
    template <int C, int B>
    void operator()() {
        const SmemLayout L = smem_layout(MODE == kStylize ? a->radius : 0, a->levels);
        err = launch_tiles<frame_kernel<C, B, MODE>>(L.total, a->W, a->H, s, *a);
    }
};

// validation shared by sb_assign_chunks and sb_stylize
static sb_status check_frame(const sb_guide *tgt, const sb_guide *src, const sb_lut *lut,
                             int32_t levels) {
    sb_status st = check_guide(tgt, "tgt_guide", false);
    if (st != SB_OK) return st;
    if ((st = check_guide(src, "src_guide", true)) != SB_OK) return st;
    if (tgt->channels != src->channels || tgt->bits != src->bits)
        return fail(SB_ERR_INVALID_ARG, "target and source guides differ in channels or bits");
    if (!lut) return fail(SB_ERR_INVALID_ARG, "lut: NULL");
    if (lut->channels != src->channels || lut->bits != src->bits || lut->src_w != src->width ||
        lut->src_h != src->height)
        return fail(SB_ERR_INVALID_ARG, "lut was built for a different source guide format/size");
    if (levels < 1 || levels > kMaxLevels)
        return fail(SB_ERR_INVALID_ARG, "levels must be in [1, 12]");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != lut->device) return fail(SB_ERR_INVALID_ARG, "lut lives on another device");
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    return SB_OK;
}

static FrameArgs frame_args(const sb_guide *tgt, const sb_guide *src, const sb_lut *lut,
                            int32_t levels, uint64_t threshold, uint32_t seed) {
    FrameArgs a{};
    a.tgt = static_cast<const uint8_t *>(tgt->data);
    a.tgt_stride = tgt->row_stride;
    a.W = tgt->width;
    a.H = tgt->height;
    a.src = static_cast<const uint8_t *>(src->data);
    a.src_stride = src->row_stride;
    a.Ws = src->width;
    a.Hs = src->height;
    a.lut = lut->entries;
    a.key_bits = lut->key_bits;
    a.levels = levels;
    a.threshold = threshold;
    a.seed = seed;
    return a;
}

}  // namespace sb

using namespace sb;

extern "C" sb_status sb_assign_chunks(const sb_guide *tgt_guide, const sb_guide *src_guide,
                                      const sb_lut *lut, int32_t levels, uint64_t threshold,
                                      uint32_t seed, uint32_t *assign_out, uint8_t *level_out,
                                      sb_stream stream) {
    sb_status st = check_frame(tgt_guide, src_guide, lut, levels);
    if (st != SB_OK) return st;
    if ((int64_t)tgt_guide->width * tgt_guide->height == 0) return ok();
    if (!assign_out) return fail(SB_ERR_INVALID_ARG, "assign_out: NULL");
    if ((uintptr_t)assign_out % 4) return fail(SB_ERR_INVALID_ARG, "assign_out: misaligned");
    FrameArgs a = frame_args(tgt_guide, src_guide, lut, levels, threshold, seed);
    a.assign_out = assign_out;
    a.level_out = level_out;
    FrameLaunch<kAssign> f{&a, static_cast<cudaStream_t>(stream)};
    dispatch_format(tgt_guide->channels, tgt_guide->bits, f);
    if (f.err != cudaSuccess) return cuda_fail(f.err, "sb_assign_chunks");
    return ok();
}

extern "C" sb_status sb_stylize(const sb_guide *tgt_guide, const sb_guide *src_guide,
                                const sb_rgba8 *src_style, const sb_lut *lut, int32_t levels,
                                uint64_t threshold, int32_t blend_radius, uint32_t seed,
                                uint8_t *rgba8_out, sb_stream stream) {
    sb_status st = check_frame(tgt_guide, src_guide, lut, levels);
    if (st != SB_OK) return st;
    if ((st = check_style(src_style, "src_style")) != SB_OK) return st;
    if (src_style->width != src_guide->width || src_style->height != src_guide->height)
        return fail(SB_ERR_INVALID_ARG, "src_style and src_guide differ in size");
    if (blend_radius < 0 || blend_radius > kMaxFusedRadius)
        return fail(SB_ERR_INVALID_ARG, "blend_radius must be in [0, 7]");
    if ((int64_t)tgt_guide->width * tgt_guide->height == 0) return ok();
    if (!rgba8_out || ((uintptr_t)rgba8_out % 4))
        return fail(SB_ERR_INVALID_ARG, "rgba8_out: NULL or not 4-byte aligned");
    FrameArgs a = frame_args(tgt_guide, src_guide, lut, levels, threshold, seed);
    a.style = src_style->data;
    a.style_stride = src_style->row_stride;
    a.radius = blend_radius;
    a.rgba_out = reinterpret_cast<uint32_t *>(rgba8_out);
    FrameLaunch<kStylize> f{&a, static_cast<cudaStream_t>(stream)};
    dispatch_format(tgt_guide->channels, tgt_guide->bits, f);
    if (f.err != cudaSuccess) return cuda_fail(f.err, "sb_stylize");
    return ok();
}

extern "C" sb_status sb_blend(const uint32_t *assign, int32_t tgt_w, int32_t tgt_h,
                              const sb_rgba8 *src_style, int32_t blend_radius,
                              uint8_t *rgba8_out, float *rgba32f_out, sb_stream stream) {
    sb_status st = check_style(src_style, "src_style");
    if (st != SB_OK) return st;
    if (tgt_w < 0 || tgt_h < 0 || tgt_w > kMaxTargetSide || tgt_h > kMaxTargetSide)
        return fail(SB_ERR_INVALID_ARG, "target size out of range");
    if (blend_radius < 0 || blend_radius > kMaxBlendRadius)
        return fail(SB_ERR_INVALID_ARG, "blend_radius must be in [0, 15]");
    if ((rgba8_out == nullptr) == (rgba32f_out == nullptr))
        return fail(SB_ERR_INVALID_ARG, "exactly one of rgba8_out / rgba32f_out must be set");
    if ((int64_t)tgt_w * tgt_h == 0) return ok();
    if (!assign || ((uintptr_t)assign % 4))
        return fail(SB_ERR_INVALID_ARG, "assign: NULL or misaligned");
    if (rgba8_out && ((uintptr_t)rgba8_out % 4))
        return fail(SB_ERR_INVALID_ARG, "rgba8_out: not 4-byte aligned");
    if (rgba32f_out && ((uintptr_t)rgba32f_out % 16))
        return fail(SB_ERR_INVALID_ARG, "rgba32f_out: not 16-byte aligned");
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    FrameArgs a{};
    a.W = tgt_w;
    a.H = tgt_h;
    a.Ws = src_style->width;
    a.Hs = src_style->height;
    a.style = src_style->data;
    a.style_stride = src_style->row_stride;
    a.radius = blend_radius;
    a.assign_in = assign;
    a.rgba_out = reinterpret_cast<uint32_t *>(rgba8_out);
    a.f32_out = reinterpret_cast<float4 *>(rgba32f_out);
    const SmemLayout L = smem_layout(blend_radius, 0);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = rgba32f_out ? launch_tiles<blend_kernel<true>>(L.total, tgt_w, tgt_h, s, a)
                    : launch_tiles<blend_kernel<false>>(L.total, tgt_w, tgt_h, s, a);
    if (e != cudaSuccess) return cuda_fail(e, "sb_blend");
    return ok();
}
