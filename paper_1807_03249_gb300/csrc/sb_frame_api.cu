// C ABI entry points of the per-frame StyleBlit path (Algorithm 2 and the
// voting step of Section 3.2): argument validation and kernel dispatch.  The
// frame kernels live in sb_frame.cuh; the blend kernels are instantiated here.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <mutex>
#include <string>
#include <unordered_map>

#include "sb_frame.cuh"

namespace sb {

static cudaError_t launch_frame_any(int channels, int bits, int mode, const FrameArgs &a,
                                    cudaStream_t s) {
    if (bits == 8) {
        switch (channels) {
            case 1: return launch_frame_c1b8(mode, a, s);
            case 2: return launch_frame_c2b8(mode, a, s);
            case 3: return launch_frame_c3b8(mode, a, s);
            case 4: return launch_frame_c4b8(mode, a, s);
        }
    } else if (bits == 16) {
        switch (channels) {
            case 1: return launch_frame_c1b16(mode, a, s);
            case 2: return launch_frame_c2b16(mode, a, s);
        }
    }
    return cudaErrorInvalidValue;
}

static cudaError_t launch_batch_any(int channels, int bits, const BatchArgs &b, int r, int th,
                                    TileQueue *queue, int max_levels, cudaStream_t s) {
    if (bits == 8) {
        switch (channels) {
            case 1: return launch_batch_c1b8(b, r, th, max_levels, queue, s);
            case 2: return launch_batch_c2b8(b, r, th, max_levels, queue, s);
            case 3: return launch_batch_c3b8(b, r, th, max_levels, queue, s);
            case 4: return launch_batch_c4b8(b, r, th, max_levels, queue, s);
        }
    } else if (bits == 16) {
        switch (channels) {
            case 1: return launch_batch_c1b16(b, r, th, max_levels, queue, s);
            case 2: return launch_batch_c2b16(b, r, th, max_levels, queue, s);
        }
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Work queues of persistent batch launches.  Two launches must never share a
// queue while both may run.  Launches on one stream run one after the other,
// so an eager launch uses the queue its stream owns (assigned on the stream's
// first persistent launch and kept).  A launch captured into a CUDA graph may
// be replayed at any time on any stream, so it gets a queue of its own that no
// other launch ever receives; replays of one executable graph are ordered by
// CUDA, so they never overlap each other.  All formats and radii draw from one
// array per device.
// ---------------------------------------------------------------------------
constexpr int kQueueSlots = 1024;
__device__ TileQueue g_tile_queues[kQueueSlots];

struct QueuePool {
    std::mutex mu;
    int used = 0;                                    // slots handed out so far
    std::unordered_map<uintptr_t, int> by_stream;    // eager launches: stream -> slot
    TileQueue *base = nullptr;                       // device address of g_tile_queues
};

static sb_status acquire_queue(cudaStream_t s, TileQueue **out) {
    constexpr int kMaxDev = 64;
    static QueuePool pools[kMaxDev];
    static thread_local int per_thread_slot[kMaxDev] = {};  // slot + 1 for cudaStreamPerThread
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "sb_stylize_batch: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDev) return fail(SB_ERR_UNSUPPORTED, "device ordinal above 63");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess)
        return cuda_fail(e, "sb_stylize_batch: cudaStreamIsCapturing");
    QueuePool &P = pools[dev];
    std::lock_guard<std::mutex> lock(P.mu);
    // the array's address is looked up outside captures (a device reset may
    // move it) and reused inside them
    if (cap == cudaStreamCaptureStatusNone || !P.base) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_tile_queues)) != cudaSuccess)
            return cuda_fail(e, "sb_stylize_batch: work-queue address");
        P.base = static_cast<TileQueue *>(p);
    }
    int slot = -1;
    if (cap != cudaStreamCaptureStatusNone) {
        if (P.used < kQueueSlots) slot = P.used++;
    } else if (s == cudaStreamPerThread) {
        // one handle, a different stream on every thread
        if (!per_thread_slot[dev] && P.used < kQueueSlots) per_thread_slot[dev] = ++P.used;
        slot = per_thread_slot[dev] - 1;
    } else {
        const uintptr_t key = reinterpret_cast<uintptr_t>(s == cudaStreamLegacy ? nullptr : s);
        auto it = P.by_stream.find(key);
        if (it != P.by_stream.end()) {
            slot = it->second;
        } else if (P.used < kQueueSlots) {
            slot = P.used++;
            P.by_stream.emplace(key, slot);
        }
    }
    if (slot < 0)
        return fail(SB_ERR_UNSUPPORTED,
                    "sb_stylize_batch: no free work queue for a persistent launch (1024 per "
                    "device: one per stream plus one per captured launch)");
    *out = P.base + slot;
    return SB_OK;
}

template <bool F32, int R>
static cudaError_t launch_blend_r(const FrameArgs &a, cudaStream_t s) {
    return launch_tiles<blend_kernel<F32, R>>(smem_layout(R, 0).total, a.W, a.H, s, a);
}

template <bool F32>
static cudaError_t launch_blend(const FrameArgs &a, cudaStream_t s) {
    switch (a.radius) {
        case 0: return launch_blend_r<F32, 0>(a, s);
        case 1: return launch_blend_r<F32, 1>(a, s);
        case 2: return launch_blend_r<F32, 2>(a, s);
        case 3: return launch_blend_r<F32, 3>(a, s);
        case 4: return launch_blend_r<F32, 4>(a, s);
        case 5: return launch_blend_r<F32, 5>(a, s);
        case 6: return launch_blend_r<F32, 6>(a, s);
        case 7: return launch_blend_r<F32, 7>(a, s);
        case 8: return launch_blend_r<F32, 8>(a, s);
        case 9: return launch_blend_r<F32, 9>(a, s);
        case 10: return launch_blend_r<F32, 10>(a, s);
        case 11: return launch_blend_r<F32, 11>(a, s);
        case 12: return launch_blend_r<F32, 12>(a, s);
        case 13: return launch_blend_r<F32, 13>(a, s);
        case 14: return launch_blend_r<F32, 14>(a, s);
        case 15: return launch_blend_r<F32, 15>(a, s);
    }
    return cudaErrorInvalidValue;
}

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
        return fail(SB_ERR_INVALID_ARG, "levels must be in [1, 15]");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != lut->device) return fail(SB_ERR_INVALID_ARG, "lut lives on another device");
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    return SB_OK;
}

static FrameArgs frame_args(const sb_guide *tgt, const sb_lut *lut, int32_t levels,
                            uint64_t threshold, uint32_t seed) {
    FrameArgs a{};
    a.tgt = static_cast<const uint8_t *>(tgt->data);
    a.tgt_stride = tgt->row_stride;
    a.W = tgt->width;
    a.H = tgt->height;
    a.src_packed = lut->src_packed;
    a.Ws = lut->src_w;
    a.Hs = lut->src_h;
    a.lut = lut->entries;
    a.nn_bounds = lut->nn_bounds;
    a.key_bits = lut->key_bits;
    a.key_channels = lut->key_channels;
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
    FrameArgs a = frame_args(tgt_guide, lut, levels, threshold, seed);
    a.assign_out = assign_out;
    a.level_out = level_out;
    cudaError_t e = launch_frame_any(tgt_guide->channels, tgt_guide->bits, kAssign, a,
                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sb_assign_chunks");
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
        return fail(SB_ERR_INVALID_ARG, "blend_radius must be in [0, 15]");
    if ((int64_t)tgt_guide->width * tgt_guide->height == 0) return ok();
    if (!rgba8_out || ((uintptr_t)rgba8_out % 4))
        return fail(SB_ERR_INVALID_ARG, "rgba8_out: NULL or not 4-byte aligned");
    FrameArgs a = frame_args(tgt_guide, lut, levels, threshold, seed);
    a.style = src_style->data;
    a.style_stride_px = (int)(src_style->row_stride / 4);
    a.radius = blend_radius;
    a.rgba_out = reinterpret_cast<uint32_t *>(rgba8_out);
    cudaError_t e = launch_frame_any(tgt_guide->channels, tgt_guide->bits, kStylize, a,
                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sb_stylize");
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
    a.style_stride_px = (int)(src_style->row_stride / 4);
    a.radius = blend_radius;
    a.assign_in = assign;
    a.rgba_out = reinterpret_cast<uint32_t *>(rgba8_out);
    a.f32_out = reinterpret_cast<float4 *>(rgba32f_out);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = rgba32f_out ? launch_blend<true>(a, s) : launch_blend<false>(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "sb_blend");
    return ok();
}

// Validates a batch and fills the launch descriptor; frames go in the given
// order or, with largest_first, by decreasing tile count (each frame keeps its
// own output, so the order changes only which tiles are issued first).
static sb_status prepare_batch(const sb_frame *frames, int32_t n_frames, int32_t blend_radius,
                               bool largest_first, bool interleave_rows, int th, BatchArgs &b,
                               int &max_levels, int &channels, int &bits) {
    if (n_frames < 0 || n_frames > kMaxBatch)
        return fail(SB_ERR_INVALID_ARG, "n_frames must be in [0, 128]");
    if (n_frames == 0) return ok();
    if (!frames) return fail(SB_ERR_INVALID_ARG, "frames: NULL");
    if (blend_radius < 0 || blend_radius > kMaxFusedRadius)
        return fail(SB_ERR_INVALID_ARG, "blend_radius must be in [0, 15]");
    b.n = n_frames;
    b.rows_interleaved = 0;
    b.rows_tx = 0;
    b.tile_start[0] = 0;
    max_levels = 1;
    channels = frames[0].tgt_guide.channels;
    bits = frames[0].tgt_guide.bits;
    int order[kMaxBatch];
    int64_t tiles[kMaxBatch];
    char name[64];
    for (int k = 0; k < n_frames; ++k) {
        const sb_frame &f = frames[k];
        std::snprintf(name, sizeof name, "frames[%d].tgt_guide", k);
        sb_status st = check_guide(&f.tgt_guide, name, false);
        if (st != SB_OK) return st;
        if (f.tgt_guide.channels != channels || f.tgt_guide.bits != bits)
            return fail(SB_ERR_UNSUPPORTED, "sb_stylize_batch: frames must share one guide format");
        std::snprintf(name, sizeof name, "frames[%d]", k);
        if (!f.lut) return fail(SB_ERR_INVALID_ARG, std::string(name) + ": lut NULL");
        if (f.lut->channels != channels || f.lut->bits != bits)
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": lut built for another format");
        std::snprintf(name, sizeof name, "frames[%d].src_style", k);
        if ((st = check_style(&f.src_style, name)) != SB_OK) return st;
        if (f.src_style.width != f.lut->src_w || f.src_style.height != f.lut->src_h)
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": size differs from the lut's guide");
        std::snprintf(name, sizeof name, "frames[%d]", k);
        if (f.levels < 1 || f.levels > kMaxLevels)
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": levels must be in [1, 15]");
        const int64_t npx = (int64_t)f.tgt_guide.width * f.tgt_guide.height;
        if (npx > 0 && (!f.rgba8_out || ((uintptr_t)f.rgba8_out % 4)))
            return fail(SB_ERR_INVALID_ARG, std::string(name) + ": rgba8_out NULL or misaligned");
        const int64_t tx = (f.tgt_guide.width + kTW - 1) / kTW, ty = (f.tgt_guide.height + th - 1) / th;
        tiles[k] = npx > 0 ? tx * ty : 0;
        order[k] = k;
        max_levels = max(max_levels, (int)f.levels);
    }
    if (largest_first)
        std::stable_sort(order, order + n_frames, [&](int i, int j) { return tiles[i] > tiles[j]; });
    for (int i = 0; i < n_frames; ++i) {
        const sb_frame &f = frames[order[i]];
        const int64_t next = (int64_t)b.tile_start[i] + tiles[order[i]];
        if (next > INT_MAX) return fail(SB_ERR_INVALID_ARG, "sb_stylize_batch: too many tiles");
        b.tile_start[i + 1] = (int)next;
        b.tiles_x[i] = max(1, (f.tgt_guide.width + kTW - 1) / kTW);
        b.div_tiles_x[i] = FastDiv::of((uint32_t)b.tiles_x[i]);
        FrameArgs a = frame_args(&f.tgt_guide, f.lut, f.levels, f.threshold, f.seed);
        a.style = f.src_style.data;
        a.style_stride_px = (int)(f.src_style.row_stride / 4);
        a.radius = blend_radius;
        a.rgba_out = reinterpret_cast<uint32_t *>(f.rgba8_out);
        b.f[i] = a;
    }
    // rows interleaved only when every frame has the same tile grid
    if (interleave_rows) {
        const int tx0 = (frames[0].tgt_guide.width + kTW - 1) / kTW;
        const int ty0 = (frames[0].tgt_guide.height + th - 1) / th;
        bool same = tiles[0] > 0;
        for (int k = 1; k < n_frames && same; ++k)
            same = (frames[k].tgt_guide.width + kTW - 1) / kTW == tx0 &&
                   (frames[k].tgt_guide.height + th - 1) / th == ty0 && tiles[k] > 0;
        if (same) {
            b.rows_interleaved = 1;
            b.rows_tx = tx0;
            b.div_row = FastDiv::of((uint32_t)(n_frames * tx0));
            b.div_rows_tx = FastDiv::of((uint32_t)tx0);
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    for (int k = 0; k < n_frames; ++k)
        if (frames[k].lut->device != dev) return fail(SB_ERR_INVALID_ARG, "a lut lives on another device");
    return ok();
}

extern "C" sb_status sb_stylize_batch_sched(const sb_frame *frames, int32_t n_frames,
                                            int32_t blend_radius,
                                            const sb_batch_schedule *schedule,
                                            sb_stream stream) {
    const sb_batch_schedule sched = schedule ? *schedule : sb_batch_schedule{0, 0, 0, 0};
    const int th = sched.tile_rows == 0 ? kTH : sched.tile_rows;
    if (th != 16 && th != 32 && th != 64)
        return fail(SB_ERR_INVALID_ARG, "schedule.tile_rows must be 0, 16, 32 or 64");
    if (th != kTH && blend_radius > kMaxShapedRadius)
        return fail(SB_ERR_INVALID_ARG, "tiles of 16 or 64 rows need blend_radius <= 7");
    static thread_local BatchArgs b;  // ~19 KB: kept off the stack
    int max_levels = 1, channels = 0, bits = 0;
    sb_status st = prepare_batch(frames, n_frames, blend_radius, sched.largest_first != 0,
                                 sched.interleave_rows != 0, th, b, max_levels, channels, bits);
    if (st != SB_OK || n_frames == 0 || b.tile_start[n_frames] == 0) return st;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    TileQueue *queue = nullptr;
    if (sched.persistent &&
        (st = acquire_queue(static_cast<cudaStream_t>(stream), &queue)) != SB_OK)
        return st;
    e = launch_batch_any(channels, bits, b, blend_radius, th, queue, max_levels,
                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sb_stylize_batch");
    return ok();
}

extern "C" sb_status sb_stylize_batch(const sb_frame *frames, int32_t n_frames,
                                      int32_t blend_radius, sb_stream stream) {
    return sb_stylize_batch_sched(frames, n_frames, blend_radius, nullptr, stream);
}

extern "C" sb_status sb_autotune_batch(const sb_frame *frames, int32_t n_frames,
                                       int32_t blend_radius, int32_t reps,
                                       sb_batch_schedule *best, float *best_ms,
                                       sb_stream stream) {
    if (!best) return fail(SB_ERR_INVALID_ARG, "best: NULL");
    if (reps < 1 || reps > 1000) return fail(SB_ERR_INVALID_ARG, "reps must be in [1, 1000]");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "sb_autotune_batch");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(SB_ERR_INVALID_ARG, "sb_autotune_batch: the stream is being captured");
    // every combination of the choices: tile heights 16, 32 and 64 (the other
    // two only for blend radii up to 7), one CTA per tile or persistent, frame
    // order or largest first, and tile rows interleaved when the frames share
    // one tile grid (otherwise it is frame order again)
    const bool ok_n = n_frames > 0 && n_frames <= kMaxBatch && frames;
    sb_batch_schedule cand[24];
    int n_cand = 0;
    for (int th : {32, 16, 64}) {
        if (th != kTH && blend_radius > kMaxShapedRadius) continue;
        bool same_grid = ok_n;
        for (int k = 1; k < n_frames && same_grid; ++k)
            same_grid = (frames[k].tgt_guide.width + kTW - 1) / kTW ==
                            (frames[0].tgt_guide.width + kTW - 1) / kTW &&
                        (frames[k].tgt_guide.height + th - 1) / th ==
                            (frames[0].tgt_guide.height + th - 1) / th;
        for (int il = 0; il <= (same_grid ? 1 : 0); ++il)
            for (int pers = 0; pers <= 1; ++pers)
                for (int lf = 0; lf <= 1; ++lf) cand[n_cand++] = sb_batch_schedule{pers, lf, il, th};
    }
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return cuda_fail(e, "sb_autotune_batch");
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(e, "sb_autotune_batch");
    }
    sb_status st = SB_OK;
    float best_t = 0.f;
    int best_i = 0;
    for (int i = 0; i < n_cand && st == SB_OK; ++i) {
        // one untimed run, then reps timed runs between two events
        st = sb_stylize_batch_sched(frames, n_frames, blend_radius, &cand[i], stream);
        if (st == SB_OK) e = cudaEventRecord(ev[0], s);
        for (int k = 0; k < reps && st == SB_OK; ++k)
            st = sb_stylize_batch_sched(frames, n_frames, blend_radius, &cand[i], stream);
        if (st != SB_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "sb_autotune_batch");
            break;
        }
        if (i == 0 || t < best_t) {
            best_t = t;
            best_i = i;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != SB_OK) return st;
    *best = cand[best_i];
    if (best_ms) *best_ms = best_t / reps;
    return ok();
}
