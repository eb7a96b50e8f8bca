/*
 * styleblit.h -- C ABI of the GB300 (sm_103a) StyleBlit library.
 *
 * StyleBlit (Sykora, Jamriska, Lu, Shechtman, "StyleBlit: Fast Example-Based
 * Stylization with Local Guidance", EGSR 2018) stylises a target image from a
 * style exemplar by copying translated chunks of the exemplar.  Its problem
 * statement (inputs of Algorithms 1 and 2): a source style exemplar C_S, source
 * guides G_S, target guides G_T, a threshold t and a number of levels L; the
 * output is the stylised target C_T.
 *
 * Conventions shared by every entry point
 *   - Image pointers are DEVICE pointers owned by the caller.  Inputs are only
 *     read; outputs are fully overwritten on success and left unspecified on
 *     error (no partial-output guarantee).
 *   - Guides are interleaved HWC.  8-bit guides may have 1..4 channels, 16-bit
 *     guides 1..2 channels (16-bit samples little-endian, rows 2-byte aligned).
 *     Target and source guides must have the same channel count and depth.
 *   - Styles are RGBA8, interleaved, rows 4-byte aligned.
 *   - Sizes: 1 <= source width/height <= 32767 (positions are packed into 16
 *     bits each; the extra bit keeps packed-position arithmetic carry-free);
 *     target width/height <= 65535, zero-sized targets are a no-op.
 *   - Source positions are packed as x | y << 16 in a uint32.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *     call only enqueues work on `stream` and returns without synchronising;
 *     results are ready when the stream reaches that point.
 *   - Every call returns SB_OK (0) or a negative sb_status.  Arguments are
 *     validated on the host before anything is launched; sb_last_error()
 *     returns a message for the most recent failure on the calling thread.
 *   - The library owns sb_lut objects (created by sb_build_lut, freed by
 *     sb_lut_destroy); it allocates device memory only inside sb_build_lut.
 *
 * The reading of the paper this library computes (shared with its CPU
 * oracle): the level loop of Algorithm 2 with seed spacing 2^l for l = L..1,
 * seeds jittered by a hash of (seed, level, cell) and clamped into the
 * target, nearest seed over the 3 x 3 neighbouring cells (x outer, y inner,
 * strict <), candidate u*(q) + (p - q) accepted when it lies in the source and
 * its squared guide distance to G_T[p] is <= threshold, the finest level always
 * accepting (candidate clamped into the source); then the voting step of
 * Section 3.2 over a (2r+1) x (2r+1) window with integer sums and round-half-up
 * division.
 */
#ifndef STYLEBLIT_H
#define STYLEBLIT_H

#include <stdint.h>

#if defined(__GNUC__)
#define SB_API __attribute__((visibility("default")))
#else
#define SB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SB_OK = 0,
    SB_ERR_INVALID_ARG = -1,   /* a pointer, size or parameter is out of range */
    SB_ERR_UNSUPPORTED = -2,   /* a valid request this build does not implement */
    SB_ERR_CUDA = -3,          /* a CUDA call failed (sticky errors included) */
    SB_ERR_OOM = -4,           /* device allocation failed */
    SB_ERR_TIMEOUT = -5        /* a bounded device-side wait gave up */
} sb_status;

typedef void *sb_stream;       /* cudaStream_t */

/* A guide image G_S or G_T (device memory, interleaved HWC). */
typedef struct {
    const void *data;
    int32_t width;
    int32_t height;
    int32_t channels;          /* 1..4 for 8-bit, 1..2 for 16-bit */
    int32_t bits;              /* 8 or 16 */
    int64_t row_stride;        /* bytes between row starts, >= width*channels*bits/8 */
} sb_guide;

/* A style exemplar C_S (device memory, RGBA8). */
typedef struct {
    const uint8_t *data;
    int32_t width;
    int32_t height;
    int64_t row_stride;        /* bytes, multiple of 4, >= 4*width; height*row_stride < 2^33 */
} sb_rgba8;

/* Opaque, library-owned guide look-up table of one exemplar. */
typedef struct sb_lut sb_lut;

/*
 * sb_build_lut -- the guide look-up table of Section 3.1.
 *
 * The paper notes that the local guide (usually two values) indirectly names
 * a source position, so a look-up table can return, for a target guide value,
 * the source pixel with the nearest guide (u* = argmin_u ||G_T[q] - G_S[u]||
 * in Algorithm 2, "found via lookup").  The table quantises each guide
 * channel to its top `key_bits` bits; bin k (channel keys concatenated,
 * channel 0 lowest) maps to the source pixel minimising the squared guide
 * distance to the bin representative rep_c = (key_c << z) + ((2^z - 1) >> 1),
 * z = bits - key_bits, ties to the smallest y * width + x.  The result is
 * exact either way it is computed: 8-bit guides keyed on at most three
 * channels go through a distance transform over the grid of guide values,
 * the others through a pruned brute-force nearest-neighbour kernel.
 *
 * Keys wider than 24 bits (e.g. four 8-bit channels at 7 or 8 bits, two
 * 16-bit channels above 12 bits) get no table: the paper retrieves u* with
 * search trees when more guide channels are used, and so does this library.
 * The object then holds a search index (a two-level tree of guide-space boxes
 * over 16 x 16-pixel tiles and 4 x 4-tile super-tiles) and the frame kernels
 * query it for every seed at the seed's bin representative, which gives the
 * same source position a full table would hold (exact nearest pixel, ties to
 * the smallest y * width + x).  Such queries cost far more than a table read;
 * sb_lookup_only refuses these objects (SB_ERR_UNSUPPORTED).
 *
 *   src_guide  source guide G_S (device).  The table refers to positions in
 *              it; later calls must pass a source guide of the same size and
 *              format (checked) and the same content (not checked).
 *   key_bits   bits kept per channel, 1 <= key_bits <= bits; a table for
 *              channels * key_bits <= 24 (at most 16 Mi entries, 64 MiB), a
 *              search index above.
 *   out        receives the new table; untouched on error.
 *   stream     the build is enqueued on this stream.  Temporary device
 *              memory is allocated and freed inside the call (stream-ordered):
 *              2 * 8 * 256^kc bytes for the distance transform (268 MB for
 *              three keyed channels), 16 bytes per 16x16 source tile for the
 *              search.  A search index keeps its 16 bytes per tile (plus one
 *              box per super-tile) for the object's lifetime.
 * Errors: SB_ERR_INVALID_ARG, SB_ERR_UNSUPPORTED, SB_ERR_OOM, SB_ERR_CUDA.
 */
SB_API sb_status sb_build_lut(const sb_guide *src_guide, int32_t key_bits, sb_lut **out,
                       sb_stream stream);

/*
 * sb_build_lut_noalloc -- the table of sb_build_lut, built into memory the
 * caller owns, with no device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, e.g. a
 * host application whose pool allocator already owns the GPU's memory, or a
 * frame loop that must not call cudaMalloc (it can synchronise the device and
 * can fail under memory pressure).
 *
 *   src_guide  source guide G_S (device), as for sb_build_lut, at most 65536
 *              tiles of 16 x 16 pixels (e.g. 4096 x 4096); larger guides are
 *              rejected with SB_ERR_INVALID_ARG.
 *   key_bits   as for sb_build_lut.
 *   table_out  device uint32[2^(channels * key_bits)], 4-byte aligned, owned by
 *              the caller: receives the same entries sb_build_lut computes.
 *   stream     the build is enqueued on this stream.
 * Scratch: a fixed 1.1 MiB array inside the library (file-scope device memory,
 * held by every GPU that loads the library until the process exits).  Every
 * call looks up that array's device address on the current device (no
 * caching, so a device reset in between is harmless); the first call on a
 * device may load the library's device code, so make it before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (every call overwrites what it reads, nothing needs clearing): calls whose
 * GPU work overlaps (e.g. enqueued on different streams without ordering)
 * race on it, so serialise them.  Nothing is allocated or freed: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 * Errors: SB_ERR_INVALID_ARG, SB_ERR_UNSUPPORTED, SB_ERR_CUDA.
 */
SB_API sb_status sb_build_lut_noalloc(const sb_guide *src_guide, int32_t key_bits,
                                      uint32_t *table_out, sb_stream stream);

/* Frees a table (NULL is a no-op).  The caller must ensure no enqueued work
 * still uses it (e.g. synchronise the streams that used it first). */
SB_API sb_status sb_lut_destroy(sb_lut *lut);

/* Describes a table: device pointer to its 2^(key_channels*key_bits) uint32
 * entries (packed x | y << 16), entry count, channels and bits of the guide
 * it was built for, key_bits, key_channels, and that guide's width and height.
 * A search index (keys wider than 24 bits) reports entries = NULL and
 * n_entries = 0.  Any output pointer may be NULL. */
SB_API sb_status sb_lut_info(const sb_lut *lut, const uint32_t **entries, int64_t *n_entries,
                             int32_t *channels, int32_t *bits, int32_t *key_bits,
                             int32_t *key_channels, int32_t *src_width, int32_t *src_height);

/*
 * sb_build_lut_keyed -- sb_build_lut keyed on the first key_channels guide
 * channels only.  Section 4 adds a segmentation guide that keeps chunks inside
 * semantic regions: such channels are appended after the local guide (e.g.
 * uint8 normals + one segment channel = 4 channels) and take part only in the
 * acceptance distance of sb_assign_chunks / sb_stylize / sb_stylize_batch,
 * while the table maps the local guide to the source pixel nearest in those
 * key channels (ties to the smallest y * width + x).
 *
 *   key_channels  1..channels; above 24 key bits a search index (as
 *                 sb_build_lut) keyed on these channels.
 *   Other arguments, ownership and errors as sb_build_lut (which is this call
 *   with key_channels = channels).
 */
SB_API sb_status sb_build_lut_keyed(const sb_guide *src_guide, int32_t key_bits,
                                    int32_t key_channels, sb_lut **out, sb_stream stream);

/*
 * sb_assign_chunks -- Algorithm 2 (ParallelStyleBlit) with coordinate
 * transfer (Section 3.2): the source position every target pixel copies from.
 *
 *   tgt_guide   target guide G_T (device).
 *   src_guide   source guide G_S (device), the one `lut` was built from.
 *   lut         table from sb_build_lut for src_guide.
 *   levels      L, 1 <= L <= 15; level l uses seed spacing 2^l.
 *   threshold   t, compared as squared integer guide distance (<=).
 *   seed        frame seed of the jitter hash (re-randomise per frame for
 *               the controllable flicker of Section 3.3).
 *   assign_out  device uint32[tgt h * tgt w], row-major: A(p) = x | y << 16.
 *   level_out   device uint8[tgt h * tgt w]: the level that accepted p, or
 *               NULL.
 * Errors: SB_ERR_INVALID_ARG, SB_ERR_UNSUPPORTED, SB_ERR_CUDA.
 */
SB_API sb_status sb_assign_chunks(const sb_guide *tgt_guide, const sb_guide *src_guide,
                           const sb_lut *lut, int32_t levels, uint64_t threshold,
                           uint32_t seed, uint32_t *assign_out, uint8_t *level_out,
                           sb_stream stream);

/*
 * sb_blend -- the voting step of Section 3.2: the colour of p is the average
 * of C_S[A(p + o) - o] over the window offsets o in [-r, r]^2 whose p + o lies
 * in the target and whose A(p + o) - o lies in the source.
 *
 *   assign        device uint32[tgt_h * tgt_w] from sb_assign_chunks.
 *   src_style     C_S (device).  Every A(p) must lie inside it.
 *   blend_radius  r, 0 <= r <= 15 (r = 0 copies C_S[A(p)]).
 *   rgba8_out     device uint8[tgt_h * tgt_w * 4]: (sum + n/2) / n, or
 *   rgba32f_out   device float[tgt_h * tgt_w * 4]: sum / (255 n).
 *                 Exactly one of the two outputs must be non-NULL.
 * Errors: SB_ERR_INVALID_ARG, SB_ERR_CUDA.
 */
SB_API sb_status sb_blend(const uint32_t *assign, int32_t tgt_w, int32_t tgt_h,
                   const sb_rgba8 *src_style, int32_t blend_radius, uint8_t *rgba8_out,
                   float *rgba32f_out, sb_stream stream);

/*
 * sb_stylize -- assignment and voting fused in one kernel (Algorithm 2 plus
 * the voting step of Section 3.2); the assignment map never reaches device
 * memory.  Bit-identical to sb_assign_chunks followed by sb_blend(rgba8).
 *
 *   tgt_guide, src_guide, lut, levels, threshold, seed: as sb_assign_chunks.
 *   src_style     C_S (device), same width and height as src_guide.
 *   blend_radius  r, 0 <= r <= 15.
 *   rgba8_out     device uint8[tgt h * tgt w * 4] (row-major, tightly packed).
 * Errors: SB_ERR_INVALID_ARG, SB_ERR_UNSUPPORTED, SB_ERR_CUDA.
 */
SB_API sb_status sb_stylize(const sb_guide *tgt_guide, const sb_guide *src_guide,
                     const sb_rgba8 *src_style, const sb_lut *lut, int32_t levels,
                     uint64_t threshold, int32_t blend_radius, uint32_t seed,
                     uint8_t *rgba8_out, sb_stream stream);

/* One frame of a batch (sb_stylize_batch).  All pointers are device pointers
 * owned by the caller, as for sb_stylize. */
typedef struct {
    sb_guide tgt_guide;        /* target guide G_T of this frame */
    const sb_lut *lut;         /* table of this frame's exemplar (sb_build_lut) */
    sb_rgba8 src_style;        /* that exemplar's style C_S (same size as its guide) */
    int32_t levels;            /* L, 1..15 */
    uint64_t threshold;        /* t, squared guide distance, <= accepts */
    uint32_t seed;             /* frame seed of the jitter hash */
    uint8_t *rgba8_out;        /* tgt h * tgt w * 4 bytes, 4-byte aligned */
} sb_frame;

/*
 * sb_stylize_batch -- sb_stylize for many frames in a single launch (the
 * batched form of Algorithm 2 plus the voting step of Section 3.2).  Frames
 * may differ in size, exemplar, level count, threshold and seed; they share
 * the guide format (channels and bits) and the blend radius.  Every frame's
 * output is bit-identical to sb_stylize on that frame alone.  The tiles of all
 * frames form one grid, so the GPU starts later frames while the last tiles of
 * earlier ones finish.
 *
 *   frames        host array of n_frames descriptors (read during the call;
 *                 the device data they point to must stay valid until the
 *                 stream reaches the batch).
 *   n_frames      0..128 (0 is a no-op).
 *   blend_radius  r, 0 <= r <= 15, for every frame.
 * Allocates nothing.  Errors: SB_ERR_INVALID_ARG (a frame's arguments, as for
 * sb_stylize; the message names the frame), SB_ERR_UNSUPPORTED (frames with
 * different guide formats), SB_ERR_CUDA.
 */
SB_API sb_status sb_stylize_batch(const sb_frame *frames, int32_t n_frames, int32_t blend_radius,
                                  sb_stream stream);

/*
 * Launch schedule of a batch.  The paper has no counterpart: this is a GPU
 * scheduling choice, and every schedule gives the same pixels (each tile runs
 * the same code).
 *   persistent     0: one CTA per tile (the hardware issues tiles as CTAs
 *                  retire); 1: as many CTAs as fit on the device take tiles
 *                  from a work queue in device memory until the batch is done.
 *                  The queue resets itself at the end of a launch.  Queues
 *                  come from a fixed set of 1024 per device, assigned so that
 *                  no two launches that may run at once share one: a stream
 *                  keeps one queue for all its eager persistent launches
 *                  (they run one after another), and a launch captured into a
 *                  CUDA graph gets a queue of its own, never reused, which
 *                  every replay of that executable graph uses (CUDA orders the
 *                  replays of one executable graph).  Not supported: running
 *                  two executable graphs instantiated from the same capture at
 *                  the same time, and destroying a stream while its persistent
 *                  launch runs and launching on a new stream that received
 *                  the same handle.  Once 1024 streams and captured launches
 *                  have taken queues on a device, further persistent launches
 *                  there fail with SB_ERR_UNSUPPORTED.
 *   largest_first  0: tiles in frame order; 1: frames with more tiles first
 *                  (shorter tail for uneven batches).
 *   interleave_rows  0: each frame's tiles together; 1: when every frame of
 *                  the batch has the same tile grid (in tiles of tile_rows),
 *                  tile row r of every frame before tile row r + 1, so the
 *                  exemplar lines those rows gather stay in L2 while the frames
 *                  stream through; batches of frames with different tile grids
 *                  keep frame order.
 *   tile_rows      output rows per tile (tiles are 64 pixels wide): 0 or 32
 *                  (256 threads a CTA), 16 (128 threads) or 64 (512 threads);
 *                  16 and 64 need blend_radius <= 7.  Shorter tiles recompute
 *                  a larger share of halo rows, taller ones use more shared
 *                  memory per CTA.
 */
typedef struct {
    int32_t persistent;
    int32_t largest_first;
    int32_t interleave_rows;
    int32_t tile_rows;
} sb_batch_schedule;

/*
 * sb_stylize_batch_sched -- sb_stylize_batch with an explicit schedule
 * (NULL: {0, 0, 0, 0}, the schedule of sb_stylize_batch).  Same arguments, outputs
 * and errors as sb_stylize_batch.
 */
SB_API sb_status sb_stylize_batch_sched(const sb_frame *frames, int32_t n_frames,
                                        int32_t blend_radius, const sb_batch_schedule *schedule,
                                        sb_stream stream);

/*
 * sb_autotune_batch -- picks the fastest schedule for this batch (no
 * counterpart in the paper).  Runs each schedule (tile_rows 32, and 16 and 64
 * for blend radii up to 7, times persistent x largest_first, times
 * interleave_rows when the frames share one tile grid) once untimed and
 * `reps` times between two CUDA events on `stream`, waits for the stream, and
 * writes the fastest to *best and its mean time per batch (ms) to *best_ms
 * (nullable).  The batch's outputs are written (every run writes the same
 * pixels).  Blocks the calling thread; refuses a stream under capture.
 *   reps  1..1000.
 * Errors: those of sb_stylize_batch; SB_ERR_INVALID_ARG (NULL best, reps out
 * of range, a capturing stream); SB_ERR_CUDA.
 */
SB_API sb_status sb_autotune_batch(const sb_frame *frames, int32_t n_frames,
                                   int32_t blend_radius, int32_t reps, sb_batch_schedule *best,
                                   float *best_ms, sb_stream stream);

/*
 * sb_lookup_only -- the per-pixel mapping StyleBlit is compared with in
 * Section 4 (texture mapping; The Lit Sphere): every target pixel copies the
 * style at the table entry of its own guide value, C_T[p] = C_S[LUT(G_T[p])],
 * with no seeds, chunks or vote.  A throughput and quality comparator.
 *
 *   tgt_guide, src_guide, src_style, lut: as sb_stylize.
 *   rgba8_out  device uint8[tgt h * tgt w * 4], 4-byte aligned.
 * Errors: SB_ERR_INVALID_ARG, SB_ERR_UNSUPPORTED, SB_ERR_CUDA.
 */
SB_API sb_status sb_lookup_only(const sb_guide *tgt_guide, const sb_guide *src_guide,
                                const sb_rgba8 *src_style, const sb_lut *lut, uint8_t *rgba8_out,
                                sb_stream stream);

/*
 * sb_lookup_only_batch -- sb_lookup_only for many frames in a single launch
 * (the comparator of Section 4, batched like sb_stylize_batch).  Frames may
 * differ in size and exemplar and share the guide format.  Every frame's
 * output is bit-identical to sb_lookup_only on that frame alone.
 *
 *   frames     host array of n_frames descriptors (sb_frame; only tgt_guide,
 *              lut, src_style and rgba8_out are used: levels, threshold and
 *              seed are ignored).  Read during the call; the device data
 *              must stay valid until the stream reaches the launch.
 *   n_frames   0..128 (0 is a no-op).
 * Allocates nothing.  Errors: SB_ERR_INVALID_ARG (a frame's arguments, as for
 * sb_lookup_only; the message names the frame), SB_ERR_UNSUPPORTED (frames
 * with different guide formats), SB_ERR_CUDA.
 */
SB_API sb_status sb_lookup_only_batch(const sb_frame *frames, int32_t n_frames,
                                      sb_stream stream);

/* Static description of a status code. */
SB_API const char *sb_status_string(sb_status status);

/* Message describing the most recent failure on the calling thread ("" if
 * none).  The pointer stays valid until the next library call on the thread. */
SB_API const char *sb_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
SB_API int32_t sb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STYLEBLIT_H */
