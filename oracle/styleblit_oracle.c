/*
 * StyleBlit CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, scalar restatement of the per-pixel StyleBlit method of
 * Sykora, Jamriska, Lu and Shechtman, "StyleBlit: Fast Example-Based
 * Stylization with Local Guidance" (EGSR 2018):
 *   - the guide look-up table of Section 3.1 (a source position for every
 *     quantised guide value),
 *   - Algorithm 2 (ParallelStyleBlit): SeedPoint, NearestSeed and the
 *     coarse-to-fine level loop,
 *   - the voting step at the end of Section 3.2 (coordinate transfer, then the
 *     colour of a target pixel is the average of the co-located pixels of the
 *     source patches that cover it).
 * It is the yardstick the CUDA library is compared against element by
 * element.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header or table with the
 * CUDA library; the two meet only in the seeded input generators.
 *
 * Readings taken where the paper is silent or leaves a choice open (the
 * paper's statement is quoted in words, not verbatim):
 *   R1  distance: Euclidean over all guide channels, compared as an integer
 *       squared distance in 64 bits; a candidate is accepted when that
 *       squared distance is <= the threshold (Algorithm 2 writes e < t on a
 *       norm; a squared integer threshold with <= is the same family).
 *   R2  the finest level (l = 1) always accepts, with the candidate clamped
 *       into the source (Algorithm 2 leaves the pixel unset otherwise).
 *   R3  level l uses seed spacing h = 2^l, l = L..1 (Algorithm 2 calls
 *       NearestSeed(p, 2^l)), so the finest spacing is 2.
 *   R4  the random jitter table of SeedPoint is replaced by a stateless hash
 *       of (frame seed, level, cell): H = fmix32(fmix32(fmix32(seed ^
 *       level*0x9E3779B9) ^ bx) ^ by), fmix32 being the 32-bit finaliser of
 *       MurmurHash3 (Appleby, public domain).  The jitter j = (H & 0xFFFF,
 *       H >> 16) / 2^16 is a 16-bit fixed-point fraction, so the seed offset
 *       floor(h * j) is ((H & 0xFFFF) * h) >> 16 and ((H >> 16) * h) >> 16.
 *   R5  a seed that falls outside the target is clamped into the target.
 *   R6  NearestSeed visits x = -1, 0, 1 in the outer loop and y = -1, 0, 1
 *       in the inner loop and replaces the best only on a strict decrease,
 *       as Algorithm 2 writes it; seed distances are squared integers.
 *   R7  a candidate outside the source is rejected at levels l > 1.
 *   R8  look-up table: a guide channel value g with B bits is keyed by its
 *       top b bits (key = g >> (B - b)); the channel keys are concatenated
 *       with channel 0 in the lowest bits.  Every bin is represented by
 *       rep = (key << (B - b)) + ((2^(B - b) - 1) >> 1) and maps to the
 *       source pixel minimising the squared guide distance to rep; ties go to
 *       the smallest linear index y * W + x.  Entries are packed x | y << 16.
 *   R9  vote: uniform k x k window, k = 2r + 1; a window offset o contributes
 *       C_S[A(p + o) - o] when p + o lies in the target and A(p + o) - o lies
 *       in the source; the RGBA8 result is (sum + n / 2) / n per channel
 *       (integer division, round half up); alpha is voted like colour.  The
 *       float variant returns sum / (255 n).
 *   R10 every pixel compares single pixels (Algorithm 2), not regions.
 *   R11 extra guide channels (Section 4 adds a segmentation guide to keep
 *       chunks inside semantic regions): the table is keyed on the first
 *       key_channels channels (the local guide) and maps a bin to the source
 *       pixel nearest in those channels; the acceptance distance (R1) uses
 *       every channel.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define ORC_UNSET 0xFFFFFFFFu

typedef struct {
    const void *data;     /* interleaved HWC, little-endian 16-bit samples */
    int32_t width;
    int32_t height;
    int32_t channels;     /* 1..4 */
    int32_t bits;         /* 8 or 16 */
    int64_t row_stride;   /* bytes between the starts of consecutive rows */
} orc_guide;

typedef struct {
    const uint8_t *data;  /* RGBA8, HWC */
    int32_t width;
    int32_t height;
    int64_t row_stride;   /* bytes */
} orc_rgba8;

/* ------------------------------------------------------------------------ */
/* guide access                                                               */
/* ------------------------------------------------------------------------ */

static uint32_t guide_value(const orc_guide *g, int64_t x, int64_t y, int32_t c)
{
    const uint8_t *row = (const uint8_t *)g->data + y * g->row_stride;
    int64_t i = x * g->channels + c;
    if (g->bits == 8)
        return row[i];
    return (uint32_t)row[2 * i] | ((uint32_t)row[2 * i + 1] << 8);
}

/* squared Euclidean guide distance between two pixels (reading R1) */
static uint64_t guide_distance(const orc_guide *a, int64_t ax, int64_t ay,
                               const orc_guide *b, int64_t bx, int64_t by)
{
    uint64_t d = 0;
    for (int32_t c = 0; c < a->channels; ++c) {
        int64_t diff = (int64_t)guide_value(a, ax, ay, c) - (int64_t)guide_value(b, bx, by, c);
        d += (uint64_t)(diff * diff);
    }
    return d;
}

/* ------------------------------------------------------------------------ */
/* look-up table (Section 3.1; reading R8)                                    */
/* ------------------------------------------------------------------------ */

/* Table index of pixel (x, y): the top key_bits bits of each of the first
 * key_channels channels (the local guide; further channels, e.g. a
 * segmentation channel of Section 4, take part only in the acceptance
 * distance), concatenated with channel 0 lowest. */
uint32_t orc_lut_index_k(const orc_guide *g, int32_t x, int32_t y, int32_t key_bits,
                         int32_t key_channels)
{
    int32_t shift = g->bits - key_bits;
    uint32_t idx = 0;
    for (int32_t c = 0; c < key_channels; ++c)
        idx |= (guide_value(g, x, y, c) >> shift) << (c * key_bits);
    return idx;
}

uint32_t orc_lut_index(const orc_guide *g, int32_t x, int32_t y, int32_t key_bits)
{
    return orc_lut_index_k(g, x, y, key_bits, g->channels);
}

void orc_bin_representative(uint32_t idx, int32_t channels, int32_t bits,
                            int32_t key_bits, uint32_t *rep)
{
    int32_t shift = bits - key_bits;
    uint32_t mask = (1u << key_bits) - 1u;
    for (int32_t c = 0; c < channels; ++c) {
        uint32_t key = (idx >> (c * key_bits)) & mask;
        rep[c] = (key << shift) + (((1u << shift) - 1u) >> 1);
    }
}

/* One table entry by its definition: the source pixel whose guide is nearest
 * to the bin representative, scanning in raster order and keeping the first
 * minimum, which is the smallest linear index among ties. */
uint32_t orc_lut_entry_k(const orc_guide *src, int32_t key_bits, int32_t key_channels,
                         uint32_t idx)
{
    uint32_t rep[4];
    orc_bin_representative(idx, key_channels, src->bits, key_bits, rep);
    uint64_t best = UINT64_MAX;
    uint32_t best_xy = 0;
    for (int32_t y = 0; y < src->height; ++y) {
        for (int32_t x = 0; x < src->width; ++x) {
            uint64_t d = 0;
            for (int32_t c = 0; c < key_channels; ++c) {
                int64_t diff = (int64_t)rep[c] - (int64_t)guide_value(src, x, y, c);
                d += (uint64_t)(diff * diff);
            }
            if (d < best) {
                best = d;
                best_xy = (uint32_t)x | ((uint32_t)y << 16);
            }
        }
    }
    return best_xy;
}

uint32_t orc_lut_entry(const orc_guide *src, int32_t key_bits, uint32_t idx)
{
    return orc_lut_entry_k(src, key_bits, src->channels, idx);
}

/* A table entry, computed on first use.  Unfilled entries hold ORC_UNSET (no
 * valid entry has x = y = 65535 since source sides are at most 65535).  With
 * no table (keys too wide to tabulate, where the paper turns to search trees)
 * the entry is computed from its definition at every use: the same value. */
static uint32_t lut_lookup(uint32_t *lut, const orc_guide *src, int32_t key_bits,
                           int32_t key_channels, uint32_t idx)
{
    if (!lut)
        return orc_lut_entry_k(src, key_bits, key_channels, idx);
    uint32_t v = __atomic_load_n(&lut[idx], __ATOMIC_RELAXED);
    if (v == ORC_UNSET) {
        v = orc_lut_entry_k(src, key_bits, key_channels, idx);
        __atomic_store_n(&lut[idx], v, __ATOMIC_RELAXED);
    }
    return v;
}

int orc_build_lut(const orc_guide *src, int32_t key_bits, int32_t key_channels, uint32_t *lut,
                  int32_t n_threads)
{
    int64_t n = (int64_t)1 << (key_channels * key_bits);
    (void)n_threads;
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads > 0 ? n_threads : 1)
    for (int64_t i = 0; i < n; ++i)
        lut[i] = orc_lut_entry_k(src, key_bits, key_channels, (uint32_t)i);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* seed hierarchy (Algorithm 2; readings R3-R6)                               */
/* ------------------------------------------------------------------------ */

uint32_t orc_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

uint32_t orc_cell_hash(uint32_t seed, int32_t level, int32_t bx, int32_t by)
{
    uint32_t h = orc_fmix32(seed ^ ((uint32_t)level * 0x9E3779B9u));
    h = orc_fmix32(h ^ (uint32_t)bx);
    h = orc_fmix32(h ^ (uint32_t)by);
    return h;
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0)))
        q -= 1;
    return q;
}

static int64_t clamp64(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* SeedPoint(p, h): the jittered grid point of the cell b = floor(p / h),
 * floor(h * (b + j)) = h * b + floor(h * j), then clamped into the target. */
void orc_seed_point(int64_t px, int64_t py, int32_t level, uint32_t seed,
                    int32_t tgt_w, int32_t tgt_h, int64_t *sx, int64_t *sy)
{
    int64_t h = (int64_t)1 << level;
    int64_t bx = floor_div(px, h);
    int64_t by = floor_div(py, h);
    uint32_t j = orc_cell_hash(seed, level, (int32_t)bx, (int32_t)by);
    int64_t ox = ((int64_t)(j & 0xFFFFu) * h) >> 16;
    int64_t oy = ((int64_t)(j >> 16) * h) >> 16;
    *sx = clamp64(h * bx + ox, 0, tgt_w - 1);
    *sy = clamp64(h * by + oy, 0, tgt_h - 1);
}

/* NearestSeed(p, h): the nearest of the seeds of the 3 x 3 cells around p. */
void orc_nearest_seed(int32_t px, int32_t py, int32_t level, uint32_t seed,
                      int32_t tgt_w, int32_t tgt_h, int32_t *qx, int32_t *qy)
{
    int64_t h = (int64_t)1 << level;
    int64_t best = INT64_MAX, bx = 0, by = 0;
    for (int64_t x = -1; x <= 1; ++x) {
        for (int64_t y = -1; y <= 1; ++y) {
            int64_t sx, sy;
            orc_seed_point(px + h * x, py + h * y, level, seed, tgt_w, tgt_h, &sx, &sy);
            int64_t d = (sx - px) * (sx - px) + (sy - py) * (sy - py);
            if (d < best) {
                best = d;
                bx = sx;
                by = sy;
            }
        }
    }
    *qx = (int32_t)bx;
    *qy = (int32_t)by;
}

/* ParallelStyleBlit for one target pixel: walk the levels from L down to 1;
 * at each, take the nearest seed q, look up u* = LUT(G_T[q]), form the
 * candidate u* + (p - q) and accept it when its guide distance to G_T[p] is
 * within the threshold (R1, R7); the finest level always accepts (R2). */
static void assign_pixel(const orc_guide *tgt, const orc_guide *src, int32_t key_bits,
                         int32_t key_channels, uint32_t *lut, int32_t levels,
                         uint64_t threshold, uint32_t seed, int32_t px, int32_t py,
                         uint32_t *a_out, uint8_t *level_out)
{
    for (int32_t l = levels; l >= 1; --l) {
        int32_t qx, qy;
        orc_nearest_seed(px, py, l, seed, tgt->width, tgt->height, &qx, &qy);
        uint32_t u = lut_lookup(lut, src, key_bits, key_channels,
                                orc_lut_index_k(tgt, qx, qy, key_bits, key_channels));
        int64_t sx = (int64_t)(u & 0xFFFFu) + ((int64_t)px - qx);
        int64_t sy = (int64_t)(u >> 16) + ((int64_t)py - qy);
        if (l > 1) {
            if (sx < 0 || sy < 0 || sx >= src->width || sy >= src->height)
                continue;
            if (guide_distance(src, sx, sy, tgt, px, py) > threshold)
                continue;
        } else {
            sx = clamp64(sx, 0, src->width - 1);
            sy = clamp64(sy, 0, src->height - 1);
        }
        *a_out = (uint32_t)sx | ((uint32_t)sy << 16);
        *level_out = (uint8_t)l;
        return;
    }
}

int orc_assign(const orc_guide *tgt, const orc_guide *src, int32_t key_bits,
               int32_t key_channels, uint32_t *lut, int32_t levels, uint64_t threshold,
               uint32_t seed, uint32_t *assign, uint8_t *level, int32_t n_threads)
{
    (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
    for (int32_t y = 0; y < tgt->height; ++y) {
        for (int32_t x = 0; x < tgt->width; ++x) {
            int64_t i = (int64_t)y * tgt->width + x;
            uint8_t l;
            assign_pixel(tgt, src, key_bits, key_channels, lut, levels, threshold, seed, x, y,
                         &assign[i], &l);
            if (level)
                level[i] = l;
        }
    }
    return 0;
}

int orc_assign_points(const orc_guide *tgt, const orc_guide *src, int32_t key_bits,
                      int32_t key_channels, uint32_t *lut, int32_t levels,
                      uint64_t threshold, uint32_t seed, const int32_t *xs, const int32_t *ys,
                      int64_t n, uint32_t *assign, uint8_t *level)
{
    for (int64_t i = 0; i < n; ++i)
        assign_pixel(tgt, src, key_bits, key_channels, lut, levels, threshold, seed, xs[i],
                     ys[i], &assign[i], &level[i]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* voting (end of Section 3.2; reading R9)                                    */
/* ------------------------------------------------------------------------ */

/* Sum of the co-located source colours over the window of p; returns n. */
static uint32_t vote_sums(const uint32_t *assign, int32_t tgt_w, int32_t tgt_h,
                          const orc_rgba8 *style, int32_t radius, int32_t px, int32_t py,
                          uint32_t sum[4])
{
    uint32_t n = 0;
    sum[0] = sum[1] = sum[2] = sum[3] = 0;
    for (int32_t oy = -radius; oy <= radius; ++oy) {
        for (int32_t ox = -radius; ox <= radius; ++ox) {
            int64_t nx = (int64_t)px + ox, ny = (int64_t)py + oy;
            if (nx < 0 || ny < 0 || nx >= tgt_w || ny >= tgt_h)
                continue;
            uint32_t a = assign[ny * tgt_w + nx];
            int64_t vx = (int64_t)(a & 0xFFFFu) - ox;
            int64_t vy = (int64_t)(a >> 16) - oy;
            if (vx < 0 || vy < 0 || vx >= style->width || vy >= style->height)
                continue;
            const uint8_t *c = style->data + vy * style->row_stride + 4 * vx;
            for (int32_t ch = 0; ch < 4; ++ch)
                sum[ch] += c[ch];
            n += 1;
        }
    }
    return n;
}

int orc_blend_rgba8(const uint32_t *assign, int32_t tgt_w, int32_t tgt_h,
                    const orc_rgba8 *style, int32_t radius, uint8_t *out, int32_t n_threads)
{
    (void)n_threads;
#pragma omp parallel for schedule(static) num_threads(n_threads > 0 ? n_threads : 1)
    for (int32_t y = 0; y < tgt_h; ++y) {
        for (int32_t x = 0; x < tgt_w; ++x) {
            uint32_t sum[4];
            uint32_t n = vote_sums(assign, tgt_w, tgt_h, style, radius, x, y, sum);
            uint8_t *o = out + 4 * ((int64_t)y * tgt_w + x);
            for (int32_t ch = 0; ch < 4; ++ch)
                o[ch] = (uint8_t)((sum[ch] + n / 2) / n);
        }
    }
    return 0;
}

int orc_blend_f32(const uint32_t *assign, int32_t tgt_w, int32_t tgt_h,
                  const orc_rgba8 *style, int32_t radius, double *out, int32_t n_threads)
{
    (void)n_threads;
#pragma omp parallel for schedule(static) num_threads(n_threads > 0 ? n_threads : 1)
    for (int32_t y = 0; y < tgt_h; ++y) {
        for (int32_t x = 0; x < tgt_w; ++x) {
            uint32_t sum[4];
            uint32_t n = vote_sums(assign, tgt_w, tgt_h, style, radius, x, y, sum);
            double *o = out + 4 * ((int64_t)y * tgt_w + x);
            for (int32_t ch = 0; ch < 4; ++ch)
                o[ch] = (double)sum[ch] / (255.0 * (double)n);
        }
    }
    return 0;
}

/* Assignment plus vote for a list of target pixels, computing every window
 * neighbour's assignment from scratch: slow, but needs no full-frame buffer,
 * so it can check sampled pixels of frames of any size. */
int orc_stylize_points(const orc_guide *tgt, const orc_guide *src, const orc_rgba8 *style,
                       int32_t key_bits, int32_t key_channels, uint32_t *lut, int32_t levels,
                       uint64_t threshold,
                       int32_t radius, uint32_t seed, const int32_t *xs, const int32_t *ys,
                       int64_t n, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t sum[4] = {0, 0, 0, 0};
        uint32_t cnt = 0;
        for (int32_t oy = -radius; oy <= radius; ++oy) {
            for (int32_t ox = -radius; ox <= radius; ++ox) {
                int64_t nx = (int64_t)xs[i] + ox, ny = (int64_t)ys[i] + oy;
                if (nx < 0 || ny < 0 || nx >= tgt->width || ny >= tgt->height)
                    continue;
                uint32_t a;
                uint8_t l;
                assign_pixel(tgt, src, key_bits, key_channels, lut, levels, threshold, seed,
                             (int32_t)nx, (int32_t)ny, &a, &l);
                int64_t vx = (int64_t)(a & 0xFFFFu) - ox;
                int64_t vy = (int64_t)(a >> 16) - oy;
                if (vx < 0 || vy < 0 || vx >= style->width || vy >= style->height)
                    continue;
                const uint8_t *c = style->data + vy * style->row_stride + 4 * vx;
                for (int32_t ch = 0; ch < 4; ++ch)
                    sum[ch] += c[ch];
                cnt += 1;
            }
        }
        for (int32_t ch = 0; ch < 4; ++ch)
            out[4 * i + ch] = (uint8_t)((sum[ch] + cnt / 2) / cnt);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* lookup-only comparator (Section 4: texture mapping / The Lit Sphere)       */
/* ------------------------------------------------------------------------ */

/* Each target pixel copies the style at the table entry of its own guide
 * value, C_T[p] = C_S[LUT(G_T[p])]: the per-pixel mapping the paper compares
 * its chunk transfer against.  No seeds, levels or vote. */
int orc_lookup_only(const orc_guide *tgt, const orc_guide *src, const orc_rgba8 *style,
                    int32_t key_bits, int32_t key_channels, uint32_t *lut, uint8_t *out)
{
    for (int32_t y = 0; y < tgt->height; ++y) {
        for (int32_t x = 0; x < tgt->width; ++x) {
            uint32_t u = lut_lookup(lut, src, key_bits, key_channels,
                                    orc_lut_index_k(tgt, x, y, key_bits, key_channels));
            const uint8_t *c = style->data + (int64_t)(u >> 16) * style->row_stride + 4 * (u & 0xFFFFu);
            uint8_t *o = out + 4 * ((int64_t)y * tgt->width + x);
            for (int32_t ch = 0; ch < 4; ++ch)
                o[ch] = c[ch];
        }
    }
    return 0;
}
