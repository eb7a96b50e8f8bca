// Host-side argument validation, status strings and error plumbing of the
// StyleBlit C ABI.
#include <cstdint>
#include <cstdio>
#include <string>

#include "sb_internal.cuh"

namespace sb {

static thread_local std::string g_last_error;

sb_status fail(sb_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

sb_status ok() {
    g_last_error.clear();
    return SB_OK;
}

sb_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(SB_ERR_OOM, m);
    return fail(SB_ERR_CUDA, m);
}

int guide_format_id(int channels, int bits) {
    if (bits == 8 && channels >= 1 && channels <= 4) return channels - 1;
    if (bits == 16 && channels >= 1 && channels <= 2) return 3 + channels;
    return -1;
}

// natural alignment of one packed pixel load
static int pixel_alignment(int channels, int bits) {
    int bytes = channels * bits / 8;
    if (bytes == 3) return 1;
    return bytes;
}

sb_status check_guide(const sb_guide *g, const char *name, bool is_source) {
    char buf[256];
    if (!g) {
        std::snprintf(buf, sizeof buf, "%s: NULL guide descriptor", name);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if (g->bits != 8 && g->bits != 16) {
        std::snprintf(buf, sizeof buf, "%s: bits must be 8 or 16 (got %d)", name, g->bits);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if (g->channels < 1 || g->channels > 4) {
        std::snprintf(buf, sizeof buf, "%s: channels must be 1..4 (got %d)", name, g->channels);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if (guide_format_id(g->channels, g->bits) < 0) {
        std::snprintf(buf, sizeof buf, "%s: %d-bit guides with %d channels are not supported",
                      name, g->bits, g->channels);
        return fail(SB_ERR_UNSUPPORTED, buf);
    }
    int max_side = is_source ? kMaxSourceSide : kMaxTargetSide;
    int min_side = is_source ? 1 : 0;
    if (g->width < min_side || g->height < min_side || g->width > max_side ||
        g->height > max_side) {
        std::snprintf(buf, sizeof buf, "%s: size %dx%d outside [%d, %d]", name, g->width,
                      g->height, min_side, max_side);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if ((int64_t)g->width * g->height == 0) return SB_OK;
    int64_t row_bytes = (int64_t)g->width * g->channels * (g->bits / 8);
    if (!g->data) {
        std::snprintf(buf, sizeof buf, "%s: NULL data", name);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if (g->row_stride < row_bytes) {
        std::snprintf(buf, sizeof buf, "%s: row_stride %lld < row bytes %lld", name,
                      (long long)g->row_stride, (long long)row_bytes);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    int al = pixel_alignment(g->channels, g->bits);
    if (((uintptr_t)g->data % al) != 0 || (g->row_stride % al) != 0) {
        std::snprintf(buf, sizeof buf, "%s: data and row_stride must be %d-byte aligned", name,
                      al);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    return SB_OK;
}

sb_status check_style(const sb_rgba8 *s, const char *name) {
    char buf[256];
    if (!s || !s->data) {
        std::snprintf(buf, sizeof buf, "%s: NULL style", name);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if (s->width < 1 || s->height < 1 || s->width > kMaxSourceSide ||
        s->height > kMaxSourceSide) {
        std::snprintf(buf, sizeof buf, "%s: size %dx%d outside [1, %d]", name, s->width,
                      s->height, kMaxSourceSide);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    if (s->row_stride < 4LL * s->width || (s->row_stride % 4) != 0 ||
        ((uintptr_t)s->data % 4) != 0) {
        std::snprintf(buf, sizeof buf, "%s: row_stride must be >= 4*width and data/stride 4-byte aligned", name);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    // the kernels address the style with 32-bit pixel offsets
    if ((int64_t)s->height * (s->row_stride / 4) > INT32_MAX) {
        std::snprintf(buf, sizeof buf, "%s: height * row_stride must stay below 2^33 bytes", name);
        return fail(SB_ERR_INVALID_ARG, buf);
    }
    return SB_OK;
}

}  // namespace sb

extern "C" const char *sb_status_string(sb_status status) {
    switch (status) {
        case SB_OK: return "SB_OK";
        case SB_ERR_INVALID_ARG: return "SB_ERR_INVALID_ARG: an argument is out of range";
        case SB_ERR_UNSUPPORTED: return "SB_ERR_UNSUPPORTED: valid request not implemented";
        case SB_ERR_CUDA: return "SB_ERR_CUDA: a CUDA call failed";
        case SB_ERR_OOM: return "SB_ERR_OOM: device allocation failed";
        case SB_ERR_TIMEOUT: return "SB_ERR_TIMEOUT: a bounded device wait gave up";
    }
    return "unknown sb_status";
}

extern "C" const char *sb_last_error(void) { return sb::g_last_error.c_str(); }

extern "C" int32_t sb_version(void) { return 10000; }
