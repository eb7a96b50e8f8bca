// Internal declarations of the GB300 StyleBlit library (not installed).
//
// Guide pixels travel packed in one uint32: 8-bit guides hold channel c in
// bits [8c, 8c+8), 16-bit guides in bits [16c, 16c+16).  Supported formats:
// 8-bit with 1..4 channels and 16-bit with 1..2 channels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "styleblit.h"

struct sb_lut {
    // table: 2^(key_channels * key_bits) entries packed x | y << 16, for keys
    // of at most 24 bits; wider keys: nullptr, and nn_bounds holds the search
    // index (tile and super-tile guide boxes) queried per seed
    uint32_t *entries = nullptr;
    uint4 *nn_bounds = nullptr;
    uint32_t *src_packed = nullptr;  // device, the source guide, one packed uint32 per pixel
    int64_t n_entries = 0;
    int32_t channels = 0;
    int32_t bits = 0;
    int32_t key_bits = 0;
    int32_t key_channels = 0;      // the table keys the first key_channels guide channels
    int32_t src_w = 0;
    int32_t src_h = 0;
    int32_t device = 0;
};

namespace sb {

// No source position (a pixel outside the target).  Its x field (0xC000) stays
// above every valid coordinate (< 32767) after subtracting any window offset
// (|o| <= 15) without a borrow, so A - o of this value is always out of the
// source and never equals a valid A + o: no separate test is needed.
constexpr uint32_t kInvalid = 0xC000C000u;
constexpr int kMaxSourceSide = 32767;         // keeps packed-position arithmetic carry-free
constexpr int kMaxTargetSide = 65535;
constexpr int kMaxLevels = 15;          // 2^15 = 32768 seed spacing
constexpr int kMaxBlendRadius = 15;
constexpr int kMaxFusedRadius = 15;
constexpr int kMaxKeyBitsTotal = 24;        // widest key with a table (16 Mi entries)

// error plumbing (host)
sb_status fail(sb_status st, const std::string &msg);
sb_status ok();
sb_status cuda_fail(cudaError_t e, const char *what);
sb_status check_guide(const sb_guide *g, const char *name, bool is_source);
sb_status check_style(const sb_rgba8 *s, const char *name);
int guide_format_id(int channels, int bits);   // 0..5, or -1

// ---------------------------------------------------------------------------
// device helpers shared by the kernels of this library
// ---------------------------------------------------------------------------

// fmix32: the 32-bit finaliser of MurmurHash3 (Austin Appleby, public domain).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Jitter hash of a seed cell (replaces the random jitter table of SeedPoint in
// Algorithm 2): H = fmix32(fmix32(level_key ^ bx) ^ by) with
// level_key = fmix32(seed ^ level * 0x9E3779B9).
__device__ __forceinline__ uint32_t level_key(uint32_t seed, int level) {
    return fmix32(seed ^ ((uint32_t)level * 0x9E3779B9u));
}
__device__ __forceinline__ uint32_t cell_hash(uint32_t lkey, int bx, int by) {
    return fmix32(fmix32(lkey ^ (uint32_t)bx) ^ (uint32_t)by);
}

template <int C, int B>
struct GuideFmt {
    static_assert((B == 8 && C >= 1 && C <= 4) || (B == 16 && C >= 1 && C <= 2), "format");
    static constexpr int kBytes = C * B / 8;

    // packed pixel (x, y) of a guide; alignment checked on the host
    __device__ __forceinline__ static uint32_t load(const uint8_t *base, int64_t stride, int x,
                                                    int y) {
        const uint8_t *row = base + (int64_t)y * stride;
        if constexpr (B == 8) {
            if constexpr (C == 1) return __ldg(row + x);
            if constexpr (C == 2) return __ldg(reinterpret_cast<const uint16_t *>(row) + x);
            if constexpr (C == 3) {
                const uint8_t *p = row + 3 * (int64_t)x;
                return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8) |
                       ((uint32_t)__ldg(p + 2) << 16);
            }
            if constexpr (C == 4) return __ldg(reinterpret_cast<const uint32_t *>(row) + x);
        } else {
            if constexpr (C == 1) return __ldg(reinterpret_cast<const uint16_t *>(row) + x);
            if constexpr (C == 2) return __ldg(reinterpret_cast<const uint32_t *>(row) + x);
        }
        return 0;
    }

    __device__ __forceinline__ static uint32_t chan(uint32_t v, int c) {
        if constexpr (B == 8) return (v >> (8 * c)) & 0xFFu;
        else return (v >> (16 * c)) & 0xFFFFu;
    }

    // squared Euclidean guide distance; fits 32 bits except 16-bit x 2
    __device__ __forceinline__ static uint64_t dist(uint32_t a, uint32_t b) {
        if constexpr (B == 8) {
            // per-byte |a - b|, then the 4-way byte dot product of that with
            // itself (unused channels are zero in both); exact in 32 bits
            const uint32_t d = __vabsdiffu4(a, b);
            return __dp4a(d, d, 0u);
        } else if constexpr (C == 1) {
            // t^2 < 2^32, so the square modulo 2^32 is exact for either sign
            const uint32_t t = (a & 0xFFFFu) - (b & 0xFFFFu);
            return t * t;
        } else {
            const int t0 = (int)(a & 0xFFFFu) - (int)(b & 0xFFFFu);
            const int t1 = (int)(a >> 16) - (int)(b >> 16);
            return (uint64_t)((int64_t)t0 * t0) + (uint64_t)((int64_t)t1 * t1);
        }
    }

    // table index: keys (top key_bits bits) of the first key_channels
    // channels, channel 0 lowest
    __device__ __forceinline__ static uint32_t key(uint32_t v, int key_bits, int key_channels) {
        const int z = B - key_bits;
        uint32_t idx = 0;
#pragma unroll
        for (int c = 0; c < C; ++c)
            if (c < key_channels) idx |= (chan(v, c) >> z) << (c * key_bits);
        return idx;
    }

    // v with the channels from key_channels on cleared
    __device__ __forceinline__ static uint32_t key_part(uint32_t v, int key_channels) {
        return key_channels * B >= 32 ? v : (v & ((1u << (key_channels * B)) - 1u));
    }
};

// Dispatch a functor templated on <C, B> for a runtime guide format.
template <typename F>
__host__ bool dispatch_format(int channels, int bits, F &&f) {
    if (bits == 8) {
        switch (channels) {
            case 1: f.template operator()<1, 8>(); return true;
            case 2: f.template operator()<2, 8>(); return true;
            case 3: f.template operator()<3, 8>(); return true;
            case 4: f.template operator()<4, 8>(); return true;
        }
    } else if (bits == 16) {
        switch (channels) {
            case 1: f.template operator()<1, 16>(); return true;
            case 2: f.template operator()<2, 16>(); return true;
        }
    }
    return false;
}

}  // namespace sb
