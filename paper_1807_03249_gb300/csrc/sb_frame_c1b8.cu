// Frame kernels and 32-row batch kernels of blend radii up to 7, instantiated
// for 8-bit guides with 1 channel; the entry points of the format.
#include "sb_frame.cuh"

namespace sb {
cudaError_t launch_frame_c1b8(int mode, const FrameArgs &a, cudaStream_t s) {
    if (mode == kStylize && a.radius > kNarrowMaxRadius) return launch_frame_wide_c1b8(a, s);
    return launch_frame_narrow<1, 8>(mode, a, s);
}
cudaError_t launch_batch_c1b8(const BatchArgs &b, int r, int th, int max_levels,
                              TileQueue *queue, cudaStream_t s) {
    if (th != kTH) return launch_batch_shaped_c1b8(b, r, th, max_levels, queue, s);
    if (r > kNarrowMaxRadius) return launch_batch_wide_c1b8(b, r, max_levels, queue, s);
    return launch_batch32<1, 8, 0, kNarrowMaxRadius>(b, r, max_levels, queue, s);
}
}  // namespace sb
