// Frame and batch kernels of blend radii 8-15, instantiated for 8-bit guides with 1 channel.
#include "sb_frame.cuh"

namespace sb {
cudaError_t launch_frame_wide_c1b8(const FrameArgs &a, cudaStream_t s) {
    return launch_stylize<1, 8, kNarrowMaxRadius + 1, kMaxFusedRadius>(a, s);
}
cudaError_t launch_batch_wide_c1b8(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                                   cudaStream_t s) {
    return launch_batch32<1, 8, kNarrowMaxRadius + 1, kMaxFusedRadius>(b, r, max_levels, queue, s);
}
}  // namespace sb
