// Frame kernels instantiated for 8-bit guides with 2 channels.
#include "sb_frame.cuh"

namespace sb {
cudaError_t launch_frame_c2b8(int mode, const FrameArgs &a, cudaStream_t s) {
    return launch_frame<2, 8>(mode, a, s);
}
cudaError_t launch_batch_c2b8(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                              cudaStream_t s) {
    return launch_batch<2, 8>(b, r, max_levels, queue, s);
}
}  // namespace sb
