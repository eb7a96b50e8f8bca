// Frame kernels instantiated for 16-bit guides with 2 channels.
#include "sb_frame.cuh"

namespace sb {
cudaError_t launch_frame_c2b16(int mode, const FrameArgs &a, cudaStream_t s) {
    return launch_frame<2, 16>(mode, a, s);
}
cudaError_t launch_batch_c2b16(const BatchArgs &b, int r, int max_levels, TileQueue *queue,
                              cudaStream_t s) {
    return launch_batch<2, 16>(b, r, max_levels, queue, s);
}
}  // namespace sb
