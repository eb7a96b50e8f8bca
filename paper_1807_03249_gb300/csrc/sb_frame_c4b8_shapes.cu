// Batch kernels with 16- and 64-row tiles instantiated for 8-bit guides with 4 channels.
#include "sb_frame.cuh"

namespace sb {
cudaError_t launch_batch_shaped_c4b8(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s) {
    return launch_batch_shaped<4, 8>(b, r, th, max_levels, queue, s);
}
}  // namespace sb
