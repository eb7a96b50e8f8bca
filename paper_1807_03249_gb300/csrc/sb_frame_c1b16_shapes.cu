// Batch kernels with 16- and 64-row tiles instantiated for 16-bit guides with 1 channel.
#include "sb_frame.cuh"

namespace sb {
cudaError_t launch_batch_shaped_c1b16(const BatchArgs &b, int r, int th, int max_levels,
                                     TileQueue *queue, cudaStream_t s) {
    return launch_batch_shaped<1, 16>(b, r, th, max_levels, queue, s);
}
}  // namespace sb
