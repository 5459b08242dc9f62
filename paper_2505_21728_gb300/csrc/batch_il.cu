// batch_il.cu -- the set-interleaved order (stage 4 of the launch tuning) for
// 4x4 blocks, the block size whose neighbours in a line belong to other sets.
#include "hygt_batch_il.cuh"

namespace hygt {

bool batch_il_ok(int log2n, int layout) { return log2n == 4 && (layout == 0 || layout == 2); }

cudaError_t launch_batch_il(int kind, int log2n, const BatchParams& p, cudaStream_t stream,
                            const BatchTune& tune) {
  if (!batch_il_ok(log2n, tune.layout)) return cudaErrorInvalidConfiguration;
  if (kind == 0)
    return tune.layout == 2 ? launch_il_variant<4, 0, 2>(p, stream, tune)
                            : launch_il_variant<4, 0, 0>(p, stream, tune);
  return tune.layout == 2 ? launch_il_variant<4, 1, 2>(p, stream, tune)
                          : launch_il_variant<4, 1, 0>(p, stream, tune);
}

}  // namespace hygt
