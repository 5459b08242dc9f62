// dyn.cu -- dispatch of the bucketed kernels with a dynamic tail
// (hygt_batch_dyn.cuh).
#include "hygt_batch_dyn.cuh"

namespace hygt {

// instantiated in dyn_6_fwd.cu ... dyn_8_inv.cu
extern template cudaError_t launch_dyn_n<6, 0>(const BatchParams&, void*, int, cudaStream_t,
                                               const BatchTune&);
extern template cudaError_t launch_dyn_n<6, 1>(const BatchParams&, void*, int, cudaStream_t,
                                               const BatchTune&);
extern template cudaError_t launch_dyn_n<8, 0>(const BatchParams&, void*, int, cudaStream_t,
                                               const BatchTune&);
extern template cudaError_t launch_dyn_n<8, 1>(const BatchParams&, void*, int, cudaStream_t,
                                               const BatchTune&);

bool batch_dyn_ok(int log2n, int layout, int stage) {
  const bool lay = (log2n == 6 && (layout == 0 || layout == 3)) ||
                   (log2n == 8 && (layout == 0 || layout == 4 || layout == 5));
  return lay && stage >= -1 && stage <= 3 && (stage != 3 || layout == 0);
}

cudaError_t launch_batch_dyn(int kind, int log2n, const BatchParams& p, void* counters,
                             int tail_64ths, cudaStream_t stream, const BatchTune& tune) {
  if (!counters || tail_64ths < 1 || tail_64ths > 32 ||
      !batch_dyn_ok(log2n, tune.layout, tune.stage))
    return cudaErrorInvalidConfiguration;
  if (log2n == 6)
    return kind == 0 ? launch_dyn_n<6, 0>(p, counters, tail_64ths, stream, tune)
                     : launch_dyn_n<6, 1>(p, counters, tail_64ths, stream, tune);
  return kind == 0 ? launch_dyn_n<8, 0>(p, counters, tail_64ths, stream, tune)
                   : launch_dyn_n<8, 1>(p, counters, tail_64ths, stream, tune);
}

}  // namespace hygt
