// float32-bulk batched ensemble classes for grids below 128.
#include "spfc_batch.cuh"

namespace spfc {
BatchClassBase* make_batch_class_f32_small(int N, const std::vector<Params>& params, cudaStream_t st, int* status,
                                           std::string* err) {
  return make_batch_class_small<float>(N, params, st, status, err);
}
}  // namespace spfc
