// float32-bulk batched ensemble classes for 256 x 256 grids (every batch schedule).
#include "spfc_batch.cuh"

namespace spfc {
BatchClassBase* make_batch_class_f32_256(int sched, const std::vector<Params>& params, cudaStream_t st,
                                         int* status, std::string* err) {
  return make_batch_class_n<float, 256>(sched, params, st, status, err);
}
}  // namespace spfc
