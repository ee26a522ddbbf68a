// kern_batch_hooke.cu -- explicit instantiation of the batched inversion kernels for
// F_HOOKE (kept apart so the build compiles them in parallel).
#include "kern_batch.cuh"

namespace afm {
template struct BatchOps<F_HOOKE>;
}  // namespace afm
