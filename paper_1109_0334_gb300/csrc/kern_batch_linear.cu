// kern_batch_linear.cu -- explicit instantiation of the batched inversion kernels for
// F_LINEAR (kept apart so the build compiles them in parallel).
#include "kern_batch.cuh"

namespace afm {
template struct BatchOps<F_LINEAR>;
}  // namespace afm
