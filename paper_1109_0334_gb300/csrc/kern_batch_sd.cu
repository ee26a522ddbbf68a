// kern_batch_sd.cu -- explicit instantiation of the batched inversion kernels for
// F_SPRING_DAMPER (kept apart so the build compiles them in parallel).
#include "kern_batch.cuh"

namespace afm {
template struct BatchOps<F_SPRING_DAMPER>;
}  // namespace afm
