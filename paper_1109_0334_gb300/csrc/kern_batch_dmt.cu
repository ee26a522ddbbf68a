// kern_batch_dmt.cu -- explicit instantiation of the batched inversion kernels for
// F_DMT (kept apart so the build compiles them in parallel).
#include "kern_batch.cuh"

namespace afm {
template struct BatchOps<F_DMT>;
}  // namespace afm
