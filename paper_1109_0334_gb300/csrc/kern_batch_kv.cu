// kern_batch_kv.cu -- explicit instantiation of the batched inversion kernels for
// F_DMT_KV (kept apart so the build compiles them in parallel).
#include "kern_batch.cuh"

namespace afm {
template struct BatchOps<F_DMT_KV>;
}  // namespace afm
