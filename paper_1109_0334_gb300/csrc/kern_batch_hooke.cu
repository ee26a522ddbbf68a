// kern_batch_hooke.cu -- the batched inversion kernels instantiated for
// F_HOOKE (kept apart so the build compiles them in parallel).
#include "kern_batch.cuh"

namespace afm {
template <>
cudaError_t batch_occupancy_of<F_HOOKE>(int m, int kp, int P, int D, int spc2, bool pp,
                                  int* blocks) {
    return BatchOps<F_HOOKE>::occupancy(m, kp, P, D, spc2, pp, blocks);
}
template <>
cudaError_t batch_launch_of<F_HOOKE>(const KConst<float>& K, const PsoConst& pc, const BatchArgs& a,
                                  int kp, int grid, cudaStream_t st) {
    return BatchOps<F_HOOKE>::launch(K, pc, a, kp, grid, st);
}
}  // namespace afm
