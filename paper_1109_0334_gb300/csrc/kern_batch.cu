// kern_batch.cu -- many independent pixel inversions (IP of Sec. 2.3, one per
// pixel of an image scan) in one persistent launch.  Each block pulls pixels
// from an atomic queue (longest record first) and runs that pixel's whole
// particle swarm (Sec. 3.4, Eq. 8) on chip: positions, velocities and
// personal bests in shared memory, the global best reduced with warp shuffles
// and one shared-memory pass, every swarm evaluation the fused RK4 (Eq. 2) +
// misfit (Eq. 5) time loop with KP particles per thread.  No block waits on
// another block.  Every pixel's winner is then re-evaluated in FP64 by
// multiple shooting in time (kern_reeval_batch.cu).
// The kernels are in kern_batch.cuh; this file holds the force dispatch, the
// queue-order sort and the shared helpers.
#include <type_traits>

#include "kern_batch.cuh"

namespace afm {

int batch_threads(int P, int kp) { return ((P + kp - 1) / kp + 31) / 32 * 32; }

int batch_max_threads(int kp) { return kp == 1 ? 1024 : 512; }

size_t batch_smem(int P, int D, int spc2, bool pp) {
    const size_t tab = (size_t)((spc2 + 1 + 3) & ~3);
    const size_t kc = pp ? (size_t)batch_kc_words<true>() : 0;
    return sizeof(float) * (kc + tab + 3 * (size_t)D * P);
}

// ---------------------------------------------------------------------------
// Per-pixel drive tables (batches whose pixels differ in their problem): the
// arithmetic of build_drive_table in FP64 from each pixel's constants, also
// rounded to FP32.  One thread per (pixel, phase).
// ---------------------------------------------------------------------------
__global__ void pix_tables_kernel(const KConst<double>* __restrict__ kd, int n_pix, int spc2,
                                  int ld, double* __restrict__ tab64, float* __restrict__ tab32) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int pix = (int)(t / (spc2 + 1)), j = (int)(t % (spc2 + 1));
    if (pix >= n_pix) return;
    const int jj = j == spc2 ? 0 : j;
    const double ph = 6.283185307179586476925 * (double)jj / (double)spc2 + kd[pix].drive_phase;
    const double g = kd[pix].drive_amp * sin(ph);
    tab64[(size_t)pix * ld + j] = g;
    tab32[(size_t)pix * ld + j] = (float)g;
}

cudaError_t launch_pix_tables(const PixConst& pc, int n_pix, int spc2, cudaStream_t st) {
    if (pc.kd == nullptr || pc.ld < spc2 + 1) return cudaErrorInvalidValue;
    const long long total = (long long)n_pix * (spc2 + 1);
    const int threads = 256;
    pix_tables_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(
        pc.kd, n_pix, spc2, pc.ld, const_cast<double*>(pc.tab64), const_cast<float*>(pc.tab32));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Longest-record-first order: one block sorts (length desc, index asc) keys
// with a bitonic network in shared memory.
// ---------------------------------------------------------------------------
constexpr int SORT_MAX = 16384;

__global__ void __launch_bounds__(1024) sort_kernel(const int64_t* __restrict__ off, int n_pix,
                                                    int len, int* __restrict__ order) {
    extern __shared__ unsigned long long key[];
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        if (i < n_pix) {
            long long L = off[i + 1] - off[i];
            unsigned long long inv = 0x7fffffffull - (unsigned long long)min(max(L, 0ll), 0x7fffffffll);
            key[i] = (inv << 32) | (unsigned)i;
        } else {
            key[i] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= len; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    unsigned long long a = key[i], b = key[l];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n_pix; i += blockDim.x) order[i] = (int)(key[i] & 0xffffffffu);
}

cudaError_t batch_sort(const int64_t* off, int n_pix, int* order, cudaStream_t st) {
    if (n_pix > SORT_MAX || n_pix < 1) return cudaErrorInvalidValue;
    int len = 1;
    while (len < n_pix) len <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)len;
    cudaError_t e = cudaFuncSetAttribute(sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(unsigned long long) * SORT_MAX));
    if (e != cudaSuccess) return e;
    sort_kernel<<<1, 1024, smem, st>>>(off, n_pix, len, order);
    return cudaGetLastError();
}

int batch_sort_max() { return SORT_MAX; }

// The kernels of each force law are instantiated in kern_batch_<law>.cu (so
// that they compile in parallel); this file only calls their entry points.
#define AFM_BATCH_DECLARE(F)                                                                   \
    template <> cudaError_t batch_occupancy_of<F>(int, int, int, int, int, bool, int*);        \
    template <> cudaError_t batch_launch_of<F>(const KConst<float>&, const PsoConst&,          \
                                               const BatchArgs&, int, int, cudaStream_t);
AFM_BATCH_DECLARE(F_LINEAR)
AFM_BATCH_DECLARE(F_DMT)
AFM_BATCH_DECLARE(F_DMT_KV)
AFM_BATCH_DECLARE(F_HOOKE)
AFM_BATCH_DECLARE(F_SPRING_DAMPER)
#undef AFM_BATCH_DECLARE



template <typename F>
static cudaError_t by_force(int force, F&& f) {
    switch (force) {
        case F_LINEAR: return f(std::integral_constant<int, F_LINEAR>{});
        case F_DMT: return f(std::integral_constant<int, F_DMT>{});
        case F_DMT_KV: return f(std::integral_constant<int, F_DMT_KV>{});
        case F_HOOKE: return f(std::integral_constant<int, F_HOOKE>{});
        case F_SPRING_DAMPER: return f(std::integral_constant<int, F_SPRING_DAMPER>{});
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_occupancy(int m, int force, int kp, int P, int D, int spc2, bool pp,
                            int* blocks_per_sm) {
    return by_force(force, [&](auto Fc) {
        return batch_occupancy_of<decltype(Fc)::value>(m, kp, P, D, spc2, pp, blocks_per_sm);
    });
}

cudaError_t launch_batch(const KConst<float>& K, const PsoConst& pc, const BatchArgs& a, int kp,
                         int grid, cudaStream_t st) {
    return by_force(K.force, [&](auto Fc) {
        return batch_launch_of<decltype(Fc)::value>(K, pc, a, kp, grid, st);
    });
}

}  // namespace afm
