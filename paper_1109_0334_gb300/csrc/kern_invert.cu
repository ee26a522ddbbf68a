// kern_invert.cu -- particle-swarm optimisation (Sec. 3.4, Eq. 8) and the
// fused inversion (IP of Sec. 2.3): each launch moves every particle (Eq. 8),
// integrates its cantilever (Eq. 2, RK4), sums its misfit (Eq. 5), updates
// its personal best and folds it into the swarm's global best with one
// 64-bit atomicMin per warp.  A launch boundary separates iterations, so the
// swarm update is synchronous, as in the oracle.
#include <type_traits>

#include "../../include/afminv.h"
#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

template <typename F>
static cudaError_t dispatch_mf(int m, int force, F&& f) {
    auto byF = [&](auto Mc) -> cudaError_t {
        switch (force) {
            case F_LINEAR: return f(Mc, std::integral_constant<int, F_LINEAR>{});
            case F_DMT: return f(Mc, std::integral_constant<int, F_DMT>{});
            case F_DMT_KV: return f(Mc, std::integral_constant<int, F_DMT_KV>{});
            case F_HOOKE: return f(Mc, std::integral_constant<int, F_HOOKE>{});
            case F_SPRING_DAMPER: return f(Mc, std::integral_constant<int, F_SPRING_DAMPER>{});
        }
        return cudaErrorInvalidValue;
    };
    if (m == 1) return byF(std::integral_constant<int, 1>{});
    if (m == 3) return byF(std::integral_constant<int, 3>{});
    return byF(std::integral_constant<int, AFM_MAXM>{});
}

// Global-best key: misfit bits (non-negative floats order like their bit
// patterns) above the particle index, so the minimum key is the lowest misfit
// with the lowest index among ties.
__device__ __forceinline__ unsigned long long best_key(float S, int p) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)p;
}

__device__ __forceinline__ float sanitize_misfit(float s, int* flags) {
    if (!(s < INFINITY)) {
        if (flags) atomicAdd(flags, 1);
        return INFINITY;
    }
    return s > 0.f ? s : 0.f;
}

__device__ __forceinline__ void warp_min_atomic(unsigned long long key, unsigned long long* dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(dst, key);
}

// ---------------------------------------------------------------------------
// Swarm initialisation: x ~ U[0,1), v = (U[0,1) - x)/2 (tags 0 and 1).
// ---------------------------------------------------------------------------
__global__ void pso_init_kernel(const PsoConst pc, SwarmPtrs sw) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        *sw.gkey[0] = ~0ull;
        *sw.gkey[1] = ~0ull;
        if (sw.flags) sw.flags[0] = 0;
    }
    if (p >= pc.P) return;
    const uint32_t id = pc.p0 + (uint32_t)p;   // swarm-wide particle index
    for (int b = 0; b * 4 < pc.D; ++b) {
        uint4 w0 = philox_draw(pc.seed, id, 0u, pc.pixel, 0u, (uint32_t)b);
        uint4 w1 = philox_draw(pc.seed, id, 0u, pc.pixel, 1u, (uint32_t)b);
        for (int k = 0; k < 4 && b * 4 + k < pc.D; ++k) {
            const int d = b * 4 + k;
            const float u0 = unif24(word_of(w0, k)), u1 = unif24(word_of(w1, k));
            sw.x[(size_t)d * pc.P + p] = u0;
            sw.v[(size_t)d * pc.P + p] = (u1 - u0) * 0.5f;
        }
    }
    sw.pbS[p] = INFINITY;
}

cudaError_t launch_pso_init(const PsoConst& pc, const SwarmPtrs& sw, cudaStream_t st) {
    const int threads = 128;
    pso_init_kernel<<<(pc.P + threads - 1) / threads, threads, 0, st>>>(pc, sw);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Standalone step, part 1: personal bests and global best from given misfits.
// ---------------------------------------------------------------------------
__global__ void pso_best_kernel(const PsoConst pc, SwarmPtrs sw, const float* __restrict__ S, int it) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = ~0ull;
    if (p < pc.P) {
        const float s = sanitize_misfit(S[p], sw.flags);
        float best = sw.pbS[p];
        if (s < best || it == 0) {
            if (s < best) best = s;
            sw.pbS[p] = best;
            for (int d = 0; d < pc.D; ++d)
                sw.pb[0][(size_t)d * pc.P + p] = sw.x[(size_t)d * pc.P + p];
        }
        key = best_key(best, (int)(pc.p0 + (uint32_t)p));
    }
    warp_min_atomic(key, sw.gkey[0]);
}

// Standalone step, part 2: Eq. 8 move using the global best of part 1.
__global__ void pso_move_kernel(const PsoConst pc, SwarmPtrs sw, int it) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pc.P) return;
    const unsigned long long key = *sw.gkey[0];
    const int g = min((int)(key & 0x7fffffffu), pc.P - 1);
    float x[AFM_MAXD], v[AFM_MAXD], pb[AFM_MAXD], gb[AFM_MAXD];
    for (int d = 0; d < pc.D; ++d) {
        const size_t q = (size_t)d * pc.P;
        x[d] = sw.x[q + p];
        v[d] = sw.v[q + p];
        pb[d] = sw.pb[0][q + p];
        gb[d] = sw.pb[0][q + g];
    }
    pso_move_dev(pc, x, v, pb, gb, p, it);
    for (int d = 0; d < pc.D; ++d) {
        sw.x[(size_t)d * pc.P + p] = x[d];
        sw.v[(size_t)d * pc.P + p] = v[d];
    }
}

// The same move with the global best position given (gb [D], device): the
// particles of a slice of a swarm split across processes.
__global__ void pso_move_given_kernel(const PsoConst pc, SwarmPtrs sw, const float* __restrict__ gbp,
                                      int it) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pc.P) return;
    float x[AFM_MAXD], v[AFM_MAXD], pb[AFM_MAXD], gb[AFM_MAXD];
    for (int d = 0; d < pc.D; ++d) {
        const size_t q = (size_t)d * pc.P;
        x[d] = sw.x[q + p];
        v[d] = sw.v[q + p];
        pb[d] = sw.pb[0][q + p];
        gb[d] = gbp[d];
    }
    pso_move_dev(pc, x, v, pb, gb, (int)(pc.p0 + (uint32_t)p), it);
    for (int d = 0; d < pc.D; ++d) {
        sw.x[(size_t)d * pc.P + p] = x[d];
        sw.v[(size_t)d * pc.P + p] = v[d];
    }
}

cudaError_t launch_pso_move_given(const PsoConst& pc, const SwarmPtrs& sw, const float* gb, int it,
                                  cudaStream_t st) {
    const int threads = 128;
    pso_move_given_kernel<<<(pc.P + threads - 1) / threads, threads, 0, st>>>(pc, sw, gb, it);
    return cudaGetLastError();
}

cudaError_t launch_pso_best(const PsoConst& pc, const SwarmPtrs& sw, const float* S, int it,
                            cudaStream_t st) {
    const int threads = 128;
    pso_best_kernel<<<(pc.P + threads - 1) / threads, threads, 0, st>>>(pc, sw, S, it);
    return cudaGetLastError();
}

cudaError_t launch_pso_move(const PsoConst& pc, const SwarmPtrs& sw, int it, cudaStream_t st) {
    const int threads = 128;
    pso_move_kernel<<<(pc.P + threads - 1) / threads, threads, 0, st>>>(pc, sw, it);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused inversion iteration.  it = 0: evaluate the initial swarm.  it >= 1:
// move (Eq. 8) with the global best of iteration it-1, then evaluate.
// Personal-best positions and the global-best key are double-buffered by
// iteration parity so that no launch reads what it writes.
// ---------------------------------------------------------------------------
template <int M, int FORCE>
__global__ void __launch_bounds__(128, 1)
invert_iter_kernel(const KConst<float> K, const PsoConst pc, SwarmPtrs sw,
                   const float* __restrict__ U, float* __restrict__ history, int it) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tab = reinterpret_cast<float*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int rd = it & 1, wr = (it + 1) & 1;
    const float* pb_rd = sw.pb[rd];
    float* pb_wr = sw.pb[wr];
    unsigned long long key = ~0ull;
    if (it > 0 && p == 0 && history != nullptr)
        history[it - 1] = __uint_as_float((uint32_t)(*sw.gkey[rd] >> 32));
    if (p < pc.P) {
        float x[AFM_MAXD], v[AFM_MAXD];
        for (int d = 0; d < pc.D; ++d) {
            x[d] = sw.x[(size_t)d * pc.P + p];
            v[d] = sw.v[(size_t)d * pc.P + p];
        }
        if (it > 0) {
            const int g = min((int)(*sw.gkey[rd] & 0x7fffffffu), pc.P - 1);
            float pb[AFM_MAXD], gb[AFM_MAXD];
            for (int d = 0; d < pc.D; ++d) {
                pb[d] = pb_rd[(size_t)d * pc.P + p];
                gb[d] = pb_rd[(size_t)d * pc.P + g];
            }
            pso_move_dev(pc, x, v, pb, gb, p, it);
            for (int d = 0; d < pc.D; ++d) {
                sw.x[(size_t)d * pc.P + p] = x[d];
                sw.v[(size_t)d * pc.P + p] = v[d];
            }
        }
        Coef<float> c = make_coef<float, float>(K, x);
        float s = integrate<float, M, FORCE>(K, c, tab, U, nullptr, 0, p, K.n_steps);
        s = sanitize_misfit(s, sw.flags);
        float best = sw.pbS[p];
        const bool improved = s < best || it == 0;
        if (s < best) best = s;
        sw.pbS[p] = best;
        for (int d = 0; d < pc.D; ++d)
            pb_wr[(size_t)d * pc.P + p] = improved ? x[d] : pb_rd[(size_t)d * pc.P + p];
        key = best_key(best, p);
    }
    warp_min_atomic(key, sw.gkey[wr]);
}

cudaError_t launch_invert_iter(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                               const float* U, float* history, int it, cudaStream_t st,
                               int lanes) {
    // small swarms of rate-free force laws: several lanes per particle
    // (kern_modes.cu: modes split; kern_pair.cu: RK4 stage forces split).
    // Automatic choice, by measurement on the 3-mode DMT swarm of 1024
    // particles (per launch: one lane 4.59 ms, stages 4.53, modes over 4
    // lanes 4.41, over 2 lanes 4.30, over 3 lanes 3.66): one mode per lane
    // for 3 modes, modes over 2 lanes for 2, else stages.
    const bool m2 = modes_supported(K.m, K.force, pc.P, 2);
    const bool m4 = modes_supported(K.m, K.force, pc.P, 4);
    const bool m3 = modes_supported(K.m, K.force, pc.P, 3);
    const bool st2 = pair_supported(K.m, K.force, pc.P);
    const bool ok = lanes == AFM_LANES_ONE || (lanes == AFM_LANES_STAGES && st2) ||
                    (lanes == AFM_LANES_MODES2 && m2) || (lanes == AFM_LANES_MODES4 && m4) ||
                    (lanes == AFM_LANES_MODES3 && m3);
    if (!ok)
        lanes = (K.m == 3 && m3) ? AFM_LANES_MODES3
                : m2             ? AFM_LANES_MODES2
                : st2            ? AFM_LANES_STAGES
                                 : AFM_LANES_ONE;
    if (lanes == AFM_LANES_MODES2) return launch_invert_modes(K, pc, sw, U, history, it, 2, st);
    if (lanes == AFM_LANES_MODES4) return launch_invert_modes(K, pc, sw, U, history, it, 4, st);
    if (lanes == AFM_LANES_MODES3) return launch_invert_modes(K, pc, sw, U, history, it, 3, st);
    if (lanes == AFM_LANES_STAGES) return launch_invert_pair(K, pc, sw, U, history, it, st);
    const int threads = pc.P <= 152 * 32 * 4 ? 32 : 128;
    const int blocks = (pc.P + threads - 1) / threads;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value, FORCE = decltype(Fc)::value;
        invert_iter_kernel<M, FORCE><<<blocks, threads, smem, st>>>(K, pc, sw, U, history, it);
        return cudaGetLastError();
    });
}

// ---------------------------------------------------------------------------
// Final: FP64 re-evaluation of the winner and the result record.
// ---------------------------------------------------------------------------
template <int M, int FORCE>
__global__ void invert_final_kernel(const KConst<double> K, const PsoConst pc, SwarmPtrs sw,
                                    const float* __restrict__ U, float* __restrict__ history,
                                    afm_result* __restrict__ res) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* tab = reinterpret_cast<double*>(smem_raw);
    __shared__ double red[256];
    build_drive_table(K, tab);
    const int fin = (pc.iters + 1) & 1;
    const unsigned long long key = *sw.gkey[fin];
    const int g = min((int)(key & 0x7fffffffu), pc.P - 1);
    // sum of U^2 for J_rel
    double acc = 0.0;
    for (int n = threadIdx.x; n < K.n_steps; n += blockDim.x) acc += (double)U[n] * (double)U[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const float S32 = __uint_as_float((uint32_t)(key >> 32));
    if (history != nullptr) history[pc.iters] = S32;
    double xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < pc.D ? (double)sw.pb[fin][(size_t)d * pc.P + g] : 0.0;
    Coef<double> c = make_coef<double, double>(K, xd);
    double S64 = integrate<double, M, FORCE, float>(K, c, tab, U, nullptr, 0, 0, K.n_steps);
    for (int d = 0; d < AFM_MAXD; ++d) res->x[d] = xd[d];
    double th[AFM_MAXD];
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = K.fixed[s];
    for (int d = 0; d < K.D; ++d) {
        double v = K.lo[d] + xd[d] * K.span[d];
        th[K.slot[d]] = K.logs[d] ? exp10(v) : v;
    }
    for (int s = 0; s < AFM_MAXD; ++s) res->theta[s] = th[s];
    res->S = (double)S32;
    res->S_f64 = S64;
    res->J_rel = red[0] > 0.0 ? sqrt(S64 / red[0]) : 0.0;
    res->iters = pc.iters;
    res->winner = g;
    res->nonfinite = sw.flags ? sw.flags[0] : 0;
    res->status = (isfinite(S64) && (sw.flags == nullptr || sw.flags[0] == 0)) ? AFM_OK : AFM_ERR_NONFINITE;
    res->defect = 0.0;
    res->segments = 0;
    res->reserved = 0;
    for (int k = 0; k < 3; ++k) res->drive[k] = 0.0;
}

cudaError_t launch_invert_final(const KConst<double>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, void* result, cudaStream_t st) {
    const size_t smem = sizeof(double) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value, FORCE = decltype(Fc)::value;
        auto kern = invert_final_kernel<M, FORCE>;
        if (smem > 40 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<1, 256, smem, st>>>(K, pc, sw, U, history, reinterpret_cast<afm_result*>(result));
        return cudaGetLastError();
    });
}

}  // namespace afm
