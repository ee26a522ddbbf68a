// kern_points.cu -- deflections at several points along the cantilever (the
// paper's n_dp measurement points, Sec. 3.2): the record holds, per step, the
// deflection u_k = sum_i phi_i(xi_k) eta_i at each point x = xi_k L
// (tip-normalised mode shapes), and the misfit of Eq. 5 runs over all of
// them.  The tip force still acts through the tip deflection.  Time stepping,
// compensated sums and swarm arithmetic are those of the tip-only kernels.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

namespace {

template <typename F>
cudaError_t dispatch_mf(int m, int force, F&& f) {
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

__device__ __forceinline__ unsigned long long points_key(float S, int p) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)p;
}

}  // namespace

template <typename T, int M, int FORCE>
__global__ void fwd_points_kernel(const KConst<T> K, const T* __restrict__ x, int P,
                                  T* __restrict__ defl, const T* __restrict__ U,
                                  T* __restrict__ S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    T xd[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) xd[d] = x[(size_t)d * P + p];
    const Coef<T> c = make_coef<T, T>(K, xd);
    T s = integrate_points<T, M, FORCE>(K, c, tab, U, defl, P, p, K.n_steps);
    if (S != nullptr) S[p] = (s < (T)INFINITY) ? s : (T)INFINITY;
}

// invert_iter_kernel of kern_invert.cu with the misfit over the points.
template <int M, int FORCE>
__global__ void __launch_bounds__(128, 1)
invert_points_kernel(const KConst<float> K, const PsoConst pc, SwarmPtrs sw,
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
        const Coef<float> c = make_coef<float, float>(K, x);
        float s = integrate_points<float, M, FORCE>(K, c, tab, U, nullptr, 0, p, K.n_steps);
        if (!(s < INFINITY)) {
            if (sw.flags) atomicAdd(sw.flags, 1);
            s = INFINITY;
        } else if (!(s > 0.f)) {
            s = 0.f;
        }
        float best = sw.pbS[p];
        const bool improved = s < best || it == 0;
        if (s < best) best = s;
        sw.pbS[p] = best;
        for (int d = 0; d < pc.D; ++d)
            pb_wr[(size_t)d * pc.P + p] = improved ? x[d] : pb_rd[(size_t)d * pc.P + p];
        key = points_key(best, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(sw.gkey[wr], key);
}

// FP64 re-evaluation of the winner (one thread) and the result record.
template <int M, int FORCE>
__global__ void points_final_kernel(const KConst<double> K, const PsoConst pc, SwarmPtrs sw,
                                    const float* __restrict__ U, float* __restrict__ history,
                                    afm_result* __restrict__ res) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* tab = reinterpret_cast<double*>(smem_raw);
    __shared__ double red[256];
    build_drive_table(K, tab);
    const int nv = K.n_steps * K.np;
    double acc = 0.0;
    for (int n = threadIdx.x; n < nv; n += blockDim.x) acc += (double)U[n] * (double)U[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const int fin = (pc.iters + 1) & 1;
    const unsigned long long key = *sw.gkey[fin];
    const int g = min((int)(key & 0x7fffffffu), pc.P - 1);
    const float S32 = __uint_as_float((uint32_t)(key >> 32));
    if (history != nullptr) history[pc.iters] = S32;
    double xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < pc.D ? (double)sw.pb[fin][(size_t)d * pc.P + g] : 0.0;
    const Coef<double> c = make_coef<double, double>(K, xd);
    const double S64 = integrate_points<double, M, FORCE, float>(K, c, tab, U, nullptr, 0, 0, K.n_steps);
    double th[AFM_MAXD];
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = K.fixed[s];
    for (int d = 0; d < K.D; ++d) {
        const double v = K.lo[d] + xd[d] * K.span[d];
        th[K.slot[d]] = K.logs[d] ? exp10(v) : v;
    }
    for (int d = 0; d < AFM_MAXD; ++d) {
        res->x[d] = xd[d];
        res->theta[d] = th[d];
    }
    for (int k = 0; k < 3; ++k) res->drive[k] = 0.0;
    res->S = (double)S32;
    res->S_f64 = S64;
    res->J_rel = red[0] > 0.0 ? sqrt(S64 / red[0]) : 0.0;
    res->iters = pc.iters;
    res->winner = g;
    res->nonfinite = sw.flags ? sw.flags[0] : 0;
    res->status = (isfinite(S64) && res->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
    res->defect = 0.0;
    res->segments = 0;
    res->reserved = 0;
}

template <typename T>
static cudaError_t forward_points(const KConst<T>& K, const T* x, int P, T* defl, const T* U, T* S,
                                  cudaStream_t st) {
    const int threads = P <= 152 * 32 * 4 ? 32 : 128;
    const size_t smem = sizeof(T) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        auto kern = fwd_points_kernel<T, decltype(Mc)::value, decltype(Fc)::value>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<(P + threads - 1) / threads, threads, smem, st>>>(K, x, P, defl, U, S);
        return cudaGetLastError();
    });
}

cudaError_t launch_forward_points_f32(const KConst<float>& K, const float* x, int P, float* defl,
                                      const float* U, float* S, cudaStream_t st) {
    return forward_points<float>(K, x, P, defl, U, S, st);
}

cudaError_t launch_forward_points_f64(const KConst<double>& K, const double* x, int P, double* defl,
                                      const double* U, double* S, cudaStream_t st) {
    return forward_points<double>(K, x, P, defl, U, S, st);
}

cudaError_t launch_invert_points(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                 const float* U, float* history, int it, cudaStream_t st,
                                 int lanes) {
    // one mode per lane (kern_modes.cu) unless one lane is asked for; per
    // launch on the three-point, 3-mode DMT swarm of 512 particles over
    // 10240 steps: one lane 2.30 ms, one mode per lane 2.22 ms
    if (lanes != AFM_LANES_ONE && points_modes_supported(K.m, K.force, pc.P, K.np))
        return launch_invert_points_modes(K, pc, sw, U, history, it, st);
    const int threads = pc.P <= 152 * 32 * 4 ? 32 : 128;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        invert_points_kernel<decltype(Mc)::value, decltype(Fc)::value>
            <<<(pc.P + threads - 1) / threads, threads, smem, st>>>(K, pc, sw, U, history, it);
        return cudaGetLastError();
    });
}

cudaError_t launch_points_final(const KConst<double>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, void* result, cudaStream_t st) {
    const size_t smem = sizeof(double) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        auto kern = points_final_kernel<decltype(Mc)::value, decltype(Fc)::value>;
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
