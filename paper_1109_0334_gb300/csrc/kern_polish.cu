// kern_polish.cu -- gradient polish of the swarm's best particles: projected
// steepest descent in the normalised parameter cube with the adjoint gradient
// (kern_adjoint.cu) and a backtracking (Armijo) line search whose candidate
// step lengths are all evaluated in one batched forward launch.  Also the
// top-K selection from a finished swarm and the FP64 re-evaluation of the
// polished winner.
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

}  // namespace

// Trial points x + alpha_j * (-g / max|g|), clamped to the cube; one thread
// per (candidate k, step j); output column k * J + j of Xc [D][K*J].
__global__ void polish_cand_kernel(int D, int K, int J, const float* __restrict__ x,
                                   const float* __restrict__ G, double alpha0, double shrink,
                                   float* __restrict__ Xc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K * J) return;
    const int k = t / J, j = t % J;
    float gmax = 0.f;
    for (int d = 0; d < D; ++d) gmax = fmaxf(gmax, fabsf(G[(size_t)d * K + k]));
    const float alpha = (float)(alpha0 * pow(shrink, (double)j));
    for (int d = 0; d < D; ++d) {
        const float xd = x[(size_t)d * K + k];
        const float step = gmax > 0.f ? -alpha * (G[(size_t)d * K + k] / gmax) : 0.f;
        float xn = xd + step;
        xn = xn < 0.f ? 0.f : (xn > 1.f ? 1.f : xn);
        Xc[(size_t)d * K * J + t] = xn;
    }
}

// Largest step meeting S(x_j) <= S(x) + sigma g.(x_j - x) (with a strict
// descent direction); one thread per candidate.
__global__ void polish_select_kernel(int D, int K, int J, float sigma, float* __restrict__ x,
                                     const float* __restrict__ G, float* __restrict__ S,
                                     const float* __restrict__ Xc, const float* __restrict__ Sc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float S0 = S[k];
    for (int j = 0; j < J; ++j) {
        const int t = k * J + j;
        float lin = 0.f;
        for (int d = 0; d < D; ++d)
            lin = fmaf(G[(size_t)d * K + k], Xc[(size_t)d * K * J + t] - x[(size_t)d * K + k], lin);
        const float Sj = Sc[t];
        if (lin < 0.f && Sj <= fmaf(sigma, lin, S0)) {
            for (int d = 0; d < D; ++d) x[(size_t)d * K + k] = Xc[(size_t)d * K * J + t];
            S[k] = Sj;
            return;
        }
    }
}

// The K particles of lowest personal-best misfit (lowest index on ties), by a
// bitonic sort of (misfit bits, index) keys in one block.
__global__ void __launch_bounds__(1024) topk_kernel(const float* __restrict__ pbS,
                                                    const float* __restrict__ pb, int P, int D,
                                                    int K, int len, float* __restrict__ xk,
                                                    int* __restrict__ idx) {
    extern __shared__ unsigned long long key[];
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        if (i < P) {
            float s = pbS[i];
            s = (s < INFINITY) ? (s > 0.f ? s : 0.f) : INFINITY;
            key[i] = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)i;
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
    for (int t = threadIdx.x; t < K * D; t += blockDim.x) {
        const int k = t % K, d = t / K;
        const int p = (int)(key[k] & 0xffffffffu);
        xk[(size_t)d * K + k] = pb[(size_t)d * P + p];
        if (d == 0) idx[k] = p;
    }
}

template <int M, int FORCE>
__global__ void polish_final_kernel(const KConst<double> K, int Kn, int iters,
                                    const float* __restrict__ x, const float* __restrict__ S,
                                    const int* __restrict__ idx, const float* __restrict__ U,
                                    const int* __restrict__ flags, afm_result* __restrict__ res) {
    extern __shared__ __align__(16) double tabd[];
    __shared__ double red[256];
    build_drive_table(K, tabd);
    double acc = 0.0;
    for (int n = threadIdx.x; n < K.n_steps; n += blockDim.x) acc += (double)U[n] * (double)U[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    int kb = 0;
    for (int k = 1; k < Kn; ++k)
        if (S[k] < S[kb]) kb = k;
    double xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < K.D ? (double)x[(size_t)d * Kn + kb] : 0.0;
    Coef<double> c = make_coef<double, double>(K, xd);
    const double S64 = integrate<double, M, FORCE, float>(K, c, tabd, U, nullptr, 0, 0, K.n_steps);
    double th[AFM_MAXD];
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = K.fixed[s];
    for (int d = 0; d < K.D; ++d) {
        double v = K.lo[d] + xd[d] * K.span[d];
        th[K.slot[d]] = K.logs[d] ? exp10(v) : v;
    }
    for (int d = 0; d < AFM_MAXD; ++d) {
        res->x[d] = xd[d];
        res->theta[d] = th[d];
    }
    res->S = (double)S[kb];
    res->S_f64 = S64;
    res->J_rel = red[0] > 0.0 ? sqrt(S64 / red[0]) : 0.0;
    res->iters = iters;
    res->winner = idx != nullptr ? idx[kb] : kb;
    res->nonfinite = flags ? flags[0] : 0;
    res->status = (isfinite(S64) && res->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
    res->defect = 0.0;
    res->segments = 0;
    res->reserved = 0;
    for (int k = 0; k < 3; ++k) res->drive[k] = 0.0;
}

cudaError_t launch_polish_cand(int D, int K, int J, const float* x, const float* G, double alpha0,
                               double shrink, float* Xc, cudaStream_t st) {
    const int n = K * J, threads = 128;
    polish_cand_kernel<<<(n + threads - 1) / threads, threads, 0, st>>>(D, K, J, x, G, alpha0, shrink, Xc);
    return cudaGetLastError();
}

cudaError_t launch_polish_select(int D, int K, int J, float sigma, float* x, const float* G,
                                 float* S, const float* Xc, const float* Sc, cudaStream_t st) {
    const int threads = 32;
    polish_select_kernel<<<(K + threads - 1) / threads, threads, 0, st>>>(D, K, J, sigma, x, G, S, Xc, Sc);
    return cudaGetLastError();
}

cudaError_t launch_topk(const float* pbS, const float* pb, int P, int D, int K, float* xk, int* idx,
                        cudaStream_t st) {
    int len = 1;
    while (len < P) len <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)len;
    cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(unsigned long long) * 8192));
    if (e != cudaSuccess) return e;
    topk_kernel<<<1, 1024, smem, st>>>(pbS, pb, P, D, K, len, xk, idx);
    return cudaGetLastError();
}

cudaError_t launch_polish_final(const KConst<double>& K, int Kn, int iters, const float* x,
                                const float* S, const int* idx, const float* U, const int* flags,
                                void* result, cudaStream_t st) {
    const size_t smem = sizeof(double) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        auto kern = polish_final_kernel<decltype(Mc)::value, decltype(Fc)::value>;
        if (smem > 40 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<1, 256, smem, st>>>(K, Kn, iters, x, S, idx, U, flags,
                                   reinterpret_cast<afm_result*>(result));
        return cudaGetLastError();
    });
}

}  // namespace afm
