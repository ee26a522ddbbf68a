// kern_bpolish.cu -- gradient polish of many pixel inversions at once: the
// per-pixel top-K choice from the batched swarms, a forward + misfit kernel
// over candidates of different pixels (each against its own record), and the
// per-pixel choice of the polished winner.  The descent step itself uses the
// polish kernels of kern_polish.cu and the adjoint of kern_adjoint.cu in its
// ragged-record form, so that every candidate follows exactly the arithmetic
// of the single-inversion polish.
//
// Candidate layout: the pixels in queue order (slot s = position in the
// longest-record-first order), Kc candidates per slot, column s * Kc + k of
// [D][n_pix * Kc] arrays; a warp thus holds candidates of records of similar
// length.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_f32x2.cuh"
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

// One block per slot: the Kc personal bests of lowest misfit (lowest particle
// index on ties, the rule of topk_kernel) by a bitonic sort of (misfit bits,
// index) keys.  pb_all: per slot [D][P] positions then [P] misfits.
__global__ void __launch_bounds__(256) topk_pix_kernel(const float* __restrict__ pb_all, int P,
                                                       int D, int Kc, int len, int Nt,
                                                       float* __restrict__ xk,
                                                       float* __restrict__ Sk,
                                                       int* __restrict__ ik) {
    extern __shared__ unsigned long long key[];
    const int slot = blockIdx.x;
    const float* pb = pb_all + (size_t)slot * (D + 1) * P;
    const float* pbS = pb + (size_t)D * P;
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
                    const unsigned long long a = key[i], b = key[l];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < Kc * D; t += blockDim.x) {
        const int k = t % Kc, d = t / Kc;
        const int p = (int)(key[k] & 0xffffffffu);
        const int col = slot * Kc + k;
        xk[(size_t)d * Nt + col] = pb[(size_t)d * P + p];
        if (d == 0) {
            ik[col] = p;
            Sk[col] = pbS[p];
        }
    }
}

// Forward solve + misfit (the arithmetic of fwd_kernel) of candidates that
// belong to different pixels: candidate p of slot p / per_slot against that
// pixel's record.
// PP: each candidate's pixel has its own constants and drive table (pix),
// read from global memory.
template <bool PP>
__device__ __forceinline__ const KConst<float>& ragged_k(const KConst<float>& K0, const PixConst& pc,
                                                         int pix) {
    if constexpr (PP)
        return pc.kf[pix];
    else
        return K0;
}

template <int M, int FORCE, bool PP>
__global__ void fwd_ragged_kernel(const KConst<float> K0, const float* __restrict__ x, int Ptot,
                                  const float* __restrict__ U_cat, const int64_t* __restrict__ off,
                                  const int* __restrict__ order, int per_slot,
                                  float* __restrict__ S, const PixConst pixc) {
    extern __shared__ __align__(16) float tabs[];
    if constexpr (!PP) {
        build_drive_table(K0, tabs);
        __syncthreads();
    }
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Ptot) return;
    const int slot = p / per_slot;
    const int pix = order != nullptr ? order[slot] : slot;
    const KConst<float>& K = ragged_k<PP>(K0, pixc, pix);
    const float* tab = PP ? pixc.tab32 + (size_t)pix * pixc.ld : tabs;
    const int64_t o = off[pix];
    const int n = (int)(off[pix + 1] - o);
    float xd[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) xd[d] = x[(size_t)d * Ptot + p];
    const Coef<float> c = make_coef<float, float>(K, xd);
    float s = integrate<float, M, FORCE>(K, c, tab, U_cat + o, nullptr, Ptot, p, n);
    if (!(s < INFINITY)) s = INFINITY;
    S[p] = s;
}

// The same with candidates 2t and 2t + 1 on thread t in paired FP32
// instructions (afm_f32x2.cuh; bit-identical): with an even number of
// candidates per slot both belong to the same pixel and record.
template <int M, int FORCE, bool PP>
__global__ void fwd_ragged_x2_kernel(const KConst<float> K0, const float* __restrict__ x,
                                     int Ptot, const float* __restrict__ U_cat,
                                     const int64_t* __restrict__ off,
                                     const int* __restrict__ order, int per_slot,
                                     float* __restrict__ S, const PixConst pixc) {
    extern __shared__ __align__(16) float tabs[];
    if constexpr (!PP) {
        build_drive_table(K0, tabs);
        __syncthreads();
    }
    const int p = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (p >= Ptot) return;
    const int slot = p / per_slot;
    const int pix = order != nullptr ? order[slot] : slot;
    const KConst<float>& K = ragged_k<PP>(K0, pixc, pix);
    const float* tab = PP ? pixc.tab32 + (size_t)pix * pixc.ld : tabs;
    const int64_t o = off[pix];
    const int n = (int)(off[pix + 1] - o);
    float xa[AFM_MAXD], xb[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) {
        xa[d] = x[(size_t)d * Ptot + p];
        xb[d] = x[(size_t)d * Ptot + p + 1];
    }
    const Coef<float> ca = make_coef<float, float>(K, xa);
    const Coef<float> cb = make_coef<float, float>(K, xb);
    const float2 s = integrate_x2<M, FORCE>(K, ca, cb, tab, U_cat + o, nullptr, Ptot, p, true, n);
    S[p] = s.x < INFINITY ? s.x : INFINITY;
    S[p + 1] = s.y < INFINITY ? s.y : INFINITY;
}

// Per slot: the polished candidate of lowest misfit (first on ties) becomes
// the pixel's winner (x, FP32 S, swarm index); the FP64 re-evaluation of
// kern_reeval_batch.cu follows.
__global__ void pick_pix_kernel(int n_pix, int D, int Kc, const float* __restrict__ xk,
                                const float* __restrict__ Sk, const int* __restrict__ ik,
                                const int* __restrict__ order, int iters,
                                afm_result* __restrict__ res) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_pix) return;
    const int pix = order != nullptr ? order[slot] : slot;
    const size_t Nt = (size_t)n_pix * Kc;
    int kb = 0;
    for (int k = 1; k < Kc; ++k)
        if (Sk[(size_t)slot * Kc + k] < Sk[(size_t)slot * Kc + kb]) kb = k;
    const size_t c = (size_t)slot * Kc + kb;
    afm_result* r = res + pix;
    for (int d = 0; d < AFM_MAXD; ++d) r->x[d] = d < D ? (double)xk[(size_t)d * Nt + c] : 0.0;
    if (Sk[c] < INFINITY) r->S = (double)Sk[c];
    r->winner = ik[c];
    r->iters = iters;
}

cudaError_t launch_topk_pix(const float* pb_all, int n_pix, int P, int D, int Kc, float* xk,
                            float* Sk, int* ik, cudaStream_t st) {
    int len = 1;
    while (len < P) len <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)len;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(topk_pix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    topk_pix_kernel<<<n_pix, 256, smem, st>>>(pb_all, P, D, Kc, len, n_pix * Kc, xk, Sk, ik);
    return cudaGetLastError();
}

cudaError_t launch_forward_ragged(const KConst<float>& K, const float* x, int Ptot, const float* U_cat,
                                  const int64_t* off, const int* order, int per_slot, float* S,
                                  cudaStream_t st, const PixConst& pix) {
    const int threads = Ptot <= 152 * 32 * 4 ? 32 : 128;
    const int blocks = (Ptot + threads - 1) / threads;
    const bool pp = pix.kf != nullptr;
    const size_t smem = pp ? 0 : sizeof(float) * (size_t)(K.spc2 + 1);
    auto by_pp = [&](auto&& f) -> cudaError_t {
        return pp ? f(std::true_type{}) : f(std::false_type{});
    };
    // pairs of candidates for large DMT batches (the same rule as
    // afm_forward_batch's paired kernel)
    if (K.force == F_DMT && (K.m == 1 || K.m == 3) && per_slot % 2 == 0 && Ptot >= 65536) {
        const int pairs = Ptot / 2;
        auto go = [&](auto Mc) -> cudaError_t {
            return by_pp([&](auto Pc) -> cudaError_t {
                auto kern = fwd_ragged_x2_kernel<decltype(Mc)::value, F_DMT, decltype(Pc)::value>;
                if (smem > 48 * 1024) {
                    cudaError_t e = cudaFuncSetAttribute(
                        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e != cudaSuccess) return e;
                }
                kern<<<(pairs + 127) / 128, 128, smem, st>>>(K, x, Ptot, U_cat, off, order,
                                                              per_slot, S, pix);
                return cudaGetLastError();
            });
        };
        if (K.m == 1) return go(std::integral_constant<int, 1>{});
        return go(std::integral_constant<int, 3>{});
    }
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        return by_pp([&](auto Pc) -> cudaError_t {
            auto kern = fwd_ragged_kernel<decltype(Mc)::value, decltype(Fc)::value,
                                          decltype(Pc)::value>;
            if (smem > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(
                    kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            kern<<<blocks, threads, smem, st>>>(K, x, Ptot, U_cat, off, order, per_slot, S, pix);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_pick_pix(int n_pix, int D, int Kc, const float* xk, const float* Sk,
                            const int* ik, const int* order, int iters, afm_result* res,
                            cudaStream_t st) {
    const int threads = 128;
    pick_pix_kernel<<<(n_pix + threads - 1) / threads, threads, 0, st>>>(n_pix, D, Kc, xk, Sk, ik,
                                                                         order, iters, res);
    return cudaGetLastError();
}

}  // namespace afm
