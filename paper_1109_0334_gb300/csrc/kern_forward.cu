// kern_forward.cu -- batched forward problem (FP of Sec. 2.2): one thread per
// candidate parameter set integrates the modal cantilever (Eq. 2) with RK4
// (Sec. 3.2), fused with the misfit of Eq. 5; the standalone misfit; and the
// synthetic-record generator (Sec. 4.1's finer-step data).
#include <cooperative_groups.h>

#include <type_traits>

#include "afm_device.cuh"
#include "afm_f32x2.cuh"
#include "afm_launch.h"

namespace cg = cooperative_groups;

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

// ---------------------------------------------------------------------------
// Forward + misfit, one thread per particle.
// ---------------------------------------------------------------------------
template <typename T, int M, int FORCE>
__global__ void fwd_kernel(const KConst<T> K, const T* __restrict__ x, int P,
                           T* __restrict__ defl, const T* __restrict__ U, T* __restrict__ S,
                           int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    T xd[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) xd[d] = x[(size_t)d * P + p];
    Coef<T> c = make_coef<T, T>(K, xd);
    T s = integrate<T, M, FORCE>(K, c, tab, U, defl, P, p, K.n_steps);
    if (S != nullptr) {
        if (!(s < (T)INFINITY)) {
            s = (T)INFINITY;
            if (flags != nullptr) atomicAdd(flags, 1);
        }
        S[p] = s;
    }
}

// The same with two particles per thread in paired FP32 instructions
// (afm_f32x2.cuh; bit-identical to fwd_kernel): thread t takes particles 2t
// and 2t + 1.  (Capping it at 72 registers, seven blocks per SM, so that
// 262 144 particles run in one wave, measured 2 % slower.)
template <int M, int FORCE>
__global__ void fwd_x2_kernel(const KConst<float> K, const float* __restrict__ x, int P,
                              float* __restrict__ defl, const float* __restrict__ U,
                              float* __restrict__ S, int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tab = reinterpret_cast<float*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int p0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (p0 >= P) return;
    const bool has1 = p0 + 1 < P;
    const int p1 = has1 ? p0 + 1 : p0;
    float xa[AFM_MAXD], xb[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) {
        xa[d] = x[(size_t)d * P + p0];
        xb[d] = x[(size_t)d * P + p1];
    }
    const Coef<float> ca = make_coef<float, float>(K, xa);
    const Coef<float> cb = make_coef<float, float>(K, xb);
    const float2 s = integrate_x2<M, FORCE>(K, ca, cb, tab, U, defl, P, p0, has1, K.n_steps);
    if (S != nullptr) {
        const float sv[2] = {s.x, s.y};
        for (int k = 0; k < (has1 ? 2 : 1); ++k) {
            float sk = sv[k];
            if (!(sk < INFINITY)) {
                sk = INFINITY;
                if (flags != nullptr) atomicAdd(flags, 1);
            }
            S[p0 + k] = sk;
        }
    }
}

// Paired particles where the law and mode count allow it and the batch is
// large enough to fill the GPU with half as many threads.
static bool forward_x2_ok(int m, int force, int P, int lanes) {
    return lanes != AFM_LANES_ONE && force == F_DMT && (m == 1 || m == 3) && P >= 65536;
}

static cudaError_t launch_forward_x2(const KConst<float>& K, const float* x, int P, float* defl,
                                     const float* U, float* S, int* flags, cudaStream_t st) {
    const int threads = 128;
    const int pairs = (P + 1) / 2;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    auto go = [&](auto Mc) -> cudaError_t {
        auto kern = fwd_x2_kernel<decltype(Mc)::value, F_DMT>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<(pairs + threads - 1) / threads, threads, smem, st>>>(K, x, P, defl, U, S, flags);
        return cudaGetLastError();
    };
    if (K.m == 1) return go(std::integral_constant<int, 1>{});
    return go(std::integral_constant<int, 3>{});
}

template <typename T>
static cudaError_t launch_forward(const KConst<T>& K, const T* x, int P, T* defl, const T* U,
                                  T* S, int* flags, cudaStream_t st) {
    const int threads = P <= 152 * 32 * 4 ? 32 : 128;
    const int blocks = (P + threads - 1) / threads;
    const size_t smem = sizeof(T) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value, FORCE = decltype(Fc)::value;
        auto kern = fwd_kernel<T, M, FORCE>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, threads, smem, st>>>(K, x, P, defl, U, S, flags);
        return cudaGetLastError();
    });
}

cudaError_t launch_forward_f32(const KConst<float>& K, const float* x, int P, float* defl,
                               const float* U, float* S, int* flags, cudaStream_t st, int lanes) {
    if (forward_x2_ok(K.m, K.force, P, lanes))
        return launch_forward_x2(K, x, P, defl, U, S, flags, st);
    return launch_forward<float>(K, x, P, defl, U, S, flags, st);
}
cudaError_t launch_forward_f64(const KConst<double>& K, const double* x, int P, double* defl,
                               const double* U, double* S, int* flags, cudaStream_t st) {
    return launch_forward<double>(K, x, P, defl, U, S, flags, st);
}

// ---------------------------------------------------------------------------
// Standalone misfit (Eq. 5) of a time-major deflection array.  HBM-bound:
// a cluster of MIS_CL blocks splits the time axis of a 32-particle column;
// within a block, MIS_NL warps stride over time with coalesced 128-byte row
// reads; partial compensated sums meet in distributed shared memory and are
// combined by rank 0 in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int MIS_CL = 8;   // blocks per cluster along time
constexpr int MIS_NL = 8;   // warps per block along time

__global__ void __cluster_dims__(1, MIS_CL, 1) __launch_bounds__(32 * MIS_NL)
    misfit_kernel(const float* __restrict__ defl, const float* __restrict__ U, int N, int P,
                  float* __restrict__ S) {
    __shared__ float partS[MIS_NL][32], partC[MIS_NL][32];
    __shared__ float blkS[32], blkC[32];
    cg::cluster_group cluster = cg::this_cluster();
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    const int rank = (int)cluster.block_rank();   // 0..MIS_CL-1 along y
    const int stride = MIS_CL * MIS_NL;
    float s = 0.f, c = 0.f;
    if (p < P) {
        int n = rank * MIS_NL + wy;
#pragma unroll 4
        for (; n < N; n += stride) {
            float r = __ldg(U + n) - __ldg(defl + (size_t)n * P + p);
            float y = fmaf(r, r, -c);
            float t = __fadd_rn(s, y);
            c = __fsub_rn(__fsub_rn(t, s), y);
            s = t;
        }
    }
    partS[wy][lane] = s;
    partC[wy][lane] = c;
    __syncthreads();
    if (wy == 0) {
        float bs = 0.f, bc = 0.f;
        for (int k = 0; k < MIS_NL; ++k) {
            float y = __fsub_rn(partS[k][lane], __fadd_rn(bc, partC[k][lane]));
            float t = __fadd_rn(bs, y);
            bc = __fsub_rn(__fsub_rn(t, bs), y);
            bs = t;
        }
        blkS[lane] = bs;
        blkC[lane] = bc;
    }
    cluster.sync();
    if (rank == 0 && wy == 0) {
        float ts = 0.f, tc = 0.f;
        for (int r = 0; r < MIS_CL; ++r) {
            float* rs = cluster.map_shared_rank(blkS, r);
            float* rc = cluster.map_shared_rank(blkC, r);
            float y = __fsub_rn(rs[lane], __fadd_rn(tc, rc[lane]));
            float t = __fadd_rn(ts, y);
            tc = __fsub_rn(__fsub_rn(t, ts), y);
            ts = t;
        }
        if (p < P) S[p] = ts;
    }
    cluster.sync();   // keep every block's shared memory alive until rank 0 has read it
}

cudaError_t launch_misfit(const float* defl, const float* U, int N, int P, float* S, int num_sms,
                          cudaStream_t st) {
    (void)num_sms;
    dim3 grid((P + 31) / 32, MIS_CL, 1);
    misfit_kernel<<<grid, 32 * MIS_NL, 0, st>>>(defl, U, N, P, S);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Synthetic records: one thread per pixel integrates its truth at the fine
// step of K (FP32, compensated), samples every `sub` steps and adds
// Box-Muller noise from Philox tag 4.
// ---------------------------------------------------------------------------
template <int M, int FORCE>
__global__ void synth_kernel(const KConst<float> K, const double* __restrict__ xt, int n_pix,
                             const int64_t* __restrict__ off, int sub, float sigma,
                             uint64_t seed, uint32_t pixel0, float* __restrict__ Ucat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tab = reinterpret_cast<float*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pix) return;
    double xd[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) xd[d] = xt[(size_t)d * n_pix + i];
    Coef<float> c = make_coef<float, double>(K, xd);
    const int64_t o = off[i];
    const int n = (int)(off[i + 1] - o);
    float q[M], v[M], cq[M], cv[M];
    init_state<float, M>(K, q, v, cq, cv);
    int j = 0;
    const uint32_t pix = pixel0 + (uint32_t)i;
    for (int s = 0; s < n; ++s) {
        for (int f = 0; f < sub; ++f) {
            float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
            j += 2;
            if (j >= K.spc2) j = 0;
            rk4_step<float, M, FORCE>(K, c, q, v, cq, cv, g0, gh, g1);
        }
        float u = tip_sum<float, M>(q);
        if (sigma > 0.f) {
            uint4 w = philox_draw(seed, (uint32_t)(s >> 1), 0u, pix, 4u, 0u);
            float u1 = ((float)(w.x >> 8) + 1.0f) * (1.0f / 16777216.0f);
            float u2 = (float)(w.y >> 8) * (1.0f / 16777216.0f);
            float rr = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            u += sigma * rr * ((s & 1) ? sn : cs);
        }
        Ucat[o + s] = u;
    }
}

cudaError_t launch_synth(const KConst<float>& K, const double* x_truth, int n_pix,
                         const int64_t* off, int sub, float sigma_nm, uint64_t seed,
                         uint32_t pixel0, float* U_cat, cudaStream_t st) {
    const int threads = 32;
    const int blocks = (n_pix + threads - 1) / threads;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value, FORCE = decltype(Fc)::value;
        synth_kernel<M, FORCE><<<blocks, threads, smem, st>>>(K, x_truth, n_pix, off, sub,
                                                               sigma_nm, seed, pixel0, U_cat);
        return cudaGetLastError();
    });
}

}  // namespace afm
