// kern_batch.cuh -- kernels of the batched pixel inversion (see
// kern_batch.cu); instantiated per force law in kern_batch_*.cu so that the
// translation units compile in parallel.
#pragma once
#include "../../include/afminv.h"
#include "afm_device.cuh"
#include "afm_f32x2.cuh"
#include "afm_launch.h"

namespace afm {

namespace batch_detail {

__device__ __forceinline__ unsigned long long bkey(float S, int p) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)p;
}

__device__ __forceinline__ unsigned long long warp_min(unsigned long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xffffffffu, k, o);
        k = other < k ? other : k;
    }
    return k;
}

// The problem constants of the pixel being inverted: the launch's (shared by
// every pixel), or the per-pixel copy staged in shared memory.
template <bool PP>
__device__ __forceinline__ const KConst<float>& pick_k(const KConst<float>& K,
                                                       const KConst<float>* sK) {
    if constexpr (PP)
        return *sK;
    else
        return K;
}

}  // namespace batch_detail

// 32-bit words of dynamic shared memory before the drive table (per-pixel
// constants), a multiple of 4 so that the arrays after it stay 16-byte aligned
template <bool PP>
__host__ __device__ constexpr int batch_kc_words() {
    return PP ? (int)((sizeof(KConst<float>) + 15) / 16 * 4) : 0;
}

// ---------------------------------------------------------------------------
// Persistent swarm kernel.
// ---------------------------------------------------------------------------
// PP: the pixels' problems differ (a.pix): each pixel's constants and drive
// table are staged into shared memory when a block takes the pixel.
template <int M, int FORCE, int KP, bool PP>
__global__ void __launch_bounds__(KP == 1 ? 1024 : 512) batch_kernel(const KConst<float> K, const PsoConst pc,
                                                     const BatchArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int P = pc.P, D = pc.D;
    KConst<float>* sK = reinterpret_cast<KConst<float>*>(sm);
    float* tab = sm + batch_kc_words<PP>();
    float* sx = tab + ((K.spc2 + 1 + 3) & ~3);
    float* sv = sx + D * P;
    float* spb = sv + D * P;
    __shared__ unsigned long long wkey[32];
    __shared__ unsigned long long s_gkey;
    __shared__ int s_slot, s_bad;
    __shared__ float s_blo[AFM_MAXD], s_bspan[AFM_MAXD];   // optional per-slot box
    const bool boxed = a.box_lo != nullptr;
    if (!PP) build_drive_table(K, tab);
    const KConst<float>& KK = batch_detail::pick_k<PP>(K, sK);
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = T >> 5;
    for (;;) {
        __syncthreads();   // table built / previous pixel finished with shared memory
        if (tid == 0) {
            const int sl = atomicAdd(a.queue, 1);
            s_slot = sl;
            s_bad = 0;
            if (boxed && sl < a.n_pix)
                for (int d = 0; d < D; ++d) {
                    const float lo = a.box_lo[(size_t)sl * D + d];
                    s_blo[d] = lo;
                    s_bspan[d] = a.box_hi[(size_t)sl * D + d] - lo;
                }
        }
        __syncthreads();
        const int slot = s_slot;
        if (slot >= a.n_pix) return;
        const int pix = a.order != nullptr ? a.order[slot] : slot;
        if constexpr (PP) {   // this pixel's constants and drive table
            const unsigned* src = reinterpret_cast<const unsigned*>(a.pix.kf + pix);
            unsigned* dst = reinterpret_cast<unsigned*>(sK);
            for (int w = tid; w < (int)(sizeof(KConst<float>) / 4); w += blockDim.x) dst[w] = src[w];
            const float* t32 = a.pix.tab32 + (size_t)pix * a.pix.ld;
            for (int j = tid; j <= K.spc2; j += blockDim.x) tab[j] = t32[j];
            __syncthreads();
        }
        const int64_t o = a.off[pix];
        const int n = (int)(a.off[pix + 1] - o);
        const float* U = a.U + o;
        PsoConst pcp = pc;
        pcp.pixel = a.pixel0 + (uint32_t)pix;

        // initial swarm (tags 0 and 1), as pso_init_kernel
        float pbS[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int p = tid + k * T;
            pbS[k] = INFINITY;
            if (p >= P) continue;
            for (int b = 0; b * 4 < D; ++b) {
                uint4 w0 = philox_draw(pcp.seed, (uint32_t)p, 0u, pcp.pixel, 0u, (uint32_t)b);
                uint4 w1 = philox_draw(pcp.seed, (uint32_t)p, 0u, pcp.pixel, 1u, (uint32_t)b);
                for (int q = 0; q < 4 && b * 4 + q < D; ++q) {
                    const int d = b * 4 + q;
                    const float u0 = unif24(word_of(w0, q)), u1 = unif24(word_of(w1, q));
                    sx[d * P + p] = u0;
                    sv[d * P + p] = (u1 - u0) * 0.5f;
                }
            }
            if (a.seeds != nullptr && p < a.n_seed) {   // seed particle, at rest, box-local
                for (int d = 0; d < D; ++d) {
                    const float s = a.seeds[((size_t)slot * a.n_seed + p) * D + d];
                    const float lo = boxed ? s_blo[d] : 0.f, sp = boxed ? s_bspan[d] : 1.f;
                    float t = sp > 0.f ? (s - lo) / sp : 0.f;
                    t = t > 0.f ? (t < 1.f ? t : 1.f) : 0.f;
                    sx[d * P + p] = t;
                    sv[d * P + p] = 0.f;
                }
            }
        }
        for (int it = 0; it <= pc.iters; ++it) {
            if (it > 0) {
                const int g = min((int)(s_gkey & 0x7fffffffu), P - 1);
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int p = tid + k * T;
                    if (p >= P) continue;
                    float x[AFM_MAXD], v[AFM_MAXD], pb[AFM_MAXD], gb[AFM_MAXD];
                    for (int d = 0; d < D; ++d) {
                        x[d] = sx[d * P + p];
                        v[d] = sv[d * P + p];
                        pb[d] = spb[d * P + p];
                        gb[d] = spb[d * P + g];
                    }
                    pso_move_dev(pcp, x, v, pb, gb, p, it);
                    for (int d = 0; d < D; ++d) {
                        sx[d * P + p] = x[d];
                        sv[d * P + p] = v[d];
                    }
                }
                __syncthreads();   // every read of the global best precedes any personal-best write
            }
            Coef<float> c[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int p = min(tid + k * T, P - 1);
                float x[AFM_MAXD];
                for (int d = 0; d < D; ++d)
                    x[d] = boxed ? fmaf(sx[d * P + p], s_bspan[d], s_blo[d]) : sx[d * P + p];
                c[k] = make_coef<float, float>(KK, x);
            }
            float S[KP];
            // pairs of particles per paired FP32 instruction where the law allows
            if constexpr (KP % 2 == 0 && M <= 4 && x2::Supported<FORCE>::value)
                integrate_multi_x2<M, FORCE, KP>(KK, c, tab, U, n, S);
            else
                integrate_multi<M, FORCE, KP>(KK, c, tab, U, n, S);
            unsigned long long key = ~0ull;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int p = tid + k * T;
                if (p >= P) continue;
                float s = S[k];
                if (!(s < INFINITY)) {
                    atomicAdd(&s_bad, 1);
                    s = INFINITY;
                } else if (!(s > 0.f)) {
                    s = 0.f;
                }
                if (s < pbS[k] || it == 0) {
                    pbS[k] = fminf(s, pbS[k]);
                    for (int d = 0; d < D; ++d) spb[d * P + p] = sx[d * P + p];
                }
                const unsigned long long kk = batch_detail::bkey(pbS[k], p);
                key = kk < key ? kk : key;
            }
            key = batch_detail::warp_min(key);
            if (lane == 0) wkey[warp] = key;
            __syncthreads();
            if (warp == 0) {
                unsigned long long k2 = lane < nwarps ? wkey[lane] : ~0ull;
                k2 = batch_detail::warp_min(k2);
                if (lane == 0) s_gkey = k2;
            }
            __syncthreads();
        }
        if (a.pb_out != nullptr) {   // final personal bests of this slot (own particles only)
            float* dst = a.pb_out + (size_t)slot * (D + 1) * P;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int p = tid + k * T;
                if (p >= P) continue;
                dst[(size_t)D * P + p] = pbS[k];
                for (int d = 0; d < D; ++d)
                    dst[(size_t)d * P + p] =
                        boxed ? fmaf(spb[d * P + p], s_bspan[d], s_blo[d]) : spb[d * P + p];
            }
        }
        if (tid == 0) {
            const int g = min((int)(s_gkey & 0x7fffffffu), P - 1);
            afm_result* r = a.res + pix;
            for (int d = 0; d < AFM_MAXD; ++d)
                r->x[d] = d >= D ? 0.0
                                 : (double)(boxed ? fmaf(spb[d * P + g], s_bspan[d], s_blo[d])
                                                  : spb[d * P + g]);
            r->S = (double)__uint_as_float((uint32_t)(s_gkey >> 32));
            r->iters = pc.iters;
            r->winner = g;
            r->nonfinite = s_bad;
        }
    }
}

// Launch helpers of one force law (explicitly instantiated per force).
template <int FORCE>
struct BatchOps {
    template <typename F>
    static cudaError_t by_mk(int m, int kp, F&& f) {
        if (m == 1) {
            switch (kp) {
                case 1: return f(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{});
                case 2: return f(std::integral_constant<int, 1>{}, std::integral_constant<int, 2>{});
                case 4: return f(std::integral_constant<int, 1>{}, std::integral_constant<int, 4>{});
            }
        } else if (m == 3) {
            switch (kp) {
                case 1: return f(std::integral_constant<int, 3>{}, std::integral_constant<int, 1>{});
                case 2: return f(std::integral_constant<int, 3>{}, std::integral_constant<int, 2>{});
                case 4: return f(std::integral_constant<int, 3>{}, std::integral_constant<int, 4>{});
            }
        } else if (kp == 1) {
            return f(std::integral_constant<int, AFM_MAXM>{}, std::integral_constant<int, 1>{});
        }
        return cudaErrorInvalidValue;
    }

    template <typename F>
    static cudaError_t by_mkp(int m, int kp, bool pp, F&& f) {
        return by_mk(m, kp, [&](auto Mc, auto Kc) -> cudaError_t {
            if (pp) return f(Mc, Kc, std::true_type{});
            return f(Mc, Kc, std::false_type{});
        });
    }

    static cudaError_t occupancy(int m, int kp, int P, int D, int spc2, bool pp, int* blocks) {
        const int threads = batch_threads(P, kp);
        const size_t smem = batch_smem(P, D, spc2, pp);
        return by_mkp(m, kp, pp, [&](auto Mc, auto Kc, auto Pc) -> cudaError_t {
            auto kern = batch_kernel<decltype(Mc)::value, FORCE, decltype(Kc)::value,
                                     decltype(Pc)::value>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, threads, smem);
        });
    }

    static cudaError_t launch(const KConst<float>& K, const PsoConst& pc, const BatchArgs& a, int kp,
                              int grid, cudaStream_t st) {
        const int threads = batch_threads(pc.P, kp);
        const bool pp = a.pix.kf != nullptr;
        const size_t smem = batch_smem(pc.P, pc.D, K.spc2, pp);
        return by_mkp(K.m, kp, pp, [&](auto Mc, auto Kc, auto Pc) -> cudaError_t {
            auto kern = batch_kernel<decltype(Mc)::value, FORCE, decltype(Kc)::value,
                                     decltype(Pc)::value>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            kern<<<grid, threads, smem, st>>>(K, pc, a);
            return cudaGetLastError();
        });
    }
};


// Per-force entry points, each defined (as an explicit specialization) in
// its kern_batch_<law>.cu so that kern_batch.cu dispatches without
// instantiating any kernel.
template <int FORCE>
cudaError_t batch_occupancy_of(int m, int kp, int P, int D, int spc2, bool pp, int* blocks);
template <int FORCE>
cudaError_t batch_launch_of(const KConst<float>& K, const PsoConst& pc, const BatchArgs& a, int kp,
                            int grid, cudaStream_t st);

}  // namespace afm
