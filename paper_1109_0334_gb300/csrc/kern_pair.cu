// kern_pair.cu -- the fused inversion iteration with two lanes per particle,
// for swarms too small to fill the GPU (latency-bound: one RK4 step of every
// particle is a serial chain of four tip-force evaluations).
//
// In classic RK4 (Sec. 3.2) the tip force of stage 2 depends on the state
// only through q + (h/2) v, not on stage 1's acceleration, and stage 4's only
// through q + h (v + (h/2) a_2), not on stage 3's, when the force law has no
// rate term.  So the even lane of a pair evaluates the forces of stages 1 and
// 3 while the odd lane evaluates those of stages 2 and 4, and one shuffle
// after each pair of evaluations gives both lanes all four forces.  Every
// other quantity is computed by both lanes with the operations of rk4_step in
// the same order, so the two lanes stay bit-identical to each other and to
// the one-lane kernels (the batched-pixel kernel and afm_forward_batch).
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

namespace {

// Force-independent part of accel's mode-i acceleration (same operations).
template <int M>
__device__ __forceinline__ float lin_part(const KConst<float>& K, int i, const float* q,
                                          const float* v, float g) {
    float ai = fmaf(-K.wq[i], v[i], K.gam[i] * g);
    if (i == 0) ai = fmaf(-K.w2lo[0], q[0], ai);
    return fmaf(-K.w2[i], q[i], ai);
}

template <int M>
__device__ __forceinline__ float sum_modes(const float* q) {
    float u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u += q[i];
    return u;
}

// One RK4 step of a particle shared by the lane pair (odd: the pair's odd
// lane).  Rate-free force laws only.
template <int M, int FORCE>
__device__ __forceinline__ void rk4_step_pair(const KConst<float>& K, const Coef<float>& c,
                                              float* q, float* v, float* cq, float* cv, float g0,
                                              float gh, float g1, bool odd) {
    static_assert(!UsesRate<FORCE>::value, "the stage split needs a rate-free force law");
    static_assert(M <= 4, "tip factors are 1 for the specialised mode counts");
    float qs2[M], vs2[M], qs3[M], vs3[M], qs4[M], vs4[M], a1[M], a2[M], a3[M], a4[M], in[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        qs2[i] = fmaf(3.f, v[i], q[i]);
        in[i] = odd ? qs2[i] : q[i];
    }
    float Fo = tip_force<FORCE, float>(c, K.Zc + sum_modes<M>(in), 0.f);
    float Fx = __shfl_xor_sync(0xffffffffu, Fo, 1);
    const float F1 = odd ? Fx : Fo, F2 = odd ? Fo : Fx;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        a1[i] = add_rn(lin_part<M>(K, i, q, v, g0), F1);
        vs2[i] = fmaf(3.f, a1[i], v[i]);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        a2[i] = add_rn(lin_part<M>(K, i, qs2, vs2, gh), F2);
        qs3[i] = fmaf(3.f, vs2[i], q[i]);
        vs3[i] = fmaf(3.f, a2[i], v[i]);
        qs4[i] = fmaf(6.f, vs3[i], q[i]);
        in[i] = odd ? qs4[i] : qs3[i];
    }
    Fo = tip_force<FORCE, float>(c, K.Zc + sum_modes<M>(in), 0.f);
    Fx = __shfl_xor_sync(0xffffffffu, Fo, 1);
    const float F3 = odd ? Fx : Fo, F4 = odd ? Fo : Fx;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        a3[i] = add_rn(lin_part<M>(K, i, qs3, vs3, gh), F3);
        vs4[i] = fmaf(6.f, a3[i], v[i]);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        a4[i] = add_rn(lin_part<M>(K, i, qs4, vs4, g1), F4);
        float Kq = v[i];
        Kq = fmaf(2.f, vs2[i], Kq);
        Kq = fmaf(2.f, vs3[i], Kq);
        Kq = Kq + vs4[i];
        float Kv = a1[i];
        Kv = fmaf(2.f, a2[i], Kv);
        Kv = fmaf(2.f, a3[i], Kv);
        Kv = Kv + a4[i];
        state_add(i, q[i], cq[i], Kq);
        state_add(i, v[i], cv[i], Kv);
    }
}

// integrate() of afm_device.cuh (misfit only) on a lane pair.
template <int M, int FORCE>
__device__ __forceinline__ float integrate_pair(const KConst<float>& K, const Coef<float>& c,
                                                const float* tab, const float* __restrict__ U,
                                                int n, bool odd) {
    float q[M], v[M], cq[M], cv[M];
    init_state<float, M>(K, q, v, cq, cv);
    float S = 0.f, cS = 0.f;
    int j = 0;
    const int spc2 = K.spc2;
    float Un = n > 0 ? U[0] : 0.f;
    for (int s = 0; s < n; ++s) {
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        const float Unext = s + 1 < n ? U[s + 1] : 0.f;
        rk4_step_pair<M, FORCE>(K, c, q, v, cq, cv, g0, gh, g1, odd);
        const float u = tip_sum<float, M>(q);
        const float r = Un - u;
        const float y = fmaf(r, r, -cS);
        const float t = add_rn(S, y);
        cS = sub_rn(sub_rn(t, S), y);
        S = t;
        Un = Unext;
    }
    return S;
}

__device__ __forceinline__ unsigned long long pair_key(float S, int p) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)p;
}

}  // namespace

// invert_iter_kernel of kern_invert.cu with two lanes per particle: both
// lanes of a pair move the particle identically (the even lane stores), then
// integrate it together; the even lane updates the bests.  Pairs beyond P run
// the last particle without storing (the shuffles need every lane).
template <int M, int FORCE>
__global__ void __launch_bounds__(32, 1)
invert_pair_kernel(const KConst<float> K, const PsoConst pc, SwarmPtrs sw,
                   const float* __restrict__ U, float* __restrict__ history, int it) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tab = reinterpret_cast<float*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int p0 = t >> 1;
    const bool odd = (t & 1) != 0;
    const bool owner = p0 < pc.P && !odd;
    const int p = min(p0, pc.P - 1);
    const int rd = it & 1, wr = (it + 1) & 1;
    const float* pb_rd = sw.pb[rd];
    float* pb_wr = sw.pb[wr];
    if (it > 0 && t == 0 && history != nullptr)
        history[it - 1] = __uint_as_float((uint32_t)(*sw.gkey[rd] >> 32));
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
        // both lanes have read x and v before the even lane overwrites them
        __syncwarp();
        if (owner)
            for (int d = 0; d < pc.D; ++d) {
                sw.x[(size_t)d * pc.P + p] = x[d];
                sw.v[(size_t)d * pc.P + p] = v[d];
            }
    }
    const Coef<float> c = make_coef<float, float>(K, x);
    float s = integrate_pair<M, FORCE>(K, c, tab, U, K.n_steps, odd);
    unsigned long long key = ~0ull;
    if (owner) {
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
        key = pair_key(best, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(sw.gkey[wr], key);
}

bool pair_supported(int m, int force, int P) {
    return (m == 1 || m == 3) && (force == F_LINEAR || force == F_DMT || force == F_HOOKE) &&
           P <= 152 * 4 * 16;
}

cudaError_t launch_invert_pair(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                               const float* U, float* history, int it, cudaStream_t st) {
    if (!pair_supported(K.m, K.force, pc.P)) return cudaErrorInvalidValue;
    const int threads = 32;
    const int blocks = (2 * pc.P + threads - 1) / threads;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    auto go = [&](auto Mc, auto Fc) -> cudaError_t {
        invert_pair_kernel<decltype(Mc)::value, decltype(Fc)::value>
            <<<blocks, threads, smem, st>>>(K, pc, sw, U, history, it);
        return cudaGetLastError();
    };
    auto byF = [&](auto Mc) -> cudaError_t {
        switch (K.force) {
            case F_LINEAR: return go(Mc, std::integral_constant<int, F_LINEAR>{});
            case F_DMT: return go(Mc, std::integral_constant<int, F_DMT>{});
            case F_HOOKE: return go(Mc, std::integral_constant<int, F_HOOKE>{});
        }
        return cudaErrorInvalidValue;
    };
    if (K.m == 1) return byF(std::integral_constant<int, 1>{});
    return byF(std::integral_constant<int, 3>{});
}

}  // namespace afm
