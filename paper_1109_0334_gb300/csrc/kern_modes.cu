// kern_modes.cu -- the fused inversion iteration with the modes of a particle
// spread over L lanes (L = 2, 3 or 4), for swarms too small to fill the GPU.
//
// A swarm of ~1000 particles fills a few dozen warps, so the RK4 recurrence
// of each particle (Sec. 3.2) runs at the latency of its dependency chain,
// and every instruction a warp issues lies on that chain.  Here each lane
// keeps the state of S = ceil(M / L) modes ("slots"; slots past the last
// mode hold zero), so a warp issues the per-mode arithmetic of S modes
// instead of M.  The tip deflection of each RK4 stage is the sum over modes:
// each lane sums its slots and a butterfly of shuffles adds the lanes'
// partial sums, so every lane holds the same deflection and evaluates the
// tip force itself.  For a rate-free law the forces of stages 1 and 2 depend
// on the step's start state only, and those of stages 3 and 4 only on the
// forces of stages 1 and 2: two shuffle exchanges per step.
//
// The partial sums meet in the order of the one-lane kernels ((q0 + q1) + q2
// for three modes, q0 + q1 for two) and every per-mode operation is
// rk4_step's, so the result is bit-identical to the one-lane kernels (the
// batched-pixel kernel, afm_forward_batch).
//
// Records at several points along the beam (the n_dp points of Sec. 3.2)
// need every mode at every step: with one mode per lane (L = M) the lanes
// read the group's M modes with M shuffles, which also give the stage-1 tip
// deflection in the one-lane order, and each lane forms the point
// deflections and the misfit as integrate_points does.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

namespace {

// Per-lane constants of the lane's S mode slots (zero for empty slots).
template <int S>
struct Slots {
    float w2[S], w2lo[S], wq[S], gam[S], tip[S];
    int cmb[S];
};

// The force-independent part of accel's acceleration for one slot, then the
// force through one final rounding, as accel's non-contractible add_rn.
// With empty slots in the group the force enters as fma(tip, F, a) (tip 1
// rounds as a + F, tip 0 keeps the slot at rest); with none, tip is known to
// be 1 and the compiler would fold that fma into an add it may then fuse
// with a force law ending in a product, so add_rn is written out.
template <int S, bool ALL_REAL>
__device__ __forceinline__ float slot_accel(const Slots<S>& C, int k, float q, float v, float g,
                                            float F) {
    float ai = fmaf(-C.wq[k], v, C.gam[k] * g);
    ai = fmaf(-C.w2lo[k], q, ai);
    ai = fmaf(-C.w2[k], q, ai);
    return ALL_REAL ? add_rn(ai, F) : fmaf(C.tip[k], F, ai);
}

// Lanes of a warp per group: 32 / L groups per warp (L = 3: ten groups,
// lanes 30 and 31 idle).
template <int L>
__device__ __forceinline__ int group_base(int wl) {
    return L == 3 ? (wl / 3) * 3 : wl & ~(L - 1);
}

// Sum of the partial sums of the L lanes of a group in the one-lane order:
// xor butterfly for L = 2, 4 ((p0 + p1) + (p2 + p3), p3 = 0 for three
// modes); for L = 3 the three partials read at once, ((p0 + p1) + p2).
template <int L>
__device__ __forceinline__ float group_sum(float p) {
    if (L == 3) {
        const int g = group_base<3>(threadIdx.x & 31);
        const float a = __shfl_sync(0xffffffffu, p, g);
        const float b = __shfl_sync(0xffffffffu, p, g + 1);
        const float c = __shfl_sync(0xffffffffu, p, g + 2);
        return (a + b) + c;
    }
    p = p + __shfl_xor_sync(0xffffffffu, p, 1);
    if (L == 4) p = p + __shfl_xor_sync(0xffffffffu, p, 2);
    return p;
}

template <int S>
__device__ __forceinline__ float slot_sum(const float* x) {
    float s = x[0];
#pragma unroll
    for (int k = 1; k < S; ++k) s += x[k];
    return s;
}

// Forward solve + compensated misfit of one particle on a lane group; with
// NP > 0 the misfit runs over the NP point deflections of each step (NP = 0:
// the tip).  The record values of step s are loaded during step s - 1.
template <int M, int FORCE, int L, int NP>
__device__ __forceinline__ float integrate_modes(const KConst<float>& K, const Coef<float>& c,
                                                 const float* tab, const float* __restrict__ U,
                                                 int n, int lane) {
    constexpr int S = (M + L - 1) / L;
    constexpr bool R = S * L == M;   // every slot holds a mode
    constexpr bool POINTS = NP > 0;
    static_assert(!POINTS || L == M, "point records need one mode per lane");
    Slots<S> C;
    float q[S], v[S], cq[S], cv[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int i = lane * S + k;
        const bool real = i < M;
        C.w2[k] = real ? K.w2[i] : 0.f;
        C.w2lo[k] = (real && i == 0) ? K.w2lo[0] : 0.f;
        C.wq[k] = real ? K.wq[i] : 0.f;
        C.gam[k] = real ? K.gam[i] : 0.f;
        C.tip[k] = real ? 1.f : 0.f;
        C.cmb[k] = (real && K.cmask[i] != 0.f) ? -1 : 0;
        q[k] = real ? K.q0[i] : 0.f;
        v[k] = real ? K.v0[i] : 0.f;
        cq[k] = 0.f;
        cv[k] = 0.f;
    }
    float S2 = 0.f, cS = 0.f;
    int j = 0;
    const int spc2 = K.spc2;
    float Un = 0.f;
    float Up[POINTS ? NP : 1];
#pragma unroll
    for (int k = 0; k < (POINTS ? NP : 1); ++k) Up[k] = (POINTS && n > 0) ? U[k] : 0.f;
    for (int s = 0; s <= n; ++s) {
        float qs2[S];
#pragma unroll
        for (int k = 0; k < S; ++k) qs2[k] = fmaf(3.f, v[k], q[k]);
        // first exchange: the step's start deflection (the previous step's output)
        // and the stage-2 deflection
        float u1, u2;
        if constexpr (POINTS) {
            const int g = group_base<L>(threadIdx.x & 31);
            float qa[M];
#pragma unroll
            for (int i = 0; i < M; ++i) qa[i] = __shfl_sync(0xffffffffu, q[0], g + i);
            u1 = qa[0];
#pragma unroll
            for (int i = 1; i < M; ++i) u1 += qa[i];
            u2 = group_sum<L>(slot_sum<S>(qs2));
            if (s > 0) {
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    float uk = K.phi[k][0] * qa[0];
#pragma unroll
                    for (int i = 1; i < M; ++i) uk = fmaf(K.phi[k][i], qa[i], uk);
                    const float r = Up[k] - uk;
                    const float y = fmaf(r, r, -cS);
                    const float t = add_rn(S2, y);
                    cS = sub_rn(sub_rn(t, S2), y);
                    S2 = t;
                }
                if (s < n) {
#pragma unroll
                    for (int k = 0; k < NP; ++k) Up[k] = U[(size_t)s * NP + k];
                }
            }
        } else {
            u1 = group_sum<L>(slot_sum<S>(q));
            u2 = group_sum<L>(slot_sum<S>(qs2));
            if (s > 0) {
                const float r = Un - u1;
                const float y = fmaf(r, r, -cS);
                const float t = add_rn(S2, y);
                cS = sub_rn(sub_rn(t, S2), y);
                S2 = t;
            }
        }
        if (s == n) break;
        if constexpr (!POINTS) Un = U[s];
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        const float F1 = tip_force<FORCE, float>(c, K.Zc + u1, 0.f);
        const float F2 = tip_force<FORCE, float>(c, K.Zc + u2, 0.f);
        float a1[S], a2[S], vs2[S], qs3[S], vs3[S], qs4[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            a1[k] = slot_accel<S, R>(C, k, q[k], v[k], g0, F1);
            vs2[k] = fmaf(3.f, a1[k], v[k]);
            a2[k] = slot_accel<S, R>(C, k, qs2[k], vs2[k], gh, F2);
            qs3[k] = fmaf(3.f, vs2[k], q[k]);
            vs3[k] = fmaf(3.f, a2[k], v[k]);
            qs4[k] = fmaf(6.f, vs3[k], q[k]);
        }
        // second exchange: stage-3 and stage-4 deflections
        const float u3 = group_sum<L>(slot_sum<S>(qs3));
        const float u4 = group_sum<L>(slot_sum<S>(qs4));
        const float F3 = tip_force<FORCE, float>(c, K.Zc + u3, 0.f);
        const float F4 = tip_force<FORCE, float>(c, K.Zc + u4, 0.f);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const float a3 = slot_accel<S, R>(C, k, qs3[k], vs3[k], gh, F3);
            const float vs4 = fmaf(6.f, a3, v[k]);
            const float a4 = slot_accel<S, R>(C, k, qs4[k], vs4, g1, F4);
            float Kq = v[k];
            Kq = fmaf(2.f, vs2[k], Kq);
            Kq = fmaf(2.f, vs3[k], Kq);
            Kq = Kq + vs4;
            float Kv = a1[k];
            Kv = fmaf(2.f, a2[k], Kv);
            Kv = fmaf(2.f, a3, Kv);
            Kv = Kv + a4;
            kahan_add(q[k], cq[k], Kq);
            kahan_add(v[k], cv[k], Kv);
            // modes taking plain sums hold their compensation at zero
            // (state_add; C.cmb: the run-time mask KConst::cmask as bits)
            if (lane * S + k > 0) {
                cq[k] = __int_as_float(__float_as_int(cq[k]) & C.cmb[k]);
                cv[k] = __int_as_float(__float_as_int(cv[k]) & C.cmb[k]);
            }
        }
    }
    return S2;
}

__device__ __forceinline__ unsigned long long modes_key(float S, int p) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)p;
}

}  // namespace

// invert_iter_kernel of kern_invert.cu with L lanes per particle: all lanes
// of a group move the particle identically (lane 0 stores), integrate it
// together, and lane 0 updates the bests.  Groups beyond P run the last
// particle without storing (the shuffles need every lane).
template <int M, int FORCE, int L, int NP>
__global__ void __launch_bounds__(32, 1)
invert_modes_kernel(const KConst<float> K, const PsoConst pc, SwarmPtrs sw,
                    const float* __restrict__ U, float* __restrict__ history, int it) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tab = reinterpret_cast<float*>(smem_raw);
    build_drive_table(K, tab);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int G = 32 / L;                       // particle groups per warp
    const int wl = threadIdx.x & 31;
    const bool in_group = wl < G * L;               // L = 3: lanes 30, 31 idle
    const int p0 = in_group ? (t >> 5) * G + wl / L : pc.P;
    const int lane = in_group ? wl - group_base<L>(wl) : 0;
    const bool owner = p0 < pc.P && lane == 0;
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
        // every lane of the group has read x and v before lane 0 overwrites them
        __syncwarp();
        if (owner)
            for (int d = 0; d < pc.D; ++d) {
                sw.x[(size_t)d * pc.P + p] = x[d];
                sw.v[(size_t)d * pc.P + p] = v[d];
            }
    }
    const Coef<float> c = make_coef<float, float>(K, x);
    float s = integrate_modes<M, FORCE, L, NP>(K, c, tab, U, K.n_steps, lane);
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
        key = modes_key(best, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(sw.gkey[wr], key);
}

bool modes_supported(int m, int force, int P, int lanes) {
    return (lanes == 2 || lanes == 3 || lanes == 4) && (m == 2 || m == 3) &&
           (force == F_LINEAR || force == F_DMT || force == F_HOOKE) &&
           P <= 152 * 4 * (32 / lanes);
}

cudaError_t launch_invert_modes(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, int it, int lanes,
                                cudaStream_t st) {
    if (!modes_supported(K.m, K.force, pc.P, lanes)) return cudaErrorInvalidValue;
    const int threads = 32, per_warp = 32 / lanes;
    const int blocks = (pc.P + per_warp - 1) / per_warp;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    auto go = [&](auto Mc, auto Fc, auto Lc) -> cudaError_t {
        invert_modes_kernel<decltype(Mc)::value, decltype(Fc)::value, decltype(Lc)::value, 0>
            <<<blocks, threads, smem, st>>>(K, pc, sw, U, history, it);
        return cudaGetLastError();
    };
    auto byL = [&](auto Mc, auto Fc) -> cudaError_t {
        if (lanes == 2) return go(Mc, Fc, std::integral_constant<int, 2>{});
        if (lanes == 3) return go(Mc, Fc, std::integral_constant<int, 3>{});
        return go(Mc, Fc, std::integral_constant<int, 4>{});
    };
    auto byF = [&](auto Mc) -> cudaError_t {
        switch (K.force) {
            case F_LINEAR: return byL(Mc, std::integral_constant<int, F_LINEAR>{});
            case F_DMT: return byL(Mc, std::integral_constant<int, F_DMT>{});
            case F_HOOKE: return byL(Mc, std::integral_constant<int, F_HOOKE>{});
        }
        return cudaErrorInvalidValue;
    };
    if (K.m == 2) return byF(std::integral_constant<int, 2>{});
    return byF(std::integral_constant<int, 3>{});
}

bool points_modes_supported(int m, int force, int P, int np) {
    return np >= 1 && np <= 4 && modes_supported(m, force, P, m);
}

// The deflection-points iteration with one mode per lane (L = M).
cudaError_t launch_invert_points_modes(const KConst<float>& K, const PsoConst& pc,
                                       const SwarmPtrs& sw, const float* U, float* history, int it,
                                       cudaStream_t st) {
    if (!points_modes_supported(K.m, K.force, pc.P, K.np)) return cudaErrorInvalidValue;
    const int per_warp = 32 / K.m;
    const int blocks = (pc.P + per_warp - 1) / per_warp;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    auto go = [&](auto Mc, auto Fc, auto Nc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value;
        invert_modes_kernel<M, decltype(Fc)::value, M, decltype(Nc)::value>
            <<<blocks, 32, smem, st>>>(K, pc, sw, U, history, it);
        return cudaGetLastError();
    };
    auto byN = [&](auto Mc, auto Fc) -> cudaError_t {
        switch (K.np) {
            case 1: return go(Mc, Fc, std::integral_constant<int, 1>{});
            case 2: return go(Mc, Fc, std::integral_constant<int, 2>{});
            case 3: return go(Mc, Fc, std::integral_constant<int, 3>{});
        }
        return go(Mc, Fc, std::integral_constant<int, 4>{});
    };
    auto byF = [&](auto Mc) -> cudaError_t {
        switch (K.force) {
            case F_LINEAR: return byN(Mc, std::integral_constant<int, F_LINEAR>{});
            case F_DMT: return byN(Mc, std::integral_constant<int, F_DMT>{});
            case F_HOOKE: return byN(Mc, std::integral_constant<int, F_HOOKE>{});
        }
        return cudaErrorInvalidValue;
    };
    if (K.m == 2) return byF(std::integral_constant<int, 2>{});
    return byF(std::integral_constant<int, 3>{});
}

}  // namespace afm
