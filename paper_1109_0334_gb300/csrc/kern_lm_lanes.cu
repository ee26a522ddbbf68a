// kern_lm_lanes.cu -- the sensitivity pass of kern_lm.cu with the parameter
// directions of a candidate spread over L lanes (one direction per lane),
// for candidate counts too small to fill the GPU (the polish of one
// inversion's best particles).  Every lane runs the primal RK4 solve
// (identical arithmetic, so S is the forward kernel's bit for bit) and the
// tangent of its own direction; each step the group gathers the tip
// tangents with shuffles and lane e accumulates row e of H = sum a a^T and
// b_e = sum a_e r.  Each direction's arithmetic and every accumulation are
// the one-lane kernel's operations in the same order, so H and b are
// bit-identical to sens_kernel's.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"
#include "afm_tangent.cuh"

namespace afm {

namespace {

constexpr int kLaneThreads = 32;
constexpr int kLaneFold = 32;   // as sens_kernel: FP32 blocks of 32 steps folded into FP64

int lanes_for(int D) { return D <= 2 ? 2 : D <= 4 ? 4 : 8; }

}  // namespace

template <int M, int FORCE, int L>
__global__ void __launch_bounds__(kLaneThreads) sens_lanes_kernel(
    const KConst<float> K, const float* __restrict__ x, int P, const float* __restrict__ U,
    const int64_t* __restrict__ off, const int* __restrict__ order, int per_slot,
    float* __restrict__ S_out, double* __restrict__ H_out, double* __restrict__ b_out) {
    extern __shared__ __align__(16) float tab[];
    build_drive_table(K, tab);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int p0 = t / L;
    const int e = t % L;                     // this lane's direction
    const bool store = p0 < P;
    const int p = min(p0, P - 1);            // groups past P repeat the last candidate
    const int D = K.D;
    int n = K.n_steps;
    if (off != nullptr) {
        const int slot = p / per_slot;
        const int pix = order != nullptr ? order[slot] : slot;
        U += off[pix];
        n = (int)(off[pix + 1] - off[pix]);
    }
    // the whole warp steps to its longest record (groups with shorter records
    // idle past their end), so that every shuffle has the full warp
    int n_warp = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_warp = max(n_warp, __shfl_xor_sync(0xffffffffu, n_warp, o));
    float xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < D ? x[(size_t)d * P + p] : 0.f;
    const Coef<float> c = make_coef<float, float>(K, xd);
    float Jc[4][1];
    {
        double Jd[4][AFM_MAXD];
        coef_jacobian<float>(K, xd, Jd);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float jk = 0.f;
            for (int d = 0; d < AFM_MAXD; ++d)
                if (d == e && d < D) jk = (float)Jd[k][d];
            Jc[k][0] = jk;
        }
    }
    float q[M], v[M], cq[M], cv[M], tq[1][M], tv[1][M];
    init_state<float, M>(K, q, v, cq, cv);
#pragma unroll
    for (int i = 0; i < M; ++i) tq[0][i] = tv[0][i] = 0.f;
    double aH[L], ab = 0.0;
    float hc[L], bc = 0.f;
#pragma unroll
    for (int f = 0; f < L; ++f) {
        aH[f] = 0.0;
        hc[f] = 0.f;
    }
    float S = 0.f, cS = 0.f;
    int j = 0, fold = 0;
    const int spc2 = K.spc2;
    for (int s = 0; s < n_warp; ++s) {
        const bool act = s < n;
        float au = 0.f, r = 0.f;
        if (act) {
            const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
            j += 2;
            if (j >= spc2) j = 0;
            rk4_step_tl<M, FORCE, 1>(K, c, Jc, q, v, cq, cv, tq, tv, g0, gh, g1);
            const float u = tip_sum<float, M>(q);
            r = U[s] - u;
            const float y = fmaf(r, r, -cS);
            const float t2 = add_rn(S, y);
            cS = sub_rn(sub_rn(t2, S), y);
            S = t2;
            au = tip_sum<float, M>(tq[0]);
        }
        float af[L];
#pragma unroll
        for (int f = 0; f < L; ++f) af[f] = __shfl_sync(0xffffffffu, au, f, L);
        if (!act) continue;
        bc = fmaf(au, r, bc);
#pragma unroll
        for (int f = 0; f < L; ++f) hc[f] = fmaf(au, af[f], hc[f]);
        if (++fold == kLaneFold || s + 1 == n) {
            fold = 0;
#pragma unroll
            for (int f = 0; f < L; ++f) {
                aH[f] += (double)hc[f];
                hc[f] = 0.f;
            }
            ab += (double)bc;
            bc = 0.f;
        }
    }
    if (!store) return;
    if (e == 0) S_out[p] = (S < INFINITY) ? S : INFINITY;
    if (e < D) {
        double* H = H_out + (size_t)p * D * D;
#pragma unroll
        for (int f = 0; f < L; ++f)
            if (f <= e) {
                H[e * D + f] = aH[f];
                H[f * D + e] = aH[f];
            }
        b_out[(size_t)p * D + e] = ab;
    }
}

// ---------------------------------------------------------------------------
// Three modes, rate-free laws: one lane per (direction e, mode k) pair, 3 D
// lanes per candidate.  Each direction group of three lanes runs the primal
// step as invert_modes_kernel's three-lane layout (one mode per lane, stage
// tip sums read by three shuffles and added in the one-lane order) and the
// tangent of its direction for its own mode; the tangent tip sums are read
// the same way.  Every operation is sens_kernel's, so S, H and b are
// bit-identical to it.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float sum3(float p, int base) {
    const float a0 = __shfl_sync(0xffffffffu, p, base);
    const float a1 = __shfl_sync(0xffffffffu, p, base + 1);
    const float a2 = __shfl_sync(0xffffffffu, p, base + 2);
    return (a0 + a1) + a2;
}

// One tangent stage of one (direction, mode) lane: tl_stage's arithmetic.
__device__ __forceinline__ float tl_lane(const StagePartials& P, const float (&Jc)[4], float w2,
                                         float wq, float tq, float tv, int dbase) {
    const float su = sum3(tq, dbase);
    float dF = P.Fd * su;
#pragma unroll
    for (int c = 0; c < 4; ++c) dF = fmaf(P.Fc[c], Jc[c], dF);
    const float base = fmaf(-wq, tv, -w2 * tq);
    return base + dF;
}

// accel's acceleration of one mode with the force added as add_rn.
__device__ __forceinline__ float mode_accel(float w2, float w2lo, float wq, float gam, float q,
                                            float v, float g, float F) {
    float ai = fmaf(-wq, v, gam * g);
    ai = fmaf(-w2lo, q, ai);
    ai = fmaf(-w2, q, ai);
    return add_rn(ai, F);
}

}  // namespace

template <int FORCE, int D>
__global__ void __launch_bounds__(kLaneThreads) sens_modes_kernel(
    const KConst<float> K, const float* __restrict__ x, int P, const float* __restrict__ U,
    const int64_t* __restrict__ off, const int* __restrict__ order, int per_slot,
    float* __restrict__ S_out, double* __restrict__ H_out, double* __restrict__ b_out) {
    static_assert(!UsesRate<FORCE>::value, "rate-free force laws only");
    constexpr int L = 3 * D, G = 32 / L;
    extern __shared__ __align__(16) float tab[];
    build_drive_table(K, tab);
    __syncthreads();
    const int wl = threadIdx.x & 31;
    const bool in_group = wl < G * L;
    const int p0 = in_group ? blockIdx.x * G + wl / L : P;
    const int li = in_group ? wl % L : 0;
    const int e = li / 3, k = li % 3;                  // direction, mode
    const int gbase = in_group ? (wl / L) * L : 0;
    const int dbase = gbase + 3 * e;
    const bool store = p0 < P;
    const int p = min(p0, P - 1);
    int n = K.n_steps;
    if (off != nullptr) {
        const int slot = p / per_slot;
        const int pix = order != nullptr ? order[slot] : slot;
        U += off[pix];
        n = (int)(off[pix + 1] - off[pix]);
    }
    int n_warp = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_warp = max(n_warp, __shfl_xor_sync(0xffffffffu, n_warp, o));
    float xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < D ? x[(size_t)d * P + p] : 0.f;
    const Coef<float> c = make_coef<float, float>(K, xd);
    float Jc[4];
    {
        double Jd[4][AFM_MAXD];
        coef_jacobian<float>(K, xd, Jd);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            float jk = 0.f;
            for (int d = 0; d < D; ++d)
                if (d == e) jk = (float)Jd[cc][d];
            Jc[cc] = jk;
        }
    }
    const float w2 = K.w2[k], w2lo = k == 0 ? K.w2lo[0] : 0.f, wq = K.wq[k], gam = K.gam[k];
    float q = K.q0[k], v = K.v0[k], cq = 0.f, cv = 0.f, tq = 0.f, tv = 0.f;
    const int cmb = K.cmask[k] != 0.f ? -1 : 0;
    double aH[D], ab = 0.0;
    float hc[D], bc = 0.f;
#pragma unroll
    for (int f = 0; f < D; ++f) {
        aH[f] = 0.0;
        hc[f] = 0.f;
    }
    float S = 0.f, cS = 0.f, Un = 0.f;
    int j = 0, fold = 0;
    const int spc2 = K.spc2;
    for (int s = 0; s <= n_warp; ++s) {
        const float qs2 = fmaf(3.f, v, q);
        const float u1 = sum3(q, dbase);
        const float u2 = sum3(qs2, dbase);
        const float au = sum3(tq, dbase);   // tangent tip deflection after step s - 1
        float af[D];
#pragma unroll
        for (int f = 0; f < D; ++f) af[f] = __shfl_sync(0xffffffffu, au, gbase + 3 * f);
        if (s > 0 && s <= n) {   // the misfit and normal equations of step s - 1
            const float r = Un - u1;
            const float y = fmaf(r, r, -cS);
            const float t2 = add_rn(S, y);
            cS = sub_rn(sub_rn(t2, S), y);
            S = t2;
            bc = fmaf(au, r, bc);
#pragma unroll
            for (int f = 0; f < D; ++f) hc[f] = fmaf(au, af[f], hc[f]);
            if (++fold == kLaneFold || s == n) {
                fold = 0;
#pragma unroll
                for (int f = 0; f < D; ++f) {
                    aH[f] += (double)hc[f];
                    hc[f] = 0.f;
                }
                ab += (double)bc;
                bc = 0.f;
            }
        }
        if (s == n_warp) break;
        Un = s < n ? U[s] : 0.f;
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        // primal step of this lane's mode, with the stage force partials
        StagePartials P1, P2, P3, P4;
        force_partials<FORCE>(c, K.Zc + u1, 0.f, P1.Fd, P1.Fr, P1.Fc);
        force_partials<FORCE>(c, K.Zc + u2, 0.f, P2.Fd, P2.Fr, P2.Fc);
        const float F1 = tip_force<FORCE, float>(c, K.Zc + u1, 0.f);
        const float F2 = tip_force<FORCE, float>(c, K.Zc + u2, 0.f);
        const float a1 = mode_accel(w2, w2lo, wq, gam, q, v, g0, F1);
        const float vs2 = fmaf(3.f, a1, v);
        const float a2 = mode_accel(w2, w2lo, wq, gam, qs2, vs2, gh, F2);
        const float qs3 = fmaf(3.f, vs2, q);
        const float vs3 = fmaf(3.f, a2, v);
        const float qs4 = fmaf(6.f, vs3, q);
        const float u3 = sum3(qs3, dbase);
        const float u4 = sum3(qs4, dbase);
        force_partials<FORCE>(c, K.Zc + u3, 0.f, P3.Fd, P3.Fr, P3.Fc);
        force_partials<FORCE>(c, K.Zc + u4, 0.f, P4.Fd, P4.Fr, P4.Fc);
        const float F3 = tip_force<FORCE, float>(c, K.Zc + u3, 0.f);
        const float F4 = tip_force<FORCE, float>(c, K.Zc + u4, 0.f);
        const float a3 = mode_accel(w2, w2lo, wq, gam, qs3, vs3, gh, F3);
        const float vs4 = fmaf(6.f, a3, v);
        const float a4 = mode_accel(w2, w2lo, wq, gam, qs4, vs4, g1, F4);
        float Kq = v;
        Kq = fmaf(2.f, vs2, Kq);
        Kq = fmaf(2.f, vs3, Kq);
        Kq = Kq + vs4;
        float Kv = a1;
        Kv = fmaf(2.f, a2, Kv);
        Kv = fmaf(2.f, a3, Kv);
        Kv = Kv + a4;
        kahan_add(q, cq, Kq);
        kahan_add(v, cv, Kv);
        // modes taking plain sums hold their compensation at zero
        // (state_add; the run-time mask KConst::cmask as bits)
        if (k > 0) {
            cq = __int_as_float(__float_as_int(cq) & cmb);
            cv = __int_as_float(__float_as_int(cv) & cmb);
        }
        // the tangent of direction e for this lane's mode
        float ta = tl_lane(P1, Jc, w2, wq, tq, tv, dbase);
        float tKq = tv, tKv = ta;
        float tqs = fmaf(3.f, tv, tq), tvs = fmaf(3.f, ta, tv);
        ta = tl_lane(P2, Jc, w2, wq, tqs, tvs, dbase);
        tKq = fmaf(2.f, tvs, tKq);
        tKv = fmaf(2.f, ta, tKv);
        tqs = fmaf(3.f, tvs, tq);
        tvs = fmaf(3.f, ta, tv);
        ta = tl_lane(P3, Jc, w2, wq, tqs, tvs, dbase);
        tKq = fmaf(2.f, tvs, tKq);
        tKv = fmaf(2.f, ta, tKv);
        tqs = fmaf(6.f, tvs, tq);
        tvs = fmaf(6.f, ta, tv);
        ta = tl_lane(P4, Jc, w2, wq, tqs, tvs, dbase);
        tq = tq + (tKq + tvs);
        tv = tv + (tKv + ta);
    }
    if (!store || k != 0) return;
    if (e == 0) S_out[p] = (S < INFINITY) ? S : INFINITY;
    double* H = H_out + (size_t)p * D * D;
#pragma unroll
    for (int f = 0; f < D; ++f)
        if (f <= e) {
            H[e * D + f] = aH[f];
            H[f * D + e] = aH[f];
        }
    b_out[(size_t)p * D + e] = ab;
}

bool sens_modes_supported(int m, int force, int P, int D) {
    return m == 3 && (force == F_LINEAR || force == F_DMT || force == F_HOOKE) && D >= 1 &&
           D <= 5 && (long long)P * 3 * D <= 152LL * 4 * 32;
}

cudaError_t launch_sens_modes(const KConst<float>& K, const float* x, int P, const float* U,
                              float* S, double* H, double* b, cudaStream_t st, const int64_t* off,
                              const int* order, int per_slot) {
    const int D = K.D;
    const int per_warp = 32 / (3 * D);
    const int blocks = (P + per_warp - 1) / per_warp;
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    auto go = [&](auto Fc, auto Dc) -> cudaError_t {
        auto kern = sens_modes_kernel<decltype(Fc)::value, decltype(Dc)::value>;
        if (smem > 24 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, kLaneThreads, smem, st>>>(K, x, P, U, off, order, per_slot, S, H, b);
        return cudaGetLastError();
    };
    auto byD = [&](auto Fc) -> cudaError_t {
        switch (D) {
            case 1: return go(Fc, std::integral_constant<int, 1>{});
            case 2: return go(Fc, std::integral_constant<int, 2>{});
            case 3: return go(Fc, std::integral_constant<int, 3>{});
            case 4: return go(Fc, std::integral_constant<int, 4>{});
            case 5: return go(Fc, std::integral_constant<int, 5>{});
        }
        return cudaErrorInvalidValue;
    };
    switch (K.force) {
        case F_LINEAR: return byD(std::integral_constant<int, F_LINEAR>{});
        case F_DMT: return byD(std::integral_constant<int, F_DMT>{});
        case F_HOOKE: return byD(std::integral_constant<int, F_HOOKE>{});
    }
    return cudaErrorInvalidValue;
}

bool sens_lanes_preferred(int P, int D) {
    // one warp per SM sub-partition at most: past that the redundant primal
    // solves cost more than the shorter chains gain
    return (long long)P * lanes_for(D) <= 152LL * 4 * 32;
}

cudaError_t launch_sens_lanes(const KConst<float>& K, const float* x, int P, const float* U,
                              float* S, double* H, double* b, cudaStream_t st, const int64_t* off,
                              const int* order, int per_slot) {
    const int L = lanes_for(K.D);
    const int blocks = (int)(((long long)P * L + kLaneThreads - 1) / kLaneThreads);
    const size_t smem = sizeof(float) * (size_t)(K.spc2 + 1);
    auto go = [&](auto Mc, auto Fc, auto Lc) -> cudaError_t {
        auto kern = sens_lanes_kernel<decltype(Mc)::value, decltype(Fc)::value, decltype(Lc)::value>;
        if (smem > 24 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, kLaneThreads, smem, st>>>(K, x, P, U, off, order, per_slot, S, H, b);
        return cudaGetLastError();
    };
    auto byL = [&](auto Mc, auto Fc) -> cudaError_t {
        if (L == 2) return go(Mc, Fc, std::integral_constant<int, 2>{});
        if (L == 4) return go(Mc, Fc, std::integral_constant<int, 4>{});
        return go(Mc, Fc, std::integral_constant<int, 8>{});
    };
    auto byF = [&](auto Mc) -> cudaError_t {
        switch (K.force) {
            case F_LINEAR: return byL(Mc, std::integral_constant<int, F_LINEAR>{});
            case F_DMT: return byL(Mc, std::integral_constant<int, F_DMT>{});
            case F_DMT_KV: return byL(Mc, std::integral_constant<int, F_DMT_KV>{});
            case F_HOOKE: return byL(Mc, std::integral_constant<int, F_HOOKE>{});
            case F_SPRING_DAMPER: return byL(Mc, std::integral_constant<int, F_SPRING_DAMPER>{});
        }
        return cudaErrorInvalidValue;
    };
    if (K.m == 1) return byF(std::integral_constant<int, 1>{});
    if (K.m == 3) return byF(std::integral_constant<int, 3>{});
    return byF(std::integral_constant<int, AFM_MAXM>{});
}

}  // namespace afm
