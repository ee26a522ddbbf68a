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
