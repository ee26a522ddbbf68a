// kern_lm.cu -- Levenberg-Marquardt polish: residual sensitivities by
// tangent-linear (forward-mode) differentiation of the FP32 RK4 solve, the
// normal equations of the misfit (Eq. 5), damped Gauss-Newton trial points
// for a ladder of damping values, and the choice among them.
//
// For the misfit S = sum_n r_n^2, r_n = U_n - u_n(x), the sensitivities
// a_n = du_n/dx (D per step) give H = sum a_n a_n^T (Gauss-Newton matrix,
// half the Gauss-Newton Hessian) and b = sum a_n r_n = -dS/dx / 2.  The
// primal solve inside the sensitivity kernel is the forward kernel's
// arithmetic, so S is bit-identical to afm_forward_batch's.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"
#include "afm_tangent.cuh"

namespace afm {

namespace {

template <typename F>
cudaError_t dispatch_mfd(int m, int force, int D, F&& f) {
    auto byD = [&](auto Mc, auto Fc) -> cudaError_t {
        if (D <= 2) return f(Mc, Fc, std::integral_constant<int, 2>{});
        if (D <= 4) return f(Mc, Fc, std::integral_constant<int, 4>{});
        return f(Mc, Fc, std::integral_constant<int, AFM_MAXD>{});
    };
    auto byF = [&](auto Mc) -> cudaError_t {
        switch (force) {
            case F_LINEAR: return byD(Mc, std::integral_constant<int, F_LINEAR>{});
            case F_DMT: return byD(Mc, std::integral_constant<int, F_DMT>{});
            case F_DMT_KV: return byD(Mc, std::integral_constant<int, F_DMT_KV>{});
            case F_HOOKE: return byD(Mc, std::integral_constant<int, F_HOOKE>{});
            case F_SPRING_DAMPER: return byD(Mc, std::integral_constant<int, F_SPRING_DAMPER>{});
        }
        return cudaErrorInvalidValue;
    };
    if (m == 1) return byF(std::integral_constant<int, 1>{});
    if (m == 3) return byF(std::integral_constant<int, 3>{});
    return byF(std::integral_constant<int, AFM_MAXM>{});
}

constexpr int kThreads = 32;
constexpr int kFold = 32;   // steps summed in FP32 before folding into FP64 totals

}  // namespace

// Sensitivity pass of one particle per thread: S (as the forward kernel),
// H [P][D][D] and b [P][D] in FP64.  Ragged form as the adjoint: off !=
// nullptr gives particle p the record of pixel order[p / per_slot].
// PP (ragged form only): each particle's pixel has its own constants and
// drive table (pix), read from global memory.
template <int M, int FORCE, int ND, bool PP>
__global__ void __launch_bounds__(kThreads) sens_kernel(const KConst<float> K0,
                                                        const float* __restrict__ x, int P,
                                                        const float* __restrict__ U,
                                                        const int64_t* __restrict__ off,
                                                        const int* __restrict__ order,
                                                        int per_slot, float* __restrict__ S_out,
                                                        double* __restrict__ H_out,
                                                        double* __restrict__ b_out,
                                                        const PixConst pixc) {
    extern __shared__ __align__(16) float tabs[];
    __shared__ double accH[ND * (ND + 1) / 2][kThreads], accb[ND][kThreads];
    if constexpr (!PP) {
        build_drive_table(K0, tabs);
        __syncthreads();
    }
    const int tid = threadIdx.x;
    const int p = blockIdx.x * blockDim.x + tid;
    if (p >= P) return;
    int n = K0.n_steps, pix = 0;
    if (off != nullptr) {
        const int slot = p / per_slot;
        pix = order != nullptr ? order[slot] : slot;
        U += off[pix];
        n = (int)(off[pix + 1] - off[pix]);
    }
    const KConst<float>* Kp = &K0;
    const float* tab = tabs;
    if constexpr (PP) {
        Kp = pixc.kf + pix;
        tab = pixc.tab32 + (size_t)pix * pixc.ld;
    }
    const KConst<float>& K = *Kp;
    const int D = K.D;
    float xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < D ? x[(size_t)d * P + p] : 0.f;
    const Coef<float> c = make_coef<float, float>(K, xd);
    float Jc[4][ND];
    {
        double Jd[4][AFM_MAXD];
        coef_jacobian<float>(K, xd, Jd);
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int e = 0; e < ND; ++e) Jc[k][e] = e < D ? (float)Jd[k][e] : 0.f;
    }
    float q[M], v[M], cq[M], cv[M], tq[ND][M], tv[ND][M];
    init_state<float, M>(K, q, v, cq, cv);
#pragma unroll
    for (int e = 0; e < ND; ++e)
#pragma unroll
        for (int i = 0; i < M; ++i) tq[e][i] = tv[e][i] = 0.f;
#pragma unroll
    for (int t = 0; t < ND * (ND + 1) / 2; ++t) accH[t][tid] = 0.0;
#pragma unroll
    for (int e = 0; e < ND; ++e) accb[e][tid] = 0.0;
    float hc[ND * (ND + 1) / 2], bc[ND];
#pragma unroll
    for (int t = 0; t < ND * (ND + 1) / 2; ++t) hc[t] = 0.f;
#pragma unroll
    for (int e = 0; e < ND; ++e) bc[e] = 0.f;
    float S = 0.f, cS = 0.f;
    int j = 0, fold = 0;
    const int spc2 = K.spc2;
    for (int s = 0; s < n; ++s) {
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        rk4_step_tl<M, FORCE, ND>(K, c, Jc, q, v, cq, cv, tq, tv, g0, gh, g1);
        const float u = tip_sum<float, M>(q);
        const float r = U[s] - u;
        const float y = fmaf(r, r, -cS);
        const float t = add_rn(S, y);
        cS = sub_rn(sub_rn(t, S), y);
        S = t;
        float au[ND];
#pragma unroll
        for (int e = 0; e < ND; ++e) au[e] = tip_sum<float, M>(tq[e]);
        int w = 0;
#pragma unroll
        for (int e = 0; e < ND; ++e) {
            bc[e] = fmaf(au[e], r, bc[e]);
#pragma unroll
            for (int f = 0; f <= e; ++f) {
                hc[w] = fmaf(au[e], au[f], hc[w]);
                ++w;
            }
        }
        if (++fold == kFold || s + 1 == n) {
            fold = 0;
#pragma unroll
            for (int t2 = 0; t2 < ND * (ND + 1) / 2; ++t2) {
                accH[t2][tid] += (double)hc[t2];
                hc[t2] = 0.f;
            }
#pragma unroll
            for (int e = 0; e < ND; ++e) {
                accb[e][tid] += (double)bc[e];
                bc[e] = 0.f;
            }
        }
    }
    if (!(S < INFINITY)) S = INFINITY;
    S_out[p] = S;
    double* H = H_out + (size_t)p * D * D;
    int w = 0;
    for (int e = 0; e < ND; ++e) {
        for (int f = 0; f <= e; ++f) {
            if (e < D) {
                H[e * D + f] = accH[w][tid];
                H[f * D + e] = accH[w][tid];
            }
            ++w;
        }
        if (e < D) b_out[(size_t)p * D + e] = accb[e][tid];
    }
}

// Trial points of candidate k: clamp(x + delta_j) with (H + lambda_j W)
// delta_j = b, lambda_j = lam0 ratio^j, W = diag(max(H_dd, 1e-12 max H_ee)),
// solved by Cholesky in FP64.  Output column k * J + j of Xc [D][K*J].
__global__ void lm_cand_kernel(int D, int K, int J, const float* __restrict__ x,
                               const double* __restrict__ H, const double* __restrict__ b,
                               double lam0, double ratio, float* __restrict__ Xc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double* Hk = H + (size_t)k * D * D;
    double hmax = 0.0;
    for (int d = 0; d < D; ++d) hmax = fmax(hmax, Hk[d * D + d]);
    const size_t KJ = (size_t)K * J;
    double lam = lam0;
    for (int j = 0; j < J; ++j, lam *= ratio) {
        double L[AFM_MAXD][AFM_MAXD], y[AFM_MAXD];
        bool ok = hmax > 0.0;
        for (int r = 0; r < D && ok; ++r) {
            for (int c = 0; c <= r; ++c) {
                double s = Hk[r * D + c];
                if (r == c) s += lam * fmax(Hk[r * D + r], 1e-12 * hmax);
                for (int t = 0; t < c; ++t) s -= L[r][t] * L[c][t];
                if (r == c) {
                    if (!(s > 0.0)) {
                        ok = false;
                        break;
                    }
                    L[r][r] = sqrt(s);
                } else {
                    L[r][c] = s / L[c][c];
                }
            }
        }
        if (ok) {
            for (int r = 0; r < D; ++r) {
                double s = b[(size_t)k * D + r];
                for (int t = 0; t < r; ++t) s -= L[r][t] * y[t];
                y[r] = s / L[r][r];
            }
            for (int r = D - 1; r >= 0; --r) {
                double s = y[r];
                for (int t = r + 1; t < D; ++t) s -= L[t][r] * y[t];
                y[r] = s / L[r][r];
            }
        }
        for (int d = 0; d < D; ++d) {
            double xn = (double)x[(size_t)d * K + k] + (ok ? y[d] : 0.0);
            if (!(xn > 0.0)) xn = 0.0;
            if (xn > 1.0) xn = 1.0;
            Xc[(size_t)d * KJ + (size_t)k * J + j] = (float)xn;
        }
    }
}

// The trial point of least misfit (first on ties) replaces x if it lowers S.
__global__ void lm_select_kernel(int D, int K, int J, float* __restrict__ x, float* __restrict__ S,
                                 const float* __restrict__ Xc, const float* __restrict__ Sc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int jb = 0;
    for (int j = 1; j < J; ++j)
        if (Sc[(size_t)k * J + j] < Sc[(size_t)k * J + jb]) jb = j;
    const float Sj = Sc[(size_t)k * J + jb];
    if (Sj < S[k]) {
        const size_t KJ = (size_t)K * J;
        for (int d = 0; d < D; ++d) x[(size_t)d * K + k] = Xc[(size_t)d * KJ + (size_t)k * J + jb];
        S[k] = Sj;
    }
}

// lm_select_kernel for the fused step: the point kept also brings its normal
// equations (computed by the sensitivity pass over the trial points).
__global__ void lm_select_hb_kernel(int D, int K, int J, float* __restrict__ x, float* __restrict__ S,
                                    double* __restrict__ H, double* __restrict__ b,
                                    const float* __restrict__ Xc, const float* __restrict__ Sc,
                                    const double* __restrict__ Hc, const double* __restrict__ bc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int jb = 0;
    for (int j = 1; j < J; ++j)
        if (Sc[(size_t)k * J + j] < Sc[(size_t)k * J + jb]) jb = j;
    const float Sj = Sc[(size_t)k * J + jb];
    if (Sj < S[k]) {
        const size_t KJ = (size_t)K * J, c = (size_t)k * J + jb;
        for (int d = 0; d < D; ++d) x[(size_t)d * K + k] = Xc[(size_t)d * KJ + c];
        for (int e = 0; e < D * D; ++e) H[(size_t)k * D * D + e] = Hc[c * D * D + e];
        for (int d = 0; d < D; ++d) b[(size_t)k * D + d] = bc[c * D + d];
        S[k] = Sj;
    }
}

cudaError_t launch_lm_select_hb(int D, int K, int J, float* x, float* S, double* H, double* b,
                                const float* Xc, const float* Sc, const double* Hc,
                                const double* bc, cudaStream_t st) {
    const int threads = 64;
    lm_select_hb_kernel<<<(K + threads - 1) / threads, threads, 0, st>>>(D, K, J, x, S, H, b, Xc,
                                                                         Sc, Hc, bc);
    return cudaGetLastError();
}

cudaError_t launch_sens(const KConst<float>& K, const float* x, int P, const float* U, float* S,
                        double* H, double* b, cudaStream_t st, const int64_t* off, const int* order,
                        int per_slot, const PixConst& pix) {
    const bool pp = pix.kf != nullptr;
    if (pp && off == nullptr) return cudaErrorInvalidValue;
    if (!pp && sens_modes_supported(K.m, K.force, P, K.D))
        return launch_sens_modes(K, x, P, U, S, H, b, st, off, order, per_slot);
    if (!pp && sens_lanes_preferred(P, K.D))
        return launch_sens_lanes(K, x, P, U, S, H, b, st, off, order, per_slot);
    const int blocks = (P + kThreads - 1) / kThreads;
    const size_t smem = pp ? 0 : sizeof(float) * (size_t)(K.spc2 + 1);
    return dispatch_mfd(K.m, K.force, K.D, [&](auto Mc, auto Fc, auto Dc) -> cudaError_t {
        auto go = [&](auto Pc) -> cudaError_t {
            auto kern = sens_kernel<decltype(Mc)::value, decltype(Fc)::value, decltype(Dc)::value,
                                    decltype(Pc)::value>;
            if (smem > 24 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(
                    kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            kern<<<blocks, kThreads, smem, st>>>(K, x, P, U, off, order, per_slot, S, H, b, pix);
            return cudaGetLastError();
        };
        return pp ? go(std::true_type{}) : go(std::false_type{});
    });
}

cudaError_t launch_lm_cand(int D, int K, int J, const float* x, const double* H, const double* b,
                           double lam0, double ratio, float* Xc, cudaStream_t st) {
    const int threads = 64;
    lm_cand_kernel<<<(K + threads - 1) / threads, threads, 0, st>>>(D, K, J, x, H, b, lam0, ratio, Xc);
    return cudaGetLastError();
}

cudaError_t launch_lm_select(int D, int K, int J, float* x, float* S, const float* Xc,
                             const float* Sc, cudaStream_t st) {
    const int threads = 64;
    lm_select_kernel<<<(K + threads - 1) / threads, threads, 0, st>>>(D, K, J, x, S, Xc, Sc);
    return cudaGetLastError();
}

}  // namespace afm
