// kern_adjoint.cu -- discrete adjoint of the fused forward solve: gradient of
// the misfit S (Eq. 5) with respect to the normalised force parameters x,
// through every RK4 step of Eq. 2 (Sec. 3.2), one thread per particle.
//
// Forward pass: the RK4 loop of afm_device.cuh with every mode compensated
// (the gradient is more sensitive to the trajectory's rounding than the
// misfit; the forward kernels compensate the lowest mode only), storing the
// full state (modal deflections, rates and their Kahan compensations) every
// AFM_SEG steps.  Reverse pass: for each segment, last first, the AFM_SEG steps are
// recomputed from their checkpoint (bit-identical to the forward pass) while
// the gap d and gap rate d' of each RK4 stage and the tip deflection after
// each step are kept in shared memory; then the adjoint state runs back
// through the segment, one reverse RK4 step at a time, accumulating the
// cotangents of the four force coefficients.  A final chain rule maps them to
// d S / d x.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

constexpr int SEG = AFM_SEG;
constexpr int SEGW = 9;   // per step: (d, d') of 4 stages + tip deflection
constexpr int ADJ_THREADS = 32;

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

// Transposed Jacobian of the modal right-hand side f(q, v) = (v, a) at one
// stage, applied to w = (wq, wv); accumulates the force-coefficient
// cotangents into cb.
template <int M, int FORCE>
__device__ __forceinline__ void rhs_vjp(const KConst<float>& K, const Coef<float>& c, float d,
                                        float dd, const float* wq, const float* wv, float* oq,
                                        float* ov, float* cb) {
    float Fd, Fr, Fc[4];
    force_partials<FORCE>(c, d, dd, Fd, Fr, Fc);
    float Fbar = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) Fbar = fmaf(K.tip[i], wv[i], Fbar);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float aq = fmaf(Fbar, Fd, -K.w2[i] * wv[i]);
        if (i == 0) aq = fmaf(-K.w2lo[0], wv[0], aq);
        oq[i] = aq;
        ov[i] = wq[i] + fmaf(Fbar, Fr, -K.wq[i] * wv[i]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) cb[k] = fmaf(Fbar, Fc[k], cb[k]);
}

// One RK4 step as in rk4_step (every mode compensated), recording (d, d') of
// each stage.
template <int M, int FORCE>
__device__ __forceinline__ void rk4_step_rec(const KConst<float>& K, const Coef<float>& c, float* q,
                                             float* v, float* cq, float* cv, float g0, float gh,
                                             float g1, float* rec) {
    float a[M], qs[M], vs[M], Kq[M], Kv[M];
    auto gap = [&](const float* qq, const float* vv, int s) {
        float u = qq[0], r = vv[0];
#pragma unroll
        for (int i = 1; i < M; ++i) {
            u += qq[i];
            r += vv[i];
        }
        rec[2 * s] = K.Zc + u;
        rec[2 * s + 1] = r;
    };
    gap(q, v, 0);
    accel<float, M, FORCE>(K, c, q, v, g0, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = v[i];
        Kv[i] = a[i];
        qs[i] = fmaf(3.f, v[i], q[i]);
        vs[i] = fmaf(3.f, a[i], v[i]);
    }
    gap(qs, vs, 1);
    accel<float, M, FORCE>(K, c, qs, vs, gh, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fmaf(2.f, vs[i], Kq[i]);
        Kv[i] = fmaf(2.f, a[i], Kv[i]);
        qs[i] = fmaf(3.f, vs[i], q[i]);
        vs[i] = fmaf(3.f, a[i], v[i]);
    }
    gap(qs, vs, 2);
    accel<float, M, FORCE>(K, c, qs, vs, gh, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fmaf(2.f, vs[i], Kq[i]);
        Kv[i] = fmaf(2.f, a[i], Kv[i]);
        qs[i] = fmaf(6.f, vs[i], q[i]);
        vs[i] = fmaf(6.f, a[i], v[i]);
    }
    gap(qs, vs, 3);
    accel<float, M, FORCE>(K, c, qs, vs, g1, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = Kq[i] + vs[i];
        Kv[i] = Kv[i] + a[i];
        state_add<float, true>(i, q[i], cq[i], Kq[i]);
        state_add<float, true>(i, v[i], cv[i], Kv[i]);
    }
}

template <int M, int FORCE>
__global__ void __launch_bounds__(ADJ_THREADS) adjoint_kernel(const KConst<float> K,
                                                              const float* __restrict__ x, int P,
                                                              const float* __restrict__ U,
                                                              float* __restrict__ S_out,
                                                              float* __restrict__ G,
                                                              float* __restrict__ ckpt,
                                                              const int64_t* __restrict__ off,
                                                              const int* __restrict__ order,
                                                              int per_slot) {
    extern __shared__ __align__(16) float sma[];
    float* tab = sma;
    float* seg = sma + ((K.spc2 + 1 + 3) & ~3);   // [SEG][SEGW][ADJ_THREADS]
    build_drive_table(K, tab);
    __syncthreads();
    const int tid = threadIdx.x;
    const int p = blockIdx.x * blockDim.x + tid;
    if (p >= P) return;
    int N = K.n_steps;
    if (off != nullptr) {
        const int slot = p / per_slot;
        const int pix = order != nullptr ? order[slot] : slot;
        U += off[pix];
        N = (int)(off[pix + 1] - off[pix]);
        if (N > K.n_steps) {   // beyond the checkpoint buffer
            S_out[p] = INFINITY;
            for (int d = 0; d < K.D; ++d) G[(size_t)d * P + p] = 0.f;
            return;
        }
    }
    const int nseg = (N + SEG - 1) / SEG;
    float xd[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) xd[d] = x[(size_t)d * P + p];
    const Coef<float> c = make_coef<float, float>(K, xd);

    // forward pass with checkpoints
    float q[M], v[M], cq[M], cv[M];
    init_state<float, M>(K, q, v, cq, cv);
    float S = 0.f, cS = 0.f;
    int j = 0;
    for (int n = 0; n < N; ++n) {
        if (n % SEG == 0) {
            float* ck = ckpt + (size_t)(n / SEG) * 4 * M * P + p;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                ck[(size_t)(0 * M + i) * P] = q[i];
                ck[(size_t)(1 * M + i) * P] = v[i];
                ck[(size_t)(2 * M + i) * P] = cq[i];
                ck[(size_t)(3 * M + i) * P] = cv[i];
            }
        }
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= K.spc2) j = 0;
        rk4_step<float, M, FORCE, true>(K, c, q, v, cq, cv, g0, gh, g1);
        const float r = U[n] - tip_sum<float, M>(q);
        const float y = fmaf(r, r, -cS);
        const float t = add_rn(S, y);
        cS = sub_rn(sub_rn(t, S), y);
        S = t;
    }
    S_out[p] = S;

    // reverse pass
    // adjoint state with Kahan compensations: like the forward state it takes
    // per-step increments far smaller than itself over the whole record
    float lq[M], lv[M], clq[M], clv[M];
#pragma unroll
    for (int i = 0; i < M; ++i) lq[i] = lv[i] = clq[i] = clv[i] = 0.f;
    // force-coefficient cotangents: FP32 within a segment, folded into FP64
    // after each (the sum runs over every stage of every step)
    double cbd[4] = {0.0, 0.0, 0.0, 0.0};
    for (int sg = nseg - 1; sg >= 0; --sg) {
        float cb[4] = {0.f, 0.f, 0.f, 0.f};
        const int n0 = sg * SEG, n1 = min(N, n0 + SEG);
        const float* ck = ckpt + (size_t)sg * 4 * M * P + p;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            q[i] = ck[(size_t)(0 * M + i) * P];
            v[i] = ck[(size_t)(1 * M + i) * P];
            cq[i] = ck[(size_t)(2 * M + i) * P];
            cv[i] = ck[(size_t)(3 * M + i) * P];
        }
        int jj = (int)(((long long)2 * n0) % K.spc2);
        for (int n = n0; n < n1; ++n) {
            const float g0 = tab[jj], gh = tab[jj + 1], g1 = tab[jj + 2];
            jj += 2;
            if (jj >= K.spc2) jj = 0;
            float rec[8];
            rk4_step_rec<M, FORCE>(K, c, q, v, cq, cv, g0, gh, g1, rec);
            float* sb = seg + (size_t)(n - n0) * SEGW * ADJ_THREADS + tid;
#pragma unroll
            for (int k = 0; k < 8; ++k) sb[k * ADJ_THREADS] = rec[k];
            sb[8 * ADJ_THREADS] = tip_sum<float, M>(q);
        }
        for (int n = n1 - 1; n >= n0; --n) {
            const float* sb = seg + (size_t)(n - n0) * SEGW * ADJ_THREADS + tid;
            // misfit term of the state after step n
            const float r = U[n] - sb[8 * ADJ_THREADS];
#pragma unroll
            for (int i = 0; i < M; ++i) kahan_add(lq[i], clq[i], -2.f * r);
            // reverse RK4 step: stage cotangents kb_s (k1..k4 weights 1,2,2,1)
            float k1q[M], k1v[M], k2q[M], k2v[M], k3q[M], k3v[M], oq[M], ov[M];
            float yq[M], yv[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                yq[i] = 0.f;   // the step's increment of the adjoint state
                yv[i] = 0.f;
                k1q[i] = lq[i];
                k1v[i] = lv[i];
                k2q[i] = 2.f * lq[i];
                k2v[i] = 2.f * lv[i];
                k3q[i] = 2.f * lq[i];
                k3v[i] = 2.f * lv[i];
            }
            // stage 4 (y4 = y + 6 k3), weight 1
            rhs_vjp<M, FORCE>(K, c, sb[6 * ADJ_THREADS], sb[7 * ADJ_THREADS], lq, lv, oq, ov, cb);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                yq[i] += oq[i];
                yv[i] += ov[i];
                k3q[i] = fmaf(6.f, oq[i], k3q[i]);
                k3v[i] = fmaf(6.f, ov[i], k3v[i]);
            }
            // stage 3 (y3 = y + 3 k2)
            rhs_vjp<M, FORCE>(K, c, sb[4 * ADJ_THREADS], sb[5 * ADJ_THREADS], k3q, k3v, oq, ov, cb);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                yq[i] += oq[i];
                yv[i] += ov[i];
                k2q[i] = fmaf(3.f, oq[i], k2q[i]);
                k2v[i] = fmaf(3.f, ov[i], k2v[i]);
            }
            // stage 2 (y2 = y + 3 k1)
            rhs_vjp<M, FORCE>(K, c, sb[2 * ADJ_THREADS], sb[3 * ADJ_THREADS], k2q, k2v, oq, ov, cb);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                yq[i] += oq[i];
                yv[i] += ov[i];
                k1q[i] = fmaf(3.f, oq[i], k1q[i]);
                k1v[i] = fmaf(3.f, ov[i], k1v[i]);
            }
            // stage 1 (y)
            rhs_vjp<M, FORCE>(K, c, sb[0], sb[1 * ADJ_THREADS], k1q, k1v, oq, ov, cb);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                kahan_add(lq[i], clq[i], yq[i] + oq[i]);
                kahan_add(lv[i], clv[i], yv[i] + ov[i]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cbd[k] += (double)cb[k];
    }
    double J[4][AFM_MAXD];
    coef_jacobian<float>(K, xd, J);
    for (int d = 0; d < K.D; ++d) {
        double g = 0.0;
        for (int k = 0; k < 4; ++k) g += cbd[k] * J[k][d];
        G[(size_t)d * P + p] = (float)g;
    }
}

size_t adjoint_ckpt_floats(int m, int n_steps, int P) {
    const int M = m == 1 ? 1 : (m == 3 ? 3 : AFM_MAXM);
    return (size_t)((n_steps + SEG - 1) / SEG) * 4 * M * P;
}

cudaError_t launch_adjoint(const KConst<float>& K, const float* x, int P, const float* U, float* S,
                           float* G, float* ckpt, cudaStream_t st, const int64_t* off,
                           const int* order, int per_slot) {
    const size_t smem = sizeof(float) * ((size_t)((K.spc2 + 1 + 3) & ~3) +
                                         (size_t)SEG * SEGW * ADJ_THREADS);
    const int blocks = (P + ADJ_THREADS - 1) / ADJ_THREADS;
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        auto kern = adjoint_kernel<decltype(Mc)::value, decltype(Fc)::value>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, ADJ_THREADS, smem, st>>>(K, x, P, U, S, G, ckpt, off, order, per_slot);
        return cudaGetLastError();
    });
}

}  // namespace afm
