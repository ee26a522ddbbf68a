// afm_tangent.cuh -- tangent-linear (forward-mode) RK4 step: the primal
// arithmetic of rk4_step with the tangents of ND parameter directions
// carried along (sensitivity kernels of kern_lm.cu and kern_lm_lanes.cu).
#pragma once

#include "afm_device.cuh"

namespace afm {

// Tangent of the modal accelerations at one stage: for each direction n,
// da_i = tip_i dF - wq_i dv_i - w2_i dq_i with dF = F_d sum dq + F_r sum dv +
// sum_k F_ck dc_k/dx_n.
template <int M, int FORCE, int ND>
__device__ __forceinline__ void tl_accel(const KConst<float>& K, const Coef<float>& c,
                                         const float (&Jc)[4][ND], const float* q, const float* v,
                                         const float (&tq)[ND][M], const float (&tv)[ND][M],
                                         float (&ta)[ND][M]) {
    float u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u += q[i];
    float dd = 0.f;
    if (UsesRate<FORCE>::value) {
        dd = v[0];
#pragma unroll
        for (int i = 1; i < M; ++i) dd += v[i];
    }
    float Fd, Fr, Fc[4];
    force_partials<FORCE>(c, K.Zc + u, dd, Fd, Fr, Fc);
#pragma unroll
    for (int n = 0; n < ND; ++n) {
        float su = tq[n][0], sv = tv[n][0];
#pragma unroll
        for (int i = 1; i < M; ++i) {
            su += tq[n][i];
            sv += tv[n][i];
        }
        float dF = Fd * su;
        if (UsesRate<FORCE>::value) dF = fmaf(Fr, sv, dF);
#pragma unroll
        for (int k = 0; k < 4; ++k) dF = fmaf(Fc[k], Jc[k][n], dF);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float base = fmaf(-K.wq[i], tv[n][i], -K.w2[i] * tq[n][i]);
            ta[n][i] = (M <= 4) ? base + dF : fmaf(K.tip[i], dF, base);
        }
    }
}

// One RK4 step of rk4_step (identical primal arithmetic) with the tangents
// of ND directions carried along.
template <int M, int FORCE, int ND>
__device__ __forceinline__ void rk4_step_tl(const KConst<float>& K, const Coef<float>& c,
                                            const float (&Jc)[4][ND], float* q, float* v,
                                            float* cq, float* cv, float (&tq)[ND][M],
                                            float (&tv)[ND][M], float g0, float gh, float g1) {
    float a[M], qs[M], vs[M], Kq[M], Kv[M];
    float ta[ND][M], tqs[ND][M], tvs[ND][M], tKq[ND][M], tKv[ND][M];
    accel<float, M, FORCE>(K, c, q, v, g0, a);
    tl_accel<M, FORCE, ND>(K, c, Jc, q, v, tq, tv, ta);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = v[i];
        Kv[i] = a[i];
        qs[i] = fmaf(3.f, v[i], q[i]);
        vs[i] = fmaf(3.f, a[i], v[i]);
#pragma unroll
        for (int n = 0; n < ND; ++n) {
            tKq[n][i] = tv[n][i];
            tKv[n][i] = ta[n][i];
            tqs[n][i] = fmaf(3.f, tv[n][i], tq[n][i]);
            tvs[n][i] = fmaf(3.f, ta[n][i], tv[n][i]);
        }
    }
    accel<float, M, FORCE>(K, c, qs, vs, gh, a);
    tl_accel<M, FORCE, ND>(K, c, Jc, qs, vs, tqs, tvs, ta);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fmaf(2.f, vs[i], Kq[i]);
        Kv[i] = fmaf(2.f, a[i], Kv[i]);
        qs[i] = fmaf(3.f, vs[i], q[i]);
        vs[i] = fmaf(3.f, a[i], v[i]);
#pragma unroll
        for (int n = 0; n < ND; ++n) {
            tKq[n][i] = fmaf(2.f, tvs[n][i], tKq[n][i]);
            tKv[n][i] = fmaf(2.f, ta[n][i], tKv[n][i]);
            tqs[n][i] = fmaf(3.f, tvs[n][i], tq[n][i]);
            tvs[n][i] = fmaf(3.f, ta[n][i], tv[n][i]);
        }
    }
    accel<float, M, FORCE>(K, c, qs, vs, gh, a);
    tl_accel<M, FORCE, ND>(K, c, Jc, qs, vs, tqs, tvs, ta);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fmaf(2.f, vs[i], Kq[i]);
        Kv[i] = fmaf(2.f, a[i], Kv[i]);
        qs[i] = fmaf(6.f, vs[i], q[i]);
        vs[i] = fmaf(6.f, a[i], v[i]);
#pragma unroll
        for (int n = 0; n < ND; ++n) {
            tKq[n][i] = fmaf(2.f, tvs[n][i], tKq[n][i]);
            tKv[n][i] = fmaf(2.f, ta[n][i], tKv[n][i]);
            tqs[n][i] = fmaf(6.f, tvs[n][i], tq[n][i]);
            tvs[n][i] = fmaf(6.f, ta[n][i], tv[n][i]);
        }
    }
    accel<float, M, FORCE>(K, c, qs, vs, g1, a);
    tl_accel<M, FORCE, ND>(K, c, Jc, qs, vs, tqs, tvs, ta);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = Kq[i] + vs[i];
        Kv[i] = Kv[i] + a[i];
        kahan_add(q[i], cq[i], Kq[i]);
        kahan_add(v[i], cv[i], Kv[i]);
#pragma unroll
        for (int n = 0; n < ND; ++n) {
            tq[n][i] = tq[n][i] + (tKq[n][i] + tvs[n][i]);
            tv[n][i] = tv[n][i] + (tKv[n][i] + ta[n][i]);
        }
    }
}

}  // namespace afm
