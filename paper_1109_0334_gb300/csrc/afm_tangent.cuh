// afm_tangent.cuh -- tangent-linear (forward-mode) RK4 step: the primal
// arithmetic of rk4_step with the tangents of ND parameter directions
// carried along (sensitivity kernels of kern_lm.cu and kern_lm_lanes.cu).
#pragma once

#include "afm_device.cuh"

namespace afm {

// Partials of the tip force at one RK4 stage state (the coefficients of the
// tangent recursion at that stage).
struct StagePartials {
    float Fd, Fr, Fc[4];
};

template <int M, int FORCE>
__device__ __forceinline__ void stage_partials(const KConst<float>& K, const Coef<float>& c,
                                               const float* q, const float* v, StagePartials& P) {
    float u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u += q[i];
    float dd = 0.f;
    if (UsesRate<FORCE>::value) {
        dd = v[0];
#pragma unroll
        for (int i = 1; i < M; ++i) dd += v[i];
    }
    force_partials<FORCE>(c, K.Zc + u, dd, P.Fd, P.Fr, P.Fc);
}

// tl_accel for one direction n with the stage's partials.
template <int M, int FORCE, int ND>
__device__ __forceinline__ void tl_stage(const KConst<float>& K, const StagePartials& P,
                                         const float (&Jc)[4][ND], int n, const float* tq,
                                         const float* tv, float* ta) {
    float su = tq[0], sv = tv[0];
#pragma unroll
    for (int i = 1; i < M; ++i) {
        su += tq[i];
        sv += tv[i];
    }
    float dF = P.Fd * su;
    if (UsesRate<FORCE>::value) dF = fmaf(P.Fr, sv, dF);
#pragma unroll
    for (int k = 0; k < 4; ++k) dF = fmaf(P.Fc[k], Jc[k][n], dF);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float base = fmaf(-K.wq[i], tv[i], -K.w2[i] * tq[i]);
        ta[i] = (M <= 4) ? base + dF : fmaf(K.tip[i], dF, base);
    }
}

// One RK4 step of rk4_step (identical primal arithmetic) with the tangents
// of ND directions carried along.  The primal step runs first and keeps the
// force partials of its four stages; then each direction takes its own
// linearised step (every operation per direction as in tl_accel's stage
// order), so only one direction's stage temporaries are live at a time.
template <int M, int FORCE, int ND>
__device__ __forceinline__ void rk4_step_tl(const KConst<float>& K, const Coef<float>& c,
                                            const float (&Jc)[4][ND], float* q, float* v,
                                            float* cq, float* cv, float (&tq)[ND][M],
                                            float (&tv)[ND][M], float g0, float gh, float g1) {
    StagePartials Ps[4];
    {
        float a[M], qs[M], vs[M], Kq[M], Kv[M];
        accel<float, M, FORCE>(K, c, q, v, g0, a);
        stage_partials<M, FORCE>(K, c, q, v, Ps[0]);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            Kq[i] = v[i];
            Kv[i] = a[i];
            qs[i] = fmaf(3.f, v[i], q[i]);
            vs[i] = fmaf(3.f, a[i], v[i]);
        }
        accel<float, M, FORCE>(K, c, qs, vs, gh, a);
        stage_partials<M, FORCE>(K, c, qs, vs, Ps[1]);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            Kq[i] = fmaf(2.f, vs[i], Kq[i]);
            Kv[i] = fmaf(2.f, a[i], Kv[i]);
            qs[i] = fmaf(3.f, vs[i], q[i]);
            vs[i] = fmaf(3.f, a[i], v[i]);
        }
        accel<float, M, FORCE>(K, c, qs, vs, gh, a);
        stage_partials<M, FORCE>(K, c, qs, vs, Ps[2]);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            Kq[i] = fmaf(2.f, vs[i], Kq[i]);
            Kv[i] = fmaf(2.f, a[i], Kv[i]);
            qs[i] = fmaf(6.f, vs[i], q[i]);
            vs[i] = fmaf(6.f, a[i], v[i]);
        }
        accel<float, M, FORCE>(K, c, qs, vs, g1, a);
        stage_partials<M, FORCE>(K, c, qs, vs, Ps[3]);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            Kq[i] = Kq[i] + vs[i];
            Kv[i] = Kv[i] + a[i];
            state_add(i, q[i], cq[i], Kq[i]);
            state_add(i, v[i], cv[i], Kv[i]);
        }
    }
#pragma unroll
    for (int n = 0; n < ND; ++n) {
        float ta[M], tqs[M], tvs[M], tKq[M], tKv[M];
        tl_stage<M, FORCE, ND>(K, Ps[0], Jc, n, tq[n], tv[n], ta);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            tKq[i] = tv[n][i];
            tKv[i] = ta[i];
            tqs[i] = fmaf(3.f, tv[n][i], tq[n][i]);
            tvs[i] = fmaf(3.f, ta[i], tv[n][i]);
        }
        tl_stage<M, FORCE, ND>(K, Ps[1], Jc, n, tqs, tvs, ta);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            tKq[i] = fmaf(2.f, tvs[i], tKq[i]);
            tKv[i] = fmaf(2.f, ta[i], tKv[i]);
            tqs[i] = fmaf(3.f, tvs[i], tq[n][i]);
            tvs[i] = fmaf(3.f, ta[i], tv[n][i]);
        }
        tl_stage<M, FORCE, ND>(K, Ps[2], Jc, n, tqs, tvs, ta);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            tKq[i] = fmaf(2.f, tvs[i], tKq[i]);
            tKv[i] = fmaf(2.f, ta[i], tKv[i]);
            tqs[i] = fmaf(6.f, tvs[i], tq[n][i]);
            tvs[i] = fmaf(6.f, ta[i], tv[n][i]);
        }
        tl_stage<M, FORCE, ND>(K, Ps[3], Jc, n, tqs, tvs, ta);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            tq[n][i] = tq[n][i] + (tKq[i] + tvs[i]);
            tv[n][i] = tv[n][i] + (tKv[i] + ta[i]);
        }
    }
}

}  // namespace afm
