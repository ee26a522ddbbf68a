// afm_reeval.cuh -- device pieces of the FP64 re-evaluation by multiple
// shooting in time (kern_reeval.cu: one winner; kern_reeval_batch.cu: one
// winner per pixel of a batch): the FP64 RK4 step with the stage force
// slopes recorded, its FP32 linearisation, and the launch dispatch.
#pragma once

#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {
namespace reeval {

constexpr double kDefectTol = 1e-9;
constexpr int kSweeps = 2;
constexpr int kRec = 8;   // recorded floats per RK4 step: (dF/dd, dF/dd') x 4 stages

inline size_t a256(size_t n) { return (n + 255) & ~size_t(255); }

// State components of the kernels' template mode count for m modes.
inline int reeval_modes(int m) { return (m == 1 || m == 3) ? m : AFM_MAXM; }

__host__ __device__ inline int reeval_segments(int n_steps) { return (n_steps + AFM_SEG - 1) / AFM_SEG; }

template <typename F>
cudaError_t dispatch_m13(int m, int force, F&& f) {
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
    if (m >= 1 && m <= AFM_MAXM) return byF(std::integral_constant<int, AFM_MAXM>{});
    return cudaErrorInvalidValue;
}

// Modal accelerations of one FP64 stage (the arithmetic of accel<double>),
// also returning the gap d and its rate d'.
template <int M, int FORCE>
__device__ __forceinline__ void accel64(const KConst<double>& K, const Coef<double>& c,
                                        const double* q, const double* v, double g, double* a,
                                        double& d, double& dd) {
    double u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u += q[i];
    dd = 0.0;
    if (UsesRate<FORCE>::value) {
        dd = v[0];
#pragma unroll
        for (int i = 1; i < M; ++i) dd += v[i];
    }
    d = K.Zc + u;
    const double F = tip_force<FORCE, double>(c, d, dd);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        double ai = fma(-K.wq[i], v[i], K.gam[i] * g);
        ai = fma(-K.w2[i], q[i], ai);
        a[i] = (M <= 4) ? ai + F : fma(K.tip[i], F, ai);   // tip 0: padding modes
    }
}

// One FP64 RK4 step (the stage pattern of rk4_step, uncompensated: FP64
// needs no compensation over a segment).  REC: the force slopes of each stage
// go to rec[k * 32], k = 2 * stage (+1 for the rate slope).
template <int M, int FORCE, bool REC>
__device__ __forceinline__ void step64(const KConst<double>& K, const Coef<double>& c,
                                       const Coef<float>& cf, double* q, double* v, double g0,
                                       double gh, double g1, float* rec) {
    double a[M], qs[M], vs[M], Kq[M], Kv[M], d, dd;
    auto slope = [&](int st) {
        if (REC) {
            float Fd, Fr, Fc[4];
            force_partials<FORCE>(cf, (float)d, (float)dd, Fd, Fr, Fc);
            rec[(2 * st) * 32] = Fd;
            rec[(2 * st + 1) * 32] = Fr;
        }
    };
    accel64<M, FORCE>(K, c, q, v, g0, a, d, dd);
    slope(0);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = v[i];
        Kv[i] = a[i];
        qs[i] = fma(3.0, v[i], q[i]);
        vs[i] = fma(3.0, a[i], v[i]);
    }
    accel64<M, FORCE>(K, c, qs, vs, gh, a, d, dd);
    slope(1);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fma(2.0, vs[i], Kq[i]);
        Kv[i] = fma(2.0, a[i], Kv[i]);
        qs[i] = fma(3.0, vs[i], q[i]);
        vs[i] = fma(3.0, a[i], v[i]);
    }
    accel64<M, FORCE>(K, c, qs, vs, gh, a, d, dd);
    slope(2);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fma(2.0, vs[i], Kq[i]);
        Kv[i] = fma(2.0, a[i], Kv[i]);
        qs[i] = fma(6.0, vs[i], q[i]);
        vs[i] = fma(6.0, a[i], v[i]);
    }
    accel64<M, FORCE>(K, c, qs, vs, g1, a, d, dd);
    slope(3);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        q[i] = q[i] + (Kq[i] + vs[i]);
        v[i] = v[i] + (Kv[i] + a[i]);
    }
}

// Linearised stage: da = dA/d(q, v) . (dq, dv) with the recorded slopes.
template <int M, int FORCE>
__device__ __forceinline__ void jvp_stage(const float* w2, const float* wq, const float* tip,
                                          const float* rec, int st, const float* dq,
                                          const float* dv, float* da) {
    float su = dq[0];
#pragma unroll
    for (int i = 1; i < M; ++i) su += dq[i];
    float dF = rec[(2 * st) * 32] * su;
    if (UsesRate<FORCE>::value) {
        float sv = dv[0];
#pragma unroll
        for (int i = 1; i < M; ++i) sv += dv[i];
        dF = fmaf(rec[(2 * st + 1) * 32], sv, dF);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float base = fmaf(-wq[i], dv[i], -w2[i] * dq[i]);
        da[i] = (M <= 4) ? base + dF : fmaf(tip[i], dF, base);
    }
}

// The RK4 step of step64 linearised about its recorded stages, applied to one
// tangent direction (dq, dv) in place.
template <int M, int FORCE>
__device__ __forceinline__ void jvp_step(const float* w2, const float* wq, const float* tip,
                                         const float* rec, float* dq, float* dv) {
    float a[M], qs[M], vs[M], Kq[M], Kv[M];
    jvp_stage<M, FORCE>(w2, wq, tip, rec, 0, dq, dv, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = dv[i];
        Kv[i] = a[i];
        qs[i] = fmaf(3.f, dv[i], dq[i]);
        vs[i] = fmaf(3.f, a[i], dv[i]);
    }
    jvp_stage<M, FORCE>(w2, wq, tip, rec, 1, qs, vs, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fmaf(2.f, vs[i], Kq[i]);
        Kv[i] = fmaf(2.f, a[i], Kv[i]);
        qs[i] = fmaf(3.f, vs[i], dq[i]);
        vs[i] = fmaf(3.f, a[i], dv[i]);
    }
    jvp_stage<M, FORCE>(w2, wq, tip, rec, 2, qs, vs, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fmaf(2.f, vs[i], Kq[i]);
        Kv[i] = fmaf(2.f, a[i], Kv[i]);
        qs[i] = fmaf(6.f, vs[i], dq[i]);
        vs[i] = fmaf(6.f, a[i], dv[i]);
    }
    jvp_stage<M, FORCE>(w2, wq, tip, rec, 3, qs, vs, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        dq[i] = dq[i] + (Kq[i] + vs[i]);
        dv[i] = dv[i] + (Kv[i] + a[i]);
    }
}

__device__ __forceinline__ Coef<double> winner_coef(const ReevalWinner& w) {
    Coef<double> c;
    c.c0 = w.c[0];
    c.c1 = w.c[1];
    c.c2 = w.c[2];
    c.c3 = w.c[3];
    return c;
}

}  // namespace reeval
}  // namespace afm
