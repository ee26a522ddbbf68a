// afm_device.cuh -- device building blocks of libafminv: the Philox stream,
// the tip-sample force laws, the parameter map and one classic RK4 step of
// the modal cantilever (Eq. 2 integrated as in Sec. 3.2), in scaled units
// (see afm_internal.h).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "afm_internal.h"
#include "afm_launch.h"

namespace afm {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two round multipliers, and the key
// advances by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t a = 0xD2511F53u, b = 0xCD9E8D57u;
        uint32_t lo_a = a * c.x, hi_a = __umulhi(a, c.x);
        uint32_t lo_b = b * c.z, hi_b = __umulhi(b, c.z);
        c = make_uint4(hi_b ^ c.y ^ k.x, lo_b, hi_a ^ c.w ^ k.y, lo_a);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                             uint32_t tag, uint32_t block) {
    return philox4x32_10(make_uint4(c0, c1, c2, (tag << 16) | block),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

__device__ __forceinline__ uint32_t word_of(uint4 w, int i) {
    return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

// 24-bit uniform on [0, 1): exact in float and double.
__device__ __forceinline__ float unif24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// Arithmetic that the compiler may not contract or reorder (Kahan sums).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

// Drive table g at the 2*spc half-step phases of one period plus a wrap entry.
template <typename T>
__device__ __forceinline__ void build_drive_table(const KConst<T>& K, T* tab) {
    for (int j = threadIdx.x; j <= K.spc2; j += blockDim.x) {
        int jj = j == K.spc2 ? 0 : j;
        double ph = 6.283185307179586476925 * (double)jj / (double)K.spc2 + K.drive_phase;
        tab[j] = (T)(K.drive_amp * sin(ph));
    }
}

// Normalised coordinates -> physical slots (SI) -> scaled force coefficients.
// Computed in double for every precision (once per particle and solve).
template <typename T, typename X>
__device__ __forceinline__ Coef<T> make_coef(const KConst<T>& K, const X* xd) {
    double th[AFM_MAXD];
#pragma unroll
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = K.fixed[s];
    for (int d = 0; d < K.D; ++d) {
        if (K.slot[d] >= AFM_MAXD) continue;   // base-motion slot (kern_drive.cu)
        double v = K.lo[d] + (double)xd[d] * K.span[d];
        v = K.logs[d] ? exp10(v) : v;
        th[K.slot[d]] = v;
    }
    const double rt = 3.1622776601683794e-5;  // 10^-4.5 = sqrt(1e-9)
    Coef<T> c;
    c.c0 = c.c1 = c.c2 = c.c3 = (T)0;
    switch (K.force) {
        case F_LINEAR:
            c.c0 = (T)(th[0] / K.k * K.s1);
            c.c1 = (T)(th[1] * 1e9);
            break;
        case F_DMT:
        case F_DMT_KV: {
            double sR = sqrt(th[2]);
            c.c0 = (T)((4.0 / 3.0) * th[0] * sR * rt / K.k * K.s1);
            c.c1 = (T)(th[1] * th[2] / (6e-27 * K.k) * K.s1);
            c.c2 = (T)(th[4] * sR * rt * K.s1 / (K.k * K.tau));
            c.c3 = (T)(th[3] * 1e9);
            break;
        }
        case F_HOOKE:
            c.c0 = (T)(th[0] / K.k * K.s1);
            c.c1 = (T)(th[1] * 1e9);
            break;
        case F_SPRING_DAMPER:
            c.c0 = (T)(th[0] / K.k * K.s1);
            c.c1 = (T)(th[1] * 1e9);
            c.c2 = (T)(th[2] * K.s1 / (K.k * K.tau));
            break;
    }
    return c;
}

template <int FORCE>
struct UsesRate {
    static constexpr bool value = FORCE == F_DMT_KV || FORCE == F_SPRING_DAMPER;
};

// Tip-sample force in scaled units; branch-free for the DMT family: the van
// der Waals term saturates at d = a0, where it equals the Hertz branch's
// constant -HR/(6 a0^2), so one expression covers both branches.
template <int FORCE, typename T>
__device__ __forceinline__ T tip_force(const Coef<T>& c, T d, T dd) {
    if (FORCE == F_LINEAR) {
        return -c.c0 * (d - c.c1);
    } else if (FORCE == F_DMT || FORCE == F_DMT_KV) {
        T dm = fmax(d, c.c3);
        T r = rcp_fast(dm);
        T fv = c.c1 * (r * r);
        T del = fmax(c.c3 - d, (T)0);
        T sq = sqrt_fast(del);
        // nvcc contracts this to fma(c0, del * sq, -fv), the form the paired
        // step of afm_f32x2.cuh writes out (the batch tests compare the two
        // bit for bit); written out here as well it schedules ~1.5 % slower
        // in the small-swarm kernels
        T F = c.c0 * (del * sq) - fv;
        if (FORCE == F_DMT_KV) F = F - c.c2 * (sq * dd);
        return F;
    } else if (FORCE == F_HOOKE) {
        return c.c0 * fmax(c.c1 - d, (T)0);
    } else {
        return d < c.c1 ? c.c0 * (c.c1 - d) - c.c2 * dd : (T)0;
    }
}

// Partial derivatives of the tip force with respect to the gap (Fd), the gap
// rate (Fr) and the four coefficients (Fc[0..3]) at (d, d').  Reciprocals and
// square roots use the hardware approximations of tip_force (a relative
// error of a few FP32 ulps, far below the tangents' own rounding).
template <int FORCE>
__device__ __forceinline__ void force_partials(const Coef<float>& c, float d, float dd, float& Fd,
                                               float& Fr, float* Fc) {
    Fc[0] = Fc[1] = Fc[2] = Fc[3] = 0.f;
    Fd = Fr = 0.f;
    if (FORCE == F_LINEAR) {
        Fd = -c.c0;
        Fc[0] = -(d - c.c1);
        Fc[1] = c.c0;
    } else if (FORCE == F_DMT || FORCE == F_DMT_KV) {
        const bool contact = d < c.c3;
        const float dm = fmaxf(d, c.c3);
        const float r = rcp_fast(dm);
        const float r2 = r * r;
        Fc[1] = -r2;
        if (contact) {
            const float del = c.c3 - d;
            const float sq = sqrt_fast(del);
            const float isq = rcp_fast(sq);
            Fd = -1.5f * c.c0 * sq;
            Fc[0] = del * sq;
            Fc[3] = 1.5f * c.c0 * sq + 2.f * c.c1 * r2 * r;
            if (FORCE == F_DMT_KV) {
                Fd += 0.5f * c.c2 * dd * isq;
                Fr = -c.c2 * sq;
                Fc[2] = -sq * dd;
                Fc[3] -= 0.5f * c.c2 * dd * isq;
            }
        } else {
            Fd = 2.f * c.c1 * r2 * r;
        }
    } else if (FORCE == F_HOOKE) {
        if (d < c.c1) {
            Fd = -c.c0;
            Fc[0] = c.c1 - d;
            Fc[1] = c.c0;
        }
    } else {
        if (d < c.c1) {
            Fd = -c.c0;
            Fr = -c.c2;
            Fc[0] = c.c1 - d;
            Fc[1] = c.c0;
            Fc[2] = -dd;
        }
    }
}

// d c_k / d x_d (double) of the coefficient map in make_coef.
template <typename X>
__device__ __forceinline__ void coef_jacobian(const KConst<float>& K, const X* xd, double J[4][AFM_MAXD]) {
    double th[AFM_MAXD], dth[AFM_MAXD];
    int slot_of_dim[AFM_MAXD];
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = K.fixed[s];
    for (int d = 0; d < K.D; ++d) {
        double v = K.lo[d] + (double)xd[d] * K.span[d];
        if (K.logs[d]) {
            v = exp10(v);
            dth[d] = v * 2.302585092994045684 * K.span[d];
        } else {
            dth[d] = K.span[d];
        }
        th[K.slot[d]] = v;
        slot_of_dim[d] = K.slot[d];
    }
    double dc[4][AFM_MAXD];   // d c_k / d theta_s
    for (int k = 0; k < 4; ++k)
        for (int s = 0; s < AFM_MAXD; ++s) dc[k][s] = 0.0;
    const double rt = 3.1622776601683794e-5;
    switch (K.force) {
        case F_LINEAR:
        case F_HOOKE:
            dc[0][0] = K.s1 / K.k;
            dc[1][1] = 1e9;
            break;
        case F_SPRING_DAMPER:
            dc[0][0] = K.s1 / K.k;
            dc[1][1] = 1e9;
            dc[2][2] = K.s1 / (K.k * K.tau);
            break;
        case F_DMT:
        case F_DMT_KV: {
            const double sR = sqrt(th[2]);
            const double A = (4.0 / 3.0) * rt / K.k * K.s1;
            const double B = K.s1 / (6e-27 * K.k);
            const double C = rt * K.s1 / (K.k * K.tau);
            dc[0][0] = A * sR;
            dc[0][2] = A * th[0] / (2.0 * sR);
            dc[1][1] = B * th[2];
            dc[1][2] = B * th[1];
            dc[2][4] = C * sR;
            dc[2][2] = C * th[4] / (2.0 * sR);
            dc[3][3] = 1e9;
            break;
        }
    }
    for (int k = 0; k < 4; ++k)
        for (int d = 0; d < AFM_MAXD; ++d)
            J[k][d] = d < K.D ? dc[k][slot_of_dim[d]] * dth[d] : 0.0;
}

// Modal accelerations (Eq. 2): a_i = tip_i F + gamma_i g - w2_i q_i - wq_i q_i'.
// Mode 0's stiffness carries a low word (w2lo) so that the resonant mode's
// frequency is represented to ~1e-15 in FP32 arithmetic.
template <typename T, int M, int FORCE>
__device__ __forceinline__ void accel(const KConst<T>& K, const Coef<T>& c, const T* q, const T* v,
                                      T g, T* a) {
    T u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u += q[i];
    T dd = (T)0;
    if (UsesRate<FORCE>::value) {
        dd = v[0];
#pragma unroll
        for (int i = 1; i < M; ++i) dd += v[i];
    }
    T F = tip_force<FORCE, T>(c, K.Zc + u, dd);
    // The force-independent part first, so that F enters each mode's
    // acceleration through one final operation (shorter dependency chain).
#pragma unroll
    for (int i = 0; i < M; ++i) {
        T ai = fma(-K.wq[i], v[i], K.gam[i] * g);
        if (i == 0) ai = fma(-K.w2lo[0], q[0], ai);
        ai = fma(-K.w2[i], q[i], ai);
        // add_rn: no contraction with a product inside F (laws whose force
        // ends in a product), so every kernel rounds this sum the same way
        a[i] = (M <= 4) ? add_rn(ai, F) : fma(K.tip[i], F, ai);
    }
}

// Kahan-compensated x += inc.
template <typename T>
__device__ __forceinline__ void kahan_add(T& x, T& c, T inc) {
    T y = sub_rn(inc, c);
    T t = add_rn(x, y);
    c = sub_rn(sub_rn(t, x), y);
    x = t;
}

// The state update of mode i: compensated or plain by comp_mode.  The plain
// sum is the compensated one entered with c == 0 (y = inc exactly), which is
// how kernels holding one mode per lane run it: every lane the compensated
// form, then c masked to zero (bitwise, by the run-time KConst::cmask) where
// the lane's mode takes plain sums.  ALL: every mode compensated (the
// adjoint, whose gradient is more sensitive to the trajectory's rounding
// than the misfit is).
template <typename T, bool ALL = false>
__device__ __forceinline__ void state_add(int i, T& x, T& c, T inc) {
    if (ALL || comp_mode<T>(i))
        kahan_add(x, c, inc);
    else
        x = add_rn(x, inc);
}

// One classic RK4 step (h = 6, h/2 = 3, h/6 = 1 in scaled time) with
// compensated state update (state_add).  g0, gh, g1: drive at t, t + h/2,
// t + h.
template <typename T, int M, int FORCE, bool ALLC = false>
__device__ __forceinline__ void rk4_step(const KConst<T>& K, const Coef<T>& c, T* q, T* v, T* cq,
                                         T* cv, T g0, T gh, T g1) {
    T a[M], qs[M], vs[M], Kq[M], Kv[M];
    accel<T, M, FORCE>(K, c, q, v, g0, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = v[i];
        Kv[i] = a[i];
        qs[i] = fma((T)3, v[i], q[i]);
        vs[i] = fma((T)3, a[i], v[i]);
    }
    accel<T, M, FORCE>(K, c, qs, vs, gh, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fma((T)2, vs[i], Kq[i]);
        Kv[i] = fma((T)2, a[i], Kv[i]);
        qs[i] = fma((T)3, vs[i], q[i]);
        vs[i] = fma((T)3, a[i], v[i]);
    }
    accel<T, M, FORCE>(K, c, qs, vs, gh, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fma((T)2, vs[i], Kq[i]);
        Kv[i] = fma((T)2, a[i], Kv[i]);
        qs[i] = fma((T)6, vs[i], q[i]);
        vs[i] = fma((T)6, a[i], v[i]);
    }
    accel<T, M, FORCE>(K, c, qs, vs, g1, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = Kq[i] + vs[i];
        Kv[i] = Kv[i] + a[i];
        state_add<T, ALLC>(i, q[i], cq[i], Kq[i]);
        state_add<T, ALLC>(i, v[i], cv[i], Kv[i]);
    }
}

template <typename T, int M>
__device__ __forceinline__ void init_state(const KConst<T>& K, T* q, T* v, T* cq, T* cv) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
        q[i] = K.q0[i];
        v[i] = K.v0[i];
        cq[i] = (T)0;
        cv[i] = (T)0;
    }
}

template <typename T, int M>
__device__ __forceinline__ T tip_sum(const T* q) {
    T u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u += q[i];
    return u;
}

// Forward solve of one particle over n steps, fused with the compensated
// misfit sum of Eq. 5 (U != nullptr) and the optional time-major output.
template <typename T, int M, int FORCE, typename TU = T>
__device__ __forceinline__ T integrate(const KConst<T>& K, const Coef<T>& c, const T* tab,
                                       const TU* __restrict__ U, T* __restrict__ defl, int P, int p,
                                       int n) {
    T q[M], v[M], cq[M], cv[M];
    init_state<T, M>(K, q, v, cq, cv);
    T S = (T)0, cS = (T)0;
    int j = 0;
    const int spc2 = K.spc2;
    T Un = (U != nullptr && n > 0) ? (T)U[0] : (T)0;
    for (int s = 0; s < n; ++s) {
        T g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        T Unext = (U != nullptr && s + 1 < n) ? (T)U[s + 1] : (T)0;
        rk4_step<T, M, FORCE>(K, c, q, v, cq, cv, g0, gh, g1);
        T u = tip_sum<T, M>(q);
        if (defl != nullptr) defl[(size_t)s * P + p] = u;
        if (U != nullptr) {
            T r = Un - u;
            T y = fma(r, r, -cS);
            T t = add_rn(S, y);
            cS = sub_rn(sub_rn(t, S), y);
            S = t;
        }
        Un = Unext;
    }
    return S;
}

// integrate() with the misfit over K.np deflection points per step (K.phi:
// tip-normalised mode shapes at the points);
// U is [n][np] (step-major), defl [n][np][P].
template <typename T, int M, int FORCE, typename TU = T>
__device__ __forceinline__ T integrate_points(const KConst<T>& K, const Coef<T>& c, const T* tab,
                                              const TU* __restrict__ U, T* __restrict__ defl,
                                              int P, int p, int n) {
    T q[M], v[M], cq[M], cv[M];
    init_state<T, M>(K, q, v, cq, cv);
    T S = (T)0, cS = (T)0;
    int j = 0;
    const int spc2 = K.spc2, np = K.np;
    // the record values of step s are loaded during step s - 1, so that no
    // step waits for a global-memory load
    T Ucur[AFM_MAX_POINTS];
#pragma unroll
    for (int k = 0; k < AFM_MAX_POINTS; ++k)
        Ucur[k] = (U != nullptr && n > 0 && k < np) ? (T)U[k] : (T)0;
    for (int s = 0; s < n; ++s) {
        const T g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        T Unext[AFM_MAX_POINTS];
#pragma unroll
        for (int k = 0; k < AFM_MAX_POINTS; ++k)
            Unext[k] = (U != nullptr && s + 1 < n && k < np) ? (T)U[(size_t)(s + 1) * np + k] : (T)0;
        rk4_step<T, M, FORCE>(K, c, q, v, cq, cv, g0, gh, g1);
        // unrolled to the largest point count (a uniform guard), so that the
        // point deflections schedule alongside the step's arithmetic
#pragma unroll
        for (int k = 0; k < AFM_MAX_POINTS; ++k) {
            if (k < np) {
                T uk = K.phi[k][0] * q[0];
#pragma unroll
                for (int i = 1; i < M; ++i) uk = fma(K.phi[k][i], q[i], uk);
                const size_t idx = (size_t)s * np + k;
                if (defl != nullptr) defl[idx * P + p] = uk;
                if (U != nullptr) {
                    const T r = Ucur[k] - uk;
                    const T y = fma(r, r, -cS);
                    const T t = add_rn(S, y);
                    cS = sub_rn(sub_rn(t, S), y);
                    S = t;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < AFM_MAX_POINTS; ++k) Ucur[k] = Unext[k];
    }
    return S;
}

// K particles per thread sharing the record and drive loads: the K
// independent RK4 recurrences interleave in one instruction stream, which
// hides the dependency latency of each.  Arithmetic per particle is the same
// as integrate() (misfit only).
template <int M, int FORCE, int K>
__device__ __forceinline__ void integrate_multi(const KConst<float>& Kc, const Coef<float>* c,
                                                const float* tab, const float* __restrict__ U,
                                                int n, float* S_out) {
    float q[K][M], v[K][M], cq[K][M], cv[K][M];
    float S[K], cS[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        init_state<float, M>(Kc, q[k], v[k], cq[k], cv[k]);
        S[k] = 0.f;
        cS[k] = 0.f;
    }
    int j = 0;
    const int spc2 = Kc.spc2;
    float Un = n > 0 ? U[0] : 0.f;
    for (int s = 0; s < n; ++s) {
        float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        float Unext = s + 1 < n ? U[s + 1] : 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            rk4_step<float, M, FORCE>(Kc, c[k], q[k], v[k], cq[k], cv[k], g0, gh, g1);
            float u = tip_sum<float, M>(q[k]);
            float r = Un - u;
            float y = fmaf(r, r, -cS[k]);
            float t = add_rn(S[k], y);
            cS[k] = sub_rn(sub_rn(t, S[k]), y);
            S[k] = t;
        }
        Un = Unext;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) S_out[k] = S[k];
}

// Eq. 8 for particle p at iteration it (>= 1): r1, r2 per dimension are words
// 2d and 2d+1 (mod 4) of counter (p, it, pixel, 2<<16 | d/2).
__device__ __forceinline__ void pso_move_dev(const PsoConst& pc, float* x, float* v, const float* pb,
                                         const float* gb, int p, int it) {
    uint4 w = make_uint4(0, 0, 0, 0);
    for (int d = 0; d < pc.D; ++d) {
        if ((d & 1) == 0) w = philox_draw(pc.seed, (uint32_t)p, (uint32_t)it, pc.pixel, 2u, (uint32_t)(d >> 1));
        const int k = (2 * d) & 3;
        const float r1 = unif24(word_of(w, k)), r2 = unif24(word_of(w, k + 1));
        // explicit FMAs: the same rounding wherever this is inlined
        float vn = fmaf(pc.c2 * r2, gb[d] - x[d], fmaf(pc.c1 * r1, pb[d] - x[d], pc.w * v[d]));
        float xn = x[d] + vn;
        if (xn < 0.f) { xn = 0.f; vn = 0.f; }
        if (xn > 1.f) { xn = 1.f; vn = 0.f; }
        x[d] = xn;
        v[d] = vn;
    }
}


}  // namespace afm
