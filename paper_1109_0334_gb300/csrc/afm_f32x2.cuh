// afm_f32x2.cuh -- two particles per instruction: the RK4 step of
// afm_device.cuh (Eq. 2 integrated as in Sec. 3.2) and the compensated
// misfit of Eq. 5 on pairs of FP32 values, with sm_100-family paired
// instructions (add/mul/fma .f32x2: each half rounded as the scalar
// operation).  A thread that carries several particles (the batched-pixel
// kernel's KP) issues one paired instruction where it issued two scalar
// ones.  Every operation is the scalar step's, in the same order and with the
// same rounding (x - y as x + (-y), which IEEE rounds identically), so each
// particle's result is bit-identical to integrate_multi / rk4_step (the one
// expression of the scalar step that nvcc contracts, in the DMT law, is
// written here in its contracted form; tests compare the two bit for bit).
// The DMT law only (the laws of the batched workloads; each other law would
// need its own check of the compiler's contractions), up to 4 modes (the
// add_rn force term of accel).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "afm_device.cuh"

namespace afm {
namespace x2 {

__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, neg(b)); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }

template <int FORCE>
struct Supported {
    static constexpr bool value = FORCE == F_DMT;
};

// Per-mode constants of accel, negated where accel negates them (the drive
// factors gam stay scalar: gam g is the same for both particles).
template <int M>
struct ModeC {
    float2 nwq[M], nw2[M], nw2lo, Zc;
    float gam[M];
};

template <int M>
__device__ __forceinline__ ModeC<M> mode_consts(const KConst<float>& K) {
    ModeC<M> C;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        C.nwq[i] = bc(-K.wq[i]);
        C.gam[i] = K.gam[i];
        C.nw2[i] = bc(-K.w2[i]);
    }
    C.nw2lo = bc(-K.w2lo[0]);
    C.Zc = bc(K.Zc);
    return C;
}

// The force coefficients of two particles.
struct Coef2 {
    float2 c0, c1, c3;
};

// tip_force<F_DMT> on a pair: min/max, reciprocal and square root per half.
__device__ __forceinline__ float2 dmt_force(const Coef2& c, float2 d) {
    const float2 dm = make_float2(fmaxf(d.x, c.c3.x), fmaxf(d.y, c.c3.y));
    const float2 r = make_float2(rcp_fast(dm.x), rcp_fast(dm.y));
    const float2 t = sub(c.c3, d);
    const float2 del = make_float2(fmaxf(t.x, 0.f), fmaxf(t.y, 0.f));
    const float2 sq = make_float2(sqrt_fast(del.x), sqrt_fast(del.y));
    // the contraction nvcc makes of the scalar law's c0 (del sq) - c1 r^2
    return fma(c.c0, mul(del, sq), neg(mul(c.c1, mul(r, r))));
}

template <int M>
__device__ __forceinline__ void accel(const ModeC<M>& C, const Coef2& c, const float2* q,
                                      const float2* v, float g, float2* a) {
    float2 u = q[0];
#pragma unroll
    for (int i = 1; i < M; ++i) u = add(u, q[i]);
    const float2 F = dmt_force(c, add(C.Zc, u));
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float2 ai = fma(C.nwq[i], v[i], bc(C.gam[i] * g));
        if (i == 0) ai = fma(C.nw2lo, q[0], ai);
        ai = fma(C.nw2[i], q[i], ai);
        a[i] = add(ai, F);
    }
}

__device__ __forceinline__ void kahan_add(float2& x, float2& c, float2 inc) {
    const float2 y = sub(inc, c);
    const float2 t = add(x, y);
    c = sub(sub(t, x), y);
    x = t;
}

template <int M>
__device__ __forceinline__ void rk4_step(const ModeC<M>& C, const Coef2& c, float2* q, float2* v,
                                         float2* cq, float2* cv, float g0, float gh, float g1) {
    const float2 two = bc(2.f), three = bc(3.f), six = bc(6.f);
    float2 a[M], qs[M], vs[M], Kq[M], Kv[M];
    accel<M>(C, c, q, v, g0, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = v[i];
        Kv[i] = a[i];
        qs[i] = fma(three, v[i], q[i]);
        vs[i] = fma(three, a[i], v[i]);
    }
    accel<M>(C, c, qs, vs, gh, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fma(two, vs[i], Kq[i]);
        Kv[i] = fma(two, a[i], Kv[i]);
        qs[i] = fma(three, vs[i], q[i]);
        vs[i] = fma(three, a[i], v[i]);
    }
    accel<M>(C, c, qs, vs, gh, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = fma(two, vs[i], Kq[i]);
        Kv[i] = fma(two, a[i], Kv[i]);
        qs[i] = fma(six, vs[i], q[i]);
        vs[i] = fma(six, a[i], v[i]);
    }
    accel<M>(C, c, qs, vs, g1, a);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Kq[i] = add(Kq[i], vs[i]);
        Kv[i] = add(Kv[i], a[i]);
        if (comp_mode<float>(i)) {   // as afm::state_add
            kahan_add(q[i], cq[i], Kq[i]);
            kahan_add(v[i], cv[i], Kv[i]);
        } else {
            q[i] = add(q[i], Kq[i]);
            v[i] = add(v[i], Kv[i]);
        }
    }
}

}  // namespace x2

// integrate_multi with the KP particles taken in KP / 2 pairs (KP even).
template <int M, int FORCE, int KP>
__device__ __forceinline__ void integrate_multi_x2(const KConst<float>& Kc, const Coef<float>* c,
                                                   const float* tab, const float* __restrict__ U,
                                                   int n, float* S_out) {
    static_assert(KP % 2 == 0 && M <= 4 && x2::Supported<FORCE>::value, "paired step");
    constexpr int NP = KP / 2;
    const x2::ModeC<M> C = x2::mode_consts<M>(Kc);
    x2::Coef2 cc[NP];
    float2 q[NP][M], v[NP][M], cq[NP][M], cv[NP][M];
    float2 S[NP], cS[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const Coef<float>& a = c[2 * k];
        const Coef<float>& b = c[2 * k + 1];
        cc[k].c0 = make_float2(a.c0, b.c0);
        cc[k].c1 = make_float2(a.c1, b.c1);
        cc[k].c3 = make_float2(a.c3, b.c3);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            q[k][i] = x2::bc(Kc.q0[i]);
            v[k][i] = x2::bc(Kc.v0[i]);
            cq[k][i] = x2::bc(0.f);
            cv[k][i] = x2::bc(0.f);
        }
        S[k] = x2::bc(0.f);
        cS[k] = x2::bc(0.f);
    }
    int j = 0;
    const int spc2 = Kc.spc2;
    float Un = n > 0 ? U[0] : 0.f;
    for (int s = 0; s < n; ++s) {
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        const float Unext = s + 1 < n ? U[s + 1] : 0.f;
        const float2 U2 = x2::bc(Un);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            x2::rk4_step<M>(C, cc[k], q[k], v[k], cq[k], cv[k], g0, gh, g1);
            float2 u = q[k][0];
#pragma unroll
            for (int i = 1; i < M; ++i) u = x2::add(u, q[k][i]);
            const float2 r = x2::sub(U2, u);
            const float2 y = x2::fma(r, r, x2::neg(cS[k]));
            const float2 t = x2::add(S[k], y);
            cS[k] = x2::sub(x2::sub(t, S[k]), y);
            S[k] = t;
        }
        Un = Unext;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        S_out[2 * k] = S[k].x;
        S_out[2 * k + 1] = S[k].y;
    }
}

// integrate() (FP32) for particles p0 and p1 of a pair: the misfit (U !=
// nullptr) and the time-major output (defl != nullptr; particle p1 only if
// has1, a pair that ends an odd-sized batch repeats p0 in its second half).
template <int M, int FORCE>
__device__ __forceinline__ float2 integrate_x2(const KConst<float>& K, const Coef<float>& ca,
                                               const Coef<float>& cb, const float* tab,
                                               const float* __restrict__ U,
                                               float* __restrict__ defl, int P, int p0, bool has1,
                                               int n) {
    static_assert(M <= 4 && x2::Supported<FORCE>::value, "paired step");
    const x2::ModeC<M> C = x2::mode_consts<M>(K);
    x2::Coef2 cc;
    cc.c0 = make_float2(ca.c0, cb.c0);
    cc.c1 = make_float2(ca.c1, cb.c1);
    cc.c3 = make_float2(ca.c3, cb.c3);
    float2 q[M], v[M], cq[M], cv[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        q[i] = x2::bc(K.q0[i]);
        v[i] = x2::bc(K.v0[i]);
        cq[i] = x2::bc(0.f);
        cv[i] = x2::bc(0.f);
    }
    float2 S = x2::bc(0.f), cS = x2::bc(0.f);
    int j = 0;
    const int spc2 = K.spc2;
    float Un = (U != nullptr && n > 0) ? U[0] : 0.f;
    for (int s = 0; s < n; ++s) {
        const float g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        const float Unext = (U != nullptr && s + 1 < n) ? U[s + 1] : 0.f;
        x2::rk4_step<M>(C, cc, q, v, cq, cv, g0, gh, g1);
        float2 u = q[0];
#pragma unroll
        for (int i = 1; i < M; ++i) u = x2::add(u, q[i]);
        if (defl != nullptr) {
            float* row = defl + (size_t)s * P + p0;
            if (has1 && (reinterpret_cast<uintptr_t>(row) & 7) == 0)
                *reinterpret_cast<float2*>(row) = u;
            else {
                row[0] = u.x;
                if (has1) row[1] = u.y;
            }
        }
        if (U != nullptr) {
            const float2 r = x2::sub(x2::bc(Un), u);
            const float2 y = x2::fma(r, r, x2::neg(cS));
            const float2 t = x2::add(S, y);
            cS = x2::sub(x2::sub(t, S), y);
            S = t;
        }
        Un = Unext;
    }
    return S;
}

}  // namespace afm
