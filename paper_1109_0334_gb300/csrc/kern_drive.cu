// kern_drive.cu -- base-motion inversion (Sec. 4.1): the base moves as
// y_b = a sin(2 pi (f t + g t^2)) with (a, f, g) per particle, free or
// fixed, and the cantilever starts at rest.  There is no shared drive table:
// each thread evaluates its particle's drive g = -y_b'' at every half step
// from a phase kept in 64-bit fixed-point turns, so the reduction modulo one
// turn is exact however long the record.  The time stepping, misfit and
// swarm arithmetic are those of the steady-drive kernels (rk4_step,
// compensated sums, pso_move_dev).
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

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

// Per-particle base motion in scaled units (time tau = h/6, half step = 3 tau).
template <typename T>
struct DriveCoef {
    T A;                       // amplitude [nm]
    T w0, w1;                  // phi' tau = w0 + w1 j at half step j
    unsigned long long F, G;   // turns per half step and per (half step)^2, x 2^64
};

// Fraction of x (any sign) as unsigned 64-bit fixed point in [0, 2^64).
__device__ __forceinline__ unsigned long long frac_u64(double x) {
    const double fr = x - floor(x);
    const double v = fr * 18446744073709551616.0;
    return v >= 18446744073709551616.0 ? 0ull : __double2ull_rz(v);
}

template <typename T, typename X>
__device__ __forceinline__ DriveCoef<T> make_drive(const KConst<T>& K, const X* xd) {
    double dr[3] = {K.drv[0], K.drv[1], K.drv[2]};
    for (int d = 0; d < K.D; ++d) {
        const int s = K.slot[d];
        if (s < AFM_MAXD) continue;
        const double v = K.lo[d] + (double)xd[d] * K.span[d];
        dr[s - AFM_MAXD] = K.logs[d] ? exp10(v) : v;
    }
    const double tau = K.tau, pi = 3.14159265358979323846;
    DriveCoef<T> c;
    c.A = (T)(dr[0] * 1e9);
    c.w0 = (T)(2.0 * pi * dr[1] * tau);
    c.w1 = (T)(12.0 * pi * dr[2] * tau * tau);
    c.F = frac_u64(dr[1] * 3.0 * tau);
    c.G = frac_u64(dr[2] * 9.0 * tau * tau);
    return c;
}

// g = -y_b'' = A (phi'^2 sin phi - phi'' cos phi) at half step j, phi in
// turns = j F + j^2 G (modulo 1), phi'' tau^2 = w1 / 3.
template <typename T>
__device__ __forceinline__ T drive_at(const DriveCoef<T>& c, long long j) {
    const unsigned long long uj = (unsigned long long)j;
    const unsigned long long q = uj * c.F + uj * uj * c.G;   // modulo 2^64
    T s, co;
    if (sizeof(T) == 4) {
        // top 32 bits as a signed fraction of a turn in [-1/2, 1/2)
        const float t = (float)(int)(unsigned)(q >> 32) * 2.3283064365386963e-10f;
        float sf, cf;
        sincospif(2.f * t, &sf, &cf);
        s = (T)sf;
        co = (T)cf;
    } else {
        const double t = (double)(long long)q * 5.4210108624275222e-20;
        double sd, cd;
        sincospi(2.0 * t, &sd, &cd);
        s = (T)sd;
        co = (T)cd;
    }
    const T wp = fma(c.w1, (T)j, c.w0);
    return c.A * (wp * wp * s - (c.w1 / (T)3) * co);
}

// integrate() of afm_device.cuh with the particle's own drive, from rest.
template <typename T, int M, int FORCE, typename TU = T>
__device__ __forceinline__ T integrate_drive(const KConst<T>& K, const Coef<T>& c,
                                             const DriveCoef<T>& dc, const TU* __restrict__ U,
                                             T* __restrict__ defl, int P, int p, int n) {
    T q[M], v[M], cq[M], cv[M];
    init_state<T, M>(K, q, v, cq, cv);
    T S = (T)0, cS = (T)0;
    T g1 = drive_at<T>(dc, 0);
    T Un = (U != nullptr && n > 0) ? (T)U[0] : (T)0;
    for (int s = 0; s < n; ++s) {
        const T g0 = g1;
        const T gh = drive_at<T>(dc, 2ll * s + 1);
        g1 = drive_at<T>(dc, 2ll * s + 2);
        const T Unext = (U != nullptr && s + 1 < n) ? (T)U[s + 1] : (T)0;
        rk4_step<T, M, FORCE>(K, c, q, v, cq, cv, g0, gh, g1);
        const T u = tip_sum<T, M>(q);
        if (defl != nullptr) defl[(size_t)s * P + p] = u;
        if (U != nullptr) {
            const T r = Un - u;
            const T y = fma(r, r, -cS);
            const T t = add_rn(S, y);
            cS = sub_rn(sub_rn(t, S), y);
            S = t;
        }
        Un = Unext;
    }
    return S;
}

__device__ __forceinline__ unsigned long long drive_key(float S, int p) {
    return ((unsigned long long)__float_as_uint(S) << 32) | (unsigned)p;
}

}  // namespace

template <typename T, int M, int FORCE>
__global__ void fwd_drive_kernel(const KConst<T> K, const T* __restrict__ x, int P,
                                 T* __restrict__ defl, const T* __restrict__ U,
                                 T* __restrict__ S) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    T xd[AFM_MAXD];
    for (int d = 0; d < K.D; ++d) xd[d] = x[(size_t)d * P + p];
    const Coef<T> c = make_coef<T, T>(K, xd);
    const DriveCoef<T> dc = make_drive<T, T>(K, xd);
    T s = integrate_drive<T, M, FORCE>(K, c, dc, U, defl, P, p, K.n_steps);
    if (S != nullptr) S[p] = (s < (T)INFINITY) ? s : (T)INFINITY;
}

// invert_iter_kernel of kern_invert.cu with the particle's own drive.
template <int M, int FORCE>
__global__ void invert_drive_kernel(const KConst<float> K, const PsoConst pc, SwarmPtrs sw,
                                    const float* __restrict__ U, float* __restrict__ history,
                                    int it) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int rd = it & 1, wr = (it + 1) & 1;
    const float* pb_rd = sw.pb[rd];
    float* pb_wr = sw.pb[wr];
    unsigned long long key = ~0ull;
    if (it > 0 && p == 0 && history != nullptr)
        history[it - 1] = __uint_as_float((uint32_t)(*sw.gkey[rd] >> 32));
    if (p < pc.P) {
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
            for (int d = 0; d < pc.D; ++d) {
                sw.x[(size_t)d * pc.P + p] = x[d];
                sw.v[(size_t)d * pc.P + p] = v[d];
            }
        }
        const Coef<float> c = make_coef<float, float>(K, x);
        const DriveCoef<float> dc = make_drive<float, float>(K, x);
        float s = integrate_drive<float, M, FORCE>(K, c, dc, U, nullptr, 0, p, K.n_steps);
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
        key = drive_key(best, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(sw.gkey[wr], key);
}

// FP64 re-evaluation of the winner (one thread) and the result record.
template <int M, int FORCE>
__global__ void drive_final_kernel(const KConst<double> K, const PsoConst pc, SwarmPtrs sw,
                                   const float* __restrict__ U, float* __restrict__ history,
                                   afm_result* __restrict__ res) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int n = threadIdx.x; n < K.n_steps; n += blockDim.x) acc += (double)U[n] * (double)U[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const int fin = (pc.iters + 1) & 1;
    const unsigned long long key = *sw.gkey[fin];
    const int g = min((int)(key & 0x7fffffffu), pc.P - 1);
    const float S32 = __uint_as_float((uint32_t)(key >> 32));
    if (history != nullptr) history[pc.iters] = S32;
    double xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < pc.D ? (double)sw.pb[fin][(size_t)d * pc.P + g] : 0.0;
    const Coef<double> c = make_coef<double, double>(K, xd);
    const DriveCoef<double> dc = make_drive<double, double>(K, xd);
    const double S64 = integrate_drive<double, M, FORCE, float>(K, c, dc, U, nullptr, 0, 0, K.n_steps);
    double th[AFM_MAXD], dr[3] = {K.drv[0], K.drv[1], K.drv[2]};
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = K.fixed[s];
    for (int d = 0; d < K.D; ++d) {
        const double v = K.lo[d] + xd[d] * K.span[d];
        const double val = K.logs[d] ? exp10(v) : v;
        if (K.slot[d] < AFM_MAXD)
            th[K.slot[d]] = val;
        else
            dr[K.slot[d] - AFM_MAXD] = val;
    }
    for (int d = 0; d < AFM_MAXD; ++d) {
        res->x[d] = xd[d];
        res->theta[d] = th[d];
    }
    for (int k = 0; k < 3; ++k) res->drive[k] = dr[k];
    res->S = (double)S32;
    res->S_f64 = S64;
    res->J_rel = red[0] > 0.0 ? sqrt(S64 / red[0]) : 0.0;
    res->iters = pc.iters;
    res->winner = g;
    res->nonfinite = sw.flags ? sw.flags[0] : 0;
    res->status = (isfinite(S64) && res->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
    res->defect = 0.0;
    res->segments = 0;
    res->reserved = 0;
}

cudaError_t launch_forward_drive_f32(const KConst<float>& K, const float* x, int P, float* defl,
                                     const float* U, float* S, cudaStream_t st) {
    const int threads = P <= 152 * 32 * 4 ? 32 : 128;
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        fwd_drive_kernel<float, decltype(Mc)::value, decltype(Fc)::value>
            <<<(P + threads - 1) / threads, threads, 0, st>>>(K, x, P, defl, U, S);
        return cudaGetLastError();
    });
}

cudaError_t launch_forward_drive_f64(const KConst<double>& K, const double* x, int P, double* defl,
                                     const double* U, double* S, cudaStream_t st) {
    const int threads = P <= 152 * 32 * 4 ? 32 : 128;
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        fwd_drive_kernel<double, decltype(Mc)::value, decltype(Fc)::value>
            <<<(P + threads - 1) / threads, threads, 0, st>>>(K, x, P, defl, U, S);
        return cudaGetLastError();
    });
}

cudaError_t launch_invert_drive(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, int it, cudaStream_t st) {
    const int threads = pc.P <= 152 * 32 * 4 ? 32 : 128;
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        invert_drive_kernel<decltype(Mc)::value, decltype(Fc)::value>
            <<<(pc.P + threads - 1) / threads, threads, 0, st>>>(K, pc, sw, U, history, it);
        return cudaGetLastError();
    });
}

cudaError_t launch_drive_final(const KConst<double>& K, const PsoConst& pc, const SwarmPtrs& sw,
                               const float* U, float* history, void* result, cudaStream_t st) {
    return dispatch_mf(K.m, K.force, [&](auto Mc, auto Fc) -> cudaError_t {
        drive_final_kernel<decltype(Mc)::value, decltype(Fc)::value><<<1, 256, 0, st>>>(
            K, pc, sw, U, history, reinterpret_cast<afm_result*>(result));
        return cudaGetLastError();
    });
}

}  // namespace afm
