// kern_fe.cu -- finite-element cantilever (cubic Hermite Euler-Bernoulli
// elements) advanced by Newmark's average-acceleration scheme (beta = 1/4,
// gamma = 1/2) with the tip-sample force solved implicitly at every step.
//
// The scheme runs in the M-orthonormal eigenbasis of the element model, in
// which the Rayleigh-damped system is diagonal, so that each step is one
// scalar recursion per mode plus the tip coupling (see afm_internal.h).  The
// recursion is the same as the physical-coordinate three-term form (it is
// that form, premultiplied by Phi^T), but it does not route the resonant
// mode through a propagator whose entries are dominated by the stiff element
// modes: applied densely in physical coordinates the 64 x 128 propagator has
// a condition number of ~3e4, which turns FP32 (and TF32) rounding into
// 1e-3 errors of the resonant response.
//
// Layout: AFM_FE_LANES lanes per particle, each lane owns modes
// lane, lane + 8, ... and holds their step coefficients in registers; the
// tip deflection is a group sum (3 shuffles), the Newton solve for the tip
// force runs redundantly in the group's lanes.
//
// The kernel carries each mode scaled by its tip displacement, w_i =
// phi_i(tip) z_i.  The recursion is linear and homogeneous in (z_i, delta_i),
// so w_i obeys it with g_i and f_i multiplied by phi_i(tip) and b1_i, d2_i
// unchanged, and the tip deflection is the plain sum of the w_i: one add per
// mode instead of a product, and no per-step fetch of phi_i(tip).
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

constexpr int FEN = AFM_FE_MAXN;
// 64 threads (8 particles in FP32) per block: a C5 swarm of 8 192 particles
// is 1 024 blocks, spread over 152 SMs within 4 % of even (256-thread blocks
// left 48 SMs with half the load of the others)
constexpr int FE_THREADS = 64;
constexpr int FE_MIN_BLOCKS = 8;   // caps registers at 128 per thread
// lanes per particle: AFM_FE_LANES in FP32 (throughput), a whole warp in FP64
// (latency: one trajectory, the FP64 re-evaluation)
template <typename T>
struct FeLanes {
    static constexpr int value = sizeof(T) == 8 ? 32 : AFM_FE_LANES;
};

// Which mode slots of a lane take compensated updates.  FP64: all.  FP32:
// slot 0 only, the lowest AFM_FE_LANES modes, which hold the resonant
// response and whose step increment is a small fraction of the coordinate
// (omega h << 1), so that plain sums lose its low bits every step.  The
// stiff modes above respond quasi-statically with amplitudes ~(omega_1 /
// omega_i)^2 of the first mode's forced term and omega h ~ 1: their rounding
// stays far below FP32 resolution of the tip deflection.
template <typename T>
__host__ __device__ constexpr bool fe_comp(int j) {
    return sizeof(T) == 8 || j == 0;
}

// Drive term of the Newmark step at phase index j of the period: the base
// acceleration enters as y(t+) + 2 y(t) + y(t-), evaluated in FP64.
template <typename T>
__device__ __forceinline__ void fe_table(const FeConst& F, T* tab) {
    const double w = 6.283185307179586476925 / (double)F.spc;
    for (int j = threadIdx.x; j < F.spc; j += blockDim.x) {
        const double y0 = sin(w * (double)j + F.drive_phase);
        const double yp = sin(w * (double)(j + 1) + F.drive_phase);
        const double ym = sin(w * (double)(j - 1) + F.drive_phase);
        tab[j] = (T)(F.drive_amp * (yp + 2.0 * y0 + ym));
    }
}

// Tip force and its slope in the gap (laws without rate dependence); the
// FP32 instantiation uses the hardware reciprocal and square root (sqrt_fast,
// rcp_fast resolve to the exact FP64 operations for double).
template <int FORCE, typename T>
__device__ __forceinline__ void fe_force(const Coef<T>& c, T d, T& Fv, T& dF) {
    if (FORCE == F_LINEAR) {
        Fv = -c.c0 * (d - c.c1);
        dF = -c.c0;
    } else if (FORCE == F_DMT) {
        // branch-free (the van der Waals term saturates at d = a0, where it
        // is the contact branch's constant): particles of one warp in and out
        // of contact follow one instruction stream
        const T r = rcp_fast(fmax(d, c.c3));
        const T r2 = r * r;
        const T del = fmax(c.c3 - d, (T)0), sq = sqrt_fast(del);
        Fv = c.c0 * del * sq - c.c1 * r2;
        dF = d > c.c3 ? (T)2 * c.c1 * r2 * r : (T)(-1.5) * c.c0 * sq;
    } else {   // HOOKE
        if (d < c.c1) {
            Fv = c.c0 * (c.c1 - d);
            dF = -c.c0;
        } else {
            Fv = (T)0;
            dF = (T)0;
        }
    }
}

// sum_j wp_j (the predicted tip deflection of a lane's mode slots) as a
// pairwise tree: a dependency chain of log2(N) adds instead of N.
template <typename T, int N>
__device__ __forceinline__ T fe_sum(const T* wp) {
    T s[N];
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = wp[k];
#pragma unroll
    for (int w = N; w > 1; w = (w + 1) / 2) {
#pragma unroll
        for (int k = 0; k < w / 2; ++k) s[k] = s[2 * k] + s[2 * k + 1];
        if (w % 2) s[w / 2] = s[w - 1];
    }
    return s[0];
}

// z = base + cz F(Zc + z) by Newton from z = base + cz Fguess.
template <int FORCE, typename T>
__device__ __forceinline__ T fe_newton(const Coef<T>& c, T Zc, T base, T cz, T Fguess, int iters,
                                       T& Fz) {
    T z = fma(cz, Fguess, base), dF;
    for (int it = 0; it < iters; ++it) {
        fe_force<FORCE, T>(c, Zc + z, Fz, dF);
        const T phi = z - base - cz * Fz;
        z = z - phi * rcp_fast((T)1 - cz * dF);
    }
    fe_force<FORCE, T>(c, Zc + z, Fz, dF);
    return z;
}

// ---------------------------------------------------------------------------
// MODE 0: forward (defl, S) for P particles; MODE 1: one fused inversion
// iteration (PSO move, forward, personal/global best; T = float);
// MODE 2: FP64 re-evaluation of an inversion's winner into afm_result.
// ---------------------------------------------------------------------------
template <typename T, typename TU, int FORCE, int MODE>
__global__ void __launch_bounds__(FE_THREADS, FE_MIN_BLOCKS) fe_modal_kernel(
    const FeConst F, const PsoConst pc, SwarmPtrs sw, const T* __restrict__ xin, int P,
    T* __restrict__ defl, const TU* __restrict__ U, T* __restrict__ S_out,
    float* __restrict__ history, int it, afm_result* __restrict__ res) {
    constexpr int FEL = FeLanes<T>::value;
    constexpr int FEM = FEN / FEL;               // modes per lane
    constexpr int FE_PPB = FE_THREADS / FEL;     // particles per block
    extern __shared__ __align__(16) unsigned char fe_smem[];
    T* tab = reinterpret_cast<T*>(fe_smem);
    const int tid = threadIdx.x, lane = tid & (FEL - 1), grp = tid / FEL;
    fe_table<T>(F, tab);
    const int D = F.pm.D;
    int p = blockIdx.x * FE_PPB + grp;
    const bool active = MODE == 2 ? (blockIdx.x == 0 && grp == 0) : p < P;
    // ---- coordinates of this group's particle
    T x[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) x[d] = (T)0.5;
    if (MODE == 0) {
        if (active)
            for (int d = 0; d < D; ++d) x[d] = xin[(size_t)d * P + p];
    } else if (MODE == 1) {
        if (active && lane == 0) {
            float xf[AFM_MAXD], v[AFM_MAXD];
            const int rd = it & 1;
            for (int d = 0; d < D; ++d) {
                xf[d] = sw.x[(size_t)d * P + p];
                v[d] = sw.v[(size_t)d * P + p];
            }
            if (it > 0) {
                const int g = min((int)(*sw.gkey[rd] & 0x7fffffffu), P - 1);
                float pb[AFM_MAXD], gb[AFM_MAXD];
                for (int d = 0; d < D; ++d) {
                    pb[d] = sw.pb[rd][(size_t)d * P + p];
                    gb[d] = sw.pb[rd][(size_t)d * P + g];
                }
                pso_move_dev(pc, xf, v, pb, gb, p, it);
                for (int d = 0; d < D; ++d) {
                    sw.x[(size_t)d * P + p] = xf[d];
                    sw.v[(size_t)d * P + p] = v[d];
                }
            }
            for (int d = 0; d < D; ++d) x[d] = (T)xf[d];
        }
        for (int d = 0; d < AFM_MAXD; ++d) x[d] = __shfl_sync(0xffffffffu, x[d], (tid & 31) & ~(FEL - 1));
        if (it > 0 && blockIdx.x == 0 && tid == 0 && history != nullptr)
            history[it - 1] = __uint_as_float((uint32_t)(*sw.gkey[it & 1] >> 32));
    } else {
        const int fin = (pc.iters + 1) & 1;
        p = min((int)(*sw.gkey[fin] & 0x7fffffffu), P - 1);
        for (int d = 0; d < D; ++d) x[d] = (T)sw.pb[fin][(size_t)d * P + p];
    }
    // parameter map in T
    KConst<T> pm;
    pm.force = F.pm.force;
    pm.D = D;
    for (int d = 0; d < AFM_MAXD; ++d) {
        pm.slot[d] = F.pm.slot[d];
        pm.logs[d] = F.pm.logs[d];
        pm.lo[d] = F.pm.lo[d];
        pm.span[d] = F.pm.span[d];
        pm.fixed[d] = F.pm.fixed[d];
    }
    pm.k = F.pm.k;
    pm.s1 = F.pm.s1;
    pm.tau = F.pm.tau;
    const Coef<T> cfc = make_coef<T, T>(pm, x);
    __syncthreads();

    // ---- this lane's modes: coefficients and tip-scaled state
    T b1[FEM], d2[FEM], gq[FEM], fq[FEM];
    T z[FEM], dz[FEM], cz[FEM], cdz[FEM];
#pragma unroll
    for (int j = 0; j < FEM; ++j) {
        const int i = lane + FEL * j;
        const double pt = F.pt[i];
        b1[j] = (T)F.b1[i];
        // the uncompensated slots take 1 + d2, see the step below
        d2[j] = fe_comp<T>(j) ? (T)F.d2[i] : (T)(1.0 + F.d2[i]);
        gq[j] = (T)(F.g[i] * pt);
        fq[j] = (T)(F.f[i] * pt);
        z[j] = (T)(F.z0[i] * pt);
        dz[j] = (T)(F.dz0[i] * pt);
        cz[j] = (T)0;
        cdz[j] = (T)0;
    }
    // the low word of the lowest mode's b1 (the resonant frequency must be
    // represented to ~1e-12); zero in FP64
    const T b1lo = (T)(F.b1[lane] - (double)b1[0]);
    const T Zc = (T)F.Zc, ctip = (T)F.ctip;
    T Fn, Fm, dF;
    fe_force<FORCE, T>(cfc, Zc + (T)F.utip0, Fn, dF);
    fe_force<FORCE, T>(cfc, Zc + (T)F.utipm, Fm, dF);
    T S = (T)0, cS = (T)0, u2 = (T)0;
    const int spc = F.spc;
    // the tip coupling is a contraction of ~1e-4.  FP32: Newton from the
    // uncoupled deflection is converged to FP32 rounding after one step (a
    // second one changes no result in the tests' cases).  FP64: from the
    // deflection the step's current force would give (the predictor base +
    // cz F_n, off by cz times one step's change of the force), one step
    // leaves ~1e-12 of the deflection (a second one moved a C5 winner's
    // FP64 misfit by 1e-13 relative)
    const int newton_it = 1;
    int jn = 0;
    // the record value of step n is loaded during step n - 1, so that no
    // step waits for a global-memory load
    T Unext = (U != nullptr && F.n_steps > 0 && lane == 0) ? (T)U[0] : (T)0;
    for (int n = 0; n < F.n_steps; ++n) {
        const int jp = jn + 1 == spc ? 0 : jn + 1;
        const T Un = Unext;
        if (U != nullptr && lane == 0 && n + 1 < F.n_steps) Unext = (T)U[n + 1];
        const T G = tab[jn];
        const T Fo = (T)2 * Fn + Fm;
        // the drive and past-force terms first: they wait on no state update
        // of the previous step.  Compensated slots form the increment; the
        // others form delta_n + increment in one sum, with (1 + d2) dz.
        T incs[FEM], zps[FEM];
#pragma unroll
        for (int j = 0; j < FEM; ++j) {
            T inc = fma(fq[j], Fo, gq[j] * G);
            inc = fma(d2[j], dz[j], inc);
            if (j == 0) inc = fma(b1lo, z[j], inc);
            inc = fma(b1[j], z[j], inc);
            incs[j] = inc;
            zps[j] = fe_comp<T>(j) ? z[j] + ((dz[j] + inc) - cz[j]) : z[j] + inc;
        }
        T tsum = fe_sum<T, FEM>(zps);
#pragma unroll
        for (int o = FEL / 2; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
        T Fp;
        fe_newton<FORCE, T>(cfc, Zc, tsum, ctip, sizeof(T) == 8 ? Fn : (T)0, newton_it, Fp);
        // compensated updates of both the increment and the modal coordinate
        // (in FP32 for the lowest modes only)
#pragma unroll
        for (int j = 0; j < FEM; ++j) {
            if (fe_comp<T>(j)) {
                kahan_add(dz[j], cdz[j], fma(fq[j], Fp, incs[j]));
                kahan_add(z[j], cz[j], dz[j]);
            } else {
                dz[j] = fma(fq[j], Fp, incs[j]);
                z[j] = z[j] + dz[j];
            }
        }
        Fm = Fn;
        Fn = Fp;
        if (lane == 0 && active) {
            const T ut = fma(ctip, Fp, tsum);
            if (MODE == 0 && defl != nullptr) defl[(size_t)n * P + p] = ut;
            if (U != nullptr) {
                const T r = Un - ut;
                const T y = fma(r, r, -cS);
                const T t = add_rn(S, y);
                cS = sub_rn(sub_rn(t, S), y);
                S = t;
                if (MODE == 2) u2 = fma(Un, Un, u2);
            }
        }
        jn = jp;
    }
    // ---- outputs
    if (MODE == 0) {
        if (lane == 0 && active && S_out != nullptr) S_out[p] = (S < (T)INFINITY) ? S : (T)INFINITY;
    } else if (MODE == 1) {
        unsigned long long key = ~0ull;
        if (lane == 0 && active) {
            float s = (float)S;
            if (!(s < INFINITY)) {
                if (sw.flags != nullptr) atomicAdd(sw.flags, 1);
                s = INFINITY;
            } else if (!(s > 0.f)) {
                s = 0.f;
            }
            const int rd = it & 1, wr = (it + 1) & 1;
            float best = sw.pbS[p];
            const bool improved = s < best || it == 0;
            if (s < best) best = s;
            sw.pbS[p] = best;
            for (int d = 0; d < D; ++d)
                sw.pb[wr][(size_t)d * P + p] = improved ? (float)x[d] : sw.pb[rd][(size_t)d * P + p];
            key = ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)p;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other < key ? other : key;
        }
        if ((tid & 31) == 0) atomicMin(sw.gkey[(it + 1) & 1], key);
    } else if (active && lane == 0) {
        const int fin = (pc.iters + 1) & 1;
        double th[AFM_MAXD];
        for (int s5 = 0; s5 < AFM_MAXD; ++s5) th[s5] = pm.fixed[s5];
        for (int d = 0; d < D; ++d) {
            double v = pm.lo[d] + (double)x[d] * pm.span[d];
            th[pm.slot[d]] = pm.logs[d] ? exp10(v) : v;
        }
        for (int d = 0; d < AFM_MAXD; ++d) {
            res->x[d] = d < D ? (double)x[d] : 0.0;
            res->theta[d] = th[d];
        }
        res->S = (double)__uint_as_float((uint32_t)(*sw.gkey[fin] >> 32));
        if (history != nullptr) history[pc.iters] = (float)res->S;
        res->S_f64 = (double)S;
        res->J_rel = u2 > (T)0 ? sqrt((double)S / (double)u2) : 0.0;
        res->iters = pc.iters;
        res->winner = p;
        res->nonfinite = sw.flags ? sw.flags[0] : 0;
        res->status = (isfinite((double)S) && res->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
        res->defect = 0.0;
        res->segments = 0;
        res->reserved = 0;
        for (int k = 0; k < 3; ++k) res->drive[k] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
namespace {

template <typename Fn>
cudaError_t fe_dispatch(int force, Fn&& f) {
    switch (force) {
        case F_LINEAR: return f(std::integral_constant<int, F_LINEAR>{});
        case F_DMT: return f(std::integral_constant<int, F_DMT>{});
        case F_HOOKE: return f(std::integral_constant<int, F_HOOKE>{});
    }
    return cudaErrorInvalidValue;
}

template <typename T>
size_t fe_smem(const FeConst& F) {
    return sizeof(T) * (size_t)F.spc;
}

template <typename T, typename TU, int MODE, typename... Args>
cudaError_t fe_launch(const FeConst& F, int blocks, cudaStream_t st, Args... args) {
    const int threads = MODE == 2 ? 32 : FE_THREADS;   // the FP64 re-evaluation: one warp
    const size_t smem = fe_smem<T>(F);
    return fe_dispatch(F.pm.force, [&](auto Fc) -> cudaError_t {
        auto kern = fe_modal_kernel<T, TU, decltype(Fc)::value, MODE>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, threads, smem, st>>>(F, args...);
        return cudaGetLastError();
    });
}

}  // namespace

cudaError_t launch_fe_forward_f32(const FeConst& F, const float* x, int P, float* defl,
                                  const float* U, float* S, cudaStream_t st) {
    PsoConst pc{};
    SwarmPtrs sw{};
    constexpr int ppb = FE_THREADS / FeLanes<float>::value;
    return fe_launch<float, float, 0>(F, (P + ppb - 1) / ppb, st, pc, sw, x, P, defl, U, S,
                                      (float*)nullptr, 0, (afm_result*)nullptr);
}

cudaError_t launch_fe_forward_f64(const FeConst& F, const double* x, int P, double* defl,
                                  const double* U, double* S, cudaStream_t st) {
    PsoConst pc{};
    SwarmPtrs sw{};
    constexpr int ppb = FE_THREADS / FeLanes<double>::value;
    return fe_launch<double, double, 0>(F, (P + ppb - 1) / ppb, st, pc, sw, x, P, defl, U,
                                        S, (float*)nullptr, 0, (afm_result*)nullptr);
}

cudaError_t launch_fe_invert_iter(const FeConst& F, const PsoConst& pc, const SwarmPtrs& sw,
                                  const float* U, float* history, int it, cudaStream_t st) {
    constexpr int ppb = FE_THREADS / FeLanes<float>::value;
    return fe_launch<float, float, 1>(F, (pc.P + ppb - 1) / ppb, st, pc, sw,
                                      (const float*)nullptr, pc.P, (float*)nullptr, U,
                                      (float*)nullptr, history, it, (afm_result*)nullptr);
}

cudaError_t launch_fe_invert_final(const FeConst& F, const PsoConst& pc, const SwarmPtrs& sw,
                                   const float* U, float* history, void* result, cudaStream_t st) {
    return fe_launch<double, float, 2>(F, 1, st, pc, sw, (const double*)nullptr, pc.P,
                                       (double*)nullptr, U, (double*)nullptr, history, 0,
                                       reinterpret_cast<afm_result*>(result));
}

}  // namespace afm
