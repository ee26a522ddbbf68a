// kern_fe.cu -- finite-element cantilever (cubic Hermite Euler-Bernoulli
// elements) with Newmark's average-acceleration scheme (beta = 1/4,
// gamma = 1/2) and the tip-sample force solved implicitly at every step, in
// the increment form documented in afm_internal.h.  Each step applies the
// dense 64 x 128 propagator [B1 | D2] to the states [u_n; delta_n] of a batch
// of particles (a (64 x 128) x (128 x B) product), then a scalar Newton
// solve for each particle's tip force and a rank-one update.
//
// The propagator is built on the device, per block, in FP64 from the
// element matrices (banded Cholesky of S, S^-1 column by column, banded
// products), so no device memory beyond the caller's arrays is needed.
#include <type_traits>

#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

constexpr int FEN = AFM_FE_MAXN;      // padded DOF count (rows)
constexpr int FEK = 2 * AFM_FE_MAXN;  // propagator columns [u; delta]
constexpr int FEB = AFM_FE_BATCH;     // particles per block (FP32 / TF32)

// ---------------------------------------------------------------------------
// Propagator construction (FP64, whole block cooperates).
// ---------------------------------------------------------------------------
struct FeScratch {
    double Mb[FEN][7], Kb[FEN][7];   // bands of M and K, offset j - i + 3
    double Lb[FEN][4];               // banded Cholesky factor of S, offset j - i + 3 (j <= i)
    double Mr[FEN];                  // M r (r = 1 on deflection DOFs)
};

__device__ __forceinline__ double fe_elem(const FeConst& F, int gi, int gj, bool stiff) {
    // sum over the (at most two) elements holding both global DOFs
    const double h = F.he;
    const double me[16] = {156, 22 * h, 54, -13 * h, 22 * h, 4 * h * h, 13 * h, -3 * h * h,
                           54, 13 * h, 156, -22 * h, -13 * h, -3 * h * h, -22 * h, 4 * h * h};
    const double ke[16] = {12, 6 * h, -12, 6 * h, 6 * h, 4 * h * h, -6 * h, 2 * h * h,
                           -12, -6 * h, 12, -6 * h, 6 * h, 2 * h * h, -6 * h, 4 * h * h};
    const double ms = F.mu * h / 420.0, ks = F.EI / (h * h * h);
    double v = 0.0;
    const int lo = max(0, (max(gi, gj) - 2) / 2), hi = min(F.ne - 1, min(gi, gj) / 2);
    for (int e = lo; e <= hi; ++e) {
        const int a = gi - 2 * e, b = gj - 2 * e;
        if (a < 0 || a > 3 || b < 0 || b > 3) continue;
        v += stiff ? ks * ke[a * 4 + b] : ms * me[a * 4 + b];
    }
    return v;
}

// Builds A[k * FEN + i] (k < FEN: B1[i][k]; k >= FEN: D2[i][k - FEN]) and the
// vectors b, c in type T; Sinv is FEN x FEN doubles of shared scratch.
template <typename T>
__device__ void fe_build(const FeConst& F, FeScratch& sc, double* Sinv, T* A, T* bvec, T* cvec) {
    const int n = F.n, tid = threadIdx.x, nt = blockDim.x;
    const double sM = 1.0 + 0.5 * F.h * F.alpha, sK = 0.5 * F.h * F.beta + 0.25 * F.h * F.h;
    for (int t = tid; t < FEN * 7; t += nt) {
        const int i = t / 7, o = t % 7, j = i + o - 3;
        double m = 0.0, k = 0.0;
        if (i < n && j >= 0 && j < n) {
            m = fe_elem(F, i + 2, j + 2, false);
            k = fe_elem(F, i + 2, j + 2, true);
        }
        sc.Mb[i][o] = m;
        sc.Kb[i][o] = k;
    }
    __syncthreads();
    for (int i = tid; i < FEN; i += nt) {
        double s = 0.0;
        for (int o = 0; o < 7; ++o) {
            const int j = i + o - 3;
            if (j >= 0 && j < n && (j % 2) == 0) s += sc.Mb[i][o];
        }
        sc.Mr[i] = i < n ? s : 0.0;
    }
    if (tid == 0) {   // banded Cholesky of S = sM M + sK K
        for (int i = 0; i < n; ++i)
            for (int j = max(0, i - 3); j <= i; ++j) {
                double s = sM * sc.Mb[i][j - i + 3] + sK * sc.Kb[i][j - i + 3];
                for (int k = max(0, i - 3); k < j; ++k) s -= sc.Lb[i][k - i + 3] * sc.Lb[j][k - j + 3];
                sc.Lb[i][j - i + 3] = (i == j) ? sqrt(s) : s / sc.Lb[j][3];
            }
    }
    __syncthreads();
    for (int t = tid; t < FEN; t += nt) {   // column t of S^-1: S x = e_t
        double* x = Sinv + t;               // x[i] at Sinv[i * FEN + t]
        for (int i = 0; i < FEN; ++i) {
            if (i >= n) { x[i * FEN] = 0.0; continue; }
            double s = (i == t) ? 1.0 : 0.0;
            for (int k = max(0, i - 3); k < i; ++k) s -= sc.Lb[i][k - i + 3] * x[k * FEN];
            x[i * FEN] = s / sc.Lb[i][3];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = x[i * FEN];
            for (int k = i + 1; k <= min(n - 1, i + 3); ++k) s -= sc.Lb[k][i - k + 3] * x[k * FEN];
            x[i * FEN] = s / sc.Lb[i][3];
        }
    }
    __syncthreads();
    const double h = F.h;
    for (int t = tid; t < FEN * FEN; t += nt) {
        const int i = t % FEN, j = t / FEN;   // row i, column j
        double b1 = 0.0, d2 = 0.0;
        if (i < n && j < n) {
            for (int o = 0; o < 7; ++o) {
                const int k = j + o - 3;      // K[k][j] = Kb[j][k - j + 3] (symmetric)
                if (k < 0 || k >= n) continue;
                const double s = Sinv[i * FEN + k];
                const double kk = sc.Kb[j][o], mm = sc.Mb[j][o];
                b1 += s * kk;
                d2 += s * (F.alpha * mm + F.beta * kk);
            }
        }
        A[j * FEN + i] = (T)(-h * h * b1);
        A[(FEN + j) * FEN + i] = (T)(-h * d2);
    }
    for (int i = tid; i < FEN; i += nt) {
        double bv = 0.0;
        for (int k = 0; k < n; ++k) bv += Sinv[i * FEN + k] * sc.Mr[k];
        bvec[i] = (T)(i < n ? bv : 0.0);
        cvec[i] = (T)(i < n ? Sinv[i * FEN + F.tip] * F.cscale : 0.0);
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void fe_table(const FeConst& F, T* tab) {
    for (int j = threadIdx.x; j < F.spc; j += blockDim.x)
        tab[j] = (T)(F.drive_amp * sin(6.283185307179586476925 * (double)j / (double)F.spc + F.drive_phase));
}

// Tip force and its slope in the gap (laws without rate dependence).
template <int FORCE, typename T>
__device__ __forceinline__ void fe_force(const Coef<T>& c, T d, T& Fv, T& dF) {
    if (FORCE == F_LINEAR) {
        Fv = -c.c0 * (d - c.c1);
        dF = -c.c0;
    } else if (FORCE == F_DMT) {
        if (d > c.c3) {
            const T r = (T)1 / d;
            Fv = -c.c1 * r * r;
            dF = (T)2 * c.c1 * r * r * r;
        } else {
            const T del = c.c3 - d, sq = sqrt(del);
            const T r = (T)1 / c.c3;
            Fv = c.c0 * del * sq - c.c1 * r * r;
            dF = (T)(-1.5) * c.c0 * sq;
        }
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

// z = base + cz F(Zc + z) by Newton from z = base.
template <int FORCE, typename T>
__device__ __forceinline__ T fe_newton(const Coef<T>& c, T Zc, T base, T cz, int iters, T& Fz) {
    T z = base, dF;
    for (int it = 0; it < iters; ++it) {
        fe_force<FORCE, T>(c, Zc + z, Fz, dF);
        const T phi = z - base - cz * Fz;
        z = z - phi / ((T)1 - cz * dF);
    }
    fe_force<FORCE, T>(c, Zc + z, Fz, dF);
    return z;
}

// ---------------------------------------------------------------------------
// FP32 batch kernel: 64 particles per block, 256 threads; thread (ty, tx)
// owns rows 4ty..4ty+3 of particles 4tx..4tx+3.  MODE 0: forward (defl, S);
// MODE 1: one fused inversion iteration (PSO move, forward, bests).
// ---------------------------------------------------------------------------
template <int FORCE, int MODE>
__global__ void __launch_bounds__(256) fe_kernel_f32(const FeConst F, const PsoConst pc, SwarmPtrs sw,
                                                     const float* __restrict__ xin, int P,
                                                     float* __restrict__ defl,
                                                     const float* __restrict__ U,
                                                     float* __restrict__ S_out,
                                                     float* __restrict__ history, int it) {
    extern __shared__ __align__(16) unsigned char fe_smem[];
    float* A = reinterpret_cast<float*>(fe_smem);                 // [FEK][FEN]
    float* X = A + FEK * FEN;                                     // [FEK][FEB]
    FeScratch& sc = *reinterpret_cast<FeScratch*>(X + FEK * FEB);
    float* bvec = reinterpret_cast<float*>(&sc + 1);
    float* cvec = bvec + FEN;
    float* Fn1 = cvec + FEN;                                      // [FEB]
    float* xs = Fn1 + FEB;                                        // [AFM_MAXD][FEB] particle coords
    float* tab = xs + AFM_MAXD * FEB;                             // [spc]
    double* Sinv = reinterpret_cast<double*>(X);                  // aliases X during set-up
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int p0 = blockIdx.x * FEB;
    const int D = F.pm.D;

    // particle coordinates (PSO move in MODE 1) into shared memory
    if (tid < FEB) {
        const int p = p0 + tid;
        float x[AFM_MAXD];
        if (p < P) {
            if (MODE == 0) {
                for (int d = 0; d < D; ++d) x[d] = xin[(size_t)d * P + p];
            } else {
                float v[AFM_MAXD];
                const int rd = it & 1;
                for (int d = 0; d < D; ++d) {
                    x[d] = sw.x[(size_t)d * P + p];
                    v[d] = sw.v[(size_t)d * P + p];
                }
                if (it > 0) {
                    const int g = min((int)(*sw.gkey[rd] & 0x7fffffffu), P - 1);
                    float pb[AFM_MAXD], gb[AFM_MAXD];
                    for (int d = 0; d < D; ++d) {
                        pb[d] = sw.pb[rd][(size_t)d * P + p];
                        gb[d] = sw.pb[rd][(size_t)d * P + g];
                    }
                    pso_move_dev(pc, x, v, pb, gb, p, it);
                    for (int d = 0; d < D; ++d) {
                        sw.x[(size_t)d * P + p] = x[d];
                        sw.v[(size_t)d * P + p] = v[d];
                    }
                }
            }
        } else {
            for (int d = 0; d < D; ++d) x[d] = 0.5f;
        }
        for (int d = 0; d < D; ++d) xs[d * FEB + tid] = x[d];
    }
    if (MODE == 1 && it > 0 && blockIdx.x == 0 && tid == 0 && history != nullptr)
        history[it - 1] = __uint_as_float((uint32_t)(*sw.gkey[it & 1] >> 32));
    fe_build<float>(F, sc, Sinv, A, bvec, cvec);
    fe_table<float>(F, tab);

    // state of this thread's 4 x 4 tile
    float u[4][4], cu[4][4], dl[4][4], br[4], cr[4];
    float Fn[4], Fm[4];
    Coef<float> cf[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = 4 * ty + r;
        br[r] = bvec[row];
        cr[r] = cvec[row];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            u[r][c] = (float)F.u0[row];
            dl[r][c] = (float)F.d0[row];
            cu[r][c] = 0.f;
        }
    }
    const float Zc = (float)F.Zc;
    const float utip0 = (float)F.u0[F.tip], utipm = (float)(F.u0[F.tip] - F.d0[F.tip]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float x[AFM_MAXD];
        for (int d = 0; d < D; ++d) x[d] = xs[d * FEB + 4 * tx + c];
        cf[c] = make_coef<float, float>(F.pm, x);
        float dF;
        fe_force<FORCE, float>(cf[c], Zc + utip0, Fn[c], dF);
        fe_force<FORCE, float>(cf[c], Zc + utipm, Fm[c], dF);
    }
    __syncthreads();   // Sinv no longer needed: X may be written
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            X[(4 * ty + r) * FEB + 4 * tx + c] = u[r][c];
            X[(FEN + 4 * ty + r) * FEB + 4 * tx + c] = dl[r][c];
        }
    __syncthreads();

    const bool tip_owner = (F.tip >> 2) == ty;
    const int tr = F.tip & 3;
    const float ctip = cvec[F.tip], btip = bvec[F.tip];
    float Sacc[4] = {0.f, 0.f, 0.f, 0.f}, cS[4] = {0.f, 0.f, 0.f, 0.f};
    const int N = F.n_steps, spc = F.spc;
    int jn = 0;   // n mod spc
    for (int n = 0; n < N; ++n) {
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 8
        for (int k = 0; k < FEK; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(A + k * FEN + 4 * ty);
            const float4 x = *reinterpret_cast<const float4*>(X + k * FEB + 4 * tx);
            const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], xv[c], acc[r][c]);
        }
        const int jp = jn + 1 == spc ? 0 : jn + 1, jm = jn == 0 ? spc - 1 : jn - 1;
        const float G = tab[jp] + 2.f * tab[jn] + tab[jm];
        if (tip_owner) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float base = u[tr][c] + (dl[tr][c] + acc[tr][c] + btip * G +
                                               ctip * (2.f * Fn[c] + Fm[c]));
                float Fz;
                fe_newton<FORCE, float>(cf[c], Zc, base, ctip, 3, Fz);
                Fn1[4 * tx + c] = Fz;
            }
        }
        __syncthreads();   // all reads of X done, tip forces visible
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float Fp = Fn1[4 * tx + c];
            const float Fs = Fp + 2.f * Fn[c] + Fm[c];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float dn = dl[r][c] + (acc[r][c] + fmaf(br[r], G, cr[r] * Fs));
                kahan_add(u[r][c], cu[r][c], dn);
                dl[r][c] = dn;
                X[(4 * ty + r) * FEB + 4 * tx + c] = u[r][c];
                X[(FEN + 4 * ty + r) * FEB + 4 * tx + c] = dn;
            }
            Fm[c] = Fn[c];
            Fn[c] = Fp;
        }
        if (tip_owner) {
            const float Un = U != nullptr ? U[n] : 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int p = p0 + 4 * tx + c;
                const float ut = u[tr][c];
                if (MODE == 0 && defl != nullptr && p < P) defl[(size_t)n * P + p] = ut;
                const float rr = Un - ut;
                const float y = fmaf(rr, rr, -cS[c]);
                const float t = add_rn(Sacc[c], y);
                cS[c] = sub_rn(sub_rn(t, Sacc[c]), y);
                Sacc[c] = t;
            }
        }
        jn = jp;
        __syncthreads();   // X complete before the next product
    }

    // outputs
    unsigned long long key = ~0ull;
    if (tip_owner) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int p = p0 + 4 * tx + c;
            if (p >= P) continue;
            float s = Sacc[c];
            if (!(s < INFINITY)) {
                if (sw.flags != nullptr) atomicAdd(sw.flags, 1);
                s = INFINITY;
            } else if (!(s > 0.f)) {
                s = 0.f;
            }
            if (MODE == 0) {
                if (S_out != nullptr) S_out[p] = s;
            } else {
                const int rd = it & 1, wr = (it + 1) & 1;
                float best = sw.pbS[p];
                const bool improved = s < best || it == 0;
                if (s < best) best = s;
                sw.pbS[p] = best;
                for (int d = 0; d < D; ++d)
                    sw.pb[wr][(size_t)d * P + p] =
                        improved ? xs[d * FEB + 4 * tx + c] : sw.pb[rd][(size_t)d * P + p];
                const unsigned long long kk = ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)p;
                key = kk < key ? kk : key;
            }
        }
    }
    if (MODE == 1) {
        // keys live in the 16 tip-owning threads (one half-warp); every lane
        // takes part in the shuffles so that the warp stays converged
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other < key ? other : key;
        }
        if (tip_owner && tx == 0) atomicMin(sw.gkey[(it + 1) & 1], key);
    }
}

// ---------------------------------------------------------------------------
// FP64: one particle per block, one thread per DOF row.  Used for the FP64
// forward and the FP64 re-evaluation of an inversion's winner.
// ---------------------------------------------------------------------------
template <int FORCE>
__global__ void __launch_bounds__(64) fe_kernel_f64(const FeConst F, const double* __restrict__ xin,
                                                    int P, double* __restrict__ defl,
                                                    const double* __restrict__ U64,
                                                    const float* __restrict__ U32,
                                                    double* __restrict__ S_out,
                                                    const unsigned long long* __restrict__ wkey,
                                                    const float* __restrict__ wpb,
                                                    afm_result* __restrict__ res,
                                                    const int* __restrict__ flags, int iters,
                                                    float* __restrict__ history) {
    extern __shared__ __align__(16) unsigned char fe_smem[];
    double* A = reinterpret_cast<double*>(fe_smem);     // [FEK][FEN]
    double* Sinv = A + FEK * FEN;                       // [FEN][FEN]
    FeScratch& sc = *reinterpret_cast<FeScratch*>(Sinv + FEN * FEN);
    double* bvec = reinterpret_cast<double*>(&sc + 1);
    double* cvec = bvec + FEN;
    double* X = cvec + FEN;                             // [FEK]
    double* red = X + FEK;                              // [64] reductions / broadcast
    double* tab = red + 64;                             // [spc]
    const int tid = threadIdx.x;
    int p = blockIdx.x;
    double xd[AFM_MAXD];
    const int D = F.pm.D;
    if (wkey != nullptr) {   // winner of an inversion
        p = min((int)(*wkey & 0x7fffffffu), P - 1);
        for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < D ? (double)wpb[(size_t)d * P + p] : 0.0;
    } else {
        for (int d = 0; d < AFM_MAXD; ++d) xd[d] = d < D ? xin[(size_t)d * P + p] : 0.0;
    }
    fe_build<double>(F, sc, Sinv, A, bvec, cvec);
    fe_table<double>(F, tab);
    KConst<double> pm;
    // the parameter map only (force law, slots, bounds, conversions)
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
    const Coef<double> cf = make_coef<double, double>(pm, xd);
    const int row = tid;
    double u = F.u0[row], dl = F.d0[row], dF;
    double Fn, Fm;
    fe_force<FORCE, double>(cf, F.Zc + F.u0[F.tip], Fn, dF);
    fe_force<FORCE, double>(cf, F.Zc + F.u0[F.tip] - F.d0[F.tip], Fm, dF);
    X[row] = u;
    X[FEN + row] = dl;
    const double br = bvec[row], cr = cvec[row], btip = bvec[F.tip], ctip = cvec[F.tip];
    double S = 0.0, u2 = 0.0;
    int jn = 0;
    __syncthreads();
    for (int n = 0; n < F.n_steps; ++n) {
        double acc = 0.0;
        for (int k = 0; k < FEK; ++k) acc = fma(A[k * FEN + row], X[k], acc);
        const int jp = jn + 1 == F.spc ? 0 : jn + 1, jm = jn == 0 ? F.spc - 1 : jn - 1;
        const double G = tab[jp] + 2.0 * tab[jn] + tab[jm];
        if (row == F.tip) {
            const double base = u + dl + acc + btip * G + ctip * (2.0 * Fn + Fm);
            double Fz;
            fe_newton<FORCE, double>(cf, F.Zc, base, ctip, 6, Fz);
            red[0] = Fz;
        }
        __syncthreads();
        const double Fp = red[0];
        const double dn = dl + acc + br * G + cr * (Fp + 2.0 * Fn + Fm);
        u = u + dn;
        dl = dn;
        Fm = Fn;
        Fn = Fp;
        X[row] = u;
        X[FEN + row] = dn;
        if (row == F.tip) {
            const double Un = U64 != nullptr ? U64[n] : (U32 != nullptr ? (double)U32[n] : 0.0);
            if (defl != nullptr) defl[(size_t)n * P + p] = u;
            S += (Un - u) * (Un - u);
            u2 += Un * Un;
        }
        jn = jp;
        __syncthreads();
    }
    if (row != F.tip) return;
    if (res == nullptr) {
        if (S_out != nullptr) S_out[p] = S;
        return;
    }
    double th[AFM_MAXD];
    for (int s = 0; s < AFM_MAXD; ++s) th[s] = pm.fixed[s];
    for (int d = 0; d < D; ++d) {
        double v = pm.lo[d] + xd[d] * pm.span[d];
        th[pm.slot[d]] = pm.logs[d] ? exp10(v) : v;
    }
    for (int d = 0; d < AFM_MAXD; ++d) {
        res->x[d] = xd[d];
        res->theta[d] = th[d];
    }
    res->S = (double)__uint_as_float((uint32_t)(*wkey >> 32));
    if (history != nullptr) history[iters] = (float)res->S;
    res->S_f64 = S;
    res->J_rel = u2 > 0.0 ? sqrt(S / u2) : 0.0;
    res->iters = iters;
    res->winner = p;
    res->nonfinite = flags ? flags[0] : 0;
    res->status = (isfinite(S) && res->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
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

size_t fe_smem_f32(const FeConst& F) {
    return sizeof(float) * ((size_t)FEK * FEN + (size_t)FEK * FEB) + sizeof(FeScratch) +
           sizeof(float) * (2 * FEN + FEB + AFM_MAXD * FEB + (size_t)F.spc);
}

size_t fe_smem_f64(const FeConst& F) {
    return sizeof(double) * ((size_t)FEK * FEN + (size_t)FEN * FEN) + sizeof(FeScratch) +
           sizeof(double) * (2 * FEN + FEK + 64 + (size_t)F.spc);
}

}  // namespace

cudaError_t launch_fe_forward_f32(const FeConst& F, const float* x, int P, float* defl,
                                  const float* U, float* S, cudaStream_t st) {
    const size_t smem = fe_smem_f32(F);
    const int blocks = (P + FEB - 1) / FEB;
    PsoConst pc{};
    SwarmPtrs sw{};
    return fe_dispatch(F.pm.force, [&](auto Fc) -> cudaError_t {
        auto kern = fe_kernel_f32<decltype(Fc)::value, 0>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, 256, smem, st>>>(F, pc, sw, x, P, defl, U, S, nullptr, 0);
        return cudaGetLastError();
    });
}

cudaError_t launch_fe_invert_iter(const FeConst& F, const PsoConst& pc, const SwarmPtrs& sw,
                                  const float* U, float* history, int it, cudaStream_t st) {
    const size_t smem = fe_smem_f32(F);
    const int blocks = (pc.P + FEB - 1) / FEB;
    return fe_dispatch(F.pm.force, [&](auto Fc) -> cudaError_t {
        auto kern = fe_kernel_f32<decltype(Fc)::value, 1>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, 256, smem, st>>>(F, pc, sw, nullptr, pc.P, nullptr, U, nullptr, history, it);
        return cudaGetLastError();
    });
}

cudaError_t launch_fe_forward_f64(const FeConst& F, const double* x, int P, double* defl,
                                  const double* U, double* S, cudaStream_t st) {
    const size_t smem = fe_smem_f64(F);
    return fe_dispatch(F.pm.force, [&](auto Fc) -> cudaError_t {
        auto kern = fe_kernel_f64<decltype(Fc)::value>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<P, 64, smem, st>>>(F, x, P, defl, U, nullptr, S, nullptr, nullptr, nullptr, nullptr, 0,
                                  nullptr);
        return cudaGetLastError();
    });
}

cudaError_t launch_fe_invert_final(const FeConst& F, const PsoConst& pc, const SwarmPtrs& sw,
                                   const float* U, float* history, void* result, cudaStream_t st) {
    const size_t smem = fe_smem_f64(F);
    const int fin = (pc.iters + 1) & 1;
    return fe_dispatch(F.pm.force, [&](auto Fc) -> cudaError_t {
        auto kern = fe_kernel_f64<decltype(Fc)::value>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<1, 64, smem, st>>>(F, nullptr, pc.P, nullptr, nullptr, U, nullptr, sw.gkey[fin],
                                  sw.pb[fin], reinterpret_cast<afm_result*>(result), sw.flags, pc.iters,
                                  history);
        return cudaGetLastError();
    });
}

}  // namespace afm
