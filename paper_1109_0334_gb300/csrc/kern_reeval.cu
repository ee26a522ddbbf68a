// kern_reeval.cu -- FP64 re-evaluation of one winner's misfit (Eq. 5 on the
// RK4 solution of Eq. 2, Sec. 3.2) by multiple shooting in time.
//
// FP64 arithmetic on this GPU issues at a small fraction of the FP32 rate,
// so one thread stepping a whole record in FP64 needs ~7 us per RK4 step.
// The record is instead cut into segments of AFM_SEG steps that are
// integrated concurrently, one thread each, and the segment start states
// are made consistent by Newton's method on the matching conditions
// Z_{b+1} = Phi_b(Z_b), Phi_b being AFM_SEG FP64 RK4 steps:
//   guess  one thread integrates the winner in FP32 (compensated, as the
//          swarm kernels do) and keeps the state at every segment start;
//   sweep  (twice) every segment is integrated in FP64 from its start Z_b,
//          giving E_b = Phi_b(Z_b), while its tangent map J_b = dPhi_b/dZ_b
//          is propagated in FP32 (the RK4 step linearised about the FP64
//          stages); one warp then walks the joins in order:
//          Z'_0 = y_0,  Z'_{b+1} = E_b + J_b (Z'_b - Z_b);
//   final  the segments are integrated in FP64 from the corrected starts,
//          each summing its share of the misfit; S is the FP64 sum of the
//          shares.
// The joins are then checked: if the summed max-norm mismatch between each
// segment's end and the next segment's start exceeds 1e-9 (scaled units),
// or anything is non-finite, the final kernel integrates the whole record
// once more, sequentially, in FP64.
#include "afm_reeval.cuh"

namespace afm {

using namespace reeval;

// The swarm's global best (as invert_final_kernel selects it); one thread.
__global__ void reeval_pick_swarm_kernel(const PsoConst pc, const SwarmPtrs sw, float* history,
                                         ReevalWinner* __restrict__ w) {
    const int fin = (pc.iters + 1) & 1;
    const unsigned long long key = *sw.gkey[fin];
    const int g = min((int)(key & 0x7fffffffu), pc.P - 1);
    const float S32 = __uint_as_float((uint32_t)(key >> 32));
    if (history != nullptr) history[pc.iters] = S32;
    for (int d = 0; d < AFM_MAXD; ++d)
        w->x[d] = d < pc.D ? (double)sw.pb[fin][(size_t)d * pc.P + g] : 0.0;
    w->S32 = S32;
    w->winner = g;
}

// The lowest of Kn misfits (first index on ties); x [D][Kn]; idx maps the
// candidate to its swarm index (or nullptr).  One thread.
__global__ void reeval_pick_min_kernel(int D, int Kn, const float* __restrict__ x,
                                       const float* __restrict__ S, const int* __restrict__ idx,
                                       ReevalWinner* __restrict__ w) {
    int kb = 0;
    for (int k = 1; k < Kn; ++k)
        if (S[k] < S[kb]) kb = k;
    for (int d = 0; d < AFM_MAXD; ++d) w->x[d] = d < D ? (double)x[(size_t)d * Kn + kb] : 0.0;
    w->S32 = S[kb];
    w->winner = idx != nullptr ? idx[kb] : kb;
}

// Drive tables, sum of U^2, FP64 force coefficients of the winner, and the
// FP32 guess of the segment start states (start[0]; b = 0 is the exact FP64
// initial state).
template <int M, int FORCE>
__global__ void __launch_bounds__(256) reeval_guess_kernel(const KConst<float> Kf,
                                                           const KConst<double> Kd,
                                                           const ReevalPtrs R,
                                                           const float* __restrict__ U) {
    extern __shared__ __align__(16) float tabf[];
    __shared__ double red[256];
    build_drive_table(Kf, tabf);
    build_drive_table(Kd, R.tab);
    double acc = 0.0;
    const int nv = Kd.n_steps * (Kd.np > 0 ? Kd.np : 1);   // record values
    for (int n = threadIdx.x; n < nv; n += blockDim.x) acc += (double)U[n] * (double)U[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    *R.sumU2 = red[0];
    ReevalWinner* w = R.win;
    double xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = w->x[d];
    const Coef<double> cd = make_coef<double, double>(Kd, xd);
    w->c[0] = cd.c0;
    w->c[1] = cd.c1;
    w->c[2] = cd.c2;
    w->c[3] = cd.c3;
    const Coef<float> c = make_coef<float, double>(Kf, xd);
    constexpr int S2 = 2 * M;
    double* Y = R.start[0];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Y[i] = Kd.q0[i];
        Y[M + i] = Kd.v0[i];
    }
    float q[M], v[M], cq[M], cv[M];
    init_state<float, M>(Kf, q, v, cq, cv);
    int j = 0, b = 1, next = AFM_SEG;
    const int n = Kf.n_steps, spc2 = Kf.spc2;
    for (int s = 0; s < n; ++s) {
        const float g0 = tabf[j], gh = tabf[j + 1], g1 = tabf[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        rk4_step<float, M, FORCE>(Kf, c, q, v, cq, cv, g0, gh, g1);
        if (s + 1 == next) {
            if (b < R.B) {
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    Y[(size_t)b * S2 + i] = (double)q[i] - (double)cq[i];
                    Y[(size_t)b * S2 + M + i] = (double)v[i] - (double)cv[i];
                }
            }
            ++b;
            next += AFM_SEG;
        }
    }
}

// One thread per segment b: AFM_SEG FP64 steps from Z_b -> E_b and the
// segment's misfit share Sb_b; TANGENT: also J_b ([2m][2m], row = output
// component, column = input direction) in FP32 from the recorded slopes.
template <int M, int FORCE, bool TANGENT>
__global__ void __launch_bounds__(32) reeval_pass_kernel(const KConst<double> K,
                                                         const ReevalPtrs R,
                                                         const double* __restrict__ Z,
                                                         const float* __restrict__ U) {
    __shared__ float rec[TANGENT ? AFM_SEG * kRec * 32 : 1];
    constexpr int S2 = 2 * M;
    const int lane = threadIdx.x;
    const int b = blockIdx.x * 32 + lane;
    if (b >= R.B) return;
    const Coef<double> c = winner_coef(*R.win);
    Coef<float> cf;
    cf.c0 = (float)c.c0;
    cf.c1 = (float)c.c1;
    cf.c2 = (float)c.c2;
    cf.c3 = (float)c.c3;
    double q[M], v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        q[i] = Z[(size_t)b * S2 + i];
        v[i] = Z[(size_t)b * S2 + M + i];
    }
    const int n0 = b * AFM_SEG;
    const int n1 = min(n0 + AFM_SEG, K.n_steps);
    int j = (int)((2ll * n0) % K.spc2);
    double S = 0.0;
    for (int s = n0; s < n1; ++s) {
        const double g0 = R.tab[j], gh = R.tab[j + 1], g1 = R.tab[j + 2];
        j += 2;
        if (j >= K.spc2) j = 0;
        step64<M, FORCE, TANGENT>(K, c, cf, q, v, g0, gh, g1, rec + lane + (s - n0) * kRec * 32);
        if (K.np > 0) {   // deflection points
            for (int k = 0; k < K.np; ++k) {
                double uk = K.phi[k][0] * q[0];
#pragma unroll
                for (int i = 1; i < M; ++i) uk = fma(K.phi[k][i], q[i], uk);
                const double r = (double)U[(size_t)s * K.np + k] - uk;
                S = fma(r, r, S);
            }
        } else {
            double u = q[0];
#pragma unroll
            for (int i = 1; i < M; ++i) u += q[i];
            const double r = (double)U[s] - u;
            S = fma(r, r, S);
        }
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        R.E[(size_t)b * S2 + i] = q[i];
        R.E[(size_t)b * S2 + M + i] = v[i];
    }
    R.Sb[b] = S;
    if (TANGENT) {
        float w2[M], wq[M], tip[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            w2[i] = (float)K.w2[i];
            wq[i] = (float)K.wq[i];
            tip[i] = (float)K.tip[i];
        }
        const int ns = n1 - n0;
#pragma unroll 1
        for (int col = 0; col < S2; ++col) {
            float dq[M], dv[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                dq[i] = col == i ? 1.f : 0.f;
                dv[i] = col == M + i ? 1.f : 0.f;
            }
            for (int t = 0; t < ns; ++t) jvp_step<M, FORCE>(w2, wq, tip, rec + lane + t * kRec * 32, dq, dv);
            double* Jc = R.J + (size_t)b * S2 * S2 + col;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                Jc[i * S2] = (double)dq[i];
                Jc[(M + i) * S2] = (double)dv[i];
            }
        }
    }
}

// Newton update of the segment starts, in order over the joins:
// Znew_0 = Zold_0 (the exact initial state), Znew_{b+1} = E_b + J_b (Znew_b -
// Zold_b).  One warp; lane i < 2m owns state component i.
template <int M>
__global__ void __launch_bounds__(32) reeval_correct_kernel(const ReevalPtrs R,
                                                            const double* __restrict__ Zold,
                                                            double* __restrict__ Znew) {
    constexpr int S2 = 2 * M;
    const int i = threadIdx.x;
    const bool act = i < S2;
    const int ii = act ? i : 0;
    double z = Zold[ii];
    if (act) Znew[i] = z;
    // operands of segment b are loaded one iteration ahead
    double e = R.E[ii], y = Zold[ii], Jr[S2];
#pragma unroll
    for (int k = 0; k < S2; ++k) Jr[k] = R.J[(size_t)ii * S2 + k];
    for (int b = 0; b < R.B; ++b) {
        double en = 0.0, yn = 0.0, Jn[S2];
#pragma unroll
        for (int k = 0; k < S2; ++k) Jn[k] = 0.0;
        if (b + 1 < R.B) {
            en = R.E[(size_t)(b + 1) * S2 + ii];
            yn = Zold[(size_t)(b + 1) * S2 + ii];
#pragma unroll
            for (int k = 0; k < S2; ++k) Jn[k] = R.J[((size_t)(b + 1) * S2 + ii) * S2 + k];
        }
        const double dl = act ? z - y : 0.0;
        double acc0 = e, acc1 = 0.0;
#pragma unroll
        for (int k = 0; k < S2; ++k) {
            const double dk = __shfl_sync(0xffffffffu, dl, k);
            if (k & 1)
                acc1 = fma(Jr[k], dk, acc1);
            else
                acc0 = fma(Jr[k], dk, acc0);
        }
        z = acc0 + acc1;
        if (act) Znew[(size_t)(b + 1) * S2 + i] = z;
        e = en;
        y = yn;
#pragma unroll
        for (int k = 0; k < S2; ++k) Jr[k] = Jn[k];
    }
}

// S_f64 = sum of the segment shares, the join check (with the sequential
// fallback) and the result record.  One block of 256.
template <int M, int FORCE>
__global__ void __launch_bounds__(256) reeval_final_kernel(const KConst<double> K,
                                                           const ReevalPtrs R,
                                                           const double* __restrict__ Z,
                                                           const float* __restrict__ U, int iters,
                                                           const int* __restrict__ flags,
                                                           afm_result* __restrict__ res) {
    __shared__ double rs[256], rd[256];
    constexpr int S2 = 2 * M;
    double s = 0.0, dsum = 0.0;
    for (int b = threadIdx.x; b < R.B; b += blockDim.x) {
        s += R.Sb[b];
        if (b + 1 < R.B) {
            double mx = 0.0;
#pragma unroll
            for (int i = 0; i < S2; ++i) {
                const double e = fabs(R.E[(size_t)b * S2 + i] - Z[(size_t)(b + 1) * S2 + i]);
                if (!(e <= mx)) mx = e;   // keeps a NaN
            }
            dsum += mx;
        }
    }
    rs[threadIdx.x] = s;
    rd[threadIdx.x] = dsum;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            rs[threadIdx.x] += rs[threadIdx.x + h];
            rd[threadIdx.x] += rd[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const ReevalWinner& w = *R.win;
    double S64 = rs[0];
    const double defect = rd[0];
    int segs = R.B;
    if (!(defect <= kDefectTol) || !isfinite(S64)) {
        S64 = K.np > 0 ? integrate_points<double, M, FORCE, float>(K, winner_coef(w), R.tab, U,
                                                                   nullptr, 0, 0, K.n_steps)
                       : integrate<double, M, FORCE, float>(K, winner_coef(w), R.tab, U, nullptr,
                                                            0, 0, K.n_steps);
        segs = 0;
    }
    double th[AFM_MAXD];
    for (int s5 = 0; s5 < AFM_MAXD; ++s5) th[s5] = K.fixed[s5];
    for (int d = 0; d < K.D; ++d) {
        const double v = K.lo[d] + w.x[d] * K.span[d];
        th[K.slot[d]] = K.logs[d] ? exp10(v) : v;
    }
    for (int d = 0; d < AFM_MAXD; ++d) {
        res->x[d] = w.x[d];
        res->theta[d] = th[d];
    }
    const double u2 = *R.sumU2;
    res->S = (double)w.S32;
    res->S_f64 = S64;
    res->J_rel = u2 > 0.0 ? sqrt(S64 / u2) : 0.0;
    res->iters = iters;
    res->winner = w.winner;
    res->nonfinite = flags != nullptr ? flags[0] : 0;
    res->status = (isfinite(S64) && res->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
    res->defect = segs > 0 ? defect : (defect <= kDefectTol ? 0.0 : defect);
    res->segments = segs;
    res->reserved = 0;
    for (int k = 0; k < 3; ++k) res->drive[k] = 0.0;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
bool reeval_supported(int m, int n_steps) {
    return m >= 1 && m <= AFM_MAXM && n_steps >= 2 * AFM_SEG;
}


size_t reeval_bytes(int m, int n_steps, int spc) {
    const size_t B = (size_t)reeval_segments(n_steps), S2 = 2 * (size_t)reeval_modes(m);
    return a256(sizeof(ReevalWinner)) + a256(sizeof(double) * (2 * (size_t)spc + 1)) +
           2 * a256(sizeof(double) * (B + 1) * S2) + a256(sizeof(double) * B * S2) +
           a256(sizeof(double) * B * S2 * S2) + a256(sizeof(double) * B) + 256;
}

void reeval_carve(void* base, int m, int n_steps, int spc, ReevalPtrs* R) {
    const size_t B = (size_t)reeval_segments(n_steps), S2 = 2 * (size_t)reeval_modes(m);
    char* p = static_cast<char*>(base);
    R->win = reinterpret_cast<ReevalWinner*>(p);
    p += a256(sizeof(ReevalWinner));
    R->tab = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * (2 * (size_t)spc + 1));
    R->start[0] = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * (B + 1) * S2);
    R->start[1] = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * (B + 1) * S2);
    R->E = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * B * S2);
    R->J = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * B * S2 * S2);
    R->Sb = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * B);
    R->sumU2 = reinterpret_cast<double*>(p);
    R->B = (int)B;
}

cudaError_t launch_reeval_pick_swarm(const PsoConst& pc, const SwarmPtrs& sw, float* history,
                                     ReevalWinner* w, cudaStream_t st) {
    reeval_pick_swarm_kernel<<<1, 1, 0, st>>>(pc, sw, history, w);
    return cudaGetLastError();
}

cudaError_t launch_reeval_pick_min(int D, int Kn, const float* x, const float* S, const int* idx,
                                   ReevalWinner* w, cudaStream_t st) {
    reeval_pick_min_kernel<<<1, 1, 0, st>>>(D, Kn, x, S, idx, w);
    return cudaGetLastError();
}

cudaError_t launch_reeval(const KConst<float>& Kf, const KConst<double>& Kd, const ReevalPtrs& R,
                          const float* U, int iters, const int* flags, void* result,
                          cudaStream_t st) {
    if (!reeval_supported(Kd.m, Kd.n_steps) || R.B != reeval_segments(Kd.n_steps))
        return cudaErrorInvalidValue;
    return dispatch_m13(Kd.m, Kd.force, [&](auto Mc, auto Fc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value, FORCE = decltype(Fc)::value;
        const size_t smem = sizeof(float) * (size_t)(Kf.spc2 + 1);
        reeval_guess_kernel<M, FORCE><<<1, 256, smem, st>>>(Kf, Kd, R, U);
        cudaError_t e = cudaGetLastError();
        const int grid = (R.B + 31) / 32;
        for (int k = 0; e == cudaSuccess && k < kSweeps; ++k) {
            reeval_pass_kernel<M, FORCE, true><<<grid, 32, 0, st>>>(Kd, R, R.start[k & 1], U);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            reeval_correct_kernel<M><<<1, 32, 0, st>>>(R, R.start[k & 1], R.start[(k + 1) & 1]);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
        const double* Zf = R.start[kSweeps & 1];
        reeval_pass_kernel<M, FORCE, false><<<grid, 32, 0, st>>>(Kd, R, Zf, U);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        reeval_final_kernel<M, FORCE><<<1, 256, 0, st>>>(Kd, R, Zf, U, iters, flags,
                                                         reinterpret_cast<afm_result*>(result));
        return cudaGetLastError();
    });
}

}  // namespace afm
