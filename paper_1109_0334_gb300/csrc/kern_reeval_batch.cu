// kern_reeval_batch.cu -- the FP64 re-evaluation by multiple shooting in
// time (kern_reeval.cu) for every pixel of a batch at once: each queue
// slot's winner (the parameters in its result record) is integrated over its
// own record in segments of AFM_SEG steps.  Slot i owns segments
// [i * maxB, i * maxB + B_i), B_i = ceil(n_i / AFM_SEG), maxB that of the
// longest record; threads past B_i return at once.
//   guess    one thread per slot: FP32 run of the winner (the swarm kernels'
//            compensated step), keeping the state at every segment start;
//   sweep    (twice) one thread per segment: FP64 integration from its start
//            with the FP32 tangent map; one warp per slot walks its joins;
//   final    the FP64 pass from the corrected starts sums each segment's
//            misfit share; one thread per slot adds its shares in order,
//            checks the joins (sequential FP64 fallback past 1e-9) and fills
//            the result record.
#include "afm_reeval.cuh"

namespace afm {

using namespace reeval;

namespace {

__device__ __forceinline__ int slot_pixel(const BatchArgs& a, int i) {
    return a.order != nullptr ? a.order[i] : i;
}

__device__ __forceinline__ int slot_steps(const BatchArgs& a, int pix) {
    return (int)(a.off[pix + 1] - a.off[pix]);
}

// Segments of a slot's record; 0 for a record longer than the problem's
// n_steps (its slot has no room: the final kernel integrates it in one
// sequential FP64 pass).
__device__ __forceinline__ int slot_segments(const ReevalBatch& R, int n) {
    const int B = reeval_segments(n);
    return B <= R.maxB ? B : 0;
}

// The constants and FP64 drive table of pixel pix: the launch's, or its own
// (PP: a batch whose pixels differ in their problem).
template <bool PP, typename T>
__device__ __forceinline__ const KConst<T>& pix_k(const KConst<T>& K, const KConst<T>* per, int pix) {
    if constexpr (PP)
        return per[pix];
    else
        return K;
}

template <bool PP>
__device__ __forceinline__ const double* pix_tab64(const ReevalBatch& R, const BatchArgs& a, int pix) {
    if constexpr (PP)
        return a.pix.tab64 + (size_t)pix * a.pix.ld;
    else
        return R.tab;
}

__device__ __forceinline__ Coef<double> slot_coef(const ReevalBatch& R, int i) {
    Coef<double> c;
    c.c0 = R.coef[4 * (size_t)i];
    c.c1 = R.coef[4 * (size_t)i + 1];
    c.c2 = R.coef[4 * (size_t)i + 2];
    c.c3 = R.coef[4 * (size_t)i + 3];
    return c;
}

}  // namespace

template <int M, int FORCE, bool PP>
__global__ void __launch_bounds__(128) rb_guess_kernel(const KConst<float> Kf0,
                                                       const KConst<double> Kd0,
                                                       const ReevalBatch R, const BatchArgs a) {
    extern __shared__ __align__(16) float tabs[];
    if constexpr (!PP) {
        build_drive_table(Kf0, tabs);
        if (blockIdx.x == 0) build_drive_table(Kd0, R.tab);
        __syncthreads();
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_pix) return;
    const int pix = slot_pixel(a, i);
    const KConst<float>& Kf = pix_k<PP>(Kf0, a.pix.kf, pix);
    const KConst<double>& Kd = pix_k<PP>(Kd0, a.pix.kd, pix);
    const float* tabf = PP ? a.pix.tab32 + (size_t)pix * a.pix.ld : tabs;
    const int n = slot_steps(a, pix);
    const float* U = a.U + a.off[pix];
    double xd[AFM_MAXD];
    for (int d = 0; d < AFM_MAXD; ++d) xd[d] = a.res[pix].x[d];
    const Coef<double> cd = make_coef<double, double>(Kd, xd);
    R.coef[4 * (size_t)i] = cd.c0;
    R.coef[4 * (size_t)i + 1] = cd.c1;
    R.coef[4 * (size_t)i + 2] = cd.c2;
    R.coef[4 * (size_t)i + 3] = cd.c3;
    double u2 = 0.0;
    for (int s = 0; s < n; ++s) u2 = fma((double)U[s], (double)U[s], u2);
    R.u2[i] = u2;
    const Coef<float> c = make_coef<float, double>(Kf, xd);
    constexpr int S2 = 2 * M;
    double* Y = R.Z + (size_t)i * R.maxB * S2;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        Y[k] = Kd.q0[k];
        Y[M + k] = Kd.v0[k];
    }
    const int B = slot_segments(R, n);
    float q[M], v[M], cq[M], cv[M];
    init_state<float, M>(Kf, q, v, cq, cv);
    int j = 0, b = 1, next = AFM_SEG;
    const int spc2 = Kf.spc2;
    // the state after step (b * AFM_SEG) starts segment b; the last segment's
    // start comes from step (B - 1) * AFM_SEG
    const int n_guess = (B - 1) * AFM_SEG;
    for (int s = 0; s < n_guess; ++s) {
        const float g0 = tabf[j], gh = tabf[j + 1], g1 = tabf[j + 2];
        j += 2;
        if (j >= spc2) j = 0;
        rk4_step<float, M, FORCE>(Kf, c, q, v, cq, cv, g0, gh, g1);
        if (s + 1 == next) {
#pragma unroll
            for (int k = 0; k < M; ++k) {
                Y[(size_t)b * S2 + k] = (double)q[k] - (double)cq[k];
                Y[(size_t)b * S2 + M + k] = (double)v[k] - (double)cv[k];
            }
            ++b;
            next += AFM_SEG;
        }
    }
}

template <int M, int FORCE, bool TANGENT, bool PP>
__global__ void __launch_bounds__(32) rb_pass_kernel(const KConst<double> K0, const ReevalBatch R,
                                                     const BatchArgs a) {
    __shared__ float rec[TANGENT ? AFM_SEG * kRec * 32 : 1];
    constexpr int S2 = 2 * M;
    const int lane = threadIdx.x;
    const long long t = (long long)blockIdx.x * 32 + lane;
    const int i = (int)(t / R.maxB), b = (int)(t % R.maxB);
    if (i >= a.n_pix) return;
    const int pix = slot_pixel(a, i);
    const int n = slot_steps(a, pix);
    if (b >= slot_segments(R, n)) return;
    const KConst<double>& K = pix_k<PP>(K0, a.pix.kd, pix);
    const double* tab = pix_tab64<PP>(R, a, pix);
    const float* U = a.U + a.off[pix];
    const Coef<double> c = slot_coef(R, i);
    Coef<float> cf;
    cf.c0 = (float)c.c0;
    cf.c1 = (float)c.c1;
    cf.c2 = (float)c.c2;
    cf.c3 = (float)c.c3;
    const size_t g = (size_t)i * R.maxB + b;   // global segment index
    double q[M], v[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        q[k] = R.Z[g * S2 + k];
        v[k] = R.Z[g * S2 + M + k];
    }
    const int n0 = b * AFM_SEG;
    const int n1 = min(n0 + AFM_SEG, n);
    int j = (int)((2ll * n0) % K.spc2);
    double S = 0.0;
    for (int s = n0; s < n1; ++s) {
        const double g0 = tab[j], gh = tab[j + 1], g1 = tab[j + 2];
        j += 2;
        if (j >= K.spc2) j = 0;
        step64<M, FORCE, TANGENT>(K, c, cf, q, v, g0, gh, g1, rec + lane + (s - n0) * kRec * 32);
        double u = q[0];
#pragma unroll
        for (int k = 1; k < M; ++k) u += q[k];
        const double r = (double)U[s] - u;
        S = fma(r, r, S);
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        R.E[g * S2 + k] = q[k];
        R.E[g * S2 + M + k] = v[k];
    }
    R.Sb[g] = S;
    if (TANGENT) {
        float w2[M], wq[M], tip[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            w2[k] = (float)K.w2[k];
            wq[k] = (float)K.wq[k];
            tip[k] = (float)K.tip[k];
        }
        const int ns = n1 - n0;
#pragma unroll 1
        for (int col = 0; col < S2; ++col) {
            float dq[M], dv[M];
#pragma unroll
            for (int k = 0; k < M; ++k) {
                dq[k] = col == k ? 1.f : 0.f;
                dv[k] = col == M + k ? 1.f : 0.f;
            }
            for (int s = 0; s < ns; ++s)
                jvp_step<M, FORCE>(w2, wq, tip, rec + lane + s * kRec * 32, dq, dv);
            float* Jc = R.J + g * S2 * S2 + col;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                Jc[k * S2] = dq[k];
                Jc[(M + k) * S2] = dv[k];
            }
        }
    }
}

// Newton update of one slot's segment starts, in place, in order over its
// joins: Z'_{b+1} = E_b + J_b (Z'_b - Z_b).  One warp per slot; lane k < 2m
// owns state component k.
template <int M>
__global__ void __launch_bounds__(128) rb_correct_kernel(const ReevalBatch R, const BatchArgs a) {
    constexpr int S2 = 2 * M;
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int k = threadIdx.x & 31;
    if (i >= a.n_pix) return;
    const int B = slot_segments(R, slot_steps(a, slot_pixel(a, i)));
    const bool act = k < S2;
    const int kk = act ? k : 0;
    double* Z = R.Z + (size_t)i * R.maxB * S2;
    const double* E = R.E + (size_t)i * R.maxB * S2;
    const float* J = R.J + (size_t)i * R.maxB * S2 * S2;
    double z = Z[kk];
    double e = B > 0 ? E[kk] : 0.0, y = z;
    float Jr[S2];
#pragma unroll
    for (int c = 0; c < S2; ++c) Jr[c] = B > 0 ? J[(size_t)kk * S2 + c] : 0.f;
    for (int b = 0; b + 1 < B; ++b) {
        // the next join's operands, read before segment b + 1's start is replaced
        const double en = E[(size_t)(b + 1) * S2 + kk];
        const double yn = Z[(size_t)(b + 1) * S2 + kk];
        float Jn[S2];
#pragma unroll
        for (int c = 0; c < S2; ++c) Jn[c] = J[((size_t)(b + 1) * S2 + kk) * S2 + c];
        const double dl = act ? z - y : 0.0;
        double acc0 = e, acc1 = 0.0;
#pragma unroll
        for (int c = 0; c < S2; ++c) {
            const double dc = __shfl_sync(0xffffffffu, dl, c);
            if (c & 1)
                acc1 = fma((double)Jr[c], dc, acc1);
            else
                acc0 = fma((double)Jr[c], dc, acc0);
        }
        z = acc0 + acc1;
        __syncwarp();
        if (act) Z[(size_t)(b + 1) * S2 + k] = z;
        e = en;
        y = yn;
#pragma unroll
        for (int c = 0; c < S2; ++c) Jr[c] = Jn[c];
    }
}

// Per slot: S_f64 = sum of the shares in order, the join check (sequential
// FP64 fallback), and the result record.
template <int M, int FORCE, bool PP>
__global__ void __launch_bounds__(128) rb_final_kernel(const KConst<double> K0, const ReevalBatch R,
                                                       const BatchArgs a) {
    constexpr int S2 = 2 * M;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_pix) return;
    const int pix = slot_pixel(a, i);
    const KConst<double>& K = pix_k<PP>(K0, a.pix.kd, pix);
    const int n = slot_steps(a, pix);
    const int B = slot_segments(R, n);
    const size_t g0 = (size_t)i * R.maxB;
    double S64 = B > 0 || n == 0 ? 0.0 : NAN, defect = 0.0;   // NaN: no room, sequential
    for (int b = 0; b < B; ++b) {
        S64 += R.Sb[g0 + b];
        if (b + 1 < B) {
            double mx = 0.0;
#pragma unroll
            for (int k = 0; k < S2; ++k) {
                const double d = fabs(R.E[(g0 + b) * S2 + k] - R.Z[(g0 + b + 1) * S2 + k]);
                if (!(d <= mx)) mx = d;   // keeps a NaN
            }
            defect += mx;
        }
    }
    int segs = B;
    if (!(defect <= kDefectTol) || !isfinite(S64)) {
        S64 = integrate<double, M, FORCE, float>(K, slot_coef(R, i), pix_tab64<PP>(R, a, pix),
                                                 a.U + a.off[pix], nullptr, 0, 0, n);
        segs = 0;
    }
    afm_result* r = a.res + pix;
    double th[AFM_MAXD];
    for (int s5 = 0; s5 < AFM_MAXD; ++s5) th[s5] = K.fixed[s5];
    for (int d = 0; d < K.D; ++d) {
        const double v = K.lo[d] + r->x[d] * K.span[d];
        th[K.slot[d]] = K.logs[d] ? exp10(v) : v;
    }
    for (int s5 = 0; s5 < AFM_MAXD; ++s5) r->theta[s5] = th[s5];
    const double u2 = R.u2[i];
    r->S_f64 = S64;
    r->J_rel = u2 > 0.0 ? sqrt(S64 / u2) : 0.0;
    r->status = (isfinite(S64) && r->nonfinite == 0) ? AFM_OK : AFM_ERR_NONFINITE;
    r->defect = segs > 0 ? defect : (defect <= kDefectTol ? 0.0 : defect);
    r->segments = segs;
    r->reserved = 0;
    for (int k = 0; k < 3; ++k) r->drive[k] = 0.0;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t reeval_batch_bytes(int m, int n_steps, int spc, int n_pix) {
    const size_t B = (size_t)reeval_segments(n_steps), S2 = 2 * (size_t)reeval_modes(m);
    const size_t segs = B * (size_t)n_pix;
    return a256(sizeof(double) * 4 * (size_t)n_pix) + a256(sizeof(double) * (2 * (size_t)spc + 1)) +
           a256(sizeof(double) * segs * S2) * 2 + a256(sizeof(float) * segs * S2 * S2) +
           a256(sizeof(double) * segs) + a256(sizeof(double) * (size_t)n_pix) + 256;
}

void reeval_batch_carve(void* base, int m, int n_steps, int spc, int n_pix, ReevalBatch* R) {
    const size_t B = (size_t)reeval_segments(n_steps), S2 = 2 * (size_t)reeval_modes(m);
    const size_t segs = B * (size_t)n_pix;
    char* p = static_cast<char*>(base);
    R->coef = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * 4 * (size_t)n_pix);
    R->tab = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * (2 * (size_t)spc + 1));
    R->Z = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * segs * S2);
    R->E = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * segs * S2);
    R->J = reinterpret_cast<float*>(p);
    p += a256(sizeof(float) * segs * S2 * S2);
    R->Sb = reinterpret_cast<double*>(p);
    p += a256(sizeof(double) * segs);
    R->u2 = reinterpret_cast<double*>(p);
    R->maxB = (int)B;
}

cudaError_t launch_reeval_batch(const KConst<float>& Kf, const KConst<double>& Kd,
                                const ReevalBatch& R, const BatchArgs& a, cudaStream_t st) {
    if (R.maxB != reeval_segments(Kd.n_steps) || Kd.np > 0) return cudaErrorInvalidValue;
    const bool pp = a.pix.kf != nullptr;
    return dispatch_m13(Kd.m, Kd.force, [&](auto Mc, auto Fc) -> cudaError_t {
        constexpr int M = decltype(Mc)::value, FORCE = decltype(Fc)::value;
        auto run = [&](auto Pc) -> cudaError_t {
            constexpr bool PP = decltype(Pc)::value;
            const size_t smem = PP ? 0 : sizeof(float) * (size_t)(Kf.spc2 + 1);
            rb_guess_kernel<M, FORCE, PP><<<(a.n_pix + 127) / 128, 128, smem, st>>>(Kf, Kd, R, a);
            cudaError_t e = cudaGetLastError();
            const long long segs = (long long)a.n_pix * R.maxB;
            const int grid = (int)((segs + 31) / 32);
            const int cgrid = (a.n_pix * 32 + 127) / 128;
            for (int k = 0; e == cudaSuccess && k < kSweeps; ++k) {
                rb_pass_kernel<M, FORCE, true, PP><<<grid, 32, 0, st>>>(Kd, R, a);
                if ((e = cudaGetLastError()) != cudaSuccess) break;
                rb_correct_kernel<M><<<cgrid, 128, 0, st>>>(R, a);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) return e;
            rb_pass_kernel<M, FORCE, false, PP><<<grid, 32, 0, st>>>(Kd, R, a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            rb_final_kernel<M, FORCE, PP><<<(a.n_pix + 127) / 128, 128, 0, st>>>(Kd, R, a);
            return cudaGetLastError();
        };
        return pp ? run(std::true_type{}) : run(std::false_type{});
    });
}

}  // namespace afm
