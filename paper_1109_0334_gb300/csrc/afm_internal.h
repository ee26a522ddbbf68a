// afm_internal.h -- structures shared by the host set-up (afminv_api.cpp) and
// the CUDA kernels.  Not part of the public ABI.
//
// Units inside the kernels ("scaled units"):
//   length  1 nm
//   time    tau = h / 6, where h = 1 / (f1 * steps_per_cycle) is the RK4 step,
//           so that the RK4 constants h/2 = 3, h = 6 and h/6 = 1 are exact
//           binary numbers (an FP32 rounding of h/6 would detune the resonant
//           mode against the index-exact drive by ~3e-8 per step, which a
//           quality factor of 400 amplifies to ~6e-6 of the deflection)
//   force   k * 1 nm * (omega_1 tau)^2, so the modal equation (Eq. 2) reads
//             q_i'' = tip_i F + gamma_i g - w2_i q_i - wq_i q_i'
//           with w2_i = (omega_i tau)^2, wq_i = omega_i tau / Q_i.
#pragma once
#include <stdint.h>

#define AFM_MAXM 8
#define AFM_MAXD 5
#define AFM_TAB_MAX 4096   // half-step drive phases per period (2 * steps_per_cycle)
#define AFM_SEG 32         // adjoint checkpoint interval (RK4 steps)

#if defined(__CUDACC__)
#define AFM_HD __host__ __device__
#else
#define AFM_HD
#endif

namespace afm {

// Which modes take compensated (Kahan) state updates.  FP64: all.  FP32: the
// lowest mode only.  It carries the resonant response, and its RK4 increment
// is a small fraction of the state (omega_1 h << 1), so that a plain sum
// drops low bits of the deflection every step; the higher modes are driven
// far off resonance, with amplitudes ~(omega_1 / omega_i)^2 / Q of the first
// mode's, and their plain-sum rounding stays far below FP32 resolution of
// the tip deflection.
template <typename T>
AFM_HD constexpr bool comp_mode(int i) {
    return sizeof(T) == 8 || i == 0;
}

enum ForceKind { F_LINEAR = 0, F_DMT = 1, F_DMT_KV = 2, F_HOOKE = 3, F_SPRING_DAMPER = 4 };

// Force-law coefficients of one particle in scaled units.
//   LINEAR        F = -c0 (d - c1)
//   DMT           F = c0 max(c3 - d, 0)^1.5 - c1 / max(d, c3)^2      (c0 = hz, c1 = vdw, c3 = a0)
//   DMT_KV        DMT - c2 sqrt(max(c3 - d, 0)) d'                    (c2 = kv)
//   HOOKE         F = c0 max(c1 - d, 0)
//   SPRING_DAMPER F = (d < c1) ? c0 (c1 - d) - c2 d' : 0
template <typename T>
struct Coef {
    T c0, c1, c2, c3;
};

// Constants of one problem in the arithmetic type of a kernel (float or
// double), filled on the host by the per-problem set-up.
template <typename T>
struct KConst {
    T w2[AFM_MAXM], w2lo[AFM_MAXM], wq[AFM_MAXM], gam[AFM_MAXM], tip[AFM_MAXM];
    T cmask[AFM_MAXM];              // 1: mode i takes compensated sums (comp_mode), else 0
    T q0[AFM_MAXM], v0[AFM_MAXM];
    T Zc;
    double drive_amp, drive_phase;  // g = drive_amp * sin(2 pi j / spc2 + drive_phase)
    int m, spc2, n_steps, force, D;
    int slot[AFM_MAXD], logs[AFM_MAXD];
    double lo[AFM_MAXD], span[AFM_MAXD], fixed[AFM_MAXD];
    double k, s1, tau;
    int drive_mode;                 // 1: per-particle base motion from rest (kern_drive.cu)
    double drv[3];                  // fixed base amplitude [m], frequency [Hz], chirp [Hz/s]
    int np;                         // deflection points (kern_points.cu), 0: the tip
    T phi[4][AFM_MAXM];             // tip-normalised mode shapes at the points
};

// Finite-element cantilever (cubic Hermite elements, clamped node removed)
// advanced by Newmark's average-acceleration scheme (beta = 1/4, gamma = 1/2)
// with the tip force implicit.  With Rayleigh damping, M, K and C are
// diagonal in the M-orthonormal eigenbasis (u = Phi z, Phi^T M Phi = I), so
// the scheme decouples exactly into one scalar recursion per mode, written in
// increment form (delta = z_n - z_{n-1}):
//   delta_{n+1} = delta_n + b1_i z_n + d2_i delta_n + g_i G_n
//                 + f_i (F_{n+1} + 2 F_n + F_{n-1}),   z_{n+1} = z_n + delta_{n+1}
// with s_i = 1 + h/2 c_i + h^2/4 lambda_i, b1_i = -h^2 lambda_i / s_i,
// d2_i = -h c_i / s_i (c_i = alpha + beta lambda_i), g_i = (phi_i^T M r) / s_i
// (G_n = table_{n+1} + 2 table_n + table_{n-1}, table = h^2/4 g in nm) and
// f_i = (h^2/4) k phi_i(tip) / s_i (force in units of k * 1 nm); the tip
// deflection is sum_i phi_i(tip) z_i.
#define AFM_FE_MAXN 64      // DOFs = modes (2 per node)
#define AFM_FE_LANES 8      // lanes per particle in the FE kernels

struct FeConst {
    int ne, n, spc, n_steps;
    double h;                   // Newmark step (s)
    double Zc;                  // rest gap [nm]
    double drive_amp, drive_phase;   // table_j = drive_amp sin(2 pi j / spc + phase)
    double b1[AFM_FE_MAXN], d2[AFM_FE_MAXN], g[AFM_FE_MAXN], f[AFM_FE_MAXN], pt[AFM_FE_MAXN];
    // b1 of the lowest AFM_FE_LANES modes carries a low word in FP32 (the
    // resonant mode's frequency must be represented to ~1e-12)
    double z0[AFM_FE_MAXN], dz0[AFM_FE_MAXN];   // initial modal state and increment
    double ctip;                // sum_i pt_i f_i: tip response to the step's own tip force
    double utip0, utipm;        // tip deflection at steps 0 and -1 [nm]
    KConst<float> pm;           // force law and parameter map (s1 = 1)
};

}  // namespace afm
