/*
 * afm_oracle.c -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see afm_oracle.h).
 *
 * Plain double-precision restatement, in SI units, of:
 *   - the modal reduction of the Euler-Bernoulli cantilever (Eq. 1 -> Eq. 2,
 *     App. B) with the paper's overflow-safe exponential mode shapes
 *     (Sec. 3.2, Eqs. 6-7), Newton roots and Simpson integration (Sec. 3.2);
 *   - the explicit classic 4th-order Runge-Kutta time loop (Sec. 3.2);
 *   - the L2 cost functional J^2 = int (U - u)^2 dt (Eq. 5), as a sum over the
 *     sampled record;
 *   - particle-swarm optimisation with the velocity update of Eq. 8 (Sec. 3.4);
 *   - synthetic records made at a finer step than the solver (the paper's
 *     inverse-crime measure, Sec. 4.1);
 *   - the DMT and DMT + Kelvin-Voigt tip-sample laws (Hertz contact and van
 *     der Waals, named as the richer force models in Sec. 2.2 and Sec. 5),
 *     the paper's Hooke and spring-damper laws (Eqs. 3-4), and a linear test
 *     spring whose response has a closed form.
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written
 * here from its published definition.
 *
 * Nothing here is blocked, fused or reordered beyond what the method states.
 */
#include "afm_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* ======================================================================== */
/* Philox4x32-10 (SC'11): ten rounds of two 32x32->64 multiplies, xor with  */
/* the other counter words and the round key; the key is bumped by the Weyl  */
/* constants between rounds.                                                 */
/* ======================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Top 24 bits of a word scaled by 2^-24: a uniform on [0, 1) that is exact in
 * both float and double. */
double orc_uniform(uint32_t word) { return (double)(word >> 8) * (1.0 / 16777216.0); }

/* One uniform from the stream: key = seed, counter = (c0, c1, c2, tag<<16|block),
 * word `word` of the four outputs. */
double orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                uint32_t tag, uint32_t block, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, (tag << 16) | block};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return orc_uniform(out[word]);
}

/* ======================================================================== */
/* Modal setup (Sec. 3.2): beta_i L by Newton, mode shapes in exponential    */
/* form, Simpson integrals.                                                  */
/* ======================================================================== */

/* i-th root (i >= 1) of cos x cosh x + 1 = 0, found by Newton on the
 * equivalent cos x + 1/cosh x = 0 (no overflow for large x). */
double orc_beam_root(int i)
{
    double x = (2.0 * i - 1.0) * M_PI / 2.0;
    for (int it = 0; it < 200; ++it) {
        double f = cos(x) + 1.0 / cosh(x);
        double fp = -sin(x) - tanh(x) / cosh(x);
        double dx = f / fp;
        x -= dx;
        if (fabs(dx) < 1e-16 * x) break;
    }
    return x;
}

/* Paper's exponential form of the clamped-free mode shape (Eq. 6), as a
 * function of xi = x / L for b = beta L:
 *   Phi = [2 sin(b xi) - 2G cos(b xi) + (G-1) e^{b xi} + (G+1) e^{-b xi}] / 2
 * with G from Eq. 7.  The printed denominator of Eq. 7 has "- e^{-2 beta L}";
 * the free-end conditions require "+ e^{-2 beta L}" (reading R2).  G - 1 is
 * formed directly (same algebra) so that it keeps its relative precision. */
double orc_mode_shape(double b, double xi)
{
    double e1 = exp(-b), e2 = exp(-2.0 * b);
    double num = 1.0 - e2 + 2.0 * e1 * sin(b);
    double den = 1.0 + e2 + 2.0 * e1 * cos(b);
    double Gm1 = (-2.0 * e2 + 2.0 * e1 * (sin(b) - cos(b))) / den;  /* = num/den - 1 */
    double G = num / den;
    double bx = b * xi;
    return (2.0 * sin(bx) - 2.0 * G * cos(bx) + Gm1 * exp(bx) + (G + 1.0) * exp(-bx)) / 2.0;
}

/* Composite Simpson rule on [0, 1] with n_points (odd) samples. */
static double simpson(const double* f, int n_points)
{
    int n = n_points - 1;
    double h = 1.0 / n, s = f[0] + f[n];
    for (int j = 1; j < n; ++j) s += (j % 2 ? 4.0 : 2.0) * f[j];
    return s * h / 3.0;
}

/* For each mode: beta_i L, gamma_i = <phi,1>/<phi,phi> and <phi,phi>/L of the
 * tip-normalised shape phi = Phi / Phi(L), and Phi(L).  Integrals by Simpson
 * on n_points samples (Sec. 3.2; App. A uses 501 points). */
int orc_modal_factors(int n_modes, int n_points, double* bL, double* gam,
                      double* int_phi2, double* phi_tip)
{
    if (n_modes < 1 || n_modes > ORC_MAXM || n_points < 3 || n_points % 2 == 0) return -1;
    double* f1 = (double*)malloc(sizeof(double) * n_points);
    double* f2 = (double*)malloc(sizeof(double) * n_points);
    for (int i = 0; i < n_modes; ++i) {
        double b = orc_beam_root(i + 1);
        double tip = orc_mode_shape(b, 1.0);
        for (int j = 0; j < n_points; ++j) {
            double p = orc_mode_shape(b, (double)j / (n_points - 1)) / tip;
            f1[j] = p;
            f2[j] = p * p;
        }
        double I1 = simpson(f1, n_points), I2 = simpson(f2, n_points);
        bL[i] = b;
        gam[i] = I1 / I2;
        if (int_phi2) int_phi2[i] = I2;
        if (phi_tip) phi_tip[i] = tip;
    }
    free(f1);
    free(f2);
    return 0;
}

/* Problem setup for the modal models (R3, R4, R6):
 *   omega_i = omega_1 (beta_i / beta_1)^2, modal mass m = k / omega_1^2,
 *   base y_b = a sin(w t + psi) with w = omega_1, and a, psi such that the free
 *   linear steady tip deflection is A0 cos(w t); the initial state is that
 *   steady state at t = 0.  Point mass: one mode with gamma = 1. */
int orc_setup(const orc_case* c, orc_modal* md)
{
    memset(md, 0, sizeof(*md));
    int m = c->model == ORC_POINT_MASS ? 1 : c->n_modes;
    if (m < 1 || m > ORC_MAXM || c->spc < 2) return -1;
    md->m = m;
    double w1 = 2.0 * M_PI * c->f1;
    if (c->model == ORC_POINT_MASS) {
        md->w[0] = w1;
        md->gam[0] = 1.0;
    } else {
        double bL[ORC_MAXM], gam[ORC_MAXM];
        if (orc_modal_factors(m, 501, bL, gam, NULL, NULL)) return -1;
        for (int i = 0; i < m; ++i) {
            md->w[i] = w1 * (bL[i] / bL[0]) * (bL[i] / bL[0]);
            md->gam[i] = gam[i];
        }
    }
    md->mass = c->k / (w1 * w1);
    md->wd = w1;
    double w = md->wd;
    double complex H[ORC_MAXM], Hs = 0.0;
    for (int i = 0; i < m; ++i) {
        H[i] = md->gam[i] / (md->w[i] * md->w[i] - w * w + I * w * md->w[i] / c->Q[i]);
        Hs += H[i];
    }
    md->a = c->A0 / (w * w * cabs(Hs));
    md->psi = M_PI / 2.0 - carg(Hs);
    for (int i = 0; i < m; ++i) {
        double complex ci = md->a * w * w * H[i] * cexp(I * md->psi);
        md->eta0[i] = cimag(ci);
        md->etad0[i] = w * creal(ci);
    }
    md->dt = 1.0 / (c->f1 * c->spc);
    if (c->drive == 1) {          /* base motion set per parameter vector; start at rest */
        if (c->dt <= 0.0 || c->model == ORC_FE_HERMITE) return -1;
        md->dt = c->dt;
        md->a = md->psi = 0.0;
        for (int i = 0; i < m; ++i) md->eta0[i] = md->etad0[i] = 0.0;
    }
    return 0;
}

/* Drive mode 1 (reading R18): g = -d^2 y_b/dt^2 for y_b = a sin(phi),
 * phi = 2 pi (f t + g t^2):  g(t) = a (phi'^2 sin phi - phi'' cos phi) with
 * phi' = 2 pi (f + 2 g t), phi'' = 4 pi g; (a, f, g) = th[5..7]. */
double orc_drive_chirp(const double th[ORC_NSLOT], double t)
{
    double a = th[5], f = th[6], g = th[7];
    double phi = 2.0 * M_PI * (f * t + g * t * t);
    double dphi = 2.0 * M_PI * (f + 2.0 * g * t);
    double ddphi = 4.0 * M_PI * g;
    return a * (dphi * dphi * sin(phi) - ddphi * cos(phi));
}

/* g = -d^2 y_b/dt^2 at the half-step index j, i.e. t = j dt / 2, with the
 * phase reduced modulo one drive period (2 spc half steps). */
double orc_drive_half(const orc_modal* md, int spc, long j)
{
    long jj = j % (2L * spc);
    double t = (double)jj * (md->dt / 2.0);
    return md->a * md->wd * md->wd * sin(md->wd * t + md->psi);
}

/* ======================================================================== */
/* Tip-sample forces.  d is the gap, ddot its rate; F > 0 pushes the tip     */
/* away from the sample.                                                     */
/* ======================================================================== */
double orc_force(int kind, const double th[ORC_NSLOT], double d, double ddot)
{
    switch (kind) {
    case ORC_F_LINEAR:
        return -th[0] * (d - th[1]);
    case ORC_F_DMT:
    case ORC_F_DMT_KV: {
        double E = th[0], H = th[1], R = th[2], a0 = th[3];
        if (d > a0) return -H * R / (6.0 * d * d);
        double delta = a0 - d;
        double F = (4.0 / 3.0) * E * sqrt(R) * pow(delta, 1.5) - H * R / (6.0 * a0 * a0);
        if (kind == ORC_F_DMT_KV) F -= th[4] * sqrt(R * delta) * ddot;
        return F;
    }
    case ORC_F_HOOKE:
        return d < th[1] ? th[0] * (th[1] - d) : 0.0;
    case ORC_F_SPRING_DAMPER:
        return d < th[1] ? th[0] * (th[1] - d) - th[2] * ddot : 0.0;
    default:
        return 0.0;
    }
}

/* Right-hand side of the modal system (Eq. 2 with 2 zeta omega_i = omega_i/Q,
 * reading R4):  eta_i'' = F/m + gamma_i g - omega_i^2 eta_i - (omega_i/Q_i) eta_i'
 * with the gap d = Zc + sum_i eta_i (tip-normalised shapes, reading R5). */
static void rhs(const orc_case* c, const orc_modal* md, const double th[ORC_NSLOT], double g,
                const double* y, double* f)
{
    int m = md->m;
    double u = 0.0, ud = 0.0;
    for (int i = 0; i < m; ++i) { u += y[i]; ud += y[m + i]; }
    double F = orc_force(c->force, th, c->Zc + u, ud);
    for (int i = 0; i < m; ++i) {
        f[i] = y[m + i];
        f[m + i] = F / md->mass + md->gam[i] * g - md->w[i] * md->w[i] * y[i]
                   - (md->w[i] / c->Q[i]) * y[m + i];
    }
}

/* Classic RK4 (Sec. 3.2) over n_steps record steps, each split into `sub`
 * equal sub-steps (sub = 1: the solver's own step; sub = 4: the finer step of
 * the synthetic records, reading R10).  u[n] = tip deflection at the end of
 * record step n + 1.  state (optional) receives [n_steps + 1][2m] modal states
 * at the record instants, starting with t = 0. */
int orc_forward(const orc_case* c, const double th[ORC_NSLOT], int n_steps, int sub,
                double* u, double* state)
{
    orc_case cf = *c;
    cf.spc = c->spc * sub;
    cf.dt = c->dt / sub;
    orc_modal md;
    if (orc_setup(&cf, &md)) return -1;
    int m = md.m, n2 = 2 * m;
    /* deflection points: tip-normalised mode shapes phi_i(xi_k) */
    int np = c->n_points;
    double phi[4][ORC_MAXM];
    if (np < 0 || np > 4 || (np > 0 && c->model != ORC_MODAL_EB)) return -1;
    if (np > 0) {
        double bL[ORC_MAXM], gam[ORC_MAXM];
        if (orc_modal_factors(m, 501, bL, gam, NULL, NULL)) return -1;
        for (int k = 0; k < np; ++k)
            for (int i = 0; i < m; ++i)
                phi[k][i] = orc_mode_shape(bL[i], c->point_xi[k]) / orc_mode_shape(bL[i], 1.0);
    }
    double y[2 * ORC_MAXM], k1[2 * ORC_MAXM], k2[2 * ORC_MAXM], k3[2 * ORC_MAXM],
        k4[2 * ORC_MAXM], yt[2 * ORC_MAXM];
    for (int i = 0; i < m; ++i) { y[i] = md.eta0[i]; y[m + i] = md.etad0[i]; }
    if (state) memcpy(state, y, sizeof(double) * n2);
    double h = md.dt;
    long step = 0;
    for (int n = 0; n < n_steps; ++n) {
        for (int s = 0; s < sub; ++s, ++step) {
            double g0, gh, g1;
            if (c->drive == 1) {
                double t = (double)step * h;
                g0 = orc_drive_chirp(th, t);
                gh = orc_drive_chirp(th, t + 0.5 * h);
                g1 = orc_drive_chirp(th, t + h);
            } else {
                g0 = orc_drive_half(&md, cf.spc, 2 * step);
                gh = orc_drive_half(&md, cf.spc, 2 * step + 1);
                g1 = orc_drive_half(&md, cf.spc, 2 * step + 2);
            }
            rhs(&cf, &md, th, g0, y, k1);
            for (int q = 0; q < n2; ++q) yt[q] = y[q] + 0.5 * h * k1[q];
            rhs(&cf, &md, th, gh, yt, k2);
            for (int q = 0; q < n2; ++q) yt[q] = y[q] + 0.5 * h * k2[q];
            rhs(&cf, &md, th, gh, yt, k3);
            for (int q = 0; q < n2; ++q) yt[q] = y[q] + h * k3[q];
            rhs(&cf, &md, th, g1, yt, k4);
            for (int q = 0; q < n2; ++q)
                y[q] = y[q] + (h / 6.0) * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
        }
        if (np > 0) {
            for (int k = 0; k < np; ++k) {
                double uk = 0.0;
                for (int i = 0; i < m; ++i) uk += phi[k][i] * y[i];
                u[(size_t)n * np + k] = uk;
            }
        } else {
            double tip = 0.0;
            for (int i = 0; i < m; ++i) tip += y[i];
            u[n] = tip;
        }
        if (state) memcpy(state + (size_t)(n + 1) * n2, y, sizeof(double) * n2);
    }
    return 0;
}

/* Eq. 5 on the sampled record (reading R8): S = sum_n (U_n - u_n)^2, so that
 * J^2 = dt * S. */
double orc_misfit(const double* U, const double* u, int n)
{
    double S = 0.0;
    for (int j = 0; j < n; ++j) S += (U[j] - u[j]) * (U[j] - u[j]);
    return S;
}

/* Normalised coordinates x in [0,1]^D -> physical slots (reading R12):
 * log10-linear for log dims, linear otherwise. */
void orc_map(const orc_pmap* pm, const double* x, double th[ORC_NSLOT])
{
    for (int s = 0; s < ORC_NSLOT; ++s) th[s] = pm->fixed[s];
    for (int d = 0; d < pm->D; ++d) {
        double lo = pm->lo[d], hi = pm->hi[d];
        if (pm->logs[d])
            th[pm->slot[d]] = pow(10.0, log10(lo) + x[d] * (log10(hi) - log10(lo)));
        else
            th[pm->slot[d]] = lo + x[d] * (hi - lo);
    }
}

int orc_fe_forward(const orc_case* c, const double th[ORC_NSLOT], int n_steps, int sub, double* u,
                   double* setup_out);

static int forward_any(const orc_case* c, const double th[ORC_NSLOT], int n, double* u)
{
    if (c->model == ORC_FE_HERMITE) return c->n_points ? -1 : orc_fe_forward(c, th, n, 1, u, NULL);
    return orc_forward(c, th, n, 1, u, NULL);
}

int orc_misfit_x(const orc_case* c, const orc_pmap* pm, const double* x,
                 const double* U, int n, double* S)
{
    double th[ORC_NSLOT];
    orc_map(pm, x, th);
    const int nv = n * (c->n_points > 0 ? c->n_points : 1);   /* record values */
    double* u = (double*)malloc(sizeof(double) * nv);
    int rc = forward_any(c, th, n, u);
    *S = rc ? INFINITY : orc_misfit(U, u, nv);
    free(u);
    return rc;
}

/* Misfit of P candidates; x is [D][P] (dimension-major). Non-finite -> +inf. */
int orc_misfit_batch(const orc_case* c, const orc_pmap* pm, const double* x,
                     int P, const double* U, int n, double* S)
{
    int D = pm->D, bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads) reduction(+ : bad)
#endif
    for (int p = 0; p < P; ++p) {
        double xp[5];
        for (int d = 0; d < D; ++d) xp[d] = x[(size_t)d * P + p];
        double s;
        bad += orc_misfit_x(c, pm, xp, U, n, &s) != 0;
        S[p] = isfinite(s) ? s : INFINITY;
    }
    return bad ? -1 : 0;
}

/* ======================================================================== */
/* Particle swarm (Sec. 3.4, Eq. 8; reading R12).                           */
/* Counter words: (particle, iteration, pixel, tag<<16 | block);            */
/* tags 0 = initial x, 1 = initial v, 2 = r1/r2.                            */
/* ======================================================================== */
/* Particles p0 .. p0 + P - 1 of a swarm (a slice of it; the counters carry
 * the swarm-wide index), stored as columns 0 .. P - 1. */
void orc_pso_init_slice(int P, int p0, int D, uint64_t seed, uint32_t pixel, double* x, double* v)
{
    for (int p = 0; p < P; ++p)
        for (int d = 0; d < D; ++d) {
            const uint32_t id = (uint32_t)(p0 + p);
            double u0 = orc_draw(seed, id, 0, pixel, 0, (uint32_t)(d / 4), d % 4);
            double u1 = orc_draw(seed, id, 0, pixel, 1, (uint32_t)(d / 4), d % 4);
            x[(size_t)d * P + p] = u0;
            v[(size_t)d * P + p] = (u1 - u0) / 2.0;
        }
}

void orc_pso_init(int P, int D, uint64_t seed, uint32_t pixel, double* x, double* v)
{
    orc_pso_init_slice(P, 0, D, seed, pixel, x, v);
}

/* Eq. 8: v <- w v + c1 r1 (b_l - x) + c2 r2 (b_g - x); x <- x + v; a
 * coordinate that leaves [0, 1] is put on the bound and its velocity zeroed.
 * r1, r2 per particle and dimension: words 2d and 2d+1 of the tag-2 stream. */
void orc_pso_update_slice(int P, int p0, int D, uint32_t it, uint64_t seed, uint32_t pixel,
                          double w, double c1, double c2, double* x, double* v,
                          const double* pbest_x, const double* gbest_x)
{
    for (int p = 0; p < P; ++p)
        for (int d = 0; d < D; ++d) {
            size_t q = (size_t)d * P + p;
            uint32_t blk = (uint32_t)((2 * d) / 4);
            const uint32_t id = (uint32_t)(p0 + p);
            double r1 = orc_draw(seed, id, it, pixel, 2, blk, (2 * d) % 4);
            double r2 = orc_draw(seed, id, it, pixel, 2, blk, (2 * d + 1) % 4);
            double vn = w * v[q] + c1 * r1 * (pbest_x[q] - x[q]) + c2 * r2 * (gbest_x[d] - x[q]);
            double xn = x[q] + vn;
            if (xn < 0.0) { xn = 0.0; vn = 0.0; }
            if (xn > 1.0) { xn = 1.0; vn = 0.0; }
            x[q] = xn;
            v[q] = vn;
        }
}

void orc_pso_update(int P, int D, uint32_t it, uint64_t seed, uint32_t pixel,
                    double w, double c1, double c2, double* x, double* v,
                    const double* pbest_x, const double* gbest_x)
{
    orc_pso_update_slice(P, 0, D, it, seed, pixel, w, c1, c2, x, v, pbest_x, gbest_x);
}

static int argmin_first(const double* S, int P)
{
    int b = 0;
    for (int p = 1; p < P; ++p)
        if (S[p] < S[b]) b = p;
    return b;
}

/* Synchronous PSO: evaluate all, update personal bests (strictly better),
 * global best = lowest personal best (lowest index on ties), then move.
 * iters counts position updates: P * (iters + 1) forward solves.
 * hist (optional) receives the global-best misfit after each evaluation. */
int orc_invert(const orc_case* c, const orc_pmap* pm, const double* U, int n,
               const orc_pso* cfg, double* best_x, double* best_S, double* hist)
{
    int P = cfg->P, D = pm->D;
    size_t sz = (size_t)P * D;
    double* x = (double*)malloc(sizeof(double) * sz);
    double* v = (double*)malloc(sizeof(double) * sz);
    double* pb = (double*)malloc(sizeof(double) * sz);
    double* S = (double*)malloc(sizeof(double) * P);
    double* pbS = (double*)malloc(sizeof(double) * P);
    double gb[5];
    orc_pso_init(P, D, cfg->seed, cfg->pixel, x, v);
    orc_misfit_batch(c, pm, x, P, U, n, S);
    memcpy(pb, x, sizeof(double) * sz);
    memcpy(pbS, S, sizeof(double) * P);
    int g = argmin_first(pbS, P);
    for (int d = 0; d < D; ++d) gb[d] = pb[(size_t)d * P + g];
    if (hist) hist[0] = pbS[g];
    for (int it = 1; it <= cfg->iters; ++it) {
        orc_pso_update(P, D, (uint32_t)it, cfg->seed, cfg->pixel, cfg->w, cfg->c1, cfg->c2,
                       x, v, pb, gb);
        orc_misfit_batch(c, pm, x, P, U, n, S);
        for (int p = 0; p < P; ++p)
            if (S[p] < pbS[p]) {
                pbS[p] = S[p];
                for (int d = 0; d < D; ++d) pb[(size_t)d * P + p] = x[(size_t)d * P + p];
            }
        g = argmin_first(pbS, P);
        for (int d = 0; d < D; ++d) gb[d] = pb[(size_t)d * P + g];
        if (hist) hist[it] = pbS[g];
    }
    for (int d = 0; d < D; ++d) best_x[d] = gb[d];
    *best_S = pbS[g];
    free(x); free(v); free(pb); free(S); free(pbS);
    return 0;
}

/* ======================================================================== */
/* Synthetic records (reading R9-R11).                                       */
/* ======================================================================== */

/* Truth drawn from tag 3 in the interior [0.1, 0.9]^D of the cube. */
void orc_truth_x(int D, uint64_t seed, uint32_t pixel, double* x)
{
    for (int d = 0; d < D; ++d)
        x[d] = 0.1 + 0.8 * orc_draw(seed, 0, 0, pixel, 3, (uint32_t)(d / 4), d % 4);
}

/* Record length in drive cycles, uniform on the integers lo..hi: tag 3,
 * block 2, word 0, scaled by integer multiply-high. */
int orc_cycles(uint64_t seed, uint32_t pixel, int lo, int hi)
{
    uint32_t ctr[4] = {0, 0, pixel, (3u << 16) | 2u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    uint32_t span = (uint32_t)(hi - lo + 1);
    return lo + (int)(((uint64_t)out[0] * span) >> 32);
}

/* Record: tip deflection of the truth integrated at dt/sub, sampled every
 * `sub` fine steps, plus Gaussian noise of std sigma.  Noise sample n uses
 * the tag-4 counter (n/2, 0, pixel, 4<<16) and Box-Muller on words 0, 1:
 *   u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1],  u2 = (w1 >> 8) 2^-24,
 *   z = sqrt(-2 ln u1) * (cos 2 pi u2 for even n, sin 2 pi u2 for odd n). */
int orc_record(const orc_case* c, const orc_pmap* pm, const double* x, int n,
               int sub, double sigma, uint64_t seed, uint32_t pixel, double* U)
{
    double th[ORC_NSLOT];
    orc_map(pm, x, th);
    int rc = c->model == ORC_FE_HERMITE ? orc_fe_forward(c, th, n, sub, U, NULL)
                                        : orc_forward(c, th, n, sub, U, NULL);
    if (rc) return -1;
    if (sigma > 0.0) {
        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
        const int nv = n * (c->n_points > 0 ? c->n_points : 1);   /* record values */
        for (int j = 0; j < nv; ++j) {
            uint32_t ctr[4] = {(uint32_t)(j / 2), 0, pixel, 4u << 16};
            uint32_t out[4];
            orc_philox4x32_10(ctr, key, out);
            double u1 = ((double)(out[0] >> 8) + 1.0) * (1.0 / 16777216.0);
            double u2 = (double)(out[1] >> 8) * (1.0 / 16777216.0);
            double r = sqrt(-2.0 * log(u1));
            double z = (j % 2 == 0) ? r * cos(2.0 * M_PI * u2) : r * sin(2.0 * M_PI * u2);
            U[j] += sigma * z;
        }
    }
    return 0;
}

/* The complex-step paths cover the force-law slots of the steady drive. */
static int complex_step_unsupported(const orc_case* c, const orc_pmap* pm)
{
    if (c->drive != 0 || c->n_points != 0) return 1;
    for (int d = 0; d < pm->D; ++d)
        if (pm->slot[d] < 0 || pm->slot[d] >= 5) return 1;
    return 0;
}

/* ======================================================================== */
/* Complex-step gradient of S(x) (the oracle side of the adjoint check).     */
/* The whole forward solve is repeated in complex arithmetic with the        */
/* perturbation i*h on one coordinate; branches are taken on real parts.     */
/* ======================================================================== */
static double complex cforce(int kind, const double complex th[5], double complex d,
                             double complex ddot)
{
    switch (kind) {
    case ORC_F_LINEAR:
        return -th[0] * (d - th[1]);
    case ORC_F_DMT:
    case ORC_F_DMT_KV: {
        double complex E = th[0], H = th[1], R = th[2], a0 = th[3];
        if (creal(d) > creal(a0)) return -H * R / (6.0 * d * d);
        double complex delta = a0 - d;
        double complex F = (4.0 / 3.0) * E * csqrt(R) * delta * csqrt(delta)
                           - H * R / (6.0 * a0 * a0);
        if (kind == ORC_F_DMT_KV) F -= th[4] * csqrt(R * delta) * ddot;
        return F;
    }
    case ORC_F_HOOKE:
        return creal(d) < creal(th[1]) ? th[0] * (th[1] - d) : 0.0;
    case ORC_F_SPRING_DAMPER:
        return creal(d) < creal(th[1]) ? th[0] * (th[1] - d) - th[2] * ddot : 0.0;
    default:
        return 0.0;
    }
}

static void cmap(const orc_pmap* pm, const double complex* x, double complex th[5])
{
    for (int s = 0; s < 5; ++s) th[s] = pm->fixed[s];
    for (int d = 0; d < pm->D; ++d) {
        double lo = pm->lo[d], hi = pm->hi[d];
        if (pm->logs[d])
            th[pm->slot[d]] = cexp(log(10.0) * (log10(lo) + x[d] * (log10(hi) - log10(lo))));
        else
            th[pm->slot[d]] = lo + x[d] * (hi - lo);
    }
}

static double complex cmisfit(const orc_case* c, const orc_modal* md,
                              const double complex th[5], const double* U, int n)
{
    int m = md->m, n2 = 2 * m;
    double complex y[2 * ORC_MAXM], k[4][2 * ORC_MAXM], yt[2 * ORC_MAXM];
    for (int i = 0; i < m; ++i) { y[i] = md->eta0[i]; y[m + i] = md->etad0[i]; }
    double h = md->dt;
    double complex S = 0.0;
    for (int step = 0; step < n; ++step) {
        double g[3] = {orc_drive_half(md, c->spc, 2L * step),
                       orc_drive_half(md, c->spc, 2L * step + 1),
                       orc_drive_half(md, c->spc, 2L * step + 2)};
        const double cs[4] = {0.0, 0.5, 0.5, 1.0};
        const int gi[4] = {0, 1, 1, 2};
        for (int s = 0; s < 4; ++s) {
            for (int q = 0; q < n2; ++q) yt[q] = s == 0 ? y[q] : y[q] + cs[s] * h * k[s - 1][q];
            double complex u = 0.0, ud = 0.0;
            for (int i = 0; i < m; ++i) { u += yt[i]; ud += yt[m + i]; }
            double complex F = cforce(c->force, th, c->Zc + u, ud);
            for (int i = 0; i < m; ++i) {
                k[s][i] = yt[m + i];
                k[s][m + i] = F / md->mass + md->gam[i] * g[gi[s]]
                              - md->w[i] * md->w[i] * yt[i] - (md->w[i] / c->Q[i]) * yt[m + i];
            }
        }
        for (int q = 0; q < n2; ++q)
            y[q] = y[q] + (h / 6.0) * (k[0][q] + 2.0 * k[1][q] + 2.0 * k[2][q] + k[3][q]);
        double complex tip = 0.0;
        for (int i = 0; i < m; ++i) tip += y[i];
        S += (U[step] - tip) * (U[step] - tip);
    }
    return S;
}

static void grad_cs_serial(const orc_case* c, const orc_modal* md, const orc_pmap* pm,
                           const double* x, const double* U, int n, double* S, double* grad)
{
    const double h = 1e-30;
    int D = pm->D;
    for (int d = 0; d < D; ++d) {
        double complex xc[5], th[5];
        for (int e = 0; e < D; ++e) xc[e] = x[e] + (e == d ? I * h : 0.0);
        cmap(pm, xc, th);
        double complex Sc = cmisfit(c, md, th, U, n);
        grad[d] = cimag(Sc) / h;
        if (d == 0) *S = creal(Sc);
    }
}

/* dS/dx_d = Im S(x + i h e_d) / h with h = 1e-30 (no subtractive error). */
int orc_grad_cs(const orc_case* c, const orc_pmap* pm, const double* x,
                const double* U, int n, double* S, double* grad)
{
    if (complex_step_unsupported(c, pm)) return -1;
    orc_modal md;
    if (orc_setup(c, &md)) return -1;
    const double h = 1e-30;
    int D = pm->D;
    double Sr = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
    for (int d = 0; d < D; ++d) {
        double complex xc[5], th[5];
        for (int e = 0; e < D; ++e) xc[e] = x[e] + (e == d ? I * h : 0.0);
        cmap(pm, xc, th);
        double complex Sc = cmisfit(c, &md, th, U, n);
        grad[d] = cimag(Sc) / h;
        if (d == 0) Sr = creal(Sc);
    }
    *S = Sr;
    return 0;
}

/* ======================================================================== */
/* Gradient polish of K candidates (reading R14): projected steepest descent */
/* in the normalised cube.  Per step and candidate: g = dS/dx (complex step), */
/* direction -g / max|g_d|, trial points clamp(x + alpha_j dir) for           */
/* alpha_j = alpha0 shrink^j (j < n_cand); the largest step meeting the       */
/* Armijo condition S(x_j) <= S(x) + sigma g.(x_j - x) is taken, else x stays.*/
/* x is [D][K]; S [K] receives the final misfits.                             */
/* ======================================================================== */
int orc_polish(const orc_case* c, const orc_pmap* pm, const double* U, int n, double* x, int K,
               int steps, int n_cand, double alpha0, double shrink, double sigma, double* S)
{
    if (complex_step_unsupported(c, pm)) return -1;
    orc_modal md;
    if (orc_setup(c, &md)) return -1;
    int D = pm->D;
    double* g = (double*)malloc(sizeof(double) * (size_t)D * K);
    double* Xc = (double*)malloc(sizeof(double) * (size_t)D * K * n_cand);
    double* Sc = (double*)malloc(sizeof(double) * (size_t)K * n_cand);
    int KJ = K * n_cand;
    for (int st = 0; st <= steps; ++st) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
        for (int k = 0; k < K; ++k) {
            double xk[5], gk[5], Sk = 0.0;
            for (int d = 0; d < D; ++d) xk[d] = x[(size_t)d * K + k];
            grad_cs_serial(c, &md, pm, xk, U, n, &Sk, gk);
            S[k] = Sk;
            for (int d = 0; d < D; ++d) g[(size_t)d * K + k] = gk[d];
        }
        if (st == steps) break;
        for (int k = 0; k < K; ++k) {
            double gmax = 0.0;
            for (int d = 0; d < D; ++d) gmax = fmax(gmax, fabs(g[(size_t)d * K + k]));
            for (int j = 0; j < n_cand; ++j) {
                double alpha = alpha0 * pow(shrink, j);
                for (int d = 0; d < D; ++d) {
                    double xd = x[(size_t)d * K + k];
                    double step = gmax > 0.0 ? -alpha * g[(size_t)d * K + k] / gmax : 0.0;
                    double xn = xd + step;
                    if (xn < 0.0) xn = 0.0;
                    if (xn > 1.0) xn = 1.0;
                    Xc[(size_t)d * KJ + (size_t)k * n_cand + j] = xn;
                }
            }
        }
        orc_misfit_batch(c, pm, Xc, KJ, U, n, Sc);
        for (int k = 0; k < K; ++k) {
            for (int j = 0; j < n_cand; ++j) {
                double lin = 0.0;
                for (int d = 0; d < D; ++d)
                    lin += g[(size_t)d * K + k] *
                           (Xc[(size_t)d * KJ + (size_t)k * n_cand + j] - x[(size_t)d * K + k]);
                double Sj = Sc[(size_t)k * n_cand + j];
                if (Sj <= S[k] + sigma * lin && lin < 0.0) {
                    for (int d = 0; d < D; ++d)
                        x[(size_t)d * K + k] = Xc[(size_t)d * KJ + (size_t)k * n_cand + j];
                    break;
                }
            }
        }
    }
    free(g);
    free(Xc);
    free(Sc);
    return 0;
}

/* ======================================================================== */
/* Finite-element cantilever (reading R13): cubic Hermite Euler-Bernoulli    */
/* elements, consistent mass, clamped node removed; Rayleigh damping with Q */
/* on modes 1 and 2; Newmark beta = 1/4, gamma = 1/2 in the displacement-    */
/* only three-term form                                                      */
/*   S u_{n+1} = (2M - h^2/2 K) u_n - (M - h/2 C + h^2/4 K) u_{n-1}           */
/*               + h^2/4 (f_{n+1} + 2 f_n + f_{n-1}),                         */
/*   S = M + h/2 C + h^2/4 K,  f = M r g + e_tip F_ts,                        */
/* g = -(base acceleration), r = 1 on deflection DOFs; the tip force at step */
/* n+1 is implicit and found by Newton on the tip deflection.                */
/* ======================================================================== */
#define ORC_FE_MAXN 128

typedef struct {
    int n;                        /* DOFs = 2 n_elem                         */
    double M[ORC_FE_MAXN * ORC_FE_MAXN], K[ORC_FE_MAXN * ORC_FE_MAXN],
        C[ORC_FE_MAXN * ORC_FE_MAXN];
    double w1, w2;                /* first two natural frequencies [rad/s]   */
    double alpha, beta;           /* Rayleigh coefficients                   */
    double thick, width, mu;      /* derived section                          */
} orc_fe_mats;

/* Dense LU with partial pivoting (in place), and its solve. */
static int lu_factor(double* A, int n, int* piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0) return -1;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
        for (int i = k + 1; i < n; ++i) {
            A[i * n + k] /= A[k * n + k];
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(const double* LU, int n, const int* piv, double* b)
{
    for (int k = 0; k < n; ++k) {
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

/* Complex dense solve by Gaussian elimination with partial pivoting. */
static int csolve(double complex* A, int n, double complex* b)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (cabs(A[i * n + k]) > cabs(A[p * n + k])) p = i;
        if (cabs(A[p * n + k]) == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double complex t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
            double complex t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double complex f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) b[i] -= A[i * n + j] * b[j];
        b[i] /= A[i * n + i];
    }
    return 0;
}

/* Eigenvalues of the symmetric matrix A (n x n, destroyed) by cyclic Jacobi
 * rotations; returned in ascending order in ev. */
static void jacobi_eig(double* A, int n, double* ev)
{
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (fabs(apq) < 1e-300) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (ev[j] < ev[i]) { double t = ev[i]; ev[i] = ev[j]; ev[j] = t; }
}

int orc_fe_dofs(const orc_case* c) { return 2 * c->n_elem; }

/* Double-double accumulation (hi + lo): s += a, and s += a * b exactly
 * before the final rounding of each partial sum (Knuth's two-sum, the
 * product's error from one fma). */
static void dd_add(double* hi, double* lo, double a)
{
    double s = *hi + a;
    double z = s - *hi;
    double e = (*hi - (s - z)) + (a - z);
    e += *lo;
    *hi = s + e;
    *lo = e - (*hi - s);
}

static void dd_add_prod(double* hi, double* lo, double a, double b)
{
    double p = a * b;
    dd_add(hi, lo, p);
    dd_add(hi, lo, fma(a, b, -p));
}

/* phi^T A phi in double-double: y = A phi row by row, then phi . y. */
static double dd_quad(const double* A, int n, const double* phi, double* lo_out)
{
    double hi = 0.0, lo = 0.0;
    for (int i = 0; i < n; ++i) {
        double yh = 0.0, yl = 0.0;
        for (int j = 0; j < n; ++j) dd_add_prod(&yh, &yl, A[i * n + j], phi[j]);
        dd_add_prod(&hi, &lo, phi[i], yh);
        dd_add_prod(&hi, &lo, phi[i], yl);
    }
    *lo_out = lo;
    return hi;
}

/* Reading R13 drives the beam at its own first frequency.  An FP64
 * eigensolver fixes the lowest eigenvalues of K x = w^2 M x only to about
 * eps * lambda_max / lambda (a few 1e-9 for 32 elements), and the resonant
 * response (Q = 400) turns that into ~1e-6 of the deflection over 50
 * cycles.  So each eigenvalue in use is refined: its eigenvector by inverse
 * iteration at the solver's value, then the Rayleigh quotient
 * phi^T K phi / phi^T M phi with both forms summed in double-double, exact
 * to rounding (the quotient's error is quadratic in the eigenvector's). */
static double rayleigh_refined(const orc_fe_mats* fe, double sigma)
{
    int n = fe->n;
    double* A = (double*)malloc(sizeof(double) * n * n);
    int* piv = (int*)malloc(sizeof(int) * n);
    double* x = (double*)malloc(sizeof(double) * n);
    double* y = (double*)malloc(sizeof(double) * n);
    double shift = sigma;
    for (int tries = 0; tries < 8; ++tries) {
        for (int i = 0; i < n * n; ++i) A[i] = fe->K[i] - shift * fe->M[i];
        if (lu_factor(A, n, piv) == 0) break;
        shift = sigma * (1.0 - 1e-12 * (double)(tries + 1));   /* exactly singular: step off */
    }
    for (int i = 0; i < n; ++i) x[i] = 1.0;
    for (int it = 0; it < 4; ++it) {
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int j = 0; j < n; ++j) t += fe->M[i * n + j] * x[j];
            y[i] = t;
        }
        lu_solve(A, n, piv, y);
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm = fmax(nrm, fabs(y[i]));
        for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    double kl, ml;
    double kh = dd_quad(fe->K, n, x, &kl);
    double mh = dd_quad(fe->M, n, x, &ml);
    double lam = kh / mh;
    lam += lam * (kl / kh - ml / mh);
    free(A); free(piv); free(x); free(y);
    return lam;
}

/* Section from the targets: 3 E I / L^3 = k and the Euler-Bernoulli first
 * frequency (beta_1 L)^2 sqrt(E I / (mu L^4)) = 2 pi f1; rho A = mu. */
static int fe_build(const orc_case* c, orc_fe_mats* fe)
{
    int ne = c->n_elem, n = 2 * ne;
    if (ne < 1 || n > ORC_FE_MAXN) return -1;
    double L = c->L, E = c->E;
    double Iz = c->fe_k * L * L * L / (3.0 * E);
    double b1 = orc_beam_root(1) / L;
    double w1t = 2.0 * M_PI * c->fe_f1;
    double mu = E * Iz * pow(b1, 4) / (w1t * w1t);
    double A = mu / c->rho;
    fe->thick = sqrt(12.0 * Iz / A);
    fe->width = A / fe->thick;
    fe->mu = mu;
    fe->n = n;
    double h = L / ne;
    int N2 = n + 2;   /* with the clamped node */
    double* Mf = (double*)calloc((size_t)N2 * N2, sizeof(double));
    double* Kf = (double*)calloc((size_t)N2 * N2, sizeof(double));
    const double me[16] = {156, 22 * h, 54, -13 * h, 22 * h, 4 * h * h, 13 * h, -3 * h * h,
                           54, 13 * h, 156, -22 * h, -13 * h, -3 * h * h, -22 * h, 4 * h * h};
    const double ke[16] = {12, 6 * h, -12, 6 * h, 6 * h, 4 * h * h, -6 * h, 2 * h * h,
                           -12, -6 * h, 12, -6 * h, 6 * h, 2 * h * h, -6 * h, 4 * h * h};
    double ms = mu * h / 420.0, ks = E * Iz / (h * h * h);
    for (int e = 0; e < ne; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                int ga = 2 * e + a, gb = 2 * e + b;
                Mf[ga * N2 + gb] += ms * me[a * 4 + b];
                Kf[ga * N2 + gb] += ks * ke[a * 4 + b];
            }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            fe->M[i * n + j] = Mf[(i + 2) * N2 + (j + 2)];
            fe->K[i * n + j] = Kf[(i + 2) * N2 + (j + 2)];
        }
    free(Mf);
    free(Kf);
    /* generalized eigenvalues of K x = w^2 M x via Cholesky M = L L^T */
    double* Lc = (double*)calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s2 = fe->M[i * n + j];
            for (int k = 0; k < j; ++k) s2 -= Lc[i * n + k] * Lc[j * n + k];
            if (i == j) {
                if (s2 <= 0) { free(Lc); return -1; }
                Lc[i * n + i] = sqrt(s2);
            } else {
                Lc[i * n + j] = s2 / Lc[j * n + j];
            }
        }
    /* B = L^-1 K L^-T */
    double* T = (double*)calloc((size_t)n * n, sizeof(double));
    double* B = (double*)calloc((size_t)n * n, sizeof(double));
    for (int col = 0; col < n; ++col)     /* T = L^-1 K (column by column) */
        for (int i = 0; i < n; ++i) {
            double s2 = fe->K[i * n + col];
            for (int k = 0; k < i; ++k) s2 -= Lc[i * n + k] * T[k * n + col];
            T[i * n + col] = s2 / Lc[i * n + i];
        }
    for (int row = 0; row < n; ++row)     /* B = T L^-T: solve L B^T = T^T */
        for (int i = 0; i < n; ++i) {
            double s2 = T[row * n + i];
            for (int k = 0; k < i; ++k) s2 -= Lc[i * n + k] * B[row * n + k];
            B[row * n + i] = s2 / Lc[i * n + i];
        }
    double* ev = (double*)malloc(sizeof(double) * n);
    jacobi_eig(B, n, ev);
    fe->w1 = sqrt(rayleigh_refined(fe, ev[0]));
    fe->w2 = n > 1 ? sqrt(rayleigh_refined(fe, ev[1])) : 3.0 * fe->w1;
    free(ev); free(B); free(T); free(Lc);
    /* Rayleigh: 1/(2Q) = alpha/(2 w_i) + beta w_i / 2, i = 1, 2 */
    double z = 1.0 / (2.0 * c->fe_Q);
    fe->beta = 2.0 * z / (fe->w1 + fe->w2);
    fe->alpha = fe->beta * fe->w1 * fe->w2;
    for (int i = 0; i < n * n; ++i) fe->C[i] = fe->alpha * fe->M[i] + fe->beta * fe->K[i];
    return 0;
}

/* Geometry and frequencies of the FE model: geom = (thickness, width, mu,
 * w1, w2, alpha, beta); M, K, C (n x n) if non-NULL. */
int orc_fe_matrices(const orc_case* c, double* M, double* K, double* C, double* w12,
                    double* geom)
{
    orc_fe_mats* fe = (orc_fe_mats*)malloc(sizeof(orc_fe_mats));
    if (fe_build(c, fe)) { free(fe); return -1; }
    int n = fe->n;
    if (M) memcpy(M, fe->M, sizeof(double) * n * n);
    if (K) memcpy(K, fe->K, sizeof(double) * n * n);
    if (C) memcpy(C, fe->C, sizeof(double) * n * n);
    if (w12) { w12[0] = fe->w1; w12[1] = fe->w2; }
    if (geom) {
        geom[0] = fe->thick; geom[1] = fe->width; geom[2] = fe->mu;
        geom[3] = fe->w1; geom[4] = fe->w2; geom[5] = fe->alpha; geom[6] = fe->beta;
    }
    free(fe);
    return 0;
}

/* d F / d d for the tip-force laws without rate dependence. */
static double force_slope(int kind, const double th[ORC_NSLOT], double d)
{
    switch (kind) {
    case ORC_F_LINEAR:
        return -th[0];
    case ORC_F_DMT: {
        double H = th[1], R = th[2], a0 = th[3];
        if (d > a0) return H * R / (3.0 * d * d * d);
        return -1.5 * (4.0 / 3.0) * th[0] * sqrt(R) * sqrt(a0 - d);
    }
    case ORC_F_HOOKE:
        return d < th[1] ? -th[0] : 0.0;
    default:
        return 0.0;
    }
}

/* FE forward solve: u[n] = tip deflection after step n+1 (record steps of
 * h = 1 / (f_1 spc) with f_1 the FE model's own first frequency, each split
 * into `sub` Newmark steps).  setup_out (optional, 8 values): w1, w2, alpha,
 * beta, a, psi, h, thickness. */
int orc_fe_forward(const orc_case* c, const double th[ORC_NSLOT], int n_steps, int sub, double* u,
                   double* setup_out)
{
    if (c->drive != 0) return -1;
    if (c->force == ORC_F_DMT_KV || c->force == ORC_F_SPRING_DAMPER) return -1;
    orc_fe_mats* fe = (orc_fe_mats*)malloc(sizeof(orc_fe_mats));
    if (fe_build(c, fe)) { free(fe); return -1; }
    int n = fe->n, tip = n - 2;
    double w = fe->w1;
    int spc = c->spc * sub;
    double h = 2.0 * M_PI / (w * spc);
    double* r = (double*)calloc(n, sizeof(double));
    for (int i = 0; i < n; i += 2) r[i] = 1.0;
    double* Mr = (double*)calloc(n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Mr[i] += fe->M[i * n + j] * r[j];
    /* free steady state: (K - w^2 M + i w C) X = M r */
    double complex* Z = (double complex*)malloc(sizeof(double complex) * n * n);
    double complex* X = (double complex*)malloc(sizeof(double complex) * n);
    for (int i = 0; i < n * n; ++i) Z[i] = fe->K[i] - w * w * fe->M[i] + I * w * fe->C[i];
    for (int i = 0; i < n; ++i) X[i] = Mr[i];
    if (csolve(Z, n, X)) { free(Z); free(X); free(r); free(Mr); free(fe); return -1; }
    double a = c->A0 / (w * w * cabs(X[tip]));
    double psi = M_PI / 2.0 - carg(X[tip]);
    double* u0 = (double*)malloc(sizeof(double) * n);
    double* um = (double*)malloc(sizeof(double) * n);
    double* up = (double*)malloc(sizeof(double) * n);
    double* rhs = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) {
        u0[i] = cimag(a * w * w * X[i] * cexp(I * psi));
        um[i] = cimag(a * w * w * X[i] * cexp(I * (psi - w * h)));
    }
    /* S, its LU, and s = S^-1 e_tip */
    double* S = (double*)malloc(sizeof(double) * n * n);
    double* P1 = (double*)malloc(sizeof(double) * n * n);
    double* P2 = (double*)malloc(sizeof(double) * n * n);
    int* piv = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n * n; ++i) {
        S[i] = fe->M[i] + 0.5 * h * fe->C[i] + 0.25 * h * h * fe->K[i];
        P1[i] = 2.0 * fe->M[i] - 0.5 * h * h * fe->K[i];
        P2[i] = fe->M[i] - 0.5 * h * fe->C[i] + 0.25 * h * h * fe->K[i];
    }
    lu_factor(S, n, piv);
    double* s = (double*)calloc(n, sizeof(double));
    s[tip] = 1.0;
    lu_solve(S, n, piv, s);
    double q = 0.25 * h * h;
    double Fm = orc_force(c->force, th, c->Zc + um[tip], 0.0);
    double F0 = orc_force(c->force, th, c->Zc + u0[tip], 0.0);
    long step = 0;
    for (int nrec = 0; nrec < n_steps; ++nrec) {
        for (int f = 0; f < sub; ++f, ++step) {
            double gm = a * w * w * sin(w * h * (double)((step - 1 + spc) % spc) + psi);
            double g0 = a * w * w * sin(w * h * (double)(step % spc) + psi);
            double gp = a * w * w * sin(w * h * (double)((step + 1) % spc) + psi);
            double G = gp + 2.0 * g0 + gm;
            for (int i = 0; i < n; ++i) {
                double acc = q * (Mr[i] * G);
                for (int j = 0; j < n; ++j) acc += P1[i * n + j] * u0[j] - P2[i * n + j] * um[j];
                if (i == tip) acc += q * (2.0 * F0 + Fm);
                rhs[i] = acc;
            }
            lu_solve(S, n, piv, rhs);             /* rhs = S^-1 (known part) */
            /* tip: z = rhs_tip + q s_tip F(Zc + z), Newton */
            double z = rhs[tip];
            for (int it = 0; it < 60; ++it) {
                double Fz = orc_force(c->force, th, c->Zc + z, 0.0);
                double phi = z - rhs[tip] - q * s[tip] * Fz;
                double dphi = 1.0 - q * s[tip] * force_slope(c->force, th, c->Zc + z);
                double dz = phi / dphi;
                z -= dz;
                if (fabs(dz) <= 1e-15 * (fabs(z) + 1e-30)) break;
            }
            double Fp = orc_force(c->force, th, c->Zc + z, 0.0);
            for (int i = 0; i < n; ++i) up[i] = rhs[i] + q * s[i] * Fp;
            double* t = um; um = u0; u0 = up; up = t;
            Fm = F0;
            F0 = Fp;
        }
        u[nrec] = u0[tip];
    }
    if (setup_out) {
        setup_out[0] = fe->w1; setup_out[1] = fe->w2; setup_out[2] = fe->alpha;
        setup_out[3] = fe->beta; setup_out[4] = a; setup_out[5] = psi; setup_out[6] = h;
        setup_out[7] = fe->thick;
    }
    free(S); free(P1); free(P2); free(piv); free(s); free(u0); free(um); free(up); free(rhs);
    free(Z); free(X); free(r); free(Mr); free(fe);
    return 0;
}


/* ======================================================================== */
/* Normal equations of the misfit (reading R15).  The residual sensitivities */
/* a_nd = d u_n / d x_d come from the complex step applied to the whole      */
/* trajectory: u_n(x + i h e_d) = u_n + i h a_nd + O(h^2), h = 1e-30, with   */
/* branches taken on real parts (as cmisfit).                                */
/* ======================================================================== */
static void ctraj(const orc_case* c, const orc_modal* md, const double complex th[5], int n,
                  double complex* tip_out)
{
    int m = md->m, n2 = 2 * m;
    double complex y[2 * ORC_MAXM], k[4][2 * ORC_MAXM], yt[2 * ORC_MAXM];
    for (int i = 0; i < m; ++i) { y[i] = md->eta0[i]; y[m + i] = md->etad0[i]; }
    double h = md->dt;
    for (int step = 0; step < n; ++step) {
        double g[3] = {orc_drive_half(md, c->spc, 2L * step),
                       orc_drive_half(md, c->spc, 2L * step + 1),
                       orc_drive_half(md, c->spc, 2L * step + 2)};
        const double cs[4] = {0.0, 0.5, 0.5, 1.0};
        const int gi[4] = {0, 1, 1, 2};
        for (int s = 0; s < 4; ++s) {
            for (int q = 0; q < n2; ++q) yt[q] = s == 0 ? y[q] : y[q] + cs[s] * h * k[s - 1][q];
            double complex u = 0.0, ud = 0.0;
            for (int i = 0; i < m; ++i) { u += yt[i]; ud += yt[m + i]; }
            double complex F = cforce(c->force, th, c->Zc + u, ud);
            for (int i = 0; i < m; ++i) {
                k[s][i] = yt[m + i];
                k[s][m + i] = F / md->mass + md->gam[i] * g[gi[s]]
                              - md->w[i] * md->w[i] * yt[i] - (md->w[i] / c->Q[i]) * yt[m + i];
            }
        }
        for (int q = 0; q < n2; ++q)
            y[q] = y[q] + (h / 6.0) * (k[0][q] + 2.0 * k[1][q] + 2.0 * k[2][q] + k[3][q]);
        double complex tip = 0.0;
        for (int i = 0; i < m; ++i) tip += y[i];
        tip_out[step] = tip;
    }
}

static int normal_eq_serial(const orc_case* c, const orc_modal* md, const orc_pmap* pm,
                            const double* x, const double* U, int n, double* S, double* H,
                            double* b, int parallel)
{
    const double hs = 1e-30;
    int D = pm->D;
    double complex* ut = (double complex*)malloc(sizeof(double complex) * (size_t)n * D);
    if (!ut) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads) if (parallel)
#endif
    for (int d = 0; d < D; ++d) {
        double complex xc[5], th[5];
        for (int e = 0; e < D; ++e) xc[e] = x[e] + (e == d ? I * hs : 0.0);
        cmap(pm, xc, th);
        ctraj(c, md, th, n, ut + (size_t)d * n);
    }
    (void)parallel;
    double Sr = 0.0;
    for (int i = 0; i < D * D; ++i) H[i] = 0.0;
    for (int d = 0; d < D; ++d) b[d] = 0.0;
    for (int t = 0; t < n; ++t) {
        double r = U[t] - creal(ut[t]);
        double a[5];
        for (int d = 0; d < D; ++d) a[d] = cimag(ut[(size_t)d * n + t]) / hs;
        Sr += r * r;
        for (int d = 0; d < D; ++d) {
            b[d] += a[d] * r;
            for (int e = 0; e < D; ++e) H[d * D + e] += a[d] * a[e];
        }
    }
    *S = Sr;
    free(ut);
    return 0;
}

int orc_normal_eq(const orc_case* c, const orc_pmap* pm, const double* x, const double* U,
                  int n, double* S, double* H, double* b)
{
    if (complex_step_unsupported(c, pm)) return -1;
    orc_modal md;
    if (orc_setup(c, &md)) return -1;
    return normal_eq_serial(c, &md, pm, x, U, n, S, H, b, 1);
}

/* ======================================================================== */
/* Levenberg-Marquardt polish of K candidates (reading R15); see the header. */
/* ======================================================================== */
int orc_lm_polish(const orc_case* c, const orc_pmap* pm, const double* U, int n, double* x,
                  int K, int steps, int n_lambda, double lam0, double lam_ratio, double* S)
{
    if (complex_step_unsupported(c, pm)) return -1;
    orc_modal md;
    if (orc_setup(c, &md)) return -1;
    int D = pm->D, J = n_lambda, KJ = K * n_lambda;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)D * KJ);
    double* Sc = (double*)malloc(sizeof(double) * (size_t)KJ);
    if (!Xc || !Sc) { free(Xc); free(Sc); return -1; }
    int rc = 0;
    for (int st = 0; st < steps && rc == 0; ++st) {
        for (int k = 0; k < K; ++k) {
            double xk[5], H[25], b[5], Sk = 0.0;
            for (int d = 0; d < D; ++d) xk[d] = x[(size_t)d * K + k];
            if (normal_eq_serial(c, &md, pm, xk, U, n, &Sk, H, b, 1)) { rc = -1; break; }
            S[k] = Sk;
            double hmax = 0.0;
            for (int d = 0; d < D; ++d) hmax = fmax(hmax, H[d * D + d]);
            for (int j = 0; j < J; ++j) {
                double lam = lam0 * pow(lam_ratio, j);
                double A[25], delta[5];
                int piv[5];
                for (int d = 0; d < D; ++d) {
                    for (int e = 0; e < D; ++e) A[d * D + e] = H[d * D + e];
                    A[d * D + d] += lam * fmax(H[d * D + d], 1e-12 * hmax);
                    delta[d] = b[d];
                }
                int ok = hmax > 0.0 && lu_factor(A, D, piv) == 0;
                if (ok) lu_solve(A, D, piv, delta);
                for (int d = 0; d < D; ++d) {
                    double xn = xk[d] + (ok ? delta[d] : 0.0);
                    if (!(xn > 0.0)) xn = 0.0;   /* also a NaN step */
                    if (xn > 1.0) xn = 1.0;
                    Xc[(size_t)d * KJ + (size_t)k * J + j] = xn;
                }
            }
        }
        if (rc) break;
        orc_misfit_batch(c, pm, Xc, KJ, U, n, Sc);
        for (int k = 0; k < K; ++k) {
            int jb = argmin_first(Sc + (size_t)k * J, J);
            if (Sc[(size_t)k * J + jb] < S[k])
                for (int d = 0; d < D; ++d)
                    x[(size_t)d * K + k] = Xc[(size_t)d * KJ + (size_t)k * J + jb];
        }
    }
    if (rc == 0) orc_misfit_batch(c, pm, x, K, U, n, S);
    free(Xc);
    free(Sc);
    return rc;
}


/* ======================================================================== */
/* Swarm inside a box, with seed particles (reading R17: the cross-pixel     */
/* warm start of image scans).  The swarm of Eq. 8 moves in box-local        */
/* coordinates y in [0, 1]^D; a particle's parameters are x = lo + y (hi -   */
/* lo) in the normalised cube.  Particles p < n_seed start at the seed points */
/* (seeds [n_seed][D], normalised, clamped into the box) with zero velocity;  */
/* the others start as in orc_pso_init.  best_x is returned in the cube.      */
/* ======================================================================== */
int orc_invert_boxed(const orc_case* c, const orc_pmap* pm, const double* U, int n,
                     const orc_pso* cfg, const double* lo, const double* hi,
                     const double* seeds, int n_seed, double* best_x, double* best_S)
{
    int P = cfg->P, D = pm->D;
    size_t sz = (size_t)P * D;
    double* y = (double*)malloc(sizeof(double) * sz);
    double* v = (double*)malloc(sizeof(double) * sz);
    double* pb = (double*)malloc(sizeof(double) * sz);
    double* X = (double*)malloc(sizeof(double) * sz);
    double* S = (double*)malloc(sizeof(double) * P);
    double* pbS = (double*)malloc(sizeof(double) * P);
    if (!y || !v || !pb || !X || !S || !pbS) {
        free(y); free(v); free(pb); free(X); free(S); free(pbS);
        return -1;
    }
    double gb[5];
    orc_pso_init(P, D, cfg->seed, cfg->pixel, y, v);
    for (int p = 0; p < n_seed && p < P; ++p)
        for (int d = 0; d < D; ++d) {
            double t = (seeds[(size_t)p * D + d] - lo[d]) / (hi[d] - lo[d]);
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            y[(size_t)d * P + p] = t;
            v[(size_t)d * P + p] = 0.0;
        }
    for (int it = 0; it <= cfg->iters; ++it) {
        if (it > 0)
            orc_pso_update(P, D, (uint32_t)it, cfg->seed, cfg->pixel, cfg->w, cfg->c1, cfg->c2,
                           y, v, pb, gb);
        for (int d = 0; d < D; ++d)
            for (int p = 0; p < P; ++p)
                X[(size_t)d * P + p] = lo[d] + y[(size_t)d * P + p] * (hi[d] - lo[d]);
        orc_misfit_batch(c, pm, X, P, U, n, S);
        for (int p = 0; p < P; ++p)
            if (it == 0 || S[p] < pbS[p]) {
                pbS[p] = S[p];
                for (int d = 0; d < D; ++d) pb[(size_t)d * P + p] = y[(size_t)d * P + p];
            }
        int g = argmin_first(pbS, P);
        for (int d = 0; d < D; ++d) gb[d] = pb[(size_t)d * P + g];
        *best_S = pbS[g];
    }
    for (int d = 0; d < D; ++d) best_x[d] = lo[d] + gb[d] * (hi[d] - lo[d]);
    free(y); free(v); free(pb); free(X); free(S); free(pbS);
    return 0;
}
