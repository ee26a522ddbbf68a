/*
 * afm_oracle.h -- FP64 CPU oracle for the tip-sample force inversion of
 * Busch, Zou & Ganapathysubramanian, "A near real-time framework for
 * extracting tip-sample forces in dynamic AFM" (arXiv 1109.0334).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is a plain, slow, obviously correct
 * restatement of the method in double precision and SI units.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Citations name the paper's section / equation.  Readings of passages the
 * paper leaves open are labelled R1..R17 and listed in the repository's
 * design notes.
 *
 * Parity status per function:
 *   orc_philox4x32_10      pinned (cuRAND host generator, same published function)
 *   orc_beam_root          pinned (textbook roots of cos x cosh x + 1 = 0)
 *   orc_mode_shape         pinned (clamped/free end conditions, orthogonality)
 *   orc_modal_factors      pinned (closed-form gamma_i, L/4 modal mass, App. A f1
 *                                  and steady amplitude)
 *   orc_setup              pinned (free steady state = closed-form transfer)
 *   orc_forward            pinned (linear-spring closed form, matrix exponential,
 *                                  energy balance, step-halving order)
 *   orc_misfit             pinned (brute-force sum in the tests)
 *   orc_invert / pso       pinned (grid search on the 2-parameter case)
 *   orc_record             pinned (noise statistics, truth interior, sub-step
 *                                  convergence)
 *   orc_grad_cs            pinned (central differences of orc_misfit_x)
 *   orc_fe_matrices        pinned (static stiffness 3EI/L^3, Euler-Bernoulli
 *                                  frequencies, Rayleigh Q of modes 1-2)
 *   orc_fe_forward         pinned (free steady state, modal-model agreement,
 *                                  Newmark energy conservation, order 2)
 *   orc_polish             pinned (monotone descent, Armijo sufficient decrease,
 *                                  stationarity at an interior optimum)
 *   orc_normal_eq          pinned (central differences of orc_forward; b = -grad/2
 *                                  of orc_grad_cs)
 *   orc_invert_boxed       pinned (whole-cube box = orc_invert; result inside the box;
 *                                  an exact seed is kept; a box around the optimum
 *                                  reaches it with a fraction of the swarm)
 *   orc_lm_polish          pinned (one step to the closed-form least-squares point
 *                                  of a problem affine in its parameter; descent;
 *                                  diagonally scaled gradient for large damping)
 */
#ifndef AFM_ORACLE_H
#define AFM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXM 8
/* Parameter slots th[ORC_NSLOT]: 0..4 the force law's (below); 5..7 the
 * base motion of drive mode 1 (reading R18): amplitude a [m], frequency f
 * [Hz], chirp rate g [Hz/s], y_b(t) = a sin(2 pi (f t + g t^2)). */
#define ORC_NSLOT 8

/* Cantilever model families. */
enum { ORC_POINT_MASS = 0, ORC_MODAL_EB = 1, ORC_FE_HERMITE = 2 };

/* Tip-sample force laws.  Parameter slots th[5]:
 *   LINEAR_SPRING : th[0] = k_s [N/m], th[1] = d_s [m]; F = -k_s (d - d_s) everywhere
 *   DMT           : th = (E* [Pa], H [J], R [m], a0 [m], -)
 *   DMT_KV        : th = (E*, H, R, a0, eta [Pa s])
 *   HOOKE         : th[0] = k [N/m], th[1] = h [m]; F = k (h - d) while d < h, else 0
 *   SPRING_DAMPER : th[0] = k, th[1] = h, th[2] = zeta_s [N s/m];
 *                   F = k (h - d) - zeta_s * ddot while d < h, else 0          */
enum { ORC_F_LINEAR = 0, ORC_F_DMT = 1, ORC_F_DMT_KV = 2, ORC_F_HOOKE = 3,
       ORC_F_SPRING_DAMPER = 4 };

typedef struct {
    int model;            /* ORC_POINT_MASS, ORC_MODAL_EB or ORC_FE_HERMITE      */
    int n_modes;          /* modal models: 1..8 (point mass: 1)                  */
    double f1;            /* first natural frequency [Hz] (modal models)         */
    double k;             /* mode-1 modal stiffness [N/m] (R3)                   */
    double Q[ORC_MAXM];   /* quality factor per mode                            */
    double A0;            /* free tip amplitude [m]                              */
    double Zc;            /* rest tip-sample gap [m]                             */
    int spc;              /* integration steps per drive cycle                   */
    int force;            /* ORC_F_*                                            */
    /* finite-element beam (model == ORC_FE_HERMITE) */
    int n_elem;
    double L, E, rho;     /* length [m], Young's modulus [Pa], density [kg/m^3]  */
    double fe_k;          /* static stiffness 3EI/L^3 target [N/m]               */
    double fe_f1;         /* first natural frequency target [Hz]                 */
    double fe_Q;          /* Rayleigh damping: Q of modes 1 and 2                */
    double nm_beta;       /* Newmark beta (gamma = 1/2)                          */
    /* base motion: 0 = driven at f1 with free amplitude A0, starting on the
     * free steady state (R6); 1 = y_b = a sin(2 pi (f t + g t^2)) with (a, f,
     * g) in slots 5..7, starting at rest (R18; modal models only) */
    int drive;
    double dt;            /* drive 1: step [s] (spc is not used)                 */
    /* deflection points (reading R19): n_points = 0 records the tip only;
     * n_points in 1..4 records the deflection at x = point_xi[k] L, the
     * record then holding n_points values per step (step-major) */
    int n_points;
    double point_xi[4];
} orc_case;

/* Derived modal quantities (SI). */
typedef struct {
    int m;                          /* number of modes                      */
    double w[ORC_MAXM];             /* omega_i [rad/s]                      */
    double gam[ORC_MAXM];           /* base participation gamma_i           */
    double mass;                    /* modal mass k / omega_1^2 [kg]        */
    double wd;                      /* drive angular frequency [rad/s]      */
    double a;                       /* base amplitude [m]                   */
    double psi;                     /* base phase [rad]                     */
    double eta0[ORC_MAXM], etad0[ORC_MAXM];  /* initial modal state          */
    double dt;                      /* step [s]                             */
} orc_modal;

/* Parameter map from the normalised PSO cube to physical slots. */
typedef struct {
    int D;                /* number of free parameters                          */
    int slot[5];          /* theta slot of free dim d                           */
    double lo[5], hi[5];  /* bounds of free dim d (SI)                          */
    int logs[5];          /* 1: log10 map, 0: linear                            */
    double fixed[ORC_NSLOT];  /* values of all slots (free ones are overwritten) */
} orc_pmap;

typedef struct {
    int P, iters;
    double w, c1, c2;
    uint64_t seed;
    uint32_t pixel;
} orc_pso;

/* ---- Philox4x32-10 and the draws built on it ---------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t word);
double orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                uint32_t tag, uint32_t block, int word);

/* ---- modal setup (Sec. 3.2, App. B) -------------------------------------- */
double orc_beam_root(int i);
double orc_mode_shape(double bL, double xi);
int orc_modal_factors(int n_modes, int n_points, double* bL, double* gam,
                      double* int_phi2, double* phi_tip);
int orc_setup(const orc_case* c, orc_modal* md);
double orc_drive_half(const orc_modal* md, int spc, long j);
double orc_drive_chirp(const double th[ORC_NSLOT], double t);

/* ---- force, forward, misfit (Eqs. 2-5) ----------------------------------- */
double orc_force(int kind, const double th[ORC_NSLOT], double d, double ddot);
int orc_forward(const orc_case* c, const double th[ORC_NSLOT], int n_steps, int sub,
                double* u, double* state);
double orc_misfit(const double* U, const double* u, int n);
void orc_map(const orc_pmap* pm, const double* x, double th[ORC_NSLOT]);
int orc_misfit_x(const orc_case* c, const orc_pmap* pm, const double* x,
                 const double* U, int n, double* S);
int orc_misfit_batch(const orc_case* c, const orc_pmap* pm, const double* x,
                     int P, const double* U, int n, double* S);

/* ---- particle swarm (Sec. 3.4, Eq. 8) ------------------------------------ */
void orc_pso_init(int P, int D, uint64_t seed, uint32_t pixel, double* x, double* v);
/* the same for particles p0 .. p0 + P - 1 of a larger swarm (columns 0 .. P - 1) */
void orc_pso_init_slice(int P, int p0, int D, uint64_t seed, uint32_t pixel, double* x, double* v);
void orc_pso_update_slice(int P, int p0, int D, uint32_t it, uint64_t seed, uint32_t pixel,
                          double w, double c1, double c2, double* x, double* v,
                          const double* pbest_x, const double* gbest_x);
void orc_pso_update(int P, int D, uint32_t it, uint64_t seed, uint32_t pixel,
                    double w, double c1, double c2, double* x, double* v,
                    const double* pbest_x, const double* gbest_x);
/* The swarm of orc_invert searching the box [lo, hi] (normalised
 * coordinates, [D] each) with particles p < n_seed started at seeds
 * [n_seed][D] (reading R17); best_x in the normalised cube. */
int orc_invert_boxed(const orc_case* c, const orc_pmap* pm, const double* U, int n,
                     const orc_pso* cfg, const double* lo, const double* hi,
                     const double* seeds, int n_seed, double* best_x, double* best_S);
int orc_invert(const orc_case* c, const orc_pmap* pm, const double* U, int n,
               const orc_pso* cfg, double* best_x, double* best_S, double* hist);

/* ---- synthetic records (Sec. 4.1 inverse-crime measure) ------------------ */
void orc_truth_x(int D, uint64_t seed, uint32_t pixel, double* x);
int orc_cycles(uint64_t seed, uint32_t pixel, int lo, int hi);
int orc_record(const orc_case* c, const orc_pmap* pm, const double* x, int n,
               int sub, double sigma, uint64_t seed, uint32_t pixel, double* U);

/* ---- gradients ---------------------------------------------------------- */
int orc_grad_cs(const orc_case* c, const orc_pmap* pm, const double* x,
                const double* U, int n, double* S, double* grad);
/* Residual sensitivities a_n = d u_n / d x (complex step on the whole
 * trajectory) and the normal equations of the misfit: S = sum r_n^2,
 * H = sum a_n a_n^T ([D][D]), b = sum a_n r_n ([D]), r_n = U_n - u_n. */
int orc_normal_eq(const orc_case* c, const orc_pmap* pm, const double* x, const double* U,
                  int n, double* S, double* H, double* b);
/* Levenberg-Marquardt polish of K candidates x [D][K] (reading R15): per step
 * and candidate the normal equations at x, trial points clamp(x + delta_j)
 * with (H + lambda_j W) delta_j = b, lambda_j = lam0 * lam_ratio^j (j <
 * n_lambda), W = diag(max(H_dd, 1e-12 max_e H_ee)); the trial point of least
 * misfit (first on ties) replaces x if its misfit is lower.  S [K] receives
 * the final misfits. */
int orc_lm_polish(const orc_case* c, const orc_pmap* pm, const double* U, int n, double* x,
                  int K, int steps, int n_lambda, double lam0, double lam_ratio, double* S);
int orc_polish(const orc_case* c, const orc_pmap* pm, const double* U, int n, double* x, int K,
               int steps, int n_cand, double alpha0, double shrink, double sigma, double* S);

/* ---- finite-element Hermite beam with Newmark time stepping (R13) ----- */
int orc_fe_dofs(const orc_case* c);
int orc_fe_matrices(const orc_case* c, double* M, double* K, double* C, double* w12,
                    double* geom);
int orc_fe_forward(const orc_case* c, const double th[ORC_NSLOT], int n_steps, int sub, double* u,
                   double* setup_out);

void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
