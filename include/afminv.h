/*
 * afminv.h -- C ABI of libafminv: GPU (sm_103a) tip-sample force inversion for
 * dynamic AFM, after Busch, Zou & Ganapathysubramanian, "A near real-time
 * framework for extracting tip-sample forces in dynamic atomic force
 * microscopy" (arXiv 1109.0334).
 *
 * Problem statement (Sec. 2.2 "FP", Sec. 2.3 "IP"):
 *   FP  given the cantilever, its base motion and a parametrised tip-sample
 *       force, compute the tip deflection u(t) (modal reduction Eq. 2 of the
 *       Euler-Bernoulli beam Eq. 1, RK4 of Sec. 3.2);
 *   IP  given the cantilever, the base motion and a measured deflection U(t),
 *       find the force parameters F* minimising J^2 = int (U - u)^2 dt (Eq. 5),
 *       by particle-swarm optimisation (Sec. 3.4, Eq. 8).
 *
 * Conventions
 *   - Every call returns afm_status and never aborts.  On failure,
 *     afm_last_error() holds a message for the calling thread.
 *   - Argument errors are reported as AFM_ERR_INVALID_ARG before any work is
 *     queued.  CUDA errors are AFM_ERR_CUDA.
 *   - Host structs are in SI units, double precision.
 *   - Device arrays are owned by the caller; the library never allocates,
 *     frees or retains them beyond the call's queued work.  "device" below
 *     means a pointer usable by kernels on the context's GPU.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous with respect to the host unless their
 *     name ends in _sync; results land in device memory in stream order.
 *   - Swarm coordinates x live in the normalised cube [0,1]^D and are stored
 *     dimension-major: x[d * P + p].
 *   - Time-major deflection arrays: defl[n * P + p] is particle p's tip
 *     deflection [nm] after step n + 1 (n = 0 .. n_steps-1).
 *   - Records U[n] [nm] are samples at the ends of steps 1 .. n_steps.
 *   - Misfits S are sum_n (U_n - u_n)^2 in nm^2 (Eq. 5 times 1/dt).
 */
#ifndef AFMINV_H
#define AFMINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AFM_MAX_MODES 8
#define AFM_MAX_PARAMS 5
#define AFM_DRIVE_SLOT 5        /* slots 5, 6, 7: base amplitude, frequency, chirp rate */
#define AFM_MAX_POINTS 4        /* deflection points along the cantilever */
#define AFM_MAX_SPC 2048

typedef enum {
    AFM_OK = 0,
    AFM_ERR_INVALID_ARG = 1,
    AFM_ERR_CUDA = 2,
    AFM_ERR_NONFINITE = 3,   /* a state or misfit became NaN/Inf (flagged, run completed) */
    AFM_ERR_TIMEOUT = 4,
    AFM_ERR_UNSUPPORTED = 5
} afm_status;

/* Cantilever models.  POINT_MASS: one mode, participation 1.  MODAL_EB:
 * n_modes clamped-free Euler-Bernoulli modes, tip-normalised (Eq. 2, App. B;
 * mode shapes of Eqs. 6-7).  FE_HERMITE: cubic Hermite beam elements. */
typedef enum { AFM_POINT_MASS = 0, AFM_MODAL_EB = 1, AFM_FE_HERMITE = 2 } afm_model;

/* Tip-sample laws.  d = gap = Zc + u (u = tip deflection, positive away from
 * the sample); F > 0 pushes the tip away from the sample.  Parameter slots:
 *   AFM_LINEAR_SPRING  (k_s [N/m], d_s [m])         F = -k_s (d - d_s)
 *   AFM_DMT            (E* [Pa], H [J], R [m], a0 [m])
 *                      F = -H R / (6 d^2)                              d > a0
 *                      F = 4/3 E* sqrt(R) (a0 - d)^1.5 - H R/(6 a0^2)  d <= a0
 *   AFM_DMT_KV         DMT slots + eta [Pa s]: adds -eta sqrt(R (a0-d)) d'
 *                      in contact
 *   AFM_HOOKE          (k [N/m], h [m])            F = k (h - d) for d < h (Eq. 3)
 *   AFM_SPRING_DAMPER  (k, h, zeta_s [N s/m])      F = k (h - d) - zeta_s d'
 *                                                  for d < h (Eq. 4)            */
typedef enum {
    AFM_LINEAR_SPRING = 0,
    AFM_DMT = 1,
    AFM_DMT_KV = 2,
    AFM_HOOKE = 3,
    AFM_SPRING_DAMPER = 4
} afm_force;

/* Problem descriptor (host, SI). */
typedef struct {
    int model;                  /* afm_model                                       */
    int n_modes;                /* MODAL_EB: 1..AFM_MAX_MODES                      */
    double f1_hz;               /* first natural frequency; the base is driven here */
    double k_N_per_m;           /* mode-1 modal stiffness (FE: static 3EI/L^3)     */
    double Q[AFM_MAX_MODES];    /* quality factor per mode (FE: Q[0] for modes 1,2) */
    /* FE_HERMITE only */
    int n_elem;
    double L_m, E_Pa, rho_kg_m3, newmark_beta;
    /* drive and set-point */
    double A0_m;                /* free tip amplitude                              */
    double Zc_m;                /* rest gap                                        */
    int steps_per_cycle;        /* 4 .. AFM_MAX_SPC                                */
    int n_steps;                /* record length in steps                          */
    /* force law and its parameters */
    int force;                  /* afm_force                                       */
    double fixed[AFM_MAX_PARAMS];   /* values of all slots (free ones ignored)     */
    int n_free;                 /* D: number of free (optimised) parameters        */
    int slot[AFM_MAX_PARAMS];   /* slot of free dimension d                        */
    double lo[AFM_MAX_PARAMS];  /* bounds of free dimension d (SI)                 */
    double hi[AFM_MAX_PARAMS];
    int log_scale[AFM_MAX_PARAMS];  /* 1: log10-uniform map, 0: linear             */
    /* Base motion.  drive_mode 0: driven at f1_hz with free tip amplitude A0_m,
     * starting on that free steady state (steps_per_cycle sets the step).
     * drive_mode 1 (base-motion inversion, Sec. 4.1): y_b(t) = a sin(2 pi
     * (f t + g t^2)) starting at rest, step dt_s; a, f, g are slots 5, 6, 7
     * of slot[] (free) or drive_a_m, drive_f_hz, drive_g_hz_s (fixed); in
     * this mode only afm_forward_batch(_f64) and afm_invert run, on modal
     * models, and steps_per_cycle and A0_m are not used. */
    int drive_mode;
    double dt_s;
    double drive_a_m, drive_f_hz, drive_g_hz_s;
    /* Deflection points (the paper's n_dp, Sec. 3.2): n_points = 0 records
     * the tip; n_points in 1..AFM_MAX_POINTS records the deflection at
     * x = point_xi[k] * L (0 < xi <= 1, MODAL_EB, drive_mode 0): records U
     * are then [n_steps][n_points] and deflection outputs [n_steps][n_points][P];
     * only afm_forward_batch(_f64) and afm_invert run in this mode. */
    int n_points;
    double point_xi[AFM_MAX_POINTS];
} afm_problem;

/* Particle-swarm settings (Sec. 3.4, Eq. 8). */
typedef struct {
    int P;                      /* particles                                       */
    int iters;                  /* position updates (P * (iters+1) forward solves) */
    double w, c1, c2;           /* inertia and acceleration weights                */
    uint64_t seed;              /* Philox4x32-10 key                               */
    uint32_t pixel;             /* counter word 2 (independent pixel streams)      */
} afm_pso_cfg;

/* Device-resident swarm state (caller-owned, see afm_pso_step). */
typedef struct {
    int P, D;
    float* x;                   /* [D][P]                                          */
    float* v;                   /* [D][P]                                          */
    float* pbest_x;             /* [D][P]                                          */
    float* pbest_S;             /* [P]                                             */
    unsigned long long* gbest;  /* 1 word: (float bits of S) << 32 | particle      */
} afm_swarm;

/* Result of one inversion (written to device memory by afm_invert). */
typedef struct {
    double x[AFM_MAX_PARAMS];       /* normalised winner                          */
    double theta[AFM_MAX_PARAMS];   /* all parameter slots, SI                    */
    double S;                       /* FP32 misfit of the winner [nm^2]           */
    double S_f64;                   /* FP64 re-evaluation of the winner [nm^2]    */
    double J_rel;                   /* sqrt(S_f64 / sum U^2)                      */
    int32_t iters;                  /* updates performed                          */
    int32_t winner;                 /* particle index of the winner               */
    int32_t nonfinite;              /* count of non-finite misfits seen           */
    int32_t status;                 /* afm_status of the device-side run          */
    /* How S_f64 was computed.  segments > 0: by multiple shooting over that
     * many time segments (afm_invert, afm_invert_polished; modal models,
     * records of 64 steps or more);
     * defect is then the sum over the segment joins of the max-norm mismatch
     * between one segment's FP64 end state and the next one's start [scaled
     * state units: nm and nm per tau], at most 1e-9.  segments = 0: one
     * sequential FP64 integration (defect = the mismatch that made the
     * multiple-shooting run fall back to it, else 0). */
    double defect;
    int32_t segments;
    int32_t reserved;               /* 0                                          */
    double drive[3];                /* drive_mode 1: the winner's a [m], f [Hz], g [Hz/s]; else 0 */
} afm_result;

typedef struct afm_ctx afm_ctx;

/* ---- context ----------------------------------------------------------- */
/* Binds a CUDA device (queries its SM count).  Owns no device memory. */
afm_status afm_ctx_create(int device, afm_ctx** out);
afm_status afm_ctx_destroy(afm_ctx* ctx);

/* Lanes per particle of the fused inversion iteration (afm_invert,
 * afm_invert_polished, deflection-point records included).  For
 * afm_forward_batch, AFM_LANES_ONE also keeps one particle per thread where
 * large FP32 DMT batches (1 or 3 modes, P >= 65536) otherwise run two
 * particles per thread in paired FP32 instructions (bit-identical).
 * A swarm too small to fill the GPU is latency-bound
 * along each particle's RK4 recurrence (Sec. 3.2); spreading a particle over
 * several lanes of a warp shortens the chain.  Every variant is bit-identical
 * to the one-lane arithmetic; a variant the problem does not support runs
 * the automatic choice.
 *   AFM_LANES_AUTO    the library's choice (default)
 *   AFM_LANES_ONE     one lane per particle
 *   AFM_LANES_STAGES  two lanes, the tip forces of RK4 stages 1/3 and 2/4
 *                     evaluated by one lane each (rate-free force laws,
 *                     1 or 3 modes, P <= 9728)
 *   AFM_LANES_MODES2  two lanes, the modes split between them (rate-free
 *                     laws, 2 or 3 modes, P <= 9728)
 *   AFM_LANES_MODES4  four lanes, one mode each (rate-free laws, 2 or 3
 *                     modes, P <= 4864)
 *   AFM_LANES_MODES3  three lanes, one mode each, ten particles per warp
 *                     (rate-free laws, 2 or 3 modes, P <= 6080)
 * Returns AFM_ERR_INVALID_ARG for an unknown value. */
typedef enum {
    AFM_LANES_AUTO = 0,
    AFM_LANES_ONE = 1,
    AFM_LANES_STAGES = 2,
    AFM_LANES_MODES2 = 3,
    AFM_LANES_MODES4 = 4,
    AFM_LANES_MODES3 = 5
} afm_lanes;
afm_status afm_set_lanes(afm_ctx* ctx, int lanes);
/* Message of the last failed call on the calling host thread ("" if none).
 * The message is thread-local, not per context: every entry point clears it
 * on entry and sets it when it returns a status other than AFM_OK, so a
 * thread that drives several contexts reads the message of its own most
 * recent call, whichever context that call used; other threads' calls never
 * change it.  The pointer stays valid until the thread's next library call. */
const char* afm_last_error(void);
const char* afm_status_string(int status);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int afm_version(void);

/* Kernel timing (tracing aid).  While enabled, the FP32 forward kernel of
 * afm_forward_batch, each fused iteration kernel of afm_invert (and
 * afm_invert_noalloc), the persistent swarm kernel of afm_invert_batch
 * (event-record nodes of its launch graph) and the polish passes of the
 * polished inversions are bracketed by CUDA events on the call's stream.  afm_profile_read waits for
 * the recorded events and returns the summed device time [ms] and the number
 * of timed launches since the previous read. */
afm_status afm_profile_enable(afm_ctx* ctx, int on);
afm_status afm_profile_read(afm_ctx* ctx, double* ms, int* launches);

/* ---- forward problem FP (Sec. 2.2; Eq. 2; RK4 of Sec. 3.2) --------------
 * P candidate parameter sets x [D][P] (device, normalised) are integrated for
 * prob->n_steps steps in FP32: the lowest (resonant) mode's state with
 * Kahan-compensated updates, the others with plain sums (FE beam: the
 * lowest 8 modes compensated), the misfit compensated.  Outputs (each
 * optional, NULL to skip):
 *   defl [n_steps][P]  tip deflection after every step (device)
 *   S    [P]           misfit against U (device; requires U [n_steps])
 * A misfit that is not finite (a diverging candidate) is stored as +inf. */
afm_status afm_forward_batch(afm_ctx* ctx, const afm_problem* prob, const float* x, int P,
                             float* defl, const float* U, float* S, void* stream);
/* The same in FP64 throughout (x, defl, U, S all double; every mode
 * compensated). */
afm_status afm_forward_batch_f64(afm_ctx* ctx, const afm_problem* prob, const double* x,
                                 int P, double* defl, const double* U, double* S,
                                 void* stream);

/* ---- cost functional (Eq. 5) -------------------------------------------
 * S[p] = sum_{n < N} (U[n] - defl[n * P + p])^2, compensated summation.
 * defl [N][P], U [N], S [P]: device. */
afm_status afm_misfit(afm_ctx* ctx, const float* defl, const float* U, int N, int P, float* S,
                      void* stream);

/* ---- particle swarm (Sec. 3.4, Eq. 8) ----------------------------------
 * afm_pso_init: x ~ U[0,1), v = (U[0,1) - x)/2 from the Philox stream
 *   (counter (particle, 0, pixel, tag<<16 | d/4), tags 0 and 1), pbest_S =
 *   +inf, gbest = all ones.
 * afm_pso_step: given the misfits S_new [P] (device) of the current x,
 *   (1) personal bests: pbest <- x where S_new < pbest_S (strictly);
 *   (2) global best = lowest pbest_S, lowest particle index on ties;
 *   (3) unless iter == cfg->iters (the final evaluation): the move of
 *       swarm generation iter + 1, v <- w v + c1 r1 (pbest - x) + c2 r2
 *       (gbest - x), x <- x + v, a coordinate leaving [0,1] is clamped and
 *       its velocity zeroed; r1, r2 per particle and dimension from counter
 *       (particle, iter + 1, pixel, 2<<16 | d/2), words 2d mod 4 and
 *       2d+1 mod 4.
 *   Evaluating the misfits of the current x and calling afm_pso_step with
 *   iter = 0, 1, ..., iters reproduces afm_invert's swarm bit for bit.  The
 *   swarm struct is the whole state: copied out after any step and restored
 *   later, it resumes the run exactly (the draws are keyed by particle,
 *   generation and pixel). */
afm_status afm_pso_init(afm_ctx* ctx, const afm_pso_cfg* cfg, afm_swarm* sw, void* stream);
afm_status afm_pso_step(afm_ctx* ctx, const afm_pso_cfg* cfg, afm_swarm* sw,
                        const float* S_new, uint32_t iter, void* stream);

/* ---- one swarm split across processes (Sec. 3.4, Eq. 8) ------------------
 * The synchronous swarm of cfg->P particles in contiguous slices, one per
 * process (GPU): a process holds particles p0 .. p0 + sw->P - 1 in its own
 * afm_swarm (arrays of sw->P columns) and evaluates their misfits itself
 * (e.g. afm_forward_batch).  Per generation iter = 0 .. cfg->iters:
 *   afm_pso_best_slice   personal bests of the slice from its misfits S_new
 *                        [sw->P] (as afm_pso_step's part 1), and *sw->gbest
 *                        = the slice's best key: (float bits of the misfit)
 *                        << 32 | swarm-wide particle index;
 *   the processes then reduce their keys to the minimum (the swarm's global
 *   best: lowest misfit, lowest index on ties; the paper's synchronous
 *   global best) and the process owning that particle sends its personal
 *   best position, a column of its pbest_x, to the others (D floats);
 *   afm_pso_move_slice   unless iter == cfg->iters: the Eq. 8 move of the
 *                        slice for generation iter + 1 with that global-best
 *                        position gbest_x [D] (device).
 * afm_pso_init_slice starts the slice as afm_pso_init.  The Philox counters
 * carry the swarm-wide index p0 + p, so slices covering 0 .. P - 1 give the
 * swarm of afm_pso_step (and afm_invert) bit for bit.  Errors:
 * AFM_ERR_INVALID_ARG for a slice outside the swarm, a NULL array, or (move)
 * iter >= cfg->iters. */
afm_status afm_pso_init_slice(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              void* stream);
afm_status afm_pso_best_slice(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              const float* S_new, uint32_t iter, void* stream);
afm_status afm_pso_move_slice(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              const float* gbest_x, uint32_t iter, void* stream);

/* ---- inverse problem IP (Sec. 2.3) --------------------------------------
 * One fused inversion: initial swarm, (iters + 1) fused evaluations (PSO
 * move + RK4 forward + misfit + personal/global best), then the winner is
 * re-evaluated in FP64 on the GPU.  U [n_steps] (device).  The caller
 * provides `workspace` (device, >= afm_invert_workspace_size bytes, 256-byte
 * aligned) and `result` (device afm_result).  The winner's misfit history
 * (iters + 1 floats) is written to `history` if non-NULL (device). */
afm_status afm_invert_workspace_size(const afm_problem* prob, const afm_pso_cfg* cfg,
                                     size_t* bytes);
afm_status afm_invert(afm_ctx* ctx, const afm_problem* prob, const float* U,
                      const afm_pso_cfg* cfg, void* workspace, size_t workspace_bytes,
                      afm_result* result, float* history, void* stream);

/* ---- gradient of the misfit (discrete adjoint) --------------------------
 * For P parameter sets x [D][P] (device, normalised): S [P] and dS_dx [D][P]
 * = d S / d x, the exact derivative of the FP32 RK4 recurrence (Eq. 2, Sec.
 * 3.2) and compensated sum (Eq. 5), by the discrete adjoint: the state is
 * checkpointed every 32 steps and each 32-step segment is recomputed during
 * the reverse sweep.  The adjoint compensates the state update of every
 * mode (afm_forward_batch: the lowest mode only), so its S agrees with
 * afm_forward_batch's within 1e-4 relative, not bit for bit.  The Kahan
 * compensation is treated as exact addition.  workspace: device,
 * >= afm_adjoint_workspace_size (the checkpoints: ceil(n_steps/32) x 4 x
 * modes x P floats). */
afm_status afm_adjoint_workspace_size(const afm_problem* prob, int P, size_t* bytes);
afm_status afm_adjoint(afm_ctx* ctx, const afm_problem* prob, const float* x, int P,
                       const float* U, float* S, float* dS_dx, void* workspace,
                       size_t workspace_bytes, void* stream);

/* ---- residual sensitivities (forward mode) ---------------------------------
 * For P parameter sets x [D][P] (device, normalised): S [P] (bit-identical
 * to afm_forward_batch), and the normal equations of the misfit Eq. 5,
 * H [P][D][D] = sum_n a_n a_n^T and b [P][D] = sum_n a_n (U_n - u_n), with
 * a_n = du_n/dx the tangent-linear sensitivities of the FP32 RK4 recurrence
 * (Eq. 2, Sec. 3.2) accumulated in FP32 blocks of 32 steps and FP64 totals.
 * -2 b is the misfit gradient (as afm_adjoint's dS_dx); 2 H is the
 * Gauss-Newton Hessian.  H and b are device FP64 arrays. */
afm_status afm_normal_equations(afm_ctx* ctx, const afm_problem* prob, const float* x, int P,
                                const float* U, float* S, double* H, double* b, void* stream);

/* ---- gradient polish ------------------------------------------------------
 * K candidates x [D][K] (device, in/out) take `steps` steps in the
 * normalised cube; S [K] (device) receives the final misfits.
 *   AFM_POLISH_STEEPEST: gradient g by afm_adjoint, direction -g / max_d |g_d|,
 *     trial points clamp(x + a_j dir) with a_j = 0.05 * 0.5^j (j < n_cand);
 *     the largest step with S(x_j) <= S(x) + 1e-4 g.(x_j - x) is taken, else
 *     x stays.
 *   AFM_POLISH_LM (Levenberg-Marquardt): normal equations by
 *     afm_normal_equations, trial points clamp(x + delta_j) with
 *     (H + lambda_j W) delta_j = b, lambda_j = 1e-7 * 10^j (j < n_cand),
 *     W = diag(max(H_dd, 1e-12 max_e H_ee)); the trial point of least misfit
 *     replaces x if it lowers the misfit.
 * All trial points of a step are evaluated in one batched forward launch.
 * workspace >= afm_polish_workspace_size.
 * afm_invert_polished: the inversion of afm_invert (cfg->iters updates), then
 * the polish_k particles of lowest personal-best misfit are polished for
 * polish_steps steps and the best of them is re-evaluated in FP64 into
 * `result` (result->winner = its swarm index).  history as afm_invert. */
typedef enum { AFM_POLISH_STEEPEST = 0, AFM_POLISH_LM = 1 } afm_polish_method;
afm_status afm_polish_workspace_size(const afm_problem* prob, int K, int n_cand, int method,
                                     size_t* bytes);
afm_status afm_polish(afm_ctx* ctx, const afm_problem* prob, const float* U, float* x, float* S,
                      int K, int steps, int n_cand, int method, void* workspace,
                      size_t workspace_bytes, void* stream);
afm_status afm_invert_polished_workspace_size(const afm_problem* prob, const afm_pso_cfg* cfg,
                                              int polish_k, int n_cand, int method, size_t* bytes);
afm_status afm_invert_polished(afm_ctx* ctx, const afm_problem* prob, const float* U,
                               const afm_pso_cfg* cfg, int polish_k, int polish_steps, int n_cand,
                               int method, void* workspace, size_t workspace_bytes,
                               afm_result* result, float* history, void* stream);

/* ---- many pixel inversions in one launch (image scans) -------------------
 * n_pix independent IPs, pixel i with record U_cat[off[i] .. off[i+1]) (its
 * own length) and Philox counter word 2 = pixel0 + i.  Each pixel runs the
 * same swarm as afm_invert with cfg->P particles (<= 4096) and cfg->iters
 * updates (cfg->pixel is ignored).
 * Problems (the IP statement of Sec. 2.3, per pixel): probs[n_prob] with
 * n_prob = 1 (one problem for every pixel) or n_prob = n_pix (pixel i
 * inverts against probs[i]: an image scan whose set-point, free amplitude
 * or cantilever calibration drifts from pixel to pixel).  Per-pixel
 * problems must agree with probs[0] in model, n_modes, force law,
 * steps_per_cycle, drive_mode 0, n_points 0 and the swarm's
 * parametrisation (n_free, slot, lo, hi, log_scale); they may differ in
 * f1_hz, k_N_per_m, Q, A0_m, Zc_m, the fixed parameter values and n_steps
 * (the largest n_steps sizes the FP64 re-evaluation, so no record may be
 * longer than it).  Else AFM_ERR_INVALID_ARG.  With per-pixel problems
 * each pixel's constants are uploaded from host memory into the workspace
 * on `stream` before the launch (the call returns once they are staged),
 * and pixel i's result equals afm_invert on probs[i] alone bit for bit.
 * One persistent kernel: blocks pull pixels from a queue, longest record
 * first, and keep the whole swarm of a pixel on chip; then every winner is
 * re-evaluated in FP64.  results [n_pix] (device afm_result) are indexed by
 * pixel.  The launch sequence is captured once into a CUDA graph (cached in
 * the context per argument set) and replayed on `stream`.
 * Particles per thread: *particles_per_thread = 1, 2 or 4 forces a choice;
 * NULL or 0 selects the autotuner, which on the first call for a new (modes,
 * force, P, D, steps per cycle) times one evaluation of the first wave of
 * pixels per candidate (synchronous: make that call before any capture of
 * `stream`), scales it by the waves the batch needs at that candidate's
 * occupancy and caches the fastest in the context.  With 2 or 4 particles
 * per thread, DMT swarms step two particles per paired FP32 instruction
 * (bit-identical to one per thread).  The choice used is written back to
 * *particles_per_thread if non-NULL.
 * workspace: device, >= afm_invert_batch_workspace_size(probs, n_prob,
 * n_pix), 256-aligned (the queue, the FP64 re-evaluation of every pixel's
 * winner by multiple shooting: ~250 bytes per 32-step segment of the
 * longest record and pixel, 1.6 GB for 4096 records of 51 200 steps; with
 * per-pixel problems ~6 KB per pixel of constants and drive tables). */
afm_status afm_invert_batch_workspace_size(const afm_problem* probs, int n_prob, int n_pix,
                                           size_t* bytes);
afm_status afm_invert_batch(afm_ctx* ctx, const afm_problem* probs, int n_prob,
                            const float* U_cat, const int64_t* off, int n_pix, uint32_t pixel0,
                            const afm_pso_cfg* cfg, void* workspace, size_t workspace_bytes,
                            afm_result* results, int* particles_per_thread, void* stream);

/* Optional selection and prior of a polished batch (image scans):
 * pixels [n_run] (device) lists the pixels to invert, in this order (no
 * longest-first sorting); box_lo / box_hi [n_run][D] (device, normalised
 * cube, or both NULL) restrict each listed pixel's swarm to a box, which it
 * searches in box-local coordinates; seeds [n_run][n_seed][D] (device,
 * normalised, or NULL with n_seed = 0) start the first n_seed particles,
 * clamped into the box, at rest.  Unlisted pixels' results are untouched. */
typedef struct {
    const int* pixels;
    int n_run;
    const float* box_lo;
    const float* box_hi;
    const float* seeds;
    int n_seed;
} afm_batch_select;

/* ---- many pixel inversions with gradient polish --------------------------
 * afm_invert_batch (same problems, queue, swarms and autotuner; no graph
 * capture), then
 * for every pixel the polish_k personal bests of lowest misfit (lowest index
 * on ties) take polish_steps steps of the polish of afm_polish (`method`,
 * n_cand trial points), all pixels' candidates together in each launch;
 * the candidate of lowest misfit is the pixel's winner
 * (results[i].winner = its swarm index) and is re-evaluated in FP64 as in
 * afm_invert_batch.  Per candidate the arithmetic equals afm_invert_polished
 * on that pixel alone.  AFM_POLISH_STEEPEST: prob->n_steps must be >= the
 * longest record, as it sizes the adjoint checkpoints (a longer record keeps
 * its swarm winner).  Per-pixel problems (n_prob = n_pix) are polished by
 * AFM_POLISH_LM only (else AFM_ERR_UNSUPPORTED).  select (or NULL): a subset
 * of the n_pix pixels and a prior for each (afm_batch_select).
 * workspace: device, >= afm_invert_batch_polished_workspace_size(probs,
 * n_prob, ..., n_run) with n_run the number of pixels inverted
 * (select->n_run, else n_pix), 256-aligned. */
afm_status afm_invert_batch_polished_workspace_size(const afm_problem* probs, int n_prob,
                                                    const afm_pso_cfg* cfg, int n_run,
                                                    int polish_k, int n_cand, int method,
                                                    size_t* bytes);
afm_status afm_invert_batch_polished(afm_ctx* ctx, const afm_problem* probs, int n_prob,
                                     const float* U_cat, const int64_t* off, int n_pix,
                                     uint32_t pixel0, const afm_pso_cfg* cfg, int polish_k,
                                     int polish_steps, int n_cand, int method,
                                     const afm_batch_select* select, void* workspace,
                                     size_t workspace_bytes, afm_result* results,
                                     int* particles_per_thread, void* stream);

/* ---- image scans with cross-pixel warm start ------------------------------
 * A row-major width x height image (pixel id = row * width + column; record
 * of pixel i at U_cat[off[i] .. off[i+1])) in two polished batches: the
 * coarse pixels (rows and columns multiple of `stride`) with swarm `coarse`,
 * then every other pixel with swarm `fine` inside a box spanning the winners
 * of its (up to 4) surrounding coarse pixels, widened by `margin`
 * (normalised units), those winners seeding 4 particles.  Philox counter
 * word 2 of pixel i is pixel0 + i (the cfg's pixel fields are ignored).
 * results [width * height] (device). */
typedef struct {
    int width, height, stride;
    double margin;
    afm_pso_cfg coarse, fine;
    int coarse_polish_k, coarse_polish_steps;
    int fine_polish_k, fine_polish_steps;
    int n_cand, method;
} afm_image_cfg;
afm_status afm_invert_image_workspace_size(const afm_problem* prob, const afm_image_cfg* icfg,
                                           size_t* bytes);
afm_status afm_invert_image(afm_ctx* ctx, const afm_problem* prob, const float* U_cat,
                            const int64_t* off, uint32_t pixel0, const afm_image_cfg* icfg,
                            void* workspace, size_t workspace_bytes, afm_result* results,
                            void* stream);

/* ---- inversion without any device allocation ----------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at all, such as a real-time AFM feedback
 * loop that forbids allocator calls once scanning has started, or a plug-in
 * whose host application owns the whole device-memory budget.  It runs the
 * same fused inversion as afm_invert (with the context's afm_set_lanes
 * choice; its iteration launches are timed by afm_profile_* like
 * afm_invert's), but its swarm state lives in a
 * fixed array of AFM_NOALLOC_SCRATCH_BYTES inside the library's device data
 * (held by every GPU that loads the library until the process exits)
 * instead of a caller workspace; the caller still passes U, result and
 * history.  The swarm state must fit (about P * D <= 200 000), else
 * AFM_ERR_INVALID_ARG.  The winner's FP64 re-evaluation runs by multiple
 * shooting in the rest of the array when its segments fit (~440 bytes per
 * 32 steps of record for 3 modes: records up to ~200 000 steps next to a
 * C2-size swarm), else as one sequential FP64 pass (~7 us per step); the
 * result's `segments` says which.  It calls no cudaMalloc/cudaFree.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) once; make that first call before any stream
 *     capture.
 *   - All calls share the one array, and it keeps the last call's contents
 *     (each call re-initialises the swarm state it needs).  Calls whose work
 *     overlaps on the GPU (different streams or host threads) race on it:
 *     serialise them. */
#define AFM_NOALLOC_SCRATCH_BYTES (4u << 20)
afm_status afm_invert_noalloc(afm_ctx* ctx, const afm_problem* prob, const float* U,
                              const afm_pso_cfg* cfg, afm_result* result, float* history,
                              void* stream);

/* ---- synthetic records (Sec. 4.1: data made by a different integration) --
 * For each of n_pix pixels, the truth x* (normalised, [D][n_pix] device
 * double; mapped to force coefficients in FP64) is integrated in FP32 with
 * the compensated RK4 step of the solver (the same arithmetic as
 * afm_forward_batch) at 1/sub of the solver step, and sampled every `sub`
 * fine steps; then Gaussian noise of std sigma_m is added (Box-Muller in
 * FP32 on Philox counter (n/2, 0, pixel0 + i, 4<<16), words 0/1: the cosine
 * branch for even n, the sine branch for odd n).  The finer step is the
 * paper's guard against the inverse crime (Sec. 4.1); records that need an
 * FP64 truth come from afm_forward_batch_f64 on a problem with the finer
 * step instead.
 * Records are concatenated: pixel i has n_i = off[i+1] - off[i] samples at
 * U_cat[off[i] ..] (device; off is a device int64 array [n_pix + 1]). */
afm_status afm_synth_records(afm_ctx* ctx, const afm_problem* prob, const double* x_truth,
                             int n_pix, const int64_t* off, int sub, double sigma_m,
                             uint64_t seed, uint32_t pixel0, float* U_cat, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AFMINV_H */
