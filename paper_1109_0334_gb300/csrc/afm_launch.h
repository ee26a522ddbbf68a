// afm_launch.h -- host-side launchers of the CUDA kernels (C++ linkage,
// internal to libafminv).  Each returns the cudaError_t of its launch.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/afminv.h"
#include "afm_internal.h"

namespace afm {

struct SwarmPtrs {
    float* x;                  // [D][P]
    float* v;                  // [D][P]
    float* pb[2];              // personal-best positions, double-buffered by iteration parity
    float* pbS;                // [P]
    unsigned long long* gkey[2];  // global-best key words (S bits << 32 | particle), by parity
    int* flags;                // [1] non-finite counter
};

struct PsoConst {
    int P, D, iters;
    float w, c1, c2;
    uint64_t seed;
    uint32_t pixel;
    uint32_t p0;   // swarm-wide index of particle 0 (a slice of a split swarm; else 0)
};

// forward + optional misfit; lanes (afm_lanes): AFM_LANES_ONE keeps one
// particle per thread, any other value pairs particles in paired FP32
// instructions for large DMT batches (1 or 3 modes, P >= 65 536;
// bit-identical)
cudaError_t launch_forward_f32(const KConst<float>& K, const float* x, int P, float* defl,
                               const float* U, float* S, int* flags, cudaStream_t st,
                               int lanes = 0);
cudaError_t launch_forward_f64(const KConst<double>& K, const double* x, int P, double* defl,
                               const double* U, double* S, int* flags, cudaStream_t st);
// standalone misfit of a time-major deflection array
cudaError_t launch_misfit(const float* defl, const float* U, int N, int P, float* S, int num_sms,
                          cudaStream_t st);
// synthetic records: FP32 at the fine step of K, sampled every `sub`, plus noise
cudaError_t launch_synth(const KConst<float>& K, const double* x_truth, int n_pix,
                         const int64_t* off, int sub, float sigma_nm, uint64_t seed,
                         uint32_t pixel0, float* U_cat, cudaStream_t st);

// Per-pixel problem constants of a batch whose pixels differ in their
// cantilever or set-point (afm_problem per pixel): indexed by pixel id, with
// each pixel's drive table at its 2 spc half-step phases (+ wrap entry) in
// FP64 and rounded to FP32.  kf == nullptr: every pixel uses the launch's
// constants.
struct PixConst {
    const KConst<float>* kf;    // [n_pix]
    const KConst<double>* kd;   // [n_pix]
    const double* tab64;        // [n_pix][ld]
    const float* tab32;         // [n_pix][ld]
    int ld;
};
// fills tab64 / tab32 of n_pix pixels from kd (the formula of build_drive_table)
cudaError_t launch_pix_tables(const PixConst& pc, int n_pix, int spc2, cudaStream_t st);

// many independent pixel inversions in one persistent launch
struct BatchArgs {
    const float* U;        // concatenated records
    const int64_t* off;    // [n_pix + 1]
    const int* order;      // queue order of pixels (longest first) or nullptr
    int n_pix;
    uint32_t pixel0;       // Philox counter word 2 of pixel 0
    int* queue;            // pixel counter (zeroed before the launch)
    afm_result* res;       // [n_pix]
    float* pb_out;         // nullptr, or per queue slot the final personal bests
                           // [D][P] (normalised cube) followed by their misfits [P]
    // optional prior per queue slot (image scans): the swarm searches the box
    // [box_lo, box_hi] ([slot][D], normalised) in box-local coordinates, and
    // particles p < n_seed start at seeds [slot][n_seed][D]
    const float* box_lo;
    const float* box_hi;
    const float* seeds;
    int n_seed;
    PixConst pix;          // per-pixel constants (pix.kf == nullptr: shared)
};
int batch_threads(int P, int kp);
// largest block of the batch kernel with kp particles per thread (the
// paired-instruction kernels of kp = 2, 4 are built for up to 128 registers)
int batch_max_threads(int kp);
// dynamic shared memory of the batch kernel (pp: per-pixel constants)
size_t batch_smem(int P, int D, int spc2, bool pp = false);
int batch_sort_max();
cudaError_t batch_sort(const int64_t* off, int n_pix, int* order, cudaStream_t st);
cudaError_t batch_occupancy(int m, int force, int kp, int P, int D, int spc2, bool pp,
                            int* blocks_per_sm);
cudaError_t launch_batch(const KConst<float>& K, const PsoConst& pc, const BatchArgs& a, int kp,
                         int grid, cudaStream_t st);

// discrete adjoint (gradient of the misfit wrt the normalised parameters)
// Ragged form (off != nullptr): particle p belongs to queue slot p / per_slot,
// pixel order[slot] (or the slot itself), and is compared with that pixel's
// record U + off[pix] of length off[pix+1] - off[pix] <= K.n_steps; records
// longer than K.n_steps give S = inf and a zero gradient.
size_t adjoint_ckpt_floats(int m, int n_steps, int P);
cudaError_t launch_adjoint(const KConst<float>& K, const float* x, int P, const float* U, float* S,
                           float* G, float* ckpt, cudaStream_t st, const int64_t* off = nullptr,
                           const int* order = nullptr, int per_slot = 1);

// Levenberg-Marquardt polish (kern_lm.cu): sensitivity pass (S [P], H
// [P][D][D], b [P][D]; ragged form as launch_adjoint), damped trial points,
// choice of the best trial point
// (pix: per-pixel constants of the ragged form, pix.kf == nullptr: K for all)
cudaError_t launch_sens(const KConst<float>& K, const float* x, int P, const float* U, float* S,
                        double* H, double* b, cudaStream_t st, const int64_t* off = nullptr,
                        const int* order = nullptr, int per_slot = 1,
                        const PixConst& pix = PixConst{});
// the same pass with one lane per parameter direction (kern_lm_lanes.cu);
// launch_sens uses it when P x lanes fits one warp per SM sub-partition
bool sens_lanes_preferred(int P, int D);
// ... and with one lane per (direction, mode) pair for three modes and
// rate-free laws (kern_lm_lanes.cu), preferred over the above where it fits
bool sens_modes_supported(int m, int force, int P, int D);
cudaError_t launch_sens_modes(const KConst<float>& K, const float* x, int P, const float* U,
                              float* S, double* H, double* b, cudaStream_t st, const int64_t* off,
                              const int* order, int per_slot);
cudaError_t launch_sens_lanes(const KConst<float>& K, const float* x, int P, const float* U,
                              float* S, double* H, double* b, cudaStream_t st, const int64_t* off,
                              const int* order, int per_slot);
cudaError_t launch_lm_cand(int D, int K, int J, const float* x, const double* H, const double* b,
                           double lam0, double ratio, float* Xc, cudaStream_t st);
cudaError_t launch_lm_select(int D, int K, int J, float* x, float* S, const float* Xc,
                             const float* Sc, cudaStream_t st);
// the choice of the fused step (trial points through the sensitivity pass):
// the point kept brings its H [D][D] and b [D] from Hc [K*J][D][D], bc [K*J][D]
cudaError_t launch_lm_select_hb(int D, int K, int J, float* x, float* S, double* H, double* b,
                                const float* Xc, const float* Sc, const double* Hc,
                                const double* bc, cudaStream_t st);

// image scans (kern_image.cu): coarse and fine pixel lists of a row-major
// width x height image with coarse spacing `stride`; per fine pixel a box
// around its (up to 4) coarse neighbours' winners, widened by `margin`, and
// those winners as 4 seed points
void image_counts(int width, int height, int stride, int* n_coarse, int* n_fine);
cudaError_t launch_image_plan(int width, int height, int stride, int* coarse, int* fine,
                              cudaStream_t st);
cudaError_t launch_image_prior(int width, int height, int stride, int D, float margin,
                               const afm_result* res, const int* fine, int n_fine, float* box_lo,
                               float* box_hi, float* seeds, cudaStream_t st);

// batched polish (kern_bpolish.cu): candidates of queue slot s are columns
// s * Kc .. s * Kc + Kc - 1 of [D][n_pix * Kc] arrays
cudaError_t launch_topk_pix(const float* pb_all, int n_pix, int P, int D, int Kc, float* xk,
                            float* Sk, int* ik, cudaStream_t st);
cudaError_t launch_forward_ragged(const KConst<float>& K, const float* x, int Ptot, const float* U_cat,
                                  const int64_t* off, const int* order, int per_slot, float* S,
                                  cudaStream_t st, const PixConst& pix = PixConst{});
cudaError_t launch_pick_pix(int n_pix, int D, int Kc, const float* xk, const float* Sk,
                            const int* ik, const int* order, int iters, afm_result* res,
                            cudaStream_t st);

// gradient polish
cudaError_t launch_polish_cand(int D, int K, int J, const float* x, const float* G, double alpha0,
                               double shrink, float* Xc, cudaStream_t st);
cudaError_t launch_polish_select(int D, int K, int J, float sigma, float* x, const float* G,
                                 float* S, const float* Xc, const float* Sc, cudaStream_t st);
cudaError_t launch_topk(const float* pbS, const float* pb, int P, int D, int K, float* xk, int* idx,
                        cudaStream_t st);
cudaError_t launch_polish_final(const KConst<double>& K, int Kn, int iters, const float* x,
                                const float* S, const int* idx, const float* U, const int* flags,
                                void* result, cudaStream_t st);

// finite-element cantilever
cudaError_t launch_fe_forward_f32(const FeConst& F, const float* x, int P, float* defl,
                                  const float* U, float* S, cudaStream_t st);
cudaError_t launch_fe_forward_f64(const FeConst& F, const double* x, int P, double* defl,
                                  const double* U, double* S, cudaStream_t st);
cudaError_t launch_fe_invert_iter(const FeConst& F, const PsoConst& pc, const SwarmPtrs& sw,
                                  const float* U, float* history, int it, cudaStream_t st);
cudaError_t launch_fe_invert_final(const FeConst& F, const PsoConst& pc, const SwarmPtrs& sw,
                                   const float* U, float* history, void* result, cudaStream_t st);

// particle swarm
cudaError_t launch_pso_init(const PsoConst& pc, const SwarmPtrs& sw, cudaStream_t st);
cudaError_t launch_pso_best(const PsoConst& pc, const SwarmPtrs& sw, const float* S, int it,
                            cudaStream_t st);
cudaError_t launch_pso_move(const PsoConst& pc, const SwarmPtrs& sw, int it, cudaStream_t st);
// the move with a given global-best position gb [D] (a slice of a split swarm)
cudaError_t launch_pso_move_given(const PsoConst& pc, const SwarmPtrs& sw, const float* gb, int it,
                                  cudaStream_t st);
// fused inversion iteration (it = 0: initial evaluation); `lanes` picks the
// lanes-per-particle variant (afm_lanes of afminv.h; all are bit-identical,
// a variant the problem does not support runs the automatic choice)
cudaError_t launch_invert_iter(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                               const float* U, float* history, int it, cudaStream_t st,
                               int lanes = 0);
// the same iteration with two lanes per particle, the RK4 stage forces split
// between them (rate-free laws, 1 or 3 modes, P <= 9728)
bool pair_supported(int m, int force, int P);
cudaError_t launch_invert_pair(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                               const float* U, float* history, int it, cudaStream_t st);
// the same iteration with the modes of a particle spread over 2 or 4 lanes
// (rate-free laws, 2 or 3 modes, P <= 19456 / lanes)
bool modes_supported(int m, int force, int P, int lanes);
cudaError_t launch_invert_modes(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, int it, int lanes,
                                cudaStream_t st);
// base-motion inversion (drive_mode 1, kern_drive.cu)
cudaError_t launch_forward_drive_f32(const KConst<float>& K, const float* x, int P, float* defl,
                                     const float* U, float* S, cudaStream_t st);
cudaError_t launch_forward_drive_f64(const KConst<double>& K, const double* x, int P, double* defl,
                                     const double* U, double* S, cudaStream_t st);
cudaError_t launch_invert_drive(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, int it, cudaStream_t st);
cudaError_t launch_drive_final(const KConst<double>& K, const PsoConst& pc, const SwarmPtrs& sw,
                               const float* U, float* history, void* result, cudaStream_t st);
// deflections at several points along the cantilever (n_points > 0, kern_points.cu)
cudaError_t launch_forward_points_f32(const KConst<float>& K, const float* x, int P, float* defl,
                                      const float* U, float* S, cudaStream_t st);
cudaError_t launch_forward_points_f64(const KConst<double>& K, const double* x, int P, double* defl,
                                      const double* U, double* S, cudaStream_t st);
// (lanes: AFM_LANES_ONE runs one lane per particle, any other value one
// mode per lane where points_modes_supported; bit-identical)
cudaError_t launch_invert_points(const KConst<float>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                 const float* U, float* history, int it, cudaStream_t st,
                                 int lanes = 0);
// the points iteration with one mode per lane (rate-free laws, 2 or 3
// modes, lanes = modes, P <= 19456 / modes)
bool points_modes_supported(int m, int force, int P, int np);
cudaError_t launch_invert_points_modes(const KConst<float>& K, const PsoConst& pc,
                                       const SwarmPtrs& sw, const float* U, float* history, int it,
                                       cudaStream_t st);
cudaError_t launch_points_final(const KConst<double>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, void* result, cudaStream_t st);
// winner re-evaluation in FP64 and result record
cudaError_t launch_invert_final(const KConst<double>& K, const PsoConst& pc, const SwarmPtrs& sw,
                                const float* U, float* history, void* result, cudaStream_t st);

// FP64 re-evaluation of one winner by multiple shooting in time
// (kern_reeval.cu): segments of AFM_SEG steps, B = ceil(n_steps / AFM_SEG).
struct ReevalWinner {
    double x[AFM_MAXD];   // normalised parameters
    double c[4];          // FP64 force coefficients (written by the guess kernel)
    float S32;            // FP32 misfit that selected the winner
    int winner;           // its particle index
};
struct ReevalPtrs {
    ReevalWinner* win;
    double* tab;          // [spc2 + 1] FP64 drive table
    double* start[2];     // [B + 1][2m] segment start states (alternating sweeps)
    double* E;            // [B][2m] segment end states
    double* J;            // [B][2m][2m] segment tangent maps
    double* Sb;           // [B] segment misfit shares
    double* sumU2;        // [1]
    int B;
};
// The same for every queue slot of a batch (kern_reeval_batch.cu): slot i
// owns segments [i maxB, (i + 1) maxB) of the segment arrays.
struct ReevalBatch {
    double* coef;   // [n_pix][4] FP64 force coefficients of each slot's winner
    double* tab;    // [spc2 + 1] FP64 drive table
    double* Z;      // [n_pix * maxB][2m] segment start states (corrected in place)
    double* E;      // [n_pix * maxB][2m] segment end states
    float* J;       // [n_pix * maxB][2m][2m] segment tangent maps (FP32)
    double* Sb;     // [n_pix * maxB] segment misfit shares
    double* u2;     // [n_pix] sum of U^2 of each slot's record
    int maxB;       // segments of the longest record (problem n_steps)
};
size_t reeval_batch_bytes(int m, int n_steps, int spc, int n_pix);
void reeval_batch_carve(void* base, int m, int n_steps, int spc, int n_pix, ReevalBatch* R);
// fills each slot's result record (S_f64, J_rel, theta, status, defect,
// segments) from the parameters already in it
cudaError_t launch_reeval_batch(const KConst<float>& Kf, const KConst<double>& Kd,
                                const ReevalBatch& R, const BatchArgs& a, cudaStream_t st);
bool reeval_supported(int m, int n_steps);
size_t reeval_bytes(int m, int n_steps, int spc);
void reeval_carve(void* base, int m, int n_steps, int spc, ReevalPtrs* R);
cudaError_t launch_reeval_pick_swarm(const PsoConst& pc, const SwarmPtrs& sw, float* history,
                                     ReevalWinner* w, cudaStream_t st);
cudaError_t launch_reeval_pick_min(int D, int Kn, const float* x, const float* S, const int* idx,
                                   ReevalWinner* w, cudaStream_t st);
cudaError_t launch_reeval(const KConst<float>& Kf, const KConst<double>& Kd, const ReevalPtrs& R,
                          const float* U, int iters, const int* flags, void* result,
                          cudaStream_t st);

}  // namespace afm
