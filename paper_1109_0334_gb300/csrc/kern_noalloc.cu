// kern_noalloc.cu -- the allocation-free variant of the fused inversion
// (afm_invert_noalloc).  Its scratch memory is a fixed-size array in the
// library's own device data instead of a caller-provided workspace, so that
// callers that may not allocate device memory at all can still invert.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/afminv.h"
#include "afm_internal.h"
#include "afm_launch.h"

namespace afm {
namespace detail {
afm_status set_error(afm_status st, const char* msg);
afm_status prepare_invert(afm_ctx* ctx, const afm_problem* prob, const afm_pso_cfg* cfg,
                          KConst<float>* Kf, KConst<double>* Kd, PsoConst* pc,
                          size_t* scratch_bytes, size_t* reeval_bytes, int* device);
void carve_swarm(void* base, int P, int D, SwarmPtrs* sw);
void clear_error();
// one fused iteration launch with the context's lanes-per-particle choice,
// bracketed by the profiling events when afm_profile_enable is on
cudaError_t invert_iter_timed(afm_ctx* ctx, const KConst<float>& K, const PsoConst& pc,
                              const SwarmPtrs& sw, const float* U, float* history, int it,
                              cudaStream_t s);
void trace_push(const char* name);
void trace_pop();
}  // namespace detail
}  // namespace afm

namespace {

// Swarm state of one inversion (positions, velocities, two personal-best
// buffers, personal-best misfits, global-best keys, non-finite counter).
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(4) << 20;   // AFM_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(kScratchBytes == AFM_NOALLOC_SCRATCH_BYTES, "header and library disagree");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// The device address of g_scratch on `device` (which must be current).  The
// host-side name g_scratch is only a stand-in; kernels must be given this
// address.  Looked up once per device.
afm_status scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices)
        return afm::detail::set_error(AFM_ERR_INVALID_ARG, "device index beyond 64");
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_addr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || p == nullptr)
            return afm::detail::set_error(AFM_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return AFM_OK;
}

// NVTX range over the call, as every other compute entry point has.
struct Trace {
    Trace() { afm::detail::trace_push("afm_invert_noalloc"); }
    ~Trace() { afm::detail::trace_pop(); }
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;
};

}  // namespace

extern "C" afm_status afm_invert_noalloc(afm_ctx* ctx, const afm_problem* prob, const float* U,
                                         const afm_pso_cfg* cfg, afm_result* result,
                                         float* history, void* stream) {
    Trace trace;
    afm::detail::clear_error();
    afm::KConst<float> Kf;
    afm::KConst<double> Kd;
    afm::PsoConst pc;
    size_t need = 0, reeval = 0;
    int device = 0;
    afm_status st = afm::detail::prepare_invert(ctx, prob, cfg, &Kf, &Kd, &pc, &need, &reeval,
                                                &device);
    if (st) return st;
    if (!U || !result) return afm::detail::set_error(AFM_ERR_INVALID_ARG, "NULL U or result");
    if (need > kScratchBytes)
        return afm::detail::set_error(
            AFM_ERR_INVALID_ARG,
            "swarm too large for the static scratch of afm_invert_noalloc (4 MiB): reduce P "
            "or use afm_invert with a workspace");
    void* base = nullptr;
    if ((st = scratch_address(device, &base))) return st;
    afm::SwarmPtrs sw;
    afm::detail::carve_swarm(base, pc.P, pc.D, &sw);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = afm::launch_pso_init(pc, sw, s);
    for (int it = 0; e == cudaSuccess && it <= pc.iters; ++it)
        e = afm::detail::invert_iter_timed(ctx, Kf, pc, sw, U, history, it, s);
    // the winner's FP64 re-evaluation by multiple shooting where the rest of
    // the scratch holds its segments, else one sequential FP64 pass
    const size_t at = (need + 255) & ~size_t(255);
    if (e == cudaSuccess && reeval > 0 && at + reeval <= kScratchBytes) {
        afm::ReevalPtrs R;
        afm::reeval_carve(static_cast<char*>(base) + at, Kd.m, Kd.n_steps, Kd.spc2 / 2, &R);
        e = afm::launch_reeval_pick_swarm(pc, sw, history, R.win, s);
        if (e == cudaSuccess) e = afm::launch_reeval(Kf, Kd, R, U, pc.iters, sw.flags, result, s);
    } else if (e == cudaSuccess) {
        e = afm::launch_invert_final(Kd, pc, sw, U, history, result, s);
    }
    if (e != cudaSuccess) return afm::detail::set_error(AFM_ERR_CUDA, cudaGetErrorString(e));
    return AFM_OK;
}
