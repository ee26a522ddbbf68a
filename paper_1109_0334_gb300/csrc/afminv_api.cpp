// afminv_api.cpp -- the C ABI of libafminv: argument validation, the
// per-problem set-up in double precision on the host (modal constants of
// Eq. 2, drive and initial state, scaled units), and the launch sequences.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>

#include "../../include/afminv.h"
#include "afm_internal.h"
#include "afm_launch.h"

using afm::KConst;

#include <map>
#include <tuple>
#include <vector>

// One instantiated launch graph of afm_invert_batch and the argument bytes it
// was built from.  Two event-record nodes bracket the swarm kernel: they
// record the graph's own events, or, while profiling is on, a fresh pair per
// launch (afm_profile_read).
struct afm_batch_graph {
    std::vector<unsigned char> key;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t ev_node[2];
    cudaEvent_t ev_own[2];
};

struct afm_ctx {
    int device;
    int num_sms;
    // afm_invert_batch: particles per thread chosen by the autotuner, per
    // (modes, force, particles, free parameters, steps per cycle, per-pixel
    // problems)
    std::map<std::tuple<int, int, int, int, int, int>, int> batch_kp;
    cudaStream_t capture_stream = nullptr;
    std::vector<afm_batch_graph> batch_graphs;
    // kernel timing (afm_profile_*): events around each fused iteration launch
    bool profiling = false;
    // lanes per particle of the fused inversion iteration (afm_lanes)
    int lanes = AFM_LANES_AUTO;
    std::vector<cudaEvent_t> ev_pool;   // reusable events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
};

namespace {

// NVTX range over each compute entry point (a tracing aid: near-free when no
// profiler is attached; the NVTX v3 headers need no library)
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};
#define AFM_TRACE(name) TraceRange afm_trace_range_(name)

thread_local char g_err[512] = "";

afm_status fail(afm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

afm_status cuda_fail(cudaError_t e, const char* where) {
    return fail(AFM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define AFM_CUDA(call, where)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Clamped-free beam: i-th root of cos b cosh b + 1 = 0 (Sec. 3.2), by
// bisection of cos b + sech b on [(2i-1) pi/2 - 1/2, (2i-1) pi/2 + 1/2].
// ---------------------------------------------------------------------------
double beam_root(int i) {
    double lo = (2 * i - 1) * kPi / 2 - 0.5, hi = lo + 1.0;
    auto f = [](double b) { return std::cos(b) + 1.0 / std::cosh(b); };
    double flo = f(lo);
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        double mid = 0.5 * (lo + hi), fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

// Base participation of the tip-normalised mode i (closed form of
// <phi,1>/<phi,phi>): 4 sigma_i / (beta_i L) (-1)^(i+1), with sigma_i written
// in decaying exponentials so that it stays finite for high modes.
double participation(int i, double b) {
    double e1 = std::exp(-b), e2 = e1 * e1;
    double sigma = (1.0 + e2 + 2.0 * e1 * std::cos(b)) / (1.0 - e2 + 2.0 * e1 * std::sin(b));
    return 4.0 * sigma / b * ((i % 2 == 1) ? 1.0 : -1.0);
}

// Clamped-free mode shape of root b at xi = x / L, normalised to 1 at the
// tip: cosh - cos - s (sinh - sin) with s = (cosh b + cos b) / (sinh b +
// sin b), its growing exponentials combined so that nothing large cancels:
// cosh z - s sinh z = ((1 - s) e^z + (1 + s) e^-z) / 2 with
// 1 - s = (sin b - cos b - e^-b) / (sinh b + sin b).
double shape_raw(double b, double xi) {
    const double den = std::sinh(b) + std::sin(b);
    const double s = (std::cosh(b) + std::cos(b)) / den;
    const double oms = (std::sin(b) - std::cos(b) - std::exp(-b)) / den;
    const double z = b * xi;
    return 0.5 * oms * std::exp(z) + 0.5 * (1.0 + s) * std::exp(-z) - std::cos(z) + s * std::sin(z);
}

double shape_tip_normalised(double b, double xi) { return shape_raw(b, xi) / shape_raw(b, 1.0); }

struct Setup {
    int m;
    double w[AFM_MAXM], gam[AFM_MAXM];
    double wd, a, psi, h;
    double q0[AFM_MAXM], v0[AFM_MAXM];  // SI
};

void modal_setup(const afm_problem& pr, int spc, Setup& s) {
    std::memset(&s, 0, sizeof(s));
    s.m = pr.model == AFM_POINT_MASS ? 1 : pr.n_modes;
    const double w1 = 2.0 * kPi * pr.f1_hz;
    if (pr.model == AFM_POINT_MASS) {
        s.w[0] = w1;
        s.gam[0] = 1.0;
    } else {
        const double b1 = beam_root(1);
        for (int i = 0; i < s.m; ++i) {
            double b = beam_root(i + 1);
            s.w[i] = w1 * (b / b1) * (b / b1);
            s.gam[i] = participation(i + 1, b);
        }
    }
    // Drive at the first resonance; amplitude and phase such that the free
    // linear steady state at the tip is A0 cos(w t); start on that state.
    s.wd = w1;
    std::complex<double> H[AFM_MAXM], Hs(0.0, 0.0);
    for (int i = 0; i < s.m; ++i) {
        H[i] = s.gam[i] / std::complex<double>(s.w[i] * s.w[i] - s.wd * s.wd,
                                                s.wd * s.w[i] / pr.Q[i]);
        Hs += H[i];
    }
    s.a = pr.A0_m / (s.wd * s.wd * std::abs(Hs));
    s.psi = kPi / 2 - std::arg(Hs);
    const std::complex<double> rot = std::polar(1.0, s.psi);
    for (int i = 0; i < s.m; ++i) {
        std::complex<double> c = s.a * s.wd * s.wd * H[i] * rot;
        s.q0[i] = c.imag();
        s.v0[i] = s.wd * c.real();
    }
    s.h = 1.0 / (pr.f1_hz * spc);
}

template <typename T>
void fill_kconst(const afm_problem& pr, int spc, int n_steps, KConst<T>& K) {
    Setup s;
    modal_setup(pr, spc, s);
    std::memset(&K, 0, sizeof(K));
    const bool drv = pr.drive_mode == 1;
    const double tau = (drv ? pr.dt_s : s.h) / 6.0, nm = 1e-9;
    const double w1t = s.w[0] * tau;
    for (int i = 0; i < AFM_MAXM; ++i) {
        if (i < s.m) {
            double w2 = (s.w[i] * tau) * (s.w[i] * tau);
            K.w2[i] = (T)w2;
            K.w2lo[i] = (T)(w2 - (double)K.w2[i]);
            K.wq[i] = (T)(s.w[i] * tau / pr.Q[i]);
            K.gam[i] = (T)s.gam[i];
            K.tip[i] = (T)1;
            K.cmask[i] = afm::comp_mode<T>(i) ? (T)1 : (T)0;
            K.q0[i] = drv ? (T)0 : (T)(s.q0[i] / nm);        // drive mode 1 starts at rest
            K.v0[i] = drv ? (T)0 : (T)(s.v0[i] * tau / nm);
        }
    }
    K.Zc = (T)(pr.Zc_m / nm);
    K.drive_amp = (s.a / nm) * (s.wd * tau) * (s.wd * tau);
    K.drive_phase = s.psi;
    K.m = s.m;
    K.spc2 = 2 * spc;
    K.n_steps = n_steps;
    K.force = pr.force;
    K.D = pr.n_free;
    for (int s5 = 0; s5 < AFM_MAXD; ++s5) K.fixed[s5] = pr.fixed[s5];
    for (int d = 0; d < pr.n_free; ++d) {
        K.slot[d] = pr.slot[d];
        K.logs[d] = pr.log_scale[d] ? 1 : 0;
        if (K.logs[d]) {
            K.lo[d] = std::log10(pr.lo[d]);
            K.span[d] = std::log10(pr.hi[d]) - std::log10(pr.lo[d]);
        } else {
            K.lo[d] = pr.lo[d];
            K.span[d] = pr.hi[d] - pr.lo[d];
        }
    }
    K.k = pr.k_N_per_m;
    K.s1 = w1t * w1t;
    K.tau = tau;
    K.drive_mode = drv ? 1 : 0;
    K.drv[0] = pr.drive_a_m;
    K.drv[1] = pr.drive_f_hz;
    K.drv[2] = pr.drive_g_hz_s;
    K.np = pr.n_points;
    for (int k = 0; k < pr.n_points && k < AFM_MAX_POINTS; ++k)
        for (int i = 0; i < s.m; ++i)
            K.phi[k][i] = (T)shape_tip_normalised(beam_root(i + 1), pr.point_xi[k]);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// ---------------------------------------------------------------------------
// Finite-element set-up (host, FP64): section from the targets, element
// assembly, the two lowest frequencies (Householder tridiagonalisation and
// Sturm bisection of L^-1 K L^-T), Rayleigh damping, the free steady state
// (complex solve) as initial state, and the drive table scale.
// ---------------------------------------------------------------------------
// Householder reduction of the symmetric A (row-major, destroyed) to
// tridiagonal (d, e), accumulating the orthogonal Q with A_orig = Q T Q^T.
void householder_tridiag(std::vector<double>& A, int n, std::vector<double>& d,
                         std::vector<double>& e, std::vector<double>& Q) {
    std::vector<double> v(n), p(n), q(n);
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int k = 0; k + 2 < n; ++k) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        if (A[(size_t)(k + 1) * n + k] > 0) alpha = -alpha;
        for (int i = 0; i < n; ++i) v[i] = i <= k ? 0.0 : A[(size_t)i * n + k];
        v[k + 1] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < n; ++i) vn2 += v[i] * v[i];
        if (vn2 == 0.0) continue;
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int j = 0; j < n; ++j) t += A[(size_t)i * n + j] * v[j];
            p[i] = 2.0 * t / vn2;
        }
        double K = 0.0;
        for (int i = 0; i < n; ++i) K += v[i] * p[i];
        K /= vn2;
        for (int i = 0; i < n; ++i) q[i] = p[i] - K * v[i];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] -= v[i] * q[j] + q[i] * v[j];
        // Q <- Q H, H = I - 2 v v^T / |v|^2
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int j = 0; j < n; ++j) t += Q[(size_t)i * n + j] * v[j];
            t *= 2.0 / vn2;
            for (int j = 0; j < n; ++j) Q[(size_t)i * n + j] -= t * v[j];
        }
    }
    d.assign(n, 0.0);
    e.assign(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
}

int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (size_t i = 1; i < d.size(); ++i) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// k-th smallest eigenvalue of the tridiagonal (d, e) by Sturm bisection.
double kth_eigenvalue(const std::vector<double>& d, const std::vector<double>& e, int k) {
    double lo = 1e300, hi = -1e300;
    const int n = (int)d.size();
    for (int i = 0; i < n; ++i) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e, mid) > k) hi = mid; else lo = mid;
        if (hi - lo <= 1e-16 * std::fabs(hi)) break;
    }
    return 0.5 * (lo + hi);
}

// Eigenvector of the tridiagonal (d, e) for eigenvalue lam, by two steps of
// inverse iteration (tridiagonal elimination with partial pivoting).
void tridiag_eigvec(const std::vector<double>& d, const std::vector<double>& e, double lam,
                    std::vector<double>& x) {
    const int n = (int)d.size();
    const double shift = lam + 1e-13 * std::fabs(lam) + 1e-300;
    x.assign(n, 1.0);
    for (int iter = 0; iter < 3; ++iter) {
        // rows: (sub, diag, sup, sup2) after pivoting
        std::vector<double> a(n, 0.0), b(n), c(n, 0.0), c2(n, 0.0), r = x;
        for (int i = 0; i < n; ++i) {
            a[i] = i > 0 ? e[i - 1] : 0.0;
            b[i] = d[i] - shift;
            c[i] = i + 1 < n ? e[i] : 0.0;
        }
        for (int i = 0; i + 1 < n; ++i) {
            // eliminate a[i+1] using row i, pivoting rows i and i+1 if needed
            if (std::fabs(a[i + 1]) > std::fabs(b[i])) {
                std::swap(b[i], a[i + 1]);
                std::swap(c[i], b[i + 1]);
                std::swap(c2[i], c[i + 1]);
                std::swap(r[i], r[i + 1]);
            }
            if (b[i] == 0.0) b[i] = 1e-300;
            const double m = a[i + 1] / b[i];
            a[i + 1] = 0.0;
            b[i + 1] -= m * c[i];
            c[i + 1] -= m * c2[i];
            r[i + 1] -= m * r[i];
        }
        if (b[n - 1] == 0.0) b[n - 1] = 1e-300;
        for (int i = n - 1; i >= 0; --i) {
            double t = r[i];
            if (i + 1 < n) t -= c[i] * x[i + 1];
            if (i + 2 < n) t -= c2[i] * x[i + 2];
            x[i] = t / b[i];
        }
        double nrm = 0.0;
        for (double v : x) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (double& v : x) v /= nrm;
    }
}

// Compensated accumulator: a running sum carried as an unevaluated pair
// (s + c), each addition exact before the final rounding (two-sum), each
// product split into its rounded value and its exact error by one fma.
struct CompSum {
    double s = 0.0, c = 0.0;
    void add(double a) {
        const double t = s + a;
        const double bp = t - s;
        c += (s - (t - bp)) + (a - bp);
        s = t;
    }
    void add_prod(double a, double b) {
        const double p = a * b;
        add(p);
        c += std::fma(a, b, -p);
    }
    double value() const { return s + c; }
};

// Rayleigh quotient phi^T K phi / phi^T M phi of an eigenvector, both forms
// accumulated with compensation.  The lowest eigenvalues of a stiff FE pair
// come out of an FP64 eigensolver with relative errors ~ eps * lambda_max /
// lambda (a few 1e-9 for 32 elements); the quotient of the computed vector
// is exact to rounding (its error is quadratic in the vector's), which keeps
// the resonant mode's frequency right to ~1e-15.
double rayleigh_quotient(const std::vector<double>& K, const std::vector<double>& M, int n,
                         const std::vector<double>& Phi, int md) {
    CompSum num, den;
    for (int i = 0; i < n; ++i) {
        CompSum kp, mp;
        for (int j = 0; j < n; ++j) {
            const double pj = Phi[(size_t)j * n + md];
            kp.add_prod(K[(size_t)i * n + j], pj);
            mp.add_prod(M[(size_t)i * n + j], pj);
        }
        const double pi = Phi[(size_t)i * n + md];
        num.add_prod(pi, kp.s);
        num.add_prod(pi, kp.c);
        den.add_prod(pi, mp.s);
        den.add_prod(pi, mp.c);
    }
    return num.value() / den.value();
}

afm_status fe_setup(const afm_problem& pr, int spc, int n_steps, afm::FeConst& F) {
    std::memset(&F, 0, sizeof(F));
    const int ne = pr.n_elem, n = 2 * ne;
    const double L = pr.L_m, E = pr.E_Pa, k = pr.k_N_per_m;
    const double I = k * L * L * L / (3.0 * E);
    const double b1 = beam_root(1) / L;
    const double w1t = 2.0 * kPi * pr.f1_hz;
    const double mu = E * I * b1 * b1 * b1 * b1 / (w1t * w1t);
    const double he = L / ne;
    std::vector<double> M((size_t)n * n, 0.0), K((size_t)n * n, 0.0);
    const double me[16] = {156, 22 * he, 54, -13 * he, 22 * he, 4 * he * he, 13 * he, -3 * he * he,
                           54, 13 * he, 156, -22 * he, -13 * he, -3 * he * he, -22 * he, 4 * he * he};
    const double ke[16] = {12, 6 * he, -12, 6 * he, 6 * he, 4 * he * he, -6 * he, 2 * he * he,
                           -12, -6 * he, 12, -6 * he, 6 * he, 2 * he * he, -6 * he, 4 * he * he};
    const double ms = mu * he / 420.0, ks = E * I / (he * he * he);
    for (int e = 0; e < ne; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const int i = 2 * e + a - 2, j = 2 * e + b - 2;   // drop the clamped node
                if (i < 0 || j < 0) continue;
                M[(size_t)i * n + j] += ms * me[a * 4 + b];
                K[(size_t)i * n + j] += ks * ke[a * 4 + b];
            }
    // M-orthonormal eigenvectors: M = Lc Lc^T, B = Lc^-1 K Lc^-T = Q T Q^T,
    // T y = lambda y, phi = Lc^-T Q y
    std::vector<double> Lc((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s2 = M[(size_t)i * n + j];
            for (int q = 0; q < j; ++q) s2 -= Lc[(size_t)i * n + q] * Lc[(size_t)j * n + q];
            if (i == j) {
                if (!(s2 > 0)) return fail(AFM_ERR_INVALID_ARG, "FE mass matrix not positive definite");
                Lc[(size_t)i * n + i] = std::sqrt(s2);
            } else {
                Lc[(size_t)i * n + j] = s2 / Lc[(size_t)j * n + j];
            }
        }
    std::vector<double> T((size_t)n * n), B((size_t)n * n);
    for (int col = 0; col < n; ++col)
        for (int i = 0; i < n; ++i) {
            double s2 = K[(size_t)i * n + col];
            for (int q = 0; q < i; ++q) s2 -= Lc[(size_t)i * n + q] * T[(size_t)q * n + col];
            T[(size_t)i * n + col] = s2 / Lc[(size_t)i * n + i];
        }
    for (int row = 0; row < n; ++row)
        for (int i = 0; i < n; ++i) {
            double s2 = T[(size_t)row * n + i];
            for (int q = 0; q < i; ++q) s2 -= Lc[(size_t)i * n + q] * B[(size_t)row * n + q];
            B[(size_t)row * n + i] = s2 / Lc[(size_t)i * n + i];
        }
    std::vector<double> d, e, Q;
    householder_tridiag(B, n, d, e, Q);
    std::vector<double> lam(n), Phi((size_t)n * n);   // Phi[i * n + mode]
    std::vector<double> y, wv(n);
    for (int md = 0; md < n; ++md) {
        lam[md] = kth_eigenvalue(d, e, md);
        tridiag_eigvec(d, e, lam[md], y);
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int j = 0; j < n; ++j) t += Q[(size_t)i * n + j] * y[j];
            wv[i] = t;
        }
        for (int i = n - 1; i >= 0; --i) {   // Lc^T phi = w
            double t = wv[i];
            for (int j = i + 1; j < n; ++j) t -= Lc[(size_t)j * n + i] * Phi[(size_t)j * n + md];
            Phi[(size_t)i * n + md] = t / Lc[(size_t)i * n + i];
        }
        lam[md] = rayleigh_quotient(K, M, n, Phi, md);
    }
    const double wA = std::sqrt(lam[0]), wB = n > 1 ? std::sqrt(lam[1]) : 3.0 * wA;
    const double zeta = 1.0 / (2.0 * pr.Q[0]);
    const double beta = 2.0 * zeta / (wA + wB), alpha = beta * wA * wB;
    const double w = wA, h = 2.0 * kPi / (w * spc);
    const int tip = n - 2;
    // modal drive participation (M r), free steady state per mode, tip shape
    std::vector<double> Mr(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; j += 2) Mr[i] += M[(size_t)i * n + j];
    std::complex<double> Htip(0.0, 0.0);
    std::vector<std::complex<double>> Hm(n);
    std::vector<double> Gam(n);
    for (int md = 0; md < n; ++md) {
        double gm = 0.0;
        for (int i = 0; i < n; ++i) gm += Phi[(size_t)i * n + md] * Mr[i];
        Gam[md] = gm;
        const double cm = alpha + beta * lam[md];
        Hm[md] = gm / std::complex<double>(lam[md] - w * w, w * cm);   // z = Hm a w^2 e^{i(wt+psi)}
        Htip += Phi[(size_t)tip * n + md] * Hm[md];
    }
    const double a = pr.A0_m / (w * w * std::abs(Htip));
    const double psi = kPi / 2 - std::arg(Htip);
    double ctip = 0.0;
    for (int md = 0; md < AFM_FE_MAXN; ++md) {
        if (md >= n) continue;
        const double cm = alpha + beta * lam[md];
        const double sm = 1.0 + 0.5 * h * cm + 0.25 * h * h * lam[md];
        const double pt = Phi[(size_t)tip * n + md];
        F.b1[md] = -h * h * lam[md] / sm;
        F.d2[md] = -h * cm / sm;
        F.g[md] = Gam[md] / sm;
        F.f[md] = 0.25 * h * h * k * pt / sm;
        F.pt[md] = pt;
        ctip += pt * F.f[md];
        const std::complex<double> z0 = a * w * w * Hm[md] * std::polar(1.0, psi) / 1e-9;
        const std::complex<double> zm = a * w * w * Hm[md] * std::polar(1.0, psi - w * h) / 1e-9;
        F.z0[md] = z0.imag();
        F.dz0[md] = z0.imag() - zm.imag();
        F.utip0 += pt * z0.imag();
        F.utipm += pt * zm.imag();
    }
    F.ctip = ctip;
    F.ne = ne;
    F.n = n;
    F.spc = spc;
    F.n_steps = n_steps;
    F.h = h;
    F.Zc = pr.Zc_m / 1e-9;
    F.drive_amp = 0.25 * h * h * a * w * w / 1e-9;
    F.drive_phase = psi;
    KConst<float>& P = F.pm;
    std::memset(&P, 0, sizeof(P));
    P.force = pr.force;
    P.D = pr.n_free;
    for (int s5 = 0; s5 < AFM_MAXD; ++s5) P.fixed[s5] = pr.fixed[s5];
    for (int dd = 0; dd < pr.n_free; ++dd) {
        P.slot[dd] = pr.slot[dd];
        P.logs[dd] = pr.log_scale[dd] ? 1 : 0;
        P.lo[dd] = P.logs[dd] ? std::log10(pr.lo[dd]) : pr.lo[dd];
        P.span[dd] = P.logs[dd] ? std::log10(pr.hi[dd]) - std::log10(pr.lo[dd]) : pr.hi[dd] - pr.lo[dd];
    }
    P.k = k;
    P.s1 = 1.0;
    P.tau = 1.0;
    return AFM_OK;
}

afm_status check_problem(const afm_problem* pr) {
    if (!pr) return fail(AFM_ERR_INVALID_ARG, "problem is NULL");
    if (pr->model != AFM_POINT_MASS && pr->model != AFM_MODAL_EB && pr->model != AFM_FE_HERMITE)
        return fail(AFM_ERR_INVALID_ARG, "unknown model %d", pr->model);
    if (pr->model == AFM_FE_HERMITE) {
        if (pr->n_elem < 1 || 2 * pr->n_elem > AFM_FE_MAXN)
            return fail(AFM_ERR_INVALID_ARG, "n_elem %d outside 1..%d", pr->n_elem, AFM_FE_MAXN / 2);
        if (!finite_pos(pr->L_m) || !finite_pos(pr->E_Pa) || !finite_pos(pr->rho_kg_m3))
            return fail(AFM_ERR_INVALID_ARG, "FE beam needs L_m, E_Pa, rho_kg_m3 > 0");
        if (pr->newmark_beta != 0.25)
            return fail(AFM_ERR_UNSUPPORTED, "only Newmark beta = 1/4 (average acceleration)");
        if (pr->force != AFM_LINEAR_SPRING && pr->force != AFM_DMT && pr->force != AFM_HOOKE)
            return fail(AFM_ERR_UNSUPPORTED, "FE beam supports rate-independent force laws only");
    }
    const int m = pr->model == AFM_POINT_MASS ? 1 : (pr->model == AFM_FE_HERMITE ? 1 : pr->n_modes);
    if (m < 1 || m > AFM_MAX_MODES) return fail(AFM_ERR_INVALID_ARG, "n_modes %d outside 1..8", m);
    if (!finite_pos(pr->f1_hz)) return fail(AFM_ERR_INVALID_ARG, "f1_hz must be > 0");
    if (!finite_pos(pr->k_N_per_m)) return fail(AFM_ERR_INVALID_ARG, "k_N_per_m must be > 0");
    for (int i = 0; i < m; ++i)
        if (!finite_pos(pr->Q[i])) return fail(AFM_ERR_INVALID_ARG, "Q[%d] must be > 0", i);
    const bool drv = pr->drive_mode == 1;
    if (pr->drive_mode != 0 && !drv)
        return fail(AFM_ERR_INVALID_ARG, "drive_mode %d is neither 0 nor 1", pr->drive_mode);
    if (drv) {
        if (pr->model == AFM_FE_HERMITE)
            return fail(AFM_ERR_UNSUPPORTED, "drive_mode 1 runs on the modal models");
        if (!finite_pos(pr->dt_s)) return fail(AFM_ERR_INVALID_ARG, "drive_mode 1 needs dt_s > 0");
    } else {
        if (!finite_pos(pr->A0_m)) return fail(AFM_ERR_INVALID_ARG, "A0_m must be > 0");
        if (pr->steps_per_cycle < 4 || pr->steps_per_cycle > AFM_TAB_MAX / 2)
            return fail(AFM_ERR_INVALID_ARG, "steps_per_cycle %d outside 4..%d",
                        pr->steps_per_cycle, AFM_TAB_MAX / 2);
    }
    if (!std::isfinite(pr->Zc_m)) return fail(AFM_ERR_INVALID_ARG, "Zc_m must be finite");
    if (pr->n_points < 0 || pr->n_points > AFM_MAX_POINTS)
        return fail(AFM_ERR_INVALID_ARG, "n_points %d outside 0..%d", pr->n_points, AFM_MAX_POINTS);
    if (pr->n_points > 0) {
        if (pr->model != AFM_MODAL_EB || drv)
            return fail(AFM_ERR_UNSUPPORTED, "deflection points need MODAL_EB and drive_mode 0");
        for (int k = 0; k < pr->n_points; ++k)
            if (!(pr->point_xi[k] > 0.0 && pr->point_xi[k] <= 1.0))
                return fail(AFM_ERR_INVALID_ARG, "point_xi[%d] outside (0, 1]", k);
    }
    if (pr->n_steps < 1) return fail(AFM_ERR_INVALID_ARG, "n_steps must be >= 1");
    if (pr->force < AFM_LINEAR_SPRING || pr->force > AFM_SPRING_DAMPER)
        return fail(AFM_ERR_INVALID_ARG, "unknown force %d", pr->force);
    if (pr->n_free < 0 || pr->n_free > AFM_MAX_PARAMS)
        return fail(AFM_ERR_INVALID_ARG, "n_free %d outside 0..5", pr->n_free);
    int used = 0;
    for (int d = 0; d < pr->n_free; ++d) {
        int s = pr->slot[d];
        const int n_slots = drv ? AFM_DRIVE_SLOT + 3 : AFM_MAX_PARAMS;
        if (s < 0 || s >= n_slots || (used >> s) & 1)
            return fail(AFM_ERR_INVALID_ARG, "slot[%d] = %d invalid or repeated", d, s);
        used |= 1 << s;
        if (!std::isfinite(pr->lo[d]) || !std::isfinite(pr->hi[d]) || !(pr->lo[d] < pr->hi[d]))
            return fail(AFM_ERR_INVALID_ARG, "bounds of dim %d need lo < hi", d);
        if (pr->log_scale[d] && !(pr->lo[d] > 0))
            return fail(AFM_ERR_INVALID_ARG, "log-scaled dim %d needs lo > 0", d);
    }
    for (int s = 0; s < AFM_MAX_PARAMS; ++s)
        if (!((used >> s) & 1) && !std::isfinite(pr->fixed[s]))
            return fail(AFM_ERR_INVALID_ARG, "fixed[%d] must be finite", s);
    if (drv && !(std::isfinite(pr->drive_a_m) && std::isfinite(pr->drive_f_hz) &&
                 std::isfinite(pr->drive_g_hz_s)))
        return fail(AFM_ERR_INVALID_ARG, "drive_a_m, drive_f_hz, drive_g_hz_s must be finite");
    if (pr->force == AFM_DMT || pr->force == AFM_DMT_KV) {
        // R (slot 2) and a0 (slot 3) must stay positive everywhere in the box
        for (int s = 2; s <= 3; ++s) {
            bool ok = true;
            if ((used >> s) & 1) {
                for (int d = 0; d < pr->n_free; ++d)
                    if (pr->slot[d] == s && !(pr->lo[d] > 0)) ok = false;
            } else if (!(pr->fixed[s] > 0)) {
                ok = false;
            }
            if (!ok) return fail(AFM_ERR_INVALID_ARG, "DMT needs R and a0 > 0");
        }
    }
    return AFM_OK;
}

afm_status modal_only(const afm_problem* pr, const char* what) {
    if (pr->model == AFM_FE_HERMITE)
        return fail(AFM_ERR_UNSUPPORTED, "%s: the FE beam runs in afm_forward_batch(_f64) and afm_invert", what);
    if (pr->drive_mode != 0)
        return fail(AFM_ERR_UNSUPPORTED, "%s: drive_mode 1 runs in afm_forward_batch(_f64) and afm_invert", what);
    if (pr->n_points != 0)
        return fail(AFM_ERR_UNSUPPORTED, "%s: deflection points run in afm_forward_batch(_f64) and afm_invert", what);
    return AFM_OK;
}

afm_status check_ctx(afm_ctx* ctx) {
    if (!ctx) return fail(AFM_ERR_INVALID_ARG, "context is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return AFM_OK;
}

afm_status check_pso(const afm_pso_cfg* cfg, int D) {
    if (!cfg) return fail(AFM_ERR_INVALID_ARG, "pso cfg is NULL");
    if (cfg->P < 1) return fail(AFM_ERR_INVALID_ARG, "P must be >= 1");
    if (cfg->iters < 0) return fail(AFM_ERR_INVALID_ARG, "iters must be >= 0");
    if (!std::isfinite(cfg->w) || !std::isfinite(cfg->c1) || !std::isfinite(cfg->c2))
        return fail(AFM_ERR_INVALID_ARG, "w, c1, c2 must be finite");
    if (D < 1) return fail(AFM_ERR_INVALID_ARG, "the swarm needs at least one free parameter");
    return AFM_OK;
}

afm::PsoConst pso_const(const afm_pso_cfg& c, int D) {
    afm::PsoConst pc;
    pc.P = c.P;
    pc.D = D;
    pc.iters = c.iters;
    pc.w = (float)c.w;
    pc.c1 = (float)c.c1;
    pc.c2 = (float)c.c2;
    pc.seed = c.seed;
    pc.pixel = c.pixel;
    pc.p0 = 0;
    return pc;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

cudaError_t take_event(afm_ctx* ctx, cudaEvent_t* e) {
    if (!ctx->ev_pool.empty()) {
        *e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Launch `fn` on stream s, bracketed by timing events when profiling is on.
template <typename Fn>
cudaError_t timed_launch(afm_ctx* ctx, cudaStream_t s, Fn&& fn) {
    if (!ctx->profiling) return fn();
    cudaEvent_t a, b;
    cudaError_t e = take_event(ctx, &a);
    if (e == cudaSuccess) e = take_event(ctx, &b);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(a, s)) != cudaSuccess) return e;
    if ((e = fn()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b, s)) != cudaSuccess) return e;
    ctx->ev_pending.emplace_back(a, b);
    return cudaSuccess;
}

struct InvLayout {
    size_t x, v, pb0, pb1, pbS, gkey, flags, total;
};

InvLayout invert_layout(int P, int D) {
    InvLayout L;
    size_t off = 0;
    const size_t xs = align256(sizeof(float) * (size_t)P * D);
    L.x = off; off += xs;
    L.v = off; off += xs;
    L.pb0 = off; off += xs;
    L.pb1 = off; off += xs;
    L.pbS = off; off += align256(sizeof(float) * (size_t)P);
    L.gkey = off; off += 256;
    L.flags = off; off += 256;
    L.total = off;
    return L;
}

// Bytes of the multiple-shooting FP64 re-evaluation appended to the
// inversion workspaces (0 where the sequential re-evaluation is used).
int problem_modes(const afm_problem& pr) { return pr.model == AFM_POINT_MASS ? 1 : pr.n_modes; }

size_t reeval_extra(const afm_problem& pr) {
    if (pr.model == AFM_FE_HERMITE || pr.drive_mode != 0) return 0;
    const int m = problem_modes(pr);
    if (!afm::reeval_supported(m, pr.n_steps)) return 0;
    return afm::reeval_bytes(m, pr.n_steps, pr.steps_per_cycle);
}

struct BatchLayout {
    size_t order, queue, total;
};

BatchLayout batch_layout(int n_pix) {
    BatchLayout L;
    L.order = 0;
    L.queue = align256(sizeof(int) * (size_t)n_pix);
    L.total = L.queue + 256;
    return L;
}

// The queue, then the FP64 re-evaluation of every slot's winner (segments
// for the longest record, problem n_steps).
size_t batch_ws_bytes(const afm_problem& pr, int n_run) {
    return batch_layout(n_run).total +
           align256(afm::reeval_batch_bytes(problem_modes(pr), pr.n_steps, pr.steps_per_cycle,
                                            n_run));
}

// Per-pixel problems of a batch (an afm_problem per pixel): their constants
// and drive tables at the end of the workspace, indexed by pixel id.
struct PixLayout {
    size_t kf, kd, t64, t32, total;
    int ld;
};

PixLayout pix_layout(int n_prob, int spc) {
    PixLayout L{};
    if (n_prob <= 1) return L;
    const size_t n = (size_t)n_prob;
    L.ld = (2 * spc + 1 + 3) & ~3;
    L.kf = 0;
    L.kd = align256(sizeof(KConst<float>) * n);
    L.t64 = L.kd + align256(sizeof(KConst<double>) * n);
    L.t32 = L.t64 + align256(sizeof(double) * n * L.ld);
    L.total = L.t32 + align256(sizeof(float) * n * L.ld);
    return L;
}

// Checks a batch's problem array: 1 (shared) or one per pixel, each valid,
// all with the same model, modes, force law, steps per cycle and swarm
// parametrisation (free slots, bounds and scales); they may differ in the
// cantilever (f1, k, Q), the free amplitude, the set-point, the fixed
// parameter values and n_steps.  *eff receives probs[0] with n_steps the
// largest of them (it sizes the FP64 re-evaluation).
afm_status check_batch_probs(const afm_problem* probs, int n_prob, int n_pix, afm_problem* eff) {
    if (!probs) return fail(AFM_ERR_INVALID_ARG, "problem array is NULL");
    if (n_prob != 1 && n_prob != n_pix)
        return fail(AFM_ERR_INVALID_ARG, "n_prob = %d: 1 (shared) or n_pix = %d problems", n_prob,
                    n_pix);
    const afm_problem& a = probs[0];
    afm_status st = check_problem(&a);
    if (st) return st;
    *eff = a;
    for (int i = 1; i < n_prob; ++i) {
        const afm_problem& b = probs[i];
        if ((st = check_problem(&b))) {
            char msg[sizeof(g_err)];
            std::snprintf(msg, sizeof(msg), "%s", g_err);
            return fail(st, "problem %d: %s", i, msg);
        }
        bool same = b.model == a.model && b.n_modes == a.n_modes && b.force == a.force &&
                    b.steps_per_cycle == a.steps_per_cycle && b.n_free == a.n_free &&
                    b.drive_mode == a.drive_mode && b.n_points == a.n_points;
        for (int d = 0; same && d < a.n_free; ++d)
            same = b.slot[d] == a.slot[d] && b.lo[d] == a.lo[d] && b.hi[d] == a.hi[d] &&
                   b.log_scale[d] == a.log_scale[d];
        if (!same)
            return fail(AFM_ERR_INVALID_ARG,
                        "problem %d differs from problem 0 in model, modes, force law, steps per "
                        "cycle or swarm parametrisation",
                        i);
        eff->n_steps = std::max(eff->n_steps, b.n_steps);
    }
    return AFM_OK;
}

template <typename T>
void append_bytes(std::vector<unsigned char>& v, const T& x) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&x);
    v.insert(v.end(), p, p + sizeof(T));
}

// Autotuner of afm_invert_batch: times one swarm evaluation of the first wave
// of pixels for each particles-per-thread choice and keeps the one with the
// lowest estimated batch time (the wave's time x the waves the batch needs).
afm_status batch_tune(afm_ctx* ctx, const KConst<float>& Kf, const afm::PsoConst& pc,
                      const afm::BatchArgs& a, cudaStream_t s, int* kp_out, int* occ_out) {
    const bool pp = a.pix.kf != nullptr;
    const auto key = std::make_tuple(Kf.m, Kf.force, pc.P, pc.D, Kf.spc2, (int)pp);
    auto it = ctx->batch_kp.find(key);
    if (it != ctx->batch_kp.end()) {
        *kp_out = it->second;
        AFM_CUDA(afm::batch_occupancy(Kf.m, Kf.force, *kp_out, pc.P, pc.D, Kf.spc2, pp, occ_out),
                 "batch occupancy");
        return AFM_OK;
    }
    float best_ms = 1e30f;
    int best_kp = 0, best_occ = 0;
    cudaEvent_t e0, e1;
    AFM_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    AFM_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    for (int kp : {1, 2, 4}) {
        const int threads = afm::batch_threads(pc.P, kp);
        if (threads > afm::batch_max_threads(kp) || (kp > 1 && Kf.m > 3)) continue;
        int occ = 0;
        if (afm::batch_occupancy(Kf.m, Kf.force, kp, pc.P, pc.D, Kf.spc2, pp, &occ) != cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            continue;
        }
        afm::PsoConst probe = pc;
        probe.iters = 0;
        afm::BatchArgs pa = a;
        pa.n_pix = std::min(a.n_pix, ctx->num_sms * occ);
        const int grid = pa.n_pix;
        AFM_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), s), "cudaMemsetAsync");
        AFM_CUDA(cudaEventRecord(e0, s), "cudaEventRecord");
        AFM_CUDA(afm::launch_batch(Kf, probe, pa, kp, grid, s), "batch probe kernel");
        AFM_CUDA(cudaEventRecord(e1, s), "cudaEventRecord");
        AFM_CUDA(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        AFM_CUDA(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        // the probe is one wave of the resident pixels (num_sms x occ, which
        // differs between candidates): estimate the whole batch as that
        // wave's time per resident pixel times the pixels
        ms *= std::max(1.0f, (float)a.n_pix / (float)pa.n_pix);
        if (ms < best_ms) {
            best_ms = ms;
            best_kp = kp;
            best_occ = occ;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_kp == 0) return fail(AFM_ERR_UNSUPPORTED, "no batch kernel configuration fits P = %d", pc.P);
    ctx->batch_kp[key] = best_kp;
    *kp_out = best_kp;
    *occ_out = best_occ;
    return AFM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Hooks for other translation units of the library (the allocation-free
// inversion entry point shares this file's validation and set-up).
// ---------------------------------------------------------------------------
namespace afm {
namespace detail {

afm_status set_error(afm_status st, const char* msg) { return fail(st, "%s", msg); }

void clear_error() { g_err[0] = 0; }

cudaError_t invert_iter_timed(afm_ctx* ctx, const KConst<float>& K, const PsoConst& pc,
                              const SwarmPtrs& sw, const float* U, float* history, int it,
                              cudaStream_t s) {
    return timed_launch(ctx, s, [&] {
        return afm::launch_invert_iter(K, pc, sw, U, history, it, s, ctx->lanes);
    });
}

void trace_push(const char* name) { nvtxRangePushA(name); }
void trace_pop() { nvtxRangePop(); }

afm_status prepare_invert(afm_ctx* ctx, const afm_problem* prob, const afm_pso_cfg* cfg,
                          KConst<float>* Kf, KConst<double>* Kd, PsoConst* pc,
                          size_t* scratch_bytes, size_t* reeval_bytes, int* device) {
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = modal_only(prob, "afm_invert_noalloc"))) return st;
    if ((st = check_ctx(ctx))) return st;
    if ((st = check_pso(cfg, prob->n_free))) return st;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, *Kf);
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, *Kd);
    *pc = pso_const(*cfg, prob->n_free);
    *scratch_bytes = invert_layout(cfg->P, prob->n_free).total;
    *reeval_bytes = reeval_extra(*prob);
    *device = ctx->device;
    return AFM_OK;
}

void carve_swarm(void* base, int P, int D, SwarmPtrs* sw) {
    const InvLayout L = invert_layout(P, D);
    char* ws = static_cast<char*>(base);
    sw->x = reinterpret_cast<float*>(ws + L.x);
    sw->v = reinterpret_cast<float*>(ws + L.v);
    sw->pb[0] = reinterpret_cast<float*>(ws + L.pb0);
    sw->pb[1] = reinterpret_cast<float*>(ws + L.pb1);
    sw->pbS = reinterpret_cast<float*>(ws + L.pbS);
    sw->gkey[0] = reinterpret_cast<unsigned long long*>(ws + L.gkey);
    sw->gkey[1] = sw->gkey[0] + 1;
    sw->flags = reinterpret_cast<int*>(ws + L.flags);
}

}  // namespace detail
}  // namespace afm

extern "C" {

int afm_version(void) { return 100; }

const char* afm_last_error(void) { return g_err; }

const char* afm_status_string(int st) {
    switch (st) {
        case AFM_OK: return "AFM_OK";
        case AFM_ERR_INVALID_ARG: return "AFM_ERR_INVALID_ARG";
        case AFM_ERR_CUDA: return "AFM_ERR_CUDA";
        case AFM_ERR_NONFINITE: return "AFM_ERR_NONFINITE";
        case AFM_ERR_TIMEOUT: return "AFM_ERR_TIMEOUT";
        case AFM_ERR_UNSUPPORTED: return "AFM_ERR_UNSUPPORTED";
    }
    return "AFM_ERR_UNKNOWN";
}

afm_status afm_ctx_create(int device, afm_ctx** out) {
    g_err[0] = 0;
    if (!out) return fail(AFM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    AFM_CUDA(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(AFM_ERR_INVALID_ARG, "device %d of %d", device, n);
    AFM_CUDA(cudaSetDevice(device), "cudaSetDevice");
    int sms = 0;
    AFM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "SM count");
    afm_ctx* c = new (std::nothrow) afm_ctx;
    if (!c) return fail(AFM_ERR_INVALID_ARG, "out of host memory");
    c->device = device;
    c->num_sms = sms;
    *out = c;
    return AFM_OK;
}

afm_status afm_ctx_destroy(afm_ctx* ctx) {
    g_err[0] = 0;
    if (ctx) {
        for (auto& pr : ctx->ev_pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
        for (auto& g : ctx->batch_graphs) {
            cudaGraphExecDestroy(g.exec);
            cudaGraphDestroy(g.graph);
            cudaEventDestroy(g.ev_own[0]);
            cudaEventDestroy(g.ev_own[1]);
        }
        if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    }
    delete ctx;
    return AFM_OK;
}

afm_status afm_profile_enable(afm_ctx* ctx, int on) {
    g_err[0] = 0;
    if (!ctx) return fail(AFM_ERR_INVALID_ARG, "context is NULL");
    ctx->profiling = on != 0;
    return AFM_OK;
}

afm_status afm_set_lanes(afm_ctx* ctx, int lanes) {
    g_err[0] = 0;
    if (!ctx) return fail(AFM_ERR_INVALID_ARG, "context is NULL");
    if (lanes < AFM_LANES_AUTO || lanes > AFM_LANES_MODES3)
        return fail(AFM_ERR_INVALID_ARG, "unknown lanes variant %d", lanes);
    ctx->lanes = lanes;
    return AFM_OK;
}

afm_status afm_profile_read(afm_ctx* ctx, double* ms, int* launches) {
    g_err[0] = 0;
    afm_status st = check_ctx(ctx);
    if (st) return st;
    if (!ms || !launches) return fail(AFM_ERR_INVALID_ARG, "NULL output");
    double total = 0.0;
    int n = 0;
    for (auto& pr : ctx->ev_pending) {
        AFM_CUDA(cudaEventSynchronize(pr.second), "cudaEventSynchronize");
        float t = 0.f;
        AFM_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second), "cudaEventElapsedTime");
        total += t;
        ++n;
        ctx->ev_pool.push_back(pr.first);
        ctx->ev_pool.push_back(pr.second);
    }
    ctx->ev_pending.clear();
    *ms = total;
    *launches = n;
    return AFM_OK;
}

afm_status afm_forward_batch(afm_ctx* ctx, const afm_problem* prob, const float* x, int P,
                             float* defl, const float* U, float* S, void* stream) {
    AFM_TRACE("afm_forward_batch");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = check_ctx(ctx))) return st;
    if (P < 1) return fail(AFM_ERR_INVALID_ARG, "P must be >= 1");
    if (prob->n_free > 0 && !x) return fail(AFM_ERR_INVALID_ARG, "x is NULL");
    if (S && !U) return fail(AFM_ERR_INVALID_ARG, "S requested without a record U");
    if (!S && !defl) return fail(AFM_ERR_INVALID_ARG, "nothing to compute (defl and S NULL)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (prob->model == AFM_FE_HERMITE) {
        afm::FeConst F;
        if ((st = fe_setup(*prob, prob->steps_per_cycle, prob->n_steps, F))) return st;
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_fe_forward_f32(F, x, P, defl, U, S, s); }),
                 "FE forward kernel");
        return AFM_OK;
    }
    KConst<float> K;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, K);
    if (prob->drive_mode == 1) {
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_forward_drive_f32(K, x, P, defl, U, S, s); }),
                 "drive forward kernel");
        return AFM_OK;
    }
    if (prob->n_points > 0) {
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_forward_points_f32(K, x, P, defl, U, S, s); }),
                 "points forward kernel");
        return AFM_OK;
    }
    AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_forward_f32(K, x, P, defl, U, S, nullptr, s, ctx->lanes); }),
             "forward kernel");
    return AFM_OK;
}

afm_status afm_forward_batch_f64(afm_ctx* ctx, const afm_problem* prob, const double* x, int P,
                                 double* defl, const double* U, double* S, void* stream) {
    AFM_TRACE("afm_forward_batch_f64");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = check_ctx(ctx))) return st;
    if (P < 1) return fail(AFM_ERR_INVALID_ARG, "P must be >= 1");
    if (prob->n_free > 0 && !x) return fail(AFM_ERR_INVALID_ARG, "x is NULL");
    if (S && !U) return fail(AFM_ERR_INVALID_ARG, "S requested without a record U");
    if (!S && !defl) return fail(AFM_ERR_INVALID_ARG, "nothing to compute (defl and S NULL)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (prob->model == AFM_FE_HERMITE) {
        afm::FeConst F;
        if ((st = fe_setup(*prob, prob->steps_per_cycle, prob->n_steps, F))) return st;
        AFM_CUDA(afm::launch_fe_forward_f64(F, x, P, defl, U, S, s), "FE forward f64 kernel");
        return AFM_OK;
    }
    KConst<double> K;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, K);
    if (prob->drive_mode == 1) {
        AFM_CUDA(afm::launch_forward_drive_f64(K, x, P, defl, U, S, s), "drive forward f64 kernel");
        return AFM_OK;
    }
    if (prob->n_points > 0) {
        AFM_CUDA(afm::launch_forward_points_f64(K, x, P, defl, U, S, s), "points forward f64 kernel");
        return AFM_OK;
    }
    AFM_CUDA(afm::launch_forward_f64(K, x, P, defl, U, S, nullptr, s), "forward f64 kernel");
    return AFM_OK;
}

afm_status afm_misfit(afm_ctx* ctx, const float* defl, const float* U, int N, int P, float* S,
                      void* stream) {
    AFM_TRACE("afm_misfit");
    g_err[0] = 0;
    afm_status st = check_ctx(ctx);
    if (st) return st;
    if (!defl || !U || !S) return fail(AFM_ERR_INVALID_ARG, "NULL array");
    if (N < 1 || P < 1) return fail(AFM_ERR_INVALID_ARG, "N and P must be >= 1");
    AFM_CUDA(afm::launch_misfit(defl, U, N, P, S, ctx->num_sms,
                                reinterpret_cast<cudaStream_t>(stream)),
             "misfit kernel");
    return AFM_OK;
}

static afm_status swarm_ptrs(const afm_swarm* sw, afm::SwarmPtrs& p) {
    if (!sw || !sw->x || !sw->v || !sw->pbest_x || !sw->pbest_S || !sw->gbest)
        return fail(AFM_ERR_INVALID_ARG, "swarm has NULL arrays");
    p.x = sw->x;
    p.v = sw->v;
    p.pb[0] = p.pb[1] = sw->pbest_x;
    p.pbS = sw->pbest_S;
    p.gkey[0] = p.gkey[1] = sw->gbest;
    p.flags = nullptr;
    return AFM_OK;
}

afm_status afm_pso_init(afm_ctx* ctx, const afm_pso_cfg* cfg, afm_swarm* sw, void* stream) {
    AFM_TRACE("afm_pso_init");
    g_err[0] = 0;
    afm_status st = check_ctx(ctx);
    if (st) return st;
    if (!sw) return fail(AFM_ERR_INVALID_ARG, "swarm is NULL");
    if ((st = check_pso(cfg, sw->D))) return st;
    if (sw->P != cfg->P || sw->D > AFM_MAX_PARAMS)
        return fail(AFM_ERR_INVALID_ARG, "swarm shape (P %d, D %d) does not match", sw->P, sw->D);
    afm::SwarmPtrs p;
    if ((st = swarm_ptrs(sw, p))) return st;
    AFM_CUDA(afm::launch_pso_init(pso_const(*cfg, sw->D), p, reinterpret_cast<cudaStream_t>(stream)),
             "pso init kernel");
    return AFM_OK;
}

afm_status afm_pso_step(afm_ctx* ctx, const afm_pso_cfg* cfg, afm_swarm* sw, const float* S_new,
                        uint32_t iter, void* stream) {
    AFM_TRACE("afm_pso_step");
    g_err[0] = 0;
    afm_status st = check_ctx(ctx);
    if (st) return st;
    if (!sw) return fail(AFM_ERR_INVALID_ARG, "swarm is NULL");
    if ((st = check_pso(cfg, sw->D))) return st;
    if (sw->P != cfg->P || sw->D > AFM_MAX_PARAMS)
        return fail(AFM_ERR_INVALID_ARG, "swarm shape (P %d, D %d) does not match", sw->P, sw->D);
    if (!S_new) return fail(AFM_ERR_INVALID_ARG, "S_new is NULL");
    if ((int)iter > cfg->iters) return fail(AFM_ERR_INVALID_ARG, "iter %u > iters", iter);
    afm::SwarmPtrs p;
    if ((st = swarm_ptrs(sw, p))) return st;
    const afm::PsoConst pc = pso_const(*cfg, sw->D);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AFM_CUDA(afm::launch_pso_best(pc, p, S_new, (int)iter, s), "pso best kernel");
    if ((int)iter < cfg->iters) AFM_CUDA(afm::launch_pso_move(pc, p, (int)iter + 1, s), "pso move kernel");
    return AFM_OK;
}

// A slice of a split swarm: particles p0 .. p0 + sw->P - 1 of cfg->P.
static afm_status slice_setup(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              afm::SwarmPtrs& p, afm::PsoConst& pc) {
    afm_status st = check_ctx(ctx);
    if (st) return st;
    if (!sw) return fail(AFM_ERR_INVALID_ARG, "swarm is NULL");
    if ((st = check_pso(cfg, sw->D))) return st;
    if (sw->P < 1 || sw->D > AFM_MAX_PARAMS || p0 < 0 || (long long)p0 + sw->P > cfg->P)
        return fail(AFM_ERR_INVALID_ARG, "slice p0 %d of %d particles outside the swarm of %d",
                    p0, sw->P, cfg->P);
    if ((st = swarm_ptrs(sw, p))) return st;
    pc = pso_const(*cfg, sw->D);
    pc.P = sw->P;
    pc.p0 = (uint32_t)p0;
    return AFM_OK;
}

afm_status afm_pso_init_slice(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              void* stream) {
    AFM_TRACE("afm_pso_init_slice");
    g_err[0] = 0;
    afm::SwarmPtrs p;
    afm::PsoConst pc;
    afm_status st = slice_setup(ctx, cfg, p0, sw, p, pc);
    if (st) return st;
    AFM_CUDA(afm::launch_pso_init(pc, p, reinterpret_cast<cudaStream_t>(stream)), "pso init kernel");
    return AFM_OK;
}

afm_status afm_pso_best_slice(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              const float* S_new, uint32_t iter, void* stream) {
    AFM_TRACE("afm_pso_best_slice");
    g_err[0] = 0;
    afm::SwarmPtrs p;
    afm::PsoConst pc;
    afm_status st = slice_setup(ctx, cfg, p0, sw, p, pc);
    if (st) return st;
    if (!S_new) return fail(AFM_ERR_INVALID_ARG, "S_new is NULL");
    if ((int)iter > cfg->iters) return fail(AFM_ERR_INVALID_ARG, "iter %u > iters", iter);
    AFM_CUDA(afm::launch_pso_best(pc, p, S_new, (int)iter, reinterpret_cast<cudaStream_t>(stream)),
             "pso best kernel");
    return AFM_OK;
}

afm_status afm_pso_move_slice(afm_ctx* ctx, const afm_pso_cfg* cfg, int p0, afm_swarm* sw,
                              const float* gbest_x, uint32_t iter, void* stream) {
    AFM_TRACE("afm_pso_move_slice");
    g_err[0] = 0;
    afm::SwarmPtrs p;
    afm::PsoConst pc;
    afm_status st = slice_setup(ctx, cfg, p0, sw, p, pc);
    if (st) return st;
    if (!gbest_x) return fail(AFM_ERR_INVALID_ARG, "gbest_x is NULL");
    if ((int)iter >= cfg->iters)
        return fail(AFM_ERR_INVALID_ARG, "iter %u: the last evaluation (iters) has no move", iter);
    AFM_CUDA(afm::launch_pso_move_given(pc, p, gbest_x, (int)iter + 1,
                                        reinterpret_cast<cudaStream_t>(stream)),
             "pso move kernel");
    return AFM_OK;
}

afm_status afm_invert_workspace_size(const afm_problem* prob, const afm_pso_cfg* cfg,
                                     size_t* bytes) {
    g_err[0] = 0;
    if (!bytes) return fail(AFM_ERR_INVALID_ARG, "bytes is NULL");
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = check_pso(cfg, prob->n_free))) return st;
    *bytes = invert_layout(cfg->P, prob->n_free).total + reeval_extra(*prob);
    return AFM_OK;
}

afm_status afm_invert(afm_ctx* ctx, const afm_problem* prob, const float* U,
                      const afm_pso_cfg* cfg, void* workspace, size_t workspace_bytes,
                      afm_result* result, float* history, void* stream) {
    AFM_TRACE("afm_invert");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = check_ctx(ctx))) return st;
    if ((st = check_pso(cfg, prob->n_free))) return st;
    if (!U || !result || !workspace) return fail(AFM_ERR_INVALID_ARG, "NULL U, result or workspace");
    if (reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(AFM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const int D = prob->n_free, P = cfg->P;
    const InvLayout L = invert_layout(P, D);
    const size_t need = L.total + reeval_extra(*prob);
    if (workspace_bytes < need)
        return fail(AFM_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    char* ws = static_cast<char*>(workspace);
    afm::SwarmPtrs sw;
    sw.x = reinterpret_cast<float*>(ws + L.x);
    sw.v = reinterpret_cast<float*>(ws + L.v);
    sw.pb[0] = reinterpret_cast<float*>(ws + L.pb0);
    sw.pb[1] = reinterpret_cast<float*>(ws + L.pb1);
    sw.pbS = reinterpret_cast<float*>(ws + L.pbS);
    sw.gkey[0] = reinterpret_cast<unsigned long long*>(ws + L.gkey);
    sw.gkey[1] = sw.gkey[0] + 1;
    sw.flags = reinterpret_cast<int*>(ws + L.flags);
    const afm::PsoConst pc = pso_const(*cfg, D);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (prob->model == AFM_FE_HERMITE) {
        afm::FeConst F;
        if ((st = fe_setup(*prob, prob->steps_per_cycle, prob->n_steps, F))) return st;
        AFM_CUDA(afm::launch_pso_init(pc, sw, s), "pso init kernel");
        for (int it = 0; it <= cfg->iters; ++it)
            AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_fe_invert_iter(F, pc, sw, U, history, it, s); }),
                     "FE invert iteration kernel");
        AFM_CUDA(afm::launch_fe_invert_final(F, pc, sw, U, history, result, s), "FE invert final kernel");
        return AFM_OK;
    }
    KConst<float> Kf;
    KConst<double> Kd;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, Kf);
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, Kd);
    AFM_CUDA(afm::launch_pso_init(pc, sw, s), "pso init kernel");
    if (prob->drive_mode == 1) {
        for (int it = 0; it <= cfg->iters; ++it)
            AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_invert_drive(Kf, pc, sw, U, history, it, s); }),
                     "drive inversion kernel");
        AFM_CUDA(afm::launch_drive_final(Kd, pc, sw, U, history, result, s), "drive final kernel");
        return AFM_OK;
    }
    for (int it = 0; it <= cfg->iters; ++it)
        AFM_CUDA(timed_launch(ctx, s, [&] {
                     return prob->n_points > 0 ? afm::launch_invert_points(Kf, pc, sw, U, history, it, s, ctx->lanes)
                                               : afm::launch_invert_iter(Kf, pc, sw, U, history, it, s,
                                                                         ctx->lanes);
                 }),
                 "invert iteration kernel");
    if (reeval_extra(*prob) > 0) {
        afm::ReevalPtrs R;
        afm::reeval_carve(ws + L.total, problem_modes(*prob), prob->n_steps, prob->steps_per_cycle, &R);
        AFM_CUDA(afm::launch_reeval_pick_swarm(pc, sw, history, R.win, s), "winner pick kernel");
        AFM_CUDA(afm::launch_reeval(Kf, Kd, R, U, cfg->iters, sw.flags, result, s),
                 "FP64 re-evaluation kernels");
        return AFM_OK;
    }
    if (prob->n_points > 0)
        AFM_CUDA(afm::launch_points_final(Kd, pc, sw, U, history, result, s), "points final kernel");
    else
        AFM_CUDA(afm::launch_invert_final(Kd, pc, sw, U, history, result, s), "invert final kernel");
    return AFM_OK;
}

afm_status afm_adjoint_workspace_size(const afm_problem* prob, int P, size_t* bytes) {
    g_err[0] = 0;
    if (!bytes || P < 1) return fail(AFM_ERR_INVALID_ARG, "P >= 1 and bytes needed");
    afm_status st = check_problem(prob);
    if (st) return st;
    const int m = prob->model == AFM_POINT_MASS ? 1 : prob->n_modes;
    *bytes = align256(sizeof(float) * afm::adjoint_ckpt_floats(m, prob->n_steps, P));
    return AFM_OK;
}

afm_status afm_adjoint(afm_ctx* ctx, const afm_problem* prob, const float* x, int P,
                       const float* U, float* S, float* dS_dx, void* workspace,
                       size_t workspace_bytes, void* stream) {
    AFM_TRACE("afm_adjoint");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = modal_only(prob, "afm_adjoint"))) return st;
    if ((st = check_ctx(ctx))) return st;
    if (P < 1 || prob->n_free < 1) return fail(AFM_ERR_INVALID_ARG, "P >= 1 and n_free >= 1 needed");
    if (!x || !U || !S || !dS_dx || !workspace)
        return fail(AFM_ERR_INVALID_ARG, "NULL x, U, S, dS_dx or workspace");
    size_t need = 0;
    if ((st = afm_adjoint_workspace_size(prob, P, &need))) return st;
    if (workspace_bytes < need)
        return fail(AFM_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    KConst<float> K;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, K);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AFM_CUDA(timed_launch(ctx, s, [&] {
                 return afm::launch_adjoint(K, x, P, U, S, dS_dx, static_cast<float*>(workspace), s);
             }),
             "adjoint kernel");
    return AFM_OK;
}

afm_status afm_normal_equations(afm_ctx* ctx, const afm_problem* prob, const float* x, int P,
                                const float* U, float* S, double* H, double* b, void* stream) {
    AFM_TRACE("afm_normal_equations");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = modal_only(prob, "afm_normal_equations"))) return st;
    if ((st = check_ctx(ctx))) return st;
    if (!x || !U || !S || !H || !b || P < 1 || prob->n_free < 1)
        return fail(AFM_ERR_INVALID_ARG, "NULL array, P < 1 or no free parameter");
    KConst<float> K32;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, K32);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_sens(K32, x, P, U, S, H, b, s); }),
             "sensitivity kernel");
    return AFM_OK;
}

// Polish workspace.  Steepest descent: gradient [D][K], adjoint checkpoints
// of K particles; Levenberg-Marquardt: normal equations H [K][D][D], b
// [K][D] (FP64); both: trial points [D][K*J] and their misfits [K*J].
// Fused Levenberg-Marquardt step (few candidates, `fused`): the trial points
// go through the sensitivity pass instead of a plain forward, which gives
// their misfits (the forward's, bit for bit) and their normal equations at
// once, so the point kept carries its H and b into the next step; also H_c
// [K*J][D][D], b_c [K*J][D].
struct PolishLayout {
    size_t G, ckpt, H, b, Hc, bc, Xc, Sc, total;
    bool fused;
};

// The fused step pays for the trial points' tangents; it wins while they fit
// the GPU's sub-partitions (latency regime), as the lane-split sensitivities.
bool lm_fused(int K, int J, int D) { return afm::sens_lanes_preferred(K * J, D); }

PolishLayout polish_layout(const afm_problem& pr, int K, int J, int method, bool fused_ok) {
    PolishLayout L;
    const size_t D = (size_t)pr.n_free;
    const int m = pr.model == AFM_POINT_MASS ? 1 : pr.n_modes;
    size_t off = 0;
    L.G = L.ckpt = L.H = L.b = L.Hc = L.bc = 0;
    L.fused = fused_ok && method == AFM_POLISH_LM && lm_fused(K, J, (int)D);
    if (method == AFM_POLISH_LM) {
        L.H = off; off += align256(sizeof(double) * (size_t)K * D * D);
        L.b = off; off += align256(sizeof(double) * (size_t)K * D);
        if (L.fused) {
            L.Hc = off; off += align256(sizeof(double) * (size_t)K * J * D * D);
            L.bc = off; off += align256(sizeof(double) * (size_t)K * J * D);
        }
    } else {
        L.G = off; off += align256(sizeof(float) * D * K);
        L.ckpt = off; off += align256(sizeof(float) * afm::adjoint_ckpt_floats(m, pr.n_steps, K));
    }
    L.Xc = off; off += align256(sizeof(float) * D * K * J);
    L.Sc = off; off += align256(sizeof(float) * (size_t)K * J);
    L.total = off;
    return L;
}

const double kPolishAlpha0 = 0.05, kPolishShrink = 0.5, kPolishSigma = 1e-4;
const double kLmLambda0 = 1e-7, kLmRatio = 10.0;

// One polish step of Kn candidates x [D][Kn] (S [Kn] receives the misfit at
// the step's start, then that of the point kept).  Ragged form (off !=
// nullptr): candidate k is compared with the record of pixel order[k / per].
afm_status polish_step(afm_ctx* ctx, const KConst<float>& K, int method, const float* U,
                       const int64_t* off, const int* order, int per, float* x, float* S, int Kn,
                       int J, const PolishLayout& L, char* ws, cudaStream_t s,
                       const afm::PixConst& pix = afm::PixConst{}) {
    float* Xc = reinterpret_cast<float*>(ws + L.Xc);
    float* Sc = reinterpret_cast<float*>(ws + L.Sc);
    const int D = K.D;
    if (method == AFM_POLISH_LM) {
        double* H = reinterpret_cast<double*>(ws + L.H);
        double* b = reinterpret_cast<double*>(ws + L.b);
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_sens(K, x, Kn, U, S, H, b, s, off, order, per, pix); }),
                 "sensitivity kernel");
        AFM_CUDA(afm::launch_lm_cand(D, Kn, J, x, H, b, kLmLambda0, kLmRatio, Xc, s), "LM trial kernel");
    } else {
        if (pix.kf != nullptr)
            return fail(AFM_ERR_UNSUPPORTED, "the steepest-descent polish needs one problem for all pixels");
        float* G = reinterpret_cast<float*>(ws + L.G);
        float* ck = reinterpret_cast<float*>(ws + L.ckpt);
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_adjoint(K, x, Kn, U, S, G, ck, s, off, order, per); }),
                 "adjoint kernel");
        AFM_CUDA(afm::launch_polish_cand(D, Kn, J, x, G, kPolishAlpha0, kPolishShrink, Xc, s),
                 "polish candidate kernel");
    }
    if (off != nullptr)
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_forward_ragged(K, Xc, Kn * J, U, off, order, per * J, Sc, s, pix); }),
                 "ragged forward kernel");
    else
        AFM_CUDA(afm::launch_forward_f32(K, Xc, Kn * J, nullptr, U, Sc, nullptr, s), "forward kernel");
    if (method == AFM_POLISH_LM) {
        AFM_CUDA(afm::launch_lm_select(D, Kn, J, x, S, Xc, Sc, s), "LM select kernel");
    } else {
        const float* G = reinterpret_cast<const float*>(ws + L.G);
        AFM_CUDA(afm::launch_polish_select(D, Kn, J, (float)kPolishSigma, x, G, S, Xc, Sc, s),
                 "polish select kernel");
    }
    return AFM_OK;
}

afm_status polish_run(afm_ctx* ctx, const afm_problem& pr, const KConst<float>& K, const float* U,
                      float* x, float* S, int Kn, int steps, int J, int method, char* ws,
                      cudaStream_t s) {
    const PolishLayout L = polish_layout(pr, Kn, J, method, true);
    if (L.fused && steps > 0) {
        float* Xc = reinterpret_cast<float*>(ws + L.Xc);
        float* Sc = reinterpret_cast<float*>(ws + L.Sc);
        double* H = reinterpret_cast<double*>(ws + L.H);
        double* b = reinterpret_cast<double*>(ws + L.b);
        double* Hc = reinterpret_cast<double*>(ws + L.Hc);
        double* bc = reinterpret_cast<double*>(ws + L.bc);
        const int D = K.D;
        AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_sens(K, x, Kn, U, S, H, b, s); }),
                 "sensitivity kernel");
        for (int st = 0; st < steps; ++st) {
            AFM_CUDA(afm::launch_lm_cand(D, Kn, J, x, H, b, kLmLambda0, kLmRatio, Xc, s), "LM trial kernel");
            AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_sens(K, Xc, Kn * J, U, Sc, Hc, bc, s); }),
                     "sensitivity kernel");
            AFM_CUDA(afm::launch_lm_select_hb(D, Kn, J, x, S, H, b, Xc, Sc, Hc, bc, s), "LM select kernel");
        }
        return AFM_OK;
    }
    for (int st = 0; st < steps; ++st) {
        afm_status e = polish_step(ctx, K, method, U, nullptr, nullptr, 1, x, S, Kn, J, L, ws, s);
        if (e) return e;
    }
    if (steps == 0)
        AFM_CUDA(afm::launch_forward_f32(K, x, Kn, nullptr, U, S, nullptr, s), "forward kernel");
    return AFM_OK;
}

afm_status afm_polish_workspace_size(const afm_problem* prob, int K, int n_cand, int method,
                                     size_t* bytes) {
    g_err[0] = 0;
    if (!bytes || K < 1 || n_cand < 1 || n_cand > 64)
        return fail(AFM_ERR_INVALID_ARG, "K >= 1, 1 <= n_cand <= 64 and bytes needed");
    afm_status st = check_problem(prob);
    if (st) return st;
    if (method != AFM_POLISH_STEEPEST && method != AFM_POLISH_LM)
        return fail(AFM_ERR_INVALID_ARG, "unknown polish method %d", method);
    *bytes = polish_layout(*prob, K, n_cand, method, true).total;
    return AFM_OK;
}

afm_status afm_polish(afm_ctx* ctx, const afm_problem* prob, const float* U, float* x, float* S,
                      int K, int steps, int n_cand, int method, void* workspace,
                      size_t workspace_bytes, void* stream) {
    AFM_TRACE("afm_polish");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = modal_only(prob, "afm_polish"))) return st;
    if ((st = check_ctx(ctx))) return st;
    if (!U || !x || !S || !workspace || K < 1 || steps < 0 || prob->n_free < 1)
        return fail(AFM_ERR_INVALID_ARG, "NULL array, K < 1, steps < 0 or no free parameter");
    size_t need = 0;
    if ((st = afm_polish_workspace_size(prob, K, n_cand, method, &need))) return st;
    if (workspace_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(AFM_ERR_INVALID_ARG, "workspace too small (%zu < %zu) or misaligned",
                    workspace_bytes, need);
    KConst<float> K32;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, K32);
    return polish_run(ctx, *prob, K32, U, x, S, K, steps, n_cand, method,
                      static_cast<char*>(workspace), reinterpret_cast<cudaStream_t>(stream));
}

afm_status afm_invert_polished_workspace_size(const afm_problem* prob, const afm_pso_cfg* cfg,
                                              int polish_k, int n_cand, int method, size_t* bytes) {
    g_err[0] = 0;
    if (!bytes) return fail(AFM_ERR_INVALID_ARG, "bytes is NULL");
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = check_pso(cfg, prob->n_free))) return st;
    if (polish_k < 1 || polish_k > cfg->P || n_cand < 1 || n_cand > 64)
        return fail(AFM_ERR_INVALID_ARG, "1 <= polish_k <= P and 1 <= n_cand <= 64 needed");
    if (method != AFM_POLISH_STEEPEST && method != AFM_POLISH_LM)
        return fail(AFM_ERR_INVALID_ARG, "unknown polish method %d", method);
    const size_t inv = invert_layout(cfg->P, prob->n_free).total;
    const size_t xk = align256(sizeof(float) * (size_t)prob->n_free * polish_k);
    const size_t sk = align256(sizeof(float) * (size_t)polish_k);
    const size_t ik = align256(sizeof(int) * (size_t)polish_k);
    *bytes = inv + xk + sk + ik + polish_layout(*prob, polish_k, n_cand, method, true).total +
             reeval_extra(*prob);
    return AFM_OK;
}

afm_status afm_invert_polished(afm_ctx* ctx, const afm_problem* prob, const float* U,
                               const afm_pso_cfg* cfg, int polish_k, int polish_steps, int n_cand,
                               int method, void* workspace, size_t workspace_bytes,
                               afm_result* result, float* history, void* stream) {
    AFM_TRACE("afm_invert_polished");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = modal_only(prob, "afm_invert_polished"))) return st;
    if ((st = check_ctx(ctx))) return st;
    if ((st = check_pso(cfg, prob->n_free))) return st;
    if (!U || !result || !workspace || polish_steps < 0)
        return fail(AFM_ERR_INVALID_ARG, "NULL U, result or workspace, or polish_steps < 0");
    if (cfg->P > 8192) return fail(AFM_ERR_INVALID_ARG, "polished inversion supports P <= 8192");
    size_t need = 0;
    if ((st = afm_invert_polished_workspace_size(prob, cfg, polish_k, n_cand, method, &need)))
        return st;
    if (workspace_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(AFM_ERR_INVALID_ARG, "workspace too small (%zu < %zu) or misaligned",
                    workspace_bytes, need);
    const int D = prob->n_free, P = cfg->P;
    char* ws = static_cast<char*>(workspace);
    const InvLayout L = invert_layout(P, D);
    afm::SwarmPtrs sw;
    afm::detail::carve_swarm(ws, P, D, &sw);
    char* pol = ws + L.total;
    float* xk = reinterpret_cast<float*>(pol);
    pol += align256(sizeof(float) * (size_t)D * polish_k);
    float* sk = reinterpret_cast<float*>(pol);
    pol += align256(sizeof(float) * (size_t)polish_k);
    int* ik = reinterpret_cast<int*>(pol);
    pol += align256(sizeof(int) * (size_t)polish_k);
    KConst<float> Kf;
    KConst<double> Kd;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, Kf);
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, Kd);
    const afm::PsoConst pc = pso_const(*cfg, D);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AFM_CUDA(afm::launch_pso_init(pc, sw, s), "pso init kernel");
    for (int it = 0; it <= cfg->iters; ++it)
        AFM_CUDA(timed_launch(ctx, s, [&] {
                     return afm::launch_invert_iter(Kf, pc, sw, U, history, it, s, ctx->lanes);
                 }),
                 "invert iteration kernel");
    const int fin = (cfg->iters + 1) & 1;
    AFM_CUDA(afm::launch_topk(sw.pbS, sw.pb[fin], P, D, polish_k, xk, ik, s), "top-k kernel");
    if ((st = polish_run(ctx, *prob, Kf, U, xk, sk, polish_k, polish_steps, n_cand, method, pol, s)))
        return st;
    if (reeval_extra(*prob) > 0) {
        afm::ReevalPtrs R;
        afm::reeval_carve(pol + polish_layout(*prob, polish_k, n_cand, method, true).total, problem_modes(*prob),
                          prob->n_steps, prob->steps_per_cycle, &R);
        AFM_CUDA(afm::launch_reeval_pick_min(D, polish_k, xk, sk, ik, R.win, s), "winner pick kernel");
        AFM_CUDA(afm::launch_reeval(Kf, Kd, R, U, cfg->iters, sw.flags, result, s),
                 "FP64 re-evaluation kernels");
        return AFM_OK;
    }
    AFM_CUDA(afm::launch_polish_final(Kd, polish_k, cfg->iters, xk, sk, ik, U, sw.flags, result, s),
             "polish final kernel");
    return AFM_OK;
}

afm_status afm_invert_batch_workspace_size(const afm_problem* probs, int n_prob, int n_pix,
                                           size_t* bytes) {
    g_err[0] = 0;
    if (!bytes || n_pix < 1) return fail(AFM_ERR_INVALID_ARG, "n_pix >= 1 and bytes needed");
    afm_problem eff;
    afm_status st = check_batch_probs(probs, n_prob, n_pix, &eff);
    if (st) return st;
    *bytes = batch_ws_bytes(eff, n_pix) + pix_layout(n_prob, eff.steps_per_cycle).total;
    return AFM_OK;
}

}  // extern "C"

namespace {

// Validation and launch set-up shared by the batched inversions: constants,
// the argument block (queue order sorted on `s`), and the particles per
// thread (forced or autotuned) with the persistent grid size.
struct BatchSetup {
    KConst<float> Kf;
    KConst<double> Kd;
    afm::PsoConst pc;
    afm::BatchArgs a;
    afm::ReevalBatch R;   // FP64 re-evaluation of the winners (after the queue)
    int kp, grid;
};

afm_status batch_setup(afm_ctx* ctx, const afm_problem* probs, int n_prob, const float* U_cat,
                       const int64_t* off, int n_pix, uint32_t pixel0, const afm_pso_cfg* cfg,
                       void* workspace, size_t pix_at, afm_result* results,
                       int* particles_per_thread, cudaStream_t s, const char* who, BatchSetup* out,
                       const afm_batch_select* select = nullptr) {
    afm_problem eff;
    afm_status st = check_batch_probs(probs, n_prob, n_pix, &eff);
    if (st) return st;
    const afm_problem* prob = &eff;
    if ((st = modal_only(prob, who))) return st;
    if ((st = check_ctx(ctx))) return st;
    if ((st = check_pso(cfg, prob->n_free))) return st;
    if (!U_cat || !off || !results || !workspace || n_pix < 1)
        return fail(AFM_ERR_INVALID_ARG, "NULL U_cat, off, results or workspace, or n_pix < 1");
    if (reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(AFM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (cfg->P > 4096) return fail(AFM_ERR_INVALID_ARG, "batched swarms hold at most 4096 particles");
    const size_t smem = afm::batch_smem(cfg->P, prob->n_free, 2 * prob->steps_per_cycle, n_prob > 1);
    if (smem > 200 * 1024)
        return fail(AFM_ERR_INVALID_ARG, "swarm state of %zu bytes exceeds shared memory", smem);
    // queue (and sort order) sized for the pixels inverted
    const int n_run = select != nullptr ? select->n_run : n_pix;
    const BatchLayout L = batch_layout(n_run);
    char* ws = static_cast<char*>(workspace);
    BatchSetup& B = *out;
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, B.Kf);
    fill_kconst(*prob, prob->steps_per_cycle, prob->n_steps, B.Kd);
    afm::reeval_batch_carve(ws + L.total, problem_modes(*prob), prob->n_steps,
                            prob->steps_per_cycle, n_run, &B.R);
    B.pc = pso_const(*cfg, prob->n_free);
    afm::BatchArgs& a = B.a;
    std::memset(&a, 0, sizeof(a));   // also the padding: the struct is part of a graph key
    a.U = U_cat;
    a.off = off;
    a.order = n_pix <= afm::batch_sort_max() ? reinterpret_cast<int*>(ws + L.order) : nullptr;
    a.n_pix = n_pix;
    a.pixel0 = pixel0;
    a.queue = reinterpret_cast<int*>(ws + L.queue);
    a.res = results;
    a.pb_out = nullptr;
    if (select != nullptr) {
        if (!select->pixels || select->n_run < 1 || select->n_seed < 0 ||
            select->n_seed > cfg->P || (select->n_seed > 0 && !select->seeds) ||
            ((select->box_lo == nullptr) != (select->box_hi == nullptr)))
            return fail(AFM_ERR_INVALID_ARG,
                        "select: pixels and n_run >= 1, 0 <= n_seed <= P with seeds, box_lo and "
                        "box_hi both or neither needed");
        a.order = select->pixels;
        a.n_pix = select->n_run;
        a.box_lo = select->box_lo;
        a.box_hi = select->box_hi;
        a.seeds = select->n_seed > 0 ? select->seeds : nullptr;
        a.n_seed = select->n_seed;
    }
    if (n_prob > 1) {
        // every pixel's constants (FP32 and FP64), uploaded to the workspace,
        // and its drive tables computed there
        const PixLayout X = pix_layout(n_prob, prob->steps_per_cycle);
        char* pw = ws + pix_at;
        std::vector<KConst<float>> kf(n_prob);
        std::vector<KConst<double>> kd(n_prob);
        for (int i = 0; i < n_prob; ++i) {
            fill_kconst(probs[i], prob->steps_per_cycle, prob->n_steps, kf[i]);
            fill_kconst(probs[i], prob->steps_per_cycle, prob->n_steps, kd[i]);
        }
        AFM_CUDA(cudaMemcpyAsync(pw + X.kf, kf.data(), sizeof(KConst<float>) * (size_t)n_prob,
                                 cudaMemcpyHostToDevice, s),
                 "per-pixel constants upload");
        AFM_CUDA(cudaMemcpyAsync(pw + X.kd, kd.data(), sizeof(KConst<double>) * (size_t)n_prob,
                                 cudaMemcpyHostToDevice, s),
                 "per-pixel constants upload");
        a.pix.kf = reinterpret_cast<const KConst<float>*>(pw + X.kf);
        a.pix.kd = reinterpret_cast<const KConst<double>*>(pw + X.kd);
        a.pix.tab64 = reinterpret_cast<const double*>(pw + X.t64);
        a.pix.tab32 = reinterpret_cast<const float*>(pw + X.t32);
        a.pix.ld = X.ld;
        AFM_CUDA(afm::launch_pix_tables(a.pix, n_prob, 2 * prob->steps_per_cycle, s),
                 "per-pixel drive tables");
    }
    // queue order (longest record first) is needed by the tuner's probe too
    if (a.order && select == nullptr)
        AFM_CUDA(afm::batch_sort(off, n_pix, const_cast<int*>(a.order), s), "sort kernel");
    int kp = 0, occ = 0;
    const int want = particles_per_thread ? *particles_per_thread : 0;
    const afm::PsoConst& pc = B.pc;
    if (want == 1 || want == 2 || want == 4) {
        if (afm::batch_threads(pc.P, want) > afm::batch_max_threads(want) || (want > 1 && B.Kf.m > 3))
            return fail(AFM_ERR_INVALID_ARG, "particles_per_thread %d unsupported here", want);
        kp = want;
        AFM_CUDA(afm::batch_occupancy(B.Kf.m, B.Kf.force, kp, pc.P, pc.D, B.Kf.spc2, n_prob > 1,
                                      &occ),
                 "batch occupancy");
        if (occ < 1) return fail(AFM_ERR_UNSUPPORTED, "batch kernel does not fit (P = %d)", pc.P);
    } else if (want != 0) {
        return fail(AFM_ERR_INVALID_ARG, "particles_per_thread must be 0 (tune), 1, 2 or 4");
    } else if ((st = batch_tune(ctx, B.Kf, pc, a, s, &kp, &occ))) {
        return st;
    }
    B.kp = kp;
    B.grid = std::min(a.n_pix, ctx->num_sms * occ);
    if (particles_per_thread) *particles_per_thread = kp;
    return AFM_OK;
}

}  // namespace

extern "C" {

afm_status afm_invert_batch(afm_ctx* ctx, const afm_problem* probs, int n_prob,
                            const float* U_cat, const int64_t* off, int n_pix, uint32_t pixel0,
                            const afm_pso_cfg* cfg, void* workspace, size_t workspace_bytes,
                            afm_result* results, int* particles_per_thread, void* stream) {
    AFM_TRACE("afm_invert_batch");
    g_err[0] = 0;
    if (n_pix < 1) return fail(AFM_ERR_INVALID_ARG, "n_pix must be >= 1");
    afm_problem eff;
    afm_status st0;
    if ((st0 = check_batch_probs(probs, n_prob, n_pix, &eff))) return st0;
    const size_t pix_at = batch_ws_bytes(eff, n_pix);
    const size_t need = pix_at + pix_layout(n_prob, eff.steps_per_cycle).total;
    if (workspace_bytes < need)
        return fail(AFM_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchSetup B;
    afm_status st = batch_setup(ctx, probs, n_prob, U_cat, off, n_pix, pixel0, cfg, workspace,
                                pix_at, results, particles_per_thread, s, "afm_invert_batch", &B);
    if (st) return st;
    const KConst<float>& Kf = B.Kf;
    const KConst<double>& Kd = B.Kd;
    const afm::PsoConst& pc = B.pc;
    const afm::BatchArgs& a = B.a;
    const int kp = B.kp, grid = B.grid;
    // one graph: zero the queue, sort, persistent swarm kernel, FP64 winners
    std::vector<unsigned char> key;
    append_bytes(key, Kf);
    append_bytes(key, Kd);
    append_bytes(key, pc);
    append_bytes(key, a);
    append_bytes(key, kp);
    append_bytes(key, grid);
    afm_batch_graph* G = nullptr;
    for (auto& g : ctx->batch_graphs)
        if (g.key == key) G = &g;
    if (!G) {
        if (!ctx->capture_stream)
            AFM_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking),
                     "cudaStreamCreate");
        afm_batch_graph g{};
        g.key = key;
        AFM_CUDA(cudaEventCreate(&g.ev_own[0]), "cudaEventCreate");
        if (cudaEventCreate(&g.ev_own[1]) != cudaSuccess) {
            cudaEventDestroy(g.ev_own[0]);
            return fail(AFM_ERR_CUDA, "cudaEventCreate failed");
        }
        auto drop = [&](cudaError_t err, const char* where) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            cudaEventDestroy(g.ev_own[0]);
            cudaEventDestroy(g.ev_own[1]);
            return cuda_fail(err, where);
        };
        cudaStream_t c = ctx->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return drop(e, "begin capture");
        e = cudaMemsetAsync(a.queue, 0, sizeof(int), c);
        if (e == cudaSuccess && a.order) e = afm::batch_sort(off, n_pix, const_cast<int*>(a.order), c);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(g.ev_own[0], c, cudaEventRecordExternal);
        if (e == cudaSuccess) e = afm::launch_batch(Kf, pc, a, kp, grid, c);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(g.ev_own[1], c, cudaEventRecordExternal);
        if (e == cudaSuccess) e = afm::launch_reeval_batch(Kf, Kd, B.R, a, c);
        cudaError_t e2 = cudaStreamEndCapture(c, &g.graph);
        if (e != cudaSuccess) return drop(e, "batch graph capture");
        if (e2 != cudaSuccess) return drop(e2, "cudaStreamEndCapture");
        // the two event-record nodes around the swarm kernel
        size_t n_nodes = 0;
        if ((e = cudaGraphGetNodes(g.graph, nullptr, &n_nodes)) != cudaSuccess)
            return drop(e, "cudaGraphGetNodes");
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if ((e = cudaGraphGetNodes(g.graph, nodes.data(), &n_nodes)) != cudaSuccess)
            return drop(e, "cudaGraphGetNodes");
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            cudaEvent_t ev = nullptr;
            if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord ||
                cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess)
                continue;
            if (ev == g.ev_own[0]) g.ev_node[0] = nd;
            if (ev == g.ev_own[1]) g.ev_node[1] = nd;
        }
        if (!g.ev_node[0] || !g.ev_node[1])
            return drop(cudaErrorInvalidValue, "batch graph: event nodes not found");
        if ((e = cudaGraphInstantiate(&g.exec, g.graph, 0)) != cudaSuccess)
            return drop(e, "cudaGraphInstantiate");
        if (ctx->batch_graphs.size() >= 8) {
            afm_batch_graph& old = ctx->batch_graphs.front();
            cudaGraphExecDestroy(old.exec);
            cudaGraphDestroy(old.graph);
            cudaEventDestroy(old.ev_own[0]);
            cudaEventDestroy(old.ev_own[1]);
            ctx->batch_graphs.erase(ctx->batch_graphs.begin());
        }
        ctx->batch_graphs.push_back(g);
        G = &ctx->batch_graphs.back();
    }
    if (ctx->profiling) {
        // a fresh event pair per launch, read back by afm_profile_read
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        AFM_CUDA(take_event(ctx, &e0), "cudaEventCreate");
        AFM_CUDA(take_event(ctx, &e1), "cudaEventCreate");
        AFM_CUDA(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_node[0], e0), "event node");
        AFM_CUDA(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_node[1], e1), "event node");
        AFM_CUDA(cudaGraphLaunch(G->exec, s), "cudaGraphLaunch");
        ctx->ev_pending.emplace_back(e0, e1);
        return AFM_OK;
    }
    AFM_CUDA(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_node[0], G->ev_own[0]), "event node");
    AFM_CUDA(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_node[1], G->ev_own[1]), "event node");
    AFM_CUDA(cudaGraphLaunch(G->exec, s), "cudaGraphLaunch");
    return AFM_OK;
}

// Workspace of the polished batch: the batch queue, every slot's final
// personal bests, the Kc candidates per slot, then the polish workspace of
// all n_pix * Kc candidates (polish_layout, checkpoints for the longest
// record).
struct BatchPolishLayout {
    size_t pb, xk, Sk, ik, pol, total;
    PolishLayout P;
};

static BatchPolishLayout batch_polish_layout(const afm_problem& pr, const afm_pso_cfg& cfg, int n_pix,
                                             int Kc, int J, int method) {
    BatchPolishLayout L;
    const size_t D = (size_t)pr.n_free, P = (size_t)cfg.P, Nt = (size_t)n_pix * Kc;
    size_t off = batch_ws_bytes(pr, n_pix);
    L.pb = off; off += align256(sizeof(float) * (size_t)n_pix * (D + 1) * P);
    L.xk = off; off += align256(sizeof(float) * D * Nt);
    L.Sk = off; off += align256(sizeof(float) * Nt);
    L.ik = off; off += align256(sizeof(int) * Nt);
    L.pol = off;
    L.P = polish_layout(pr, (int)Nt, J, method, false);
    L.total = off + L.P.total;
    return L;
}

static afm_status check_batch_polish(const afm_problem* prob, const afm_pso_cfg* cfg, int n_pix,
                                     int polish_k, int n_cand, int method) {
    if (!prob || !cfg) return fail(AFM_ERR_INVALID_ARG, "NULL prob or cfg");
    if (method != AFM_POLISH_STEEPEST && method != AFM_POLISH_LM)
        return fail(AFM_ERR_INVALID_ARG, "unknown polish method %d", method);
    if (n_pix < 1 || polish_k < 1 || polish_k > cfg->P || n_cand < 1 || n_cand > 64)
        return fail(AFM_ERR_INVALID_ARG, "n_pix >= 1, 1 <= polish_k <= P and 1 <= n_cand <= 64 needed");
    if ((size_t)n_pix * polish_k * n_cand > (size_t)1 << 30)
        return fail(AFM_ERR_INVALID_ARG, "n_pix x polish_k x n_cand too large");
    if (cfg->P > 4096) return fail(AFM_ERR_INVALID_ARG, "batched swarms hold at most 4096 particles");
    return AFM_OK;
}

afm_status afm_invert_batch_polished_workspace_size(const afm_problem* probs, int n_prob,
                                                    const afm_pso_cfg* cfg, int n_run,
                                                    int polish_k, int n_cand, int method,
                                                    size_t* bytes) {
    g_err[0] = 0;
    if (!bytes) return fail(AFM_ERR_INVALID_ARG, "bytes is NULL");
    afm_status st = check_batch_polish(probs, cfg, n_run, polish_k, n_cand, method);
    if (st) return st;
    afm_problem eff;
    if ((st = check_batch_probs(probs, n_prob, n_prob > 1 ? n_prob : 1, &eff))) return st;
    *bytes = batch_polish_layout(eff, *cfg, n_run, polish_k, n_cand, method).total +
             pix_layout(n_prob, eff.steps_per_cycle).total;
    return AFM_OK;
}

static afm_status batch_polished_run(afm_ctx* ctx, const afm_problem* prob, const BatchSetup& B,
                                     const BatchPolishLayout& PL, const float* U_cat,
                                     const int64_t* off, const afm_pso_cfg* cfg, int polish_k,
                                     int polish_steps, int n_cand, int method, char* ws,
                                     afm_result* results, cudaStream_t s);

afm_status afm_invert_batch_polished(afm_ctx* ctx, const afm_problem* probs, int n_prob,
                                     const float* U_cat, const int64_t* off, int n_pix,
                                     uint32_t pixel0, const afm_pso_cfg* cfg, int polish_k,
                                     int polish_steps, int n_cand, int method,
                                     const afm_batch_select* select, void* workspace,
                                     size_t workspace_bytes, afm_result* results,
                                     int* particles_per_thread, void* stream) {
    AFM_TRACE("afm_invert_batch_polished");
    g_err[0] = 0;
    const int n_run = select ? select->n_run : n_pix;
    afm_status st = check_batch_polish(probs, cfg, n_run, polish_k, n_cand, method);
    if (st) return st;
    if (polish_steps < 0) return fail(AFM_ERR_INVALID_ARG, "polish_steps < 0");
    afm_problem eff;
    if ((st = check_batch_probs(probs, n_prob, n_pix, &eff))) return st;
    if (n_prob > 1 && method != AFM_POLISH_LM)
        return fail(AFM_ERR_UNSUPPORTED,
                    "per-pixel problems are polished by Levenberg-Marquardt (AFM_POLISH_LM) only");
    const BatchPolishLayout PL = batch_polish_layout(eff, *cfg, n_run, polish_k, n_cand, method);
    const size_t need = PL.total + pix_layout(n_prob, eff.steps_per_cycle).total;
    if (workspace_bytes < need)
        return fail(AFM_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchSetup B;
    if ((st = batch_setup(ctx, probs, n_prob, U_cat, off, n_pix, pixel0, cfg, workspace, PL.total,
                          results, particles_per_thread, s, "afm_invert_batch_polished", &B,
                          select)))
        return st;
    return batch_polished_run(ctx, &eff, B, PL, U_cat, off, cfg, polish_k, polish_steps, n_cand,
                              method, static_cast<char*>(workspace), results, s);
}

static afm_status batch_polished_run(afm_ctx* ctx, const afm_problem* prob, const BatchSetup& B,
                                     const BatchPolishLayout& PL, const float* U_cat,
                                     const int64_t* off, const afm_pso_cfg* cfg, int polish_k,
                                     int polish_steps, int n_cand, int method, char* ws,
                                     afm_result* results, cudaStream_t s) {
    afm_status st = AFM_OK;
    afm::BatchArgs a = B.a;
    const int n_pix = a.n_pix;   // queue slots
    a.pb_out = reinterpret_cast<float*>(ws + PL.pb);
    float* xk = reinterpret_cast<float*>(ws + PL.xk);
    float* Sk = reinterpret_cast<float*>(ws + PL.Sk);
    int* ik = reinterpret_cast<int*>(ws + PL.ik);
    const int D = prob->n_free, Kc = polish_k, J = n_cand, Nt = n_pix * Kc;
    AFM_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), s), "cudaMemsetAsync");
    AFM_CUDA(timed_launch(ctx, s, [&] { return afm::launch_batch(B.Kf, B.pc, a, B.kp, B.grid, s); }),
             "batch kernel");
    AFM_CUDA(afm::launch_topk_pix(a.pb_out, n_pix, cfg->P, D, Kc, xk, Sk, ik, s), "top-k kernel");
    for (int k = 0; k < polish_steps; ++k)
        if ((st = polish_step(ctx, B.Kf, method, U_cat, off, a.order, Kc, xk, Sk, Nt, J, PL.P,
                              ws + PL.pol, s, a.pix)))
            return st;
    AFM_CUDA(afm::launch_pick_pix(n_pix, D, Kc, xk, Sk, ik, a.order, cfg->iters, results, s),
             "winner pick kernel");
    AFM_CUDA(afm::launch_reeval_batch(B.Kf, B.Kd, B.R, a, s), "batch FP64 re-evaluation");
    return AFM_OK;
}

// Image scan workspace: the coarse and fine pixel lists, the fine pixels'
// boxes and seeds, then one polished-batch workspace for the larger pass.
struct ImageLayout {
    size_t coarse, fine, blo, bhi, seeds, batch, total;
    int n_coarse, n_fine;
};

static afm_status image_layout(const afm_problem& pr, const afm_image_cfg& ic, ImageLayout* L) {
    if (ic.width < 1 || ic.height < 1 || ic.stride < 2 || !(ic.margin >= 0.0) || ic.margin > 1.0)
        return fail(AFM_ERR_INVALID_ARG, "width, height >= 1, stride >= 2, 0 <= margin <= 1 needed");
    if ((size_t)ic.width * ic.height > (size_t)1 << 26)
        return fail(AFM_ERR_INVALID_ARG, "image too large");
    afm::image_counts(ic.width, ic.height, ic.stride, &L->n_coarse, &L->n_fine);
    const size_t D = (size_t)pr.n_free;
    const int nf = std::max(L->n_fine, 1);
    size_t off = 0;
    L->coarse = off; off += align256(sizeof(int) * (size_t)L->n_coarse);
    L->fine = off; off += align256(sizeof(int) * (size_t)nf);
    L->blo = off; off += align256(sizeof(float) * (size_t)nf * D);
    L->bhi = off; off += align256(sizeof(float) * (size_t)nf * D);
    L->seeds = off; off += align256(sizeof(float) * (size_t)nf * 4 * D);
    L->batch = off;
    afm_status st = check_batch_polish(&pr, &ic.coarse, L->n_coarse, ic.coarse_polish_k, ic.n_cand,
                                       ic.method);
    if (st) return st;
    if (L->n_fine > 0 &&
        (st = check_batch_polish(&pr, &ic.fine, L->n_fine, ic.fine_polish_k, ic.n_cand, ic.method)))
        return st;
    if (ic.fine.P < 4 && L->n_fine > 0)
        return fail(AFM_ERR_INVALID_ARG, "the fine swarm needs P >= 4 (4 seed particles)");
    const size_t bc = batch_polish_layout(pr, ic.coarse, L->n_coarse, ic.coarse_polish_k, ic.n_cand,
                                          ic.method).total;
    const size_t bf = L->n_fine > 0 ? batch_polish_layout(pr, ic.fine, L->n_fine, ic.fine_polish_k,
                                                          ic.n_cand, ic.method).total
                                    : 0;
    L->total = off + std::max(bc, bf);
    return AFM_OK;
}

afm_status afm_invert_image_workspace_size(const afm_problem* prob, const afm_image_cfg* icfg,
                                           size_t* bytes) {
    g_err[0] = 0;
    if (!prob || !icfg || !bytes) return fail(AFM_ERR_INVALID_ARG, "NULL prob, icfg or bytes");
    afm_status st = check_problem(prob);
    if (st) return st;
    ImageLayout L;
    if ((st = image_layout(*prob, *icfg, &L))) return st;
    *bytes = L.total;
    return AFM_OK;
}

afm_status afm_invert_image(afm_ctx* ctx, const afm_problem* prob, const float* U_cat,
                            const int64_t* off, uint32_t pixel0, const afm_image_cfg* icfg,
                            void* workspace, size_t workspace_bytes, afm_result* results,
                            void* stream) {
    AFM_TRACE("afm_invert_image");
    g_err[0] = 0;
    if (!prob || !icfg) return fail(AFM_ERR_INVALID_ARG, "NULL prob or icfg");
    afm_status st = check_problem(prob);
    if (st) return st;
    ImageLayout L;
    if ((st = image_layout(*prob, *icfg, &L))) return st;
    if (!workspace || workspace_bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(AFM_ERR_INVALID_ARG, "workspace NULL, misaligned or < %zu bytes", L.total);
    const afm_image_cfg& ic = *icfg;
    const int n_pix = ic.width * ic.height, D = prob->n_free;
    char* ws = static_cast<char*>(workspace);
    int* coarse = reinterpret_cast<int*>(ws + L.coarse);
    int* fine = reinterpret_cast<int*>(ws + L.fine);
    float* blo = reinterpret_cast<float*>(ws + L.blo);
    float* bhi = reinterpret_cast<float*>(ws + L.bhi);
    float* seeds = reinterpret_cast<float*>(ws + L.seeds);
    char* bws = ws + L.batch;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AFM_CUDA(afm::launch_image_plan(ic.width, ic.height, ic.stride, coarse, fine, s), "image plan kernel");
    // pass 1: the coarse pixels, full search
    afm_batch_select sel{};
    sel.pixels = coarse;
    sel.n_run = L.n_coarse;
    BatchSetup B;
    if ((st = batch_setup(ctx, prob, 1, U_cat, off, n_pix, pixel0, &ic.coarse, bws, 0, results,
                          nullptr, s, "afm_invert_image", &B, &sel)))
        return st;
    BatchPolishLayout PL = batch_polish_layout(*prob, ic.coarse, L.n_coarse, ic.coarse_polish_k,
                                               ic.n_cand, ic.method);
    if ((st = batch_polished_run(ctx, prob, B, PL, U_cat, off, &ic.coarse, ic.coarse_polish_k,
                                 ic.coarse_polish_steps, ic.n_cand, ic.method, bws, results, s)))
        return st;
    if (L.n_fine == 0) return AFM_OK;
    // pass 2: every other pixel inside the box of its coarse neighbours' winners
    AFM_CUDA(afm::launch_image_prior(ic.width, ic.height, ic.stride, D, (float)ic.margin, results, fine,
                                     L.n_fine, blo, bhi, seeds, s),
             "image prior kernel");
    sel.pixels = fine;
    sel.n_run = L.n_fine;
    sel.box_lo = blo;
    sel.box_hi = bhi;
    sel.seeds = seeds;
    sel.n_seed = 4;
    if ((st = batch_setup(ctx, prob, 1, U_cat, off, n_pix, pixel0, &ic.fine, bws, 0, results,
                          nullptr, s, "afm_invert_image", &B, &sel)))
        return st;
    PL = batch_polish_layout(*prob, ic.fine, L.n_fine, ic.fine_polish_k, ic.n_cand, ic.method);
    return batch_polished_run(ctx, prob, B, PL, U_cat, off, &ic.fine, ic.fine_polish_k,
                              ic.fine_polish_steps, ic.n_cand, ic.method, bws, results, s);
}

afm_status afm_synth_records(afm_ctx* ctx, const afm_problem* prob, const double* x_truth,
                             int n_pix, const int64_t* off, int sub, double sigma_m,
                             uint64_t seed, uint32_t pixel0, float* U_cat, void* stream) {
    AFM_TRACE("afm_synth_records");
    g_err[0] = 0;
    afm_status st = check_problem(prob);
    if (st) return st;
    if ((st = modal_only(prob, "afm_synth_records"))) return st;
    if ((st = check_ctx(ctx))) return st;
    if (n_pix < 1 || !off || !U_cat || (prob->n_free > 0 && !x_truth))
        return fail(AFM_ERR_INVALID_ARG, "n_pix >= 1 and non-NULL off, U_cat, x_truth needed");
    if (sub < 1 || (long)prob->steps_per_cycle * sub > AFM_TAB_MAX / 2)
        return fail(AFM_ERR_INVALID_ARG, "sub %d: steps_per_cycle * sub must be <= %d", sub,
                    AFM_TAB_MAX / 2);
    if (!(sigma_m >= 0) || !std::isfinite(sigma_m)) return fail(AFM_ERR_INVALID_ARG, "sigma must be >= 0");
    KConst<float> K;
    fill_kconst(*prob, prob->steps_per_cycle * sub, prob->n_steps * sub, K);
    AFM_CUDA(afm::launch_synth(K, x_truth, n_pix, off, sub, (float)(sigma_m / 1e-9), seed, pixel0,
                               U_cat, reinterpret_cast<cudaStream_t>(stream)),
             "synth kernel");
    return AFM_OK;
}

}  // extern "C"
