// Host set-up and C ABI of the FDLB solver (see include/fdlb.h).
//
// Everything here is built from the paper's definitions, independently of any
// other implementation:
//  * Gauss rules (Sec. III A 2 half-range, App. A full-range): recurrence
//    coefficients of the orthonormal polynomials by the Stieltjes procedure on a
//    discretised weight (composite Gauss-Legendre), nodes as eigenvalues of the
//    Jacobi matrix (Sturm-sequence bisection, Newton polish), Christoffel weights.
//  * 6th-order gradient stencils (Sec. III B 3) with one-sided / biased 7-point
//    stencils at the 3 nodes next to a wall (solved from the moment conditions).
//  * Grid mapping, time step, workspace layout, work lists, error handling.
#include "fdlb_internal.h"
#include "fdlb_launch.h"
#include "fdlb_ctx_internal.h"
#include "../../include/fdlb.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace fdlb;

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

struct fdlb_ctx {
    int count = 0;
    std::vector<fdlb_params> prm;
    std::vector<Inst> inst;           // host copies (device pointers inside)
    Inst* d_inst = nullptr;
    Work* d_upd = nullptr;
    Work* d_nod = nullptr;
    int n_upd = 0, n_nod = 0, qmax = 1;
    int* d_list = nullptr;            // count ints: instances in resident-cluster order
    int* d_status_all = nullptr;      // count ints (Inst::status points here)
    long long* d_steps_all = nullptr;
    double* d_resid_all = nullptr;    // count doubles (misc[M_RESID] copies)
    cudaStream_t stream = nullptr;
    size_t smem_upd_f64 = 0, smem_upd_f32 = 0;
    bool any_fp32 = false, any_fp64 = false;
    int ukc_max = 1;
    // schedule (FDLB_SCHED_*): requested, and the one in use once chosen (0 = not yet)
    int sched_req = FDLB_SCHED_AUTO, sched = 0;
    int cs = 0;                       // CTAs per cluster of the resident schedule (0: unavailable)
    size_t res_smem = 0;
    // shared-memory-resident schedule (part of FDLB_SCHED_MIXED): the instances whose three RK
    // buffers fit in one block's shared memory, stepped by k_smemres on a second stream
    int* d_smem_list = nullptr;       // count ints (the first n_smem used)
    std::vector<int> smem_idx;
    int n_smem = 0, smem_qmax = 1;
    size_t smem_scratch = 0, smem_dyn = 0;
    bool smem_flags = false;          // smem_res set on the device for the listed instances
    std::string smem_note;            // how the set was chosen (for the error message)
    cudaStream_t stream2 = nullptr;   // created on first use of FDLB_SCHED_MIXED
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    // update blocks of 16 warps (the same results as 8) while the active instances' update blocks
    // fit on the SMs at once: a 16-warp block holds a whole SM's registers, so with more blocks
    // than SMs it would run in waves
    int n_sms = 0;
    std::vector<int> upd_blocks;      // update work items of each instance
    bool upd_wide = false;            // in use: fdlb_step keeps the choice made at creation (all
    bool upd_wide_all = false;        // instances active); fdlb_run re-chooses at each status check
    // CUDA graph of GRAPH_STEPS steps for one freeze tolerance and update width (replayed by
    // fdlb_step)
    cudaGraphExec_t graph = nullptr;
    double graph_tol = -1.0;
    bool graph_wide = false;
    bool graph_failed = false;
    // optional per-kernel-class event timing (fdlb_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev[KK_COUNT];
    size_t nev[KK_COUNT] = {0, 0, 0, 0};
    ~fdlb_ctx() {
        for (auto& v : ev)
            for (auto e : v) cudaEventDestroy(e);
        if (graph) cudaGraphExecDestroy(graph);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (stream2) cudaStreamDestroy(stream2);
    }
};

static void choose_cluster(fdlb_ctx* c);
static void choose_smem_resident(fdlb_ctx* c);
static void choose_update_width(fdlb_ctx* c, const int* st);

// Record a start/stop event pair around one launch of class `kind` when profiling is on.
static cudaError_t prof_mark(fdlb_ctx* c, int kind) {
    if (!c->prof) return cudaSuccess;
    auto& v = c->ev[kind];
    if (c->nev[kind] >= v.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        v.push_back(e);
    }
    return cudaEventRecord(v[c->nev[kind]++], c->stream);
}

// One TVD-RK3 step (Eq. rk3): three stages of moments -> closure -> update, then the
// moments of the new state and the residual/status pass.  The stage-1 moments are the
// end-of-step moments of the previous step.
static cudaError_t step_once(fdlb_ctx* c, double freeze_tol) {
    cudaError_t e = cudaSuccess;
    auto guard = [&](int kind, auto&& fn) {
        if (e != cudaSuccess) return;
        e = prof_mark(c, kind);
        if (e == cudaSuccess) e = fn();
        if (e == cudaSuccess) e = prof_mark(c, kind);
    };
    // the update kernel's epilogue computes the moments of each stage's result
    for (int stage = 1; stage <= 3; ++stage) {
        guard(KK_NODAL, [&] { return launch_nodal(c->d_inst, c->d_nod, c->n_nod, c->qmax, c->stream); });
        guard(KK_UPDATE, [&] { return launch_update(c->d_inst, c->d_upd, c->n_upd, stage, c->smem_upd_f64, c->smem_upd_f32,
                                                    c->any_fp64, c->any_fp32, c->upd_wide, c->stream); });
    }
    guard(KK_RESID, [&] { return launch_resid(c->d_inst, c->count, -2, freeze_tol, c->d_resid_all, c->stream); });
    return e;
}

static int fail(fdlb_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    g_err = msg;
    return code;
}

static int cuda_check(fdlb_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FDLB_OK;
    return fail(c, FDLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" int32_t fdlb_abi_version(void) { return FDLB_ABI_VERSION; }

extern "C" const char* fdlb_last_error(const fdlb_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

// ---------------------------------------------------------------------------
// quadrature
// ---------------------------------------------------------------------------
namespace {

// Gauss-Legendre rule on [-1, 1] (Newton on the Legendre three-term recurrence).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs((double)dz) < 1e-19) break;
        }
        x[i] = (double)z;
        w[i] = (double)(2 / ((1 - z * z) * dp * dp));
    }
}

// Monic recurrence pi_{l+1} = (p - alpha_l) pi_l - beta_l pi_{l-1}, l = 0..L-1, for the
// half-range weight omega(p) = exp(-p^2/2)/sqrt(2 pi) on [0, inf), by the Stieltjes
// procedure on the discrete measure of a composite Gauss-Legendre rule on [0, 32] (panels
// of width 1/4; the weight is below 1e-222 beyond, where the polynomials of the orders up to
// 101 have long passed their largest zero, ~22.3 at order 101); beta_0 = mass = 1/2.  The
// monic values stay below 32^101 and their squares times the weight in range.
void half_range_recurrence(int L, std::vector<double>& alpha, std::vector<double>& beta) {
    std::vector<double> gx, gw;
    const int npt = 24, panels = 128;
    gauss_legendre(npt, gx, gw);
    const double hi = 32.0, h = hi / panels;
    std::vector<double> t, W;
    for (int pnl = 0; pnl < panels; ++pnl)
        for (int j = 0; j < npt; ++j) {
            double x = (pnl + 0.5) * h + 0.5 * h * gx[j];
            t.push_back(x);
            W.push_back(0.5 * h * gw[j] * std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI));
        }
    const size_t P = t.size();
    std::vector<double> pm(P, 0.0), pc(P, 1.0), pn(P);
    alpha.assign(L, 0.0);
    beta.assign(L, 0.0);
    double norm_prev = 1.0;
    // the inner products summed with Neumaier's compensated summation (the terms span many
    // orders of magnitude at high degree)
    auto csum = [](double& s, double& c, double v) {
        const double t2 = s + v;
        c += std::fabs(s) >= std::fabs(v) ? (s - t2) + v : (v - t2) + s;
        s = t2;
    };
    for (int l = 0; l < L; ++l) {
        double nrm = 0, xn = 0, cn = 0, cx = 0;
        for (size_t j = 0; j < P; ++j) {
            const double q = W[j] * pc[j] * pc[j];
            csum(nrm, cn, q);
            csum(xn, cx, q * t[j]);
        }
        nrm += cn;
        xn += cx;
        alpha[l] = (double)(xn / nrm);
        beta[l] = (double)(l == 0 ? nrm : nrm / norm_prev);
        for (size_t j = 0; j < P; ++j) pn[j] = (t[j] - (double)alpha[l]) * pc[j] - (double)beta[l] * pm[j];
        pm.swap(pc);
        pc.swap(pn);
        norm_prev = nrm;
    }
}

struct Rule {
    std::vector<double> x, w;     // nodes (ascending), weights
    std::vector<double> alpha;    // alpha_l, l < Q+1
    std::vector<double> beta;     // beta_l (beta_0 = total mass), l < Q+1
};

// Eigenvalues of the symmetric tridiagonal Jacobi matrix (diag alpha, off-diagonal
// sqrt(beta_l), l = 1..Q-1) by Sturm-count bisection, polished by Newton on pi_Q.
void jacobi_nodes(int Q, const std::vector<double>& alpha, const std::vector<double>& beta, std::vector<double>& x) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < Q; ++i) {
        double r = (i > 0 ? std::sqrt(beta[i]) : 0.0) + (i + 1 < Q ? std::sqrt(beta[i + 1]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    auto count_below = [&](double s) {
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < Q; ++i) {
            d = (alpha[i] - s) - (i > 0 ? beta[i] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0) ++cnt;
        }
        return cnt;
    };
    x.assign(Q, 0.0);
    for (int k = 0; k < Q; ++k) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, std::fabs(a)); ++it) {
            double m = 0.5 * (a + b);
            if (count_below(m) > k) b = m; else a = m;
        }
        double z = 0.5 * (a + b);
        for (int it = 0; it < 5; ++it) {      // Newton on the monic pi_Q
            double p0 = 1, p1 = z - alpha[0], d0 = 0, d1 = 1;
            for (int l = 1; l < Q; ++l) {
                double p2 = (z - alpha[l]) * p1 - beta[l] * p0;
                double d2 = p1 + (z - alpha[l]) * d1 - beta[l] * d0;
                p0 = p1; p1 = p2; d0 = d1; d1 = d2;
            }
            if (Q == 1) { p1 = z - alpha[0]; d1 = 1; }
            if (d1 == 0) break;
            z -= p1 / d1;
        }
        x[k] = (double)z;
    }
}

// Orthonormal polynomial values h_0..h_{L-1} at x from the monic recurrence.
void ortho_values(int L, const std::vector<double>& alpha, const std::vector<double>& beta, double x,
                  std::vector<double>& h) {
    h.assign(L, 0.0);
    double hm = 0.0, hc = 1.0 / std::sqrt((double)beta[0]);
    for (int l = 0; l < L; ++l) {
        h[l] = hc;
        if (l + 1 < L) {
            double bn = std::sqrt((double)beta[l + 1]);
            double b = l > 0 ? std::sqrt((double)beta[l]) : 0.0;
            double hn = ((x - alpha[l]) * hc - b * hm) / bn;
            hm = hc;
            hc = hn;
        }
    }
}

Rule make_rule_uncached(int kind, int Q) {
    Rule r;
    if (kind == 0) {
        half_range_recurrence(Q + 1, r.alpha, r.beta);
    } else {
        r.alpha.assign(Q + 1, 0.0);
        r.beta.resize(Q + 1);
        r.beta[0] = 1.0;
        for (int l = 1; l <= Q; ++l) r.beta[l] = l;     // He_{l+1} = p He_l - l He_{l-1}
    }
    jacobi_nodes(Q, r.alpha, r.beta, r.x);
    r.w.resize(Q);
    std::vector<double> h;
    for (int k = 0; k < Q; ++k) {
        ortho_values(Q, r.alpha, r.beta, r.x[k], h);
        double s = 0;
        for (int l = 0; l < Q; ++l) s += h[l] * h[l];
        r.w[k] = (double)(1.0 / s);
    }
    return r;
}

// Rules depend only on (kind, Q): cache them (large batches repeat a few orders).
Rule make_rule(int kind, int Q) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, Rule> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(kind, Q);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    Rule r = make_rule_uncached(kind, Q);
    cache.emplace(key, r);
    return r;
}

// Weights c_j, j = 0..6, with sum_j c_j F(j) = F'(x0) for polynomials of degree <= 6:
// c_j = l_j'(x0) for the Lagrange basis on the integer nodes 0..6.  Every product below is
// an exact integer in double arithmetic; each term is rounded once.
void stencil7(int x0, double* c) {
    for (int j = 0; j < 7; ++j) {
        double den = 1.0;
        for (int l = 0; l < 7; ++l)
            if (l != j) den *= (double)(j - l);
        double num = 0.0;
        for (int m = 0; m < 7; ++m) {
            if (m == j) continue;
            double prod = 1.0;
            for (int l = 0; l < 7; ++l)
                if (l != j && l != m) prod *= (double)(x0 - l);
            num += prod;
        }
        c[j] = num / den;
    }
}

double chi_cs(double eta) { return (2.0 - eta) / (2.0 * (1.0 - eta) * (1.0 - eta) * (1.0 - eta)); }

int validate(const fdlb_params& p, std::string& why) {
    auto bad = [&](const char* m) { why = m; return FDLB_EINVAL; };
    if (p.struct_size != sizeof(fdlb_params)) return bad("struct_size != sizeof(fdlb_params)");
    if (p.nx < 8 || p.nx > 4096) return bad("nx must be in [8, 4096]");
    if (p.qx_half < 1) return bad("qx_half must be >= 1");
    if (p.x_quadrature == FDLB_XQ_HALF && p.qx_half > QX_HALF_MAX) return bad("qx_half must be in [1, 100] (half-range x)");
    if (p.qy != 0 && (p.qy < 2 || p.qy > QYMAX)) return bad("qy must be 0 or in [2, 8]");
    if (p.qz != 0 && (p.qz < 3 || p.qz > QZMAX)) return bad("qz must be 0 or in [3, 8]");
    if (p.qy == 0 && p.qz != 0) return bad("qy == 0 (1D reduced) requires qz == 0");
    if (p.qy == 0 && (p.U_left != 0 || p.U_right != 0 || p.accel_y != 0))
        return bad("the 1D reduced form (qy == 0) has no y motion: walls at rest, no force");
    if (p.grid != FDLB_GRID_UNIFORM && p.grid != FDLB_GRID_TANH) return bad("unknown grid");
    if (p.grid == FDLB_GRID_TANH && !(p.stretch > 0)) return bad("stretch must be > 0");
    if (p.precision != FDLB_FP64 && p.precision != FDLB_FP32_STORAGE && p.precision != FDLB_FP32_THEN_FP64)
        return bad("unknown precision");
    if (p.j1_shear != 0 && p.j1_shear != 1) return bad("j1_shear must be 0 or 1");
    if (p.chi_model != FDLB_CHI_SET && p.chi_model != FDLB_CHI_RET_FM) return bad("unknown chi_model");
    if (p.chi_model == FDLB_CHI_RET_FM && !(p.eta0 > 0)) return bad("chi_model RET-FM needs eta0 > 0");
    if (p.x_quadrature != FDLB_XQ_HALF && p.x_quadrature != FDLB_XQ_FULL) return bad("unknown x_quadrature");
    if (p.x_quadrature == FDLB_XQ_FULL && p.qx_half > QX_FULL_MAX)
        return bad("the full-range x quadrature needs qx_half <= 100 (order 2 qx_half <= 200)");
    if (!(p.kn > 0) || !std::isfinite(p.kn)) return bad("kn must be > 0");
    if (!(p.eta0 >= 0 && p.eta0 < 0.5)) return bad("eta0 must be in [0, 0.5)");
    if (!(p.T_left > 0) || !(p.T_right > 0)) return bad("wall temperatures must be > 0");
    if (!std::isfinite(p.U_left) || !std::isfinite(p.U_right) || !std::isfinite(p.accel_y)) return bad("non-finite wall speed or force");
    if (!(p.dt >= 0) || (p.dt == 0 && !(p.cfl > 0))) return bad("need dt > 0 or cfl > 0");
    if (!(p.T_init >= 0)) return bad("T_init must be >= 0");
    return FDLB_OK;
}

// Fischer-Methfessel averaging weights (Eq. chi_ret) as sparse rows: n-bar_i = sum_e w[e]
// n[col[e]].  The density is constant on each cell [x(s_j), x(s_{j+1})] and zero beyond the
// walls; w = 3/(4 sigma^3) times the exact integral of sigma^2 - t^2 over the cell's part of
// |t| < sigma around x_i, sigma = 6 sqrt(2) eta0 chi(eta0) Kn.
void fm_weights(const fdlb_params& p, std::vector<int>& ptr, std::vector<int>& col, std::vector<double>& w) {
    const int N = p.nx;
    const double ds = 2.0 / N;
    auto xmap = [&](double s) {
        return p.grid == FDLB_GRID_UNIFORM ? 0.5 * s : 0.5 * std::tanh(p.stretch * s) / std::tanh(p.stretch);
    };
    std::vector<double> faces(N + 1);
    for (int j = 0; j <= N; ++j) faces[j] = xmap(-1.0 + j * ds);
    const double eta = p.eta0, chi0 = (2.0 - eta) / (2.0 * (1.0 - eta) * (1.0 - eta) * (1.0 - eta));
    const double sg = 6.0 * std::sqrt(2.0) * eta * chi0 * p.kn;
    const double c = 3.0 / (4.0 * sg * sg * sg);
    auto K = [&](double t) { return sg * sg * t - t * t * t / 3.0; };
    ptr.assign(1, 0);
    col.clear();
    w.clear();
    for (int i = 0; i < N; ++i) {
        const double xi = xmap(-1.0 + (i + 0.5) * ds);
        for (int j = 0; j < N; ++j) {
            const double lo = std::min(std::max(faces[j] - xi, -sg), sg), hi = std::min(std::max(faces[j + 1] - xi, -sg), sg);
            if (hi > lo) {
                col.push_back(j);
                w.push_back(c * (K(hi) - K(lo)));
            }
        }
        ptr.push_back((int)col.size());
    }
}

// Byte layout of one instance inside the workspace.
struct Layout {
    size_t tables = 0, fbuf = 0, node = 0, tab = 0, tab32 = 0, misc = 0, msum = 0, mcnt = 0, total = 0;
    int ld = 0, K = 0, Tc = 0, form = 0, ntab = 0, trows = 0, My = 0, Mz = 0, groups = 1, ukc = 1;
    int fm_nnz = 0;            // entries of the Fischer-Methfessel weights (RET-FM only)
};

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

// FNV-1a over the fields of a parameter set (field by field, so that struct padding never
// enters).  fp32_alike: FDLB_FP32_STORAGE and FDLB_FP32_THEN_FP64 hash alike (the stochastic
// rounding seed, so that both round identically while both store FP32).
static uint64_t params_fnv(const fdlb_params& p, bool fp32_alike) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* v, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(v);
        for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    };
    int32_t prec = p.precision;
    if (fp32_alike && prec == FDLB_FP32_THEN_FP64) prec = FDLB_FP32_STORAGE;
    const int32_t iv[] = {p.flow, p.nx, p.grid, p.qx_half, p.qy, p.qz, prec, p.j1_shear, p.chi_model, p.x_quadrature};
    const double dv[] = {p.stretch, p.kn, p.eta0, p.T_left, p.T_right, p.U_left, p.U_right, p.accel_y, p.cfl, p.dt, p.T_init};
    mix(iv, sizeof(iv));
    mix(dv, sizeof(dv));
    return h;
}

namespace {

// Velocities per update block: small batches split a tile's velocities into chunks (16 for
// fewer than 38 tiles, a quarter of the SMs; 32 up to 1216 tiles) to occupy the GPU; large
// batches give a block the whole tile (the node table is loaded once), at most 256
// velocities (the block keeps its outputs in shared memory for the moments).
constexpr int UKC_MAX = 256;
constexpr size_t UPD_SMEM_LIMIT = 220 * 1024;   // dynamic shared memory of one update block, at most
int upd_chunk(const std::vector<fdlb_params>& ps) {
    long tiles = 0;
    for (auto& p : ps) tiles += (p.nx + TILE - 1) / TILE;
    return tiles >= 1216 ? UKC_MAX : (tiles < 38 ? 16 : 32);
}

Layout layout_of(const fdlb_params& p, int ukc) {
    Layout L;
    L.form = p.qz > 0 ? FORM_UNREDUCED : (p.qy > 0 ? FORM_REDUCED2D : FORM_REDUCED1D);
    L.Tc = L.form == FORM_UNREDUCED ? p.qy * p.qz : (L.form == FORM_REDUCED2D ? 2 * p.qy : 2);
    L.K = 2 * p.qx_half * L.Tc;
    L.ld = (p.nx + TILE - 1) / TILE * TILE;
    L.ntab = 8 * p.qx_half + 4 * L.Tc + 1;
    L.My = p.qy > 0 ? (p.qy + 5) / 2 : 0;     // 2 My - 1 >= qy + 2
    L.Mz = p.qz > 0 ? (p.qz + 5) / 2 : 0;
    const int Q = p.qx_half, Lx = p.x_quadrature == FDLB_XQ_FULL ? 2 * Q : Q;
    size_t nd = 0;
    // tables (doubles), each padded to 256 B
    auto add = [&](size_t n) { nd += al256(n * 8) / 8; };
    const int mxa = std::max(MX, p.x_quadrature == FDLB_XQ_FULL ? Q + 2 : aux_points_half(Lx));   // aux x rule
    add(2 * Q); add(mxa); add(mxa); add(MX8); add(MX8); add(Lx); add(Lx + 1); add(Lx + 1); add(Lx * Q);
    add(QYMAX); add(MYMAX); add(MYMAX); add(QYMAX * QYMAX);
    add(QZMAX); add(MYMAX); add(MYMAX); add(QZMAX * QZMAX);
    add(QYMAX * QYMAX);
    add(L.Tc); add(L.Tc); add(L.Tc);
    add(p.nx); add(p.nx); add(21);
    add(L.K); add(L.K);
    add(QYMAX + 2); add(QYMAX + 2);
    auto add32 = [&](size_t n) { nd += al256(n * 4) / 8; };
    add(6 * L.Tc); add32(6 * L.Tc); add32(6 * L.Tc);
    const bool f32 = p.precision != FDLB_FP64;             // FP32 tables (FP32 and two-phase)
    if (f32) {
        add32(2 * Q); add32(p.nx); add32(QYMAX * QYMAX); add32(L.K); add32(L.K);
        // float pairs: xq, xw, xq8, xw8, xa, xb, xib, xH, yq, yw, yH, zq, zw, zH, fsq, fisq
        add32(2 * mxa); add32(2 * mxa); add32(2 * MX8); add32(2 * MX8); add32(2 * Lx); add32(2 * (Lx + 1));
        add32(2 * (Lx + 1)); add32(2 * Lx * Q); add32(2 * MYMAX); add32(2 * MYMAX); add32(2 * QYMAX * QYMAX);
        add32(2 * MYMAX); add32(2 * MYMAX); add32(2 * QZMAX * QZMAX); add32(2 * (QYMAX + 2)); add32(2 * (QYMAX + 2));
        add32(2 * 2 * Q);   // px pairs
    }
    if (p.chi_model == FDLB_CHI_RET_FM) {
        std::vector<int> pt, cl;
        std::vector<double> ww;
        fm_weights(p, pt, cl, ww);
        L.fm_nnz = (int)cl.size();
        add32(p.nx + 1); add32(L.fm_nnz); add(L.fm_nnz);
    }
    L.tables = nd * 8;
    const size_t es = p.precision == FDLB_FP32_STORAGE ? 4 : 8;
    L.fbuf = al256((size_t)L.K * L.ld * es);
    L.node = al256((size_t)NROWS * L.ld * 8);
    L.tab = al256((size_t)L.ntab * L.ld * 8);
    L.misc = al256(8 * 8);
    L.tab32 = f32 ? al256((size_t)L.ntab * L.ld * 4) : 0;
    L.ukc = std::min(L.K, ukc);
    // the update block stages its chunk's rows and the table rows it uses in shared memory:
    // halve the chunk of the largest velocity sets until a block fits in the per-block limit
    // (with room for the static part)
    auto trows = [&](int kc) {
        const int nkx = std::min(2 * p.qx_half, (kc + L.Tc - 1) / L.Tc + 1);   // x-velocities a chunk spans
        return std::min(L.ntab, 4 * nkx + 4 * L.Tc + 1);
    };
    {
        const size_t s_max = p.precision == FDLB_FP32_STORAGE ? 4 : 8;
        while (L.ukc > 8 && update_smem_bytes(trows(L.ukc), L.ukc, s_max, s_max) > UPD_SMEM_LIMIT) L.ukc = (L.ukc + 1) / 2;
    }
    L.trows = trows(L.ukc);
    L.groups = (L.K + L.ukc - 1) / L.ukc;
    L.msum = L.groups > 1 ? al256((size_t)L.groups * MOM_SUMS * L.ld * 8) : 0;
    L.mcnt = al256((size_t)(L.ld / TILE) * 4);
    L.total = L.tables + 3 * L.fbuf + L.node + L.tab + L.tab32 + L.misc + L.msum + L.mcnt;
    return L;
}

size_t global_bytes(int count, int n_upd, int n_nod) {
    return al256(sizeof(Inst) * count) + al256(sizeof(Work) * n_upd) + al256(sizeof(Work) * n_nod) +
           al256(sizeof(int) * count) + al256(sizeof(long long) * count) + al256(sizeof(double) * count) +
           al256(sizeof(int) * count) + al256(sizeof(int) * count);
}

void count_work(const std::vector<fdlb_params>& p, int& n_upd, int& n_nod) {
    n_upd = n_nod = 0;
    const int ukc = upd_chunk(p);
    for (auto& q : p) {
        Layout L = layout_of(q, ukc);
        int tiles = (q.nx + TILE - 1) / TILE;
        n_upd += tiles * L.groups;
        n_nod += tiles * 3;
    }
}

}  // namespace

extern "C" int fdlb_quadrature(int32_t kind, int32_t q, double* nodes, double* weights) {
    if ((kind != 0 && kind != 1) || q < 1 || q > (kind == 0 ? QX_HALF_MAX : LXMAX) || !nodes || !weights)
        return fail(nullptr, FDLB_EINVAL, "fdlb_quadrature: bad arguments");
    Rule r = make_rule(kind, q);
    for (int k = 0; k < q; ++k) { nodes[k] = r.x[k]; weights[k] = r.w[k]; }
    return FDLB_OK;
}

extern "C" size_t fdlb_workspace_bytes(const fdlb_params* params, int32_t count) {
    if (!params || count < 1) { g_err = "fdlb_workspace_bytes: need params and count >= 1"; return 0; }
    std::vector<fdlb_params> p(params, params + count);
    for (int i = 0; i < count; ++i) {
        std::string why;
        if (validate(p[i], why) != FDLB_OK) { g_err = "instance " + std::to_string(i) + ": " + why; return 0; }
    }
    int n_upd, n_nod;
    count_work(p, n_upd, n_nod);
    size_t tot = global_bytes(count, n_upd, n_nod);
    const int ukc = upd_chunk(p);
    for (auto& q : p) tot += layout_of(q, ukc).total;
    return tot;
}

extern "C" int fdlb_create(fdlb_ctx** out, const fdlb_params* params, int32_t count, void* dev_workspace,
                           size_t ws_bytes, void* stream) {
    if (!out || !params || count < 1) return fail(nullptr, FDLB_EINVAL, "fdlb_create: bad arguments");
    *out = nullptr;
    size_t need = fdlb_workspace_bytes(params, count);
    if (need == 0) return fail(nullptr, FDLB_EINVAL, g_err);
    if (!dev_workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(dev_workspace) & 255))
        return fail(nullptr, FDLB_ENOMEM, "fdlb_create: workspace missing, smaller than fdlb_workspace_bytes, or not 256-byte aligned");
    fdlb_ctx* c = new fdlb_ctx();
    c->count = count;
    c->prm.assign(params, params + count);
    c->stream = reinterpret_cast<cudaStream_t>(stream);

    int n_upd, n_nod;
    count_work(c->prm, n_upd, n_nod);
    c->n_upd = n_upd;
    c->n_nod = n_nod;
    char* base = reinterpret_cast<char*>(dev_workspace);
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base + off; off += al256(bytes); return p; };
    c->d_inst = reinterpret_cast<Inst*>(take(sizeof(Inst) * count));
    c->d_upd = reinterpret_cast<Work*>(take(sizeof(Work) * n_upd));
    c->d_nod = reinterpret_cast<Work*>(take(sizeof(Work) * n_nod));
    c->d_status_all = reinterpret_cast<int*>(take(sizeof(int) * count));
    c->d_steps_all = reinterpret_cast<long long*>(take(sizeof(long long) * count));
    c->d_resid_all = reinterpret_cast<double*>(take(sizeof(double) * count));
    c->d_list = reinterpret_cast<int*>(take(sizeof(int) * count));
    c->d_smem_list = reinterpret_cast<int*>(take(sizeof(int) * count));

    std::vector<Work> wu, wn;
    std::vector<std::pair<int*, size_t>> counters;
    std::vector<char> staging;        // host image of all table regions
    std::vector<std::pair<size_t, size_t>> regions;   // (offset, size) of table regions
    size_t max_smem64 = 0, max_smem32 = 0;

    const int ukc = upd_chunk(c->prm);
    for (int ii = 0; ii < count; ++ii) {
        const fdlb_params& p = c->prm[ii];
        Layout L = layout_of(p, ukc);
        const int Q = p.qx_half, N = p.nx;
        Inst I;
        std::memset(&I, 0, sizeof(I));
        I.N = N; I.ld = L.ld; I.Q = Q; I.Qy = p.qy; I.Qz = p.qz; I.form = L.form; I.Tc = L.Tc; I.K = L.K;
        I.Mx = aux_points_half(p.x_quadrature == FDLB_XQ_FULL ? 2 * p.qx_half : p.qx_half); I.My = L.My; I.Mz = L.Mz;
        I.precision = p.precision == FDLB_FP64 ? FDLB_FP64 : FDLB_FP32_STORAGE;
        I.two_phase = p.precision == FDLB_FP32_THEN_FP64;
        I.j1_shear = p.j1_shear;
        I.chi_model = p.chi_model; I.ntab = L.ntab; I.trows = L.trows; I.mgroups = L.groups; I.ukc = L.ukc;
        {
            const uint64_t h = params_fnv(p, true);
            I.sr_key = (uint32_t)(h ^ (h >> 32));
        }
        const bool xfull = p.x_quadrature == FDLB_XQ_FULL;
        const int Lx = xfull ? 2 * Q : Q;
        I.xfull = xfull; I.Lx = Lx;
        // full range: (p - u)^a h_l(p) g is a polynomial of degree <= Lx + 2 in the Gaussian
        // variable, integrated exactly by the Gauss-Hermite rule of Q + 2 points
        if (xfull) I.Mx = Q + 2;
        I.kn = p.kn; I.eta0 = p.eta0; I.chi0 = chi_cs(p.eta0);
        I.mu0c = (5.0 / 16.0) * std::sqrt(2.0 * M_PI) * I.chi0 * p.kn;
        I.accel_y = p.accel_y;
        I.T_L = p.T_left; I.T_R = p.T_right; I.U_L = p.U_left; I.U_R = p.U_right;
        I.T_init = p.T_init > 0 ? p.T_init : 0.5 * (p.T_left + p.T_right);
        I.ds = 2.0 / N;

        // ---- host tables
        size_t tab_off = off;
        std::vector<double> img(L.tables / 8, 0.0);
        size_t pos = 0;
        auto put = [&](const double** dst, size_t n) -> double* {
            double* h = img.data() + pos;
            *dst = reinterpret_cast<const double*>(base + tab_off + pos * 8);
            pos += al256(n * 8) / 8;
            return h;
        };
        auto put32 = [&](const float** dst, size_t n) -> float* {
            float* h = reinterpret_cast<float*>(img.data() + pos);
            *dst = reinterpret_cast<const float*>(base + tab_off + pos * 8);
            pos += al256(n * 4) / 8;
            return h;
        };
        auto putw = [&](double** dst, size_t n) -> double* {
            double* h = img.data() + pos;
            *dst = reinterpret_cast<double*>(base + tab_off + pos * 8);
            pos += al256(n * 8) / 8;
            return h;
        };
        // x axis: the half-range rule of order Q, or the full-range rule of order 2Q whose
        // positive nodes (the upper half of its ascending list) play the same part
        Rule xr = xfull ? make_rule(1, Lx) : make_rule(0, Q);
        const int kpos = xfull ? Q : 0;            // index of +p_1 in xr.x
        Rule xa = make_rule(xfull ? 1 : 0, I.Mx);
        const int mxa = std::max(MX, I.Mx);
        {
            double* h = put(&I.px, 2 * Q);
            for (int k = 0; k < Q; ++k) { h[k] = xr.x[kpos + k]; h[Q + k] = -xr.x[kpos + k]; }
            h = put(&I.xq, mxa); for (int m = 0; m < I.Mx; ++m) h[m] = xa.x[m];
            h = put(&I.xw, mxa); for (int m = 0; m < I.Mx; ++m) h[m] = xa.w[m];
            Rule xa8 = make_rule(0, MX8);
            h = put(&I.xq8, MX8); for (int m = 0; m < MX8; ++m) h[m] = xa8.x[m];
            h = put(&I.xw8, MX8); for (int m = 0; m < MX8; ++m) h[m] = xa8.w[m];
            h = put(&I.xa, Lx); for (int l = 0; l < Lx; ++l) h[l] = xr.alpha[l];
            double* hb = put(&I.xb, Lx + 1);
            double* hib = put(&I.xib, Lx + 1);
            for (int l = 0; l <= Lx; ++l) {
                hb[l] = l ? std::sqrt(xr.beta[l]) : 0.0;
                hib[l] = l ? 1.0 / std::sqrt(xr.beta[l]) : 0.0;
            }
            I.x_h0 = 1.0 / std::sqrt(xr.beta[0]);
            h = put(&I.xH, Lx * Q);
            std::vector<double> hv;
            for (int k = 0; k < Q; ++k) {
                ortho_values(Lx, xr.alpha, xr.beta, xr.x[kpos + k], hv);
                for (int l = 0; l < Lx; ++l) h[l * Q + k] = (double)(xr.w[kpos + k] * hv[l]);
            }
        }
        auto full_tables = [&](int Qn, int M, const double** nn, const double** aq, const double** aw, const double** H) {
            double* hn = put(nn, QYMAX);
            double* hq = put(aq, MYMAX);
            double* hw = put(aw, MYMAX);
            double* hH = put(H, QYMAX * QYMAX);
            if (Qn == 0) return;
            Rule r = make_rule(1, Qn), a = make_rule(1, M);
            for (int k = 0; k < Qn; ++k) hn[k] = r.x[k];
            for (int m = 0; m < M; ++m) { hq[m] = a.x[m]; hw[m] = a.w[m]; }
            std::vector<double> hv;
            for (int k = 0; k < Qn; ++k) {
                ortho_values(Qn, r.alpha, r.beta, r.x[k], hv);
                for (int l = 0; l < Qn; ++l) hH[l * Qn + k] = (double)(r.w[k] * hv[l]);
            }
        };
        full_tables(p.qy, L.My, &I.yn, &I.yq, &I.yw, &I.yH);
        full_tables(p.qz, L.Mz, &I.zn, &I.zq, &I.zw, &I.zH);
        {
            // momentum-derivative kernel on y (App. A, Eq. kernel_H):
            // K[k][k'] = -w_k sum_{l=0}^{Q-2} He_{l+1}(p_k) He_l(p_k')/l!
            double* h = put(&I.Ky, QYMAX * QYMAX);
            if (p.qy > 0) {
                Rule r = make_rule(1, p.qy);
                const int Qy = p.qy;
                std::vector<std::vector<double>> He(Qy + 1, std::vector<double>(Qy));
                for (int k = 0; k < Qy; ++k) {
                    He[0][k] = 1;
                    He[1][k] = r.x[k];
                    for (int l = 1; l < Qy; ++l) He[l + 1][k] = r.x[k] * He[l][k] - l * He[l - 1][k];
                }
                for (int k = 0; k < Qy; ++k)
                    for (int kp = 0; kp < Qy; ++kp) {
                        double s = 0, fact = 1;
                        for (int l = 0; l <= Qy - 2; ++l) {
                            if (l > 0) fact *= l;
                            s += He[l + 1][k] * He[l][kp] / fact;
                        }
                        h[k * Qy + kp] = (double)(-r.w[k] * s);
                    }
            }
        }
        {
            double* hm = put(&I.tmt, L.Tc);
            double* hy = put(&I.tpy, L.Tc);
            double* he = put(&I.tet, L.Tc);
            if (L.form == FORM_UNREDUCED) {
                Rule ry = make_rule(1, p.qy), rz = make_rule(1, p.qz);
                for (int ky = 0; ky < p.qy; ++ky)
                    for (int kz = 0; kz < p.qz; ++kz) {
                        int t = ky * p.qz + kz;
                        hm[t] = 1.0; hy[t] = ry.x[ky]; he[t] = 0.5 * rz.x[kz] * rz.x[kz];
                    }
            } else if (L.form == FORM_REDUCED2D) {
                Rule ry = make_rule(1, p.qy);
                for (int ky = 0; ky < p.qy; ++ky) {
                    hm[2 * ky] = 1.0; hy[2 * ky] = ry.x[ky]; he[2 * ky] = 0.0;
                    hm[2 * ky + 1] = 0.0; hy[2 * ky + 1] = ry.x[ky]; he[2 * ky + 1] = 0.5;
                }
            } else {
                hm[0] = 1.0; hy[0] = 0.0; he[0] = 0.0;
                hm[1] = 0.0; hy[1] = 0.0; he[1] = 0.5;
            }
        }
        {
            double* hxi = put(&I.xpinv, N);
            double* hdx = put(&I.dxw, N);
            double xpmin = 1e300;
            for (int i = 0; i < N; ++i) {
                double s = -1.0 + (i + 0.5) * I.ds, xp;
                if (p.grid == FDLB_GRID_UNIFORM) xp = 0.5;
                else { double ch = std::cosh(p.stretch * s); xp = 0.5 * p.stretch / (ch * ch * std::tanh(p.stretch)); }
                hxi[i] = 1.0 / (xp * I.ds);
                hdx[i] = xp * I.ds;
                xpmin = std::min(xpmin, xp);
            }
            I.dt = p.dt > 0 ? p.dt : p.cfl * xpmin * I.ds / xr.x[kpos + Q - 1];
            double* hg = put(&I.gst, 21);
            for (int r = 0; r < 3; ++r) stencil7(r, hg + 7 * r);
        }
        putw(&I.gL, L.K);
        putw(&I.gR, L.K);
        {
            // sqrt(l) and 1/sqrt(l): recurrence of the orthonormal He_l/sqrt(l!)
            double* hb = put(&I.fsq, QYMAX + 2);
            double* hib = put(&I.fisq, QYMAX + 2);
            for (int l = 0; l < QYMAX + 2; ++l) { hb[l] = std::sqrt((double)l); hib[l] = l ? 1.0 / std::sqrt((double)l) : 0.0; }
        }
        {
            // transverse weights of the factorised moment sums, and their float head/tail split
            const double* hm = reinterpret_cast<const double*>(img.data()) + ((const char*)I.tmt - (base + tab_off)) / 8;
            const double* hy = reinterpret_cast<const double*>(img.data()) + ((const char*)I.tpy - (base + tab_off)) / 8;
            const double* he = reinterpret_cast<const double*>(img.data()) + ((const char*)I.tet - (base + tab_off)) / 8;
            double* tw = put(&I.tw, 6 * L.Tc);
            float* twh = put32(&I.twh, 6 * L.Tc);
            float* twl = put32(&I.twl, 6 * L.Tc);
            for (int t = 0; t < L.Tc; ++t) {
                const double w6[6] = {hm[t], hm[t] * hy[t], hm[t] * hy[t] * hy[t], hm[t] * hy[t] * hy[t] * hy[t], he[t], he[t] * hy[t]};
                for (int j = 0; j < 6; ++j) {
                    tw[j * L.Tc + t] = w6[j];
                    twh[j * L.Tc + t] = (float)w6[j];
                    twl[j * L.Tc + t] = (float)(w6[j] - (double)(float)w6[j]);
                }
            }
        }
        if (p.precision != FDLB_FP64) {
            const double* img0 = reinterpret_cast<const double*>(img.data());
            auto host_of = [&](const double* dev) { return img0 + ((const char*)dev - (base + tab_off)) / 8; };
            float* h = put32(&I.px32, 2 * Q);
            for (int k = 0; k < 2 * Q; ++k) h[k] = (float)host_of(I.px)[k];
            h = put32(&I.xpinv32, N);
            for (int i = 0; i < N; ++i) h[i] = (float)host_of(I.xpinv)[i];
            h = put32(&I.Ky32, QYMAX * QYMAX);
            for (int k = 0; k < QYMAX * QYMAX; ++k) h[k] = (float)host_of(I.Ky)[k];
            const float* g32;
            put32(&g32, L.K);
            I.gL32 = const_cast<float*>(g32);
            put32(&g32, L.K);
            I.gR32 = const_cast<float*>(g32);
            // float-pair copies: hi = nearest float, lo = the float nearest to the remainder
            auto pairs = [&](const float2** dst, const double* dev, size_t n) {
                const float** d = reinterpret_cast<const float**>(dst);
                float* h2 = put32(d, 2 * n);
                const double* src = host_of(dev);
                for (size_t k = 0; k < n; ++k) {
                    const float hi = (float)src[k];
                    h2[2 * k] = hi;
                    h2[2 * k + 1] = (float)(src[k] - (double)hi);
                }
            };
            pairs(&I.xq2, I.xq, std::max(MX, I.Mx));
            pairs(&I.xw2, I.xw, std::max(MX, I.Mx));
            pairs(&I.xq82, I.xq8, MX8);
            pairs(&I.xw82, I.xw8, MX8);
            pairs(&I.xa2, I.xa, Lx);
            pairs(&I.xb2, I.xb, Lx + 1);
            pairs(&I.xib2, I.xib, Lx + 1);
            pairs(&I.xH2, I.xH, (size_t)Lx * Q);
            pairs(&I.yq2, I.yq, MYMAX);
            pairs(&I.yw2, I.yw, MYMAX);
            pairs(&I.yH2, I.yH, QYMAX * QYMAX);
            pairs(&I.zq2, I.zq, MYMAX);
            pairs(&I.zw2, I.zw, MYMAX);
            pairs(&I.zH2, I.zH, QZMAX * QZMAX);
            pairs(&I.fsq2, I.fsq, QYMAX + 2);
            pairs(&I.fisq2, I.fisq, QYMAX + 2);
            pairs(&I.px2, I.px, 2 * Q);
            const float h0 = (float)I.x_h0;
            I.x_h02 = make_float2(h0, (float)(I.x_h0 - (double)h0));
        }
        if (p.chi_model == FDLB_CHI_RET_FM) {
            std::vector<int> pt, cl;
            std::vector<double> ww;
            fm_weights(p, pt, cl, ww);
            float* hp = put32(reinterpret_cast<const float**>(&I.fm_ptr), pt.size());
            std::memcpy(hp, pt.data(), sizeof(int) * pt.size());
            float* hc = put32(reinterpret_cast<const float**>(&I.fm_col), cl.size());
            std::memcpy(hc, cl.data(), sizeof(int) * cl.size());
            double* hw = put(&I.fm_w, ww.size());
            std::memcpy(hw, ww.data(), sizeof(double) * ww.size());
        }
        if (pos * 8 != L.tables) { delete c; return fail(nullptr, FDLB_EINVAL, "internal: table layout mismatch"); }
        regions.push_back({tab_off, L.tables});
        {
            size_t o = staging.size();
            staging.resize(o + L.tables);
            std::memcpy(staging.data() + o, img.data(), L.tables);
        }
        off += L.tables;
        // state
        for (int b = 0; b < 3; ++b) I.f[b] = take(L.fbuf);
        I.node = reinterpret_cast<double*>(take(L.node));
        I.tab = reinterpret_cast<double*>(take(L.tab));
        I.tab32 = L.tab32 ? reinterpret_cast<float*>(take(L.tab32)) : nullptr;
        I.misc = reinterpret_cast<double*>(take(L.misc));
        I.msum = L.msum ? reinterpret_cast<double*>(take(L.msum)) : nullptr;
        I.mcnt = reinterpret_cast<int*>(take(L.mcnt));
        counters.push_back({I.mcnt, L.mcnt});
        I.status = c->d_status_all + ii;
        I.steps = c->d_steps_all + ii;
        c->inst.push_back(I);

        int tiles = (N + TILE - 1) / TILE;
        const size_t nu0 = wu.size();
        for (int t = 0; t < tiles; ++t) {
            for (int k0 = 0; k0 < L.K; k0 += L.ukc) wu.push_back({ii, t * TILE, k0, std::min(L.K, k0 + L.ukc)});
            for (int role = 0; role < 3; ++role) wn.push_back({ii, t * TILE, role, 0});
        }
        c->upd_blocks.push_back((int)(wu.size() - nu0));
        c->qmax = std::max(c->qmax, Lx);      // register and shared arrays hold Lx polynomials
        c->ukc_max = std::max(c->ukc_max, L.ukc);
        if (p.precision != FDLB_FP32_STORAGE) max_smem64 = std::max(max_smem64, update_smem_bytes(L.trows, L.ukc, 8, 8)), c->any_fp64 = true;
        if (p.precision != FDLB_FP64) max_smem32 = std::max(max_smem32, update_smem_bytes(L.trows, L.ukc, 4, 4)), c->any_fp32 = true;
    }
    if (off > need) { delete c; return fail(nullptr, FDLB_EINVAL, "internal: workspace layout overflow"); }
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            c->n_sms = 0;             // unknown: 8-warp update blocks throughout
        }
        choose_update_width(c, nullptr);
        c->upd_wide_all = c->upd_wide;
    }
    c->smem_upd_f64 = max_smem64;
    c->smem_upd_f32 = max_smem32;

    // ---- upload
    cudaStream_t s = c->stream;
    int rc;
    size_t so = 0;
    for (auto& r : regions) {
        rc = cuda_check(c, cudaMemcpyAsync(base + r.first, staging.data() + so, r.second, cudaMemcpyHostToDevice, s), "upload tables");
        if (rc) { int e = rc; g_err = c->err; delete c; return e; }
        so += r.second;
    }
    // resident clusters take the largest instances (nodes x velocities) first
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long)c->inst[a].N * c->inst[a].K > (long)c->inst[b].N * c->inst[b].K;
    });
    rc = cuda_check(c, cudaMemcpyAsync(c->d_list, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s), "upload list");
    if (!rc) {
        choose_smem_resident(c);
        if (c->n_smem > 0)
            rc = cuda_check(c, cudaMemcpyAsync(c->d_smem_list, c->smem_idx.data(), sizeof(int) * c->n_smem, cudaMemcpyHostToDevice, s),
                            "upload list");
    }
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(s), "upload list");
    if (rc) { int e = rc; g_err = c->err; delete c; return e; }
    rc = cuda_check(c, cudaMemcpyAsync(c->d_inst, c->inst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, s), "upload descriptors");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(c->d_upd, wu.data(), sizeof(Work) * n_upd, cudaMemcpyHostToDevice, s), "upload work");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(c->d_nod, wn.data(), sizeof(Work) * n_nod, cudaMemcpyHostToDevice, s), "upload work");
    for (auto& cn : counters)
        if (!rc) rc = cuda_check(c, cudaMemsetAsync(cn.first, 0, cn.second, s), "clear counters");
    if (!rc) rc = cuda_check(c, prepare_kernels(c->smem_upd_f64, c->smem_upd_f32, c->qmax), "kernel attributes");
    if (!rc) choose_cluster(c);
    if (!rc) rc = cuda_check(c, launch_setup(c->d_inst, count, s), "setup kernel");
    if (!rc) rc = cuda_check(c, launch_moments(c->d_inst, c->d_upd, n_upd, 0, c->ukc_max, c->any_fp64, c->any_fp32, s), "moments kernel");
    if (!rc) rc = cuda_check(c, launch_resid(c->d_inst, count, -1, 0.0, c->d_resid_all, s), "residual kernel");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(s), "fdlb_create synchronize");
    if (rc) { int e = rc; g_err = c->err; delete c; return e; }
    *out = c;
    return FDLB_OK;
}

extern "C" void fdlb_destroy(fdlb_ctx* ctx) { delete ctx; }

extern "C" int fdlb_info(const fdlb_ctx* ctx, int32_t inst, int32_t* nx, int32_t* nvel, double* dt) {
    if (!ctx) return fail(nullptr, FDLB_EINVAL, "fdlb_info: null context");
    if (inst < 0 || inst >= ctx->count) return fail(const_cast<fdlb_ctx*>(ctx), FDLB_EINVAL, "fdlb_info: instance out of range");
    if (nx) *nx = ctx->inst[inst].N;
    if (nvel) *nvel = ctx->inst[inst].K;
    if (dt) *dt = ctx->inst[inst].dt;
    return FDLB_OK;
}

extern "C" int fdlb_layout(const fdlb_ctx* ctx, int32_t inst, int32_t* chunk, int32_t* chunks_per_tile, int32_t* tiles) {
    if (!ctx) return fail(nullptr, FDLB_EINVAL, "fdlb_layout: null context");
    if (inst < 0 || inst >= ctx->count) return fail(const_cast<fdlb_ctx*>(ctx), FDLB_EINVAL, "fdlb_layout: instance out of range");
    const Inst& I = ctx->inst[inst];
    if (chunk) *chunk = I.ukc;
    if (chunks_per_tile) *chunks_per_tile = I.mgroups;
    if (tiles) *tiles = (I.N + TILE - 1) / TILE;
    return FDLB_OK;
}

static const int GRAPH_STEPS = 16;
static const int RESIDENT_CHUNK = 256;     // steps per resident launch

// Cluster size of the resident schedule: the largest candidate (at most the largest
// instance's 3 x tiles nodal items) whose clusters for the whole batch fit on the GPU at once;
// failing that, the candidate with the most CTAs resident at once.  cs = 0: unavailable.
static void choose_cluster(fdlb_ctx* c) {
    int items = 1;
    for (auto& I : c->inst) items = std::max(items, 3 * ((I.N + TILE - 1) / TILE));
    int best = 0, best_ctas = 0;
    size_t best_smem = 0;
    for (int cs : {16, 8, 4, 2, 1}) {
        if (cs > items && cs > 1) continue;
        size_t smem = 0;
        int n = 0;
        if (prepare_resident(c->qmax, std::max(c->smem_upd_f64, c->smem_upd_f32), cs, &smem) != cudaSuccess ||
            resident_max_clusters(c->qmax, smem, cs, &n) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (n < 1) continue;
        if (n >= c->count) {
            best = cs;
            best_smem = smem;
            break;
        }
        if (n * cs > best_ctas) {
            best = cs;
            best_ctas = n * cs;
            best_smem = smem;
        }
    }
    c->cs = best;
    c->res_smem = best_smem;
    // the kernel attribute must match the size used at launch
    if (best) {
        size_t smem;
        if (prepare_resident(c->qmax, std::max(c->smem_upd_f64, c->smem_upd_f32), best, &smem) != cudaSuccess) {
            cudaGetLastError();
            c->cs = 0;
        }
    }
}

// Instances for the shared-memory-resident kernel: not two-phase, and the item scratch plus the
// three RK buffers fit in one block's dynamic shared memory.  The kernel is launched with one
// size for all of them (the largest scratch and buffers of the set), so the instances with the
// largest need leave the set until that size fits.  Largest first in the launch order.
static void choose_smem_resident(fdlb_ctx* c) {
    c->n_smem = 0;
    c->smem_idx.clear();
    struct Cand { int idx, Lx; size_t upd, fb, need; };
    std::vector<Cand> cand;
    size_t limit = 0;
    int qall = 1;
    for (auto& I : c->inst) qall = std::max(qall, I.Lx);
    if (smemres_dynamic_limit(qall, &limit) != cudaSuccess) { cudaGetLastError(); return; }
    for (int i = 0; i < c->count; ++i) {
        const Inst& I = c->inst[i];
        if (I.two_phase) continue;
        const size_t sz = I.precision == FDLB_FP32_STORAGE ? 4 : 8;
        const size_t upd = update_smem_bytes(I.trows, I.ukc, sz, sz);
        const size_t fb = smemres_buffer_bytes(I.K, I.ld, sz);
        const size_t need = smemres_scratch_bytes(I.Lx, upd) + 3 * fb;
        if (need <= limit) cand.push_back({i, I.Lx, upd, fb, need});
    }
    std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.need > b.need; });
    size_t first = 0;
    int qm = 1;
    size_t scratch = 0, dyn = 0;
    cudaError_t attr = cudaSuccess;
    while (first < cand.size()) {
        size_t um = 0, fm = 0;
        qm = 1;
        for (size_t j = first; j < cand.size(); ++j) { qm = std::max(qm, cand[j].Lx); um = std::max(um, cand[j].upd); fm = std::max(fm, cand[j].fb); }
        scratch = smemres_scratch_bytes(qm, um);
        dyn = scratch + 3 * fm;
        if (dyn <= limit) {
            attr = prepare_smemres(qm, dyn);
            if (attr == cudaSuccess) break;
            cudaGetLastError();
        }
        ++first;
    }
    size_t least = 0;
    for (auto& cd : cand) least = least ? std::min(least, cd.need) : cd.need;
    c->smem_note = "dynamic shared memory per block " + std::to_string(limit) + " B; " + std::to_string(cand.size()) +
                   " candidates" + (cand.empty() ? "" : ", smallest need " + std::to_string(least) + " B") +
                   (attr != cudaSuccess ? std::string(", attribute: ") + cudaGetErrorString(attr) : std::string());
    if (first >= cand.size()) return;
    for (size_t j = first; j < cand.size(); ++j) c->smem_idx.push_back(cand[j].idx);
    c->n_smem = (int)c->smem_idx.size();
    c->smem_qmax = qm;
    c->smem_scratch = scratch;
    c->smem_dyn = dyn;
}

// smem_res of the listed instances on the device (the tiled kernels skip flagged instances).
static int set_smem_flags(fdlb_ctx* c, bool on) {
    if (c->smem_flags == on || c->n_smem == 0) return FDLB_OK;
    int rc = cuda_check(c, launch_set_smem_flags(c->d_inst, c->d_smem_list, c->n_smem, on ? 1 : 0, c->stream), "schedule flags");
    if (!rc) c->smem_flags = on;
    return rc;
}

// Capture GRAPH_STEPS steps into an executable graph (kernels only; no host synchronisation
// inside).  The legacy default stream cannot be captured: then steps are launched directly.
static bool ensure_graph(fdlb_ctx* c, double tol) {
    if (c->graph && c->graph_tol == tol && c->graph_wide == c->upd_wide) return true;
    if (c->graph_failed || c->stream == nullptr) return false;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        c->graph_failed = true;
        cudaGetLastError();
        return false;
    }
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < GRAPH_STEPS && e == cudaSuccess; ++s) e = step_once(c, tol);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        c->graph_failed = true;
        cudaGetLastError();
        return false;
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        c->graph_failed = true;
        cudaGetLastError();
        return false;
    }
    c->graph_tol = tol;
    c->graph_wide = c->upd_wide;
    return true;
}

// Update width from the instances still active (st: statuses, null = all active).
static void choose_update_width(fdlb_ctx* c, const int* st) {
    long blocks = 0;
    for (int i = 0; i < c->count; ++i)
        if (!st || st[i] == FDLB_ACTIVE) blocks += c->upd_blocks[i];
    c->upd_wide = c->n_sms > 0 && blocks <= c->n_sms;
}

static int step_tiled(fdlb_ctx* c, int64_t nsteps, double freeze_tol) {
    if (!c->prof && nsteps >= GRAPH_STEPS && ensure_graph(c, freeze_tol)) {
        while (nsteps >= GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
            if (e != cudaSuccess) return cuda_check(c, e, "fdlb_step graph launch");
            nsteps -= GRAPH_STEPS;
        }
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaError_t e = step_once(c, freeze_tol);
        if (e != cudaSuccess) return cuda_check(c, e, "fdlb_step launch");
    }
    return FDLB_OK;
}

static int step_resident(fdlb_ctx* c, int64_t nsteps, double freeze_tol) {
    while (nsteps > 0) {
        const int n = (int)std::min<int64_t>(nsteps, RESIDENT_CHUNK);
        cudaError_t e = launch_resident(c->d_inst, c->d_list, c->count, c->cs, c->qmax, c->res_smem, n, freeze_tol,
                                        c->d_resid_all, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "fdlb_step resident launch");
        nsteps -= n;
    }
    return FDLB_OK;
}

// Mixed schedule: the shared-memory-resident instances advance in one k_smemres launch on the
// second stream while the others take the tiled steps on the context's stream; the call's work
// is joined back into the context's stream.
static int step_mixed(fdlb_ctx* c, int64_t nsteps, double freeze_tol) {
    int rc = FDLB_OK;
    if (!c->stream2) {
        rc = cuda_check(c, cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking), "second stream");
        if (!rc) rc = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "stream events");
        if (!rc) rc = cuda_check(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "stream events");
        if (rc) return rc;
    }
    rc = set_smem_flags(c, true);
    if (!rc) rc = cuda_check(c, cudaEventRecord(c->ev_fork, c->stream), "fork");
    if (!rc) rc = cuda_check(c, cudaStreamWaitEvent(c->stream2, c->ev_fork, 0), "fork");
    int64_t left = nsteps;
    while (!rc && left > 0) {
        const int n = (int)std::min<int64_t>(left, 1 << 20);
        rc = cuda_check(c, launch_smemres(c->d_inst, c->d_smem_list, c->n_smem, c->smem_qmax, c->smem_scratch, c->smem_dyn, n,
                                          freeze_tol, c->d_resid_all, c->stream2), "shared-memory-resident launch");
        left -= n;
    }
    if (!rc && c->n_smem < c->count) rc = step_tiled(c, nsteps, freeze_tol);
    if (!rc) rc = cuda_check(c, cudaEventRecord(c->ev_join, c->stream2), "join");
    if (!rc) rc = cuda_check(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join");
    return rc;
}

static int step_schedule(fdlb_ctx* c, int sched, int64_t nsteps, double freeze_tol) {
    if (sched == FDLB_SCHED_MIXED) return step_mixed(c, nsteps, freeze_tol);
    int rc = set_smem_flags(c, false);
    if (rc) return rc;
    return sched == FDLB_SCHED_RESIDENT ? step_resident(c, nsteps, freeze_tol) : step_tiled(c, nsteps, freeze_tol);
}

// Times TUNE steps of each available schedule (after WARM warm-up steps of each) and keeps the
// fastest: tiled, cluster-resident, and mixed (shared-memory-resident for the instances that fit).
static int autotune(fdlb_ctx* c, double freeze_tol) {
    std::vector<int> cands = {FDLB_SCHED_TILED};
    if (c->cs > 0) cands.push_back(FDLB_SCHED_RESIDENT);
    if (c->n_smem > 0) cands.push_back(FDLB_SCHED_MIXED);
    const int WARM = 16, TUNE = (FDLB_AUTOTUNE_STEPS - (int)cands.size() * WARM) / (int)cands.size();
    std::vector<cudaEvent_t> ev(2 * cands.size(), nullptr);
    int rc = FDLB_OK;
    for (auto& e : ev)
        if (!rc) rc = cuda_check(c, cudaEventCreate(&e), "autotune events");
    for (size_t j = 0; j < cands.size() && !rc; ++j) {
        rc = step_schedule(c, cands[j], WARM, freeze_tol);
        if (!rc) rc = cuda_check(c, cudaEventRecord(ev[2 * j], c->stream), "autotune events");
        if (!rc) rc = step_schedule(c, cands[j], TUNE, freeze_tol);
        if (!rc) rc = cuda_check(c, cudaEventRecord(ev[2 * j + 1], c->stream), "autotune events");
    }
    if (!rc) rc = cuda_check(c, cudaEventSynchronize(ev.back()), "autotune synchronize");
    float best = 0.0f;
    int pick = FDLB_SCHED_TILED;
    for (size_t j = 0; j < cands.size() && !rc; ++j) {
        float t = 0.0f;
        rc = cuda_check(c, cudaEventElapsedTime(&t, ev[2 * j], ev[2 * j + 1]), "autotune timing");
        if (!rc && (j == 0 || t < best)) { best = t; pick = cands[j]; }
    }
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    if (!rc) c->sched = pick;
    return rc;
}

extern "C" int fdlb_step(fdlb_ctx* c, int64_t nsteps, double freeze_tol) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_step: null context");
    if (nsteps < 0 || !(freeze_tol >= 0)) return fail(c, FDLB_EINVAL, "fdlb_step: nsteps >= 0 and freeze_tol >= 0 required");
    if (c->prof) return step_schedule(c, FDLB_SCHED_TILED, nsteps, freeze_tol);
    if (c->sched == 0) {
        if (c->sched_req != FDLB_SCHED_AUTO) {
            c->sched = c->sched_req;
        } else if (c->cs == 0 && c->n_smem == 0) {
            c->sched = FDLB_SCHED_TILED;
        } else if (nsteps >= FDLB_AUTOTUNE_STEPS) {
            int rc = autotune(c, freeze_tol);
            if (rc) return rc;
            nsteps -= FDLB_AUTOTUNE_STEPS;
        }
    }
    return step_schedule(c, c->sched == 0 ? FDLB_SCHED_TILED : c->sched, nsteps, freeze_tol);
}

extern "C" int fdlb_set_schedule(fdlb_ctx* c, int32_t schedule) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_set_schedule: null context");
    if (schedule != FDLB_SCHED_AUTO && schedule != FDLB_SCHED_TILED && schedule != FDLB_SCHED_RESIDENT &&
        schedule != FDLB_SCHED_MIXED)
        return fail(c, FDLB_EINVAL, "fdlb_set_schedule: unknown schedule");
    if (schedule == FDLB_SCHED_RESIDENT && c->cs == 0)
        return fail(c, FDLB_EINVAL, "fdlb_set_schedule: the resident cluster kernel cannot be launched for this batch");
    if (schedule == FDLB_SCHED_MIXED && c->n_smem == 0)
        return fail(c, FDLB_EINVAL, "fdlb_set_schedule: no instance of this batch fits in one block's shared memory (" +
                                        c->smem_note + ")");
    c->sched_req = schedule;
    c->sched = schedule == FDLB_SCHED_AUTO ? 0 : schedule;
    return FDLB_OK;
}

extern "C" int fdlb_get_schedule(const fdlb_ctx* c, int32_t* schedule, int32_t* cluster_ctas) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_get_schedule: null context");
    if (schedule) *schedule = c->sched;
    if (cluster_ctas) *cluster_ctas = c->cs;
    return FDLB_OK;
}

extern "C" int fdlb_get_schedule_mix(const fdlb_ctx* c, int32_t* smem_resident, int32_t* n) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_get_schedule_mix: null context");
    if (n) *n = c->n_smem;
    if (smem_resident) {
        for (int i = 0; i < c->count; ++i) smem_resident[i] = 0;
        for (int i : c->smem_idx) smem_resident[i] = 1;
    }
    return FDLB_OK;
}

extern "C" int fdlb_status(fdlb_ctx* c, double* residual, int32_t* status, int64_t* steps) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_status: null context");
    int rc = FDLB_OK;
    if (residual && !rc) rc = cuda_check(c, cudaMemcpyAsync(residual, c->d_resid_all, sizeof(double) * c->count, cudaMemcpyDeviceToHost, c->stream), "status copy");
    if (status && !rc) rc = cuda_check(c, cudaMemcpyAsync(status, c->d_status_all, sizeof(int) * c->count, cudaMemcpyDeviceToHost, c->stream), "status copy");
    std::vector<long long> st(c->count);
    if (steps && !rc) rc = cuda_check(c, cudaMemcpyAsync(st.data(), c->d_steps_all, sizeof(long long) * c->count, cudaMemcpyDeviceToHost, c->stream), "status copy");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "status synchronize");
    if (!rc && steps) for (int i = 0; i < c->count; ++i) steps[i] = st[i];
    return rc;
}

extern "C" int fdlb_residual(fdlb_ctx* c, double* host_out) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_residual: null context");
    if (!host_out) return fail(c, FDLB_EINVAL, "fdlb_residual: null output");
    return fdlb_status(c, host_out, nullptr, nullptr);
}

extern "C" int fdlb_run(fdlb_ctx* c, double tol, int64_t max_steps, int64_t check_every, double timeout_s) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_run: null context");
    if (!(tol > 0) || max_steps < 0 || check_every < 1 || !(timeout_s > 0)) return fail(c, FDLB_EINVAL, "fdlb_run: bad arguments");
    auto t0 = std::chrono::steady_clock::now();
    std::vector<int> st(c->count);
    std::vector<long long> steps(c->count);
    int64_t done = 0;
    // the width chosen from the active instances holds only inside this call
    struct RestoreWidth {
        fdlb_ctx* c;
        ~RestoreWidth() { c->upd_wide = c->upd_wide_all; }
    } restore{c};
    while (true) {
        int rc = fdlb_status(c, nullptr, st.data(), nullptr);
        if (rc) return rc;
        bool active = false, nonfinite = false, unphys = false, stagnated = false, copy = false;
        for (int s : st) {
            active |= s == FDLB_ACTIVE;
            nonfinite |= s == FDLB_FAILED_NONFINITE;
            unphys |= s == FDLB_FAILED_UNPHYSICAL;
            stagnated |= s == FDLB_STAGNATED;
            copy |= s == FDLB_FAILED_COPY;
        }
        if (copy) return fail(c, FDLB_ETIMEOUT, "an asynchronous copy into shared memory did not complete (FDLB_FAILED_COPY)");
        if (!active || done >= max_steps) {
            if (nonfinite) return fail(c, FDLB_ENONFINITE, "an instance produced a non-finite moment");
            if (unphys) return fail(c, FDLB_EUNPHYSICAL, "an instance produced n <= 0 or T <= 0");
            return active ? 1 : (stagnated ? 2 : FDLB_OK);
        }
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(c, FDLB_ETIMEOUT, "fdlb_run: wall-clock limit reached");
        choose_update_width(c, st.data());
        int64_t chunk = std::min<int64_t>(check_every, max_steps - done);
        rc = fdlb_step(c, chunk, tol);
        if (rc) return rc;
        done += chunk;
    }
}

extern "C" int fdlb_moments(fdlb_ctx* c, int32_t inst, double* host_out) {
    if (!c || !host_out) return fail(c, FDLB_EINVAL, "fdlb_moments: bad arguments");
    if (inst < 0 || inst >= c->count) return fail(c, FDLB_EINVAL, "fdlb_moments: instance out of range");
    const Inst& I = c->inst[inst];
    int rc = cuda_check(c, cudaMemcpy2DAsync(host_out, sizeof(double) * I.N, I.node, sizeof(double) * I.ld,
                                             sizeof(double) * I.N, 8, cudaMemcpyDeviceToHost, c->stream), "moments copy");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "moments synchronize");
    return rc;
}

extern "C" int fdlb_set_profiles(fdlb_ctx* c, int32_t inst, const double* n, const double* uy, const double* T) {
    if (!c || !n || !uy || !T) return fail(c, FDLB_EINVAL, "fdlb_set_profiles: bad arguments");
    if (inst < 0 || inst >= c->count) return fail(c, FDLB_EINVAL, "fdlb_set_profiles: instance out of range");
    const Inst& I = c->inst[inst];
    std::vector<double> rows((size_t)4 * I.ld, 0.0);
    for (int i = 0; i < I.N; ++i) {
        if (!(n[i] > 0) || !(T[i] > 0) || !std::isfinite(uy[i])) return fail(c, FDLB_EINVAL, "fdlb_set_profiles: need n > 0, T > 0, finite u_y");
        rows[0 * I.ld + i] = n[i];
        rows[1 * I.ld + i] = 0.0;
        rows[2 * I.ld + i] = uy[i];
        rows[3 * I.ld + i] = T[i];
    }
    if (I.form == FORM_REDUCED1D) for (int i = 0; i < I.N; ++i) rows[2 * I.ld + i] = 0.0;
    int rc = cuda_check(c, cudaMemcpyAsync(I.node, rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice, c->stream), "profiles upload");
    if (!rc) rc = cuda_check(c, launch_set_profiles(c->d_inst, inst, c->stream), "profiles kernel");
    if (!rc) rc = cuda_check(c, launch_moments(c->d_inst, c->d_upd, c->n_upd, 0, c->ukc_max, c->any_fp64, c->any_fp32, c->stream), "moments kernel");
    if (!rc) rc = cuda_check(c, launch_resid(c->d_inst, c->count, inst, 0.0, c->d_resid_all, c->stream), "residual kernel");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "profiles synchronize");
    return rc;
}

// ---- checkpoint: [magic u64][hash u64][steps i64][f bytes]
static uint64_t param_hash(const fdlb_params& p) { return params_fnv(p, false); }

// Two-phase instances add [storage i64][switch step i64] after the header and always carry f
// at its FP64 size.
static size_t phase_bytes(const Inst& I) { return I.two_phase ? 16 : 0; }

static size_t f_bytes_of(const Inst& I) {
    return (size_t)I.K * I.ld * (I.precision == FDLB_FP32_STORAGE && !I.two_phase ? 4 : 8);
}

extern "C" size_t fdlb_state_bytes(const fdlb_ctx* c, int32_t inst) {
    if (!c || inst < 0 || inst >= c->count) return 0;
    const Inst& I = c->inst[inst];
    return 24 + phase_bytes(I) + f_bytes_of(I);
}

// Device copies of an instance's current storage precision and switch step.
static int read_phase(fdlb_ctx* c, int inst, int32_t* storage, int64_t* sw) {
    const Inst& I = c->inst[inst];
    if (!I.two_phase) {
        *storage = I.precision;
        *sw = -1;
        return FDLB_OK;
    }
    int32_t pr = 0;
    double swd = -1.0;
    const char* dI = reinterpret_cast<const char*>(c->d_inst + inst);
    int rc = cuda_check(c, cudaMemcpyAsync(&pr, dI + offsetof(Inst, precision), sizeof(pr), cudaMemcpyDeviceToHost, c->stream), "phase copy");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(&swd, I.misc + M_SWITCH, sizeof(swd), cudaMemcpyDeviceToHost, c->stream), "phase copy");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "phase synchronize");
    *storage = pr;
    *sw = (int64_t)swd;
    return rc;
}

extern "C" int fdlb_precision(fdlb_ctx* c, int32_t* storage, int64_t* switch_step) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_precision: null context");
    for (int i = 0; i < c->count; ++i) {
        int32_t pr;
        int64_t sw;
        int rc = read_phase(c, i, &pr, &sw);
        if (rc) return rc;
        if (storage) storage[i] = pr;
        if (switch_step) switch_step[i] = sw;
    }
    return FDLB_OK;
}

extern "C" int fdlb_get_state(fdlb_ctx* c, int32_t inst, void* host, size_t bytes) {
    if (!c || !host) return fail(c, FDLB_EINVAL, "fdlb_get_state: bad arguments");
    size_t need = fdlb_state_bytes(c, inst);
    if (need == 0 || bytes < need) return fail(c, FDLB_EINVAL, "fdlb_get_state: instance out of range or buffer too small");
    const Inst& I = c->inst[inst];
    uint64_t hdr[3] = {0x46444c42u, param_hash(c->prm[inst]), 0};
    const size_t ph = phase_bytes(I);
    int64_t phase[2] = {0, -1};
    if (ph) {
        int32_t pr;
        int rc = read_phase(c, inst, &pr, &phase[1]);
        if (rc) return rc;
        phase[0] = pr;
    }
    long long st = 0;
    // in the FP32 phase only the first half of a two-phase f buffer is state; the rest is zeroed
    const size_t fb = need - 24 - ph, used = (ph && phase[0] == FDLB_FP32_STORAGE) ? fb / 2 : fb;
    if (used < fb) std::memset(static_cast<char*>(host) + 24 + ph + used, 0, fb - used);
    int rc = cuda_check(c, cudaMemcpyAsync(&st, I.steps, sizeof(st), cudaMemcpyDeviceToHost, c->stream), "state copy");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(static_cast<char*>(host) + 24 + ph, I.f[0], used, cudaMemcpyDeviceToHost, c->stream), "state copy");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "state synchronize");
    if (rc) return rc;
    hdr[2] = (uint64_t)st;
    std::memcpy(host, hdr, 24);
    if (ph) std::memcpy(static_cast<char*>(host) + 24, phase, 16);
    return FDLB_OK;
}

extern "C" int fdlb_set_state(fdlb_ctx* c, int32_t inst, const void* host, size_t bytes) {
    if (!c || !host) return fail(c, FDLB_EINVAL, "fdlb_set_state: bad arguments");
    size_t need = fdlb_state_bytes(c, inst);
    if (need == 0 || bytes != need) return fail(c, FDLB_ESTATE, "fdlb_set_state: size does not match this instance");
    uint64_t hdr[3];
    std::memcpy(hdr, host, 24);
    if (hdr[0] != 0x46444c42u || hdr[1] != param_hash(c->prm[inst])) return fail(c, FDLB_ESTATE, "fdlb_set_state: state belongs to other parameters");
    const Inst& I = c->inst[inst];
    long long st = (long long)hdr[2];
    const size_t ph = phase_bytes(I);
    int rc = FDLB_OK;
    // kept alive until the synchronisation below (the copies are asynchronous)
    int32_t pr = 0;
    double swd = -1.0;
    if (ph) {
        int64_t phase[2];
        std::memcpy(phase, static_cast<const char*>(host) + 24, 16);
        if (phase[0] != FDLB_FP64 && phase[0] != FDLB_FP32_STORAGE) return fail(c, FDLB_ESTATE, "fdlb_set_state: bad storage phase");
        pr = (int32_t)phase[0];
        swd = (double)phase[1];
        char* dI = reinterpret_cast<char*>(c->d_inst + inst);
        rc = cuda_check(c, cudaMemcpyAsync(dI + offsetof(Inst, precision), &pr, sizeof(pr), cudaMemcpyHostToDevice, c->stream), "state upload");
        if (!rc) rc = cuda_check(c, cudaMemcpyAsync(I.misc + M_SWITCH, &swd, sizeof(swd), cudaMemcpyHostToDevice, c->stream), "state upload");
    }
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(I.f[0], static_cast<const char*>(host) + 24 + ph, need - 24 - ph, cudaMemcpyHostToDevice, c->stream), "state upload");
    if (!rc) rc = cuda_check(c, launch_moments(c->d_inst, c->d_upd, c->n_upd, 0, c->ukc_max, c->any_fp64, c->any_fp32, c->stream), "moments kernel");
    if (!rc) rc = cuda_check(c, launch_resid(c->d_inst, c->count, inst, 0.0, c->d_resid_all, c->stream), "residual kernel");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(I.steps, &st, sizeof(st), cudaMemcpyHostToDevice, c->stream), "state upload");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "state synchronize");
    return rc;
}

extern "C" int fdlb_profile(fdlb_ctx* c, int32_t on) {
    if (!c) return fail(nullptr, FDLB_EINVAL, "fdlb_profile: null context");
    c->prof = on != 0;
    for (int k = 0; k < KK_COUNT; ++k) c->nev[k] = 0;
    return FDLB_OK;
}

extern "C" int fdlb_profile_read(fdlb_ctx* c, int32_t kind, double* total_ms, int64_t* launches) {
    if (!c || kind < 0 || kind >= KK_COUNT) return fail(c, FDLB_EINVAL, "fdlb_profile_read: bad arguments");
    int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "profile synchronize");
    if (rc) return rc;
    double tot = 0.0;
    for (size_t j = 0; j + 1 < c->nev[kind]; j += 2) {
        float ms = 0.0f;
        rc = cuda_check(c, cudaEventElapsedTime(&ms, c->ev[kind][j], c->ev[kind][j + 1]), "profile elapsed");
        if (rc) return rc;
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (int64_t)(c->nev[kind] / 2);
    return FDLB_OK;
}

// ---------------------------------------------------------------------------
// internal accessors (fdlb_ctx_internal.h)
// ---------------------------------------------------------------------------
namespace fdlb {

int ctx_f_buffer(fdlb_ctx* c, int inst, void** f, size_t* bytes) {
    if (!c || inst < 0 || inst >= c->count) return fail(c, FDLB_EINVAL, "internal: bad instance");
    const Inst& I = c->inst[inst];
    *f = I.f[0];
    *bytes = f_bytes_of(I);
    return FDLB_OK;
}

int ctx_reanchor(fdlb_ctx* c, int inst) {
    if (!c || inst < 0 || inst >= c->count) return fail(c, FDLB_EINVAL, "internal: bad instance");
    static const int active = FDLB_ACTIVE;
    const Inst& I = c->inst[inst];
    int rc = cuda_check(c, cudaMemcpyAsync(I.status, &active, sizeof(int), cudaMemcpyHostToDevice, c->stream), "status reset");
    if (!rc) rc = cuda_check(c, launch_moments(c->d_inst, c->d_upd, c->n_upd, 0, c->ukc_max, c->any_fp64, c->any_fp32, c->stream), "moments kernel");
    if (!rc) rc = cuda_check(c, launch_resid(c->d_inst, c->count, inst, 0.0, c->d_resid_all, c->stream), "residual kernel");
    return rc;
}

int ctx_moment_rows(fdlb_ctx* c, int inst, const double** rows, int* ld, int* nx) {
    if (!c || inst < 0 || inst >= c->count) return fail(c, FDLB_EINVAL, "internal: bad instance");
    const Inst& I = c->inst[inst];
    *rows = I.node;
    *ld = I.ld;
    *nx = I.N;
    return FDLB_OK;
}

cudaStream_t ctx_stream(fdlb_ctx* c) { return c->stream; }

// fdlb_step then launches every step's kernels directly: no stream capture, no graph
// instantiation (which may allocate inside the driver).
void ctx_direct_launches(fdlb_ctx* c) { c->graph_failed = true; }

void set_global_error(const std::string& msg) { g_err = msg; }

}  // namespace fdlb
