// CUDA kernels of the FDLB solver for the simplified Enskog equation (sm_103a).
//
// One TVD-RK3 stage (Eq. rk3) is two kernels over a batch of independent channel problems:
//   k_nodal    per node: chi (Eq. chi), Pr (Eq. prandtl), tau (Eqs. viscosity, tau),
//              6th-order gradients (Sec. III B 3), the 13 monomial coefficients of
//              f^S + tau J1 (Sec. II A, Eq. j1) and their projections onto the
//              half-range (Sec. III A 2) and full-range (App. A) velocity sets (on x
//              either rule);
//              per instance: the wall densities n_w (Sec. III B);
//   k_update   per (velocity, node): WENO-5 fluxes (Sec. III B 2) with the
//              diffuse-reflection closure, the p_y-derivative force (App. A,
//              Eq. kernel_H), relaxation to the projected target and the RK3
//              combination; its epilogue reduces the new values to the moments
//              n, u, T, q, Pi of every node (Eq. macro_LB) for the next stage.
// After stage 3, k_resid (per-step residual, status).  k_moments computes the moments
// from scratch (creation, new profiles, a loaded state) with the epilogue's arithmetic.
// k_resident runs whole steps of one instance per thread-block cluster with the same item
// functions.
//
// Storage type S (double | float) holds f; compute type C of the per-velocity work is
// double for FDLB_FP64 and float for FDLB_FP32_STORAGE.  FP64 instances do all the rest in
// double; FP32-storage instances run the moment sums and the velocity projections in
// double-float (float pairs) and keep the closure chain, the moment finalisation and the
// residual in double.
#include "fdlb_internal.h"
#include "fdlb_launch.h"
#include "../../include/fdlb.h"

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <mutex>

namespace fdlb {

__constant__ double c_inv[13] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12};

__constant__ int c_mono[NTERMS][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0},
                                      {3, 0, 0}, {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {0, 3, 0}, {0, 1, 2}};

__device__ __forceinline__ double chi_cs(double eta) {
    const double om = 1.0 - eta;
    return (2.0 - eta) / (2.0 * om * om * om);
}

// ---------------------------------------------------------------------------
// projections of (p - u)^a g(p; u, T), a = 0..3
// ---------------------------------------------------------------------------

// Half-range axis (Sec. III A 2): value at node +p_k (half = 0) of
//   int_0^inf l_k(p) (p - u)^a g(p; u, T) dp,
// or at node -p_k (half = 1), which is (-1)^a times the same with u -> -u.  Evaluated in
// the orthonormal basis, value_k = w_k sum_l h_l(p_k) G_l, with
//   G_l = int_0^inf h_l(p) (p - u)^a g dp = sum_m W_m exp(q_m v - v^2/2) h_l(sqrt(T) q_m) y_m^a,
// p = sqrt(T) q, v = u/sqrt(T), y_m = sqrt(T) q_m - u, on the MX-point auxiliary rule.
// Full-range x axis (App. A, I.xfull): the integrals run over the whole line with the
// 2Q-node basis, G_l = sum_m W_m h_l(u + sqrt(T) y_m) (sqrt(T) y_m)^a on the Mx-point
// Gauss-Hermite rule (exact); the rule is symmetric, so the mirror relation for -p_k holds
// as well.
__device__ void proj_x(const Inst& I, double u, double T, int half, double* out, int stride) {
    const int Q = I.Q, Lx = I.Lx;
    const bool full = I.xfull;
    const double uu = half ? -u : u;
    const double sT = sqrt(T), v = uu / sT, ev = -0.5 * v * v;
    const int M = I.Mx;
    // the polynomials in blocks of QMAX; the H products continue one chain across blocks
    // (kept in out, signed at the end)
    for (int lb = 0; lb < Lx; lb += QMAX) {
        const int nl = min(QMAX, Lx - lb);
        double G[4][QMAX];
#pragma unroll
        for (int a = 0; a < 4; ++a)
            for (int l = 0; l < QMAX; ++l) G[a][l] = 0.0;
        for (int m = 0; m < M; ++m) {
            const double q = I.xq[m];
            const double x = full ? fma(sT, q, uu) : sT * q;
            const double E = full ? I.xw[m] : I.xw[m] * exp(fma(q, v, ev));
            const double y = full ? sT * q : x - uu;
            const double e1 = E * y, e2 = e1 * y, e3 = e2 * y;
            double hm = 0.0, h = I.x_h0;
            for (int l = 0; l < lb; ++l) {
                const double hn = ((x - I.xa[l]) * h - I.xb[l] * hm) * I.xib[l + 1];
                hm = h;
                h = hn;
            }
            for (int j = 0; j < nl; ++j) {
                const int l = lb + j;
                G[0][j] = fma(E, h, G[0][j]);
                G[1][j] = fma(e1, h, G[1][j]);
                G[2][j] = fma(e2, h, G[2][j]);
                G[3][j] = fma(e3, h, G[3][j]);
                const double hn = ((x - I.xa[l]) * h - I.xb[l] * hm) * I.xib[l + 1];
                hm = h;
                h = hn;
            }
        }
        const bool last = lb + nl == Lx;
        for (int a = 0; a < 4; ++a) {
            const double sgn = (half && (a & 1)) ? -1.0 : 1.0;
            for (int k = 0; k < Q; ++k) {
                double* o = out + (a * 2 * Q + half * Q + k) * stride;
                double s = lb == 0 ? 0.0 : *o;
                for (int j = 0; j < nl; ++j) s = fma(I.xH[(lb + j) * Q + k], G[a][j], s);
                *o = last ? sgn * s : s;
            }
        }
    }
}

// Full-range axis (App. A): out[a*Qn + k] = int_R l_k(p) (p - u)^a g(p; u, T) dp, exact
// with p = u + sqrt(T) y on the M-point Gauss-Hermite rule (2M - 1 >= Qn + 2).
__device__ void proj_full(const Inst& I, const double* aq, const double* aw, const double* H, int Qn, int M, double u,
                          double T, int amax, double* out) {
    double G[4][QYMAX];
#pragma unroll
    for (int a = 0; a < 4; ++a)
        for (int l = 0; l < QYMAX; ++l) G[a][l] = 0.0;
    const double sT = sqrt(T);
    for (int m = 0; m < M; ++m) {
        const double y = sT * aq[m], x = u + y, E = aw[m];
        const double e1 = E * y, e2 = e1 * y, e3 = e2 * y;
        double hm = 0.0, h = 1.0;
        for (int l = 0; l < Qn; ++l) {
            G[0][l] = fma(E, h, G[0][l]);
            G[1][l] = fma(e1, h, G[1][l]);
            G[2][l] = fma(e2, h, G[2][l]);
            G[3][l] = fma(e3, h, G[3][l]);
            const double hn = (x * h - I.fsq[l] * hm) * I.fisq[l + 1];
            hm = h;
            h = hn;
        }
    }
    for (int a = 0; a <= amax; ++a)
        for (int k = 0; k < Qn; ++k) {
            double s = 0.0;
            for (int l = 0; l < Qn; ++l) s = fma(H[l * Qn + k], G[a][l], s);
            out[a * Qn + k] = s;
        }
}

// E[xi^j] of a centred Gaussian of variance T.
__device__ __forceinline__ double gmom(int j, double T) {
    switch (j) {
        case 0: return 1.0;
        case 2: return T;
        case 4: return 3.0 * T * T;
        case 6: return 15.0 * T * T * T;
        default: return 0.0;
    }
}

// Transverse factors: out[(a*Tc + t)*stride] = nscale * sum_{terms with x-power a} c_term * Ytrans(t).
__device__ void build_Y(const Inst& I, const double* c, double uy, double T, double nscale, double* out, int stride) {
    const int Tc = I.Tc;
    if (I.form == FORM_REDUCED1D) {
        for (int a = 0; a < 4; ++a)
            for (int slot = 0; slot < 2; ++slot) {
                double s = 0.0;
                for (int j = 0; j < NTERMS; ++j) {
                    if (c_mono[j][0] != a) continue;
                    const int b = c_mono[j][1], cc = c_mono[j][2];
                    const double e = slot == 0 ? gmom(b, T) * gmom(cc, T)
                                               : gmom(b + 2, T) * gmom(cc, T) + gmom(b, T) * gmom(cc + 2, T);
                    s = fma(c[j], e, s);
                }
                out[(a * Tc + slot) * stride] = nscale * s;
            }
        return;
    }
    double Py[4 * QYMAX];
    proj_full(I, I.yq, I.yw, I.yH, I.Qy, I.My, uy, T, 3, Py);
    const int Qy = I.Qy;
    if (I.form == FORM_UNREDUCED) {
        double Pz[3 * QZMAX];
        const int Qz = I.Qz;
        proj_full(I, I.zq, I.zw, I.zH, Qz, I.Mz, 0.0, T, 2, Pz);
        for (int a = 0; a < 4; ++a)
            for (int t = 0; t < Tc; ++t) {
                const int ky = t / Qz, kz = t - ky * Qz;
                double s = 0.0;
                for (int j = 0; j < NTERMS; ++j) {
                    if (c_mono[j][0] != a) continue;
                    s = fma(c[j], Py[c_mono[j][1] * Qy + ky] * Pz[c_mono[j][2] * Qz + kz], s);
                }
                out[(a * Tc + t) * stride] = nscale * s;
            }
    } else {
        for (int a = 0; a < 4; ++a)
            for (int t = 0; t < Tc; ++t) {
                const int ky = t >> 1, slot = t & 1;
                double s = 0.0;
                for (int j = 0; j < NTERMS; ++j) {
                    if (c_mono[j][0] != a) continue;
                    const int cc = c_mono[j][2];
                    const double zf = slot == 0 ? gmom(cc, T) : gmom(cc + 2, T);
                    s = fma(c[j], Py[c_mono[j][1] * Qy + ky] * zf, s);
                }
                out[(a * Tc + t) * stride] = nscale * s;
            }
    }
}

// ---------------------------------------------------------------------------
// set-up: wall Maxwellians, initial state
// ---------------------------------------------------------------------------
__device__ void wall_maxwellian(const Inst& I, double U, double T, double* g) {
    double Px[4 * 2 * QX_FULL_MAX];
    proj_x(I, 0.0, T, 0, Px, 1);
    proj_x(I, 0.0, T, 1, Px, 1);
    double c[NTERMS];
    for (int j = 0; j < NTERMS; ++j) c[j] = 0.0;
    c[0] = 1.0;
    double Y[4 * TCMAX];
    build_Y(I, c, U, T, 1.0, Y, 1);
    for (int k = 0; k < I.K; ++k) {
        const int kx = k / I.Tc, t = k - kx * I.Tc;
        g[k] = Px[kx] * Y[t];
    }
}

__global__ void k_setup(Inst* insts) {
    Inst& I = insts[blockIdx.x];
    if (threadIdx.x == 0) wall_maxwellian(I, I.U_L, I.T_L, I.gL);
    if (threadIdx.x == 32) wall_maxwellian(I, I.U_R, I.T_R, I.gR);
    __syncthreads();
    if (I.gL32)
        for (int k = threadIdx.x; k < I.K; k += blockDim.x) {
            I.gL32[k] = (float)I.gL[k];
            I.gR32[k] = (float)I.gR[k];
        }
    if (threadIdx.x == 0) {
        const int Q = I.Q, Tc = I.Tc;
        double inL = 0.0, inR = 0.0;
        for (int k = 0; k < I.K; ++k) {
            const int kx = k / Tc, t = k - kx * Tc;
            const double mp = I.tmt[t] * I.px[kx];
            if (kx < Q) inL = fma(mp, I.gL[k], inL);
            else inR = fma(mp, I.gR[k], inR);
        }
        I.misc[M_INL] = inL;
        I.misc[M_INR] = inR;
        I.misc[M_NWL] = 1.0;
        I.misc[M_NWR] = 1.0;
        I.misc[M_RESID] = CUDART_INF;
        I.misc[M_WIN_STEP] = -1.0;
        I.misc[M_WIN_RESID] = CUDART_INF;
        I.misc[M_SWITCH] = -1.0;
        *I.status = FDLB_ACTIVE;
        *I.steps = 0;
    }
    const double T0 = I.T_init;
    for (int i = threadIdx.x; i < I.ld; i += blockDim.x) {
        I.node[R_N * I.ld + i] = 1.0;
        I.node[R_UX * I.ld + i] = 0.0;
        I.node[R_UY * I.ld + i] = 0.0;
        I.node[R_T * I.ld + i] = T0;
    }
}

// Projected local equilibrium from the profile rows into F (all instances when inst < 0).
template <typename S>
__global__ void k_profiles(Inst* insts, int inst) {
    Inst& I = insts[inst < 0 ? blockIdx.x : inst];
    if (I.two_phase) {
        // a two-phase instance restarts in its FP32 phase: the FP64 launch (first in stream
        // order) resets the phase, the FP32 launch writes f
        if (sizeof(S) == 8) {
            if (threadIdx.x == 0) {
                I.precision = FDLB_FP32_STORAGE;
                I.misc[M_SWITCH] = -1.0;
            }
            return;
        }
    } else if ((I.precision == FDLB_FP64) != (sizeof(S) == 8)) {
        return;
    }
    const int ld = I.ld, Q = I.Q, Tc = I.Tc;
    double c[NTERMS];
    for (int j = 0; j < NTERMS; ++j) c[j] = 0.0;
    c[0] = 1.0;
    for (int i = threadIdx.x; i < I.N; i += blockDim.x) {
        const double n = I.node[R_N * ld + i], uy = I.node[R_UY * ld + i], T = I.node[R_T * ld + i];
        proj_x(I, 0.0, T, 0, I.tab + i, ld);
        proj_x(I, 0.0, T, 1, I.tab + i, ld);
        build_Y(I, c, uy, T, n, I.tab + 8 * Q * ld + i, ld);
    }
    __syncthreads();
    S* F = static_cast<S*>(I.f[0]);
    for (int k = 0; k < I.K; ++k) {
        const int kx = k / Tc, t = k - kx * Tc;
        for (int i = threadIdx.x; i < ld; i += blockDim.x) {
            double v = 0.0;
            if (i < I.N)
                for (int a = 0; a < 4; ++a) v = fma(I.tab[(a * 2 * Q + kx) * ld + i], I.tab[(8 * Q + a * Tc + t) * ld + i], v);
            F[(size_t)k * ld + i] = (S)v;
        }
    }
    if (threadIdx.x == 0) {
        *I.status = FDLB_ACTIVE;
        *I.steps = 0;
    }
}

// ---------------------------------------------------------------------------
// moments
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// double-float arithmetic (unevaluated float pairs hi + lo, ~2^-46 relative) for the
// projections of FP32-storage instances: their tables are rounded to FP32, and FP32 FMAs run
// 64 times faster than FP64 FMAs on this GPU.  Error-free transformations (TwoSum, FMA
// products, Dekker's fast two-sum) use the _rn intrinsics so that no contraction changes them.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_fast(float a, float b) {      // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fadd_rn(b, __fsub_rn(a, s))};
}
__device__ __forceinline__ df operator+(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df_fast(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast(p, e);
}
__device__ __forceinline__ df df_of(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ df df_of(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ float df_float(df a) { return __fadd_rn(a.hi, a.lo); }

constexpr int NTW = 6;     // transverse weights: mt, mt py, mt py^2, mt py^3, et, et py

// Inner (transverse) running sum of w(t) f over t.  FP64 storage: an FP64 FMA.  FP32
// storage: an unevaluated pair hi + lo of floats (error-free product of f with the float
// head of w, the tail of w applied in float, TwoSum accumulation), ~1e-13 relative.
template <typename S>
struct InnerSum;

template <>
struct InnerSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double f, double w, float, float) { s = fma(w, f, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct InnerSum<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float f, double, float wh, float wl) {
        const float p = f * wh;
        float e = fmaf(f, wh, -p);
        e = fmaf(f, wl, e);
        const float t = hi + p;
        const float bb = t - hi;
        const float err = (hi - (t - bb)) + (p - bb);
        hi = t;
        lo += err + e;
    }
    // adds a value known exactly (a product by a power of two), TwoSum on the head: the same
    // result as add() with a zero product error
    __device__ __forceinline__ void add_exact(float p) {
        const float t = hi + p;
        const float bb = t - hi;
        const float err = (hi - (t - bb)) + (p - bb);
        hi = t;
        lo += err;
    }
    // adds another pair's value h + l (TwoSum on the heads)
    __device__ __forceinline__ void add_pair(float h, float l) {
        const float t = hi + h;
        const float bb = t - hi;
        const float err = (hi - (t - bb)) + (h - bb);
        hi = t;
        lo += err + l;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Per node: the 14 raw sums over all velocities, factorised as sum_kx px^a (sum_t w_j(t) f),
// and the moments they give.

// Temperature from the raw sums (the same operations wherever it is needed).
__device__ __forceinline__ double sums_temperature(double n, double s1, double s2, double s3, double s4, double s6,
                                                   double s7) {
    const double ux = (s1 + s2) / n, uy = s3 / n;
    const double Pxx = s4 - n * ux * ux, Pyy = s6 - n * uy * uy;
    const double E = 0.5 * (Pxx + Pyy) + s7;
    return E / (1.5 * n);
}

// Moments of the nodes of tile i0 from the raw sums ss[MOM_SUMS][TILE], by 128 threads: warp 0
// writes the primitive rows, warps 1..3 ln n, ln T and ln chi(eta0 n) (independent FP64
// chains on different schedulers).
__device__ void finalize_tile(const Inst& I, int i0, const double* ss, int tid) {
    const int lane = tid & 31, g = tid >> 5, i = i0 + lane;
    if (i >= I.N) return;
    const int ld = I.ld;
    double* nd = I.node;
    double s[MOM_SUMS];
#pragma unroll
    for (int j = 0; j < MOM_SUMS; ++j) s[j] = ss[j * TILE + lane];
    const double n = s[0];
    if (g == 1) {
        nd[R_LNN * ld + i] = log(n);
    } else if (g == 2) {
        nd[R_LNT * ld + i] = log(sums_temperature(n, s[1], s[2], s[3], s[4], s[6], s[7]));
    } else if (g == 3) {
        nd[R_LNCHI * ld + i] = log(chi_cs(I.eta0 * n));
    } else {
        const double sx = s[1] + s[2];
        const double ux = sx / n, uy = s[3] / n;
        const double Pxx = s[4] - n * ux * ux, Pxy = s[5] - n * ux * uy;
        const double T = sums_temperature(n, s[1], s[2], s[3], s[4], s[6], s[7]);
        const double cx3 = s[8] - 3.0 * ux * s[4] + 2.0 * n * ux * ux * ux;
        const double cxyy = s[9] - 2.0 * uy * s[5] - ux * s[6] + 2.0 * n * ux * uy * uy;
        const double cxxy = s[10] - 2.0 * ux * s[5] - uy * s[4] + 2.0 * n * ux * ux * uy;
        const double cy3 = s[11] - 3.0 * uy * s[6] + 2.0 * n * uy * uy * uy;
        const double qx = 0.5 * (cx3 + cxyy) + (s[12] - ux * s[7]);
        const double qy = 0.5 * (cy3 + cxxy) + (s[13] - uy * s[7]);
        nd[R_N * ld + i] = n;
        nd[R_UX * ld + i] = ux;
        nd[R_UY * ld + i] = uy;
        nd[R_T * ld + i] = T;
        nd[R_QX * ld + i] = qx;
        nd[R_QY * ld + i] = qy;
        nd[R_PXX * ld + i] = Pxx;
        nd[R_PXY * ld + i] = Pxy;
        nd[R_SNEG * ld + i] = s[1];
        nd[R_SPOS * ld + i] = s[2];
    }
}

// Programmatic dependent launch: a stepping kernel launched with programmatic stream
// serialization may start while its predecessor in the stream drains; it waits here, before
// reading anything, until the predecessor has completed and its writes are visible (a no-op
// for a kernel launched without the attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Named barrier over `n` threads (moment finalisation runs on 128-thread parts of a block).
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }


// Adds the x-velocity p's contribution to the 14 raw sums from the 6 transverse sums S.
__device__ __forceinline__ void outer_sums(double* o, const double* S, double p, bool neg) {
    const double p2 = p * p, p3 = p2 * p;
    o[0] += S[0];
    if (neg) o[1] = fma(p, S[0], o[1]); else o[2] = fma(p, S[0], o[2]);
    o[3] += S[1];
    o[4] = fma(p2, S[0], o[4]);
    o[5] = fma(p, S[1], o[5]);
    o[6] += S[2];
    o[7] += S[4];
    o[8] = fma(p3, S[0], o[8]);
    o[9] = fma(p, S[2], o[9]);
    o[10] = fma(p2, S[1], o[10]);
    o[11] += S[3];
    o[12] = fma(p, S[4], o[12]);
    o[13] += S[5];
}


// Outer sums in double-float (FP32 storage): as outer_sums, p and S as float pairs.
__device__ __forceinline__ void outer_sums_df(df* o, const df* S, df p, bool neg) {
    const df p2 = p * p, p3 = p2 * p;
    o[0] = o[0] + S[0];
    if (neg) o[1] = p * S[0] + o[1]; else o[2] = p * S[0] + o[2];
    o[3] = o[3] + S[1];
    o[4] = p2 * S[0] + o[4];
    o[5] = p * S[1] + o[5];
    o[6] = o[6] + S[2];
    o[7] = o[7] + S[4];
    o[8] = p3 * S[0] + o[8];
    o[9] = p * S[2] + o[9];
    o[10] = p2 * S[1] + o[10];
    o[11] = o[11] + S[3];
    o[12] = p * S[4] + o[12];
    o[13] = o[13] + S[5];
}

// Normalised pair of an InnerSum<float> (TwoSum of head and tail).
__device__ __forceinline__ df df_norm(float h, float l) {
    const float s = __fadd_rn(h, l);
    const float bb = __fsub_rn(s, h);
    return {s, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(l, bb))};
}

// Moments of tile i0 from the I.mgroups partials of its update chunks, added in chunk order,
// by 128 threads (barrier `bar`); ss: MOM_SUMS x TILE doubles of shared memory.
// nw warps (tid < 32 nw, barrier `bar` over them, nw >= 4) share the sums; FP32 storage keeps
// the partials as float pairs and adds them in double-float, FP64 storage in FP64.
template <typename S>
__device__ void moments_final_tile(const Inst& I, int i0, double* ss, int tid, int nw, int bar) {
    const int lane = tid & 31, g = tid >> 5, i = i0 + lane;
    const int ld = I.ld, G = I.mgroups;
    named_sync(bar, 32 * nw);             // the previous item's readers of `ss` are done
    for (int j = g; j < MOM_SUMS; j += nw) {
        double v = 0.0;
        if (i < I.N) {
            if constexpr (sizeof(S) == 4) {
                const float2* ms = reinterpret_cast<const float2*>(I.msum);
                df a = {0.0f, 0.0f};
                for (int q = 0; q < G; ++q) a = a + df_of(__ldcg(ms + ((size_t)q * MOM_SUMS + j) * ld + i));
                v = (double)a.hi + (double)a.lo;
            } else {
                for (int q = 0; q < G; ++q) v += __ldcg(I.msum + ((size_t)q * MOM_SUMS + j) * ld + i);
            }
        }
        ss[j * TILE + lane] = v;
    }
    named_sync(bar, 32 * nw);
    if (tid < 128) finalize_tile(I, i0, ss, tid);
}

// ---------------------------------------------------------------------------
// per-node closure and projection tables
// ---------------------------------------------------------------------------
// Three independent block roles per 32-node tile (lane = node, so every FP64 instruction runs
// with full lanes): role 0 / 1 = x projection onto the nodes +p_k / -p_k (half-range rules,
// or the full-range rule of order 2Q), role 2 = gradients, closure, coefficients, y and z
// projections and the transverse factors.
// Shared doubles: role 0/1: [NOD_WARPS][4 Lx][32] partials + [4 Lx][32] sums (Lx = Q or 2Q);
//                 role 2:   [20][32] scalars + Py [4 QYMAX][32] + Pz [3 QZMAX][32] + A [8 QYMAX][32].
constexpr int CL_ROWS = 5 + 8 + 15;    // closure item: gradients, scalars, coefficients

__host__ __device__ inline int nodal_smem_doubles(int qmax) {
    // larger x orders run in blocks of QMAX polynomials, with the recurrence state of every
    // auxiliary point kept between blocks: [M][2][32] more (M bounded for either x rule)
    const int mst = qmax > QMAX ? (aux_points_half(qmax) > qmax / 2 + 2 ? aux_points_half(qmax) : qmax / 2 + 2) : 0;
    if (qmax > QMAX) qmax = QMAX;
    const int r01 = (NOD_WARPS + 1) * 4 * qmax * TILE + 2 * mst * TILE;
    const int r2 = (CL_ROWS + 4 * QYMAX + 3 * QZMAX + 8 * QYMAX + 2 * MYMAX * (QYMAX + 1)) * TILE;
    return r01 > r2 ? r01 : r2;
}

// 1/j as float pairs, j = 0..16 (set by prepare_kernels)
constexpr int NINV2 = 17;
__constant__ float2 c_inv2[NINV2];

// exp of a double-float: z = k ln 2 + r with |r| <= ln 2 / 2, e^r from its Taylor series to
// r^14/14! (the rest is below 2^-57 relative), then the exact scaling by 2^k.  For |z| < 80.
__device__ __forceinline__ df df_exp(df z) {
    const df ln2 = {0.693147182464599609375f, -1.90465429995776787e-09f};
    const float k = rintf(z.hi * 1.44269504088896341f);
    const df r = z - ln2 * df{k, 0.0f};
    const df one = {1.0f, 0.0f};
    df e = one;
#pragma unroll
    for (int j = 14; j >= 1; --j) e = e * r * df_of(c_inv2[j]) + one;
    const int ki = (int)k;
    return {ldexpf(e.hi, ki), ldexpf(e.lo, ki)};
}

// Half-range x projection of an FP32-storage tile (roles 0 / 1 of nodal_item) in double-float:
// the same steps as the FP64 branch, with the per-node scalars sqrt(T), u and v computed once
// by warp 0 and shared.
template <int QB>
__device__ void xproj_df(const Inst& I, int i0, int role, double* nsm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = i0 + lane, N = I.N, ld = I.ld, Q = I.Q;
    const bool valid = i < N;
    const int ic = valid ? i : N - 1;
    __shared__ float2 xs[4][TILE];                   // sqrt(T), u, v, v^2/2 as pairs
    __shared__ int use_short;
    if (wid == 0) {
        // sqrt T and u / sqrt T in double-float: one Newton correction of the FP32 root and
        // quotient (both ~1e-14)
        const double ux = I.node[R_UX * ld + ic];
        const df T = df_of(I.node[R_T * ld + ic]), uu = df_of(role ? -ux : ux);
        const float s0 = sqrtf(T.hi);
        const df r0 = T - df{s0, 0.0f} * df{s0, 0.0f};
        const df sT = df_fast(s0, __fdiv_rn(r0.hi, 2.0f * s0));
        const float q0 = __fdiv_rn(uu.hi, sT.hi);
        const df r1 = uu - df{q0, 0.0f} * sT;
        const df v = df_fast(q0, __fdiv_rn(r1.hi, sT.hi));
        const df d = df{0.5f, 0.0f} * v * v;
        xs[0][lane] = make_float2(sT.hi, sT.lo);
        xs[1][lane] = make_float2(uu.hi, uu.lo);
        xs[2][lane] = make_float2(v.hi, v.lo);
        xs[3][lane] = make_float2(d.hi, d.lo);
        float av = valid ? fabsf(v.hi) : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) av = fmaxf(av, __shfl_xor_sync(0xffffffffu, av, o));
        if (lane == 0) use_short = av < 0.02f ? 1 : 2;
    }
    __syncthreads();
    const bool full = I.xfull;               // full-range x: as in the FP64 branch
    const int Lx = I.Lx;
    const bool short_rule = !full && use_short == 1 && Q <= 12;
    const int M = full ? I.Mx : (short_rule ? MX8 : I.Mx);
    const df sT = df_of(xs[0][lane]), uu = df_of(xs[1][lane]), v = df_of(xs[2][lane]), hv2 = df_of(xs[3][lane]);
    const df one = {1.0f, 0.0f};
    float2* part = reinterpret_cast<float2*>(nsm);                  // [NOD_WARPS][4 nl][32]
    float2* hst = part + (NOD_WARPS + 1) * 4 * QB * TILE;           // [M][2][32] recurrence state (Lx > QB)
    // blocks of QB polynomials as in the FP64 branch; the chain of H products continues across
    // blocks as float pairs in the instance's FP64 table rows (8 bytes each), and the last
    // block rounds it into the FP32 table
    float2* acc = reinterpret_cast<float2*>(I.tab);
    for (int lb = 0; lb < Lx; lb += QB) {
        const int nl = min(QB, Lx - lb);
        float2* sum = part + NOD_WARPS * 4 * nl * TILE;             // [4 nl][32]
        df G[4][QB];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int l = 0; l < QB; ++l) G[a][l] = {0.0f, 0.0f};
        for (int m = wid; m < M; m += NOD_WARPS) {
            const df q = df_of(short_rule ? I.xq82[m] : I.xq2[m]);
            const df Wm = df_of(short_rule ? I.xw82[m] : I.xw2[m]);
            df x, E, y;
            if (full) {
                y = sT * q;
                x = uu + y;
                E = Wm;
            } else {
                const df z = q * v - hv2;
                df ez;
                if (short_rule) {
                    ez = one;
#pragma unroll
                    for (int j = 12; j >= 1; --j) ez = ez * z * df_of(c_inv2[j]) + one;
                } else {
                    ez = df_exp(z);
                }
                x = sT * q;
                E = Wm * ez;
                y = x - uu;
            }
            const df e1 = E * y, e2 = e1 * y, e3 = e2 * y;
            df hm = {0.0f, 0.0f}, h = df_of(I.x_h02);
            if (lb > 0) {
                hm = df_of(hst[(2 * m) * TILE + lane]);
                h = df_of(hst[(2 * m + 1) * TILE + lane]);
            }
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                if (j < nl) {
                    const int l = lb + j;
                    G[0][j] = E * h + G[0][j];
                    G[1][j] = e1 * h + G[1][j];
                    G[2][j] = e2 * h + G[2][j];
                    G[3][j] = e3 * h + G[3][j];
                    const df hn = ((x - df_of(I.xa2[l])) * h - df_of(I.xb2[l]) * hm) * df_of(I.xib2[l + 1]);
                    hm = h;
                    h = hn;
                }
            }
            if (lb + nl < Lx) {
                hst[(2 * m) * TILE + lane] = make_float2(hm.hi, hm.lo);
                hst[(2 * m + 1) * TILE + lane] = make_float2(h.hi, h.lo);
            }
        }
        if (lb > 0) __syncthreads();              // the previous block's readers of part and sum are done
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < QB; ++j)
                if (j < nl) part[((wid * 4 + a) * nl + j) * TILE + lane] = make_float2(G[a][j].hi, G[a][j].lo);
        __syncthreads();
        for (int r = wid; r < 4 * nl; r += NOD_WARPS) {
            df t = {0.0f, 0.0f};
            for (int q = 0; q < NOD_WARPS; ++q) t = t + df_of(part[(q * 4 * nl + r) * TILE + lane]);
            sum[r * TILE + lane] = make_float2(t.hi, t.lo);
        }
        __syncthreads();
        const bool last = lb + nl == Lx;
        for (int o = wid; o < 4 * Q; o += NOD_WARPS) {
            const int a = o / Q, k = o - a * Q;
            const size_t r = (size_t)(a * 2 * Q + role * Q + k) * ld + i;
            df t = (lb > 0 && valid) ? df_of(acc[r]) : df{0.0f, 0.0f};
            for (int j = 0; j < nl; ++j) t = df_of(I.xH2[(lb + j) * Q + k]) * df_of(sum[(a * nl + j) * TILE + lane]) + t;
            if (last && role && (a & 1)) t = -t;
            if (valid) {
                if (last) I.tab32[r] = df_float(t);
                else acc[r] = make_float2(t.hi, t.lo);
            }
        }
    }
}

// Arithmetic of the closure item's projections: FP64 for FP64 storage, double-float for FP32
// storage (whose tables are rounded to FP32).
__device__ __forceinline__ double r_of(double x, double) { return x; }
__device__ __forceinline__ df r_of(double x, df) { return df_of(x); }
__device__ __forceinline__ double r_tab(const double* d, const float2*, int k, double) { return d[k]; }
__device__ __forceinline__ df r_tab(const double*, const float2* p, int k, df) { return df_of(p[k]); }
__device__ __forceinline__ double r_dbl(double x) { return x; }
__device__ __forceinline__ double r_dbl(df x) { return (double)x.hi + (double)x.lo; }

// Output rows of the projection table in the closure's arithmetic type.
__device__ __forceinline__ double* r_out(const Inst& I, double) { return I.tab; }
__device__ __forceinline__ float* r_out(const Inst& I, df) { return I.tab32; }
__device__ __forceinline__ void r_put(double* p, size_t r, double v) { p[r] = v; }
__device__ __forceinline__ void r_put(float* p, size_t r, df v) { p[r] = df_float(v); }

// Role 2 of a tile: gradients (Sec. III B 3), closure (Eqs. chi, prandtl, viscosity, tau), the
// 13 coefficients of f^S + tau J1 = n g(xi) sum_j c_j xi^(a_j, b_j, c_j) (Eq. j1), the y and z
// projections (App. A) and the transverse factors n Y[a][t]; wall densities (Sec. III B).
// Phase A: warps 0..4 one gradient each, warp 5 sqrt T, warp 6 the wall densities, warp 7 the
// FP64 closure chain; warps 0..6 then run the projections (the recurrence at each auxiliary
// point, then the rows) while warp 7 is still busy.  Phase B: the coefficients; phase C:
// assembly.
template <typename R>
__device__ void closure_item(const Inst& I, int i0, double* nsm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = i0 + lane, N = I.N, ld = I.ld, Q = I.Q, Tc = I.Tc, Qy = I.Qy, Qz = I.Qz;
    const bool valid = i < N;
    const int ic = valid ? i : N - 1;           // padding lanes work on a real node, write nothing
    const double* nd = I.node;
    double* gr = nsm;                           // [5][32] d/dx of ln n, ln chi, ln T, u_x, u_y
    double* cs = gr + 5 * TILE;                 // [8][32] W = -tau b rho chi, A, 1/T, tau, -, n; sqrt T, u_y as R
    R* sc = reinterpret_cast<R*>(cs + 8 * TILE);        // [15][32] coefficients, n, 1/tau
    R* Py = sc + 15 * TILE;                             // [4 QYMAX][32]
    R* Pz = Py + 4 * QYMAX * TILE;                      // [3 QZMAX][32]
    R* Ay = Pz + 3 * QZMAX * TILE;                      // [8 QYMAX][32]
    R* hp = Ay + 8 * QYMAX * TILE;                      // [2 MYMAX][QYMAX][32] h_l at the auxiliary points
    R* yp = hp + 2 * MYMAX * QYMAX * TILE;              // [2 MYMAX][32] p - u0 at the auxiliary points
    // Fischer-Methfessel contact value (Eq. chi_ret): the averaged density n-bar and ln chi(n-bar)
    // on the tile and a halo of 7 nodes each side (what the gradient stencils reach)
    constexpr int FH = 7;
    __shared__ double fm_nbar[TILE + 2 * FH], fm_lnchi[TILE + 2 * FH];
    const bool fm = I.chi_model == FDLB_CHI_RET_FM;
    const int h0 = i0 - FH;
    if (fm) {
        for (int h = wid; h < TILE + 2 * FH; h += NOD_WARPS) {
            const int j = h0 + h;
            double v = 0.0;
            if (j >= 0 && j < N)
                for (int e = I.fm_ptr[j] + lane; e < I.fm_ptr[j + 1]; e += 32) v = fma(I.fm_w[e], nd[R_N * ld + I.fm_col[e]], v);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) fm_nbar[h] = v;
        }
        __syncthreads();
        if (threadIdx.x < TILE + 2 * FH) {
            const int j = h0 + threadIdx.x;
            fm_lnchi[threadIdx.x] = (j >= 0 && j < N) ? log(chi_cs(I.eta0 * fm_nbar[threadIdx.x])) : 0.0;
        }
        __syncthreads();
    }
    if (wid < 5) {
        const int row = wid == 0 ? R_LNN : (wid == 1 ? R_LNCHI : (wid == 2 ? R_LNT : (wid == 3 ? R_UX : R_UY)));
        const double cen[7] = {-1.0 / 60.0, 3.0 / 20.0, -0.75, 0.0, 0.75, -3.0 / 20.0, 1.0 / 60.0};
        double g = 0.0;
        for (int j = 0; j < 7; ++j) {
            int idx;
            double wj;
            if (ic < 3) { idx = j; wj = I.gst[ic * 7 + j]; }
            else if (ic > N - 4) { const int m = N - 1 - ic; idx = N - 1 - j; wj = -I.gst[m * 7 + j]; }
            else { idx = ic - 3 + j; wj = cen[j]; }
            g = fma(wj, (fm && wid == 1) ? fm_lnchi[idx - h0] : nd[row * ld + idx], g);
        }
        gr[wid * TILE + lane] = g * I.xpinv[ic];
    } else if (wid == 5) {
        // sqrt T and u_y in the projections' arithmetic, converted once
        R* cr = reinterpret_cast<R*>(cs + 6 * TILE);
        cr[lane] = r_of(sqrt(nd[R_T * ld + ic]), R{});
        cr[TILE + lane] = r_of(nd[R_UY * ld + ic], R{});
    } else if (wid == 6) {
        if (i0 == 0 && lane == 0) {
            // zero net mass flux through each wall (Sec. III B): the outgoing wall-face flux is
            // the quadratic reconstruction (11 f_1 - 7 f_2 + 2 f_3)/6 of outgoing populations.
            const double oL = (11.0 * nd[R_SNEG * ld + 0] - 7.0 * nd[R_SNEG * ld + 1] + 2.0 * nd[R_SNEG * ld + 2]) / 6.0;
            const double oR = (11.0 * nd[R_SPOS * ld + N - 1] - 7.0 * nd[R_SPOS * ld + N - 2] + 2.0 * nd[R_SPOS * ld + N - 3]) / 6.0;
            I.misc[M_NWL] = -oL / I.misc[M_INL];
            I.misc[M_NWR] = -oR / I.misc[M_INR];
        }
    } else {
        const double k_mu = (4.0 / 25.0) * (1.0 + 12.0 / CUDART_PI);
        const double k_pd = (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * CUDART_PI));
        const double n = nd[R_N * ld + ic], T = nd[R_T * ld + ic];
        const double eta = I.eta0 * n, chi = chi_cs(fm ? I.eta0 * fm_nbar[ic - h0] : eta), br = 4.0 * eta, brc = br * chi;
        const double Pr = (2.0 / 3.0) * (1.0 + 0.8 * brc + k_mu * brc * brc) / (1.0 + 1.2 * brc + k_pd * brc * brc);
        const double iT = 1.0 / T, in = 1.0 / n;
        // tau = mu/(n T) = mu0c X sqrt T / (T n), W = -tau b rho chi
        const double tau = I.mu0c * (1.0 / chi + 0.8 * br + k_mu * br * br * chi) * iT * in * sqrt(T);
        cs[0 * TILE + lane] = -tau * brc;
        cs[1 * TILE + lane] = (1.0 - Pr) * 0.2 * iT * iT * in;
        cs[2 * TILE + lane] = iT;
        cs[3 * TILE + lane] = tau;
        cs[5 * TILE + lane] = n;
    }
    // warps 0..6 go on to the projections (they need sqrt T and u_y only) while warp 7 still
    // runs the closure chain; named barrier 1 synchronises the 7 warps
    if (wid < NOD_WARPS - 1) {
        const R z = r_of(0.0, R{});
        named_sync(1, (NOD_WARPS - 1) * TILE);
        // full-range projections, step 1: the orthonormal recurrence h_l at each auxiliary point
        // (y points first, then z points), one point per warp of warps 0..6
        if (I.form != FORM_REDUCED1D) {
            const int My = I.My, Mz = I.form == FORM_UNREDUCED ? I.Mz : 0;
            const R* cr = reinterpret_cast<const R*>(cs + 6 * TILE);
            const R sT = cr[lane], uy = cr[TILE + lane], one = r_of(1.0, z);
            for (int pt = wid; pt < My + Mz; pt += NOD_WARPS - 1) {
                const bool ydir = pt < My;
                const int m = ydir ? pt : pt - My, Qn = ydir ? Qy : Qz;
                const R y = sT * (ydir ? r_tab(I.yq, I.yq2, m, z) : r_tab(I.zq, I.zq2, m, z));
                const R x = ydir ? uy + y : y;
                yp[pt * TILE + lane] = y;
                R hm = z, h = one;
#pragma unroll
                for (int l = 0; l < QYMAX; ++l) {
                    if (l < Qn) {
                        hp[(pt * QYMAX + l) * TILE + lane] = h;
                        const R hn = (x * h - r_tab(I.fsq, I.fsq2, l, z) * hm) * r_tab(I.fisq, I.fisq2, l + 1, z);
                        hm = h;
                        h = hn;
                    }
                }
            }
        }
        named_sync(1, (NOD_WARPS - 1) * TILE);
        if (I.form != FORM_REDUCED1D && (wid < 4 || I.form == FORM_UNREDUCED)) {
            // step 2: warps 0..3 rows a = wid of Py ((p_y - u_y)^a g), warps 4..6 rows a = wid - 4 of
            // Pz (p_z^a g): sum over the auxiliary points of w y^a h_l, then the H matrix (App. A)
            const bool ydir = wid < 4;
            const int a = ydir ? wid : wid - 4, Qn = ydir ? Qy : Qz, M = ydir ? I.My : I.Mz, p0 = ydir ? 0 : I.My;
            const double* aw = ydir ? I.yw : I.zw;
            const float2* aw2 = ydir ? I.yw2 : I.zw2;
            R G[QYMAX];
#pragma unroll
            for (int l = 0; l < QYMAX; ++l) G[l] = z;
            for (int m = 0; m < M; ++m) {
                const R y = yp[(p0 + m) * TILE + lane];
                R e = r_tab(aw, aw2, m, z);
                for (int j = 0; j < a; ++j) e = e * y;
#pragma unroll
                for (int l = 0; l < QYMAX; ++l)
                    if (l < Qn) G[l] = e * hp[((p0 + m) * QYMAX + l) * TILE + lane] + G[l];
            }
            const double* H = ydir ? I.yH : I.zH;
            const float2* H2 = ydir ? I.yH2 : I.zH2;
            R* P = ydir ? Py + a * QYMAX * TILE : Pz + a * QZMAX * TILE;
            for (int k2 = 0; k2 < Qn; ++k2) {
                R t = z;
#pragma unroll
                for (int l = 0; l < QYMAX; ++l)
                    if (l < Qn) t = r_tab(H, H2, l * Qn + k2, z) * G[l] + t;
                P[k2 * TILE + lane] = t;
            }
        }
    }
    __syncthreads();
    {
        // coefficients: warp w computes a few, reading only what they need
        const R z = r_of(0.0, R{});
        const double* W = cs + 0 * TILE;
        const double* A = cs + 1 * TILE;
        const double* iT = cs + 2 * TILE;
        switch (wid) {
            case 0:
                sc[0 * TILE + lane] = r_of(1.0 - W[lane] * gr[3 * TILE + lane], z);
                sc[13 * TILE + lane] = r_of(cs[5 * TILE + lane], z);
                break;
            case 1: {
                const double Gr = 2.0 * gr[0 * TILE + lane] + gr[1 * TILE + lane] + gr[2 * TILE + lane];
                sc[1 * TILE + lane] = r_of(-5.0 * A[lane] * nd[R_QX * ld + ic] + W[lane] * (Gr - 1.5 * gr[2 * TILE + lane]), z);
                break;
            }
            case 2:
                sc[2 * TILE + lane] = r_of(-5.0 * A[lane] * nd[R_QY * ld + ic], z);
                sc[6 * TILE + lane] = I.j1_shear ? r_of(W[lane] * 0.4 * gr[4 * TILE + lane] * iT[lane], z) : z;
                break;
            case 3: {
                const double u = W[lane] * gr[3 * TILE + lane] * iT[lane];
                sc[3 * TILE + lane] = r_of(0.6 * u, z);
                sc[4 * TILE + lane] = r_of(0.2 * u, z);
                sc[5 * TILE + lane] = sc[4 * TILE + lane];
                break;
            }
            case 4: {
                const R c3 = r_of(A[lane] * nd[R_QX * ld + ic] * iT[lane] + W[lane] * 0.3 * gr[2 * TILE + lane] * iT[lane], z);
                sc[7 * TILE + lane] = c3;
                sc[8 * TILE + lane] = c3;
                sc[9 * TILE + lane] = c3;
                break;
            }
            case 5: {
                const R cy = r_of(A[lane] * nd[R_QY * ld + ic] * iT[lane], z);
                sc[10 * TILE + lane] = cy;
                sc[11 * TILE + lane] = cy;
                sc[12 * TILE + lane] = cy;
                break;
            }
            case 6: sc[14 * TILE + lane] = r_of(1.0 / cs[3 * TILE + lane], z); break;
            default: break;
        }
    }
    __syncthreads();
    auto* out = r_out(I, R{});
    const int form = I.form;
    if (form != FORM_REDUCED1D) {
        // A[a][c'][ky] = n sum over the monomials (a, b, c = 2 c') of coef * Py[b][ky]; with the
        // monomial order of c_mono: (0,0,0) (1,0,0) (0,1,0) (2,0,0) (0,2,0) (0,0,2) (1,1,0)
        // (3,0,0) (1,2,0) (1,0,2) (2,1,0) (0,3,0) (0,1,2)
        for (int ky = wid; ky < Qy; ky += NOD_WARPS) {
            R c[NTERMS];
#pragma unroll
            for (int j = 0; j < NTERMS; ++j) c[j] = sc[j * TILE + lane];
            const R n = sc[13 * TILE + lane];
            const R P0 = Py[(0 * QYMAX + ky) * TILE + lane], P1 = Py[(1 * QYMAX + ky) * TILE + lane];
            const R P2 = Py[(2 * QYMAX + ky) * TILE + lane], P3 = Py[(3 * QYMAX + ky) * TILE + lane];
            const R zero = r_of(0.0, R{});
            Ay[(0 * Qy + ky) * TILE + lane] = n * (c[0] * P0 + c[2] * P1 + c[4] * P2 + c[11] * P3);   // a = 0, c' = 0
            Ay[(1 * Qy + ky) * TILE + lane] = n * (c[5] * P0 + c[12] * P1);                          // a = 0, c' = 1
            Ay[(2 * Qy + ky) * TILE + lane] = n * (c[1] * P0 + c[6] * P1 + c[8] * P2);               // a = 1, c' = 0
            Ay[(3 * Qy + ky) * TILE + lane] = n * (c[9] * P0);                                       // a = 1, c' = 1
            Ay[(4 * Qy + ky) * TILE + lane] = n * (c[3] * P0 + c[10] * P1);                          // a = 2, c' = 0
            Ay[(5 * Qy + ky) * TILE + lane] = zero;                                                  // a = 2, c' = 1
            Ay[(6 * Qy + ky) * TILE + lane] = n * (c[7] * P0);                                       // a = 3, c' = 0
            Ay[(7 * Qy + ky) * TILE + lane] = zero;                                                  // a = 3, c' = 1
        }
        __syncthreads();
        // transverse factors n Y[a][t] = A[a][0][ky] Z0(t) + A[a][1][ky] Z2(t), t = ky Tz + kz;
        // a warp takes (a, ky) pairs and runs over kz (no per-output index divisions)
        const double T = nd[R_T * ld + ic];
        const R Tr = r_of(T, R{}), one = r_of(1.0, R{}), T23 = r_of(3.0 * T * T, R{});
        const bool unred = form == FORM_UNREDUCED;
        const int Tz = unred ? Qz : 2;
        for (int pr = wid; pr < 4 * Qy; pr += NOD_WARPS) {
            const int a = pr / Qy, ky = pr - a * Qy;
            const R A0 = Ay[((2 * a) * Qy + ky) * TILE + lane], A1 = Ay[((2 * a + 1) * Qy + ky) * TILE + lane];
            auto* row = out + (size_t)(8 * Q + a * Tc + ky * Tz) * ld + i;
            if (unred) {
                for (int kz = 0; kz < Qz; ++kz) {
                    const R v = A0 * Pz[(0 * QZMAX + kz) * TILE + lane] + A1 * Pz[(2 * QZMAX + kz) * TILE + lane];
                    if (valid) r_put(row, (size_t)kz * ld, v);
                }
            } else {
                const R v0 = A0 * one + A1 * Tr, v1 = A0 * Tr + A1 * T23;
                if (valid) {
                    r_put(row, 0, v0);
                    r_put(row, (size_t)ld, v1);
                }
            }
        }
    } else {
        // 1D reduced (Sec. II B 1): slots phi, theta carry the (p_y, p_z) Gaussian moments
        const int a = wid >> 1, slot = wid & 1;
        const double T = nd[R_T * ld + ic];
        double t = 0.0;
        for (int j = 0; j < NTERMS; ++j) {
            if (c_mono[j][0] != a) continue;
            const int b = c_mono[j][1], cc = c_mono[j][2];
            const double e = slot == 0 ? gmom(b, T) * gmom(cc, T) : gmom(b + 2, T) * gmom(cc, T) + gmom(b, T) * gmom(cc + 2, T);
            t = fma(r_dbl(sc[j * TILE + lane]), e, t);
        }
        if (valid) r_put(out, (size_t)(8 * Q + a * Tc + slot) * ld + i, r_of(r_dbl(sc[13 * TILE + lane]) * t, R{}));
    }
    if (wid == 0 && valid) r_put(out, (size_t)(8 * Q + 4 * Tc) * ld + i, sc[14 * TILE + lane]);
}

// One (tile, role) item by a block of NOD_WARPS warps; nsm holds nodal_smem_doubles(QB)
// doubles; fp32: the instance stores f in FP32 (tables go to tab32).
template <int QB>
__device__ void nodal_item(const Inst& I, int i0, int role, double* nsm, bool fp32) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = i0 + lane;
    __syncthreads();                      // the previous item's readers of nsm are done
    // FP32 storage: the half-range x projection in double-float, up to 32 polynomials.  Larger
    // orders keep the FP64 projection below (writing the FP32 table): the orthonormal
    // polynomials grow to ~e^(x^2/4) at the auxiliary points x = sqrt(T) q, beyond the float
    // range (3e38) once x > ~18.8 -- the full-range rule of order 200 has |q| up to ~19, the
    // half-range aux rule of order 100 q up to ~17 (overflow from T ~ 1.2); at 32 polynomials
    // the aux rule ends near q = 11, which would need T > 3.
    if (fp32 && role < 2 && !I.xfull && I.Lx <= 32) {
        xproj_df<QB>(I, i0, role, nsm);
        return;
    }
    const int N = I.N, ld = I.ld, Q = I.Q, Tc = I.Tc;
    const bool valid = i < N;
    const int ic = valid ? i : N - 1;           // padding lanes work on a real node, write nothing
    const double* nd = I.node;
    if (role < 2) {
        // ---- half-range x projection (Sec. III A 2), half-axis `role`.  With |v| < 0.02 and
        // Q <= 12 the 8-point auxiliary rule is used (exact for v = 0 up to degree 15 >= Q + 2;
        // the neglected part of exp(q v) is below 1e-14 relative) with exp(q v - v^2/2) from its
        // Taylor series (|argument| < 0.12, 12 terms).  Warp w takes auxiliary points w, w + 8.
        // sqrt T, u and v = u / sqrt T once per node (warp 0), shared; one rule per block so that
        // the warps agree: the largest |v| of the tile decides
        __shared__ double xs[3][TILE];
        __shared__ int use_short;
        if (wid == 0) {
            const double T = nd[R_T * ld + ic], ux = nd[R_UX * ld + ic];
            const double sT0 = sqrt(T), uu0 = role ? -ux : ux, v0 = uu0 / sT0;
            xs[0][lane] = sT0;
            xs[1][lane] = uu0;
            xs[2][lane] = v0;
            double av = valid ? fabs(v0) : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) av = fmax(av, __shfl_xor_sync(0xffffffffu, av, o));
            if (lane == 0) use_short = av < 0.02 ? 1 : 2;
        }
        __syncthreads();
        const double sT = xs[0][lane], uu = xs[1][lane], v = xs[2][lane];
        // full-range x (App. A): Lx = 2Q polynomials, x = u + sqrt(T) q on the exact Mx-point
        // Gauss-Hermite rule, no exponential (the Maxwellian is the rule's weight)
        const bool full = I.xfull;
        const int Lx = I.Lx;
        const bool short_rule = !full && use_short == 1 && Q <= 12;
        const int M = full ? I.Mx : (short_rule ? MX8 : I.Mx);
        double* part = nsm;                                  // [NOD_WARPS][4 nl][32]
        double* hst = nsm + (NOD_WARPS + 1) * 4 * QB * TILE; // [M][2][32] recurrence state (Lx > QB)
        // the polynomials in blocks of QB: per block the sums over the auxiliary points (the
        // recurrence continued from the previous block's state), then the H products, whose
        // chain continues across blocks in the instance's FP64 table rows (signed and written at
        // the last block)
        for (int lb = 0; lb < Lx; lb += QB) {
            const int nl = min(QB, Lx - lb);
            double* sum = nsm + NOD_WARPS * 4 * nl * TILE;   // [4 nl][32]
            double G[4][QB];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int l = 0; l < QB; ++l) G[a][l] = 0.0;
            for (int m = wid; m < M; m += NOD_WARPS) {
                const double q = short_rule ? I.xq8[m] : I.xq[m];
                const double Wm = short_rule ? I.xw8[m] : I.xw[m];
                double x, E, y;
                if (full) {
                    y = sT * q;
                    x = uu + y;
                    E = Wm;
                } else {
                    const double z = fma(q, v, -0.5 * v * v);
                    double ez;
                    if (short_rule) {
                        ez = 1.0;
#pragma unroll
                        for (int j = 12; j >= 1; --j) ez = fma(ez * z, c_inv[j], 1.0);
                    } else {
                        ez = exp(z);
                    }
                    x = sT * q;
                    E = Wm * ez;
                    y = x - uu;
                }
                const double e1 = E * y, e2 = e1 * y, e3 = e2 * y;
                // recurrence state at the block's first polynomial: from the start, or as the
                // previous block left it (this thread stored it)
                double hm = 0.0, h = I.x_h0;
                if (lb > 0) {
                    hm = hst[(2 * m) * TILE + lane];
                    h = hst[(2 * m + 1) * TILE + lane];
                }
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    if (j < nl) {
                        const int l = lb + j;
                        G[0][j] = fma(E, h, G[0][j]);
                        G[1][j] = fma(e1, h, G[1][j]);
                        G[2][j] = fma(e2, h, G[2][j]);
                        G[3][j] = fma(e3, h, G[3][j]);
                        const double hn = ((x - I.xa[l]) * h - I.xb[l] * hm) * I.xib[l + 1];
                        hm = h;
                        h = hn;
                    }
                }
                if (lb + nl < Lx) {
                    hst[(2 * m) * TILE + lane] = hm;
                    hst[(2 * m + 1) * TILE + lane] = h;
                }
            }
            if (lb > 0) __syncthreads();          // the previous block's readers of part and sum are done
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int j = 0; j < QB; ++j)
                    if (j < nl) part[((wid * 4 + a) * nl + j) * TILE + lane] = G[a][j];
            __syncthreads();
            for (int r = wid; r < 4 * nl; r += NOD_WARPS) {
                double s = 0.0;
                for (int q = 0; q < NOD_WARPS; ++q) s += part[(q * 4 * nl + r) * TILE + lane];
                sum[r * TILE + lane] = s;
            }
            __syncthreads();
            const bool last = lb + nl == Lx;
            for (int o = wid; o < 4 * Q; o += NOD_WARPS) {
                const int a = o / Q, k = o - a * Q;
                const size_t r = (size_t)(a * 2 * Q + role * Q + k) * ld + i;
                double s = (lb > 0 && valid) ? I.tab[r] : 0.0;
                for (int j = 0; j < nl; ++j) s = fma(I.xH[(lb + j) * Q + k], sum[(a * nl + j) * TILE + lane], s);
                if (last && role && (a & 1)) s = -s;
                if (valid) {
                    if (last && fp32) I.tab32[r] = (float)s;
                    else I.tab[r] = s;
                }
            }
        }
        return;
    }
    if (fp32) closure_item<df>(I, i0, nsm);
    else closure_item<double>(I, i0, nsm);
}

template <int QB>
__global__ void __launch_bounds__(TILE * NOD_WARPS) k_nodal(const Inst* __restrict__ insts, const Work* __restrict__ work) {
    extern __shared__ __align__(16) double nsm[];
    pdl_wait();
    const Work w = work[blockIdx.x];
    const Inst& I = insts[w.inst];
    if (*I.status != FDLB_ACTIVE || I.smem_res) return;
    nodal_item<QB>(I, w.i0, w.k0, nsm, I.precision == FDLB_FP32_STORAGE);
}

// ---------------------------------------------------------------------------
// per-step residual and status
// ---------------------------------------------------------------------------
// Stagnation of a two-phase instance in its FP32 phase (window rule of FDLB_FP32_THEN_FP64).
__device__ int stagnated(Inst& I, double r, double step) {
    if (r == 0.0) return 1;
    double* m = I.misc;
    if (m[M_WIN_STEP] < 0.0) {
        m[M_WIN_STEP] = step;
        m[M_WIN_RESID] = r;
        return 0;
    }
    if (step - m[M_WIN_STEP] < FDLB_STAGNATION_WINDOW) return 0;
    if (!(r < FDLB_STAGNATION_FACTOR * m[M_WIN_RESID])) return 1;
    m[M_WIN_STEP] = step;
    m[M_WIN_RESID] = r;
    return 0;
}

// Residual, status and (two-phase) precision switch of instance I (batch index idx) after a
// step, by a block of 256 threads.
__device__ void resid_item(Inst& I, int idx, double tol, double* resid_all) {
    const int ld = I.ld, N = I.N;
    double* nd = I.node;
    constexpr int RT = 256;                   // threads of the calling block
    __shared__ double red[7][RT];
    __shared__ double tot[7], term[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    int bad_nf = 0, bad_ph = 0;
    for (int i = threadIdx.x; i < N; i += RT) {
        const double n = nd[R_N * ld + i], ux = nd[R_UX * ld + i], uy = nd[R_UY * ld + i], T = nd[R_T * ld + i];
        if (!isfinite(n) || !isfinite(ux) || !isfinite(uy) || !isfinite(T)) bad_nf = 1;
        else if (!(n > 0.0) || !(T > 0.0)) bad_ph = 1;
        const double w = I.dxw[i];
        const double dn = n - nd[R_PREV_N * ld + i], dT = T - nd[R_PREV_T * ld + i];
        const double dux = ux - nd[R_PREV_UX * ld + i], duy = uy - nd[R_PREV_UY * ld + i];
        s[0] += w * dn * dn;
        s[1] += w * n * n;
        s[2] += w * dT * dT;
        s[3] += w * T * T;
        s[4] += w * dux * dux;
        s[5] += w * duy * duy;
        s[6] += w * n;
        nd[R_PREV_N * ld + i] = n;
        nd[R_PREV_UX * ld + i] = ux;
        nd[R_PREV_UY * ld + i] = uy;
        nd[R_PREV_T * ld + i] = T;
    }
    __shared__ int flags[3];
    __shared__ double scale;
    if (threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; flags[2] = 0; }
#pragma unroll
    for (int j = 0; j < 7; ++j) red[j][threadIdx.x] = s[j];
    __syncthreads();
    if (bad_nf) atomicOr(&flags[0], 1);
    if (bad_ph) atomicOr(&flags[1], 1);
    // sum j over the block by warp j (independent FP64 chains on different schedulers)
    if (wid < 7) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < RT / 32; ++q) v += red[wid][q * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) tot[wid] = v;
    }
    __syncthreads();
    // the four terms of the residual on four warps
    if (lane == 0 && wid < 4)
        term[wid] = wid == 0 ? sqrt(tot[0] / tot[1]) : (wid == 1 ? sqrt(tot[2] / tot[3]) : sqrt(tot[wid + 2]));
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = fmax(fmax(term[0], term[1]), fmax(term[2], term[3]));
        *I.steps += 1;
        I.misc[M_RESID] = r;
        resid_all[idx] = r;
        const bool fp32 = I.precision == FDLB_FP32_STORAGE;
        if (flags[0]) *I.status = FDLB_FAILED_NONFINITE;
        else if (flags[1]) *I.status = FDLB_FAILED_UNPHYSICAL;
        else if (fp32 && r == 0.0 && I.two_phase) flags[2] = 1;   // FP32 f stopped changing
        else if (fp32 && r == 0.0 && tol > 0.0) *I.status = FDLB_STAGNATED;
        else if (tol > 0.0 && r < tol) *I.status = FDLB_CONVERGED;
        else if (I.two_phase && fp32) flags[2] = stagnated(I, r, (double)*I.steps);
        scale = I.misc[M_MASS0] / tot[6];
    }
    __syncthreads();
    if (!flags[2]) return;
    // Up-cast f: floats of F -> doubles in the stage buffer A, then back into F (which holds
    // K ld doubles in a two-phase instance; A is free between steps), times the factor that
    // restores the channel mass of the last anchor.  The discrete scheme conserves mass, but
    // FP32 rounding near stagnation drops the same small updates step after step and lets the
    // mass drift, which would move the FP64 steady state.  The node rows are rescaled alike
    // (extensive rows by the factor, ln n and ln chi(eta0 n) anew; u and T are unchanged),
    // so the next stage sees the moments of the rescaled f.
    const double c = scale;
    const size_t nf = (size_t)I.K * ld;
    const float* src = static_cast<const float*>(I.f[0]);
    double* tmp = static_cast<double*>(I.f[1]);
    for (size_t e = threadIdx.x; e < nf; e += blockDim.x) tmp[e] = (double)src[e] * c;
    __syncthreads();
    double* dst = static_cast<double*>(I.f[0]);
    for (size_t e = threadIdx.x; e < nf; e += blockDim.x) dst[e] = tmp[e];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double n = nd[R_N * ld + i] * c;
        nd[R_N * ld + i] = n;
        nd[R_PREV_N * ld + i] *= c;
        nd[R_QX * ld + i] *= c;
        nd[R_QY * ld + i] *= c;
        nd[R_PXX * ld + i] *= c;
        nd[R_PXY * ld + i] *= c;
        nd[R_SNEG * ld + i] *= c;
        nd[R_SPOS * ld + i] *= c;
        nd[R_LNN * ld + i] = log(n);
        nd[R_LNCHI * ld + i] = log(chi_cs(I.eta0 * n));
    }
    if (threadIdx.x == 0) {
        I.precision = FDLB_FP64;
        I.misc[M_SWITCH] = (double)*I.steps;
    }
}


__global__ void __launch_bounds__(256) k_resid(Inst* insts, int anchor, double tol, double* resid_all) {
    pdl_wait();
    Inst& I = insts[blockIdx.x];
    const int ld = I.ld, N = I.N;
    double* nd = I.node;
    __shared__ double red[7][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (anchor >= -1) {
        if (anchor >= 0 && anchor != (int)blockIdx.x) return;
        double m = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            nd[R_PREV_N * ld + i] = nd[R_N * ld + i];
            nd[R_PREV_UX * ld + i] = nd[R_UX * ld + i];
            nd[R_PREV_UY * ld + i] = nd[R_UY * ld + i];
            nd[R_PREV_T * ld + i] = nd[R_T * ld + i];
            m = fma(I.dxw[i], nd[R_N * ld + i], m);
        }
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0) red[0][wid] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[0][q];
            I.misc[M_MASS0] = t;
            I.misc[M_RESID] = CUDART_INF;
            I.misc[M_WIN_STEP] = -1.0;
            resid_all[blockIdx.x] = CUDART_INF;
        }
        return;
    }
    if (*I.status != FDLB_ACTIVE || I.smem_res) return;
    resid_item(I, blockIdx.x, tol, resid_all);
}

// ---------------------------------------------------------------------------
// update: WENO-5 advection + walls + force + relaxation + RK3 combination
// ---------------------------------------------------------------------------

// Upwind-biased WENO-5 face value from (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}) taken in the
// upwind direction (Sec. III B 2).  Weights delta_q/phi_q^2 without epsilon; a vanishing
// indicator takes the weight in the limit (the normalised weights are continuous there).
__device__ __forceinline__ double weno_face(double a, double b, double c, double d, double e) {
    const double F1 = fma(1.0 / 3.0, a, fma(-7.0 / 6.0, b, 11.0 / 6.0 * c));
    const double F2 = fma(-1.0 / 6.0, b, fma(5.0 / 6.0, c, 1.0 / 3.0 * d));
    const double F3 = fma(1.0 / 3.0, c, fma(5.0 / 6.0, d, -1.0 / 6.0 * e));
    const double t1 = a - 2.0 * b + c, t2 = a - 4.0 * b + 3.0 * c;
    const double u1 = b - 2.0 * c + d, u2 = b - d;
    const double v1 = c - 2.0 * d + e, v2 = 3.0 * c - 4.0 * d + e;
    const double s1 = fma(13.0 / 12.0, t1 * t1, 0.25 * t2 * t2);
    const double s2 = fma(13.0 / 12.0, u1 * u1, 0.25 * u2 * u2);
    const double s3 = fma(13.0 / 12.0, v1 * v1, 0.25 * v2 * v2);
    const double smax = fmax(s1, fmax(s2, s3));
    double w1, w2, w3;
    if (smax == 0.0) {
        w1 = 0.1; w2 = 0.6; w3 = 0.3;
    } else {
        // omega_q ~ delta_q / phi_q^2 ~ delta_q prod_{r != q} phi_r^2 (phi scaled by the max)
        const double r = 1.0 / smax;
        const double a1 = s1 * r, a2 = s2 * r, a3 = s3 * r;
        const double p1 = a1 * a1, p2 = a2 * a2, p3 = a3 * a3;
        w1 = 0.1 * p2 * p3;
        w2 = 0.6 * p1 * p3;
        w3 = 0.3 * p1 * p2;
        double sum = w1 + w2 + w3;
        if (sum == 0.0) {
            // two indicators vanish (or underflow): weight on the smallest ones
            const double smin = fmin(s1, fmin(s2, s3));
            w1 = s1 == smin ? 0.1 : 0.0;
            w2 = s2 == smin ? 0.6 : 0.0;
            w3 = s3 == smin ? 0.3 : 0.0;
            sum = w1 + w2 + w3;
        }
        const double is = 1.0 / sum;
        w1 *= is; w2 *= is; w3 *= is;
    }
    return fma(w1, F1, fma(w2, F2, w3 * F3));
}

__device__ __forceinline__ float weno_face(float a, float b, float c, float d, float e) {
    const float F1 = fmaf(1.0f / 3.0f, a, fmaf(-7.0f / 6.0f, b, 11.0f / 6.0f * c));
    const float F2 = fmaf(-1.0f / 6.0f, b, fmaf(5.0f / 6.0f, c, 1.0f / 3.0f * d));
    const float F3 = fmaf(1.0f / 3.0f, c, fmaf(5.0f / 6.0f, d, -1.0f / 6.0f * e));
    const float t1 = a - 2.0f * b + c, t2 = a - 4.0f * b + 3.0f * c;
    const float u1 = b - 2.0f * c + d, u2 = b - d;
    const float v1 = c - 2.0f * d + e, v2 = 3.0f * c - 4.0f * d + e;
    const float s1 = fmaf(13.0f / 12.0f, t1 * t1, 0.25f * t2 * t2);
    const float s2 = fmaf(13.0f / 12.0f, u1 * u1, 0.25f * u2 * u2);
    const float s3 = fmaf(13.0f / 12.0f, v1 * v1, 0.25f * v2 * v2);
    const float smax = fmaxf(s1, fmaxf(s2, s3));
    float w1, w2, w3;
    if (smax < 1e-30f) {
        // uniform to FP32 resolution (indicators zero or below any meaningful difference): the
        // candidates agree, the ideal weights are the limit
        w1 = 0.1f; w2 = 0.6f; w3 = 0.3f;
    } else {
        // omega_q ~ delta_q / phi_q^2 ~ delta_q prod_{r != q} phi_r^2, phi scaled by the largest
        // (one reciprocal; fast division: the FP32 form's tolerance is far above its error)
        const float r = __fdividef(1.0f, smax);
        const float a1 = s1 * r, a2 = s2 * r, a3 = s3 * r;
        const float p1 = a1 * a1, p2 = a2 * a2, p3 = a3 * a3;
        w1 = 0.1f * p2 * p3;
        w2 = 0.6f * p1 * p3;
        w3 = 0.3f * p1 * p2;
        if (w1 + w2 + w3 < 1e-30f) {
            // two indicators vanish relative to the third (or underflow): weight on the smallest
            const float smin = fminf(s1, fminf(s2, s3));
            w1 = s1 == smin ? 0.1f : 0.0f;
            w2 = s2 == smin ? 0.6f : 0.0f;
            w3 = s3 == smin ? 0.3f : 0.0f;
        }
    }
    const float is = __fdividef(1.0f, w1 + w2 + w3);
    return fmaf(w1 * is, F1, fmaf(w2 * is, F2, w3 * is * F3));
}

constexpr int UPD_WARPS = 8;          // warps of an update block; the moment epilogue's partials
constexpr int UPD_WARPS_WIDE = 16;    // wide update blocks: the velocity loop on 16 warps

// ---------------------------------------------------------------------------
// stochastic rounding of FP32 storage
// ---------------------------------------------------------------------------
// With round-to-nearest, FP32 storage drops every per-step change below half an ulp of f, so a
// solve stalls at a distance ~ ulp / (2 eps) from the steady state (eps = decay per step of its
// slowest mode; ~5e-5 on the Couette sweep), and the dropped changes no longer sum to zero
// over the channel, which drifts the mass.  Rounding base + inc up or down at random, with the
// probabilities that make the expected stored value the exact sum (Connolly, Higham & Mary,
// SIAM J. Sci. Comput. 43, 2021), keeps small changes in expectation: no stall, and a mass
// error that only random-walks.  The random bits come from a counter-based hash of (the
// instance's parameters, step, stage, velocity, node), so runs are reproducible, both schedules
// round alike, and an instance rounds the same way whatever batch it is in.

// MurmurHash3's 32-bit finalizer (Appleby, public domain): a bijective avalanche mix.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Per-launch seed of instance I for RK stage `stage` of the current step.
__device__ __forceinline__ uint32_t sr_seed(const Inst& I, int stage) {
    const unsigned long long step = (unsigned long long)*(volatile long long*)I.steps;
    return fmix32((uint32_t)(step * 3ull + (unsigned long long)stage) ^ fmix32(I.sr_key));
}

// base + inc stored as a float: the exact sum s + err (TwoSum) goes to its round-to-nearest
// value s, or to the neighbouring float on the side of err with probability |err| / gap, so
// that its expectation is the exact sum.
__device__ __forceinline__ float sr_add(float base, float inc, uint32_t bits) {
    const float s = __fadd_rn(base, inc);
    const float bb = __fsub_rn(s, base);
    const float err = __fadd_rn(__fsub_rn(base, __fsub_rn(s, bb)), __fsub_rn(inc, bb));
    if (err == 0.0f) return s;
    // the neighbouring float on the side of err: one unit in the last place of s's magnitude
    // bits, up when s and err have the same sign, down otherwise (s = 0: the smallest
    // subnormal with err's sign)
    const uint32_t sb = __float_as_uint(s);
    const float nb = s == 0.0f ? copysignf(__uint_as_float(1u), err)
                               : __uint_as_float((s > 0.0f) == (err > 0.0f) ? sb + 1u : sb - 1u);
    const float gap = fabsf(__fsub_rn(nb, s));
    const float u = __uint2float_rz(bits >> 8) * 0x1p-24f;        // uniform on [0, 1), exact
    return __fmul_rn(u, gap) < fabsf(err) ? nb : s;
}

// Tables read by the update kernel in its compute type (FP32 copies for FP32 storage).
template <typename C>
struct Tabs;
template <>
struct Tabs<double> {
    __device__ static const double* tab(const Inst& I) { return I.tab; }
    __device__ static const double* px(const Inst& I) { return I.px; }
    __device__ static const double* gL(const Inst& I) { return I.gL; }
    __device__ static const double* gR(const Inst& I) { return I.gR; }
    __device__ static const double* xpinv(const Inst& I) { return I.xpinv; }
    __device__ static const double* Ky(const Inst& I) { return I.Ky; }
};
template <>
struct Tabs<float> {
    __device__ static const float* tab(const Inst& I) { return I.tab32; }
    __device__ static const float* px(const Inst& I) { return I.px32; }
    __device__ static const float* gL(const Inst& I) { return I.gL32; }
    __device__ static const float* gR(const Inst& I) { return I.gR32; }
    __device__ static const float* xpinv(const Inst& I) { return I.xpinv32; }
    __device__ static const float* Ky(const Inst& I) { return I.Ky32; }
};

// Shared memory of one update item: the projection table, the transverse moment weights, the
// staged source rows of the chunk (each with a 4-node halo on either side: 40 values per row;
// the epilogue's per-warp sums reuse this space once the rows are consumed), and the step's F
// values, which the outputs replace (the epilogue reads them there).
constexpr size_t TW_BYTES = (size_t)NTW * TCMAX * sizeof(double);
constexpr int SW = 40;                // staged row: nodes i0 - 4 .. i0 + 35
__host__ __device__ inline size_t upd_table_bytes(int ntab, size_t c) { return ((size_t)ntab * TILE * c + 15) / 16 * 16; }
__host__ __device__ inline size_t upd_ex_bytes() { return (size_t)(UPD_WARPS + 1) * MOM_SUMS * TILE * sizeof(double); }
__host__ __device__ inline size_t upd_stage_bytes(int ukc, size_t s) {
    const size_t rows = (size_t)ukc * SW * s, ex = upd_ex_bytes();
    return ((rows > ex ? rows : ex) + 15) / 16 * 16;
}
__host__ __device__ inline size_t upd_stage_offset(int ntab, size_t c) { return upd_table_bytes(ntab, c) + TW_BYTES; }
__host__ __device__ inline size_t upd_fo_offset(int ntab, int ukc, size_t c, size_t s) {
    return upd_stage_offset(ntab, c) + upd_stage_bytes(ukc, s);
}
__host__ __device__ inline size_t upd_smem_bytes(int ntab, int ukc, size_t c, size_t s) {
    return upd_fo_offset(ntab, ukc, c, s) + (size_t)ukc * TILE * s;
}

// Transverse moment weights of the epilogue into shared memory (FP32 storage: float heads
// and tails, FP64: doubles), by the whole block.
template <typename S>
__device__ __forceinline__ void load_tw(const Inst& I, void* tws, int tid, int nthreads) {
    const int n = NTW * I.Tc;
    if constexpr (sizeof(S) == 4) {
        float* h = static_cast<float*>(tws);
        for (int e = tid; e < n; e += nthreads) {
            h[e] = I.twh[e];
            h[n + e] = I.twl[e];
        }
    } else {
        double* d = static_cast<double*>(tws);
        for (int e = tid; e < n; e += nthreads) d[e] = I.tw[e];
    }
}

// Epilogue of an update item: raw moment sums of the chunk's values fo[k - k0][lane] with the
// factorisation of the moments (per x-velocity the transverse sums, then the outer sums over
// x-velocities; FP32 pairs and double-float for FP32 storage), summed over the warps, then
// the moments (one chunk per tile) or the chunk's partial sums in msum[grp].
template <typename S>
__device__ void chunk_moments(const Inst& I, int i0, int k0, int k1, int grp, const S* fo, double* ex, const void* tws,
                              int lane, int wy, int nwb = UPD_WARPS) {
    const int i = i0 + lane, ld = I.ld, Tc = I.Tc, Q = I.Q, G = I.mgroups;
    const bool valid = i < I.N;
    // warp wy < UPD_WARPS takes the velocities [ka, kb) of the chunk (warps beyond, in a wide
    // block, take none and only join the cross-warp sums: the same arithmetic in any block)
    const int per = (k1 - k0 + UPD_WARPS - 1) / UPD_WARPS;
    const int ka = min(k1, k0 + wy * per), kb = min(k1, ka + per);
    double* ss = ex + UPD_WARPS * MOM_SUMS * TILE;
    if constexpr (sizeof(S) == 4) {
        df o[MOM_SUMS];
#pragma unroll
        for (int j = 0; j < MOM_SUMS; ++j) o[j] = {0.0f, 0.0f};
        for (int kk = ka; kk < kb;) {
            const int kx = kk / Tc, ta = kk - kx * Tc, tb = min(Tc, kb - kx * Tc);
            kk = kx * Tc + tb;
            const float* twh = static_cast<const float*>(tws);
            const float* twl = twh + NTW * Tc;
            InnerSum<float> a[NTW];
            for (int t = ta; t < tb; ++t) {
                const float fv = fo[(kx * Tc + t - k0) * TILE + lane];
#pragma unroll
                for (int j = 0; j < NTW; ++j) {
                    // the weight is the same for every lane: zero weights (the mass and energy
                    // flags of the reduced slots) are skipped, power-of-two weights with no
                    // tail give exact products; both leave the sum's bits as add() would
                    const float wh = twh[j * Tc + t], wl = twl[j * Tc + t];
                    if (wh == 0.0f) continue;
                    if (wl == 0.0f && (__float_as_uint(wh) & 0x007fffffu) == 0u) a[j].add_exact(fv * wh);
                    else a[j].add(fv, 0.0, wh, wl);
                }
            }
            df Sd[NTW];
#pragma unroll
            for (int j = 0; j < NTW; ++j) Sd[j] = df_norm(a[j].hi, a[j].lo);
            outer_sums_df(o, Sd, df_of(I.px2[kx]), kx >= Q);
        }
        float2* pe = reinterpret_cast<float2*>(ex);
        if (wy < UPD_WARPS)
#pragma unroll
            for (int j = 0; j < MOM_SUMS; ++j) pe[(wy * MOM_SUMS + j) * TILE + lane] = make_float2(o[j].hi, o[j].lo);
        __syncthreads();
        for (int j = wy; j < MOM_SUMS; j += nwb) {
            df v = {0.0f, 0.0f};
            for (int q = 0; q < UPD_WARPS; ++q) v = v + df_of(pe[(q * MOM_SUMS + j) * TILE + lane]);
            if (G > 1) {
                if (valid) reinterpret_cast<float2*>(I.msum)[((size_t)grp * MOM_SUMS + j) * ld + i] = make_float2(v.hi, v.lo);
            } else {
                ss[j * TILE + lane] = (double)v.hi + (double)v.lo;
            }
        }
    } else {
        double o[MOM_SUMS];
#pragma unroll
        for (int j = 0; j < MOM_SUMS; ++j) o[j] = 0.0;
        for (int kk = ka; kk < kb;) {
            const int kx = kk / Tc, ta = kk - kx * Tc, tb = min(Tc, kb - kx * Tc);
            kk = kx * Tc + tb;
            const double* tw = static_cast<const double*>(tws);
            InnerSum<double> a[NTW];
            for (int t = ta; t < tb; ++t) {
                const double fv = fo[(kx * Tc + t - k0) * TILE + lane];
#pragma unroll
                for (int j = 0; j < NTW; ++j) {
                    const double w = tw[j * Tc + t];
                    if (w != 0.0) a[j].add(fv, w, 0.0f, 0.0f);     // same for every lane
                }
            }
            double Sv[NTW];
#pragma unroll
            for (int j = 0; j < NTW; ++j) Sv[j] = a[j].value();
            outer_sums(o, Sv, I.px[kx], kx >= Q);
        }
        if (wy < UPD_WARPS)
#pragma unroll
            for (int j = 0; j < MOM_SUMS; ++j) ex[(wy * MOM_SUMS + j) * TILE + lane] = o[j];
        __syncthreads();
        for (int j = wy; j < MOM_SUMS; j += nwb) {
            double v = 0.0;
            for (int q = 0; q < UPD_WARPS; ++q) v += ex[(q * MOM_SUMS + j) * TILE + lane];
            if (G > 1) {
                if (valid) I.msum[((size_t)grp * MOM_SUMS + j) * ld + i] = v;
            } else {
                ss[j * TILE + lane] = v;
            }
        }
    }
    if (G > 1) return;
    __syncthreads();
    const int tid = wy * TILE + lane;
    if (tid < 128) finalize_tile(I, i0, ss, tid);
}

// Tiled schedule, tiles split into several chunks: the last chunk block of the tile to arrive
// (ticket) adds the chunks' partial sums in chunk order -- the result does not depend on the
// arrival order -- and resets the ticket.  ss: MOM_SUMS x TILE shared doubles.
template <typename S>
__device__ void chunk_ticket_final(const Inst& I, int i0, double* ss, int nwb = UPD_WARPS) {
    __shared__ int last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, tile = i0 / TILE;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(I.mcnt + tile, 1) == I.mgroups - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid == 0) I.mcnt[tile] = 0;
    moments_final_tile<S>(I, i0, ss, tid, nwb, 1);
}

// ---- bulk asynchronous copies into shared memory (cp.async.bulk with an mbarrier) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bytes (a multiple of 16) from global src to shared dst (both 16-byte aligned), completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Phase `parity` of bar complete?  Each poll may suspend the thread for up to ~1 us.
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return done != 0;
}

constexpr long COPY_WAIT_POLLS = 2000000;      // ~2 s at the suspend hint

// Rows [k0, k0 + nrows) of one tile into shared memory: the source stage's values of nodes
// i0 - 4 .. i0 + 35 (clipped to the row) into Sw[r][0..SW), and, with F, the step's values of
// nodes i0 .. i0 + 31 into Fo[r][0..TILE).  BULK: one cp.async.bulk per row, all of the block's
// rows in flight at once, completion counted in bytes on an mbarrier (the tiled schedule);
// otherwise plain loads (the resident schedule).  Both leave the same values in shared memory.
// Window bounds are multiples of 4 nodes, so every bulk copy starts on a 16-byte boundary and
// moves a multiple of 16 bytes.  Returns false if the copies did not complete within the wait
// limit (the instance is then marked FDLB_FAILED_COPY).
template <typename S, bool BULK>
__device__ bool stage_rows(const Inst& I, int i0, int k0, int nrows, int stage, S* Sw, S* Fo, int lane, int wy,
                           int nwb = UPD_WARPS) {
    const int ld = I.ld;
    const int lo = max(0, i0 - 4), hi = min(ld, i0 + 36);
    const int off = lo - (i0 - 4);
    const S* src = static_cast<const S*>(I.f[stage - 1]);
    const S* F = static_cast<const S*>(I.f[0]);
    const bool withF = stage != 1;
    if constexpr (BULK) {
        __shared__ __align__(8) uint64_t bar;
        const uint32_t rowbytes = (uint32_t)(hi - lo) * sizeof(S), fbytes = TILE * sizeof(S);
        const int tid = wy * TILE + lane;
        if (tid == 0) {
            mbar_init(&bar, 1);
            mbar_expect_tx(&bar, (uint32_t)nrows * (rowbytes + (withF ? fbytes : 0u)));
        }
        // earlier generic accesses of this shared memory come before the copies' writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (lane == 0)
            for (int r = wy; r < nrows; r += nwb) {
                bulk_g2s(Sw + r * SW + off, src + (size_t)(k0 + r) * ld + lo, rowbytes, &bar);
                if (withF) bulk_g2s(Fo + r * TILE, F + (size_t)(k0 + r) * ld + i0, fbytes, &bar);
            }
        bool ok = false;
        for (long it = 0; it < COPY_WAIT_POLLS && !ok; ++it) ok = mbar_poll(&bar, 0);
        if (__syncthreads_or(!ok)) {          // the same decision in every thread of the block
            if (tid == 0) atomicExch(I.status, FDLB_FAILED_COPY);
            // give copies still in flight a second bounded wait before the block leaves
            for (long it = 0; it < COPY_WAIT_POLLS && !mbar_poll(&bar, 0); ++it) {
            }
            __syncthreads();
            return false;
        }
        if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(&bar)) : "memory");
        return true;
    } else {
        __syncthreads();
        const int n = hi - lo;
        for (int r = wy; r < nrows; r += nwb) {
            const S* row = src + (size_t)(k0 + r) * ld + lo;
            for (int j = lane; j < n; j += TILE) Sw[r * SW + off + j] = row[j];
            if (withF) Fo[r * TILE + lane] = F[(size_t)(k0 + r) * ld + i0 + lane];
        }
        __syncthreads();
        return true;
    }
}

// Velocities [k0, k1) of one tile for RK stage `stage`, by W warps (lane, warp wy; the
// velocity loop on all W, the moment partials on UPD_WARPS of them, so that W = 8 and 16 give
// the same results bit for bit);
// smem_raw holds upd_smem_bytes(ntab, ukc, sizeof(C), sizeof(S)).  The chunk's source rows (and
// F) are staged in shared memory first (stage_rows); the stencil, the ghost cells of the diffuse
// walls and F are then read from there.  The epilogue computes the moments of the new values
// (chunk_moments).  Returns false when the staging copies failed.
template <typename S, typename C, bool BULK, int W = UPD_WARPS>
__device__ bool update_item(const Inst& I, int i0, int k0, int k1, int stage, unsigned char* smem_raw, int lane, int wy) {
    C* stab = reinterpret_cast<C*>(smem_raw);
    void* tws = smem_raw + upd_table_bytes(I.trows, sizeof(C));
    S* Sw = reinterpret_cast<S*>(smem_raw + upd_stage_offset(I.trows, sizeof(C)));
    double* ex = reinterpret_cast<double*>(Sw);                 // after the rows are consumed
    S* fo = reinterpret_cast<S*>(smem_raw + upd_fo_offset(I.trows, I.ukc, sizeof(C), sizeof(S)));
    const int i = i0 + lane;
    const int N = I.N, ld = I.ld, Q = I.Q, Tc = I.Tc, trows = I.trows;
    // compact table: the x-projection rows of the NKX x-velocities from kx0 on (the chunk's),
    // then the 4 Tc transverse rows and 1/tau; NKX = 2Q (kx0 = 0) is the whole table
    const int NKX = (trows - 4 * Tc - 1) / 4;
    const int kx0 = NKX == 2 * Q ? 0 : k0 / Tc;
    const bool valid = i < N;
    const C* tabc = Tabs<C>::tab(I);
    const C* pxc = Tabs<C>::px(I);
    const C* gLc = Tabs<C>::gL(I);
    const C* gRc = Tabs<C>::gR(I);
    const C* Kyc = Tabs<C>::Ky(I);
    __syncthreads();                      // the previous item's readers of shared memory are done
    if (!stage_rows<S, BULK>(I, i0, k0, k1 - k0, stage, Sw, fo, lane, wy, W)) return false;
    // rows in batches: all loads of a batch are issued before its shared-memory stores
    constexpr int TB = 16;
    for (int r0 = wy; r0 < trows; r0 += W * TB) {
        C tmp[TB];
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int r = r0 + b * W;
            int gr = -1;                              // row of the instance's table
            if (r < 4 * NKX) {
                const int a = r / NKX, kx = kx0 + (r - a * NKX);
                if (kx < 2 * Q) gr = a * 2 * Q + kx;
            } else if (r < trows) {
                gr = 8 * Q + (r - 4 * NKX);
            }
            tmp[b] = (valid && gr >= 0) ? tabc[(size_t)gr * ld + i] : (C)0;
        }
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int r = r0 + b * W;
            if (r < trows) stab[r * TILE + lane] = tmp[b];
        }
    }
    load_tw<S>(I, tws, wy * TILE + lane, W * TILE);
    __syncthreads();
    const S* src = static_cast<const S*>(I.f[stage - 1]);
    S* dst = static_cast<S*>(I.f[stage % 3]);
    const C ca = stage == 1 ? (C)0 : (stage == 2 ? (C)0.75 : (C)(1.0 / 3.0));
    const C cb = stage == 1 ? (C)1 : (stage == 2 ? (C)0.25 : (C)(2.0 / 3.0));
    const C dt = (C)I.dt;
    const uint32_t seed = sizeof(S) == 4 ? sr_seed(I, stage) : 0u;
    const C nwL = (C)I.misc[M_NWL], nwR = (C)I.misc[M_NWR];
    const C xpi = valid ? Tabs<C>::xpinv(I)[i] : (C)0;
    const C invtau = stab[(4 * NKX + 4 * Tc) * TILE + lane];
    const bool force = I.accel_y != 0.0 && I.form != FORM_REDUCED1D;
    const int Tz = I.form == FORM_UNREDUCED ? I.Qz : 2;
    const C ay = (C)I.accel_y;
    const C sixth = (C)(1.0 / 6.0);
    // every stencil node of the tile inside the domain: no ghost cells (block-uniform)
    const bool interior = i0 >= 3 && i0 + TILE + 3 <= N;
    // (kx, t) of the warp's velocities k = k0 + wy + W m, stepped without divisions
    int kx = (k0 + wy) / Tc, t = (k0 + wy) - kx * Tc;
    for (int k = k0 + wy; k < k1; k += W) {
        const bool pos = kx < Q;
        const C p = pxc[kx];
        // node values i-3 .. i+3 (staged node j at row index j - i0 + 4) with the ghost cells of
        // the diffuse walls (Sec. III B): incoming populations take the wall Maxwellian n_w g,
        // outgoing ones the quadratic extrapolation of the three nodes next to the wall
        const S* row = Sw + (k - k0) * SW + 4 - i0;
        C v[7];
#pragma unroll
        for (int jj = 0; jj < 7; ++jj) {
            const int j = i - 3 + jj;
            C val;
            if (interior || (j >= 0 && j < N)) {
                val = (C)row[j];
            } else if (j < 0) {
                if (pos) {
                    val = nwL * gLc[k];
                } else {
                    const C f0 = (C)row[0], f1 = (C)row[1], f2 = (C)row[2];
                    val = j == -1 ? 3 * f0 - 3 * f1 + f2 : (j == -2 ? 6 * f0 - 8 * f1 + 3 * f2 : 10 * f0 - 15 * f1 + 6 * f2);
                }
            } else {
                if (!pos) {
                    val = nwR * gRc[k];
                } else {
                    const C f0 = (C)row[N - 1], f1 = (C)row[N - 2], f2 = (C)row[N - 3];
                    val = j == N ? 3 * f0 - 3 * f1 + f2 : (j == N + 1 ? 6 * f0 - 8 * f1 + 3 * f2 : 10 * f0 - 15 * f1 + 6 * f2);
                }
            }
            v[jj] = val;
        }
        // right face (i + 1/2)
        C fr;
        if (i + 1 == N) fr = pos ? (11 * v[3] - 7 * v[2] + 2 * v[1]) * sixth : nwR * gRc[k];
        else fr = pos ? weno_face(v[1], v[2], v[3], v[4], v[5]) : weno_face(v[6], v[5], v[4], v[3], v[2]);
        C fl = __shfl_up_sync(0xffffffffu, fr, 1);
        if (lane == 0) {
            if (i == 0) fl = pos ? nwL * gLc[k] : (11 * v[3] - 7 * v[4] + 2 * v[5]) * sixth;
            else fl = pos ? weno_face(v[0], v[1], v[2], v[3], v[4]) : weno_face(v[5], v[4], v[3], v[2], v[1]);
        }
        S* fk = fo + (k - k0) * TILE + lane;
        if (valid) {
            C L = -xpi * p * (fr - fl);
            if (force) {
                const int ky = t / Tz, kz = t - ky * Tz;
                const C* Kr = Kyc + ky * I.Qy;
                C d = 0;
                for (int kp = 0; kp < I.Qy; ++kp) d += Kr[kp] * (C)src[(size_t)(kx * Tc + kp * Tz + kz) * ld + i];
                L -= ay * d;
            }
            C tgt = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) tgt += stab[(a * NKX + kx - kx0) * TILE + lane] * stab[(4 * NKX + a * Tc + t) * TILE + lane];
            const C fi = v[3];
            const C Fk = stage == 1 ? (C)0 : (C)*fk;
            L += (tgt - fi) * invtau;
            C out;
            if constexpr (sizeof(C) == 4) {
                // FP32: the same combination written as an increment of F, F + cb ((f - F) + dt L)
                // (stage 1: f + dt L).  In the printed form ca F + cb (f + dt L) the rounded
                // weights (float) 1/3 + (float) 2/3 = 1 + 3e-8 scale a steady f up by half an ulp
                // every step, a mass drift of ~1e-3 over a solve; the increment form has no such
                // bias.  The sum is stored with stochastic rounding (sr_add).
                const C base = stage == 1 ? fi : Fk;
                const C inc = stage == 1 ? dt * L : cb * ((fi - Fk) + dt * L);
                out = sr_add(base, inc, fmix32(((uint32_t)k * (uint32_t)ld + (uint32_t)i) ^ seed));
            } else {
                out = cb * (fi + dt * L);
                if (stage != 1) out += ca * Fk;
            }
            dst[(size_t)k * ld + i] = (S)out;
            *fk = (S)out;
        } else {
            *fk = (S)0;
        }
        t += W;
        while (t >= Tc) {
            t -= Tc;
            ++kx;
        }
    }
    __syncthreads();                      // every warp is done with the staged rows (ex aliases them)
    chunk_moments<S>(I, i0, k0, k1, k0 / I.ukc, fo, ex, tws, lane, wy, W);
    return true;
}

template <typename S, typename C, int W>
__global__ void __launch_bounds__(TILE * W) k_update(const Inst* __restrict__ insts, const Work* __restrict__ work, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const Work w = work[blockIdx.x];
    const Inst& I = insts[w.inst];
    if (*I.status != FDLB_ACTIVE || I.smem_res) return;
    if ((I.precision == FDLB_FP64) != (sizeof(S) == 8)) return;
    if (!update_item<S, C, true, W>(I, w.i0, w.k0, w.k1, stage, smem_raw, threadIdx.x, threadIdx.y)) return;
    if (I.mgroups > 1)
        chunk_ticket_final<S>(I, w.i0, reinterpret_cast<double*>(smem_raw + upd_stage_offset(I.trows, sizeof(C))) + UPD_WARPS * MOM_SUMS * TILE, W);
}

// Moments of buffer `buf` from scratch (creation, new profiles, a loaded state): one block per
// update chunk of a tile with exactly the arithmetic of the update epilogue, so that the
// moments of a state do not depend on how it was reached (restarts are bitwise).
template <typename S>
__global__ void __launch_bounds__(TILE * UPD_WARPS) k_moments(const Inst* __restrict__ insts, const Work* __restrict__ work, int buf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Work w = work[blockIdx.x];
    const Inst& I = insts[w.inst];
    if (*I.status != FDLB_ACTIVE) return;
    if ((I.precision == FDLB_FP64) != (sizeof(S) == 8)) return;
    const int lane = threadIdx.x, wy = threadIdx.y, i = w.i0 + lane, ld = I.ld;
    const bool valid = i < I.N;
    void* tws = smem_raw;
    S* fo = reinterpret_cast<S*>(smem_raw + TW_BYTES);
    double* ex = reinterpret_cast<double*>(smem_raw + TW_BYTES + (size_t)I.ukc * TILE * sizeof(S));
    const S* f = static_cast<const S*>(I.f[buf]);
    for (int k = w.k0 + wy; k < w.k1; k += UPD_WARPS) fo[(k - w.k0) * TILE + lane] = valid ? f[(size_t)k * ld + i] : (S)0;
    load_tw<S>(I, tws, wy * TILE + lane, UPD_WARPS * TILE);
    __syncthreads();
    chunk_moments<S>(I, w.i0, w.k0, w.k1, w.k0 / I.ukc, fo, ex, tws, lane, wy);
    if (I.mgroups > 1) chunk_ticket_final<S>(I, w.i0, ex + UPD_WARPS * MOM_SUMS * TILE);
}

// ---------------------------------------------------------------------------
// resident schedule: one thread-block cluster per instance runs whole steps
// ---------------------------------------------------------------------------
// The phases of a step are the items of the tiled kernels (identical arithmetic), spread over
// the cluster's CTAs and separated by cluster barriers instead of kernel boundaries.  Every
// CTA of a cluster passes the same barriers: the trip counts depend only on the instance and
// on values broadcast from rank 0's shared memory.  Clusters never wait on each other.
namespace cg = cooperative_groups;

constexpr int RES_THREADS = TILE * NOD_WARPS;    // 256 = UPD_WARPS warps = two moment halves

__host__ __device__ inline size_t resident_smem_bytes(int qmax, size_t upd_max) {
    const size_t fin = (size_t)2 * MOM_SUMS * TILE * sizeof(double);
    const size_t nod = (size_t)nodal_smem_doubles(qmax) * sizeof(double);
    size_t m = fin > nod ? fin : nod;
    return m > upd_max ? m : upd_max;
}

// Moments of tiles whose update was split into chunks: the chunk partials, by 128-thread halves.
template <typename S>
__device__ void res_final(const Inst& I, int rank, int CS, unsigned char* sm, cg::cluster_group& cl) {
    const int tiles = (I.N + TILE - 1) / TILE, half = threadIdx.x >> 7;
    double* ss = reinterpret_cast<double*>(sm) + half * MOM_SUMS * TILE;
    for (int tl = 2 * rank + half; tl < tiles; tl += 2 * CS) moments_final_tile<S>(I, tl * TILE, ss, threadIdx.x & 127, 4, 1 + half);
    cl.sync();
}

template <int QB, typename S>
__device__ void res_step(Inst& I, int idx, double tol, double* resid_all, int rank, int CS, unsigned char* sm,
                         cg::cluster_group& cl) {
    const int tiles = (I.N + TILE - 1) / TILE, K = I.K, KC = I.ukc, nch = I.mgroups;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    // the update items' epilogue computes the moments of each stage's result
    for (int stage = 1; stage <= 3; ++stage) {
        for (int it = rank; it < 3 * tiles; it += CS)
            nodal_item<QB>(I, (it / 3) * TILE, it % 3, reinterpret_cast<double*>(sm), sizeof(S) == 4);
        cl.sync();
        for (int it = rank; it < tiles * nch; it += CS) {
            const int tl = it / nch, c = it - tl * nch, k0 = c * KC;
            update_item<S, S, false>(I, tl * TILE, k0, min(K, k0 + KC), stage, sm, lane, wy);
        }
        cl.sync();
        if (nch > 1) res_final<S>(I, rank, CS, sm, cl);
    }
    if (rank == 0) resid_item(I, idx, tol, resid_all);
}

// Cluster c of the grid advances instance list[c] by up to nsteps steps (it stops early when
// the instance leaves ACTIVE).
template <int QB>
__global__ void __launch_bounds__(RES_THREADS, 1) k_resident(Inst* insts, const int* list, int nsteps, double tol, double* resid_all) {
    extern __shared__ __align__(16) unsigned char rsm[];
    __shared__ int bc[2];
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int idx = list[blockIdx.x / CS];
    Inst& I = insts[idx];
    for (int s = 0; s < nsteps; ++s) {
        if (rank == 0 && threadIdx.x == 0) {
            bc[0] = *(volatile int*)I.status;
            bc[1] = *(volatile int*)&I.precision;
        }
        cl.sync();
        const int* b0 = cl.map_shared_rank(bc, 0);
        const int st = b0[0], prec = b0[1];
        if (st != FDLB_ACTIVE) {
            cl.sync();                    // nobody reads rank 0's shared memory after it exits
            break;
        }
        if (prec == FDLB_FP64) res_step<QB, double>(I, idx, tol, resid_all, rank, CS, rsm, cl);
        else res_step<QB, float>(I, idx, tol, resid_all, rank, CS, rsm, cl);
    }
}

// ---------------------------------------------------------------------------
// shared-memory-resident schedule: one CTA per instance keeps f in shared memory
// ---------------------------------------------------------------------------
// The CTA runs whole steps of its instance with the items of the tiled kernels (identical
// arithmetic) on a block-local copy of the instance record whose three RK buffers point into
// dynamic shared memory: f crosses HBM only when the launch starts and ends.  Tables, node rows
// and partial sums stay in global memory (L2).  Stages are separated by block barriers.
__host__ __device__ inline size_t smemres_f_bytes(int K, int ld, size_t s) { return ((size_t)K * ld * s + 15) / 16 * 16; }

template <int QB, typename S>
__device__ void smem_step(Inst& I, int idx, double tol, double* resid_all, unsigned char* sm) {
    const int tiles = (I.N + TILE - 1) / TILE, K = I.K, KC = I.ukc, nch = I.mgroups;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    for (int stage = 1; stage <= 3; ++stage) {
        for (int it = 0; it < 3 * tiles; ++it)
            nodal_item<QB>(I, (it / 3) * TILE, it % 3, reinterpret_cast<double*>(sm), sizeof(S) == 4);
        __syncthreads();
        for (int it = 0; it < tiles * nch; ++it) {
            const int tl = it / nch, c = it - tl * nch, k0 = c * KC;
            update_item<S, S, false>(I, tl * TILE, k0, min(K, k0 + KC), stage, sm, lane, wy);
        }
        __syncthreads();
        if (nch > 1) {
            // moments of chunked tiles from their partials, by 128-thread halves
            const int half = threadIdx.x >> 7;
            double* ss = reinterpret_cast<double*>(sm) + half * MOM_SUMS * TILE;
            for (int tl = half; tl < tiles; tl += 2) moments_final_tile<S>(I, tl * TILE, ss, threadIdx.x & 127, 4, 1 + half);
            __syncthreads();
        }
    }
    resid_item(I, idx, tol, resid_all);
    __syncthreads();
}

// Block b advances instance list[b] by up to nsteps steps; dynamic shared memory = scratch
// bytes for the items, then the three RK buffers.
template <int QB>
__global__ void __launch_bounds__(RES_THREADS, 1) k_smemres(Inst* insts, const int* list, int nsteps, double tol, double* resid_all,
                                                            size_t scratch) {
    extern __shared__ __align__(16) unsigned char rsm[];
    __shared__ Inst Is;
    const int idx = list[blockIdx.x];
    Inst& Ig = insts[idx];
    if (*(volatile int*)Ig.status != FDLB_ACTIVE) return;
    if (threadIdx.x == 0) Is = Ig;
    __syncthreads();
    const bool fp32 = Is.precision == FDLB_FP32_STORAGE;
    const size_t bytes = (size_t)Is.K * Is.ld * (fp32 ? 4 : 8);          // a multiple of 128
    const size_t fb = smemres_f_bytes(Is.K, Is.ld, fp32 ? 4 : 8);
    unsigned char* fs = rsm + scratch;
    uint4* gF = static_cast<uint4*>(Ig.f[0]);
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < 3; ++b) Is.f[b] = fs + b * fb;
    uint4* sF = reinterpret_cast<uint4*>(fs);
    for (size_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) sF[e] = gF[e];
    __syncthreads();
    for (int step = 0; step < nsteps; ++step) {
        if (*(volatile int*)Is.status != FDLB_ACTIVE) break;              // written by this block
        if (fp32) smem_step<QB, float>(Is, idx, tol, resid_all, rsm);
        else smem_step<QB, double>(Is, idx, tol, resid_all, rsm);
    }
    for (size_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) gF[e] = sF[e];
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
// The stepping kernels (closure, update, residual) are launched with programmatic stream
// serialization: the next kernel of a step is set up while the previous one finishes.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Kernel attributes (dynamic shared memory above 48 KB, non-portable cluster sizes) and the
// __constant__ tables are per device: each device keeps its own record of what was set, and
// a mutex serialises the updates.  Attributes only ever grow, so contexts created earlier on
// a device keep launching.
namespace {
constexpr int kMaxDevices = 64;
struct DevAttr {
    bool consts = false;
    int nodal = 0;
    size_t mom64 = 0, mom32 = 0, upd64 = 0, upd32 = 0;
    size_t res[2] = {0, 0};
    size_t smemres[2] = {0, 0};
    bool nonport[2] = {false, false};
};
std::mutex g_attr_mu;
DevAttr g_attr[kMaxDevices];

// Record of the current device (the caller holds g_attr_mu).
cudaError_t dev_attr(DevAttr** out) {
    int d = -1;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDevices) return cudaErrorInvalidDevice;
    *out = &g_attr[d];
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_setup(const Inst* d_inst, int count, cudaStream_t s) {
    k_setup<<<count, 128, 0, s>>>(const_cast<Inst*>(d_inst));
    k_profiles<double><<<count, 128, 0, s>>>(const_cast<Inst*>(d_inst), -1);
    k_profiles<float><<<count, 128, 0, s>>>(const_cast<Inst*>(d_inst), -1);
    return cudaGetLastError();
}

cudaError_t launch_set_profiles(const Inst* d_inst, int inst, cudaStream_t s) {
    k_profiles<double><<<1, 128, 0, s>>>(const_cast<Inst*>(d_inst), inst);
    k_profiles<float><<<1, 128, 0, s>>>(const_cast<Inst*>(d_inst), inst);
    return cudaGetLastError();
}

size_t moments_smem_bytes(int ukc, size_t s) {
    return TW_BYTES + (size_t)ukc * TILE * s + (size_t)(UPD_WARPS + 1) * MOM_SUMS * TILE * sizeof(double);
}

size_t update_smem_bytes(int ntab, int ukc, size_t c, size_t s) { return upd_smem_bytes(ntab, ukc, c, s); }

cudaError_t launch_moments(const Inst* d_inst, const Work* d_upd, int n_upd, int buf, int ukc_max, bool f64, bool f32,
                           cudaStream_t s) {
    const size_t m64 = moments_smem_bytes(ukc_max, 8), m32 = moments_smem_bytes(ukc_max, 4);
    {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        DevAttr* A = nullptr;
        cudaError_t e = dev_attr(&A);
        if (e == cudaSuccess && f64 && m64 > 48 * 1024 && m64 > A->mom64) {
            e = cudaFuncSetAttribute(k_moments<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m64);
            if (e == cudaSuccess) A->mom64 = m64;
        }
        if (e == cudaSuccess && f32 && m32 > 48 * 1024 && m32 > A->mom32) {
            e = cudaFuncSetAttribute(k_moments<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m32);
            if (e == cudaSuccess) A->mom32 = m32;
        }
        if (e != cudaSuccess) return e;
    }
    dim3 blk(TILE, UPD_WARPS);
    if (f64) k_moments<double><<<n_upd, blk, m64, s>>>(d_inst, d_upd, buf);
    if (f32) k_moments<float><<<n_upd, blk, m32, s>>>(d_inst, d_upd, buf);
    return cudaGetLastError();
}

cudaError_t launch_resid(const Inst* d_inst, int count, int anchor_inst, double freeze_tol, double* d_resid_all, cudaStream_t s) {
    if (anchor_inst != -2) {
        k_resid<<<count, 256, 0, s>>>(const_cast<Inst*>(d_inst), anchor_inst, freeze_tol, d_resid_all);
        return cudaGetLastError();
    }
    return launch_pdl(k_resid, (unsigned)count, dim3(256), 0, s, const_cast<Inst*>(d_inst), anchor_inst, freeze_tol, d_resid_all);
}

// (the caller holds g_attr_mu)
static cudaError_t set_smem(DevAttr* A, size_t smem64, size_t smem32) {
    cudaError_t e = cudaSuccess;
    if (smem64 > 48 * 1024 && smem64 > A->upd64) {
        e = cudaFuncSetAttribute(k_update<double, double, UPD_WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_update<double, double, UPD_WARPS_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
        if (e == cudaSuccess) A->upd64 = smem64;
    }
    if (e == cudaSuccess && smem32 > 48 * 1024 && smem32 > A->upd32) {
        e = cudaFuncSetAttribute(k_update<float, float, UPD_WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_update<float, float, UPD_WARPS_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32);
        if (e == cudaSuccess) A->upd32 = smem32;
    }
    return e;
}

cudaError_t launch_nodal(const Inst* d_inst, const Work* d_nod, int n_nod, int qmax, cudaStream_t s) {
    const size_t smem = (size_t)nodal_smem_doubles(qmax) * sizeof(double);
    if (qmax <= 8) return launch_pdl(k_nodal<8>, (unsigned)n_nod, dim3(TILE * NOD_WARPS), smem, s, d_inst, d_nod);
    return launch_pdl(k_nodal<QMAX>, (unsigned)n_nod, dim3(TILE * NOD_WARPS), smem, s, d_inst, d_nod);
}

cudaError_t prepare_kernels(size_t smem64, size_t smem32, int qmax) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    DevAttr* A = nullptr;
    cudaError_t ed = dev_attr(&A);
    if (ed != cudaSuccess) return ed;
    if (!A->consts) {
        float2 h[NINV2];
        h[0] = make_float2(0.0f, 0.0f);
        for (int j = 1; j < NINV2; ++j) {
            const double v = 1.0 / j;
            const float hi = (float)v;
            h[j] = make_float2(hi, (float)(v - (double)hi));
        }
        // synchronous copy: the table is in place before any kernel of this device uses it
        cudaError_t e = cudaMemcpyToSymbol(c_inv2, h, sizeof(h));
        if (e != cudaSuccess) return e;
        A->consts = true;
    }
    const int smem = nodal_smem_doubles(qmax) * (int)sizeof(double);
    if (smem > 48 * 1024 && smem > A->nodal) {
        cudaError_t e = cudaFuncSetAttribute(k_nodal<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_nodal<QMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        A->nodal = smem;
    }
    return set_smem(A, smem64, smem32);
}

// Attributes only ever grow, so that contexts created earlier keep launching; slot 0 records
// k_resident<8>, slot 1 k_resident<QMAX>.
template <int QB>
static cudaError_t resident_config(size_t smem, int cs) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    DevAttr* A = nullptr;
    cudaError_t e = dev_attr(&A);
    if (e != cudaSuccess) return e;
    const int slot = QB == 8 ? 0 : 1;
    if (smem > A->res[slot]) {
        e = cudaFuncSetAttribute(k_resident<QB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) A->res[slot] = smem;
    }
    if (e == cudaSuccess && cs > 8 && !A->nonport[slot]) {
        e = cudaFuncSetAttribute(k_resident<QB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) A->nonport[slot] = true;
    }
    return e;
}

cudaError_t prepare_resident(int qmax, size_t upd_max, int cs, size_t* smem) {
    *smem = resident_smem_bytes(qmax, upd_max);
    return qmax <= 8 ? resident_config<8>(*smem, cs) : resident_config<QMAX>(*smem, cs);
}

template <int QB>
static cudaError_t max_clusters(size_t smem, int cs, int* n) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(RES_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(n, k_resident<QB>, &cfg);
}

cudaError_t resident_max_clusters(int qmax, size_t smem, int cs, int* n) {
    return qmax <= 8 ? max_clusters<8>(smem, cs, n) : max_clusters<QMAX>(smem, cs, n);
}

cudaError_t launch_resident(Inst* d_inst, const int* d_list, int nclusters, int cs, int qmax, size_t smem, int nsteps,
                            double freeze_tol, double* d_resid_all, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(nclusters * cs);
    cfg.blockDim = dim3(RES_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (qmax <= 8) return cudaLaunchKernelEx(&cfg, k_resident<8>, d_inst, d_list, nsteps, freeze_tol, d_resid_all);
    return cudaLaunchKernelEx(&cfg, k_resident<QMAX>, d_inst, d_list, nsteps, freeze_tol, d_resid_all);
}

__global__ void k_set_smem_flags(Inst* insts, const int* list, int n, int on) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) insts[list[j]].smem_res = on;
}

cudaError_t launch_set_smem_flags(Inst* d_inst, const int* d_list, int n, int on, cudaStream_t s) {
    if (n > 0) k_set_smem_flags<<<(n + 255) / 256, 256, 0, s>>>(d_inst, d_list, n, on);
    return cudaGetLastError();
}

size_t smemres_scratch_bytes(int qmax, size_t upd_max) { return resident_smem_bytes(qmax, upd_max); }
size_t smemres_buffer_bytes(int K, int ld, size_t s) { return smemres_f_bytes(K, ld, s); }

// Dynamic shared memory available to k_smemres<QB>: the per-block maximum minus its static part.
cudaError_t smemres_dynamic_limit(int qmax, size_t* limit) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = qmax <= 8 ? cudaFuncGetAttributes(&fa, k_smemres<8>) : cudaFuncGetAttributes(&fa, k_smemres<QMAX>);
    if (e != cudaSuccess) return e;
    *limit = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    return cudaSuccess;
}

cudaError_t prepare_smemres(int qmax, size_t dyn) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    DevAttr* A = nullptr;
    cudaError_t e = dev_attr(&A);
    if (e != cudaSuccess) return e;
    const int slot = qmax <= 8 ? 0 : 1;
    if (dyn > A->smemres[slot]) {
        e = qmax <= 8 ? cudaFuncSetAttribute(k_smemres<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)
                      : cudaFuncSetAttribute(k_smemres<QMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e == cudaSuccess) A->smemres[slot] = dyn;
    }
    return e;
}

cudaError_t launch_smemres(Inst* d_inst, const int* d_list, int n, int qmax, size_t scratch, size_t dyn, int nsteps,
                           double freeze_tol, double* d_resid_all, cudaStream_t s) {
    if (qmax <= 8) k_smemres<8><<<n, RES_THREADS, dyn, s>>>(d_inst, d_list, nsteps, freeze_tol, d_resid_all, scratch);
    else k_smemres<QMAX><<<n, RES_THREADS, dyn, s>>>(d_inst, d_list, nsteps, freeze_tol, d_resid_all, scratch);
    return cudaGetLastError();
}

cudaError_t launch_update(const Inst* d_inst, const Work* d_upd, int n_upd, int stage, size_t smem64, size_t smem32,
                          bool f64, bool f32, bool wide, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (wide) {
        const dim3 blk(TILE, UPD_WARPS_WIDE);
        if (f64) e = launch_pdl(k_update<double, double, UPD_WARPS_WIDE>, (unsigned)n_upd, blk, smem64, s, d_inst, d_upd, stage);
        if (e == cudaSuccess && f32)
            e = launch_pdl(k_update<float, float, UPD_WARPS_WIDE>, (unsigned)n_upd, blk, smem32, s, d_inst, d_upd, stage);
    } else {
        const dim3 blk(TILE, UPD_WARPS);
        if (f64) e = launch_pdl(k_update<double, double, UPD_WARPS>, (unsigned)n_upd, blk, smem64, s, d_inst, d_upd, stage);
        if (e == cudaSuccess && f32) e = launch_pdl(k_update<float, float, UPD_WARPS>, (unsigned)n_upd, blk, smem32, s, d_inst, d_upd, stage);
    }
    return e;
}

}  // namespace fdlb
