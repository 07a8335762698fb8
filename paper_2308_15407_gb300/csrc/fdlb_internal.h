// Internal layout shared by the host set-up (fdlb_host.cpp) and the kernels
// (fdlb_kernels.cu).  Not part of the ABI.
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <vector_types.h>

namespace fdlb {

constexpr int QMAX = 16;        // x polynomials per block of the x projections (register block)
constexpr int QX_HALF_MAX = 100; // half-range order per side, at most (Sec. IV uses 100 for Kn > 1)
constexpr int QX_FULL_MAX = 100;  // half the full-range x order (order 2 x 100 = 200), at most
constexpr int LXMAX = 2 * QX_FULL_MAX;  // orthonormal x polynomials of a projection, at most
constexpr int QYMAX = 8;        // full-range order on y
constexpr int QZMAX = 8;        // full-range order on z
constexpr int TCMAX = QYMAX * QZMAX;
constexpr int MX = 16;          // auxiliary half-range rule of the x projections, at least
// Points of the auxiliary half-range rule for Lx half-range polynomials: the integrand is a
// polynomial of degree Lx + 2 times exp(q v - v^2/2); 16 points up to Lx = 16, beyond that
// enough for exactness on the polynomial part with the same margin for the exponential.
__host__ __device__ inline int aux_points_half(int Lx) { return Lx <= 16 ? MX : (Lx + 21) / 2; }
constexpr int MX8 = 8;          // shorter auxiliary rule when |u_x|/sqrt(T) is small (see k_nodal)
constexpr int MYMAX = 8;        // auxiliary full-range rule (exact: 2M > Q + 2)
constexpr int NTERMS = 13;      // monomials of f^S + tau J1
constexpr int TILE = 32;        // nodes per tile (one warp lane per node)
constexpr int NOD_WARPS = 8;    // warps per k_nodal block (a block serves one 32-node tile)
constexpr int MOM_SUMS = 14;    // raw moment sums per node

enum Form : int { FORM_UNREDUCED = 0, FORM_REDUCED2D = 1, FORM_REDUCED1D = 2 };

// Rows of the per-node primitive array (each row has ld doubles).
enum NodeRow : int {
    R_N = 0, R_UX, R_UY, R_T, R_QX, R_QY, R_PXX, R_PXY, R_SNEG, R_SPOS,
    R_PREV_N, R_PREV_UX, R_PREV_UY, R_PREV_T,
    R_LNN, R_LNT, R_LNCHI,     // ln n, ln T, ln chi(eta0 n) of the current moments
    NROWS
};

// Per-instance misc slots (doubles).
// M_WIN_STEP / M_WIN_RESID: step and residual at the start of the current stagnation window
// (M_WIN_STEP < 0: open a window at the next step); M_SWITCH: step of the FP32 -> FP64 up-cast
// of a two-phase instance, or -1; M_MASS0: channel mass sum_i dx_i n_i at the last anchor.
enum Misc : int { M_NWL = 0, M_NWR, M_RESID, M_INL, M_INR, M_WIN_STEP, M_WIN_RESID, M_SWITCH, M_MASS0, NMISC };

// One channel problem as the kernels see it.  All pointers are device addresses
// inside the caller's workspace.
struct Inst {
    int N, ld, Q, Qy, Qz, form, Tc, K;
    int Mx, My, Mz;
    int precision;             // storage in use now: FDLB_FP64 or FDLB_FP32_STORAGE (changes once
                               // on the device for two-phase instances)
    int j1_shear;
    int chi_model;             // FDLB_CHI_SET | FDLB_CHI_RET_FM
    int xfull;                 // x axis: 0 = half-range rules of order Q per side, 1 = one full-range
                               // rule of order 2Q (App. A)
    int Lx;                    // orthonormal x polynomials in the projection: Q (half), 2Q (full)
    int two_phase;             // FDLB_FP32_THEN_FP64: tables and buffers exist for both storages
    int ntab;                  // doubles per node in the projection table
    int trows;                 // rows of an update block's compact table: 4 NKX x-projection rows
                               // (the chunk's x-velocities), 4 Tc transverse rows, 1/tau
    uint32_t sr_key;           // hash of the parameters: seeds the stochastic rounding of FP32 storage
    int ukc;                   // velocities per update block (chunk) of a tile
    int mgroups;               // update chunks per tile (> 1: partial moment sums in msum)
    int smem_res;              // 1: stepped by the shared-memory-resident kernel (the tiled kernels skip it)
    double kn, eta0, chi0, mu0c, dt, ds, accel_y;
    double T_L, T_R, U_L, U_R, T_init;
    double x_h0;               // h_0 of the x axis' orthonormal family
    // tables
    const double* px;          // [2Q]: +p_1..+p_Q, -p_1..-p_Q
    const double* xq;          // [Mx] aux nodes: half-range rule (half), Gauss-Hermite rule (full)
    const double* xw;          // [Mx] aux weights (Mx = aux_points_half(Lx) or Q + 2)
    const double* xq8;         // [MX8] 8-point aux half-range nodes
    const double* xw8;         // [MX8] 8-point aux half-range weights
    const double* xa;          // [Lx]   recurrence alpha_l
    const double* xb;          // [Lx+1] recurrence b_l = sqrt(beta_l), b_0 = 0
    const double* xib;         // [Lx+1] 1/b_l (l >= 1)
    const double* xH;          // [Lx*Q] w_k h_l(p_k) at the positive nodes, index l*Q + k
    const double* yn;          // [Qy] nodes
    const double* yq;          // [My] aux full-range nodes
    const double* yw;          // [My] aux full-range weights
    const double* yH;          // [Qy*Qy] w_k h_l(p_k) with h_l = He_l/sqrt(l!)
    const double* zn;          // [Qz]
    const double* zq;          // [Mz]
    const double* zw;          // [Mz]
    const double* zH;          // [Qz*Qz]
    const double* Ky;          // [Qy*Qy] d/dp_y kernel, row k, column k'
    const double* tmt;         // [Tc] mass flag of transverse index t
    const double* tpy;         // [Tc] p_y of t
    const double* tet;         // [Tc] internal (z / theta) energy weight of t
    const double* xpinv;       // [N] 1/(x'(s_i) ds)
    const double* dxw;         // [N] x'(s_i) ds
    const double* gst;         // [3*7] gradient weights (in s) for nodes 0,1,2 on nodes 0..6
    const double* tw;          // [6*Tc] transverse moment weights mt, mt py, mt py^2, mt py^3, et, et py
    const float* twh;          // [6*Tc] float head of tw
    const float* twl;          // [6*Tc] float tail of tw (tw - twh)
    const double* fsq;         // [QYMAX+2] sqrt(l)
    const double* fisq;        // [QYMAX+2] 1/sqrt(l) (l >= 1)
    double* gL;                // [K] unit-density wall Maxwellians
    double* gR;                // [K]
    // FP32 copies read by the update kernel of FP32-storage instances (null otherwise)
    const float* px32;         // [2Q]
    const float* xpinv32;      // [N]
    const float* Ky32;         // [Qy*Qy]
    float* gL32;               // [K]
    float* gR32;               // [K]
    float* tab32;              // [ntab*ld]
    // (hi, lo) float pairs of the projection tables for the double-float closure of FP32
    // storage (null otherwise); same lengths as the FP64 tables
    const float2* xq2;
    const float2* xw2;
    const float2* xq82;
    const float2* xw82;
    const float2* xa2;
    const float2* xb2;
    const float2* xib2;
    const float2* xH2;
    const float2* yq2;
    const float2* yw2;
    const float2* yH2;
    const float2* zq2;
    const float2* zw2;
    const float2* zH2;
    const float2* fsq2;
    const float2* fisq2;
    const float2* px2;         // [2Q] x-velocities
    // Fischer-Methfessel averaging n-bar_i = sum_e w[e] n[col[e]], e in [ptr[i], ptr[i+1]) (RET-FM only)
    const int* fm_ptr;         // [N+1]
    const int* fm_col;         // [nnz]
    const double* fm_w;        // [nnz]
    float2 x_h02;
    void* f[3];                // RK buffers F, A, B; each K*ld elements of the storage type
    double* node;              // [NROWS*ld]
    double* tab;               // [ntab*ld] projection table (see below)
    double* misc;              // [NMISC]
    double* msum;              // [mgroups][14][ld] partial raw moment sums (mgroups > 1 only; FP32
                               // storage keeps them as float pairs in the same space)
    int* mcnt;                 // [tiles] arrival tickets of the update chunks of a tile (zero between uses)
    int* status;
    long long* steps;
};
// Projection table layout per node i (column i of a row-major [ntab][ld] array):
//   rows 0 .. 8Q-1          : Px[a][kx], a = 0..3, kx = 0..2Q-1   (row a*2Q + kx)
//   rows 8Q .. 8Q+4Tc-1     : n * Y[a][t]                         (row 8Q + a*Tc + t)
//   row  8Q+4Tc             : 1/tau
// Target value at (kx, t) = sum_a Px[a][kx] * nY[a][t].

// Work item for the tiled kernels.
struct Work {
    int inst;
    int i0;      // first node of the tile
    int k0, k1;  // velocity range [k0, k1)
};

}  // namespace fdlb
