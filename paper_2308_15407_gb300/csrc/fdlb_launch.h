// Kernel launch wrappers (fdlb_kernels.cu), called by the host set-up.
#pragma once
#include <cuda_runtime.h>
#include "fdlb_internal.h"

namespace fdlb {

// Wall Maxwellians, initial uniform equilibrium, status/steps reset, for all instances.
cudaError_t launch_setup(const Inst* d_inst, int count, cudaStream_t s);

// Moments of RK buffer `buf` (0 = F, 1 = A, 2 = B) of every ACTIVE instance.
cudaError_t launch_moments(const Inst* d_inst, const Work* d_mom, int n_mom, int buf, bool f64, bool f32,
                           cudaStream_t s);

// Residual / status pass after a step (anchor_inst = -2), or re-anchor instance `anchor_inst`
// (-1 = all): previous moments := current, residual := +inf, without a status change.
cudaError_t launch_resid(const Inst* d_inst, int count, int anchor_inst, double freeze_tol, double* d_resid_all,
                         cudaStream_t s);

// Projected local equilibrium from the profile rows (n, u_x, u_y, T) of instance `inst` into F.
cudaError_t launch_set_profiles(const Inst* d_inst, int inst, cudaStream_t s);

// Per-node closure (chi, Pr, tau, gradients, projection tables, wall densities).
cudaError_t launch_nodal(const Inst* d_inst, const Work* d_nod, int n_nod, int qmax, cudaStream_t s);

// RK stage `stage` (1..3) update of every ACTIVE instance.
cudaError_t launch_update(const Inst* d_inst, const Work* d_upd, int n_upd, int stage, size_t smem64, size_t smem32,
                          bool f64, bool f32, cudaStream_t s);

// Shared-memory attributes of the kernels that need more than 48 KB (call outside any capture).
cudaError_t prepare_kernels(size_t smem64, size_t smem32, int qmax);

// Kernel classes for the optional event timing of fdlb_profile.
enum KernelKind : int { KK_MOMENTS = 0, KK_NODAL = 1, KK_UPDATE = 2, KK_RESID = 3, KK_COUNT = 4 };

}  // namespace fdlb
