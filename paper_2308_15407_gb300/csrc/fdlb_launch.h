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

// One full TVD-RK3 step of every ACTIVE instance, ending with the moments of the new state
// and the residual/status pass.
cudaError_t launch_step(const Inst* d_inst, int count, const Work* d_mom, int n_mom, const Work* d_upd, int n_upd,
                        size_t smem64, size_t smem32, bool f64, bool f32, double freeze_tol, double* d_resid_all,
                        cudaStream_t s);

}  // namespace fdlb
