// Kernel launch wrappers (fdlb_kernels.cu), called by the host set-up.
#pragma once
#include <cuda_runtime.h>
#include "fdlb_internal.h"

namespace fdlb {

// Wall Maxwellians, initial uniform equilibrium, status/steps reset, for all instances.
cudaError_t launch_setup(const Inst* d_inst, int count, cudaStream_t s);

// Moments of RK buffer `buf` (0 = F, 1 = A, 2 = B) of every ACTIVE instance from scratch
// (during steps the update kernel's epilogue computes them): one block per update work item;
// ukc_max = largest update chunk of the batch.  Not inside a stream capture (it may set a
// kernel attribute).
cudaError_t launch_moments(const Inst* d_inst, const Work* d_upd, int n_upd, int buf, int ukc_max, bool f64, bool f32,
                           cudaStream_t s);

// Shared memory of one update item (table of ntab rows in type size c, ukc outputs of size s).
size_t update_smem_bytes(int ntab, int ukc, size_t c, size_t s);

// Residual / status pass after a step (anchor_inst = -2), or re-anchor instance `anchor_inst`
// (-1 = all): previous moments := current, residual := +inf, without a status change.
cudaError_t launch_resid(const Inst* d_inst, int count, int anchor_inst, double freeze_tol, double* d_resid_all,
                         cudaStream_t s);

// Projected local equilibrium from the profile rows (n, u_x, u_y, T) of instance `inst` into F.
cudaError_t launch_set_profiles(const Inst* d_inst, int inst, cudaStream_t s);

// Per-node closure (chi, Pr, tau, gradients, projection tables, wall densities).
cudaError_t launch_nodal(const Inst* d_inst, const Work* d_nod, int n_nod, int qmax, cudaStream_t s);

// RK stage `stage` (1..3) update of every ACTIVE instance; wide: blocks of 16 warps instead of
// 8 (the same results bit for bit; faster when the active blocks fit on the SMs at once).
cudaError_t launch_update(const Inst* d_inst, const Work* d_upd, int n_upd, int stage, size_t smem64, size_t smem32,
                          bool f64, bool f32, bool wide, cudaStream_t s);

// Resident schedule: attributes (shared memory, cluster size cs) of the cluster kernel for
// the batch's largest half-range order and update-item shared memory; *smem receives its
// dynamic shared memory.
cudaError_t prepare_resident(int qmax, size_t upd_max, int cs, size_t* smem);

// Clusters of cs CTAs that can be resident at once.
cudaError_t resident_max_clusters(int qmax, size_t smem, int cs, int* n);

// nclusters clusters of cs CTAs; cluster c advances instance d_list[c] by up to nsteps steps
// (residual, status and freezing as fdlb_step).
cudaError_t launch_resident(Inst* d_inst, const int* d_list, int nclusters, int cs, int qmax, size_t smem, int nsteps,
                            double freeze_tol, double* d_resid_all, cudaStream_t s);

// Shared-memory-resident schedule: one CTA per instance of d_list[0..n) keeps the instance's
// three RK buffers in dynamic shared memory (after `scratch` bytes of item scratch) and runs up
// to nsteps steps.  smemres_scratch_bytes: the item scratch for the batch's largest x order and
// update-item shared memory; smemres_buffer_bytes: one RK buffer; smemres_dynamic_limit: the
// dynamic shared memory a block of the kernel can have on this device.
size_t smemres_scratch_bytes(int qmax, size_t upd_max);
size_t smemres_buffer_bytes(int K, int ld, size_t s);
cudaError_t smemres_dynamic_limit(int qmax, size_t* limit);
cudaError_t prepare_smemres(int qmax, size_t dyn);
// smem_res := on for the instances d_list[0..n) (the tiled kernels skip flagged instances).
cudaError_t launch_set_smem_flags(Inst* d_inst, const int* d_list, int n, int on, cudaStream_t s);
cudaError_t launch_smemres(Inst* d_inst, const int* d_list, int n, int qmax, size_t scratch, size_t dyn, int nsteps,
                           double freeze_tol, double* d_resid_all, cudaStream_t s);

// Shared-memory attributes of the kernels that need more than 48 KB (call outside any capture).
cudaError_t prepare_kernels(size_t smem64, size_t smem32, int qmax);

// Kernel classes for the optional event timing of fdlb_profile.
enum KernelKind : int { KK_MOMENTS = 0, KK_NODAL = 1, KK_UPDATE = 2, KK_RESID = 3, KK_COUNT = 4 };

}  // namespace fdlb
