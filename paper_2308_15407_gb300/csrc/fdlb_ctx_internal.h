// Internal accessors of a context (fdlb_host.cpp) used by the static-scratch entry point.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <string>
#include "../../include/fdlb.h"

namespace fdlb {
int ctx_f_buffer(fdlb_ctx* c, int inst, void** f, size_t* bytes);            // device address and size of F
int ctx_reanchor(fdlb_ctx* c, int inst);                                      // moments of F, residual anchor, ACTIVE
int ctx_moment_rows(fdlb_ctx* c, int inst, const double** rows, int* ld, int* nx);
cudaStream_t ctx_stream(fdlb_ctx* c);
void ctx_direct_launches(fdlb_ctx* c);                                        // never capture or instantiate a graph
void set_global_error(const std::string& msg);
}  // namespace fdlb
