// xf_internal.h -- helpers shared by the translation units of libxf.so
// (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>

#include "xf.h"
#include "xf_device.cuh"

// Validate (grid, thermo, opts) and build the kernels' parameter block.
xf_status xf_internal_fill_params(const xf_grid* g, const xf_thermo* th, const xf_opts* o,
                                  xf::Params* p);
// Record the message returned by xf_last_error on this thread.
void xf_internal_set_error(const char* msg);
void xf_internal_set_cuda_error(const char* what, cudaError_t e);
