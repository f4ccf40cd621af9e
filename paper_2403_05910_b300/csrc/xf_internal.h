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

// Launchers of the reverse-mode kernels of one (dim, N), filled by the
// translation unit that instantiates them (xf_adjoint_launch.cu). The face
// adjoints are indexed [reconstruction - 5][direction].
using XfFaceAdjFn = void (*)(const xf::Params&, const double*, const double*, double, double*,
                             cudaStream_t);
using XfFaceAdjPosFn = void (*)(const xf::Params&, const double*, const double*, double, double*,
                                const double*, cudaStream_t);
using XfFaceAdjPosTFn = void (*)(const xf::Params&, const double*, const double*, double,
                                 double*, const double*, const double*, cudaStream_t);
using XfGradAdjFn = void (*)(const xf::Params&, double*, cudaStream_t);
using XfCellAdjFn = void (*)(const xf::Params&, const double*, const double*, double*,
                             cudaStream_t);
using XfMixFn = void (*)(const xf::Params&, const double*, int, double, double*, double*,
                         cudaStream_t);
struct XfAdjTable {
  XfFaceAdjFn face_adj[3][3];
  XfFaceAdjPosFn face_adj_pos[3][3];  // inside an RK stage with the positivity blend
  XfFaceAdjPosTFn face_adj_pos_tape[3][3];  // the same, reading the flux tape
  XfGradAdjFn grad_adj;
  XfCellAdjFn prim_adj;
  XfCellAdjFn from_prim_adj;
  XfMixFn mixing;
};
// fill the reconstruction-5/6/7 entries (the 5 one also the cell, gradient
// and objective adjoints); false when (dim, N) has no instantiation
bool xf_internal_adj_fill5(int dim, int N, XfAdjTable* t);
bool xf_internal_adj_fill6(int dim, int N, XfAdjTable* t);
bool xf_internal_adj_fill7(int dim, int N, XfAdjTable* t);
