// xf_adjoint_launch.cu -- launchers of the reverse-mode kernels (xf_adjoint.cuh)
// for every (dim, N). Compiled once per reconstruction (-DXF_ADJ_REC=5, 6 or
// 7) so that the library's translation units build in parallel; the REC = 5
// object also holds the cell, gradient and objective adjoints.
#include "xf_adjoint.cuh"
#include "xf_internal.h"

#ifndef XF_ADJ_REC
#error "compile with -DXF_ADJ_REC=5, 6 or 7"
#endif
#define XF_ADJ_CAT2(a, b) a##b
#define XF_ADJ_CAT(a, b) XF_ADJ_CAT2(a, b)
#define XF_ADJ_FILL XF_ADJ_CAT(xf_internal_adj_fill, XF_ADJ_REC)

namespace {

inline unsigned blocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <int DIM, int NS>
struct AdjLaunch {
  template <int D, int REC>
  static void face_adj(const xf::Params& p, const double* Q, const double* Rb, double scale,
                       double* Qb, cudaStream_t s) {
    if constexpr (D < DIM) {
      const long long nf =
          (long long)(p.n[0] + (D == 0)) * (p.n[1] + (D == 1)) * (p.n[2] + (D == 2));
      xf::k_face_adj<DIM, NS, D, REC><<<blocks(nf, 128), 128, 0, s>>>(p, Q, Rb, scale, Qb);
    }
  }
  template <int D, int REC>
  static void face_adj_pos(const xf::Params& p, const double* Q, const double* Rb, double scale,
                           double* Qb, const double* dt, cudaStream_t s) {
    if constexpr (D < DIM) {
      const long long nf =
          (long long)(p.n[0] + (D == 0)) * (p.n[1] + (D == 1)) * (p.n[2] + (D == 2));
      xf::k_face_adj_pos<DIM, NS, D, REC><<<blocks(nf, 128), 128, 0, s>>>(p, Q, Rb, scale, Qb,
                                                                         dt);
    }
  }
  template <int D, int REC>
  static void face_adj_pos_tape(const xf::Params& p, const double* Q, const double* Rb,
                                double scale, double* Qb, const double* dt, const double* Fh,
                                cudaStream_t s) {
    if constexpr (D < DIM) {
      const long long nf =
          (long long)(p.n[0] + (D == 0)) * (p.n[1] + (D == 1)) * (p.n[2] + (D == 2));
      xf::k_face_adj_pos_tape<DIM, NS, D, REC><<<blocks(nf, 128), 128, 0, s>>>(p, Q, Rb, scale,
                                                                              Qb, dt, Fh);
    }
  }
  static void grad_adj(const xf::Params& p, double* Qb, cudaStream_t s) {
    xf::k_grad_adj<DIM, NS><<<blocks(p.pcells, 256), 256, 0, s>>>(p, Qb);
  }
  static void prim_adj(const xf::Params& p, const double* Q, const double* Qb, double* Ub,
                       cudaStream_t s) {
    xf::k_prim_adj<DIM, NS><<<blocks(p.pcells, 128), 128, 0, s>>>(p, Q, Qb, Ub);
  }
  static void from_prim_adj(const xf::Params& p, const double* P, const double* Ub, double* Pb,
                            cudaStream_t s) {
    xf::k_from_prim_adj<DIM, NS><<<blocks(p.cells, 256), 256, 0, s>>>(p, P, Ub, Pb);
  }
  static void mixing(const xf::Params& p, const double* U, int sp, double dV, double* part,
                     double* Ub, cudaStream_t s) {
    xf::k_mixing<DIM, NS><<<blocks(p.cells, 256), 256, 0, s>>>(p, U, sp, dV, part, Ub);
  }
  static void fill(XfAdjTable* t) {
    constexpr int R = XF_ADJ_REC;
    t->face_adj[R - 5][0] = face_adj<0, R>;
    t->face_adj[R - 5][1] = face_adj<1, R>;
    t->face_adj[R - 5][2] = face_adj<2, R>;
    t->face_adj_pos[R - 5][0] = face_adj_pos<0, R>;
    t->face_adj_pos[R - 5][1] = face_adj_pos<1, R>;
    t->face_adj_pos[R - 5][2] = face_adj_pos<2, R>;
    t->face_adj_pos_tape[R - 5][0] = face_adj_pos_tape<0, R>;
    t->face_adj_pos_tape[R - 5][1] = face_adj_pos_tape<1, R>;
    t->face_adj_pos_tape[R - 5][2] = face_adj_pos_tape<2, R>;
#if XF_ADJ_REC == 5
    t->grad_adj = grad_adj;
    t->prim_adj = prim_adj;
    t->from_prim_adj = from_prim_adj;
    t->mixing = mixing;
#endif
  }
};

template <int DIM>
bool pick_n(int N, XfAdjTable* t) {
  switch (N) {
    case 2: AdjLaunch<DIM, 2>::fill(t); return true;
    case 3: AdjLaunch<DIM, 3>::fill(t); return true;
    case 4: AdjLaunch<DIM, 4>::fill(t); return true;
    case 5: AdjLaunch<DIM, 5>::fill(t); return true;
    default: return false;
  }
}

}  // namespace

bool XF_ADJ_FILL(int dim, int N, XfAdjTable* t) {
  switch (dim) {
    case 1: return pick_n<1>(N, t);
    case 2: return pick_n<2>(N, t);
    case 3: return pick_n<3>(N, t);
    default: return false;
  }
}
