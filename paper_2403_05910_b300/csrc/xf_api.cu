// xf_api.cu -- C-ABI entry points (include/xf.h) and kernel dispatch.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "xf.h"
#include "xf_device.cuh"
#include "xf_internal.h"

namespace {

thread_local std::string g_err;

void set_err(const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  g_err = buf;
}

#define XF_CUDA(call)        \
  do {                       \
    cudaError_t e_ = (call); \
    if (e_ != cudaSuccess) { \
      set_err(#call, e_);    \
      return XF_ERR_CUDA;    \
    }                        \
  } while (0)

inline unsigned blocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Multiprocessors of the current device (queried once).
int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 148;
    }
    return v;
  }();
  return n;
}

// Threads per block for n work items: the kernel's usual size, halved (down
// to one warp) while the grid would give fewer than two blocks per SM. The
// kernels are FP64-bound, and a single warp issues FP64 work slowly, so on
// small grids spreading the items over more SMs shortens every launch.
inline int bsize(long long n, int maxbs) {
  int bs = maxbs;
  while (bs > 32 && (n + bs - 1) / bs < 2LL * sm_count()) bs >>= 1;
  return bs;
}

// reduction of the per-block partial sums of the mixing objective (one block)
__global__ void k_sum_partials(const double* __restrict__ part, int n, double* out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// out = a x + b y + c z (elementwise; any of x, y, z may alias out)
__global__ void k_lincomb(long long n, double a, const double* x, double b, const double* y,
                          double c, const double* z, double* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = a * x[i];
  if (y) r = fma(b, y[i], r);
  if (z) r = fma(c, z[i], r);
  out[i] = r;
}


using PrimFn = void (*)(const xf::Params&, const double*, const double*, double*, double*,
                        uint32_t*, unsigned long long*, int, cudaStream_t);
using GradFn = void (*)(const xf::Params&, double*, cudaStream_t);
using FaceFn = void (*)(const xf::Params&, const double*, double*, uint32_t*, const double*,
                        cudaStream_t);
using UpdFn = void (*)(const xf::Params&, const double*, const double*, const double*,
                       const double*, const double*, double*, const double*, int, cudaStream_t);
// the same on an index range [b, e) (padded cells, faces of one direction,
// interior cells): the slabs of xf_step_rk3_host
using PrimRFn = void (*)(const xf::Params&, const double*, const double*, double*, double*,
                         uint32_t*, unsigned long long*, int, long long, long long, cudaStream_t);
using FaceRFn = void (*)(const xf::Params&, const double*, double*, uint32_t*, const double*,
                         long long, long long, cudaStream_t);
using UpdRFn = void (*)(const xf::Params&, const double*, const double*, const double*,
                        const double*, const double*, double*, const double*, int, long long,
                        long long, cudaStream_t);
using FromPrimFn = void (*)(const xf::Params&, const double*, double*, double*, cudaStream_t);
using GhostRFn = void (*)(const xf::Params&, double*, long long, long long, cudaStream_t);
using FaceTFn = void (*)(const xf::Params&, const double*, double*, uint32_t*, const double*,
                         double*, cudaStream_t);


struct Table {
  PrimFn prim;
  GradFn grad;
  FaceFn face[3];   // WENO5-JS reconstruction
  FaceFn face6[3];  // WENO-CU6
  FaceFn face7[3];  // WENO7-JS
  UpdFn update;
  FromPrimFn from_prim;
  int nq;
  XfAdjTable adj;  // reverse-mode launchers (xf_adjoint_launch.cu)
  PrimRFn prim_r;
  GhostRFn ghost_r;
  FaceRFn face_r[3][3];  // [weno - 5][direction]
  UpdRFn update_r;
  FaceTFn face_tape[3][3];  // [weno - 5][direction]: also write the flux tape
};

template <int DIM, int NS>
struct Launch {
  // primitive recovery of interior cells [b, e)
  static void prim_r(const xf::Params& p, const double* U, const double* Tin, double* Tout,
                     double* Q, uint32_t* fl, unsigned long long* red, int cfl, long long b,
                     long long e, cudaStream_t s) {
    if (e <= b) return;
    const int bs = bsize(e - b, 256);
    xf::k_prim<DIM, NS><<<blocks(e - b, bs), bs, 0, s>>>(p, U, Tin, Tout, Q, fl, red, cfl, b, e);
  }
  // ghost cells among padded cells [b, e), copied from their interior images
  static void ghost_r(const xf::Params& p, double* Q, long long b, long long e, cudaStream_t s) {
    if (e <= b || p.pcells == p.cells) return;
    xf::k_ghost<DIM, NS><<<blocks(e - b, 256), 256, 0, s>>>(p, Q, b, e);
  }
  static void prim(const xf::Params& p, const double* U, const double* Tin, double* Tout,
                   double* Q, uint32_t* fl, unsigned long long* red, int cfl, cudaStream_t s) {
    prim_r(p, U, Tin, Tout, Q, fl, red, cfl, 0, p.cells, s);
    ghost_r(p, Q, 0, p.pcells, s);
  }
  static void grad(const xf::Params& p, double* Q, cudaStream_t s) {
    const int bs = bsize(p.pcells, 256);
    xf::k_grad<DIM, NS><<<blocks(p.pcells, bs), bs, 0, s>>>(p, Q);
  }
  template <int D, int REC = 5>
  static void face_r(const xf::Params& p, const double* Q, double* G, uint32_t* fl,
                     const double* dt, long long b, long long e, cudaStream_t s) {
    if constexpr (D < DIM) {
      if (e <= b) return;
      const int bs = bsize(e - b, XF_FACE_THREADS);
      xf::k_face<DIM, NS, D, REC><<<blocks(e - b, bs), bs, 0, s>>>(p, Q, G, fl, dt, b, e);
    }
  }
  template <int D, int REC = 5>
  static void face(const xf::Params& p, const double* Q, double* G, uint32_t* fl, const double* dt,
                   cudaStream_t s) {
    const long long nf =
        (long long)(p.n[0] + (D == 0)) * (p.n[1] + (D == 1)) * (p.n[2] + (D == 2));
    face_r<D, REC>(p, Q, G, fl, dt, 0, nf, s);
  }
  template <int D, int REC = 5>
  static void face_tape(const xf::Params& p, const double* Q, double* G, uint32_t* fl,
                        const double* dt, double* Fh, cudaStream_t s) {
    if constexpr (D < DIM) {
      const long long nf =
          (long long)(p.n[0] + (D == 0)) * (p.n[1] + (D == 1)) * (p.n[2] + (D == 2));
      xf::k_face_tape<DIM, NS, D, REC><<<blocks(nf, XF_FACE_THREADS), XF_FACE_THREADS, 0, s>>>(
          p, Q, G, fl, dt, Fh);
    }
  }
  static void update_r(const xf::Params& p, const double* Gx, const double* Gy, const double* Gz,
                       const double* Un, const double* Us, double* out, const double* dt,
                       int mode, long long b, long long e, cudaStream_t s) {
    if (e <= b) return;
    const int bs = bsize(e - b, 256);
    xf::k_update<DIM, NS, true><<<blocks(e - b, bs), bs, 0, s>>>(p, Gx, Gy, Gz, Un, Us, out,
                                                                  dt, mode, b, e);
  }
  static void update(const xf::Params& p, const double* Gx, const double* Gy, const double* Gz,
                     const double* Un, const double* Us, double* out, const double* dt, int mode,
                     cudaStream_t s) {
    const int bs = bsize(p.cells, 256);
    xf::k_update<DIM, NS><<<blocks(p.cells, bs), bs, 0, s>>>(p, Gx, Gy, Gz, Un, Us, out, dt,
                                                              mode, 0, p.cells);
  }
  static void from_prim(const xf::Params& p, const double* P, double* U, double* T,
                        cudaStream_t s) {
    xf::k_from_prim<DIM, NS><<<blocks(p.cells, 256), 256, 0, s>>>(p, P, U, T);
  }
  static Table table() {
    Table t{prim, grad, {face<0>, face<1>, face<2>}, {face<0, 6>, face<1, 6>, face<2, 6>},
            {face<0, 7>, face<1, 7>, face<2, 7>}, update, from_prim, xf::Lay<DIM, NS>::NQ,
            XfAdjTable{}, prim_r, ghost_r,
            {{face_r<0>, face_r<1>, face_r<2>}, {face_r<0, 6>, face_r<1, 6>, face_r<2, 6>},
             {face_r<0, 7>, face_r<1, 7>, face_r<2, 7>}},
            update_r,
            {{face_tape<0>, face_tape<1>, face_tape<2>},
             {face_tape<0, 6>, face_tape<1, 6>, face_tape<2, 6>},
             {face_tape<0, 7>, face_tape<1, 7>, face_tape<2, 7>}}};
    xf_internal_adj_fill5(DIM, NS, &t.adj);
    xf_internal_adj_fill6(DIM, NS, &t.adj);
    xf_internal_adj_fill7(DIM, NS, &t.adj);
    return t;
  }
};

// face-flux launchers of the handle's reconstruction
inline const FaceFn* faces_of(const Table& t, int weno) {
  return weno == 7 ? t.face7 : (weno == 6 ? t.face6 : t.face);
}

template <int DIM>
bool pick_n(int N, Table* t) {
  switch (N) {
    case 2: *t = Launch<DIM, 2>::table(); return true;
    case 3: *t = Launch<DIM, 3>::table(); return true;
    case 4: *t = Launch<DIM, 4>::table(); return true;
    case 5: *t = Launch<DIM, 5>::table(); return true;
    default: return false;
  }
}

bool pick(int dim, int N, Table* t) {
  switch (dim) {
    case 1: return pick_n<1>(N, t);
    case 2: return pick_n<2>(N, t);
    case 3: return pick_n<3>(N, t);
    default: return false;
  }
}

// dt from the reduced maxima (one thread); resets the accumulators.
__global__ void k_dt_finalize(const __grid_constant__ xf::Params p, unsigned long long* red,
                              double* dt_out, double* dt_copy) {
  const double dt = xf::dt_from_red(p, red);
  *dt_out = dt;
  if (dt_copy) *dt_copy = dt;
  red[0] = 0ull;
  red[1] = 0ull;
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

__global__ void k_fill(double* p, long long n, double v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct xf_handle {
  xf::Params p;
  xf::Params* pdev = nullptr;  // p in device memory (p.dev)
  Table tab;
  int tcur = 0;  // which temperature buffer holds the latest warm start
  long long nf[3] = {0, 0, 0};
  double* U = nullptr;   // U^n
  double* Us = nullptr;  // stage state (also staging for host primitives)
  double* T[2] = {nullptr, nullptr};
  double* Q = nullptr;   // padded per-cell fields
  double* G[3] = {nullptr, nullptr, nullptr};  // per-direction face fluxes
  double* dt = nullptr;
  unsigned long long* red = nullptr;
  uint32_t* flags = nullptr;
  // adjoint buffers (allocated on first use): per-cell adjoint fields, the two
  // stage states and two stage adjoints of xf_step_rk3_adjoint, reduction partials
  double* Qb = nullptr;
  double* A1 = nullptr;
  double* A2 = nullptr;
  double* B1 = nullptr;
  double* B2 = nullptr;
  double* part = nullptr;
  // per-cell fields of U^n and U1 kept by xf_step_rk3_adjoint (allocated on
  // its first call), so its reverse does not recompute them
  double* QS[2] = {nullptr, nullptr};
  // xf_step_rk3_n: one captured step per temperature-buffer parity, for the
  // step size it was captured with (0 = CFL), replayed on the caller's stream
  cudaStream_t cap = nullptr;
  // xf_step_rk3_host: the copy stream and its events (reused across calls)
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> hev;
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  double step_graph_dt[2] = {-1.0, -1.0};
  // per-kernel event timing (xf_profile_enable / xf_profile_read)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int slot; cudaEvent_t a, b; };
  std::vector<Rec> recs;
};

namespace {

xf_status fill_params(const xf_grid* g, const xf_thermo* th, const xf_opts* o, xf::Params* p) {
  if (!g || !th || !o) return XF_ERR_ARG;
  if (g->dim < 1 || g->dim > 3) return XF_ERR_ARG;
  if (th->n_species < 2 || th->n_species > XF_MAX_SPECIES) return XF_ERR_ARG;
  if (o->weno < 5 || o->weno > 7 || o->split != 0) return XF_ERR_ARG;
  if (!(o->cfl > 0.0) || o->newton_max < 1 || !(o->newton_rtol > 0.0) || !(o->weno_eps > 0.0))
    return XF_ERR_ARG;
  if (!th->W || !th->cp_coef || !th->h_off) return XF_ERR_ARG;
  if (o->viscous && (!th->mu_coef || !th->kappa_coef || !(th->lewis > 0.0))) return XF_ERR_ARG;
  if (!(th->T_hi > th->T_lo) || !(th->a_ref2 > 0.0) || !(th->rho_ref > 0.0) || !(th->L_ref > 0.0))
    return XF_ERR_ARG;
  std::memset(p, 0, sizeof *p);
  const int dim = g->dim, N = th->n_species;
  p->dim = dim;
  p->N = N;
  p->nv = dim + 2 + N - 1;
  long long cells = 1, pcells = 1;
  double hmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      const int G = xf::ghosts(o->weno);
      if (g->n[a] < G || g->n[a] > (1 << 24)) return XF_ERR_ARG;
      if (!(g->hi[a] > g->lo[a])) return XF_ERR_ARG;
      for (int s = 0; s < 2; ++s)
        if (g->bc[a][s] < 0 || g->bc[a][s] > 2) return XF_ERR_ARG;
      if ((g->bc[a][0] == XF_BC_PERIODIC) != (g->bc[a][1] == XF_BC_PERIODIC)) return XF_ERR_ARG;
      p->n[a] = (int)g->n[a];
      p->np[a] = p->n[a] + 2 * G;
      p->go[a] = G;
      const double dx = (g->hi[a] - g->lo[a]) / (double)g->n[a];
      p->inv_dx[a] = 1.0 / dx;
      hmin = std::fmin(hmin, dx);
      p->bc[a][0] = g->bc[a][0];
      p->bc[a][1] = g->bc[a][1];
    } else {
      p->n[a] = 1;
      p->np[a] = 1;
      p->go[a] = 0;
      p->inv_dx[a] = 0.0;
    }
    cells *= p->n[a];
    pcells *= p->np[a];
  }
  if (pcells > (1ll << 31)) return XF_ERR_ARG;
  p->cells = cells;
  p->pcells = pcells;
  p->hmin2_over_2dim = hmin * hmin / (2.0 * dim);
  const double Ru = 8.314462618;
  p->T_lo = th->T_lo;
  p->span = th->T_hi - th->T_lo;
  p->inv_span = 1.0 / p->span;
  p->tau0 = -th->T_lo * p->inv_span;
  for (int j = 0; j < 5; ++j) p->hsj[j] = p->span / (j + 1);
  for (int s = 0; s < N; ++s) {
    if (!(th->W[s] > 0.0)) return XF_ERR_ARG;
    const double r = Ru / th->W[s] / th->a_ref2;
    p->r[s] = r;
    for (int j = 0; j < 5; ++j) {
      const double cj = th->cp_coef[s * 5 + j];
      p->rcp[s][j] = r * cj;
      p->rh[s][j] = r * p->span * cj / (j + 1);
    }
    p->rhoff[s] = r * th->h_off[s];
    p->invW[s] = 1.0 / th->W[s];
    p->Wm[s] = th->W[s];
    if (o->viscous) {
      for (int j = 0; j < 4; ++j) {
        p->lnmu[s][j] = th->mu_coef[s * 4 + j];
        p->lnka[s][j] = th->kappa_coef[s * 4 + j];
      }
    }
  }
  for (int s = 0; s < N; ++s)
    for (int t = 0; t < N; ++t) {
      p->wA[s][t] = (1.0 / std::sqrt(8.0)) * std::pow(1.0 + th->W[s] / th->W[t], -0.5);
      p->wB[s][t] = std::pow(th->W[t] / th->W[s], 0.25);
      p->wAB[s][t] = p->wA[s][t] * p->wB[s][t];
      p->wABB[s][t] = p->wA[s][t] * p->wB[s][t] * p->wB[s][t];
    }
  // coefficients of h_s - h_N and c_p,s - c_p,N (the face's heat flux by
  // diffusion); zero beyond s = N - 2
  for (int s = 0; s < xf::MAXN; ++s) {
    const bool in = s < N - 1;
    for (int j = 0; j < 5; ++j) {
      p->rcpd[s][j] = in ? p->rcp[s][j] - p->rcp[N - 1][j] : 0.0;
      p->rhd[s][j] = in ? p->rh[s][j] - p->rh[N - 1][j] : 0.0;
    }
    p->rhoffd[s] = in ? p->rhoff[s] - p->rhoff[N - 1] : 0.0;
    p->rdN[s] = in ? p->r[s] - p->r[N - 1] : 0.0;
  }
  const double a_ref = std::sqrt(th->a_ref2);
  p->fmu = 1.0 / (th->rho_ref * a_ref * th->L_ref);
  p->fka = 1.0 / (th->rho_ref * a_ref * th->a_ref2 * th->L_ref);
  p->inv_lewis = o->viscous ? 1.0 / th->lewis : 0.0;
  p->cfl = o->cfl;
  p->weno_eps = o->weno_eps;
  if (o->weno == 7) {
    const double e240 = 240.0 * o->weno_eps;
    p->wenoe[0] = e240 * xf::kW7c0; p->wenoe[1] = e240 * xf::kW7c1;
    p->wenoe[2] = e240 * xf::kW7c2; p->wenoe[3] = e240 * xf::kW7c3;
  } else {
    const double e12 = 12.0 * o->weno_eps;
    p->wenoe[0] = e12 * xf::kWc0; p->wenoe[1] = e12 * xf::kWc1; p->wenoe[2] = e12 * xf::kWc2;
    p->wenoe[3] = e12;
  }
  for (int k = 0; k < 4; ++k) p->wenoe4[k] = 0.25 * p->wenoe[k];
  p->weno = o->weno;
  for (int j = 0; j < 32; ++j) p->kface[j] = j < xf::kFaceCoefN ? xf::kFaceCoef[j] : 0.0;
  p->kface[14] = o->weno == 7 ? xf::rec_scale<7>() : xf::rec_scale<5>();
  for (int j = 0; j < 8; ++j) p->kexp[j] = xf::kExpCoef[j];
  for (int j = 0; j < 9; ++j) p->klog[j] = xf::kLogCoef[j];
  p->dev = nullptr;  // set by the owner of the struct
  p->newton_rtol = o->newton_rtol;
  p->newton_max = o->newton_max;
  p->viscous = o->viscous ? 1 : 0;
  p->convective = o->convective ? 1 : 0;
  p->positivity = o->positivity ? 1 : 0;
  if (o->positivity && !(o->pos_eps >= 0.0)) return XF_ERR_ARG;
  p->pos_eps = o->pos_eps;
  if (o->diffusion != 0 && o->diffusion != 1) return XF_ERR_ARG;
  p->diffusion = (o->viscous && o->diffusion == 1) ? 1 : 0;
  if (p->diffusion) {
    if (!th->dbin_coef) return XF_ERR_ARG;
    for (int s = 0; s < N; ++s)
      for (int t = 0; t < N; ++t)
        for (int j = 0; j < 4; ++j) p->dbin[s][t][j] = th->dbin_coef[(s * N + t) * 4 + j];
  }
  p->fdsm = th->rho_ref * th->a_ref2 * a_ref * th->L_ref;
  return XF_OK;
}

// per-cell fields of a handle's padded block (the D_sm fields ride along
// only with the mixture-averaged model)
inline size_t nq_of(const Table& t, const xf::Params& p) {
  return (size_t)t.nq + (p.diffusion ? (size_t)p.N : 0);
}

cudaEvent_t pool_event(xf_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch `fn` on stream s; with profiling on, bracket it by two events that
// xf_profile_read later turns into a duration for `slot` (XF_PROF_*).
template <class F>
void timed(xf_handle* h, int slot, cudaStream_t s, F&& fn) {
  if (!h->prof) {
    fn();
    return;
  }
  xf_handle::Rec r{slot, pool_event(h), pool_event(h)};
  cudaEventRecord(r.a, s);
  fn();
  cudaEventRecord(r.b, s);
  h->recs.push_back(r);
}

// Flux tape of one RK stage: the unblended convective fluxes of every face,
// direction by direction, each [n_v][faces of that direction].
long long tape_dir_off(const xf::Params& p, int d) {
  long long off = 0;
  for (int e = 0; e < d; ++e)
    off += (long long)p.nv * (p.n[0] + (e == 0)) * (p.n[1] + (e == 1)) * (p.n[2] + (e == 2));
  return off;
}
long long tape_stage_len(const xf::Params& p) { return tape_dir_off(p, p.dim); }

// Primitive recovery + (viscous) nodal gradients + every face flux of Uin.
// Inside an RK stage (`stepping`) the face kernels see the stage dt, which the
// positivity-preserving blend needs; a plain RHS has no dt.
xf_status stage_fluxes(xf_handle* h, const double* Uin, int do_cfl, cudaStream_t s,
                       bool stepping = false, double* Fh = nullptr) {
  const xf::Params& p = h->p;
  timed(h, XF_PROF_PRIM, s, [&] {
    h->tab.prim(p, Uin, h->T[h->tcur], h->T[1 - h->tcur], h->Q, h->flags, h->red, do_cfl, s);
  });
  h->tcur = 1 - h->tcur;
  if (do_cfl)
    timed(h, XF_PROF_DT, s, [&] { k_dt_finalize<<<1, 1, 0, s>>>(p, h->red, h->dt, nullptr); });
  if (p.viscous) timed(h, XF_PROF_GRAD, s, [&] { h->tab.grad(p, h->Q, s); });
  for (int d = 0; d < p.dim; ++d)
    timed(h, XF_PROF_FACE_X + d, s,
          [&] {
            if (Fh)
              h->tab.face_tape[p.weno - 5][d](p, h->Q, h->G[d], h->flags,
                                              stepping ? h->dt : nullptr,
                                              Fh + tape_dir_off(p, d), s);
            else
              faces_of(h->tab, p.weno)[d](p, h->Q, h->G[d], h->flags,
                                          stepping ? h->dt : nullptr, s);
          });
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

// Per-cell fields (and nodal gradients) of Uin, without the faces.
xf_status cell_fields(xf_handle* h, const double* Uin, cudaStream_t s) {
  const xf::Params& p = h->p;
  timed(h, XF_PROF_PRIM, s, [&] {
    h->tab.prim(p, Uin, h->T[h->tcur], h->T[1 - h->tcur], h->Q, h->flags, h->red, 0, s);
  });
  h->tcur = 1 - h->tcur;
  if (p.viscous) timed(h, XF_PROF_GRAD, s, [&] { h->tab.grad(p, h->Q, s); });
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status ensure_adjoint_buffers(xf_handle* h) {
  if (h->Qb) return XF_OK;
  const xf::Params& p = h->p;
  const size_t sb = sizeof(double) * (size_t)p.nv * p.cells;
  void* ptrs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const size_t bytes[6] = {sizeof(double) * nq_of(h->tab, p) * p.pcells, sb, sb, sb, sb,
                           sizeof(double) * (size_t)blocks(p.cells, 256)};
  for (int k = 0; k < 6; ++k) {
    if (cudaMalloc(&ptrs[k], bytes[k]) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < k; ++j) cudaFree(ptrs[j]);
      g_err = "adjoint buffers: cudaMalloc failed";
      return XF_ERR_OOM;
    }
  }
  h->Qb = (double*)ptrs[0];
  h->A1 = (double*)ptrs[1];
  h->A2 = (double*)ptrs[2];
  h->B1 = (double*)ptrs[3];
  h->B2 = (double*)ptrs[4];
  h->part = (double*)ptrs[5];
  return XF_OK;
}

// Ubar += scale (dL/dU)^T Rbar at the state U. With fields_ready the block
// h->Q already holds the per-cell fields of U. dtp (device, nullable): the
// RK stage's time step, for the reverse of the positivity blend.
xf_status rhs_adjoint_impl(xf_handle* h, const double* U, const double* Rbar, double scale,
                           double* Ubar, cudaStream_t s, bool fields_ready = false,
                           const double* dtp = nullptr, const double* Fh = nullptr) {
  xf_status st = ensure_adjoint_buffers(h);
  if (st != XF_OK) return st;
  if (!fields_ready) {
    st = cell_fields(h, U, s);
    if (st != XF_OK) return st;
  }
  const xf::Params& p = h->p;
  XF_CUDA(cudaMemsetAsync(h->Qb, 0, sizeof(double) * nq_of(h->tab, p) * p.pcells, s));
  for (int d = 0; d < p.dim; ++d)
    timed(h, XF_PROF_FACE_ADJ, s, [&] {
      const int r = p.weno - 5;
      if (p.positivity && dtp && Fh)
        h->tab.adj.face_adj_pos_tape[r][d](p, h->Q, Rbar, scale, h->Qb, dtp,
                                           Fh + tape_dir_off(p, d), s);
      else if (p.positivity && dtp)
        h->tab.adj.face_adj_pos[r][d](p, h->Q, Rbar, scale, h->Qb, dtp, s);
      else h->tab.adj.face_adj[r][d](p, h->Q, Rbar, scale, h->Qb, s);
    });
  if (p.viscous) timed(h, XF_PROF_GRAD, s, [&] { h->tab.adj.grad_adj(p, h->Qb, s); });
  timed(h, XF_PROF_PRIM_ADJ, s, [&] { h->tab.adj.prim_adj(p, h->Q, h->Qb, Ubar, s); });
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

void lincomb(const xf_handle* h, double a, const double* x, double b, const double* y, double c,
             const double* z, double* out, cudaStream_t s) {
  const long long n = (long long)h->p.nv * h->p.cells;
  k_lincomb<<<blocks(n, 256), 256, 0, s>>>(n, a, x, b, y, c, z, out);
}

// rcp_nr beside the correctly rounded division, element by element
__global__ void k_probe_rcp(const double* __restrict__ x, double* __restrict__ y,
                            double* __restrict__ ref, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = xf::rcp_nr(x[i]);
  ref[i] = 1.0 / x[i];
}

// exp_t beside CUDA's exp, element by element
__global__ void k_probe_exp(const double* __restrict__ x, double* __restrict__ y,
                            double* __restrict__ ref, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = xf::exp_t(x[i]);
  ref[i] = exp(x[i]);
}

// log_t beside CUDA's log, element by element
__global__ void k_probe_log(const double* __restrict__ x, double* __restrict__ y,
                            double* __restrict__ ref, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = xf::log_t(x[i]);
  ref[i] = log(x[i]);
}

__global__ void k_probe_fp64(double* out, long long iters, double a) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4,
         x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (long long i = 0; i < iters; ++i) {
    x0 = fma(x0, a, -a); x1 = fma(x1, a, -a); x2 = fma(x2, a, -a); x3 = fma(x3, a, -a);
    x4 = fma(x4, a, -a); x5 = fma(x5, a, -a); x6 = fma(x6, a, -a); x7 = fma(x7, a, -a);
  }
  const double r = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (r == 12345.678) out[0] = r;  // keeps the chains live; never true in practice
}

}  // namespace

xf_status xf_internal_fill_params(const xf_grid* g, const xf_thermo* th, const xf_opts* o,
                                  xf::Params* p) {
  return fill_params(g, th, o, p);
}
void xf_internal_set_error(const char* msg) { g_err = msg; }
void xf_internal_set_cuda_error(const char* what, cudaError_t e) { set_err(what, e); }

namespace {
// ---- xf_step_rk3_host: slabs of the slowest active axis a. Each slab j holds
// interior planes [z_j, z_{j+1}) of a; the copies of slab j run on the handle's
// copy stream while the compute stream works on other slabs.
struct Slabs {
  int a = 0, S = 1, G = 0;
  long long n = 1, cs = 1, ps = 1;  // planes, interior / padded cells per plane
  long long zb[9] = {0};            // slab j holds planes [zb[j], zb[j+1])
  long long z(int j) const { return zb[j]; }
};

Slabs slabs_of(const xf::Params& p) {
  Slabs sl;
  sl.a = p.dim - 1;
  sl.n = p.n[sl.a];
  sl.G = p.go[sl.a];
  sl.cs = p.cells / sl.n;
  sl.ps = p.pcells / p.np[sl.a];
  // slabs of >= 16 planes and >= 2^18 cells, at most 8: below that the copies
  // are short and one slab (no overlap) costs fewer launches
  long long S = std::min<long long>(8, sl.n / 16);
  S = std::min<long long>(S, p.cells >> 18);
  sl.S = (int)std::max<long long>(1, S);
  // from 4 slabs on, the first and the last are a quarter of the others: the
  // first slab's upload and the last one's read-back are the copies that no
  // compute hides (each still >= 3 planes: n >= 16 S)
  const long long m = sl.S - 2, units = 4 * m + 2;
  for (int j = 0; j <= sl.S; ++j) {
    long long u = j;
    if (sl.S >= 4) u = j == 0 ? 0 : (j == sl.S ? units : 1 + 4 * (long long)(j - 1));
    sl.zb[j] = sl.S >= 4 ? sl.n * u / units : sl.n * j / sl.S;
  }
  return sl;
}

// faces of direction d on face planes [z0, z1) of axis a (n planes when
// d != a, n + 1 when d == a), in the face kernels' order
void face_range(const xf::Params& p, const Slabs& sl, int d, long long z0, long long z1,
                long long* b, long long* e) {
  long long ps = 1;
  for (int k = 0; k < sl.a; ++k) ps *= p.n[k] + (k == d);
  *b = z0 * ps;
  *e = z1 * ps;
}

xf_status host_events(xf_handle* h, int need) {
  while ((int)h->hev.size() < need) {
    cudaEvent_t e;
    XF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->hev.push_back(e);
  }
  if (!h->cs) XF_CUDA(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
  return XF_OK;
}

}  // namespace

extern "C" {

const char* xf_status_str(xf_status s) {
  switch (s) {
    case XF_OK: return "ok";
    case XF_ERR_ARG: return "invalid argument";
    case XF_ERR_CUDA: return "CUDA error";
    case XF_ERR_NONPHYS: return "non-physical state (NaN/inf, rho<=0, p<=0 or T<=0)";
    case XF_ERR_NEWTON: return "temperature Newton solve did not converge";
    case XF_ERR_EIGEN: return "face sound speed squared <= 0";
    case XF_ERR_TIMEOUT: return "bounded device wait gave up";
    case XF_ERR_OOM: return "out of device memory";
  }
  return "unknown status";
}

const char* xf_last_error(void) { return g_err.c_str(); }

xf_status xf_create(const xf_grid* grid, const xf_thermo* thermo, const xf_opts* opts,
                    xf_handle** out) {
  if (!out) return XF_ERR_ARG;
  *out = nullptr;
  xf::Params p;
  xf_status st = fill_params(grid, thermo, opts, &p);
  if (st != XF_OK) return st;
  Table tab;
  if (!pick(p.dim, p.N, &tab)) return XF_ERR_ARG;
  xf_handle* h = new xf_handle();
  h->p = p;
  h->tab = tab;
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t st_bytes = sizeof(double) * (size_t)p.nv * p.cells;
  bool ok = alloc((void**)&h->pdev, sizeof(xf::Params)) &&
            alloc((void**)&h->U, st_bytes) && alloc((void**)&h->Us, st_bytes) &&
            alloc((void**)&h->T[0], sizeof(double) * p.cells) &&
            alloc((void**)&h->T[1], sizeof(double) * p.cells) &&
            alloc((void**)&h->Q, sizeof(double) * nq_of(tab, p) * p.pcells) &&
            alloc((void**)&h->dt, sizeof(double)) &&
            alloc((void**)&h->red, 2 * sizeof(unsigned long long)) &&
            alloc((void**)&h->flags, sizeof(uint32_t));
  for (int d = 0; ok && d < p.dim; ++d) {
    h->nf[d] = (long long)(p.n[0] + (d == 0)) * (p.n[1] + (d == 1)) * (p.n[2] + (d == 2));
    ok = alloc((void**)&h->G[d], sizeof(double) * (size_t)p.nv * h->nf[d]);
  }
  if (!ok) {
    xf_destroy(h);
    g_err = "cudaMalloc failed";
    return XF_ERR_OOM;
  }
  h->p.dev = h->pdev;
  if (cudaMemcpy(h->pdev, &h->p, sizeof(xf::Params), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->red, 0, 2 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(h->flags, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(h->dt, 0, sizeof(double)) != cudaSuccess ||
      cudaMemset(h->Q, 0, sizeof(double) * nq_of(tab, p) * p.pcells) != cudaSuccess) {
    xf_destroy(h);
    g_err = "cudaMemcpy or cudaMemset failed";
    return XF_ERR_CUDA;
  }
  k_fill<<<blocks(p.cells, 256), 256>>>(h->T[0], p.cells, 300.0);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    xf_destroy(h);
    g_err = "initialisation failed";
    return XF_ERR_CUDA;
  }
  *out = h;
  return XF_OK;
}

void xf_destroy(xf_handle* h) {
  if (!h) return;
  cudaFree(h->pdev);
  cudaFree(h->U);
  cudaFree(h->Us);
  cudaFree(h->T[0]);
  cudaFree(h->T[1]);
  cudaFree(h->Q);
  for (int d = 0; d < 3; ++d) cudaFree(h->G[d]);
  cudaFree(h->dt);
  cudaFree(h->red);
  cudaFree(h->flags);
  cudaFree(h->Qb);
  cudaFree(h->QS[0]);
  cudaFree(h->QS[1]);
  cudaFree(h->A1);
  cudaFree(h->A2);
  cudaFree(h->B1);
  cudaFree(h->B2);
  cudaFree(h->part);
  for (auto& r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k)
    if (h->step_graph[k]) cudaGraphExecDestroy(h->step_graph[k]);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (auto e : h->hev) cudaEventDestroy(e);
  if (h->cs) cudaStreamDestroy(h->cs);
  delete h;
}

int xf_nv(const xf_handle* h) { return h ? h->p.nv : 0; }
int64_t xf_cells(const xf_handle* h) { return h ? h->p.cells : 0; }

xf_status xf_set_state(xf_handle* h, const double* U, const double* T_guess, void* stream) {
  if (!h || !U) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const xf::Params& p = h->p;
  XF_CUDA(cudaMemcpyAsync(h->U, U, sizeof(double) * (size_t)p.nv * p.cells, cudaMemcpyDefault, s));
  if (T_guess) {
    XF_CUDA(cudaMemcpyAsync(h->T[h->tcur], T_guess, sizeof(double) * p.cells, cudaMemcpyDefault, s));
  } else {
    k_fill<<<blocks(p.cells, 256), 256, 0, s>>>(h->T[h->tcur], p.cells, 300.0);
    XF_CUDA(cudaGetLastError());
  }
  return XF_OK;
}

xf_status xf_set_primitive(xf_handle* h, const double* P, void* stream) {
  if (!h || !P) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const xf::Params& p = h->p;
  const double* src = P;
  if (!is_device_ptr(P)) {
    XF_CUDA(cudaMemcpyAsync(h->Us, P, sizeof(double) * (size_t)p.nv * p.cells, cudaMemcpyDefault, s));
    src = h->Us;
  }
  h->tab.from_prim(p, src, h->U, h->T[h->tcur], s);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_get_state(xf_handle* h, double* U, double* T, void* stream) {
  if (!h) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const xf::Params& p = h->p;
  if (U) XF_CUDA(cudaMemcpyAsync(U, h->U, sizeof(double) * (size_t)p.nv * p.cells, cudaMemcpyDefault, s));
  if (T) XF_CUDA(cudaMemcpyAsync(T, h->T[h->tcur], sizeof(double) * p.cells, cudaMemcpyDefault, s));
  return XF_OK;
}

xf_status xf_rhs(xf_handle* h, const double* U, double* dUdt, void* stream) {
  if (!h || !U || !dUdt) return XF_ERR_ARG;
  if (!is_device_ptr(U) || !is_device_ptr(dUdt)) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  xf_status st = stage_fluxes(h, U, 0, s);
  if (st != XF_OK) return st;
  const xf::Params& p = h->p;
  timed(h, XF_PROF_UPDATE, s, [&] {
    h->tab.update(p, h->G[0], h->G[1], h->G[2], nullptr, nullptr, dUdt, h->dt, 0, s);
  });
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_compute_dt(xf_handle* h, double* dt_dev, void* stream) {
  if (!h || !dt_dev) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const xf::Params& p = h->p;
  h->tab.prim(p, h->U, h->T[h->tcur], h->T[1 - h->tcur], h->Q, h->flags, h->red, 1, s);
  h->tcur = 1 - h->tcur;
  k_dt_finalize<<<1, 1, 0, s>>>(p, h->red, h->dt, dt_dev);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

// One SSP-RK3 step (Eq. 16) of the handle's state on stream s (dt <= 0: the
// CFL step of U^n, computed on the device).
// One SSP-RK3 step. The stage states go to U1 and U2 when given (the taped
// step), else both to the handle's stage buffer.
static xf_status step_impl(xf_handle* h, double dt, double* dt_dev_out, cudaStream_t s,
                           double* U1 = nullptr, double* U2 = nullptr, double* Fhat = nullptr) {
  const xf::Params& p = h->p;
  const bool cfl = !(dt > 0.0);
  double* S1 = U1 ? U1 : h->Us;
  double* S2 = U2 ? U2 : h->Us;
  const long long tl = tape_stage_len(p);
  if (!cfl) k_set_scalar<<<1, 1, 0, s>>>(h->dt, dt);
  // Eq. 16: three stages, U^n kept in U
  xf_status st = stage_fluxes(h, h->U, cfl ? 1 : 0, s, true, Fhat);
  if (st != XF_OK) return st;
  timed(h, XF_PROF_UPDATE, s, [&] {
    h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, h->U, S1, h->dt, 1, s);
  });
  st = stage_fluxes(h, S1, 0, s, true, Fhat ? Fhat + tl : nullptr);
  if (st != XF_OK) return st;
  timed(h, XF_PROF_UPDATE, s, [&] {
    h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, S1, S2, h->dt, 2, s);
  });
  st = stage_fluxes(h, S2, 0, s, true, Fhat ? Fhat + 2 * tl : nullptr);
  if (st != XF_OK) return st;
  timed(h, XF_PROF_UPDATE, s, [&] {
    h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, S2, h->U, h->dt, 3, s);
  });
  XF_CUDA(cudaGetLastError());
  if (dt_dev_out)
    XF_CUDA(cudaMemcpyAsync(dt_dev_out, h->dt, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return XF_OK;
}

xf_status xf_step_rk3(xf_handle* h, double dt, double* dt_dev_out, void* stream) {
  if (!h || !(dt == dt)) return XF_ERR_ARG;
  return step_impl(h, dt, dt_dev_out, (cudaStream_t)stream);
}

xf_status xf_step_rk3_host(xf_handle* h, const double* U_in, const double* T_in, double* U_out,
                           double* T_out, double dt, double* dt_dev_out, void* stream) {
  if (!h || !U_in || !U_out || !(dt == dt)) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const xf::Params& p = h->p;
  const Slabs sl = slabs_of(p);
  const int S = sl.S;
  xf_status st = host_events(h, 2 * S + 3);
  if (st != XF_OK) return st;
  cudaEvent_t* ev = h->hev.data();  // [0, S) uploads, [S, 2S) updates, then T, start, end
  cudaEvent_t ev_T = ev[2 * S], ev_start = ev[2 * S + 1], ev_end = ev[2 * S + 2];
  cudaStream_t cs = h->cs;
  const size_t row = sizeof(double) * (size_t)p.cells;
  // the uploads overwrite the state: they wait for the work already on `stream`
  XF_CUDA(cudaEventRecord(ev_start, s));
  XF_CUDA(cudaStreamWaitEvent(cs, ev_start, 0));
  double* Tn = h->T[h->tcur];
  if (!T_in) k_fill<<<blocks(p.cells, 256), 256, 0, cs>>>(Tn, p.cells, 300.0);
  for (int j = 0; j < S; ++j) {
    const long long c0 = sl.z(j) * sl.cs, nc = (sl.z(j + 1) - sl.z(j)) * sl.cs;
    XF_CUDA(cudaMemcpy2DAsync(h->U + c0, row, U_in + c0, row, sizeof(double) * nc, p.nv,
                              cudaMemcpyDefault, cs));
    if (T_in)
      XF_CUDA(cudaMemcpyAsync(Tn + c0, T_in + c0, sizeof(double) * nc, cudaMemcpyDefault, cs));
    XF_CUDA(cudaEventRecord(ev[j], cs));
  }
  const bool cfl = !(dt > 0.0);
  if (!cfl) k_set_scalar<<<1, 1, 0, s>>>(h->dt, dt);
  // stage 1: the primitive recovery of each slab's interior planes as soon
  // as its upload lands, then the ghosts inside those planes (their images
  // lie in the same plane); the ghost planes of axis a (whose images are on
  // any slab) after the last one
  double* Tout = h->T[1 - h->tcur];
  for (int j = 0; j < S; ++j) {
    XF_CUDA(cudaStreamWaitEvent(s, ev[j], 0));
    timed(h, XF_PROF_PRIM, s, [&] {
      h->tab.prim_r(p, h->U, Tn, Tout, h->Q, h->flags, h->red, cfl ? 1 : 0,
                    sl.z(j) * sl.cs, sl.z(j + 1) * sl.cs, s);
      h->tab.ghost_r(p, h->Q, (sl.z(j) + sl.G) * sl.ps, (sl.z(j + 1) + sl.G) * sl.ps, s);
    });
  }
  timed(h, XF_PROF_PRIM, s, [&] {
    h->tab.ghost_r(p, h->Q, 0, sl.G * sl.ps, s);
    h->tab.ghost_r(p, h->Q, (sl.n + sl.G) * sl.ps, p.pcells, s);
  });
  h->tcur = 1 - h->tcur;
  if (cfl) timed(h, XF_PROF_DT, s, [&] { k_dt_finalize<<<1, 1, 0, s>>>(p, h->red, h->dt, nullptr); });
  if (p.viscous) timed(h, XF_PROF_GRAD, s, [&] { h->tab.grad(p, h->Q, s); });
  for (int d = 0; d < p.dim; ++d)
    timed(h, XF_PROF_FACE_X + d, s, [&] {
      faces_of(h->tab, p.weno)[d](p, h->Q, h->G[d], h->flags, h->dt, s);
    });
  timed(h, XF_PROF_UPDATE, s, [&] {
    h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, h->U, h->Us, h->dt, 1, s);
  });
  // stage 2 as in xf_step_rk3
  st = stage_fluxes(h, h->Us, 0, s, true);
  if (st != XF_OK) return st;
  timed(h, XF_PROF_UPDATE, s, [&] {
    h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, h->Us, h->Us, h->dt, 2, s);
  });
  // stage 3: the warm start it leaves goes out during the faces; each slab's
  // U^{n+1} goes out as soon as its faces and update are done
  st = cell_fields(h, h->Us, s);
  if (st != XF_OK) return st;
  if (T_out) {
    XF_CUDA(cudaEventRecord(ev_T, s));
    XF_CUDA(cudaStreamWaitEvent(cs, ev_T, 0));
    XF_CUDA(cudaMemcpyAsync(T_out, h->T[h->tcur], row, cudaMemcpyDefault, cs));
  }
  const FaceRFn* fr = h->tab.face_r[p.weno - 5];
  for (int j = 0; j < S; ++j) {
    const long long z0 = sl.z(j), z1 = sl.z(j + 1);
    for (int d = 0; d < p.dim; ++d) {
      long long b, e;
      if (d == sl.a) {  // face planes (z0, z1], and plane 0 with the first slab
        face_range(p, sl, d, j == 0 ? 0 : z0 + 1, z1 + 1, &b, &e);
      } else {
        face_range(p, sl, d, z0, z1, &b, &e);
      }
      timed(h, XF_PROF_FACE_X + d, s, [&] { fr[d](p, h->Q, h->G[d], h->flags, h->dt, b, e, s); });
    }
    timed(h, XF_PROF_UPDATE, s, [&] {
      h->tab.update_r(p, h->G[0], h->G[1], h->G[2], h->U, h->Us, h->U, h->dt, 3, z0 * sl.cs,
                      z1 * sl.cs, s);
    });
    XF_CUDA(cudaEventRecord(ev[S + j], s));
    XF_CUDA(cudaStreamWaitEvent(cs, ev[S + j], 0));
    const long long c0 = z0 * sl.cs, nc = (z1 - z0) * sl.cs;
    XF_CUDA(cudaMemcpy2DAsync(U_out + c0, row, h->U + c0, row, sizeof(double) * nc, p.nv,
                              cudaMemcpyDefault, cs));
  }
  // the caller's stream sees the copies done
  XF_CUDA(cudaEventRecord(ev_end, cs));
  XF_CUDA(cudaStreamWaitEvent(s, ev_end, 0));
  if (dt_dev_out)
    XF_CUDA(cudaMemcpyAsync(dt_dev_out, h->dt, sizeof(double), cudaMemcpyDeviceToDevice, s));
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_step_rk3_n(xf_handle* h, int nsteps, double dt, void* stream) {
  if (!h || nsteps < 0 || !(dt == dt)) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->prof) {  // event timing cannot sit inside a graph: plain launches
    for (int k = 0; k < nsteps; ++k) {
      xf_status st = step_impl(h, dt, nullptr, s);
      if (st != XF_OK) return st;
    }
    return XF_OK;
  }
  const double key = dt > 0.0 ? dt : 0.0;
  if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->cap = nullptr;
    g_err = "xf_step_rk3_n: capture stream";
    return XF_ERR_CUDA;
  }
  for (int k = 0; k < nsteps; ++k) {
    const int par = h->tcur;
    if (!h->step_graph[par] || h->step_graph_dt[par] != key) {
      if (h->step_graph[par]) cudaGraphExecDestroy(h->step_graph[par]);
      h->step_graph[par] = nullptr;
      // the capture records one step as it would run from this parity; the
      // host-side parity it advanced is put back, the replay advances it
      XF_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
      xf_status st = step_impl(h, key, nullptr, h->cap);
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(h->cap, &g);
      h->tcur = par;
      if (st != XF_OK || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != XF_OK ? st : XF_ERR_CUDA;
      }
      const cudaError_t ei = cudaGraphInstantiate(&h->step_graph[par], g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        h->step_graph[par] = nullptr;
        set_err("cudaGraphInstantiate", ei);
        return XF_ERR_CUDA;
      }
      h->step_graph_dt[par] = key;
    }
    XF_CUDA(cudaGraphLaunch(h->step_graph[par], s));
    h->tcur = 1 - par;  // a step runs three primitive recoveries
  }
  return XF_OK;
}


xf_status xf_get_status(xf_handle* h, uint32_t* flags, void* stream) {
  if (!h) return XF_ERR_ARG;
  uint32_t f = 0;
  XF_CUDA(cudaMemcpyAsync(&f, h->flags, sizeof f, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  XF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (flags) *flags = f;
  if (f & XF_FLAG_NONPHYS) return XF_ERR_NONPHYS;
  if (f & XF_FLAG_NEWTON) return XF_ERR_NEWTON;
  if (f & XF_FLAG_EIGEN) return XF_ERR_EIGEN;
  if (f & XF_FLAG_TIMEOUT) return XF_ERR_TIMEOUT;
  return XF_OK;
}

xf_status xf_clear_status(xf_handle* h, void* stream) {
  if (!h) return XF_ERR_ARG;
  XF_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), (cudaStream_t)stream));
  return XF_OK;
}

xf_status xf_rhs_adjoint(xf_handle* h, const double* U, const double* dUdt_bar, double* U_bar,
                         void* stream) {
  if (!h || !U || !dUdt_bar || !U_bar) return XF_ERR_ARG;
  if (!is_device_ptr(U) || !is_device_ptr(dUdt_bar) || !is_device_ptr(U_bar)) return XF_ERR_ARG;
  return rhs_adjoint_impl(h, U, dUdt_bar, 1.0, U_bar, (cudaStream_t)stream);
}

// The two extra per-cell field blocks of the step adjoints (allocated on
// first use, kept with the handle).
static xf_status ensure_stage_fields(xf_handle* h) {
  const size_t qbytes = sizeof(double) * nq_of(h->tab, h->p) * h->p.pcells;
  for (int k = 0; k < 2; ++k) {
    if (!h->QS[k] && cudaMalloc((void**)&h->QS[k], qbytes) != cudaSuccess) {
      cudaGetLastError();
      h->QS[k] = nullptr;
      g_err = "step adjoint buffers: cudaMalloc failed";
      return XF_ERR_OOM;
    }
  }
  return XF_OK;
}

// Restores the handle's own field block on every return of a step adjoint.
struct QGuard {
  xf_handle* h;
  double* q;
  ~QGuard() { h->Q = q; }
};

xf_status xf_step_rk3_adjoint(xf_handle* h, double dt, double* U_bar, void* stream) {
  if (!h || !U_bar || !(dt > 0.0)) return XF_ERR_ARG;
  if (!is_device_ptr(U_bar)) return XF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  xf_status st = ensure_adjoint_buffers(h);
  if (st != XF_OK) return st;
  const xf::Params& p = h->p;
  st = ensure_stage_fields(h);
  if (st != XF_OK) return st;
  // the forward passes write U^n's and U1's per-cell fields into QS[0], QS[1];
  // h->Q is restored on every return
  QGuard guard{h, h->Q};
  k_set_scalar<<<1, 1, 0, s>>>(h->dt, dt);
  // forward stage states U1 (A1) and U2 (A2) from U^n (h->U)
  h->Q = h->QS[0];
  st = stage_fluxes(h, h->U, 0, s, true);
  if (st != XF_OK) return st;
  h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, h->U, h->A1, h->dt, 1, s);
  h->Q = h->QS[1];
  st = stage_fluxes(h, h->A1, 0, s, true);
  if (st != XF_OK) return st;
  h->tab.update(p, h->G[0], h->G[1], h->G[2], h->U, h->A1, h->A2, h->dt, 2, s);
  // reverse of U3 = U/3 + 2/3 (U2 + dt L(U2)), U2 = 3/4 U + 1/4 (U1 + dt L(U1)),
  // U1 = U + dt L(U); a = Ubar(U3) on entry
  lincomb(h, 2.0 / 3.0, U_bar, 0.0, nullptr, 0.0, nullptr, h->B2, s);
  h->Q = guard.q;
  st = rhs_adjoint_impl(h, h->A2, U_bar, 2.0 / 3.0 * dt, h->B2, s, false, h->dt);
  if (st != XF_OK) return st;
  lincomb(h, 0.25, h->B2, 0.0, nullptr, 0.0, nullptr, h->B1, s);
  h->Q = h->QS[1];
  st = rhs_adjoint_impl(h, h->A1, h->B2, 0.25 * dt, h->B1, s, true, h->dt);
  if (st != XF_OK) return st;
  lincomb(h, 1.0 / 3.0, U_bar, 0.75, h->B2, 1.0, h->B1, U_bar, s);
  h->Q = h->QS[0];
  st = rhs_adjoint_impl(h, h->U, h->B1, dt, U_bar, s, true, h->dt);
  if (st != XF_OK) return st;
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_step_rk3_tape(xf_handle* h, double dt, double* U1, double* U2, void* stream) {
  if (!h || !U1 || !U2 || U1 == U2 || !(dt > 0.0)) return XF_ERR_ARG;
  if (!is_device_ptr(U1) || !is_device_ptr(U2)) return XF_ERR_ARG;
  return step_impl(h, dt, nullptr, (cudaStream_t)stream, U1, U2);
}

static xf_status step_adjoint_tape_impl(xf_handle* h, double dt, const double* U1,
                                        const double* U2, const double* Fhat, double* U_bar,
                                        cudaStream_t s) {
  const long long tl = tape_stage_len(h->p);
  const double* F0 = Fhat;
  const double* F1 = Fhat ? Fhat + tl : nullptr;
  const double* F2 = Fhat ? Fhat + 2 * tl : nullptr;
  xf_status st = ensure_adjoint_buffers(h);
  if (st != XF_OK) return st;
  st = ensure_stage_fields(h);
  if (st != XF_OK) return st;
  QGuard guard{h, h->Q};
  k_set_scalar<<<1, 1, 0, s>>>(h->dt, dt);
  // the three stages' per-cell fields in the forward step's order, so that
  // each Newton solve starts from the warm start the forward step gave it
  // and the fields are bitwise those the forward faces saw
  h->Q = h->QS[0];
  st = cell_fields(h, h->U, s);
  if (st != XF_OK) return st;
  h->Q = h->QS[1];
  st = cell_fields(h, U1, s);
  if (st != XF_OK) return st;
  h->Q = guard.q;
  st = cell_fields(h, U2, s);
  if (st != XF_OK) return st;
  // the reverse of xf_step_rk3_adjoint on those fields
  lincomb(h, 2.0 / 3.0, U_bar, 0.0, nullptr, 0.0, nullptr, h->B2, s);
  st = rhs_adjoint_impl(h, U2, U_bar, 2.0 / 3.0 * dt, h->B2, s, true, h->dt, F2);
  if (st != XF_OK) return st;
  lincomb(h, 0.25, h->B2, 0.0, nullptr, 0.0, nullptr, h->B1, s);
  h->Q = h->QS[1];
  st = rhs_adjoint_impl(h, U1, h->B2, 0.25 * dt, h->B1, s, true, h->dt, F1);
  if (st != XF_OK) return st;
  lincomb(h, 1.0 / 3.0, U_bar, 0.75, h->B2, 1.0, h->B1, U_bar, s);
  h->Q = h->QS[0];
  st = rhs_adjoint_impl(h, h->U, h->B1, dt, U_bar, s, true, h->dt, F0);
  if (st != XF_OK) return st;
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_step_rk3_adjoint_tape(xf_handle* h, double dt, const double* U1, const double* U2,
                                   double* U_bar, void* stream) {
  if (!h || !U1 || !U2 || !U_bar || !(dt > 0.0)) return XF_ERR_ARG;
  if (!is_device_ptr(U1) || !is_device_ptr(U2) || !is_device_ptr(U_bar)) return XF_ERR_ARG;
  return step_adjoint_tape_impl(h, dt, U1, U2, nullptr, U_bar, (cudaStream_t)stream);
}

int64_t xf_tape_flux_len(const xf_handle* h) {
  return h ? (int64_t)(3 * tape_stage_len(h->p)) : -1;
}

xf_status xf_step_rk3_tape_flux(xf_handle* h, double dt, double* U1, double* U2, double* Fhat,
                                void* stream) {
  if (!h || !U1 || !U2 || !Fhat || U1 == U2 || !(dt > 0.0)) return XF_ERR_ARG;
  if (!is_device_ptr(U1) || !is_device_ptr(U2) || !is_device_ptr(Fhat)) return XF_ERR_ARG;
  return step_impl(h, dt, nullptr, (cudaStream_t)stream, U1, U2, Fhat);
}

xf_status xf_step_rk3_adjoint_tape_flux(xf_handle* h, double dt, const double* U1,
                                        const double* U2, const double* Fhat, double* U_bar,
                                        void* stream) {
  if (!h || !U1 || !U2 || !Fhat || !U_bar || !(dt > 0.0)) return XF_ERR_ARG;
  if (!is_device_ptr(U1) || !is_device_ptr(U2) || !is_device_ptr(Fhat) || !is_device_ptr(U_bar))
    return XF_ERR_ARG;
  return step_adjoint_tape_impl(h, dt, U1, U2, Fhat, U_bar, (cudaStream_t)stream);
}

xf_status xf_objective_mixing(xf_handle* h, const double* U, int species, double* J_dev,
                              double* U_bar, void* stream) {
  if (!h || !U || !J_dev || !U_bar || species < 0 || species >= h->p.N) return XF_ERR_ARG;
  if (!is_device_ptr(U) || !is_device_ptr(J_dev) || !is_device_ptr(U_bar)) return XF_ERR_ARG;
  xf_status st = ensure_adjoint_buffers(h);
  if (st != XF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const xf::Params& p = h->p;
  double dV = 1.0;
  for (int a = 0; a < p.dim; ++a) dV /= p.inv_dx[a];
  h->tab.adj.mixing(p, U, species, dV, h->part, U_bar, s);
  k_sum_partials<<<1, 256, 0, s>>>(h->part, (int)blocks(p.cells, 256), J_dev);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_set_primitive_adjoint(xf_handle* h, const double* P, const double* U_bar,
                                   double* P_bar, void* stream) {
  if (!h || !P || !U_bar || !P_bar) return XF_ERR_ARG;
  if (!is_device_ptr(P) || !is_device_ptr(U_bar) || !is_device_ptr(P_bar)) return XF_ERR_ARG;
  h->tab.adj.from_prim_adj(h->p, P, U_bar, P_bar, (cudaStream_t)stream);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_profile_enable(xf_handle* h, int on) {
  if (!h) return XF_ERR_ARG;
  h->prof = on != 0;
  return XF_OK;
}

xf_status xf_profile_read(xf_handle* h, double* ms, int64_t* launches) {
  if (!h || !ms || !launches) return XF_ERR_ARG;
  for (int k = 0; k < XF_PROF_SLOTS; ++k) { ms[k] = 0.0; launches[k] = 0; }
  xf_status st = XF_OK;
  for (auto& r : h->recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) {
      set_err("xf_profile_read", e);
      st = XF_ERR_CUDA;
    } else {
      ms[r.slot] += t;
      launches[r.slot] += 1;
    }
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  h->recs.clear();
  return st;
}

xf_status xf_probe_rcp(const double* x, double* y, double* ref, int64_t n, void* stream) {
  if (!x || !y || !ref || n < 0) return XF_ERR_ARG;
  if (n == 0) return XF_OK;
  if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(ref)) return XF_ERR_ARG;
  k_probe_rcp<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(x, y, ref, n);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_probe_exp(const double* x, double* y, double* ref, int64_t n, void* stream) {
  if (!x || !y || !ref || n < 0) return XF_ERR_ARG;
  if (n == 0) return XF_OK;
  if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(ref)) return XF_ERR_ARG;
  k_probe_exp<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(x, y, ref, n);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_probe_log(const double* x, double* y, double* ref, int64_t n, void* stream) {
  if (!x || !y || !ref || n < 0) return XF_ERR_ARG;
  if (n == 0) return XF_OK;
  if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(ref)) return XF_ERR_ARG;
  k_probe_log<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(x, y, ref, n);
  XF_CUDA(cudaGetLastError());
  return XF_OK;
}

xf_status xf_probe_fp64(int64_t iters, int blocks_per_sm, double* tflops) {
  if (iters < 1 || blocks_per_sm < 1 || !tflops) return XF_ERR_ARG;
  int dev = 0, sms = 0;
  XF_CUDA(cudaGetDevice(&dev));
  XF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* out = nullptr;
  XF_CUDA(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int threads = 256;
  const long long nb = (long long)sms * blocks_per_sm;
  k_probe_fp64<<<(unsigned)nb, threads>>>(out, iters / 10 + 1, 1.0 - 1e-9);  // warm-up
  cudaEventRecord(a);
  k_probe_fp64<<<(unsigned)nb, threads>>>(out, iters, 1.0 - 1e-9);
  cudaEventRecord(b);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) {
    set_err("xf_probe_fp64", e);
    return XF_ERR_CUDA;
  }
  const double flops = 2.0 * 8.0 * (double)iters * (double)(nb * threads);
  *tflops = flops / (ms * 1e-3) / 1e12;
  return XF_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free right-hand side (xf_rhs_static). Scratch for the padded
// per-cell fields, the face fluxes, the temperature warm start and the status
// word lives in one file-scope device array of fixed size instead of memory
// obtained from cudaMalloc. Host code never uses the array's name as a device
// address: each device's address comes from cudaGetSymbolAddress, looked up on
// that device's first call and cached.
namespace {

constexpr size_t kStaticScratchDoubles = size_t(4) << 20;  // 32 MiB per device
static __device__ __align__(256) double xf_static_scratch[kStaticScratchDoubles];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kStaticMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on first use).
xf_status static_scratch(double** out) {
  int dev = 0;
  XF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) {
    g_err = "xf_rhs_static: device ordinal beyond the supported range";
    return XF_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    XF_CUDA(cudaGetSymbolAddress(&ptr, xf_static_scratch));
    g_static_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_static_ptr[dev];
  return XF_OK;
}

}  // namespace

extern "C" {

int64_t xf_rhs_static_capacity_bytes(void) {
  return (int64_t)(kStaticScratchDoubles * sizeof(double));
}

xf_status xf_rhs_static(const xf_grid* grid, const xf_thermo* thermo, const xf_opts* opts,
                        const double* U, const double* T_guess, double* dUdt,
                        uint32_t* flags_out, void* stream) {
  if (!U || !dUdt) {
    g_err = "xf_rhs_static: U and dUdt must not be null";
    return XF_ERR_ARG;
  }
  xf::Params p;
  xf_status st = fill_params(grid, thermo, opts, &p);
  if (st != XF_OK) {
    g_err = "xf_rhs_static: invalid grid, thermo tables or options";
    return st;
  }
  Table tab;
  if (!pick(p.dim, p.N, &tab)) {
    g_err = "xf_rhs_static: unsupported dimension and species count";
    return XF_ERR_ARG;
  }
  if (!is_device_ptr(U) || !is_device_ptr(dUdt) || (T_guess && !is_device_ptr(T_guess))) {
    g_err = "xf_rhs_static: U, dUdt and T_guess must be device pointers";
    return XF_ERR_ARG;
  }
  // scratch plan (in doubles): Params | Q | G_x | G_y | G_z | T_in | T_out | dt | red[2] |
  // flags, the Params slot rounded up to 256 bytes
  constexpr size_t kParamSlot = (sizeof(xf::Params) + 255) / 256 * 32;
  long long nf[3] = {0, 0, 0};
  size_t need = kParamSlot + nq_of(tab, p) * p.pcells;
  for (int d = 0; d < p.dim; ++d) {
    nf[d] = (long long)(p.n[0] + (d == 0)) * (p.n[1] + (d == 1)) * (p.n[2] + (d == 2));
    need += (size_t)p.nv * nf[d];
  }
  need += 2 * (size_t)p.cells + 1 + 2 + 1;
  if (need > kStaticScratchDoubles) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "xf_rhs_static: this grid needs %zu bytes of scratch; the static scratch holds "
             "%zu bytes",
             need * sizeof(double), kStaticScratchDoubles * sizeof(double));
    g_err = buf;
    return XF_ERR_ARG;
  }
  double* base = nullptr;
  st = static_scratch(&base);
  if (st != XF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  p.dev = reinterpret_cast<const xf::Params*>(base);
  double* Q = base + kParamSlot;
  double* cur = Q + nq_of(tab, p) * p.pcells;
  double* G[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < p.dim; ++d) {
    G[d] = cur;
    cur += (size_t)p.nv * nf[d];
  }
  double* Tin = cur;
  double* Tout = Tin + p.cells;
  double* dt = Tout + p.cells;
  unsigned long long* red = reinterpret_cast<unsigned long long*>(dt + 1);
  uint32_t* flags = reinterpret_cast<uint32_t*>(dt + 3);
  // the parameters' device copy (from pageable memory: staged before the call
  // returns); the array keeps the previous call's contents: zero the accumulators
  XF_CUDA(cudaMemcpyAsync(base, &p, sizeof(xf::Params), cudaMemcpyHostToDevice, s));
  XF_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), s));
  XF_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
  if (T_guess) {
    XF_CUDA(cudaMemcpyAsync(Tin, T_guess, sizeof(double) * p.cells, cudaMemcpyDeviceToDevice, s));
  } else {
    k_fill<<<blocks(p.cells, 256), 256, 0, s>>>(Tin, p.cells, 300.0);
  }
  tab.prim(p, U, Tin, Tout, Q, flags, red, 0, s);
  if (p.viscous) tab.grad(p, Q, s);
  for (int d = 0; d < p.dim; ++d) faces_of(tab, p.weno)[d](p, Q, G[d], flags, nullptr, s);
  tab.update(p, G[0], G[1], G[2], nullptr, nullptr, dUdt, dt, 0, s);
  XF_CUDA(cudaGetLastError());
  if (flags_out) {
    XF_CUDA(cudaMemcpyAsync(flags_out, flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    XF_CUDA(cudaStreamSynchronize(s));
  }
  return XF_OK;
}

}  // extern "C"
