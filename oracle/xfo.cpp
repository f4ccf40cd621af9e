// xfo.cpp -- CPU oracle for the multicomponent RHS / SSP-RK3 stage
// (TEST INFRASTRUCTURE ONLY; see xfo.h). Plain FP64, ghost-cell arrays,
// dense eigen-matrices (the full-eigensystem "EEO" route of Sec. III.D.3),
// serial loops with OpenMP only over independent cells/faces.
//
// Every function is templated on the scalar S so that a forward-mode dual
// number (Dual<K>) gives exact Jacobian-vector products through the same code.
//
// Readings where the paper is silent or garbled are marked "Reading:".
#include "xfo.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kRu = 8.314462618;  // J/(mol K), Eq. 7
// ghost layers: the flux at i+1/2 reads cells i-G+1 .. i+G (WENO5 and
// WENO-CU6: 6 cells; WENO7: 8 cells)
inline int ghosts(int weno) { return weno == 7 ? 4 : 3; }

// ------------------------------------------------------------ dual numbers --
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0.0) { for (int k = 0; k < K; ++k) d[k] = 0.0; }
  Dual(double x) : v(x) { for (int k = 0; k < K; ++k) d[k] = 0.0; }  // NOLINT
};
template <int K> Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v + b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v - b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r; r.v = -a.v; for (int k = 0; k < K; ++k) r.d[k] = -a.d[k]; return r; }
template <int K> Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v * b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int K> Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v / b.v;
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
  return r; }
template <int K> Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> Dual<K> operator*(const Dual<K>& a, double b) {
  Dual<K> r; r.v = a.v * b; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b; return r; }
template <int K> Dual<K> operator*(double a, const Dual<K>& b) { return b * a; }
template <int K> Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> Dual<K>& operator+=(Dual<K>& a, const Dual<K>& b) { a = a + b; return a; }
template <int K> Dual<K>& operator-=(Dual<K>& a, const Dual<K>& b) { a = a - b; return a; }
template <int K> Dual<K>& operator*=(Dual<K>& a, const Dual<K>& b) { a = a * b; return a; }
template <int K> bool operator<(const Dual<K>& a, const Dual<K>& b) { return a.v < b.v; }
template <int K> bool operator>(const Dual<K>& a, const Dual<K>& b) { return a.v > b.v; }
template <int K> bool operator<(const Dual<K>& a, double b) { return a.v < b; }
template <int K> bool operator>(const Dual<K>& a, double b) { return a.v > b; }
template <int K> bool operator<=(const Dual<K>& a, double b) { return a.v <= b; }
template <int K> Dual<K> sqrt(const Dual<K>& a) {
  Dual<K> r; r.v = std::sqrt(a.v); for (int k = 0; k < K; ++k) r.d[k] = a.d[k] / (2.0 * r.v); return r; }
template <int K> Dual<K> exp(const Dual<K>& a) {
  Dual<K> r; r.v = std::exp(a.v); for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * r.v; return r; }
template <int K> Dual<K> log(const Dual<K>& a) {
  Dual<K> r; r.v = std::log(a.v); for (int k = 0; k < K; ++k) r.d[k] = a.d[k] / a.v; return r; }
// d|x|/dx = sign(x), taken as 0 at x = 0
template <int K> Dual<K> fabs(const Dual<K>& a) {
  if (a.v > 0.0) return a;
  if (a.v < 0.0) return -a;
  return Dual<K>(0.0); }

inline double val(double x) { return x; }
template <int K> double val(const Dual<K>& x) { return x.v; }
using std::exp; using std::fabs; using std::log; using std::sqrt;

using D8 = Dual<XFO_KDIR>;

// first maximum wins on ties
template <class S> S max_first(const S& a, const S& b) { return (b > a) ? b : a; }

// ------------------------------------------------------------ layout -------
struct Layout {
  int dim, N, nv, G;
  int64_t n[3], np[3], cells, pcells;
  double dx[3];
  int iE() const { return 1 + dim; }
  int iY(int s) const { return 2 + dim + s; }
  explicit Layout(const xfo_params& p) {
    dim = p.dim; N = p.N; nv = dim + 2 + N - 1; G = ghosts(p.weno);
    cells = 1; pcells = 1;
    for (int a = 0; a < 3; ++a) {
      n[a] = (a < dim) ? p.n[a] : 1;
      np[a] = (a < dim) ? n[a] + 2 * G : 1;
      cells *= n[a]; pcells *= np[a];
      dx[a] = (a < dim) ? (p.hi[a] - p.lo[a]) / (double)p.n[a] : 1.0;
    }
  }
  int64_t g(int64_t i, int64_t j, int64_t k) const {  // interior index
    return (k * n[1] + j) * n[0] + i; }
  int64_t pg(int64_t i, int64_t j, int64_t k) const {  // padded index, i in [-G, n+G)
    int64_t oi = dim > 0 ? G : 0, oj = dim > 1 ? G : 0, ok = dim > 2 ? G : 0;
    return ((k + ok) * np[1] + (j + oj)) * np[0] + (i + oi); }
};

// Ghost mapping of one axis: interior source index and whether the normal
// velocity of that axis flips sign (symmetric wall).
inline int64_t map_axis(int64_t i, int64_t n, int bclo, int bchi, bool* flip) {
  *flip = false;
  if (i >= 0 && i < n) return i;
  int bc = (i < 0) ? bclo : bchi;
  if (bc == XFO_BC_PERIODIC) return (i < 0) ? i + n : i - n;
  if (bc == XFO_BC_SYMMETRIC) { *flip = true; return (i < 0) ? -1 - i : 2 * n - 1 - i; }
  return (i < 0) ? 0 : n - 1;  // transmissive: zero-gradient copy
}

// ------------------------------------------------------------ thermo -------
struct Thermo {
  int N;
  double Rs[XFO_MAXN];  // R_s / a_ref^2  (1/K)
  double W[XFO_MAXN];
  const xfo_params* p;
  explicit Thermo(const xfo_params& pp) : N(pp.N), p(&pp) {
    for (int s = 0; s < N; ++s) { Rs[s] = kRu / pp.W[s] / pp.a_ref2; W[s] = pp.W[s]; }
  }
  // c_p,s / R_s at T: the degree-4 polynomial in tau on [T_lo, T_hi], held at
  // its end values outside (Reading: the paper gives no extrapolation rule).
  template <class S> S cpR(int s, const S& T) const {
    S tau = (T - p->T_lo) / (p->T_hi - p->T_lo);
    if (tau < 0.0) tau = S(0.0);
    if (tau > 1.0) tau = S(1.0);
    S sum(0.0), pw(1.0);
    for (int j = 0; j < 5; ++j) { sum = sum + p->cp[s][j] * pw; pw = pw * tau; }
    return sum;
  }
  // h_s / R_s (K): h_off + integral of c_p/R from T_lo, continued linearly with
  // the end-point c_p outside the range.
  template <class S> S hR(int s, const S& T) const {
    double span = p->T_hi - p->T_lo;
    S tau = (T - p->T_lo) / span;
    if (tau < 0.0) return p->h_off[s] + p->cp[s][0] * span * tau;
    if (tau > 1.0) {
      double top = 0.0, cp1 = 0.0;
      for (int j = 0; j < 5; ++j) { top += p->cp[s][j] / (j + 1); cp1 += p->cp[s][j]; }
      return p->h_off[s] + span * top + cp1 * span * (tau - 1.0);
    }
    S sum(0.0), pw = tau;
    for (int j = 0; j < 5; ++j) { sum = sum + (p->cp[s][j] / (j + 1)) * pw; pw = pw * tau; }
    return p->h_off[s] + span * sum;
  }
  template <class S> S e_s(int s, const S& T) const { return Rs[s] * (hR(s, T) - T); }
  template <class S> S h_s(int s, const S& T) const { return Rs[s] * hR(s, T); }
  template <class S> S cv_s(int s, const S& T) const { return Rs[s] * (cpR(s, T) - 1.0); }
  template <class S> S cp_s(int s, const S& T) const { return Rs[s] * cpR(s, T); }
};

// Newton iteration of Eq. 21 for T(e, Y), warm-started at T0.
// Stop when |T_{k+1} - T_k| <= rtol T_{k+1}; a non-positive iterate is replaced
// by half the previous one (Reading: safeguard the paper does not state).
template <class S>
S newton_T(const Thermo& th, const xfo_params& p, const S& e, const S* Y, double T0,
           int* iters, uint32_t* st) {
  S T(T0);
  bool conv = false;
  int it = 0;
  for (; it < p.newton_max; ++it) {
    S eT(0.0), cv(0.0);
    for (int s = 0; s < th.N; ++s) { eT = eT + Y[s] * th.e_s(s, T); cv = cv + Y[s] * th.cv_s(s, T); }
    S Tn = T + (e - eT) / cv;
    if (!(val(Tn) > 0.0)) Tn = 0.5 * T;
    conv = std::fabs(val(Tn) - val(T)) <= p.newton_rtol * val(Tn);
    T = Tn;
    if (conv) { ++it; break; }
  }
  if (!conv) *st |= XFO_FLAG_NEWTON;
  if (iters) *iters = it;
  return T;
}

// ------------------------------------------------------------ cell state ---
template <class S>
struct Prim {
  S rho, u[3], p, T, c2, c, H, E, cv, cp, Rm;
  S Y[XFO_MAXN];
  S mu, kap, D;
  S Ds[XFO_MAXN];  // per-species diffusion coefficients of the selected model
  S U[XFO_MAXV];  // conserved values of this (possibly ghost) cell
};

// Primitive recovery of one cell (Eq. 7, Eq. 21): rho, u = m/rho, Y_s, Y_N =
// 1 - sum, e = E/rho - |u|^2/2, Newton T, p = rho R T, c^2 = (cp/cv) p/rho,
// H = (E + p)/rho.
template <class S>
void recover(const Layout& L, const Thermo& th, const xfo_params& p, const S* Uc,
             double Twarm, Prim<S>& q, uint32_t* st) {
  bool finite = true;
  for (int v = 0; v < L.nv; ++v) { q.U[v] = Uc[v]; finite = finite && std::isfinite(val(Uc[v])); }
  q.rho = Uc[0];
  S ke(0.0);
  for (int a = 0; a < 3; ++a) q.u[a] = S(0.0);
  for (int a = 0; a < L.dim; ++a) { q.u[a] = Uc[1 + a] / q.rho; ke = ke + q.u[a] * q.u[a]; }
  q.E = Uc[L.iE()];
  S ysum(0.0);
  for (int s = 0; s < L.N - 1; ++s) { q.Y[s] = Uc[L.iY(s)] / q.rho; ysum = ysum + q.Y[s]; }
  q.Y[L.N - 1] = 1.0 - ysum;
  S e = q.E / q.rho - 0.5 * ke;
  q.T = newton_T(th, p, e, q.Y, Twarm, nullptr, st);
  S Rm(0.0), cv(0.0), cp(0.0);
  for (int s = 0; s < L.N; ++s) {
    Rm = Rm + q.Y[s] * th.Rs[s];
    cv = cv + q.Y[s] * th.cv_s(s, q.T);
    cp = cp + q.Y[s] * th.cp_s(s, q.T);
  }
  q.Rm = Rm; q.cv = cv; q.cp = cp;
  q.p = q.rho * Rm * q.T;
  q.c2 = (cp / cv) * q.p / q.rho;
  q.c = sqrt(q.c2);
  q.H = (q.E + q.p) / q.rho;
  if (!finite || !(val(q.rho) > 0.0) || !(val(q.p) > 0.0) || !(val(q.T) > 0.0))
    *st |= XFO_FLAG_NONPHYS;
}

// Mixture transport of one cell: Eq. 29 fits for mu_s and kappa_s, the Wilke
// rule of Eq. 22 for mu and kappa, and the species diffusivities D_s: either
// a constant-Lewis-number D = kappa/(rho c_p Le) for every species, or the
// mixture-averaged D_sm of Eq. 26 from the binary D_st of Eq. 25 (fits of
// ln(p D_st) in ln T, the form of Eq. 29). Reading for Eq. 26: the mole
// fractions enter as X~_t = (max(X_t, 0) + 1e-12) normalised to sum 1, which
// keeps D_sm finite in pure species s (where Eq. 26 is 0/0) and changes
// nothing above round-off elsewhere. Returned dimensionless.
template <class S>
void transport(const Thermo& th, const xfo_params& p, Prim<S>& q) {
  int N = th.N;
  S lnT = log(q.T);
  S mus[XFO_MAXN], kas[XFO_MAXN], X[XFO_MAXN];
  S ysw(0.0);
  for (int s = 0; s < N; ++s) {
    S lm(0.0), lk(0.0), pw(1.0);
    for (int j = 0; j < 4; ++j) { lm = lm + p.mu[s][j] * pw; lk = lk + p.kap[s][j] * pw; pw = pw * lnT; }
    mus[s] = exp(lm);
    kas[s] = exp(lk);
    ysw = ysw + q.Y[s] / th.W[s];
  }
  for (int s = 0; s < N; ++s) X[s] = (q.Y[s] / th.W[s]) / ysw;
  auto wilke = [&](const S* al) {
    S mix(0.0);
    for (int s = 0; s < N; ++s) {
      S den(0.0);
      for (int t = 0; t < N; ++t) {
        S ph = (1.0 / std::sqrt(8.0)) * std::pow(1.0 + th.W[s] / th.W[t], -0.5);
        S br = 1.0 + sqrt(al[s] / al[t]) * std::pow(th.W[t] / th.W[s], 0.25);
        den = den + X[t] * (ph * br * br);
      }
      mix = mix + X[s] * al[s] / den;
    }
    return mix;
  };
  double a_ref = std::sqrt(p.a_ref2);
  q.mu = wilke(mus) / (p.rho_ref * a_ref * p.L_ref);
  q.kap = wilke(kas) / (p.rho_ref * a_ref * p.a_ref2 * p.L_ref);
  q.D = q.kap / (q.rho * q.cp * p.lewis);
  if (p.diffusion == 1) {
    S Xt[XFO_MAXN], xs(0.0);
    for (int t = 0; t < N; ++t) {
      Xt[t] = (X[t] > 0.0 ? X[t] : S(0.0)) + 1e-12;
      xs = xs + Xt[t];
    }
    S Wb(0.0);
    for (int t = 0; t < N; ++t) { Xt[t] = Xt[t] / xs; Wb = Wb + Xt[t] * th.W[t]; }
    S pd = q.rho * q.Rm * q.T * (p.rho_ref * p.a_ref2);  // pressure in Pa
    for (int s = 0; s < N; ++s) {
      S num(0.0), den(0.0);
      for (int t = 0; t < N; ++t) {
        if (t == s) continue;
        S l(0.0), pw(1.0);
        for (int j = 0; j < 4; ++j) { l = l + p.dbin[s][t][j] * pw; pw = pw * lnT; }
        S Dst = exp(l) / pd;  // m^2/s
        num = num + Xt[t] * th.W[t];
        den = den + Xt[t] / Dst;
      }
      q.Ds[s] = num / (Wb * den) / (a_ref * p.L_ref);
    }
  } else {
    for (int s = 0; s < N; ++s) q.Ds[s] = q.D;
  }
}

// Physical flux of direction d (Eq. 2) from the cell primitives.
template <class S>
void phys_flux(const Layout& L, const Prim<S>& q, int d, S* F) {
  S un = q.u[d];
  F[0] = q.rho * un;
  for (int a = 0; a < L.dim; ++a) F[1 + a] = q.rho * un * q.u[a] + (a == d ? q.p : S(0.0));
  F[L.iE()] = (q.E + q.p) * un;
  for (int s = 0; s < L.N - 1; ++s) F[L.iY(s)] = q.rho * q.Y[s] * un;
}

// ------------------------------------------------------- eigensystem ------
// Dense face eigensystem of direction d between states qa (left) and qb
// (right), in storage order. Reading of the "multicomponent Roe average":
// sqrt(rho) weights for u, H, Y_s, T; Gamma = R/c_v(T, Y); phi_s = R_s T -
// Gamma (e_s(T) - |u|^2/2); c^2 = sum Y_s phi_s + Gamma (H - |u|^2).
// Columns/rows k: 0 = u-c, 1 = u+c, 2 = entropy, 3.. = tangential momenta,
// then species s = 1..N-1. lamtype[k]: 0 u-c, 1 u+c, 2 u.
template <class S>
void eigen(const Layout& L, const Thermo& th, const Prim<S>& qa, const Prim<S>& qb, int d,
           S* Lm, S* Rm, S* lam, int* lamtype, S* c2out, uint32_t* st) {
  int nv = L.nv, N = L.N, dim = L.dim;
  S wa = sqrt(qa.rho), wb = sqrt(qb.rho);
  S ta = wa / (wa + wb), tb = wb / (wa + wb);
  S u[3], Y[XFO_MAXN];
  S q2(0.0);
  for (int a = 0; a < 3; ++a) u[a] = S(0.0);
  for (int a = 0; a < dim; ++a) { u[a] = ta * qa.u[a] + tb * qb.u[a]; q2 = q2 + u[a] * u[a]; }
  S H = ta * qa.H + tb * qb.H;
  S T = ta * qa.T + tb * qb.T;
  for (int s = 0; s < N; ++s) Y[s] = ta * qa.Y[s] + tb * qb.Y[s];
  S Rbar(0.0), cv(0.0);
  for (int s = 0; s < N; ++s) { Rbar = Rbar + Y[s] * th.Rs[s]; cv = cv + Y[s] * th.cv_s(s, T); }
  S Gam = Rbar / cv;
  S phi[XFO_MAXN];
  for (int s = 0; s < N; ++s) phi[s] = th.Rs[s] * T - Gam * (th.e_s(s, T) - 0.5 * q2);
  S c2(0.0);
  for (int s = 0; s < N; ++s) c2 = c2 + Y[s] * phi[s];
  c2 = c2 + Gam * (H - q2);
  if (!(val(c2) > 0.0)) {  // Reading: flag and fall back to the mean cell c^2
    *st |= XFO_FLAG_EIGEN;
    c2 = 0.5 * (qa.c2 + qb.c2);
  }
  *c2out = c2;
  S c = sqrt(c2);
  for (int i = 0; i < nv * nv; ++i) { Lm[i] = S(0.0); Rm[i] = S(0.0); }
  // p-gradient g = dp/dU
  S g[XFO_MAXV];
  g[0] = phi[N - 1];
  for (int a = 0; a < dim; ++a) g[1 + a] = -Gam * u[a];
  g[L.iE()] = Gam;
  for (int s = 0; s < N - 1; ++s) g[L.iY(s)] = phi[s] - phi[N - 1];
  int im = 1 + d;
  // right eigenvectors (columns)
  for (int sg = 0; sg < 2; ++sg) {  // k = 0: u - c, k = 1: u + c
    double sgn = sg == 0 ? -1.0 : 1.0;
    int k = sg;
    Rm[0 * nv + k] = S(1.0);
    for (int a = 0; a < dim; ++a) Rm[(1 + a) * nv + k] = u[a] + (a == d ? sgn * c : S(0.0));
    Rm[L.iE() * nv + k] = H + sgn * u[d] * c;
    for (int s = 0; s < N - 1; ++s) Rm[L.iY(s) * nv + k] = Y[s];
  }
  Rm[0 * nv + 2] = S(1.0);
  for (int a = 0; a < dim; ++a) Rm[(1 + a) * nv + 2] = u[a];
  Rm[L.iE() * nv + 2] = H - c2 / Gam;
  for (int s = 0; s < N - 1; ++s) Rm[L.iY(s) * nv + 2] = Y[s];
  int k = 3;
  int tang[2], nt = 0;
  for (int a = 0; a < dim; ++a) if (a != d) tang[nt++] = a;
  for (int t = 0; t < nt; ++t, ++k) {
    Rm[(1 + tang[t]) * nv + k] = S(1.0);
    Rm[L.iE() * nv + k] = u[tang[t]];
  }
  int kspec = k;
  for (int s = 0; s < N - 1; ++s) {
    Rm[L.iE() * nv + kspec + s] = -(phi[s] - phi[N - 1]) / Gam;
    Rm[L.iY(s) * nv + kspec + s] = S(1.0);
  }
  // left eigenvectors (rows)
  S inv2c2 = 1.0 / (2.0 * c2);
  for (int sg = 0; sg < 2; ++sg) {
    double sgn = sg == 0 ? -1.0 : 1.0;
    for (int j = 0; j < nv; ++j) {
      S vj(0.0);
      if (j == 0) vj = -u[d];
      if (j == im) vj = S(1.0);
      Lm[sg * nv + j] = (g[j] + sgn * c * vj) * inv2c2;
    }
  }
  for (int j = 0; j < nv; ++j) Lm[2 * nv + j] = (j == 0 ? S(1.0) : S(0.0)) - g[j] / c2;
  k = 3;
  for (int t = 0; t < nt; ++t, ++k) {
    Lm[k * nv + 0] = -u[tang[t]];
    Lm[k * nv + 1 + tang[t]] = S(1.0);
  }
  for (int s = 0; s < N - 1; ++s) {
    Lm[(kspec + s) * nv + 0] = -Y[s];
    Lm[(kspec + s) * nv + L.iY(s)] = S(1.0);
  }
  for (int kk = 0; kk < nv; ++kk) {
    lamtype[kk] = kk < 2 ? kk : 2;
    lam[kk] = kk == 0 ? u[d] - c : (kk == 1 ? u[d] + c : u[d]);
  }
}

// WENO5-JS reconstruction at i+1/2 from f[0..4] = f_{i-2..i+2}.
// Reading: the Jiang-Shu smoothness indicators, linear weights (0.1, 0.6, 0.3)
// and an absolute epsilon (1e-6 by default) on dimensionless data.
template <class S>
S weno5(const S* f, double eps) {
  S b0 = (13.0 / 12.0) * (f[0] - 2.0 * f[1] + f[2]) * (f[0] - 2.0 * f[1] + f[2]) +
         0.25 * (f[0] - 4.0 * f[1] + 3.0 * f[2]) * (f[0] - 4.0 * f[1] + 3.0 * f[2]);
  S b1 = (13.0 / 12.0) * (f[1] - 2.0 * f[2] + f[3]) * (f[1] - 2.0 * f[2] + f[3]) +
         0.25 * (f[1] - f[3]) * (f[1] - f[3]);
  S b2 = (13.0 / 12.0) * (f[2] - 2.0 * f[3] + f[4]) * (f[2] - 2.0 * f[3] + f[4]) +
         0.25 * (3.0 * f[2] - 4.0 * f[3] + f[4]) * (3.0 * f[2] - 4.0 * f[3] + f[4]);
  S a0 = 0.1 / ((eps + b0) * (eps + b0));
  S a1 = 0.6 / ((eps + b1) * (eps + b1));
  S a2 = 0.3 / ((eps + b2) * (eps + b2));
  S q0 = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
  S q1 = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
  S q2 = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// WENO-CU6 at i+1/2 from f[0..5] = f_{i-2..i+3} (central-upwind, ref. 34).
// Reading: candidates q_0..q_2 of WENO5 plus the downwind q_3 on {i+1, i+2,
// i+3}; linear weights (1, 9, 9, 1)/20 (they make the 6-point central
// scheme); beta_0..beta_2 the Jiang-Shu indicators; beta_3 = beta_6, the
// Jiang-Shu indicator of the degree-5 polynomial on the whole stencil (integer
// table below, /120960); tau_6 = beta_6 - (beta_0 + beta_2 + 4 beta_1)/6;
// alpha_k = d_k (C + tau_6/(beta_k + eps)) with C = 20 and q = 1. The paper
// gives no eps; the one of WENO5 is used (absolute, 1e-6 by default). With
// the original 1e-40 the weights leave their linear values near extrema of a
// smooth wave (beta_k -> 0) and a density wave converges at order ~3.8 only;
// with 1e-6 it converges at sixth order.
template <class S>
S cu6_beta6(const S* f) {
  static const int e[21][2] = {{0,0},{0,1},{0,2},{0,3},{0,4},{0,5},{1,1},{1,2},{1,3},{1,4},{1,5},
                               {2,2},{2,3},{2,4},{2,5},{3,3},{3,4},{3,5},{4,4},{4,5},{5,5}};
  static const double c[21] = {271779, -2380800, 4086352, -3462252, 1458762, -245620, 5653317,
                               -20427884, 17905032, -7727988, 1325006, 19510972, -35817664,
                               15929912, -2792660, 17195652, -15880404, 2863984, 3824847,
                               -1429976, 139633};
  // beta_6 integrates derivatives only, so it is invariant to a constant
  // shift: evaluate the form on g = f - f_i, which keeps smooth data (small
  // variations about an offset) from cancelling away most of its digits
  S g[6];
  for (int k = 0; k < 6; ++k) g[k] = f[k] - f[2];
  S b(0.0);
  for (int k = 0; k < 21; ++k) b = b + c[k] * g[e[k][0]] * g[e[k][1]];
  return b / 120960.0;
}

template <class S>
S weno_cu6(const S* f, double eps) {
  const double C = 20.0, d[4] = {0.05, 0.45, 0.45, 0.05};
  S b[4];
  b[0] = (13.0 / 12.0) * (f[0] - 2.0 * f[1] + f[2]) * (f[0] - 2.0 * f[1] + f[2]) +
         0.25 * (f[0] - 4.0 * f[1] + 3.0 * f[2]) * (f[0] - 4.0 * f[1] + 3.0 * f[2]);
  b[1] = (13.0 / 12.0) * (f[1] - 2.0 * f[2] + f[3]) * (f[1] - 2.0 * f[2] + f[3]) +
         0.25 * (f[1] - f[3]) * (f[1] - f[3]);
  b[2] = (13.0 / 12.0) * (f[2] - 2.0 * f[3] + f[4]) * (f[2] - 2.0 * f[3] + f[4]) +
         0.25 * (3.0 * f[2] - 4.0 * f[3] + f[4]) * (3.0 * f[2] - 4.0 * f[3] + f[4]);
  b[3] = cu6_beta6(f);
  S tau = b[3] - (b[0] + b[2] + 4.0 * b[1]) / 6.0;
  S q[4];
  q[0] = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
  q[1] = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
  q[2] = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
  q[3] = (11.0 * f[3] - 7.0 * f[4] + 2.0 * f[5]) / 6.0;
  S a[4], as(0.0), aq(0.0);
  for (int k = 0; k < 4; ++k) {
    a[k] = d[k] * (C + tau / (b[k] + eps));
    as = as + a[k];
    aq = aq + a[k] * q[k];
  }
  return aq / as;
}

// WENO7-JS at i+1/2 from f[0..6] = f_{i-3..i+3} (ref. 36; reading): the four
// cubic candidates on {i-3+k .. i+k}, linear weights (1, 12, 18, 4)/35 (they
// make the 7-point upwind scheme), Jiang-Shu indicators of the cubics (the
// integer tables below, /240), alpha_k = d_k/(eps + beta_k)^2 with the WENO5
// epsilon. The indicators are evaluated on f - f_i (they integrate derivatives
// only).
template <class S>
S weno7_beta(const S* g, int k) {
  // beta_0 on g[0..3]; beta_3 is beta_0 mirrored (g[6..3]); beta_2 mirrors beta_1
  static const int e[10][2] = {{0,0},{0,1},{0,2},{0,3},{1,1},{1,2},{1,3},{2,2},{2,3},{3,3}};
  static const double c0[10] = {547, -3882, 4642, -1854, 7043, -17246, 7042, 11003, -9402, 2107};
  static const double c1[10] = {267, -1642, 1602, -494, 2843, -5966, 1922, 3443, -2522, 547};
  S h[4];
  for (int m = 0; m < 4; ++m) {
    if (k == 0) h[m] = g[m];
    else if (k == 1) h[m] = g[1 + m];
    else if (k == 2) h[m] = g[5 - m];
    else h[m] = g[6 - m];
  }
  const double* c = (k == 0 || k == 3) ? c0 : c1;
  S b(0.0);
  for (int t = 0; t < 10; ++t) b = b + c[t] * h[e[t][0]] * h[e[t][1]];
  return b / 240.0;
}

template <class S>
S weno7(const S* f, double eps) {
  const double d[4] = {1.0 / 35.0, 12.0 / 35.0, 18.0 / 35.0, 4.0 / 35.0};
  S g[7];
  for (int m = 0; m < 7; ++m) g[m] = f[m] - f[3];
  S q[4];
  q[0] = (-3.0 * f[0] + 13.0 * f[1] - 23.0 * f[2] + 25.0 * f[3]) / 12.0;
  q[1] = (f[1] - 5.0 * f[2] + 13.0 * f[3] + 3.0 * f[4]) / 12.0;
  q[2] = (-f[2] + 7.0 * f[3] + 7.0 * f[4] - f[5]) / 12.0;
  q[3] = (3.0 * f[3] + 13.0 * f[4] - 5.0 * f[5] + f[6]) / 12.0;
  S as(0.0), aq(0.0);
  for (int k = 0; k < 4; ++k) {
    S b = weno7_beta(g, k);
    S a = d[k] / ((eps + b) * (eps + b));
    as = as + a;
    aq = aq + a * q[k];
  }
  return aq / as;
}

// ------------------------------------------------------------ the RHS -----
template <class S>
struct Work {
  std::vector<Prim<S>> q;  // padded cells
};

template <class S>
void fill_padded(const Layout& L, const Thermo& th, const xfo_params& p, const S* U,
                 const double* Twarm, std::vector<Prim<S>>& q, double* Tout, uint32_t* st) {
  q.resize(L.pcells);
  uint32_t s_all = 0;
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) { lo[a] = (a < L.dim) ? -L.G : 0; hi[a] = (a < L.dim) ? L.n[a] + L.G : 1; }
  int64_t nx = hi[0] - lo[0], ny = hi[1] - lo[1], nz = hi[2] - lo[2];
#pragma omp parallel for schedule(static) reduction(| : s_all)
  for (int64_t t = 0; t < nx * ny * nz; ++t) {
    int64_t i = lo[0] + t % nx, j = lo[1] + (t / nx) % ny, k = lo[2] + t / (nx * ny);
    bool f[3];
    int64_t si = map_axis(i, L.n[0], p.bc[0][0], p.bc[0][1], &f[0]);
    int64_t sj = map_axis(j, L.n[1], p.bc[1][0], p.bc[1][1], &f[1]);
    int64_t sk = map_axis(k, L.n[2], p.bc[2][0], p.bc[2][1], &f[2]);
    int64_t src = L.g(si, sj, sk);
    S Uc[XFO_MAXV];
    for (int v = 0; v < L.nv; ++v) Uc[v] = U[(int64_t)v * L.cells + src];
    for (int a = 0; a < L.dim; ++a) if (f[a]) Uc[1 + a] = -Uc[1 + a];
    uint32_t sl = 0;
    Prim<S>& c = q[L.pg(i, j, k)];
    recover(L, th, p, Uc, Twarm[src], c, &sl);
    if (p.viscous) transport(th, p, c);
    if (i == si && j == sj && k == sk && Tout) Tout[src] = val(c.T);
    s_all |= sl;
  }
  *st |= s_all;
}

// unit step of axis a in padded indexing
inline int64_t pstride(const Layout& L, int a) {
  return a == 0 ? 1 : (a == 1 ? L.np[0] : L.np[0] * L.np[1]);
}

// Viscous face flux of direction d at the face between padded cells c0 and
// c0 + e_d (Reading of the "central 4th-order" viscous scheme): face values by
// (-1, 9, 9, -1)/16; normal derivatives by (1, -15, 15, -1)/(12 dx); tangential
// velocity derivatives by the nodal (1, -8, 0, 8, -1)/(12 dx) difference then
// the same face interpolation. Species rows carry -J_s (down-gradient).
template <class S>
void viscous_face(const Layout& L, const Thermo& th, const std::vector<Prim<S>>& q,
                  int64_t c0, int d, S* Fv) {
  int dim = L.dim, N = L.N;
  int64_t sd = pstride(L, d);
  const Prim<S>* c[4] = {&q[c0 - sd], &q[c0], &q[c0 + sd], &q[c0 + 2 * sd]};
  double h = L.dx[d];
  auto I = [&](auto get) { return (-get(*c[0]) + 9.0 * get(*c[1]) + 9.0 * get(*c[2]) - get(*c[3])) / 16.0; };
  auto Dn = [&](auto get) { return (get(*c[0]) - 15.0 * get(*c[1]) + 15.0 * get(*c[2]) - get(*c[3])) / (12.0 * h); };
  S mu = I([](const Prim<S>& x) { return x.mu; });
  S kap = I([](const Prim<S>& x) { return x.kap; });
  S Dsf[XFO_MAXN];
  for (int s = 0; s < N; ++s) Dsf[s] = I([s](const Prim<S>& x) { return x.Ds[s]; });
  S rho = I([](const Prim<S>& x) { return x.rho; });
  S T = I([](const Prim<S>& x) { return x.T; });
  S u[3], Yf[XFO_MAXN], dY[XFO_MAXN];
  for (int a = 0; a < dim; ++a) u[a] = I([a](const Prim<S>& x) { return x.u[a]; });
  for (int s = 0; s < N; ++s) {
    Yf[s] = I([s](const Prim<S>& x) { return x.Y[s]; });
    dY[s] = Dn([s](const Prim<S>& x) { return x.Y[s]; });
  }
  S dT = Dn([](const Prim<S>& x) { return x.T; });
  // velocity gradient at the face: grad[a][b] = d u_a / d x_b
  S grad[3][3];
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) {
      if (b == d) {
        grad[a][b] = Dn([a](const Prim<S>& x) { return x.u[a]; });
      } else {
        int64_t sb = pstride(L, b);
        double hb = L.dx[b];
        S nod[4];
        for (int m = 0; m < 4; ++m) {
          int64_t cm = c0 + (m - 1) * sd;
          nod[m] = (q[cm - 2 * sb].u[a] - 8.0 * q[cm - sb].u[a] + 8.0 * q[cm + sb].u[a] -
                    q[cm + 2 * sb].u[a]) / (12.0 * hb);
        }
        grad[a][b] = (-nod[0] + 9.0 * nod[1] + 9.0 * nod[2] - nod[3]) / 16.0;
      }
    }
  S div(0.0);
  for (int a = 0; a < dim; ++a) div = div + grad[a][a];
  S tau[3];
  for (int a = 0; a < dim; ++a) {
    tau[a] = mu * (grad[d][a] + grad[a][d]);
    if (a == d) tau[a] = tau[a] - (2.0 / 3.0) * mu * div;
  }
  // species diffusion with the mixture correction (Eq. 6)
  S corr(0.0);
  for (int s = 0; s < N; ++s) corr = corr + Dsf[s] * dY[s];
  S J[XFO_MAXN];
  for (int s = 0; s < N; ++s) J[s] = -rho * (Dsf[s] * dY[s] - Yf[s] * corr);
  Fv[0] = S(0.0);
  S work(0.0);
  for (int a = 0; a < dim; ++a) { Fv[1 + a] = tau[a]; work = work + tau[a] * u[a]; }
  S qd(0.0);
  for (int s = 0; s < N; ++s) qd = qd + th.h_s(s, T) * J[s];
  Fv[L.iE()] = work + kap * dT - qd;
  for (int s = 0; s < N - 1; ++s) Fv[L.iY(s)] = -J[s];
}

// Positivity-preserving blend of one face (Eq. 17-20; reading): the blended
// flux F* = (1 - theta) F_LF + theta F_hat, with F_LF the local Lax-Friedrichs
// flux of Eq. 19 (alpha = max over the two cells of |u_d| + c), keeps every
// partial density rho Y_s (s = 1..N) of the two one-sided states
// U_i - 2 lam F* and U_{i+1} + 2 lam F* (Eq. 18) at or above
// eps = min(pos_eps, its value with F_LF); lam = dim dt / dx_d. theta is the
// smallest admissible value over those 2N conditions.
template <class S>
void positivity_blend(const Layout& L, const xfo_params& p, const Prim<S>& a, const Prim<S>& b,
                      int d, double lam, S* Fh) {
  int nv = L.nv, N = L.N;
  S Fa[XFO_MAXV], Fb[XFO_MAXV];
  phys_flux(L, a, d, Fa);
  phys_flux(L, b, d, Fb);
  S al = max_first(S(fabs(a.u[d]) + a.c), S(fabs(b.u[d]) + b.c));
  S Flf[XFO_MAXV];
  for (int v = 0; v < nv; ++v) Flf[v] = 0.5 * (Fa[v] + Fb[v] + al * (a.U[v] - b.U[v]));
  S theta(1.0);
  for (int s = 0; s < N; ++s) {
    // partial density s and its flux components (the last one from rho - sum)
    S qa, qb, fh, fl;
    if (s < N - 1) {
      qa = a.U[L.iY(s)]; qb = b.U[L.iY(s)]; fh = Fh[L.iY(s)]; fl = Flf[L.iY(s)];
    } else {
      qa = a.U[0]; qb = b.U[0]; fh = Fh[0]; fl = Flf[0];
      for (int k = 0; k < N - 1; ++k) {
        qa = qa - a.U[L.iY(k)]; qb = qb - b.U[L.iY(k)];
        fh = fh - Fh[L.iY(k)]; fl = fl - Flf[L.iY(k)];
      }
    }
    for (int side = 0; side < 2; ++side) {
      double sg = side == 0 ? -2.0 * lam : 2.0 * lam;  // left cell: q - 2 lam F, right: q + 2 lam F
      S q = side == 0 ? qa : qb;
      S hi = q + sg * fh, lo = q + sg * fl;
      S eps = lo < p.pos_eps ? lo : S(p.pos_eps);
      if (hi < eps) {
        S th = (lo - eps) / (lo - hi);
        if (th < 0.0) th = S(0.0);
        if (th < theta) theta = th;
      }
    }
  }
  if (theta < 1.0)
    for (int v = 0; v < nv; ++v) Fh[v] = (1.0 - theta) * Flf[v] + theta * Fh[v];
}

template <class S>
void rhs_impl(const xfo_params& p, const S* U, double* T, S* dUdt, uint32_t* st, double dt = 0.0) {
  Layout L(p);
  Thermo th(p);
  int nv = L.nv, dim = L.dim;
  std::vector<Prim<S>> q;
  std::vector<double> Tw(T, T + L.cells);
  fill_padded(L, th, p, U, Tw.data(), q, T, st);
  for (int64_t i = 0; i < (int64_t)nv * L.cells; ++i) dUdt[i] = S(0.0);
  uint32_t s_all = 0;
  for (int d = 0; d < dim; ++d) {
    // faces i + 1/2 for i = -1 .. n_d - 1 at every interior transverse position
    int64_t nf[3] = {L.n[0], L.n[1], L.n[2]};
    nf[d] += 1;
    int64_t nfaces = nf[0] * nf[1] * nf[2];
    std::vector<S> Fh((size_t)nfaces * nv);
    int64_t sd = pstride(L, d);
#pragma omp parallel for schedule(dynamic, 64) reduction(| : s_all)
    for (int64_t f = 0; f < nfaces; ++f) {
      int64_t idx[3] = {f % nf[0], (f / nf[0]) % nf[1], f / (nf[0] * nf[1])};
      idx[d] -= 1;  // left cell of the face
      int64_t c0 = L.pg(idx[0], idx[1], idx[2]);
      S Ft[XFO_MAXV];
      for (int v = 0; v < nv; ++v) Ft[v] = S(0.0);
      uint32_t sl = 0;
      if (p.convective) {
        S Lm[XFO_MAXV * XFO_MAXV], Rm[XFO_MAXV * XFO_MAXV], lam[XFO_MAXV], c2;
        int lt[XFO_MAXV];
        eigen(L, th, q[c0], q[c0 + sd], d, Lm, Rm, lam, lt, &c2, &sl);
        // stencil m = i-2 .. i+3: characteristic projections (Eq. 14)
        const int W = 2 * L.G;  // stencil cells i-G+1 .. i+G
        S LU[8][XFO_MAXV], LF[8][XFO_MAXV];
        S amax[3] = {S(0.0), S(0.0), S(0.0)};
        for (int m = 0; m < W; ++m) {
          const Prim<S>& cm = q[c0 + (m - L.G + 1) * sd];
          S F[XFO_MAXV];
          phys_flux(L, cm, d, F);
          for (int kk = 0; kk < nv; ++kk) {
            S a(0.0), b(0.0);
            for (int j = 0; j < nv; ++j) { a = a + Lm[kk * nv + j] * cm.U[j]; b = b + Lm[kk * nv + j] * F[j]; }
            LU[m][kk] = a; LF[m][kk] = b;
          }
          // LLF: alpha_k = max over the stencil of |lambda_k| (per-cell eigenvalues)
          amax[0] = max_first(amax[0], S(fabs(cm.u[d] - cm.c)));
          amax[1] = max_first(amax[1], S(fabs(cm.u[d] + cm.c)));
          amax[2] = max_first(amax[2], S(fabs(cm.u[d])));
        }
        S Fc[XFO_MAXV];
        for (int kk = 0; kk < nv; ++kk) {
          S al = amax[lt[kk]];
          S wp[8], wm[8];
          for (int m = 0; m < W; ++m) {
            wp[m] = 0.5 * (LF[m][kk] + al * LU[m][kk]);                   // m -> i-G+1+m
            wm[m] = 0.5 * (LF[W - 1 - m][kk] - al * LU[W - 1 - m][kk]);   // mirrored: i+G-m
          }
          if (p.weno == 7)
            Fc[kk] = weno7(wp, p.weno_eps) + weno7(wm, p.weno_eps);
          else if (p.weno == 6)
            Fc[kk] = weno_cu6(wp, p.weno_eps) + weno_cu6(wm, p.weno_eps);
          else
            Fc[kk] = weno5(wp, p.weno_eps) + weno5(wm, p.weno_eps);
        }
        for (int j = 0; j < nv; ++j) {  // back-projection (Eq. 15)
          S a(0.0);
          for (int kk = 0; kk < nv; ++kk) a = a + Rm[j * nv + kk] * Fc[kk];
          Ft[j] = a;
        }
        if (p.positivity && dt > 0.0)
          positivity_blend(L, p, q[c0], q[c0 + sd], d, L.dim * dt / L.dx[d], Ft);
      }
      if (p.viscous) {
        S Fv[XFO_MAXV];
        viscous_face(L, th, q, c0, d, Fv);
        for (int v = 0; v < nv; ++v) Ft[v] = Ft[v] - Fv[v];
      }
      for (int v = 0; v < nv; ++v) Fh[(size_t)f * nv + v] = Ft[v];
      s_all |= sl;
    }
    // conservative difference (Eq. 13): dU/dt -= (G_{i+1/2} - G_{i-1/2}) / dx_d
    double h = L.dx[d];
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < L.cells; ++c) {
      int64_t idx[3] = {c % L.n[0], (c / L.n[0]) % L.n[1], c / (L.n[0] * L.n[1])};
      int64_t fl[3] = {idx[0], idx[1], idx[2]};
      int64_t fr[3] = {idx[0], idx[1], idx[2]};
      fr[d] += 1;
      int64_t il = (fl[2] * nf[1] + fl[1]) * nf[0] + fl[0];
      int64_t ir = (fr[2] * nf[1] + fr[1]) * nf[0] + fr[0];
      for (int v = 0; v < nv; ++v)
        dUdt[(int64_t)v * L.cells + c] =
            dUdt[(int64_t)v * L.cells + c] - (Fh[(size_t)ir * nv + v] - Fh[(size_t)il * nv + v]) / h;
    }
  }
  *st |= s_all;
}

template <class S>
void rk3_impl(const xfo_params& p, S* U, double* T, double dt, uint32_t* st) {
  Layout L(p);
  int64_t n = (int64_t)L.nv * L.cells;
  std::vector<S> U0(U, U + n), U1(n), U2(n), R(n);
  // Eq. 16
  rhs_impl(p, U0.data(), T, R.data(), st, dt);
  for (int64_t i = 0; i < n; ++i) U1[i] = U0[i] + dt * R[i];
  rhs_impl(p, U1.data(), T, R.data(), st, dt);
  for (int64_t i = 0; i < n; ++i) U2[i] = 0.75 * U0[i] + 0.25 * (U1[i] + dt * R[i]);
  rhs_impl(p, U2.data(), T, R.data(), st, dt);
  for (int64_t i = 0; i < n; ++i) U[i] = (1.0 / 3.0) * U0[i] + (2.0 / 3.0) * (U2[i] + dt * R[i]);
}

int check(const xfo_params* p) {
  if (!p || p->dim < 1 || p->dim > 3 || p->N < 2 || p->N > XFO_MAXN) return -1;
  if (p->weno != 5 && p->weno != 6 && p->weno != 7) return -1;
  if (p->diffusion != 0 && p->diffusion != 1) return -1;
  for (int a = 0; a < p->dim; ++a) if (p->n[a] < 1) return -1;
  for (int a = 0; a < p->dim; ++a)
    for (int s = 0; s < 2; ++s)
      if (p->bc[a][s] != XFO_BC_TRANSMISSIVE && p->n[a] < ghosts(p->weno)) return -1;
#ifdef _OPENMP
  if (p->threads > 0) omp_set_num_threads(p->threads);
#endif
  return 0;
}

}  // namespace

extern "C" {

int xfo_nv(const xfo_params* p) { return p->dim + 2 + p->N - 1; }

int xfo_prim_to_cons(const xfo_params* p, const double* P, double* U, double* T) {
  if (check(p)) return -1;
  Layout L(*p);
  Thermo th(*p);
  for (int64_t c = 0; c < L.cells; ++c) {
    double rho = P[c], pr = P[(int64_t)(1 + L.dim) * L.cells + c];
    double Y[XFO_MAXN], ysum = 0.0, Rm = 0.0, ke = 0.0;
    for (int s = 0; s < L.N - 1; ++s) { Y[s] = P[(int64_t)L.iY(s) * L.cells + c]; ysum += Y[s]; }
    Y[L.N - 1] = 1.0 - ysum;
    for (int s = 0; s < L.N; ++s) Rm += Y[s] * th.Rs[s];
    double Tc = pr / (rho * Rm);  // Eq. 7
    double e = 0.0;
    for (int s = 0; s < L.N; ++s) e += Y[s] * th.e_s(s, Tc);
    U[c] = rho;
    for (int a = 0; a < L.dim; ++a) {
      double u = P[(int64_t)(1 + a) * L.cells + c];
      U[(int64_t)(1 + a) * L.cells + c] = rho * u;
      ke += u * u;
    }
    U[(int64_t)L.iE() * L.cells + c] = rho * (e + 0.5 * ke);
    for (int s = 0; s < L.N - 1; ++s) U[(int64_t)L.iY(s) * L.cells + c] = rho * Y[s];
    if (T) T[c] = Tc;
  }
  return 0;
}

int xfo_cons_to_prim(const xfo_params* p, const double* U, double* T, double* P,
                     uint32_t* status) {
  if (check(p)) return -1;
  Layout L(*p);
  Thermo th(*p);
  uint32_t st = 0;
  for (int64_t c = 0; c < L.cells; ++c) {
    double Uc[XFO_MAXV];
    for (int v = 0; v < L.nv; ++v) Uc[v] = U[(int64_t)v * L.cells + c];
    Prim<double> q;
    recover(L, th, *p, Uc, T[c], q, &st);
    T[c] = q.T;
    P[c] = q.rho;
    for (int a = 0; a < L.dim; ++a) P[(int64_t)(1 + a) * L.cells + c] = q.u[a];
    P[(int64_t)(1 + L.dim) * L.cells + c] = q.p;
    for (int s = 0; s < L.N - 1; ++s) P[(int64_t)L.iY(s) * L.cells + c] = q.Y[s];
  }
  if (status) *status |= st;
  return 0;
}

int xfo_rhs(const xfo_params* p, const double* U, double* T, double* dUdt, uint32_t* status) {
  if (check(p)) return -1;
  uint32_t st = 0;
  rhs_impl<double>(*p, U, T, dUdt, &st);
  if (status) *status |= st;
  return 0;
}

double xfo_dt(const xfo_params* p, const double* U, double* T, uint32_t* status) {
  if (check(p)) return -1.0;
  Layout L(*p);
  Thermo th(*p);
  double smax = 0.0, numax = 0.0;
  uint32_t st = 0;
  for (int64_t c = 0; c < L.cells; ++c) {
    double Uc[XFO_MAXV];
    for (int v = 0; v < L.nv; ++v) Uc[v] = U[(int64_t)v * L.cells + c];
    Prim<double> q;
    recover(L, th, *p, Uc, T[c], q, &st);
    T[c] = q.T;
    double s = 0.0;
    for (int a = 0; a < L.dim; ++a) s += (std::fabs(q.u[a]) + q.c) / L.dx[a];
    smax = std::max(smax, s);
    if (p->viscous) {
      transport(th, *p, q);
      double nu = std::max(4.0 * q.mu / (3.0 * q.rho), q.kap / (q.rho * q.cv));
      for (int k = 0; k < p->N; ++k) nu = std::max(nu, q.Ds[k]);
      numax = std::max(numax, nu);
    }
  }
  if (status) *status |= st;
  // Reading of the multi-D CFL condition (Eq. 17: lambda = CFL / Lambda)
  double dt = p->cfl / smax;
  if (p->viscous && numax > 0.0) {
    double hmin = L.dx[0];
    for (int a = 1; a < L.dim; ++a) hmin = std::min(hmin, L.dx[a]);
    dt = std::min(dt, p->cfl * hmin * hmin / (2.0 * L.dim * numax));
  }
  return dt;
}

double xfo_step_rk3(const xfo_params* p, double* U, double* T, double dt, uint32_t* status) {
  if (check(p)) return -1.0;
  uint32_t st = 0;
  if (dt <= 0.0) dt = xfo_dt(p, U, T, &st);
  rk3_impl<double>(*p, U, T, dt, &st);
  if (status) *status |= st;
  return dt;
}

int xfo_run_to(const xfo_params* p, double* U, double* T, double t_end, int max_steps,
               uint32_t* status) {
  if (check(p)) return -1;
  double t = 0.0;
  int steps = 0;
  while (t < t_end && steps < max_steps) {
    uint32_t st = 0;
    double dt = xfo_dt(p, U, T, &st);
    if (t + dt >= t_end) dt = t_end - t;
    rk3_impl<double>(*p, U, T, dt, &st);
    if (status) *status |= st;
    t += dt;
    ++steps;
    if (t_end - t <= 1e-14 * t_end) break;
  }
  return steps;
}

int xfo_thermo(const xfo_params* p, double T, const double* Y, double* e, double* cv,
               double* cp, double* e_s, double* h_s) {
  if (check(p)) return -1;
  Thermo th(*p);
  double a = 0.0, b = 0.0, c = 0.0;
  for (int s = 0; s < p->N; ++s) {
    a += Y[s] * th.e_s(s, T); b += Y[s] * th.cv_s(s, T); c += Y[s] * th.cp_s(s, T);
    if (e_s) e_s[s] = th.e_s(s, T);
    if (h_s) h_s[s] = th.h_s(s, T);
  }
  if (e) *e = a;
  if (cv) *cv = b;
  if (cp) *cp = c;
  return 0;
}

double xfo_temperature(const xfo_params* p, double e, const double* Y, double T0, int* iters,
                       uint32_t* status) {
  if (check(p)) return -1.0;
  Thermo th(*p);
  uint32_t st = 0;
  double T = newton_T(th, *p, e, Y, T0, iters, &st);
  if (status) *status |= st;
  return T;
}

int xfo_eigen(const xfo_params* p, int d, const double* UL, const double* UR, double TL,
              double TR, double* Lo, double* Ro, double* lam, double* c2, uint32_t* status) {
  if (check(p) || d < 0 || d >= p->dim) return -1;
  Layout L(*p);
  Thermo th(*p);
  uint32_t st = 0;
  Prim<double> a, b;
  recover(L, th, *p, UL, TL, a, &st);
  recover(L, th, *p, UR, TR, b, &st);
  int lt[XFO_MAXV];
  eigen(L, th, a, b, d, Lo, Ro, lam, lt, c2, &st);
  if (status) *status |= st;
  return 0;
}

int xfo_flux(const xfo_params* p, int d, const double* U1, double T, double* F, uint32_t* status) {
  if (check(p) || d < 0 || d >= p->dim) return -1;
  Layout L(*p);
  Thermo th(*p);
  uint32_t st = 0;
  Prim<double> a;
  recover(L, th, *p, U1, T, a, &st);
  phys_flux(L, a, d, F);
  if (status) *status |= st;
  return 0;
}

double xfo_weno5(const double* f) { return weno5(f, 1e-6); }
double xfo_weno_cu6(const double* f, double eps) { return weno_cu6(f, eps); }
double xfo_weno7(const double* f, double eps) { return weno7(f, eps); }
double xfo_cu6_beta6(const double* f) { return cu6_beta6(f); }

int xfo_species_diffusion(const xfo_params* p, double T, double rho, const double* Y,
                          double* Ds) {
  if (check(p)) return -1;
  Thermo th(*p);
  Prim<double> q;
  q.T = T; q.rho = rho;
  double cp = 0.0, Rm = 0.0;
  for (int s = 0; s < p->N; ++s) { q.Y[s] = Y[s]; cp += Y[s] * th.cp_s(s, T); Rm += Y[s] * th.Rs[s]; }
  q.cp = cp; q.Rm = Rm;
  transport(th, *p, q);
  for (int s = 0; s < p->N; ++s) Ds[s] = q.Ds[s];
  return 0;
}

int xfo_transport(const xfo_params* p, double T, double rho, const double* Y, double* mu,
                  double* kappa, double* D) {
  if (check(p)) return -1;
  Thermo th(*p);
  Prim<double> q;
  q.T = T; q.rho = rho;
  double cp = 0.0, Rm = 0.0;
  for (int s = 0; s < p->N; ++s) { q.Y[s] = Y[s]; cp += Y[s] * th.cp_s(s, T); Rm += Y[s] * th.Rs[s]; }
  q.cp = cp; q.Rm = Rm;
  transport(th, *p, q);
  *mu = q.mu; *kappa = q.kap; *D = q.D;
  return 0;
}

int xfo_rhs_jvp(const xfo_params* p, const double* U, const double* V, double* T, double* dUdt,
                double* JV, uint32_t* status) {
  if (check(p)) return -1;
  Layout L(*p);
  int64_t n = (int64_t)L.nv * L.cells;
  std::vector<D8> Ud(n), Rd(n);
  for (int64_t i = 0; i < n; ++i) {
    Ud[i].v = U[i];
    for (int k = 0; k < XFO_KDIR; ++k) Ud[i].d[k] = V[(int64_t)k * n + i];
  }
  uint32_t st = 0;
  rhs_impl<D8>(*p, Ud.data(), T, Rd.data(), &st);
  for (int64_t i = 0; i < n; ++i) {
    dUdt[i] = Rd[i].v;
    for (int k = 0; k < XFO_KDIR; ++k) JV[(int64_t)k * n + i] = Rd[i].d[k];
  }
  if (status) *status |= st;
  return 0;
}

int xfo_rk3_jvp(const xfo_params* p, double* U, double* V, double* T, double dt, int steps,
                uint32_t* status) {
  if (check(p) || dt <= 0.0) return -1;
  Layout L(*p);
  int64_t n = (int64_t)L.nv * L.cells;
  std::vector<D8> Ud(n);
  for (int64_t i = 0; i < n; ++i) {
    Ud[i].v = U[i];
    for (int k = 0; k < XFO_KDIR; ++k) Ud[i].d[k] = V[(int64_t)k * n + i];
  }
  uint32_t st = 0;
  for (int s = 0; s < steps; ++s) rk3_impl<D8>(*p, Ud.data(), T, dt, &st);
  for (int64_t i = 0; i < n; ++i) {
    U[i] = Ud[i].v;
    for (int k = 0; k < XFO_KDIR; ++k) V[(int64_t)k * n + i] = Ud[i].d[k];
  }
  if (status) *status |= st;
  return 0;
}

}  // extern "C"
