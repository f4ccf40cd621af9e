/* xfo.h -- C interface of the CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * A plain, slow FP64 implementation of the per-stage right-hand side and
 * SSP-RK3 step of the multicomponent compressible solver of arXiv 2403.05910
 * (XFluids), written from the paper's equations: primitive recovery with the
 * Newton temperature solve (Eq. 21), ideal-gas mixture EOS (Eq. 7),
 * characteristic LLF flux splitting (Eq. 14), WENO5-JS reconstruction and
 * back-projection (Eq. 15), the full-eigensystem (EEO) dense projection,
 * mixture-averaged transport (Eq. 22, Eq. 29), viscous and species-diffusion
 * fluxes (Eq. 3-6), the conservative difference (Eq. 13) and SSP-RK3 (Eq. 16).
 *
 * Also: WENO-CU6 and WENO7-JS reconstructions (refs. 34, 36), the
 * positivity-preserving flux blend (Eq. 17-20) and the mixture-averaged
 * diffusion of Eq. 25-26.
 *
 * Parity unpinned vs the paper: the basis of the degenerate u-eigenspace
 * (xfo_eigen), the paper's choice being in references it only cites; it is
 * pinned for self-consistency (L.R = I, A r = lambda r), so results that
 * depend on it match the paper's method up to that choice. The
 * multicomponent Roe average of the face state (also only cited) is pinned
 * by what the mathematics fixes: it is an exact Roe matrix for mixtures of
 * calorically perfect species (R diag(lambda) L dU = dF to round-off) and a
 * consistent second-order linearisation when c_p,s depends on T.
 *
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark use
 * this library; the product path never links or calls it. It shares no code
 * with the CUDA path.
 *
 * Arrays are FP64 SoA [n_v][nz][ny][nx] (i fastest), interior cells only, with
 * rows (rho, rho u_1..rho u_dim, E, rho Y_1..rho Y_{N-1}); primitive arrays use
 * (rho, u_1..u_dim, p, Y_1..Y_{N-1}). Functions return 0 on success and a
 * negative value on an argument error; device-free status bits are OR-ed into
 * *status (XFO_FLAG_*).
 */
#ifndef XFO_H
#define XFO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XFO_MAXN 8
#define XFO_MAXV (3 + 2 + XFO_MAXN - 1)

#define XFO_BC_TRANSMISSIVE 0
#define XFO_BC_PERIODIC 1
#define XFO_BC_SYMMETRIC 2

#define XFO_FLAG_NONPHYS 1u /* NaN/inf in U, rho<=0, p<=0 or T<=0 */
#define XFO_FLAG_NEWTON 2u  /* temperature solve did not converge */
#define XFO_FLAG_EIGEN 4u   /* face sound speed squared <= 0 */

typedef struct {
  int dim;
  int64_t n[3];
  double lo[3], hi[3];
  int bc[3][2];
  int N;                          /* species count, 2..XFO_MAXN */
  double W[XFO_MAXN];             /* kg/mol */
  double T_lo, T_hi;              /* K, c_p polynomial range */
  double cp[XFO_MAXN][5];         /* c_p/R_s monomials in tau */
  double h_off[XFO_MAXN];         /* h_s/R_s at T_lo, K */
  double mu[XFO_MAXN][4];         /* ln mu_s [Pa s] cubic in ln T */
  double kap[XFO_MAXN][4];        /* ln kappa_s [W/(m K)] cubic in ln T */
  double lewis;
  double a_ref2, rho_ref, L_ref;  /* reference scales */
  double cfl;
  int viscous;                    /* viscous + diffusion fluxes on/off */
  int convective;                 /* convective fluxes on/off (tests) */
  int newton_max;
  double newton_rtol;
  double weno_eps;
  int threads;                    /* OpenMP threads, 0 = default */
  int positivity;                 /* positivity-preserving flux blend (Eq. 17-20) */
  int weno;                       /* 5: WENO5-JS, 6: WENO-CU6, 7: WENO7-JS */
  double pos_eps;                 /* target floor of the partial densities */
  int diffusion;                  /* 0: D = kappa/(rho c_p Le) for every species;
                                     1: mixture-averaged D_sm (Eq. 25-26) */
  double dbin[XFO_MAXN][XFO_MAXN][4]; /* ln(p D_st [Pa m^2/s]) cubic in ln T */
} xfo_params;

int xfo_nv(const xfo_params *p);

/* primitive (rho,u,p,Y) -> conserved U; also T (K) per cell */
int xfo_prim_to_cons(const xfo_params *p, const double *P, double *U, double *T);
/* conserved -> primitive with the Newton solve warm-started from T (in/out) */
int xfo_cons_to_prim(const xfo_params *p, const double *U, double *T, double *P,
                     uint32_t *status);
/* dUdt = L(U); T is the warm start (in) and the recovered temperature (out) */
int xfo_rhs(const xfo_params *p, const double *U, double *T, double *dUdt,
            uint32_t *status);
/* CFL time step of the state U (convective and viscous limits) */
double xfo_dt(const xfo_params *p, const double *U, double *T, uint32_t *status);
/* one SSP-RK3 step of size dt (dt <= 0: the CFL step of U^n); returns dt used */
double xfo_step_rk3(const xfo_params *p, double *U, double *T, double dt,
                    uint32_t *status);
/* march to t_end with CFL steps, the last one clipped; returns step count */
int xfo_run_to(const xfo_params *p, double *U, double *T, double t_end,
               int max_steps, uint32_t *status);

/* single-state helpers for the self-checks */
int xfo_thermo(const xfo_params *p, double T, const double *Y, double *e,
               double *cv, double *cp, double *e_s, double *h_s);
double xfo_temperature(const xfo_params *p, double e, const double *Y,
                       double T0, int *iters, uint32_t *status);
/* face eigensystem of direction d between two conserved states (dense,
 * storage order); L, R are n_v x n_v row-major, lam n_v, c2 scalar */
int xfo_eigen(const xfo_params *p, int d, const double *UL, const double *UR,
              double TL, double TR, double *L, double *R, double *lam,
              double *c2, uint32_t *status);
/* physical flux of direction d at one conserved state */
int xfo_flux(const xfo_params *p, int d, const double *U1, double T, double *F,
             uint32_t *status);
double xfo_weno5(const double *f);
/* WENO-CU6 at i+1/2 from f[0..5] = f_{i-2..i+3}; beta6 of the 6-point stencil */
double xfo_weno_cu6(const double *f, double eps);
double xfo_cu6_beta6(const double *f);
/* WENO7-JS at i+1/2 from f[0..6] = f_{i-3..i+3} */
double xfo_weno7(const double *f, double eps);
/* per-species diffusion coefficients D_s (dimensionless) of the selected
 * model at (T, rho, Y): the mixture-averaged D_sm of Eq. 26 or the common D */
int xfo_species_diffusion(const xfo_params *p, double T, double rho, const double *Y,
                          double *Ds);
/* per-cell mixture transport (dimensionless mu, kappa, D) */
int xfo_transport(const xfo_params *p, double T, double rho, const double *Y,
                  double *mu, double *kappa, double *D);

/* Forward-mode derivatives with XFO_KDIR directions per call (dual numbers).
 * V is [XFO_KDIR][n_v*cells]; JV gets [XFO_KDIR][n_v*cells]. */
#define XFO_KDIR 8
int xfo_rhs_jvp(const xfo_params *p, const double *U, const double *V, double *T,
                double *dUdt, double *JV, uint32_t *status);
/* `steps` RK3 steps of fixed dt, propagating XFO_KDIR tangents V (in/out) */
int xfo_rk3_jvp(const xfo_params *p, double *U, double *V, double *T, double dt,
                int steps, uint32_t *status);

#ifdef __cplusplus
}
#endif
#endif
