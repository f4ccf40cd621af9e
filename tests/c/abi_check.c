/* Plain C99 use of the C-ABI: the header compiles as C, the library links,
 * and the calls that need no device behave (argument errors, status
 * strings). Built and run by tests/test_c_abi.py. */
#include <stdio.h>
#include <string.h>

#include "xf.h"

int main(void) {
  const double W[2] = {0.028, 0.004};
  const double cp[10] = {3.5, 0, 0, 0, 0, 2.5, 0, 0, 0, 0};
  const double h_off[2] = {0.0, 0.0};
  xf_grid g;
  xf_thermo t;
  xf_opts o;
  xf_handle *h = NULL;
  memset(&g, 0, sizeof g);
  memset(&t, 0, sizeof t);
  memset(&o, 0, sizeof o);
  g.dim = 1;
  g.n[0] = 2; /* too small: at least 3 cells per axis */
  g.hi[0] = 1.0;
  t.n_species = 2;
  t.W = W;
  t.T_lo = 200.0;
  t.T_hi = 4000.0;
  t.cp_coef = cp;
  t.h_off = h_off;
  t.lewis = 1.0;
  t.a_ref2 = 89079.0;
  t.rho_ref = 1.0;
  t.L_ref = 1.0;
  o.cfl = 0.5;
  o.weno = 5;
  o.newton_max = 50;
  o.newton_rtol = 1e-13;
  o.weno_eps = 1e-6;
  if (xf_create(&g, &t, &o, &h) != XF_ERR_ARG || h != NULL) return 1;
  g.n[0] = 64;
  o.weno = 4; /* no such scheme */
  if (xf_create(&g, &t, &o, &h) != XF_ERR_ARG) return 2;
  if (xf_step_rk3(NULL, 0.0, NULL, NULL) != XF_ERR_ARG) return 3;
  if (xf_nv(NULL) != 0 || xf_cells(NULL) != 0) return 4;
  if (strncmp(xf_status_str(XF_ERR_ARG), "invalid", 7) != 0) return 5;
  printf("ok %s\n", xf_status_str(XF_OK));
  return 0;
}
