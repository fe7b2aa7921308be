// esmm_3d.h -- the 3D RMHD handle (esmm_3d.cu) behind the C ABI: esmm_api.cu
// forwards the calls of dim = 3 grids here.  Arguments as in include/esmm.h
// with [8][N] states, [3][N] meshes and mesh velocities.
#pragma once

#include "esmm.h"

struct esmm3;

int esmm3_create(esmm3 **out, const int n[3], const double lo[3], const double hi[3], const int bc[3], void *stream);
void esmm3_destroy(esmm3 *g);
int esmm3_set_stream(esmm3 *g, void *stream);
int esmm3_set_eos(esmm3 *g, double gamma);
int esmm3_set_order(esmm3 *g, int p, int w);
int esmm3_set_params(esmm3 *g, const esmm_params *prm);
int esmm3_get_params(const esmm3 *g, esmm_params *prm);
int esmm3_state_set(esmm3 *g, const double *prim, const double *x, int mem);
int esmm3_state_set_cons(esmm3 *g, const double *cons, const double *J, const double *x, double t, int mem);
int esmm3_state_get(esmm3 *g, int what, double *out, int mem);
int esmm3_get_time(esmm3 *g, double *t);
int esmm3_rhs(esmm3 *g, const double *cons, const double *J, const double *x, const double *xdot, double *dcons,
              double *dJ, int mem);
int esmm3_cfl_dt(esmm3 *g, double *dt);
int esmm3_mesh_redistribute(esmm3 *g, double dt, double *xdot, double *dtau, double *dt_used, int mem);
int esmm3_rk_step(esmm3 *g, double dt, double *dt_used);
int esmm3_rk_step_given(esmm3 *g, const double *xdot, double dt, int mem);
int esmm3_advance(esmm3 *g, int nsteps, double dt);
int esmm3_set_inflow(esmm3 *g, const double *prim);
int esmm3_totals(esmm3 *g, double out[3]);
int esmm3_last_error(esmm3 *g, int *n_c2p_fail, char *msg, int len);
long long esmm3_launches(const esmm3 *g);
int esmm3_rhs_vjp(esmm3 *g, const double *cons, const double *J, const double *x, const double *xdot,
                  const double *mu, double *lam, int mem);
int esmm3_adjoint_record(esmm3 *g, int nsteps, double dt);
int esmm3_adjoint_steps(esmm3 *g, int *nsteps, double *dt);
int esmm3_adjoint_checkpoint(esmm3 *g, int step, int what, double *out, int mem);
int esmm3_adjoint_replay(esmm3 *g, int nsteps);
int esmm3_adjoint_vjp(esmm3 *g, const double *lam_final, double *lam_cons0, double *lam_prim0, int mem);
int esmm3_profile(esmm3 *g, int mask);
int esmm3_profile_read(esmm3 *g, double ms[ESMM_NKINDS], long long launches[ESMM_NKINDS],
                       long long timed[ESMM_NKINDS]);
