/*
 * oracle.h -- plain single-threaded FP64 CPU oracle for RK4 subcycling in time
 * on nested refined boxes with dense-output ghost filling (arXiv:2503.09629).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (all indices are cell indices, cell-centred grids):
 *   level l has spacing h_l = h0 / 2^l and index space [0, ncells0 * 2^l) per dim;
 *   cell i of level l has centre origin + (i + 1/2) h_l;
 *   every box carries 3 ghost cells per side; arrays are x fastest;
 *   one FP64 array per field ("SoA").
 * Every function returns 0 on success and a negative code on error.
 */
#ifndef SUBCYC_ORACLE_H
#define SUBCYC_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_WAVE = 0, ORC_Z4C = 1 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_RADIATIVE = 1, ORC_BC_CALLBACK = 2 };
enum { ORC_ID_STANDING_WAVE = 0, ORC_ID_GAUSSIAN = 1, ORC_ID_BRILL_LINDQUIST = 2,
       ORC_ID_MINKOWSKI = 3, ORC_ID_SPHERICAL_GAUSSIAN = 4, ORC_ID_BRILL_LINDQUIST_AVG_LAPSE = 5 };

/* Physical boundary callback (ORC_BC_CALLBACK, level 0 only): fill out[f*npts+p]
 * with the value the stage state should take at the given cell centres.
 * which = 1..s: stage state Y_which of the step that starts at t_n with step dt;
 * which = 0: the state y(t_n + dt) after the step. */
typedef void (*orc_bc_fn)(void* user, int which, double t_n, double dt, int npts,
                          const double* xyz, double* out);

int orc_create(int system, int nlevels, const int* nboxes, const int* boxes,
               const int* ncells0, const double* origin, double h0, int bc,
               double cfl, int subcycle, const double* params, void** out);
/* As orc_create with the finite-difference order of the right-hand sides,
 * fd_order = 4 (3 ghost cells per box) or 8 (the paper's production setting,
 * 4 ghost cells; Kreiss-Oliger dissipation stays r = 4), and the Runge-Kutta
 * method, rk_order = 4 (classic RK4, Sec. II), 3 (Heun's third-order method)
 * or 2 (explicit midpoint), each subcycled with its own dense output. */
int orc_create_ex(int system, int nlevels, const int* nboxes, const int* boxes,
                  const int* ncells0, const double* origin, double h0, int bc,
                  double cfl, int subcycle, const double* params, int fd_order, int rk_order,
                  void** out);
void orc_destroy(void* h);
int orc_nfields(void* h);
int orc_set_bc_callback(void* h, orc_bc_fn fn, void* user);
/* Gamma-driver damping eta(r) = (eta_c - eta_o) exp(-(r/eta_s)^4) + eta_o (Sec. III.A). */
int orc_set_eta_profile(void* h, double eta_c, double eta_s, double eta_o);
int orc_set_initial_data(void* h, int kind, const double* params, int nparams);
int orc_set_field(void* h, int level, int box, int field, const double* src);
int orc_get_field(void* h, int level, int box, int field, double* dst);
int orc_set_field_ghosted(void* h, int level, int box, int field, const double* src);
int orc_get_field_ghosted(void* h, int level, int box, int field, double* dst);
int orc_advance(void* h, int ncoarse);
double orc_time(void* h);
int orc_zone_updates(void* h, double* finest_equiv, double* actual);

/* Pieces of the method, exposed for the pin tests. */
void orc_dense_b(double theta, int m, double* b4);
double orc_amr_value(double y, const double* k4, double H, double theta0, int which);
void orc_dense_b_rk(int rk, double theta, int m, double* b4);
double orc_amr_value_rk(int rk, double y, const double* k4, double H, double theta0, int which);
int orc_rhs_box(void* h, int level, int box, const double* state_ghosted, double* rhs_ghosted);
int orc_constraints(void* h, int level, int box, double* out);
int orc_debug_set_vector(void* h, int level, int box, int vec, int field, const double* src);
int orc_debug_get_vector(void* h, int level, int box, int vec, int field, double* dst);
int orc_debug_prolong(void* h, int level);
int orc_debug_fill_amr(void* h, int level, int vec, double theta0, int which);
int orc_debug_restrict(void* h, int level);
int orc_debug_fill_ghosts(void* h);
void orc_flop_counts(double* counts);
/* Moving boxes: new boxes for every level (level 0 unchanged); see oracle.cpp. */
int orc_regrid(void* h, const int* nboxes, const int* boxes);
int orc_interpolate(void* h, int npts, const double* xyz, int field, double* out);

#ifdef __cplusplus
}
#endif
#endif
