/* btdf_oracle.h - plain FP64 CPU oracle of the BTDF immersed-boundary lattice
 * Boltzmann time step (M. Jiang, Z. Liu, "A Boundary Thickening-based Direct
 * Forcing Immersed Boundary Method for Fully Resolved Simulation of
 * Particle-laden Flows", arXiv 1806.09403).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no source,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded inputs they are both given.
 *
 * Lattice units: dh = dt = c = 1, rho0 = 1.  Populations are stored
 * array-of-structures, f[(y*nx + x)*9 + a], in full (not as deviations).
 * D2Q9 ordering (Eq. 8): 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
 * 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *
 * Parity status of each function is stated in the file that implements it.
 */
#ifndef BTDF_ORACLE_H
#define BTDF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_sim ora_sim;

/* bc_x: 0 periodic, 1 inlet (x = 0, velocity u_in) / zero-gradient outlet,
 * 2 the same inlet with a convective outlet (d f / dt + u_in d f / dx = 0,
 * implicit upwind in time and space), 3 a prescribed-velocity box (every
 * outer node by non-equilibrium extrapolation to the velocity set with
 * oracle_set_boundary_velocity; bc_y is then ignored).
 * bc_y: 0 periodic, 1 free-slip walls, 2 no-slip walls (half-way bounce-back).
 * delta: 2, 3, 4 (Eqs. 37-39) or 5 (4-point cosine).  nf: forcing passes. */
ora_sim *oracle_create(int nx, int ny, double tau, double u_in, int bc_x, int bc_y,
                       double gx, double gy, int delta, int nf);
void oracle_destroy(ora_sim *s);

/* f = f_eq(rho, u) at every node (Eq. 6); arrays are ny*nx, x fastest. */
void oracle_init_fields(ora_sim *s, const double *rho, const double *ux, const double *uy);
/* Raw population access, ny*nx*9 doubles, AoS. */
void oracle_get_pops(const ora_sim *s, double *out);
void oracle_set_pops(ora_sim *s, const double *in);
/* Re-applies the inlet rule (non-equilibrium extrapolation from column 1,
 * Sec. 5.2 inflow) to the current post-streaming populations with the
 * simulation's own u_in; no effect without an inlet.  A state taken from a
 * simulation with another inlet speed then continues as if that speed had
 * been in force at the last streaming. */
void oracle_apply_inlet(ora_sim *s);
/* Outer-node velocities of a bc_x = 3 lattice, 2 nx + 2 (ny - 2) values each
 * in perimeter order: row 0 (x = 0..nx-1), row ny-1, column 0 (y = 1..ny-2),
 * column nx-1 (y = 1..ny-2).  Zero until set. */
void oracle_set_boundary_velocity(ora_sim *s, const double *ubx, const double *uby);

/* One body of n markers; drs <= 0 takes the paper's constant for the delta.
 * Returns the body index. */
int oracle_add_body(ora_sim *s, int n, const double *X, const double *Y,
                    const double *Ubx, const double *Uby, double ds, double drs);
void oracle_set_marker_velocity(ora_sim *s, int body, const double *Ubx, const double *Uby);

void oracle_step(ora_sim *s, int64_t nsteps);
int64_t oracle_step_count(const ora_sim *s);

/* rho and unforced velocity u* (Eqs. 9-10) of the current populations. */
void oracle_moments(const ora_sim *s, double *rho, double *ux, double *uy);
/* IB force density f on the Eulerian nodes from the last step (ny*nx each). */
void oracle_force_field(const ora_sim *s, double *fx, double *fy);
/* Body force F_p per step (Eq. 27, force on the body); returns count copied. */
int64_t oracle_history(const ora_sim *s, int body, int64_t first, int64_t n,
                       double *Fx, double *Fy);
/* Per-marker diagnostics of the last step: U* interpolated from the unforced
 * field (first pass), total F_b, interpolated corrected velocity D_I u after
 * forcing, interpolated density. Any pointer may be NULL. */
void oracle_marker_diag(const ora_sim *s, int body, double *Usx, double *Usy,
                        double *Fbx, double *Fby, double *Ux, double *Uy, double *rho_l);
double oracle_body_drs(const ora_sim *s, int body);

/* Building blocks, exported for the pins. */
double oracle_delta(int kind, double r);                 /* Eqs. 37-39, cosine */
double oracle_drs_paper(int kind);                       /* Sec. 4.4 constants */
int oracle_support_width(int kind);
/* Support nodes of a point (X, Y) under this lattice's boundary rules:
 * node indices (y*nx + x) and weights delta(x-X) delta(y-Y) (Eq. 14). */
int oracle_support(const ora_sim *s, double X, double Y, int64_t *nodes, double *w);
/* D_I of body b applied to arbitrary Eulerian fields (Eq. 12/14). */
void oracle_interp(const ora_sim *s, int body, const double *fx, const double *fy,
                   double *Ux, double *Uy);
/* D_E of body b applied to arbitrary Lagrangian forces (Eq. 13/15);
 * accumulates into the Eulerian arrays. */
void oracle_spread(const ora_sim *s, int body, const double *Fx, const double *Fy,
                   double *fx, double *fy);
/* Local thickness of every marker of body b from Eqs. 22, 24, 25 (solved
 * densely); returns 0 on success, -1 if the matrix is singular. */
int oracle_drs_local(const ora_sim *s, int body, double *drs_out);
/* Equilibrium (Eq. 6) and Guo forcing term (Eq. 7) at one node. */
void oracle_feq(double rho, double ux, double uy, double *out9);
void oracle_guo(double tau, double ux, double uy, double fx, double fy, double *out9);

void oracle_set_threads(int n);
int oracle_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
