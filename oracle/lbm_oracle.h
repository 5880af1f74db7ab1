/*
 * FP64 CPU oracle for the site-based particle-suspension lattice Boltzmann method
 * (dos Santos & Philippi, "An alternative method for simulating particle suspensions
 * using lattice Boltzmann", arXiv:1105.2904).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, plain reference that the CUDA
 * path is checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.
 *
 * Units are lattice units (dx = dt = 1). Distributions are stored as f[i][z][y][x]
 * (x fastest), i = 0..Q-1 in the velocity order documented in lbm_oracle.c.
 * Tags use the encoding (class << 30) | particle_id with class 0 = IS (internal site),
 * 1 = BS (boundary site), 2 = IN (other solid site); 0xFFFFFFFF = fluid.
 *
 * Parity-pinned by tests/test_oracle_*.py (closed forms, invariants, brute force).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osim osim;

/* lattice: 0 = D2Q9 (nz must be 1), 1 = D3Q19. F = fluid body-force density (Guo). */
osim* osim_create(int lattice, int nx, int ny, int nz, double tau, const double F[3]);
void osim_destroy(osim* s);

/* walls[k] = 1: no-slip halfway bounce-back walls at both ends of axis k, 0: periodic. */
int osim_set_walls(osim* s, const int walls[3]);
/* Tangential velocity of a wall face (0..5 = -x,+x,-y,+y,-z,+z); the face must be a wall.
 * Returns 0, or <0 if the face is periodic or u has a normal component. */
int osim_set_wall_velocity(osim* s, int face, const double u[3]);
/* Makes a wall face an equilibrium face (R16) imposing velocity u (any direction): fluid
 * sites on it take f^eq(rho, u) after the collision; moves through it bounce back without a
 * wall-momentum term. Later osim_set_wall_velocity calls on the face change u. Returns 0, or
 * <0 if the face is periodic. */
int osim_set_equilibrium_face(osim* s, int face, const double u[3]);
/* gravity on particles (net buoyant), contact gap, whether F also acts on particles (F/rho_p). */
void osim_set_particle_options(osim* s, const double g[3], double gap, int body_force_on_particles);

/* Adds n particles (before the first step). density = +INFINITY marks a fixed particle.
 * vel / omega may be NULL (zero). Returns 0 on success, <0 on invalid input. */
int osim_add_particles(osim* s, int n, const double* centers, const double* radii,
                       const double* densities, const double* vel, const double* omega);

void osim_step(osim* s, int nsteps);

void osim_get_f(const osim* s, double* f);
void osim_set_f(osim* s, const double* f);
/* rho[N], u[N*3] with u = (sum f c + F/2)/rho, the velocity the collision uses. */
void osim_get_fields(const osim* s, double* rho, double* u);
/* x,u,omega: n*3; force = -dP_B and torque = -dL_B of the last step (n*3 each). */
void osim_get_particles(const osim* s, double* x, double* u, double* omega,
                        double* force, double* torque);
void osim_get_tags(const osim* s, unsigned* tags);
/* Orientation of each particle, n*4: unit quaternion (w, x, y, z), identity when added,
 * turned every step by |omega| about omega (space frame) after the acceleration. */
void osim_get_orientations(const osim* s, double* q);
/* Momentum handed to the fluid in the last step: diag[0..2] = sum of dP_B over all
 * particles, diag[3..5] = momentum change caused by the IS imposition. */
void osim_get_diagnostics(const osim* s, double* diag);
int osim_num_particles(const osim* s);
/* Template of particle p: number of solid sites, and (if out != NULL) the entries as
 * 4 ints each (ox, oy, oz, class) in z,y,x lexicographic order. */
int osim_get_template(const osim* s, int p, int* out);

/* Test hook: runs only the particle-particle / particle-wall contact step (Eqs. 16-19)
 * on the given velocities, with the positions currently held. u is n*3, in/out. */
void osim_resolve_contacts(osim* s, double* u);

/* Single-site collision (Eq. 3 with Guo forcing): fin[Q] -> fout[Q]. */
void osim_collide_site(const osim* s, const double* fin, double* fout);

#ifdef __cplusplus
}
#endif
#endif
