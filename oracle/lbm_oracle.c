/*
 * FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).
 *
 * A literal, single-threaded restatement of the site-based particle-suspension method of
 * dos Santos & Philippi (arXiv:1105.2904). One time step follows the paper's order:
 *
 *   1. collide every site, solids included (Sec. 2.1, Eq. 3; Sec. 2.2 "all sites will be
 *      updated by the usual collision/propagation steps"),
 *   2. particle-fluid momentum transfer at the boundary sites (Sec. 2.2, Eqs. 5-9),
 *   3. particle acceleration (Eqs. 10-11),
 *   4. hard-core particle-particle and particle-wall collisions (Sec. 2.3, Eqs. 16-19),
 *      "part of the particle's acceleration substep",
 *   5. position update (Eqs. 13-15) and orientation (a unit quaternion turned by the angular
 *      velocity over the step),
 *   6. velocity of the internal sites at the new position (Eq. 12),
 *   7. propagation (Eq. 3, left-hand side), with halfway bounce-back at solid walls.
 *
 * Readings of points the paper leaves silent or garbled (each one is documented in the
 * project's design notes, and pinned by a test where a pin exists):
 *   R1 equilibrium: standard second-order polynomial with c_s^2 = 1/3 (Sec. 2.1; tau = 0.6
 *      giving nu = 1/30 in Sec. 3.2 fixes c_s^2 = 1/3 through Eq. 4).
 *   R2 particle sites: S = {y : |y - x_p0|^2 <= r^2}; BS = sites of S with a lattice
 *      neighbour (model velocity set) outside S; IS = other sites of S with a neighbour in
 *      BS; IN = the rest of S.
 *   R3 moving sites: x_B(t) = x_B0 + (x_p(t) - x_p0) (Eqs. 14-15), so [x_B] is the initial
 *      set translated by the integer shift s = floor(x_p - x_p0 + 1/2); the lever arm
 *      x_B - x_p = y0 - x_p0 is constant.
 *   R4 Eq. 5 / Eq. 12 sign: u' = u_p + omega_p x (x_B - x_p) (a rigid-body velocity; the
 *      printed operand order would spin a particle up in still fluid).
 *   R5 rho in f^eq(rho, u'): the site's own density (rho_B, rho_I).
 *   R6 u_B: post-collision momentum over rho_B.
 *   R7 overlapping claims: one owner per site, IS beats BS beats IN, then the lowest id;
 *      the owner map is rebuilt after every position update.
 *   R8 fluid body force: Guo forcing at every site; optionally F/rho_p on particles.
 *   R9 gravity on particles: net buoyant acceleration (1 - rho_f/rho_p) g, rho_f = 1.
 *   R10 particle-wall: the wall is an infinite-mass hard-core partner.
 *   R11 contact trigger: predicted overlap |(x_i+u_i')-(x_j+u_j')| < r_i+r_j+gap with the
 *      post-acceleration velocities; candidate pairs processed once in (i,j) order, each
 *      reflected only if still approaching.
 *   R12 mass and inertia: continuum values of a sphere (3D) or disk (2D).
 *   R15 moving walls (velocity-imposed boundaries of Secs. 3.1-3.2, mechanism not given):
 *      halfway bounce-back with the wall-momentum term -6 w_i (c_i . u_w), density 1.
 *   R16 equilibrium faces (the paper's own way of imposing a velocity at a site, Sec. 2.2,
 *      applied to a domain face): moves that leave the domain through such a face bounce
 *      back (no wall-momentum term); after the collision every fluid site lying on the
 *      face takes f^eq(rho, u_face), rho its post-collision density. A site on several
 *      equilibrium faces takes the first of -x, +x, -y, +y, -z, +z.
 *
 * Distribution layout f[i][z][y][x]; lattice velocity order below.
 * Compile with -ffp-contract=off: the arithmetic is meant to be evaluated exactly as written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "lbm_oracle.h"

#define MAXQ 19
#define TAG_FLUID 0xFFFFFFFFu
#define CLS_IS 0u
#define CLS_BS 1u
#define CLS_IN 2u
#define ORACLE_PI 3.14159265358979323846

typedef struct {
    int Q, D;
    int c[MAXQ][3];
    double w[MAXQ];
    int opp[MAXQ];
} olat;

typedef struct {
    double x0[3];    /* centre when the particle was added */
    int A[3];        /* floor(x0) */
    double phi[3];   /* x0 - A, fractional part */
    double x[3], u[3], om[3];
    double r, inv_m, inv_I, inv_rho, ext[3];
    double q[4];     /* orientation, unit quaternion (w, x, y, z); identity when added */
    int s[3];        /* integer shift of the site set (R3) */
    int nt;          /* number of solid sites in the template */
    int* tmpl;       /* nt entries of (ox, oy, oz, class) relative to A */
    double dP[3], dL[3];
} opart;

struct osim {
    olat L;
    int nx, ny, nz;
    long N;
    double tau, omega, F[3];
    int walls[3];
    double wall_u[6][3]; /* velocity of each face (-x,+x,-y,+y,-z,+z); tangential */
    int eqface[6];       /* 1: equilibrium face (R16) */
    double eq_u[6][3];   /* velocity imposed on an equilibrium face */
    double g[3], gap;
    int bfp;
    double* f;    /* state at the start of a step (pre-collision), [Q][N] */
    double* fp;   /* post-collision work array, [Q][N] */
    unsigned* tag;
    int np, started;
    opart* P;
    double diag[6];
};

/* D2Q9 and D3Q19 velocity sets (Fig. 1 for D2Q9; D3Q19 is the 3D set the method is run
 * with here) and their weights. */
static void lattice_init(olat* L, int lattice)
{
    memset(L, 0, sizeof(*L));
    if (lattice == 0) {
        static const int c2[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                     {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
        L->Q = 9;
        L->D = 2;
        for (int i = 0; i < 9; i++) {
            L->c[i][0] = c2[i][0];
            L->c[i][1] = c2[i][1];
            L->c[i][2] = 0;
            L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else {
        static const int c3[19][3] = {
            {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
            {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
            {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        L->Q = 19;
        L->D = 3;
        for (int i = 0; i < 19; i++) {
            for (int k = 0; k < 3; k++) L->c[i][k] = c3[i][k];
            L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
    }
    for (int i = 0; i < L->Q; i++)
        for (int j = 0; j < L->Q; j++)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
}

/* Second-order equilibrium (R1). */
static double feq(const olat* L, int i, double rho, const double u[3])
{
    double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

/* BGK collision of one site with Guo forcing (Eq. 3 right-hand side, R8):
 * rho = sum f (Eq. 1), rho u = sum f c + F/2 (Eq. 2 plus the half-force shift). */
static void collide(const osim* s, const double* fin, double* fout)
{
    const olat* L = &s->L;
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3];
    for (int i = 0; i < L->Q; i++) rho += fin[i];
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < L->Q; i++) j[k] += fin[i] * L->c[i][k];
    for (int k = 0; k < 3; k++) u[k] = (j[k] + 0.5 * s->F[k]) / rho;
    double pre = 1.0 - 0.5 / s->tau;
    double uF = u[0] * s->F[0] + u[1] * s->F[1] + u[2] * s->F[2];
    for (int i = 0; i < L->Q; i++) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        double cF = L->c[i][0] * s->F[0] + L->c[i][1] * s->F[1] + L->c[i][2] * s->F[2];
        double Si = pre * L->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
        fout[i] = fin[i] - s->omega * (fin[i] - feq(L, i, rho, u)) + Si;
    }
}

static int axis_len(const osim* s, int k) { return k == 0 ? s->nx : (k == 1 ? s->ny : s->nz); }

/* Lattice site of template offset o of particle p at its current shift, or -1 when the
 * site lies beyond a solid wall (such sites are skipped). Periodic axes wrap. */
static long site_of(const osim* s, const opart* p, const int* o)
{
    long idx = 0, stride = 1;
    for (int k = 0; k < 3; k++) {
        int n = axis_len(s, k);
        long v = (long)p->A[k] + p->s[k] + o[k];
        if (s->walls[k]) {
            if (v < 0 || v >= n) return -1;
        } else {
            v %= n;
            if (v < 0) v += n;
        }
        idx += v * stride;
        stride *= n;
    }
    return idx;
}

/* Classifies the solid sites of a particle around its initial centre (R2) and stores them
 * in z, y, x lexicographic order of their offsets from A = floor(x0). */
static int build_template(const osim* s, opart* p)
{
    const olat* L = &s->L;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, ex[3];
    for (int k = 0; k < L->D; k++) {
        lo[k] = (int)floor(p->phi[k] - p->r) - 1;
        hi[k] = (int)ceil(p->phi[k] + p->r) + 1;
    }
    for (int k = 0; k < 3; k++) ex[k] = hi[k] - lo[k] + 1;
    long box = (long)ex[0] * ex[1] * ex[2];
    unsigned char* inS = calloc((size_t)box, 1);
    unsigned char* cls = calloc((size_t)box, 1); /* 0 none, 1 BS, 2 IS, 3 IN */
    if (!inS || !cls) return -1;
    double r2 = p->r * p->r;
#define BOXI(a, b, c) ((((long)(c)-lo[2]) * ex[1] + ((b)-lo[1])) * ex[0] + ((a)-lo[0]))
    for (int oz = lo[2]; oz <= hi[2]; oz++)
        for (int oy = lo[1]; oy <= hi[1]; oy++)
            for (int ox = lo[0]; ox <= hi[0]; ox++) {
                double dx = (double)ox - p->phi[0];
                double dy = (double)oy - p->phi[1];
                double dz = (double)oz - p->phi[2];
                double d2 = dx * dx + dy * dy + dz * dz;
                inS[BOXI(ox, oy, oz)] = (d2 <= r2);
            }
    /* BS: solid site with at least one neighbour outside S. */
    for (int oz = lo[2]; oz <= hi[2]; oz++)
        for (int oy = lo[1]; oy <= hi[1]; oy++)
            for (int ox = lo[0]; ox <= hi[0]; ox++) {
                if (!inS[BOXI(ox, oy, oz)]) continue;
                int bs = 0;
                for (int i = 1; i < L->Q; i++)
                    if (!inS[BOXI(ox + L->c[i][0], oy + L->c[i][1], oz + L->c[i][2])]) bs = 1;
                if (bs) cls[BOXI(ox, oy, oz)] = 1;
            }
    /* IS: remaining solid site with at least one neighbour in BS; IN: the rest. */
    for (int oz = lo[2]; oz <= hi[2]; oz++)
        for (int oy = lo[1]; oy <= hi[1]; oy++)
            for (int ox = lo[0]; ox <= hi[0]; ox++) {
                long b = BOXI(ox, oy, oz);
                if (!inS[b] || cls[b] == 1) continue;
                int is = 0;
                for (int i = 1; i < L->Q; i++)
                    if (cls[BOXI(ox + L->c[i][0], oy + L->c[i][1], oz + L->c[i][2])] == 1) is = 1;
                cls[b] = is ? 2 : 3;
            }
    int nt = 0;
    for (long b = 0; b < box; b++) nt += inS[b];
    p->tmpl = malloc(sizeof(int) * 4 * (size_t)(nt > 0 ? nt : 1));
    if (!p->tmpl) return -1;
    int e = 0;
    for (int oz = lo[2]; oz <= hi[2]; oz++)
        for (int oy = lo[1]; oy <= hi[1]; oy++)
            for (int ox = lo[0]; ox <= hi[0]; ox++) {
                long b = BOXI(ox, oy, oz);
                if (!inS[b]) continue;
                unsigned c = cls[b] == 1 ? CLS_BS : (cls[b] == 2 ? CLS_IS : CLS_IN);
                p->tmpl[4 * e + 0] = ox;
                p->tmpl[4 * e + 1] = oy;
                p->tmpl[4 * e + 2] = oz;
                p->tmpl[4 * e + 3] = (int)c;
                e++;
            }
#undef BOXI
    p->nt = nt;
    free(inS);
    free(cls);
    return 0;
}

/* Owner map (R7): lowest (class << 30 | id) wins. Rebuilt from scratch. */
static void rebuild_tags(osim* s)
{
    for (long x = 0; x < s->N; x++) s->tag[x] = TAG_FLUID;
    for (int p = 0; p < s->np; p++) {
        opart* P = &s->P[p];
        for (int e = 0; e < P->nt; e++) {
            long y = site_of(s, P, &P->tmpl[4 * e]);
            if (y < 0) continue;
            unsigned code = ((unsigned)P->tmpl[4 * e + 3] << 30) | (unsigned)p;
            if (code < s->tag[y]) s->tag[y] = code;
        }
    }
}

/* Rigid-body velocity at lever arm r (R4): u + omega x r. */
static void rigid_velocity(const double u[3], const double om[3], const double r[3], double out[3])
{
    out[0] = u[0] + (om[1] * r[2] - om[2] * r[1]);
    out[1] = u[1] + (om[2] * r[0] - om[0] * r[2]);
    out[2] = u[2] + (om[0] * r[1] - om[1] * r[0]);
}

static void lever_arm(const opart* P, const int* o, double r[3])
{
    for (int k = 0; k < 3; k++) r[k] = (double)o[k] - P->phi[k];
}

/* Orientation update of the rigid-body integration (Sec. 2.2: the particle moves with the
 * velocities of Eqs. 10-11 over the step, Eq. 13 for the position). The orientation is the
 * unit quaternion q = (w, x, y, z); turning at the angular velocity omega (space frame),
 * held over the step dt = 1, rotates the body by theta = |omega| about omega/|omega|:
 * q' = dq q with dq = (cos(theta/2), sin(theta/2) omega/|omega|) (Hamilton product,
 * dq applied in the space frame), then q' is divided by its norm. The spheres' dynamics
 * do not depend on it; it is bookkeeping of the body's attitude. */
static void rotate_orientation(double q[4], const double om[3])
{
    double th = sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
    if (th == 0.0) return;
    double c = cos(0.5 * th), sn = sin(0.5 * th) / th;
    double d[4] = {c, sn * om[0], sn * om[1], sn * om[2]};
    double r[4];
    r[0] = d[0] * q[0] - (d[1] * q[1] + d[2] * q[2] + d[3] * q[3]);
    r[1] = d[0] * q[1] + q[0] * d[1] + (d[2] * q[3] - d[3] * q[2]);
    r[2] = d[0] * q[2] + q[0] * d[2] + (d[3] * q[1] - d[1] * q[3]);
    r[3] = d[0] * q[3] + q[0] * d[3] + (d[1] * q[2] - d[2] * q[1]);
    double nrm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int k = 0; k < 4; k++) q[k] = r[k] / nrm;
}

static double min_image(double d, int n, int periodic)
{
    if (!periodic) return d;
    return d - (double)n * floor(d / (double)n + 0.5);
}

osim* osim_create(int lattice, int nx, int ny, int nz, double tau, const double F[3])
{
    if (lattice != 0 && lattice != 1) return NULL;
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == 0 && nz != 1) || !(tau > 0.5)) return NULL;
    osim* s = calloc(1, sizeof(osim));
    if (!s) return NULL;
    lattice_init(&s->L, lattice);
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->N = (long)nx * ny * nz;
    s->tau = tau;
    s->omega = 1.0 / tau;
    for (int k = 0; k < 3; k++) s->F[k] = F ? F[k] : 0.0;
    if (lattice == 0) s->F[2] = 0.0;
    s->f = malloc(sizeof(double) * (size_t)s->L.Q * (size_t)s->N);
    s->fp = malloc(sizeof(double) * (size_t)s->L.Q * (size_t)s->N);
    s->tag = malloc(sizeof(unsigned) * (size_t)s->N);
    if (!s->f || !s->fp || !s->tag) {
        osim_destroy(s);
        return NULL;
    }
    for (int i = 0; i < s->L.Q; i++)
        for (long x = 0; x < s->N; x++) s->f[(long)i * s->N + x] = s->L.w[i];
    for (long x = 0; x < s->N; x++) s->tag[x] = TAG_FLUID;
    return s;
}

void osim_destroy(osim* s)
{
    if (!s) return;
    for (int p = 0; p < s->np; p++) free(s->P[p].tmpl);
    free(s->P);
    free(s->f);
    free(s->fp);
    free(s->tag);
    free(s);
}

int osim_set_walls(osim* s, const int walls[3])
{
    if (s->np > 0) return -1;
    for (int k = 0; k < 3; k++) s->walls[k] = walls[k] ? 1 : 0;
    if (s->L.D == 2) s->walls[2] = 0;
    return 0;
}

int osim_set_equilibrium_face(osim* s, int face, const double u[3])
{
    if (face < 0 || face > 5 || !s->walls[face / 2]) return -1;
    s->eqface[face] = 1;
    for (int k = 0; k < 3; k++) {
        s->eq_u[face][k] = (s->L.D == 2 && k == 2) ? 0.0 : u[k];
        s->wall_u[face][k] = 0.0;
    }
    return 0;
}

int osim_set_wall_velocity(osim* s, int face, const double u[3])
{
    if (face < 0 || face > 5 || !s->walls[face / 2]) return -1;
    if (s->eqface[face]) return osim_set_equilibrium_face(s, face, u);
    if (u[face / 2] != 0.0) return -2; /* the wall plane does not move along its normal */
    for (int k = 0; k < 3; k++) s->wall_u[face][k] = (s->L.D == 2 && k == 2) ? 0.0 : u[k];
    return 0;
}

void osim_set_particle_options(osim* s, const double g[3], double gap, int bfp)
{
    for (int k = 0; k < 3; k++) s->g[k] = g ? g[k] : 0.0;
    if (s->L.D == 2) s->g[2] = 0.0;
    s->gap = gap;
    s->bfp = bfp ? 1 : 0;
}

int osim_add_particles(osim* s, int n, const double* centers, const double* radii,
                       const double* densities, const double* vel, const double* omega)
{
    const int D = s->L.D;
    if (s->started) return -1;
    if (n < 0) return -2;
    opart* P = realloc(s->P, sizeof(opart) * (size_t)(s->np + n + 1));
    if (!P) return -7;
    s->P = P;
    int built = 0, err = 0;
    for (int q = 0; q < n; q++) {
        opart* p = &s->P[s->np + q];
        memset(p, 0, sizeof(*p));
        p->r = radii[q];
        double rho = densities[q];
        if (!(p->r >= 1.5)) { err = -2; goto fail; }
        if (!(rho > 0.0)) { err = -3; goto fail; }
        for (int k = 0; k < 3; k++) {
            p->x0[k] = (k < D) ? centers[3 * q + k] : 0.0;
            p->x[k] = p->x0[k];
            p->u[k] = (vel && k < D) ? vel[3 * q + k] : 0.0;
            p->om[k] = omega ? omega[3 * q + k] : 0.0;
            if (D == 2 && k < 2) p->om[k] = 0.0;
            p->A[k] = (int)floor(p->x0[k]);
            p->phi[k] = p->x0[k] - (double)p->A[k];
            p->s[k] = 0;
        }
        p->q[0] = 1.0;
        p->q[1] = p->q[2] = p->q[3] = 0.0;
        for (int k = 0; k < D; k++) {
            int nk = axis_len(s, k);
            if (s->walls[k]) {
                if (p->x0[k] + 0.5 < p->r || ((double)nk - 0.5) - p->x0[k] < p->r) { err = -5; goto fail; }
            } else if (2.0 * (p->r + 2.0) >= (double)nk) {
                err = -4;
                goto fail;
            }
        }
        /* R12: continuum mass and moment of inertia; infinite density = fixed particle. */
        if (isinf(rho)) {
            p->inv_rho = 0.0;
            p->inv_m = 0.0;
            p->inv_I = 0.0;
        } else {
            double vol = (D == 3) ? (4.0 / 3.0) * ORACLE_PI * p->r * p->r * p->r : ORACLE_PI * p->r * p->r;
            double m = rho * vol;
            double I = (D == 3) ? 0.4 * m * p->r * p->r : 0.5 * m * p->r * p->r;
            p->inv_rho = 1.0 / rho;
            p->inv_m = 1.0 / m;
            p->inv_I = 1.0 / I;
        }
        for (int k = 0; k < 3; k++) {
            if (p->inv_rho == 0.0)
                p->ext[k] = 0.0;
            else
                p->ext[k] = s->g[k] * (1.0 - p->inv_rho) + (s->bfp ? s->F[k] * p->inv_rho : 0.0);
        }
        /* Hard-core particles may not overlap (Sec. 2.3). */
        for (int o = 0; o < s->np + q; o++) {
            opart* b = &s->P[o];
            double d2 = 0.0;
            for (int k = 0; k < 3; k++) {
                double d = min_image(p->x0[k] - b->x[k], axis_len(s, k), !s->walls[k] && k < D);
                d2 += d * d;
            }
            if (d2 < (p->r + b->r) * (p->r + b->r)) { err = -6; goto fail; }
        }
        if (build_template(s, p) != 0) { err = -7; goto fail; }
        built++;
    }
    s->np += n;
    rebuild_tags(s);
    return 0;
fail:
    for (int q = 0; q < built; q++) free(s->P[s->np + q].tmpl);
    return err;
}

/* Hard-core collisions (Sec. 2.3, Eqs. 16-19; readings R10, R11). In the centre-of-mass
 * frame the normal components reverse and the tangential ones are kept; with inverse
 * masses a_i, a_j and approach rate w = (u_j - u_i).n < 0 this is
 * u_i += 2 a_i w/(a_i+a_j) n, u_j -= 2 a_j w/(a_i+a_j) n. */
static void contacts(osim* s, double* u)
{
    const int D = s->L.D;
    int np = s->np;
    int cap = 64, npair = 0;
    int* pairs = malloc(sizeof(int) * 2 * (size_t)cap);
    for (int i = 0; i < np; i++)
        for (int j = i + 1; j < np; j++) {
            opart *a = &s->P[i], *b = &s->P[j];
            double d2 = 0.0;
            for (int k = 0; k < 3; k++) {
                double pd = (b->x[k] + u[3 * j + k]) - (a->x[k] + u[3 * i + k]);
                pd = min_image(pd, axis_len(s, k), !s->walls[k] && k < D);
                d2 += pd * pd;
            }
            double R = a->r + b->r + s->gap;
            if (d2 < R * R) {
                if (npair == cap) {
                    cap *= 2;
                    pairs = realloc(pairs, sizeof(int) * 2 * (size_t)cap);
                }
                pairs[2 * npair] = i;
                pairs[2 * npair + 1] = j;
                npair++;
            }
        }
    for (int q = 0; q < npair; q++) {
        int i = pairs[2 * q], j = pairs[2 * q + 1];
        opart *a = &s->P[i], *b = &s->P[j];
        double den = a->inv_m + b->inv_m;
        if (den == 0.0) continue;
        double d[3], n[3];
        for (int k = 0; k < 3; k++) d[k] = min_image(b->x[k] - a->x[k], axis_len(s, k), !s->walls[k] && k < D);
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (dn == 0.0) continue;
        for (int k = 0; k < 3; k++) n[k] = d[k] / dn;
        double w = (u[3 * j + 0] - u[3 * i + 0]) * n[0] + (u[3 * j + 1] - u[3 * i + 1]) * n[1] +
                   (u[3 * j + 2] - u[3 * i + 2]) * n[2];
        if (!(w < 0.0)) continue;
        double ci = 2.0 * a->inv_m * w / den;
        double cj = 2.0 * b->inv_m * w / den;
        for (int k = 0; k < 3; k++) {
            u[3 * i + k] = u[3 * i + k] + ci * n[k];
            u[3 * j + k] = u[3 * j + k] - cj * n[k];
        }
    }
    free(pairs);
    /* Walls: planes at -1/2 and n - 1/2 of each no-slip axis. */
    for (int p = 0; p < np; p++) {
        opart* a = &s->P[p];
        if (a->inv_m == 0.0) continue;
        double R = a->r + s->gap;
        for (int k = 0; k < D; k++) {
            if (!s->walls[k]) continue;
            double xp = a->x[k] + u[3 * p + k];
            double lo = xp + 0.5;
            double hi = ((double)axis_len(s, k) - 0.5) - xp;
            if (lo < R && u[3 * p + k] < 0.0)
                u[3 * p + k] = -u[3 * p + k];
            else if (hi < R && u[3 * p + k] > 0.0)
                u[3 * p + k] = -u[3 * p + k];
        }
    }
}

void osim_resolve_contacts(osim* s, double* u) { contacts(s, u); }

static void step_once(osim* s)
{
    const olat* L = &s->L;
    const int Q = L->Q, D = L->D;
    const long N = s->N;
    s->started = 1;
    for (int k = 0; k < 6; k++) s->diag[k] = 0.0;

    /* 1. Collision at every site. (The sites are independent; an OpenMP build splits this
     * loop and the propagation loop between threads without changing any site's arithmetic.) */
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; x++) {
        double fin[MAXQ] = {0}, fout[MAXQ] = {0};
        for (int i = 0; i < Q; i++) fin[i] = s->f[(long)i * N + x];
        collide(s, fin, fout);
        for (int i = 0; i < Q; i++) s->fp[(long)i * N + x] = fout[i];
    }

    /* 1b. Equilibrium faces (R16): fluid sites on such a face take f^eq(rho, u_face). */
    if (s->eqface[0] || s->eqface[1] || s->eqface[2] || s->eqface[3] || s->eqface[4] || s->eqface[5]) {
        for (int z = 0; z < s->nz; z++)
            for (int y = 0; y < s->ny; y++)
                for (int x = 0; x < s->nx; x++) {
                    const int pos[3] = {x, y, z}, n3[3] = {s->nx, s->ny, s->nz};
                    int face = -1;
                    for (int f = 0; f < 6 && face < 0; f++)
                        if (s->eqface[f] && pos[f / 2] == ((f & 1) ? n3[f / 2] - 1 : 0)) face = f;
                    const long site = ((long)z * s->ny + y) * s->nx + x;
                    if (face < 0 || (s->np > 0 && s->tag[site] != TAG_FLUID)) continue;
                    double rho = 0.0;
                    for (int i = 0; i < Q; i++) rho += s->fp[(long)i * N + site];
                    for (int i = 0; i < Q; i++) s->fp[(long)i * N + site] = feq(L, i, rho, s->eq_u[face]);
                }
    }

    /* 2. Particle-fluid momentum transfer at the BS sites (Eqs. 5-9). */
    for (int p = 0; p < s->np; p++) {
        opart* P = &s->P[p];
        for (int k = 0; k < 3; k++) P->dP[k] = P->dL[k] = 0.0;
        for (int e = 0; e < P->nt; e++) {
            const int* o = &P->tmpl[4 * e];
            if ((unsigned)o[3] != CLS_BS) continue;
            long y = site_of(s, P, o);
            if (y < 0 || s->tag[y] != ((CLS_BS << 30) | (unsigned)p)) continue;
            double rhoB = 0.0, jB[3] = {0.0, 0.0, 0.0}, uB[3], r[3], uBp[3], du[3], cr[3];
            for (int i = 0; i < Q; i++) rhoB += s->fp[(long)i * N + y];
            for (int k = 0; k < 3; k++)
                for (int i = 0; i < Q; i++) jB[k] += s->fp[(long)i * N + y] * L->c[i][k];
            for (int k = 0; k < 3; k++) uB[k] = jB[k] / rhoB;
            lever_arm(P, o, r);
            rigid_velocity(P->u, P->om, r, uBp);
            for (int i = 0; i < Q; i++) s->fp[(long)i * N + y] = feq(L, i, rhoB, uBp);
            for (int k = 0; k < 3; k++) du[k] = uBp[k] - uB[k];
            cr[0] = r[1] * du[2] - r[2] * du[1];
            cr[1] = r[2] * du[0] - r[0] * du[2];
            cr[2] = r[0] * du[1] - r[1] * du[0];
            for (int k = 0; k < 3; k++) {
                P->dP[k] += rhoB * du[k];
                P->dL[k] += rhoB * cr[k];
            }
        }
        for (int k = 0; k < 3; k++) s->diag[k] += P->dP[k];
    }

    /* 3. Particle acceleration (Eqs. 10-11, R8, R9). */
    double* un = malloc(sizeof(double) * 3 * (size_t)(s->np > 0 ? s->np : 1));
    for (int p = 0; p < s->np; p++) {
        opart* P = &s->P[p];
        for (int k = 0; k < 3; k++) {
            un[3 * p + k] = (P->u[k] - P->dP[k] * P->inv_m) + P->ext[k];
            P->om[k] = P->om[k] - P->dL[k] * P->inv_I;
        }
    }
    /* 4. Hard-core contacts, part of the acceleration substep (Sec. 2.3). */
    if (s->np > 0) contacts(s, un);
    /* 5. Position update (Eq. 13) and the integer shift of the site set (R3). */
    for (int p = 0; p < s->np; p++) {
        opart* P = &s->P[p];
        for (int k = 0; k < 3; k++) P->u[k] = un[3 * p + k];
        for (int k = 0; k < D; k++) {
            P->x[k] = P->x[k] + P->u[k];
            P->s[k] = (int)floor((P->x[k] - P->x0[k]) + 0.5);
        }
        rotate_orientation(P->q, P->om);
    }
    free(un);
    if (s->np > 0) rebuild_tags(s);

    /* 6. Velocity of the internal sites at the new position (Eq. 12). */
    for (int p = 0; p < s->np; p++) {
        opart* P = &s->P[p];
        for (int e = 0; e < P->nt; e++) {
            const int* o = &P->tmpl[4 * e];
            if ((unsigned)o[3] != CLS_IS) continue;
            long y = site_of(s, P, o);
            if (y < 0 || s->tag[y] != ((CLS_IS << 30) | (unsigned)p)) continue;
            double rhoI = 0.0, r[3], uI[3];
            for (int i = 0; i < Q; i++) rhoI += s->fp[(long)i * N + y];
            lever_arm(P, o, r);
            rigid_velocity(P->u, P->om, r, uI);
            for (int i = 0; i < Q; i++) {
                double old = s->fp[(long)i * N + y];
                double nw = feq(L, i, rhoI, uI);
                s->fp[(long)i * N + y] = nw;
                for (int k = 0; k < 3; k++) s->diag[3 + k] += (nw - old) * L->c[i][k];
            }
        }
    }

    /* 7. Propagation; halfway bounce-back where a move would cross a solid wall. Every
     * (site, direction) has its own target, so z-planes are independent. */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long src = ((long)z * s->ny + y) * s->nx + x;
                int pos[3] = {x, y, z}, n3[3] = {s->nx, s->ny, s->nz};
                for (int i = 0; i < Q; i++) {
                    int t[3], bounce = 0, face = -1;
                    for (int k = 0; k < 3; k++) {
                        t[k] = pos[k] + L->c[i][k];
                        if (t[k] < 0 || t[k] >= n3[k]) {
                            if (s->walls[k]) {
                                bounce = 1;
                                if (face < 0) face = 2 * k + (t[k] >= n3[k] ? 1 : 0);
                            } else {
                                t[k] = (t[k] + n3[k]) % n3[k];
                            }
                        }
                    }
                    double v = s->fp[(long)i * N + src];
                    if (bounce) {
                        /* R15 moving wall (halfway bounce-back with the momentum of a wall moving
                         * at u_w, reference density 1): f_opp(i) = f*_i - 6 w_i (c_i . u_w); a move
                         * crossing two walls takes the wall of its lowest axis. */
                        const double* uw = s->wall_u[face];
                        const double cuw = L->c[i][0] * uw[0] + L->c[i][1] * uw[1] + L->c[i][2] * uw[2];
                        s->f[(long)L->opp[i] * N + src] = v - 6.0 * L->w[i] * cuw;
                    } else
                        s->f[(long)i * N + ((long)t[2] * s->ny + t[1]) * s->nx + t[0]] = v;
                }
            }
}

void osim_step(osim* s, int nsteps)
{
    for (int n = 0; n < nsteps; n++) step_once(s);
}

void osim_get_f(const osim* s, double* f)
{
    memcpy(f, s->f, sizeof(double) * (size_t)s->L.Q * (size_t)s->N);
}

void osim_set_f(osim* s, const double* f)
{
    memcpy(s->f, f, sizeof(double) * (size_t)s->L.Q * (size_t)s->N);
}

void osim_get_fields(const osim* s, double* rho, double* u)
{
    const olat* L = &s->L;
    for (long x = 0; x < s->N; x++) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < L->Q; i++) r += s->f[(long)i * s->N + x];
        for (int k = 0; k < 3; k++)
            for (int i = 0; i < L->Q; i++) j[k] += s->f[(long)i * s->N + x] * L->c[i][k];
        rho[x] = r;
        for (int k = 0; k < 3; k++) u[3 * x + k] = (j[k] + 0.5 * s->F[k]) / r;
    }
}

void osim_get_particles(const osim* s, double* x, double* u, double* omega, double* force,
                        double* torque)
{
    for (int p = 0; p < s->np; p++) {
        const opart* P = &s->P[p];
        for (int k = 0; k < 3; k++) {
            if (x) x[3 * p + k] = P->x[k];
            if (u) u[3 * p + k] = P->u[k];
            if (omega) omega[3 * p + k] = P->om[k];
            if (force) force[3 * p + k] = -P->dP[k];
            if (torque) torque[3 * p + k] = -P->dL[k];
        }
    }
}

void osim_get_orientations(const osim* s, double* q)
{
    for (int p = 0; p < s->np; p++)
        for (int k = 0; k < 4; k++) q[4 * p + k] = s->P[p].q[k];
}

void osim_get_tags(const osim* s, unsigned* tags) { memcpy(tags, s->tag, sizeof(unsigned) * (size_t)s->N); }

void osim_get_diagnostics(const osim* s, double* diag) { memcpy(diag, s->diag, sizeof(double) * 6); }

int osim_num_particles(const osim* s) { return s->np; }

int osim_get_template(const osim* s, int p, int* out)
{
    if (p < 0 || p >= s->np) return -1;
    if (out) memcpy(out, s->P[p].tmpl, sizeof(int) * 4 * (size_t)s->P[p].nt);
    return s->P[p].nt;
}

void osim_collide_site(const osim* s, const double* fin, double* fout) { collide(s, fin, fout); }
