/*
 * lbmp — C-ABI of the GB300 (sm_103a) site-based particle-suspension lattice Boltzmann
 * library (dos Santos & Philippi, "An alternative method for simulating particle
 * suspensions using lattice Boltzmann", arXiv:1105.2904).
 *
 * One time step (lbm_step) is, in the paper's order:
 *   - BGK collision of every lattice site, solids included (Sec. 2.1, Eq. 3), with Guo
 *     body forcing, fused with the pull-propagation of the previous step (Eq. 3 LHS);
 *   - momentum transfer at each particle's boundary sites, BS (Sec. 2.2, Eqs. 5-7) and the
 *     per-particle reduction of the exchanged momentum and angular momentum (Eqs. 8-9);
 *   - particle acceleration (Eqs. 10-11) and hard-core particle-particle and
 *     particle-wall collisions (Sec. 2.3, Eqs. 16-19);
 *   - position update (Eqs. 13-15) and the re-marking of each particle's BS / IS sites;
 *   - equilibrium imposition at the internal sites, IS (Eq. 12), applied as the next
 *     step pulls its populations.
 *
 * Conventions shared by every call:
 *   - Lattice units: dx = dt = 1. Sites are indexed x fastest: idx = x + nx*(y + ny*z).
 *     D2Q9 uses nz = 1 and ignores z components of vectors (omega uses only z).
 *   - Host arrays passed in or out are caller-owned, plain C arrays of double unless
 *     stated; the library copies them synchronously and never keeps the pointers.
 *     Device memory is owned by the library and freed by lbm_destroy.
 *   - Distribution arrays are f[i][z][y][x] with i in the velocity order below.
 *       D2Q9 : (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *       D3Q19: (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1) (1,1,0) (-1,-1,0)
 *              (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1)
 *              (0,1,-1) (0,-1,1)
 *   - Every call returns an lbm_status; none exits, traps or asserts on the device.
 *     Kernels report faults (capacity overflow, a particle moving more than one site per
 *     step, ...) through a device status word that lbm_synchronize and the getters read.
 *     lbm_last_error gives a one-line description of the last non-OK status.
 *   - The library fails loudly: if no CUDA device is usable, lbm_create returns
 *     LBM_E_CUDA. There is no CPU fallback.
 */
#ifndef LBMP_H
#define LBMP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;     /* opaque, library-owned */
typedef struct lbm_batch lbm_batch; /* opaque, library-owned: an ensemble of contexts */

typedef enum {
    LBM_OK = 0,
    LBM_E_INVALID = 1,  /* bad argument (size, tau <= 1/2, radius, wall crossing, ...) */
    LBM_E_OOM = 2,      /* device allocation failed */
    LBM_E_CUDA = 3,     /* a CUDA call failed (no device, launch error, ...) */
    LBM_E_OVERLAP = 4,  /* particles overlap when added */
    LBM_E_TIMEOUT = 5,  /* reserved for a bounded device wait that expired; no kernel of this
                           version waits on another (a step's phases are separate launches in
                           stream order), so none returns it */
    LBM_E_STATE = 6,    /* call not allowed in the current state (e.g. configure after step) */
    LBM_E_NAN = 7,      /* non-finite value detected in the state */
    LBM_E_CAPACITY = 8, /* a device work list overflowed (e.g. contact pairs) */
    LBM_E_UNSTABLE = 9, /* a particle moved by more than one site in one step */
    LBM_E_BOUNDS = 10   /* only in the bounds-checked build (LBM_DEBUG): a kernel found an index
                           out of range and skipped that access */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* Storage precision of the distributions. Arithmetic is FP64 for LBM_FP64 and FP32
 * otherwise; particle state and force/torque sums are FP64 in every mode.
 *   LBM_FP64    : f stored as is (the parity build; evaluates the same IEEE operations as
 *                 a plain FP64 implementation, reductions in a fixed order);
 *   LBM_FP32    : deviation g_i = f_i - w_i stored in FP32;
 *   LBM_FP16DEV : (f_i - w_i)/w_i stored in IEEE half;
 *   LBM_BF16DEV : (f_i - w_i)/w_i stored in bfloat16. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16DEV = 2, LBM_BF16DEV = 3 } lbm_precision;

/* Kinds of domain face. LBM_NOSLIP: halfway bounce-back wall (optionally moving in its own
 * plane, lbm_set_wall_velocity). LBM_EQUILIBRIUM: imposes a velocity the way the method
 * imposes one at a particle's sites (Sec. 2.2, Eqs. 5 and 12): after the collision every
 * fluid site lying on the face takes f^eq(rho, u_face), rho its own post-collision density;
 * moves that leave the domain through it bounce back (no wall-momentum term). The paper
 * imposes free-stream velocities on the faces of its drag runs (Sec. 3.1) without stating
 * the mechanism; this face is the reading that uses the method's own. A site on several
 * equilibrium faces takes the first of -x, +x, -y, +y, -z, +z; particle sites keep the
 * particle treatment. */
typedef enum { LBM_PERIODIC = 0, LBM_NOSLIP = 1, LBM_EQUILIBRIUM = 2 } lbm_face;

/* Creates a simulation of an nx*ny*nz lattice (D2Q9: nz = 1) of BGK fluid with relaxation
 * time tau (viscosity nu = (tau - 1/2)/3, Sec. 2.1 Eq. 4) at rest (f_i = w_i, rho = 1).
 * body_force: force density F applied at every site by Guo forcing; may be NULL (zero).
 * Defaults: LBM_FP32, all faces periodic, no particle gravity, contact gap 0, F not applied
 * to particles, a library-created non-blocking stream.
 * Errors: LBM_E_INVALID (sizes < 1, nz != 1 for D2Q9, tau <= 1/2, more than 2^31 sites),
 *         LBM_E_CUDA (no usable device). *out is NULL on error. */
lbm_status lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau,
                      const double body_force[3]);

/* Sets the storage precision (lbm_precision), the kind of each face (lbm_face; order -x,+x,
 * -y,+y,-z,+z; an axis is periodic on both faces or on neither; NULL = all periodic), the acceleration g of
 * gravity on particles (net buoyant: (1 - 1/rho_p) g, Sec. 3.3-3.4 settling runs; NULL =
 * none), the contact gap added to r_i + r_j in the hard-core trigger (Sec. 2.3), whether F
 * also accelerates particles (F/rho_p), and the CUDA stream (cudaStream_t, may be NULL) on
 * which every later call enqueues its work. Walls are halfway bounce-back planes at -1/2
 * and n - 1/2 (the bounce-back solid of Sec. 3.1).
 * Only allowed before particles are added, distributions set, or a step is taken
 * (LBM_E_STATE). LBM_E_INVALID on a bad enum value or mismatched faces. */
lbm_status lbm_configure(lbm_ctx* ctx, int precision, const int faces[6],
                         const double particle_gravity[3], double contact_gap,
                         int body_force_on_particles, void* cuda_stream);

/* Moves wall face `face` (0..5 = -x,+x,-y,+y,-z,+z) in its own plane with velocity u
 * (xyz; u[face/2] must be 0), or, for an LBM_EQUILIBRIUM face, sets the velocity it imposes
 * (any direction; it applies from the collision of the next step on). The paper drives its shear and channel flows through
 * velocity-imposed walls (Secs. 3.1-3.2) without stating the mechanism; here a population
 * that bounces off a moving wall gains the wall momentum -6 w_i (c_i . u_w) at reference
 * density 1 (halfway bounce-back). A move crossing two walls takes the wall of its lowest
 * axis. The velocity applies from the streaming of the next step on (lbm_get_* still see the
 * last step streamed with the velocity it was taken with); the first step after creation or
 * lbm_set_distributions pulls the given populations as they are. Allowed at any time
 * between steps (the stream is synchronised); lbm_configure clears the velocity of faces it
 * makes periodic.
 * Errors: LBM_E_INVALID (face out of range or periodic, u NULL, not finite, or with a
 * normal component on a no-slip face); LBM_E_CUDA. */
lbm_status lbm_set_wall_velocity(lbm_ctx* ctx, int face, const double u[3]);

/* Adds n rigid spheres (disks for D2Q9) (Sec. 2.2: centre x_p, radius r_p, mass and
 * moment of inertia from the density). centers, velocities and omegas are n*3 (xyz);
 * radii and densities are n. densities are particle/fluid density ratios; +INFINITY makes
 * a fixed particle that never moves. velocities / omegas may be NULL (zero).
 * The particle's lattice sites are classified once, around the given centre, into BS
 * (solid sites with a neighbour outside the sphere), IS (solid sites next to BS) and the
 * rest, and this set then translates rigidly with the particle (Eqs. 14-15).
 * *first_id (may be NULL) receives the id of the first added particle; ids are dense.
 * Only before the first lbm_step (LBM_E_STATE). Errors: LBM_E_INVALID (radius < 1.5 or
 * > 120, density <= 0, sphere wider than half a periodic axis, sphere crossing a wall),
 * LBM_E_OVERLAP (two spheres overlap). On error nothing is added. */
lbm_status lbm_add_particles(lbm_ctx* ctx, int n, const double* centers, const double* radii,
                             const double* densities, const double* velocities,
                             const double* omegas, int* first_id);

/* Enqueues n time steps on the context's stream (replays of a captured CUDA graph) and
 * returns without waiting. Steps never leave the device. n = 0 is a no-op. */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* Waits for the context's stream and returns the device status word (LBM_OK, or the first
 * fault a kernel recorded: LBM_E_CAPACITY, LBM_E_UNSTABLE, ...). */
lbm_status lbm_synchronize(lbm_ctx* ctx);

/* Macroscopic fields of the current state: rho[N] (Eq. 1) and u[N*3] (site-major, xyz)
 * with rho u = sum_i f_i c_i + F/2 (Eq. 2 with the Guo half-force). Synchronizes. */
lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho, double* u);

/* Particle state after the last step, n*3 each (any pointer may be NULL): centre x_p
 * (continuous, not wrapped into periodic boxes), velocity u_p, angular velocity omega_p,
 * force = -dP_B and torque = -dL_B exchanged with the fluid in the last step (Eqs. 8-9,
 * dt = 1). Synchronizes. */
lbm_status lbm_get_particles(lbm_ctx* ctx, double* x, double* u, double* omega,
                             double* force, double* torque);

/* Orientation of each particle after the last step, q[n*4]: the unit quaternion (w, x, y, z)
 * of the rotation from the particle's attitude when it was added (the identity) to its
 * attitude now. It is the angular part of the rigid-body integration (Sec. 2.2: the particle
 * moves with the velocities Eqs. 10-11 give, Eq. 13 for the position): every step the
 * quaternion is turned by |omega| about omega, omega the angular velocity after that step's
 * acceleration (space frame, held over dt = 1), q <- dq q with dq = (cos(|omega|/2),
 * sin(|omega|/2) omega/|omega|), and renormalised; FP64 on the device in every storage
 * precision. The spheres' dynamics do not depend on it. Synchronizes.
 * LBM_E_INVALID for a NULL argument. */
lbm_status lbm_get_orientations(lbm_ctx* ctx, double* q);

/* Asynchronous form of lbm_get_particles (the same quantities, Eqs. 8-9 and 10-13; the
 * asynchrony has no counterpart in the paper) for loops that read the particles every step
 * without stalling the device: enqueues on the context's stream, after the work so far, the
 * packing of x, u, omega, force and torque and their copy into dst, then returns at once.
 * dst: page-locked host memory (cudaMallocHost, cudaHostRegister, or a pinned torch tensor)
 * of 15 np + 1 doubles, caller-owned, untouched by the caller until the read-back is waited
 * for: the five arrays of lbm_get_particles as consecutive [np][3] blocks, then the device
 * status word. *ticket identifies the read-back. At most 8 may be outstanding.
 * Errors: LBM_E_INVALID (null argument, no particles, 8 outstanding), LBM_E_CUDA. */
lbm_status lbm_get_particles_async(lbm_ctx* ctx, double* dst, long long* ticket);

/* Waits until read-back `ticket` has landed in its buffer (work enqueued after it may still
 * run) and returns the device status it carries (as lbm_synchronize would, for the steps
 * before it). LBM_E_INVALID for an unknown or already waited ticket. */
lbm_status lbm_wait_particles(lbm_ctx* ctx, long long ticket);

/* Full distribution state f[Q][N] at the current step boundary: the populations f_i(x, t)
 * of Sec. 2.1 (Eq. 3) after propagation, with the IS imposition of Eq. 12 applied, converted
 * to double. Synchronizes. */
lbm_status lbm_get_distributions(lbm_ctx* ctx, double* f);

/* Replaces the distribution state, the populations f_i(x, t) of Sec. 2.1 (Eq. 3) at a step
 * boundary, by f[Q][N] (same layout as lbm_get_distributions). Values are rounded to the
 * storage precision. Synchronizes. */
lbm_status lbm_set_distributions(lbm_ctx* ctx, const double* f);

/* Owner map of the lattice sites, tags[N] (unsigned 32-bit): the boundary sites (BS) and
 * internal sites (IS) of each particle (Sec. 2.2, Fig. 2) at its current whole-site shift
 * (Eqs. 14-15): (class << 30) | particle id with class 0 = IS, 1 = BS, 2 = other solid
 * site; 0xFFFFFFFF = fluid. Where the site
 * sets of close particles meet, IS wins over BS over the rest, then the lower id.
 * Synchronizes. */
lbm_status lbm_get_masks(lbm_ctx* ctx, unsigned* tags);

/* Introspection: out[0] = number of particles, out[1] = steps taken, out[2] = kernel
 * launches per step in the captured graph, out[3] = device bytes held by the context,
 * out[4] = bytes of distribution storage per site (2 Q b in the pull scheme; Q b plus
 * two densities with in-place streaming, see lbm_set_streaming), out[5] = precision. Returns LBM_E_INVALID if out is NULL. */
lbm_status lbm_get_info(lbm_ctx* ctx, long long out[6]);

/* Runs n steps like lbm_step but without graph capture, timing kernel groups with CUDA
 * events on the context's stream: out_ms[0] = mean duration of the main sweep kernel (the
 * fused propagation + collision + boundary-site transfer over every site), out_ms[1] =
 * mean duration of the particle phase (its kernels back to back, launch gaps included),
 * out_ms[2] = mean duration of a whole step. Advances the simulation by n steps and
 * synchronizes. Errors as lbm_step; LBM_E_INVALID if n < 1 or out_ms is NULL. */
lbm_status lbm_profile_steps(lbm_ctx* ctx, int n, double out_ms[3]);

/* Shape of the main sweep kernel (a tuning knob with no counterpart in the paper, which
 * describes a serial algorithm; results agree to FP32 rounding). For the
 * FP32 / FP16 / BF16 storages on a lattice with even nx, threads_x = 16, 32, 64 or 128
 * selects the two-site kernel (each thread updates the sites x, x + 1 with paired 8- or
 * 4-byte accesses and packed FP32 pair arithmetic; blocks of 128 threads, threads_x of them
 * along x, 128 / threads_x rows); 0 selects the one-site kernel; -1 (the default) picks
 * the two-site kernel with 16 threads along x (the one-site kernel where nx is odd). FP64
 * storage always uses the one-site kernel. Drops the captured step graphs. LBM_E_INVALID for
 * other values. */
lbm_status lbm_set_sweep_shape(lbm_ctx* ctx, int threads_x);

/* Streaming scheme (no counterpart in the paper, whose Eq. 4 only states that f*_i(x) moves
 * to x + c_i; results agree bit for bit in FP64 storage):
 *   LBM_STREAM_PULL (default): two distribution buffers; each sweep gathers f_i(x) from
 *     x - c_i of the buffer the previous sweep wrote into the other one. 2 Q b bytes of
 *     distribution storage per site (b = bytes per stored value).
 *   LBM_STREAM_INPLACE: one buffer, two kinds of sweep taken in turn. The neighbour sweep
 *     gathers f_i(x) from slot i of x - c_i and writes f*_i(x) into slot opp(i) of x + c_i
 *     (slot i of x where x + c_i lies beyond a wall); the local sweep reads f_i(x) from slot
 *     opp(i) of x and writes f*_i(x) into slot i of x. Q b bytes per site plus two arrays of
 *     one density per site (4 bytes each in FP32 / FP16 / BF16 storage, 8 in FP64) that hold
 *     the post-collision densities of the IS sites, which keep their populations in this
 *     scheme. The sweep is always the one-site kernel (lbm_set_sweep_shape is ignored); the
 *     getters, lbm_set_distributions, the closure inputs and checkpoints see the same state
 *     as in the pull scheme. Single contexts only (a batch refuses such a cell).
 * Must be called after lbm_configure and before particles, distributions, steps or anything
 * that allocates the context's buffers: LBM_E_STATE otherwise; LBM_E_INVALID for an unknown
 * mode. */
typedef enum { LBM_STREAM_PULL = 0, LBM_STREAM_INPLACE = 1 } lbm_streaming;
lbm_status lbm_set_streaming(lbm_ctx* ctx, int mode);

/* Diagnostics of the state at the current step boundary (no counterpart in the paper; for
 * monitoring long runs). The site moments are those of lbm_get_fields (Eqs. 1-2 with the Guo
 * half-force, on the populations with the pending IS imposition): out[0] = total mass sum rho
 * over all sites (fluid and particle sites alike), out[1..3] = total momentum sum rho u,
 * out[4] = max |u|, out[5] = the lattice Mach number max |u| / c_s (c_s = 1/sqrt(3)), out[6] =
 * the number of sites whose rho or u is not finite (their moments are left out of out[0..5]).
 * Sums in a fixed order: the same state gives the same values. Synchronizes.
 * Returns LBM_E_NAN, with out filled, when out[6] > 0; LBM_E_INVALID if out is NULL; otherwise
 * the errors of lbm_synchronize. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, double out[7]);

/* ---- Checkpoint and resume ------------------------------------------------------------------
 * No counterpart in the paper. For long runs that must survive the end of a job (the paper's longest sedimentation runs
 * take about 10^5 steps). A checkpoint holds the state at a step boundary: the distributions the
 * next step streams (storage format), the owner map and IS-source masks, each particle's
 * velocities, angular velocities, site-set anchor, position and last force and torque, the
 * pending-imposition flag and the wall velocities. The constant set-up (lattice, sizes, tau,
 * forces, faces, particle constants, site templates) is not stored but fingerprinted: a
 * checkpoint loads only into a context created, configured and given particles by the same
 * calls with the same arguments (its own steps, if any, are overwritten). The byte layout is
 * this version's of the library, on this machine; it is not a portable file format. */

/* Size in bytes of a checkpoint of ctx. */
lbm_status lbm_checkpoint_size(lbm_ctx* ctx, unsigned long long* bytes);

/* Copies the state at the current step boundary into buf (host memory, caller-owned, at
 * least lbm_checkpoint_size bytes). Synchronizes; returns a recorded device error first.
 * LBM_E_INVALID if bytes is too small. */
lbm_status lbm_checkpoint_save(lbm_ctx* ctx, void* buf, unsigned long long bytes);

/* Restores a checkpoint written by lbm_checkpoint_save: the next lbm_step continues exactly
 * (bit for bit) where the saved context stood. Synchronizes. LBM_E_INVALID if buf is not a
 * checkpoint written by this version of the library, is truncated, or was taken from a
 * context set up differently. */
lbm_status lbm_checkpoint_load(lbm_ctx* ctx, const void* buf, unsigned long long bytes);

/* Largest particle count lbm_bs_exchange_noalloc accepts. */
#define LBM_NOALLOC_MAX_PARTICLES 65536

/* Boundary-site momentum exchange without any device allocation.
 *
 * The paper has no counterpart of this call; it exists for callers that cannot call
 * cudaMalloc: code that owns its device memory through its own pool or arena (a host
 * framework that forbids foreign allocations), code running where allocation is not
 * allowed or must not stall (a real-time loop, work being recorded into a CUDA graph),
 * and callers holding the state in buffers they allocated themselves. They pass every
 * input and output; the library uses no memory of its own beyond a fixed array that is
 * part of the library's device image.
 *
 * Computes, for a state given by the caller, what one step hands each particle through its
 * boundary sites: at every site the owner map tags BS of particle p, the post-collision
 * density and momentum (rho and sum_i f_i c_i + F) meet the rigid-body velocity
 * u_p + omega_p x r, r the minimum-image offset of the site from centers[p]; the momentum
 * change of the fluid there is summed per particle and returned as force = -sum dp and
 * torque = -sum r x dp (the force and torque lbm_get_particles reports for a step taken
 * from that state).
 *
 * centers[p] is the centre of particle p's site set, not its position x_p: the sites are
 * the set classified around the centre x_p0 at which the particle was added, translated by
 * the whole-site shift s_p = floor(x_p - x_p0 + 1/2) per axis (Eqs. 14-15), and the lever
 * arms of a step are taken from x_p0 + s_p. Before a particle first moves that is x_p0;
 * a caller who passes the x_p that lbm_get_particles reports after the particle has moved
 * by a fraction of a site gets other rigid-body velocities and torques.
 *
 * Arguments: lattice and sizes as lbm_create; walls[3] (may be NULL: all periodic) flags the
 * axes with solid walls (no minimum image there); body_force[3] the fluid force density F
 * (may be NULL). Device pointers, caller-owned: g[Q][N] FP32 deviations f_i - w_i of the
 * populations at the start of the step (velocity order and site order as in this header),
 * tags[N] the owner map in the encoding of lbm_get_masks, centers / velocities / omegas
 * [n][3] doubles, force / torque [n][3] doubles written by the call. cuda_stream: the
 * stream the work is enqueued on (NULL = default stream); the call returns after enqueueing.
 *
 * Limits and rules: n <= LBM_NOALLOC_MAX_PARTICLES, else LBM_E_INVALID (as for sizes
 * lbm_create rejects). The per-particle accumulators live in one fixed device array (3 MiB,
 * held by every GPU that loads the library until the process exits) shared by all calls:
 * each call clears the part it uses before accumulating, and the array keeps the last
 * call's sums afterwards. Calls that overlap on the GPU (different streams, or devices
 * sharing nothing else) race on that array and must be serialised by the caller. The first
 * call on each device looks up the array's device address (a CUDA runtime query, no
 * allocation) and keeps it for the life of the process; make that first call before any
 * stream capture. A device reset (cudaDeviceReset) reloads the library's device image at
 * another address, so the call is not supported on a device that was reset after its first
 * call there. No cudaMalloc, cudaFree or allocating library routine is called.
 * LBM_E_CUDA, with nothing enqueued, if a CUDA error from earlier work is still pending on
 * the calling thread (it is left for its owner to read) or the device query fails; LBM_E_CUDA
 * if one of the call's own launches fails. */
lbm_status lbm_bs_exchange_noalloc(int lattice, int nx, int ny, int nz, const int walls[3],
                                   const double body_force[3], const float* g,
                                   const unsigned* tags, int n, const double* centers,
                                   const double* velocities, const double* omegas,
                                   double* force, double* torque, void* cuda_stream);

/* ---- Batched ensembles ------------------------------------------------------------------
 * Many independent simulations ("cells", e.g. periodic boxes of different sizes, each with
 * its own tau, body force and particles) advanced together. The paper simulates one box at
 * a time; the batch only changes how the work is launched: every step runs one sweep
 * launch over all cells (a schedule table of 128-thread tiles, each tile one rectangle of
 * one x-y plane of one cell) and one launch per particle-phase kernel (the cell as the
 * second grid index), captured in CUDA graphs of one or several steps. Each cell's result
 * is bit for bit the result of stepping it alone with the one-site sweep kernel
 * (lbm_set_sweep_shape(ctx, 0)); the batch sweep is that kernel. */

/* Creates ncells contexts sharing the lattice, storage precision, face kinds, particle
 * gravity, contact gap and force-on-particles flag (meaning as lbm_configure); dims
 * (ncells*3: nx, ny, nz), tau (ncells) and body_force (ncells*3, may be NULL = 0) are per
 * cell. All cells enqueue on one library-created stream (lbm_batch_stream).
 * Errors as lbm_create / lbm_configure; *out is NULL on error. */
lbm_status lbm_batch_create(lbm_batch** out, int lattice, int ncells, const int* dims, const double* tau,
                            const double* body_force, int precision, const int faces[6],
                            const double particle_gravity[3], double contact_gap,
                            int body_force_on_particles);

/* lbm_add_particles on cell `cell` (before the first step). Errors as lbm_add_particles,
 * LBM_E_INVALID for a cell index out of range. */
lbm_status lbm_batch_add_particles(lbm_batch* b, int cell, int n, const double* centers, const double* radii,
                                   const double* densities, const double* velocities, const double* omegas);

/* The context of one cell (owned by the batch; NULL if out of range). Every single-context
 * getter and setter works on it (lbm_get_fields, lbm_get_particles, lbm_set_distributions,
 * lbm_set_wall_velocity, ...); lbm_step on it advances that cell alone with its own graph.
 * Cells must share their buffer parity when the batch steps (an odd number of single-cell
 * steps on one cell makes lbm_batch_step return LBM_E_STATE). */
lbm_ctx* lbm_batch_cell(lbm_batch* b, int cell);

/* Launch tuning (results do not depend on it):
 *   tile_width[ncells]: sites along x of a cell's tiles, 32, 64 or 128 (the tile then spans
 *     128/width rows in y); NULL = 128 for every cell;
 *   order: 0 cells one after another, 1 one tile of each cell in turn, 2 largest cell first;
 *   grid: 0 = one block per tile, > 0 = that many resident blocks striding over the table;
 *   steps_per_graph: steps captured in one graph launch (1..256).
 * Re-captures the step graphs at the next step. LBM_E_INVALID on a bad value. */
lbm_status lbm_batch_set_tuning(lbm_batch* b, const int* tile_width, int order, int grid, int steps_per_graph);

/* Advances every cell by n steps (asynchronous, like lbm_step). */
lbm_status lbm_batch_step(lbm_batch* b, int n);

/* Waits for the batch's stream; returns the first non-OK device status of any cell. */
lbm_status lbm_batch_synchronize(lbm_batch* b);

/* As lbm_profile_steps, for the whole batch: out_ms = mean sweep, particle phase, step. */
lbm_status lbm_batch_profile_steps(lbm_batch* b, int n, double out_ms[3]);

/* out[0] cells, out[1] lattice sites of all cells, out[2] particles, out[3] sweep tiles,
 * out[4] kernels launched per step. Captures the step graphs if needed. */
lbm_status lbm_batch_get_info(lbm_batch* b, long long out[5]);

/* The cudaStream_t every cell of the batch enqueues on. */
void* lbm_batch_stream(lbm_batch* b);

/* Host-only (no device needed): the sweep schedule of a batch. Returns the number of tiles
 * for ncells cells of sizes dims[ncells*3] with tile_width[ncells] (NULL = 128) in the given
 * order (as lbm_batch_set_tuning), or -1 on a bad argument. If out != NULL it receives 4
 * ints per tile in launch order: cell, x0, y0 | (log2(width) << 16), z. */
long long lbm_schedule_tiles(int ncells, const int* dims, const int* tile_width, int order, int* out);

/* Description of the last non-OK status of b (never NULL). */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Destroys the batch and all of its cells (NULL is a no-op). */
void lbm_batch_destroy(lbm_batch* b);

/* Inputs of the learned closure for every particle of ctx, enqueued on the context's stream:
 * the moments (rho - 1, u - u_p) / u_ref at the n_side^3 nodes x_p + spacing (i - (n_side-1)/2,
 * j - .., k - ..), trilinearly interpolated from the 8 surrounding sites of the current state
 * (periodic axes wrap, walled axes clamp to the domain; u as lbm_get_fields), followed by the
 * fractional part x_p0 - floor(x_p0) of the particle's reference centre (3 values), which
 * with the radius fixes the particle's discrete site set. out: device pointer to
 * np * (4 n_side^3 + 3) floats, [p][(k n_side + j) n_side + i][4] then the 3 offsets. D2Q9:
 * nodes that differ only in k carry the same values.
 * Errors: LBM_E_INVALID (n_side outside 1..8, spacing <= 0, u_ref zero or not finite). */
lbm_status lbm_closure_features(lbm_ctx* ctx, int n_side, double spacing, double u_ref, float* out);

/* ---- Learned drag / torque closure network -------------------------------------------------
 * Not in the paper: a multilayer perceptron x -> relu(W1 x + b1) -> ... -> W_L h + b_L that
 * predicts the correction to the force and torque a coarse-resolution particle feels. It is
 * trained and evaluated on the GPU: weights and activations in bfloat16, tensor-core products
 * accumulated in FP32, FP32 master weights, Adam (Kingma & Ba 2015) and a mean-squared-error
 * loss. Parameters are laid out layer by layer, W_l (sizes[l+1] x sizes[l], row-major) then
 * b_l. Data arrays are caller-owned device pointers (FP32, row-major); every call enqueues on
 * the stream given at creation and returns after enqueueing unless it returns host values. */
typedef struct lbm_mlp lbm_mlp;

/* nlayers (1..8) weight layers of widths sizes[0..nlayers] (each 1..4096). Parameters start at
 * zero (set them with lbm_mlp_set_params). Errors: LBM_E_INVALID, LBM_E_CUDA, LBM_E_OOM. */
lbm_status lbm_mlp_create(lbm_mlp** out, int nlayers, const int* sizes, void* cuda_stream);

/* Number of parameters (weights and biases), or -1 for NULL. */
long long lbm_mlp_num_params(const lbm_mlp* net);

/* Host FP64 parameters in (rounded to FP32 masters and bfloat16 copies); resets Adam. */
lbm_status lbm_mlp_set_params(lbm_mlp* net, const double* params);

/* Input standardisation applied by every call that reads inputs (forward, loss, training):
 * the network sees (x_c - shift[c]) * scale[c] for each of the sizes[0] inputs (host arrays,
 * copied). Both NULL removes it. Errors: LBM_E_INVALID (one NULL, non-finite entries). */
lbm_status lbm_mlp_set_input_scaling(lbm_mlp* net, const double* shift, const double* scale);

/* Host copies of the FP32 masters and / or of the last gradients (either may be NULL). */
lbm_status lbm_mlp_get_params(lbm_mlp* net, double* params, double* grads);

/* y[rows][sizes[L]] = network(x[rows][sizes[0]]) (device pointers). */
lbm_status lbm_mlp_forward(lbm_mlp* net, const float* x, int rows, float* y);

/* Mean-squared error of the network on (x, t) over all rows x outputs, and its gradient
 * (kept for lbm_mlp_adam_step / lbm_mlp_get_params); *loss (host, may be NULL) receives
 * the loss, which synchronizes. */
lbm_status lbm_mlp_loss_grad(lbm_mlp* net, const float* x, const float* t, int rows, double* loss);

/* One Adam step with the last gradients. */
lbm_status lbm_mlp_adam_step(lbm_mlp* net, double lr, double beta1, double beta2, double eps);

/* Trains on n rows (x, t) for `epochs` epochs of shuffled minibatches of `batch` rows (the
 * shuffle is seeded; a last partial minibatch is skipped), Adam with beta1 0.9, beta2 0.999,
 * eps 1e-8. epoch_loss (host, may be NULL) receives the mean minibatch loss of each epoch. */
lbm_status lbm_mlp_train(lbm_mlp* net, const float* x, const float* t, int n, int batch, int epochs, double lr,
                         unsigned seed, double* epoch_loss);

const char* lbm_mlp_last_error(const lbm_mlp* net);
void lbm_mlp_destroy(lbm_mlp* net);

/* Description of the last non-OK status of ctx (static storage; never NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Frees every device and host resource of ctx (NULL is a no-op). Synchronizes first. */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBMP_H */
