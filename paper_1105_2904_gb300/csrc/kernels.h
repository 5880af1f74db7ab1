// Host-side interface between the translation units of the CUDA path: argument records
// and launch functions. The sweep family is compiled once per storage format (double in
// a TU built with -fmad=false so that it evaluates the same IEEE operations as a plain
// FP64 implementation; float / half / bfloat16 in another).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lbmp {

struct SweepArgs {
    int lattice;               // 0 = D2Q9, 1 = D3Q19
    Geom g;
    const void* fin;           // [Q][N] storage format
    void* fout;                // [Q][N]
    PartView pv;               // tag == nullptr: no particles
    void* bs_scratch;          // per-site BS records: FP64 mode [N][6] doubles (dP, dL); other
                               // modes float4 (dP, owner tag bits: 16 bytes) at the site index
                               // (16-bit storages) or its brick index (FP32, rec_brick_index)
    double omega, pre, F[3];   // 1/tau, 1 - 1/(2 tau), body force
    float omega_f, pre_f, F_f[3];  // the same in FP32 (reduced-storage sweeps)
    int moving_walls;          // 1: wall faces may move (uw is read)
    const WallVel* uw;         // wall velocities of the streaming that the pull completes
    int pair_bx;               // deviation storage, even nx: two-site kernel with this many
                               // threads along x (16, 32, 64 or 128); 0: one-site kernel
    // In-place streaming (fin == fout, one buffer): 0 = the pull scheme above; 1 = the
    // neighbour phase (site x reads slot i of x - c_i, writes f*_i into slot opp(i) of
    // x + c_i); 2 = the local phase (site x reads slot opp(i) of x, writes f*_i into slot i).
    // The IS sites keep their populations; their post-collision densities go to is_rho_out
    // and the pulls from IS sources read is_rho_in ([N] compute type each).
    int aa;
    const void* is_rho_in;
    void* is_rho_out;
};

struct MaterializeArgs {
    int lattice;
    Geom g;
    const void* fin;
    PartView pv;
    double F[3];
    int moving_walls;
    const WallVel* uw;
    unsigned s0, count;        // site range [s0, s0 + count)
    int mode;                  // 0: rho[count], u[count][3]; 1: f[Q][count]
    int aa;                    // 0: pull-source layout; 1: in-place layout after a neighbour
                               // phase (slot opp(i) of x holds the pulled f_i(x))
    const void* is_rho;        // in-place streaming: densities of the IS sites ([N] compute type)
    double* out0;
    double* out1;
};

struct ConvertArgs {
    int lattice;
    Geom g;
    const double* f;           // [Q][count] plain distributions
    void* dst;                 // [Q][N] storage format, unshifted
    unsigned s0, count;
    int opp;                   // 1: f_i goes to slot opp(i) (in-place layout after a neighbour phase)
};

struct UnstreamArgs {
    int lattice;
    Geom g;
    const void* src;           // [Q][N] storage format holding f at unshifted sites
    void* dst;                 // [Q][N] pull-source layout
};

// The IS-site bookkeeping of one step (see k_is_density, k_is_restore, k_is_fix). Every
// site tagged IS when a sweep runs stores its post-collision density (in the compute form:
// rho, or rho - 1 for deviation storage) in all Q of its slots instead of its populations,
// which no pull ever uses raw (every pull from an IS site takes the imposed equilibrium).
// When a particle's shift changes, the sites that stop being IS get their populations back
// and the sites that become IS get their density.
struct ISFixArgs {
    SweepArgs s;               // the step's sweep, with the particle view it ran with (prev copies)
    void* dens;                // [N] compute type: densities of the sites visited
    const PKern* pk;           // current particle records (new anchors)
    const PConst* pc;
    const int* tmpl;
    const int* Kold;           // [np][3] anchors the sweep ran with
    const int* list;           // particles whose shift changed
    const Counters* cnt;       // cnt->nchanged entries of list
};

struct MaskArgs {
    int lattice;
    Geom g;
    const unsigned* tag;
    unsigned* ismask;          // [N]
    const PKern* pk;
    const PConst* pc;
    const int* tmpl;
    const int* list;           // particles whose sites need new masks (nullptr = all np)
    const Counters* cnt;       // cnt->nrestamp entries of list
    int np;
};

// One sweep launch over a batch of independent cells. Entry e of the schedule table is one
// 128-thread tile of one cell: (cell, x0, y0 | log2(tile width) << 16, z); the tile covers
// x0 .. x0 + w - 1 and y0 .. y0 + 128/w - 1 of plane z (w = 32, 64 or 128).
struct BatchSweepArgs {
    int lattice;
    const SweepArgs* cells;    // device [ncells], this step's buffer parity
    const int4* table;         // device [ntiles]
    int ntiles;
    int walls;                 // some cell has walls
    int part;                  // some cell has particles
    int grid;                  // 0: one block per tile; > 0: that many blocks stride over the table
};

// Inputs of the closure network: stencil moments around each particle (see k_features).
struct FeatureArgs {
    MaterializeArgs m;         // the state (buffer, particle view, walls, F)
    const double* x;           // [np][3] centres
    const PKern* pk;           // particle velocities
    int np;
    int n_side;                // stencil nodes per axis
    double h;                  // node spacing
    double u_ref;              // velocity scale
    float* out;                // [np][n_side^3][4]
};

struct KernelTable {
    void (*sweep)(const SweepArgs&, cudaStream_t);
    void (*update_masks)(const MaskArgs&, cudaStream_t);
    void (*materialize)(const MaterializeArgs&, cudaStream_t);
    void (*convert_in)(const ConvertArgs&, cudaStream_t);
    void (*unstream)(const UnstreamArgs&, cudaStream_t);
    void (*fill_rest)(int lattice, void* dst, unsigned N, cudaStream_t);
    void (*is_save)(const ISFixArgs&, cudaStream_t);   // densities, then populations restored
    void (*is_fix)(const ISFixArgs&, cudaStream_t);    // densities into the new IS sites
    void (*sweep_batch)(const BatchSweepArgs&, cudaStream_t);
    // per-cell argument arrays on the device, blockIdx.y = cell
    void (*is_save_batch)(int lattice, const ISFixArgs* cells, int ncells, cudaStream_t);
    void (*is_fix_batch)(int lattice, const ISFixArgs* cells, int ncells, cudaStream_t);
    void (*update_masks_batch)(int lattice, const MaskArgs* cells, int ncells, cudaStream_t);
    void (*features)(const FeatureArgs&, cudaStream_t);
    // In-place streaming: after re-marking, the densities of the sites that are now IS
    // (ISFixArgs.dens = the density array the next sweep reads; s.aa = the layout the sweep
    // left: 1 after a neighbour phase, 2 after a local phase).
    void (*inplace_fix)(const ISFixArgs&, cudaStream_t);
    int elem_bytes;
    int compute_bytes;
};

const KernelTable* kernels_f64();
const KernelTable* kernels_f32();
const KernelTable* kernels_f16();
const KernelTable* kernels_bf16();

// ---- particle phase (particles.cu, FP64, -fmad=false) ---------------------------------------
struct CellGrid {
    int n[3];          // cells per axis
    double size[3];    // cell edge per axis
    int total;
};

struct ParticleArgs {
    int lattice;
    Geom g;
    int np;
    PKern* pk;
    PKernF* pkf;        // FP32 copy of pk, refreshed after the move
    PKern* pk_prev;     // [np] pk, pkf and *pending as the step's sweep saw them (copied
    PKernF* pkf_prev;   // at the start of the particle phase)
    int* pending_prev;
    const PConst* pc;
    const int* tmpl;
    unsigned* tag;
    double* x;          // [np][3] centres
    double* q;          // [np][4] orientations, unit quaternions (w, x, y, z)
    int* Kold;          // [np][3] anchor before this step's move
    double* un;         // [np][3] velocity during the contact step
    float4* xpf;        // [np] predicted centre x + u' in FP32 and the radius (pair pre-test)
    double* acc;        // [np][6]
    double* force;      // [np][6] -dP, -dL of the last step
    void* bs_scratch;        // per-site BS records (layout as in SweepArgs)
    int scratch_f64;         // 1: bs_scratch holds doubles (FP64 mode)
    int rec_brick;           // 1: float4 records at rec_brick_index (FP32 storage)
    Counters* cnt;
    int* status;        // device status word (first fault wins)
    int* pending;
    CellGrid cg;
    int* cell_of;       // [np]
    int* cell_count;    // [total]
    int* cell_start;    // [total + 1]
    int* cell_cursor;   // [total]
    int* cell_items;    // [np]
    unsigned long long* pairs;  // [pair_cap]
    int pair_cap;
    int* changed;       // [np]
    int* restamp;       // [np]
    int* restamp_flag;  // [np]
    double gap;
};

// Enqueues the particle phase of one step after the sweep in two parts: (a) snapshot of the
// sweep's particle view, reduction, acceleration, contacts, move, the list of particles to
// re-mark; (b) re-marking of the owner map. The IS-site bookkeeping (ISFixArgs) runs between
// them, while the owner map is still the one the sweep used. Return the kernels launched.
int launch_particle_phase_a(const ParticleArgs& a, cudaStream_t s);
int launch_particle_phase_b(const ParticleArgs& a, cudaStream_t s);
// Stamps every particle's site set into a cleared owner map (after lbm_add_particles).
void launch_stamp_all(const ParticleArgs& a, cudaStream_t s);

// Shape of a batched particle phase: the largest per-cell counts size the grids
// (blockIdx.y = cell; blocks beyond a cell's own counts return at once).
struct PhaseShape {
    int ncells;
    int max_np;       // particles of the most populated cell
    int max_cells;    // contact-grid cells of the largest cell
    int pair_cap;     // contact-pair capacity of every cell (its resolve buffer)
    int scratch_f64;  // FP64 storage: ordered per-particle sums
};
int launch_particle_phase_batch_a(const ParticleArgs* cells, const PhaseShape& sh, cudaStream_t s);
int launch_particle_phase_batch_b(const ParticleArgs* cells, const PhaseShape& sh, cudaStream_t s);
// After a sweep with moving walls: the current wall velocities become those of the streaming
// that the next pull completes (wv[0] <- wv[1]), and the pulled values await streaming.
void launch_wall_advance(WallVel* wv, int* pending, cudaStream_t s);
// Packs x, u, omega, force, torque of every particle into out (five [np][3] blocks) and the
// device status word into out[15 np].
void launch_pack_particles(const ParticleArgs& a, double* out, cudaStream_t s);
// Opts the contact kernel into the shared memory its pair list needs.
cudaError_t prepare_particle_kernels(int pair_cap);



}  // namespace lbmp
