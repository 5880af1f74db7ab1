// Host side of the C-ABI declared in include/lbmp.h: argument checks, device allocation,
// particle set-up (classification of each particle's lattice sites, Sec. 2.2 / Fig. 2),
// capture of one time step into CUDA graphs, and the synchronous getters/setters.
// Host arithmetic that must agree with a plain FP64 implementation (site classification,
// masses) is compiled with -ffp-contract=off.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"

using namespace lbmp;
using namespace lbmp::host;

namespace lbmp {
namespace host {

const KernelTable* table_for(int precision)
{
    switch (precision) {
    case LBM_FP64: return kernels_f64();
    case LBM_FP32: return kernels_f32();
    case LBM_FP16DEV: return kernels_f16();
    case LBM_BF16DEV: return kernels_bf16();
    default: return nullptr;
    }
}

int lat_c(int lattice, int i, int k) { return lattice == 0 ? D2Q9::c(i, k) : D3Q19::c(i, k); }

WallVel wall_vel(const lbm_ctx* ctx)
{
    WallVel w{};
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k) {
            w.u[f][k] = ctx->uw[f][k];
            w.uf[f][k] = (float)ctx->uw[f][k];
        }
    return w;
}

lbm_status ensure_alloc(lbm_ctx* ctx)
{
    if (ctx->allocated) return LBM_OK;
    ctx->kt = table_for(ctx->precision);
    const size_t N = ctx->g.N;
    const size_t fbytes = (size_t)ctx->Q * N * (size_t)ctx->kt->elem_bytes;
    CS(dev_alloc(ctx, &ctx->f[0], fbytes));
    if (ctx->inplace) {
        for (int c = 0; c < 2; ++c) {
            CS(dev_alloc(ctx, &ctx->is_rho[c], (size_t)ctx->kt->compute_bytes * N));
            CK(cudaMemsetAsync(ctx->is_rho[c], 0, (size_t)ctx->kt->compute_bytes * N, ctx->stream));
        }
    } else {
        CS(dev_alloc(ctx, &ctx->f[1], fbytes));
    }
    CS(dev_alloc(ctx, &ctx->status, sizeof(int)));
    CS(dev_alloc(ctx, &ctx->pending, sizeof(int)));
    CS(dev_alloc(ctx, &ctx->pending_prev, sizeof(int)));
    CS(dev_alloc(ctx, &ctx->wv, 2 * sizeof(WallVel)));
    CS(dev_alloc(ctx, &ctx->staging, STAGING_BYTES));
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(ctx->pending, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(ctx->pending_prev, 0, sizeof(int), ctx->stream));
    {
        const WallVel w[2] = {wall_vel(ctx), wall_vel(ctx)};
        CK(cudaMemcpyAsync(ctx->wv, w, sizeof(w), cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->kt->fill_rest(ctx->lattice, ctx->f[0], ctx->g.N, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->cur = 0;
    ctx->allocated = true;
    return LBM_OK;
}

// Classification of the solid sites of one particle around its initial centre (Sec. 2.2,
// Fig. 2): S = {o : |o - phi|^2 <= r^2} (offsets o from floor(x0)); BS = sites of S with a
// neighbour (model velocity set) outside S; IS = other sites of S with a neighbour in BS;
// the rest of S is interior. Entries are emitted grouped BS, IS, interior, each group in
// z, y, x lexicographic order; n_bs and n_is count the first two groups.
void classify(int lattice, const double phi[3], double r, std::vector<int>& out, int& n_bs, int& n_is)
{
    const int D = lattice == 0 ? 2 : 3, Q = lattice == 0 ? 9 : 19;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) {
        lo[k] = (int)std::floor(phi[k] - r) - 1;
        hi[k] = (int)std::ceil(phi[k] + r) + 1;
    }
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const size_t cells = (size_t)ex * ey * ez;
    // neighbour i of box cell b is b + off[i] (the box has a one-cell margin around S)
    long long off[19];
    for (int i = 0; i < Q; ++i)
        off[i] = ((long long)lat_c(lattice, i, 2) * ey + lat_c(lattice, i, 1)) * ex + lat_c(lattice, i, 0);
    std::vector<unsigned char> cls(cells, 0);  // 0 outside S, 1 BS, 2 IS, 3 interior, 4 S unclassified
    const double r2 = r * r;
    size_t b = 0;
    for (int oz = lo[2]; oz <= hi[2]; ++oz)
        for (int oy = lo[1]; oy <= hi[1]; ++oy)
            for (int ox = lo[0]; ox <= hi[0]; ++ox, ++b) {
                const double dx = (double)ox - phi[0];
                const double dy = (double)oy - phi[1];
                const double dz = (double)oz - phi[2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                cls[b] = d2 <= r2 ? 4 : 0;
            }
    for (size_t c = 0; c < cells; ++c) {
        if (cls[c] != 4) continue;
        for (int i = 1; i < Q; ++i)
            if (cls[c + off[i]] == 0) {
                cls[c] = 1;  // BS: a neighbour outside S
                break;
            }
    }
    for (size_t c = 0; c < cells; ++c) {
        if (cls[c] != 4) continue;
        bool is = false;
        for (int i = 1; i < Q && !is; ++i) is = cls[c + off[i]] == 1;
        cls[c] = is ? 2 : 3;  // IS: a neighbour in BS
    }
    // grouped BS, IS, interior; z, y, x lexicographic order inside each group
    out.clear();
    n_bs = n_is = 0;
    for (unsigned char want : {1, 2, 3}) {
        b = 0;
        for (int oz = lo[2]; oz <= hi[2]; ++oz)
            for (int oy = lo[1]; oy <= hi[1]; ++oy)
                for (int ox = lo[0]; ox <= hi[0]; ++ox, ++b) {
                    if (cls[b] != want) continue;
                    out.push_back(tmpl_pack(ox, oy, oz, want == 1 ? CLS_BS : (want == 2 ? CLS_IS : CLS_IN)));
                }
        if (want == 1) n_bs = (int)out.size();
        if (want == 2) n_is = (int)out.size() - n_bs;
    }
}

double min_image_h(double d, int n, bool periodic)
{
    if (!periodic) return d;
    return d - (double)n * std::floor(d / (double)n + 0.5);
}

int axis_n(const lbm_ctx* c, int k) { return k == 0 ? c->g.nx : (k == 1 ? c->g.ny : c->g.nz); }

ParticleArgs particle_args(lbm_ctx* ctx)
{
    ParticleArgs a{};
    a.lattice = ctx->lattice;
    a.g = ctx->g;
    a.np = ctx->np;
    a.pk = ctx->pk;
    a.pkf = ctx->pkf;
    a.pk_prev = ctx->pk_prev;
    a.pkf_prev = ctx->pkf_prev;
    a.pending_prev = ctx->pending_prev;
    a.pc = ctx->pc;
    a.tmpl = ctx->tmpl;
    a.tag = ctx->tag;
    a.x = ctx->x;
    a.q = ctx->q;
    a.xpf = ctx->xpf;
    a.Kold = ctx->Kold;
    a.un = ctx->un;
    a.acc = ctx->acc;
    a.force = ctx->force;
    a.bs_scratch = ctx->bs_scratch;
    a.scratch_f64 = ctx->precision == LBM_FP64;
    a.rec_brick = ctx->precision == LBM_FP32;
    a.cnt = ctx->cnt;
    a.status = ctx->status;
    a.pending = ctx->pending;
    a.cg = ctx->cg;
    a.cell_of = ctx->cell_of;
    a.cell_count = ctx->cell_count;
    a.cell_start = ctx->cell_start;
    a.cell_cursor = ctx->cell_cursor;
    a.cell_items = ctx->cell_items;
    a.pairs = ctx->pairs;
    a.pair_cap = PAIR_CAP;
    a.changed = ctx->changed;
    a.restamp = ctx->restamp;
    a.restamp_flag = ctx->restamp_flag;
    a.gap = ctx->gap;
    return a;
}

MaskArgs mask_args(lbm_ctx* ctx, bool restamp_list)
{
    MaskArgs m{};
    m.lattice = ctx->lattice;
    m.g = ctx->g;
    m.tag = ctx->tag;
    m.ismask = ctx->ismask;
    m.pk = ctx->pk;
    m.pc = ctx->pc;
    m.tmpl = ctx->tmpl;
    m.list = restamp_list ? ctx->restamp : nullptr;
    m.cnt = ctx->cnt;
    m.np = ctx->np;
    return m;
}

PartView part_view(lbm_ctx* ctx)
{
    PartView v{};
    v.tag = ctx->np > 0 ? ctx->tag : nullptr;
    v.pk = ctx->pk;
    v.pkf = ctx->pkf;
    v.pending = ctx->pending;
    v.ismask = ctx->ismask;
    v.np = ctx->np;
    v.status = ctx->status;
    return v;
}

// Arguments of the sweep that reads buffer c and writes buffer 1 - c.
SweepArgs sweep_args(lbm_ctx* ctx, int c)
{
    SweepArgs a{};
    a.lattice = ctx->lattice;
    a.g = ctx->g;
    a.fin = ctx->f[c];
    a.fout = ctx->f[1 - c];
    a.pv = part_view(ctx);
    a.bs_scratch = ctx->bs_scratch;
    a.omega = 1.0 / ctx->tau;
    a.pre = 1.0 - 0.5 / ctx->tau;
    for (int k = 0; k < 3; ++k) a.F[k] = ctx->F[k];
    a.omega_f = (float)a.omega;
    a.pre_f = (float)a.pre;
    for (int k = 0; k < 3; ++k) a.F_f[k] = (float)ctx->F[k];
    wall_args(ctx, a);
    // automatic shape: the two-site kernel with 16 threads along x for every deviation storage
    // (fastest at the 512^3 suspension: FP32 3.63 ms against 3.87 ms for the one-site kernel,
    // which also takes odd nx and is the batch sweep's form)
    a.pair_bx = ctx->sweep_bx < 0 ? 16 : ctx->sweep_bx;
    if (ctx->inplace) {
        // parity 0: natural layout, neighbour phase next; parity 1: local phase next
        a.fin = ctx->f[0];
        a.fout = ctx->f[0];
        a.aa = 1 + c;
        a.is_rho_in = ctx->is_rho[c];
        a.is_rho_out = ctx->is_rho[1 - c];
        a.pair_bx = 0;
    }
    return a;
}

// Arguments of the IS-site bookkeeping after the sweep that read buffer c and wrote 1 - c:
// that sweep's arguments with the particle view it ran with (the copies taken at the start
// of the particle phase).
ISFixArgs is_fix_args(lbm_ctx* ctx, int c)
{
    ISFixArgs s{};
    s.s = sweep_args(ctx, c);
    s.s.pv.pk = ctx->pk_prev;
    s.s.pv.pkf = ctx->pkf_prev;
    s.s.pv.pending = ctx->pending_prev;
    s.dens = ctx->dens;
    s.pk = ctx->pk;
    s.pc = ctx->pc;
    s.tmpl = ctx->tmpl;
    s.Kold = ctx->Kold;
    s.list = ctx->changed;
    s.cnt = ctx->cnt;
    return s;
}

// One time step on ctx->stream, reading buffer c and writing buffer 1 - c. With ev != nullptr
// CUDA events are recorded before the sweep, after it, and after the particle phase.
int enqueue_step(lbm_ctx* ctx, int c, cudaEvent_t* ev = nullptr)
{
    const SweepArgs a = sweep_args(ctx, c);
    if (ev) cudaEventRecord(ev[0], ctx->stream);
    {
        NvtxRange r("lbm sweep");
        ctx->kt->sweep(a, ctx->stream);
    }
    if (ev) cudaEventRecord(ev[1], ctx->stream);
    int launches = 1;
    NvtxRange rp("lbm particle phase");
    if (ctx->np > 0) {
        const ParticleArgs pa = particle_args(ctx);
        const ISFixArgs fa = is_fix_args(ctx, c);
        launches += launch_particle_phase_a(pa, ctx->stream);
        if (ctx->inplace) {
            // in-place streaming: the IS sites kept their populations; only the sites that
            // became IS need their density in the array the next sweep reads
            launches += launch_particle_phase_b(pa, ctx->stream);
            ISFixArgs fi = fa;
            fi.dens = ctx->is_rho[1 - c];
            ctx->kt->inplace_fix(fi, ctx->stream);
            ctx->kt->update_masks(mask_args(ctx, true), ctx->stream);
            launches += 2;
        } else {
            ctx->kt->is_save(fa, ctx->stream);
            launches += launch_particle_phase_b(pa, ctx->stream);
            ctx->kt->is_fix(fa, ctx->stream);
            ctx->kt->update_masks(mask_args(ctx, true), ctx->stream);
            launches += 4;
        }
    }
    if (ctx->moving_walls) {
        launch_wall_advance(ctx->wv, ctx->pending, ctx->stream);
        launches += 1;
    }
    if (ev) cudaEventRecord(ev[2], ctx->stream);
    return launches;
}

lbm_status build_graphs(lbm_ctx* ctx)
{
    for (int c = 0; c < 2; ++c) {
        if (ctx->gexec[c]) continue;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const int launches = enqueue_step(ctx, c);
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
        if (le != cudaSuccess) return cuda_fail(ctx, le, "kernel launch during capture");
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
        cudaError_t ie = cudaGraphInstantiate(&ctx->gexec[c], graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ctx, ie, "cudaGraphInstantiate");
        ctx->launches_per_step = launches;
    }
    return LBM_OK;
}

lbm_status sync_status(lbm_ctx* ctx)
{
    CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->allocated) return LBM_OK;
    int st = 0;
    CK(cudaMemcpy(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == ERR_CAPACITY) return fail(ctx, LBM_E_CAPACITY, "a device work list overflowed (contact pairs)");
    if (st == ERR_UNSTABLE)
        return fail(ctx, LBM_E_UNSTABLE, "a particle moved by more than one lattice site in one step");
    if (st == ERR_BOUNDS)
        return fail(ctx, LBM_E_BOUNDS, "a kernel of the bounds-checked build met an index out of range");
    if (st != 0) return fail(ctx, (lbm_status)st, "device status " + std::to_string(st));
    return LBM_OK;
}

}  // namespace host
}  // namespace lbmp

extern "C" {

lbm_status lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double body_force[3])
{
    if (!out) return LBM_E_INVALID;
    *out = nullptr;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) return LBM_E_INVALID;
    if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535) return LBM_E_INVALID;
    if (lattice == LBM_D2Q9 && nz != 1) return LBM_E_INVALID;
    if (!(tau > 0.5) || !std::isfinite(tau)) return LBM_E_INVALID;
    const unsigned long long N = (unsigned long long)nx * ny * nz;
    if (N >= (1ull << 31)) return LBM_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    lbm_ctx* ctx = new lbm_ctx();
    ctx->lattice = lattice;
    ctx->Q = lattice == 0 ? 9 : 19;
    ctx->D = lattice == 0 ? 2 : 3;
    ctx->g.nx = nx;
    ctx->g.ny = ny;
    ctx->g.nz = nz;
    ctx->g.N = (unsigned)N;
    ctx->tau = tau;
    for (int k = 0; k < 3; ++k) ctx->F[k] = body_force ? body_force[k] : 0.0;
    if (lattice == 0) ctx->F[2] = 0.0;
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete ctx;
        return LBM_E_CUDA;
    }
    ctx->own_stream = true;
    *out = ctx;
    return LBM_OK;
}

lbm_status lbm_configure(lbm_ctx* ctx, int precision, const int faces[6], const double particle_gravity[3],
                         double contact_gap, int body_force_on_particles, void* cuda_stream)
{
    if (!ctx) return LBM_E_INVALID;
    if (ctx->allocated || ctx->np > 0 || ctx->stepped)
        return fail(ctx, LBM_E_STATE, "lbm_configure must precede particles, distributions and steps");
    if (!table_for(precision)) return fail(ctx, LBM_E_INVALID, "unknown precision");
    int walls[3] = {0, 0, 0}, eq = 0;
    if (faces) {
        for (int f = 0; f < 6; ++f)
            if (faces[f] != LBM_PERIODIC && faces[f] != LBM_NOSLIP && faces[f] != LBM_EQUILIBRIUM)
                return fail(ctx, LBM_E_INVALID, "unknown face kind");
        for (int k = 0; k < 3; ++k) {
            if ((faces[2 * k] == LBM_PERIODIC) != (faces[2 * k + 1] == LBM_PERIODIC))
                return fail(ctx, LBM_E_INVALID, "an axis is periodic on both faces or on neither");
            walls[k] = faces[2 * k] != LBM_PERIODIC;
        }
        for (int f = 0; f < 6; ++f)
            if (faces[f] == LBM_EQUILIBRIUM && (ctx->D == 3 || f < 4)) eq |= 1 << f;
    }
    if (ctx->D == 2) walls[2] = 0;
    if (!std::isfinite(contact_gap)) return fail(ctx, LBM_E_INVALID, "contact gap must be finite");
    ctx->precision = precision;
    ctx->g.eqface = eq;
    for (int k = 0; k < 3; ++k) {
        ctx->g.wall[k] = walls[k];
        ctx->grav[k] = particle_gravity ? particle_gravity[k] : 0.0;
    }
    if (ctx->D == 2) ctx->grav[2] = 0.0;
    ctx->gap = contact_gap;
    ctx->bfp = body_force_on_particles ? 1 : 0;
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k)
            if (!walls[f / 2]) ctx->uw[f][k] = 0.0;
    if (cuda_stream) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        ctx->stream = (cudaStream_t)cuda_stream;
        ctx->own_stream = false;
    }
    return LBM_OK;
}

lbm_status lbm_set_wall_velocity(lbm_ctx* ctx, int face, const double u[3])
{
    if (!ctx) return LBM_E_INVALID;
    if (face < 0 || face > 5 || !u) return fail(ctx, LBM_E_INVALID, "face must be 0..5 and u non-null");
    if (!ctx->g.wall[face / 2]) return fail(ctx, LBM_E_INVALID, "the face is periodic, not a wall");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(u[k])) return fail(ctx, LBM_E_INVALID, "wall velocity must be finite");
    const bool eq_face = (ctx->g.eqface >> face) & 1;
    if (!eq_face && u[face / 2] != 0.0) return fail(ctx, LBM_E_INVALID, "a wall moves only in its own plane");
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 3; ++k) ctx->uw[face][k] = (ctx->D == 2 && k == 2) ? 0.0 : u[k];
    bool moving = false;  // a moving no-slip wall: the bounce-back gains the wall momentum
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k) moving = moving || (ctx->uw[f][k] != 0.0 && !((ctx->g.eqface >> f) & 1));
    if (ctx->allocated) {
        // Only the current set changes: the streaming still pending (the values the next pull
        // completes) keeps the velocities it was taken with.
        const WallVel w = wall_vel(ctx);
        CK(cudaMemcpy(ctx->wv + 1, &w, sizeof(w), cudaMemcpyHostToDevice));
    }
    if (moving && !ctx->moving_walls) {
        ctx->moving_walls = true;  // the step graphs gain the wall term and its advance
        for (int c = 0; c < 2; ++c)
            if (ctx->gexec[c]) {
                cudaGraphExecDestroy(ctx->gexec[c]);
                ctx->gexec[c] = nullptr;
            }
    }
    return LBM_OK;
}

lbm_status lbm_add_particles(lbm_ctx* ctx, int n, const double* centers, const double* radii,
                             const double* densities, const double* velocities, const double* omegas,
                             int* first_id)
{
    if (!ctx) return LBM_E_INVALID;
    if (ctx->stepped) return fail(ctx, LBM_E_STATE, "particles must be added before the first step");
    if (n < 0 || (n > 0 && (!centers || !radii || !densities)))
        return fail(ctx, LBM_E_INVALID, "null particle arrays");
    if ((long long)ctx->np + n >= (long long)PID_MASK) return fail(ctx, LBM_E_INVALID, "too many particles");
    if (n == 0) {
        if (first_id) *first_id = ctx->np;
        return LBM_OK;
    }
    CS(ensure_alloc(ctx));
    const int D = ctx->D;
    std::vector<PConst> pc(n);
    std::vector<PKern> pk(n);
    std::vector<PKernF> pkf(n);
    std::vector<double> xs(3 * (size_t)n);
    for (int q = 0; q < n; ++q) {
        PConst& c = pc[q];
        PKern& k = pk[q];
        std::memset(&c, 0, sizeof(c));
        std::memset(&k, 0, sizeof(k));
        const double r = radii[q], rho = densities[q];
        if (!(r >= 1.5) || !(r <= 120.0)) return fail(ctx, LBM_E_INVALID, "radius must lie in [1.5, 120]");
        if (!(rho > 0.0)) return fail(ctx, LBM_E_INVALID, "density must be positive");
        c.r = r;
        for (int a = 0; a < 3; ++a) {
            c.x0[a] = a < D ? centers[3 * q + a] : 0.0;
            if (!std::isfinite(c.x0[a])) return fail(ctx, LBM_E_INVALID, "non-finite centre");
            c.A[a] = (int)std::floor(c.x0[a]);
            k.phi[a] = c.x0[a] - (double)c.A[a];
            k.K[a] = c.A[a];
            const int na = axis_n(ctx, a);
            k.Kw[a] = ctx->g.wall[a] ? c.A[a] : ((c.A[a] % na) + na) % na;
            k.u[a] = (velocities && a < D) ? velocities[3 * q + a] : 0.0;
            k.om[a] = omegas ? omegas[3 * q + a] : 0.0;
            if (D == 2 && a < 2) k.om[a] = 0.0;
            xs[3 * (size_t)q + a] = c.x0[a];
            pkf[q].u[a] = (float)k.u[a];
            pkf[q].om[a] = (float)k.om[a];
            pkf[q].phi[a] = (float)k.phi[a];
            pkf[q].Kw[a] = k.Kw[a];
        }
        for (int a = 0; a < D; ++a) {
            const int na = axis_n(ctx, a);
            if (ctx->g.wall[a]) {
                if (c.x0[a] + 0.5 < r || ((double)na - 0.5) - c.x0[a] < r)
                    return fail(ctx, LBM_E_INVALID, "particle crosses a wall");
            } else if (2.0 * (r + 2.0) >= (double)na) {
                return fail(ctx, LBM_E_INVALID, "particle wider than half the periodic box");
            }
        }
        // Continuum mass and moment of inertia of a sphere (3D) or disk (2D).
        if (std::isinf(rho)) {
            c.inv_m = 0.0;
            c.inv_I = 0.0;
            for (int a = 0; a < 3; ++a) c.ext[a] = 0.0;
        } else {
            const double vol = D == 3 ? (4.0 / 3.0) * LBM_PI * r * r * r : LBM_PI * r * r;
            const double m = rho * vol;
            const double I = D == 3 ? 0.4 * m * r * r : 0.5 * m * r * r;
            const double inv_rho = 1.0 / rho;
            c.inv_m = 1.0 / m;
            c.inv_I = 1.0 / I;
            for (int a = 0; a < 3; ++a)
                c.ext[a] = ctx->grav[a] * (1.0 - inv_rho) + (ctx->bfp ? ctx->F[a] * inv_rho : 0.0);
        }
    }
    // Hard-core particles may not overlap (Sec. 2.3). Candidates come from a uniform grid of
    // cells at least 2 r_max wide, so each new particle is tested against 27 cells.
    std::vector<double> allx(ctx->h_x);
    allx.insert(allx.end(), xs.begin(), xs.end());
    std::vector<double> allr;
    for (auto& c : ctx->h_pc) allr.push_back(c.r);
    for (auto& c : pc) allr.push_back(c.r);
    const int tot = ctx->np + n;
    {
        double rmax_all = 0.0;
        for (double rr : allr) rmax_all = std::max(rmax_all, rr);
        int nc[3];
        double cs[3];
        for (int a = 0; a < 3; ++a) {
            const int na = axis_n(ctx, a);
            nc[a] = a < D ? std::max(1, std::min(1024, (int)std::floor((double)na / (2.0 * rmax_all + 1e-9)))) : 1;
            cs[a] = (double)na / nc[a];
        }
        auto cell_of = [&](int i, int a) {
            const int na = axis_n(ctx, a);
            double v = allx[3 * (size_t)i + a];
            if (a >= D) return 0;
            v = ctx->g.wall[a] ? v + 0.5 : v - (double)na * std::floor(v / (double)na);
            int c = (int)std::floor(v / cs[a]);
            return std::min(std::max(c, 0), nc[a] - 1);
        };
        std::vector<std::vector<int>> cells((size_t)nc[0] * nc[1] * nc[2]);
        for (int i = 0; i < tot; ++i)
            cells[((size_t)cell_of(i, 2) * nc[1] + cell_of(i, 1)) * nc[0] + cell_of(i, 0)].push_back(i);
        for (int i = ctx->np; i < tot; ++i) {
            const int ci[3] = {cell_of(i, 0), cell_of(i, 1), cell_of(i, 2)};
            std::vector<size_t> seen;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                        bool skip = false;
                        for (int a = 0; a < 3; ++a) {
                            if (cc[a] < 0 || cc[a] >= nc[a]) {
                                if (ctx->g.wall[a] || a >= D) skip = true;
                                cc[a] = (cc[a] + nc[a]) % nc[a];
                            }
                        }
                        if (skip) continue;
                        const size_t cid = ((size_t)cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
                        if (std::find(seen.begin(), seen.end(), cid) != seen.end()) continue;
                        seen.push_back(cid);
                        for (int j : cells[cid]) {
                            if (j >= i) continue;
                            double d2 = 0.0;
                            for (int a = 0; a < 3; ++a) {
                                const double d = min_image_h(allx[3 * (size_t)i + a] - allx[3 * (size_t)j + a],
                                                             axis_n(ctx, a), a < D && !ctx->g.wall[a]);
                                d2 += d * d;
                            }
                            const double R = allr[i] + allr[j];
                            if (d2 < R * R)
                                return fail(ctx, LBM_E_OVERLAP, "particles " + std::to_string(j) + " and " +
                                                                    std::to_string(i) + " overlap");
                        }
                    }
        }
    }
    // Site classification of each new particle (independent, spread over host threads).
    std::vector<std::vector<int>> tm(n);
    std::vector<int> nbs(n), nis(n);
    {
        const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t]() {
                for (int q = (int)t; q < n; q += (int)nt)
                    classify(ctx->lattice, pk[q].phi, pc[q].r, tm[q], nbs[q], nis[q]);
            });
        for (auto& t : th) t.join();
    }
    size_t total = ctx->h_tmpl.size();
    for (int q = 0; q < n; ++q) total += tm[q].size();
    if (total >= (1ull << 31)) return fail(ctx, LBM_E_INVALID, "too many particle sites");
    ctx->h_tmpl.reserve(total);
    for (int q = 0; q < n; ++q) {
        pc[q].tmpl_off = (int)ctx->h_tmpl.size();
        pc[q].tmpl_n = (int)tm[q].size();
        pc[q].n_bs = nbs[q];
        pc[q].n_is = nis[q];
        ctx->h_tmpl.insert(ctx->h_tmpl.end(), tm[q].begin(), tm[q].end());
    }
    ctx->h_pc.insert(ctx->h_pc.end(), pc.begin(), pc.end());
    ctx->h_pk.insert(ctx->h_pk.end(), pk.begin(), pk.end());
    ctx->h_pkf.insert(ctx->h_pkf.end(), pkf.begin(), pkf.end());
    ctx->h_x.insert(ctx->h_x.end(), xs.begin(), xs.end());
    for (int q = 0; q < n; ++q) ctx->h_q.insert(ctx->h_q.end(), {1.0, 0.0, 0.0, 0.0});
    const int first = ctx->np;
    ctx->np = tot;

    // (Re)build the device-side particle arrays.
    CK(cudaStreamSynchronize(ctx->stream));
    auto release = [&](void* p) {
        if (!p) return;
        auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
        if (it != ctx->allocs.end()) {
            const size_t k = (size_t)(it - ctx->allocs.begin());
            ctx->dev_bytes -= ctx->alloc_bytes[k];
            ctx->allocs.erase(it);
            ctx->alloc_bytes.erase(ctx->alloc_bytes.begin() + (std::ptrdiff_t)k);
        }
        cudaFree(p);
    };
    for (void* p : {(void*)ctx->pk, (void*)ctx->pkf, (void*)ctx->pk_prev, (void*)ctx->pkf_prev, (void*)ctx->pc, (void*)ctx->tmpl, (void*)ctx->x, (void*)ctx->q, (void*)ctx->xpf, (void*)ctx->un,
                    (void*)ctx->acc, (void*)ctx->force, (void*)ctx->Kold, (void*)ctx->cell_of,
                    (void*)ctx->cell_count, (void*)ctx->cell_start, (void*)ctx->cell_cursor,
                    (void*)ctx->cell_items, (void*)ctx->changed, (void*)ctx->restamp,
                    (void*)ctx->restamp_flag, (void*)ctx->pout})
        release(p);
    const size_t np = (size_t)ctx->np;
    CS(dev_alloc(ctx, &ctx->pk, sizeof(PKern) * np));
    CS(dev_alloc(ctx, &ctx->pkf, sizeof(PKernF) * np));
    CS(dev_alloc(ctx, &ctx->pk_prev, sizeof(PKern) * np));
    CS(dev_alloc(ctx, &ctx->pkf_prev, sizeof(PKernF) * np));
    CS(dev_alloc(ctx, &ctx->pc, sizeof(PConst) * np));
    CS(dev_alloc(ctx, &ctx->tmpl, sizeof(int) * ctx->h_tmpl.size()));
    CS(dev_alloc(ctx, &ctx->x, sizeof(double) * 3 * np));
    CS(dev_alloc(ctx, &ctx->q, sizeof(double) * 4 * np));
    CS(dev_alloc(ctx, &ctx->xpf, sizeof(float4) * np));
    CS(dev_alloc(ctx, &ctx->un, sizeof(double) * 3 * np));
    CS(dev_alloc(ctx, &ctx->acc, sizeof(double) * 6 * np));
    CS(dev_alloc(ctx, &ctx->force, sizeof(double) * 6 * np));
    CS(dev_alloc(ctx, &ctx->Kold, sizeof(int) * 3 * np));
    CS(dev_alloc(ctx, &ctx->cell_of, sizeof(int) * np));
    CS(dev_alloc(ctx, &ctx->cell_items, sizeof(int) * np));
    CS(dev_alloc(ctx, &ctx->changed, sizeof(int) * np));
    CS(dev_alloc(ctx, &ctx->restamp, sizeof(int) * np));
    CS(dev_alloc(ctx, &ctx->restamp_flag, sizeof(int) * np));
    CS(dev_alloc(ctx, &ctx->pout, sizeof(double) * (15 * np + 1)));
    if (!ctx->tag) {
        CS(dev_alloc(ctx, &ctx->tag, sizeof(unsigned) * (size_t)ctx->g.N));
        if (!ctx->inplace) CS(dev_alloc(ctx, &ctx->dens, (size_t)ctx->kt->compute_bytes * ctx->g.N));
        CS(dev_alloc(ctx, &ctx->cnt, sizeof(Counters)));
        CS(dev_alloc(ctx, &ctx->pairs, sizeof(unsigned long long) * PAIR_CAP));
        CS(dev_alloc(ctx, &ctx->ismask, sizeof(unsigned) * (size_t)ctx->g.N));
        CS(dev_alloc(ctx, (char**)&ctx->bs_scratch, bs_record_bytes(ctx)));
        CK(prepare_particle_kernels(PAIR_CAP));
    }
    // Cell grid for contact and neighbour searches: cells at least 2 r_max + gap + 4 wide.
    double rmax = 0.0;
    for (auto& c : ctx->h_pc) rmax = std::max(rmax, c.r);
    const double h = 2.0 * rmax + std::max(ctx->gap, 0.0) + 4.0;
    ctx->cg.total = 1;
    for (int a = 0; a < 3; ++a) {
        const int na = axis_n(ctx, a);
        ctx->cg.n[a] = a < D ? std::max(1, (int)std::floor((double)na / h)) : 1;
        ctx->cg.size[a] = a < D ? (double)na / ctx->cg.n[a] : 1e300;
        ctx->cg.total *= ctx->cg.n[a];
    }
    CS(dev_alloc(ctx, &ctx->cell_count, sizeof(int) * (size_t)ctx->cg.total));
    CS(dev_alloc(ctx, &ctx->cell_start, sizeof(int) * ((size_t)ctx->cg.total + 1)));
    CS(dev_alloc(ctx, &ctx->cell_cursor, sizeof(int) * (size_t)ctx->cg.total));

    CK(cudaMemcpyAsync(ctx->pk, ctx->h_pk.data(), sizeof(PKern) * np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pkf, ctx->h_pkf.data(), sizeof(PKernF) * np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pc, ctx->h_pc.data(), sizeof(PConst) * np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->tmpl, ctx->h_tmpl.data(), sizeof(int) * ctx->h_tmpl.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->x, ctx->h_x.data(), sizeof(double) * 3 * np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->q, ctx->h_q.data(), sizeof(double) * 4 * np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 6 * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->force, 0, sizeof(double) * 6 * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->tag, 0xFF, sizeof(unsigned) * (size_t)ctx->g.N, ctx->stream));
    // no record may carry a BS code before the first sweep writes them
    CK(cudaMemsetAsync(ctx->bs_scratch, 0, bs_record_bytes(ctx), ctx->stream));
    launch_stamp_all(particle_args(ctx), ctx->stream);
    ctx->kt->update_masks(mask_args(ctx, false), ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < 2; ++c)
        if (ctx->gexec[c]) {
            cudaGraphExecDestroy(ctx->gexec[c]);
            ctx->gexec[c] = nullptr;
        }
    if (first_id) *first_id = first;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int n)
{
    if (!ctx) return LBM_E_INVALID;
    if (n < 0) return fail(ctx, LBM_E_INVALID, "negative step count");
    if (n == 0) return LBM_OK;
    CS(ensure_alloc(ctx));
    CS(build_graphs(ctx));
    ctx->stepped = true;
    NvtxRange r("lbm_step");
    for (int s = 0; s < n; ++s) {
        CK(cudaGraphLaunch(ctx->gexec[ctx->cur], ctx->stream));
        ctx->cur ^= 1;
        ++ctx->steps;
    }
    return LBM_OK;
}

lbm_status lbm_set_streaming(lbm_ctx* ctx, int mode)
{
    if (!ctx) return LBM_E_INVALID;
    if (mode != LBM_STREAM_PULL && mode != LBM_STREAM_INPLACE)
        return fail(ctx, LBM_E_INVALID, "streaming mode must be LBM_STREAM_PULL or LBM_STREAM_INPLACE");
    if (ctx->allocated || ctx->np > 0 || ctx->stepped)
        return fail(ctx, LBM_E_STATE, "lbm_set_streaming must precede particles, distributions and steps");
    ctx->inplace = mode == LBM_STREAM_INPLACE;
    return LBM_OK;
}

lbm_status lbm_set_sweep_shape(lbm_ctx* ctx, int threads_x)
{
    if (!ctx) return LBM_E_INVALID;
    if (!(threads_x == -1 || threads_x == 0 || threads_x == 16 || threads_x == 32 || threads_x == 64 ||
          threads_x == 128))
        return fail(ctx, LBM_E_INVALID, "sweep shape: threads_x must be -1, 0, 16, 32, 64 or 128");
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    ctx->sweep_bx = threads_x;
    for (auto& ge : ctx->gexec)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
    return LBM_OK;
}

lbm_status lbm_profile_steps(lbm_ctx* ctx, int n, double out_ms[3])
{
    if (!ctx || !out_ms || n < 1) return LBM_E_INVALID;
    CS(ensure_alloc(ctx));
    CS(build_graphs(ctx));
    ctx->stepped = true;
    std::vector<cudaEvent_t> ev(3 * (size_t)n, nullptr);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    for (int s = 0; s < n; ++s) {
        enqueue_step(ctx, ctx->cur, &ev[3 * (size_t)s]);
        ctx->cur ^= 1;
        ++ctx->steps;
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    double acc[3] = {0, 0, 0};
    for (int s = 0; s < n && le == cudaSuccess && se == cudaSuccess; ++s) {
        float a = 0, b = 0, c = 0;
        cudaEventElapsedTime(&a, ev[3 * (size_t)s], ev[3 * (size_t)s + 1]);
        cudaEventElapsedTime(&b, ev[3 * (size_t)s + 1], ev[3 * (size_t)s + 2]);
        cudaEventElapsedTime(&c, ev[3 * (size_t)s], ev[3 * (size_t)s + 2]);
        acc[0] += a;
        acc[1] += b;
        acc[2] += c;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (le != cudaSuccess) return cuda_fail(ctx, le, "kernel launch");
    if (se != cudaSuccess) return cuda_fail(ctx, se, "cudaStreamSynchronize");
    for (int k = 0; k < 3; ++k) out_ms[k] = acc[k] / n;
    return sync_status(ctx);
}

lbm_status lbm_synchronize(lbm_ctx* ctx)
{
    if (!ctx) return LBM_E_INVALID;
    return sync_status(ctx);
}

static lbm_status materialize(lbm_ctx* ctx, int mode, double* out_a, double* out_b)
{
    CS(ensure_alloc(ctx));
    CS(sync_status(ctx));
    const size_t N = ctx->g.N;
    const size_t per_site = mode == 0 ? 4 : (size_t)ctx->Q;
    const size_t chunk = std::min(N, STAGING_BYTES / (per_site * sizeof(double)));
    for (size_t s0 = 0; s0 < N; s0 += chunk) {
        const size_t cnt = std::min(chunk, N - s0);
        MaterializeArgs a{};
        a.lattice = ctx->lattice;
        a.g = ctx->g;
        a.fin = ctx->f[ctx->inplace ? 0 : ctx->cur];
        a.aa = ctx->inplace ? ctx->cur : 0;
        a.is_rho = ctx->inplace ? ctx->is_rho[ctx->cur] : nullptr;
        a.pv = part_view(ctx);
        for (int k = 0; k < 3; ++k) a.F[k] = ctx->F[k];
        wall_args(ctx, a);
        a.s0 = (unsigned)s0;
        a.count = (unsigned)cnt;
        a.mode = mode;
        a.out0 = ctx->staging;
        a.out1 = ctx->staging + cnt;
        ctx->kt->materialize(a, ctx->stream);
        CK(cudaGetLastError());
        if (mode == 0) {
            if (out_a) CK(cudaMemcpyAsync(out_a + s0, ctx->staging, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
            if (out_b)
                CK(cudaMemcpyAsync(out_b + 3 * s0, ctx->staging + cnt, sizeof(double) * 3 * cnt,
                                   cudaMemcpyDeviceToHost, ctx->stream));
        } else {
            for (int i = 0; i < ctx->Q; ++i)
                CK(cudaMemcpyAsync(out_a + (size_t)i * N + s0, ctx->staging + (size_t)i * cnt, sizeof(double) * cnt,
                                   cudaMemcpyDeviceToHost, ctx->stream));
        }
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return LBM_OK;
}

lbm_status lbm_closure_features(lbm_ctx* ctx, int n_side, double spacing, double u_ref, float* out)
{
    if (!ctx || !out || n_side < 1 || n_side > 8 || !(spacing > 0.0) || !(u_ref != 0.0) || !std::isfinite(u_ref))
        return LBM_E_INVALID;
    if (ctx->np == 0) return LBM_OK;
    CS(ensure_alloc(ctx));
    FeatureArgs f{};
    f.m.lattice = ctx->lattice;
    f.m.g = ctx->g;
    f.m.fin = ctx->f[ctx->inplace ? 0 : ctx->cur];
    f.m.aa = ctx->inplace ? ctx->cur : 0;
    f.m.is_rho = ctx->inplace ? ctx->is_rho[ctx->cur] : nullptr;
    f.m.pv = part_view(ctx);
    for (int k = 0; k < 3; ++k) f.m.F[k] = ctx->F[k];
    wall_args(ctx, f.m);
    f.x = ctx->x;
    f.pk = ctx->pk;
    f.np = ctx->np;
    f.n_side = n_side;
    f.h = spacing;
    f.u_ref = u_ref;
    f.out = out;
    ctx->kt->features(f, ctx->stream);
    CK(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho, double* u)
{
    if (!ctx) return LBM_E_INVALID;
    return materialize(ctx, 0, rho, u);
}

lbm_status lbm_get_distributions(lbm_ctx* ctx, double* f)
{
    if (!ctx || !f) return LBM_E_INVALID;
    return materialize(ctx, 1, f, nullptr);
}

lbm_status lbm_set_distributions(lbm_ctx* ctx, const double* f)
{
    if (!ctx || !f) return LBM_E_INVALID;
    CS(ensure_alloc(ctx));
    CS(sync_status(ctx));
    const size_t N = ctx->g.N;
    const size_t chunk = std::min(N, STAGING_BYTES / ((size_t)ctx->Q * sizeof(double)));
    // pull scheme: into the other buffer, then shifted so that the pull returns f; in-place
    // streaming: straight into the layout a neighbour phase leaves (slot opp(i) of x holds f_i(x))
    void* tmp = ctx->inplace ? ctx->f[0] : ctx->f[1 - ctx->cur];
    for (size_t s0 = 0; s0 < N; s0 += chunk) {
        const size_t cnt = std::min(chunk, N - s0);
        for (int i = 0; i < ctx->Q; ++i)
            CK(cudaMemcpyAsync(ctx->staging + (size_t)i * cnt, f + (size_t)i * N + s0, sizeof(double) * cnt,
                               cudaMemcpyHostToDevice, ctx->stream));
        ConvertArgs a{};
        a.lattice = ctx->lattice;
        a.g = ctx->g;
        a.f = ctx->staging;
        a.dst = tmp;
        a.s0 = (unsigned)s0;
        a.count = (unsigned)cnt;
        a.opp = ctx->inplace ? 1 : 0;
        ctx->kt->convert_in(a, ctx->stream);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->inplace) {
        ctx->cur = 1;
    } else {
        UnstreamArgs u{};
        u.lattice = ctx->lattice;
        u.g = ctx->g;
        u.src = tmp;
        u.dst = ctx->f[ctx->cur];
        ctx->kt->unstream(u, ctx->stream);
        CK(cudaGetLastError());
    }
    CK(cudaMemsetAsync(ctx->pending, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_get_particles(lbm_ctx* ctx, double* x, double* u, double* omega, double* force, double* torque)
{
    if (!ctx) return LBM_E_INVALID;
    const size_t np = (size_t)ctx->np;
    if (np == 0) return sync_status(ctx);
    // One kernel packs x, u, omega, force, torque into the staging buffer; one copy brings
    // them to a pinned host buffer.
    const size_t bytes = sizeof(double) * 15 * np;
    if (ctx->pinned_bytes < bytes) {
        if (ctx->pinned) cudaFreeHost(ctx->pinned);
        ctx->pinned = nullptr;
        ctx->pinned_bytes = 0;
        CK(cudaMallocHost(&ctx->pinned, bytes));
        ctx->pinned_bytes = bytes;
    }
    launch_pack_particles(particle_args(ctx), ctx->pout, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->pinned, ctx->pout, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CS(sync_status(ctx));
    const double* h = (const double*)ctx->pinned;
    double* outs[5] = {x, u, omega, force, torque};
    for (int k = 0; k < 5; ++k)
        if (outs[k]) std::memcpy(outs[k], h + (size_t)k * 3 * np, sizeof(double) * 3 * np);
    return LBM_OK;
}

lbm_status lbm_get_orientations(lbm_ctx* ctx, double* q)
{
    if (!ctx || !q) return LBM_E_INVALID;
    const size_t np = (size_t)ctx->np;
    if (np == 0) return sync_status(ctx);
    const size_t bytes = sizeof(double) * 4 * np;
    if (ctx->pinned_bytes < bytes) {
        if (ctx->pinned) cudaFreeHost(ctx->pinned);
        ctx->pinned = nullptr;
        ctx->pinned_bytes = 0;
        CK(cudaMallocHost(&ctx->pinned, bytes));
        ctx->pinned_bytes = bytes;
    }
    CK(cudaMemcpyAsync(ctx->pinned, ctx->q, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CS(sync_status(ctx));
    std::memcpy(q, ctx->pinned, bytes);
    return LBM_OK;
}

lbm_status lbm_get_particles_async(lbm_ctx* ctx, double* dst, long long* ticket)
{
    if (!ctx || !dst || !ticket) return LBM_E_INVALID;
    if (ctx->np == 0) return fail(ctx, LBM_E_INVALID, "no particles");
    int slot = -1;
    for (int k = 0; k < lbm_ctx::RB_SLOTS; ++k)
        if (!ctx->rb_busy[k]) {
            slot = k;
            break;
        }
    if (slot < 0) return fail(ctx, LBM_E_INVALID, "8 particle read-backs are outstanding; wait for one first");
    if (!ctx->rb_ev[slot]) CK(cudaEventCreateWithFlags(&ctx->rb_ev[slot], cudaEventDisableTiming));
    const size_t bytes = sizeof(double) * (15 * (size_t)ctx->np + 1);
    launch_pack_particles(particle_args(ctx), ctx->pout, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dst, ctx->pout, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaEventRecord(ctx->rb_ev[slot], ctx->stream));
    ctx->rb_busy[slot] = true;
    ctx->rb_dst[slot] = dst;
    ctx->rb_ticket[slot] = ++ctx->rb_count;
    *ticket = ctx->rb_count;
    return LBM_OK;
}

lbm_status lbm_wait_particles(lbm_ctx* ctx, long long ticket)
{
    if (!ctx) return LBM_E_INVALID;
    for (int k = 0; k < lbm_ctx::RB_SLOTS; ++k) {
        if (!ctx->rb_busy[k] || ctx->rb_ticket[k] != ticket) continue;
        ctx->rb_busy[k] = false;
        CK(cudaEventSynchronize(ctx->rb_ev[k]));
        const int st = (int)ctx->rb_dst[k][15 * (size_t)ctx->np];
        if (st == ERR_CAPACITY) return fail(ctx, LBM_E_CAPACITY, "a device work list overflowed (contact pairs)");
        if (st == ERR_UNSTABLE)
            return fail(ctx, LBM_E_UNSTABLE, "a particle moved by more than one lattice site in one step");
        if (st != 0) return fail(ctx, (lbm_status)st, "device status " + std::to_string(st));
        return LBM_OK;
    }
    return fail(ctx, LBM_E_INVALID, "no outstanding particle read-back with this ticket");
}

lbm_status lbm_get_masks(lbm_ctx* ctx, unsigned* tags)
{
    if (!ctx || !tags) return LBM_E_INVALID;
    CS(sync_status(ctx));
    if (ctx->np == 0 || !ctx->tag) {
        std::memset(tags, 0xFF, sizeof(unsigned) * (size_t)ctx->g.N);
        return LBM_OK;
    }
    CK(cudaMemcpy(tags, ctx->tag, sizeof(unsigned) * (size_t)ctx->g.N, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_ctx* ctx, long long out[6])
{
    if (!ctx || !out) return LBM_E_INVALID;
    const int eb = table_for(ctx->precision)->elem_bytes;
    if (!ctx->gexec[0] && ctx->allocated) build_graphs(ctx);
    out[0] = ctx->np;
    out[1] = ctx->steps;
    out[2] = ctx->launches_per_step;
    out[3] = (long long)ctx->dev_bytes;
    out[4] = ctx->inplace ? (long long)ctx->Q * eb + 2LL * table_for(ctx->precision)->compute_bytes
                          : 2LL * ctx->Q * eb;
    out[5] = ctx->precision;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

void lbm_destroy(lbm_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (int c = 0; c < 2; ++c)
        if (ctx->gexec[c]) cudaGraphExecDestroy(ctx->gexec[c]);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (auto& e : ctx->rb_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
