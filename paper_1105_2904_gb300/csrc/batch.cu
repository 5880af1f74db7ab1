// Batched ensembles of independent cells (the C-ABI lbm_batch_* of include/lbmp.h).
//
// Every cell is an ordinary simulation context (its own lattice, storage, particles and
// owner map), so the single-context getters and setters work on it unchanged. The batch
// replaces the cells' separate step graphs by one: a single sweep launch over a schedule
// table of (cell, tile) entries, and one launch per particle-phase kernel with the cell in
// blockIdx.y. Per-cell kernel arguments live in small device arrays; the arithmetic per site
// and per particle is the single-context code, so a batch gives the same bits as its cells
// stepped one by one.
#include <algorithm>
#include <numeric>

#include "ctx.h"

using namespace lbmp;
using namespace lbmp::host;

struct lbm_batch {
    int lattice = 1;
    int precision = LBM_FP32;
    std::vector<lbm_ctx*> cells;
    cudaStream_t stream = nullptr;
    const KernelTable* kt = nullptr;

    // tuning
    std::vector<int> tile_w;  // per cell: 32, 64 or 128 sites along x per tile
    int order = 0;
    int grid = 0;
    int steps_per_graph = 1;

    // device-side argument arrays and schedule
    SweepArgs* d_sweep[2] = {nullptr, nullptr};
    ISFixArgs* d_isfix[2] = {nullptr, nullptr};
    ParticleArgs* d_part = nullptr;
    MaskArgs* d_mask = nullptr;
    int4* d_table = nullptr;
    int ntiles = 0;
    PhaseShape shape{};
    bool any_part = false, any_walls = false;
    std::vector<int> moving;  // cells with moving walls
    std::vector<int> built_np;  // particles of each cell when the arrays were built

    cudaGraphExec_t g1[2] = {nullptr, nullptr};
    cudaGraphExec_t gk[2] = {nullptr, nullptr};
    bool built = false;
    int launches_per_step = 0;
    long long steps = 0;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& msg)
{
    if (b) b->err = msg;
    return s;
}

#define BK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define BS(call)                                     \
    do {                                             \
        lbm_status s_ = (call);                      \
        if (s_ != LBM_OK) return s_;                 \
    } while (0)

// Status of a call on cell i, with the cell's message carried into the batch.
lbm_status from_cell(lbm_batch* b, int i, lbm_status s)
{
    if (s != LBM_OK) b->err = "cell " + std::to_string(i) + ": " + lbm_last_error(b->cells[(size_t)i]);
    return s;
}

void drop_graphs(lbm_batch* b)
{
    for (int c = 0; c < 2; ++c) {
        if (b->g1[c]) cudaGraphExecDestroy(b->g1[c]);
        if (b->gk[c]) cudaGraphExecDestroy(b->gk[c]);
        b->g1[c] = b->gk[c] = nullptr;
    }
}

void release_device(lbm_batch* b)
{
    drop_graphs(b);
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
    b->d_sweep[0] = b->d_sweep[1] = nullptr;
    b->d_isfix[0] = b->d_isfix[1] = nullptr;
    b->d_part = nullptr;
    b->d_mask = nullptr;
    b->d_table = nullptr;
    b->built = false;
}

template <typename T>
lbm_status upload(lbm_batch* b, T** dst, const std::vector<T>& src)
{
    void* q = nullptr;
    BK(cudaMalloc(&q, std::max<size_t>(16, sizeof(T) * src.size())));
    b->allocs.push_back(q);
    *dst = (T*)q;
    if (!src.empty()) BK(cudaMemcpy(q, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return LBM_OK;
}

int log2_width(int w) { return w == 32 ? 5 : (w == 64 ? 6 : 7); }

// One step of every cell from buffer parity c.
int enqueue_batch_step(lbm_batch* b, int c, cudaEvent_t* ev = nullptr)
{
    BatchSweepArgs a{};
    a.lattice = b->lattice;
    a.cells = b->d_sweep[c];
    a.table = b->d_table;
    a.ntiles = b->ntiles;
    a.walls = b->any_walls ? 1 : 0;
    a.part = b->any_part ? 1 : 0;
    a.grid = b->grid;
    if (ev) cudaEventRecord(ev[0], b->stream);
    b->kt->sweep_batch(a, b->stream);
    if (ev) cudaEventRecord(ev[1], b->stream);
    int launches = 1;
    if (b->any_part) {
        const int nc = (int)b->cells.size();
        launches += launch_particle_phase_batch_a(b->d_part, b->shape, b->stream);
        b->kt->is_save_batch(b->lattice, b->d_isfix[c], nc, b->stream);
        launches += launch_particle_phase_batch_b(b->d_part, b->shape, b->stream);
        b->kt->is_fix_batch(b->lattice, b->d_isfix[c], nc, b->stream);
        b->kt->update_masks_batch(b->lattice, b->d_mask, nc, b->stream);
        launches += 4;
    }
    for (int i : b->moving) {
        launch_wall_advance(b->cells[(size_t)i]->wv, b->cells[(size_t)i]->pending, b->stream);
        ++launches;
    }
    if (ev) cudaEventRecord(ev[2], b->stream);
    return launches;
}

lbm_status capture(lbm_batch* b, int c, int nsteps, cudaGraphExec_t* out)
{
    cudaGraph_t graph = nullptr;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    for (int s = 0; s < nsteps; ++s) launches = enqueue_batch_step(b, (c + s) & 1);
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (le != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("kernel launch during capture: ") + cudaGetErrorString(le));
    if (ce != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    b->launches_per_step = launches;
    return LBM_OK;
}

// Device argument arrays, the schedule table and the step graphs.
lbm_status build(lbm_batch* b)
{
    if (b->built) return LBM_OK;
    const int nc = (int)b->cells.size();
    const int cur = b->cells[0]->cur;
    for (int i = 0; i < nc; ++i) {
        lbm_ctx* ctx = b->cells[(size_t)i];
        if (ctx->inplace) return bfail(b, LBM_E_STATE, "in-place streaming is for single contexts, not batch cells");
        BS(from_cell(b, i, ensure_alloc(ctx)));
        if (ctx->cur != cur)
            return bfail(b, LBM_E_STATE, "the cells of a batch must share their buffer parity (step them together)");
    }
    release_device(b);
    b->any_part = b->any_walls = false;
    b->moving.clear();
    b->shape = PhaseShape{};
    b->shape.ncells = nc;
    b->shape.scratch_f64 = b->precision == LBM_FP64 ? 1 : 0;
    long long max_pairs = 1;
    for (int i = 0; i < nc; ++i) {
        lbm_ctx* ctx = b->cells[(size_t)i];
        b->any_part = b->any_part || ctx->np > 0;
        b->any_walls = b->any_walls || ctx->g.wall[0] || ctx->g.wall[1] || ctx->g.wall[2];
        if (ctx->moving_walls) b->moving.push_back(i);
        b->shape.max_np = std::max(b->shape.max_np, ctx->np);
        if (ctx->np > 0) b->shape.max_cells = std::max(b->shape.max_cells, ctx->cg.total);
        max_pairs = std::max(max_pairs, (long long)ctx->np * (ctx->np - 1) / 2);
    }
    // Each cell's resolve buffer holds all its possible pairs (up to the single-context cap).
    int cap = 32;
    while (cap < max_pairs && cap < PAIR_CAP) cap <<= 1;
    b->shape.pair_cap = std::min(cap, PAIR_CAP);
    b->built_np.clear();
    for (lbm_ctx* ctx : b->cells) b->built_np.push_back(ctx->np);

    std::vector<SweepArgs> sw[2];
    std::vector<ISFixArgs> st[2];
    std::vector<ParticleArgs> pa;
    std::vector<MaskArgs> ma;
    for (int i = 0; i < nc; ++i) {
        lbm_ctx* ctx = b->cells[(size_t)i];
        for (int c = 0; c < 2; ++c) {
            sw[c].push_back(sweep_args(ctx, c));
            st[c].push_back(ctx->np > 0 ? is_fix_args(ctx, c) : ISFixArgs{});
        }
        if (ctx->np > 0) {
            ParticleArgs p = particle_args(ctx);
            p.pair_cap = b->shape.pair_cap;
            pa.push_back(p);
            ma.push_back(mask_args(ctx, true));
        } else {
            pa.push_back(ParticleArgs{});
            ma.push_back(MaskArgs{});
        }
    }
    std::vector<int> dims(3 * (size_t)nc);
    for (int i = 0; i < nc; ++i) {
        dims[3 * (size_t)i] = b->cells[(size_t)i]->g.nx;
        dims[3 * (size_t)i + 1] = b->cells[(size_t)i]->g.ny;
        dims[3 * (size_t)i + 2] = b->cells[(size_t)i]->g.nz;
    }
    const long long nt = lbm_schedule_tiles(nc, dims.data(), b->tile_w.data(), b->order, nullptr);
    if (nt < 0) return bfail(b, LBM_E_INVALID, "schedule");
    if (nt >= (1ll << 31)) return bfail(b, LBM_E_INVALID, "too many tiles");
    std::vector<int4> table((size_t)nt);
    lbm_schedule_tiles(nc, dims.data(), b->tile_w.data(), b->order, (int*)table.data());
    b->ntiles = (int)nt;
    for (int c = 0; c < 2; ++c) {
        BS(upload(b, &b->d_sweep[c], sw[c]));
        BS(upload(b, &b->d_isfix[c], st[c]));
    }
    BS(upload(b, &b->d_part, pa));
    BS(upload(b, &b->d_mask, ma));
    BS(upload(b, &b->d_table, table));
    for (int c = 0; c < 2; ++c) {
        BS(capture(b, c, 1, &b->g1[c]));
        if (b->steps_per_graph > 1) BS(capture(b, c, b->steps_per_graph, &b->gk[c]));
    }
    b->built = true;
    return LBM_OK;
}

// The argument arrays and graphs follow the cells: a cell that gained particles or a moving
// wall through its own context since they were built makes them stale.
void drop_if_stale(lbm_batch* b)
{
    if (!b->built) return;
    for (size_t i = 0; i < b->cells.size(); ++i) {
        const bool mv = std::find(b->moving.begin(), b->moving.end(), (int)i) != b->moving.end();
        if (b->cells[i]->np != b->built_np[i] || b->cells[i]->moving_walls != mv) {
            release_device(b);
            return;
        }
    }
}

lbm_status same_parity(lbm_batch* b)
{
    for (lbm_ctx* ctx : b->cells)
        if (ctx->cur != b->cells[0]->cur)
            return bfail(b, LBM_E_STATE, "the cells of a batch must share their buffer parity (step them together)");
    return LBM_OK;
}

void advance_cells(lbm_batch* b, int n)
{
    for (lbm_ctx* ctx : b->cells) {
        ctx->stepped = true;
        ctx->steps += n;
        if (n & 1) ctx->cur ^= 1;
    }
    b->steps += n;
}

}  // namespace

extern "C" {

long long lbm_schedule_tiles(int ncells, const int* dims, const int* tile_width, int order, int* out)
{
    if (ncells < 1 || !dims || order < 0 || order > 2) return -1;
    std::vector<std::vector<int4>> per((size_t)ncells);
    for (int i = 0; i < ncells; ++i) {
        const int nx = dims[3 * (size_t)i], ny = dims[3 * (size_t)i + 1], nz = dims[3 * (size_t)i + 2];
        if (nx < 1 || ny < 1 || nz < 1 || ny > 65535) return -1;
        const int w = tile_width ? tile_width[i] : 128;
        if (w != 32 && w != 64 && w != 128) return -1;
        const int h = 128 / w, lw = log2_width(w);
        if (!out) {
            per[(size_t)i].resize((size_t)((nx + w - 1) / w) * ((ny + h - 1) / h) * nz);
            continue;
        }
        for (int z = 0; z < nz; ++z)
            for (int y0 = 0; y0 < ny; y0 += h)
                for (int x0 = 0; x0 < nx; x0 += w) per[(size_t)i].push_back(make_int4(i, x0, y0 | (lw << 16), z));
    }
    long long total = 0;
    for (auto& v : per) total += (long long)v.size();
    if (!out) return total;
    std::vector<int> seq((size_t)ncells);
    std::iota(seq.begin(), seq.end(), 0);
    if (order == 2)  // largest cell first (ties by index)
        std::stable_sort(seq.begin(), seq.end(), [&](int a, int c) {
            const long long sa = (long long)dims[3 * (size_t)a] * dims[3 * (size_t)a + 1] * dims[3 * (size_t)a + 2];
            const long long sc = (long long)dims[3 * (size_t)c] * dims[3 * (size_t)c + 1] * dims[3 * (size_t)c + 2];
            return sa > sc;
        });
    size_t k = 0;
    auto put = [&](const int4& t) {
        out[4 * k] = t.x;
        out[4 * k + 1] = t.y;
        out[4 * k + 2] = t.z;
        out[4 * k + 3] = t.w;
        ++k;
    };
    if (order == 1) {  // one tile of each cell in turn
        size_t longest = 0;
        for (auto& v : per) longest = std::max(longest, v.size());
        for (size_t j = 0; j < longest; ++j)
            for (int i = 0; i < ncells; ++i)
                if (j < per[(size_t)i].size()) put(per[(size_t)i][j]);
    } else {
        for (int i : seq)
            for (const int4& t : per[(size_t)i]) put(t);
    }
    return total;
}

lbm_status lbm_batch_create(lbm_batch** out, int lattice, int ncells, const int* dims, const double* tau,
                            const double* body_force, int precision, const int faces[6],
                            const double particle_gravity[3], double contact_gap, int body_force_on_particles)
{
    if (!out) return LBM_E_INVALID;
    *out = nullptr;
    if (ncells < 1 || !dims || !tau) return LBM_E_INVALID;
    lbm_batch* b = new lbm_batch();
    b->lattice = lattice;
    b->precision = precision;
    b->kt = table_for(precision);
    if (!b->kt) {
        delete b;
        return LBM_E_INVALID;
    }
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return LBM_E_CUDA;
    }
    for (int i = 0; i < ncells; ++i) {
        lbm_ctx* c = nullptr;
        lbm_status s = lbm_create(&c, lattice, dims[3 * (size_t)i], dims[3 * (size_t)i + 1], dims[3 * (size_t)i + 2],
                                  tau[i], body_force ? body_force + 3 * (size_t)i : nullptr);
        if (s == LBM_OK) {
            s = lbm_configure(c, precision, faces, particle_gravity, contact_gap, body_force_on_particles, b->stream);
            if (s != LBM_OK) lbm_destroy(c);
        }
        if (s != LBM_OK) {
            lbm_batch_destroy(b);
            return s;
        }
        b->cells.push_back(c);
    }
    b->tile_w.assign((size_t)ncells, 128);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_add_particles(lbm_batch* b, int cell, int n, const double* centers, const double* radii,
                                   const double* densities, const double* velocities, const double* omegas)
{
    if (!b) return LBM_E_INVALID;
    if (cell < 0 || cell >= (int)b->cells.size()) return bfail(b, LBM_E_INVALID, "no such cell");
    release_device(b);
    return from_cell(b, cell, lbm_add_particles(b->cells[(size_t)cell], n, centers, radii, densities, velocities,
                                                omegas, nullptr));
}

lbm_ctx* lbm_batch_cell(lbm_batch* b, int cell)
{
    if (!b || cell < 0 || cell >= (int)b->cells.size()) return nullptr;
    return b->cells[(size_t)cell];
}

lbm_status lbm_batch_set_tuning(lbm_batch* b, const int* tile_width, int order, int grid, int steps_per_graph)
{
    if (!b) return LBM_E_INVALID;
    const int nc = (int)b->cells.size();
    if (order < 0 || order > 2) return bfail(b, LBM_E_INVALID, "order must be 0, 1 or 2");
    if (grid < 0) return bfail(b, LBM_E_INVALID, "grid must be >= 0");
    if (steps_per_graph < 1 || steps_per_graph > 256) return bfail(b, LBM_E_INVALID, "steps_per_graph in 1..256");
    if (tile_width)
        for (int i = 0; i < nc; ++i)
            if (tile_width[i] != 32 && tile_width[i] != 64 && tile_width[i] != 128)
                return bfail(b, LBM_E_INVALID, "tile width must be 32, 64 or 128");
    BK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < nc; ++i) b->tile_w[(size_t)i] = tile_width ? tile_width[i] : 128;
    b->order = order;
    b->grid = grid;
    b->steps_per_graph = steps_per_graph;
    release_device(b);
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n)
{
    if (!b) return LBM_E_INVALID;
    if (n < 0) return bfail(b, LBM_E_INVALID, "negative step count");
    if (n == 0) return LBM_OK;
    drop_if_stale(b);
    BS(build(b));
    BS(same_parity(b));
    const int K = b->steps_per_graph;
    NvtxRange r("lbm_batch_step");
    while (n > 0) {
        const int cur = b->cells[0]->cur;
        if (K > 1 && n >= K) {
            BK(cudaGraphLaunch(b->gk[cur], b->stream));
            advance_cells(b, K);
            n -= K;
        } else {
            BK(cudaGraphLaunch(b->g1[cur], b->stream));
            advance_cells(b, 1);
            n -= 1;
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch* b)
{
    if (!b) return LBM_E_INVALID;
    BK(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < b->cells.size(); ++i) BS(from_cell(b, (int)i, lbm_synchronize(b->cells[i])));
    return LBM_OK;
}

lbm_status lbm_batch_profile_steps(lbm_batch* b, int n, double out_ms[3])
{
    if (!b || !out_ms || n < 1) return LBM_E_INVALID;
    drop_if_stale(b);
    BS(build(b));
    BS(same_parity(b));
    std::vector<cudaEvent_t> ev(3 * (size_t)n, nullptr);
    for (auto& e : ev) BK(cudaEventCreate(&e));
    for (int s = 0; s < n; ++s) {
        enqueue_batch_step(b, b->cells[0]->cur, &ev[3 * (size_t)s]);
        advance_cells(b, 1);
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(b->stream);
    double acc[3] = {0, 0, 0};
    for (int s = 0; s < n && le == cudaSuccess && se == cudaSuccess; ++s) {
        float x = 0, y = 0, z = 0;
        cudaEventElapsedTime(&x, ev[3 * (size_t)s], ev[3 * (size_t)s + 1]);
        cudaEventElapsedTime(&y, ev[3 * (size_t)s + 1], ev[3 * (size_t)s + 2]);
        cudaEventElapsedTime(&z, ev[3 * (size_t)s], ev[3 * (size_t)s + 2]);
        acc[0] += x;
        acc[1] += y;
        acc[2] += z;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (le != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(le));
    if (se != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("synchronize: ") + cudaGetErrorString(se));
    for (int k = 0; k < 3; ++k) out_ms[k] = acc[k] / n;
    return lbm_batch_synchronize(b);
}

lbm_status lbm_batch_get_info(lbm_batch* b, long long out[5])
{
    if (!b || !out) return LBM_E_INVALID;
    BS(build(b));
    long long sites = 0, np = 0;
    for (lbm_ctx* c : b->cells) {
        sites += (long long)c->g.N;
        np += c->np;
    }
    out[0] = (long long)b->cells.size();
    out[1] = sites;
    out[2] = np;
    out[3] = b->ntiles;
    out[4] = b->launches_per_step;
    return LBM_OK;
}

void* lbm_batch_stream(lbm_batch* b) { return b ? (void*)b->stream : nullptr; }

const char* lbm_batch_last_error(const lbm_batch* b)
{
    if (!b) return "null batch";
    return b->err.c_str();
}

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    release_device(b);
    for (lbm_ctx* c : b->cells) lbm_destroy(c);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
