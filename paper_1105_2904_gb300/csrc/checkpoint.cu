// Checkpoint and resume of a simulation context (lbm_checkpoint_* in include/lbmp.h).
//
// A checkpoint is the state at a step boundary: the distribution buffer the next sweep reads
// (in the storage format, IS sites carrying their density), the owner map and the IS-source
// masks, the particles' kinematic records, positions, orientations and last forces, the
// pending-imposition flag and the wall velocities; with in-place streaming also the layout
// parity and the IS-site densities the next sweep reads. Everything else a step uses is
// rebuilt inside the step. The constant part of the set-up (lattice, sizes,
// tau, forces, faces, particle constants and templates) is not stored: it is fingerprinted,
// and a checkpoint loads only into a context set up with the same calls.
#include <cstring>
#include <string>

#include "ctx.h"

using namespace lbmp;
using namespace lbmp::host;

namespace {

constexpr char kMagic[8] = {'L', 'B', 'M', 'P', 'C', 'K', 'P', '1'};
constexpr int kVersion = 5;

struct CkptHeader {
    char magic[8];
    int version;
    int lattice, nx, ny, nz, precision, Q, elem_bytes, np;
    int moving_walls;
    int inplace, parity;       // in-place streaming and its layout parity (ctx->cur)
    long long steps;
    unsigned long long fingerprint;
    unsigned long long bytes_total;
    double uw[6][3];
};

// FNV-1a over the values of the set-up (field by field: no struct padding enters the hash).
struct Fnv {
    unsigned long long h = 1469598103934665603ull;
    void bytes(const void* p, size_t n)
    {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
    template <class T> void val(const T& v) { bytes(&v, sizeof(T)); }
};

unsigned long long fingerprint(const lbm_ctx* ctx)
{
    Fnv f;
    f.val(ctx->lattice);
    f.val(ctx->g.nx);
    f.val(ctx->g.ny);
    f.val(ctx->g.nz);
    for (int k = 0; k < 3; ++k) f.val(ctx->g.wall[k]);
    f.val(ctx->g.eqface);  // no-slip and equilibrium faces both set wall[k]
    f.val(ctx->precision);
    f.val(ctx->inplace);
    f.val(ctx->tau);
    for (int k = 0; k < 3; ++k) f.val(ctx->F[k]);
    for (int k = 0; k < 3; ++k) f.val(ctx->grav[k]);
    f.val(ctx->gap);
    f.val(ctx->bfp);
    f.val(ctx->np);
    for (const PConst& c : ctx->h_pc) {
        for (int k = 0; k < 3; ++k) f.val(c.x0[k]);
        f.val(c.r);
        f.val(c.inv_m);
        f.val(c.inv_I);
        for (int k = 0; k < 3; ++k) f.val(c.ext[k]);
        for (int k = 0; k < 3; ++k) f.val(c.A[k]);
        f.val(c.tmpl_off);
        f.val(c.tmpl_n);
        f.val(c.n_bs);
        f.val(c.n_is);
    }
    if (!ctx->h_tmpl.empty()) f.bytes(ctx->h_tmpl.data(), sizeof(int) * ctx->h_tmpl.size());
    return f.h;
}

// The state's sections, in file order: device pointer and byte count.
struct Section {
    void* dev;
    size_t bytes;
};

std::vector<Section> sections(lbm_ctx* ctx)
{
    const size_t N = ctx->g.N;
    const size_t np = (size_t)ctx->np;
    std::vector<Section> s;
    s.push_back({ctx->f[ctx->inplace ? 0 : ctx->cur], (size_t)ctx->Q * N * (size_t)ctx->kt->elem_bytes});
    if (ctx->inplace) s.push_back({ctx->is_rho[ctx->cur], (size_t)ctx->kt->compute_bytes * N});
    if (np > 0) {
        s.push_back({ctx->tag, sizeof(unsigned) * N});
        s.push_back({ctx->ismask, sizeof(unsigned) * N});
        s.push_back({ctx->pk, sizeof(PKern) * np});
        s.push_back({ctx->pkf, sizeof(PKernF) * np});
        s.push_back({ctx->x, sizeof(double) * 3 * np});
        s.push_back({ctx->q, sizeof(double) * 4 * np});
        s.push_back({ctx->force, sizeof(double) * 6 * np});
    }
    s.push_back({ctx->pending, sizeof(int)});
    s.push_back({ctx->wv, 2 * sizeof(WallVel)});
    return s;
}

unsigned long long total_bytes(lbm_ctx* ctx)
{
    unsigned long long t = sizeof(CkptHeader);
    for (const Section& s : sections(ctx)) t += s.bytes;
    return t;
}

CkptHeader header_of(lbm_ctx* ctx)
{
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.lattice = ctx->lattice;
    h.nx = ctx->g.nx;
    h.ny = ctx->g.ny;
    h.nz = ctx->g.nz;
    h.precision = ctx->precision;
    h.Q = ctx->Q;
    h.elem_bytes = ctx->kt->elem_bytes;
    h.np = ctx->np;
    h.moving_walls = ctx->moving_walls ? 1 : 0;
    h.inplace = ctx->inplace ? 1 : 0;
    h.parity = ctx->cur;
    h.steps = ctx->steps;
    h.fingerprint = fingerprint(ctx);
    h.bytes_total = total_bytes(ctx);
    std::memcpy(h.uw, ctx->uw, sizeof(h.uw));
    return h;
}

}  // namespace

extern "C" {

lbm_status lbm_checkpoint_size(lbm_ctx* ctx, unsigned long long* bytes)
{
    if (!ctx || !bytes) return LBM_E_INVALID;
    CS(ensure_alloc(ctx));
    *bytes = total_bytes(ctx);
    return LBM_OK;
}

lbm_status lbm_checkpoint_save(lbm_ctx* ctx, void* buf, unsigned long long bytes)
{
    if (!ctx || !buf) return LBM_E_INVALID;
    CS(ensure_alloc(ctx));
    CS(sync_status(ctx));
    const CkptHeader h = header_of(ctx);
    if (bytes < h.bytes_total)
        return fail(ctx, LBM_E_INVALID, "checkpoint buffer holds " + std::to_string(bytes) + " bytes, " +
                                            std::to_string(h.bytes_total) + " needed");
    char* p = (char*)buf;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    for (const Section& s : sections(ctx)) {
        CK(cudaMemcpy(p, s.dev, s.bytes, cudaMemcpyDeviceToHost));
        p += s.bytes;
    }
    return LBM_OK;
}

lbm_status lbm_checkpoint_load(lbm_ctx* ctx, const void* buf, unsigned long long bytes)
{
    if (!ctx || !buf) return LBM_E_INVALID;
    CS(ensure_alloc(ctx));
    CS(sync_status(ctx));
    if (bytes < sizeof(CkptHeader)) return fail(ctx, LBM_E_INVALID, "checkpoint: truncated header");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const CkptHeader mine = header_of(ctx);
    if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != kVersion)
        return fail(ctx, LBM_E_INVALID, "checkpoint: not a checkpoint of this library version");
    if (h.lattice != mine.lattice || h.nx != mine.nx || h.ny != mine.ny || h.nz != mine.nz ||
        h.precision != mine.precision || h.Q != mine.Q || h.elem_bytes != mine.elem_bytes || h.np != mine.np ||
        h.inplace != mine.inplace)
        return fail(ctx, LBM_E_INVALID, "checkpoint: lattice, sizes, precision, streaming or particle count differ");
    if (h.parity != 0 && h.parity != 1) return fail(ctx, LBM_E_INVALID, "checkpoint: bad layout parity");
    if (h.fingerprint != mine.fingerprint)
        return fail(ctx, LBM_E_INVALID, "checkpoint: the context's set-up (tau, forces, faces, particles) differs");
    if (h.bytes_total != mine.bytes_total || bytes < h.bytes_total)
        return fail(ctx, LBM_E_INVALID, "checkpoint: truncated or inconsistent size");
    // in-place streaming: the layout (and the density array the next sweep reads) follow the
    // saved parity
    if (ctx->inplace) ctx->cur = h.parity;
    const char* p = (const char*)buf + sizeof(h);
    for (const Section& s : sections(ctx)) {
        CK(cudaMemcpy(s.dev, p, s.bytes, cudaMemcpyHostToDevice));
        p += s.bytes;
    }
    // a copy from pageable memory may still be in flight when cudaMemcpy returns, and the
    // library's stream need not be ordered with the copies' stream
    CK(cudaDeviceSynchronize());
    // the BS records of the context's own past steps may not match the loaded owner map: clear
    // them (the next sweep rewrites the record of every BS site)
    if (ctx->np > 0) CK(cudaMemset(ctx->bs_scratch, 0, bs_record_bytes(ctx)));
    ctx->steps = h.steps;
    ctx->stepped = ctx->stepped || h.steps > 0;
    std::memcpy(ctx->uw, h.uw, sizeof(h.uw));
    ctx->moving_walls = h.moving_walls != 0;
    // the captured step graphs depend on the moving-wall flag: capture them again
    for (auto& ge : ctx->gexec)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
    return LBM_OK;
}

}  // extern "C"
