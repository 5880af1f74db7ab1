// Host-side state of a simulation context and the helpers shared by the single-context
// entry points (api.cu) and the batched ensemble (batch.cu). Internal: not installed.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "lbmp.h"

namespace lbmp {
namespace host {
constexpr double LBM_PI = 3.14159265358979323846;
constexpr int PAIR_CAP = 16384;
constexpr size_t STAGING_BYTES = 64ull << 20;
}  // namespace host
}  // namespace lbmp

// One simulation: the lattice, its storage and particles, and the captured step graphs.
struct lbm_ctx {
    int lattice = 1, Q = 19, D = 3;
    lbmp::Geom g{};
    double tau = 0.6, F[3] = {0, 0, 0};
    int precision = LBM_FP32;
    int sweep_bx = -1;         // lbm_set_sweep_shape
    const lbmp::KernelTable* kt = nullptr;
    double grav[3] = {0, 0, 0};
    double uw[6][3] = {};      // tangential velocity of each wall face (host copy)
    bool moving_walls = false; // set once a face is given a velocity; never cleared
    lbmp::WallVel* wv = nullptr;     // device: [0] velocities of the pending streaming, [1] current
    double gap = 0.0;
    int bfp = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool allocated = false;
    bool stepped = false;

    void* f[2] = {nullptr, nullptr};  // in-place streaming: f[0] only
    bool inplace = false;      // lbm_set_streaming(LBM_STREAM_INPLACE); cur = 1 after a neighbour phase
    void* is_rho[2] = {nullptr, nullptr};  // in-place streaming: [N] compute type, IS-site densities
                               // (the sweep from parity c reads is_rho[c] and writes is_rho[1 - c])
    void* dens = nullptr;      // [N] compute type: site densities for the IS bookkeeping
    unsigned* tag = nullptr;
    unsigned* ismask = nullptr;
    void* bs_scratch = nullptr;
    int cur = 0;

    int np = 0;
    std::vector<lbmp::PConst> h_pc;
    std::vector<lbmp::PKern> h_pk;
    std::vector<lbmp::PKernF> h_pkf;
    std::vector<double> h_x;
    std::vector<double> h_q;   // orientations (w, x, y, z) when added: the identity
    std::vector<int> h_tmpl;
    lbmp::PKern* pk = nullptr;
    lbmp::PKernF* pkf = nullptr;
    lbmp::PKern* pk_prev = nullptr;
    lbmp::PKernF* pkf_prev = nullptr;
    lbmp::PConst* pc = nullptr;
    int* tmpl = nullptr;
    double *x = nullptr, *un = nullptr, *acc = nullptr, *force = nullptr;
    double* q = nullptr;       // [np][4] orientation quaternions (w, x, y, z)
    float4* xpf = nullptr;     // [np] predicted centres in FP32 and radii (contact pre-test)
    int* Kold = nullptr;
    lbmp::Counters* cnt = nullptr;
    int* status = nullptr;
    int* pending = nullptr;
    int* pending_prev = nullptr;
    lbmp::CellGrid cg{};
    int *cell_of = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_cursor = nullptr,
        *cell_items = nullptr;
    unsigned long long* pairs = nullptr;
    int *changed = nullptr, *restamp = nullptr, *restamp_flag = nullptr;

    double* staging = nullptr;
    void* pinned = nullptr;  // page-locked host staging for particle read-backs
    size_t pinned_bytes = 0;
    double* pout = nullptr;  // [15][np] packed particle state on the device, + the status word
    // asynchronous particle read-backs (lbm_get_particles_async): a ring of events
    static constexpr int RB_SLOTS = 8;
    cudaEvent_t rb_ev[RB_SLOTS] = {};
    long long rb_ticket[RB_SLOTS] = {};
    const double* rb_dst[RB_SLOTS] = {};
    bool rb_busy[RB_SLOTS] = {};
    long long rb_count = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int launches_per_step = 0;
    long long steps = 0;
    size_t dev_bytes = 0;            // bytes of the allocations below
    std::vector<void*> allocs;
    std::vector<size_t> alloc_bytes; // size of allocs[k]
    std::string err;
};

namespace lbmp {
namespace host {

// NVTX range for the duration of a scope: names the host-side enqueue of a step and of its
// kernel groups (sweep, particle phase) in a profiler's timeline. Header-only NVTX: without a
// tool attached the calls return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

inline lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

inline lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, LBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                       \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);       \
    } while (0)

template <typename T>
lbm_status dev_alloc(lbm_ctx* ctx, T** p, size_t bytes)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LBM_E_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " +
                                        cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    ctx->alloc_bytes.push_back(bytes);
    ctx->dev_bytes += bytes;
    *p = (T*)q;
    return LBM_OK;
}

#define CS(call)                                 \
    do {                                         \
        lbm_status s_ = (call);                  \
        if (s_ != LBM_OK) return s_;             \
    } while (0)

template <class A>
void wall_args(const lbm_ctx* ctx, A& a)
{
    a.moving_walls = ctx->moving_walls ? 1 : 0;
    a.uw = ctx->wv;
}

// Bytes of the per-site BS records: 6 doubles (FP64 storage) or one float4 per site (in
// bricks of 2 x 2 x 2 sites for FP32 storage, rec_brick_index).
inline size_t bs_record_bytes(const lbm_ctx* ctx)
{
    if (ctx->precision == LBM_FP64) return 6 * sizeof(double) * (size_t)ctx->g.N;
    if (ctx->precision == LBM_FP32) return sizeof(float4) * lbmp::rec_brick_count(ctx->g);
    return sizeof(float4) * (size_t)ctx->g.N;
}

const KernelTable* table_for(int precision);
lbm_status ensure_alloc(lbm_ctx* ctx);
lbm_status sync_status(lbm_ctx* ctx);
ParticleArgs particle_args(lbm_ctx* ctx);
MaskArgs mask_args(lbm_ctx* ctx, bool restamp_list);
PartView part_view(lbm_ctx* ctx);
SweepArgs sweep_args(lbm_ctx* ctx, int c);
ISFixArgs is_fix_args(lbm_ctx* ctx, int c);

}  // namespace host
}  // namespace lbmp
