// C ABI of the GB300 lattice-Boltzmann + immersed-boundary library (see
// include/lbibm.h).  Host-side responsibilities: argument validation, the
// membrane topology (node rings, wing vertices, rest lengths / angles / areas
// in FP64), device memory, and the order of the four kernels of one cycle of
// Sec. 2.2 (area/volume sums -> forces + spreading -> stream-collide ->
// interpolation + advance), launched directly or replayed as CUDA graphs.
#include "lbibm.h"
#include "lbibm_internal.cuh"

#include <algorithm>
#include <thread>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

using namespace lbibm;

namespace {

constexpr int CHUNK_TRIS = 128;     // triangles per block of the area/volume reduction (one per thread;
                                    // measured on GB300: 256 -> 128 took the element pass 18.2 -> 16.5 us, 64 slower)
constexpr int MAX_VALENCE = 64;

struct ChannelHost {
    lb_params p;
    ChannelDev d;
    int n_blocks = 0;
    std::vector<float> spheres;   // bead spheres of lb_set_obstacles (cx, cy, cz, r)
};

struct MeshHost {
    int ch = 0;
    int node0 = 0, n = 0;
    int tri0 = 0, nt = 0;
    int cell = 0;
    double S0 = 0, V0 = 0;
};

// The connectivity-derived tables of a mesh, in its own node, triangle and
// edge numbering: edges (a, b, c, d) with a < b in triangle order, and per
// node its ring slots (3 t + position of the node in t, 4 e + role as a / b,
// 4 e' + role as c / d, t).  They depend on the triangles only, so meshes
// that share a template (every red cell of a scene) are checked and indexed
// once per context.
struct MeshConn {
    int n = 0, nt = 0;
    std::vector<int32_t> tris;   // the key
    std::vector<int4> edges;
    std::vector<int4> slots;
    std::vector<int> ring_off, valence;
};

// A mesh added to the context: its connectivity and where its nodes,
// triangles, edges and ring slots go in the context's tables.
struct PendingMesh {
    const MeshConn* conn;
    int node0, tri0, e0, slot0, cell, ch;
    float ks, kb;
};

struct EventPair {
    cudaEvent_t a, b;
    int cls;
};

}  // namespace

struct lb_ctx {
    std::string err = "no error";
    bool poisoned = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lb_storage storage = LB_F32;
    std::vector<ChannelHost> ch;
    int cur = 0;
    long long Ntot = 0;
    long long plane = 0;   // population plane stride (>= Ntot)
    int total_blocks = 0;
    int n_groups = 0;        // row groups of the staged stream-collide variant
    int sm_count = 152;
    // lattice
    void* h[2] = {nullptr, nullptr};
    uint32_t* mask = nullptr;
    uint8_t* slow = nullptr;
    uint32_t* links = nullptr;   // bounce-back link mask per node
    float4* g[2] = {nullptr, nullptr};
    uint8_t* fl[2] = {nullptr, nullptr};
    float4* u = nullptr;
    ChannelDev* d_ch = nullptr;
    double* diag_partials = nullptr;
    double* diag_out = nullptr;
    int diag_blocks = 0;
    // immersed boundary, host staging
    std::vector<Q4> hq0, hq;
    std::vector<int4> hinfo;
    std::vector<int4> hslots;      // ring CSR: element outputs of each ring slot
    std::vector<int4> hedges;      // (a, b, c, d)
    std::vector<float4> hedge_rest;  // (L0, theta0, ks, kb)
    std::vector<int4> htris;
    std::vector<float> htriS0;
    std::vector<int4> hchunks;
    std::vector<CellDev> hcells;
    std::vector<double> hrest;     // rest positions (x, y, z per node)
    std::vector<std::unique_ptr<MeshConn>> conn_cache;   // connectivity per distinct triangle list
    std::vector<PendingMesh> pending_meshes;             // meshes whose tables the commit writes
    int n_tris_staged = 0, n_edges_staged = 0, n_slots_staged = 0;
    float* fields_buf = nullptr;   // device scratch of lb_get_fields (4 floats per node of the largest channel)
    std::vector<MeshHost> meshes;
    std::vector<std::vector<int>> ch_meshes;
    bool committed = false;
    // immersed boundary, device
    int M = 0, C = 0, T = 0, NCH = 0, K = 0, E = 0;
    Q4* q[2] = {nullptr, nullptr};
    Q4* q0 = nullptr;
    float4* F = nullptr;
    Q4* hq_pinned = nullptr;       // page-locked staging of positions for readback [M]
    double* d_xyz = nullptr;       // [3M] device staging of asynchronous readbacks
    cudaEvent_t rb_ev[2] = {nullptr, nullptr};
    int4* info = nullptr;
    int4* slots = nullptr;
    int4* edges = nullptr;
    float4* edge_rest = nullptr;
    float4 *eS = nullptr, *eB = nullptr, *tA = nullptr, *tN = nullptr;
    int4* tris = nullptr;
    float* triS0 = nullptr;
    int4* chunks = nullptr;
    longlong2* partials = nullptr;
    unsigned* counters = nullptr;
    double2* cell_sums = nullptr;
    float2* cell_rel = nullptr;
    CellDev* d_cells = nullptr;
    // stream-collide variant and its grid
    K3Config k3 = {1, 256};
    // stepping
    long long step = 0;
    bool started = false;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec_blk[2] = {nullptr, nullptr};   // GRAPH_BLOCK consecutive cycles from parity p
    // overlapped schedule: the immersed-boundary chain on a second stream of
    // higher priority, concurrent with the bulk of the stream-collide
    bool overlap = false;          // chosen by the caller (lb_set_schedule)
    bool pdl = true;               // sequential cycle: programmatic dependent launches
    bool dvalid = false;           // the stencil set of the next step is current
    cudaStream_t ib_stream = nullptr;
    cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork2[2] = {nullptr, nullptr}, ev_join2[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec_ov[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [parity][leading interpolation]
    uint8_t* dmap[2] = {nullptr, nullptr};
    int* dlist[2] = {nullptr, nullptr};
    int* dcount = nullptr;         // [2]
    int* sched_err = nullptr;      // [2]: overlapped-schedule check, TMA-variant waits
    CUtensorMap tma_maps[2];       // TMA-staged stream-collide: h[0], h[1]
    bool tma_ready = false;
    int list_blocks = 0;
    // collisions (soft sphere): off while rep_k == 0
    float rep_k = 0.f, rep_dc = 0.f;
    double ib_m = 0.0, ib_gamma = 0.0;   // IB points with mass (ib_m > 0) and drag
    bool deterministic = false;          // fixed-point spreading, run-to-run identical results
    unsigned long long* gfix = nullptr;  // [3][Ntot] its sums
    float4* W = nullptr;                 // [M] their velocities
    int rep_cap = 0, rep_nb = 0;
    float4 *rep_R = nullptr, *rep_bounds = nullptr;
    int2* rep_pairs = nullptr;
    int *rep_count = nullptr, *rep_near = nullptr, *rep_near_count = nullptr, *rep_err = nullptr, *rep_bead_ch = nullptr;
    Q4* rep_bead_q = nullptr;
    float* rep_bead_r = nullptr;
    // differentiable variant
    float* phi = nullptr;          // bead solid fraction per node (null: off)
    float alpha = 0.f, delta = 0.f;
    std::vector<double> beads;     // cx, cy, cz, r per bead (host)
    float* d_beads = nullptr;
    // adjoint workspace (allocated by the first lb_adjoint of a given size)
    struct AdjWork {
        int K = 0, n_ck = 0;
        float *ck_h = nullptr, *seg_h = nullptr, *fin_h = nullptr, *lam[2] = {nullptr, nullptr}, *Lphi = nullptr;
        Q4 *ck_q = nullptr, *seg_q = nullptr, *fin_q = nullptr;
        float4 *seg_F = nullptr, *seg_g = nullptr, *seg_u = nullptr, *lam_u = nullptr, *lam_g = nullptr;
        float4 *lamX[2] = {nullptr, nullptr}, *lamF = nullptr, *tri_dS = nullptr, *tri_n = nullptr;
        float4 *fin_u = nullptr, *fin_F = nullptr;
        uint8_t *seg_fl = nullptr, *fl_zero = nullptr;
        // captured segment sweeps: forward (key: len, start parity) and
        // reverse (key: len, population / position adjoint buffer parity)
        std::map<std::pair<int, int>, cudaGraphExec_t> g_fwd, g_bwd;
        float2* seg_rel = nullptr;
        double *lam_c = nullptr, *grad = nullptr;
    } adj;
    int bulk_res = 10;             // resident bulk blocks per SM (128 threads)
    int pf_nodes = 0;              // stream-collide L2 prefetch distance (lattice nodes, 0 = off)
    long long smem_per_sm = 0;
    // timing
    int timing = 0;          // bit k: record events around kernel class k (no graph)
    double ms[4] = {0, 0, 0, 0};
    long long launches[4] = {0, 0, 0, 0};
    std::vector<EventPair> pending;
    std::vector<cudaEvent_t> free_events;
    std::vector<void*> allocations;
    // debug guard zones (lb_set_guard_zones): bytes of pattern before and
    // after every allocation of this context, and the guarded allocations
    size_t guard = 0;
    struct Guarded {
        char* base;
        size_t bytes, guard;
    };
    std::vector<Guarded> guarded;
};

namespace lbibm {
// Message of the last failed call of this thread that has no context to hold
// it (lb_create, lb_create_batch, ibm_check_mesh, bead_forces, bead_relax).
thread_local std::string context_free_err = "no error";
lb_status context_free_error(lb_status s, const char* msg) {
    context_free_err = msg;
    return s;
}
}  // namespace lbibm

namespace {

lb_status fail(lb_ctx* c, lb_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* where) {
    if (c) {
        c->poisoned = true;
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
}

#define LB_CUDA(expr)                                            \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

#define LB_GUARD(ctx)                                                         \
    do {                                                                      \
        if (!(ctx)) return LB_ERR_ARG;                                        \
        if ((ctx)->poisoned) return LB_ERR_CUDA;                              \
    } while (0)

// Guard zones of the contexts created from now on (lb_set_guard_zones).
std::atomic<size_t> g_guard_bytes{0};
constexpr unsigned char GUARD_PATTERN = 0xA5;

// Device allocation owned by the context.  With guard zones, `guard` bytes of
// GUARD_PATTERN sit before and after the returned block (which keeps the
// 256-byte alignment of cudaMalloc: guards are multiples of 256).
template <class T>
cudaError_t dalloc(lb_ctx* ctx, T** p, size_t count) {
    void* v = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    const size_t gz = ctx->guard;
    cudaError_t e = cudaMalloc(&v, bytes + 2 * gz);
    if (e == cudaSuccess && gz) {
        e = cudaMemset(v, GUARD_PATTERN, gz);
        if (e == cudaSuccess) e = cudaMemset((char*)v + gz + bytes, GUARD_PATTERN, gz);
        if (e != cudaSuccess) {
            cudaFree(v);
            v = nullptr;
        }
    }
    if (e == cudaSuccess) {
        *p = (T*)((char*)v + gz);
        ctx->allocations.push_back(v);
        if (gz) ctx->guarded.push_back({(char*)v, bytes, gz});
    } else {
        *p = nullptr;
    }
    return e;
}

void dfree(lb_ctx* ctx, void* p) {
    if (!p) return;
    void* base = (char*)p - ctx->guard;
    auto it = std::find(ctx->allocations.begin(), ctx->allocations.end(), base);
    if (it != ctx->allocations.end()) ctx->allocations.erase(it);
    ctx->guarded.erase(std::remove_if(ctx->guarded.begin(), ctx->guarded.end(),
                                      [&](const lb_ctx::Guarded& g) { return g.base == base; }),
                       ctx->guarded.end());
    cudaFree(base);
}

// Bytes of [p, p + n) that differ from the guard pattern, added to *count.
__global__ void k_guard_count(const unsigned char* __restrict__ p, size_t n, unsigned long long* count) {
    unsigned long long c = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += p[i] != GUARD_PATTERN;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

size_t pop_bytes(lb_storage s) { return s == LB_F32 ? 4 : 2; }

LatticeArgs lattice_args(const lb_ctx* ctx, int par) {
    LatticeArgs a;
    std::memset(&a, 0, sizeof(a));
    for (size_t k = 0; k < ctx->ch.size() && k < (size_t)MAXCH_P; ++k) a.chp[k] = ctx->ch[k].d;
    a.ch = ctx->d_ch;
    a.n_ch = (int)ctx->ch.size();
    a.storage = (int)ctx->storage;
    a.par = par;
    a.has_last = ctx->step > 0;
    a.h0 = ctx->h[0];
    a.h1 = ctx->h[1];
    a.Ntot = ctx->plane;
    a.mask = ctx->mask;
    a.slow = ctx->slow;
    a.links = ctx->links;
    a.g0 = ctx->g[0];
    a.g1 = ctx->g[1];
    a.fl0 = ctx->fl[0];
    a.fl1 = ctx->fl[1];
    a.u = ctx->u;
    a.n_groups = ctx->n_groups;
    a.phi = ctx->phi;
    a.alpha = ctx->alpha;
    a.dmap = ctx->dmap[par];
    a.dlist = ctx->dlist[par];
    a.dcount = ctx->dcount ? ctx->dcount + par : nullptr;
    a.tma_err = ctx->sched_err ? ctx->sched_err + 1 : nullptr;
    a.pf_nodes = ctx->pf_nodes;
    return a;
}

// the stream-collide launch of the context's variant
cudaError_t k3_launch(const lb_ctx* ctx, const LatticeArgs& la, K3Config c, cudaStream_t s) {
    if (c.npt == -2) {
        if (!ctx->tma_ready) return cudaErrorNotSupported;
        return launch_stream_collide_tma(la, c.bs, ctx->tma_maps, ctx->total_blocks, s);
    }
    return launch_stream_collide(la, c, ctx->total_blocks, s);
}

IbmArgs ibm_args(const lb_ctx* ctx, int par, bool overlapped = false) {
    IbmArgs a;
    std::memset(&a, 0, sizeof(a));
    for (size_t k = 0; k < ctx->ch.size() && k < (size_t)MAXCH_P; ++k) a.chp[k] = ctx->ch[k].d;
    a.n_nodes = ctx->M;
    a.n_cells = ctx->C;
    a.par = par;
    a.n_ch = (int)ctx->ch.size();
    a.ch = ctx->d_ch;
    a.cells = ctx->d_cells;
    a.info = ctx->info;
    a.qa = ctx->q[0];
    a.qb = ctx->q[1];
    a.q0 = ctx->q0;
    a.slots = ctx->slots;
    a.edges = ctx->edges;
    a.edge_rest = ctx->edge_rest;
    a.n_edges = ctx->E;
    a.eS = ctx->eS;
    a.eB = ctx->eB;
    a.tA = ctx->tA;
    a.tN = ctx->tN;
    a.F = ctx->F;
    a.tris = ctx->tris;
    a.tri_S0 = ctx->triS0;
    a.chunks = ctx->chunks;
    a.n_chunks = ctx->NCH;
    a.partials = ctx->partials;
    a.counters = ctx->counters;
    a.cell_sums = ctx->cell_sums;
    a.cell_rel = ctx->cell_rel;
    a.mask = ctx->mask;
    a.g0 = ctx->g[0];
    a.g1 = ctx->g[1];
    a.fl0 = ctx->fl[0];
    a.fl1 = ctx->fl[1];
    a.u = ctx->u;
    a.R = ctx->rep_k > 0.f ? ctx->rep_R : nullptr;
    if (ctx->deterministic && ctx->gfix) {
        a.gfix = ctx->gfix;
        a.gfix_stride = ctx->Ntot;
    }
    if (ctx->ib_m > 0.0 && ctx->W) {
        // kick / exact drag drift constants: a = gamma / m, p1 = (1 - e^-a) / a, E = e^-a
        const double m = ctx->ib_m, gam = ctx->ib_gamma, aa = gam / m;
        const double p1 = aa < 1e-4 ? 1.0 - aa * (0.5 - aa * (1.0 / 6.0 - aa / 24.0)) : -std::expm1(-aa) / aa;
        a.W = ctx->W;
        a.ib_inv_m = (float)(1.0 / m);
        a.ib_gp1 = (float)(gam * p1);
        a.ib_p1 = (float)p1;
        a.ib_E = (float)std::exp(-aa);
    }
    a.dmark = ctx->dmap[1 - par];
    a.dcur = overlapped ? ctx->dmap[par] : nullptr;
    a.sched_err = ctx->sched_err;
    return a;
}

lb_status validate_params(const lb_params& p, std::string& why) {
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) { why = "lattice dimensions must be >= 1"; return LB_ERR_ARG; }
    const long long n = (long long)p.nx * p.ny * p.nz;
    if (n > 2147483647LL) { why = "nx*ny*nz must be < 2^31"; return LB_ERR_ARG; }
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) { why = "tau must be > 1/2"; return LB_ERR_ARG; }
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p.body_force[d])) { why = "body force must be finite"; return LB_ERR_ARG; }
    for (int w = 0; w < 2; ++w)
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(p.wall_velocity[w][d])) { why = "wall velocities must be finite"; return LB_ERR_ARG; }
    if (p.storage != LB_F32 && p.storage != LB_F16_SHIFTED && p.storage != LB_BF16_SHIFTED) {
        why = "unknown storage";
        return LB_ERR_ARG;
    }
    for (int k = 0; k < 4; ++k)
        if (p.reserved[k]) { why = "reserved fields must be zero"; return LB_ERR_ARG; }
    return LB_OK;
}

// ---- timing helpers ----
cudaEvent_t take_event(lb_ctx* ctx) {
    if (!ctx->free_events.empty()) {
        cudaEvent_t e = ctx->free_events.back();
        ctx->free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// ---- one cycle (Sec. 2.2) ----
lb_status enqueue_step(lb_ctx* ctx, int par) {
    LatticeArgs la = lattice_args(ctx, par);
    IbmArgs ia = ibm_args(ctx, par);
    // each kernel of the cycle is scheduled during its predecessor's last wave
    // and waits for it before touching what it wrote (not under per-kernel
    // timing, whose events separate the launches).  The stream-collide reads
    // the previous cycle's populations before its wait, so it is a
    // programmatic dependent only when the spreading kernel precedes it.
    ia.pdl = ctx->pdl && ctx->timing == 0;
    la.pdl = ia.pdl && ctx->M > 0;
    const bool ibm = ctx->M > 0;
    if (ibm && ctx->rep_k > 0.f) {
        // collisions (Sec. 2.4), added to the membrane forces in the spreading kernel
        RepArgs ra;
        std::memset(&ra, 0, sizeof(ra));
        ra.k = ctx->rep_k;
        ra.dc = ctx->rep_dc;
        ra.n_cells = ctx->C;
        ra.n_nodes = ctx->M;
        ra.n_beads = ctx->rep_nb;
        ra.pair_cap = ctx->rep_cap;
        ra.q = ctx->q[par];
        ra.cells = ctx->d_cells;
        ra.info = ctx->info;
        ra.ch = ctx->d_ch;
        ra.bounds = ctx->rep_bounds;
        ra.pairs = ctx->rep_pairs;
        ra.pair_count = ctx->rep_count;
        ra.near = ctx->rep_near;
        ra.near_count = ctx->rep_near_count;
        ra.bead_q = ctx->rep_bead_q;
        ra.bead_r = ctx->rep_bead_r;
        ra.bead_ch = ctx->rep_bead_ch;
        ra.R = ctx->rep_R;
        ra.err = ctx->rep_err;
        for (size_t k = 0; k < ctx->ch.size() && k < (size_t)MAXCH_P; ++k) ra.chp[k] = ctx->ch[k].d;
        LB_CUDA(cudaMemsetAsync(ctx->rep_R, 0, sizeof(float4) * ctx->M, ctx->stream));
        LB_CUDA(cudaMemsetAsync(ctx->rep_count, 0, sizeof(int), ctx->stream));
        LB_CUDA(cudaMemsetAsync(ctx->rep_near_count, 0, sizeof(int) * ctx->C, ctx->stream));
        cudaError_t e = launch_repulsion(ra, ctx->sm_count, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
        ctx->launches[1] += 4;
    }
    for (int k = 0; k < 4; ++k) {
        if (!ibm && k != 2) continue;
        if (k == 3 && ctx->W) continue;   // points with mass move in the spreading kernel
        EventPair ep{};
        const bool timed = (ctx->timing >> k) & 1;
        ctx->launches[k] += (k == 1 && ctx->deterministic) ? 2 : 1;   // + the fixed-point conversion
        if (timed) {
            ep.a = take_event(ctx);
            ep.b = take_event(ctx);
            ep.cls = k;
            LB_CUDA(cudaEventRecord(ep.a, ctx->stream));
        }
        cudaError_t e = cudaSuccess;
        switch (k) {
            case 0: e = launch_elements(ia, ctx->stream); break;
            case 1:
                e = launch_forces_spread(ia, ctx->stream);
                if (e == cudaSuccess && ia.gfix) e = launch_gfix_to_g(ia, ctx->stream);
                break;
            case 2: e = k3_launch(ctx, la, ctx->k3, ctx->stream); break;
            case 3: e = launch_interp_advance(ia, ctx->stream); break;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
        if (timed) {
            LB_CUDA(cudaEventRecord(ep.b, ctx->stream));
            ctx->pending.push_back(ep);
        }
    }
    return LB_OK;
}

// Cycles per block graph: within a block every kernel, the first of each
// cycle included, is a programmatic dependent of the one before it.
constexpr int GRAPH_BLOCK = 8;

lb_status build_graphs(lb_ctx* ctx) {
    for (int blk = 0; blk < 2; ++blk)
        for (int par = 0; par < 2; ++par) {
            cudaGraphExec_t& ge = blk ? ctx->gexec_blk[par] : ctx->gexec[par];
            if (ge) continue;
            cudaGraph_t g = nullptr;
            long long saved[4];
            std::copy(ctx->launches, ctx->launches + 4, saved);   // capture launches nothing
            LB_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            lb_status s = LB_OK;
            for (int k = 0; k < (blk ? GRAPH_BLOCK : 1) && s == LB_OK; ++k) s = enqueue_step(ctx, (par + k) & 1);
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            std::copy(saved, saved + 4, ctx->launches);
            if (s != LB_OK) return s;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
    return LB_OK;
}

// One cycle in the overlapped schedule.  Only the 32-node groups of the
// stencil set D (the groups any IB point can reach within one step, computed
// during the previous step) depend on this step's IB forces, so
//   ib stream:   [interpolation + advance of the previous step], elements,
//                forces + spreading (which also marks the next step's D),
//                compaction of the next D into a list
//   main stream: stream-collide of every group outside D
// run concurrently; after the join the groups of D are updated.  The result is
// the same as the sequential cycle: D contains every group that receives force
// or is interpolated, and the spreading kernel counts any target outside D.
// Unused dynamic shared memory per bulk block that caps the bulk at
// bulk_res resident 128-thread blocks per SM, keeping 8 KB for the blocks of
// the immersed-boundary kernels (0 when registers cap it first).
size_t bulk_smem(const lb_ctx* ctx) {
    const int res = std::max(1, ctx->bulk_res * 128 / ctx->k3.bs);
    const long long per_block = (ctx->smem_per_sm - 8192) / res - 1024;
    return per_block > 0 ? (size_t)per_block : 0;
}

size_t bulk_smem_max(const lb_ctx* ctx) {
    const long long per_block = (ctx->smem_per_sm - 8192) - 1024;
    return per_block > 0 ? (size_t)per_block : 0;
}

lb_status enqueue_step_overlap(lb_ctx* ctx, int par, bool lead_interp) {
    const LatticeArgs la = lattice_args(ctx, par);
    const IbmArgs ia = ibm_args(ctx, par, true);
    const long long NG = ctx->Ntot / GROUP;
    cudaStream_t m = ctx->stream, ib = ctx->ib_stream;
    LB_CUDA(cudaEventRecord(ctx->ev_fork[par], m));
    LB_CUDA(cudaStreamWaitEvent(ib, ctx->ev_fork[par], 0));
    LB_CUDA(cudaMemsetAsync(ctx->dmap[1 - par], 0, (size_t)NG, ib));
    LB_CUDA(cudaMemsetAsync(ctx->dcount + (1 - par), 0, sizeof(int), ib));
    cudaError_t e = cudaSuccess;
    if (lead_interp && e == cudaSuccess) e = launch_interp_advance(ibm_args(ctx, 1 - par), ib);
    if (e == cudaSuccess) e = launch_elements(ia, ib);
    if (e == cudaSuccess) e = launch_forces_spread(ia, ib);
    if (e == cudaSuccess) e = launch_compact_groups(ctx->dmap[1 - par], (int)NG, ctx->dlist[1 - par], ctx->dcount + (1 - par), ib);
    if (e == cudaSuccess) e = launch_stream_collide_split(la, ctx->k3.bs, 1, ctx->total_blocks, bulk_smem(ctx), m);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    LB_CUDA(cudaEventRecord(ctx->ev_join[par], ib));
    LB_CUDA(cudaStreamWaitEvent(m, ctx->ev_join[par], 0));
    // stencil groups: one warp per list entry on the main stream; entries
    // beyond that grid (none on the workloads here) by a looping grid on the
    // second stream, concurrently
    const int covered = ctx->list_blocks * ctx->k3.bs / 32;
    LB_CUDA(cudaEventRecord(ctx->ev_fork2[par], m));
    LB_CUDA(cudaStreamWaitEvent(ib, ctx->ev_fork2[par], 0));
    e = launch_stream_collide_split(la, ctx->k3.bs, 3, ctx->sm_count, (size_t)covered, ib);
    if (e == cudaSuccess) e = launch_stream_collide_split(la, ctx->k3.bs, 2, ctx->list_blocks, 0, m);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    LB_CUDA(cudaEventRecord(ctx->ev_join2[par], ib));
    LB_CUDA(cudaStreamWaitEvent(m, ctx->ev_join2[par], 0));
    return LB_OK;
}

bool use_overlap(const lb_ctx* ctx) {
    const long long m = ctx->committed ? ctx->M : (long long)ctx->hq0.size();
    return ctx->overlap && m > 0 && ctx->phi == nullptr && ctx->rep_k == 0.f && ctx->ib_m == 0.0 && !ctx->deterministic &&
           ctx->k3.npt == 1 &&
           ctx->timing == 0 && ctx->ib_stream != nullptr;
}

lb_status build_graphs_overlap(lb_ctx* ctx) {
    for (int par = 0; par < 2; ++par)
        for (int lead = 0; lead < 2; ++lead) {
            if (ctx->gexec_ov[par][lead]) continue;
            cudaGraph_t g = nullptr;
            LB_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            lb_status s = enqueue_step_overlap(ctx, par, lead != 0);
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            if (s != LB_OK) return s;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
            // every kernel but the bulk stream-collide at the highest priority, so
            // that the immersed-boundary chain takes SM slots as bulk blocks retire
            int lo = 0, hi = 0;
            cudaDeviceGetStreamPriorityRange(&lo, &hi);
            const void* bulk = stream_collide_bulk_func((int)ctx->storage, ctx->k3.bs);
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
                cudaKernelNodeParams kp;
                if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
                cudaLaunchAttributeValue v;
                std::memset(&v, 0, sizeof(v));
                v.priority = kp.func == bulk ? lo : hi;
                cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v);
            }
            cudaGetLastError();
            // node priorities only take effect with this flag
            e = cudaGraphInstantiateWithFlags(&ctx->gexec_ov[par][lead], g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
    return LB_OK;
}

// Stencil set of the coming step from the current positions (after setup,
// after positions or a checkpoint were loaded, or after sequential steps).
lb_status prepare_stencil_set(lb_ctx* ctx) {
    const int par = (int)(ctx->step & 1);
    const long long NG = ctx->Ntot / GROUP;
    LB_CUDA(cudaMemsetAsync(ctx->dmap[par], 0, (size_t)NG, ctx->stream));
    LB_CUDA(cudaMemsetAsync(ctx->dcount + par, 0, sizeof(int), ctx->stream));
    LB_CUDA(launch_mark_stencils(ibm_args(ctx, par), ctx->dmap[par], ctx->stream));
    LB_CUDA(launch_compact_groups(ctx->dmap[par], (int)NG, ctx->dlist[par], ctx->dcount + par, ctx->stream));
    ctx->launches[1] += 2;
    ctx->dvalid = true;
    return LB_OK;
}

void drop_graphs(lb_ctx* ctx) {
    for (int par = 0; par < 2; ++par) {
        if (ctx->gexec[par]) {
            cudaGraphExecDestroy(ctx->gexec[par]);
            ctx->gexec[par] = nullptr;
        }
        if (ctx->gexec_blk[par]) {
            cudaGraphExecDestroy(ctx->gexec_blk[par]);
            ctx->gexec_blk[par] = nullptr;
        }
        for (int lead = 0; lead < 2; ++lead)
            if (ctx->gexec_ov[par][lead]) {
                cudaGraphExecDestroy(ctx->gexec_ov[par][lead]);
                ctx->gexec_ov[par][lead] = nullptr;
            }
    }
}

// ---- membrane topology on the host (FP64) ----
double dihedral_host(const double* xa, const double* xb, const double* xc, const double* xd) {
    double e[3], ac[3], ba[3], bd[3], n1[3], n2[3], m[3];
    for (int k = 0; k < 3; ++k) {
        e[k] = xb[k] - xa[k];
        ac[k] = xc[k] - xa[k];
        ba[k] = xa[k] - xb[k];
        bd[k] = xd[k] - xb[k];
    }
    auto cr = [](const double* a, const double* b, double* o) {
        o[0] = a[1] * b[2] - a[2] * b[1];
        o[1] = a[2] * b[0] - a[0] * b[2];
        o[2] = a[0] * b[1] - a[1] * b[0];
    };
    cr(e, ac, n1);
    cr(ba, bd, n2);
    cr(n1, n2, m);
    const double le = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    return std::atan2((m[0] * e[0] + m[1] * e[1] + m[2] * e[2]) / le, n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
}

double tri_area_host(const double* a, const double* b, const double* c) {
    const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    return 0.5 * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
}

long long to_fixed(double x) { return std::llround(x * FIX_SCALE); }

// Extra nodes between population planes.  Planes of exactly 2^k nodes put all
// 38 read / write streams of the stream-collide kernel at identical large
// power-of-two offsets; a pad (a multiple of 64 nodes) staggers them across
// DRAM channels.
constexpr long long PLANE_PAD = 1088;
long long plane_pad() { return PLANE_PAD; }

// Grid of the stream-collide kernel for a (nodes per thread, block size)
// variant: channel k's blocks start at blk0 and cover its padded node range.
bool k3_config_valid(const lb_ctx* ctx, K3Config c) {
    if (!k3_config_supported((int)ctx->storage, c)) return false;
    if (ctx->phi && c.npt != 1) return false;   // the differentiable variant runs one node per thread
    if (c.npt == -2) return ctx->ch.size() == 1 && tma_variant_ok(ctx->ch[0].d, (int)ctx->storage, 1, c.bs);
    // the 16-bit quad variant addresses the populations with 32-bit element offsets
    if (c.npt == 4 && ctx->storage != LB_F32 && (long long)Q * ctx->plane >= (1LL << 32)) return false;
    for (const auto& ch : ctx->ch) {
        if (c.npt == 0) {
            if (staged_rows(ch.d.nx, (int)pop_bytes(ctx->storage)) == 0) return false;
        } else if (c.npt > 0 && ch.d.nx % c.npt != 0) {
            return false;
        }
    }
    return true;
}

// Default variant: one node per thread (FP32); for 16-bit storage four nodes
// per thread in blocks of 64 where every nx is a multiple of 4 (measured on
// GB300, FP16: 55.3 vs 57.5 us on 256x128x64, 357 vs 396 us on 512x256x128).
K3Config default_k3_config(const lb_ctx* ctx) {
    if (ctx->storage != LB_F32 && k3_config_valid(ctx, K3Config{4, 64})) return K3Config{4, 64};
    const K3Config pref[] = {{1, 128}};
    for (const K3Config& c : pref)
        if (k3_config_valid(ctx, c)) return c;
    return K3Config{1, 256};
}

void apply_k3_config(lb_ctx* ctx, K3Config c) {
    ctx->k3 = c;
    if (c.npt == -2) {
        // TMA-staged: bs-node tiles, persistent grid at full residency; the
        // tensor maps address the two population arrays
        const ChannelDev& d = ctx->ch[0].d;
        const int tiles = d.ny / (c.bs / d.nx) * d.nz;
        ctx->ch[0].d.blk0 = 0;
        ctx->n_groups = tiles;
        ctx->total_blocks = std::min(tiles, tma_blocks_per_sm(c.bs) * ctx->sm_count);
        ctx->tma_ready = ctx->h[0] && ctx->h[1] &&
                         encode_tma_maps(d, c.bs, ctx->h[0], ctx->h[1], ctx->plane, ctx->tma_maps) == cudaSuccess;
        return;
    }
    if (c.npt == 0) {
        // staged: row groups per channel, persistent grid of two blocks per SM
        int grp = 0;
        for (auto& ch : ctx->ch) {
            ch.d.srows = staged_rows(ch.d.nx, (int)pop_bytes(ctx->storage));
            ch.d.sg0 = grp;
            ch.d.blk0 = 0;
            const int rows = ch.d.ny * ch.d.nz;
            grp += ch.d.srows > 0 ? (rows + ch.d.srows - 1) / ch.d.srows : 0;
        }
        ctx->n_groups = grp;
        ctx->total_blocks = std::min(grp, 2 * ctx->sm_count);
        return;
    }
    if (c.npt == -1) {
        // pipelined: 32-node groups per channel, persistent grid at full residency
        int grp = 0;
        for (auto& ch : ctx->ch) {
            ch.d.blk0 = grp;
            grp += (ch.d.n + GROUP - 1) / GROUP;
        }
        ctx->n_groups = grp;
        const int warps_per_block = c.bs / 32;
        const int needed = (grp + warps_per_block - 1) / warps_per_block;
        ctx->total_blocks = std::min(needed, ctx->sm_count * (512 / c.bs));
        return;
    }
    const int per_block = c.npt * c.bs;
    int blk = 0;
    for (auto& ch : ctx->ch) {
        ch.d.blk0 = blk;
        ch.n_blocks = (ch.d.n + per_block - 1) / per_block;
        blk += ch.n_blocks;
    }
    ctx->total_blocks = blk;
}

// The element and ring tables of every mesh (triangles with their rest
// areas, edges with rest length and rest dihedral angle (the bending's
// theta0, Sec. 2.3.1), each node's ring slots), written at the commit, the
// meshes spread over up to 16 host threads (each writes only its own ranges).
void build_tables(lb_ctx* ctx) {
    ctx->htris.resize(ctx->n_tris_staged);
    ctx->htriS0.resize(ctx->n_tris_staged);
    ctx->hedges.resize(ctx->n_edges_staged);
    ctx->hedge_rest.resize(ctx->n_edges_staged);
    ctx->hslots.resize(ctx->n_slots_staged);
    ctx->hinfo.resize(ctx->hq0.size());
    const double* x = ctx->hrest.data();
    auto one = [ctx, x](const PendingMesh& pm) {
        const MeshConn& c = *pm.conn;
        const int node0 = pm.node0;
        for (int t = 0; t < c.nt; ++t) {
            const int v[3] = {c.tris[3 * t], c.tris[3 * t + 1], c.tris[3 * t + 2]};
            ctx->htris[pm.tri0 + t] = make_int4(node0 + v[0], node0 + v[1], node0 + v[2], pm.cell);
            ctx->htriS0[pm.tri0 + t] =
                (float)tri_area_host(x + 3 * (node0 + v[0]), x + 3 * (node0 + v[1]), x + 3 * (node0 + v[2]));
        }
        for (size_t k = 0; k < c.edges.size(); ++k) {
            const int4 e = c.edges[k];
            const int4 g = make_int4(node0 + e.x, node0 + e.y, node0 + e.z, node0 + e.w);
            const double* xa = x + 3 * g.x;
            const double* xb = x + 3 * g.y;
            const double L0 = std::sqrt((xb[0] - xa[0]) * (xb[0] - xa[0]) + (xb[1] - xa[1]) * (xb[1] - xa[1]) +
                                        (xb[2] - xa[2]) * (xb[2] - xa[2]));
            const double th0 = dihedral_host(xa, xb, x + 3 * g.z, x + 3 * g.w);
            ctx->hedges[pm.e0 + k] = g;
            ctx->hedge_rest[pm.e0 + k] = make_float4((float)L0, (float)th0, pm.ks, pm.kb);
        }
        for (int i = 0; i < c.n; ++i)
            ctx->hinfo[node0 + i] = make_int4(pm.cell, node0, pm.slot0 + c.ring_off[i], c.valence[i] | (pm.ch << 8));
        for (size_t k = 0; k < c.slots.size(); ++k) {
            const int4 sl = c.slots[k];
            ctx->hslots[pm.slot0 + k] = make_int4(3 * pm.tri0 + sl.x, 4 * pm.e0 + sl.y, 4 * pm.e0 + sl.z, pm.tri0 + sl.w);
        }
    };
    const int nm = (int)ctx->pending_meshes.size();
    const int nth = std::max(1, std::min({16, (int)std::thread::hardware_concurrency(), nm / 4}));
    // thread t takes meshes t, t + nth, ...; a thread that cannot be started
    // leaves its meshes to this one (no exception leaves the library)
    std::vector<std::thread> th;
    std::vector<int> serial;
    for (int t = 1; t < nth; ++t) {
        try {
            th.emplace_back([&, t] {
                for (int m = t; m < nm; m += nth) one(ctx->pending_meshes[m]);
            });
        } catch (...) {
            serial.push_back(t);
        }
    }
    for (int m = 0; m < nm; m += nth) one(ctx->pending_meshes[m]);
    for (int t : serial)
        for (int m = t; m < nm; m += nth) one(ctx->pending_meshes[m]);
    for (auto& t : th) t.join();
    ctx->pending_meshes.clear();
}

lb_status commit_ibm(lb_ctx* ctx) {
    if (ctx->committed) return LB_OK;
    ctx->committed = true;
    build_tables(ctx);
    ctx->M = (int)ctx->hq0.size();
    ctx->C = (int)ctx->hcells.size();
    ctx->T = (int)ctx->htris.size();
    ctx->NCH = (int)ctx->hchunks.size();
    ctx->K = (int)ctx->hslots.size();
    ctx->E = (int)ctx->hedges.size();
    if (ctx->M == 0) return LB_OK;
    auto up = [&](auto** dst, const auto& src) -> cudaError_t {
        using T = typename std::remove_reference<decltype(src)>::type::value_type;
        cudaError_t e = dalloc(ctx, (T**)dst, src.size());
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
    };
    LB_CUDA(up(&ctx->q0, ctx->hq0));
    LB_CUDA(up(&ctx->q[0], ctx->hq));
    LB_CUDA(up(&ctx->q[1], ctx->hq));
    LB_CUDA(up(&ctx->info, ctx->hinfo));
    LB_CUDA(up(&ctx->slots, ctx->hslots));
    if (ctx->rep_k > 0.f) {
        std::vector<Q4> bq;
        std::vector<float> br;
        std::vector<int> bc;
        for (size_t k = 0; k < ctx->ch.size(); ++k)
            for (size_t b = 0; b + 3 < ctx->ch[k].spheres.size(); b += 4) {
                Q4 q;
                q.x = to_fixed(ctx->ch[k].spheres[b]);
                q.y = to_fixed(ctx->ch[k].spheres[b + 1]);
                q.z = to_fixed(ctx->ch[k].spheres[b + 2]);
                q.w = 0;
                bq.push_back(q);
                br.push_back(ctx->ch[k].spheres[b + 3]);
                bc.push_back((int)k);
            }
        ctx->rep_nb = (int)bq.size();
        ctx->rep_cap = 32 * std::max(ctx->C, 1);
        LB_CUDA(dalloc(ctx, &ctx->rep_R, ctx->M));
        LB_CUDA(dalloc(ctx, &ctx->rep_bounds, ctx->C));
        LB_CUDA(dalloc(ctx, &ctx->rep_pairs, ctx->rep_cap));
        LB_CUDA(dalloc(ctx, &ctx->rep_count, 1));
        LB_CUDA(dalloc(ctx, &ctx->rep_near, (size_t)ctx->C * REP_NEARB));
        LB_CUDA(dalloc(ctx, &ctx->rep_near_count, ctx->C));
        LB_CUDA(dalloc(ctx, &ctx->rep_err, 1));
        LB_CUDA(cudaMemsetAsync(ctx->rep_err, 0, sizeof(int), ctx->stream));
        if (!bq.empty()) {
            LB_CUDA(up(&ctx->rep_bead_q, bq));
            LB_CUDA(up(&ctx->rep_bead_r, br));
            LB_CUDA(up(&ctx->rep_bead_ch, bc));
        }
    }
    LB_CUDA(up(&ctx->edges, ctx->hedges));
    LB_CUDA(up(&ctx->edge_rest, ctx->hedge_rest));
    LB_CUDA(dalloc(ctx, &ctx->eS, ctx->E));
    LB_CUDA(dalloc(ctx, &ctx->eB, 4 * (size_t)ctx->E));
    LB_CUDA(dalloc(ctx, &ctx->tA, 3 * (size_t)ctx->T));
    LB_CUDA(dalloc(ctx, &ctx->tN, ctx->T));
    LB_CUDA(up(&ctx->tris, ctx->htris));
    LB_CUDA(up(&ctx->triS0, ctx->htriS0));
    LB_CUDA(up(&ctx->chunks, ctx->hchunks));
    LB_CUDA(up(&ctx->d_cells, ctx->hcells));
    LB_CUDA(dalloc(ctx, &ctx->F, ctx->M));
    if (ctx->ib_m > 0.0) {
        LB_CUDA(dalloc(ctx, &ctx->W, ctx->M));
        LB_CUDA(cudaMemsetAsync(ctx->W, 0, sizeof(float4) * ctx->M, ctx->stream));
    }
    LB_CUDA(cudaMallocHost((void**)&ctx->hq_pinned, sizeof(Q4) * (size_t)ctx->M));
    LB_CUDA(cudaMemsetAsync(ctx->F, 0, sizeof(float4) * ctx->M, ctx->stream));
    LB_CUDA(dalloc(ctx, &ctx->partials, ctx->NCH));
    LB_CUDA(dalloc(ctx, &ctx->counters, ctx->C));
    LB_CUDA(cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned) * ctx->C, ctx->stream));
    LB_CUDA(dalloc(ctx, &ctx->cell_sums, ctx->C));
    LB_CUDA(cudaMemsetAsync(ctx->cell_sums, 0, sizeof(double2) * ctx->C, ctx->stream));
    LB_CUDA(dalloc(ctx, &ctx->cell_rel, ctx->C));
    LB_CUDA(cudaMemsetAsync(ctx->cell_rel, 0, sizeof(float2) * ctx->C, ctx->stream));
    return LB_OK;
}

lb_status upload_channels(lb_ctx* ctx) {
    std::vector<ChannelDev> v;
    for (auto& c : ctx->ch) v.push_back(c.d);
    LB_CUDA(cudaMemcpyAsync(ctx->d_ch, v.data(), sizeof(ChannelDev) * v.size(), cudaMemcpyHostToDevice, ctx->stream));
    return LB_OK;
}

lb_status check_channel_mesh(lb_ctx* ctx, int mesh_id, const MeshHost** out) {
    const auto& ids = ctx->ch_meshes[ctx->cur];
    if (mesh_id < 0 || mesh_id >= (int)ids.size()) return fail(ctx, LB_ERR_ARG, "mesh id out of range");
    *out = &ctx->meshes[ids[mesh_id]];
    return LB_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

int lb_version(void) { return 10000; }

lb_status lb_set_guard_zones(size_t bytes) {
    if (bytes > ((size_t)1 << 30)) return context_free_error(LB_ERR_ARG, "guard zone larger than 1 GiB");
    g_guard_bytes.store((bytes + 255) / 256 * 256);
    return LB_OK;
}

lb_status lb_check_guard_zones(lb_ctx* ctx, int self_test, int64_t* damaged_bytes) {
    LB_GUARD(ctx);
    if (!damaged_bytes) return fail(ctx, LB_ERR_ARG, "damaged_bytes is NULL");
    *damaged_bytes = 0;
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->guarded.empty()) return LB_OK;
    unsigned long long* d_count = nullptr;
    LB_CUDA(cudaMalloc(&d_count, sizeof(unsigned long long)));   // outside the guarded set
    cudaError_t e = cudaMemset(d_count, 0, sizeof(unsigned long long));
    // self test: one byte of every zone changed from the host first, then restored
    for (const auto& g : ctx->guarded) {
        if (e == cudaSuccess && self_test) e = cudaMemset(g.base + g.guard - 1, 0, 1);
        if (e == cudaSuccess && self_test) e = cudaMemset(g.base + g.guard + g.bytes, 0, 1);
        if (e == cudaSuccess) k_guard_count<<<8, 256, 0, ctx->stream>>>((const unsigned char*)g.base, g.guard, d_count);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess)
            k_guard_count<<<8, 256, 0, ctx->stream>>>((const unsigned char*)g.base + g.guard + g.bytes, g.guard, d_count);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_count, sizeof(h), cudaMemcpyDeviceToHost);
    if (self_test) {
        for (const auto& g : ctx->guarded) {
            if (e == cudaSuccess) e = cudaMemset(g.base + g.guard - 1, GUARD_PATTERN, 1);
            if (e == cudaSuccess) e = cudaMemset(g.base + g.guard + g.bytes, GUARD_PATTERN, 1);
        }
    }
    cudaFree(d_count);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lb_check_guard_zones");
    *damaged_bytes = (int64_t)h;
    return LB_OK;
}

const char* lb_last_error(const lb_ctx* ctx) { return ctx ? ctx->err.c_str() : context_free_err.c_str(); }

lb_status lb_create_batch(const lb_params* params, int n_channels, void* cuda_stream, lb_ctx** out) {
    if (!out) return context_free_error(LB_ERR_ARG, "null output handle");
    *out = nullptr;
    if (!params || n_channels < 1 || n_channels > 4096)
        return context_free_error(LB_ERR_ARG, "need 1 to 4096 channel parameter sets");
    for (int k = 0; k < n_channels; ++k) {
        std::string why;
        if (validate_params(params[k], why) != LB_OK)
            return context_free_error(LB_ERR_ARG, ("channel " + std::to_string(k) + ": " + why).c_str());
        if (params[k].storage != params[0].storage)
            return context_free_error(LB_ERR_ARG, "every channel of a batch needs the same storage");
    }
    lb_ctx* ctx = new lb_ctx();
    ctx->guard = g_guard_bytes.load();
    ctx->storage = params[0].storage;
    long long base = 0;
    for (int k = 0; k < n_channels; ++k) {
        const lb_params& p = params[k];
        ChannelHost c;
        c.p = p;
        ChannelDev& d = c.d;
        std::memset(&d, 0, sizeof(d));
        d.nx = p.nx; d.ny = p.ny; d.nz = p.nz;
        d.dnx = make_fastdiv(p.nx);
        d.dny = make_fastdiv(p.ny);
        for (int a = 0; a < 3; ++a) d.per[a] = p.periodic[a] ? 1 : 0;
        d.n = p.nx * p.ny * p.nz;
        d.base = base;
        d.omega = (float)(1.0 / p.tau);
        d.fpre = (float)(1.0 - 1.0 / (2.0 * p.tau));
        for (int a = 0; a < 3; ++a) d.G[a] = (float)p.body_force[a];
        d.has_uw = 0;
        for (int w = 0; w < 2; ++w)
            for (int a = 0; a < 3; ++a) {
                d.uw[w][a] = (float)p.wall_velocity[w][a];
                if (p.wall_velocity[w][a] != 0.0) d.has_uw = 1;
            }
        base += ((long long)d.n + CH_ALIGN - 1) / CH_ALIGN * CH_ALIGN;
        ctx->ch.push_back(c);
    }
    ctx->Ntot = base;
    ctx->plane = base + plane_pad();
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (ctx->sm_count <= 0) ctx->sm_count = 152;
        cudaGetLastError();
        if (prepare_staged((int)ctx->storage) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return context_free_error(LB_ERR_CUDA, "kernel setup failed (no usable CUDA device?)");
        }
    }
    if (ctx->plane >= (1LL << 31)) {   // node indices are 32-bit inside the kernels
        delete ctx;
        return context_free_error(LB_ERR_ARG, "lattice too large: the padded node count must be < 2^31");
    }
    apply_k3_config(ctx, default_k3_config(ctx));
    ctx->ch_meshes.resize(n_channels);
    cudaStream_t us = (cudaStream_t)cuda_stream;
    if (us == nullptr || us == cudaStreamLegacy || us == cudaStreamPerThread) {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return context_free_error(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, cudaGetErrorString(e));
        }
        ctx->own_stream = true;
    } else {
        ctx->stream = us;
    }
    const long long NT = ctx->Ntot;
    const long long NG = NT / GROUP;
    cudaError_t e = cudaSuccess;
#define TRY(x) if (e == cudaSuccess) e = (x)
    TRY(dalloc(ctx, (char**)&ctx->h[0], (size_t)Q * ctx->plane * pop_bytes(ctx->storage)));
    TRY(dalloc(ctx, (char**)&ctx->h[1], (size_t)Q * ctx->plane * pop_bytes(ctx->storage)));
    TRY(dalloc(ctx, &ctx->mask, NG));
    TRY(dalloc(ctx, &ctx->slow, NG));
    TRY(dalloc(ctx, &ctx->links, NT));
    TRY(dalloc(ctx, &ctx->g[0], NT));
    TRY(dalloc(ctx, &ctx->g[1], NT));
    TRY(dalloc(ctx, &ctx->fl[0], NG));
    TRY(dalloc(ctx, &ctx->fl[1], NG));
    TRY(dalloc(ctx, &ctx->u, NT));
    TRY(dalloc(ctx, &ctx->dmap[0], NG));
    TRY(dalloc(ctx, &ctx->dmap[1], NG));
    TRY(dalloc(ctx, &ctx->dlist[0], NG));
    TRY(dalloc(ctx, &ctx->dlist[1], NG));
    TRY(dalloc(ctx, &ctx->dcount, 2));
    TRY(dalloc(ctx, &ctx->sched_err, 2));
    TRY(dalloc(ctx, &ctx->d_ch, ctx->ch.size()));
    ctx->diag_blocks = 152 * 4;
    TRY(dalloc(ctx, &ctx->diag_partials, (size_t)ctx->diag_blocks * 6));
    TRY(dalloc(ctx, &ctx->diag_out, 6));
    TRY(cudaMemsetAsync(ctx->h[0], 0, (size_t)Q * ctx->plane * pop_bytes(ctx->storage), ctx->stream));
    TRY(cudaMemsetAsync(ctx->h[1], 0, (size_t)Q * ctx->plane * pop_bytes(ctx->storage), ctx->stream));
    TRY(cudaMemsetAsync(ctx->mask, 0, NG * 4, ctx->stream));
    TRY(cudaMemsetAsync(ctx->slow, 0, NG, ctx->stream));
    TRY(cudaMemsetAsync(ctx->links, 0, NT * sizeof(uint32_t), ctx->stream));
    TRY(cudaMemsetAsync(ctx->g[0], 0, NT * sizeof(float4), ctx->stream));
    TRY(cudaMemsetAsync(ctx->g[1], 0, NT * sizeof(float4), ctx->stream));
    TRY(cudaMemsetAsync(ctx->fl[0], 0, NG, ctx->stream));
    TRY(cudaMemsetAsync(ctx->fl[1], 0, NG, ctx->stream));
    TRY(cudaMemsetAsync(ctx->u, 0, NT * sizeof(float4), ctx->stream));
    TRY(cudaMemsetAsync(ctx->dmap[0], 0, NG, ctx->stream));
    TRY(cudaMemsetAsync(ctx->dmap[1], 0, NG, ctx->stream));
    TRY(cudaMemsetAsync(ctx->dcount, 0, 2 * sizeof(int), ctx->stream));
    TRY(cudaMemsetAsync(ctx->sched_err, 0, 2 * sizeof(int), ctx->stream));
    {
        int lo = 0, hi = 0;
        TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        TRY(cudaStreamCreateWithPriority(&ctx->ib_stream, cudaStreamNonBlocking, hi));
        for (int k = 0; k < 2; ++k) {
            TRY(cudaEventCreateWithFlags(&ctx->ev_fork[k], cudaEventDisableTiming));
            TRY(cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming));
            TRY(cudaEventCreateWithFlags(&ctx->ev_fork2[k], cudaEventDisableTiming));
            TRY(cudaEventCreateWithFlags(&ctx->ev_join2[k], cudaEventDisableTiming));
        }
    }
    ctx->list_blocks = ctx->sm_count * 16;   // 2 waves of 128-thread blocks at 64 registers
    {
        int dev = 0, smem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        ctx->smem_per_sm = smem;
        cudaGetLastError();
        if (smem > 0) TRY(prepare_bulk((int)ctx->storage, (int)bulk_smem_max(ctx)));
    }
#undef TRY
    if (e != cudaSuccess) {
        lb_status s = e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
        cudaGetLastError();
        lb_destroy(ctx);
        return context_free_error(s, cudaGetErrorString(e));
    }
    const char* setup_err = "lattice setup failed (CUDA error)";
    if (upload_channels(ctx) != LB_OK) { lb_destroy(ctx); return context_free_error(LB_ERR_CUDA, setup_err); }
    for (size_t k = 0; k < ctx->ch.size(); ++k)
        if (launch_slow_flags(ctx->ch[k].d, ctx->mask, ctx->slow, ctx->links, ctx->stream) != cudaSuccess) {
            lb_destroy(ctx);
            return context_free_error(LB_ERR_CUDA, setup_err);
        }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        lb_destroy(ctx);
        return context_free_error(LB_ERR_CUDA, setup_err);
    }
    *out = ctx;
    return LB_OK;
}

lb_status lb_create(const lb_params* params, void* cuda_stream, lb_ctx** out) {
    return lb_create_batch(params, 1, cuda_stream, out);
}

lb_status lb_select_channel(lb_ctx* ctx, int channel) {
    LB_GUARD(ctx);
    if (channel < 0 || channel >= (int)ctx->ch.size()) return fail(ctx, LB_ERR_ARG, "channel out of range");
    ctx->cur = channel;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx* ctx) {
    if (!ctx) return LB_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    for (auto& kv : ctx->adj.g_fwd) cudaGraphExecDestroy(kv.second);
    for (auto& kv : ctx->adj.g_bwd) cudaGraphExecDestroy(kv.second);
    for (void* p : ctx->allocations) cudaFree(p);
    if (ctx->hq_pinned) cudaFreeHost(ctx->hq_pinned);
    ctx->allocations.clear();
    for (auto& ep : ctx->pending) { cudaEventDestroy(ep.a); cudaEventDestroy(ep.b); }
    for (auto e : ctx->free_events) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->ib_stream) {
        cudaStreamSynchronize(ctx->ib_stream);
        cudaStreamDestroy(ctx->ib_stream);
    }
    for (int k = 0; k < 2; ++k) {
        if (ctx->rb_ev[k]) cudaEventDestroy(ctx->rb_ev[k]);
        if (ctx->ev_fork[k]) cudaEventDestroy(ctx->ev_fork[k]);
        if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
        if (ctx->ev_fork2[k]) cudaEventDestroy(ctx->ev_fork2[k]);
        if (ctx->ev_join2[k]) cudaEventDestroy(ctx->ev_join2[k]);
    }
    delete ctx;
    return LB_OK;
}

lb_status lb_set_repulsion(lb_ctx* ctx, double k, double dc) {
    LB_GUARD(ctx);
    if (ctx->started || ctx->committed) return fail(ctx, LB_ERR_STATE, "collisions must be set before the first step");
    if (!(k >= 0.0) || !(dc > 0.0) || !std::isfinite(k) || !std::isfinite(dc))
        return fail(ctx, LB_ERR_ARG, "need k >= 0 and dc > 0");
    if (k > 0.0 && ctx->phi) return fail(ctx, LB_ERR_STATE, "collisions are not part of the differentiable variant");
    if (k > 0.0 && ctx->deterministic) return fail(ctx, LB_ERR_STATE, "collisions accumulate with float atomics");
    ctx->rep_k = (float)k;
    ctx->rep_dc = (float)dc;
    drop_graphs(ctx);
    return LB_OK;
}

lb_status lb_set_ib_dynamics(lb_ctx* ctx, double mass, double gamma) {
    LB_GUARD(ctx);
    if (ctx->started || ctx->committed)
        return fail(ctx, LB_ERR_STATE, "the IB point dynamics must be set before the first step");
    if (!(mass >= 0.0) || !(gamma >= 0.0) || !std::isfinite(mass) || !std::isfinite(gamma))
        return fail(ctx, LB_ERR_ARG, "need finite mass >= 0 and gamma >= 0");
    if (mass > 0.0 && ctx->phi) return fail(ctx, LB_ERR_STATE, "the differentiable variant has massless points");
    ctx->ib_m = mass;
    ctx->ib_gamma = gamma;
    drop_graphs(ctx);
    return LB_OK;
}

lb_status lb_set_deterministic(lb_ctx* ctx, int on) {
    LB_GUARD(ctx);
    if (on != 0 && on != 1) return fail(ctx, LB_ERR_ARG, "on must be 0 or 1");
    if (on && ctx->rep_k > 0.f) return fail(ctx, LB_ERR_STATE, "collisions accumulate with float atomics");
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (on && !ctx->gfix) {
        LB_CUDA(dalloc(ctx, &ctx->gfix, 3 * (size_t)ctx->Ntot));
        LB_CUDA(cudaMemsetAsync(ctx->gfix, 0, sizeof(unsigned long long) * 3 * (size_t)ctx->Ntot, ctx->stream));
    }
    if ((on != 0) != ctx->deterministic) drop_graphs(ctx);
    ctx->deterministic = on != 0;
    ctx->dvalid = false;
    return LB_OK;
}

lb_status ibm_get_velocities(lb_ctx* ctx, int mesh_id, double* v) {
    LB_GUARD(ctx);
    const MeshHost* mh;
    if (check_channel_mesh(ctx, mesh_id, &mh) != LB_OK) return LB_ERR_ARG;
    if (!v) return fail(ctx, LB_ERR_ARG, "null output");
    lb_status st = commit_ibm(ctx);
    if (st != LB_OK) return st;
    if (!ctx->W) {
        for (int j = 0; j < 3 * mh->n; ++j) v[j] = 0.0;
        return LB_OK;
    }
    std::vector<float4> w(mh->n);
    LB_CUDA(cudaMemcpyAsync(w.data(), ctx->W + mh->node0, sizeof(float4) * mh->n, cudaMemcpyDeviceToHost, ctx->stream));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < mh->n; ++j) {
        v[3 * j] = w[j].x;
        v[3 * j + 1] = w[j].y;
        v[3 * j + 2] = w[j].z;
    }
    return LB_OK;
}

lb_status lb_set_brinkman(lb_ctx* ctx, const double* beads, int n, double alpha, double delta) {
    LB_GUARD(ctx);
    if (ctx->started) return fail(ctx, LB_ERR_STATE, "the Brinkman beads must be set before the first step");
    if (ctx->ch.size() != 1) return fail(ctx, LB_ERR_ARG, "the differentiable variant takes a single-channel context");
    if (ctx->rep_k > 0.f) return fail(ctx, LB_ERR_STATE, "collisions are not part of the differentiable variant");
    if (ctx->ib_m > 0.0) return fail(ctx, LB_ERR_STATE, "the differentiable variant has massless points");
    if (n < 0 || (n > 0 && !beads) || !(alpha >= 0.0) || !(delta > 0.0))
        return fail(ctx, LB_ERR_ARG, "bad bead list, alpha or delta");
    for (int k = 0; k < 4 * n; ++k)
        if (!std::isfinite(beads[k]) || (k % 4 == 3 && beads[k] < 0))
            return fail(ctx, LB_ERR_ARG, "bead data must be finite with r >= 0");
    if (!k3_config_valid(ctx, K3Config{1, ctx->k3.npt == 1 ? ctx->k3.bs : 128}))
        return fail(ctx, LB_ERR_ARG, "no one-node-per-thread stream-collide variant for this lattice");
    if (ctx->k3.npt != 1) apply_k3_config(ctx, K3Config{1, 128});
    ctx->beads.assign(beads, beads + 4 * n);
    ctx->alpha = (float)alpha;
    ctx->delta = (float)delta;
    const ChannelHost& c = ctx->ch[0];
    if (!ctx->phi) LB_CUDA(dalloc(ctx, &ctx->phi, ctx->Ntot));
    LB_CUDA(cudaMemsetAsync(ctx->phi, 0, sizeof(float) * ctx->Ntot, ctx->stream));
    std::vector<float> fb(4 * (size_t)n);
    for (int k = 0; k < 4 * n; ++k) fb[k] = (float)beads[k];
    if (ctx->d_beads) dfree(ctx, ctx->d_beads);
    ctx->d_beads = nullptr;
    LB_CUDA(dalloc(ctx, &ctx->d_beads, std::max(4 * n, 4)));
    if (n > 0) {
        LB_CUDA(cudaMemcpyAsync(ctx->d_beads, fb.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice, ctx->stream));
        LB_CUDA(launch_brinkman_phi(c.d, ctx->d_beads, n, (float)delta, ctx->phi, ctx->stream));
    }
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);
    return upload_channels(ctx);
}

// ---- discrete adjoint of the differentiable variant ----
namespace {

// Forward cycle k of a segment run directly on the segment store: it pulls
// from populations slot k and writes slot k + 1, advances positions slot k to
// k + 1, and leaves its node forces, spread force density (zeroed first, no
// previous-cycle flags to clear), velocity and cells' (dS/S0, dV/V0) in slot
// k: everything the reverse sweep of that cycle reads.
lb_status store_step(lb_ctx* ctx, int k) {
    auto& W = ctx->adj;
    const int par = (int)(ctx->step & 1);
    const size_t hN = (size_t)Q * ctx->plane;
    cudaStream_t s = ctx->stream;
    float* hs = W.seg_h + (size_t)k * hN;
    float* hd = W.seg_h + (size_t)(k + 1) * hN;
    Q4* qs = W.seg_q + (size_t)k * ctx->M;
    Q4* qd = W.seg_q + (size_t)(k + 1) * ctx->M;
    float4* gk = W.seg_g + (size_t)k * ctx->Ntot;
    float4* uk = W.seg_u + (size_t)k * ctx->Ntot;
    uint8_t* flk = W.seg_fl + (size_t)k * (ctx->Ntot / GROUP);
    LatticeArgs la = lattice_args(ctx, par);
    IbmArgs ia = ibm_args(ctx, par);
    la.h0 = par ? (void*)hd : (void*)hs;
    la.h1 = par ? (void*)hs : (void*)hd;
    la.u = uk;
    la.g0 = la.g1 = gk;
    ia.g0 = ia.g1 = gk;
    la.fl0 = ia.fl0 = par ? W.fl_zero : flk;
    la.fl1 = ia.fl1 = par ? flk : W.fl_zero;
    ia.u = uk;
    ia.qa = par ? qd : qs;
    ia.qb = par ? qs : qd;
    ia.F = W.seg_F + (size_t)k * ctx->M;
    ia.cell_rel = W.seg_rel + (size_t)k * ctx->C;
    ia.gfix = nullptr;   // the adjoint's forward spreads with float atomics
    // programmatic dependents as in the plain cycle, except the segment's
    // first kernel (it follows the zeroing of the segment's force slots)
    ia.pdl = ctx->pdl && k > 0;
    LB_CUDA(launch_elements(ia, s));
    ia.pdl = la.pdl = ctx->pdl;
    LB_CUDA(launch_forces_spread(ia, s));
    LB_CUDA(k3_launch(ctx, la, ctx->k3, s));
    LB_CUDA(launch_interp_advance(ia, s));
    ctx->step++;
    return LB_OK;
}

// The forward cycles 0 .. len-1 of a segment on the segment store, as one
// CUDA graph per (len, parity of the first cycle), launched on the stream.
// Every cycle's force density and flags start from zero.
lb_status run_segment_forward(lb_ctx* ctx, int len) {
    auto& W = ctx->adj;
    const std::pair<int, int> key(len, (int)(ctx->step & 1));
    auto it = W.g_fwd.find(key);
    if (it == W.g_fwd.end()) {
        const long long step_saved = ctx->step;
        cudaGraph_t g = nullptr;
        LB_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e0 = cudaMemsetAsync(W.seg_g, 0, sizeof(float4) * ctx->Ntot * (size_t)len, ctx->stream);
        if (e0 == cudaSuccess) e0 = cudaMemsetAsync(W.seg_fl, 0, (size_t)(ctx->Ntot / GROUP) * len, ctx->stream);
        lb_status st = e0 == cudaSuccess ? LB_OK : LB_ERR_CUDA;
        for (int k = 0; k < len && st == LB_OK; ++k) st = store_step(ctx, k);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        ctx->step = step_saved;
        if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "cudaMemsetAsync");
        if (st != LB_OK) return st;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        it = W.g_fwd.emplace(key, ge).first;
    }
    LB_CUDA(cudaGraphLaunch(it->second, ctx->stream));
    ctx->step += len;
    return LB_OK;
}

// Positions + populations of the current step into (h_dst, q_dst) or back.
lb_status copy_state(lb_ctx* ctx, float* h, Q4* q, bool save) {
    const int par = (int)(ctx->step & 1);
    const size_t hb = sizeof(float) * Q * (size_t)ctx->plane;
    cudaStream_t s = ctx->stream;
    if (save) {
        LB_CUDA(cudaMemcpyAsync(h, ctx->h[par], hb, cudaMemcpyDeviceToDevice, s));
        LB_CUDA(cudaMemcpyAsync(q, ctx->q[par], sizeof(Q4) * ctx->M, cudaMemcpyDeviceToDevice, s));
    } else {
        LB_CUDA(cudaMemcpyAsync(ctx->h[par], h, hb, cudaMemcpyDeviceToDevice, s));
        LB_CUDA(cudaMemcpyAsync(ctx->q[par], q, sizeof(Q4) * ctx->M, cudaMemcpyDeviceToDevice, s));
        // force fields and flags as at the start of any step: nothing pending
        for (int k = 0; k < 2; ++k) {
            LB_CUDA(cudaMemsetAsync(ctx->g[k], 0, sizeof(float4) * ctx->Ntot, s));
            LB_CUDA(cudaMemsetAsync(ctx->fl[k], 0, (size_t)(ctx->Ntot / GROUP), s));
        }
    }
    return LB_OK;
}

double mean_x(const Q4* qdev, const MeshHost& m) {
    std::vector<Q4> q(m.n);
    cudaMemcpy(q.data(), qdev + m.node0, sizeof(Q4) * m.n, cudaMemcpyDeviceToHost);
    double s = 0.0;
    for (const Q4& v : q) s += (double)v.x / FIX_SCALE;
    return s / m.n;
}

}  // namespace

lb_status lb_adjoint(lb_ctx* ctx, int n_steps, int ckpt_every, int objective_mesh, double* J, double* grad_beads,
                     double* grad_ks, double* grad_kb) {
    LB_GUARD(ctx);
    if (!ctx->phi) return fail(ctx, LB_ERR_STATE, "lb_adjoint needs the differentiable variant (lb_set_brinkman)");
    if (ctx->ib_m > 0.0) return fail(ctx, LB_ERR_STATE, "lb_adjoint needs massless IB points");
    if (ctx->storage != LB_F32) return fail(ctx, LB_ERR_ARG, "lb_adjoint needs FP32 populations");
    if (n_steps < 1 || ckpt_every < 1) return fail(ctx, LB_ERR_ARG, "n_steps and ckpt_every must be >= 1");
    if (ctx->timing) return fail(ctx, LB_ERR_STATE, "per-kernel timing is on");
    lb_status st = commit_ibm(ctx);
    if (st != LB_OK) return st;
    const MeshHost* mo;
    if (check_channel_mesh(ctx, objective_mesh, &mo) != LB_OK) return LB_ERR_ARG;
    const int nb = (int)ctx->beads.size() / 4;
    if (nb > 64) return fail(ctx, LB_ERR_ARG, "at most 64 beads");
    auto& W = ctx->adj;
    const int K = std::min(ckpt_every, n_steps);
    const int n_ck = (n_steps + K - 1) / K;
    const size_t hN = (size_t)Q * ctx->plane;
    if (W.K != K || W.n_ck != n_ck) {
        for (void* p : {(void*)W.ck_h, (void*)W.seg_h, (void*)W.fin_h, (void*)W.lam[0], (void*)W.lam[1], (void*)W.Lphi,
                        (void*)W.ck_q, (void*)W.seg_q, (void*)W.fin_q, (void*)W.seg_F, (void*)W.seg_g, (void*)W.seg_u,
                        (void*)W.lam_u, (void*)W.lam_g, (void*)W.lamX[0], (void*)W.lamX[1], (void*)W.lamF,
                        (void*)W.tri_dS, (void*)W.tri_n, (void*)W.seg_rel, (void*)W.lam_c, (void*)W.grad,
                        (void*)W.fin_u, (void*)W.fin_F, (void*)W.seg_fl, (void*)W.fl_zero})
            dfree(ctx, p);
        for (auto& kv : W.g_fwd) cudaGraphExecDestroy(kv.second);
        for (auto& kv : W.g_bwd) cudaGraphExecDestroy(kv.second);
        W = lb_ctx::AdjWork();
        cudaError_t e = cudaSuccess;
#define ATRY(x) if (e == cudaSuccess) e = (x)
        ATRY(dalloc(ctx, &W.ck_h, (size_t)n_ck * hN));
        ATRY(dalloc(ctx, &W.ck_q, (size_t)n_ck * ctx->M));
        ATRY(dalloc(ctx, &W.seg_h, (size_t)(K + 1) * hN));
        ATRY(dalloc(ctx, &W.seg_q, (size_t)(K + 1) * ctx->M));
        ATRY(dalloc(ctx, &W.seg_fl, (size_t)K * (ctx->Ntot / GROUP)));
        ATRY(dalloc(ctx, &W.fl_zero, (size_t)(ctx->Ntot / GROUP)));
        if (e == cudaSuccess) e = cudaMemsetAsync(W.fl_zero, 0, (size_t)(ctx->Ntot / GROUP), ctx->stream);
        ATRY(dalloc(ctx, &W.seg_F, (size_t)K * ctx->M));
        ATRY(dalloc(ctx, &W.seg_g, (size_t)K * ctx->Ntot));
        ATRY(dalloc(ctx, &W.seg_u, (size_t)K * ctx->Ntot));
        ATRY(dalloc(ctx, &W.seg_rel, (size_t)K * ctx->C));
        ATRY(dalloc(ctx, &W.fin_h, hN));
        ATRY(dalloc(ctx, &W.fin_q, ctx->M));
        ATRY(dalloc(ctx, &W.fin_u, ctx->Ntot));
        ATRY(dalloc(ctx, &W.fin_F, ctx->M));
        ATRY(dalloc(ctx, &W.lam[0], hN));
        ATRY(dalloc(ctx, &W.lam[1], hN));
        ATRY(dalloc(ctx, &W.Lphi, ctx->Ntot));
        ATRY(dalloc(ctx, &W.lam_u, ctx->Ntot));
        ATRY(dalloc(ctx, &W.lam_g, ctx->Ntot));
        ATRY(dalloc(ctx, &W.lamX[0], ctx->M));
        ATRY(dalloc(ctx, &W.lamX[1], ctx->M));
        ATRY(dalloc(ctx, &W.lamF, ctx->M));
        ATRY(dalloc(ctx, &W.tri_dS, 2 * (size_t)ctx->T));
        ATRY(dalloc(ctx, &W.tri_n, ctx->T));
        ATRY(dalloc(ctx, &W.lam_c, 2 * (size_t)ctx->C));
        ATRY(dalloc(ctx, &W.grad, 2 + 3 * 64));
#undef ATRY
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "adjoint workspace");
        }
        W.K = K;
        W.n_ck = n_ck;
    }
    cudaStream_t s = ctx->stream;
    const long long step0 = ctx->step;
    const double x0 = mean_x(ctx->q[ctx->step & 1], *mo);
    const size_t hb = sizeof(float) * hN;
    // forward: checkpoints at the start of every segment; the last segment
    // runs on the segment store, so its reverse sweep needs no recompute
    for (int c = 0; c + 1 < n_ck; ++c) {
        if (copy_state(ctx, W.ck_h + (size_t)c * hN, W.ck_q + (size_t)c * ctx->M, true) != LB_OK) return LB_ERR_CUDA;
        st = lb_step(ctx, K);
        if (st != LB_OK) return st;
    }
    const int last = n_ck - 1;
    const int len_last = n_steps - last * K;
    if (copy_state(ctx, W.seg_h, W.seg_q, true) != LB_OK) return LB_ERR_CUDA;
    st = run_segment_forward(ctx, len_last);
    if (st != LB_OK) return st;
    // the final state, restored into the context at the end
    LB_CUDA(cudaMemcpyAsync(W.fin_h, W.seg_h + (size_t)len_last * hN, hb, cudaMemcpyDeviceToDevice, s));
    LB_CUDA(cudaMemcpyAsync(W.fin_q, W.seg_q + (size_t)len_last * ctx->M, sizeof(Q4) * ctx->M, cudaMemcpyDeviceToDevice, s));
    LB_CUDA(cudaMemcpyAsync(W.fin_u, W.seg_u + (size_t)(len_last - 1) * ctx->Ntot, sizeof(float4) * ctx->Ntot,
                            cudaMemcpyDeviceToDevice, s));
    LB_CUDA(cudaMemcpyAsync(W.fin_F, W.seg_F + (size_t)(len_last - 1) * ctx->M, sizeof(float4) * ctx->M,
                            cudaMemcpyDeviceToDevice, s));
    LB_CUDA(cudaStreamSynchronize(s));
    const double Jv = mean_x(W.fin_q, *mo) - x0;
    // reverse sweep
    LB_CUDA(cudaMemsetAsync(W.lam[0], 0, sizeof(float) * hN, s));
    LB_CUDA(cudaMemsetAsync(W.lam[1], 0, sizeof(float) * hN, s));
    LB_CUDA(cudaMemsetAsync(W.Lphi, 0, sizeof(float) * ctx->Ntot, s));
    LB_CUDA(cudaMemsetAsync(W.lam_u, 0, sizeof(float4) * ctx->Ntot, s));
    LB_CUDA(cudaMemsetAsync(W.lam_g, 0, sizeof(float4) * ctx->Ntot, s));
    LB_CUDA(cudaMemsetAsync(W.grad, 0, sizeof(double) * (2 + 3 * 64), s));
    {
        std::vector<float4> l0(ctx->M, make_float4(0.f, 0.f, 0.f, 0.f));
        for (int i = 0; i < mo->n; ++i) l0[mo->node0 + i].x = (float)(1.0 / mo->n);   // dJ / dX^T
        LB_CUDA(cudaMemcpyAsync(W.lamX[0], l0.data(), sizeof(float4) * ctx->M, cudaMemcpyHostToDevice, s));
        LB_CUDA(cudaStreamSynchronize(s));
    }
    AdjArgs A;
    std::memset(&A, 0, sizeof(A));
    A.ch = ctx->ch[0].d;
    A.M = ctx->M;
    A.n_edges = ctx->E;
    A.n_tris = ctx->T;
    A.n_beads = nb;
    A.obj_cell = mo->cell;
    A.n_cells = ctx->C;
    A.plane = ctx->plane;
    A.mask = ctx->mask;
    A.links = ctx->links;
    A.slow = ctx->slow;
    A.phi = ctx->phi;
    A.alpha = ctx->alpha;
    A.delta = ctx->delta;
    A.beads = reinterpret_cast<const float4*>(ctx->d_beads);
    A.lam_u = W.lam_u;
    A.lam_g = W.lam_g;
    A.Lphi = W.Lphi;
    A.lamF = W.lamF;
    A.edges = ctx->edges;
    A.edge_rest = ctx->edge_rest;
    A.tris = ctx->tris;
    A.tri_S0 = ctx->triS0;
    A.info = ctx->info;
    A.cells = ctx->d_cells;
    A.tri_dS = W.tri_dS;
    A.tri_n = W.tri_n;
    A.lam_c = W.lam_c;
    A.grad = W.grad;
    int lc = 0, xc = 0;
    for (int c = n_ck - 1; c >= 0; --c) {
        const int len = std::min(K, n_steps - c * K);
        if (c < last) {
            // recompute the segment from its checkpoint on the segment store
            ctx->step = step0 + (long long)c * K;
            LB_CUDA(cudaMemcpyAsync(W.seg_h, W.ck_h + (size_t)c * hN, hb, cudaMemcpyDeviceToDevice, s));
            LB_CUDA(cudaMemcpyAsync(W.seg_q, W.ck_q + (size_t)c * ctx->M, sizeof(Q4) * ctx->M, cudaMemcpyDeviceToDevice, s));
            st = run_segment_forward(ctx, len);
            if (st != LB_OK) return st;
        }
        {
            const std::pair<int, int> key(len, lc + 2 * xc);
            auto it = W.g_bwd.find(key);
            if (it == W.g_bwd.end()) {
                cudaGraph_t g = nullptr;
                LB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                int l = lc, x = xc;
                cudaError_t e = cudaSuccess;
                for (int k = len - 1; k >= 0 && e == cudaSuccess; --k) {
                    A.q_t = W.seg_q + (size_t)k * ctx->M;
                    A.F_t = W.seg_F + (size_t)k * ctx->M;
                    A.g_t = W.seg_g + (size_t)k * ctx->Ntot;
                    A.u_t = W.seg_u + (size_t)k * ctx->Ntot;
                    A.h_t = W.seg_h + (size_t)k * hN;
                    A.rel_t = W.seg_rel + (size_t)k * ctx->C;
                    A.fl_t = W.seg_fl + (size_t)k * (ctx->Ntot / GROUP);
                    A.lam_in = W.lam[l];
                    A.lam_out = W.lam[1 - l];
                    A.lamX = W.lamX[x];
                    A.lamX_out = W.lamX[1 - x];
                    // each kernel a programmatic dependent of the one before it,
                    // except the graph's first
                    A.pdl = ctx->pdl && k < len - 1;
                    e = launch_adj_interp(A, s);
                    A.pdl = ctx->pdl;
                    if (e == cudaSuccess) e = launch_adj_collide(A, s);
                    if (e == cudaSuccess) e = launch_adj_spread(A, s);
                    if (e == cudaSuccess) e = launch_adj_membrane(A, s);
                    l = 1 - l;
                    x = 1 - x;
                }
                cudaError_t e2 = cudaStreamEndCapture(s, &g);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint launch");
                if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
                cudaGraphExec_t ge = nullptr;
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
                it = W.g_bwd.emplace(key, ge).first;
            }
            LB_CUDA(cudaGraphLaunch(it->second, s));
            if (len & 1) {
                lc = 1 - lc;
                xc = 1 - xc;
            }
        }
    }
    A.pdl = 0;
    LB_CUDA(launch_adj_bead_grad(A, s));
    std::vector<double> g(2 + 3 * 64);
    LB_CUDA(cudaMemcpyAsync(g.data(), W.grad, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, s));
    // leave the context in the state after the n_steps forward steps
    ctx->step = step0 + n_steps;
    if (copy_state(ctx, W.fin_h, W.fin_q, false) != LB_OK) return LB_ERR_CUDA;
    LB_CUDA(cudaMemcpyAsync(ctx->u, W.fin_u, sizeof(float4) * ctx->Ntot, cudaMemcpyDeviceToDevice, s));
    LB_CUDA(cudaMemcpyAsync(ctx->F, W.fin_F, sizeof(float4) * ctx->M, cudaMemcpyDeviceToDevice, s));
    LB_CUDA(cudaStreamSynchronize(s));
    if (J) *J = Jv;
    if (grad_ks) *grad_ks = g[0];
    if (grad_kb) *grad_kb = g[1];
    if (grad_beads)
        for (int k = 0; k < 3 * nb; ++k) grad_beads[k] = g[2 + k];
    return LB_OK;
}

lb_status lb_set_obstacles(lb_ctx* ctx, const float* spheres, int n, const uint8_t* extra_mask) {
    LB_GUARD(ctx);
    if (ctx->started) return fail(ctx, LB_ERR_STATE, "obstacles must be set before the first step");
    if (n < 0 || (n > 0 && !spheres)) return fail(ctx, LB_ERR_ARG, "bad sphere list");
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < 4; ++j)
            if (!std::isfinite(spheres[4 * k + j]) || (j == 3 && spheres[4 * k + 3] < 0))
                return fail(ctx, LB_ERR_ARG, "sphere data must be finite with r >= 0");
    const ChannelHost& c = ctx->ch[ctx->cur];
    const long long w0 = c.d.base / GROUP;
    const long long nw = (c.d.n + GROUP - 1) / GROUP;
    LB_CUDA(cudaMemsetAsync(ctx->mask + w0, 0, nw * 4, ctx->stream));
    LB_CUDA(cudaMemsetAsync(ctx->slow + w0, 0, nw, ctx->stream));
    float* dsph = nullptr;
    uint8_t* dext = nullptr;
    if (n > 0) {
        LB_CUDA(dalloc(ctx, &dsph, (size_t)4 * n));
        LB_CUDA(cudaMemcpyAsync(dsph, spheres, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    }
    if (extra_mask) {
        LB_CUDA(dalloc(ctx, &dext, (size_t)c.d.n));
        LB_CUDA(cudaMemcpyAsync(dext, extra_mask, (size_t)c.d.n, cudaMemcpyHostToDevice, ctx->stream));
    }
    LB_CUDA(launch_rasterise(dsph, n, dext, c.d, ctx->mask, ctx->stream));
    ctx->ch[ctx->cur].spheres.assign(spheres, spheres + 4 * (size_t)n);
    LB_CUDA(launch_slow_flags(c.d, ctx->mask, ctx->slow, ctx->links, ctx->stream));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, dsph);
    dfree(ctx, dext);
    return LB_OK;
}

lb_status lb_get_mask(lb_ctx* ctx, uint8_t* solid) {
    LB_GUARD(ctx);
    if (!solid) return LB_ERR_ARG;
    const ChannelDev& d = ctx->ch[ctx->cur].d;
    std::vector<uint32_t> mask((size_t)((d.n + 31) / 32));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    LB_CUDA(cudaMemcpy(mask.data(), ctx->mask + d.base / GROUP, sizeof(uint32_t) * mask.size(), cudaMemcpyDeviceToHost));
    for (long long p = 0; p < d.n; ++p) solid[p] = (mask[p >> 5] >> (p & 31)) & 1u;
    return LB_OK;
}

namespace {
// Directed edges a -> b of one mesh with an int each, stored per tail node in
// one flat array (a node's slots are as many as the triangles around it, at
// most the valence limit, so a lookup scans a handful of entries).
struct DirEdges {
    std::vector<int> off, cnt, key, val;
    DirEdges(int n, const int32_t* tris, int nt) : off(n + 1, 0), cnt(n, 0), key(3 * (size_t)nt), val(3 * (size_t)nt) {
        for (int k = 0; k < 3 * nt; ++k) off[tris[k] + 1]++;
        for (int i = 0; i < n; ++i) off[i + 1] += off[i];
    }
    int size(int a) const { return cnt[a]; }
    int* find(int a, int b) {
        for (int i = off[a]; i < off[a] + cnt[a]; ++i)
            if (key[i] == b) return &val[i];
        return nullptr;
    }
    void put(int a, int b, int v) {
        if (int* p = find(a, b)) {
            *p = v;
            return;
        }
        key[off[a] + cnt[a]] = b;
        val[off[a] + cnt[a]] = v;
        cnt[a]++;
    }
    int at(int a, int b) {
        int* p = find(a, b);
        return p ? *p : -1;
    }
    void sort_node(int a) {   // by head vertex (insertion sort: a handful of entries)
        for (int i = off[a] + 1; i < off[a] + cnt[a]; ++i)
            for (int j = i; j > off[a] && key[j - 1] > key[j]; --j) {
                std::swap(key[j - 1], key[j]);
                std::swap(val[j - 1], val[j]);
            }
    }
    int first(int a) const { return key[off[a]]; }
};
}  // namespace

namespace {
// A cell mesh checked for use: directed edge a -> b with the third vertex of
// its triangle, every node's ring of neighbours, the rest area and volume.
struct MeshTopology {
    DirEdges third;
    std::vector<int> out_deg;
    std::vector<std::vector<int>> ringv;
    double S0 = 0.0, V0 = 0.0;
    MeshTopology(int n, const int32_t* tris, int nt) : third(n, tris, nt), out_deg(n, 0), ringv(n) {}
};

// The rest area and volume (FP64) of a mesh whose connectivity is valid;
// refuses non-finite positions and an inward orientation.
const char* mesh_geometry(const double* x, int n, const int32_t* tris, int nt, double& S0, double& V0) {
    for (int k = 0; k < 3 * n; ++k)
        if (!std::isfinite(x[k]) || std::fabs(x[k]) > 4.0e6) return "node positions must be finite and |x| < 4e6";
    S0 = 0.0;
    V0 = 0.0;
    for (int t = 0; t < nt; ++t) {
        const double* a = x + 3 * tris[3 * t];
        const double* b = x + 3 * tris[3 * t + 1];
        const double* c = x + 3 * tris[3 * t + 2];
        S0 += tri_area_host(a, b, c);
        V0 += (a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
               a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
    }
    if (!(V0 > 0.0)) return "mesh volume must be positive (outward orientation)";
    return nullptr;
}

// Checks that (x, tris) is a closed, outward, oriented 2-manifold whose every
// node is a single fan of at most MAX_VALENCE triangles, and builds its
// topology into *topo.  Returns nullptr, or why the mesh is refused.  Host
// code only.
const char* mesh_topology(const double* x, int n, const int32_t* tris, int nt, std::unique_ptr<MeshTopology>& topo) {
    if (!x || !tris || n < 4 || nt < 4) return "mesh needs >= 4 nodes and triangles";
    for (int k = 0; k < 3 * n; ++k)
        if (!std::isfinite(x[k]) || std::fabs(x[k]) > 4.0e6) return "node positions must be finite and |x| < 4e6";
    for (int k = 0; k < 3 * nt; ++k)
        if (tris[k] < 0 || tris[k] >= n) return "triangle index out of range";
    topo.reset(new MeshTopology(n, tris, nt));
    DirEdges& third = topo->third;
    std::vector<int>& out_deg = topo->out_deg;
    for (int t = 0; t < nt; ++t) {
        const int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        for (int k = 0; k < 3; ++k) {
            const int a = v[k], b = v[(k + 1) % 3];
            if (a == b) return "degenerate triangle";
            if (third.find(a, b)) return "mesh is not an oriented 2-manifold (edge used twice)";
            third.put(a, b, v[(k + 2) % 3]);
            out_deg[a]++;
        }
    }
    for (int a = 0; a < n; ++a) {
        if (out_deg[a] > MAX_VALENCE) return "mesh vertex is not a single fan (non-manifold) or valence > 64";
        third.sort_node(a);
        for (int i = third.off[a]; i < third.off[a] + third.cnt[a]; ++i)
            if (!third.find(third.key[i], a)) return "mesh is not closed";
    }
    // node rings, counter-clockwise seen from outside: ring[j+1] = third(i -> ring[j]),
    // each starting at the node's smallest neighbour
    for (int i = 0; i < n; ++i) {
        if (third.size(i) == 0) continue;
        int a = third.first(i);
        std::vector<int>& r = topo->ringv[i];
        r.reserve((size_t)out_deg[i] + 1);
        for (int guard = 0; guard <= MAX_VALENCE; ++guard) {
            r.push_back(a);
            a = third.at(i, a);
            if (a < 0 || a == r[0]) break;
        }
        if ((int)r.size() != out_deg[i] || (int)r.size() > MAX_VALENCE || a != r[0])
            return "mesh vertex is not a single fan (non-manifold) or valence > 64";
    }
    for (int i = 0; i < n; ++i)
        if (topo->ringv[i].empty()) return "mesh has an isolated node";
    return mesh_geometry(x, n, tris, nt, topo->S0, topo->V0);
}

// Checks a mesh and builds its connectivity tables into c (and its rest area
// and volume); nullptr, or why the mesh is refused.
const char* build_conn(const double* x, int n, const int32_t* tris, int nt, MeshConn& c, double& S0, double& V0) {
    std::unique_ptr<MeshTopology> topo;
    if (const char* err = mesh_topology(x, n, tris, nt, topo)) return err;
    S0 = topo->S0;
    V0 = topo->V0;
    DirEdges& third = topo->third;
    c.n = n;
    c.nt = nt;
    c.tris.assign(tris, tris + 3 * (size_t)nt);
    DirEdges tri_of(n, tris, nt);    // directed edge -> 3 t + position
    DirEdges edge_of(n, tris, nt);   // (a, b), a < b -> edge index
    for (int t = 0; t < nt; ++t) {
        const int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        for (int k = 0; k < 3; ++k) {
            const int a = v[k], b = v[(k + 1) % 3];
            tri_of.put(a, b, 3 * t + k);
            if (a < b) {
                edge_of.put(a, b, (int)c.edges.size());
                c.edges.push_back(make_int4(a, b, third.at(a, b), third.at(b, a)));
            }
        }
    }
    auto edge_id = [&](int u, int v) { return edge_of.at(std::min(u, v), std::max(u, v)); };
    c.ring_off.resize(n);
    c.valence.resize(n);
    for (int i = 0; i < n; ++i) {
        const std::vector<int>& r = topo->ringv[i];
        const int k = (int)r.size();
        c.ring_off[i] = (int)c.slots.size();
        c.valence[i] = k;
        for (int j = 0; j < k; ++j) {
            // slot j: triangle (i, nb, nx), edge (i, nb), opposite edge (nb, nx)
            const int nb = r[j], nx = r[(j + 1) % k];
            const int tk = tri_of.at(i, nb);
            const int role1 = i < nb ? 0 : 1;    // i is a or b of edge (i, nb)
            const int role2 = nb < nx ? 2 : 3;   // i is c or d of edge (nb, nx)
            c.slots.push_back(make_int4(tk, 4 * edge_id(i, nb) + role1, 4 * edge_id(nb, nx) + role2, tk / 3));
        }
    }
    return nullptr;
}
}  // namespace

lb_status ibm_check_mesh(const double* rest_xyz, int n, const int32_t* tris, int nt, char* why, int why_len) {
    std::unique_ptr<MeshTopology> topo;
    const char* err = mesh_topology(rest_xyz, n, tris, nt, topo);
    if (err) context_free_error(LB_ERR_ARG, err);
    if (why && why_len > 0) {
        std::strncpy(why, err ? err : "", (size_t)why_len - 1);
        why[why_len - 1] = '\0';
    }
    return err ? LB_ERR_ARG : LB_OK;
}

lb_status ibm_add_mesh(lb_ctx* ctx, const double* rest_xyz, int n, const int32_t* tris, int nt,
                       const ibm_moduli* mod, int* mesh_id) {
    LB_GUARD(ctx);
    if (ctx->started || ctx->committed) return fail(ctx, LB_ERR_STATE, "meshes must be added before the first step");
    if (!mod) return fail(ctx, LB_ERR_ARG, "null moduli");
    const double mv[5] = {mod->ks, mod->kb, mod->kal, mod->kag, mod->kv};
    for (double v : mv)
        if (!std::isfinite(v)) return fail(ctx, LB_ERR_ARG, "moduli must be finite");
    // the connectivity: from the context's cache when a mesh with the same
    // triangles was added before (then only the positions are checked)
    if (!rest_xyz || !tris || n < 4 || nt < 4) return fail(ctx, LB_ERR_ARG, "mesh needs >= 4 nodes and triangles");
    const MeshConn* conn = nullptr;
    for (const auto& c : ctx->conn_cache)
        if (c->n == n && c->nt == nt && std::memcmp(c->tris.data(), tris, sizeof(int32_t) * 3 * (size_t)nt) == 0) {
            conn = c.get();
            break;
        }
    double S0 = 0.0, V0 = 0.0;
    if (conn) {
        if (const char* err = mesh_geometry(rest_xyz, n, tris, nt, S0, V0)) return fail(ctx, LB_ERR_ARG, err);
    } else {
        std::unique_ptr<MeshConn> c(new MeshConn);
        if (const char* err = build_conn(rest_xyz, n, tris, nt, *c, S0, V0)) return fail(ctx, LB_ERR_ARG, err);
        ctx->conn_cache.push_back(std::move(c));
        conn = ctx->conn_cache.back().get();
    }
    const double* x = rest_xyz;
    const int node0 = (int)ctx->hq0.size();
    const int cell = (int)ctx->hcells.size();
    const int tri0 = ctx->n_tris_staged;
    for (int i = 0; i < n; ++i) {
        Q4 q;   // fixed-point rest position
        q.x = to_fixed(x[3 * i]);
        q.y = to_fixed(x[3 * i + 1]);
        q.z = to_fixed(x[3 * i + 2]);
        q.w = 0;
        ctx->hq0.push_back(q);
        ctx->hq.push_back(q);
    }
    ctx->hrest.insert(ctx->hrest.end(), x, x + 3 * (size_t)n);
    // the element and ring tables are written when the context commits
    // (every mesh's ranges at once, on host threads)
    PendingMesh pm;
    pm.conn = conn;
    pm.node0 = node0;
    pm.tri0 = tri0;
    pm.e0 = ctx->n_edges_staged;
    pm.slot0 = ctx->n_slots_staged;
    pm.cell = cell;
    pm.ch = ctx->cur;
    pm.ks = (float)mod->ks;
    pm.kb = (float)mod->kb;
    ctx->pending_meshes.push_back(pm);
    ctx->n_tris_staged += nt;
    ctx->n_edges_staged += (int)conn->edges.size();
    ctx->n_slots_staged += (int)conn->slots.size();
    CellDev cd;
    std::memset(&cd, 0, sizeof(cd));
    cd.ch = ctx->cur;
    cd.ref = node0;
    cd.node0 = node0;
    cd.n_nodes = n;
    cd.chunk0 = (int)ctx->hchunks.size();
    const int nch = (nt + CHUNK_TRIS - 1) / CHUNK_TRIS;
    for (int b = 0; b < nt; b += CHUNK_TRIS)
        ctx->hchunks.push_back(make_int4(cell, tri0 + b, tri0 + std::min(nt, b + CHUNK_TRIS), nch));
    cd.n_chunks = nch;
    cd.ks = (float)mod->ks; cd.kb = (float)mod->kb; cd.kal = (float)mod->kal; cd.kag = (float)mod->kag; cd.kv = (float)mod->kv;
    cd.S0 = S0;
    cd.V0 = V0;
    cd.kag_S0 = (float)(mod->kag / S0);
    cd.kv_6V0 = (float)(mod->kv / (6.0 * V0));
    ctx->hcells.push_back(cd);
    MeshHost mh;
    mh.ch = ctx->cur; mh.node0 = node0; mh.n = n; mh.tri0 = tri0; mh.nt = nt; mh.cell = cell; mh.S0 = S0; mh.V0 = V0;
    ctx->meshes.push_back(mh);
    ctx->ch_meshes[ctx->cur].push_back((int)ctx->meshes.size() - 1);
    if (mesh_id) *mesh_id = (int)ctx->ch_meshes[ctx->cur].size() - 1;
    return LB_OK;
}

lb_status ibm_set_nodes(lb_ctx* ctx, int mesh_id, const double* xyz) {
    LB_GUARD(ctx);
    const MeshHost* m;
    if (check_channel_mesh(ctx, mesh_id, &m) != LB_OK) return LB_ERR_ARG;
    if (!xyz) return fail(ctx, LB_ERR_ARG, "null positions");
    std::vector<Q4> q(m->n);
    for (int i = 0; i < m->n; ++i) {
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(xyz[3 * i + k]) || std::fabs(xyz[3 * i + k]) > 4.0e6)
                return fail(ctx, LB_ERR_ARG, "positions must be finite and |x| < 4e6");
        q[i].x = to_fixed(xyz[3 * i]);
        q[i].y = to_fixed(xyz[3 * i + 1]);
        q[i].z = to_fixed(xyz[3 * i + 2]);
        q[i].w = 0;
    }
    if (!ctx->committed) {
        std::copy(q.begin(), q.end(), ctx->hq.begin() + m->node0);
        return LB_OK;
    }
    const int par = (int)(ctx->step & 1);
    LB_CUDA(cudaMemcpyAsync(ctx->q[par] + m->node0, q.data(), sizeof(Q4) * m->n, cudaMemcpyHostToDevice, ctx->stream));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->dvalid = false;
    return LB_OK;
}

lb_status lb_step(lb_ctx* ctx, int n_steps) {
    LB_GUARD(ctx);
    if (n_steps < 0) return fail(ctx, LB_ERR_ARG, "n_steps < 0");
    if (n_steps == 0) return LB_OK;
    lb_status s = commit_ibm(ctx);
    if (s != LB_OK) return s;
    ctx->started = true;
    if (use_overlap(ctx)) {
        s = build_graphs_overlap(ctx);
        if (s != LB_OK) return s;
        if (!ctx->dvalid) {
            s = prepare_stencil_set(ctx);
            if (s != LB_OK) return s;
        }
        for (int k = 0; k < n_steps; ++k) {
            const int par = (int)(ctx->step & 1);
            LB_CUDA(cudaGraphLaunch(ctx->gexec_ov[par][k > 0 ? 1 : 0], ctx->stream));
            ctx->launches[0] += 1;
            ctx->launches[1] += 2;
            ctx->launches[2] += 3;
            if (k > 0) ctx->launches[3] += 1;
            ctx->step++;
        }
        // interpolation + advance of the last step
        LB_CUDA(launch_interp_advance(ibm_args(ctx, (int)((ctx->step - 1) & 1)), ctx->stream));
        ctx->launches[3] += 1;
        LB_CUDA(cudaGetLastError());
        return LB_OK;
    }
    ctx->dvalid = false;
    if (!ctx->timing) {
        s = build_graphs(ctx);
        if (s != LB_OK) return s;
    }
    for (int k = 0; k < n_steps;) {
        const int par = (int)(ctx->step & 1);
        if (ctx->timing) {
            s = enqueue_step(ctx, par);
            if (s != LB_OK) return s;
            ctx->step++;
            ++k;
            continue;
        }
        const int n = n_steps - k >= GRAPH_BLOCK ? GRAPH_BLOCK : 1;
        LB_CUDA(cudaGraphLaunch(n > 1 ? ctx->gexec_blk[par] : ctx->gexec[par], ctx->stream));
        for (int c = 0; c < 4; ++c)
            if ((ctx->M > 0 || c == 2) && !(c == 3 && ctx->W))
                ctx->launches[c] += (c == 1 && ctx->deterministic) ? 2 * n : n;   // + the fixed-point conversion
        if (ctx->M > 0 && ctx->rep_k > 0.f) ctx->launches[1] += 4 * n;   // collision kernels
        ctx->step += n;
        k += n;
    }
    LB_CUDA(cudaGetLastError());
    return LB_OK;
}

lb_status lb_set_kernel_config(lb_ctx* ctx, int nodes_per_thread, int block_size) {
    LB_GUARD(ctx);
    const K3Config c{nodes_per_thread, block_size};
    if (!k3_config_valid(ctx, c)) return fail(ctx, LB_ERR_ARG, "unsupported stream-collide variant for this lattice");
    if (c.npt == ctx->k3.npt && c.bs == ctx->k3.bs) return LB_OK;
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    apply_k3_config(ctx, c);
    drop_graphs(ctx);
    return upload_channels(ctx);
}

lb_status lb_set_prefetch(lb_ctx* ctx, int nodes_ahead) {
    LB_GUARD(ctx);
    if (nodes_ahead < 0 || nodes_ahead % 256 != 0 || nodes_ahead > (1 << 24))
        return fail(ctx, LB_ERR_ARG, "prefetch distance must be a multiple of 256 in 0..2^24");
    if (nodes_ahead == ctx->pf_nodes) return LB_OK;
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->pf_nodes = nodes_ahead;
    drop_graphs(ctx);
    return LB_OK;
}

lb_status lb_get_prefetch(lb_ctx* ctx, int* nodes_ahead) {
    LB_GUARD(ctx);
    if (nodes_ahead) *nodes_ahead = ctx->pf_nodes;
    return LB_OK;
}

lb_status lb_set_schedule(lb_ctx* ctx, int overlapped) {
    LB_GUARD(ctx);
    if (overlapped < 0 || overlapped > 2) return fail(ctx, LB_ERR_ARG, "schedule must be 0, 1 or 2");
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->overlap = overlapped == 1;
    const bool pdl = overlapped != 2;
    if (pdl != ctx->pdl) drop_graphs(ctx);
    ctx->pdl = pdl;
    ctx->dvalid = false;
    return LB_OK;
}

lb_status lb_get_schedule(lb_ctx* ctx, int* overlapped) {
    LB_GUARD(ctx);
    if (overlapped) *overlapped = use_overlap(ctx) ? 1 : ctx->pdl ? 0 : 2;
    return LB_OK;
}

lb_status lb_get_kernel_config(lb_ctx* ctx, int* nodes_per_thread, int* block_size) {
    LB_GUARD(ctx);
    if (nodes_per_thread) *nodes_per_thread = ctx->k3.npt;
    if (block_size) *block_size = ctx->k3.bs;
    return LB_OK;
}

lb_status lb_autotune(lb_ctx* ctx, int repeats, int* nodes_per_thread, int* block_size, double* ms) {
    LB_GUARD(ctx);
    if (ctx->step != 0) return fail(ctx, LB_ERR_STATE, "autotune runs only before the first step");
    if (repeats < 1) repeats = 1;
    lb_status st = commit_ibm(ctx);
    if (st != LB_OK) return st;
    cudaEvent_t e0, e1;
    LB_CUDA(cudaEventCreate(&e0));
    LB_CUDA(cudaEventCreate(&e1));
    const K3Config keep = ctx->k3;
    K3Config best = keep;
    double best_ms = 1e30;
    for (int k = 0; k < k3_config_count((int)ctx->storage); ++k) {
        const K3Config c = k3_config_at((int)ctx->storage, k);
        if (!k3_config_valid(ctx, c)) continue;
        apply_k3_config(ctx, c);
        if (ctx->ch.size() > (size_t)MAXCH_P && upload_channels(ctx) != LB_OK) return LB_ERR_CUDA;
        const LatticeArgs la = lattice_args(ctx, 0);
        cudaError_t e = k3_launch(ctx, la, c, ctx->stream);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < repeats && e == cudaSuccess; ++r) e = k3_launch(ctx, la, c, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(ctx, e, "lb_autotune");
        }
        if (t / repeats < best_ms) {
            best_ms = t / repeats;
            best = c;
        }
    }
    // then the L2 prefetch distance of the winner (variants with 1, 2 or 4
    // nodes per thread); the distance kept is the fastest, 0 on a tie
    apply_k3_config(ctx, best);
    if (ctx->ch.size() > (size_t)MAXCH_P && upload_channels(ctx) != LB_OK) return LB_ERR_CUDA;
    const int keep_pf = ctx->pf_nodes;
    int best_pf = 0;
    if (best.npt > 0) {
        const int dists[] = {0, 65536, 131072, 262144};
        double best_pf_ms = 1e30;
        for (int d : dists) {
            ctx->pf_nodes = d;
            const LatticeArgs la = lattice_args(ctx, 0);
            cudaError_t e = k3_launch(ctx, la, best, ctx->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
            for (int r = 0; r < repeats && e == cudaSuccess; ++r) e = k3_launch(ctx, la, best, ctx->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) {
                ctx->pf_nodes = keep_pf;
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(ctx, e, "lb_autotune");
            }
            if (t / repeats < 0.99 * best_pf_ms) {
                best_pf_ms = t / repeats;
                best_pf = d;
            }
        }
        if (best_pf_ms < best_ms) best_ms = best_pf_ms;
    }
    ctx->pf_nodes = best_pf;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graphs(ctx);
    st = upload_channels(ctx);
    if (st != LB_OK) return st;
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (nodes_per_thread) *nodes_per_thread = best.npt;
    if (block_size) *block_size = best.bs;
    if (ms) *ms = best_ms;
    return LB_OK;
}

lb_status lb_synchronize(lb_ctx* ctx) {
    LB_GUARD(ctx);
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    return LB_OK;
}

lb_status lb_get_step(lb_ctx* ctx, int64_t* step) {
    LB_GUARD(ctx);
    if (!step) return LB_ERR_ARG;
    *step = ctx->step;
    return LB_OK;
}

lb_status lb_get_fields(lb_ctx* ctx, float* rho, float* u, int dst_is_device) {
    LB_GUARD(ctx);
    if (!rho && !u) return LB_OK;
    const ChannelHost& c = ctx->ch[ctx->cur];
    const long long n = c.d.n;
    LatticeArgs a = lattice_args(ctx, (int)(ctx->step & 1));
    if (dst_is_device) {
        LB_CUDA(launch_fields(a, ctx->cur, rho, u, ctx->stream));
        LB_CUDA(cudaStreamSynchronize(ctx->stream));
        return LB_OK;
    }
    if (!ctx->fields_buf) {
        // one device scratch for every later call: 4 floats per node of the largest channel
        long long nmax = 0;
        for (const ChannelHost& ch : ctx->ch) nmax = std::max<long long>(nmax, ch.d.n);
        LB_CUDA(dalloc(ctx, &ctx->fields_buf, (size_t)4 * nmax));
    }
    float* buf = ctx->fields_buf;
    cudaError_t e = launch_fields(a, ctx->cur, rho ? buf : nullptr, u ? buf + n : nullptr, ctx->stream);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, buf, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, buf + n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lb_get_fields");
    return LB_OK;
}

lb_status lb_get_populations(lb_ctx* ctx, double* f) {
    LB_GUARD(ctx);
    if (!f) return LB_ERR_ARG;
    const ChannelHost& c = ctx->ch[ctx->cur];
    const long long n = c.d.n;
    float* buf = nullptr;
    LB_CUDA(dalloc(ctx, &buf, (size_t)Q * n));
    std::vector<float> h((size_t)Q * n);
    cudaError_t e = launch_pull_populations(lattice_args(ctx, (int)(ctx->step & 1)), ctx->cur, buf, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), buf, sizeof(float) * Q * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, buf);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lb_get_populations");
    std::vector<uint32_t> mask((size_t)((n + 31) / 32));
    LB_CUDA(cudaMemcpy(mask.data(), ctx->mask + c.d.base / GROUP, sizeof(uint32_t) * mask.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < Q; ++i)
        for (long long p = 0; p < n; ++p) {
            const bool solid = (mask[p >> 5] >> (p & 31)) & 1u;
            f[(size_t)i * n + p] = wgt_d(i) + (solid ? 0.0 : (double)h[(size_t)i * n + p]);
        }
    return LB_OK;
}

lb_status lb_set_populations(lb_ctx* ctx, const double* f) {
    LB_GUARD(ctx);
    if (!f) return LB_ERR_ARG;
    const ChannelHost& c = ctx->ch[ctx->cur];
    const ChannelDev& d = c.d;
    const long long n = d.n;
    for (long long k = 0; k < (long long)Q * n; ++k)
        if (!std::isfinite(f[k])) return fail(ctx, LB_ERR_ARG, "populations must be finite");
    std::vector<uint32_t> mask((size_t)((n + 31) / 32));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    LB_CUDA(cudaMemcpy(mask.data(), ctx->mask + d.base / GROUP, sizeof(uint32_t) * mask.size(), cudaMemcpyDeviceToHost));
    auto solid = [&](long long p) { return (bool)((mask[p >> 5] >> (p & 31)) & 1u); };
    // inverse of the pull step: h*_i(x) = h_i(x + e_i) where x + e_i is fluid and
    // inside the domain; otherwise h*_i(x) = h_opp(i)(x) minus the wall term.
    std::vector<float> hs((size_t)Q * n, 0.0f);
    const int dims[3] = {d.nx, d.ny, d.nz};
    for (int z = 0; z < d.nz; ++z)
        for (int y = 0; y < d.ny; ++y)
            for (int xx = 0; xx < d.nx; ++xx) {
                const long long p = xx + (long long)d.nx * (y + (long long)d.ny * z);
                if (solid(p)) continue;
                for (int i = 0; i < Q; ++i) {
                    int cc[3] = {xx + ex(i), y + ey(i), z + ez(i)};
                    bool ok = true;
                    for (int a = 0; a < 3; ++a)
                        if (cc[a] < 0 || cc[a] >= dims[a]) {
                            if (d.per[a]) cc[a] = (cc[a] + dims[a]) % dims[a];
                            else ok = false;
                        }
                    long long q = 0;
                    if (ok) {
                        q = cc[0] + (long long)d.nx * (cc[1] + (long long)d.ny * cc[2]);
                        ok = !solid(q);
                    }
                    double v;
                    if (ok) {
                        v = f[(size_t)i * n + q] - wgt_d(i);
                    } else {
                        const int o = opp(i);
                        v = f[(size_t)o * n + p] - wgt_d(o);
                        if (d.has_uw && !d.per[1]) {
                            int wall = -1;
                            if (ey(o) == 1 && y == 0) wall = 0;
                            if (ey(o) == -1 && y == d.ny - 1) wall = 1;
                            if (wall >= 0)
                                v -= 6.0 * wgt_d(o) * (ex(o) * c.p.wall_velocity[wall][0] + ey(o) * c.p.wall_velocity[wall][1] +
                                                       ez(o) * c.p.wall_velocity[wall][2]);
                        }
                    }
                    hs[(size_t)i * n + p] = (float)v;
                }
            }
    const int par = (int)(ctx->step & 1);
    const size_t eb = pop_bytes(ctx->storage);
    for (int i = 0; i < Q; ++i) {
        char* dst = (char*)ctx->h[par] + ((size_t)i * ctx->plane + d.base) * eb;
        if (ctx->storage == LB_F32) {
            LB_CUDA(cudaMemcpy(dst, hs.data() + (size_t)i * n, sizeof(float) * n, cudaMemcpyHostToDevice));
        } else {
            std::vector<uint16_t> tmp(n);
            for (long long p = 0; p < n; ++p) {
                const float s = hs[(size_t)i * n + p] * (1.0f / wgt(i));
                if (ctx->storage == LB_F16_SHIFTED) {
                    __half hv = __float2half_rn(s);
                    std::memcpy(&tmp[p], &hv, 2);
                } else {
                    __nv_bfloat16 bv = __float2bfloat16_rn(s);
                    std::memcpy(&tmp[p], &bv, 2);
                }
            }
            LB_CUDA(cudaMemcpy(dst, tmp.data(), 2 * n, cudaMemcpyHostToDevice));
        }
    }
    return LB_OK;
}

// Copy node ranges of the current positions into the page-locked staging
// buffer (adjacent ranges merged into one copy), wait once, convert.
lb_status read_positions(lb_ctx* ctx, const std::vector<const MeshHost*>& ms, double* xyz) {
    if (!ctx->committed) {
        size_t o = 0;
        for (const MeshHost* m : ms)
            for (int i = 0; i < m->n; ++i, ++o) {
                const Q4& q = ctx->hq[m->node0 + i];
                xyz[3 * o] = (double)q.x / FIX_SCALE;
                xyz[3 * o + 1] = (double)q.y / FIX_SCALE;
                xyz[3 * o + 2] = (double)q.z / FIX_SCALE;
            }
        return LB_OK;
    }
    const Q4* src = ctx->q[ctx->step & 1];
    size_t k = 0;
    while (k < ms.size()) {
        size_t e = k + 1;
        while (e < ms.size() && ms[e]->node0 == ms[e - 1]->node0 + ms[e - 1]->n) ++e;
        const int n0 = ms[k]->node0, n1 = ms[e - 1]->node0 + ms[e - 1]->n;
        LB_CUDA(cudaMemcpyAsync(ctx->hq_pinned + n0, src + n0, sizeof(Q4) * (size_t)(n1 - n0), cudaMemcpyDeviceToHost,
                                ctx->stream));
        k = e;
    }
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    size_t o = 0;
    for (const MeshHost* m : ms)
        for (int i = 0; i < m->n; ++i, ++o) {
            const Q4& q = ctx->hq_pinned[m->node0 + i];
            xyz[3 * o] = (double)q.x / FIX_SCALE;
            xyz[3 * o + 1] = (double)q.y / FIX_SCALE;
            xyz[3 * o + 2] = (double)q.z / FIX_SCALE;
        }
    return LB_OK;
}

lb_status ibm_get_nodes(lb_ctx* ctx, int mesh_id, double* xyz) {
    LB_GUARD(ctx);
    const MeshHost* m;
    if (check_channel_mesh(ctx, mesh_id, &m) != LB_OK) return LB_ERR_ARG;
    if (!xyz) return LB_ERR_ARG;
    return read_positions(ctx, {m}, xyz);
}

lb_status ibm_get_all_nodes(lb_ctx* ctx, double* xyz) {
    LB_GUARD(ctx);
    if (!xyz) return LB_ERR_ARG;
    std::vector<const MeshHost*> ms;
    for (int id : ctx->ch_meshes[ctx->cur]) ms.push_back(&ctx->meshes[id]);
    if (ms.empty()) return LB_OK;
    return read_positions(ctx, ms, xyz);
}

lb_status ibm_get_all_nodes_async(lb_ctx* ctx, double* xyz, int slot) {
    LB_GUARD(ctx);
    if (!xyz || (slot != 0 && slot != 1)) return fail(ctx, LB_ERR_ARG, "null output or slot not 0 or 1");
    lb_status st = commit_ibm(ctx);
    if (st != LB_OK) return st;
    std::vector<const MeshHost*> ms;
    for (int id : ctx->ch_meshes[ctx->cur]) ms.push_back(&ctx->meshes[id]);
    if (!ctx->rb_ev[slot]) LB_CUDA(cudaEventCreateWithFlags(&ctx->rb_ev[slot], cudaEventDisableTiming));
    if (!ms.empty()) {
        if (!ctx->d_xyz) LB_CUDA(dalloc(ctx, &ctx->d_xyz, 3 * (size_t)ctx->M));
        const Q4* src = ctx->q[ctx->step & 1];
        size_t k = 0, o = 0;
        while (k < ms.size()) {
            size_t e = k + 1;
            while (e < ms.size() && ms[e]->node0 == ms[e - 1]->node0 + ms[e - 1]->n) ++e;
            const int n0 = ms[k]->node0, n1 = ms[e - 1]->node0 + ms[e - 1]->n;
            LB_CUDA(launch_positions_to_double(src + n0, n1 - n0, ctx->d_xyz + 3 * (size_t)n0, ctx->stream));
            LB_CUDA(cudaMemcpyAsync(xyz + 3 * o, ctx->d_xyz + 3 * (size_t)n0, sizeof(double) * 3 * (size_t)(n1 - n0),
                                    cudaMemcpyDeviceToHost, ctx->stream));
            o += (size_t)(n1 - n0);
            k = e;
        }
    }
    LB_CUDA(cudaEventRecord(ctx->rb_ev[slot], ctx->stream));
    return LB_OK;
}

lb_status lb_readback_wait(lb_ctx* ctx, int slot) {
    LB_GUARD(ctx);
    if (slot != 0 && slot != 1) return fail(ctx, LB_ERR_ARG, "slot not 0 or 1");
    if (!ctx->rb_ev[slot]) return LB_OK;
    LB_CUDA(cudaEventSynchronize(ctx->rb_ev[slot]));
    return LB_OK;
}

lb_status ibm_get_forces(lb_ctx* ctx, int mesh_id, double* f) {
    LB_GUARD(ctx);
    const MeshHost* m;
    if (check_channel_mesh(ctx, mesh_id, &m) != LB_OK) return LB_ERR_ARG;
    if (!f) return LB_ERR_ARG;
    lb_status s = commit_ibm(ctx);
    if (s != LB_OK) return s;
    std::vector<float4> F(m->n);
    LB_CUDA(cudaMemcpyAsync(F.data(), ctx->F + m->node0, sizeof(float4) * m->n, cudaMemcpyDeviceToHost, ctx->stream));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < m->n; ++i) {
        f[3 * i] = F[i].x;
        f[3 * i + 1] = F[i].y;
        f[3 * i + 2] = F[i].z;
    }
    return LB_OK;
}

lb_status ibm_get_area_volume(lb_ctx* ctx, double* area, double* volume) {
    LB_GUARD(ctx);
    lb_status s = commit_ibm(ctx);
    if (s != LB_OK) return s;
    const auto& ids = ctx->ch_meshes[ctx->cur];
    if (ids.empty()) return LB_OK;
    LB_CUDA(launch_cell_sums(ibm_args(ctx, (int)(ctx->step & 1)), ctx->stream));
    std::vector<double2> cs(ctx->C);
    LB_CUDA(cudaMemcpyAsync(cs.data(), ctx->cell_sums, sizeof(double2) * ctx->C, cudaMemcpyDeviceToHost, ctx->stream));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (size_t k = 0; k < ids.size(); ++k) {
        const MeshHost& m = ctx->meshes[ids[k]];
        if (area) area[k] = m.S0 + cs[m.cell].x;
        if (volume) volume[k] = m.V0 + cs[m.cell].y;
    }
    return LB_OK;
}

lb_status lb_diagnostics(lb_ctx* ctx, double u_max, double out[6]) {
    LB_GUARD(ctx);
    if (!out) return LB_ERR_ARG;
    const ChannelHost& c = ctx->ch[ctx->cur];
    LB_CUDA(launch_diagnostics(lattice_args(ctx, (int)(ctx->step & 1)), ctx->cur, ctx->diag_partials,
                               ctx->diag_blocks, ctx->diag_out, ctx->stream));
    LB_CUDA(cudaMemcpyAsync(out, ctx->diag_out, sizeof(double) * 6, cudaMemcpyDeviceToHost, ctx->stream));
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (out[4] > 0) return fail(ctx, LB_ERR_NUMERIC, "non-finite populations");
    int serr = 0;
    if (ctx->rep_err) {
        LB_CUDA(cudaMemcpy(&serr, ctx->rep_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (serr > 0) return fail(ctx, LB_ERR_STATE, "collision candidate lists overflowed (more than 32 neighbour cells or 256 beads)");
    }
    int serr2[2] = {0, 0};
    LB_CUDA(cudaMemcpy(serr2, ctx->sched_err, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    if (serr2[0] > 0)
        return fail(ctx, LB_ERR_NUMERIC, "an IB point moved a lattice unit or more in one step (overlapped schedule)");
    if (serr2[1] > 0) return fail(ctx, LB_ERR_TIMEOUT, "a TMA-staged stream-collide block gave up waiting for its copies");
    if (u_max > 0 && !(out[5] <= u_max)) return fail(ctx, LB_ERR_NUMERIC, "velocity above the stability bound");
    return LB_OK;
}

// ---- checkpoint ----
namespace {
struct StateHeader {
    uint64_t magic;
    int64_t step;
    int64_t Ntot;
    int32_t storage;
    int32_t M;
    int32_t massive;   // 1: points with mass; their velocities W and the fluid
                       // velocity u of the last collision (read by the next
                       // spreading) follow F
    int32_t reserved;
};
constexpr uint64_t STATE_MAGIC = 0x4c4249424d535432ULL;
}  // namespace

lb_status lb_save_state(lb_ctx* ctx, void* buf, size_t* bytes) {
    LB_GUARD(ctx);
    if (!bytes) return LB_ERR_ARG;
    lb_status s = commit_ibm(ctx);
    if (s != LB_OK) return s;
    const size_t hb = (size_t)Q * ctx->plane * pop_bytes(ctx->storage);
    const size_t gb = (size_t)ctx->Ntot * sizeof(float4);
    const size_t fb = (size_t)ctx->Ntot / GROUP;
    const size_t qb = (size_t)ctx->M * sizeof(Q4);
    const size_t Fb = (size_t)ctx->M * sizeof(float4);
    const size_t Wb = ctx->W ? Fb : 0;
    const size_t ub = ctx->W ? (size_t)ctx->Ntot * sizeof(float4) : 0;
    const size_t total = sizeof(StateHeader) + hb + gb + fb + qb + Fb + Wb + ub;
    if (!buf) { *bytes = total; return LB_OK; }
    if (*bytes < total) return fail(ctx, LB_ERR_ARG, "checkpoint buffer too small");
    StateHeader hd{STATE_MAGIC, ctx->step, ctx->Ntot, (int32_t)ctx->storage, ctx->M, ctx->W ? 1 : 0, 0};
    char* p = (char*)buf;
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const int par = (int)(ctx->step & 1);
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    LB_CUDA(cudaMemcpy(p, ctx->h[par], hb, cudaMemcpyDeviceToHost)); p += hb;
    LB_CUDA(cudaMemcpy(p, ctx->g[1 - par], gb, cudaMemcpyDeviceToHost)); p += gb;
    LB_CUDA(cudaMemcpy(p, ctx->fl[1 - par], fb, cudaMemcpyDeviceToHost)); p += fb;
    if (ctx->M) {
        LB_CUDA(cudaMemcpy(p, ctx->q[par], qb, cudaMemcpyDeviceToHost)); p += qb;
        LB_CUDA(cudaMemcpy(p, ctx->F, Fb, cudaMemcpyDeviceToHost)); p += Fb;
        if (ctx->W) {
            LB_CUDA(cudaMemcpy(p, ctx->W, Wb, cudaMemcpyDeviceToHost)); p += Wb;
            LB_CUDA(cudaMemcpy(p, ctx->u, ub, cudaMemcpyDeviceToHost)); p += ub;
        }
    }
    *bytes = total;
    return LB_OK;
}

lb_status lb_load_state(lb_ctx* ctx, const void* buf, size_t bytes) {
    LB_GUARD(ctx);
    if (!buf || bytes < sizeof(StateHeader)) return LB_ERR_ARG;
    lb_status s = commit_ibm(ctx);
    if (s != LB_OK) return s;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != STATE_MAGIC || hd.Ntot != ctx->Ntot || hd.storage != (int32_t)ctx->storage || hd.M != ctx->M ||
        hd.massive != (ctx->W ? 1 : 0))
        return fail(ctx, LB_ERR_ARG, "checkpoint does not match this context");
    const size_t hb = (size_t)Q * ctx->plane * pop_bytes(ctx->storage);
    const size_t gb = (size_t)ctx->Ntot * sizeof(float4);
    const size_t fb = (size_t)ctx->Ntot / GROUP;
    const size_t qb = (size_t)ctx->M * sizeof(Q4);
    const size_t Fb = (size_t)ctx->M * sizeof(float4);
    const size_t Wb = ctx->W ? Fb : 0;
    const size_t ub = ctx->W ? (size_t)ctx->Ntot * sizeof(float4) : 0;
    if (bytes < sizeof(StateHeader) + hb + gb + fb + qb + Fb + Wb + ub)
        return fail(ctx, LB_ERR_ARG, "checkpoint truncated");
    const char* p = (const char*)buf + sizeof(hd);
    ctx->step = hd.step;
    const int par = (int)(ctx->step & 1);
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    LB_CUDA(cudaMemcpy(ctx->h[par], p, hb, cudaMemcpyHostToDevice)); p += hb;
    LB_CUDA(cudaMemcpy(ctx->g[1 - par], p, gb, cudaMemcpyHostToDevice)); p += gb;
    LB_CUDA(cudaMemcpy(ctx->fl[1 - par], p, fb, cudaMemcpyHostToDevice)); p += fb;
    LB_CUDA(cudaMemset(ctx->g[par], 0, gb));
    LB_CUDA(cudaMemset(ctx->fl[par], 0, fb));
    if (ctx->M) {
        LB_CUDA(cudaMemcpy(ctx->q[par], p, qb, cudaMemcpyHostToDevice)); p += qb;
        LB_CUDA(cudaMemcpy(ctx->F, p, Fb, cudaMemcpyHostToDevice)); p += Fb;
        if (ctx->W) {
            LB_CUDA(cudaMemcpy(ctx->W, p, Wb, cudaMemcpyHostToDevice)); p += Wb;
            LB_CUDA(cudaMemcpy(ctx->u, p, ub, cudaMemcpyHostToDevice)); p += ub;
        }
        ctx->dvalid = false;
    }
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->started = ctx->step > 0 || ctx->started;
    return LB_OK;
}

// ---- timing ----
lb_status lb_set_timing(lb_ctx* ctx, int kernel_mask) {
    LB_GUARD(ctx);
    if (kernel_mask < 0 || kernel_mask > 15) return fail(ctx, LB_ERR_ARG, "timing mask outside 0..15");
    ctx->timing = kernel_mask;
    return LB_OK;
}

lb_status lb_kernel_times(lb_ctx* ctx, double ms[4], int64_t launches[4]) {
    LB_GUARD(ctx);
    LB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& ep : ctx->pending) {
        float t = 0.f;
        LB_CUDA(cudaEventElapsedTime(&t, ep.a, ep.b));
        ctx->ms[ep.cls] += t;
        ctx->free_events.push_back(ep.a);
        ctx->free_events.push_back(ep.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = ctx->ms[k];
        if (launches) launches[k] = ctx->launches[k];
        ctx->ms[k] = 0;
        ctx->launches[k] = 0;
    }
    return LB_OK;
}

}  // extern "C"
