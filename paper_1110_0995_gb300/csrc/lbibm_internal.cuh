// Internal declarations of the GB300 lattice-Boltzmann + immersed-boundary
// library: device data layout, kernel argument blocks and launchers.
//
// Data layout in HBM (one context = one batch of channels):
//   populations  h[2][19][Ntot]   SoA, direction-major; Ntot is the padded sum
//                                 of all channels' node counts; channel k's
//                                 nodes start at a multiple of CH_ALIGN.
//                                 Storage type float (h = f - w), half or
//                                 bfloat16 (h / w).  Step parity p reads
//                                 h[p] and writes h[1-p] (pull scheme).
//   obstacle mask uint32[Ntot/32] one bit per node (1 = solid)
//   slow flags   uint8[Ntot/32]   nonzero if a node of the 32-node group is
//                                 solid or has a link leaving the domain or
//                                 ending on a solid node (bit 0 wall, bit 1 obstacle)
//   link masks   uint32[Ntot]     per node: bit i = population i is bounced
//                                 back, bit 0 = node solid; read only by the
//                                 warps of slow groups
//   force fields float4 g[2][Ntot] IB force density (x, y, z, 0), double-
//                                 buffered by step parity, sparse in use
//   force flags  uint8[2][Ntot/32] group's g[parity] holds forces of the step
//                                 with that parity; cleared by the warp that
//                                 owns the group one step later
//   velocity     float4 u[Ntot]   (ux, uy, uz, rho), written only for flagged
//                                 groups (the stencils of the IB points)
//   IB nodes     int64 q[2][M]x4  positions in 2^-40 lu fixed point (by parity)
//                int64 q0[M]x4    rest positions
//                int4 info        (cell, reference node, ring offset, valence | channel << 8)
//   ring CSR     int4 per slot of a node's ring: where the node's share of the
//                incident triangle, edge and opposite edge lies in the
//                element outputs below
//   edges        int4 (a, b, c, d), a < b: edge (a, b) between triangles
//                (a, b, c) and (b, a, d); float4 (L0, theta0, ks, kb)
//   element outputs (rewritten every step, read by the node gather):
//                float4 eS[E]     stretching force on a (on b: its negative)
//                float4 eB[4E]    bending force on a, b, c, d
//                float4 tA[3T]    area direction a_k of vertex k, .w = kal dS_t/S0_t
//                float4 tN[T]     unnormalised outward normal of the triangle
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <utility>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbibm {

// ---- programmatic dependent launch ----
// A kernel of the cycle may be launched before its predecessor in the stream
// has finished.  pdl_wait returns once the predecessor has completed and its
// writes are visible; pdl_trigger, issued by every block only after its
// pdl_wait, lets the next kernel be scheduled.  So when a kernel starts, every
// kernel before its predecessor has completed: before pdl_wait it may read
// anything but what its immediate predecessor writes.  Both are no-ops for a
// kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_entry() {
    pdl_wait();
    pdl_trigger();
}

template <typename... K, typename... A>
inline cudaError_t launch_ex(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                             A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}


constexpr int Q = 19;
constexpr int GROUP = 32;           // nodes per mask word / flag
// Channel node ranges start at, and are padded to, multiples of this.  Every
// stream-collide block covers whole groups inside one channel's padded range,
// so lanes past the channel's end still index valid flag / mask words.
constexpr int CH_ALIGN = 2048;
constexpr int MAXCH_P = 32;         // channels carried in the kernel parameter block
constexpr double FIX_SCALE = 1099511627776.0;   // 2^40
constexpr float FIX_SCALE_F = 1099511627776.0f;
constexpr float FIX_INV_F = 9.094947017729282e-13f;  // 2^-40
constexpr int FIX_BITS = 40;
constexpr int SUB = 8;              // lanes per IB node in the node-parallel kernels

// Exact division of 31-bit non-negative integers by a fixed divisor d >= 1 via
// multiply-high (Granlund-Montgomery, round-up variant): with l = ceil(log2 d)
// and m = ceil(2^(31+l) / d), floor(n / d) = (n * m) >> (31 + l) for n < 2^31.
struct FastDiv {
    unsigned m;
    int s;   // l - 1, or -1 for d == 1
};

inline FastDiv make_fastdiv(int d) {
    FastDiv f;
    if (d <= 1) {
        f.m = 0;
        f.s = -1;
        return f;
    }
    int l = 0;
    while ((1LL << l) < d) ++l;
    const unsigned long long num = 1ULL << (31 + l);
    f.m = (unsigned)((num + (unsigned long long)d - 1) / (unsigned long long)d);
    f.s = l - 1;
    return f;
}

__device__ __forceinline__ int fdiv(int n, FastDiv f) {
    return f.s < 0 ? n : (int)(__umulhi((unsigned)n, f.m) >> f.s);
}

struct ChannelDev {
    int nx, ny, nz;
    FastDiv dnx, dny;     // division by nx and by ny
    int per[3];
    long long base;       // first global node index
    int n;                // nx * ny * nz (< 2^31)
    int blk0;             // first block of the stream-collide grid for this channel
    int sg0;              // first row group of the staged stream-collide variant
    int srows;            // rows per staged group (0: channel not stageable)
    float omega;          // 1 / tau
    float fpre;           // 1 - 1 / (2 tau)
    float G[3];           // uniform body force
    float uw[2][3];       // y-low / y-high wall velocity
    int has_uw;
};

struct __align__(32) Q4 {
    long long x, y, z, w;
};

struct CellDev {
    int ch;               // channel
    int ref;              // global index of the reference node (first node of the cell)
    int node0, n_nodes;
    int chunk0, n_chunks; // triangle chunks of the area/volume reduction
    float ks, kb, kal, kag, kv;
    float kag_S0, kv_6V0; // kag / S0 and kv / (6 V0) in FP32
    float pad;
    double S0, V0;        // rest area and volume (FP64)
};

struct LatticeArgs {
    const ChannelDev* ch; // all channels (global memory)
    int n_ch;
    int pdl;              // launched as a programmatic dependent of the previous kernel
    int storage;          // lb_storage
    int par;              // step parity: read h[par], write h[1-par]; forces in g[par]
    int has_last;         // a step has completed (fields / diagnostics)
    void* h0;
    void* h1;
    long long Ntot;
    const uint32_t* mask;
    const uint8_t* slow;
    const uint32_t* links;  // [Ntot] bounce-back link mask per node (bit 0: solid)
    float4* g0;
    float4* g1;
    uint8_t* fl0;
    uint8_t* fl1;
    float4* u;
    int n_groups;         // row groups of the staged stream-collide variant
    // overlapped schedule: the step's stencil set (groups that may hold IB
    // force or be interpolated) as a byte map and as a list
    const uint8_t* dmap;
    const int* dlist;
    const int* dcount;
    // differentiable variant: bead solid fraction per node (null: off) and
    // the Brinkman coefficient alpha
    const float* phi;
    float alpha;
    int* tma_err;         // TMA variant: mbarrier waits that ran out
    // stream-collide: L2 prefetch distance in lattice nodes (0: off).  A block
    // asks L2 for the source rows of the nodes pf_nodes past its own, so the
    // blocks that run a wave later find them there instead of in DRAM.
    int pf_nodes;
    ChannelDev chp[MAXCH_P];   // copy of the first channels (constant bank)
};

struct IbmArgs {
    int pdl;              // launched as a programmatic dependent of the previous kernel
    int n_nodes;          // M
    int n_cells;
    int par;              // step parity: positions q[par] are current, q[1-par] receive the advance
    int n_ch;
    const ChannelDev* ch;
    const CellDev* cells;
    const int4* info;     // [M] (cell, ref, ring offset, valence | channel << 8)
    Q4* qa;               // [M] positions, even steps
    Q4* qb;               // [M] positions, odd steps
    const Q4* q0;         // [M] rest positions
    const int4* slots;    // [K] (3 t + role in t, 4 e + role in e, 4 e' + role in e', t) per ring slot
    const int4* edges;    // [E] (a, b, c, d)
    const float4* edge_rest;  // [E] (L0, theta0, ks, kb)
    int n_edges;
    float4* eS;           // [E]
    float4* eB;           // [4E]
    float4* tA;           // [3T]
    float4* tN;           // [T]
    float4* F;            // [M] last node forces
    // area / volume reduction
    const int4* tris;     // [T] (a, b, c, cell) global node indices
    const float* tri_S0;  // [T] rest area of each triangle
    const int4* chunks;   // [NCH] (cell, t_begin, t_end, chunks of that cell)
    int n_chunks;
    longlong2* partials;  // [NCH] (dS, 6 dV) per chunk, 2^-40 units
    unsigned* counters;   // [C]
    double2* cell_sums;   // [C] (dS, dV)
    float2* cell_rel;     // [C] (dS / S0, dV / V0)
    // lattice pieces used by spread / interpolation
    const uint32_t* mask;
    float4* g0;
    float4* g1;
    uint8_t* fl0;
    uint8_t* fl1;
    const float4* u;
    const float4* R;      // [M] collision forces added to the membrane forces (null: none)
    // IB points with mass (null W: massless points advected by k_interp_advance):
    // kick V = W + F / m, drift X += U + p1 (V - U), W <- U + E (V - U), the
    // fluid receiving J = gamma p1 (V - U); U interpolated at X from u
    float4* W;            // [M] point velocities carried between steps
    float ib_inv_m, ib_gp1, ib_p1, ib_E;
    // deterministic spreading (null: float atomics): force density in 2^-40
    // fixed point, [3][gfix_stride], converted to g by k_gfix_to_g
    unsigned long long* gfix;
    long long gfix_stride;
    // overlapped schedule: map receiving the next step's stencil set, the
    // current step's set (every spread target must lie in it) and the count
    // of spread targets found outside it
    uint8_t* dmark;
    const uint8_t* dcur;
    int* sched_err;
    ChannelDev chp[MAXCH_P];
};

// Arguments of the adjoint kernels (one step of the reverse sweep of the
// differentiable variant; single channel, FP32 populations).
struct AdjArgs {
    ChannelDev ch;
    int M, n_edges, n_tris, n_beads, obj_cell;
    int n_cells;
    int pdl;                  // launched as a programmatic dependent of the previous kernel
    long long plane;          // population plane stride
    // the forward step t (recomputed and stored)
    const Q4* q_t;            // [M] positions at the start of step t
    const float4* F_t;        // [M] node forces of step t
    const float4* g_t;        // [plane] spread force density of step t
    const float4* u_t;        // [plane] velocity of step t's collision
    const float* h_t;         // [19][plane] populations at the start of step t
    const float2* rel_t;      // [C] (dS/S0, dV/V0) of step t
    const uint8_t* fl_t;      // [plane / 32] groups that received IB force in step t (the stencil groups)
    const uint32_t* mask;
    const uint32_t* links;
    const uint8_t* slow;      // per 32-node group: any bounce-back link
    const float* phi;
    float alpha, delta;
    const float4* beads;      // [n_beads] (cx, cy, cz, r)
    // adjoint state
    const float* lam_in;      // [19][plane] adjoint of step t+1's pulled populations
    float* lam_out;           // [19][plane] adjoint of step t's pulled populations
    float4* lam_u;            // [plane] adjoint of step t's velocity (from the interpolation); the
                              // stream-collide adjoint zeroes what it read
    float4* lam_g;            // [plane] adjoint of step t's force density
    float* Lphi;              // [plane] accumulated adjoint of phi
    const float4* lamX;       // [M] adjoint of X^{t+1}
    float4* lamX_out;         // [M] adjoint of X^t
    float4* lamF;             // [M] adjoint of F^t
    // membrane topology
    const int4* edges;
    const float4* edge_rest;
    const int4* tris;
    const float* tri_S0;
    const int4* info;
    const CellDev* cells;
    float4* tri_dS;           // [2T]
    float4* tri_n;            // [T]
    double* lam_c;            // [2C]
    double* grad;             // [2 + 3 n_beads] (ks, kb of the objective cell, bead centres)
};

// Arguments of the collision kernels (repulsion.cu).
constexpr int REP_NEARB = 256;      // candidate beads per cell
struct RepArgs {
    float k, dc;                    // force k (dc - d) for d < dc
    int n_cells, n_nodes, n_beads, pair_cap;
    const Q4* q;                    // current positions
    const CellDev* cells;
    const int4* info;
    const ChannelDev* ch;
    float4* bounds;                 // [C] centre (absolute), radius
    int2* pairs;                    // [pair_cap] ordered candidate cell pairs
    int* pair_count;
    int* near;                      // [C][REP_NEARB] candidate beads per cell
    int* near_count;                // [C]
    const Q4* bead_q;               // [nb] bead centres in fixed point
    const float* bead_r;            // [nb]
    const int* bead_ch;             // [nb]
    float4* R;                      // [M] collision force per node (accumulated)
    int* err;                       // candidate list overflows
    ChannelDev chp[MAXCH_P];
};

// D3Q19 velocity set (Sec. 2.1): rest, +-x, +-y, +-z, then the 12 diagonals,
// opposite directions adjacent.
__host__ __device__ constexpr int ex(int i) {
    return i == 1 || i == 7 || i == 9 || i == 11 || i == 13 ? 1 : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return i == 3 || i == 7 || i == 10 || i == 15 || i == 17 ? 1 : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18 ? -1 : 0);
}
__host__ __device__ constexpr int ez(int i) {
    return i == 5 || i == 11 || i == 14 || i == 15 || i == 18 ? 1 : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f)); }
__host__ __device__ constexpr double wgt_d(int i) { return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0)); }

// Stream-collide kernel variants: nodes per thread along x and block size.
// npt = 0 selects the staged variant (rows copied to shared memory with
// asynchronous copies, persistent grid of bs-thread blocks), npt = -1 the
// pipelined one, npt = -2 the TMA-staged one (tensor copies of every
// direction's source rows into shared memory, FP32, one channel; bs = tile).
struct K3Config {
    int npt;
    int bs;
};
constexpr int SG_NODES = 512;       // nodes per row group of the staged variant
// Rows per staged group for a row of nx nodes of `bytes`-byte populations, or 0
// when the row is not 16-byte copyable or no whole number of rows fills a
// group with a multiple of 32 nodes.
__host__ __device__ inline int staged_rows(int nx, int bytes) {
    if ((nx * bytes) % 16 != 0 || nx > SG_NODES) return 0;
    int r = SG_NODES / nx;
    while (r > 0 && (r * nx) % 32 != 0) --r;
    return r;
}
cudaError_t prepare_staged(int storage);
bool k3_config_supported(int storage, K3Config c);
int k3_config_count(int storage);
K3Config k3_config_at(int storage, int k);

// ---- launchers (defined in lattice_kernels.cu / ibm_kernels.cu) ----
cudaError_t launch_brinkman_phi(const ChannelDev& ch, const float* beads, int nb, float delta, float* phi,
                               cudaStream_t s);
cudaError_t launch_rasterise(const float* spheres, int n_spheres, const uint8_t* extra, const ChannelDev& ch,
                             uint32_t* mask, cudaStream_t s);
cudaError_t launch_slow_flags(const ChannelDev& ch, const uint32_t* mask, uint8_t* slow, uint32_t* links,
                              cudaStream_t s);
cudaError_t launch_stream_collide(const LatticeArgs& a, K3Config cfg, int total_blocks, cudaStream_t s);
// TMA-staged variant: tile geometry, descriptor encoding and launch
// (tile = nodes per tile = threads per block, 256 or 512: R = tile / nx whole rows)
bool tma_variant_ok(const ChannelDev& C, int storage, int n_ch, int tile);
cudaError_t encode_tma_maps(const ChannelDev& C, int tile, void* h0, void* h1, long long plane, CUtensorMap* maps);
int tma_blocks_per_sm(int tile);
cudaError_t launch_stream_collide_tma(const LatticeArgs& a, int tile, const CUtensorMap* maps, int blocks,
                                      cudaStream_t s);
// mode 1: bulk (groups outside a.dmap; `smem` bytes of unused dynamic shared
// memory per block cap its residency), mode 2: the first (blocks * bs / 32)
// groups of a.dlist, mode 3: the groups of a.dlist from entry `smem` on
cudaError_t launch_stream_collide_split(const LatticeArgs& a, int bs, int mode, int blocks, size_t smem,
                                        cudaStream_t s);
const void* stream_collide_bulk_func(int storage, int bs);
cudaError_t prepare_bulk(int storage, int max_smem);   // allow up to max_smem dynamic bytes per bulk block
cudaError_t launch_fields(const LatticeArgs& a, int ch_index, float* rho, float* u, cudaStream_t s);
cudaError_t launch_pull_populations(const LatticeArgs& a, int ch_index, float* h_out, cudaStream_t s);
cudaError_t launch_diagnostics(const LatticeArgs& a, int ch_index, double* partials, int n_blocks, double* out,
                               cudaStream_t s);

cudaError_t launch_cell_sums(const IbmArgs& a, cudaStream_t s);
cudaError_t launch_elements(const IbmArgs& a, cudaStream_t s);
cudaError_t launch_forces_spread(const IbmArgs& a, cudaStream_t s);
cudaError_t launch_gfix_to_g(const IbmArgs& a, cudaStream_t s);
cudaError_t launch_interp_advance(const IbmArgs& a, cudaStream_t s);
cudaError_t launch_positions_to_double(const Q4* q, int n, double* out, cudaStream_t s);

cudaError_t launch_repulsion(const RepArgs& a, int sm_count, cudaStream_t s);
cudaError_t launch_adj_interp(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_collide(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_spread(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_membrane(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_bead_grad(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_mark_stencils(const IbmArgs& a, uint8_t* map, cudaStream_t s);
cudaError_t launch_compact_groups(const uint8_t* map, int n_groups, int* list, int* count, cudaStream_t s);

}  // namespace lbibm
