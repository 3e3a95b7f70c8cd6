// Collisions between cells and with walls and beads (Gusenbauer et al.,
// arXiv:1110.0995, Sec. 2.4: a soft potential between mesh nodes of different
// cells and between cells and walls, cut at an interaction radius; form and
// constants not printed).  Reading: harmonic soft sphere, a force
// k (d_c - d) along the separation for d < d_c, between
//   * nodes of different cells of the same channel (equal and opposite,
//     x minimum image on a periodic axis),
//   * a node and a bead surface (d = |x - c| - r),
//   * a node and a wall of a non-periodic axis (walls half a link outside the
//     first and last lattice node).
// Per step: each cell's bounding sphere (k_rep_bounds), candidate cell pairs
// and cell-bead pairs from the bounding spheres (k_rep_pairs), node-node forces
// for each ordered candidate pair, one block per pair with the partner's nodes
// staged in shared memory (k_rep_nodes), then node-bead and node-wall forces
// (k_rep_walls_beads).  The result R is added to the membrane forces before
// spreading.  Distances come from exact fixed-point differences.
#include "lbibm_internal.cuh"

namespace lbibm {

__device__ __forceinline__ float rfx(long long v) {   // v * 2^-40 (|v| < 2^51)
    const int hi = (int)(v >> 20);
    const int lo = (int)(v & 0xFFFFF);
    return fmaf((float)hi, 9.5367431640625e-07f, (float)lo * FIX_INV_F);
}

__device__ __forceinline__ const ChannelDev& rchan(const RepArgs& a, int c) {
    return c < MAXCH_P ? a.chp[c] : a.ch[c];
}

__device__ __forceinline__ float min_image(float d, int per, int n) {
    return per ? d - (float)n * rintf(d / (float)n) : d;
}

// (1) bounding sphere of every cell: centre (relative to the reference node,
// plus the reference node's absolute position) and radius.
__global__ void k_rep_bounds(const __grid_constant__ RepArgs a) {
    const CellDev& C = a.cells[blockIdx.x];
    const Q4 qr = a.q[C.ref];
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int i = threadIdx.x; i < C.n_nodes; i += blockDim.x) {
        const Q4 q = a.q[C.node0 + i];
        sx += rfx(q.x - qr.x); sy += rfx(q.y - qr.y); sz += rfx(q.z - qr.z);
    }
    __shared__ float sh[3][32];
    __shared__ float cen[3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) { sh[0][wid] = sx; sh[1][wid] = sy; sh[2][wid] = sz; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t[3] = {0.f, 0.f, 0.f};
        for (int w = 0; w < (int)blockDim.x / 32; ++w)
            for (int d = 0; d < 3; ++d) t[d] += sh[d][w];
        for (int d = 0; d < 3; ++d) cen[d] = t[d] / (float)C.n_nodes;
    }
    __syncthreads();
    float r2 = 0.f;
    for (int i = threadIdx.x; i < C.n_nodes; i += blockDim.x) {
        const Q4 q = a.q[C.node0 + i];
        const float dx = rfx(q.x - qr.x) - cen[0], dy = rfx(q.y - qr.y) - cen[1], dz = rfx(q.z - qr.z) - cen[2];
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    __syncthreads();
    if (lane == 0) sh[0][wid] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) m = fmaxf(m, sh[0][w]);
        // absolute centre as float (a coarse test with a margin; distances
        // between nodes themselves use fixed point)
        a.bounds[blockIdx.x] = make_float4(rfx(qr.x) + cen[0], rfx(qr.y) + cen[1], rfx(qr.z) + cen[2], sqrtf(m));
    }
}

// (2) candidate pairs: threads [0, C*C) test ordered cell pairs (a != b, same
// channel), threads [C*C, C*C + C*nb) test (cell, bead) pairs.  Margin 0.5 lu
// covers the float rounding of the absolute centres.
__global__ void k_rep_pairs(const __grid_constant__ RepArgs a) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nC = a.n_cells;
    const long long np = nC * nC;
    if (t < np) {
        const int ca = (int)(t / nC), cb = (int)(t - (t / nC) * nC);
        if (ca == cb || a.cells[ca].ch != a.cells[cb].ch) return;
        const ChannelDev& Ch = rchan(a, a.cells[ca].ch);
        const float4 A = a.bounds[ca], B = a.bounds[cb];
        const float dx = min_image(A.x - B.x, Ch.per[0], Ch.nx), dy = min_image(A.y - B.y, Ch.per[1], Ch.ny),
                    dz = min_image(A.z - B.z, Ch.per[2], Ch.nz);
        const float lim = A.w + B.w + a.dc + 0.5f;
        if (dx * dx + dy * dy + dz * dz < lim * lim) {
            const int k = atomicAdd(a.pair_count, 1);
            if (k < a.pair_cap) a.pairs[k] = make_int2(ca, cb);
            else atomicAdd(a.err, 1);
        }
    } else if (t < np + nC * a.n_beads) {
        const long long u = t - np;
        const int c = (int)(u / a.n_beads), b = (int)(u - (u / a.n_beads) * a.n_beads);
        if (a.bead_ch[b] != a.cells[c].ch) return;
        const ChannelDev& Ch = rchan(a, a.cells[c].ch);
        const float4 A = a.bounds[c];
        const Q4 bq = a.bead_q[b];
        const float dx = min_image(A.x - rfx(bq.x), Ch.per[0], Ch.nx), dy = min_image(A.y - rfx(bq.y), Ch.per[1], Ch.ny),
                    dz = min_image(A.z - rfx(bq.z), Ch.per[2], Ch.nz);
        const float lim = A.w + a.bead_r[b] + a.dc + 0.5f;
        if (dx * dx + dy * dy + dz * dz < lim * lim) {
            const int k = atomicAdd(a.near_count + c, 1);
            if (k < REP_NEARB) a.near[c * REP_NEARB + k] = b;
            else atomicAdd(a.err, 1);
        }
    }
}

// (3) node-node forces of ordered candidate pairs (a, b): forces on a's nodes,
// b's nodes staged in shared memory relative to a's reference node.
constexpr int RN_THREADS = 256;
constexpr int RN_TILE = 512;

__global__ void __launch_bounds__(RN_THREADS) k_rep_nodes(const __grid_constant__ RepArgs a) {
    __shared__ float3 tile[RN_TILE];
    const int n_pairs = min(*a.pair_count, a.pair_cap);
    const float k = a.k, dc = a.dc, dc2 = a.dc * a.dc;
    for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        const int2 pr = a.pairs[p];
        const CellDev& A = a.cells[pr.x];
        const CellDev& B = a.cells[pr.y];
        const ChannelDev& Ch = rchan(a, A.ch);
        const Q4 qr = a.q[A.ref];
        for (int i0 = 0; i0 < A.n_nodes; i0 += RN_THREADS) {
            const int i = i0 + threadIdx.x;
            float3 xi = make_float3(0.f, 0.f, 0.f);
            if (i < A.n_nodes) {
                const Q4 q = a.q[A.node0 + i];
                xi = make_float3(rfx(q.x - qr.x), rfx(q.y - qr.y), rfx(q.z - qr.z));
            }
            float fx = 0.f, fy = 0.f, fz = 0.f;
            for (int j0 = 0; j0 < B.n_nodes; j0 += RN_TILE) {
                __syncthreads();
                for (int j = threadIdx.x; j < RN_TILE && j0 + j < B.n_nodes; j += RN_THREADS) {
                    const Q4 q = a.q[B.node0 + j0 + j];
                    tile[j] = make_float3(rfx(q.x - qr.x), rfx(q.y - qr.y), rfx(q.z - qr.z));
                }
                __syncthreads();
                const int nj = min(RN_TILE, B.n_nodes - j0);
                if (i < A.n_nodes) {
                    for (int j = 0; j < nj; ++j) {
                        const float3 xj = tile[j];
                        const float dx = min_image(xi.x - xj.x, Ch.per[0], Ch.nx);
                        const float dy = min_image(xi.y - xj.y, Ch.per[1], Ch.ny);
                        const float dz = min_image(xi.z - xj.z, Ch.per[2], Ch.nz);
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        if (d2 < dc2 && d2 > 0.f) {
                            const float d = sqrtf(d2);
                            const float f = k * (dc - d) / d;
                            fx += f * dx; fy += f * dy; fz += f * dz;
                        }
                    }
                }
            }
            if (i < A.n_nodes && (fx != 0.f || fy != 0.f || fz != 0.f)) {
                float* r = reinterpret_cast<float*>(a.R + A.node0 + i);
                atomicAdd(r, fx);
                atomicAdd(r + 1, fy);
                atomicAdd(r + 2, fz);
            }
        }
    }
}

// (4) node-bead (the cell's candidate beads) and node-wall forces.
__global__ void k_rep_walls_beads(const __grid_constant__ RepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_nodes) return;
    const int c = a.info[i].x;
    const CellDev& C = a.cells[c];
    const ChannelDev& Ch = rchan(a, C.ch);
    const Q4 q = a.q[i];
    const float k = a.k, dc = a.dc;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int nb = min(a.near_count[c], REP_NEARB);
    for (int t = 0; t < nb; ++t) {
        const int b = a.near[c * REP_NEARB + t];
        const Q4 bq = a.bead_q[b];
        const float dx = min_image(rfx(q.x - bq.x), Ch.per[0], Ch.nx);
        const float dy = min_image(rfx(q.y - bq.y), Ch.per[1], Ch.ny);
        const float dz = min_image(rfx(q.z - bq.z), Ch.per[2], Ch.nz);
        const float d2 = dx * dx + dy * dy + dz * dz;
        const float rr = a.bead_r[b] + dc;
        if (d2 < rr * rr && d2 > 0.f) {
            const float d = sqrtf(d2);
            const float f = k * (dc - (d - a.bead_r[b])) / d;
            fx += f * dx; fy += f * dy; fz += f * dz;
        }
    }
    // walls at -1/2 and n - 1/2 on the non-periodic axes
    const long long half = 1LL << (FIX_BITS - 1);
    const long long qq[3] = {q.x, q.y, q.z};
    const int n[3] = {Ch.nx, Ch.ny, Ch.nz};
    float fw[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (Ch.per[d]) continue;
        const float lo = rfx(qq[d] + half);
        const float hi = rfx(((long long)n[d] << FIX_BITS) - half - qq[d]);
        if (lo < dc) fw[d] += k * (dc - lo);
        if (hi < dc) fw[d] -= k * (dc - hi);
    }
    float4 r = a.R[i];
    r.x += fx + fw[0];
    r.y += fy + fw[1];
    r.z += fz + fw[2];
    a.R[i] = r;
}

cudaError_t launch_repulsion(const RepArgs& a, int sm_count, cudaStream_t s) {
    if (a.n_cells <= 0) return cudaSuccess;
    k_rep_bounds<<<a.n_cells, 256, 0, s>>>(a);
    const long long np = (long long)a.n_cells * a.n_cells + (long long)a.n_cells * a.n_beads;
    k_rep_pairs<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(a);
    k_rep_nodes<<<2 * sm_count, RN_THREADS, 0, s>>>(a);
    k_rep_walls_beads<<<(a.n_nodes + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbibm
