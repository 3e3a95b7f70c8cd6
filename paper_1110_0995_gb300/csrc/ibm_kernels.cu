// Immersed-boundary kernels (Gusenbauer et al., arXiv:1110.0995, Sec. 2.2-2.3):
//   k_cell_sums      per-cell change of surface area and volume, FP32 per-triangle
//                    terms added as exact 2^-40 fixed-point integers (Sec. 2.3.3:
//                    the global area and volume constraints need every node of a cell)
//   k_elements       the same per-triangle pass plus each triangle's area and
//                    volume force terms, and per edge its stretching and
//                    bending forces (Sec. 2.3.1), every element evaluated once
//   k_forces_spread  node forces gathered from the element outputs of the
//                    node's ring (deterministic order, no force atomics), then
//                    spread with the trilinear delta function (Sec. 2.2 step 3)
//   k_interp_advance trilinear velocity interpolation (Sec. 2.2 step 1) and the
//                    point advance X <- X + U (massless points)
// The force kernel gives each IB node eight lanes: one ring slot and one
// stencil corner per lane, so every load of a node is in flight at once.
//
// Positions are 64-bit fixed point (2^-40 lu); element geometry is FP32 formed
// from exact fixed-point differences (see Pt below).
#include "lbibm_internal.cuh"

namespace lbibm {

__device__ __forceinline__ float3 f3(const float4& v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return make_float3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------------------
// fixed point -> FP32 with 32-bit integer and FP32 operations only (64-bit
// integer <-> float conversions run on the FP64 pipe, which GB300 keeps small)
// ---------------------------------------------------------------------------

// v * 2^-40, correctly rounded for |v| < 2^44 (16 lu), faithfully up to 2^51:
// v = hi 2^20 + lo with 0 <= lo < 2^20, both exact in FP32, one rounding.
__device__ __forceinline__ float fx(long long v) {
    const int hi = (int)(v >> 20);
    const int lo = (int)(v & 0xFFFFF);
    return fmaf((float)hi, 9.5367431640625e-07f, (float)lo * FIX_INV_F);   // 2^-20, 2^-40
}

// round(u * 2^40) for |u| < 2^15: u * 2^16 = m + f with m integral and |f| <= 1/2
// (both exact in FP32), so round(u * 2^40) = m * 2^24 + round(f * 2^24).
__device__ __forceinline__ long long float_to_fixed(float u) {
    const float s = u * 65536.0f;
    const float m = rintf(s);
    const float f = (s - m) * 16777216.0f;
    return ((long long)__float2int_rn(m) << 24) + (long long)__float2int_rn(f);
}

// One IB point for the element terms: fixed-point position q and displacement
// from rest D = q - q0.  Edge vectors and displacement differences are formed
// exactly as integer differences and rounded once (fx), so an edge is accurate
// to FP32 rounding of its own length however far the cell has moved, and
// |e|^2 - L0^2 = 2 e0.de + de.de keeps its relative accuracy when the change
// is small.
struct Pt {
    long long x, y, z;      // q
    long long dx, dy, dz;   // D
};

__device__ __forceinline__ Pt load_pt(const IbmArgs& a, const Q4* qc, int i) {
    const Q4 q = qc[i], q0 = a.q0[i];
    Pt p;
    p.x = q.x; p.y = q.y; p.z = q.z;
    p.dx = q.x - q0.x; p.dy = q.y - q0.y; p.dz = q.z - q0.z;
    return p;
}

__device__ __forceinline__ const Q4* cur_q(const IbmArgs& a) { return a.par ? a.qb : a.qa; }

// x_b - x_a
__device__ __forceinline__ float3 edge(const Pt& A, const Pt& B) {
    return make_float3(fx(B.x - A.x), fx(B.y - A.y), fx(B.z - A.z));
}
// D_b - D_a
__device__ __forceinline__ float3 ddisp(const Pt& A, const Pt& B) {
    return make_float3(fx(B.dx - A.dx), fx(B.dy - A.dy), fx(B.dz - A.dz));
}
// rest position q0_b - q0_a
__device__ __forceinline__ float3 rest_edge(const Pt& A, const Pt& B) {
    return make_float3(fx((B.x - B.dx) - (A.x - A.dx)), fx((B.y - B.dy) - (A.y - A.dy)), fx((B.z - B.dz) - (A.z - A.dz)));
}

__device__ __forceinline__ const ChannelDev& chan(const IbmArgs& a, int c) {
    return c < MAXCH_P ? a.chp[c] : a.ch[c];
}

// ---------------------------------------------------------------------------
// element terms
// ---------------------------------------------------------------------------

// The element terms divide with __fdividef and take square roots as x
// rsqrt(x) (a few ulp, against the ~10 instructions of a correctly rounded
// division; every argument is positive for a non-degenerate element).
__device__ __forceinline__ float sqrt_fast(float x) { return x * rsqrtf(x); }

// Stretching (neo-Hookean bond, Dupin et al.): tension ks kappa(lambda)(lambda-1)
// with kappa = (lambda^1/2 + lambda^-5/2)/(lambda + lambda^-3)
//            = lambda^1/2 (lambda^3 + 1)/(lambda^4 + 1);
// returns the force on a (the force on b is its negative).  a < b in global index.
__device__ __forceinline__ float3 stretch_on_a(const Pt& A, const Pt& B, float L0, float ks) {
    const float3 d = edge(A, B);
    const float3 de = ddisp(A, B);
    const float3 d0 = d - de;
    const float num = 2.0f * dot(d0, de) + dot(de, de);   // |d|^2 - |d0|^2
    const float L = sqrt_fast(L0 * L0 + num);
    const float lm1 = __fdividef(num, (L + L0) * L0);      // lambda - 1
    const float lam = 1.0f + lm1;
    const float lam2 = lam * lam;
    const float kappa = __fdividef(sqrt_fast(lam) * (lam2 * lam + 1.0f), lam2 * lam2 + 1.0f);
    const float T = ks * kappa * lm1;
    return (T * rsqrtf(dot(d, d))) * d;
}

// Bending: E = (kb/2)(theta - theta0)^2 at edge (a, b) between triangle (a, b, c)
// and triangle (b, a, d); theta = atan2((n1 x n2).e_hat, n1.n2).  Writes the
// forces on a, b, c, d (they sum to zero up to rounding).
__device__ __forceinline__ void bend_all(const Pt& A, const Pt& B, const Pt& Cc, const Pt& D, float th0,
                                         float kb, float3 f[4]) {
    const float3 e = edge(A, B);
    const float3 ac = edge(A, Cc);
    const float3 ad = edge(A, D);
    const float3 bd = ad - e;
    const float3 n1 = cross(e, ac);
    const float3 n2 = cross(-e, bd);
    const float l2 = dot(e, e);
    const float rl = rsqrtf(l2);
    const float l = l2 * rl;
    const float theta = atan2f(dot(cross(n1, n2), e) * rl, dot(n1, n2));
    const float coef = -kb * (theta - th0);
    const float3 gc = __fdividef(-l, dot(n1, n1)) * n1;
    const float3 gd = __fdividef(-l, dot(n2, n2)) * n2;
    const float il2 = __fdividef(1.0f, l2);
    const float sc = dot(ac, e) * il2;
    const float sd = dot(ad, e) * il2;
    f[0] = coef * ((-(1.0f - sc)) * gc - (1.0f - sd) * gd);
    f[1] = coef * ((-sc) * gc - sd * gd);
    f[2] = coef * gc;
    f[3] = coef * gd;
}

// Area change of triangle (0, 1, 2) from rest: S_t - S0_t from
// |n|^2 - |n0|^2 = 2 n0.dn + dn.dn, dn = a1 x b2 + b1 x a2 + b1 x b2.
__device__ __forceinline__ float tri_dS(const float3& e1, const float3& e2, const float3& b1, const float3& b2,
                                        float S0t) {
    const float3 a1 = e1 - b1, a2 = e2 - b2;
    const float3 n0 = cross(a1, a2);
    const float3 dn = cross(a1, b2) + cross(b1, a2) + cross(b1, b2);
    const float num = 2.0f * dot(n0, dn) + dot(dn, dn);
    const float nn0 = 2.0f * S0t;
    const float nn = sqrt_fast(nn0 * nn0 + num);
    return __fdividef(num, 2.0f * (nn + nn0));
}

// Volume change of the tetrahedron (reference node R, 0, 1, 2) from rest, times 6:
// (r0 + d0).((r1 + d1) x (r2 + d2)) - r0.(r1 x r2), expanded, with r_k the rest
// position and d_k the displacement of point k relative to R's.
__device__ __forceinline__ float tri_dV6(const Pt& R, const Pt& P0, const Pt& P1, const Pt& P2) {
    const float3 r0 = rest_edge(R, P0), r1 = rest_edge(R, P1), r2 = rest_edge(R, P2);
    const float3 d0 = ddisp(R, P0), d1 = ddisp(R, P1), d2 = ddisp(R, P2);
    const float3 r1r2 = cross(r1, r2), d1r2 = cross(d1, r2), r1d2 = cross(r1, d2), d1d2 = cross(d1, d2);
    return dot(d0, r1r2) + dot(r0, d1r2) + dot(r0, r1d2) + dot(d0, d1r2) + dot(d0, r1d2) + dot(r0, d1d2) +
           dot(d0, d1d2);
}

// ---------------------------------------------------------------------------
// Per-cell dS, dV, one block per chunk of one cell's triangles, one triangle
// per thread.  The per-triangle terms are added as 64-bit integers in 2^-40
// units (each rounded once, far below its FP32 rounding; the sums are exact
// and independent of their order, and run on the integer pipe: this GPU's
// FP64 pipe retires about two operations per clock per SM).  The last block
// of a cell adds the cell's partials and forms dS, dV in FP64 once.  With
// FORCES the same pass
// writes each triangle's area and volume force terms:
//   area (local + global, homocentric): F_k = (kal dS_t/S0_t + kag dS/S0) a_k,
//     a_k = -(2 S_t / sum_j |w_j|^2) w_k, w_k = x_k - centroid;
//   volume: F_k = -kv (dV/V0) n_t / 6, n_t = (x_1 - x_0) x (x_2 - x_0).
// The cell totals dS/S0 and dV/V0 are applied in the node gather.
// ---------------------------------------------------------------------------
// Block size and register budget of the immersed-boundary kernels: 128
// threads within 64 registers (8192 per block), so that one such block fits
// in what a retiring stream-collide block frees on an SM that is full of
// them (6144 registers plus the 4096 left over; overlapped schedule).
constexpr int CS_BLOCK = 128;
constexpr int IB_MIN_BLOCKS = 8;

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The cell's partial sums (dS, 6 dV in 2^-40 units) of one chunk: block
// reduction, then the last block of the cell adds the cell's partials.
__device__ __forceinline__ void chunk_sums(const IbmArgs& a, int chunk, const int4& ck, long long s, long long v) {
    __shared__ long long sh[2][CS_BLOCK / 32];
    __shared__ bool last;
    s = warp_sum_ll(s);
    v = warp_sum_ll(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = s; sh[1][wid] = v; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long S = 0, V = 0;
        for (int w = 0; w < CS_BLOCK / 32; ++w) { S += sh[0][w]; V += sh[1][w]; }
        a.partials[chunk] = make_longlong2(S, V);
        __threadfence();
        const unsigned done = atomicAdd(a.counters + ck.x, 1u);
        last = (done + 1 == (unsigned)ck.w);
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        // the last block of the cell: one warp loads all partials at once
        __threadfence();
        const int c0 = a.cells[ck.x].chunk0, nc = ck.w;
        long long Si = 0, Vi = 0;
        for (int k = threadIdx.x; k < nc; k += 32) {
            const longlong2 pv = __ldcg(a.partials + c0 + k);
            Si += pv.x;
            Vi += pv.y;
        }
        Si = warp_sum_ll(Si);
        Vi = warp_sum_ll(Vi);
        if (threadIdx.x == 0) {
            const double S = (double)Si * (1.0 / FIX_SCALE), V = (double)Vi * (1.0 / (6.0 * FIX_SCALE));
            a.cell_sums[ck.x] = make_double2(S, V);
            a.cell_rel[ck.x] = make_float2((float)(S / a.cells[ck.x].S0), (float)(V / a.cells[ck.x].V0));
            a.counters[ck.x] = 0u;
        }
    }
}

// The static data of one triangle (indices, rest area, the cell's reference
// node and local-area modulus), which the element pass loads before waiting
// for the previous advance.
struct TriStatic {
    int4 tr;
    float S0t, kal;
    int ref;
};

__device__ __forceinline__ TriStatic tri_static(const IbmArgs& a, int t) {
    TriStatic d;
    d.tr = a.tris[t];
    d.S0t = a.tri_S0[t];
    d.ref = a.cells[d.tr.w].ref;
    d.kal = a.cells[d.tr.w].kal;
    return d;
}

// dS_t and dV_t (x 6) of one triangle; with FORCES also its area and volume
// force terms.
template <bool FORCES>
__device__ __forceinline__ void tri_terms(const IbmArgs& a, int t, const TriStatic& d, long long& s, long long& v) {
    const Q4* qc = cur_q(a);
    const Pt R = load_pt(a, qc, d.ref);
    const Pt P0 = load_pt(a, qc, d.tr.x), P1 = load_pt(a, qc, d.tr.y), P2 = load_pt(a, qc, d.tr.z);
    const float3 e1 = edge(P0, P1), e2 = edge(P0, P2);
    const float dSt = tri_dS(e1, e2, ddisp(P0, P1), ddisp(P0, P2), d.S0t);
    s += float_to_fixed(dSt);
    v += float_to_fixed(tri_dV6(R, P0, P1, P2));
    if constexpr (FORCES) {
        const float St = d.S0t + dSt;
        const float3 third = (1.0f / 3.0f) * (e1 + e2);
        const float3 w0 = -third, w1 = e1 - third, w2 = e2 - third;
        const float ww = dot(w0, w0) + dot(w1, w1) + dot(w2, w2);
        const float c = __fdividef(-2.0f * St, ww);
        const float sl = __fdividef(d.kal * dSt, d.S0t);
        a.tA[3 * t] = make_float4(c * w0.x, c * w0.y, c * w0.z, sl);
        a.tA[3 * t + 1] = make_float4(c * w1.x, c * w1.y, c * w1.z, sl);
        a.tA[3 * t + 2] = make_float4(c * w2.x, c * w2.y, c * w2.z, sl);
        const float3 n = cross(e1, e2);
        a.tN[t] = make_float4(n.x, n.y, n.z, 0.f);
    }
}

template <bool FORCES>
__device__ __forceinline__ void tri_chunk(const IbmArgs& a, int chunk) {
    const int4 ck = a.chunks[chunk];
    long long s = 0, v = 0;
    for (int t = ck.y + (int)threadIdx.x; t < ck.z; t += CS_BLOCK) tri_terms<FORCES>(a, t, tri_static(a, t), s, v);
    chunk_sums(a, chunk, ck, s, v);
}

__global__ void __launch_bounds__(CS_BLOCK, 6) k_cell_sums(const __grid_constant__ IbmArgs a) {
    tri_chunk<false>(a, blockIdx.x);
}

cudaError_t launch_cell_sums(const IbmArgs& a, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_cell_sums<<<a.n_chunks, CS_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Element pass: blocks [0, n_chunks) are the triangle chunks above (with their
// force terms), the blocks after them take one edge per thread: stretching
// (neo-Hookean bond) and bending of edge (a, b), each evaluated once.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CS_BLOCK, 6) k_elements(const __grid_constant__ IbmArgs a) {
    if ((int)blockIdx.x < a.n_chunks) {
        // a chunk holds at most one triangle per thread: its static data
        // before the previous advance has finished, then its positions
        const int4 ck = a.chunks[blockIdx.x];
        const int t = ck.y + (int)threadIdx.x;
        const bool live = t < ck.z;
        TriStatic d = {};
        if (live) d = tri_static(a, t);
        pdl_entry();
        long long s = 0, v = 0;
        if (live) tri_terms<true>(a, t, d, s, v);
        chunk_sums(a, blockIdx.x, ck, s, v);
        return;
    }
    // the edge's static data before the previous advance has finished
    const int e = ((int)blockIdx.x - a.n_chunks) * CS_BLOCK + (int)threadIdx.x;
    const bool live = e < a.n_edges;
    int4 ev = make_int4(0, 0, 0, 0);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);   // (L0, theta0, ks, kb)
    if (live) {
        ev = a.edges[e];
        r = a.edge_rest[e];
    }
    pdl_entry();
    if (!live) return;
    const Q4* qc = cur_q(a);
    const Pt A = load_pt(a, qc, ev.x), B = load_pt(a, qc, ev.y), Cc = load_pt(a, qc, ev.z), D = load_pt(a, qc, ev.w);
    const float3 fs = stretch_on_a(A, B, r.x, r.z);
    a.eS[e] = make_float4(fs.x, fs.y, fs.z, 0.f);
    float3 fb[4];
    bend_all(A, B, Cc, D, r.y, r.w, fb);
#pragma unroll
    for (int k = 0; k < 4; ++k) a.eB[4 * e + k] = make_float4(fb[k].x, fb[k].y, fb[k].z, 0.f);
}

cudaError_t launch_elements(const IbmArgs& a, cudaStream_t s) {
    const int blocks = a.n_chunks + (a.n_edges + CS_BLOCK - 1) / CS_BLOCK;
    if (blocks <= 0) return cudaSuccess;
    return launch_ex(k_elements, blocks, CS_BLOCK, 0, s, a.pdl, a);
}

// ---------------------------------------------------------------------------
// one corner of the trilinear stencil of a fixed-point position
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool corner(const ChannelDev& C, const Q4& q, int c, long long& g, float& w) {
    const long long qq[3] = {q.x, q.y, q.z};
    const int n[3] = {C.nx, C.ny, C.nz};
    const int cc[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    int ic[3];
    w = 1.0f;
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // fractional part: top 24 of the 40 fraction bits (exact in FP32)
        const unsigned f24 = (unsigned)((qq[d] >> (FIX_BITS - 24)) & 0xFFFFFF);
        const float fr = __uint2float_rn(f24) * 5.9604644775390625e-08f;   // 2^-24
        w *= cc[d] ? fr : 1.0f - fr;
        int v = (int)(qq[d] >> FIX_BITS) + cc[d];
        if (v < 0 || v >= n[d]) {
            if (C.per[d]) {
                v %= n[d];
                if (v < 0) v += n[d];
            } else {
                ok = false;
            }
        }
        ic[d] = v;
    }
    g = ok ? C.base + ic[0] + (long long)C.nx * (ic[1] + (long long)C.ny * ic[2]) : 0;
    return ok;
}

// Stencil set of the overlapped schedule.  A point at X with base node
// floor(X) = (ix, iy, iz) has its stencil in [ix, ix+1]^3 now and, as long as
// it moves less than one lattice unit per step, in [ix-1, ix+2]^3 after the
// next advance.  Lane sl (0..7) of the point marks the 32-node groups of the
// nodes of that box in the rows (dy, dz) = (c & 3, c >> 2) - 1, c = 2 sl, 2 sl + 1.
__device__ __forceinline__ void mark_box(const ChannelDev& C, const Q4& q, int sl, uint8_t* map) {
    const int bx = (int)(q.x >> FIX_BITS), by = (int)(q.y >> FIX_BITS), bz = (int)(q.z >> FIX_BITS);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = 2 * sl + h;
        int y = by + (c & 3) - 1, z = bz + (c >> 2) - 1;
        if (y < 0 || y >= C.ny) {
            if (!C.per[1]) continue;
            y = ((y % C.ny) + C.ny) % C.ny;
        }
        if (z < 0 || z >= C.nz) {
            if (!C.per[2]) continue;
            z = ((z % C.nz) + C.nz) % C.nz;
        }
        const long long row = C.base + (long long)C.nx * (y + (long long)C.ny * z);
        long long last = -1;
#pragma unroll
        for (int dx = -1; dx <= 2; ++dx) {
            int x = bx + dx;
            if (x < 0 || x >= C.nx) {
                if (!C.per[0]) continue;
                x = ((x % C.nx) + C.nx) % C.nx;
            }
            const long long g = (row + x) >> 5;
            if (g != last) map[g] = 1;
            last = g;
        }
    }
}

__global__ void __launch_bounds__(128, IB_MIN_BLOCKS) k_mark_stencils(const __grid_constant__ IbmArgs a, uint8_t* map) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / SUB;
    if (i >= a.n_nodes) return;
    const int chn = a.info[i].w >> 8;
    mark_box(chan(a, chn), (a.par ? a.qb : a.qa)[i], threadIdx.x & (SUB - 1), map);
}

cudaError_t launch_mark_stencils(const IbmArgs& a, uint8_t* map, cudaStream_t s) {
    if (a.n_nodes <= 0) return cudaSuccess;
    const long long threads = (long long)a.n_nodes * SUB;
    k_mark_stencils<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a, map);
    return cudaGetLastError();
}

// Marked groups of a byte map as a list (order unspecified), one atomic per warp.
__global__ void __launch_bounds__(128, IB_MIN_BLOCKS) k_compact_groups(const uint8_t* map, int n_groups, int* list, int* count) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = g < n_groups && map[g] != 0;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    if (!b) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(count, __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[base + __popc(b & ((1u << lane) - 1u))] = g;
}

cudaError_t launch_compact_groups(const uint8_t* map, int n_groups, int* list, int* count, cudaStream_t s) {
    if (n_groups <= 0) return cudaSuccess;
    k_compact_groups<<<(n_groups + 127) / 128, 128, 0, s>>>(map, n_groups, list, count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// node forces + spreading, eight lanes per IB node: each lane gathers the
// node's share of the elements of some ring slots (incident triangle, edge and
// opposite edge; fixed order, no atomics), the eight partial sums are added by
// shuffles, then each lane spreads to one stencil corner.
// ---------------------------------------------------------------------------
constexpr int FS_BLOCK = 128;

#ifndef LBIBM_FS_MINB
#define LBIBM_FS_MINB 10
#endif
// (massless points: 48 registers, 10 blocks of 128 per SM; with mass: 64, 8)
template <bool MASSIVE>
__global__ void __launch_bounds__(FS_BLOCK, MASSIVE ? IB_MIN_BLOCKS : LBIBM_FS_MINB) k_forces_spread(const __grid_constant__ IbmArgs a) {
    const int i = (blockIdx.x * FS_BLOCK + threadIdx.x) / SUB;
    const int sl = threadIdx.x & (SUB - 1);
    const bool live = i < a.n_nodes;
    // before the element pass has finished: the node's static data, its
    // position (advanced in the previous cycle) and this lane's stencil corner
    // (Sec. 2.2 step 3) with its obstacle bit
    // and the lane's first ring slot
    int4 inf = make_int4(0, 0, 0, 0);
    int4 sr0 = make_int4(0, 0, 0, 0);
    Q4 qi = {};
    long long g = 0;
    float w = 0.f;
    bool hit = false;
    if (live) {
        inf = a.info[i];
        if (sl < (inf.w & 0xff)) sr0 = a.slots[inf.z + sl];
        qi = (a.par ? a.qb : a.qa)[i];
        hit = corner(chan(a, inf.w >> 8), qi, sl, g, w);
        if (hit) hit = !((__ldg(a.mask + (g >> 5)) >> (g & 31)) & 1u);
    }
    pdl_entry();
    if (!live) return;   // whole groups of eight lanes leave together
    const unsigned smask = 0xffu << (threadIdx.x & 24);
    const int cid = inf.x, k0 = inf.z, k = inf.w & 0xff, chn = inf.w >> 8;
    const CellDev& C = a.cells[cid];
    const float2 rel = a.cell_rel[cid];
    const ChannelDev Ch = chan(a, chn);
    if (a.dcur) {
        // overlapped schedule: the target must be in this step's stencil set
        // (it is whenever no point moved a lattice unit in one step), and the
        // next step's set is marked around the current position
        if (hit && !__ldg(a.dcur + (g >> 5))) atomicAdd(a.sched_err, 1);
        mark_box(Ch, qi, sl, a.dmark);
    }

    const float kag_dS = C.kag * rel.x;
    const float kv_dV6 = C.kv * rel.y * (1.0f / 6.0f);
    float3 F = make_float3(0.f, 0.f, 0.f);
    for (int s = sl; s < k; s += SUB) {
        const int4 sr = s == sl ? sr0 : a.slots[k0 + s];
        const float4 ta = a.tA[sr.x];
        const float4 tn = a.tN[sr.w];
        const float4 es = a.eS[sr.y >> 2];
        const float4 b1 = a.eB[sr.y];
        const float4 b2 = a.eB[sr.z];
        const float sg = (sr.y & 3) == 0 ? 1.0f : -1.0f;   // stretching acts on a, its negative on b
        const float ca = ta.w + kag_dS;
        F.x += ((ca * ta.x - kv_dV6 * tn.x) + sg * es.x) + (b1.x + b2.x);
        F.y += ((ca * ta.y - kv_dV6 * tn.y) + sg * es.y) + (b1.y + b2.y);
        F.z += ((ca * ta.z - kv_dV6 * tn.z) + sg * es.z) + (b1.z + b2.z);
    }
#pragma unroll
    for (int o = SUB / 2; o > 0; o >>= 1) {
        F.x += __shfl_xor_sync(smask, F.x, o);
        F.y += __shfl_xor_sync(smask, F.y, o);
        F.z += __shfl_xor_sync(smask, F.z, o);
    }
    if (a.R) {
        // collisions (Sec. 2.4): every lane holds the reduced total, add to each
        const float4 r = a.R[i];
        F.x += r.x; F.y += r.y; F.z += r.z;
    }
    if (sl == 0) a.F[i] = make_float4(F.x, F.y, F.z, 0.f);

    uint8_t* fl = a.par ? a.fl1 : a.fl0;
    const unsigned active = __activemask();
    float3 S = F;   // what reaches the fluid
    if (MASSIVE) {
        // points with mass (Sec. 2.2 Newton equation): the fluid velocity of
        // the last collision at X (this lane's corner, summed over the eight
        // lanes), kick by F, exact drag drift; the fluid receives the drag's
        // impulse and the point moves now (no interpolation kernel follows)
        float4 uc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (hit) uc = a.u[g];
        float3 U = make_float3(w * uc.x, w * uc.y, w * uc.z);
#pragma unroll
        for (int o = SUB / 2; o > 0; o >>= 1) {
            U.x += __shfl_xor_sync(smask, U.x, o);
            U.y += __shfl_xor_sync(smask, U.y, o);
            U.z += __shfl_xor_sync(smask, U.z, o);
        }
        const float4 W = a.W[i];
        const float3 D = make_float3(W.x + F.x * a.ib_inv_m - U.x, W.y + F.y * a.ib_inv_m - U.y,
                                     W.z + F.z * a.ib_inv_m - U.z);   // V - U
        S = make_float3(a.ib_gp1 * D.x, a.ib_gp1 * D.y, a.ib_gp1 * D.z);
        Q4 qn = qi;
        qn.x += float_to_fixed(U.x + a.ib_p1 * D.x);
        qn.y += float_to_fixed(U.y + a.ib_p1 * D.y);
        qn.z += float_to_fixed(U.z + a.ib_p1 * D.z);
        if (sl == 0) {
            a.W[i] = make_float4(U.x + a.ib_E * D.x, U.y + a.ib_E * D.y, U.z + a.ib_E * D.z, 0.f);
            (a.par ? a.qa : a.qb)[i] = qn;
        }
        // the stencil at the new position needs this step's velocity there:
        // flag its groups so that the stream-collide writes it
        long long g2;
        float w2;
        const long long grp2 = corner(Ch, qn, sl, g2, w2) ? (g2 >> 5) : -1;
        const unsigned same2 = __match_any_sync(active, grp2);
        if (grp2 >= 0 && (__ffs(same2) - 1) == (int)(threadIdx.x & 31)) fl[grp2] = 1;
    }

    // spreading: g(x) += w(x - X) S at this lane's corner; in 2^-40 fixed
    // point when deterministic (integer sums do not depend on their order)
    if (hit) {
        if (a.gfix) {
            const float c[3] = {w * S.x, w * S.y, w * S.z};
#pragma unroll
            for (int d = 0; d < 3; ++d)
                atomicAdd(a.gfix + d * a.gfix_stride + g, (unsigned long long)__float2ll_rn(c[d] * FIX_SCALE_F));
        } else {
            atomicAdd((a.par ? a.g1 : a.g0) + g, make_float4(w * S.x, w * S.y, w * S.z, 0.f));
        }
    }
    // flag the 32-node groups that received force: one store per distinct group of this warp
    const long long grp = hit ? (g >> 5) : -1;
    const unsigned same = __match_any_sync(active, grp);
    if (hit && (__ffs(same) - 1) == (int)(threadIdx.x & 31)) fl[grp] = 1;
}

// The massless node forces + spreading with four lanes per IB node (each
// lane two ring slots and two stencil corners): half the threads of the
// eight-lane kernel for the sequential schedule (the overlapped schedule's
// stencil marking and points with mass keep eight lanes).
constexpr int FS4 = 4;

__global__ void __launch_bounds__(FS_BLOCK, 9) k_forces_spread4(const __grid_constant__ IbmArgs a) {
    const int i = (blockIdx.x * FS_BLOCK + threadIdx.x) / FS4;
    const int sl = threadIdx.x & (FS4 - 1);
    const bool live = i < a.n_nodes;
    // before the element pass has finished: the node's static data, its
    // position (advanced in the previous cycle), this lane's two stencil
    // corners with their obstacle bits and its first two ring slots
    int4 inf = make_int4(0, 0, 0, 0);
    int4 sr0 = make_int4(0, 0, 0, 0), sr1 = make_int4(0, 0, 0, 0);
    long long g[2] = {0, 0};
    float w[2] = {0.f, 0.f};
    bool hit[2] = {false, false};
    if (live) {
        inf = a.info[i];
        const int k = inf.w & 0xff;
        if (sl < k) sr0 = a.slots[inf.z + sl];
        if (sl + FS4 < k) sr1 = a.slots[inf.z + sl + FS4];
        const Q4 qi = (a.par ? a.qb : a.qa)[i];
        const ChannelDev& Ch = chan(a, inf.w >> 8);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            hit[c] = corner(Ch, qi, sl + c * FS4, g[c], w[c]);
            if (hit[c]) hit[c] = !((__ldg(a.mask + (g[c] >> 5)) >> (g[c] & 31)) & 1u);
        }
    }
    pdl_entry();
    if (!live) return;   // whole groups of four lanes leave together
    const unsigned smask = 0xfu << (threadIdx.x & 28);
    const int cid = inf.x, k0 = inf.z, k = inf.w & 0xff;
    const CellDev& C = a.cells[cid];
    const float2 rel = a.cell_rel[cid];
    const float kag_dS = C.kag * rel.x;
    const float kv_dV6 = C.kv * rel.y * (1.0f / 6.0f);
    float3 F = make_float3(0.f, 0.f, 0.f);
    for (int s = sl; s < k; s += FS4) {
        const int4 sr = s == sl ? sr0 : (s == sl + FS4 ? sr1 : a.slots[k0 + s]);
        const float4 ta = a.tA[sr.x];
        const float4 tn = a.tN[sr.w];
        const float4 es = a.eS[sr.y >> 2];
        const float4 b1 = a.eB[sr.y];
        const float4 b2 = a.eB[sr.z];
        const float sg = (sr.y & 3) == 0 ? 1.0f : -1.0f;   // stretching acts on a, its negative on b
        const float ca = ta.w + kag_dS;
        F.x += ((ca * ta.x - kv_dV6 * tn.x) + sg * es.x) + (b1.x + b2.x);
        F.y += ((ca * ta.y - kv_dV6 * tn.y) + sg * es.y) + (b1.y + b2.y);
        F.z += ((ca * ta.z - kv_dV6 * tn.z) + sg * es.z) + (b1.z + b2.z);
    }
#pragma unroll
    for (int o = FS4 / 2; o > 0; o >>= 1) {
        F.x += __shfl_xor_sync(smask, F.x, o);
        F.y += __shfl_xor_sync(smask, F.y, o);
        F.z += __shfl_xor_sync(smask, F.z, o);
    }
    if (a.R) {
        const float4 r = a.R[i];
        F.x += r.x; F.y += r.y; F.z += r.z;
    }
    if (sl == 0) a.F[i] = make_float4(F.x, F.y, F.z, 0.f);
    uint8_t* fl = a.par ? a.fl1 : a.fl0;
    const unsigned active = __activemask();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (hit[c]) {
            if (a.gfix) {
                const float cc[3] = {w[c] * F.x, w[c] * F.y, w[c] * F.z};
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    atomicAdd(a.gfix + d * a.gfix_stride + g[c],
                              (unsigned long long)__float2ll_rn(cc[d] * FIX_SCALE_F));
            } else {
                atomicAdd((a.par ? a.g1 : a.g0) + g[c], make_float4(w[c] * F.x, w[c] * F.y, w[c] * F.z, 0.f));
            }
        }
        // flag the 32-node groups that received force: one store per distinct group of this warp
        const long long grp = hit[c] ? (g[c] >> 5) : -1;
        const unsigned same = __match_any_sync(active, grp);
        if (hit[c] && (__ffs(same) - 1) == (int)(threadIdx.x & 31)) fl[grp] = 1;
    }
}

cudaError_t launch_forces_spread(const IbmArgs& a, cudaStream_t s) {
    if (a.n_nodes <= 0) return cudaSuccess;
    const long long threads = (long long)a.n_nodes * SUB;
    if (a.W) return launch_ex(k_forces_spread<true>, (unsigned)((threads + FS_BLOCK - 1) / FS_BLOCK), FS_BLOCK, 0, s, a.pdl, a);
    if (!a.dcur) {
        const long long t4 = (long long)a.n_nodes * FS4;
        return launch_ex(k_forces_spread4, (unsigned)((t4 + FS_BLOCK - 1) / FS_BLOCK), FS_BLOCK, 0, s, a.pdl, a);
    }
    return launch_ex(k_forces_spread<false>, (unsigned)((threads + FS_BLOCK - 1) / FS_BLOCK), FS_BLOCK, 0, s, a.pdl, a);
}

// Deterministic spreading: the fixed-point force density of the flagged
// 32-node groups into g (one warp per group; a group's flag is the same for
// all its lanes), clearing the fixed-point sums for the next step.
__global__ void __launch_bounds__(256) k_gfix_to_g(const __grid_constant__ IbmArgs a) {
    pdl_entry();
    const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= a.gfix_stride) return;
    if (!(a.par ? a.fl1 : a.fl0)[gi >> 5]) return;
    unsigned long long* p = a.gfix + gi;
    const long long x = (long long)p[0], y = (long long)p[a.gfix_stride], z = (long long)p[2 * a.gfix_stride];
    const float inv = 1.0f / FIX_SCALE_F;
    (a.par ? a.g1 : a.g0)[gi] = make_float4((float)x * inv, (float)y * inv, (float)z * inv, 0.f);
    p[0] = 0ull;
    p[a.gfix_stride] = 0ull;
    p[2 * a.gfix_stride] = 0ull;
}

cudaError_t launch_gfix_to_g(const IbmArgs& a, cudaStream_t s) {
    if (!a.gfix || a.gfix_stride <= 0) return cudaSuccess;
    return launch_ex(k_gfix_to_g, (unsigned)((a.gfix_stride + 255) / 256), 256, 0, s, a.pdl, a);
}

// ---------------------------------------------------------------------------
// interpolation + advance (Sec. 2.2 steps 1 and 4), one thread per IB node:
// the eight stencil velocities are loaded at once, U = sum w u, and the
// position advances by the exact fixed-point addition X <- X + U.  Obstacle
// and out-of-domain stencil nodes contribute nothing.
// ---------------------------------------------------------------------------
constexpr int IA_BLOCK = 128;

__global__ void __launch_bounds__(IA_BLOCK, IB_MIN_BLOCKS) k_interp_advance(const __grid_constant__ IbmArgs a) {
    const int i = blockIdx.x * IA_BLOCK + threadIdx.x;
    const bool live = i < a.n_nodes;
    // before the stream-collide has finished: position and stencil weights
    Q4 q = {};
    long long g[8];
    float w[8];
    bool ok[8];
    if (live) {
        const ChannelDev Ch = chan(a, a.info[i].w >> 8);
        q = cur_q(a)[i];
#pragma unroll
        for (int c = 0; c < 8; ++c) ok[c] = corner(Ch, q, c, g[c], w[c]);
    }
    pdl_entry();
    if (!live) return;
    float4 u[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) u[c] = ok[c] ? a.u[g[c]] : make_float4(0.f, 0.f, 0.f, 0.f);
    float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        ux = fmaf(w[c], u[c].x, ux);
        uy = fmaf(w[c], u[c].y, uy);
        uz = fmaf(w[c], u[c].z, uz);
    }
    Q4 qn = q;
    qn.x += float_to_fixed(ux);
    qn.y += float_to_fixed(uy);
    qn.z += float_to_fixed(uz);
    (a.par ? a.qa : a.qb)[i] = qn;
}

cudaError_t launch_interp_advance(const IbmArgs& a, cudaStream_t s) {
    if (a.n_nodes <= 0) return cudaSuccess;
    return launch_ex(k_interp_advance, (unsigned)((a.n_nodes + IA_BLOCK - 1) / IA_BLOCK), IA_BLOCK, 0, s, a.pdl, a);
}

// Positions as doubles (x, y, z per node) for an asynchronous readback; the
// 2^-40 fixed point converts exactly for |x| < 2^13 lu.
__global__ void k_positions_to_double(const Q4* __restrict__ q, int n, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Q4 v = q[i];
    out[3 * i] = (double)v.x * (1.0 / FIX_SCALE);
    out[3 * i + 1] = (double)v.y * (1.0 / FIX_SCALE);
    out[3 * i + 2] = (double)v.z * (1.0 / FIX_SCALE);
}

cudaError_t launch_positions_to_double(const Q4* q, int n, double* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_positions_to_double<<<(n + 255) / 256, 256, 0, s>>>(q, n, out);
    return cudaGetLastError();
}

}  // namespace lbibm
