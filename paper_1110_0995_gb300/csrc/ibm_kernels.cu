// Immersed-boundary kernels (Gusenbauer et al., arXiv:1110.0995, Sec. 2.2-2.3):
//   k_cell_sums      per-cell change of surface area and volume, FP32 per-triangle
//                    terms accumulated in FP64 (Sec. 2.3.3: the global area and
//                    volume constraints need every node of a cell)
//   k_forces_spread  node forces (Sec. 2.3.1: stretching, bending, local/global
//                    area, volume), one thread per node gathering its incident
//                    elements (deterministic, no force atomics), then spreading
//                    with the trilinear delta function (Sec. 2.2 step 3)
//   k_interp_advance trilinear velocity interpolation (Sec. 2.2 step 1) and the
//                    point advance X <- X + U (massless points)
//
// Positions are 64-bit fixed point (2^-40 lu).  Element geometry is evaluated
// in FP32 relative to each cell's reference node; length and area changes use
// the displacement from rest (d = (x - x0) - (x_ref - x0_ref)) so that
// |x_b - x_a|^2 - L0^2 = 2 d0.de + de.de keeps its relative accuracy when the
// change is small.  Every element is evaluated in a canonical vertex order so
// that all threads touching it compute bit-identical contributions.
#include "lbibm_internal.cuh"

namespace lbibm {

__device__ __forceinline__ float3 f3(const float4& v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

struct NodeF {
    float3 x;   // position relative to the cell's reference node
    float3 d;   // displacement from rest relative to the reference node's
    float3 r;   // rest position relative to the reference node's rest position
};

__device__ __forceinline__ NodeF load_node(const IbmArgs& a, int i) {
    NodeF n;
    n.x = f3(a.xr[i]);
    n.d = f3(a.dl[i]);
    n.r = f3(a.r0[i]);
    return n;
}

// ---------------------------------------------------------------------------
// element terms
// ---------------------------------------------------------------------------

// Stretching (neo-Hookean bond, Dupin et al.): tension ks kappa(lambda)(lambda-1)
// with kappa = (lambda^1/2 + lambda^-5/2)/(lambda + lambda^-3); returns the force
// on a (the force on b is its negative).  a < b in global index.
__device__ __forceinline__ float3 stretch_on_a(const NodeF& A, const NodeF& B, float L0, float ks) {
    const float3 d = B.x - A.x;
    const float3 de = B.d - A.d;
    const float3 d0 = B.r - A.r;
    const float num = 2.0f * dot(d0, de) + dot(de, de);   // |d|^2 - L0^2
    const float L = sqrtf(L0 * L0 + num);
    const float lm1 = num / ((L + L0) * L0);               // lambda - 1
    const float lam = 1.0f + lm1;
    const float sl = sqrtf(lam);
    const float kappa = (sl + 1.0f / (lam * lam * sl)) / (lam + 1.0f / (lam * lam * lam));
    const float T = ks * kappa * lm1;
    return (T / sqrtf(dot(d, d))) * d;
}

// Bending: E = (kb/2)(theta - theta0)^2 at edge (a, b) between triangle (a, b, c)
// and triangle (b, a, d); theta = atan2((n1 x n2).e_hat, n1.n2).  Returns the
// force on vertex `role` (0..3 = a, b, c, d).
__device__ __forceinline__ float3 bend_on(const float3& xa, const float3& xb, const float3& xc, const float3& xd,
                                          float th0, float kb, int role) {
    const float3 e = xb - xa;
    const float3 ac = xc - xa;
    const float3 ad = xd - xa;
    const float3 n1 = cross(e, ac);
    const float3 n2 = cross(xa - xb, xd - xb);
    const float l2 = dot(e, e);
    const float l = sqrtf(l2);
    const float theta = atan2f(dot(cross(n1, n2), e) / l, dot(n1, n2));
    const float coef = -kb * (theta - th0);
    const float3 gc = (-l / dot(n1, n1)) * n1;
    const float3 gd = (-l / dot(n2, n2)) * n2;
    const float sc = dot(ac, e) / l2;
    const float sd = dot(ad, e) / l2;
    const float3 ga = (-(1.0f - sc)) * gc - (1.0f - sd) * gd;
    const float3 gb = (-sc) * gc - sd * gd;
    const float3 g = role == 0 ? ga : (role == 1 ? gb : (role == 2 ? gc : gd));
    return coef * g;
}

// Area change of triangle (0, 1, 2) from rest: S_t - S0_t with
// |n|^2 - |n0|^2 = 2 n0.dn + dn.dn, dn = a1 x b2 + b1 x a2 + b1 x b2.
__device__ __forceinline__ float tri_dS(const NodeF& P0, const NodeF& P1, const NodeF& P2, float S0t) {
    const float3 a1 = P1.r - P0.r, a2 = P2.r - P0.r;
    const float3 b1 = P1.d - P0.d, b2 = P2.d - P0.d;
    const float3 n0 = cross(a1, a2);
    const float3 dn = cross(a1, b2) + cross(b1, a2) + cross(b1, b2);
    const float num = 2.0f * dot(n0, dn) + dot(dn, dn);
    const float nn0 = 2.0f * S0t;
    const float nn = sqrtf(nn0 * nn0 + num);
    return num / (2.0f * (nn + nn0));
}

// Volume change of the tetrahedron (origin, 0, 1, 2) from rest, times 6:
// (r0 + d0).((r1 + d1) x (r2 + d2)) - r0.(r1 x r2), expanded.
__device__ __forceinline__ float tri_dV6(const NodeF& P0, const NodeF& P1, const NodeF& P2) {
    const float3 r1r2 = cross(P1.r, P2.r), d1r2 = cross(P1.d, P2.r), r1d2 = cross(P1.r, P2.d), d1d2 = cross(P1.d, P2.d);
    return dot(P0.d, r1r2) + dot(P0.r, d1r2) + dot(P0.r, r1d2) + dot(P0.d, d1r2) + dot(P0.d, r1d2) + dot(P0.r, d1d2) +
           dot(P0.d, d1d2);
}

// Area (local + global) and volume forces of triangle (0, 1, 2) on vertex `role`:
// homocentric area force along w_k = x_k - centroid with magnitude
// k dA (2 S_t / sum |w|^2); volume force -kv dV/V0 n/6.
__device__ __forceinline__ float3 tri_on(const NodeF& P0, const NodeF& P1, const NodeF& P2, float S0t, float kal,
                                         float kag_dS, float kv_dV6, int role) {
    const float dSt = tri_dS(P0, P1, P2, S0t);
    const float St = S0t + dSt;
    const float3 c = (1.0f / 3.0f) * (P0.x + P1.x + P2.x);
    const float3 w0 = P0.x - c, w1 = P1.x - c, w2 = P2.x - c;
    const float ww = dot(w0, w0) + dot(w1, w1) + dot(w2, w2);
    const float coefA = (-kal * dSt / S0t - kag_dS) * 2.0f * St / ww;
    const float3 n = cross(P1.x - P0.x, P2.x - P0.x);
    const float3 w = role == 0 ? w0 : (role == 1 ? w1 : w2);
    return coefA * w - kv_dV6 * n;
}

// ---------------------------------------------------------------------------
// R1: per-cell dS, dV (FP64 accumulation), one block per triangle chunk; the
// last block of a cell adds the cell's partials in chunk order.
// ---------------------------------------------------------------------------
constexpr int CS_BLOCK = 128;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(CS_BLOCK) k_cell_sums(IbmArgs a) {
    const int4 ck = a.chunks[blockIdx.x];
    double s = 0.0, v = 0.0;
    for (int t = ck.y + threadIdx.x; t < ck.z; t += CS_BLOCK) {
        const int4 tr = a.tris[t];
        const NodeF P0 = load_node(a, tr.x), P1 = load_node(a, tr.y), P2 = load_node(a, tr.z);
        s += (double)tri_dS(P0, P1, P2, a.tri_S0[t]);
        v += (double)tri_dV6(P0, P1, P2);
    }
    __shared__ double sh[2][CS_BLOCK / 32];
    __shared__ bool last;
    s = warp_sum_d(s);
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = s; sh[1][wid] = v; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, V = 0.0;
        for (int w = 0; w < CS_BLOCK / 32; ++w) { S += sh[0][w]; V += sh[1][w]; }
        a.partials[blockIdx.x] = make_double2(S, V / 6.0);
        __threadfence();
        const unsigned done = atomicAdd(a.counters + ck.x, 1u);
        last = (done + 1 == (unsigned)a.cells[ck.x].n_chunks);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const CellDev C = a.cells[ck.x];
        double S = 0.0, V = 0.0;
        for (int k = 0; k < C.n_chunks; ++k) {
            const volatile double* pv = (const volatile double*)(a.partials + C.chunk0 + k);
            S += pv[0];
            V += pv[1];
        }
        a.cell_sums[ck.x] = make_double2(S, V);
        a.counters[ck.x] = 0u;
    }
}

cudaError_t launch_cell_sums(const IbmArgs& a, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_cell_sums<<<a.n_chunks, CS_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// lattice coordinates of a fixed-point position
// ---------------------------------------------------------------------------
struct Corner {
    long long g[8];
    float w[8];
    bool ok[8];
};

__device__ __forceinline__ void stencil(const ChannelDev& C, const Q4& q, const uint32_t* mask, Corner& s) {
    const long long qq[3] = {q.x, q.y, q.z};
    const int n[3] = {C.nx, C.ny, C.nz};
    long long base[3];
    float fr[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        base[d] = qq[d] >> FIX_BITS;
        fr[d] = __ll2float_rn(qq[d] & ((1LL << FIX_BITS) - 1)) * FIX_INV_F;
    }
    long long ic[3][2];
    bool ok[3][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            long long v = base[d] + k;
            bool good = true;
            if (v < 0 || v >= n[d]) {
                if (C.per[d]) { v %= n[d]; if (v < 0) v += n[d]; }
                else good = false;
            }
            ic[d][k] = v;
            ok[d][k] = good;
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const float w = (cx ? fr[0] : 1.0f - fr[0]) * (cy ? fr[1] : 1.0f - fr[1]) * (cz ? fr[2] : 1.0f - fr[2]);
        bool good = ok[0][cx] && ok[1][cy] && ok[2][cz];
        long long g = 0;
        if (good) {
            g = C.base + ic[0][cx] + (long long)C.nx * (ic[1][cy] + (long long)C.ny * ic[2][cz]);
            good = !((__ldg(mask + (g >> 5)) >> (g & 31)) & 1u);
        }
        s.g[c] = g;
        s.w[c] = w;
        s.ok[c] = good;
    }
}

// ---------------------------------------------------------------------------
// forces + spreading, one thread per IB node
// ---------------------------------------------------------------------------
constexpr int FS_BLOCK = 128;

__global__ void __launch_bounds__(FS_BLOCK) k_forces_spread(IbmArgs a) {
    const int i = blockIdx.x * FS_BLOCK + threadIdx.x;
    if (i >= a.n_nodes) return;
    const int cid = a.cell_of[i];
    const CellDev C = a.cells[cid];
    const double2 cs = a.cell_sums[cid];
    const float kag_dS = C.kag * (float)(cs.x / C.S0);
    const float kv_dV6 = C.kv * (float)(cs.y / C.V0) * (1.0f / 6.0f);
    const NodeF I = load_node(a, i);
    const int k0 = a.ring_off[i], k1 = a.ring_off[i + 1];
    const int k = k1 - k0;

    int nb_prev = a.ring[k1 - 1].x;
    int nb_cur = a.ring[k0].x;
    NodeF Pprev = load_node(a, nb_prev);
    NodeF Pcur = load_node(a, nb_cur);
    float3 F = make_float3(0.f, 0.f, 0.f);
    for (int s = 0; s < k; ++s) {
        const int j = k0 + s;
        const int2 rg = a.ring[j];
        const float4 rest = a.ring_rest[j];   // L0(i,cur), theta0(i,cur), theta0(cur,next), S0(i,cur,next)
        const int nb_next = a.ring[k0 + (s + 1 == k ? 0 : s + 1)].x;
        const NodeF Pnext = load_node(a, nb_next);
        const NodeF Pout = load_node(a, rg.y);

        // stretching of edge (i, cur)
        if (i < nb_cur) F = F + stretch_on_a(I, Pcur, rest.x, C.ks);
        else F = F - stretch_on_a(Pcur, I, rest.x, C.ks);

        // bending of edge (i, cur): triangle (i, cur, next) and triangle (cur, i, prev)
        if (i < nb_cur) F = F + bend_on(I.x, Pcur.x, Pnext.x, Pprev.x, rest.y, C.kb, 0);
        else F = F + bend_on(Pcur.x, I.x, Pprev.x, Pnext.x, rest.y, C.kb, 1);

        // bending of the opposite edge (cur, next): triangle (cur, next, i), triangle (next, cur, out)
        if (nb_cur < nb_next) F = F + bend_on(Pcur.x, Pnext.x, I.x, Pout.x, rest.z, C.kb, 2);
        else F = F + bend_on(Pnext.x, Pcur.x, Pout.x, I.x, rest.z, C.kb, 3);

        // triangle (i, cur, next), rotated to start at its smallest index
        if (i < nb_cur && i < nb_next) F = F + tri_on(I, Pcur, Pnext, rest.w, C.kal, kag_dS, kv_dV6, 0);
        else if (nb_cur < nb_next) F = F + tri_on(Pcur, Pnext, I, rest.w, C.kal, kag_dS, kv_dV6, 2);
        else F = F + tri_on(Pnext, I, Pcur, rest.w, C.kal, kag_dS, kv_dV6, 1);

        Pprev = Pcur; Pcur = Pnext;
        nb_prev = nb_cur; nb_cur = nb_next;
    }
    a.F[i] = make_float4(F.x, F.y, F.z, 0.f);

    // spreading (Sec. 2.2 step 3): g(x) += w(x - X) F
    const ChannelDev Ch = a.ch[C.ch];
    float4* g = a.par ? a.g1 : a.g0;
    uint8_t* fl = a.par ? a.fl1 : a.fl0;
    Corner sc;
    stencil(Ch, (a.par ? a.qb : a.qa)[i], a.mask, sc);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (!sc.ok[c]) continue;
        const float w = sc.w[c];
        atomicAdd(g + sc.g[c], make_float4(w * F.x, w * F.y, w * F.z, 0.f));
        fl[sc.g[c] >> 5] = 1;
    }
}

cudaError_t launch_forces_spread(const IbmArgs& a, cudaStream_t s) {
    if (a.n_nodes <= 0) return cudaSuccess;
    k_forces_spread<<<(a.n_nodes + FS_BLOCK - 1) / FS_BLOCK, FS_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// interpolation + advance (Sec. 2.2 steps 1 and 4), one thread per IB node.
// Every thread of a cell also advances the cell's reference node (identical
// arithmetic) so that the relative coordinates of the next step can be formed
// without a second pass.
// ---------------------------------------------------------------------------
constexpr int IA_BLOCK = 128;

__device__ __forceinline__ Q4 advanced(const IbmArgs& a, const ChannelDev& Ch, int i) {
    const Q4 q = (a.par ? a.qb : a.qa)[i];
    Corner sc;
    stencil(Ch, q, a.mask, sc);
    float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (!sc.ok[c]) continue;
        const float4 u = a.u[sc.g[c]];
        ux += sc.w[c] * u.x;
        uy += sc.w[c] * u.y;
        uz += sc.w[c] * u.z;
    }
    Q4 o = q;
    o.x += __float2ll_rn(ux * FIX_SCALE_F);
    o.y += __float2ll_rn(uy * FIX_SCALE_F);
    o.z += __float2ll_rn(uz * FIX_SCALE_F);
    return o;
}

__device__ __forceinline__ float4 rel(const Q4& a, const Q4& b) {
    return make_float4(__ll2float_rn(a.x - b.x) * FIX_INV_F, __ll2float_rn(a.y - b.y) * FIX_INV_F,
                       __ll2float_rn(a.z - b.z) * FIX_INV_F, 0.f);
}

__device__ __forceinline__ float4 disp(const Q4& q, const Q4& q0, const Q4& qr, const Q4& q0r) {
    return make_float4(__ll2float_rn((q.x - q0.x) - (qr.x - q0r.x)) * FIX_INV_F,
                       __ll2float_rn((q.y - q0.y) - (qr.y - q0r.y)) * FIX_INV_F,
                       __ll2float_rn((q.z - q0.z) - (qr.z - q0r.z)) * FIX_INV_F, 0.f);
}

__global__ void __launch_bounds__(IA_BLOCK) k_interp_advance(IbmArgs a) {
    const int i = blockIdx.x * IA_BLOCK + threadIdx.x;
    if (i >= a.n_nodes) return;
    const CellDev C = a.cells[a.cell_of[i]];
    const ChannelDev Ch = a.ch[C.ch];
    const Q4 qn = advanced(a, Ch, i);
    const Q4 qr = (i == C.ref) ? qn : advanced(a, Ch, C.ref);
    (a.par ? a.qa : a.qb)[i] = qn;
    a.xr[i] = rel(qn, qr);
    a.dl[i] = disp(qn, a.q0[i], qr, a.q0[C.ref]);
}

cudaError_t launch_interp_advance(const IbmArgs& a, cudaStream_t s) {
    if (a.n_nodes <= 0) return cudaSuccess;
    k_interp_advance<<<(a.n_nodes + IA_BLOCK - 1) / IA_BLOCK, IA_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// Relative coordinates from the current fixed-point positions (after setup or
// after positions are overwritten).
__global__ void k_prepare_nodes(IbmArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_nodes) return;
    const CellDev C = a.cells[a.cell_of[i]];
    const Q4* qc = a.par ? a.qb : a.qa;
    const Q4 q = qc[i], qr = qc[C.ref];
    a.xr[i] = rel(q, qr);
    a.dl[i] = disp(q, a.q0[i], qr, a.q0[C.ref]);
}

cudaError_t launch_prepare_nodes(const IbmArgs& a, cudaStream_t s) {
    if (a.n_nodes <= 0) return cudaSuccess;
    k_prepare_nodes<<<(a.n_nodes + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbibm
