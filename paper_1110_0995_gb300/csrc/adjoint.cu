// Discrete adjoint of the differentiable variant of the immersed-boundary
// cycle (Brinkman beads, Sec. 2.1-2.3.1 with the bead reading stated in
// include/lbibm.h): per step, in reverse,
//   interpolation + advance  X' = X + sum_c w_c(X) u(x_c)
//   stream-collide           h'(x) = C(pull(h)(x), g(x), phi(x))
//   spreading                g(x) = sum_j w(x - X_j) F_j + G
//   membrane forces          F = F(X; ks, kb, ...)
// each as a vector-Jacobian product written out by hand.  The adjoint of the
// pull is a gather from the neighbours (the push, read backwards).  Element
// Jacobians are taken in forward mode (float dual numbers), so no second
// derivative is derived by hand: for the energy-derived edge forces one
// evaluation along the adjoint (symmetric Jacobian), for the triangle forces
// (the homocentric area force is not a gradient) one per input coordinate.
// Populations are FP32 (shifted storage h = f - w; the shift is a constant).
#include "lbibm_internal.cuh"

namespace lbibm {

constexpr unsigned AFULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// float dual number (value, tangent)
// ---------------------------------------------------------------------------
struct DF {
    float v, d;
};
__device__ __forceinline__ DF mk(float v, float d = 0.f) { return DF{v, d}; }
__device__ __forceinline__ DF operator+(DF a, DF b) { return DF{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ DF operator-(DF a, DF b) { return DF{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ DF operator-(DF a) { return DF{-a.v, -a.d}; }
__device__ __forceinline__ DF operator*(DF a, DF b) { return DF{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ DF operator*(float a, DF b) { return DF{a * b.v, a * b.d}; }
__device__ __forceinline__ DF operator/(DF a, DF b) { return DF{a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
__device__ __forceinline__ DF operator/(DF a, float b) { return DF{a.v / b, a.d / b}; }
__device__ __forceinline__ DF operator/(float a, DF b) { return DF{a / b.v, -a * b.d / (b.v * b.v)}; }
__device__ __forceinline__ DF operator+(float a, DF b) { return DF{a + b.v, b.d}; }
__device__ __forceinline__ DF operator+(DF a, float b) { return DF{a.v + b, a.d}; }
__device__ __forceinline__ DF operator-(float a, DF b) { return DF{a - b.v, -b.d}; }
__device__ __forceinline__ DF dsqrt(DF a) {
    const float r = sqrtf(a.v);
    return DF{r, 0.5f * a.d / r};
}
__device__ __forceinline__ DF datan2(DF y, DF x) {
    return DF{atan2f(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
}

struct V3 {
    DF x, y, z;
};
__device__ __forceinline__ V3 operator+(const V3& a, const V3& b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(const V3& a, const V3& b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(const V3& a) { return V3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(DF s, const V3& a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ DF dot(const V3& a, const V3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(const V3& a, const V3& b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{mk(x), mk(y), mk(z)}; }
__device__ __forceinline__ float tdot(const V3& a, float4 l) { return a.x.d * l.x + a.y.d * l.y + a.z.d * l.z; }
__device__ __forceinline__ float vdot(const V3& a, float4 l) { return a.x.v * l.x + a.y.v * l.y + a.z.v * l.z; }
__device__ __forceinline__ void seed(V3& a, int k) {
    if (k == 0) a.x.d = 1.f;
    else if (k == 1) a.y.d = 1.f;
    else a.z.d = 1.f;
}

// v * 2^-40 as float (v a small fixed-point difference)
__device__ __forceinline__ float fxa(long long v) {
    const int hi = (int)(v >> 20);
    const int lo = (int)(v & 0xFFFFF);
    return fmaf((float)hi, 9.5367431640625e-07f, (float)lo * FIX_INV_F);
}
__device__ __forceinline__ V3 rel(const Q4& a, const Q4& b) {   // x_b - x_a
    return v3(fxa(b.x - a.x), fxa(b.y - a.y), fxa(b.z - a.z));
}

__device__ __forceinline__ void atomic_add3(float4* p, float x, float y, float z) {
    atomicAdd(p, make_float4(x, y, z, 0.f));   // one 16-byte vector reduction
}

__device__ __forceinline__ const ChannelDev& achan(const AdjArgs& a) { return a.ch; }

// ---------------------------------------------------------------------------
// trilinear stencil of a fixed-point position (same weights as the forward:
// 24-bit fractions), with the gradient of each weight
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool acorner(const ChannelDev& C, const Q4& q, int c, long long& g, float& w, float3& dw) {
    const long long qq[3] = {q.x, q.y, q.z};
    const int n[3] = {C.nx, C.ny, C.nz};
    float fr[3], f1[3];
    int ic[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const unsigned f24 = (unsigned)((qq[d] >> (FIX_BITS - 24)) & 0xFFFFFF);
        const float f = __uint2float_rn(f24) * 5.9604644775390625e-08f;
        const int cc = (c >> d) & 1;
        fr[d] = cc ? f : 1.0f - f;                 // factor of this axis
        f1[d] = cc ? 1.0f : -1.0f;                 // its derivative
        int v = (int)(qq[d] >> FIX_BITS) + cc;
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
    w = fr[0] * fr[1] * fr[2];
    dw = make_float3(f1[0] * fr[1] * fr[2], fr[0] * f1[1] * fr[2], fr[0] * fr[1] * f1[2]);
    g = ok ? C.base + ic[0] + (long long)C.nx * (ic[1] + (long long)C.ny * ic[2]) : 0;
    return ok;
}

// Eight lanes per IB node, lane c taking stencil corner c; partial sums are
// added over the eight lanes by shuffles.
constexpr int ADJ_SUB = 8;

__device__ __forceinline__ float sub_sum(float v, unsigned smask) {
#pragma unroll
    for (int o = ADJ_SUB / 2; o > 0; o >>= 1) v += __shfl_xor_sync(smask, v, o);
    return v;
}

// (B1) interpolation + advance, reversed: lam_u(x_c) += w_c lamX, and
// lamX_out = lamX + sum_c grad w_c (u(x_c) . lamX).
__global__ void k_adj_interp(const __grid_constant__ AdjArgs a) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // the cycle's per-cell sums (B5) start from zero; the previous cycle's
    // reader (B6) has completed
    for (int k = t; k < 2 * a.n_cells; k += gridDim.x * blockDim.x) a.lam_c[k] = 0.0;
    const int j = t / ADJ_SUB, c = t & (ADJ_SUB - 1);
    if (j >= a.M) return;   // whole groups of eight lanes leave together
    const unsigned smask = 0xffu << (threadIdx.x & 24);
    const Q4 q = a.q_t[j];
    const float4 l = a.lamX[j];
    float gx = 0.f, gy = 0.f, gz = 0.f;
    long long g;
    float w;
    float3 dw;
    if (acorner(a.ch, q, c, g, w, dw)) {
        const float4 u = a.u_t[g];
        const float s = u.x * l.x + u.y * l.y + u.z * l.z;
        gx = dw.x * s; gy = dw.y * s; gz = dw.z * s;
        atomicAdd(a.lam_u + g, make_float4(w * l.x, w * l.y, w * l.z, 0.f));
    }
    gx = sub_sum(gx, smask);
    gy = sub_sum(gy, smask);
    gz = sub_sum(gz, smask);
    if (c == 0) a.lamX_out[j] = make_float4(l.x + gx, l.y + gy, l.z + gz, 0.f);
}

// (B3) spreading, reversed: lamF_j = sum_c w_c lam_g(x_c);
// lamX_out += sum_c grad w_c (F_j . lam_g(x_c)).
__global__ void k_adj_spread(const __grid_constant__ AdjArgs a) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = t / ADJ_SUB, c = t & (ADJ_SUB - 1);
    if (j >= a.M) return;
    const unsigned smask = 0xffu << (threadIdx.x & 24);
    const Q4 q = a.q_t[j];
    const float4 F = a.F_t[j];
    float lx = 0.f, ly = 0.f, lz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    long long g;
    float w;
    float3 dw;
    if (acorner(a.ch, q, c, g, w, dw) && !((__ldg(a.mask + (g >> 5)) >> (g & 31)) & 1u)) {
        const float4 lg = a.lam_g[g];
        lx = w * lg.x; ly = w * lg.y; lz = w * lg.z;
        const float s = F.x * lg.x + F.y * lg.y + F.z * lg.z;
        gx = dw.x * s; gy = dw.y * s; gz = dw.z * s;
    }
    lx = sub_sum(lx, smask);
    ly = sub_sum(ly, smask);
    lz = sub_sum(lz, smask);
    gx = sub_sum(gx, smask);
    gy = sub_sum(gy, smask);
    gz = sub_sum(gz, smask);
    if (c == 0) {
        a.lamF[j] = make_float4(lx, ly, lz, 0.f);
        float4 o = a.lamX_out[j];
        o.x += gx; o.y += gy; o.z += gz;
        a.lamX_out[j] = o;
    }
}

// ---------------------------------------------------------------------------
// (B4) edges: stretching + bending, reversed.  Positions relative to vertex a
// (the forces depend on differences only, so the column of a is minus the sum
// of the others).  9 forward-mode columns per edge.
// ---------------------------------------------------------------------------
template <bool VALUES>
__device__ __forceinline__ void edge_forces(const V3& xb, const V3& xc, const V3& xd, float L0, float th0, float ks,
                                            float kb, V3 fs[2], V3 fb[4]) {
    // stretching (neo-Hookean bond): tension ks kappa(lambda) (lambda - 1) along the edge
    const DF L = dsqrt(dot(xb, xb));
    const DF lam = L / L0;
    const DF sl = dsqrt(lam);
    const DF l2 = lam * lam;
    const DF kappa = (sl + 1.0f / (l2 * sl)) / (lam + 1.0f / (l2 * lam));
    const DF T = ks * (kappa * (lam + (-1.0f)));
    fs[0] = (T / L) * xb;
    fs[1] = -fs[0];
    // bending: E = kb/2 (theta - theta0)^2 at edge (a, b), triangles (a, b, c), (b, a, d)
    const V3 e = xb, ac = xc, ad = xd;
    const V3 bd = ad - e;
    const V3 n1 = cross(e, ac);
    const V3 n2 = cross(-e, bd);
    const DF el2 = dot(e, e);
    const DF el = dsqrt(el2);
    const DF theta = datan2(dot(cross(n1, n2), e) / el, dot(n1, n2));
    const DF coef = -kb * (theta + (-th0));
    const V3 gc = (-(el / dot(n1, n1))) * n1;
    const V3 gd = (-(el / dot(n2, n2))) * n2;
    const DF sc = dot(ac, e) / el2;
    const DF sd = dot(ad, e) / el2;
    fb[0] = coef * ((-(1.0f - sc)) * gc - (1.0f - sd) * gd);
    fb[1] = coef * ((-sc) * gc - sd * gd);
    fb[2] = coef * gc;
    fb[3] = coef * gd;
}

// Stretching and bending forces are minus the gradients of energies
// (E = L0 int T(lambda) dlambda per bond, E = kb/2 (theta - theta0)^2 per
// edge), so their Jacobian with respect to the four vertices is symmetric
// (minus the Hessian) and the vector-Jacobian product with lamF is the
// Jacobian-vector product along lamF: one forward-mode evaluation per edge,
// seeded with the adjoint itself (relative to vertex a, the seeds are
// lamF_v - lamF_a).
__device__ __forceinline__ void adj_edges_block(const AdjArgs& a, int blk) {
    const int e = blk * blockDim.x + threadIdx.x;
    float gks = 0.f, gkb = 0.f;   // (FP32 within a warp, FP64 across warps and steps)
    if (e < a.n_edges) {
        const int4 ev = a.edges[e];
        const float4 er = a.edge_rest[e];   // (L0, theta0, ks, kb)
        const Q4 qa = a.q_t[ev.x], qb = a.q_t[ev.y], qc = a.q_t[ev.z], qd = a.q_t[ev.w];
        const float4 la = a.lamF[ev.x], lb = a.lamF[ev.y], lc = a.lamF[ev.z], ld = a.lamF[ev.w];
        V3 xb = rel(qa, qb), xc = rel(qa, qc), xd = rel(qa, qd);
        xb.x.d = lb.x - la.x; xb.y.d = lb.y - la.y; xb.z.d = lb.z - la.z;
        xc.x.d = lc.x - la.x; xc.y.d = lc.y - la.y; xc.z.d = lc.z - la.z;
        xd.x.d = ld.x - la.x; xd.y.d = ld.y - la.y; xd.z.d = ld.z - la.z;
        V3 fs[2], fb[4];
        edge_forces<false>(xb, xc, xd, er.x, er.y, er.z, er.w, fs, fb);
        atomic_add3(a.lamX_out + ev.x, fs[0].x.d + fb[0].x.d, fs[0].y.d + fb[0].y.d, fs[0].z.d + fb[0].z.d);
        atomic_add3(a.lamX_out + ev.y, fs[1].x.d + fb[1].x.d, fs[1].y.d + fb[1].y.d, fs[1].z.d + fb[1].z.d);
        atomic_add3(a.lamX_out + ev.z, fb[2].x.d, fb[2].y.d, fb[2].z.d);
        atomic_add3(a.lamX_out + ev.w, fb[3].x.d, fb[3].y.d, fb[3].z.d);
        if (a.info[ev.x].x == a.obj_cell) {
            // parameter gradients (the forces are linear in ks and kb)
            if (er.z != 0.f) gks = (vdot(fs[0], la) + vdot(fs[1], lb)) / er.z;
            if (er.w != 0.f) gkb = (vdot(fb[0], la) + vdot(fb[1], lb) + vdot(fb[2], lc) + vdot(fb[3], ld)) / er.w;
        }
    }
    if (!__any_sync(AFULL, gks != 0.f || gkb != 0.f)) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gks += __shfl_down_sync(AFULL, gks, o);
        gkb += __shfl_down_sync(AFULL, gkb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.grad + 0, (double)gks);
        atomicAdd(a.grad + 1, (double)gkb);
    }
}

// ---------------------------------------------------------------------------
// (B5) triangles: local area (with the cell's global terms held fixed),
// global area and volume, reversed.  Force on vertex i:
//   F_i = (kal dS_t/S0_t + c1) a_i - c2 n_t,   a_i = -(2 S_t / sum |w|^2) w_i,
//   c1 = kag (S - S0)/S0, c2 = kv (V - V0)/(6 V0).
// Writes the column products, accumulates per cell lam_c1 = sum lamF . a_i and
// lam_c2 = -sum lamF . n_t, and keeps dS_t/dx_b, dS_t/dx_c and n_t for (B6).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_forces(const V3& xb, const V3& xc, float S0t, float kal, float c1, float c2,
                                           V3 f[3], V3 av[3], V3& n, DF& St) {
    n = cross(xb, xc);
    St = 0.5f * dsqrt(dot(n, n));
    const V3 third = V3{(xb.x + xc.x) / 3.0f, (xb.y + xc.y) / 3.0f, (xb.z + xc.z) / 3.0f};
    const V3 w0 = -third, w1 = xb - third, w2 = xc - third;
    const DF ww = dot(w0, w0) + dot(w1, w1) + dot(w2, w2);
    const DF cw = -(2.0f * St) / ww;
    av[0] = cw * w0; av[1] = cw * w1; av[2] = cw * w2;
    const DF ca = kal * ((St + (-S0t)) / S0t) + c1;
    f[0] = ca * av[0] - mk(c2) * n;
    f[1] = ca * av[1] - mk(c2) * n;
    f[2] = ca * av[2] - mk(c2) * n;
}

// One thread per (triangle, column): column v*3+k seeds coordinate k of vertex
// b or c (v = 0, 1); the column of a is minus their sum.  The column-0 thread
// also forms the per-cell products and keeps the normal.
__device__ __forceinline__ void adj_tris_block(const AdjArgs& a, int blk) {
    const int tid = blk * blockDim.x + threadIdx.x;
    const int t = tid / 6, col = tid - 6 * (tid / 6);
    const bool valid = t < a.n_tris;   // every lane stays for the per-cell warp sums
    int cell = -1;
    float lc1 = 0.f, lc2 = 0.f;
    if (valid) {
        const int4 tr = a.tris[t];
        const CellDev& C = a.cells[tr.w];
        const float2 rel_sv = a.rel_t[tr.w];   // (dS/S0, dV/V0) of this step
        const float c1 = C.kag * rel_sv.x, c2 = C.kv * rel_sv.y / 6.0f;
        const Q4 qa = a.q_t[tr.x], qb = a.q_t[tr.y], qc = a.q_t[tr.z];
        const float4 la = a.lamF[tr.x], lb = a.lamF[tr.y], lc = a.lamF[tr.z];
        V3 xb = rel(qa, qb), xc = rel(qa, qc);
        const int v = col / 3, k = col % 3;
        if (v == 0) seed(xb, k);
        else seed(xc, k);
        V3 f[3], av[3], n;
        DF St;
        tri_forces(xb, xc, a.tri_S0[t], C.kal, c1, c2, f, av, n, St);
        const float acc = tdot(f[0], la) + tdot(f[1], lb) + tdot(f[2], lc);
        atomicAdd(reinterpret_cast<float*>(a.lamX_out + (v == 0 ? tr.y : tr.z)) + k, acc);
        atomicAdd(reinterpret_cast<float*>(a.lamX_out + tr.x) + k, -acc);
        reinterpret_cast<float*>(a.tri_dS)[6 * t + col] = St.d;
        if (col == 0) {
            cell = tr.w;
            lc1 = vdot(av[0], la) + vdot(av[1], lb) + vdot(av[2], lc);
            lc2 = -(vdot(n, la) + vdot(n, lb) + vdot(n, lc));
            a.tri_n[t] = make_float4(n.x.v, n.y.v, n.z.v, 0.f);
        }
    }
    // per-cell sums lam_c1, lam_c2 over the column-0 lanes: one atomic per cell per warp
    const bool has = cell >= 0;
    const int lane = threadIdx.x & 31;
    unsigned rem = __ballot_sync(AFULL, has);
    while (rem) {
        const int l0 = __ffs(rem) - 1;
        const int c = __shfl_sync(AFULL, cell, l0);
        const bool mine = has && cell == c;
        float s1 = mine ? lc1 : 0.f, s2 = mine ? lc2 : 0.f;   // (FP32 within a warp)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(AFULL, s1, o);
            s2 += __shfl_xor_sync(AFULL, s2, o);
        }
        if (lane == l0) {
            atomicAdd(a.lam_c + 2 * c, (double)s1);
            atomicAdd(a.lam_c + 2 * c + 1, (double)s2);
        }
        rem &= ~__ballot_sync(AFULL, mine);
    }
}

// (B4) + (B5) in one launch: blocks [0, edge_blocks) take the edges, the rest
// the triangle columns (the two are independent; B6 follows).
__global__ void __launch_bounds__(128, 6) k_adj_membrane(const __grid_constant__ AdjArgs a, int edge_blocks) {
    pdl_entry();
    if ((int)blockIdx.x < edge_blocks) adj_edges_block(a, blockIdx.x);
    else adj_tris_block(a, (int)blockIdx.x - edge_blocks);
}

// (B6) the cell's global terms: lam_S = lam_c1 kag / S0, lam_V = lam_c2 kv / (6 V0);
// dS/dx from the triangles' areas, dV/dx_k = sum over triangles at k of n_t / 6.
__global__ void k_adj_tris_global(const __grid_constant__ AdjArgs a) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tris) return;
    const int4 tr = a.tris[t];
    const CellDev& C = a.cells[tr.w];
    const float lS = (float)a.lam_c[2 * tr.w] * C.kag_S0;
    const float lV = (float)a.lam_c[2 * tr.w + 1] * C.kv_6V0;
    const float* ds = reinterpret_cast<const float*>(a.tri_dS) + 6 * t;
    const float3 db = make_float3(ds[0], ds[1], ds[2]), dc = make_float3(ds[3], ds[4], ds[5]);
    const float4 n = a.tri_n[t];
    const float vn = lV / 6.0f;
    atomic_add3(a.lamX_out + tr.y, lS * db.x + vn * n.x, lS * db.y + vn * n.y, lS * db.z + vn * n.z);
    atomic_add3(a.lamX_out + tr.z, lS * dc.x + vn * n.x, lS * dc.y + vn * n.y, lS * dc.z + vn * n.z);
    atomic_add3(a.lamX_out + tr.x, -lS * (db.x + dc.x) + vn * n.x, -lS * (db.y + dc.y) + vn * n.y,
                -lS * (db.z + dc.z) + vn * n.z);
}

// dJ/dc_k = sum_x Lphi(x) dphi(x)/dc_k, with phi = 1 - prod_j (1 - phi_j):
// dphi/dc_k = prod_{j != k} (1 - phi_j) dphi_k/dc_k,
// dphi_k/dc_k = (1 - tanh^2 s) / (2 delta) (x - c_k)/|x - c_k|, s = (|x - c_k| - r_k)/delta.
constexpr int BG_MAXB = 64;
__global__ void k_adj_bead_grad(const __grid_constant__ AdjArgs a) {
    const ChannelDev& C = a.ch;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int nb = a.n_beads;
    float lp = 0.f;
    int x = 0, y = 0, z = 0;
    if (p < C.n) {
        lp = a.Lphi[C.base + p];
        const int r = fdiv(p, C.dnx);
        x = p - r * C.nx;
        z = fdiv(r, C.dny);
        y = r - z * C.ny;
    }
    float om[BG_MAXB];   // 1 - phi_j
    float prod = 1.f;
    for (int k = 0; k < nb; ++k) {
        const float4 b = a.beads[k];
        const float dx = (float)x - b.x, dy = (float)y - b.y, dz = (float)z - b.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);
        om[k] = 1.0f - 0.5f * (1.0f - tanhf((d - b.w) / a.delta));
        prod *= om[k];
    }
    for (int k = 0; k < nb; ++k) {
        const float4 b = a.beads[k];
        const float dx = (float)x - b.x, dy = (float)y - b.y, dz = (float)z - b.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (p < C.n && d > 0.f && lp != 0.f) {
            float others = 1.f;
            for (int j = 0; j < nb; ++j)
                if (j != k) others *= om[j];
            const float t = tanhf((d - b.w) / a.delta);
            const float s = lp * others * 0.5f * (1.0f - t * t) / a.delta / d;
            gx = s * dx; gy = s * dy; gz = s * dz;
        }
        float sx = gx, sy = gy, sz = gz;   // (FP32 within a warp)
        if (!__any_sync(AFULL, sx != 0.f || sy != 0.f || sz != 0.f)) continue;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_down_sync(AFULL, sx, o);
            sy += __shfl_down_sync(AFULL, sy, o);
            sz += __shfl_down_sync(AFULL, sz, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.grad + 2 + 3 * k, (double)sx);
            atomicAdd(a.grad + 3 + 3 * k, (double)sy);
            atomicAdd(a.grad + 4 + 3 * k, (double)sz);
        }
    }
    (void)prod;
}

// ---- launchers ----
cudaError_t launch_adj_interp(const AdjArgs& a, cudaStream_t s) {
    return launch_ex(k_adj_interp, (ADJ_SUB * a.M + 127) / 128, 128, 0, s, a.pdl, a);
}
cudaError_t launch_adj_spread(const AdjArgs& a, cudaStream_t s) {
    return launch_ex(k_adj_spread, (ADJ_SUB * a.M + 127) / 128, 128, 0, s, a.pdl, a);
}
cudaError_t launch_adj_membrane(const AdjArgs& a, cudaStream_t s) {
    const int eb = (a.n_edges + 127) / 128, tb = (6 * a.n_tris + 127) / 128;
    if (eb + tb == 0) return cudaSuccess;
    cudaError_t e = launch_ex(k_adj_membrane, eb + tb, 128, 0, s, a.pdl, a, eb);
    if (a.n_tris > 0 && e == cudaSuccess) e = launch_ex(k_adj_tris_global, (a.n_tris + 127) / 128, 128, 0, s, a.pdl, a);
    return e;
}
cudaError_t launch_adj_bead_grad(const AdjArgs& a, cudaStream_t s) {
    if (a.n_beads <= 0) return cudaSuccess;
    if (a.n_beads > BG_MAXB) return cudaErrorInvalidValue;
    k_adj_bead_grad<<<(a.ch.n + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbibm
