// Discrete adjoint of the differentiable variant of the immersed-boundary
// cycle (Brinkman beads, Sec. 2.1-2.3.1 with the bead reading stated in
// include/lbibm.h): per step, in reverse,
//   interpolation + advance  X' = X + sum_c w_c(X) u(x_c)
//   stream-collide           h'(x) = C(pull(h)(x), g(x), phi(x))
//   spreading                g(x) = sum_j w(x - X_j) F_j + G
//   membrane forces          F = F(X; ks, kb, ...)
// each as a vector-Jacobian product written out by hand.  The adjoint of the
// pull is a gather from the neighbours (the push, read backwards).  Element
// Jacobians are taken column by column in forward mode (a float dual number
// per input coordinate), so no second derivative is derived by hand.
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
    float* f = reinterpret_cast<float*>(p);
    atomicAdd(f, x);
    atomicAdd(f + 1, y);
    atomicAdd(f + 2, z);
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

// (B1) interpolation + advance, reversed: lam_u(x_c) += w_c lamX, and
// lamX_out = lamX + sum_c grad w_c (u(x_c) . lamX).
__global__ void k_adj_interp(const __grid_constant__ AdjArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.M) return;
    const Q4 q = a.q_t[j];
    const float4 l = a.lamX[j];
    float gx = l.x, gy = l.y, gz = l.z;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        long long g;
        float w;
        float3 dw;
        if (!acorner(a.ch, q, c, g, w, dw)) continue;
        const float4 u = a.u_t[g];
        const float s = u.x * l.x + u.y * l.y + u.z * l.z;
        gx += dw.x * s; gy += dw.y * s; gz += dw.z * s;
        atomic_add3(a.lam_u + g, w * l.x, w * l.y, w * l.z);
    }
    a.lamX_out[j] = make_float4(gx, gy, gz, 0.f);
}

// (B3) spreading, reversed: lamF_j = sum_c w_c lam_g(x_c);
// lamX_out += sum_c grad w_c (F_j . lam_g(x_c)).
__global__ void k_adj_spread(const __grid_constant__ AdjArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.M) return;
    const Q4 q = a.q_t[j];
    const float4 F = a.F_t[j];
    float lx = 0.f, ly = 0.f, lz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        long long g;
        float w;
        float3 dw;
        if (!acorner(a.ch, q, c, g, w, dw)) continue;
        if ((__ldg(a.mask + (g >> 5)) >> (g & 31)) & 1u) continue;
        const float4 lg = a.lam_g[g];
        lx += w * lg.x; ly += w * lg.y; lz += w * lg.z;
        const float s = F.x * lg.x + F.y * lg.y + F.z * lg.z;
        gx += dw.x * s; gy += dw.y * s; gz += dw.z * s;
    }
    a.lamF[j] = make_float4(lx, ly, lz, 0.f);
    float4 o = a.lamX_out[j];
    o.x += gx; o.y += gy; o.z += gz;
    a.lamX_out[j] = o;
}

// ---------------------------------------------------------------------------
// (B2) stream-collide, reversed, one node per thread.  Gathers the adjoint of
// this step's output h'(x) from the adjoint of the next step's pulled
// populations (lam_in): the next step pulled h'_k(x) at x + e_k, or at x
// itself as direction opp(k) when that link bounces back.  Then the
// vector-Jacobian product of the collision with respect to the pulled
// populations (lam_out), the force density (lam_g) and the solid fraction
// (accumulated into Lphi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int nb_off(const ChannelDev& C, int x, int y, int z, int dx, int dy, int dz, bool& ok) {
    ok = true;
    int xs = x + dx, ys = y + dy, zs = z + dz;
    if (xs < 0 || xs >= C.nx) { if (C.per[0]) xs = (xs + C.nx) % C.nx; else ok = false; }
    if (ys < 0 || ys >= C.ny) { if (C.per[1]) ys = (ys + C.ny) % C.ny; else ok = false; }
    if (zs < 0 || zs >= C.nz) { if (C.per[2]) zs = (zs + C.nz) % C.nz; else ok = false; }
    return ok ? (xs - x) + C.nx * ((ys - y) + C.ny * (zs - z)) : 0;
}

__global__ void __launch_bounds__(128) k_adj_collide(const __grid_constant__ AdjArgs a) {
    const ChannelDev& C = a.ch;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const long long gp = C.base + p;
    if ((__ldg(a.mask + (gp >> 5)) >> (gp & 31)) & 1u) return;   // bitmask obstacle nodes do not update
    const int r = fdiv(p, C.dnx);
    const int x = p - r * C.nx;
    const int z = fdiv(r, C.dny);
    const int y = r - z * C.ny;
    const long long NT = a.plane;
    const uint32_t lk = __ldg(a.links + gp);
    float f[Q], lh[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // pulled population (forward): from x - e_i, or bounced back
        bool ok;
        const int o = nb_off(C, x, y, z, -ex(i), -ey(i), -ez(i), ok);
        if ((lk >> i) & 1u) ok = false;
        float v = ok ? __ldg(a.h_t + (long long)i * NT + gp + o) : __ldg(a.h_t + (long long)opp(i) * NT + gp);
        if (!ok && C.has_uw && !C.per[1]) {
            const int wall = (ey(i) == 1 && y == 0) ? 0 : ((ey(i) == -1 && y == C.ny - 1) ? 1 : -1);
            if (wall >= 0) v += 6.0f * wgt(i) * (ex(i) * C.uw[wall][0] + ey(i) * C.uw[wall][1] + ez(i) * C.uw[wall][2]);
        }
        f[i] = v;
        // adjoint of this node's output h'_i: the next step pulled it at x + e_i,
        // unless that link bounces (bit opp(i) of this node's mask)
        bool ok2;
        const int o2 = nb_off(C, x, y, z, ex(i), ey(i), ez(i), ok2);
        if ((lk >> opp(i)) & 1u) ok2 = false;
        lh[i] = ok2 ? __ldg(a.lam_in + (long long)i * NT + gp + o2) : __ldg(a.lam_in + (long long)opp(i) * NT + gp);
    }
    // forward quantities (shifted populations: rho = 1 + sum h)
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += f[i];
        jx += ex(i) * f[i]; jy += ey(i) * f[i]; jz += ez(i) * f[i];
    }
    const float rho = 1.0f + drho;
    const float4 gs = a.g_t[gp];
    const float gx = gs.x + C.G[0], gy = gs.y + C.G[1], gz = gs.z + C.G[2];
    const float phi = a.phi ? __ldg(a.phi + gp) : 0.f;
    const float al = a.alpha * phi;
    const float D = 1.0f + 0.5f * al;
    const float vx = jx + 0.5f * gx, vy = jy + 0.5f * gy, vz = jz + 0.5f * gz;
    const float ux = vx / (rho * D), uy = vy / (rho * D), uz = vz / (rho * D);
    const float tx = gx - al * vx / D, ty = gy - al * vy / D, tz = gz - al * vz / D;   // g_tot
    const float uu = ux * ux + uy * uy + uz * uz;
    const float om = C.omega, fp = C.fpre;   // omega = 1/tau, fp = 1 - omega/2
    // sums over the outputs h'_i = (1 - om) f_i + om feq_i(rho, u) + S_i(u, g_tot)
    float lrho = 0.f, lux = 0.f, luy = 0.f, luz = 0.f, ltx = 0.f, lty = 0.f, ltz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float L = lh[i];
        const float w = wgt(i);
        const float eu = ex(i) * ux + ey(i) * uy + ez(i) * uz;
        const float et = ex(i) * tx + ey(i) * ty + ez(i) * tz;
        // d feq_i / d rho = w (1 + 3 eu + 4.5 eu^2 - 1.5 uu)
        lrho += L * om * w * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
        // d feq_i / d u = w rho (3 e + 9 eu e - 3 u);  d S_i / d u = fp w (-3 t + 9 et e)
        const float a1 = om * w * rho * (3.0f + 9.0f * eu) + fp * w * 9.0f * et;
        const float a2 = -3.0f * om * w * rho;
        const float a3 = -3.0f * fp * w;
        lux += L * (a1 * ex(i) + a2 * ux + a3 * tx);
        luy += L * (a1 * ey(i) + a2 * uy + a3 * ty);
        luz += L * (a1 * ez(i) + a2 * uz + a3 * tz);
        // d S_i / d g_tot = fp w (3 (e - u) + 9 eu e)
        const float b1 = fp * w * (3.0f + 9.0f * eu);
        const float b2 = -3.0f * fp * w;
        ltx += L * (b1 * ex(i) + b2 * ux);
        lty += L * (b1 * ey(i) + b2 * uy);
        ltz += L * (b1 * ez(i) + b2 * uz);
    }
    // the interpolation's use of u
    const float4 lu = a.lam_u[gp];
    lux += lu.x; luy += lu.y; luz += lu.z;
    // u = v / (rho D), g_tot = g - al v / D, v = j + g/2
    const float irD = 1.0f / (rho * D);
    const float lvx = lux * irD - ltx * al / D, lvy = luy * irD - lty * al / D, lvz = luz * irD - ltz * al / D;
    lrho -= (lux * ux + luy * uy + luz * uz) / rho;
    const float lgx = 0.5f * lvx + ltx, lgy = 0.5f * lvy + lty, lgz = 0.5f * lvz + ltz;
    // pulled populations: direct (1 - om), through rho (1) and j (e_i)
    float* lo = a.lam_out;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        lo[(long long)i * NT + gp] = (1.0f - om) * lh[i] + lrho + ex(i) * lvx + ey(i) * lvy + ez(i) * lvz;
    a.lam_g[gp] = make_float4(lgx, lgy, lgz, 0.f);
    if (a.phi) {
        // d u / d phi = -(alpha/2) v / (rho D^2);  d g_tot / d phi = -alpha v / D^2
        const float iD2 = 1.0f / (D * D);
        const float lphi = -0.5f * a.alpha * (lux * vx + luy * vy + luz * vz) * iD2 / rho -
                           a.alpha * (ltx * vx + lty * vy + ltz * vz) * iD2;
        a.Lphi[gp] += lphi;
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

__global__ void k_adj_edges(const __grid_constant__ AdjArgs a) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double gks = 0.0, gkb = 0.0;
    if (e < a.n_edges) {
        const int4 ev = a.edges[e];
        const float4 er = a.edge_rest[e];   // (L0, theta0, ks, kb)
        const Q4 qa = a.q_t[ev.x], qb = a.q_t[ev.y], qc = a.q_t[ev.z], qd = a.q_t[ev.w];
        const float4 la = a.lamF[ev.x], lb = a.lamF[ev.y], lc = a.lamF[ev.z], ld = a.lamF[ev.w];
        const V3 xb0 = rel(qa, qb), xc0 = rel(qa, qc), xd0 = rel(qa, qd);
        float acc[3][3];
#pragma unroll 1
        for (int col = 0; col < 9; ++col) {
            V3 xb = xb0, xc = xc0, xd = xd0;
            const int v = col / 3, k = col % 3;
            if (v == 0) seed(xb, k);
            else if (v == 1) seed(xc, k);
            else seed(xd, k);
            V3 fs[2], fb[4];
            edge_forces<false>(xb, xc, xd, er.x, er.y, er.z, er.w, fs, fb);
            acc[v][k] = tdot(fs[0], la) + tdot(fs[1], lb) + tdot(fb[0], la) + tdot(fb[1], lb) + tdot(fb[2], lc) +
                        tdot(fb[3], ld);
            if (col == 0 && a.info[ev.x].x == a.obj_cell) {
                // parameter gradients (values are linear in ks and kb)
                if (er.z != 0.f) gks = (double)((vdot(fs[0], la) + vdot(fs[1], lb)) / er.z);
                if (er.w != 0.f)
                    gkb = (double)((vdot(fb[0], la) + vdot(fb[1], lb) + vdot(fb[2], lc) + vdot(fb[3], ld)) / er.w);
            }
        }
        atomic_add3(a.lamX_out + ev.y, acc[0][0], acc[0][1], acc[0][2]);
        atomic_add3(a.lamX_out + ev.z, acc[1][0], acc[1][1], acc[1][2]);
        atomic_add3(a.lamX_out + ev.w, acc[2][0], acc[2][1], acc[2][2]);
        atomic_add3(a.lamX_out + ev.x, -(acc[0][0] + acc[1][0] + acc[2][0]), -(acc[0][1] + acc[1][1] + acc[2][1]),
                    -(acc[0][2] + acc[1][2] + acc[2][2]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gks += __shfl_down_sync(AFULL, gks, o);
        gkb += __shfl_down_sync(AFULL, gkb, o);
    }
    if ((threadIdx.x & 31) == 0 && (gks != 0.0 || gkb != 0.0)) {
        atomicAdd(a.grad + 0, gks);
        atomicAdd(a.grad + 1, gkb);
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

__global__ void k_adj_tris(const __grid_constant__ AdjArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tris) return;
    const int4 tr = a.tris[t];
    const CellDev& C = a.cells[tr.w];
    const float2 rel_sv = a.rel_t[tr.w];   // (dS/S0, dV/V0) of this step
    const float c1 = C.kag * rel_sv.x, c2 = C.kv * rel_sv.y / 6.0f;
    const Q4 qa = a.q_t[tr.x], qb = a.q_t[tr.y], qc = a.q_t[tr.z];
    const float4 la = a.lamF[tr.x], lb = a.lamF[tr.y], lc = a.lamF[tr.z];
    const V3 xb0 = rel(qa, qb), xc0 = rel(qa, qc);
    const float S0t = a.tri_S0[t];
    float acc[2][3], dS[2][3];
    float lc1 = 0.f, lc2 = 0.f;
    V3 n0;
#pragma unroll 1
    for (int col = 0; col < 6; ++col) {
        V3 xb = xb0, xc = xc0;
        const int v = col / 3, k = col % 3;
        if (v == 0) seed(xb, k);
        else seed(xc, k);
        V3 f[3], av[3], n;
        DF St;
        tri_forces(xb, xc, S0t, C.kal, c1, c2, f, av, n, St);
        acc[v][k] = tdot(f[0], la) + tdot(f[1], lb) + tdot(f[2], lc);
        dS[v][k] = St.d;
        if (col == 0) {
            lc1 = vdot(av[0], la) + vdot(av[1], lb) + vdot(av[2], lc);
            lc2 = -(vdot(n, la) + vdot(n, lb) + vdot(n, lc));
            n0 = n;
        }
    }
    atomic_add3(a.lamX_out + tr.y, acc[0][0], acc[0][1], acc[0][2]);
    atomic_add3(a.lamX_out + tr.z, acc[1][0], acc[1][1], acc[1][2]);
    atomic_add3(a.lamX_out + tr.x, -(acc[0][0] + acc[1][0]), -(acc[0][1] + acc[1][1]), -(acc[0][2] + acc[1][2]));
    a.tri_dS[2 * t] = make_float4(dS[0][0], dS[0][1], dS[0][2], 0.f);
    a.tri_dS[2 * t + 1] = make_float4(dS[1][0], dS[1][1], dS[1][2], 0.f);
    a.tri_n[t] = make_float4(n0.x.v, n0.y.v, n0.z.v, 0.f);
    atomicAdd(a.lam_c + 2 * tr.w, (double)lc1);
    atomicAdd(a.lam_c + 2 * tr.w + 1, (double)lc2);
}

// (B6) the cell's global terms: lam_S = lam_c1 kag / S0, lam_V = lam_c2 kv / (6 V0);
// dS/dx from the triangles' areas, dV/dx_k = sum over triangles at k of n_t / 6.
__global__ void k_adj_tris_global(const __grid_constant__ AdjArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tris) return;
    const int4 tr = a.tris[t];
    const CellDev& C = a.cells[tr.w];
    const float lS = (float)(a.lam_c[2 * tr.w] * (double)C.kag / C.S0);
    const float lV = (float)(a.lam_c[2 * tr.w + 1] * (double)C.kv / (6.0 * C.V0));
    const float4 db = a.tri_dS[2 * t], dc = a.tri_dS[2 * t + 1], n = a.tri_n[t];
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
        double sx = gx, sy = gy, sz = gz;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_down_sync(AFULL, sx, o);
            sy += __shfl_down_sync(AFULL, sy, o);
            sz += __shfl_down_sync(AFULL, sz, o);
        }
        if ((threadIdx.x & 31) == 0 && (sx != 0.0 || sy != 0.0 || sz != 0.0)) {
            atomicAdd(a.grad + 2 + 3 * k, sx);
            atomicAdd(a.grad + 3 + 3 * k, sy);
            atomicAdd(a.grad + 4 + 3 * k, sz);
        }
    }
    (void)prod;
}

// ---- launchers ----
cudaError_t launch_adj_interp(const AdjArgs& a, cudaStream_t s) {
    k_adj_interp<<<(a.M + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_adj_collide(const AdjArgs& a, cudaStream_t s) {
    k_adj_collide<<<(a.ch.n + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_adj_spread(const AdjArgs& a, cudaStream_t s) {
    k_adj_spread<<<(a.M + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_adj_membrane(const AdjArgs& a, cudaStream_t s) {
    if (a.n_edges > 0) k_adj_edges<<<(a.n_edges + 127) / 128, 128, 0, s>>>(a);
    if (a.n_tris > 0) {
        k_adj_tris<<<(a.n_tris + 127) / 128, 128, 0, s>>>(a);
        k_adj_tris_global<<<(a.n_tris + 127) / 128, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}
cudaError_t launch_adj_bead_grad(const AdjArgs& a, cudaStream_t s) {
    if (a.n_beads <= 0) return cudaSuccess;
    if (a.n_beads > BG_MAXB) return cudaErrorInvalidValue;
    k_adj_bead_grad<<<(a.ch.n + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbibm
