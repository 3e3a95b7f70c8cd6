// Lattice kernels: obstacle rasterisation, the fused pull-scheme
// stream-collide-force step, field / population export and FP64 diagnostics.
//
// Method: Gusenbauer et al., arXiv:1110.0995, Sec. 2.1 (D3Q19 LB equation with
// external force F_i), Sec. 2.4 (bounce-back at walls and obstacle nodes; no
// inside/outside distinction for the force).  Readings: second-order
// equilibrium, Guo forcing with the half-force velocity, halfway bounce-back
// with Ladd's moving-wall term (rho0 = 1).
//
// Storage is shifted: h_i = f_i - w_i (rho0 = 1), so the moments are sums of
// small numbers (FP32 keeps ~1e-7 relative accuracy on u ~ 1e-3 instead of
// ~1e-5 with f_i ~ 0.05).  The half/bfloat16 modes store h_i / w_i.
//
// The stream-collide kernel handles NPT consecutive x-nodes per thread: every
// direction is one aligned NPT-wide vector load (128-bit for FP32 with NPT = 4)
// of the source row; the +-x shifted directions take their missing element
// from the neighbouring lane with a warp shuffle.  Warps whose 32-node groups
// touch an obstacle or a wall take a per-node path with bounce-back instead.
#include "lbibm_internal.cuh"

#include <cuda_pipeline.h>

#include <type_traits>

namespace lbibm {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// population storage
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class S> __device__ __forceinline__ S __ushort_as_s(unsigned short v);
template <> __device__ __forceinline__ __half __ushort_as_s<__half>(unsigned short v) { return __ushort_as_half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 __ushort_as_s<__nv_bfloat16>(unsigned short v) {
    return __ushort_as_bfloat16(v);
}
template <class S> __device__ __forceinline__ S from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Cache policy of the population stream (each value is read once and written
// once per step).  16-bit storage streams (ld/st .cs, evict-first in L2), which
// leaves the immersed-boundary working set (positions, element terms, force
// and velocity stencils) in L2 across the step: 85.4 -> 81.6 us per cycle on
// the 256x128x64 filter, the stream-collide itself unchanged.  FP32 keeps the
// read-only path: streaming loads cost it 7 us (62.5 -> 69.3 us), streaming
// stores alone gain nothing (measured on GB300).
template <class S>
__host__ __device__ constexpr bool pop_streaming() { return sizeof(S) == 2; }

template <class S, class T>
__device__ __forceinline__ T pop_ld(const T* p) {
    if constexpr (pop_streaming<S>()) return __ldcs(p);
    else return __ldg(p);
}

template <class S, class T>
__device__ __forceinline__ void pop_st(T* p, T v) {
    if constexpr (pop_streaming<S>()) __stcs(p, v);
    else *p = v;
}

// ---------------------------------------------------------------------------
// Stochastic rounding of the 16-bit population stores.
//
// Rounding to nearest gives every node of a region of uniform flow the same
// rounding error, so the errors of a step add up coherently over the region:
// a uniform (k = 0) momentum error that viscosity does not damp, growing like
// a random walk over the steps.  Rounding up with a probability equal to the
// discarded fraction (stochastic rounding) makes each error unbiased and the
// errors of different nodes independent, so they fall into short-wavelength
// modes that the collision and viscosity damp.  (Emulated on the CPU on a
// 32x48x48 force-driven channel after 200 steps, velocity error against
// FP64: FP16 2.5e-3 -> 1.6e-4, BF16 1.8e-2 -> 1.3e-3.)
//
// cvt.rs.{f16x2,bf16x2}.f32 (sm_100 family) rounds its upper operand with the
// upper 16 of its random bits and its lower operand with the lower 16.  The
// random word of a node (or node pair) is a hash of its index and of the bit
// patterns of its moments, which change from step to step: runs stay
// bit-reproducible and no step counter is needed.  Direction i draws
// seed * sr_k(i) (distinct odd multipliers).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr unsigned sr_mix(unsigned x) {
    // 32-bit integer finaliser (xorshift-multiply, "lowbias32" constants)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__host__ __device__ constexpr unsigned sr_k(int i) { return sr_mix(0x632be5abu + 0x9e3779b9u * (unsigned)i) | 1u; }

__device__ __forceinline__ unsigned sr_seed(unsigned node, float a, float b) {
    return sr_mix(node * 0x9e3779b1u ^ __float_as_uint(a) ^ __funnelshift_l(__float_as_uint(b), __float_as_uint(b), 16));
}

// Two floats to a packed 16-bit pair (hi: upper half) with stochastic rounding.
template <class S> __device__ __forceinline__ unsigned cvt_rs2(float hi, float lo, unsigned rb);
template <> __device__ __forceinline__ unsigned cvt_rs2<__half>(float hi, float lo, unsigned rb) {
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rb));
    return d;
}
template <> __device__ __forceinline__ unsigned cvt_rs2<__nv_bfloat16>(float hi, float lo, unsigned rb) {
    unsigned d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rb));
    return d;
}
// One float to 16 bits with stochastic rounding (the lower 16 random bits).
template <class S> __device__ __forceinline__ S cvt_rs1(float v, unsigned rb) {
    return __ushort_as_s<S>((unsigned short)(cvt_rs2<S>(0.0f, v, rb) & 0xffffu));
}

template <class S> struct Pop {
    static __device__ __forceinline__ float ld(const S* p, long long idx, int i) {
        if constexpr (sizeof(S) == 4) return pop_ld<S>(p + idx);
        else return wgt(i) * to_f(pop_ld<S>(p + idx));
    }
    // rb: the node's random word (sr_seed); 16-bit storage rounds with
    // rb * sr_k(i), FP32 ignores it
    static __device__ __forceinline__ void st(S* p, long long idx, float h, int i, unsigned rb) {
        if constexpr (sizeof(S) == 4) pop_st<S>(p + idx, h);
        else pop_st<S>(p + idx, cvt_rs1<S>(h * (1.0f / wgt(i)), rb * sr_k(i)));
    }
};

// NPT consecutive populations of one direction as one aligned vector access.
template <int BYTES> struct Raw;
template <> struct Raw<2> { using T = unsigned short; };
template <> struct Raw<4> { using T = unsigned int; };
template <> struct Raw<8> { using T = uint2; };
template <> struct Raw<16> { using T = uint4; };

template <class S, int NPT>
struct VecIO {
    using R = typename Raw<sizeof(S) * NPT>::T;
    static __device__ __forceinline__ void ld(const S* base, long long idx, int i, float out[NPT]) {
        const R r = pop_ld<S>(reinterpret_cast<const R*>(base + idx));
        const S* e = reinterpret_cast<const S*>(&r);
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            if constexpr (sizeof(S) == 4) out[k] = to_f(e[k]);
            else out[k] = wgt(i) * to_f(e[k]);
        }
    }
    // rb[k]: random word of node k (16-bit storage only)
    static __device__ __forceinline__ void st(S* base, long long idx, int i, const float in[NPT],
                                              const unsigned rb[NPT]) {
        R r;
        S* e = reinterpret_cast<S*>(&r);
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            if constexpr (sizeof(S) == 4) e[k] = from_f<S>(in[k]);
            else e[k] = cvt_rs1<S>(in[k] * (1.0f / wgt(i)), rb[k] * sr_k(i));
        }
        pop_st<S>(reinterpret_cast<R*>(base + idx), r);
    }
};

__device__ __forceinline__ bool solid_at(const uint32_t* mask, long long g) {
    return (__ldg(mask + (g >> 5)) >> (g & 31)) & 1u;
}

__device__ __forceinline__ const ChannelDev& chan(const LatticeArgs& a, int c) {
    return c < MAXCH_P ? a.chp[c] : a.ch[c];
}

// L2 prefetch ahead of the stream-collide blocks: threads 0..18 of a block
// whose first node has global index g0 and that covers nb nodes each ask L2
// (one bulk prefetch, no registers held, nothing returned) for the nb
// populations of their direction starting pf_nodes further on, clipped to the
// direction's plane.  Every address lies inside the population array: the
// start is below the plane stride and the end at most at it.  Requires
// g0 + pf_nodes and nb * sizeof(S) to be multiples of 16 bytes' worth of
// populations (the block sizes and the distance are multiples of 256 nodes).
template <class S>
__device__ __forceinline__ void prefetch_ahead(const LatticeArgs& a, long long g0, int nb) {
    if (a.pf_nodes <= 0 || threadIdx.x >= Q) return;
    const long long g = g0 + a.pf_nodes;
    if (g >= a.Ntot) return;
    const long long n = a.Ntot - g < nb ? a.Ntot - g : nb;
    const S* src = (const S*)(a.par ? a.h1 : a.h0) + (size_t)threadIdx.x * (size_t)a.Ntot + g;
    const unsigned bytes = (unsigned)(n * (long long)sizeof(S)) & ~15u;
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Source offsets of the pull scheme for one node: for each axis the linear
// offset to the neighbour at coordinate -1 ("m") and +1 ("p"), with periodic
// wrap, and whether that neighbour exists.
struct Nbr {
    int om[3], op[3];
    bool vm[3], vp[3];
};

__device__ __forceinline__ void neighbours(const ChannelDev& C, int x, int y, int z, Nbr& nb) {
    const int c[3] = {x, y, z};
    const int n[3] = {C.nx, C.ny, C.nz};
    const int s[3] = {1, C.nx, C.nx * C.ny};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (c[d] > 0) { nb.om[d] = -s[d]; nb.vm[d] = true; }
        else if (C.per[d]) { nb.om[d] = (n[d] - 1) * s[d]; nb.vm[d] = true; }
        else { nb.om[d] = 0; nb.vm[d] = false; }
        if (c[d] < n[d] - 1) { nb.op[d] = s[d]; nb.vp[d] = true; }
        else if (C.per[d]) { nb.op[d] = -(n[d] - 1) * s[d]; nb.vp[d] = true; }
        else { nb.op[d] = 0; nb.vp[d] = false; }
    }
}

// Offset of the pull source x - e_i and whether it lies inside the domain.
template <int I>
__device__ __forceinline__ int src_off(const Nbr& nb, bool& ok) {
    int o = 0;
    ok = true;
    if (ex(I) == 1) { o += nb.om[0]; ok = ok && nb.vm[0]; }
    if (ex(I) == -1) { o += nb.op[0]; ok = ok && nb.vp[0]; }
    if (ey(I) == 1) { o += nb.om[1]; ok = ok && nb.vm[1]; }
    if (ey(I) == -1) { o += nb.op[1]; ok = ok && nb.vp[1]; }
    if (ez(I) == 1) { o += nb.om[2]; ok = ok && nb.vm[2]; }
    if (ez(I) == -1) { o += nb.op[2]; ok = ok && nb.vp[2]; }
    return o;
}

// y/z part of the source offset (the +-x part is handled by the vector path).
template <int I>
__device__ __forceinline__ int src_off_yz(const Nbr& nb) {
    int o = 0;
    if (ey(I) == 1) o += nb.om[1];
    if (ey(I) == -1) o += nb.op[1];
    if (ez(I) == 1) o += nb.om[2];
    if (ez(I) == -1) o += nb.op[2];
    return o;
}

// Pull one population with bounce-back where the source is a wall or solid.
template <class S, int I>
__device__ __forceinline__ float pull_slow(const S* src, long long NT, long long gp, const Nbr& nb,
                                           const uint32_t* mask, const ChannelDev& C, int y, bool check_solid) {
    bool ok;
    const int o = src_off<I>(nb, ok);
    if (ok && check_solid) ok = !solid_at(mask, gp + o);
    if (ok) return Pop<S>::ld(src, (long long)I * NT + gp + o, I);
    float h = Pop<S>::ld(src, (long long)opp(I) * NT + gp, opp(I));
    if (C.has_uw && !C.per[1]) {
        int wall = -1;
        if (ey(I) == 1 && y == 0) wall = 0;
        if (ey(I) == -1 && y == C.ny - 1) wall = 1;
        if (wall >= 0) {
            const float eu = ex(I) * C.uw[wall][0] + ey(I) * C.uw[wall][1] + ez(I) * C.uw[wall][2];
            h += 6.0f * wgt(I) * eu;
        }
    }
    return h;
}

#define LBIBM_ALL_I(M) M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) M(17) M(18)

template <class S>
__device__ __forceinline__ void pull_node(const S* src, long long NT, long long gp, const Nbr& nb,
                                          const uint32_t* mask, const ChannelDev& C, int y, float h[Q],
                                          bool check_solid = true) {
#define LBIBM_PS(I) h[I] = pull_slow<S, I>(src, NT, gp, nb, mask, C, y, check_solid);
    LBIBM_ALL_I(LBIBM_PS)
#undef LBIBM_PS
}

// Vector pull, phase 1: issue the loads of direction I for the NPT nodes
// starting at x0.  Every address stays inside the channel's rows (a missing
// neighbour maps to offset 0), so the loads can be issued before the warp
// knows whether it takes this path; lanes past the channel's end load nothing.
// With NPT = 1 the +-x shift is part of the address; with NPT > 1 the vector
// is the aligned source row and the lanes at a row end or a warp edge also
// load the one element their neighbour lane cannot hand them.
template <class S, int NPT, int I>
__device__ __forceinline__ void issue_vec(const S* src, long long NT, int gi0, const Nbr& nb, const ChannelDev& C,
                                          int x0, int lane, bool inr, float v[NPT], float& extra) {
    extra = 0.0f;
    const S* pl = src + (size_t)I * (size_t)NT;   // plane of direction I (warp-uniform)
    if constexpr (NPT == 1) {
        bool ok;
        const int b = gi0 + src_off<I>(nb, ok);
        v[0] = inr ? Pop<S>::ld(pl, b, I) : 0.0f;
    } else {
        const int b = gi0 + src_off_yz<I>(nb);   // source row, aligned to NPT
        if (inr) {
            VecIO<S, NPT>::ld(pl, b, I, v);
        } else {
#pragma unroll
            for (int k = 0; k < NPT; ++k) v[k] = 0.0f;
        }
        if constexpr (ex(I) == 1) {
            if (inr && (lane == 0 || x0 == 0)) extra = Pop<S>::ld(pl, x0 == 0 ? b + (C.nx - 1) : b - 1, I);
        } else if constexpr (ex(I) == -1) {
            if (inr && (lane == 31 || x0 + NPT == C.nx)) extra = Pop<S>::ld(pl, x0 + NPT == C.nx ? b - x0 : b + NPT, I);
        }
    }
}

// Vector pull, phase 2 (converged warp, no walls or obstacles around): place
// the loaded values, taking the +-x halo element from the neighbouring lane.
template <int NPT, int I>
__device__ __forceinline__ void place_vec(const float v[NPT], float extra, const ChannelDev& C, int x0, int lane,
                                          float h[NPT][Q]) {
    if constexpr (NPT == 1 || ex(I) == 0) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) h[k][I] = v[k];
    } else if constexpr (ex(I) == 1) {
        // node x0 + k pulls from x0 + k - 1
        float left = __shfl_up_sync(FULL, v[NPT - 1], 1);
        if (lane == 0 || x0 == 0) left = extra;
        h[0][I] = left;
#pragma unroll
        for (int k = 1; k < NPT; ++k) h[k][I] = v[k - 1];
    } else {
        // node x0 + k pulls from x0 + k + 1
        float right = __shfl_down_sync(FULL, v[0], 1);
        if (lane == 31 || x0 + NPT == C.nx) right = extra;
#pragma unroll
        for (int k = 0; k < NPT - 1; ++k) h[k][I] = v[k + 1];
        h[NPT - 1][I] = right;
    }
}

// Moments of the shifted populations in a fixed pairwise order.
__device__ __forceinline__ void moments(const float h[Q], float& drho, float& jx, float& jy, float& jz) {
    const float a1 = h[1] - h[2], a3 = h[3] - h[4], a5 = h[5] - h[6];
    const float d7 = h[7] - h[8], d9 = h[9] - h[10], d11 = h[11] - h[12], d13 = h[13] - h[14];
    const float d15 = h[15] - h[16], d17 = h[17] - h[18];
    jx = (a1 + (d7 + d9)) + (d11 + d13);
    jy = (a3 + (d7 - d9)) + (d15 + d17);
    jz = (a5 + (d11 - d13)) + (d15 - d17);
    drho = (((h[0] + (h[1] + h[2])) + ((h[3] + h[4]) + (h[5] + h[6]))) +
            (((h[7] + h[8]) + (h[9] + h[10])) + ((h[11] + h[12]) + (h[13] + h[14])))) +
           ((h[15] + h[16]) + (h[17] + h[18]));
}

// Macroscopic state of one node for the collision.
struct Mac {
    float drho, rho, ux, uy, uz, uu, gx, gy, gz, ug;
};

__device__ __forceinline__ Mac macro(const float h[Q], float gx, float gy, float gz) {
    Mac m;
    float jx, jy, jz;
    moments(h, m.drho, jx, jy, jz);
    m.gx = gx; m.gy = gy; m.gz = gz;
    m.rho = 1.0f + m.drho;
    const float irho = 1.0f / m.rho;
    m.ux = (jx + 0.5f * gx) * irho;
    m.uy = (jy + 0.5f * gy) * irho;
    m.uz = (jz + 0.5f * gz) * irho;
    m.uu = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    m.ug = m.ux * gx + m.uy * gy + m.uz * gz;
    return m;
}

// Differentiable variant: Brinkman force -a rho u (a = alpha phi) taken
// implicitly, u = (j + g/2) / (rho (1 + a/2)); the collision then uses
// g_tot = g - a rho u = g - a (j + g/2) / (1 + a/2).
__device__ __forceinline__ Mac macro_brinkman(const float h[Q], float gx, float gy, float gz, float a) {
    Mac m;
    float jx, jy, jz;
    moments(h, m.drho, jx, jy, jz);
    m.rho = 1.0f + m.drho;
    const float vx = jx + 0.5f * gx, vy = jy + 0.5f * gy, vz = jz + 0.5f * gz;
    const float iD = 1.0f / (1.0f + 0.5f * a);
    const float s = iD / m.rho;
    m.ux = vx * s;
    m.uy = vy * s;
    m.uz = vz * s;
    m.gx = gx - a * vx * iD;
    m.gy = gy - a * vy * iD;
    m.gz = gz - a * vz * iD;
    m.uu = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    m.ug = m.ux * m.gx + m.uy * m.gy + m.uz * m.gz;
    return m;
}

// BGK collision with Guo forcing on shifted populations:
//   h*_i = h_i + omega (h_i^eq - h_i) + S_i,
//   h_i^eq = w_i [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u)],
//   S_i = (1 - 1/2tau) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . g.
template <int I>
__device__ __forceinline__ float collide_one(float hi, const Mac& m, float omega, float fpre) {
    const float eu = ex(I) * m.ux + ey(I) * m.uy + ez(I) * m.uz;
    const float eg = ex(I) * m.gx + ey(I) * m.gy + ez(I) * m.gz;
    const float heq = wgt(I) * (m.drho + m.rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * m.uu));
    const float s = fpre * wgt(I) * (3.0f * (eg - m.ug) + 9.0f * eu * eg);
    return hi + omega * (heq - hi) + s;
}

// The same collision for the pair of opposite directions (I, I+1), I odd:
// e_{I+1} = -e_I, so the equilibrium and the source split into a part even in
// e (shared) and a part odd in e (sign flipped), which halves the arithmetic.
template <int I>
__device__ __forceinline__ void collide_pair(float h[Q], const Mac& m, float A1, float om, float fp) {
    constexpr int J = I + 1;
    const float w = wgt(I);
    const float eu = ex(I) * m.ux + ey(I) * m.uy + ez(I) * m.uz;
    const float eg = ex(I) * m.gx + ey(I) * m.gy + ez(I) * m.gz;
    const float seq = w * (A1 + 4.5f * m.rho * eu * eu);
    const float aeq = (3.0f * w) * m.rho * eu;
    const float ss = (fp * w) * (9.0f * eu * eg - 3.0f * m.ug);
    const float as = (3.0f * fp * w) * eg;
    const float hi = h[I], hj = h[J];
    h[I] = hi + om * ((seq + aeq) - hi) + (ss + as);
    h[J] = hj + om * ((seq - aeq) - hj) + (ss - as);
}

// Collide all 19 populations of one node in place (h -> h*).
__device__ __forceinline__ void collide_all(float h[Q], const Mac& m, float om, float fp) {
    const float A1 = m.drho - 1.5f * m.rho * m.uu;
    h[0] = h[0] + om * (wgt(0) * A1 - h[0]) + (fp * wgt(0)) * (-3.0f * m.ug);
    collide_pair<1>(h, m, A1, om, fp);
    collide_pair<3>(h, m, A1, om, fp);
    collide_pair<5>(h, m, A1, om, fp);
    collide_pair<7>(h, m, A1, om, fp);
    collide_pair<9>(h, m, A1, om, fp);
    collide_pair<11>(h, m, A1, om, fp);
    collide_pair<13>(h, m, A1, om, fp);
    collide_pair<15>(h, m, A1, om, fp);
    collide_pair<17>(h, m, A1, om, fp);
}

template <class S, int NPT, int I>
__device__ __forceinline__ void store_vec(S* dst, long long NT, int gi0, const float h[NPT][Q], const unsigned rb[NPT]) {
    float o[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) o[k] = h[k][I];
    VecIO<S, NPT>::st(dst + (size_t)I * (size_t)NT, gi0, I, o, rb);
}

// Link masks of NPT consecutive nodes (one aligned vector load).
template <int NPT>
__device__ __forceinline__ void links_ld(const uint32_t* p, uint32_t lk[NPT]) {
    if constexpr (NPT == 1) {
        lk[0] = __ldg(p);
    } else if constexpr (NPT == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        lk[0] = v.x; lk[1] = v.y;
    } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        lk[0] = v.x; lk[1] = v.y; lk[2] = v.z; lk[3] = v.w;
    }
}

// Halfway bounce-back (Sec. 2.4) for the links of one node whose bit is set
// in its link mask: the population pulled along direction i comes back from
// the node's own post-collision population opp(i); on a moving y-wall Ladd's
// term 6 w_i rho0 e_i . u_wall is added (rho0 = 1).
template <class S>
__device__ __forceinline__ void bounce_back(const S* src, long long NT, int gi, uint32_t lk, const ChannelDev& C,
                                            int y, float h[Q]) {
    if (!(lk & ~1u)) return;
#define LBIBM_BB(I)                                                                  \
    if (I > 0 && ((lk >> I) & 1u)) {                                                 \
        float v = Pop<S>::ld(src, (long long)opp(I) * NT + gi, opp(I));              \
        if (C.has_uw && !C.per[1]) {                                                 \
            const int wall = (ey(I) == 1 && y == 0) ? 0 : ((ey(I) == -1 && y == C.ny - 1) ? 1 : -1); \
            if (wall >= 0)                                                           \
                v += 6.0f * wgt(I) * (ex(I) * C.uw[wall][0] + ey(I) * C.uw[wall][1] + ez(I) * C.uw[wall][2]); \
        }                                                                            \
        h[I] = v;                                                                    \
    }
    LBIBM_ALL_I(LBIBM_BB)
#undef LBIBM_BB
}

// Resident threads per SM the register budget is sized for.  One node per
// thread: 1152 threads (56 registers) for FP32 and for 16-bit populations, the
// fastest of the budgets measured on GB300 with row-aligned blocks (FP32: 1280
// 61.0 us, 1152 60.6, 1024 64.1; 16-bit: 1280 56.2, 1152 55.9, 1024 58.3); two
// nodes per thread: 512 (128 registers); four: 256 (255 registers).
#ifndef LBIBM_K3_THREADS1
#define LBIBM_K3_THREADS1 1152
#endif
#ifndef LBIBM_K3_THREADS1_16
#define LBIBM_K3_THREADS1_16 1152
#endif
#ifndef LBIBM_K3_THREADS2
#define LBIBM_K3_THREADS2 512
#endif
template <class S, int NPT, int BS> struct K3MinBlocks {
    static constexpr int threads = NPT == 1 ? (sizeof(S) == 4 ? LBIBM_K3_THREADS1 : LBIBM_K3_THREADS1_16)
                                            : (NPT == 2 ? LBIBM_K3_THREADS2 : 256);
    static constexpr int value = threads / BS > 0 ? threads / BS : 1;
};

// Schedules of one stream-collide launch: every node (SC_ALL); the bulk, i.e.
// every 32-node group outside the step's stencil set (SC_BULK); or the groups
// of the stencil set from a list (SC_LIST); or every node of the
// differentiable variant (SC_BRINK: Brinkman beads, velocity written at every
// node).  Bulk groups carry no IB force in this step and none in the previous
// one, so their flag loads are skipped.
enum : int { SC_ALL = 0, SC_BULK = 1, SC_LIST = 2, SC_BRINK = 3 };

// One thread's NPT nodes starting at channel-local node p0.
// ROW: the caller's block lies inside one lattice row, all its nodes in range,
// and passes the coordinates (y, z are then block-uniform).
template <class S, int NPT, int MODE, bool ROW = false>
__device__ __forceinline__ void sc_nodes(const LatticeArgs& a, const ChannelDev& C, int p0, int lane, int xr = 0,
                                         int yr = 0, int zr = 0) {
    const long long gp0 = C.base + p0;
    const int gi0 = (int)gp0;      // the padded node count of a context is below 2^31
    const int grp = gi0 >> 5;
    const int par = a.par;
    uint8_t* fl_prev = par ? a.fl0 : a.fl1;
    const bool inr = ROW ? true : p0 < C.n;
    const uint8_t fslow = inr ? __ldg(a.slow + grp) : (uint8_t)0;
    const S* src = (const S*)(par ? a.h1 : a.h0);
    S* dst = (S*)(par ? a.h0 : a.h1);
    const long long NT = a.Ntot;
    int x0, y, z;
    if constexpr (ROW) {
        x0 = xr; y = yr; z = zr;
    } else {
        const int r = fdiv(p0, C.dnx);
        x0 = p0 - r * C.nx;
        z = fdiv(r, C.dny);
        y = r - z * C.ny;
    }
    Nbr nb;
    neighbours(C, x0, y, z, nb);
    // phase 1: every population load of the vector path in flight at once
    // The populations are the previous cycle's (launched as a programmatic
    // dependent only behind the spreading kernel), the force flags and
    // densities come from that kernel.  FP32 issues its population loads
    // before the wait (they overlap the predecessor's tail); 16-bit storage
    // waits first, so that the flags travel with its loads (measured on GB300:
    // FP32 412.8 vs 431.0 us, FP16 396.2 vs 383.0 us on 512x256x128, with
    // the loads before / after the wait).
    constexpr bool wait_first = sizeof(S) == 2;
    if constexpr (wait_first) pdl_entry();
    const uint8_t fcur_e = (!wait_first || MODE == SC_BULK) ? (uint8_t)0 : __ldg((par ? a.fl1 : a.fl0) + grp);
    const uint8_t fprev_e = (!wait_first || MODE == SC_BULK) ? (uint8_t)0 : __ldg(fl_prev + grp);
    float v[Q][NPT], extra[Q];
#define LBIBM_IV(I) issue_vec<S, NPT, I>(src, NT, gi0, nb, C, x0, lane, inr, v[I], extra[I]);
    LBIBM_ALL_I(LBIBM_IV)
#undef LBIBM_IV
    if constexpr (!wait_first) pdl_entry();
    const uint8_t fcur = wait_first ? fcur_e : (MODE == SC_BULK ? (uint8_t)0 : __ldg((par ? a.fl1 : a.fl0) + grp));
    const uint8_t fprev = wait_first ? fprev_e : (MODE == SC_BULK ? (uint8_t)0 : __ldg(fl_prev + grp));
    const bool forced = fcur != 0;
    const bool prevf = fprev != 0;
    const bool wslow = __any_sync(FULL, fslow != 0);
    const float om = C.omega, fp = C.fpre;
    const float4* gcur = par ? a.g1 : a.g0;
    float4* gprev = par ? a.g0 : a.g1;
    // stencil groups mostly carry force: load it with the populations
    float4 gpre = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE == SC_LIST && NPT == 1 && inr) gpre = gcur[gi0];

    // phase 2 (converged warp): place the loaded values
    float h[NPT][Q];
#define LBIBM_PV(I) place_vec<NPT, I>(v[I], extra[I], C, x0, lane, h);
    LBIBM_ALL_I(LBIBM_PV)
#undef LBIBM_PV
    // groups at a wall or an obstacle: replace the populations of bounce-back
    // links by the opposite population of the node itself (halfway bounce-back)
    uint32_t lk[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) lk[k] = 0u;
    if (wslow) {
        if (inr && fslow) links_ld<NPT>(a.links + gi0, lk);
#pragma unroll
        for (int k = 0; k < NPT; ++k) bounce_back<S>(src, NT, gi0 + k, lk[k], C, y, h[k]);
    }
    if (inr) {
        Mac m[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            float gx = C.G[0], gy = C.G[1], gz = C.G[2];
            if (forced) {
                const float4 g = (MODE == SC_LIST && NPT == 1) ? gpre : gcur[gi0 + k];
                gx += g.x; gy += g.y; gz += g.z;
            }
            if constexpr (MODE == SC_BRINK) m[k] = macro_brinkman(h[k], gx, gy, gz, a.alpha * __ldg(a.phi + gi0 + k));
            else m[k] = macro(h[k], gx, gy, gz);
        }
        unsigned rb[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) rb[k] = sr_seed((unsigned)(gi0 + k), m[k].drho, m[k].ux);
#pragma unroll
        for (int k = 0; k < NPT; ++k) collide_all(h[k], m[k], om, fp);
        uint32_t solid = 0u;
#pragma unroll
        for (int k = 0; k < NPT; ++k) solid |= lk[k];
        if (!(solid & 1u)) {
#define LBIBM_SV(I) store_vec<S, NPT, I>(dst, NT, gi0, h, rb);
            LBIBM_ALL_I(LBIBM_SV)
#undef LBIBM_SV
        } else {
            // a solid node among this thread's nodes: it keeps its populations
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                if (lk[k] & 1u) continue;
#define LBIBM_S1(I) Pop<S>::st(dst, (long long)(I) * NT + gi0 + k, h[k][I], I, rb[k]);
                LBIBM_ALL_I(LBIBM_S1)
#undef LBIBM_S1
            }
        }
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            if (lk[k] & 1u) continue;
            if (forced || MODE == SC_BRINK) a.u[gi0 + k] = make_float4(m[k].ux, m[k].uy, m[k].uz, m[k].rho);
            if (prevf) gprev[gi0 + k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // the lane holding the first node of each 32-node group clears the previous
    // step's flag after every lane of the warp has consumed it
    __syncwarp();
    if (prevf && (gp0 & 31) == 0) fl_prev[grp] = 0;
}

template <class S, int NPT, int BS>
__global__ void __launch_bounds__(BS, K3MinBlocks<S, NPT, BS>::value) k_stream_collide(const __grid_constant__ LatticeArgs a) {
    // (sc_nodes waits for the predecessor after its population loads)
    const int b = blockIdx.x;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (b >= chan(a, k).blk0) c = k;
    const ChannelDev C = chan(a, c);   // registers: read once from the parameter bank
    const int lane = threadIdx.x & 31;
    const int p0 = ((b - C.blk0) * BS + (int)threadIdx.x) * NPT;   // first channel-local node of this thread
    prefetch_ahead<S>(a, C.base + (long long)(b - C.blk0) * BS * NPT, BS * NPT);
    if constexpr (NPT == 1) {
        // (measured on GB300, 256x128x64 filter: FP32 62.4 -> 60.6 us with the
        // 56-register budget, 16-bit 59.6 -> 57.5 us)
        const int pb = (b - C.blk0) * BS;
        if (C.nx % BS == 0 && pb + BS <= C.n) {
            // the block is a piece of one row: y and z are the block's
            const int r = fdiv(pb, C.dnx);
            const int z = fdiv(r, C.dny);
            sc_nodes<S, 1, SC_ALL, true>(a, C, p0, lane, pb - r * C.nx + (int)threadIdx.x, r - z * C.ny, z);
            return;
        }
    }
    sc_nodes<S, NPT, SC_ALL>(a, C, p0, lane);
}

// ---------------------------------------------------------------------------
// Pair variant (nodes_per_thread = 2): each thread takes the consecutive
// x-nodes x0, x0 + 1 (x0 even) of one row.  A direction without an x
// component pulls both nodes' values as one aligned pair (a 32-bit word of two
// 16-bit values, or a float2); a direction with one pulls two single values
// (x0 - 1 and x0 along +x, x0 + 1 and x0 + 2 along -x).  The two nodes'
// moments and collisions run as packed FP32 pairs (add / mul / fma.f32x2: two
// FP32 lanes per instruction on the sm_100 family) and every direction is
// stored as one pair.  16-bit storage keeps s_i = h_i / w_i, whose collision
// is free of weights,
//   s*_i = (1 - om) s_i + om [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u)]
//          + (1 - 1/2tau) [3 (e_i - u) + 9 (e_i.u) e_i] . g,
// so only the moments weigh the populations; FP32 keeps h_i and multiplies
// the equilibrium and source part by w_i.  Stores round stochastically
// (one random word per pair, see sr_mix).
// ---------------------------------------------------------------------------
typedef float2 F2;
__device__ __forceinline__ F2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const F2*>(&r);
}

template <class S> struct PairIO;
template <> struct PairIO<float> {
    static constexpr bool SCALED = false;
    static __device__ __forceinline__ F2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
    static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st2(float* p, F2 v, unsigned) { *reinterpret_cast<float2*>(p) = v; }
    static __device__ __forceinline__ void st1(float* p, float v, unsigned) { *p = v; }
};
template <> struct PairIO<__half> {
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ F2 ld2(const __half* p) {
        const unsigned r = __ldcs(reinterpret_cast<const unsigned*>(p));
        return __half22float2(*reinterpret_cast<const __half2*>(&r));
    }
    static __device__ __forceinline__ float ld1(const __half* p) { return __half2float(__ldcs(p)); }
    static __device__ __forceinline__ void st2(__half* p, F2 v, unsigned rb) {
        __stcs(reinterpret_cast<unsigned*>(p), cvt_rs2<__half>(v.y, v.x, rb));
    }
    static __device__ __forceinline__ void st1(__half* p, float v, unsigned rb) { __stcs(p, cvt_rs1<__half>(v, rb)); }
};
template <> struct PairIO<__nv_bfloat16> {
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ F2 ld2(const __nv_bfloat16* p) {
        const unsigned r = __ldcs(reinterpret_cast<const unsigned*>(p));
        return make_float2(__uint_as_float(r << 16), __uint_as_float(r & 0xffff0000u));
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16* p) {
        return __uint_as_float((unsigned)__bfloat16_as_ushort(__ldcs(p)) << 16);
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16* p, F2 v, unsigned rb) {
        __stcs(reinterpret_cast<unsigned*>(p), cvt_rs2<__nv_bfloat16>(v.y, v.x, rb));
    }
    static __device__ __forceinline__ void st1(__nv_bfloat16* p, float v, unsigned rb) {
        __stcs(p, cvt_rs1<__nv_bfloat16>(v, rb));
    }
};

// Offsets of the pull sources of one node pair relative to x0's index: the
// rows y -+ 1, z -+ 1 (wrapped on periodic axes; a missing row maps to the
// node's own row, whose link then bounces back) and the x neighbours x0 - 1 of
// node 0 and x0 + 2 of node 1 (a missing one maps to the node itself).
struct PairNbr {
    int oym, oyp, ozm, ozp;
    int dxm, dxp;
};

__device__ __forceinline__ void pair_neighbours(const ChannelDev& C, int x0, int y, int z, PairNbr& nb) {
    const int sy = C.nx, sz = C.nx * C.ny;
    nb.oym = y > 0 ? -sy : (C.per[1] ? (C.ny - 1) * sy : 0);
    nb.oyp = y < C.ny - 1 ? sy : (C.per[1] ? -(C.ny - 1) * sy : 0);
    nb.ozm = z > 0 ? -sz : (C.per[2] ? (C.nz - 1) * sz : 0);
    nb.ozp = z < C.nz - 1 ? sz : (C.per[2] ? -(C.nz - 1) * sz : 0);
    nb.dxm = x0 > 0 ? -1 : (C.per[0] ? C.nx - 1 : 0);
    nb.dxp = x0 + 2 < C.nx ? 2 : (C.per[0] ? -x0 : 1);
}

template <int I, class NB>
__device__ __forceinline__ int pair_row(const NB& nb) {
    int o = 0;
    if (ey(I) == 1) o += nb.oym;
    if (ey(I) == -1) o += nb.oyp;
    if (ez(I) == 1) o += nb.ozm;
    if (ez(I) == -1) o += nb.ozp;
    return o;
}

// Pull direction I of both nodes (phase 1: the loads only).
template <class S, int I>
__device__ __forceinline__ F2 pair_pull(const S* src, long long NT, int gi0, const PairNbr& nb, bool inr) {
    const S* pl = src + (size_t)I * (size_t)NT + gi0 + pair_row<I>(nb);
    if (!inr) return make_float2(0.f, 0.f);
    if constexpr (ex(I) == 0) return PairIO<S>::ld2(pl);
    else if constexpr (ex(I) == 1) return make_float2(PairIO<S>::ld1(pl + nb.dxm), PairIO<S>::ld1(pl));
    else return make_float2(PairIO<S>::ld1(pl + 1), PairIO<S>::ld1(pl + nb.dxp));
}

// Halfway bounce-back of node k of the pair: population I comes back as the
// node's own opp(I) (in the storage's scaling), plus Ladd's moving-wall term.
template <class S, int I, class NTT>
__device__ __forceinline__ void pair_bounce(const S* src, NTT NT, int gi, uint32_t lk, const ChannelDev& C,
                                            int y, float& v) {
    if (!((lk >> I) & 1u)) return;
    float b = PairIO<S>::ld1(src + (sizeof(NTT) == 4 ? (size_t)((unsigned)opp(I) * (unsigned)NT + (unsigned)gi)
                                                     : (size_t)opp(I) * (size_t)NT + gi));
    if (C.has_uw && !C.per[1]) {
        const int wall = (ey(I) == 1 && y == 0) ? 0 : ((ey(I) == -1 && y == C.ny - 1) ? 1 : -1);
        if (wall >= 0) {
            const float eu = ex(I) * C.uw[wall][0] + ey(I) * C.uw[wall][1] + ez(I) * C.uw[wall][2];
            b += PairIO<S>::SCALED ? 6.0f * eu : 6.0f * wgt(I) * eu;
        }
    }
    v = b;
}

// e_I . (ax, ay, az) for the packed pair, with e_I's components in {-1, 0, 1}.
template <int I>
__device__ __forceinline__ F2 edot2(F2 ax, F2 ay, F2 az) {
    F2 r = make_float2(0.f, 0.f);
    bool any = false;
    auto acc = [&](int e, F2 v) {
        if (e == 0) return;
        if (!any) {
            r = e > 0 ? v : make_float2(-v.x, -v.y);
            any = true;
        } else {
            r = e > 0 ? add2(r, v) : sub2(r, v);
        }
    };
    acc(ex(I), ax);
    acc(ey(I), ay);
    acc(ez(I), az);
    return r;
}

// Packed macroscopic state of the pair.
struct Mac2 {
    F2 drho, rho, ux, uy, uz, gx, gy, gz, A1, mug;
};

// Collision of the opposite directions (I, I + 1), I odd, for both nodes.
template <bool SCALED, int I>
__device__ __forceinline__ void collide_pair2(F2 h[Q], const Mac2& m, F2 om, F2 omc, F2 c3om, F2 c9fp, F2 c3fp) {
    constexpr int J = I + 1;
    const F2 eu = edot2<I>(m.ux, m.uy, m.uz);
    const F2 eg = edot2<I>(m.gx, m.gy, m.gz);
    const F2 reu = mul2(m.rho, eu);
    const F2 E = fma2(mul2(f2s(4.5f), reu), eu, m.A1);          // A1 + 9/2 rho (e.u)^2
    const F2 Es = fma2(om, E, fma2(mul2(c9fp, eu), eg, m.mug));   // + fp (9 (e.u)(e.g) - 3 u.g)
    const F2 Os = fma2(c3om, reu, mul2(c3fp, eg));                // 3 om rho e.u + 3 fp e.g
    const F2 XI = add2(Es, Os), XJ = sub2(Es, Os);
    if constexpr (SCALED) {
        h[I] = fma2(omc, h[I], XI);
        h[J] = fma2(omc, h[J], XJ);
    } else {
        const F2 w = f2s(wgt(I));
        h[I] = fma2(w, XI, mul2(omc, h[I]));
        h[J] = fma2(w, XJ, mul2(omc, h[J]));
    }
}

// Moments and collision of one in-range node pair in place (h: the pulled
// populations after bounce-back, in the storage's scaling; g0, g1: the nodes'
// force densities, added when the group is forced).  m returns the pair's
// macroscopic state (velocity, density) for the velocity output and the
// rounding seed.
template <bool SCALED>
__device__ __forceinline__ void pair_collide(const ChannelDev& C, float4 g0, float4 g1, bool forced, F2 h[Q],
                                             Mac2& m) {
    m.gx = make_float2(C.G[0], C.G[0]);
    m.gy = make_float2(C.G[1], C.G[1]);
    m.gz = make_float2(C.G[2], C.G[2]);
    if (forced) {
        m.gx = add2(m.gx, make_float2(g0.x, g1.x));
        m.gy = add2(m.gy, make_float2(g0.y, g1.y));
        m.gz = add2(m.gz, make_float2(g0.z, g1.z));
    }
    // moments (pairwise differences of opposite directions first)
    {
        const F2 a1 = sub2(h[1], h[2]), a3 = sub2(h[3], h[4]), a5 = sub2(h[5], h[6]);
        const F2 d7 = sub2(h[7], h[8]), d9 = sub2(h[9], h[10]), d11 = sub2(h[11], h[12]);
        const F2 d13 = sub2(h[13], h[14]), d15 = sub2(h[15], h[16]), d17 = sub2(h[17], h[18]);
        const F2 sa = add2(add2(add2(h[1], h[2]), add2(h[3], h[4])), add2(h[5], h[6]));
        const F2 sd = add2(add2(add2(add2(h[7], h[8]), add2(h[9], h[10])), add2(add2(h[11], h[12]), add2(h[13], h[14]))),
                           add2(add2(h[15], h[16]), add2(h[17], h[18])));
        const F2 dx = add2(add2(d7, d9), add2(d11, d13));
        const F2 dy = add2(sub2(d7, d9), add2(d15, d17));
        const F2 dz = add2(sub2(d11, d13), sub2(d15, d17));
        F2 jx, jy, jz;
        if constexpr (SCALED) {
            const F2 w1 = f2s(wgt(1)), w2 = f2s(wgt(7));
            jx = fma2(w1, a1, mul2(w2, dx));
            jy = fma2(w1, a3, mul2(w2, dy));
            jz = fma2(w1, a5, mul2(w2, dz));
            m.drho = fma2(f2s(wgt(0)), h[0], fma2(w1, sa, mul2(w2, sd)));
        } else {
            jx = add2(a1, dx);
            jy = add2(a3, dy);
            jz = add2(a5, dz);
            m.drho = add2(h[0], add2(sa, sd));
        }
        m.rho = add2(f2s(1.0f), m.drho);
        const F2 irho = make_float2(1.0f / m.rho.x, 1.0f / m.rho.y);
        const F2 half = f2s(0.5f);
        m.ux = mul2(fma2(half, m.gx, jx), irho);
        m.uy = mul2(fma2(half, m.gy, jy), irho);
        m.uz = mul2(fma2(half, m.gz, jz), irho);
    }
    const F2 uu = fma2(m.uz, m.uz, fma2(m.uy, m.uy, mul2(m.ux, m.ux)));
    const F2 ug = fma2(m.uz, m.gz, fma2(m.uy, m.gy, mul2(m.ux, m.gx)));
    const float om_s = C.omega, fp_s = C.fpre;
    m.A1 = fma2(mul2(f2s(-1.5f), m.rho), uu, m.drho);   // drho - 3/2 rho u.u
    m.mug = mul2(f2s(-3.0f * fp_s), ug);                // -3 fp u.g
    const F2 om = f2s(om_s), omc = f2s(1.0f - om_s), c3om = f2s(3.0f * om_s);
    const F2 c9fp = f2s(9.0f * fp_s), c3fp = f2s(3.0f * fp_s);
    // rest population: (1 - om) h0 + w0 [om A1 - 3 fp u.g]
    {
        const F2 X0 = fma2(om, m.A1, m.mug);
        if constexpr (SCALED) h[0] = fma2(omc, h[0], X0);
        else h[0] = fma2(f2s(wgt(0)), X0, mul2(omc, h[0]));
    }
    collide_pair2<SCALED, 1>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 3>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 5>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 7>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 9>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 11>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 13>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 15>(h, m, om, omc, c3om, c9fp, c3fp);
    collide_pair2<SCALED, 17>(h, m, om, omc, c3om, c9fp, c3fp);
}

// Moments, collision and stores of one in-range node pair (h: the pulled
// populations after bounce-back; lk0 / lk1: the nodes' link masks).
template <class S>
__device__ __forceinline__ void pair_collide_store(const LatticeArgs& a, const ChannelDev& C, int gi0, F2 h[Q],
                                                   uint32_t lk0, uint32_t lk1, bool forced, bool prevf) {
    using IO = PairIO<S>;
    const int par = a.par;
    S* dst = (S*)(par ? a.h0 : a.h1);
    const long long NT = a.Ntot;
    float4* gprev = par ? a.g0 : a.g1;
    Mac2 m;
    const float4* gcur = par ? a.g1 : a.g0;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    pair_collide<IO::SCALED>(C, forced ? gcur[gi0] : z4, forced ? gcur[gi0 + 1] : z4, forced, h, m);
    const unsigned seed = sr_seed((unsigned)gi0, m.drho.x, m.ux.y);
    const bool s0 = lk0 & 1u, s1 = lk1 & 1u;
    if (!(s0 || s1)) {
#define LBIBM_P2(I) IO::st2(dst + (size_t)(I) * (size_t)NT + gi0, h[I], seed * sr_k(I));
        LBIBM_ALL_I(LBIBM_P2)
#undef LBIBM_P2
    } else {
        // a solid node keeps its populations; the other one is stored alone
        if (!s0) {
#define LBIBM_P1(I) IO::st1(dst + (size_t)(I) * (size_t)NT + gi0, h[I].x, seed * sr_k(I));
            LBIBM_ALL_I(LBIBM_P1)
#undef LBIBM_P1
        }
        if (!s1) {
#define LBIBM_P1(I) IO::st1(dst + (size_t)(I) * (size_t)NT + gi0 + 1, h[I].y, (seed * sr_k(I)) >> 16);
            LBIBM_ALL_I(LBIBM_P1)
#undef LBIBM_P1
        }
    }
    if (forced) {
        if (!s0) a.u[gi0] = make_float4(m.ux.x, m.uy.x, m.uz.x, m.rho.x);
        if (!s1) a.u[gi0 + 1] = make_float4(m.ux.y, m.uy.y, m.uz.y, m.rho.y);
    }
    if (prevf) {
        if (!s0) gprev[gi0] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!s1) gprev[gi0 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <class S, bool ROW>
__device__ __forceinline__ void sc_pair(const LatticeArgs& a, const ChannelDev& C, int p0, int xr, int yr, int zr) {
    const int gi0 = (int)(C.base + p0);   // even; the padded node count of a context is below 2^31
    const int grp = gi0 >> 5;
    const int par = a.par;
    uint8_t* fl_prev = par ? a.fl0 : a.fl1;
    const bool inr = ROW ? true : p0 < C.n;
    const uint8_t fslow = inr ? __ldg(a.slow + grp) : (uint8_t)0;
    const S* src = (const S*)(par ? a.h1 : a.h0);
    const long long NT = a.Ntot;
    int x0, y, z;
    if constexpr (ROW) {
        x0 = xr; y = yr; z = zr;
    } else {
        const int r = fdiv(p0, C.dnx);
        x0 = p0 - r * C.nx;
        z = fdiv(r, C.dny);
        y = r - z * C.ny;
    }
    PairNbr nb;
    pair_neighbours(C, x0, y, z, nb);
    // phase 1: every population load in flight at once
    F2 h[Q];
#define LBIBM_PP(I) h[I] = pair_pull<S, I>(src, NT, gi0, nb, inr);
    LBIBM_ALL_I(LBIBM_PP)
#undef LBIBM_PP
    // the populations are the previous cycle's; flags and force densities come
    // from the spreading kernel this launch may overlap
    pdl_entry();
    const uint8_t fcur = __ldg((par ? a.fl1 : a.fl0) + grp);
    const uint8_t fprev = __ldg(fl_prev + grp);
    const bool forced = fcur != 0;
    const bool prevf = fprev != 0;
    const bool wslow = __any_sync(FULL, fslow != 0);
    uint32_t lk0 = 0u, lk1 = 0u;
    if (wslow) {
        if (inr && fslow) {
            const uint2 l = __ldg(reinterpret_cast<const uint2*>(a.links + gi0));
            lk0 = l.x;
            lk1 = l.y;
        }
        if (lk0 & ~1u) {
#define LBIBM_PB(I) if (I > 0) pair_bounce<S, I>(src, NT, gi0, lk0, C, y, h[I].x);
            LBIBM_ALL_I(LBIBM_PB)
#undef LBIBM_PB
        }
        if (lk1 & ~1u) {
#define LBIBM_PB(I) if (I > 0) pair_bounce<S, I>(src, NT, gi0 + 1, lk1, C, y, h[I].y);
            LBIBM_ALL_I(LBIBM_PB)
#undef LBIBM_PB
        }
    }
    if (inr) pair_collide_store<S>(a, C, gi0, h, lk0, lk1, forced, prevf);
    // the lane holding the first node of each 32-node group clears the previous
    // step's flag after every lane of the warp has consumed it
    __syncwarp();
    if (prevf && (gi0 & 31) == 0) fl_prev[grp] = 0;
}

// Resident threads per SM of the pair variant's register budget (512: the
// kernel's 122 registers without spills).
#ifndef LBIBM_K3_PAIR_THREADS
#define LBIBM_K3_PAIR_THREADS 512
#endif

template <class S, int BS>
__global__ void __launch_bounds__(BS, LBIBM_K3_PAIR_THREADS / BS) k_stream_collide_pair(const __grid_constant__ LatticeArgs a) {
    // (sc_pair waits for the predecessor after its population loads)
    const int b = blockIdx.x;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (b >= chan(a, k).blk0) c = k;
    const ChannelDev C = chan(a, c);
    const int pb = (b - C.blk0) * (2 * BS);                  // first channel-local node of the block
    const int p0 = pb + 2 * (int)threadIdx.x;
    prefetch_ahead<S>(a, C.base + pb, 2 * BS);
    if (C.nx % (2 * BS) == 0 && pb + 2 * BS <= C.n) {
        // the block is a piece of one row: y and z are the block's
        const int r = fdiv(pb, C.dnx);
        const int z = fdiv(r, C.dny);
        sc_pair<S, true>(a, C, p0, pb - r * C.nx + 2 * (int)threadIdx.x, r - z * C.ny, z);
        return;
    }
    sc_pair<S, false>(a, C, p0, 0, 0, 0);
}

// ---------------------------------------------------------------------------
// Quad variant for 16-bit storage (nodes_per_thread = 4): each thread takes
// the consecutive x-nodes x0 .. x0 + 3 (x0 a multiple of 4) of one row and
// pulls every direction as one aligned 64-bit word of four 16-bit values.  A
// direction with an x component takes the value its first (+x) or last (-x)
// node needs from the neighbouring lane's word by a shuffle, or, at a warp's
// or a row's edge, from one extra aligned 32-bit word.  The words stay packed
// (two registers per direction for four nodes) until the two node pairs are
// unpacked in turn for the packed-FP32 moments and collision, and each
// direction is stored as one 64-bit word.  The 16-bit kernel with one node per
// thread holds too few population bytes in flight per register to cover HBM
// latency; packed words hold four nodes' loads in the registers one node's
// floats would take.
// ---------------------------------------------------------------------------
template <class S> struct QuadIO;
template <> struct QuadIO<__half> {
    // two packed halves (lo: first node) to floats
    static __device__ __forceinline__ F2 unpack(unsigned w) {
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    }
};
template <> struct QuadIO<__nv_bfloat16> {
    static __device__ __forceinline__ F2 unpack(unsigned w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
};

// Row offsets of the pull sources (as PairNbr) and the element offsets, from
// the thread's first node in the source row, of the aligned 32-bit words that
// hold the x-neighbours x0 - 1 (hi half of the word at wxm) and x0 + 4 (lo
// half of the word at wxp).  A missing neighbour (non-periodic x) maps to the
// thread's own word; its link bounces back.
struct QuadNbr {
    int oym, oyp, ozm, ozp;
    int wxm, wxp;
};

__device__ __forceinline__ void quad_neighbours(const ChannelDev& C, int x0, int y, int z, QuadNbr& nb) {
    const int sy = C.nx, sz = C.nx * C.ny;
    nb.oym = y > 0 ? -sy : (C.per[1] ? (C.ny - 1) * sy : 0);
    nb.oyp = y < C.ny - 1 ? sy : (C.per[1] ? -(C.ny - 1) * sy : 0);
    nb.ozm = z > 0 ? -sz : (C.per[2] ? (C.nz - 1) * sz : 0);
    nb.ozp = z < C.nz - 1 ? sz : (C.per[2] ? -(C.nz - 1) * sz : 0);
    nb.wxm = x0 > 0 ? -2 : (C.per[0] ? C.nx - 2 : 0);
    nb.wxp = x0 + 4 < C.nx ? 4 : (C.per[0] ? -x0 : 0);
}

// Phase 1 of direction I: the thread's aligned word of the source row and,
// on an edge lane of a direction with an x component, the extra word.
template <class S, int I>
__device__ __forceinline__ void quad_pull(const S* src, unsigned NT, int gi0, const QuadNbr& nb, bool inr,
                                          bool edge_lo, bool edge_hi, uint2& w, unsigned& e) {
    const S* pl = src + ((unsigned)I * NT + (unsigned)(gi0 + pair_row<I>(nb)));
    w = inr ? __ldcs(reinterpret_cast<const uint2*>(pl)) : make_uint2(0u, 0u);
    e = 0u;
    if constexpr (ex(I) == 1) {
        if (inr && edge_lo) e = __ldcs(reinterpret_cast<const unsigned*>(pl + nb.wxm));
    } else if constexpr (ex(I) == -1) {
        if (inr && edge_hi) e = __ldcs(reinterpret_cast<const unsigned*>(pl + nb.wxp));
    }
}

// Phase 2 (converged warp): shift the word of a direction with an x component
// by one node.  +x: nodes x0 .. x0 + 3 pull x0 - 1 .. x0 + 2; -x: x0 + 1 .. x0 + 4.
template <int I>
__device__ __forceinline__ void quad_shift(uint2& w, unsigned e, bool edge_lo, bool edge_hi) {
    if constexpr (ex(I) == 1) {
        unsigned prev = __shfl_up_sync(FULL, w.y, 1);   // hi half: element x0 - 1
        if (edge_lo) prev = e;
        w = make_uint2(__byte_perm(prev, w.x, 0x5432), __byte_perm(w.x, w.y, 0x5432));
    } else if constexpr (ex(I) == -1) {
        unsigned next = __shfl_down_sync(FULL, w.x, 1);  // lo half: element x0 + 4
        if (edge_hi) next = e;
        w = make_uint2(__byte_perm(w.x, w.y, 0x5432), __byte_perm(w.y, next, 0x5432));
    }
}

// One node pair of the quad (k = 0: nodes x0, x0 + 1 from the words' lo
// halves; k = 1: x0 + 2, x0 + 3): unpack, bounce-back, moments, collision and
// the pair's stores (one 32-bit word per direction, rounded stochastically;
// a solid node keeps its populations).
template <class S>
__device__ __forceinline__ void quad_half(const ChannelDev& C, const S* src, S* dst, unsigned NT, int gi, int y,
                                          const uint2 w[Q], int k, uint32_t lk0, uint32_t lk1, bool forced,
                                          float4 g0, float4 g1, Mac2& m) {
    F2 h[Q];
#define LBIBM_QU(I) h[I] = QuadIO<S>::unpack(k ? w[I].y : w[I].x);
    LBIBM_ALL_I(LBIBM_QU)
#undef LBIBM_QU
    if (lk0 & ~1u) {
#define LBIBM_PB(I) if (I > 0) pair_bounce<S, I>(src, NT, gi, lk0, C, y, h[I].x);
        LBIBM_ALL_I(LBIBM_PB)
#undef LBIBM_PB
    }
    if (lk1 & ~1u) {
#define LBIBM_PB(I) if (I > 0) pair_bounce<S, I>(src, NT, gi + 1, lk1, C, y, h[I].y);
        LBIBM_ALL_I(LBIBM_PB)
#undef LBIBM_PB
    }
    pair_collide<true>(C, g0, g1, forced, h, m);
    const unsigned seed = sr_seed((unsigned)gi, m.drho.x, m.ux.y);
    using IO = PairIO<S>;
    if (!((lk0 | lk1) & 1u)) {
#define LBIBM_P2(I) IO::st2(dst + ((unsigned)(I) * NT + (unsigned)gi), h[I], seed * sr_k(I));
        LBIBM_ALL_I(LBIBM_P2)
#undef LBIBM_P2
    } else {
        if (!(lk0 & 1u)) {
#define LBIBM_P1(I) IO::st1(dst + ((unsigned)(I) * NT + (unsigned)gi), h[I].x, seed * sr_k(I));
            LBIBM_ALL_I(LBIBM_P1)
#undef LBIBM_P1
        }
        if (!(lk1 & 1u)) {
#define LBIBM_P1(I) IO::st1(dst + ((unsigned)(I) * NT + (unsigned)(gi + 1)), h[I].y, (seed * sr_k(I)) >> 16);
            LBIBM_ALL_I(LBIBM_P1)
#undef LBIBM_P1
        }
    }
}

template <class S, bool ROW>
__device__ __forceinline__ void sc_quad(const LatticeArgs& a, const ChannelDev& C, int p0, int lane, int xr, int yr,
                                        int zr) {
    static_assert(sizeof(S) == 2, "the quad variant packs 16-bit populations");
    const int gi0 = (int)(C.base + p0);   // a multiple of 4; the padded node count is below 2^31
    const int grp = gi0 >> 5;
    const int par = a.par;
    uint8_t* fl_prev = par ? a.fl0 : a.fl1;
    const bool inr = ROW ? true : p0 < C.n;
    const uint8_t fslow = inr ? __ldg(a.slow + grp) : (uint8_t)0;
    const S* src = (const S*)(par ? a.h1 : a.h0);
    S* dst = (S*)(par ? a.h0 : a.h1);
    const unsigned NT = (unsigned)a.Ntot;   // Q * plane stride < 2^32 (checked on the host)
    int x0, y, z;
    if constexpr (ROW) {
        x0 = xr; y = yr; z = zr;
    } else {
        const int r = fdiv(p0, C.dnx);
        x0 = p0 - r * C.nx;
        z = fdiv(r, C.dny);
        y = r - z * C.ny;
    }
    QuadNbr nb;
    quad_neighbours(C, x0, y, z, nb);
    const bool edge_lo = lane == 0 || x0 == 0;
    const bool edge_hi = lane == 31 || x0 + 4 == C.nx;
    // phase 1: every population word in flight at once
    // wait for the spreading kernel first, so that this cycle's group flags
    // travel with the population loads instead of after them (the populations
    // are the previous cycle's and could be loaded earlier, but on GB300 the
    // flags' round trip costs more than the overlap with the predecessor's
    // tail gains: 512x256x128 FP16 354.8 -> 343.9 us)
    pdl_entry();
    const uint8_t fcur = __ldg((par ? a.fl1 : a.fl0) + grp);
    const uint8_t fprev = __ldg(fl_prev + grp);
    uint2 w[Q];
    unsigned e[Q];
#define LBIBM_QP(I) quad_pull<S, I>(src, NT, gi0, nb, inr, edge_lo, edge_hi, w[I], e[I]);
    LBIBM_ALL_I(LBIBM_QP)
#undef LBIBM_QP
    const bool forced = fcur != 0;
    const bool prevf = fprev != 0;
    const bool wslow = __any_sync(FULL, fslow != 0);
#define LBIBM_QS(I) quad_shift<I>(w[I], e[I], edge_lo, edge_hi);
    LBIBM_ALL_I(LBIBM_QS)
#undef LBIBM_QS
    uint4 lk = make_uint4(0u, 0u, 0u, 0u);
    if (wslow && inr && fslow) lk = __ldg(reinterpret_cast<const uint4*>(a.links + gi0));
    if (inr) {
        Mac2 m0, m1;
        const float4* gcur = par ? a.g1 : a.g0;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        quad_half<S>(C, src, dst, NT, gi0, y, w, 0, lk.x, lk.y, forced, forced ? gcur[gi0] : z4,
                     forced ? gcur[gi0 + 1] : z4, m0);
        quad_half<S>(C, src, dst, NT, gi0 + 2, y, w, 1, lk.z, lk.w, forced, forced ? gcur[gi0 + 2] : z4,
                     forced ? gcur[gi0 + 3] : z4, m1);
        float4* gprev = par ? a.g0 : a.g1;
        if (forced) {
            if (!(lk.x & 1u)) a.u[gi0] = make_float4(m0.ux.x, m0.uy.x, m0.uz.x, m0.rho.x);
            if (!(lk.y & 1u)) a.u[gi0 + 1] = make_float4(m0.ux.y, m0.uy.y, m0.uz.y, m0.rho.y);
            if (!(lk.z & 1u)) a.u[gi0 + 2] = make_float4(m1.ux.x, m1.uy.x, m1.uz.x, m1.rho.x);
            if (!(lk.w & 1u)) a.u[gi0 + 3] = make_float4(m1.ux.y, m1.uy.y, m1.uz.y, m1.rho.y);
        }
        if (prevf) {
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!(lk.x & 1u)) gprev[gi0] = z4;
            if (!(lk.y & 1u)) gprev[gi0 + 1] = z4;
            if (!(lk.z & 1u)) gprev[gi0 + 2] = z4;
            if (!(lk.w & 1u)) gprev[gi0 + 3] = z4;
        }
    }
    // the lane holding the first node of each 32-node group clears the previous
    // step's flag after every lane of the warp has consumed it
    __syncwarp();
    if (prevf && (gi0 & 31) == 0) fl_prev[grp] = 0;
}

// Resident threads per SM of the quad variant's register budget.
#ifndef LBIBM_K3_QUAD_THREADS
#define LBIBM_K3_QUAD_THREADS 640
#endif

template <class S, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_stream_collide_quad(const __grid_constant__ LatticeArgs a) {
    // (sc_quad waits for the predecessor after its population loads)
    const int b = blockIdx.x;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (b >= chan(a, k).blk0) c = k;
    const ChannelDev C = chan(a, c);
    const int lane = threadIdx.x & 31;
    const int pb = (b - C.blk0) * (4 * BS);                  // first channel-local node of the block
    const int p0 = pb + 4 * (int)threadIdx.x;
    prefetch_ahead<S>(a, C.base + pb, 4 * BS);
    if (C.nx % (4 * BS) == 0 && pb + 4 * BS <= C.n) {
        // the block is a piece of one row: y and z are the block's
        const int r = fdiv(pb, C.dnx);
        const int z = fdiv(r, C.dny);
        sc_quad<S, true>(a, C, p0, lane, pb - r * C.nx + 4 * (int)threadIdx.x, r - z * C.ny, z);
        return;
    }
    sc_quad<S, false>(a, C, p0, lane, 0, 0, 0);
}

// Bulk of the overlapped schedule (one node per thread; a warp is one group).
// Launched with dynamic shared memory it does not use, sized so that fewer
// blocks are resident per SM than registers would allow: the room left over
// takes the blocks of the immersed-boundary kernels running concurrently.
template <class S, int BS>
__global__ void __launch_bounds__(BS, K3MinBlocks<S, 1, BS>::value) k_stream_collide_bulk(const __grid_constant__ LatticeArgs a) {
    const int b = blockIdx.x;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (b >= chan(a, k).blk0) c = k;
    const ChannelDev C = chan(a, c);
    const int lane = threadIdx.x & 31;
    const int p0 = (b - C.blk0) * BS + (int)threadIdx.x;
    if (__ldg(a.dmap + ((C.base + p0) >> 5))) return;   // a stencil group: the list launch takes it
    sc_nodes<S, 1, SC_BULK>(a, C, p0, lane);
}

// Stencil groups of the overlapped schedule: warp w of the grid takes list
// entry `first + w`; k_stream_collide_list_rest takes the entries beyond the
// first grid's warps, if any (a loop, which costs registers, so kept apart).
template <class S>
__device__ __forceinline__ void sc_list_entry(const LatticeArgs& a, int li, int lane) {
    const long long g0 = (long long)__ldg(a.dlist + li) * GROUP;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (g0 >= chan(a, k).base) c = k;
    const ChannelDev C = chan(a, c);
    sc_nodes<S, 1, SC_LIST>(a, C, (int)(g0 - C.base) + lane, lane);
}

template <class S, int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) k_stream_collide_list(const __grid_constant__ LatticeArgs a) {
    const int li = (int)(blockIdx.x * BS + threadIdx.x) >> 5;
    if (li >= __ldg(a.dcount)) return;
    sc_list_entry<S>(a, li, threadIdx.x & 31);
}

template <class S, int BS>
__global__ void __launch_bounds__(BS) k_stream_collide_list_rest(const __grid_constant__ LatticeArgs a, int first) {
    const int nl = __ldg(a.dcount);
    const int nw = (int)(gridDim.x * BS) >> 5;
    for (int li = first + ((int)(blockIdx.x * BS + threadIdx.x) >> 5); li < nl; li += nw)
        sc_list_entry<S>(a, li, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// Staged variant: a persistent block walks over groups of whole lattice rows
// (SG_NODES nodes) of one channel.  For each group it copies, for every
// direction i, the source rows (y - ey_i, z - ez_i) of plane i into shared
// memory with asynchronous 16-byte copies, double-buffered so that the copies
// of the next group are in flight while the current one is computed: the
// bytes in flight are bounded by shared memory, not by registers.  The +-x
// shift is an index into the staged row.  Nodes of groups that touch a wall
// or an obstacle take the per-node path with bounce-back from global memory.
// ---------------------------------------------------------------------------
constexpr int SG_THREADS = 256;

template <class S>
__device__ __forceinline__ int staged_channel(const LatticeArgs& a, int g) {
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (g >= chan(a, k).sg0) c = k;
    return c;
}

template <class S>
__device__ __forceinline__ void staged_issue(const LatticeArgs& a, const S* src, int g, S* B) {
    const ChannelDev& C = chan(a, staged_channel<S>(a, g));
    const int R = C.srows;
    const int r0 = (g - C.sg0) * R;
    const int rows = min(R, C.ny * C.nz - r0);
    const int cpr = C.nx * (int)sizeof(S) / 16;   // 16-byte chunks per row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ij = warp; ij < Q * rows; ij += SG_THREADS / 32) {
        const int i = ij / rows, j = ij - i * rows;
        const int r = r0 + j;
        const int z = fdiv(r, C.dny), y = r - z * C.ny;
        int ys = y - ey(i), zs = z - ez(i);
        bool ok = true;
        if (ys < 0 || ys >= C.ny) {
            if (C.per[1]) ys = (ys + C.ny) % C.ny;
            else ok = false;
        }
        if (zs < 0 || zs >= C.nz) {
            if (C.per[2]) zs = (zs + C.nz) % C.nz;
            else ok = false;
        }
        if (!ok) continue;   // only wall-adjacent rows pull from here; they take the per-node path
        const char* g0 = (const char*)(src + (size_t)i * (size_t)a.Ntot + C.base + (long long)(ys + C.ny * zs) * C.nx);
        char* s0 = (char*)(B + i * SG_NODES + j * C.nx);
        for (int k = lane; k < cpr; k += 32) __pipeline_memcpy_async(s0 + 16 * k, g0 + 16 * k, 16);
    }
}

template <class S>
__device__ __forceinline__ float sm_pop(const S* B, int idx, int i) {
    if constexpr (sizeof(S) == 4) return B[idx];
    else return wgt(i) * to_f(B[idx]);
}

template <class S>
__device__ __forceinline__ void staged_compute(const LatticeArgs& a, const S* src, S* dst, int g, const S* B) {
    const ChannelDev C = chan(a, staged_channel<S>(a, g));
    const int R = C.srows;
    const int r0 = (g - C.sg0) * R;
    const int rows = min(R, C.ny * C.nz - r0);
    const int nn = rows * C.nx;
    const int par = a.par;
    uint8_t* fl_prev = par ? a.fl0 : a.fl1;
    const uint8_t* fl_cur = par ? a.fl1 : a.fl0;
    const float4* gcur = par ? a.g1 : a.g0;
    float4* gprev = par ? a.g0 : a.g1;
    const float om = C.omega, fp = C.fpre;
    const long long NT = a.Ntot;
#pragma unroll 1
    for (int half = 0; half < SG_NODES / SG_THREADS; ++half) {
        const int n = threadIdx.x + half * SG_THREADS;
        const bool inr = n < nn;
        const int p = r0 * C.nx + n;
        const long long gp = C.base + p;
        const int grp = (int)(gp >> 5);
        bool prevf = false;
        if (inr) {
            const bool forced = fl_cur[grp] != 0;
            prevf = fl_prev[grp] != 0;
            const bool slow = __ldg(a.slow + grp) != 0;
            const int j = fdiv(n, C.dnx), x = n - j * C.nx;
            bool active = true;
            float h[Q];
            if (!slow) {
#define LBIBM_SM(I)                                 \
    {                                               \
        int xs = x - ex(I);                         \
        xs += xs < 0 ? C.nx : 0;                    \
        xs -= xs >= C.nx ? C.nx : 0;                \
        h[I] = sm_pop<S>(B, I * SG_NODES + j * C.nx + xs, I); \
    }
                LBIBM_ALL_I(LBIBM_SM)
#undef LBIBM_SM
            } else if (!solid_at(a.mask, gp)) {
                const int z = fdiv(r0 + j, C.dny), y = (r0 + j) - z * C.ny;
                Nbr nb;
                neighbours(C, x, y, z, nb);
                pull_node<S>(src, NT, gp, nb, a.mask, C, y, h);
            } else {
                active = false;
            }
            if (active) {
                float gx = C.G[0], gy = C.G[1], gz = C.G[2];
                if (forced) {
                    const float4 gg = gcur[gp];
                    gx += gg.x; gy += gg.y; gz += gg.z;
                }
                const Mac m = macro(h, gx, gy, gz);
                const unsigned rb = sr_seed((unsigned)gp, m.drho, m.ux);
                collide_all(h, m, om, fp);
#define LBIBM_C1(I) Pop<S>::st(dst, (long long)(I) * NT + gp, h[I], I, rb);
                LBIBM_ALL_I(LBIBM_C1)
#undef LBIBM_C1
                if (forced) a.u[gp] = make_float4(m.ux, m.uy, m.uz, m.rho);
                if (prevf) gprev[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        // the warp holding a 32-node group clears its previous-step flag after use
        __syncwarp();
        if (inr && prevf && (gp & 31) == 0) fl_prev[grp] = 0;
    }
}

template <class S>
__global__ void __launch_bounds__(SG_THREADS, 2) k_stream_collide_staged(const __grid_constant__ LatticeArgs a) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char sm[];
    S* B0 = reinterpret_cast<S*>(sm);
    S* B1 = B0 + Q * SG_NODES;
    const S* src = (const S*)(a.par ? a.h1 : a.h0);
    S* dst = (S*)(a.par ? a.h0 : a.h1);
    int g = blockIdx.x;
    if (g >= a.n_groups) return;
    staged_issue<S>(a, src, g, B0);
    __pipeline_commit();
    int cur = 0;
    for (; g < a.n_groups; g += gridDim.x) {
        const int gn = g + gridDim.x;
        if (gn < a.n_groups) staged_issue<S>(a, src, gn, cur ? B0 : B1);
        __pipeline_commit();
        __pipeline_wait_prior(1);   // the current group's copies have landed
        __syncthreads();
        staged_compute<S>(a, src, dst, g, cur ? B1 : B0);
        __syncthreads();            // every thread is done with this buffer before it is refilled
        cur ^= 1;
    }
}

// ---------------------------------------------------------------------------
// Pipelined variant: a persistent grid of warps walks over 32-node groups
// (one node per lane).  Each warp issues the 19 loads of its next group before
// it computes the current one, so loads are in flight continuously instead of
// only during a load phase; warps whose group touches a wall or an obstacle
// compute it with the per-node path.
// ---------------------------------------------------------------------------
struct PipeNode {
    long long gp;
    int c, x, y, z;
    bool inr;
    uint8_t fcur, fprev, fslow;
};

template <class S>
__device__ __forceinline__ void pipe_issue(const LatticeArgs& a, const S* src, int G, int lane, PipeNode& P,
                                           float v[Q]) {
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (G >= chan(a, k).blk0) c = k;
    const ChannelDev& C = chan(a, c);
    const int p = (G - C.blk0) * 32 + lane;
    P.c = c;
    P.inr = p < C.n;
    P.gp = C.base + p;
    const int gi = (int)P.gp;
    const int grp = gi >> 5;
    P.fcur = __ldg((a.par ? a.fl1 : a.fl0) + grp);
    P.fprev = __ldg((a.par ? a.fl0 : a.fl1) + grp);
    P.fslow = P.inr ? __ldg(a.slow + grp) : (uint8_t)0;
    const int r = fdiv(p, C.dnx);
    P.x = p - r * C.nx;
    P.z = fdiv(r, C.dny);
    P.y = r - P.z * C.ny;
    Nbr nb;
    neighbours(C, P.x, P.y, P.z, nb);
    float extra;
#define LBIBM_IP(I) issue_vec<S, 1, I>(src, a.Ntot, gi, nb, C, P.x, lane, P.inr, &v[I], extra);
    LBIBM_ALL_I(LBIBM_IP)
#undef LBIBM_IP
}

template <class S>
__device__ __forceinline__ void pipe_process(const LatticeArgs& a, const S* src, S* dst, const PipeNode& P,
                                             const float v[Q]) {
    const ChannelDev& C = chan(a, P.c);
    const bool forced = P.fcur != 0, prevf = P.fprev != 0;
    const bool wslow = __any_sync(FULL, P.fslow != 0);
    const long long NT = a.Ntot;
    const long long gp = P.gp;
    const float4* gcur = a.par ? a.g1 : a.g0;
    float4* gprev = a.par ? a.g0 : a.g1;
    bool active = P.inr;
    float h[Q];
    if (!wslow) {
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = v[i];
    } else if (active) {
        const bool obst = (P.fslow & 2) != 0;
        if (obst && solid_at(a.mask, gp)) {
            active = false;
        } else {
            Nbr nb;
            neighbours(C, P.x, P.y, P.z, nb);
            pull_node<S>(src, NT, gp, nb, a.mask, C, P.y, h, obst);
        }
    }
    if (active) {
        float gx = C.G[0], gy = C.G[1], gz = C.G[2];
        if (forced) {
            const float4 g = gcur[gp];
            gx += g.x; gy += g.y; gz += g.z;
        }
        const Mac m = macro(h, gx, gy, gz);
        const float om = C.omega, fp = C.fpre;
        const unsigned rb = sr_seed((unsigned)gp, m.drho, m.ux);
        collide_all(h, m, om, fp);
#define LBIBM_C1(I) Pop<S>::st(dst, (long long)(I) * NT + gp, h[I], I, rb);
        LBIBM_ALL_I(LBIBM_C1)
#undef LBIBM_C1
        if (forced) a.u[gp] = make_float4(m.ux, m.uy, m.uz, m.rho);
        if (prevf) gprev[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    if (P.inr && prevf && (gp & 31) == 0) (a.par ? a.fl0 : a.fl1)[gp >> 5] = 0;
}

template <class S, int BS>
__global__ void __launch_bounds__(BS, 512 / BS) k_stream_collide_pipe(const __grid_constant__ LatticeArgs a) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int n_warps = gridDim.x * (BS / 32);
    int G = blockIdx.x * (BS / 32) + (threadIdx.x >> 5);
    if (G >= a.n_groups) return;   // whole warps leave together
    const S* src = (const S*)(a.par ? a.h1 : a.h0);
    S* dst = (S*)(a.par ? a.h0 : a.h1);
    PipeNode P0, P1;
    float v0[Q], v1[Q];
    pipe_issue<S>(a, src, G, lane, P0, v0);
    // ping-pong between two register sets: the next group's loads are issued
    // before the current group is computed
    for (;;) {
        int Gn = G + n_warps;
        if (Gn < a.n_groups) pipe_issue<S>(a, src, Gn, lane, P1, v1);
        pipe_process<S>(a, src, dst, P0, v0);
        if (Gn >= a.n_groups) break;
        G = Gn;
        Gn = G + n_warps;
        if (Gn < a.n_groups) pipe_issue<S>(a, src, Gn, lane, P0, v0);
        pipe_process<S>(a, src, dst, P1, v1);
        if (Gn >= a.n_groups) break;
        G = Gn;
    }
}

// Differentiable variant (one node per thread).
template <class S, int BS>
__global__ void __launch_bounds__(BS, K3MinBlocks<S, 1, BS>::value) k_stream_collide_brinkman(const __grid_constant__ LatticeArgs a) {
    pdl_entry();
    const int b = blockIdx.x;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (b >= chan(a, k).blk0) c = k;
    const ChannelDev C = chan(a, c);
    sc_nodes<S, 1, SC_BRINK>(a, C, (b - C.blk0) * BS + (int)threadIdx.x, threadIdx.x & 31);
}

// Solid fraction of the differentiable variant at every node of a channel:
// phi = 1 - prod_k (1 - phi_k), phi_k = 1/2 (1 - tanh((|x - c_k| - r_k) / delta)).
__global__ void k_brinkman_phi(ChannelDev C, const float4* beads, int nb, float inv_delta, float* phi) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const int r = fdiv(p, C.dnx);
    const int x = p - r * C.nx;
    const int z = fdiv(r, C.dny);
    const int y = r - z * C.ny;
    float prod = 1.0f;
    for (int k = 0; k < nb; ++k) {
        const float4 bk = beads[k];
        const float dx = (float)x - bk.x, dy = (float)y - bk.y, dz = (float)z - bk.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);
        prod *= 1.0f - 0.5f * (1.0f - tanhf((d - bk.w) * inv_delta));
    }
    phi[C.base + p] = 1.0f - prod;
}

cudaError_t launch_brinkman_phi(const ChannelDev& ch, const float* beads, int nb, float delta, float* phi,
                               cudaStream_t s) {
    k_brinkman_phi<<<(unsigned)((ch.n + 255) / 256), 256, 0, s>>>(ch, reinterpret_cast<const float4*>(beads), nb,
                                                                  1.0f / delta, phi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// TMA-staged variant (FP32, one channel, walls in y and z, nx dividing 512).
// A tile is R = 512 / nx whole rows of one z-plane.  For every direction i the
// R source rows (y - ey_i, z - ez_i) of plane i are one box of a 4-D tensor
// map (x, y, z, direction) copied by the tensor-memory accelerator into shared
// memory; rows outside the channel arrive zero-filled (their links bounce
// back, read from global memory).  Persistent blocks double-buffer: the
// copies of the next tile are in flight while the current one is collided.
// The +-x shift is a wrapped index into the staged row.  Every wait on the
// tile's mbarrier is bounded; a wait that runs out sets tma_err and the block
// stops.
// ---------------------------------------------------------------------------
constexpr unsigned TMA_WAIT_LIMIT = 1u << 20;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// all 19 boxes of tile t into buffer `buf`, one expect_tx for their bytes
template <int TILE>
__device__ __forceinline__ void tma_issue(const CUtensorMap* map, const ChannelDev& C, int R, int t, float* buf,
                                          uint64_t* bar) {
    const int tpz = C.ny / R;
    const int z = t / tpz, y0 = (t - z * tpz) * R;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier generic reads of buf before the async writes
    mbar_expect_tx(bar, (unsigned)(Q * TILE * sizeof(float)));
#pragma unroll
    for (int i = 0; i < Q; ++i) tma_load_4d(buf + i * TILE, map, 0, y0 - ey(i), z - ez(i), i, bar);
}

template <int TILE, int I>
__device__ __forceinline__ float tma_pop(const float* buf, int j, int x, int nx) {
    int xs = x - ex(I);
    xs += xs < 0 ? nx : 0;
    xs -= xs >= nx ? nx : 0;
    return buf[I * TILE + j * nx + xs];
}

// one thread per node of a TILE-node tile; STAGES tiles in a ring of buffers
template <int TILE, int STAGES>
__global__ void __launch_bounds__(TILE, 1024 / TILE) k_stream_collide_tma(const __grid_constant__ LatticeArgs a,
                                                                    const __grid_constant__ CUtensorMap map0,
                                                                    const __grid_constant__ CUtensorMap map1) {
    pdl_entry();
    extern __shared__ __align__(128) unsigned char tma_sm[];
    float* bufs = reinterpret_cast<float*>(tma_sm);                 // [STAGES][19][TILE]
    uint64_t* bars = reinterpret_cast<uint64_t*>(tma_sm + STAGES * Q * TILE * sizeof(float));
    const ChannelDev C = a.chp[0];
    const int R = TILE / C.nx;
    const int tiles = (C.ny / R) * C.nz;
    const int par = a.par;
    const CUtensorMap* map = par ? &map1 : &map0;
    const float* src = (const float*)(par ? a.h1 : a.h0);
    float* dst = (float*)(par ? a.h0 : a.h1);
    uint8_t* fl_prev = par ? a.fl0 : a.fl1;
    const uint8_t* fl_cur = par ? a.fl1 : a.fl0;
    const float4* gcur = par ? a.g1 : a.g0;
    float4* gprev = par ? a.g0 : a.g1;
    const long long NT = a.Ntot;
    const float om = C.omega, fp = C.fpre;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < STAGES; ++k) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // prologue: the block's first STAGES tiles
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < STAGES; ++k) {
            const int t = (int)blockIdx.x + k * (int)gridDim.x;
            if (t < tiles) tma_issue<TILE>(map, C, R, t, bufs + k * Q * TILE, &bars[k]);
        }
    }
    unsigned phase = 0u;   // bit k: parity of buffer k's next completion
    int sidx = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        // bounded wait for this tile's boxes
        unsigned it = 0;
        while (!mbar_try_wait(&bars[sidx], (phase >> sidx) & 1u) && ++it < TMA_WAIT_LIMIT) {
        }
        phase ^= 1u << sidx;
        const float* buf = bufs + sidx * Q * TILE;
        const int tpz = C.ny / R;
        const int z = t / tpz, y0 = (t - z * tpz) * R;
        {
            const int n = threadIdx.x;
            const int j = n / C.nx, x = n - j * C.nx;
            const int y = y0 + j;
            const int gi = (int)C.base + x + C.nx * (y + C.ny * z);
            const int grp = gi >> 5;
            const bool forced = fl_cur[grp] != 0;
            const bool prevf = fl_prev[grp] != 0;
            const bool slow = __ldg(a.slow + grp) != 0;
            float h[Q];
#define LBIBM_TP(I) h[I] = tma_pop<TILE, I>(buf, j, x, C.nx);
            LBIBM_ALL_I(LBIBM_TP)
#undef LBIBM_TP
            // every thread has its populations in registers: the buffer is free.
            // A wait that ran out ends the block (all threads together).
            if (__syncthreads_or(it >= TMA_WAIT_LIMIT)) {
                if (threadIdx.x == 0) {
                    atomicAdd(a.tma_err, 1);
                    // copies still in flight into this block's buffers: wait, bounded, before leaving
                    for (int k = 0; k < STAGES; ++k) {
                        const int tk = t + k * (int)gridDim.x;
                        const int bk = (sidx + k) % STAGES;
                        const unsigned pk = ((phase >> bk) & 1u) ^ (k == 0 ? 1u : 0u);
                        unsigned w = 0;
                        while (tk < tiles && !mbar_try_wait(&bars[bk], pk) && ++w < TMA_WAIT_LIMIT) {
                        }
                    }
                }
                return;
            }
            const int nt = t + STAGES * (int)gridDim.x;
            if (threadIdx.x == 0 && nt < tiles) tma_issue<TILE>(map, C, R, nt, bufs + sidx * Q * TILE, &bars[sidx]);
            uint32_t lk = 0u;
            if (slow) {
                lk = __ldg(a.links + gi);
                bounce_back<float>(src, NT, gi, lk, C, y, h);
            }
            if (!(lk & 1u)) {
                float gx = C.G[0], gy = C.G[1], gz = C.G[2];
                if (forced) {
                    const float4 g = gcur[gi];
                    gx += g.x; gy += g.y; gz += g.z;
                }
                const Mac m = macro(h, gx, gy, gz);
                collide_all(h, m, om, fp);
#define LBIBM_TS(I) dst[(long long)(I) * NT + gi] = h[I];
                LBIBM_ALL_I(LBIBM_TS)
#undef LBIBM_TS
                if (forced) a.u[gi] = make_float4(m.ux, m.uy, m.uz, m.rho);
                if (prevf) gprev[gi] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncwarp();
            if (prevf && (gi & 31) == 0) fl_prev[grp] = 0;
        }
        sidx = sidx == STAGES - 1 ? 0 : sidx + 1;
    }
}

static size_t tma_smem(int tile, int stages) { return stages * ((size_t)Q * tile * sizeof(float) + sizeof(uint64_t)); }

bool tma_variant_ok(const ChannelDev& C, int storage, int n_ch, int tile) {
    return (tile == 256 || tile == 512) && storage == 0 && n_ch == 1 && !C.per[1] && !C.per[2] && C.nx >= 32 &&
           C.nx <= 256 && tile % C.nx == 0 && C.ny % (tile / C.nx) == 0;
}

cudaError_t encode_tma_maps(const ChannelDev& C, int tile, void* h0, void* h1, long long plane, CUtensorMap* maps) {
    using Enc = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)C.nx, (cuuint64_t)C.ny, (cuuint64_t)C.nz, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {(cuuint64_t)C.nx * 4, (cuuint64_t)C.nx * C.ny * 4, (cuuint64_t)plane * 4};
    const cuuint32_t box[4] = {(cuuint32_t)C.nx, (cuuint32_t)(tile / C.nx), 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    void* bases[2] = {h0, h1};
    for (int k = 0; k < 2; ++k) {
        float* base = reinterpret_cast<float*>(bases[k]) + C.base;
        const CUresult r = reinterpret_cast<Enc>(fn)(&maps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides,
                                                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

template <int TILE, int STAGES>
static cudaError_t launch_tma_typed(const LatticeArgs& a, const CUtensorMap* maps, int blocks, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_stream_collide_tma<TILE, STAGES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem(TILE, STAGES));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_ex(k_stream_collide_tma<TILE, STAGES>, blocks, TILE, tma_smem(TILE, STAGES), s, a.pdl, a, maps[0],
                     maps[1]);
}

// (measured on GB300, 256x128x64 filter, tile 256: two buffers at 4 blocks per
// SM and 64 registers, 65.5 us; three buffers 71.5 us, four 91.6 us -- each
// costs a block of residency, and the kernel is issue-bound, not waiting on
// its copies; 48 registers spill, 72.2 us)
constexpr int TMA_STAGES = 2;

template <int TILE>
static int tma_occ() {
    int n = 0;
    cudaError_t e = cudaFuncSetAttribute(k_stream_collide_tma<TILE, TMA_STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem(TILE, TMA_STAGES));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stream_collide_tma<TILE, TMA_STAGES>, TILE,
                                                          tma_smem(TILE, TMA_STAGES));
    return e == cudaSuccess && n > 0 ? n : 1;
}

int tma_blocks_per_sm(int tile) { return tile == 256 ? tma_occ<256>() : tma_occ<512>(); }

cudaError_t launch_stream_collide_tma(const LatticeArgs& a, int tile, const CUtensorMap* maps, int blocks,
                                      cudaStream_t s) {
    if (tile == 256) return launch_tma_typed<256, TMA_STAGES>(a, maps, blocks, s);
    if (tile == 512) return launch_tma_typed<512, TMA_STAGES>(a, maps, blocks, s);
    return cudaErrorInvalidConfiguration;
}


template <class S>
static size_t staged_smem() { return 2 * (size_t)Q * SG_NODES * sizeof(S); }

cudaError_t prepare_staged(int storage) {
    if (storage == 0)
        return cudaFuncSetAttribute(k_stream_collide_staged<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)staged_smem<float>());
    if (storage == 1)
        return cudaFuncSetAttribute(k_stream_collide_staged<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)staged_smem<__half>());
    return cudaFuncSetAttribute(k_stream_collide_staged<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)staged_smem<__nv_bfloat16>());
}

// Supported (nodes per thread, block size) pairs per storage type; npt = 0 is
// the staged variant, npt = -1 the pipelined one.
static const K3Config CFG_F32[] = {{-2, 256}, {-2, 512}, {-1, 128}, {-1, 256}, {0, 256}, {1, 256}, {2, 256}, {4, 256}, {4, 128}, {2, 128}, {1, 128}};
static const K3Config CFG_16[] = { {-1, 128}, {-1, 256}, {0, 256}, {2, 256}, {4, 128}, {4, 64}, {2, 128}, {1, 256}, {1, 128}};

int k3_config_count(int storage) { return storage == 0 ? 11 : 9; }
K3Config k3_config_at(int storage, int k) { return storage == 0 ? CFG_F32[k] : CFG_16[k]; }
bool k3_config_supported(int storage, K3Config c) {
    for (int k = 0; k < k3_config_count(storage); ++k) {
        const K3Config d = k3_config_at(storage, k);
        if (d.npt == c.npt && d.bs == c.bs) return true;
    }
    return false;
}

template <class S>
static cudaError_t launch_sc_typed(const LatticeArgs& a, K3Config c, int blocks, cudaStream_t s) {
#define LBIBM_CASE(N, B)                                   \
    if (c.npt == N && c.bs == B) {                         \
        return launch_ex(k_stream_collide<S, N, B>, blocks, B, 0, s, a.pdl, a); \
    }
    if (c.npt == 2) {
        if (c.bs == 128) return launch_ex(k_stream_collide_pair<S, 128>, blocks, 128, 0, s, a.pdl, a);
        if (c.bs == 256) return launch_ex(k_stream_collide_pair<S, 256>, blocks, 256, 0, s, a.pdl, a);
        return cudaErrorInvalidConfiguration;
    }
    if constexpr (sizeof(S) == 2) {
        if (c.npt == 4) {
            if (c.bs == 64) return launch_ex(k_stream_collide_quad<S, 64, 512 / 64>, blocks, 64, 0, s, a.pdl, a);
            if (c.bs == 128)
                return launch_ex(k_stream_collide_quad<S, 128, LBIBM_K3_QUAD_THREADS / 128>, blocks, 128, 0, s, a.pdl, a);
            return cudaErrorInvalidConfiguration;
        }
    }
    if (c.npt == 0) {
        return launch_ex(k_stream_collide_staged<S>, blocks, SG_THREADS, staged_smem<S>(), s, a.pdl, a);
    }
    if (c.npt == -1) {
        if (c.bs == 128) return launch_ex(k_stream_collide_pipe<S, 128>, blocks, 128, 0, s, a.pdl, a);
        return launch_ex(k_stream_collide_pipe<S, 256>, blocks, 256, 0, s, a.pdl, a);
    }
    if constexpr (sizeof(S) == 4) {
        LBIBM_CASE(1, 256) LBIBM_CASE(4, 256) LBIBM_CASE(4, 128) LBIBM_CASE(1, 128)
    } else {
        LBIBM_CASE(1, 256) LBIBM_CASE(1, 128)
    }
#undef LBIBM_CASE
    return cudaErrorInvalidConfiguration;
}

template <class S>
static cudaError_t launch_sc_split(const LatticeArgs& a, int bs, int mode, int blocks, size_t smem, cudaStream_t s) {
    if (mode == SC_BULK) {
        if (bs == 128) k_stream_collide_bulk<S, 128><<<blocks, 128, smem, s>>>(a);
        else k_stream_collide_bulk<S, 256><<<blocks, 256, smem, s>>>(a);
    } else if (mode == SC_LIST) {
        if (bs == 128) k_stream_collide_list<S, 128><<<blocks, 128, 0, s>>>(a);
        else k_stream_collide_list<S, 256><<<blocks, 256, 0, s>>>(a);
    } else {
        // entries from `smem` on (the warps of the first list grid)
        if (bs == 128) k_stream_collide_list_rest<S, 128><<<blocks, 128, 0, s>>>(a, (int)smem);
        else k_stream_collide_list_rest<S, 256><<<blocks, 256, 0, s>>>(a, (int)smem);
    }
    return cudaGetLastError();
}

template <class S>
static cudaError_t prepare_bulk_typed(int max_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_stream_collide_bulk<S, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_stream_collide_bulk<S, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t prepare_bulk(int storage, int max_smem) {
    if (storage == 0) return prepare_bulk_typed<float>(max_smem);
    if (storage == 1) return prepare_bulk_typed<__half>(max_smem);
    return prepare_bulk_typed<__nv_bfloat16>(max_smem);
}

const void* stream_collide_bulk_func(int storage, int bs) {
    if (storage == 0) return bs == 128 ? (const void*)k_stream_collide_bulk<float, 128> : (const void*)k_stream_collide_bulk<float, 256>;
    if (storage == 1) return bs == 128 ? (const void*)k_stream_collide_bulk<__half, 128> : (const void*)k_stream_collide_bulk<__half, 256>;
    return bs == 128 ? (const void*)k_stream_collide_bulk<__nv_bfloat16, 128> : (const void*)k_stream_collide_bulk<__nv_bfloat16, 256>;
}

cudaError_t launch_stream_collide_split(const LatticeArgs& a, int bs, int mode, int blocks, size_t smem,
                                        cudaStream_t s) {
    if (blocks <= 0) return cudaSuccess;
    if (bs != 128 && bs != 256) return cudaErrorInvalidConfiguration;
    if (a.storage == 0) return launch_sc_split<float>(a, bs, mode, blocks, smem, s);
    if (a.storage == 1) return launch_sc_split<__half>(a, bs, mode, blocks, smem, s);
    return launch_sc_split<__nv_bfloat16>(a, bs, mode, blocks, smem, s);
}

template <class S>
static cudaError_t launch_sc_brinkman(const LatticeArgs& a, int bs, int blocks, cudaStream_t s) {
    if (bs == 128) return launch_ex(k_stream_collide_brinkman<S, 128>, blocks, 128, 0, s, a.pdl, a);
    return launch_ex(k_stream_collide_brinkman<S, 256>, blocks, 256, 0, s, a.pdl, a);
}

cudaError_t launch_stream_collide(const LatticeArgs& a, K3Config cfg, int total_blocks, cudaStream_t s) {
    if (total_blocks <= 0) return cudaSuccess;
    if (a.phi) {
        if (cfg.npt != 1) return cudaErrorInvalidConfiguration;
        if (a.storage == 0) return launch_sc_brinkman<float>(a, cfg.bs, total_blocks, s);
        if (a.storage == 1) return launch_sc_brinkman<__half>(a, cfg.bs, total_blocks, s);
        return launch_sc_brinkman<__nv_bfloat16>(a, cfg.bs, total_blocks, s);
    }
    if (a.storage == 0) return launch_sc_typed<float>(a, cfg, total_blocks, s);
    if (a.storage == 1) return launch_sc_typed<__half>(a, cfg, total_blocks, s);
    return launch_sc_typed<__nv_bfloat16>(a, cfg, total_blocks, s);
}

// ---------------------------------------------------------------------------
// Adjoint of the stream-collide of the differentiable variant (FP32
// populations, one node per thread).  The adjoint of this step's output h'_i
// at x is gathered from the adjoint of the next step's pulled populations:
// the next step pulled h'_i at x + e_i, or at x itself as direction opp(i)
// when that link bounces back (bit opp(i) of x's link mask).  Then the
// vector-Jacobian product of h'_i = (1 - om) f_i + om f^eq_i(rho, u) + S_i(u, g_tot)
// with u = (j + g/2) / (rho D), g_tot = g - a (j + g/2) / D, D = 1 + a/2,
// a = alpha phi, with respect to the pulled populations f (lam_out), the force
// density g (lam_g) and phi (accumulated into Lphi); lam_u carries the
// interpolation's use of u.
// ---------------------------------------------------------------------------
template <int I, bool SLOW>
__device__ __forceinline__ void adj_pull(const AdjArgs& a, long long NT, int gi, const Nbr& nb, uint32_t lk,
                                         const ChannelDev& C, int y, float f[Q], float lh[Q]) {
    const float* hp = a.h_t + (size_t)I * (size_t)NT;       // plane of direction I (warp-uniform)
    const float* lp = a.lam_in + (size_t)I * (size_t)NT;
    bool ok, ok2;
    const int o = src_off<I>(nb, ok);
    const int o2 = src_off<opp(I)>(nb, ok2);   // offset to x + e_I
    if constexpr (!SLOW) {
        // no wall or obstacle link in this warp's group
        f[I] = __ldg(hp + gi + o);
        lh[I] = __ldg(lp + gi + o2);
    } else {
        if ((lk >> I) & 1u) ok = false;
        float v = ok ? __ldg(hp + gi + o) : __ldg(a.h_t + (size_t)opp(I) * (size_t)NT + gi);
        if (!ok && C.has_uw && !C.per[1]) {
            const int wall = (ey(I) == 1 && y == 0) ? 0 : ((ey(I) == -1 && y == C.ny - 1) ? 1 : -1);
            if (wall >= 0) v += 6.0f * wgt(I) * (ex(I) * C.uw[wall][0] + ey(I) * C.uw[wall][1] + ez(I) * C.uw[wall][2]);
        }
        f[I] = v;
        if ((lk >> opp(I)) & 1u) ok2 = false;
        lh[I] = ok2 ? __ldg(lp + gi + o2) : __ldg(a.lam_in + (size_t)opp(I) * (size_t)NT + gi);
    }
}

template <bool SLOW>
__device__ __forceinline__ void adj_node(const AdjArgs& a, const ChannelDev& C, int gi, int x, int y, int z) {
    const long long gp = gi;
    Nbr nb;
    neighbours(C, x, y, z, nb);
    const long long NT = a.plane;
    const uint32_t lk = SLOW ? __ldg(a.links + gp) : 0u;
    float f[Q], lh[Q];
#define LBIBM_AP(I) adj_pull<I, SLOW>(a, NT, gi, nb, lk, C, y, f, lh);
    LBIBM_ALL_I(LBIBM_AP)
#undef LBIBM_AP
    // The pulls above read the segment store and the adjoint written two kernels
    // back, complete when this kernel starts; only the interpolation's adjoint
    // lam_u comes from the kernel before it.
    pdl_entry();
    float drho, jx, jy, jz;
    moments(f, drho, jx, jy, jz);
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    // IB force, the interpolation's adjoint and lam_g live on the stencil groups only
    const bool forced = __ldg(a.fl_t + (gp >> 5)) != 0;
    float gx = C.G[0], gy = C.G[1], gz = C.G[2];
    float4 lu = make_float4(0.f, 0.f, 0.f, 0.f);
    if (forced) {
        const float4 gs = a.g_t[gp];
        gx += gs.x; gy += gs.y; gz += gs.z;
        lu = a.lam_u[gp];
        a.lam_u[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float phi = a.phi ? __ldg(a.phi + gp) : 0.f;
    const float al = a.alpha * phi;
    const float iD = 1.0f / (1.0f + 0.5f * al);
    const float vx = jx + 0.5f * gx, vy = jy + 0.5f * gy, vz = jz + 0.5f * gz;
    const float s = iD * irho;
    const float ux = vx * s, uy = vy * s, uz = vz * s;
    const float tx = gx - al * vx * iD, ty = gy - al * vy * iD, tz = gz - al * vz * iD;   // g_tot
    const float uu = ux * ux + uy * uy + uz * uz;
    const float om = C.omega, fp = C.fpre;
    // sums over the outputs, opposite directions in pairs (e_J = -e_I): with
    // S = L_I + L_J and D = L_I - L_J every term splits into an even and an odd part
    float lrho = lh[0] * (om * wgt(0)) * (1.0f - 1.5f * uu);
    float lux = lh[0] * (-3.0f * wgt(0)) * ((om * rho) * ux + fp * tx);
    float luy = lh[0] * (-3.0f * wgt(0)) * ((om * rho) * uy + fp * ty);
    float luz = lh[0] * (-3.0f * wgt(0)) * ((om * rho) * uz + fp * tz);
    float ltx = lh[0] * (-3.0f * fp * wgt(0)) * ux;
    float lty = lh[0] * (-3.0f * fp * wgt(0)) * uy;
    float ltz = lh[0] * (-3.0f * fp * wgt(0)) * uz;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float Sp = lh[i] + lh[i + 1], Dm = lh[i] - lh[i + 1];
        const float w = wgt(i);
        const float eu = ex(i) * ux + ey(i) * uy + ez(i) * uz;
        const float et = ex(i) * tx + ey(i) * ty + ez(i) * tz;
        // d feq / d rho: om w (1 + 3 eu + 4.5 eu^2 - 1.5 uu)
        lrho += (om * w) * (Sp * (1.0f + 4.5f * eu * eu - 1.5f * uu) + 3.0f * eu * Dm);
        // d h' / d u: e [3 om w rho D + 9 w (om rho eu + fp et) S] - 3 w (om rho u + fp t) S
        const float ce = 3.0f * (om * w) * rho * Dm + 9.0f * w * ((om * rho) * eu + fp * et) * Sp;
        const float cu = -3.0f * w * Sp;
        lux += ce * ex(i) + cu * ((om * rho) * ux + fp * tx);
        luy += ce * ey(i) + cu * ((om * rho) * uy + fp * ty);
        luz += ce * ez(i) + cu * ((om * rho) * uz + fp * tz);
        // d S / d g_tot: fp w (e [3 D + 9 eu S] - 3 u S)
        const float te = fp * w * (3.0f * Dm + 9.0f * eu * Sp);
        const float tu = -3.0f * fp * w * Sp;
        ltx += te * ex(i) + tu * ux;
        lty += te * ey(i) + tu * uy;
        ltz += te * ez(i) + tu * uz;
    }
    lux += lu.x; luy += lu.y; luz += lu.z;
    const float lvx = lux * s - ltx * al * iD, lvy = luy * s - lty * al * iD, lvz = luz * s - ltz * al * iD;
    lrho -= (lux * ux + luy * uy + luz * uz) * irho;
    const float lgx = 0.5f * lvx + ltx, lgy = 0.5f * lvy + lty, lgz = 0.5f * lvz + ltz;
    float* lo = a.lam_out;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        lo[(size_t)i * (size_t)NT + gi] = (1.0f - om) * lh[i] + lrho + ex(i) * lvx + ey(i) * lvy + ez(i) * lvz;
    if (forced) a.lam_g[gp] = make_float4(lgx, lgy, lgz, 0.f);
    if (al != 0.f) {   // phi is exactly 0 away from the beads (tanh saturates in FP32)
        const float iD2 = iD * iD;
        const float lphi = -0.5f * a.alpha * (lux * vx + luy * vy + luz * vz) * iD2 * irho -
                           a.alpha * (ltx * vx + lty * vy + ltz * vz) * iD2;
        a.Lphi[gp] += lphi;
    }
}

__global__ void __launch_bounds__(128, 8) k_adj_collide(const __grid_constant__ AdjArgs a) {
    // (adj_node waits for the predecessor after its pulls)
    const ChannelDev C = a.ch;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool inr = p < C.n;
    const long long gp = C.base + p;   // inside the channel's padded range
    const uint8_t fslow = inr ? __ldg(a.slow + (gp >> 5)) : (uint8_t)0;
    const bool wslow = __any_sync(0xffffffffu, fslow != 0);
    if (!inr || solid_at(a.mask, gp)) return;   // bitmask obstacle nodes do not update
    const int r = fdiv(p, C.dnx);
    const int x = p - r * C.nx;
    const int z = fdiv(r, C.dny);
    const int y = r - z * C.ny;
    if (wslow) adj_node<true>(a, C, (int)gp, x, y, z);
    else adj_node<false>(a, C, (int)gp, x, y, z);
}

cudaError_t launch_adj_collide(const AdjArgs& a, cudaStream_t s) {
    return launch_ex(k_adj_collide, (a.ch.n + 127) / 128, 128, 0, s, a.pdl, a);
}

// ---------------------------------------------------------------------------
// Fields: rho and the force-corrected velocity of the last collision, from the
// stored post-collision populations: sum_i e_i f*_i = rho u + g/2.
// ---------------------------------------------------------------------------
template <class S>
__global__ void k_fields(const __grid_constant__ LatticeArgs a, int c, float* rho_out, float* u_out) {
    const ChannelDev& C = chan(a, c);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const long long gp = C.base + p;
    if (!a.has_last || solid_at(a.mask, gp)) {
        if (rho_out) rho_out[p] = 1.0f;
        if (u_out) { u_out[p] = 0.f; u_out[(long long)C.n + p] = 0.f; u_out[2LL * C.n + p] = 0.f; }
        return;
    }
    if (a.phi) {
        // differentiable variant: the collision wrote rho and u at every node
        const float4 uu = a.u[gp];
        if (rho_out) rho_out[p] = uu.w;
        if (u_out) { u_out[p] = uu.x; u_out[(long long)C.n + p] = uu.y; u_out[2LL * C.n + p] = uu.z; }
        return;
    }
    // the last step had parity 1 - par and wrote h[par]
    const S* hs = (const S*)(a.par ? a.h1 : a.h0);
    float h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = Pop<S>::ld(hs, (long long)i * a.Ntot + gp, i);
    float drho, jx, jy, jz;
    moments(h, drho, jx, jy, jz);
    float gx = C.G[0], gy = C.G[1], gz = C.G[2];
    if ((a.par ? a.fl0 : a.fl1)[gp >> 5]) {
        const float4 g = (a.par ? a.g0 : a.g1)[gp];
        gx += g.x; gy += g.y; gz += g.z;
    }
    const float rho = 1.0f + drho;
    if (rho_out) rho_out[p] = rho;
    if (u_out) {
        u_out[p] = (jx - 0.5f * gx) / rho;
        u_out[(long long)C.n + p] = (jy - 0.5f * gy) / rho;
        u_out[2LL * C.n + p] = (jz - 0.5f * gz) / rho;
    }
}

static int chan_n_host(const LatticeArgs& a, int c) { return c < MAXCH_P ? a.chp[c].n : -1; }

cudaError_t launch_fields(const LatticeArgs& a, int c, float* rho, float* u, cudaStream_t s) {
    const int B = 256;
    const int n = chan_n_host(a, c);
    if (n < 0) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((n + B - 1) / B);
    if (a.storage == 0) k_fields<float><<<blocks, B, 0, s>>>(a, c, rho, u);
    else if (a.storage == 1) k_fields<__half><<<blocks, B, 0, s>>>(a, c, rho, u);
    else k_fields<__nv_bfloat16><<<blocks, B, 0, s>>>(a, c, rho, u);
    return cudaGetLastError();
}

// Pre-collision (post-stream) shifted populations of the next step.
template <class S>
__global__ void k_pull_populations(const __grid_constant__ LatticeArgs a, int c, float* h_out) {
    const ChannelDev& C = chan(a, c);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const long long gp = C.base + p;
    const S* src = (const S*)(a.par ? a.h1 : a.h0);
    float h[Q];
    if (solid_at(a.mask, gp)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = 0.0f;
    } else {
        const int r = fdiv(p, C.dnx);
        const int x = p - r * C.nx;
        const int z = fdiv(r, C.dny);
        const int y = r - z * C.ny;
        Nbr nb;
        neighbours(C, x, y, z, nb);
        pull_node<S>(src, a.Ntot, gp, nb, a.mask, C, y, h);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) h_out[(long long)i * C.n + p] = h[i];
}

cudaError_t launch_pull_populations(const LatticeArgs& a, int c, float* h_out, cudaStream_t s) {
    const int B = 256;
    const int n = chan_n_host(a, c);
    if (n < 0) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((n + B - 1) / B);
    if (a.storage == 0) k_pull_populations<float><<<blocks, B, 0, s>>>(a, c, h_out);
    else if (a.storage == 1) k_pull_populations<__half><<<blocks, B, 0, s>>>(a, c, h_out);
    else k_pull_populations<__nv_bfloat16><<<blocks, B, 0, s>>>(a, c, h_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conservation diagnostics: FP64 per-thread sums, FP64 block reduction, one
// partial per block, then an ordered final sum (deterministic).
// ---------------------------------------------------------------------------
constexpr int DIAG_BLOCK = 256;
constexpr int DIAG_N = 6;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, o));
    return v;
}

template <class S>
__global__ void __launch_bounds__(DIAG_BLOCK) k_diag_partial(const __grid_constant__ LatticeArgs a, int c,
                                                             double* partials) {
    const ChannelDev& C = chan(a, c);
    const S* hs = (const S*)(a.par ? a.h1 : a.h0);
    const uint8_t* fl = a.par ? a.fl0 : a.fl1;
    const float4* gg = a.par ? a.g0 : a.g1;
    double acc[DIAG_N] = {0, 0, 0, 0, 0, 0};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < C.n; p += gridDim.x * blockDim.x) {
        const long long gp = C.base + p;
        if (solid_at(a.mask, gp)) continue;
        float h[Q];
        int bad = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            h[i] = Pop<S>::ld(hs, (long long)i * a.Ntot + gp, i);
            bad += !isfinite(h[i]);
        }
        float drho, jx, jy, jz;
        moments(h, drho, jx, jy, jz);
        acc[0] += 1.0 + (double)drho;
        acc[1] += jx; acc[2] += jy; acc[3] += jz;
        acc[4] += bad;
        if (a.has_last) {
            float gx = C.G[0], gy = C.G[1], gz = C.G[2];
            if (fl[gp >> 5]) { const float4 g = gg[gp]; gx += g.x; gy += g.y; gz += g.z; }
            const double rho = 1.0 + (double)drho;
            const double ux = (jx - 0.5 * gx) / rho, uy = (jy - 0.5 * gy) / rho, uz = (jz - 0.5 * gz) / rho;
            const double um = sqrt(ux * ux + uy * uy + uz * uz);
            acc[5] = (um != um) ? INFINITY : fmax(acc[5], um);
        }
    }
    __shared__ double sh[DIAG_BLOCK / 32][DIAG_N];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < DIAG_N; ++k) {
        const double v = (k == 5) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_N) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < DIAG_BLOCK / 32; ++w) v = (k == 5) ? fmax(v, sh[w][k]) : v + sh[w][k];
        partials[(long long)blockIdx.x * DIAG_N + k] = v;
    }
}

__global__ void k_diag_final(const double* partials, int n_blocks, double* out) {
    const int k = threadIdx.x;
    if (k >= DIAG_N) return;
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) {
        const double x = partials[(long long)b * DIAG_N + k];
        v = (k == 5) ? fmax(v, x) : v + x;
    }
    out[k] = v;
}

cudaError_t launch_diagnostics(const LatticeArgs& a, int c, double* partials, int n_blocks, double* out,
                               cudaStream_t s) {
    if (a.storage == 0) k_diag_partial<float><<<n_blocks, DIAG_BLOCK, 0, s>>>(a, c, partials);
    else if (a.storage == 1) k_diag_partial<__half><<<n_blocks, DIAG_BLOCK, 0, s>>>(a, c, partials);
    else k_diag_partial<__nv_bfloat16><<<n_blocks, DIAG_BLOCK, 0, s>>>(a, c, partials);
    k_diag_final<<<1, 32, 0, s>>>(partials, n_blocks, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Obstacles (Sec. 2.4, 2.5).  One block per sphere covers the sphere's
// bounding box; the membership test |x - c|^2 <= r^2 runs in double with
// explicitly rounded operations (no contraction), so it matches a plain double
// evaluation bit for bit.  Spheres are not imaged across periodic boundaries.
// ---------------------------------------------------------------------------
__global__ void k_rasterise_spheres(const float4* sph, ChannelDev C, uint32_t* mask) {
    const float4 s = sph[blockIdx.x];
    const double cx = s.x, cy = s.y, cz = s.z, r = s.w;
    const int x0 = max(0, (int)ceil(cx - r)), x1 = min(C.nx - 1, (int)floor(cx + r));
    const int y0 = max(0, (int)ceil(cy - r)), y1 = min(C.ny - 1, (int)floor(cy + r));
    const int z0 = max(0, (int)ceil(cz - r)), z1 = min(C.nz - 1, (int)floor(cz + r));
    if (x1 < x0 || y1 < y0 || z1 < z0) return;
    const int bx = x1 - x0 + 1, by = y1 - y0 + 1, bz = z1 - z0 + 1;
    const double r2 = __dmul_rn(r, r);
    for (int k = threadIdx.x; k < bx * by * bz; k += blockDim.x) {
        const int x = x0 + k % bx, y = y0 + (k / bx) % by, z = z0 + k / (bx * by);
        const double dx = __dadd_rn((double)x, -cx), dy = __dadd_rn((double)y, -cy), dz = __dadd_rn((double)z, -cz);
        double d2 = __dmul_rn(dx, dx);
        d2 = __dadd_rn(d2, __dmul_rn(dy, dy));
        d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
        if (d2 <= r2) {
            const long long g = C.base + x + (long long)C.nx * (y + (long long)C.ny * z);
            atomicOr(mask + (g >> 5), 1u << (g & 31));
        }
    }
}

__global__ void k_rasterise_extra(const uint8_t* extra, ChannelDev C, uint32_t* mask) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n || !extra[p]) return;
    const long long g = C.base + p;
    atomicOr(mask + (g >> 5), 1u << (g & 31));
}

cudaError_t launch_rasterise(const float* spheres, int n_spheres, const uint8_t* extra, const ChannelDev& ch,
                             uint32_t* mask, cudaStream_t s) {
    if (n_spheres > 0) k_rasterise_spheres<<<n_spheres, 256, 0, s>>>((const float4*)spheres, ch, mask);
    if (extra) k_rasterise_extra<<<(unsigned)((ch.n + 255) / 256), 256, 0, s>>>(extra, ch, mask);
    return cudaGetLastError();
}

// A 32-node group is "slow" when one of its nodes is solid or has one of the
// 18 neighbours solid or outside the domain; the stream-collide kernel checks
// the mask and bounds only there.
// Link masks and slow-group flags of one channel.  Link mask of a node: bit i
// (1..18) set when the pull source x - e_i lies outside the domain on a
// non-periodic axis or on an obstacle node, i.e. population i is bounced back;
// bit 0 set when the node itself is solid.  Group flag: bit 0 = a node of the
// 32-node group has a link leaving the domain, bit 1 = an obstacle node in the
// group or next to it.
__global__ void k_slow_flags(ChannelDev C, const uint32_t* mask, uint8_t* slow, uint32_t* links) {
    // one warp covers one 32-node group (channel bases are multiples of 32)
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const long long gp = C.base + p;
    bool wall = false, obst = false;
    uint32_t lk = 0u;
    if (p < C.n) obst = solid_at(mask, gp);
    if (p < C.n && !obst) {
        const int r = fdiv(p, C.dnx);
        const int x = p - r * C.nx;
        const int z = fdiv(r, C.dny);
        const int y = r - z * C.ny;
        Nbr nb;
        neighbours(C, x, y, z, nb);
        bool ok;
#define LBIBM_CHK(I)                                        \
    {                                                       \
        const int o = src_off<I>(nb, ok);                   \
        const bool sld = ok && solid_at(mask, gp + o);      \
        wall = wall || !ok;                                 \
        obst = obst || sld;                                 \
        if (!ok || sld) lk |= 1u << I;                      \
    }
        LBIBM_CHK(1) LBIBM_CHK(2) LBIBM_CHK(3) LBIBM_CHK(4) LBIBM_CHK(5) LBIBM_CHK(6) LBIBM_CHK(7)
        LBIBM_CHK(8) LBIBM_CHK(9) LBIBM_CHK(10) LBIBM_CHK(11) LBIBM_CHK(12) LBIBM_CHK(13) LBIBM_CHK(14)
        LBIBM_CHK(15) LBIBM_CHK(16) LBIBM_CHK(17) LBIBM_CHK(18)
#undef LBIBM_CHK
    } else if (p < C.n) {
        lk = 1u;
    }
    if (p < C.n) links[gp] = lk;
    const bool any_wall = __any_sync(FULL, wall), any_obst = __any_sync(FULL, obst);
    if ((threadIdx.x & 31) == 0) slow[gp >> 5] = (uint8_t)(any_wall | (any_obst << 1));
}

cudaError_t launch_slow_flags(const ChannelDev& ch, const uint32_t* mask, uint8_t* slow, uint32_t* links,
                              cudaStream_t s) {
    k_slow_flags<<<(unsigned)((ch.n + 255) / 256), 256, 0, s>>>(ch, mask, slow, links);
    return cudaGetLastError();
}

}  // namespace lbibm
