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
#include "lbibm_internal.cuh"

namespace lbibm {

constexpr int K3_BLOCK = 256;
static_assert(CH_ALIGN % K3_BLOCK == 0, "channel padding must cover whole stream-collide blocks");
int stream_collide_block_size() { return K3_BLOCK; }

// ---------------------------------------------------------------------------
// population storage
// ---------------------------------------------------------------------------
template <class S> struct Pop;
template <> struct Pop<float> {
    static __device__ __forceinline__ float ld(const float* p, long long idx, int) { return __ldg(p + idx); }
    static __device__ __forceinline__ void st(float* p, long long idx, float h, int) { p[idx] = h; }
};
template <> struct Pop<__half> {
    static __device__ __forceinline__ float ld(const __half* p, long long idx, int i) {
        return wgt(i) * __half2float(__ldg(p + idx));
    }
    static __device__ __forceinline__ void st(__half* p, long long idx, float h, int i) {
        p[idx] = __float2half_rn(h * (1.0f / wgt(i)));
    }
};
template <> struct Pop<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, long long idx, int i) {
        return wgt(i) * __bfloat162float(__ldg(p + idx));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, long long idx, float h, int i) {
        p[idx] = __float2bfloat16_rn(h * (1.0f / wgt(i)));
    }
};

__device__ __forceinline__ bool solid_at(const uint32_t* mask, long long g) {
    return (__ldg(mask + (g >> 5)) >> (g & 31)) & 1u;
}

// Source offsets of the pull scheme for one node: for each axis the linear
// offset to the neighbour at coordinate -1 ("m") and +1 ("p"), with periodic
// wrap, and whether that neighbour exists.
struct Nbr {
    long long om[3], op[3];
    bool vm[3], vp[3];
};

__device__ __forceinline__ void neighbours(const ChannelDev& C, int x, int y, int z, Nbr& nb) {
    const long long sx = 1, sy = C.nx, sz = (long long)C.nx * C.ny;
    const int c[3] = {x, y, z};
    const int n[3] = {C.nx, C.ny, C.nz};
    const long long s[3] = {sx, sy, sz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (c[d] > 0) { nb.om[d] = -s[d]; nb.vm[d] = true; }
        else if (C.per[d]) { nb.om[d] = (long long)(n[d] - 1) * s[d]; nb.vm[d] = true; }
        else { nb.om[d] = 0; nb.vm[d] = false; }
        if (c[d] < n[d] - 1) { nb.op[d] = s[d]; nb.vp[d] = true; }
        else if (C.per[d]) { nb.op[d] = -(long long)(n[d] - 1) * s[d]; nb.vp[d] = true; }
        else { nb.op[d] = 0; nb.vp[d] = false; }
    }
}

// Offset of the pull source x - e_i and whether it lies inside the domain.
template <int I>
__device__ __forceinline__ long long src_off(const Nbr& nb, bool& ok) {
    long long o = 0;
    ok = true;
    if (ex(I) == 1) { o += nb.om[0]; ok = ok && nb.vm[0]; }
    if (ex(I) == -1) { o += nb.op[0]; ok = ok && nb.vp[0]; }
    if (ey(I) == 1) { o += nb.om[1]; ok = ok && nb.vm[1]; }
    if (ey(I) == -1) { o += nb.op[1]; ok = ok && nb.vp[1]; }
    if (ez(I) == 1) { o += nb.om[2]; ok = ok && nb.vm[2]; }
    if (ez(I) == -1) { o += nb.op[2]; ok = ok && nb.vp[2]; }
    return o;
}

// Pull one population with bounce-back where the source is a wall or solid.
template <class S, int I>
__device__ __forceinline__ float pull_slow(const S* src, long long NT, long long gp, const Nbr& nb,
                                           const uint32_t* mask, const ChannelDev& C, int y) {
    bool ok;
    const long long o = src_off<I>(nb, ok);
    if (ok) ok = !solid_at(mask, gp + o);
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

template <class S>
__device__ __forceinline__ void pull_all(const S* src, long long NT, long long gp, const Nbr& nb,
                                         const uint32_t* mask, const ChannelDev& C, int y, bool slow, float h[Q]) {
    if (slow) {
        h[0] = pull_slow<S, 0>(src, NT, gp, nb, mask, C, y);
        h[1] = pull_slow<S, 1>(src, NT, gp, nb, mask, C, y);
        h[2] = pull_slow<S, 2>(src, NT, gp, nb, mask, C, y);
        h[3] = pull_slow<S, 3>(src, NT, gp, nb, mask, C, y);
        h[4] = pull_slow<S, 4>(src, NT, gp, nb, mask, C, y);
        h[5] = pull_slow<S, 5>(src, NT, gp, nb, mask, C, y);
        h[6] = pull_slow<S, 6>(src, NT, gp, nb, mask, C, y);
        h[7] = pull_slow<S, 7>(src, NT, gp, nb, mask, C, y);
        h[8] = pull_slow<S, 8>(src, NT, gp, nb, mask, C, y);
        h[9] = pull_slow<S, 9>(src, NT, gp, nb, mask, C, y);
        h[10] = pull_slow<S, 10>(src, NT, gp, nb, mask, C, y);
        h[11] = pull_slow<S, 11>(src, NT, gp, nb, mask, C, y);
        h[12] = pull_slow<S, 12>(src, NT, gp, nb, mask, C, y);
        h[13] = pull_slow<S, 13>(src, NT, gp, nb, mask, C, y);
        h[14] = pull_slow<S, 14>(src, NT, gp, nb, mask, C, y);
        h[15] = pull_slow<S, 15>(src, NT, gp, nb, mask, C, y);
        h[16] = pull_slow<S, 16>(src, NT, gp, nb, mask, C, y);
        h[17] = pull_slow<S, 17>(src, NT, gp, nb, mask, C, y);
        h[18] = pull_slow<S, 18>(src, NT, gp, nb, mask, C, y);
    } else {
        bool ok;
#define LBIBM_PULL(I) h[I] = Pop<S>::ld(src, (long long)(I) * NT + gp + src_off<I>(nb, ok), I);
        LBIBM_PULL(0) LBIBM_PULL(1) LBIBM_PULL(2) LBIBM_PULL(3) LBIBM_PULL(4) LBIBM_PULL(5) LBIBM_PULL(6)
        LBIBM_PULL(7) LBIBM_PULL(8) LBIBM_PULL(9) LBIBM_PULL(10) LBIBM_PULL(11) LBIBM_PULL(12)
        LBIBM_PULL(13) LBIBM_PULL(14) LBIBM_PULL(15) LBIBM_PULL(16) LBIBM_PULL(17) LBIBM_PULL(18)
#undef LBIBM_PULL
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

// BGK collision with Guo forcing on shifted populations:
//   h*_i = h_i + omega (h_i^eq - h_i) + S_i,
//   h_i^eq = w_i [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u)],
//   S_i = (1 - 1/2tau) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . g.
template <int I>
__device__ __forceinline__ float collide_one(float hi, float drho, float rho, float ux, float uy, float uz, float uu,
                                             float gx, float gy, float gz, float ug, float omega, float fpre) {
    const float eu = ex(I) * ux + ey(I) * uy + ez(I) * uz;
    const float eg = ex(I) * gx + ey(I) * gy + ez(I) * gz;
    const float heq = wgt(I) * (drho + rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * uu));
    const float s = fpre * wgt(I) * (3.0f * (eg - ug) + 9.0f * eu * eg);
    return hi + omega * (heq - hi) + s;
}

template <class S>
__global__ void __launch_bounds__(K3_BLOCK) k_stream_collide(LatticeArgs a) {
    const int b = blockIdx.x;
    int c = 0;
    for (int k = 1; k < a.n_ch; ++k)
        if (b >= a.ch[k].blk0) c = k;
    const ChannelDev C = a.ch[c];
    const long long p = (long long)(b - C.blk0) * K3_BLOCK + threadIdx.x;
    const long long gp = C.base + p;
    const int grp = (int)(gp >> 5);
    const int par = a.par;
    uint8_t* fl_prev = par ? a.fl0 : a.fl1;
    const bool forced = __ldg((par ? a.fl1 : a.fl0) + grp) != 0;
    const bool prevf = __ldg(fl_prev + grp) != 0;
    const bool active = p < C.n && !solid_at(a.mask, gp);
    if (active) {
        const S* src = (const S*)(par ? a.h1 : a.h0);
        S* dst = (S*)(par ? a.h0 : a.h1);
        const long long NT = a.Ntot;
        const int x = (int)(p % C.nx);
        const long long r = p / C.nx;
        const int y = (int)(r % C.ny);
        const int z = (int)(r / C.ny);
        Nbr nb;
        neighbours(C, x, y, z, nb);
        const bool slow = __ldg(a.slow + grp) != 0;

        float h[Q];
        pull_all<S>(src, NT, gp, nb, a.mask, C, y, slow, h);

        float drho, jx, jy, jz;
        moments(h, drho, jx, jy, jz);
        float gx = C.G[0], gy = C.G[1], gz = C.G[2];
        if (forced) {
            const float4 g = (par ? a.g1 : a.g0)[gp];
            gx += g.x; gy += g.y; gz += g.z;
        }
        const float rho = 1.0f + drho;
        const float irho = 1.0f / rho;
        const float ux = (jx + 0.5f * gx) * irho;
        const float uy = (jy + 0.5f * gy) * irho;
        const float uz = (jz + 0.5f * gz) * irho;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float ug = ux * gx + uy * gy + uz * gz;
        const float om = C.omega, fp = C.fpre;
#define LBIBM_COLL(I) Pop<S>::st(dst, (long long)(I) * NT + gp, \
        collide_one<I>(h[I], drho, rho, ux, uy, uz, uu, gx, gy, gz, ug, om, fp), I);
        LBIBM_COLL(0) LBIBM_COLL(1) LBIBM_COLL(2) LBIBM_COLL(3) LBIBM_COLL(4) LBIBM_COLL(5) LBIBM_COLL(6)
        LBIBM_COLL(7) LBIBM_COLL(8) LBIBM_COLL(9) LBIBM_COLL(10) LBIBM_COLL(11) LBIBM_COLL(12)
        LBIBM_COLL(13) LBIBM_COLL(14) LBIBM_COLL(15) LBIBM_COLL(16) LBIBM_COLL(17) LBIBM_COLL(18)
#undef LBIBM_COLL
        if (forced) a.u[gp] = make_float4(ux, uy, uz, rho);
        if (prevf) (par ? a.g0 : a.g1)[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the warp owning this 32-node group clears the previous step's flag after
    // all its lanes have consumed it
    __syncwarp();
    if (prevf && (threadIdx.x & 31) == 0) fl_prev[grp] = 0;
}

cudaError_t launch_stream_collide(const LatticeArgs& a, int total_blocks, cudaStream_t s) {
    if (total_blocks <= 0) return cudaSuccess;
    if (a.storage == 0) k_stream_collide<float><<<total_blocks, K3_BLOCK, 0, s>>>(a);
    else if (a.storage == 1) k_stream_collide<__half><<<total_blocks, K3_BLOCK, 0, s>>>(a);
    else k_stream_collide<__nv_bfloat16><<<total_blocks, K3_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fields: rho and the force-corrected velocity of the last collision, from the
// stored post-collision populations: sum_i e_i f*_i = rho u + g/2.
// ---------------------------------------------------------------------------
template <class S>
__global__ void k_fields(LatticeArgs a, int c, float* rho_out, float* u_out) {
    const ChannelDev C = a.ch[c];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const long long gp = C.base + p;
    if (!a.has_last || solid_at(a.mask, gp)) {
        if (rho_out) rho_out[p] = 1.0f;
        if (u_out) { u_out[p] = 0.f; u_out[C.n + p] = 0.f; u_out[2 * C.n + p] = 0.f; }
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
        u_out[C.n + p] = (jy - 0.5f * gy) / rho;
        u_out[2 * C.n + p] = (jz - 0.5f * gz) / rho;
    }
}

cudaError_t launch_fields(const LatticeArgs& a, const ChannelDev& ch, int c, float* rho, float* u, cudaStream_t s) {
    const int B = 256;
    const long long blocks = (ch.n + B - 1) / B;
    if (a.storage == 0) k_fields<float><<<(unsigned)blocks, B, 0, s>>>(a, c, rho, u);
    else if (a.storage == 1) k_fields<__half><<<(unsigned)blocks, B, 0, s>>>(a, c, rho, u);
    else k_fields<__nv_bfloat16><<<(unsigned)blocks, B, 0, s>>>(a, c, rho, u);
    return cudaGetLastError();
}

// Pre-collision (post-stream) shifted populations of the next step.
template <class S>
__global__ void k_pull_populations(LatticeArgs a, int c, float* h_out) {
    const ChannelDev C = a.ch[c];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const long long gp = C.base + p;
    const S* src = (const S*)(a.par ? a.h1 : a.h0);
    float h[Q];
    if (solid_at(a.mask, gp)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = 0.0f;
    } else {
        const int x = (int)(p % C.nx);
        const long long r = p / C.nx;
        const int y = (int)(r % C.ny);
        const int z = (int)(r / C.ny);
        Nbr nb;
        neighbours(C, x, y, z, nb);
        pull_all<S>(src, a.Ntot, gp, nb, a.mask, C, y, true, h);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) h_out[(long long)i * C.n + p] = h[i];
}

cudaError_t launch_pull_populations(const LatticeArgs& a, const ChannelDev& ch, int c, float* h_out, cudaStream_t s) {
    const int B = 256;
    const long long blocks = (ch.n + B - 1) / B;
    if (a.storage == 0) k_pull_populations<float><<<(unsigned)blocks, B, 0, s>>>(a, c, h_out);
    else if (a.storage == 1) k_pull_populations<__half><<<(unsigned)blocks, B, 0, s>>>(a, c, h_out);
    else k_pull_populations<__nv_bfloat16><<<(unsigned)blocks, B, 0, s>>>(a, c, h_out);
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
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <class S>
__global__ void __launch_bounds__(DIAG_BLOCK) k_diag_partial(LatticeArgs a, int c, double* partials) {
    const ChannelDev C = a.ch[c];
    const S* hs = (const S*)(a.par ? a.h1 : a.h0);
    const uint8_t* fl = a.par ? a.fl0 : a.fl1;
    const float4* gg = a.par ? a.g0 : a.g1;
    double acc[DIAG_N] = {0, 0, 0, 0, 0, 0};
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < C.n;
         p += (long long)gridDim.x * blockDim.x) {
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

cudaError_t launch_diagnostics(const LatticeArgs& a, const ChannelDev& ch, int c, double* partials, int n_blocks,
                               double* out, cudaStream_t s) {
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
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n || !extra[p]) return;
    const long long g = C.base + p;
    atomicOr(mask + (g >> 5), 1u << (g & 31));
}

cudaError_t launch_rasterise(const float* spheres, int n_spheres, const uint8_t* extra, const ChannelDev& ch,
                             const ChannelDev*, int, uint32_t* mask, cudaStream_t s) {
    if (n_spheres > 0) k_rasterise_spheres<<<n_spheres, 256, 0, s>>>((const float4*)spheres, ch, mask);
    if (extra) k_rasterise_extra<<<(unsigned)((ch.n + 255) / 256), 256, 0, s>>>(extra, ch, mask);
    return cudaGetLastError();
}

// A 32-node group is "slow" when one of its nodes is solid or has one of the
// 18 neighbours solid or outside the domain; the stream-collide kernel checks
// the mask and bounds only there.
__global__ void k_slow_flags(ChannelDev C, const uint32_t* mask, uint8_t* slow) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C.n) return;
    const long long gp = C.base + p;
    bool s = solid_at(mask, gp);
    if (!s) {
        const int x = (int)(p % C.nx);
        const long long r = p / C.nx;
        const int y = (int)(r % C.ny);
        const int z = (int)(r / C.ny);
        Nbr nb;
        neighbours(C, x, y, z, nb);
        bool ok;
#define LBIBM_CHK(I) { const long long o = src_off<I>(nb, ok); s = s || !ok || solid_at(mask, gp + (ok ? o : 0)); }
        LBIBM_CHK(1) LBIBM_CHK(2) LBIBM_CHK(3) LBIBM_CHK(4) LBIBM_CHK(5) LBIBM_CHK(6) LBIBM_CHK(7)
        LBIBM_CHK(8) LBIBM_CHK(9) LBIBM_CHK(10) LBIBM_CHK(11) LBIBM_CHK(12) LBIBM_CHK(13) LBIBM_CHK(14)
        LBIBM_CHK(15) LBIBM_CHK(16) LBIBM_CHK(17) LBIBM_CHK(18)
#undef LBIBM_CHK
    }
    if (s) slow[gp >> 5] = 1;
}

cudaError_t launch_slow_flags(const ChannelDev& ch, const ChannelDev*, int, const uint32_t* mask, uint8_t* slow,
                              cudaStream_t s) {
    k_slow_flags<<<(unsigned)((ch.n + 255) / 256), 256, 0, s>>>(ch, mask, slow);
    return cudaGetLastError();
}

}  // namespace lbibm
