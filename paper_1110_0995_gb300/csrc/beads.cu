// Magnetic bead assembly (Sec. 2.5): the dipole-dipole force between beads,
// a harmonic contact force, and overdamped bead motion, all pairs on the GPU.
//
// One thread per bead b accumulates the force of the beads a of its block's
// share of the pairs; the positions and moments of a tile of BEAD_TILE beads
// at a time are staged in shared memory so that each is read from global
// memory once per block.  A second launch moves every bead by
// mobility * F * dt into the other position buffer (every bead sees the
// positions of the same step).
#include "lbibm.h"
#include "lbibm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace lbibm {
lb_status context_free_error(lb_status s, const char* msg);   // lbibm_api.cu

namespace {

constexpr int BEAD_TILE = 256;

struct BeadDev {
    float c3;         // 3 mu0 / (4 pi)
    float two_r;      // contact distance 2R
    float k;          // contact stiffness
    float mob_dt;     // mobility * dt
    float box[3];
    float inv_box[3];
    int per[3];
    int n;
};

__device__ __forceinline__ float3 bead_pair(const float4 xa, const float4 ma, const float4 xb, const float4 mb,
                                            const BeadDev& p) {
    // r = x_b - x_a (force on b from a), minimum image on periodic axes
    float r0 = xb.x - xa.x, r1 = xb.y - xa.y, r2 = xb.z - xa.z;
    if (p.per[0]) r0 -= p.box[0] * rintf(r0 * p.inv_box[0]);
    if (p.per[1]) r1 -= p.box[1] * rintf(r1 * p.inv_box[1]);
    if (p.per[2]) r2 -= p.box[2] * rintf(r2 * p.inv_box[2]);
    const float rr = r0 * r0 + r1 * r1 + r2 * r2;
    const float inv = rsqrtf(rr);
    const float inv2 = inv * inv;
    const float pre = p.c3 * inv2 * inv2 * inv;   // 3c / |r|^5
    const float mar = ma.x * r0 + ma.y * r1 + ma.z * r2;
    const float mbr = mb.x * r0 + mb.y * r1 + mb.z * r2;
    const float mab = ma.x * mb.x + ma.y * mb.y + ma.z * mb.z;
    const float s = mab - 5.0f * mar * mbr * inv2;
    float f0 = pre * (mar * mb.x + mbr * ma.x + s * r0);
    float f1 = pre * (mar * mb.y + mbr * ma.y + s * r1);
    float f2 = pre * (mar * mb.z + mbr * ma.z + s * r2);
    const float d = rr * inv;
    if (d < p.two_r) {
        const float c = p.k * (p.two_r - d) * inv;
        f0 += c * r0;
        f1 += c * r1;
        f2 += c * r2;
    }
    return make_float3(f0, f1, f2);
}

// Partial forces: block (bx, by) sums, for the BEAD_TILE beads of tile bx,
// the forces of the beads in j-tiles [by * jt, (by + 1) * jt) and adds them
// to F (zeroed before the step).  Splitting the j range over blocks keeps
// every SM busy for a few thousand beads.
__global__ void __launch_bounds__(BEAD_TILE) k_bead_forces(const float4* __restrict__ x, const float4* __restrict__ m,
                                                           BeadDev p, int jt, float4* __restrict__ F) {
    __shared__ float4 sx[BEAD_TILE], sm[BEAD_TILE];
    const int b = blockIdx.x * BEAD_TILE + threadIdx.x;
    const bool live = b < p.n;
    const float4 xb = live ? x[b] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 mb = live ? m[b] : make_float4(0.f, 0.f, 0.f, 0.f);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    const int j_end = min(p.n, (int)(blockIdx.y + 1) * jt * BEAD_TILE);
    for (int t0 = blockIdx.y * jt * BEAD_TILE; t0 < j_end; t0 += BEAD_TILE) {
        const int a = t0 + threadIdx.x;
        sx[threadIdx.x] = a < p.n ? x[a] : make_float4(0.f, 0.f, 0.f, 0.f);
        sm[threadIdx.x] = a < p.n ? m[a] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int cnt = min(BEAD_TILE, p.n - t0);
        if (live) {
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                if (t0 + j == b) continue;
                const float3 f = bead_pair(sx[j], sm[j], xb, mb, p);
                f0 += f.x;
                f1 += f.y;
                f2 += f.z;
            }
        }
        __syncthreads();
    }
    if (live) atomicAdd(F + b, make_float4(f0, f1, f2, 0.f));
}

// Overdamped move x_out = x + mobility dt F, wrapped on periodic axes; F is
// cleared for the next step.
__global__ void k_bead_move(const float4* __restrict__ x, float4* __restrict__ F, BeadDev p,
                            float4* __restrict__ x_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.n) return;
    const float4 xb = x[b];
    const float4 f = F[b];
    float v[3] = {xb.x + p.mob_dt * f.x, xb.y + p.mob_dt * f.y, xb.z + p.mob_dt * f.z};
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (p.per[d]) v[d] -= p.box[d] * floorf(v[d] / p.box[d]);
    x_out[b] = make_float4(v[0], v[1], v[2], 0.f);
    F[b] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Grid of the force kernel: (bead tiles, j chunks) with about eight blocks
// per SM over the whole grid.
dim3 force_grid(int n, int& jt) {
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    const int tiles = (n + BEAD_TILE - 1) / BEAD_TILE;
    int split = std::max(1, std::min(tiles, (8 * std::max(sms, 1) + tiles - 1) / tiles));
    jt = (tiles + split - 1) / split;
    split = (tiles + jt - 1) / jt;
    return dim3((unsigned)tiles, (unsigned)split);
}

bool params_ok(const bead_params* p, int n) {
    if (!p || n < 1) return false;
    const double v[5] = {p->mu0_4pi, p->radius, p->k_contact, p->mobility, p->dt};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    if (p->radius < 0 || p->k_contact < 0) return false;
    for (int d = 0; d < 3; ++d)
        if (p->periodic[d] && !(p->box[d] > 0 && std::isfinite(p->box[d]))) return false;
    for (int k = 0; k < 5; ++k)
        if (p->reserved[k]) return false;
    return true;
}

BeadDev dev_params(const bead_params* p, int n) {
    BeadDev d;
    d.c3 = (float)(3.0 * p->mu0_4pi);
    d.two_r = (float)(2.0 * p->radius);
    d.k = (float)p->k_contact;
    d.mob_dt = (float)(p->mobility * p->dt);
    for (int k = 0; k < 3; ++k) {
        d.box[k] = (float)p->box[k];
        d.inv_box[k] = p->periodic[k] ? (float)(1.0 / p->box[k]) : 0.f;
        d.per[k] = p->periodic[k] ? 1 : 0;
    }
    d.n = n;
    return d;
}

// Device buffers of one call: positions (two), moments, forces.
struct BeadBuffers {
    float4* x[2] = {nullptr, nullptr};
    float4* m = nullptr;
    float4* F = nullptr;
    ~BeadBuffers() {
        cudaFree(x[0]);
        cudaFree(x[1]);
        cudaFree(m);
        cudaFree(F);
    }
};

lb_status upload(const double* xyz, const double* moments, int n, BeadBuffers& B, cudaStream_t s) {
    std::vector<float4> hx(n), hm(n);
    for (int i = 0; i < n; ++i) {
        hx[i] = make_float4((float)xyz[3 * i], (float)xyz[3 * i + 1], (float)xyz[3 * i + 2], 0.f);
        hm[i] = make_float4((float)moments[3 * i], (float)moments[3 * i + 1], (float)moments[3 * i + 2], 0.f);
    }
    const size_t bytes = sizeof(float4) * (size_t)n;
    if (cudaMalloc(&B.x[0], bytes) != cudaSuccess || cudaMalloc(&B.x[1], bytes) != cudaSuccess ||
        cudaMalloc(&B.m, bytes) != cudaSuccess || cudaMalloc(&B.F, bytes) != cudaSuccess) {
        cudaGetLastError();
        return context_free_error(LB_ERR_OOM, "bead buffers: device allocation failed");
    }
    if (cudaMemcpyAsync(B.x[0], hx.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B.m, hm.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return context_free_error(LB_ERR_CUDA, "bead upload: CUDA error");
    return LB_OK;
}

lb_status download(const float4* d, int n, double* out, cudaStream_t s) {
    std::vector<float4> h(n);
    if (cudaMemcpyAsync(h.data(), d, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return context_free_error(LB_ERR_CUDA, "bead readback: CUDA error");
    for (int i = 0; i < n; ++i) {
        out[3 * i] = h[i].x;
        out[3 * i + 1] = h[i].y;
        out[3 * i + 2] = h[i].z;
    }
    return LB_OK;
}

}  // namespace
}  // namespace lbibm

using namespace lbibm;

extern "C" {

lb_status bead_forces(const double* xyz, const double* moments, int n, const bead_params* p, double* F,
                      void* cuda_stream) {
    if (!xyz || !moments || !F || !params_ok(p, n))
        return context_free_error(LB_ERR_ARG, "null array, n < 1 or invalid bead parameters");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BeadBuffers B;
    lb_status st = upload(xyz, moments, n, B, s);
    if (st != LB_OK) return st;
    const BeadDev d = dev_params(p, n);
    int jt = 1;
    const dim3 grid = force_grid(n, jt);
    if (cudaMemsetAsync(B.F, 0, sizeof(float4) * (size_t)n, s) != cudaSuccess)
        return context_free_error(LB_ERR_CUDA, "bead forces: CUDA error");
    k_bead_forces<<<grid, BEAD_TILE, 0, s>>>(B.x[0], B.m, d, jt, B.F);
    if (cudaGetLastError() != cudaSuccess) return context_free_error(LB_ERR_CUDA, "bead forces: launch failed");
    return download(B.F, n, F, s);
}

lb_status bead_relax(double* xyz, const double* moments, int n, const bead_params* p, int steps, void* cuda_stream) {
    if (!xyz || !moments || steps < 0 || !params_ok(p, n))
        return context_free_error(LB_ERR_ARG, "null array, n < 1, steps < 0 or invalid bead parameters");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    BeadBuffers B;
    lb_status st = upload(xyz, moments, n, B, s);
    if (st != LB_OK) return st;
    const BeadDev d = dev_params(p, n);
    int jt = 1;
    const dim3 grid = force_grid(n, jt);
    if (cudaMemsetAsync(B.F, 0, sizeof(float4) * (size_t)n, s) != cudaSuccess)
        return context_free_error(LB_ERR_CUDA, "bead relax: CUDA error");
    for (int k = 0; k < steps; ++k) {
        k_bead_forces<<<grid, BEAD_TILE, 0, s>>>(B.x[k & 1], B.m, d, jt, B.F);
        k_bead_move<<<(n + 255) / 256, 256, 0, s>>>(B.x[k & 1], B.F, d, B.x[(k + 1) & 1]);
        if (cudaGetLastError() != cudaSuccess) return context_free_error(LB_ERR_CUDA, "bead relax: launch failed");
    }
    return download(B.x[steps & 1], n, xyz, s);
}

}  // extern "C"
