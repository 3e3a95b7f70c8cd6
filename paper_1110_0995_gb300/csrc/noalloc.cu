// Area and volume of closed triangle meshes without any device allocation.
//
// Some callers cannot allocate device memory: code that runs under a
// framework which owns the whole device memory pool (a cudaMalloc there fails
// or fragments the pool), code in a latency-critical loop where cudaMalloc's
// implicit synchronisation is not acceptable, and embedded callers with a
// fixed memory budget.  This file gives them a variant of the library's
// per-cell area / volume reduction whose scratch space (the per-block partial
// sums) lives in a fixed, file-scope device array instead of memory the
// library allocates.  Inputs and outputs are still the caller's buffers.
//
// The scratch array exists once per device that loads the library and stays
// there until the process exits.  Every call shares it and it keeps the last
// call's contents; each call writes every partial it later reads, so nothing
// has to start at zero.  Two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on the array.
//
// The array's device address belongs to the CUDA context that loaded the
// module.  It is looked up on a device's first call and again whenever the
// context current on that device changes (a cudaDeviceReset, or a driver
// context the caller made current), keyed by the context's unique id.
#include "lbibm.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

namespace {

constexpr int NA_BLOCK = 256;                 // triangles per block (chunk)
constexpr int NA_MAX_PARTIALS = 65536;        // 65,536 x 16 B = 1 MiB of scratch
constexpr int NA_MAX_DEVICES = 64;

// Per-block partial sums (area, volume) of the reduction, indexed
// cell * max_chunks + chunk.  Host code must not pass this symbol to a kernel:
// on the host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) double2 g_noalloc_partials[NA_MAX_PARTIALS];

std::mutex g_setup_mutex;
void* g_scratch_ptr[NA_MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[NA_MAX_DEVICES] = {};

// Unique id of the context current on the calling thread (driver entry points
// through the runtime, so the library needs no link against libcuda).
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e != cudaSuccess || qa != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess || qb != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
        get_current = (ctx_get_current_fn)a;
        get_id = (ctx_get_id_fn)b;
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return cudaErrorDeviceUninitialized;
    if (get_id(c, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of the scratch array in the current context, looked up
// (under a lock) on the first call on a device and whenever that device's
// current context has changed since the last lookup.
cudaError_t scratch_address(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id) == cudaSuccess;   // false: no context current yet
    if (!have_id || !g_scratch_ptr[dev] || g_scratch_ctx[dev] != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);   // makes the primary context current if none is
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = id;
    }
    *out = (double2*)g_scratch_ptr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1: block (chunk, cell) sums area and 6 x volume of up to NA_BLOCK
// triangles of one cell in FP64 and writes one partial.
__global__ void __launch_bounds__(NA_BLOCK) k_area_volume_partials(const double* __restrict__ xyz,
                                                                  const int* __restrict__ tris,
                                                                  const int* __restrict__ cell_start,
                                                                  int max_chunks, double2* partials) {
    const int c = blockIdx.y;
    const int k = blockIdx.x;
    const int t0 = cell_start[c], t1 = cell_start[c + 1];
    const int t = t0 + k * NA_BLOCK + threadIdx.x;
    if (t0 + k * NA_BLOCK >= t1) return;   // the whole block is past this cell's triangles
    double s = 0.0, v = 0.0;
    if (t < t1) {
        const int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
        const double ax = xyz[3 * ia], ay = xyz[3 * ia + 1], az = xyz[3 * ia + 2];
        const double bx = xyz[3 * ib], by = xyz[3 * ib + 1], bz = xyz[3 * ib + 2];
        const double cx = xyz[3 * ic], cy = xyz[3 * ic + 1], cz = xyz[3 * ic + 2];
        const double ux = bx - ax, uy = by - ay, uz = bz - az;
        const double wx = cx - ax, wy = cy - ay, wz = cz - az;
        const double nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
        s = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
        v = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
    }
    __shared__ double sh[2][NA_BLOCK / 32];
    s = warp_sum(s);
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s;
        sh[1][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, V = 0.0;
        for (int w = 0; w < NA_BLOCK / 32; ++w) {
            S += sh[0][w];
            V += sh[1][w];
        }
        partials[(long long)c * max_chunks + k] = make_double2(S, V / 6.0);
    }
}

// Pass 2: one warp per cell adds the cell's partials in a fixed order.  The
// chunk count comes from the device offsets and is clamped to the row stride
// the host derived from its copy, so offsets that disagree with the host copy
// give a wrong sum but never a read outside the cell's row of partials.
__global__ void k_area_volume_final(const int* __restrict__ cell_start, int n_cells, int max_chunks,
                                    const double2* partials, double* area, double* volume) {
    const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_cells) return;
    const int nt = cell_start[c + 1] - cell_start[c];
    int nk = (nt + NA_BLOCK - 1) / NA_BLOCK;
    nk = nk < 0 ? 0 : (nk > max_chunks ? max_chunks : nk);
    double S = 0.0, V = 0.0;
    for (int k = lane; k < nk; k += 32) {
        const double2 p = partials[(long long)c * max_chunks + k];
        S += p.x;
        V += p.y;
    }
    S = warp_sum(S);
    V = warp_sum(V);
    if (lane == 0) {
        area[c] = S;
        volume[c] = V;
    }
}

}  // namespace

extern "C" lb_status ibm_area_volume_noalloc(const double* xyz, const int32_t* tris, const int32_t* cell_tri_start,
                                             const int32_t* cell_tri_start_host, int n_cells, double* area,
                                             double* volume, void* cuda_stream) {
    if (n_cells < 0 || (n_cells > 0 && (!xyz || !tris || !cell_tri_start || !cell_tri_start_host || !area || !volume)))
        return LB_ERR_ARG;
    if (n_cells == 0) return LB_OK;
    if (n_cells > 65535) return LB_ERR_ARG;                    // grid y limit
    int max_chunks = 0;
    for (int c = 0; c < n_cells; ++c) {
        const int nt = cell_tri_start_host[c + 1] - cell_tri_start_host[c];
        if (nt < 0 || cell_tri_start_host[c] < 0) return LB_ERR_ARG;
        const int nk = (nt + NA_BLOCK - 1) / NA_BLOCK;
        if (nk > max_chunks) max_chunks = nk;
    }
    if (max_chunks == 0) max_chunks = 1;
    // the scratch holds one partial per (cell, chunk of 256 triangles)
    if ((long long)n_cells * max_chunks > NA_MAX_PARTIALS) return LB_ERR_ARG;
    double2* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LB_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // each launch's own status (cudaLaunchKernel returns it; an error left over
    // from an unrelated earlier call is neither consumed nor reported here)
    const double* a_xyz = xyz;
    const int* a_tris = tris;
    const int* a_start = cell_tri_start;
    void* args1[] = {(void*)&a_xyz, (void*)&a_tris, (void*)&a_start, (void*)&max_chunks, (void*)&scratch};
    if (cudaLaunchKernel((const void*)k_area_volume_partials, dim3(max_chunks, n_cells), dim3(NA_BLOCK), args1, 0,
                         s) != cudaSuccess)
        return LB_ERR_CUDA;
    const double2* a_scr = scratch;
    void* args2[] = {(void*)&a_start, (void*)&n_cells, (void*)&max_chunks, (void*)&a_scr, (void*)&area,
                     (void*)&volume};
    if (cudaLaunchKernel((const void*)k_area_volume_final, dim3((n_cells + 7) / 8), dim3(256), args2, 0, s) !=
        cudaSuccess)
        return LB_ERR_CUDA;
    return LB_OK;
}
