// noalloc.cu -- residual norm ||b - L x||_2 that allocates no memory at all.
//
// Who needs this: callers that cannot call cudaMalloc (or any allocating library routine) at the
// point where they want the number -- e.g. code running inside a memory pool with a fixed budget,
// a host callback, or a framework hook that must not touch the allocator.  The regular
// stokes_residual_norm needs a handle, and creating a handle allocates the whole multigrid
// hierarchy; this entry point takes the grid parameters directly, reads the caller's device
// vectors in place and keeps its per-block partial sums in a fixed device array that is part of
// the library image.
//
// Scratch: g_noalloc_partials, kNoAllocMaxParts doubles (128 KiB), loaded with the library on every
// GPU that uses it and kept until the process exits.  Its device address is looked up once per
// device (cudaGetSymbolAddress with that device current) by the first call on that device, so the
// first call should not happen during a CUDA stream capture.  Every slot a call reads was written
// by the same call, so nothing has to be cleared between calls; the array keeps the last call's
// partials.  Calls that overlap on the GPU (different streams, or different host threads on one
// device) share the array and race: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "stokes_internal.cuh"
#include "stokesmg.h"

namespace {

constexpr int kNoAllocMaxParts = 16384;  // partial sums, one per thread block
constexpr int kMaxDevices = 64;
constexpr int NBX = 32, NBY = 8, NKZ = 16;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxParts];

std::mutex g_mu;
double *g_ptr[kMaxDevices] = {};  // device address of g_noalloc_partials, per device

// ||b - L x||^2 partials: cell-centric positions (i, j) of 32 x 8 blocks, NKZ planes per thread;
// reads x through the checked stencils, so entries of x off the unknowns may hold anything
__global__ void __launch_bounds__(256) k_noalloc_residual(smg::Lev L, const double *__restrict__ b,
                                                          const double *__restrict__ x, double *__restrict__ parts,
                                                          smg::Coef<double> K) {
    using namespace smg;
    int i = blockIdx.x * NBX + threadIdx.x, j = blockIdx.y * NBY + threadIdx.y;
    double acc = 0.0;
    if (i <= L.nx && j <= L.ny) {
        int k0 = blockIdx.z * NKZ, k1 = k0 + NKZ < L.nz + 1 ? k0 + NKZ : L.nz + 1;
        for (int k = k0; k < k1; ++k)
            for (int c = 0; c < 4; ++c) {
                if (!active(L, c, i, j, k)) continue;
                double v = c < 3 ? face_Lx(x, L, c, i, j, k, K) : cell_Lx(x, L, i, j, k, K);
                double r = b[pidx(L, c, i, j, k)] - v;
                acc += r * r;
            }
    }
    __shared__ double sh[256];
    int t = threadIdx.x + NBX * threadIdx.y;
    sh[t] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) sh[t] += sh[t + w];
        __syncthreads();
    }
    if (t == 0) parts[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = sh[0];
}

// fixed-order sum of the partials, square root into *out (device)
__global__ void __launch_bounds__(256) k_noalloc_finish(const double *__restrict__ parts, int nparts, double *out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) acc += parts[t];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(sh[0]);
}

// p is device (or managed) memory of device dev: memory of another GPU would be read through the
// peer path, or fault where no peer access is enabled
bool device_pointer(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int stokes_residual_norm_noalloc(int nx, int ny, int nz, double h, double viscosity, const double *b,
                                            const double *x, double *out, void *stream) {
    if (nx < 2 || ny < 2 || nz < 2 || !b || !x || !out) return STOKES_ERR_INVALID_ARG;
    if (!(viscosity > 0.0) || !std::isfinite(viscosity) || !std::isfinite(h)) return STOKES_ERR_INVALID_ARG;
    if (nx > 2047 || ny > 2047 || nz > 1023) return STOKES_ERR_INVALID_ARG;
    dim3 grid((nx + 1 + NBX - 1) / NBX, (ny + 1 + NBY - 1) / NBY, (nz + 1 + NKZ - 1) / NKZ);
    long long nparts = (long long)grid.x * grid.y * grid.z;
    if (nparts > kNoAllocMaxParts) return STOKES_ERR_INVALID_ARG;  // grid too large for the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return STOKES_ERR_CUDA;
    }
    // the caller's vectors are read in place, on the current device: staging host data would need an
    // allocation, and memory of another GPU is not this launch's to read
    if (!device_pointer(b, dev) || !device_pointer(x, dev) || !device_pointer(out, dev)) return STOKES_ERR_INVALID_ARG;
    if (stream) {
        int sdev = -1;
        if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return STOKES_ERR_INVALID_ARG;
        }
        if (sdev != dev) return STOKES_ERR_INVALID_ARG;
    }
    double *parts = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            // first call on this device: look up the array's device address with the device current
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return STOKES_ERR_CUDA;
            }
            g_ptr[dev] = (double *)p;
        }
        parts = g_ptr[dev];
    }
    smg::Lev L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    long long nu = (long long)(nx + 1) * ny * nz, nv = (long long)nx * (ny + 1) * nz, nw = (long long)nx * ny * (nz + 1);
    L.off[0] = 0; L.off[1] = nu; L.off[2] = nu + nv; L.off[3] = nu + nv + nw;
    L.n = L.off[3] + (long long)nx * ny * nz;
    L.h = h > 0 ? h : 1.0 / nx;
    L.eta = viscosity;
    L.gamma = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_residual<<<grid, dim3(NBX, NBY, 1), 0, s>>>(L, b, x, parts, smg::coef<double>(L, 0.0));
    k_noalloc_finish<<<1, 256, 0, s>>>(parts, (int)nparts, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STOKES_OK : STOKES_ERR_CUDA;
}
