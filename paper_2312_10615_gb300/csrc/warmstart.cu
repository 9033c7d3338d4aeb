// warmstart.cu -- learned initial guess for MG-SQMR: a four-level, 16-channel 3D convolutional
// network (forward map, reverse-mode gradient, Adam) in hand-written CUDA for sm_103a, and a solve
// that starts the paper's SQMR (Alg. 4) from the network's guess.
//
// Activations are channels-last, one voxel's channels contiguous ([voxel][C], x fastest among the
// voxels), stored FP32 or BF16; every convolution accumulates in FP32.  With BF16 storage the 3x3x3
// convolutions, their data gradients and weight gradients run on the tensor cores (warmstart_tc.cu:
// tcgen05 implicit GEMM with the voxels as M, and mma.sync for the weight gradient).  With FP32
// storage (and where the tensor-core form does not apply) they run on the CUDA cores: the
// convolution keeps its 27 x CI x CO weights in shared memory (read as warp-wide broadcasts) and each
// thread produces two neighbouring voxels; the weight gradient stages a halo tile of the input and a
// tile of the output gradient in shared memory and accumulates per-tap sums in registers across a
// grid-stride loop of tiles.  Per-block partial sums are added in a fixed order (deterministic).  The
// data-gradient of a convolution is the same kernel with the taps mirrored and the channel roles
// exchanged.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "stokes_internal.cuh"
#include "warmstart.h"
#include "warmstart_tc.h"

using smg::launch_k;
using smg::pdl_wait;

namespace {

typedef __nv_bfloat16 bf16;
constexpr int CH = 16;
constexpr float SLOPE = 0.1f;
constexpr int NRED = 592;        // blocks of the vector reductions
constexpr int WG_BLOCKS = 304;   // blocks of the weight-gradient kernels (2 per SM)
constexpr long long W_COUNT = 27LL * 4 * CH + 10LL * 27 * CH * CH + CH * 4;  // 70,912

long long w_off(int l) {  // offset of layer l in the flat weight vector
    if (l == 0) return 0;
    if (l <= 11) return 27LL * 4 * CH + (l - 1) * 27LL * CH * CH;
    return W_COUNT;
}

__host__ __device__ inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---- element access ----
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(bf16 v) { return __bfloat162float(v); }

// C contiguous channels (C % 4 == 0) at p, as floats
template <int C> __device__ __forceinline__ void ldc(const float *p, float *o) {
#pragma unroll
    for (int c = 0; c < C; c += 4) {
        float4 t = *reinterpret_cast<const float4 *>(p + c);
        o[c] = t.x; o[c + 1] = t.y; o[c + 2] = t.z; o[c + 3] = t.w;
    }
}
template <int C> __device__ __forceinline__ void ldc(const bf16 *p, float *o) {
#pragma unroll
    for (int c = 0; c < C; c += 4) {
        uint2 t = *reinterpret_cast<const uint2 *>(p + c);
        float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.y));
        o[c] = a.x; o[c + 1] = a.y; o[c + 2] = b.x; o[c + 3] = b.y;
    }
}
template <int C> __device__ __forceinline__ void stc(float *p, const float *v) {
#pragma unroll
    for (int c = 0; c < C; c += 4) *reinterpret_cast<float4 *>(p + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
}
template <int C> __device__ __forceinline__ void stc(bf16 *p, const float *v) {
#pragma unroll
    for (int c = 0; c < C; c += 4) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[c], v[c + 1]), b = __floats2bfloat162_rn(v[c + 2], v[c + 3]);
        uint2 t;
        t.x = *reinterpret_cast<unsigned *>(&a);
        t.y = *reinterpret_cast<unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p + c) = t;
    }
}
__device__ __forceinline__ float leaky(float z) { return z > 0.f ? z : SLOPE * z; }

// ---- 3x3x3 convolution, zero padding.  Forward: Y[v] = sum_t X[v + off_t] W[t] (W [27][CI][CO]).
// BWD: the data gradient of a layer with CO input and CI output channels, dX[v] = sum_t
// G[v - off_t] W[t]^T, evaluated as a forward convolution with weights W'[t][co][ci] =
// W[26 - t][ci][co] (off_{26-t} = -off_t).  Block 32 x 4 threads, two x-neighbours per thread.
template <int CI, int CO, class TI, class TO, bool BWD, bool ACT>
__global__ void __launch_bounds__(128) k_conv3(int nx, int ny, int nz, const TI *__restrict__ X,
                                              const float *__restrict__ Wt, TO *__restrict__ Y) {
    __shared__ __align__(16) float sw[27 * CI * CO];
    pdl_wait();
    const int tid = threadIdx.x + 32 * threadIdx.y;
    for (int e = tid; e < 27 * CI * CO; e += 128) {
        int t = e / (CI * CO), r = e - t * (CI * CO), ci = r / CO, co = r - ci * CO;
        sw[e] = BWD ? Wt[((26 - t) * CO + co) * CI + ci] : Wt[e];
    }
    __syncthreads();
    const int x0 = 2 * (blockIdx.x * 32 + threadIdx.x), y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x0 >= nx || y >= ny) return;
    float acc[2][CO];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < CO; ++c) acc[q][c] = 0.f;
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int zz = z + dz, yy = y + dy;
        const bool row = zz >= 0 && zz < nz && yy >= 0 && yy < ny;
        float in[2][CI];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int xx = x0 + q + dx;
            if (row && xx >= 0 && xx < nx) {
                ldc<CI>(X + (((long long)zz * ny + yy) * nx + xx) * CI, in[q]);
            } else {
#pragma unroll
                for (int c = 0; c < CI; ++c) in[q][c] = 0.f;
            }
        }
        const float4 *w4 = reinterpret_cast<const float4 *>(sw + t * CI * CO);
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) {
#pragma unroll
            for (int c4 = 0; c4 < CO / 4; ++c4) {
                const float4 w = w4[ci * (CO / 4) + c4];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    acc[q][4 * c4 + 0] = fmaf(in[q][ci], w.x, acc[q][4 * c4 + 0]);
                    acc[q][4 * c4 + 1] = fmaf(in[q][ci], w.y, acc[q][4 * c4 + 1]);
                    acc[q][4 * c4 + 2] = fmaf(in[q][ci], w.z, acc[q][4 * c4 + 2]);
                    acc[q][4 * c4 + 3] = fmaf(in[q][ci], w.w, acc[q][4 * c4 + 3]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (x0 + q >= nx) continue;
        float o[CO];
#pragma unroll
        for (int c = 0; c < CO; ++c) o[c] = ACT ? leaky(acc[q][c]) : acc[q][c];
        stc<CO>(Y + (((long long)z * ny + y) * nx + x0 + q) * CO, o);
    }
}

template <int CI, int CO, class TI, class TO, bool BWD, bool ACT>
void conv3(int n, const TI *X, const float *W, TO *Y, cudaStream_t s) {
    launch_k(k_conv3<CI, CO, TI, TO, BWD, ACT>, dim3(cdiv(n, 64), cdiv(n, 4), n), dim3(32, 4), 0, s, n, n, n, X, W, Y);
}

// ---- weight gradient of a 3x3x3 convolution: dW[t][ci][co] = sum_v X[v + off_t][ci] G[v][co].
// Thread (ci, co pair) owns 2 x 27 sums; tiles of 8 x 8 x 2 voxels (halo 10 x 10 x 4) in shared
// memory; per-block partials [block][27][CI][CO].
template <int CI, int CO, class TI>
__global__ void __launch_bounds__(CI *CO / 2) k_wgrad3(int n, const TI *__restrict__ X, const float *__restrict__ G,
                                                      float *__restrict__ partials) {
    constexpr int NT = CI * CO / 2, TX = 8, TY = 8, TZ = 2, HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
    __shared__ float sx[HZ * HY * HX * CI];
    __shared__ __align__(8) float sg[TZ * TY * TX * CO];
    pdl_wait();
    const int tid = threadIdx.x, ci = tid / (CO / 2), co = 2 * (tid % (CO / 2));
    float a0[27], a1[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) a0[t] = a1[t] = 0.f;
    const int ntx = cdiv(n, TX), nty = cdiv(n, TY), ntz = cdiv(n, TZ);
    const int ntiles = ntx * nty * ntz;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bx = (tile % ntx) * TX, by = ((tile / ntx) % nty) * TY, bz = (tile / (ntx * nty)) * TZ;
        for (int e = tid; e < HZ * HY * HX * CI; e += NT) {
            int h = e / CI, c = e - h * CI;
            int gx = bx + h % HX - 1, gy = by + (h / HX) % HY - 1, gz = bz + h / (HX * HY) - 1;
            bool in = gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n;
            sx[e] = in ? tof(X[(((long long)gz * n + gy) * n + gx) * CI + c]) : 0.f;
        }
        for (int e = tid; e < TZ * TY * TX * CO; e += NT) {
            int v = e / CO, c = e - v * CO;
            int gx = bx + v % TX, gy = by + (v / TX) % TY, gz = bz + v / (TX * TY);
            bool in = gx < n && gy < n && gz < n;
            sg[e] = in ? G[(((long long)gz * n + gy) * n + gx) * CO + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 1
        for (int v = 0; v < TZ * TY * TX; ++v) {
            const int vx = v % TX, vy = (v / TX) % TY, vz = v / (TX * TY);
            const float2 g = *reinterpret_cast<const float2 *>(&sg[v * CO + co]);
            const float *xb = sx + ((vz * HY + vy) * HX + vx) * CI + ci;
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;  // offsets + 1
                const float xv = xb[((dz * HY + dy) * HX + dx) * CI];
                a0[t] = fmaf(xv, g.x, a0[t]);
                a1[t] = fmaf(xv, g.y, a1[t]);
            }
        }
        __syncthreads();
    }
    float *o = partials + (long long)blockIdx.x * 27 * CI * CO;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        o[(t * CI + ci) * CO + co] = a0[t];
        o[(t * CI + ci) * CO + co + 1] = a1[t];
    }
}

// column sums of partials [nb][m] in block order -> out[m]
__global__ void __launch_bounds__(256) k_colsum(const float *__restrict__ partials, int nb, int m, float *__restrict__ out) {
    pdl_wait();
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += partials[(long long)b * m + e];
    out[e] = s;
}

template <int CI, int CO, class TI>
void wgrad3(int n, const TI *X, const float *G, float *partials, float *out, cudaStream_t s) {
    int ntiles = cdiv(n, 8) * cdiv(n, 8) * cdiv(n, 2);
    int nb = ntiles < WG_BLOCKS ? ntiles : WG_BLOCKS;
    launch_k(k_wgrad3<CI, CO, TI>, dim3(nb), dim3(CI * CO / 2), 0, s, n, X, G, partials);
    launch_k(k_colsum, dim3(cdiv(27 * CI * CO, 256)), dim3(256), 0, s, (const float *)partials, nb, 27 * CI * CO, out);
}

// ---- 1x1x1 output layer (16 -> 4) and its gradient (fused with the activation gradient of c0) ----
template <class S>
__global__ void __launch_bounds__(256) k_conv1(long long nvox, const S *__restrict__ C0, const float *__restrict__ W,
                                               float *__restrict__ P) {
    pdl_wait();
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    float c[CH], o[4] = {0.f, 0.f, 0.f, 0.f};
    ldc<CH>(C0 + v * CH, c);
#pragma unroll
    for (int ci = 0; ci < CH; ++ci)
#pragma unroll
        for (int co = 0; co < 4; ++co) o[co] = fmaf(c[ci], W[ci * 4 + co], o[co]);
    stc<4>(P + v * 4, o);
}

template <class S>
__global__ void __launch_bounds__(256) k_conv1_bwd(long long nvox, const S *__restrict__ C0, const float *__restrict__ dP,
                                                   const float *__restrict__ W, float *__restrict__ dZ,
                                                   float *__restrict__ partials) {
    __shared__ float red[8][CH * 4];
    pdl_wait();
    float acc[CH * 4];
#pragma unroll
    for (int e = 0; e < CH * 4; ++e) acc[e] = 0.f;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        float c[CH], d[4], g[CH];
        ldc<CH>(C0 + v * CH, c);
        ldc<4>(dP + v * 4, d);
#pragma unroll
        for (int ci = 0; ci < CH; ++ci) {
            float s = 0.f;
#pragma unroll
            for (int co = 0; co < 4; ++co) {
                s = fmaf(d[co], W[ci * 4 + co], s);
                acc[ci * 4 + co] = fmaf(c[ci], d[co], acc[ci * 4 + co]);
            }
            g[ci] = c[ci] > 0.f ? s : SLOPE * s;
        }
        stc<CH>(dZ + v * CH, g);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < CH * 4; ++e) {
        float x = acc[e];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][e] = x;
    }
    __syncthreads();
    if (threadIdx.x < CH * 4) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        partials[(long long)blockIdx.x * CH * 4 + threadIdx.x] = s;
    }
}

// ---- pooling / upsampling (fine grid n, coarse n/2) ----
template <class S>
__global__ void __launch_bounds__(256) k_pool(int nc, const S *__restrict__ X, S *__restrict__ Y) {
    pdl_wait();
    long long V = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long Nc = (long long)nc * nc * nc;
    if (V >= Nc) return;
    int I = (int)(V % nc), J = (int)((V / nc) % nc), K = (int)(V / ((long long)nc * nc));
    int n = 2 * nc;
    float s[CH], t[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) s[c] = 0.f;
    for (int d = 0; d < 8; ++d) {
        long long v = ((long long)(2 * K + (d >> 2)) * n + 2 * J + ((d >> 1) & 1)) * n + 2 * I + (d & 1);
        ldc<CH>(X + v * CH, t);
#pragma unroll
        for (int c = 0; c < CH; ++c) s[c] += t[c];
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) s[c] *= 0.125f;
    stc<CH>(Y + V * CH, s);
}

// Y[v] = Xc[parent(v)] + skip[v]
template <class S>
__global__ void __launch_bounds__(256) k_up_add(int n, const S *__restrict__ Xc, const S *__restrict__ skip, S *__restrict__ Y) {
    pdl_wait();
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)n * n * n) return;
    int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
    int nc = n / 2;
    long long V = ((long long)(k >> 1) * nc + (j >> 1)) * nc + (i >> 1);
    float a[CH], b[CH];
    ldc<CH>(Xc + V * CH, a);
    ldc<CH>(skip + v * CH, b);
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] += b[c];
    stc<CH>(Y + v * CH, a);
}

// gc[V] = sum of g over the 8 children (adjoint of nearest upsampling)
__global__ void __launch_bounds__(256) k_upT(int nc, const float *__restrict__ g, float *__restrict__ gc) {
    pdl_wait();
    long long V = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (V >= (long long)nc * nc * nc) return;
    int I = (int)(V % nc), J = (int)((V / nc) % nc), K = (int)(V / ((long long)nc * nc));
    int n = 2 * nc;
    float s[CH], t[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) s[c] = 0.f;
    for (int d = 0; d < 8; ++d) {
        long long v = ((long long)(2 * K + (d >> 2)) * n + 2 * J + ((d >> 1) & 1)) * n + 2 * I + (d & 1);
        ldc<CH>(g + v * CH, t);
#pragma unroll
        for (int c = 0; c < CH; ++c) s[c] += t[c];
    }
    stc<CH>(gc + V * CH, s);
}

// g[v] += gc[parent(v)] / 8 (adjoint of mean pooling, accumulated)
__global__ void __launch_bounds__(256) k_add_poolT(int n, float *__restrict__ g, const float *__restrict__ gc) {
    pdl_wait();
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)n * n * n) return;
    int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
    int nc = n / 2;
    long long V = ((long long)(k >> 1) * nc + (j >> 1)) * nc + (i >> 1);
    float a[CH], b[CH];
    ldc<CH>(g + v * CH, a);
    ldc<CH>(gc + V * CH, b);
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = fmaf(0.125f, b[c], a[c]);
    stc<CH>(g + v * CH, a);
}

// g *= act'(.) given the activation's output y (same sign as its input)
template <class S>
__global__ void __launch_bounds__(256) k_act_bwd(long long nvox, float *__restrict__ g, const S *__restrict__ y) {
    pdl_wait();
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    float a[CH], b[CH];
    ldc<CH>(g + v * CH, a);
    ldc<CH>(y + v * CH, b);
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = b[c] > 0.f ? a[c] : SLOPE * a[c];
    stc<CH>(g + v * CH, a);
}

// ---- packed MAC vector <-> cell channels ----
struct Pk {  // offsets of the u, v, w, p blocks of the packed vector of an n^3 box
    long long o1, o2, o3, npk;
};
Pk packed(int n) {
    long long N = n;
    Pk p;
    p.o1 = (N + 1) * N * N;
    p.o2 = p.o1 + N * (N + 1) * N;
    p.o3 = p.o2 + N * N * (N + 1);
    p.npk = p.o3 + N * N * N;
    return p;
}

// X0[cell] = (mean of the two u faces, two v faces, two w faces, p) / rms(b);  sc[0] = sum b^2
template <class S>
__global__ void __launch_bounds__(256) k_in_map(int n, Pk pk, const double *__restrict__ b, const double *__restrict__ sc,
                                                S *__restrict__ X0) {
    pdl_wait();
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)n * n * n) return;
    long long N = n;
    int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / (N * N));
    double inv = 1.0 / sqrt(sc[0] / (double)pk.npk);
    long long u = i + (N + 1) * (j + N * k), vv = pk.o1 + i + N * (j + (N + 1) * k), w = pk.o2 + i + N * (j + N * k);
    float o[4];
    o[0] = (float)(0.5 * (b[u] + b[u + 1]) * inv);
    o[1] = (float)(0.5 * (b[vv] + b[vv + N]) * inv);
    o[2] = (float)(0.5 * (b[w] + b[w + N * N]) * inv);
    o[3] = (float)(b[pk.o3 + v] * inv);
    stc<4>(X0 + v * 4, o);
}

// x0 = scale * rms(b) * faces(P); one thread per packed entry, blockIdx.z = 4 k + component
__global__ void __launch_bounds__(256) k_out_map(int n, Pk pk, const float *__restrict__ P, const double *__restrict__ sc,
                                                 double scale, double *__restrict__ x0) {
    pdl_wait();
    const int c = blockIdx.z & 3, k = blockIdx.z >> 2;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const long long N = n;
    const int ex = n + (c == 0), ey = n + (c == 1), ez = n + (c == 2);
    if (i >= ex || j >= ey || k >= ez) return;
    const double f = scale * sqrt(sc[0] / (double)pk.npk);
    auto cell = [&](int a, int bb, int cc) { return ((long long)cc * N + bb) * N + a; };
    double val;
    long long q;
    if (c == 3) {
        q = pk.o3 + cell(i, j, k);
        val = P[cell(i, j, k) * 4 + 3];
    } else {
        int nn = c == 0 ? i : (c == 1 ? j : k);
        long long base = c == 0 ? 0 : (c == 1 ? pk.o1 : pk.o2);
        q = base + i + (long long)ex * (j + (long long)ey * k);
        if (nn == 0 || nn == n) {
            val = 0.0;
        } else {
            long long lo = cell(i - (c == 0), j - (c == 1), k - (c == 2)), hi = cell(i, j, k);
            val = 0.5 * ((double)P[lo * 4 + c] + (double)P[hi * 4 + c]);
        }
    }
    x0[q] = f * val;
}

// per-block sums of sum (x0 - xs)^2 and sum xs^2 (x0 == NULL: only the second); partials [block][2]
__global__ void __launch_bounds__(256) k_loss_parts(long long m, const double *__restrict__ x0, const double *__restrict__ xs,
                                                    double *__restrict__ partials) {
    __shared__ double sh[2][256];
    pdl_wait();
    double a = 0.0, b = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
        double s = xs[t], d = (x0 ? x0[t] : 0.0) - s;
        a += d * d;
        b += s * s;
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sh[0][0];
        partials[2 * blockIdx.x + 1] = sh[1][0];
    }
}
// sc[k0] = sum of partials[2 b], sc[k0 + 1] = sum of partials[2 b + 1], in block order
__global__ void __launch_bounds__(256) k_finish2(const double *__restrict__ partials, int nb, double *__restrict__ sc, int k0) {
    __shared__ double sh[2][256];
    pdl_wait();
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        a += partials[2 * t];
        b += partials[2 * t + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc[k0] = sh[0][0];
        sc[k0 + 1] = sh[1][0];
    }
}

// dP = scale * rms(b) * faces^T(dx0), dx0 = 2 (a - bsub) / sc[2] (bsub may be NULL); one thread per cell
__global__ void __launch_bounds__(256) k_dP(int n, Pk pk, const double *__restrict__ a, const double *__restrict__ bsub,
                                            const double *__restrict__ sc, double scale, float *__restrict__ dP) {
    pdl_wait();
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)n * n * n) return;
    const long long N = n;
    const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / (N * N));
    const double f = scale * sqrt(sc[0] / (double)pk.npk) * 2.0 / sc[2];
    auto d = [&](long long q) { return a[q] - (bsub ? bsub[q] : 0.0); };
    const long long u = i + (N + 1) * (j + N * k), vv = pk.o1 + i + N * (j + (N + 1) * k), w = pk.o2 + i + N * (j + N * k);
    float o[4];
    o[0] = (float)(f * 0.5 * ((i >= 1 ? d(u) : 0.0) + (i + 1 <= n - 1 ? d(u + 1) : 0.0)));
    o[1] = (float)(f * 0.5 * ((j >= 1 ? d(vv) : 0.0) + (j + 1 <= n - 1 ? d(vv + N) : 0.0)));
    o[2] = (float)(f * 0.5 * ((k >= 1 ? d(w) : 0.0) + (k + 1 <= n - 1 ? d(w + N * N) : 0.0)));
    o[3] = (float)(f * d(pk.o3 + v));
    stc<4>(dP + v * 4, o);
}

// y = a - b elementwise
__global__ void __launch_bounds__(256) k_sub(long long m, const double *__restrict__ a, const double *__restrict__ b,
                                             double *__restrict__ y) {
    pdl_wait();
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x)
        y[t] = a[t] - b[t];
}

// Adam (Kingma & Ba, Algorithm 1); c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
__global__ void __launch_bounds__(256) k_adam(long long m, float *__restrict__ w, const float *__restrict__ g,
                                              float *__restrict__ mo, float *__restrict__ vo, float lr, float b1, float b2,
                                              float eps, float c1, float c2) {
    pdl_wait();
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    float gg = g[e];
    float a = b1 * mo[e] + (1.f - b1) * gg, b = b2 * vo[e] + (1.f - b2) * gg * gg;
    mo[e] = a;
    vo[e] = b;
    w[e] -= lr * (a * c1) / (sqrtf(b * c2) + eps);
}

bool is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return STOKES_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
}

}  // namespace

struct warmstart_s {
    int n = 0, storage = WARMSTART_STORE_FP32, dev = 0;
    int tensor_cores = 1;  // BF16 storage: convolutions on the tensor cores (0: CUDA cores)
    int *tcerr = nullptr;  // set by a tensor-core kernel whose bounded wait ran out
    double scale = 1.0;
    long long N[4] = {0, 0, 0, 0};
    Pk pk;
    // activations (element type by storage)
    void *X0 = nullptr, *a[4] = {}, *s[3] = {}, *p[4] = {}, *u[3] = {}, *c[3] = {}, *b3 = nullptr;
    float *P = nullptr, *dP = nullptr, *gA[4] = {}, *gB[4] = {};
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *wpart = nullptr;
    double *red = nullptr, *sc = nullptr;  // sc[0] = sum b^2; sc[1] / sc[2] = the loss
    double *xp = nullptr, *xd = nullptr, *xr = nullptr;  // packed prediction and residual-form scratch
    int step = 0;
    std::vector<void *> allocs;
    ~warmstart_s() {
        for (void *q : allocs) cudaFree(q);
    }
    int alloc(void **q, size_t bytes) {
        cudaError_t e = cudaMalloc(q, bytes ? bytes : 16);
        if (e != cudaSuccess) return cuda_rc(e);
        allocs.push_back(*q);
        return cuda_rc(cudaMemset(*q, 0, bytes ? bytes : 16));
    }
};

namespace {

const float *Wl(warmstart_s *h, int l) { return h->w + w_off(l); }
float *Gl(warmstart_s *h, int l) { return h->g + w_off(l); }

// forward convolution with activation, 16 output channels: tensor cores for BF16 activations
template <int CI, class S> void conv_fwd(warmstart_s *h, int n, const S *X, const float *W, S *Y, cudaStream_t s) {
    if constexpr (sizeof(S) == 2) {
        if (h->tensor_cores && wstc::conv3_fwd(n, CI, X, W, Y, h->tcerr, s)) return;
    }
    conv3<CI, CH, S, S, false, true>(n, X, W, Y, s);
}
// data gradient of a 16 -> 16 layer (FP32 gradients; BF16 operands on the tensor cores)
template <class S> void conv_bwd(warmstart_s *h, int n, const float *G, const float *W, float *Y, cudaStream_t s) {
    if constexpr (sizeof(S) == 2) {
        if (h->tensor_cores && wstc::conv3_bwd(n, G, W, Y, h->tcerr, s)) return;
    }
    conv3<CH, CH, float, float, true, false>(n, G, W, Y, s);
}
// weight gradient
template <int CI, class S>
void wgrad(warmstart_s *h, int n, const S *X, const float *G, float *partials, float *out, cudaStream_t s) {
    if constexpr (sizeof(S) == 2) {
        if (h->tensor_cores) {
            const int nb = wstc::wgrad3(n, CI, X, G, partials, s);
            if (nb > 0) {
                launch_k(k_colsum, dim3(cdiv(27 * CI * CH, 256)), dim3(256), 0, s, (const float *)partials, nb,
                         27 * CI * CH, out);
                return;
            }
        }
    }
    wgrad3<CI, CH, S>(n, X, G, partials, out, s);
}

template <class S> void forward(warmstart_s *h, const double *b, double *x0, cudaStream_t s) {
    const int n0 = h->n;
    const int nl[4] = {n0, n0 / 2, n0 / 4, n0 / 8};
    // sc[0] = sum b^2 (k_loss_parts with no prediction sums (0 - b)^2 and b^2)
    launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, (const double *)nullptr, b, h->red);
    launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 0);
    S *X0 = (S *)h->X0;
    S *A[4], *Sk[3], *Pl[4], *U[3], *C[3];
    for (int l = 0; l < 4; ++l) { A[l] = (S *)h->a[l]; Pl[l] = (S *)h->p[l]; }
    for (int l = 0; l < 3; ++l) { Sk[l] = (S *)h->s[l]; U[l] = (S *)h->u[l]; C[l] = (S *)h->c[l]; }
    S *B3 = (S *)h->b3;
    launch_k(k_in_map<S>, dim3(cdiv(h->N[0], 256)), dim3(256), 0, s, n0, h->pk, b, (const double *)h->sc, X0);
    conv_fwd<4, S>(h, nl[0], X0, Wl(h, 0), A[0], s);
    conv_fwd<CH, S>(h, nl[0], A[0], Wl(h, 1), Sk[0], s);
    for (int l = 1; l <= 2; ++l) {
        launch_k(k_pool<S>, dim3(cdiv(h->N[l], 256)), dim3(256), 0, s, nl[l], (const S *)Sk[l - 1], Pl[l]);
        conv_fwd<CH, S>(h, nl[l], Pl[l], Wl(h, 2 * l), A[l], s);
        conv_fwd<CH, S>(h, nl[l], A[l], Wl(h, 2 * l + 1), Sk[l], s);
    }
    launch_k(k_pool<S>, dim3(cdiv(h->N[3], 256)), dim3(256), 0, s, nl[3], (const S *)Sk[2], Pl[3]);
    conv_fwd<CH, S>(h, nl[3], Pl[3], Wl(h, 6), A[3], s);
    conv_fwd<CH, S>(h, nl[3], A[3], Wl(h, 7), B3, s);
    const S *below = B3;
    for (int l = 2; l >= 0; --l) {
        launch_k(k_up_add<S>, dim3(cdiv(h->N[l], 256)), dim3(256), 0, s, nl[l], below, (const S *)Sk[l], U[l]);
        conv_fwd<CH, S>(h, nl[l], U[l], Wl(h, 10 - l), C[l], s);
        below = C[l];
    }
    launch_k(k_conv1<S>, dim3(cdiv(h->N[0], 256)), dim3(256), 0, s, h->N[0], (const S *)C[0], Wl(h, 11), h->P);
    launch_k(k_out_map, dim3(cdiv(n0 + 1, 32), cdiv(n0 + 1, 8), 4 * (n0 + 1)), dim3(32, 8), 0, s, n0, h->pk,
             (const float *)h->P, (const double *)h->sc, h->scale, x0);
}

// dx0 of the loss: error form (st == NULL) 2 (x0 - xs) / ||xs||^2; residual form 2 L L (x0 - xs) / ||b||^2
int loss_head(warmstart_s *h, stokes_t st, const double *b, const double *x0, const double *xs, cudaStream_t s) {
    if (!st) {
        launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, x0, xs, h->red);
        launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 1);
        launch_k(k_dP, dim3(cdiv(h->N[0], 256)), dim3(256), 0, s, h->n, h->pk, x0, xs, (const double *)h->sc, h->scale,
                 h->dP);
        return STOKES_OK;
    }
    launch_k(k_sub, dim3(NRED), dim3(256), 0, s, h->pk.npk, x0, xs, h->xd);
    int rc = stokes_apply(st, h->xd, h->xr, s);  // r = L (x0 - x*)
    if (rc != STOKES_OK) return rc;
    // sc[1] = sum r^2 (as the sum of (r - 0)^2), sc[2] = sum b^2
    launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, (const double *)nullptr, (const double *)h->xr, h->red);
    launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 1);
    launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, (const double *)nullptr, b, h->red);
    launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 2);  // sc[2], sc[3] = sum b^2
    rc = stokes_apply(st, h->xr, h->xd, s);  // L r
    if (rc != STOKES_OK) return rc;
    launch_k(k_dP, dim3(cdiv(h->N[0], 256)), dim3(256), 0, s, h->n, h->pk, (const double *)h->xd, (const double *)nullptr,
             (const double *)h->sc, h->scale, h->dP);
    return STOKES_OK;
}

template <class S> void backward(warmstart_s *h, cudaStream_t s) {
    const int n0 = h->n;
    const int nl[4] = {n0, n0 / 2, n0 / 4, n0 / 8};
    S *X0 = (S *)h->X0;
    S *A[4], *Sk[3], *Pl[4], *U[3], *C[3];
    for (int l = 0; l < 4; ++l) { A[l] = (S *)h->a[l]; Pl[l] = (S *)h->p[l]; }
    for (int l = 0; l < 3; ++l) { Sk[l] = (S *)h->s[l]; U[l] = (S *)h->u[l]; C[l] = (S *)h->c[l]; }
    S *B3 = (S *)h->b3;
    float **gA = h->gA, **gB = h->gB;
    auto nb = [&](int l) { return dim3(cdiv(h->N[l], 256)); };
    // output layer (and the activation gradient of c0)
    launch_k(k_conv1_bwd<S>, dim3(NRED), dim3(256), 0, s, h->N[0], (const S *)C[0], (const float *)h->dP, Wl(h, 11),
             gA[0], h->wpart);
    launch_k(k_colsum, dim3(1), dim3(256), 0, s, (const float *)h->wpart, NRED, CH * 4, Gl(h, 11));
    // decoder, levels 0..2: gA[l] holds dz of the c_l convolution
    for (int l = 0; l <= 2; ++l) {
        wgrad<CH, S>(h, nl[l], U[l], gA[l], h->wpart, Gl(h, 10 - l), s);
        conv_bwd<S>(h, nl[l], gA[l], Wl(h, 10 - l), gB[l], s);  // du_l (also d skip_l)
        launch_k(k_upT, nb(l + 1), dim3(256), 0, s, nl[l + 1], (const float *)gB[l], gA[l + 1]);
        launch_k(k_act_bwd<S>, nb(l + 1), dim3(256), 0, s, h->N[l + 1], gA[l + 1], l + 1 <= 2 ? (const S *)C[l + 1] : (const S *)B3);
    }
    // level 3: b3 = act(conv(a3, W7)), a3 = act(conv(p3, W6))
    wgrad<CH, S>(h, nl[3], A[3], gA[3], h->wpart, Gl(h, 7), s);
    conv_bwd<S>(h, nl[3], gA[3], Wl(h, 7), gB[3], s);
    launch_k(k_act_bwd<S>, nb(3), dim3(256), 0, s, h->N[3], gB[3], (const S *)A[3]);
    wgrad<CH, S>(h, nl[3], Pl[3], gB[3], h->wpart, Gl(h, 6), s);
    conv_bwd<S>(h, nl[3], gB[3], Wl(h, 6), gA[3], s);  // d p3
    // encoder, levels 2..0: gB[l] holds du_l; add the pooled gradient to get d s_l
    const float *dpool = gA[3];
    for (int l = 2; l >= 0; --l) {
        launch_k(k_add_poolT, nb(l), dim3(256), 0, s, nl[l], gB[l], dpool);
        launch_k(k_act_bwd<S>, nb(l), dim3(256), 0, s, h->N[l], gB[l], (const S *)Sk[l]);
        wgrad<CH, S>(h, nl[l], A[l], gB[l], h->wpart, Gl(h, 2 * l + 1), s);
        conv_bwd<S>(h, nl[l], gB[l], Wl(h, 2 * l + 1), gA[l], s);
        launch_k(k_act_bwd<S>, nb(l), dim3(256), 0, s, h->N[l], gA[l], (const S *)A[l]);
        if (l > 0) {
            wgrad<CH, S>(h, nl[l], Pl[l], gA[l], h->wpart, Gl(h, 2 * l), s);
            conv_bwd<S>(h, nl[l], gA[l], Wl(h, 2 * l), gB[l], s);  // d p_l
            dpool = gB[l];
        } else {
            wgrad<4, S>(h, nl[0], X0, gA[0], h->wpart, Gl(h, 0), s);
        }
    }
}

// STOKES_ERR_TIMEOUT (and the flag cleared) if a tensor-core kernel's bounded wait ran out since the last
// check; synchronises the stream
int tc_check(warmstart_s *h, cudaStream_t s) {
    int f = 0;
    cudaError_t e = cudaMemcpyAsync(&f, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_rc(e);
    if (!f) return STOKES_OK;
    e = cudaMemsetAsync(h->tcerr, 0, sizeof(int), s);
    return e == cudaSuccess ? STOKES_ERR_TIMEOUT : cuda_rc(e);
}

}  // namespace

extern "C" {

long long warmstart_num_weights(void) { return W_COUNT; }

int warmstart_create(int n, int storage, double scale, warmstart_t *out) {
    if (!out || n < 8 || n > 1016 || n % 8 != 0 || !(scale > 0.0) ||
        (storage != WARMSTART_STORE_FP32 && storage != WARMSTART_STORE_BF16))
        return STOKES_ERR_INVALID_ARG;
    *out = nullptr;
    warmstart_s *h = new (std::nothrow) warmstart_s();
    if (!h) return STOKES_ERR_OOM;
    h->n = n;
    h->storage = storage;
    h->scale = scale;
    cudaGetDevice(&h->dev);
    h->pk = packed(n);
    for (int l = 0; l < 4; ++l) h->N[l] = (long long)(n >> l) * (n >> l) * (n >> l);
    const size_t es = storage == WARMSTART_STORE_BF16 ? 2 : 4;
    int rc = STOKES_OK;
    auto A = [&](void **q, size_t bytes) {
        if (rc == STOKES_OK) rc = h->alloc(q, bytes);
    };
    A(&h->X0, h->N[0] * 4 * es);
    for (int l = 0; l < 4; ++l) {
        A(&h->a[l], h->N[l] * CH * es);
        A((void **)&h->gA[l], h->N[l] * CH * 4);
        A((void **)&h->gB[l], h->N[l] * CH * 4);
        if (l > 0) A(&h->p[l], h->N[l] * CH * es);
    }
    for (int l = 0; l < 3; ++l) {
        A(&h->s[l], h->N[l] * CH * es);
        A(&h->u[l], h->N[l] * CH * es);
        A(&h->c[l], h->N[l] * CH * es);
    }
    A(&h->b3, h->N[3] * CH * es);
    A((void **)&h->P, h->N[0] * 4 * 4);
    A((void **)&h->dP, h->N[0] * 4 * 4);
    A((void **)&h->w, W_COUNT * 4);
    A((void **)&h->g, W_COUNT * 4);
    A((void **)&h->m, W_COUNT * 4);
    A((void **)&h->v, W_COUNT * 4);
    size_t wp = (size_t)WG_BLOCKS * 27 * CH * CH;
    if ((size_t)NRED * CH * 4 > wp) wp = (size_t)NRED * CH * 4;
    A((void **)&h->wpart, wp * 4);
    A((void **)&h->red, NRED * 2 * sizeof(double));
    A((void **)&h->sc, 16 * sizeof(double));
    A((void **)&h->xp, h->pk.npk * sizeof(double));
    A((void **)&h->xd, h->pk.npk * sizeof(double));
    A((void **)&h->xr, h->pk.npk * sizeof(double));
    A((void **)&h->tcerr, sizeof(int));
    // the zero fills above run on the legacy stream: complete them before any caller stream uses the buffers
    if (rc == STOKES_OK) rc = cuda_rc(cudaDeviceSynchronize());
    if (rc != STOKES_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return STOKES_OK;
}

int warmstart_destroy(warmstart_t h) {
    if (!h) return STOKES_ERR_INVALID_ARG;
    delete h;
    return STOKES_OK;
}

int warmstart_set_engine(warmstart_t h, int tensor_cores) {
    if (!h || (tensor_cores != 0 && tensor_cores != 1)) return STOKES_ERR_INVALID_ARG;
    h->tensor_cores = tensor_cores;
    return STOKES_OK;
}

int warmstart_set_scale(warmstart_t h, double scale) {
    if (!h || !(scale > 0.0)) return STOKES_ERR_INVALID_ARG;
    h->scale = scale;
    return STOKES_OK;
}

int warmstart_set_weights(warmstart_t h, const float *w) {
    if (!h || !w) return STOKES_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(h->w, w, W_COUNT * 4, is_device(w) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, W_COUNT * 4);
    if (e == cudaSuccess) e = cudaMemset(h->v, 0, W_COUNT * 4);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // synchronous for the caller's streams too
    h->step = 0;
    return cuda_rc(e);
}

int warmstart_get_weights(warmstart_t h, float *w) {
    if (!h || !w) return STOKES_ERR_INVALID_ARG;
    return cuda_rc(cudaMemcpy(w, h->w, W_COUNT * 4, is_device(w) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
}

int warmstart_predict(warmstart_t h, const double *b, double *x0, void *stream) {
    if (!h || !b || !x0 || !is_device(b) || !is_device(x0)) return STOKES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->storage == WARMSTART_STORE_BF16) forward<bf16>(h, b, x0, s);
    else forward<float>(h, b, x0, s);
    return cuda_rc(cudaGetLastError());
}

int warmstart_loss_grad(warmstart_t h, stokes_t st, const double *b, const double *xstar, double *loss, float *grad,
                        void *stream) {
    if (!h || !b || !xstar || !is_device(b) || !is_device(xstar)) return STOKES_ERR_INVALID_ARG;
    if (st && stokes_vector_length(st, 0) != h->pk.npk) return STOKES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (h->storage == WARMSTART_STORE_BF16) {
        forward<bf16>(h, b, h->xp, s);
        rc = loss_head(h, st, b, h->xp, xstar, s);
        if (rc == STOKES_OK) backward<bf16>(h, s);
    } else {
        forward<float>(h, b, h->xp, s);
        rc = loss_head(h, st, b, h->xp, xstar, s);
        if (rc == STOKES_OK) backward<float>(h, s);
    }
    if (rc != STOKES_OK) return rc;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, h->g, W_COUNT * 4, is_device(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && loss) {
        double sc[3];
        e = cudaMemcpyAsync(sc, h->sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) *loss = sc[2] > 0 ? sc[1] / sc[2] : 0.0;
    } else if (e == cudaSuccess && grad) {
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_rc(e);
    return (loss || grad) ? tc_check(h, s) : STOKES_OK;
}

int warmstart_adam_step(warmstart_t h, double lr, double beta1, double beta2, double eps, void *stream) {
    if (!h || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps >= 0))
        return STOKES_ERR_INVALID_ARG;
    h->step += 1;
    float c1 = (float)(1.0 / (1.0 - std::pow(beta1, h->step))), c2 = (float)(1.0 / (1.0 - std::pow(beta2, h->step)));
    launch_k(k_adam, dim3(cdiv(W_COUNT, 256)), dim3(256), 0, (cudaStream_t)stream, W_COUNT, h->w, (const float *)h->g,
             h->m, h->v, (float)lr, (float)beta1, (float)beta2, (float)eps, c1, c2);
    return cuda_rc(cudaGetLastError());
}

int warmstart_solve(warmstart_t h, stokes_t st, const double *b, double *x, double tol, int max_iter, sqmr_info_t *info,
                    int *used_guess, void *stream) {
    if (!h || !st || !b || !x || !is_device(b) || !is_device(x)) return STOKES_ERR_INVALID_ARG;
    if (stokes_vector_length(st, 0) != h->pk.npk) return STOKES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = warmstart_predict(h, b, x, stream);
    // SQMR decides convergence as always.  A guess is kept only if it lowers both the residual, ||b - L x0|| <
    // ||b|| (the tolerance is relative to ||b||, and a reduction far beyond the V-cycle's own
    // precision cannot be asked of the preconditioned iteration), and SQMR's first quantity
    // tau_0 = ||M (b - L x0)|| (M the V-cycle) below its value for x0 = 0, ||M b||
    if (rc == STOKES_OK) rc = stokes_apply(st, x, h->xr, stream);
    if (rc == STOKES_OK) {
        launch_k(k_sub, dim3(NRED), dim3(256), 0, s, h->pk.npk, b, (const double *)h->xr, h->xd);
        launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, (const double *)nullptr, (const double *)h->xd, h->red);
        launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 8);
        rc = mg_precondition(st, h->xd, h->xr, stream);
    }
    if (rc == STOKES_OK) {
        launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, (const double *)nullptr, (const double *)h->xr, h->red);
        launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 4);
        rc = mg_precondition(st, b, h->xd, stream);
    }
    if (rc != STOKES_OK) return rc;
    launch_k(k_loss_parts, dim3(NRED), dim3(256), 0, s, h->pk.npk, (const double *)nullptr, (const double *)h->xd, h->red);
    launch_k(k_finish2, dim3(1), dim3(256), 0, s, (const double *)h->red, NRED, h->sc, 6);
    double sc[10];
    cudaError_t e = cudaMemcpyAsync(sc, h->sc, 10 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_rc(e);
    rc = tc_check(h, s);
    if (rc != STOKES_OK) return rc;
    // sc[0] = ||b||^2, sc[8] = ||b - L x0||^2, sc[4] = ||M (b - L x0)||^2, sc[6] = ||M b||^2
    const int use = std::isfinite(sc[4]) && std::isfinite(sc[8]) && sc[8] < sc[0] && sc[4] < sc[6];
    if (!use) {
        e = cudaMemsetAsync(x, 0, h->pk.npk * sizeof(double), s);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    if (used_guess) *used_guess = use;
    return sqmr_solve(st, b, x, tol, max_iter, info, stream);
}


int warmstart_conv_check(int n, int ci, int op, int engine, const void *x, const float *g, const float *w, void *out,
                         void *stream) {
    if (n < 1 || n > 1024 || (ci != 4 && ci != 16) || op < 0 || op > 2 || (engine != 0 && engine != 1) || !x || !w ||
        !out || (op == 1 && ci != 16) || (op == 2 && !g) || !is_device(x) || !is_device(w) || !is_device(out) ||
        (g && !is_device(g)))
        return STOKES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = nullptr;
    float *part = nullptr;
    cudaError_t e = cudaMalloc((void **)&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess && op == 2) e = cudaMalloc((void **)&part, (size_t)WG_BLOCKS * 27 * ci * CH * sizeof(float));
    int rc = cuda_rc(e);
    if (rc == STOKES_OK) {
        bool ran = true;
        if (op == 0) {
            const bf16 *X = (const bf16 *)x;
            bf16 *Y = (bf16 *)out;
            if (engine) ran = wstc::conv3_fwd(n, ci, X, w, Y, err, s);
            else if (ci == 4) conv3<4, CH, bf16, bf16, false, true>(n, X, w, Y, s);
            else conv3<CH, CH, bf16, bf16, false, true>(n, X, w, Y, s);
        } else if (op == 1) {
            if (engine) ran = wstc::conv3_bwd(n, (const float *)x, w, (float *)out, err, s);
            else conv3<CH, CH, float, float, true, false>(n, (const float *)x, w, (float *)out, s);
        } else {
            const bf16 *X = (const bf16 *)x;
            if (engine) {
                const int nb = wstc::wgrad3(n, ci, X, g, part, s);
                ran = nb > 0;
                if (ran)
                    launch_k(k_colsum, dim3(cdiv(27 * ci * CH, 256)), dim3(256), 0, s, (const float *)part, nb,
                             27 * ci * CH, (float *)out);
            } else if (ci == 4) {
                wgrad3<4, CH, bf16>(n, X, g, part, (float *)out, s);
            } else {
                wgrad3<CH, CH, bf16>(n, X, g, part, (float *)out, s);
            }
        }
        if (!ran) rc = STOKES_ERR_UNSUPPORTED;
        e = cudaGetLastError();
        if (rc == STOKES_OK && e != cudaSuccess) rc = cuda_rc(e);
        int f = 0;
        e = cudaMemcpyAsync(&f, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (rc == STOKES_OK) rc = e != cudaSuccess ? cuda_rc(e) : (f ? STOKES_ERR_TIMEOUT : STOKES_OK);
    }
    if (err) cudaFree(err);
    if (part) cudaFree(part);
    return rc;
}

int warmstart_mma_check(const void *a, const void *b, float *d, void *stream) {
    if (!a || !b || !d || !is_device(a) || !is_device(b) || !is_device(d)) return STOKES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = nullptr;
    cudaError_t e = cudaMalloc((void **)&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) {
        if (err) cudaFree(err);
        return cuda_rc(e);
    }
    wstc::mma_selftest((const bf16 *)a, (const bf16 *)b, d, err, s);
    int rc = cuda_rc(cudaGetLastError());
    int f = 0;
    e = cudaMemcpyAsync(&f, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (rc == STOKES_OK) rc = e != cudaSuccess ? cuda_rc(e) : (f ? STOKES_ERR_TIMEOUT : STOKES_OK);
    cudaFree(err);
    return rc;
}

}  // extern "C"
