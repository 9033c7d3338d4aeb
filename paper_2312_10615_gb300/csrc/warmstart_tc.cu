// warmstart_tc.cu -- tensor-core kernels of the initial-guess network.
//
// 3x3x3 convolution (16 output channels) as an implicit GEMM on tcgen05.  A CTA stages a slab of the
// input -- tz z-planes x ty y-rows x every x, plus a one-voxel halo -- in shared memory as two
// channel halves, [half][z][y][x][8 channels] BF16, so that the 8 channels of a voxel are one 16-byte
// row and 8 consecutive voxels one 128-byte core matrix (the no-swizzle K-major operand layout).  Every
// voxel of the slab is a position p in that padded array, and tap (dx, dy, dz) of the output at p reads
// position p + dx + W dy + W Ys dz: a constant shift.  So the A operand of one MMA (M = 128 consecutive
// positions, K = the 16 input channels) for one tap is the staged array itself, addressed from a shifted
// start, and an output tile takes 27 MMAs (128 x 16 x 16, one per tap) accumulated in a 16-column FP32
// tensor-memory tile.  Positions on the halo produce values that are thrown away.  B (the tap's 16 x 16
// weights, [tap][k half][co][8 ci]) sits in shared memory for the whole kernel.  One thread issues the
// MMAs and commits them to an mbarrier; the four warps read the accumulators back with tcgen05.ld (warp
// w owns tensor-memory lanes 32w..32w+31, i.e. tile positions 32w + lane), apply the activation and
// store channels-last rows.  BF16 inputs are staged by two TMA tile loads per slab (4D tensor map over
// [z][y][x][c], box 8 x W x Ys x Zs starting at (-1, -1, -1): the zero padding is TMA's out-of-bounds
// fill); FP32 inputs (the data gradient) are converted while staged with plain loads.  The CTA is
// persistent over slabs; every wait is bounded and a wait that runs out sets the error flag.
//
// Weight gradient on mma.sync m16n8k16 (M = the 16 input channels is below tcgen05's smallest M):
// per tile of 16 x 8 x 4 voxels the CTA stages the X halo and G as BF16 channel halves; warp w
// accumulates taps w, w + 4, ... as 16 x 16 FP32 fragments over the tile's 16-voxel x-rows (ldmatrix.trans
// gives both operands from voxel-major rows); per-block partials are written in a fixed order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "stokes_internal.cuh"
#include "warmstart_tc.h"

using smg::launch_k;
using smg::pdl_wait;

namespace wstc {
namespace {

constexpr float SLOPE = 0.1f;
constexpr int kThreads = 128;
constexpr int kMaxTiles = 8;            // accumulator tiles per slab (16 columns each)
constexpr uint32_t kTmemCols = 128;     // tensor-memory columns a CTA allocates
constexpr uint32_t kWBytes = 27 * 512;  // B operands: 27 taps x 16 x 16 BF16
constexpr uint32_t kWRegion = 14336;    // kWBytes rounded up to 1 KB
static_assert(kWBytes <= kWRegion, "B operand region");
constexpr unsigned kSpinLimit = 1u << 22;
constexpr int kMaxSmem = 110 * 1024;    // two CTAs per SM
// at least this much dynamic shared memory per CTA, so that at most three CTAs (3 x 128 of the SM's 512
// tensor-memory columns) are resident on an SM and tcgen05.alloc never waits
constexpr int kMinSmem = 60 * 1024;

// ---- PTX wrappers ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (unsigned i = 0; i < kSpinLimit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// warp-wide
__device__ __forceinline__ void tmem_alloc(uint32_t holder, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
// D[tmem] (+)= A B^T, kind::f16 (BF16 operands, FP32 accumulator)
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive on the mbarrier once every MMA this thread issued has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of this thread's tensor-memory lane (warp-wide)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"((unsigned long long)(uintptr_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// asynchronous global -> shared copies of 16 or 8 bytes; an invalid source copies zeros (no bytes read)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// shared-memory matrix descriptor, no swizzle: 16-byte rows, 8-row core matrices of 128 contiguous bytes;
// lbo = byte distance between core matrices adjacent along K, sbo = along M (or N)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ float leaky(float z) { return z > 0.f ? z : SLOPE * z; }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&t);
}

// ---- convolution geometry (host-chosen) ----
struct Geom {
    int n, ty, tz, R, W, Ys, Zs, tpg, gpp, tiles, nsy, nslab, half_pos;
    uint32_t half_bytes, smem;
};

__host__ __device__ inline int tile_start(const Geom &g, int i) {
    const int grp = i / g.tpg, j = i - grp * g.tpg;
    const int zs = 1 + grp / g.gpp, ys = 1 + (grp % g.gpp) * g.R;
    return (zs * g.Ys + ys) * g.W + 1 + 128 * j;
}

// one slab's staging, the 27 x tiles MMAs and the epilogue; TI = input element type
template <class TI, class TO, int CI, bool BWD, bool ACT, bool TMA>
__global__ void __launch_bounds__(kThreads) k_conv3_tc(const __grid_constant__ CUtensorMap map, const Geom g,
                                                       const TI *__restrict__ X, const float *__restrict__ Wt,
                                                       TO *__restrict__ Y, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    pdl_wait();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(smem_raw), base = (raw + 1023u) & ~1023u;
    uint8_t *const sp = smem_raw + (base - raw);
    const uint32_t sW = base, sH0 = base + kWRegion, sH1 = sH0 + g.half_bytes;
    const uint32_t bar_tma = smem_u32(&s_bar[0]), bar_mma = smem_u32(&s_bar[1]);
    const int plane = g.Ys * g.W, staged = g.Zs * plane;

    // weights -> B operands [tap][k half][co][8 ci] (BF16); forward B[co][ci] = W[t][ci][co], data
    // gradient B[co][ci] = W[26 - t][co][ci]
    for (int e = tid; e < 27 * 256; e += kThreads) {
        const int t = e >> 8, nn = (e >> 4) & 15, k = e & 15;
        float v = 0.f;
        if (k < CI) v = BWD ? Wt[((26 - t) * 16 + nn) * 16 + k] : Wt[(t * CI + k) * 16 + nn];
        *reinterpret_cast<bf16 *>(sp + t * 512 + (k >> 3) * 256 + nn * 16 + (k & 7) * 2) = __float2bfloat16_rn(v);
    }
    // the positions past the staged slab (read only by discarded tile rows) are zero; so is all of half 1
    // for a 4-channel input (channels 8..15 do not exist)
    for (int p = (CI < 16 ? 0 : staged) + tid; p < g.half_pos; p += kThreads)
        *reinterpret_cast<uint4 *>(sp + kWRegion + (size_t)p * 16) = make_uint4(0, 0, 0, 0);
    for (int p = (CI < 16 ? 0 : staged) + tid; p < g.half_pos; p += kThreads)
        *reinterpret_cast<uint4 *>(sp + kWRegion + g.half_bytes + (size_t)p * 16) = make_uint4(0, 0, 0, 0);
    fence_async_smem();
    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    int shift[27];  // staged-position offset of tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1)
#pragma unroll
    for (int t = 0; t < 27; ++t) shift[t] = (t % 3 - 1) + ((t / 3) % 3 - 1) * g.W + (t / 9 - 1) * plane;
    uint32_t ph_tma = 0, ph_mma = 0;
    int bad = 0;
    for (int slab = blockIdx.x; slab < g.nslab; slab += gridDim.x) {
        const int y0 = (slab % g.nsy) * g.ty, z0 = (slab / g.nsy) * g.tz;
        if (TMA) {
            if (tid == 0) {
                mbar_expect_tx(bar_tma, 2u * (uint32_t)staged * 16u);
                tma_load_4d(sH0, &map, 0, -1, y0 - 1, z0 - 1, bar_tma);
                tma_load_4d(sH1, &map, 8, -1, y0 - 1, z0 - 1, bar_tma);
            }
            const bool ok = mbar_wait(bar_tma, ph_tma);
            ph_tma ^= 1;
            if (__syncthreads_or(!ok)) {
                bad = 1;
                break;
            }
        } else {
            // one warp per staged row (z, y), lanes along x.  BF16 inputs: asynchronous copies, all in flight
            // at once (a 4-channel input copies 8 bytes into half 0, whose upper 8 bytes and all of half 1
            // hold the zeros written at the start); FP32 inputs: four voxels' loads batched per lane, rounded
            // to BF16 on the way
            for (int r = warp; r < g.Zs * g.Ys; r += kThreads / 32) {
                const int zs = r / g.Ys, ys = r - zs * g.Ys;
                const int gz = z0 + zs - 1, gy = y0 + ys - 1;
                const bool row = gz >= 0 && gz < g.n && gy >= 0 && gy < g.n;
                const long long rbase = row ? ((long long)gz * g.n + gy) * g.n : 0;
                const uint32_t d0 = sH0 + (uint32_t)(r * g.W) * 16u;
                if constexpr (sizeof(TI) == 2) {
                    for (int xs = lane; xs < g.W; xs += 32) {
                        const int gx = xs - 1;
                        const bool in = row && gx >= 0 && gx < g.n;
                        const TI *src = X + (in ? (rbase + gx) * CI : 0);
                        if constexpr (CI == 16) {
                            cp_async16(d0 + (uint32_t)xs * 16u, src, in);
                            cp_async16(d0 + g.half_bytes + (uint32_t)xs * 16u, src + 8, in);
                        } else {
                            cp_async8(d0 + (uint32_t)xs * 16u, src, in);
                        }
                    }
                } else {
                    for (int x0 = lane; x0 < g.W; x0 += 128) {
                        float4 q[4][4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int xs = x0 + 32 * u, gx = xs - 1;
                            const bool in = xs < g.W && row && gx >= 0 && gx < g.n;
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                q[u][c] = in ? reinterpret_cast<const float4 *>(X + (rbase + gx) * 16)[c]
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int xs = x0 + 32 * u;
                            if (xs >= g.W) break;
                            uint8_t *dst = sp + kWRegion + (size_t)(r * g.W + xs) * 16;
                            *reinterpret_cast<uint4 *>(dst) =
                                make_uint4(pack2(q[u][0].x, q[u][0].y), pack2(q[u][0].z, q[u][0].w),
                                           pack2(q[u][1].x, q[u][1].y), pack2(q[u][1].z, q[u][1].w));
                            *reinterpret_cast<uint4 *>(dst + g.half_bytes) =
                                make_uint4(pack2(q[u][2].x, q[u][2].y), pack2(q[u][2].z, q[u][2].w),
                                           pack2(q[u][3].x, q[u][3].y), pack2(q[u][3].z, q[u][3].w));
                        }
                    }
                }
            }
            if constexpr (sizeof(TI) == 2) cp_async_wait_all();
            fence_async_smem();
            __syncthreads();
        }
        tc_fence_after();
        if (tid == 0) {
            // descriptors of a tile's first tap; tap t adds its position shift to the A start field (16-byte
            // units, the staged array lies below 256 KB so the field neither under- nor overflows) and t x 512
            // bytes to B's
            const uint64_t b0 = sdesc(sW, 256, 128);
            for (int i = 0; i < g.tiles; ++i) {
                const uint64_t a0 = sdesc(sH0 + (uint32_t)tile_start(g, i) * 16u, sH1 - sH0, 128);
                const uint32_t d = tmem + (uint32_t)i * 16u;
#pragma unroll
                for (int t = 0; t < 27; ++t)
                    mma_bf16(d, a0 + (uint64_t)(int64_t)shift[t], b0 + (uint64_t)(t * 32), kIdesc, t > 0);
            }
            mma_commit(bar_mma);
        }
        const bool ok = mbar_wait(bar_mma, ph_mma);
        ph_mma ^= 1;
        if (__syncthreads_or(!ok)) {
            bad = 2;
            break;
        }
        tc_fence_after();
        for (int i = 0; i < g.tiles; ++i) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)i * 16u, v);
            const int grp = i / g.tpg, gzs = 1 + grp / g.gpp, gys = 1 + (grp % g.gpp) * g.R;
            const int p = tile_start(g, i) + warp * 32 + lane;
            const int zs = p / plane, r = p - zs * plane, ys = r / g.W, xs = r - ys * g.W;
            const int gz = z0 + zs - 1, gy = y0 + ys - 1, gx = xs - 1;
            if (zs != gzs || ys < gys || ys >= gys + g.R || gx < 0 || gx >= g.n || gy >= g.n || gz >= g.n) continue;
            const long long vox = ((long long)gz * g.n + gy) * g.n + gx;
            if (ACT) {
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = leaky(v[c]);
            }
            if constexpr (sizeof(TO) == 2) {
                uint4 *o = reinterpret_cast<uint4 *>(Y + vox * 16);
                o[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                o[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]), pack2(v[14], v[15]));
            } else {
                float4 *o = reinterpret_cast<float4 *>(Y + vox * 16);
#pragma unroll
                for (int c = 0; c < 4; ++c) o[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (bad) {
        // a wait ran out: record it, give the operation in flight a second bounded wait, then release
        if (tid == 0) atomicExch(err, 1);
        if (bad == 1) (void)mbar_wait(bar_tma, ph_tma ^ 1);
        else (void)mbar_wait(bar_mma, ph_mma ^ 1);
        tc_fence_before();
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// D = A B^T for one 128 x 16 x 16 tile: the smallest use of the operand layouts and descriptors above
__global__ void __launch_bounds__(kThreads) k_mma_selftest(const bf16 *__restrict__ A, const bf16 *__restrict__ B,
                                                           float *__restrict__ D, int *__restrict__ err) {
    // A [k half][128][8] at 0 (4 KB), B [k half][16][8] at 36 KB; the buffer is large enough that the
    // operands stay inside it under either reading of the two descriptor offsets
    __shared__ __align__(1024) uint8_t sm[40 * 1024];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    pdl_wait();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < (int)sizeof(sm) / 16; e += kThreads) reinterpret_cast<uint4 *>(sm)[e] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int e = tid; e < 128 * 16; e += kThreads) {
        const int m = e >> 4, k = e & 15;
        *reinterpret_cast<bf16 *>(sm + (k >> 3) * 2048 + m * 16 + (k & 7) * 2) = A[e];
    }
    for (int e = tid; e < 16 * 16; e += kThreads) {
        const int nn = e >> 4, k = e & 15;
        *reinterpret_cast<bf16 *>(sm + 36 * 1024 + (k >> 3) * 256 + nn * 16 + (k & 7) * 2) = B[e];
    }
    fence_async_smem();
    const uint32_t bar = smem_u32(&s_bar);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(smem_u32(&s_tmem), 32);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem, s0 = smem_u32(sm);
    if (tid == 0) {
        mma_bf16(tmem, sdesc(s0, 2048, 128), sdesc(s0 + 36 * 1024, 256, 128), kIdesc, 0);
        mma_commit(bar);
    }
    const bool ok = mbar_wait(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(err, 1);
        (void)mbar_wait(bar, 0);
    } else {
        tc_fence_after();
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
        for (int c = 0; c < 16; ++c) D[(warp * 32 + lane) * 16 + c] = v[c];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 32);
    }
}

// ---- weight gradient on mma.sync ----
constexpr int WX = 16, WY = 8, WZ = 4, WHX = WX + 2, WHY = WY + 2, WHZ = WZ + 2;
constexpr int WXH = WHZ * WHY * WHX;  // staged X positions per half
constexpr int WGV = WZ * WY * WX;     // G voxels per half
constexpr int kWgBlocks = 304;

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t *r) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void mma16816(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, "
        "%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int CI>
__global__ void __launch_bounds__(kThreads) k_wgrad3_mma(int n, const bf16 *__restrict__ X, const float *__restrict__ G,
                                                         float *__restrict__ partials) {
    __shared__ __align__(128) uint8_t sx[2 * WXH * 16];
    __shared__ __align__(128) uint8_t sg[2 * WGV * 16];
    pdl_wait();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NT = 7;  // taps per warp: warp w owns taps w + 4 j (j < 7, t < 27)
    float acc[NT][2][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[j][b][c] = 0.f;
    const int ntx = (n + WX - 1) / WX, nty = (n + WY - 1) / WY, ntz = (n + WZ - 1) / WZ;
    const int ntiles = ntx * nty * ntz;
    const uint32_t sx0 = smem_u32(sx), sg0 = smem_u32(sg);
    if (CI < 16) {  // channels 4..15 of every staged voxel stay 0 (the copies write 8 bytes of half 0)
        for (int e = tid; e < 2 * WXH; e += kThreads) reinterpret_cast<uint4 *>(sx)[e] = make_uint4(0, 0, 0, 0);
        __syncthreads();
    }
    // ldmatrix row owned by this lane: A (X, shifted) matrices (vox 0-7, h0) (0-7, h1) (8-15, h0) (8-15, h1);
    // B (G) matrices (vox 0-7, h0) (8-15, h0) (0-7, h1) (8-15, h1)
    const int a_vox = (lane & 7) + ((lane >> 4) << 3), a_h = (lane >> 3) & 1;
    const int b_vox = (lane & 7) + (((lane >> 3) & 1) << 3), b_h = lane >> 4;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bx = (tile % ntx) * WX, by = ((tile / ntx) % nty) * WY, bz = (tile / (ntx * nty)) * WZ;
        // X halo by asynchronous copies (a 4-channel input: 8 bytes into half 0 of pre-zeroed slots)
        for (int e = tid; e < (CI == 16 ? 2 : 1) * WXH; e += kThreads) {
            const int h = CI == 16 ? (e & 1) : 0, p = CI == 16 ? (e >> 1) : e;
            const int xs = p % WHX, ys = (p / WHX) % WHY, zs = p / (WHX * WHY);
            const int gx = bx + xs - 1, gy = by + ys - 1, gz = bz + zs - 1;
            const bool in = gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n;
            const bf16 *src = X + (in ? (((long long)gz * n + gy) * n + gx) * CI + h * 8 : 0);
            const uint32_t dst = sx0 + (uint32_t)(h * WXH + p) * 16u;
            if constexpr (CI == 16) cp_async16(dst, src, in);
            else cp_async8(dst, src, in);
        }
        // G rounded to BF16, four 16-byte halves per thread loaded before any is stored
        for (int e0 = tid; e0 < 2 * WGV; e0 += 4 * kThreads) {
            float4 q[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * kThreads, h = e & 1, p = e >> 1;
                const int xs = p % WX, ys = (p / WX) % WY, zs = p / (WX * WY);
                const int gx = bx + xs, gy = by + ys, gz = bz + zs;
                const bool in = e < 2 * WGV && gx < n && gy < n && gz < n;
                const float4 *src =
                    reinterpret_cast<const float4 *>(G + (in ? (((long long)gz * n + gy) * n + gx) * 16 + h * 8 : 0));
                q[u][0] = in ? src[0] : make_float4(0.f, 0.f, 0.f, 0.f);
                q[u][1] = in ? src[1] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * kThreads, h = e & 1, p = e >> 1;
                if (e >= 2 * WGV) break;
                *reinterpret_cast<uint4 *>(sg + (size_t)h * WGV * 16 + (size_t)p * 16) =
                    make_uint4(pack2(q[u][0].x, q[u][0].y), pack2(q[u][0].z, q[u][0].w), pack2(q[u][1].x, q[u][1].y),
                               pack2(q[u][1].z, q[u][1].w));
            }
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll 1
        for (int row = 0; row < WY * WZ; ++row) {
            const int ry = row % WY, rz = row / WY;
            uint32_t bq[4];
            ldsm_x4_t(sg0 + (uint32_t)(b_h * WGV + row * WX + b_vox) * 16u, bq);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int t = warp + 4 * j;
                if (t < 27) {
                    const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;  // offsets + 1
                    const int p = ((rz + dz) * WHY + ry + dy) * WHX + a_vox + dx;
                    uint32_t aq[4];
                    ldsm_x4_t(sx0 + (uint32_t)(a_h * WXH + p) * 16u, aq);
                    mma16816(acc[j][0], aq, bq[0], bq[1]);
                    mma16816(acc[j][1], aq, bq[2], bq[3]);
                }
            }
        }
        __syncthreads();
    }
    // fragment (ci = g or g + 8, co = nb * 8 + 2 q + {0, 1}) -> partials[block][t][ci][co]
    float *o = partials + (long long)blockIdx.x * 27 * CI * 16;
    const int gq = lane >> 2, q = lane & 3;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int t = warp + 4 * j;
        if (t >= 27) continue;
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            const int co = nb * 8 + 2 * q;
            if (gq < CI) {
                o[(t * CI + gq) * 16 + co] = acc[j][nb][0];
                o[(t * CI + gq) * 16 + co + 1] = acc[j][nb][1];
            }
            if (gq + 8 < CI) {
                o[(t * CI + gq + 8) * 16 + co] = acc[j][nb][2];
                o[(t * CI + gq + 8) * 16 + co + 1] = acc[j][nb][3];
            }
        }
    }
}

// ---- host side ----
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// slab shape for an n^3 level: minimise the staged bytes plus the tile work over all slabs
bool pick_geom(int n, Geom &best) {
    if (n < 8 || n > 254) return false;
    double best_cost = -1.0;
    const int W = n + 2;
    for (int tz = 1; tz <= 16 && tz <= n; tz *= 2) {
        for (int ty = 1; ty <= n; ++ty) {
            const int R = n % 128 == 0 ? 1 : ty;
            if (ty % R) continue;
            Geom g;
            g.n = n; g.ty = ty; g.tz = tz; g.R = R; g.W = W; g.Ys = ty + 2; g.Zs = tz + 2;
            g.tpg = ((R - 1) * W + n + 127) / 128;
            g.gpp = ty / R;
            g.tiles = tz * g.gpp * g.tpg;
            if (g.tiles > kMaxTiles || g.Ys > 256 || g.Zs > 256) continue;
            const int staged = g.Zs * g.Ys * W;
            int maxread = 0;
            for (int i = 0; i < g.tiles; ++i) {
                const int m = tile_start(g, i) + 127 + 1 + W + W * g.Ys;
                if (m > maxread) maxread = m;
            }
            g.half_pos = (maxread + 1 > staged ? maxread + 1 : staged);
            g.half_pos = (g.half_pos + 63) / 64 * 64;
            g.half_bytes = (uint32_t)g.half_pos * 16u;
            g.smem = kWRegion + 2 * g.half_bytes + 1024;
            if ((int)g.smem > kMaxSmem) continue;
            if ((int)g.smem < kMinSmem) g.smem = kMinSmem;
            g.nsy = (n + ty - 1) / ty;
            g.nslab = g.nsy * ((n + tz - 1) / tz);
            const double cost = (double)g.nslab * ((double)staged * 32.0 + (double)g.tiles * 128.0 * 64.0);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best = g;
            }
        }
    }
    return best_cost >= 0;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

template <class TI, class TO, int CI, bool BWD, bool ACT, bool TMA>
bool launch_conv(const Geom &g, const CUtensorMap &map, const TI *X, const float *W, TO *Y, int *err, cudaStream_t s) {
    auto kern = k_conv3_tc<TI, TO, CI, BWD, ACT, TMA>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        attr = true;
    }
    int grid = 2 * num_sms();
    if (grid > g.nslab) grid = g.nslab;
    launch_k(kern, dim3(grid), dim3(kThreads), (size_t)g.smem, s, map, g, X, W, Y, err);
    return cudaPeekAtLastError() == cudaSuccess;
}

bool encode_act_map(CUtensorMap &map, const Geom &g, const bf16 *X) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t n = (cuuint64_t)g.n;
    const cuuint64_t dims[4] = {16, n, n, n};
    const cuuint64_t strides[3] = {32, 32 * n, 32 * n * n};
    const cuuint32_t box[4] = {8, (cuuint32_t)g.W, (cuuint32_t)g.Ys, (cuuint32_t)g.Zs};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)X, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace

bool conv3_fwd(int n, int ci, const bf16 *X, const float *W, bf16 *Y, int *err, cudaStream_t s) {
    Geom g;
    if (!pick_geom(n, g)) return false;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (ci == 16) {
        if (!encode_act_map(map, g, X)) return false;
        return launch_conv<bf16, bf16, 16, false, true, true>(g, map, X, W, Y, err, s);
    }
    if (ci == 4) return launch_conv<bf16, bf16, 4, false, true, false>(g, map, X, W, Y, err, s);
    return false;
}

bool conv3_bwd(int n, const float *G, const float *W, float *Y, int *err, cudaStream_t s) {
    Geom g;
    if (!pick_geom(n, g)) return false;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    return launch_conv<float, float, 16, true, false, false>(g, map, G, W, Y, err, s);
}

int wgrad3_max_blocks() { return kWgBlocks; }

int wgrad3(int n, int ci, const bf16 *X, const float *G, float *partials, cudaStream_t s) {
    const int ntiles = ((n + WX - 1) / WX) * ((n + WY - 1) / WY) * ((n + WZ - 1) / WZ);
    const int nb = ntiles < kWgBlocks ? ntiles : kWgBlocks;
    if (ci == 16) launch_k(k_wgrad3_mma<16>, dim3(nb), dim3(kThreads), 0, s, n, X, G, partials);
    else if (ci == 4) launch_k(k_wgrad3_mma<4>, dim3(nb), dim3(kThreads), 0, s, n, X, G, partials);
    else return 0;
    return cudaPeekAtLastError() == cudaSuccess ? nb : 0;
}

void mma_selftest(const bf16 *A, const bf16 *B, float *D, int *err, cudaStream_t s) {
    launch_k(k_mma_selftest, dim3(1), dim3(kThreads), 0, s, A, B, D, err);
}

}  // namespace wstc
