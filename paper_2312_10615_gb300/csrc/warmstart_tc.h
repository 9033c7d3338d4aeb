// warmstart_tc.h -- tensor-core kernels of the initial-guess network (warmstart_tc.cu): the 3x3x3
// convolution as an implicit GEMM on the 5th-generation tensor cores (tcgen05, accumulators in tensor
// memory, halo tiles staged by TMA) and its weight gradient on warp-level mma.sync.  BF16 operands,
// FP32 accumulation.  Activations are channels-last ([voxel][C], x fastest), n^3 cubes.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace wstc {

typedef __nv_bfloat16 bf16;

// Y = act(conv(X, W)) with CI in {4, 16} input and 16 output channels, zero padding; W [27][CI][16]
// FP32 (rounded to BF16 for the product); bwd: the data gradient of a 16 -> 16 layer (taps mirrored,
// channel roles exchanged, no activation), X FP32.  Returns false (nothing launched) where the
// tensor-core form does not apply (n outside [8, 254], shared memory, a tensor map the driver
// refuses); err: device flag set to 1 if a bounded wait ran out
bool conv3_fwd(int n, int ci, const bf16 *X, const float *W, bf16 *Y, int *err, cudaStream_t s);
bool conv3_bwd(int n, const float *G, const float *W, float *Y, int *err, cudaStream_t s);
// per-block partial sums of dW[t][ci][co] = sum_v X[v + off_t][ci] G[v][co] (X BF16, G FP32 rounded
// to BF16) into partials [nblocks][27][ci][16]; returns nblocks (0: not launched)
int wgrad3(int n, int ci, const bf16 *X, const float *G, float *partials, cudaStream_t s);
int wgrad3_max_blocks();
// one 128 x 16 x 16 tcgen05 MMA, D = A B^T (A [128][16], B [16][16] BF16 row-major, D FP32)
void mma_selftest(const bf16 *A, const bf16 *B, float *D, int *err, cudaStream_t s);

}  // namespace wstc
