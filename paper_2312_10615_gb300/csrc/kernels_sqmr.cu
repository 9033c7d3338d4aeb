// kernels_sqmr.cu -- FP64 kernels of MG-preconditioned SQMR (Tao & Sifakis, Alg. 4):
// operator apply fused with q^T L q, fused vector recurrences, deterministic dot products
// (per-block partials, warp shuffles, fixed-order final sum) and the scalar recurrences on the
// device, so an iteration needs no host round trip except the convergence flag.
#include <math.h>

#include "kernels.h"

namespace smg {

namespace {
constexpr int kBlock = 256;
constexpr int BX = 32, BY = 8;

// sum NV values over the block (warp shuffles, then warp 0 over the per-warp sums) and store them
// as partials[slot * kRedParts + m]; fixed order, so the result is reproducible
template <int NV> __device__ __forceinline__ void block_store(double (&v)[NV], double *partials, int slot) {
    __shared__ double sh[NV][kBlock / 32];
    int tid = threadIdx.x + blockDim.x * threadIdx.y;
    int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int m = 0; m < NV; ++m) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
        if (lane == 0) sh[m][warp] = v[m];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            double s = lane < kBlock / 32 ? sh[m][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) partials[slot * kRedParts + m] = s;
        }
    }
}
}  // namespace

// Cell-centric 3D launch (as k_apply): blocks of 32 x 8 positions (i, j), KZR planes marched by
// each thread, four packed entries per position; one partial sum per block.  The input vectors
// hold 0 off the unknowns (the fast stencils rely on it).
constexpr int KZR = 16;
static dim3 red_grid(const Lev &L) {
    return dim3((L.nx + 1 + BX - 1) / BX, (L.ny + 1 + BY - 1) / BY, (L.nz + 1 + KZR - 1) / KZR);
}
int reduce_parts(const Lev &L) {
    dim3 g = red_grid(L);
    return (int)(g.x * g.y * g.z);
}

template <bool RESIDUAL, bool BATCH>
__global__ void __launch_bounds__(256) k_apply_red(Lev L, const double *__restrict__ x, const double *__restrict__ b,
                                                   double *__restrict__ w, double *partials, Coef<double> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) w = bslot(w, L.bstride, zs.p);
    if constexpr (BATCH) partials = bslot(partials, L.bstride, zs.p);
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    double v[1] = {0.0};
    if (i <= L.nx && j <= L.ny) {
        int k0 = zs.z * KZR, k1 = k0 + KZR < L.nz + 1 ? k0 + KZR : L.nz + 1;
        for (int k = k0; k < k1; ++k) {
            Quad Q = quad_at(L, i, j, k);
            double o[4];
            if (L.flags) quad_eval<double, OP_APPLY, true>(x, L, i, j, k, Q, K, o);
            else quad_eval<double, OP_APPLY, false>(x, L, i, j, k, Q, K, o);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (!Q.ex[c]) continue;
                double y = 0.0;
                if (Q.act[c]) {
                    if (RESIDUAL) {
                        y = b[Q.q[c]] - o[c];
                        v[0] += y * y;
                    } else {
                        y = o[c];
                        v[0] += x[Q.q[c]] * y;
                    }
                }
                if (w) w[Q.q[c]] = y;
            }
        }
    }
    block_store<1>(v, partials, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zs.z));
}
// red_grid for all the problems of a batched level (z blocks of problem p follow those of p - 1)
static dim3 red_grid_all(const Lev &L) {
    dim3 g = red_grid(L);
    g.z *= L.nb;
    return g;
}

int launch_apply_dot(const Lev &L, const double *q, double *w, double *partials, cudaStream_t s) {
    launch_k(L.nb > 1 ? k_apply_red<false, true> : k_apply_red<false, false>, red_grid_all(L), dim3(BX, BY, 1), 0, s, L, q, nullptr, w, partials,
             coef<double>(L, 0.0));
    return reduce_parts(L);
}
int launch_residual_dot(const Lev &L, const double *b, const double *x, double *w, double *partials, cudaStream_t s) {
    launch_k(L.nb > 1 ? k_apply_red<true, true> : k_apply_red<true, false>, red_grid_all(L), dim3(BX, BY, 1), 0, s, L, x, b, w, partials, coef<double>(L, 0.0));
    return reduce_parts(L);
}

// a.a and a.b
template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_dot2(long long n, const T *__restrict__ a, const double *__restrict__ b,
                                              double *partials, long long bs) {
    pdl_enter();
    if constexpr (BATCH) a = bslot(a, bs, (int)blockIdx.y);
    if constexpr (BATCH) b = bslot(b, bs, (int)blockIdx.y);
    if constexpr (BATCH) partials = bslot(partials, bs, (int)blockIdx.y);
    double v[2] = {0.0, 0.0};
    // groups of four entries with 16-byte loads (the vectors start 256-byte aligned), then the tail
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = n >> 2;
    for (long long g = gid; g < n4; g += stride) {
        double x[4], y[4] = {0.0, 0.0, 0.0, 0.0};
        if constexpr (sizeof(T) == 4) {
            const float4 q = reinterpret_cast<const float4 *>(a)[g];
            x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
        } else {
            const double2 q0 = reinterpret_cast<const double2 *>(a)[2 * g], q1 = reinterpret_cast<const double2 *>(a)[2 * g + 1];
            x[0] = q0.x; x[1] = q0.y; x[2] = q1.x; x[3] = q1.y;
        }
        if (b) {
            const double2 r0 = reinterpret_cast<const double2 *>(b)[2 * g], r1 = reinterpret_cast<const double2 *>(b)[2 * g + 1];
            y[0] = r0.x; y[1] = r0.y; y[2] = r1.x; y[3] = r1.y;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[0] += x[k] * x[k];
            v[1] += x[k] * y[k];
        }
    }
    for (long long t = 4 * n4 + gid; t < n; t += stride) {
        double x = (double)a[t];
        v[0] += x * x;
        if (b) v[1] += x * b[t];
    }
    block_store<2>(v, partials, blockIdx.x);
}
template <class T>
void launch_dot2(long long n, const T *a, const double *b, double *partials, cudaStream_t s, const Bat &bt) {
    launch_k(bt.nb > 1 ? k_dot2<T, true> : k_dot2<T, false>, dim3(kRedBlocks, bt.nb), dim3(kBlock), 0, s, n, a, b, partials, bt.bs);
}

// scalar recurrences of Alg. 4 (one block; fixed-order sum of the nparts partials)
template <bool BATCH>
__global__ void __launch_bounds__(256) k_scalars(int stage, const double *partials, int nparts, SqmrState *st,
                                                 double *host_out, double aux, long long bs) {
    pdl_enter();
    if constexpr (BATCH) partials = bslot(partials, bs, (int)blockIdx.x);
    if constexpr (BATCH) st = bslot(st, bs, (int)blockIdx.x);
    if constexpr (BATCH) {
        host_out += 2 * blockIdx.x;
        if (st->frozen && stage <= 2) return;
    }
    __shared__ double sh[kRedParts][kBlock];
    double v[kRedParts] = {0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < nparts; t += blockDim.x)
#pragma unroll
        for (int m = 0; m < kRedParts; ++m) v[m] += partials[t * kRedParts + m];
#pragma unroll
    for (int m = 0; m < kRedParts; ++m) sh[m][threadIdx.x] = v[m];
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int m = 0; m < kRedParts; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double p0 = sh[0][0], p1 = sh[1][0];
    switch (stage) {
    case 0: {  // sigma = q^T L q, alpha = rho / sigma
        st->sigma = p0;
        if (!isfinite(p0)) st->nonfinite = 1;
        if (p0 == 0.0 || st->rho == 0.0) st->breakdown = 1;
        st->alpha = (p0 != 0.0) ? st->rho / p0 : 0.0;
        break;
    }
    case 1: {  // nu_j, c_j, tau_j, rho_j, beta_j and the coefficients of d_j
        st->tt = p0;
        st->st = p1;
        double nu = sqrt(p0) / st->tau;
        double c2 = 1.0 / (1.0 + nu * nu);
        st->nu = nu;
        st->c2 = c2;
        st->tau = st->tau * nu * sqrt(c2);
        st->coefA = c2 * st->nu_prev * st->nu_prev;
        st->coefB = c2 * st->alpha;
        st->rho_new = p1;
        st->beta = (st->rho != 0.0) ? p1 / st->rho : 0.0;
        if (!isfinite(nu) || !isfinite(p1)) st->nonfinite = 1;
        break;
    }
    case 2: {  // |r_j|^2 of the recursive true residual; advance the iteration
        st->rr = p0;
        st->rho = st->rho_new;
        st->nu_prev = st->nu;
        st->iter += 1;
        st->dx_pending = 1;  // d_j, x_j still to be applied (k_update_dx, with this iteration's coefA / coefB)
        if (!isfinite(p0)) st->nonfinite = 1;
        host_out[0] = p0;
        host_out[1] = (double)(st->breakdown | (st->nonfinite << 1));
        break;
    }
    case 3: {  // initial tau_0 = |t_0|, rho_0 = s_0^T t_0, nu_0 = 0
        st->tt = p0;
        st->tau = sqrt(p0);
        st->rho = p1;
        st->nu_prev = 0.0;
        st->iter = 0;
        st->breakdown = 0;
        st->dx_pending = 0;
        st->nonfinite = (!isfinite(p0) || !isfinite(p1)) ? 1 : 0;
        host_out[0] = p0;
        host_out[1] = p1;
        break;
    }
    case 4: {  // a plain sum (norms) to the host
        host_out[0] = p0;
        host_out[1] = p1;
        break;
    }
    case 5: {  // pressure mean (aux = number of pressures)
        st->pmean = p0 / aux;
        break;
    }
    }
}

void launch_scalars(int stage, const double *partials, int nparts, SqmrState *st, double *host_out,
                    cudaStream_t s, const Bat &bt) {
    launch_k(bt.nb > 1 ? k_scalars<true> : k_scalars<false>, dim3(bt.nb), dim3(kBlock), 0, s, stage, partials, nparts,
             st, host_out, 0.0, bt.bs);
}
void launch_scalars_aux(int stage, const double *partials, int nparts, SqmrState *st, double *host_out, double aux,
                        cudaStream_t s) {
    launch_k(k_scalars<false>, dim3(1), dim3(kBlock), 0, s, stage, partials, nparts, st, host_out, aux, 0LL);
}

// s_j = s_{j-1} - alpha t  (t = L q_{j-1}); optional narrowed copy for the V-cycle
template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_update_s(long long n, double *__restrict__ s, const double *__restrict__ w,
                                                  const SqmrState *__restrict__ st, T *__restrict__ bT, long long bs) {
    pdl_enter();
    if constexpr (BATCH) s = bslot(s, bs, (int)blockIdx.y);
    if constexpr (BATCH) w = bslot(w, bs, (int)blockIdx.y);
    if constexpr (BATCH) st = bslot(st, bs, (int)blockIdx.y);
    if constexpr (BATCH) bT = bslot(bT, bs, (int)blockIdx.y);
    if (BATCH && st->frozen) return;
    double alpha = st->alpha;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        double v = s[t] - alpha * w[t];
        s[t] = v;
        if (bT) bT[t] = cvt<T>(v);
    }
}
template <class T>
void launch_update_s(long long n, double *s, const double *w, const SqmrState *st, T *bT, cudaStream_t stream,
                     const Bat &bt) {
    launch_k(bt.nb > 1 ? k_update_s<T, true> : k_update_s<T, false>, dim3(kRedBlocks, bt.nb), dim3(kBlock), 0, stream, n, s, w, st, bT, bt.bs);
}

// d_j = c^2 nu_{j-1}^2 d_{j-1} + c^2 alpha q_{j-1};  x_j = x_{j-1} + d_j;
// r_j = (1 - c^2) r_{j-1} + c^2 s_j  (true residual of the QMR-smoothed iterate);
// q_j = t + beta q_{j-1};  partial |r_j|^2
// The d, x, r, q recurrences of Alg. 4 in two kernels.  The part the next iteration needs -- the recursive true
// residual r_j = (1 - c_j^2) r_{j-1} + c_j^2 s_j, its norm and q_j = t_j + beta_j q_{j-1} (written into the
// other of two q buffers, so q_{j-1} survives) -- and the part nothing in the iteration reads: the
// iterate, d_j = A_j d_{j-1} + B_j q_{j-1}, x_j = x_{j-1} + d_j.  The second is deferred into the next
// iteration, beside its V-cycle; it runs only while st->dx_pending is set (by the iteration's last
// scalar step; cleared when the update has been applied outside the loop).  Same arithmetic per entry.
template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_update_rq(long long n, const double *__restrict__ qo, double *__restrict__ qn,
                                                   const T *__restrict__ tv, double *__restrict__ r,
                                                   const double *__restrict__ sv, const SqmrState *__restrict__ st,
                                                   double *partials, long long bs) {
    pdl_enter();
    const int p = (int)blockIdx.y;
    if constexpr (BATCH) qo = bslot(qo, bs, p);
    if constexpr (BATCH) qn = bslot(qn, bs, p);
    if constexpr (BATCH) tv = bslot(tv, bs, p);
    if constexpr (BATCH) r = bslot(r, bs, p);
    if constexpr (BATCH) sv = bslot(sv, bs, p);
    if constexpr (BATCH) st = bslot(st, bs, p);
    if constexpr (BATCH) partials = bslot(partials, bs, p);
    if (BATCH && st->frozen) return;  // the whole block: one problem per blockIdx.y
    const double c2 = st->c2, beta = st->beta;
    double v[1] = {0.0};
#pragma unroll 1
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double q0 = qo[t];
        const double rn = (1.0 - c2) * r[t] + c2 * sv[t];
        r[t] = rn;
        qn[t] = (double)tv[t] + beta * q0;
        v[0] += rn * rn;
    }
    block_store<1>(v, partials, blockIdx.x);
}
template <bool BATCH>
__global__ void __launch_bounds__(256) k_update_dx(long long n, double *__restrict__ x, double *__restrict__ d,
                                                   const double *__restrict__ qo, const SqmrState *__restrict__ st,
                                                   long long bs) {
    pdl_enter();
    const int p = (int)blockIdx.y;
    if constexpr (BATCH) x = bslot(x, bs, p);
    if constexpr (BATCH) d = bslot(d, bs, p);
    if constexpr (BATCH) qo = bslot(qo, bs, p);
    if constexpr (BATCH) st = bslot(st, bs, p);
    if (!st->dx_pending || (BATCH && st->frozen)) return;
    const double A = st->coefA, B = st->coefB;
#pragma unroll 1
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double dn = A * d[t] + B * qo[t];
        d[t] = dn;
        x[t] += dn;
    }
}
template <class T>
void launch_update_rq(long long n, const double *qo, double *qn, const T *t, double *r, const double *sv,
                      const SqmrState *st, double *partials, cudaStream_t s, const Bat &bt) {
    launch_k(bt.nb > 1 ? k_update_rq<T, true> : k_update_rq<T, false>, dim3(kRedBlocks, bt.nb), dim3(kBlock), 0, s, n, qo, qn, t, r, sv, st, partials, bt.bs);
}
// blocks: the full reduction grid when it runs alone; a few per SM when it runs beside the V-cycle, so
// that the V-cycle's kernels keep most of every SM's thread slots
void launch_update_dx(long long n, double *x, double *d, const double *qo, const SqmrState *st, cudaStream_t s,
                      int blocks, const Bat &bt) {
    launch_k(bt.nb > 1 ? k_update_dx<true> : k_update_dx<false>, dim3(blocks > 0 ? blocks : kRedBlocks, bt.nb), dim3(kBlock), 0, s, n, x, d, qo, st, bt.bs);
}

__global__ void k_loop_check(const SqmrState *__restrict__ st, const LoopCtl *__restrict__ lc,
                             cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hi, int set_if, double *host_out) {
    if (threadIdx.x != 0) return;
    const double rr = st->rr;
    const bool stop = st->breakdown || st->nonfinite || !isfinite(rr) || sqrt(rr) / lc->nb < lc->tol ||
                      st->iter >= lc->max_iter;
    cudaGraphSetConditional(hw, stop ? 0u : 1u);
    if (set_if) cudaGraphSetConditional(hi, stop ? 0u : 1u);
    host_out[2] = (double)st->iter;
}
void launch_loop_check(const SqmrState *st, const LoopCtl *lc, cudaGraphConditionalHandle hw,
                       cudaGraphConditionalHandle hi, int set_if, double *host_out, cudaStream_t s) {
    k_loop_check<<<1, 32, 0, s>>>(st, lc, hw, hi, set_if, host_out);
}

template <class T>
__global__ void __launch_bounds__(256) k_init_q(long long n, const T *__restrict__ tv, double *__restrict__ q,
                                                double *__restrict__ d) {
    pdl_enter();
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        q[t] = (double)tv[t];
        d[t] = 0.0;
    }
}
template <class T> void launch_init_q(long long n, const T *t, double *q, double *d, cudaStream_t s) {
    launch_k(k_init_q<T>, dim3(kRedBlocks), dim3(kBlock), 0, s, n, t, q, d);
}

__global__ void __launch_bounds__(256) k_psum(Lev L, const double *__restrict__ x, double *partials) {
    pdl_enter();
    double v[1] = {0.0};
    long long np = L.n - L.off[3];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < np; t += (long long)gridDim.x * blockDim.x)
        v[0] += x[L.off[3] + t];  // pressures of non-interior cells hold 0
    block_store<1>(v, partials, blockIdx.x);
}
__global__ void __launch_bounds__(256) k_psub(Lev L, double *__restrict__ x, const SqmrState *__restrict__ st) {
    pdl_enter();
    double m = st->pmean;
    long long np = L.n - L.off[3];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < np; t += (long long)gridDim.x * blockDim.x)
        if (!L.flags || (L.flags[L.off[3] + t] & kFlagActive)) x[L.off[3] + t] -= m;
}
void launch_psum(const Lev &L, const double *x, double *partials, cudaStream_t s) {
    launch_k(k_psum, dim3(kRedBlocks), dim3(kBlock), 0, s, L, x, partials);
}
void launch_psub(const Lev &L, double *x, const SqmrState *st, cudaStream_t s) {
    launch_k(k_psub, dim3(kRedBlocks), dim3(kBlock), 0, s, L, x, st);
}

template void launch_dot2<float>(long long, const float *, const double *, double *, cudaStream_t, const Bat &);
template void launch_dot2<double>(long long, const double *, const double *, double *, cudaStream_t, const Bat &);
template void launch_update_s<float>(long long, double *, const double *, const SqmrState *, float *, cudaStream_t,
                                     const Bat &);
template void launch_update_s<double>(long long, double *, const double *, const SqmrState *, double *, cudaStream_t,
                                      const Bat &);
template void launch_update_s<bf16>(long long, double *, const double *, const SqmrState *, bf16 *, cudaStream_t,
                                    const Bat &);
template void launch_update_rq<float>(long long, const double *, double *, const float *, double *, const double *,
                                      const SqmrState *, double *, cudaStream_t, const Bat &);
template void launch_update_rq<double>(long long, const double *, double *, const double *, double *, const double *,
                                       const SqmrState *, double *, cudaStream_t, const Bat &);
// x += t (the pure-multigrid update x_{k+1} = x_k + W^+ (b - L~ x_k), t in the V-cycle's precision)
template <class T>
__global__ void __launch_bounds__(256) k_add_to(long long n, const T *__restrict__ tv, double *__restrict__ x) {
    pdl_enter();
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        x[t] += (double)tv[t];
}
template <class T> void launch_add_to(long long n, const T *t, double *x, cudaStream_t s) {
    launch_k(k_add_to<T>, dim3(kRedBlocks), dim3(kBlock), 0, s, n, t, x);
}
template void launch_add_to<float>(long long, const float *, double *, cudaStream_t);
template void launch_add_to<double>(long long, const double *, double *, cudaStream_t);
template void launch_init_q<float>(long long, const float *, double *, double *, cudaStream_t);
template void launch_init_q<double>(long long, const double *, double *, double *, cudaStream_t);

}  // namespace smg
