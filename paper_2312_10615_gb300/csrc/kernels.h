// kernels.h -- host-side launchers of the CUDA kernels (definitions in kernels_level.cu and
// kernels_sqmr.cu).  T is the V-cycle precision (float or double); SQMR kernels are FP64.
#pragma once
#include <cuda_runtime.h>

#include "stokes_internal.cuh"

namespace smg {

// ---- per-level operators (kernels_level.cu) ----
// y = L~x (gamma_on) or Lx on the unknowns, 0 elsewhere; if b != nullptr: y = b - (L~x)
// T: arithmetic precision of a level kernel; TB: storage type of the level operands b, r, g/h
// (T itself, or BF16 on the finest levels of the mixed-precision V-cycle)
template <class T, class TB> void launch_apply(const Lev &L, const T *x, const TB *b, TB *y, double gam, cudaStream_t s);
// b = f + Dirichlet folding (finest level, FP64)
void launch_rhs(const Lev &L, const double *f, const double *g, double *b, cudaStream_t s);
// symmetric DGS pieces (Alg. 2 / Eq. ldist) on the V2 set
template <class T, class TB> void launch_dgs_u(const Lev &L, T *x, const TB *b, int parity, cudaStream_t s);
// both velocity parities of one DGS stage (pa first) in one out-of-place pass X -> Y; Y receives every
// packed entry; bit-identical to launch_dgs_u(pa) then launch_dgs_u(1 - pa) in place
template <class T, class TB>
void launch_dgs_u_fused(const Lev &L, const T *X, T *Y, const TB *b, int pa, cudaStream_t s);
template <class T, class TB> bool dgs_u_fused_prepare();
template <class T, class TB>
void launch_dgs_p_fwd(const Lev &L, T *x, const TB *b, T *delta, int colour, cudaStream_t s);
template <class T> void launch_dgs_p_gather(const Lev &L, T *x, const T *delta, cudaStream_t s);
// backward pressure colours read g = b - Au (faces) and h = b - Bu (cells) precomputed into gh;
// with delta != null the same launch applies the pending neighbour-pressure part of the forward
// sweep (what launch_dgs_p_gather does)
template <class T, class TB>
void launch_dgs_p_bwd_prep(const Lev &L, T *x, const TB *b, TB *gh, const T *delta, cudaStream_t s);
template <class T, class TB> void launch_dgs_p_bwd(const Lev &L, T *x, const TB *gh, int colour, cudaStream_t s);
// colours c and c ^ 1 (i bit only) in one launch, one block per group of whole x-rows; false (nothing
// launched) if a row is longer than 512 cells of one colour
template <class T, class TB>
bool launch_dgs_p_fwd_pair(const Lev &L, T *x, const TB *b, T *delta, int colour, cudaStream_t s);
template <class T, class TB> bool launch_dgs_p_bwd_pair(const Lev &L, T *x, const TB *gh, int colour, cudaStream_t s);
// symmetric distributive weighted Jacobi on V2 (Sec. 3.1), weight w; t: level-size scratch, delta: per cell
template <class T, class TB>
void launch_dwj_sym(const Lev &L, T *x, const TB *b, T *t, T *delta, double w, cudaStream_t s);
// one colour of the multiplicative Vanka sweep on V1 (compute corrections, then add them)
// corrections scaled by w (1 for the multiplicative sweep, 1/2 for the damped additive step)
template <class T, class TB>
void launch_vanka_compute(const Lev &L, const T *x, const TB *b, const int *cells, const int *tab, int ncell,
                          const T *kinv, T *corr,
                          int cap, double w, cudaStream_t s);
template <class T>
void launch_vanka_apply(const Lev &L, T *x, const int *cells, int ncell, const T *corr, int cap, cudaStream_t s);
// a whole symmetric Vanka sweep (colours 0..7 then 7..0), `sweeps` times, in ONE cooperative
// launch: compute / grid barrier / apply / grid barrier per colour.  The barrier spins at most
// kBarrierSpinLimit polls; on expiry it sets bar->err and every block stops waiting.
struct GridBarrier {
    unsigned count, gen;
    int err, pad;
};
constexpr unsigned kBarrierSpinLimit = 1u << 22;
struct VankaLists {
    const int *cells[8];
    const int *tab[8];  // per-cell inverse-table entries (label domains with exterior cells), else nullptr
    int count[8];
};
// missing_blocks > 0 (bounded-wait self-test only): the barrier waits for that many blocks more than the
// grid has, so every wait runs out after spin_limit polls and sets bar->err
template <class T, class TB>
void launch_vanka_sweep(const Lev &L, T *x, const TB *b, const VankaLists &lists, const T *kinv, T *corr, int cap,
                        int sweeps, GridBarrier *bar, int max_blocks, cudaStream_t s, int missing_blocks = 0,
                        unsigned spin_limit = kBarrierSpinLimit);
template <class T, class TB> int vanka_sweep_blocks_per_sm();
// `sweeps` symmetric Vanka sweeps, one launch per colour step on two copies of the state (x and x2,
// ping-pong; x2 holds 0 off the unknowns), after copying the nshell DOFs the patches read or write
// (shell) from x to x2 at the start of each sweep; the result is in x, bit-identical to the
// two-launch form
template <class T, class TB>
void launch_vanka_pingpong(const Lev &L, T *x, T *x2, const TB *b, const VankaLists &lists, const int *shell,
                           int nshell, const T *kinv, int sweeps, cudaStream_t s);
// one symmetric Vanka sweep (x sweeps) in a single thread-block cluster of `cluster` CTAs x 1024
// threads separated by hardware cluster barriers (no software wait); returns the launch status
template <class T, class TB> cudaError_t vanka_cluster_prepare();
// one symmetric Vanka sweep (x sweeps) in one 1024-thread block on a shared-memory copy of the level
// (x, b, corrections); vanka_smem_prepare sets the shared-memory opt-in and says whether it fits
template <class T, class TB> bool vanka_smem_prepare(const Lev &L, int cap);
template <class T, class TB>
void launch_vanka_smem(const Lev &L, T *x, const TB *b, const VankaLists &lists, const T *kinv, int cap, int sweeps,
                       cudaStream_t s);
template <class T, class TB>
cudaError_t launch_vanka_cluster(const Lev &L, T *x, const TB *b, const VankaLists &lists, const T *kinv, T *corr,
                                 int cap, int sweeps, int cluster, cudaStream_t s);
// transfers (Sec. 2): bc = R rf,  xf += P ec
// tile of a transfer launch: thread block bx x by over the coarse level's (x, y) positions, kz coarse
// z-planes marched per thread (any tile gives the same bits)
struct Tile {
    int bx = 32, by = 8, kz = 8;
};
template <class T, class TF, class TC>
void launch_restrict(const Lev &F, const Lev &C, const TF *rf, TC *bc, cudaStream_t s, Tile t = Tile());
template <class T> void launch_prolong(const Lev &F, const Lev &C, const T *ec, T *xf, cudaStream_t s, Tile t = Tile());
// coarsest level: x = Kinv b over the compact unknown list (FP64 matrix)
template <class T>
void launch_coarse(const Lev &C, const int *cidx, int nc, const double *kinv, const T *b, T *x, cudaStream_t s);
// set every entry that is not an unknown to 0 (every internal vector keeps this invariant: the fast
// stencils read wall-normal faces as zeros)
template <class T> void launch_mask(const Lev &L, T *x, cudaStream_t s);
// precision conversion of a packed vector
template <class A, class B> void launch_convert(long long n, const A *in, B *out, cudaStream_t s);

// ---- SQMR (kernels_sqmr.cu), all FP64 except the preconditioned vector t of type T ----
struct SqmrState {
    double rho, sigma, alpha, tau, nu, nu_prev, c2, coefA, coefB, beta, rho_new;
    double tt, st, rr, bb, pmean;
    int breakdown, nonfinite, iter, dx_pending;
    int frozen, pad;  // batched solves: a problem that has converged keeps its state (its kernels return)
};
// problems of a batched launch of the SQMR kernels: nb problems, problem p's vectors, partials and state
// at byte offset p * bs from problem 0's, its two host-visible values at host_out + 2 p
struct Bat {
    int nb = 1;
    long long bs = 0;
};

constexpr int kRedBlocks = 1184;  // 152 SMs x 8 resident 256-thread blocks: grid of every reduction kernel
constexpr int kRedParts = 3;      // partial sums per block

// w = L q (FP64, gamma = 0) with per-block partials of q.w ; unknowns only.  Returns the number
// of partials written (reduce_parts(L)); the 1D vector kernels below write kRedBlocks.
int reduce_parts(const Lev &L);
int launch_apply_dot(const Lev &L, const double *q, double *w, double *partials, cudaStream_t s);
// w = b - L x (w may be null) with partials of |b - Lx|^2
int launch_residual_dot(const Lev &L, const double *b, const double *x, double *w, double *partials, cudaStream_t s);
// partials of a.a (and optionally a.b)
template <class T>
void launch_dot2(long long n, const T *a, const double *b, double *partials, cudaStream_t s, const Bat &bt = Bat());
// scalar stages on one thread block: 0 alpha (after q.Lq), 1 nu/c/tau/beta (after |t|^2, s.t),
// 2 residual norm (after |r|^2), 3 init (after |t|^2, s.t of the first V-cycle), 4 |b|^2, 5 pressure mean
void launch_scalars(int stage, const double *partials, int nparts, SqmrState *st, double *host_out,
                    cudaStream_t s, const Bat &bt = Bat());
void launch_scalars_aux(int stage, const double *partials, int nparts, SqmrState *st, double *host_out, double aux,
                        cudaStream_t s);
// s -= alpha w ; optionally b32 = (T) s for a lower-precision V-cycle
template <class T>
void launch_update_s(long long n, double *s, const double *w, const SqmrState *st, T *bT, cudaStream_t stream,
                     const Bat &bt = Bat());
// the d, x, r, q recurrences of Alg. 4 in two parts: r = (1-c2) r + c2 s ; qn = t + beta qo ; partials of
// |r|^2 (the part the next iteration needs) and, when st->dx_pending, d = coefA d + coefB qo ; x += d (the
// iterate, deferred into the next iteration)
template <class T>
void launch_update_rq(long long n, const double *qo, double *qn, const T *t, double *r, const double *sv,
                      const SqmrState *st, double *partials, cudaStream_t s, const Bat &bt = Bat());
void launch_update_dx(long long n, double *x, double *d, const double *qo, const SqmrState *st, cudaStream_t s,
                      int blocks = 0, const Bat &bt = Bat());
// the graph-resident SQMR loop (a while node around one or two iterations): after an iteration, continue
// unless it broke down, produced a non-finite value, brought the recursive residual below tol
// (sqrt(rr) / nb < tol, the host's own test) or reached max_iter; sets the while handle and, with
// set_if, the handle of the node that runs the body's second iteration; host_out[2] = iterations done
struct LoopCtl {
    double nb, tol;
    int max_iter, pad;
};
void launch_loop_check(const SqmrState *st, const LoopCtl *lc, cudaGraphConditionalHandle hw,
                       cudaGraphConditionalHandle hi, int set_if, double *host_out, cudaStream_t s);
// q = t (widening), d = 0
template <class T> void launch_init_q(long long n, const T *t, double *q, double *d, cudaStream_t s);
template <class T> void launch_add_to(long long n, const T *t, double *x, cudaStream_t s);
// partial sum of the pressure block (for the mean) and subtraction of st->pmean
void launch_psum(const Lev &L, const double *x, double *partials, cudaStream_t s);
void launch_psub(const Lev &L, double *x, const SqmrState *st, cudaStream_t s);

}  // namespace smg
