// kernels_level.cu -- per-level CUDA kernels of the symmetric multigrid V-cycle (sm_103a):
// operator apply / residual (Eq. 2, Sec. 4), Dirichlet folding (Sec. 5), symmetric distributive
// Gauss-Seidel (Alg. 2, Eq. ldist, App. A), 8-colour multiplicative Vanka (Sec. 3.2, App. C,
// Sec. 6), restriction / prolongation (Sec. 2) and the exact coarsest solve (Alg. 1).
//
// Every kernel is bandwidth-shaped: 32 x 8 thread blocks over (x, y) of one z-plane (x fastest,
// so a warp reads one 128-byte line of FP32 values), the component folded into gridDim.y, 32-bit
// coordinates taken straight from the block/thread indices (no integer division), 64-bit only in
// the final address.  No tensor cores: nothing here is a contraction.
#include <algorithm>

#include "kernels.h"

namespace smg {

namespace {
constexpr int BX = 32, BY = 8;
constexpr int KZ = 8;  // z-planes marched by one thread (fewer, longer-lived blocks)
const dim3 kBlock3(BX, BY, 1);

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }
// the batched instantiation of a kernel (problem index from the grid, per-problem offsets) only where a
// launch covers several problems; a one-problem launch runs the plain kernel
#define BSEL(nb, ...) ((nb) > 1 ? __VA_ARGS__, true> : __VA_ARGS__, false>)

// geometry of a launch over the packed entries of ncomp components: grid (x tiles, y tiles x ncomp, z)
struct Geo {
    dim3 grid;
    int gy;  // y tiles per component
};
inline Geo geo_components(const Lev &L, int ncomp) {
    int mx = L.nx + 1, my = L.ny + 1, mz = L.nz + 1;
    Geo g;
    g.gy = cdiv(my, BY);
    g.grid = dim3(cdiv(mx, BX), g.gy * ncomp, cdiv(mz, KZ));
    return g;
}

// V2 index ranges of the box problem: faces of component c with normal index in [2, n-2] and
// tangential indices in [1, n-2]; cells with every index in [1, n-2].
// cells of colour (bx, by, bz) inside the V2 cell range [1, n-2]
__host__ __device__ inline void v2_colour_range(const Lev &L, int colour, int lo[3], int cnt[3]) {
    int n[3] = {L.nx, L.ny, L.nz};
    for (int d = 0; d < 3; ++d) {
        int bit = (colour >> d) & 1;
        lo[d] = bit ? 1 : 2;
        cnt[d] = (n[d] - 2 >= lo[d]) ? (n[d] - 2 - lo[d]) / 2 + 1 : 0;
    }
}
__device__ __forceinline__ bool in_v2_cell(const Lev &L, int i, int j, int k) { return v2_cell_at(L, i, j, k); }
__device__ __forceinline__ long long cell_lin(const Lev &L, int i, int j, int k) {
    return i + (long long)L.nx * (j + (long long)L.ny * k);
}
// (c, i, j) and the z range [k0, k1) of the calling thread in a geo_components launch; false if the
// thread lies outside component c's box
__device__ __forceinline__ bool thread_entry(const Lev &L, int gy, int &c, int &i, int &j, int &k0, int &k1) {
    c = blockIdx.y / gy;
    i = blockIdx.x * BX + threadIdx.x;
    j = (blockIdx.y - c * gy) * BY + threadIdx.y;
    k0 = blockIdx.z * KZ;
    int ez = ext(L, c, 2);
    k1 = k0 + KZ < ez ? k0 + KZ : ez;
    return i < ext(L, c, 0) && j < ext(L, c, 1) && k0 < ez;
}
}  // namespace

// ------------------------------------------------------------------------------------------
// y = L~x or b - L~x on every packed entry (0 off the unknowns); x must hold 0 off the unknowns.
//
// One entry per thread, blockIdx.z = 4 k + component.  The component is dispatched once at the top
// of the kernel, so every extent, stride and guard of the entry's row is specialised at compile
// time, and offsets within a component are IDX = 32-bit integers whenever the largest component
// has fewer than 2^31 entries (the kernels are instruction-bound, not DRAM-bound: 32-bit offsets
// halve the address arithmetic of the neighbour loads).

// row C of L~x at (i,j,k) (an unknown); P = false: faces A u only, cells -div u only
template <class T, int C, bool P, class IDX>
__device__ __forceinline__ T row_at(const T *__restrict__ x, const Lev &L, int i, int j, int k, const Coef<T> &K) {
    if constexpr (C < 3) {
        const IDX sy = (IDX)(L.nx + (C == 0)), sz = sy * (IDX)(L.ny + (C == 1));
        const IDX o = (IDX)i + sy * (IDX)j + sz * (IDX)k;
        const T *xc = x + L.off[C] + o;
        T s;
        if (!L.flags) {
            s = T(6) * xc[0];
            if (C == 0) s -= xc[-1] + xc[1];
            else s -= (i > 0 ? xc[-1] : T(0)) + (i < L.nx - 1 ? xc[1] : T(0));
            if (C == 1) s -= xc[-sy] + xc[sy];
            else s -= (j > 0 ? xc[-sy] : T(0)) + (j < L.ny - 1 ? xc[sy] : T(0));
            if (C == 2) s -= xc[-sz] + xc[sz];
            else s -= (k > 0 ? xc[-sz] : T(0)) + (k < L.nz - 1 ? xc[sz] : T(0));
        } else {
            // label domains: the dropped viscous terms of a face next to exterior cells (Sec. 5 reading)
            const uint8_t f = L.flags[L.off[C] + o];
            const IDX sn = C == 0 ? (IDX)1 : (C == 1 ? sy : sz);
            s = diag_weight<T>(f) * xc[0];
            s -= ((f & kFlagDropLo) ? T(0) : xc[-sn]) + ((f & kFlagDropHi) ? T(0) : xc[sn]);
            if (C != 0) s -= (i > 0 ? xc[-1] : T(0)) + (i < L.nx - 1 ? xc[1] : T(0));
            if (C != 1) s -= (j > 0 ? xc[-sy] : T(0)) + (j < L.ny - 1 ? xc[sy] : T(0));
            if (C != 2) s -= (k > 0 ? xc[-sz] : T(0)) + (k < L.nz - 1 ? xc[sz] : T(0));
        }
        if constexpr (!P) {
            return K.eh2 * s;
        } else {
            const IDX cy = (IDX)L.nx, cz = cy * (IDX)L.ny;
            const T *pc = x + L.off[3] + ((IDX)i + cy * (IDX)j + cz * (IDX)k);
            const IDX ps = C == 0 ? (IDX)1 : (C == 1 ? cy : cz);
            return K.eh2 * s + K.ih * (pc[0] - pc[-ps]);
        }
    } else {
        const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
        const T *u = x + L.off[0] + ((IDX)i + (nx + 1) * ((IDX)j + ny * (IDX)k));
        const T *v = x + L.off[1] + ((IDX)i + nx * ((IDX)j + (ny + 1) * (IDX)k));
        const T *w = x + L.off[2] + ((IDX)i + nx * ((IDX)j + ny * (IDX)k));
        const T div = (u[1] - u[0]) + (v[nx] - v[0]) + (w[nx * ny] - w[0]);
        if constexpr (!P) return -K.ih * div;
        else return -K.ih * div - K.gam * x[L.off[3] + ((IDX)i + nx * ((IDX)j + ny * (IDX)k))];
    }
}
// does entry (C; i,j,k) exist in the packed array, and is it an unknown?
template <int C> __device__ __forceinline__ bool entry_exists(const Lev &L, int i, int j, int k) {
    return i < L.nx + (C == 0) && j < L.ny + (C == 1) && k < L.nz + (C == 2);
}
template <int C> __device__ __forceinline__ bool entry_active(const Lev &L, int i, int j, int k) {
    if (C == 0) return i >= 1 && i <= L.nx - 1;
    if (C == 1) return j >= 1 && j <= L.ny - 1;
    if (C == 2) return k >= 1 && k <= L.nz - 1;
    return true;
}
// entry_active for an existing entry at packed index q, with the label flags where the domain has them
template <int C> __device__ __forceinline__ bool entry_unknown(const Lev &L, int i, int j, int k, long long q) {
    return entry_active<C>(L, i, j, k) && (!L.flags || (L.flags[q] & kFlagActive));
}
template <int C, class IDX> __device__ __forceinline__ long long entry_index(const Lev &L, int i, int j, int k) {
    const IDX sy = (IDX)(L.nx + (C == 0)), sz = sy * (IDX)(L.ny + (C == 1));
    return L.off[C] + (long long)((IDX)i + sy * (IDX)j + sz * (IDX)k);
}
inline dim3 entry_grid(const Lev &L) { return dim3(cdiv(L.nx + 1, BX), cdiv(L.ny + 1, BY), 4 * (L.nz + 1) * L.nb); }
// offsets of every component fit 32 bits
inline bool idx32(const Lev &L) { return (long long)(L.nx + 1) * (L.ny + 1) * (L.nz + 1) < (1LL << 31); }

template <class T, class TB, int C, class IDX>
__device__ __forceinline__ void apply_entry(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                            TB *__restrict__ y, const Coef<T> &K, int i, int j, int k) {
    if (!entry_exists<C>(L, i, j, k)) return;
    const long long q = entry_index<C, IDX>(L, i, j, k);
    T v = T(0);
    if (entry_unknown<C>(L, i, j, k, q)) {
        v = row_at<T, C, true, IDX>(x, L, i, j, k, K);
        if (b) v = T(ldv(b[q])) - v;
    }
    y[q] = cvt<TB>(v);
}

template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256, 8) k_apply(Lev L, const T *__restrict__ x, const TB *__restrict__ b,
                                                  TB *__restrict__ y, Coef<T> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) y = bslot(y, L.bstride, zs.p);
    const int c = zs.z & 3, k = zs.z >> 2;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: apply_entry<T, TB, 0, IDX>(L, x, b, y, K, i, j, k); break;
    case 1: apply_entry<T, TB, 1, IDX>(L, x, b, y, K, i, j, k); break;
    case 2: apply_entry<T, TB, 2, IDX>(L, x, b, y, K, i, j, k); break;
    default: apply_entry<T, TB, 3, IDX>(L, x, b, y, K, i, j, k);
    }
}


// ------------------------------------------------------------------------------------------
// Sec. 5: b = f on the unknowns with Dirichlet data g (ghost-extended layout) folded in
__device__ __forceinline__ long long gidx(const Lev &L, int c, int i, int j, int k) {
    long long nx = L.nx, ny = L.ny, nz = L.nz;
    long long G1 = (nx + 1) * (ny + 2) * (nz + 2), G2 = G1 + (nx + 2) * (ny + 1) * (nz + 2);
    if (c == 0) return i + (nx + 1) * ((j + 1) + (ny + 2) * (long long)(k + 1));
    if (c == 1) return G1 + (i + 1) + (nx + 2) * (j + (ny + 1) * (long long)(k + 1));
    return G2 + (i + 1) + (nx + 2) * ((j + 1) + (ny + 2) * (long long)k);
}

__global__ void __launch_bounds__(256) k_rhs(Lev L, int gy, const double *__restrict__ f, const double *__restrict__ g,
                                             double *__restrict__ b, Coef<double> K) {
    pdl_enter();
    int c, i, j, k0, k1;
    if (!thread_entry(L, gy, c, i, j, k0, k1)) return;
    for (int k = k0; k < k1; ++k) {
    long long q = pidx(L, c, i, j, k);
    if (!unknown(L, c, i, j, k)) {
        b[q] = 0.0;
        continue;
    }
    double v = f ? f[q] : 0.0;
    if (g) {
        if (c < 3) {
            const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
            // a term that drops out (across an exterior cell along the normal) reads no data
            const uint8_t fq = L.flags ? L.flags[q] : (uint8_t)0;
            for (int m = 0; m < 6; ++m) {
                if ((m == 2 * c && (fq & kFlagDropLo)) || (m == 2 * c + 1 && (fq & kFlagDropHi))) continue;
                int a = i + di[m], bb = j + dj[m], cc = k + dk[m];
                if (!unknown(L, c, a, bb, cc) && dirichlet_face(L, c, a, bb, cc)) v += K.eh2 * g[gidx(L, c, a, bb, cc)];
            }
        } else {
            for (int d = 0; d < 3; ++d) {
                int hi = i + (d == 0), hj = j + (d == 1), hk = k + (d == 2);
                if (!unknown(L, d, hi, hj, hk) && dirichlet_face(L, d, hi, hj, hk)) v += K.ih * g[gidx(L, d, hi, hj, hk)];
                if (!unknown(L, d, i, j, k) && dirichlet_face(L, d, i, j, k)) v -= K.ih * g[gidx(L, d, i, j, k)];
            }
        }
    }
    b[q] = v;
    }
}

void launch_rhs(const Lev &L, const double *f, const double *g, double *b, cudaStream_t s) {
    Geo gg = geo_components(L, 4);
    launch_k(k_rhs, dim3(gg.grid), dim3(kBlock3), 0, s, L, gg.gy, f, g, b, coef<double>(L, 0.0));
}

// ------------------------------------------------------------------------------------------
// Alg. 2 velocity block: V2 faces of one parity (i+j+k), u, v, w together (A does not couple
// components; same-parity faces are not A-neighbours, pressures are not written) -- in place.
// Thread x covers every other face of a row so no thread idles.
// Cell-centric: the thread of V2 cell (i,j,k) of the given parity updates its low faces u, v, w (all
// three share the cell's parity), each if it lies in that component's V2 range.  Inside the V2
// cell range every stencil neighbour exists, so no guards are needed.
// one relaxed velocity face: x0 + (b - (eh2 (6 x0 - neighbours) + ih (p_plus - p_minus))) / (6 eh2).
// The multiply-adds are spelled out as fma() calls, so every kernel that relaxes a face (the in-place
// parity launches and the fused two-parity pass) rounds the same way and produces the same bits.
template <class T>
__device__ __forceinline__ T dgs_relax(T x0, T nxm, T nxp, T nym, T nyp, T nzm, T nzp, T pc, T pm, T bv,
                                       const Coef<T> &K) {
    T s = fma(T(6), x0, -nxm);
    s = s - nxp;
    s = s - nym;
    s = s - nyp;
    s = s - nzm;
    s = s - nzp;
    const T g = K.ih * (pc - pm);
    const T r = bv - fma(K.eh2, s, g);
    return x0 + r / (T(6) * K.eh2);
}
template <class T, class TB, class IDX>
__device__ __forceinline__ void dgs_face(T *__restrict__ xq, const TB *__restrict__ bq, IDX sy, IDX sz, T pc, T pm,
                                         const Coef<T> &K) {
    xq[0] = dgs_relax<T>(xq[0], xq[-1], xq[1], xq[-sy], xq[sy], xq[-sz], xq[sz], pc, pm, T(ldv(bq[0])), K);
}

template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256, 8) k_dgs_u(Lev L, T *__restrict__ x, const TB *__restrict__ b, int parity,
                                                  Coef<T> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    const int j = 1 + blockIdx.y * BY + threadIdx.y;
    if (j > L.ny - 2) return;
    const int k = 1 + zs.z;
    int i = 1 + 2 * (blockIdx.x * BX + threadIdx.x);
    i += (i + j + k + parity) & 1;
    if (i > L.nx - 2) return;
    const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
    const IDX uy = nx + 1, uz = (nx + 1) * ny, vz = nx * (ny + 1), wz = nx * ny;
    const IDX ci = (IDX)i, cj = (IDX)j, ck = (IDX)k;
    const T *pp = x + L.off[3] + (ci + nx * (cj + ny * ck));
    const T pc = pp[0];
    const uint8_t *fl = L.flags;  // label domains: a face is relaxed only if both its cells are V2
    {
        const IDX o = ci + uy * cj + uz * ck;
        if (i >= 2 && (!fl || (fl[L.off[0] + o] & kFlagV2)))
            dgs_face<T, TB, IDX>(x + L.off[0] + o, b + L.off[0] + o, uy, uz, pc, pp[-1], K);
    }
    {
        const IDX o = ci + nx * cj + vz * ck;
        if (j >= 2 && (!fl || (fl[L.off[1] + o] & kFlagV2)))
            dgs_face<T, TB, IDX>(x + L.off[1] + o, b + L.off[1] + o, nx, vz, pc, pp[-nx], K);
    }
    {
        const IDX o = ci + nx * cj + wz * ck;
        if (k >= 2 && (!fl || (fl[L.off[2] + o] & kFlagV2)))
            dgs_face<T, TB, IDX>(x + L.off[2] + o, b + L.off[2] + o, nx, wz, pc, pp[-wz], K);
    }
}

template <class T, class TB> void launch_dgs_u(const Lev &L, T *x, const TB *b, int parity, cudaStream_t s) {
    if (L.nx < 3 || L.ny < 3 || L.nz < 3) return;
    dim3 grid(cdiv((L.nx - 2 + 1) / 2, BX), cdiv(L.ny - 2, BY), (L.nz - 2) * L.nb);
    if (idx32(L)) launch_k(BSEL(L.nb, k_dgs_u<T, TB, int), dim3(grid), dim3(kBlock3), 0, s, L, x, b, parity, coef<T>(L, L.gamma));
    else launch_k(BSEL(L.nb, k_dgs_u<T, TB, long long), dim3(grid), dim3(kBlock3), 0, s, L, x, b, parity, coef<T>(L, L.gamma));
}

// ------------------------------------------------------------------------------------------
// The velocity block of Alg. 2 / Eq. ldist, both parities in one pass, out of place (X read, Y
// written).  Phase A relaxes the V2 faces of parity pa from X, phase B those of parity 1 - pa from
// the phase-A values -- the two in-place launches of k_dgs_u, the same arithmetic per face.
// A block is a window of FW x FH cell positions, one thread each, marching a chunk of planes in z;
// it writes the entries of the inner FTX x FTY tile (a two-position halo on every side).  The planes
// of X (u v w p) and of b stream into a ring of FNS shared-memory slots with asynchronous copies issued
// FP planes ahead, so several planes of loads are in flight while the block computes.  At step k the
// block relaxes phase A at plane k + 1 on the tile and a one-position ring (neighbours from the slots
// of planes k, k + 1, k + 2), then phase B at plane k on the tile (in-plane phase-A neighbours from
// shared memory, the z neighbours' phase-A values from the thread's own registers) and writes the
// tile's entries of Y at plane k.  The ring's phase-A values are recomputed by the neighbouring blocks
// too (overlapped tiling), so no block waits for another; one barrier per plane.  Every packed entry of
// Y is written once: an updated face, or X's value.
constexpr int FW = 32, FH = 16;            // window (threads) of one block
constexpr int FTX = FW - 4, FTY = FH - 4;  // tile written by the block
constexpr int FZMAX = 32;                  // planes per block at most
constexpr int FP = 4;                      // planes copied ahead
constexpr int FNS = FP + 2;                // plane slots: planes k - 1 .. k + FP are distinct

template <class T> struct DgsFusedSmem {
    T x[FNS][4][FH][FW];  // [plane slot][component u v w p][y][x]
    T b[FNS][3][FH][FW];  // [plane slot][component u v w][y][x]
    T a[2][3][FH][FW];    // phase-A values: [plane slot][component u v w][y][x]
};

// asynchronous copy of one N-byte value into shared memory (zero-filled when !valid; nothing is read)
template <int N> __device__ __forceinline__ void cp_async_n(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(N), "r"(valid ? N : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// is face (c; i, j, k) a V2 face (relaxed by the DGS)?  i, j, k inside the component's array
__device__ __forceinline__ bool dgs_v2_face(const Lev &L, int c, int i, int j, int k, long long q) {
    const int n[3] = {L.nx, L.ny, L.nz}, id[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int lo = d == c ? 2 : 1, hi = n[d] - 2;
        if (id[d] < lo || id[d] > hi) return false;
    }
    return !L.flags || (L.flags[q] & kFlagV2);
}

template <class T, class TB, class IDX>
__global__ void __launch_bounds__(FW * FH, sizeof(T) == 4 ? 2 : 1)
    k_dgs_u_fused(Lev L, const T *__restrict__ X, T *__restrict__ Y, const TB *__restrict__ b, int pa, int fz,
                  Coef<T> K) {
    extern __shared__ __align__(16) unsigned char fsm[];
    DgsFusedSmem<T> &S = *reinterpret_cast<DgsFusedSmem<T> *>(fsm);
    const int wx = threadIdx.x, wy = threadIdx.y;
    const int gi = (int)blockIdx.x * FTX - 2 + wx, gj = (int)blockIdx.y * FTY - 2 + wy;
    const int k0 = (int)blockIdx.z * fz, k1 = min(k0 + fz, L.nz + 1);  // phase B (and Y) at planes k0..k1-1
    const bool ring = wx >= 1 && wx <= FW - 2 && wy >= 1 && wy <= FH - 2;  // phase A here
    const bool tile = wx >= 2 && wx <= FW - 3 && wy >= 2 && wy <= FH - 3;  // phase B and Y here
    const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
    // this thread's column of each component: offset at plane 0, plane stride, planes, in the array
    IDX cb[4], cz[4];
    int ce[4];
    bool cv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const IDX syc = c == 0 ? nx + 1 : nx;
        cz[c] = c == 0 ? (nx + 1) * ny : (c == 1 ? nx * (ny + 1) : nx * ny);
        cv[c] = gi >= 0 && gj >= 0 && gi < L.nx + (c == 0) && gj < L.ny + (c == 1);
        cb[c] = cv[c] ? (IDX)gi + syc * (IDX)gj : (IDX)0;
        ce[c] = L.nz + (c == 2);
    }
    const T *Xc[4] = {X + L.off[0], X + L.off[1], X + L.off[2], X + L.off[3]};
    T *Yc[4] = {Y + L.off[0], Y + L.off[1], Y + L.off[2], Y + L.off[3]};
    const TB *Bc[3] = {b + L.off[0], b + L.off[1], b + L.off[2]};
    const int kb = k0 - 2;  // first plane staged; plane m lives in slot (m - kb) % FNS
    // copy this thread's entries of plane m (X, and b where phase A or B may relax) into its slot
    auto stage = [&](int m) {
        const int sl = (m - kb) % FNS;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool in = cv[c] && m >= 0 && m < ce[c];
            cp_async_n<sizeof(T)>(&S.x[sl][c][wy][wx], in ? Xc[c] + cb[c] + cz[c] * (IDX)m : Xc[c], in);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool in = ring && cv[c] && m >= 0 && m < ce[c];
            if constexpr (sizeof(TB) == sizeof(T))
                cp_async_n<sizeof(T)>(&S.b[sl][c][wy][wx], in ? (const void *)(Bc[c] + cb[c] + cz[c] * (IDX)m) : (const void *)Bc[c], in);
            else
                S.b[sl][c][wy][wx] = in ? T(ldv(Bc[c][cb[c] + cz[c] * (IDX)m])) : T(0);
        }
        cp_async_commit();
    };
    pdl_enter();
#pragma unroll 1
    for (int m = kb; m < kb + FP; ++m) stage(m);
    T pm1 = (cv[3] && kb - 1 >= 0) ? Xc[3][cb[3] + cz[3] * (IDX)(kb - 1)] : T(0);  // p at plane k - 1
    T am[3] = {T(0), T(0), T(0)}, a0[3] = {T(0), T(0), T(0)};                      // phase A at k - 1, k
#pragma unroll 1
    for (int k = kb, it = 0; k < k1; ++k, ++it) {
        stage(k + FP);
        cp_async_wait<FP - 2>();  // planes up to k + 2 have landed (this thread's copies)
        __syncthreads();          // ... and every thread's
        const int s0 = it % FNS, s1 = (it + 1) % FNS, s2 = (it + 2) % FNS, a1s = (it + 1) & 1, a0s = it & 1;
        // phase A at plane k + 1 (tile and ring)
        const int kp = k + 1;
        const bool parA = ((gi + gj + kp) & 1) == pa;
        T an[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T v = S.x[s1][c][wy][wx];
            if (ring && parA && cv[c] && kp >= 0 && kp < ce[c] &&
                dgs_v2_face(L, c, gi, gj, kp, L.off[c] + cb[c] + cz[c] * (IDX)kp)) {
                const T pmv = c == 0 ? S.x[s1][3][wy][wx - 1] : (c == 1 ? S.x[s1][3][wy - 1][wx] : S.x[s0][3][wy][wx]);
                v = dgs_relax<T>(v, S.x[s1][c][wy][wx - 1], S.x[s1][c][wy][wx + 1], S.x[s1][c][wy - 1][wx],
                                 S.x[s1][c][wy + 1][wx], S.x[s0][c][wy][wx], S.x[s2][c][wy][wx], S.x[s1][3][wy][wx],
                                 pmv, S.b[s1][c][wy][wx], K);
            }
            an[c] = v;
            S.a[a1s][c][wy][wx] = v;
        }
        // phase B at plane k (tile), from the phase-A values of planes k - 1, k, k + 1; Y at plane k
        const T pc = S.x[s0][3][wy][wx];
        if (tile && k >= k0) {
            const bool parB = ((gi + gj + k) & 1) == pa;  // these faces keep their phase-A value
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!cv[c] || k >= ce[c]) continue;
                const IDX o = cb[c] + cz[c] * (IDX)k;
                const T x0 = S.x[s0][c][wy][wx];
                T v = x0;
                if (parB) {
                    v = a0[c];
                } else if (dgs_v2_face(L, c, gi, gj, k, L.off[c] + o)) {
                    const T pmv = c == 0 ? S.x[s0][3][wy][wx - 1] : (c == 1 ? S.x[s0][3][wy - 1][wx] : pm1);
                    v = dgs_relax<T>(x0, S.a[a0s][c][wy][wx - 1], S.a[a0s][c][wy][wx + 1], S.a[a0s][c][wy - 1][wx],
                                     S.a[a0s][c][wy + 1][wx], am[c], an[c], pc, pmv, S.b[s0][c][wy][wx], K);
                }
                Yc[c][o] = v;
            }
            if (cv[3] && k < ce[3]) Yc[3][cb[3] + cz[3] * (IDX)k] = pc;
        }
        pm1 = pc;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            am[c] = a0[c];
            a0[c] = an[c];
        }
    }
    cp_async_wait<0>();  // no copy outlives the block
}

template <class T, class TB> size_t dgs_u_fused_smem() { return sizeof(DgsFusedSmem<T>); }

// the shared-memory opt-in of the fused kernel, set once outside any capture
template <class T, class TB> bool dgs_u_fused_prepare() {
    return cudaFuncSetAttribute(k_dgs_u_fused<T, TB, int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(DgsFusedSmem<T>)) == cudaSuccess &&
           cudaFuncSetAttribute(k_dgs_u_fused<T, TB, long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(DgsFusedSmem<T>)) == cudaSuccess;
}

template <class T, class TB>
void launch_dgs_u_fused(const Lev &L, const T *X, T *Y, const TB *b, int pa, cudaStream_t s) {
    // z chunks of at most FZMAX planes, as even as possible (every chunk re-reads two planes either side)
    const int nch = cdiv(L.nz + 1, FZMAX), fz = cdiv(L.nz + 1, nch);
    dim3 grid(cdiv(L.nx + 1, FTX), cdiv(L.ny + 1, FTY), cdiv(L.nz + 1, fz));
    if (idx32(L))
        launch_k(k_dgs_u_fused<T, TB, int>, grid, dim3(FW, FH, 1), sizeof(DgsFusedSmem<T>), s, L, X, Y, b, pa, fz,
                 coef<T>(L, L.gamma));
    else
        launch_k(k_dgs_u_fused<T, TB, long long>, grid, dim3(FW, FH, 1), sizeof(DgsFusedSmem<T>), s, L, X, Y, b, pa, fz,
                 coef<T>(L, L.gamma));
}

// Alg. 2 pressure block, one colour (i mod 2, j mod 2, k mod 2):
//   r = b_c - (L~x)_c,  delta = r / d,  d = L~_c . M_{.c} = -6 (1 + gamma eta)/h^2,
//   x += delta M_{.c}:  low faces -= delta/h, high faces += delta/h, p_c += 6 eta/h^2 delta,
//                       p of the 6 neighbours -= eta/h^2 delta.
// The neighbour-pressure part is applied in gather form: a cell first collects the deltas of
// neighbours whose colour came earlier in this sweep (pre-gather); k_dgs_p_gather applies the rest
// after the last colour.  delta is stored per cell and stays 0 outside V2.
template <class T, class TB, class IDX>
__device__ __forceinline__ void p_fwd_cell(const Lev &L, T *__restrict__ x, const TB *__restrict__ b,
                                           T *__restrict__ delta, int colour, IDX i, IDX j, IDX k, const Coef<T> &K,
                                           T dP) {
    const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
    const IDX sy = nx, sz = nx * ny;
    const IDX cl = i + nx * (j + ny * k);
    if (L.flags && !(L.flags[L.off[3] + cl] & kFlagV2)) return;  // label domains: V2 cells only
    T *dc = delta + cl;
    T g = T(0);
    if (colour & 1) g += dc[-1] + dc[1];
    if (colour & 2) g += dc[-sy] + dc[sy];
    if (colour & 4) g += dc[-sz] + dc[sz];
    T *pp = x + L.off[3] + cl;
    const T p = pp[0] - K.eh2 * g;
    T *u = x + L.off[0] + (i + (nx + 1) * (j + ny * k));
    T *v = x + L.off[1] + (i + nx * (j + (ny + 1) * k));
    T *w = x + L.off[2] + (i + nx * (j + ny * k));
    const T div = (u[1] - u[0]) + (v[sy] - v[0]) + (w[sz] - w[0]);
    const T r = T(ldv(b[L.off[3] + cl])) + K.ih * div + K.gam * p;
    const T dl = r / dP;
    const T fd = dl * K.ih;
    u[0] -= fd;
    u[1] += fd;
    v[0] -= fd;
    v[sy] += fd;
    w[0] -= fd;
    w[sz] += fd;
    pp[0] = p + T(6) * K.eh2 * dl;
    dc[0] = dl;
}
template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256) k_dgs_p_fwd(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                   T *__restrict__ delta, int colour, Coef<T> K, T dP) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) delta = bslot(delta, L.bstride, zs.p);
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    const int ti = blockIdx.x * BX + threadIdx.x, tj = blockIdx.y * BY + threadIdx.y, tk = zs.z;
    if (ti >= cnt[0] || tj >= cnt[1] || tk >= cnt[2]) return;
    p_fwd_cell<T, TB, IDX>(L, x, b, delta, colour, (IDX)(lo[0] + 2 * ti), (IDX)(lo[1] + 2 * tj), (IDX)(lo[2] + 2 * tk),
                           K, dP);
}
// Two colours that differ in the i bit only (c, then c ^ 1) in one launch.  A cell of colour c ^ 1
// reads what colour c wrote only in its own x-row: its two x-faces, written by the colour-c cells
// on either side, and their deltas; its y- and z-faces and the deltas of its y/z neighbours belong
// to colours whose j or k bit differs.  One block holds whole x-rows (thread x = cell along the
// row), so a __syncthreads orders the two colours.
template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(512) k_dgs_p_fwd_pair(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                        T *__restrict__ delta, int colour, Coef<T> K, T dP) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) delta = bslot(delta, L.bstride, zs.p);
    int lo[3], cnt[3], lo2[3], cnt2[3];
    v2_colour_range(L, colour, lo, cnt);
    v2_colour_range(L, colour ^ 1, lo2, cnt2);  // same j and k ranges
    const int ti = threadIdx.x, tj = blockIdx.y * blockDim.y + threadIdx.y, tk = zs.z;
    const bool row = tj < cnt[1] && tk < cnt[2];
    const IDX j = (IDX)(lo[1] + 2 * tj), k = (IDX)(lo[2] + 2 * tk);
    if (row && ti < cnt[0]) p_fwd_cell<T, TB, IDX>(L, x, b, delta, colour, (IDX)(lo[0] + 2 * ti), j, k, K, dP);
    __syncthreads();
    if (row && ti < cnt2[0]) p_fwd_cell<T, TB, IDX>(L, x, b, delta, colour ^ 1, (IDX)(lo2[0] + 2 * ti), j, k, K, dP);
}

template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_dgs_p_gather(Lev L, T *__restrict__ x, const T *__restrict__ delta,
                                                      Coef<T> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) delta = bslot(delta, L.bstride, zs.p);
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = zs.z;
    if (i >= L.nx || j >= L.ny || k >= L.nz) return;
    long long t = cell_lin(L, i, j, k);
    bool v2 = in_v2_cell(L, i, j, k);
    int colour = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    long long sy = L.nx, sz = (long long)L.nx * L.ny;
    T g = T(0);
    if (!v2 || !(colour & 1)) {
        if (i > 0) g += delta[t - 1];
        if (i < L.nx - 1) g += delta[t + 1];
    }
    if (!v2 || !(colour & 2)) {
        if (j > 0) g += delta[t - sy];
        if (j < L.ny - 1) g += delta[t + sy];
    }
    if (!v2 || !(colour & 4)) {
        if (k > 0) g += delta[t - sz];
        if (k < L.nz - 1) g += delta[t + sz];
    }
    if (g != T(0)) x[L.off[3] + t] -= K.eh2 * g;
}

// Eq. (ldist) backward sweep, pressure block.  Only pressures change during its colours, so the
// parts of the residual that do not depend on p are computed once (k_dgs_p_bwd_prep):
//   g_f = b_f - (A u)_f on every unknown face,   h_c = b_c - (B u)_c on every cell,
// and a colour then needs r_f = g_f - (p_plus - p_minus)/h and r_n = h_n + gamma p_n only:
//   p_c += [ sum_axes (r_high_face - r_low_face)/h + eta/h^2 (6 r_c - sum of the 6 neighbour r) ] / d
// (M_{.c}^T r with the full column of M).  Same-colour cells read none of each other's values.
// The same launch also finishes the forward sweep: the neighbour-pressure part of the last
// colours (gather form of k_dgs_p_gather), which the prep never reads.  One entry per thread as k_apply.
template <class T, class TB, int C, class IDX>
__device__ __forceinline__ void prep_entry(const Lev &L, T *__restrict__ x, const TB *__restrict__ b,
                                           TB *__restrict__ gh, const T *__restrict__ delta, const Coef<T> &K, int i,
                                           int j, int k) {
    if (!entry_exists<C>(L, i, j, k)) return;
    const long long q = entry_index<C, IDX>(L, i, j, k);
    T v = T(0);
    if (entry_unknown<C>(L, i, j, k, q)) v = T(ldv(b[q])) - row_at<T, C, false, IDX>(x, L, i, j, k, K);
    gh[q] = cvt<TB>(v);
    if (C == 3 && delta) {
        const IDX sy = (IDX)L.nx, sz = sy * (IDX)L.ny;
        const T *dc = delta + ((IDX)i + sy * (IDX)j + sz * (IDX)k);
        const bool v2 = in_v2_cell(L, i, j, k);
        const int colour = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
        T g = T(0);
        if (!v2 || !(colour & 1)) g += (i > 0 ? dc[-1] : T(0)) + (i < L.nx - 1 ? dc[1] : T(0));
        if (!v2 || !(colour & 2)) g += (j > 0 ? dc[-sy] : T(0)) + (j < L.ny - 1 ? dc[sy] : T(0));
        if (!v2 || !(colour & 4)) g += (k > 0 ? dc[-sz] : T(0)) + (k < L.nz - 1 ? dc[sz] : T(0));
        if (g != T(0)) x[q] -= K.eh2 * g;
    }
}

template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256, 8) k_dgs_p_bwd_prep(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                           TB *__restrict__ gh, const T *__restrict__ delta,
                                                           Coef<T> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) gh = bslot(gh, L.bstride, zs.p);
    if constexpr (BATCH) delta = bslot(delta, L.bstride, zs.p);
    const int c = zs.z & 3, k = zs.z >> 2;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: prep_entry<T, TB, 0, IDX>(L, x, b, gh, delta, K, i, j, k); break;
    case 1: prep_entry<T, TB, 1, IDX>(L, x, b, gh, delta, K, i, j, k); break;
    case 2: prep_entry<T, TB, 2, IDX>(L, x, b, gh, delta, K, i, j, k); break;
    default: prep_entry<T, TB, 3, IDX>(L, x, b, gh, delta, K, i, j, k);
    }
}

// ---- the residual and the backward-DGS prep, four entries per thread along x ----
// Both are bound by instruction issue with one entry per thread.  On the box (no label flags) with
// nx % 4 == 0 the rows of v, w and p start on 4-entry boundaries, so a thread takes four consecutive
// entries with 16-byte loads of the centre and of the y/z neighbour rows and two scalar loads for
// the x neighbours; index math and guards are paid once per four entries.  Each entry's arithmetic
// is the one-entry code's,
// in the same order.  The u rows (nx + 1 entries, not 4-aligned) take four entries per thread too,
// with scalar loads.
template <class T> struct V4 {
    T v[4];
};
template <class T> __device__ __forceinline__ V4<T> ld4(const T *p);
template <> __device__ __forceinline__ V4<float> ld4<float>(const float *p) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    return {{a.x, a.y, a.z, a.w}};
}
template <> __device__ __forceinline__ V4<double> ld4<double>(const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], c = reinterpret_cast<const double2 *>(p)[1];
    return {{a.x, a.y, c.x, c.y}};
}
template <> __device__ __forceinline__ V4<bf16> ld4<bf16>(const bf16 *p) {
    const __nv_bfloat162 a = reinterpret_cast<const __nv_bfloat162 *>(p)[0];
    const __nv_bfloat162 c = reinterpret_cast<const __nv_bfloat162 *>(p)[1];
    return {{a.x, a.y, c.x, c.y}};
}
template <class D, class T> __device__ __forceinline__ void st4(D *p, const T (&a)[4]) {
    if constexpr (sizeof(D) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(cvt<float>(a[0]), cvt<float>(a[1]), cvt<float>(a[2]), cvt<float>(a[3]));
    } else if constexpr (sizeof(D) == 8) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(cvt<double>(a[0]), cvt<double>(a[1]));
        reinterpret_cast<double2 *>(p)[1] = make_double2(cvt<double>(a[2]), cvt<double>(a[3]));
    } else {
        __nv_bfloat162 lo, hi;
        lo.x = cvt<bf16>(a[0]);
        lo.y = cvt<bf16>(a[1]);
        hi.x = cvt<bf16>(a[2]);
        hi.y = cvt<bf16>(a[3]);
        reinterpret_cast<__nv_bfloat162 *>(p)[0] = lo;
        reinterpret_cast<__nv_bfloat162 *>(p)[1] = hi;
    }
}
template <class T> __device__ __forceinline__ V4<T> zero4() { return {{T(0), T(0), T(0), T(0)}}; }

// rows of four consecutive entries i0..i0+3 of component C (1, 2: faces; 3: cells) at (j, k); P adds
// the pressure gradient / -gamma p as in row_at
template <class T, int C, bool P, class IDX>
__device__ __forceinline__ void rows4(const T *__restrict__ x, const Lev &L, int i0, int j, int k, const Coef<T> &K,
                                      T (&out)[4]) {
    const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
    if constexpr (C < 3) {
        const IDX sy = nx, sz = sy * (ny + (C == 1));
        const T *xc = x + L.off[C] + ((IDX)i0 + sy * (IDX)j + sz * (IDX)k);
        const V4<T> c = ld4(xc);
        const T xl = i0 > 0 ? xc[-1] : T(0), xr = i0 + 4 < L.nx ? xc[4] : T(0);
        const V4<T> ym = (C == 1 || j > 0) ? ld4(xc - sy) : zero4<T>();
        const V4<T> yp = (C == 1 || j < L.ny - 1) ? ld4(xc + sy) : zero4<T>();
        const V4<T> zm = (C == 2 || k > 0) ? ld4(xc - sz) : zero4<T>();
        const V4<T> zp = (C == 2 || k < L.nz - 1) ? ld4(xc + sz) : zero4<T>();
        V4<T> pc, pm;
        if constexpr (P) {
            const IDX cy = nx, cz = cy * ny;
            const T *pp = x + L.off[3] + ((IDX)i0 + cy * (IDX)j + cz * (IDX)k);
            pc = ld4(pp);
            pm = ld4(pp - (C == 1 ? cy : cz));
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const T lft = e == 0 ? xl : c.v[e - 1], rgt = e == 3 ? xr : c.v[e + 1];
            T s = T(6) * c.v[e];
            s -= lft + rgt;
            s -= ym.v[e] + yp.v[e];
            s -= zm.v[e] + zp.v[e];
            if constexpr (P) out[e] = K.eh2 * s + K.ih * (pc.v[e] - pm.v[e]);
            else out[e] = K.eh2 * s;
        }
    } else {
        const T *u = x + L.off[0] + ((IDX)i0 + (nx + 1) * ((IDX)j + ny * (IDX)k));
        const T *v = x + L.off[1] + ((IDX)i0 + nx * ((IDX)j + (ny + 1) * (IDX)k));
        const T *w = x + L.off[2] + ((IDX)i0 + nx * ((IDX)j + ny * (IDX)k));
        T uu[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) uu[e] = u[e];
        const V4<T> v0 = ld4(v), v1 = ld4(v + nx), w0 = ld4(w), w1 = ld4(w + nx * ny);
        V4<T> pc;
        if constexpr (P) pc = ld4(x + L.off[3] + ((IDX)i0 + nx * ((IDX)j + ny * (IDX)k)));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const T div = (uu[e + 1] - uu[e]) + (v1.v[e] - v0.v[e]) + (w1.v[e] - w0.v[e]);
            if constexpr (P) out[e] = -K.ih * div - K.gam * pc.v[e];
            else out[e] = -K.ih * div;
        }
    }
}

// u rows (nx + 1 entries, not aligned): four consecutive entries i0..i0+3 with scalar loads; e_ok[e]
// says whether entry i0 + e exists (i <= nx), act[e] whether it is an unknown (1 <= i <= nx - 1)
template <class T, bool P, class IDX>
__device__ __forceinline__ void rows4u(const T *__restrict__ x, const Lev &L, int i0, int j, int k, const Coef<T> &K,
                                       T (&out)[4]) {
    const IDX sy = (IDX)(L.nx + 1), sz = sy * (IDX)L.ny;
    const T *xc = x + L.off[0] + ((IDX)i0 + sy * (IDX)j + sz * (IDX)k);
    T c[6];  // entries i0 - 1 .. i0 + 4 of the row, 0 outside it
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int i = i0 - 1 + e;
        c[e] = (i >= 0 && i <= L.nx) ? xc[e - 1] : T(0);
    }
    const bool ym = j > 0, yp = j < L.ny - 1, zm = k > 0, zp = k < L.nz - 1;
    const IDX cy = (IDX)L.nx, cz = cy * (IDX)L.ny;
    const T *pc = x + L.off[3] + ((IDX)i0 + cy * (IDX)j + cz * (IDX)k);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = i0 + e;
        out[e] = T(0);
        if (i < 1 || i > L.nx - 1) continue;
        T s = T(6) * c[e + 1];
        s -= c[e] + c[e + 2];
        s -= (ym ? xc[e - sy] : T(0)) + (yp ? xc[e + sy] : T(0));
        s -= (zm ? xc[e - sz] : T(0)) + (zp ? xc[e + sz] : T(0));
        if constexpr (P) out[e] = K.eh2 * s + K.ih * (pc[e] - pc[e - 1]);
        else out[e] = K.eh2 * s;
    }
}

// launch shape of the four-per-thread kernels: the component in the low two bits of blockIdx.z as in
// the one-entry kernels; x tiles cover the longest row (u, nx + 1 entries) in groups of four
inline dim3 grid4(const Lev &L) { return dim3(cdiv(L.nx + 1, 4 * BX), cdiv(L.ny + 1, BY), 4 * (L.nz + 1) * L.nb); }
// box only (no label flags), rows of v, w, p on 4-entry boundaries (nx % 4 == 0 and the v block at a
// multiple of 4), and every array 16-byte aligned
inline bool al16(const void *p) { return ((uintptr_t)p & 15) == 0; }
inline bool use_x4(const Lev &L, const void *a, const void *b, const void *c, const void *d = nullptr) {
    return !L.flags && L.nx >= 4 && L.nx % 4 == 0 && L.off[1] % 4 == 0 && al16(a) && al16(b) && al16(c) && al16(d);
}
// u entries i0..i0+3 (those that exist): one-entry semantics with four entries per thread
template <class T, class TB, class IDX>
__device__ __forceinline__ void apply_u4(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                         TB *__restrict__ y, const Coef<T> &K, int i0, int j, int k) {
    if (i0 > L.nx || j >= L.ny || k >= L.nz) return;
    const long long q = entry_index<0, IDX>(L, i0, j, k);
    T v[4];
    rows4u<T, true, IDX>(x, L, i0, j, k, K, v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = i0 + e;
        if (i > L.nx) break;
        T r = v[e];
        if (b && i >= 1 && i <= L.nx - 1) r = T(ldv(b[q + e])) - r;
        y[q + e] = cvt<TB>(r);
    }
}
template <class T, class TB, int C, class IDX>
__device__ __forceinline__ void apply_entry4(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                             TB *__restrict__ y, const Coef<T> &K, int i0, int j, int k) {
    if (i0 >= L.nx || j >= L.ny + (C == 1) || k >= L.nz + (C == 2)) return;
    const long long q = entry_index<C, IDX>(L, i0, j, k);
    T v[4] = {T(0), T(0), T(0), T(0)};
    if (entry_active<C>(L, 0, j, k)) {  // the activity of v, w and p rows does not depend on i
        rows4<T, C, true, IDX>(x, L, i0, j, k, K, v);
        if (b) {
            const V4<TB> bv = ld4(b + q);
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = T(ldv(bv.v[e])) - v[e];
        }
    }
    st4(y + q, v);
}
template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256, 8) k_apply4(Lev L, const T *__restrict__ x, const TB *__restrict__ b,
                                                   TB *__restrict__ y, Coef<T> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) y = bslot(y, L.bstride, zs.p);
    const int c = zs.z & 3, k = zs.z >> 2;
    const int i = 4 * (blockIdx.x * BX + threadIdx.x), j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: apply_u4<T, TB, IDX>(L, x, b, y, K, i, j, k); break;
    case 1: apply_entry4<T, TB, 1, IDX>(L, x, b, y, K, i, j, k); break;
    case 2: apply_entry4<T, TB, 2, IDX>(L, x, b, y, K, i, j, k); break;
    default: apply_entry4<T, TB, 3, IDX>(L, x, b, y, K, i, j, k);
    }
}

template <class T, class TB, class IDX>
__device__ __forceinline__ void prep_u4(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                        TB *__restrict__ gh, const Coef<T> &K, int i0, int j, int k) {
    if (i0 > L.nx || j >= L.ny || k >= L.nz) return;
    const long long q = entry_index<0, IDX>(L, i0, j, k);
    T v[4];
    rows4u<T, false, IDX>(x, L, i0, j, k, K, v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = i0 + e;
        if (i > L.nx) break;
        gh[q + e] = cvt<TB>(i >= 1 && i <= L.nx - 1 ? T(ldv(b[q + e])) - v[e] : T(0));
    }
}
template <class T, class TB, int C, class IDX>
__device__ __forceinline__ void prep_entry4(const Lev &L, T *__restrict__ x, const TB *__restrict__ b,
                                            TB *__restrict__ gh, const T *__restrict__ delta, const Coef<T> &K, int i0,
                                            int j, int k) {
    if (i0 >= L.nx || j >= L.ny + (C == 1) || k >= L.nz + (C == 2)) return;
    const long long q = entry_index<C, IDX>(L, i0, j, k);
    T v[4] = {T(0), T(0), T(0), T(0)};
    if (entry_active<C>(L, 0, j, k)) {
        rows4<T, C, false, IDX>(x, L, i0, j, k, K, v);
        const V4<TB> bv = ld4(b + q);
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = T(ldv(bv.v[e])) - v[e];
    }
    st4(gh + q, v);
    if (C == 3 && delta) {
        // the forward sweep's pending neighbour-pressure part (gather form), as in prep_entry
        const IDX sy = (IDX)L.nx, sz = sy * (IDX)L.ny;
        const T *dc = delta + ((IDX)i0 + sy * (IDX)j + sz * (IDX)k);
        const V4<T> d0 = ld4(dc);
        const T dl = i0 > 0 ? dc[-1] : T(0), dr = i0 + 4 < L.nx ? dc[4] : T(0);
        const V4<T> dym = j > 0 ? ld4(dc - sy) : zero4<T>(), dyp = j < L.ny - 1 ? ld4(dc + sy) : zero4<T>();
        const V4<T> dzm = k > 0 ? ld4(dc - sz) : zero4<T>(), dzp = k < L.nz - 1 ? ld4(dc + sz) : zero4<T>();
        const bool v2jk = j >= 1 && k >= 1 && j <= L.ny - 2 && k <= L.nz - 2;
        T *xp = x + q;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = i0 + e;
            const bool v2 = v2jk && i >= 1 && i <= L.nx - 2;
            const int colour = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
            T g = T(0);
            if (!v2 || !(colour & 1)) g += (e == 0 ? dl : d0.v[e - 1]) + (e == 3 ? dr : d0.v[e + 1]);
            if (!v2 || !(colour & 2)) g += dym.v[e] + dyp.v[e];
            if (!v2 || !(colour & 4)) g += dzm.v[e] + dzp.v[e];
            if (g != T(0)) xp[e] -= K.eh2 * g;
        }
    }
}
template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256, 8) k_dgs_p_bwd_prep4(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                            TB *__restrict__ gh, const T *__restrict__ delta,
                                                            Coef<T> K) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) b = bslot(b, L.bstride, zs.p);
    if constexpr (BATCH) gh = bslot(gh, L.bstride, zs.p);
    if constexpr (BATCH) delta = bslot(delta, L.bstride, zs.p);
    const int c = zs.z & 3, k = zs.z >> 2;
    const int i = 4 * (blockIdx.x * BX + threadIdx.x), j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: prep_u4<T, TB, IDX>(L, x, b, gh, K, i, j, k); break;
    case 1: prep_entry4<T, TB, 1, IDX>(L, x, b, gh, delta, K, i, j, k); break;
    case 2: prep_entry4<T, TB, 2, IDX>(L, x, b, gh, delta, K, i, j, k); break;
    default: prep_entry4<T, TB, 3, IDX>(L, x, b, gh, delta, K, i, j, k);
    }
}

template <class T, class TB, class IDX>
__device__ __forceinline__ void p_bwd_cell(const Lev &L, T *__restrict__ x, const TB *__restrict__ ghs, IDX i, IDX j,
                                           IDX k, const Coef<T> &K, T dP) {
    const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
    const IDX sy = nx, sz = nx * ny;
    const IDX cl = i + nx * (j + ny * k);
    if (L.flags && !(L.flags[L.off[3] + cl] & kFlagV2)) return;  // label domains: V2 cells only
    T *pp = x + L.off[3] + cl;
    const T pc = pp[0], pxm = pp[-1], pxp = pp[1], pym = pp[-sy], pyp = pp[sy], pzm = pp[-sz], pzp = pp[sz];
    const TB *gc = ghs + L.off[3] + cl;
    const TB *gu = ghs + L.off[0] + (i + (nx + 1) * (j + ny * k));
    const TB *gv = ghs + L.off[1] + (i + nx * (j + (ny + 1) * k));
    const TB *gw = ghs + L.off[2] + (i + nx * (j + ny * k));
    auto G = [](TB v) { return T(ldv(v)); };
    // face residuals r_f = g_f - (p_plus - p_minus)/h
    const T rul = G(gu[0]) - K.ih * (pc - pxm), ruh = G(gu[1]) - K.ih * (pxp - pc);
    const T rvl = G(gv[0]) - K.ih * (pc - pym), rvh = G(gv[sy]) - K.ih * (pyp - pc);
    const T rwl = G(gw[0]) - K.ih * (pc - pzm), rwh = G(gw[sz]) - K.ih * (pzp - pc);
    // cell residuals r_n = h_n + gamma p_n
    const T rc = G(gc[0]) + K.gam * pc;
    const T rn = (G(gc[-1]) + K.gam * pxm) + (G(gc[1]) + K.gam * pxp) + (G(gc[-sy]) + K.gam * pym) +
                 (G(gc[sy]) + K.gam * pyp) + (G(gc[-sz]) + K.gam * pzm) + (G(gc[sz]) + K.gam * pzp);
    const T s = K.ih * ((ruh - rul) + (rvh - rvl) + (rwh - rwl)) + K.eh2 * (T(6) * rc - rn);
    pp[0] = pc + s / dP;
}
template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256) k_dgs_p_bwd(Lev L, T *__restrict__ x, const TB *__restrict__ ghs, int colour,
                                                   Coef<T> K, T dP) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) ghs = bslot(ghs, L.bstride, zs.p);
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    const int ti = blockIdx.x * BX + threadIdx.x, tj = blockIdx.y * BY + threadIdx.y, tk = zs.z;
    if (ti >= cnt[0] || tj >= cnt[1] || tk >= cnt[2]) return;
    p_bwd_cell<T, TB, IDX>(L, x, ghs, (IDX)(lo[0] + 2 * ti), (IDX)(lo[1] + 2 * tj), (IDX)(lo[2] + 2 * tk), K, dP);
}
// colours c and c ^ 1 of the backward pressure sweep in one launch: only pressures change, and a cell
// reads the pressures of the other colour of the pair only at its two x-neighbours (same x-row)
template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(512) k_dgs_p_bwd_pair(Lev L, T *__restrict__ x, const TB *__restrict__ ghs,
                                                        int colour, Coef<T> K, T dP) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(L) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) x = bslot(x, L.bstride, zs.p);
    if constexpr (BATCH) ghs = bslot(ghs, L.bstride, zs.p);
    int lo[3], cnt[3], lo2[3], cnt2[3];
    v2_colour_range(L, colour, lo, cnt);
    v2_colour_range(L, colour ^ 1, lo2, cnt2);
    const int ti = threadIdx.x, tj = blockIdx.y * blockDim.y + threadIdx.y, tk = zs.z;
    const bool row = tj < cnt[1] && tk < cnt[2];
    const IDX j = (IDX)(lo[1] + 2 * tj), k = (IDX)(lo[2] + 2 * tk);
    if (row && ti < cnt[0]) p_bwd_cell<T, TB, IDX>(L, x, ghs, (IDX)(lo[0] + 2 * ti), j, k, K, dP);
    __syncthreads();
    if (row && ti < cnt2[0]) p_bwd_cell<T, TB, IDX>(L, x, ghs, (IDX)(lo2[0] + 2 * ti), j, k, K, dP);
}

template <class T> static T dgs_pressure_diag(const Lev &L) {
    return T(-6.0 * (1.0 + L.gamma * L.eta) / (L.h * L.h));
}

template <class T, class TB>
void launch_dgs_p_fwd(const Lev &L, T *x, const TB *b, T *delta, int colour, cudaStream_t s) {
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    if ((long long)cnt[0] * cnt[1] * cnt[2] == 0) return;
    dim3 grid(cdiv(cnt[0], BX), cdiv(cnt[1], BY), cnt[2] * L.nb);
    if (idx32(L))
        launch_k(BSEL(L.nb, k_dgs_p_fwd<T, TB, int), dim3(grid), dim3(kBlock3), 0, s, L, x, b, delta, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
    else
        launch_k(BSEL(L.nb, k_dgs_p_fwd<T, TB, long long), dim3(grid), dim3(kBlock3), 0, s, L, x, b, delta, colour,
                 coef<T>(L, L.gamma), dgs_pressure_diag<T>(L));
}
// block shape of the colour-pair kernels: whole x-rows, rows stacked to about 256 threads; false if a
// row of one colour has more than 512 cells
inline bool pair_block(const Lev &L, int colour, dim3 &grid, dim3 &block) {
    int lo[3], cnt[3], lo2[3], cnt2[3];
    v2_colour_range(L, colour, lo, cnt);
    v2_colour_range(L, colour ^ 1, lo2, cnt2);
    const int rx = 32 * cdiv(cnt[0] > cnt2[0] ? cnt[0] : cnt2[0], 32);
    if (rx == 0 || rx > 512 || (long long)cnt[1] * cnt[2] == 0) return false;
    const int ry = rx >= 256 ? 1 : 256 / rx;
    block = dim3(rx, ry, 1);
    grid = dim3(1, cdiv(cnt[1], ry), cnt[2] * L.nb);
    return true;
}
template <class T, class TB>
bool launch_dgs_p_fwd_pair(const Lev &L, T *x, const TB *b, T *delta, int colour, cudaStream_t s) {
    dim3 grid, block;
    if (!pair_block(L, colour, grid, block)) return false;
    if (idx32(L))
        launch_k(BSEL(L.nb, k_dgs_p_fwd_pair<T, TB, int), grid, block, 0, s, L, x, b, delta, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
    else
        launch_k(BSEL(L.nb, k_dgs_p_fwd_pair<T, TB, long long), grid, block, 0, s, L, x, b, delta, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
    return true;
}
template <class T, class TB> bool launch_dgs_p_bwd_pair(const Lev &L, T *x, const TB *gh, int colour, cudaStream_t s) {
    dim3 grid, block;
    if (!pair_block(L, colour, grid, block)) return false;
    if (idx32(L))
        launch_k(BSEL(L.nb, k_dgs_p_bwd_pair<T, TB, int), grid, block, 0, s, L, x, gh, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
    else
        launch_k(BSEL(L.nb, k_dgs_p_bwd_pair<T, TB, long long), grid, block, 0, s, L, x, gh, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
    return true;
}
template <class T> void launch_dgs_p_gather(const Lev &L, T *x, const T *delta, cudaStream_t s) {
    dim3 grid(cdiv(L.nx, BX), cdiv(L.ny, BY), L.nz * L.nb);
    launch_k(BSEL(L.nb, k_dgs_p_gather<T), dim3(grid), dim3(kBlock3), 0, s, L, x, delta, coef<T>(L, L.gamma));
}
template <class T, class TB>
void launch_apply(const Lev &L, const T *x, const TB *b, TB *y, double gam, cudaStream_t s) {
    if (use_x4(L, x, b, y)) {
        if (idx32(L)) launch_k(BSEL(L.nb, k_apply4<T, TB, int), grid4(L), dim3(kBlock3), 0, s, L, x, b, y, coef<T>(L, gam));
        else launch_k(BSEL(L.nb, k_apply4<T, TB, long long), grid4(L), dim3(kBlock3), 0, s, L, x, b, y, coef<T>(L, gam));
        return;
    }
    if (idx32(L))
        launch_k(BSEL(L.nb, k_apply<T, TB, int), dim3(entry_grid(L)), dim3(kBlock3), 0, s, L, x, b, y, coef<T>(L, gam));
    else
        launch_k(BSEL(L.nb, k_apply<T, TB, long long), dim3(entry_grid(L)), dim3(kBlock3), 0, s, L, x, b, y, coef<T>(L, gam));
}
template <class T, class TB>
void launch_dgs_p_bwd_prep(const Lev &L, T *x, const TB *b, TB *gh, const T *delta, cudaStream_t s) {
    if (use_x4(L, x, b, gh, delta)) {
        if (idx32(L))
            launch_k(BSEL(L.nb, k_dgs_p_bwd_prep4<T, TB, int), grid4(L), dim3(kBlock3), 0, s, L, x, b, gh, delta, coef<T>(L, L.gamma));
        else
            launch_k(BSEL(L.nb, k_dgs_p_bwd_prep4<T, TB, long long), grid4(L), dim3(kBlock3), 0, s, L, x, b, gh, delta,
                     coef<T>(L, L.gamma));
        return;
    }
    if (idx32(L))
        launch_k(BSEL(L.nb, k_dgs_p_bwd_prep<T, TB, int), dim3(entry_grid(L)), dim3(kBlock3), 0, s, L, x, b, gh, delta,
                 coef<T>(L, L.gamma));
    else
        launch_k(BSEL(L.nb, k_dgs_p_bwd_prep<T, TB, long long), dim3(entry_grid(L)), dim3(kBlock3), 0, s, L, x, b, gh, delta,
                 coef<T>(L, L.gamma));
}
template <class T, class TB> void launch_dgs_p_bwd(const Lev &L, T *x, const TB *gh, int colour, cudaStream_t s) {
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    if ((long long)cnt[0] * cnt[1] * cnt[2] == 0) return;
    dim3 grid(cdiv(cnt[0], BX), cdiv(cnt[1], BY), cnt[2] * L.nb);
    if (idx32(L))
        launch_k(BSEL(L.nb, k_dgs_p_bwd<T, TB, int), dim3(grid), dim3(kBlock3), 0, s, L, x, gh, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
    else
        launch_k(BSEL(L.nb, k_dgs_p_bwd<T, TB, long long), dim3(grid), dim3(kBlock3), 0, s, L, x, gh, colour, coef<T>(L, L.gamma),
                 dgs_pressure_diag<T>(L));
}

// ------------------------------------------------------------------------------------------
// Vanka (Sec. 3.2): patch of cell c = its active faces [u_lo, u_hi, v_lo, v_hi, w_lo, w_hi] and
// p_c; correction = (C L~ C^T)^{-1} C (b - L~x) with the inverse of the cell's configuration
// (which faces are unknowns: 6-bit mask, 64 pre-factorised 7x7 inverses per level, Sec. 6).
// Corrections of one colour are computed from the pre-colour state, stored, then added.
// Cell lists hold packed coordinates i | j << 11 | k << 22.
__device__ __forceinline__ void unpack_cell(int w, int &i, int &j, int &k) {
    i = w & 2047;
    j = (w >> 11) & 2047;
    k = (w >> 22) & 1023;
}

// 8 lanes per cell: lane a < 6 owns face a of the patch, lane 6 the pressure, lane 7 idles; the
// 7 residuals are exchanged with width-8 shuffles and lane a forms row a of K^{-1} r.  The six face
// lanes run one code path with the component as data (strides, base and guards selected per lane),
// so a warp's four cells diverge only between face lanes and the pressure lane.
template <class T, class TB>
__device__ __forceinline__ T vanka_face_residual(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b, int a,
                                                 int i, int j, int k, const Coef<T> &K) {
    const int d = a >> 1, side = a & 1;
    const int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
    const long long nx = L.nx, ny = L.ny;
    const long long sy = nx + (d == 0), sz = sy * (ny + (d == 1));
    const long long q = (d == 0 ? L.off[0] : (d == 1 ? L.off[1] : L.off[2])) + fi + sy * fj + sz * fk;
    const T *xc = x + q;
    // neighbours along the face normal always exist (wall faces hold 0); tangential ones only inside
    const bool xm = d == 0 || fi > 0, xp = d == 0 || fi < L.nx - 1;
    const bool ym = d == 1 || fj > 0, yp = d == 1 || fj < L.ny - 1;
    const bool zm = d == 2 || fk > 0, zp = d == 2 || fk < L.nz - 1;
    T s = T(6) * xc[0];
    T xl = xm ? xc[-1] : T(0), xh = xp ? xc[1] : T(0), yl = ym ? xc[-sy] : T(0), yh = yp ? xc[sy] : T(0);
    T zl = zm ? xc[-sz] : T(0), zh = zp ? xc[sz] : T(0);
    if (L.flags) {
        // label domains: the dropped viscous terms of a face next to exterior cells (Sec. 5 reading)
        const uint8_t f = L.flags[q];
        s = diag_weight<T>(f) * xc[0];
        if (f & kFlagDropLo) (d == 0 ? xl : (d == 1 ? yl : zl)) = T(0);
        if (f & kFlagDropHi) (d == 0 ? xh : (d == 1 ? yh : zh)) = T(0);
    }
    s -= xl + xh;
    s -= yl + yh;
    s -= zl + zh;
    const T *pc = x + L.off[3] + (fi + nx * (fj + ny * fk));
    const long long ps = d == 0 ? 1 : (d == 1 ? nx : nx * ny);
    return T(ldv(b[q])) - (K.eh2 * s + K.ih * (pc[0] - pc[-ps]));
}

// the face-lane residual of vanka_face_residual and the pressure-lane residual of cell_Lx_fast with
// IDX-wide offsets (32-bit where the level allows): the same loads and the same arithmetic in the
// same order, fewer address instructions
template <class T, class TB, class IDX>
__device__ __forceinline__ T vanka_residual_idx(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b, int a,
                                                int i, int j, int k, const Coef<T> &K) {
    const IDX nx = (IDX)L.nx, ny = (IDX)L.ny;
    if (a == 6) {
        const IDX cl = (IDX)i + nx * ((IDX)j + ny * (IDX)k);
        const T *u = x + L.off[0] + ((IDX)i + (nx + 1) * ((IDX)j + ny * (IDX)k));
        const T *v = x + L.off[1] + ((IDX)i + nx * ((IDX)j + (ny + 1) * (IDX)k));
        const T *w = x + L.off[2] + cl;
        const T div = (u[1] - u[0]) + (v[nx] - v[0]) + (w[nx * ny] - w[0]);
        return T(ldv(b[L.off[3] + cl])) - (-K.ih * div - K.gam * x[L.off[3] + cl]);
    }
    const int d = a >> 1, side = a & 1;
    const int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
    const IDX sy = nx + (IDX)(d == 0), sz = sy * (ny + (IDX)(d == 1));
    const long long base = d == 0 ? L.off[0] : (d == 1 ? L.off[1] : L.off[2]);
    const IDX o = (IDX)fi + sy * (IDX)fj + sz * (IDX)fk;
    const T *xc = x + base + o;
    const bool xm = d == 0 || fi > 0, xp = d == 0 || fi < L.nx - 1;
    const bool ym = d == 1 || fj > 0, yp = d == 1 || fj < L.ny - 1;
    const bool zm = d == 2 || fk > 0, zp = d == 2 || fk < L.nz - 1;
    T s = T(6) * xc[0];
    T xl = xm ? xc[-1] : T(0), xh = xp ? xc[1] : T(0), yl = ym ? xc[-sy] : T(0), yh = yp ? xc[sy] : T(0);
    T zl = zm ? xc[-sz] : T(0), zh = zp ? xc[sz] : T(0);
    if (L.flags) {
        const uint8_t f = L.flags[base + o];
        s = diag_weight<T>(f) * xc[0];
        if (f & kFlagDropLo) (d == 0 ? xl : (d == 1 ? yl : zl)) = T(0);
        if (f & kFlagDropHi) (d == 0 ? xh : (d == 1 ? yh : zh)) = T(0);
    }
    s -= xl + xh;
    s -= yl + yh;
    s -= zl + zh;
    const T *pc = x + L.off[3] + ((IDX)fi + nx * ((IDX)fj + ny * (IDX)fk));
    const IDX ps = d == 0 ? (IDX)1 : (d == 1 ? nx : nx * ny);
    return T(ldv(b[base + o])) - (K.eh2 * s + K.ih * (pc[0] - pc[-ps]));
}

// the part of a Vanka lane that reads only the level's static data (cell list, label flags, inverse
// table): the cell, its 6-bit face configuration and where the lane's row of the local inverse lies.
// Nothing here is written during a solve, so kernels read it before waiting for the previous kernel.
template <class T> struct VankaLane {
    int i, j, k, cfg;
    const T *Ki;
};
template <class T>
__device__ __forceinline__ void vanka_lane_setup(const Lev &L, int cellw, int a, const T *__restrict__ kinv,
                                                 const int *__restrict__ tab, int slot, VankaLane<T> &v) {
    unpack_cell(cellw, v.i, v.j, v.k);
    const int i = v.i, j = v.j, k = v.k;
    // which of the cell's six faces are unknowns (6-bit configuration of the pre-factorised inverses);
    // on the box a face of a cell is one unless it lies on a wall
    v.cfg = L.flags ? ((int)unknown(L, 0, i, j, k) | ((int)unknown(L, 0, i + 1, j, k) << 1) |
                       ((int)unknown(L, 1, i, j, k) << 2) | ((int)unknown(L, 1, i, j + 1, k) << 3) |
                       ((int)unknown(L, 2, i, j, k) << 4) | ((int)unknown(L, 2, i, j, k + 1) << 5))
                    : ((int)(i > 0) | ((int)(i < L.nx - 1) << 1) | ((int)(j > 0) << 2) | ((int)(j < L.ny - 1) << 3) |
                       ((int)(k > 0) << 4) | ((int)(k < L.nz - 1) << 5));
    // label domains with exterior cells: the cell's own entry of the level's inverse table (its faces'
    // dropped terms change the local matrix); otherwise the 6-bit configuration indexes it
    const int id = tab ? tab[slot] : v.cfg;
    v.Ki = kinv + id * 49 + (a < 7 ? a : 6) * 7;
}
// the rest of the lane: its residual from the current state, row a of K^{-1} r, the stored correction
template <class T, class TB, class IDX>
__device__ __forceinline__ void vanka_lane_finish(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                                  const VankaLane<T> &v, int a, unsigned gmask, T *__restrict__ corr,
                                                  int cap, int slot, const Coef<T> &K, T w) {
    T r = T(0);
    if (a == 6 || (a < 6 && ((v.cfg >> a) & 1))) r = vanka_residual_idx<T, TB, IDX>(L, x, b, a, v.i, v.j, v.k, K);
    T s = T(0);
#pragma unroll
    for (int bb = 0; bb < 7; ++bb) s += v.Ki[bb] * __shfl_sync(gmask, r, bb, 8);
    if (a < 7) corr[(long long)a * cap + slot] = w * s;  // w = 1 (multiplicative) is exact
}
template <class T, class TB, class IDX = long long>
__device__ __forceinline__ void vanka_compute_lane(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                                   int cellw, int a, unsigned gmask, const T *__restrict__ kinv,
                                                   T *__restrict__ corr, int cap, int slot, const Coef<T> &K,
                                                   T w = T(1), const int *__restrict__ tab = nullptr) {
    VankaLane<T> v;
    vanka_lane_setup<T>(L, cellw, a, kinv, tab, slot, v);
    vanka_lane_finish<T, TB, IDX>(L, x, b, v, a, gmask, corr, cap, slot, K, w);
}

// the entry a Vanka lane updates (static: cell list and label flags); false for lane 7 and for faces that
// are not unknowns
__device__ __forceinline__ bool vanka_apply_target(const Lev &L, int cellw, int a, long long &q) {
    if (a == 7) return false;
    int i, j, k;
    unpack_cell(cellw, i, j, k);
    const long long nx = L.nx, ny = L.ny;
    if (a == 6) {
        q = L.off[3] + (i + nx * (j + ny * k));
        return true;
    }
    const int d = a >> 1, side = a & 1;
    const int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
    const long long sy = nx + (d == 0), sz = sy * (ny + (d == 1));
    q = (d == 0 ? L.off[0] : (d == 1 ? L.off[1] : L.off[2])) + fi + sy * fj + sz * fk;
    const int nrm = d == 0 ? fi : (d == 1 ? fj : fk), nn = d == 0 ? L.nx : (d == 1 ? L.ny : L.nz);
    return nrm >= 1 && nrm <= nn - 1 && (!L.flags || (L.flags[q] & kFlagActive));
}
template <class T>
__device__ __forceinline__ void vanka_apply_lane(const Lev &L, T *__restrict__ x, int cellw, int a,
                                                 const T *__restrict__ corr, int cap, int slot) {
    long long q;
    if (vanka_apply_target(L, cellw, a, q)) x[q] += corr[(long long)a * cap + slot];
}

template <class T, class TB, class IDX, bool BATCH>
__global__ void __launch_bounds__(256) k_vanka_compute(Lev L, const T *__restrict__ x, const TB *__restrict__ b,
                                                       const int *__restrict__ cells, const int *__restrict__ tab,
                                                       int ncell, const T *__restrict__ kinv, T *__restrict__ corr,
                                                       int cap, Coef<T> K, T w) {
    if constexpr (BATCH) x = bslot(x, L.bstride, (int)blockIdx.y);
    if constexpr (BATCH) b = bslot(b, L.bstride, (int)blockIdx.y);
    if constexpr (BATCH) corr = bslot(corr, L.bstride, (int)blockIdx.y);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = t >> 3, a = t & 7;
    if (slot >= ncell) return;  // whole 8-lane groups leave together
    // the static part (cell, configuration, inverse table entry) overlaps the previous kernel's tail
    VankaLane<T> v;
    vanka_lane_setup<T>(L, cells[slot], a, kinv, tab, slot, v);
    pdl_enter();
    vanka_lane_finish<T, TB, IDX>(L, x, b, v, a, 0xffu << (threadIdx.x & 24), corr, cap, slot, K, w);
}

template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_vanka_apply(Lev L, T *__restrict__ x, const int *__restrict__ cells,
                                                     int ncell, const T *__restrict__ corr, int cap) {
    if constexpr (BATCH) x = bslot(x, L.bstride, (int)blockIdx.y);
    if constexpr (BATCH) corr = bslot(corr, L.bstride, (int)blockIdx.y);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = t >> 3;
    long long q;
    if (slot >= ncell || !vanka_apply_target(L, cells[slot], t & 7, q)) return;  // static: before the wait
    pdl_enter();
    x[q] += corr[(long long)(t & 7) * cap + slot];
}

template <class T, class TB>
void launch_vanka_compute(const Lev &L, const T *x, const TB *b, const int *cells, const int *tab, int ncell,
                          const T *kinv, T *corr, int cap, double w, cudaStream_t s) {
    if (ncell <= 0) return;
    if (idx32(L))
        launch_k(BSEL(L.nb, k_vanka_compute<T, TB, int), dim3(cdiv(8LL * ncell, 256), L.nb), dim3(256), 0, s, L, x, b, cells, tab, ncell,
                 kinv, corr, cap, coef<T>(L, L.gamma), T(w));
    else
        launch_k(BSEL(L.nb, k_vanka_compute<T, TB, long long), dim3(cdiv(8LL * ncell, 256), L.nb), dim3(256), 0, s, L, x, b, cells, tab,
                 ncell, kinv, corr, cap, coef<T>(L, L.gamma), T(w));
}
template <class T>
void launch_vanka_apply(const Lev &L, T *x, const int *cells, int ncell, const T *corr, int cap, cudaStream_t s) {
    if (ncell <= 0) return;
    launch_k(BSEL(L.nb, k_vanka_apply<T), dim3(cdiv(8LL * ncell, 256), L.nb), dim3(256), 0, s, L, x, cells, ncell, corr, cap);
}

// ---- one launch per colour step: two copies of the level's Vanka state (ping-pong) ----
// Step t (colour c) reads the state R and writes W: every DOF of a colour-c patch gets R + its patch
// correction (computed from R, the pre-colour state, exactly as the two-launch form), and every DOF of a
// patch of the previous step's colour that no colour-c patch holds gets R's value; W already equals R
// everywhere else (it was the state of the step before, which differed from R only on the previous
// colour's patches).  So W is the post-colour state and no grid-wide order is needed inside the step.
// Same-colour patches share no DOF and a DOF of the previous colour's patch shared with a colour-c
// patch is written by the colour-c lane only, so every entry of W is written by at most one thread.
// Lane a of slot s does both: DOF a of the s-th colour-c patch and DOF a of the s-th patch of the previous
// colour, so a step has as many threads as the longer of the two cell lists.
// Both copies agree on the ring of V2 DOFs the patches read (k_vanka_shell_copy at the start of each
// sweep) and hold 0 off the unknowns.  An even number of steps (16 per symmetric sweep) returns the
// state to the level's own vector.
template <class T>
__device__ __forceinline__ bool vanka_dof(const Lev &L, int cellw, int a, long long &q, int &d) {
    int i, j, k;
    unpack_cell(cellw, i, j, k);
    const long long nx = L.nx, ny = L.ny;
    if (a == 6) {
        q = L.off[3] + (i + nx * (j + ny * k));
        d = -1;
        return true;
    }
    d = a >> 1;
    const int side = a & 1;
    const int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
    const long long sy = nx + (d == 0), sz = sy * (ny + (d == 1));
    q = (d == 0 ? L.off[0] : (d == 1 ? L.off[1] : L.off[2])) + fi + sy * fj + sz * fk;
    const int nrm = d == 0 ? fi : (d == 1 ? fj : fk), nn = d == 0 ? L.nx : (d == 1 ? L.ny : L.nz);
    return nrm >= 1 && nrm <= nn - 1 && (!L.flags || (L.flags[q] & kFlagActive));
}
// is the cell across face a of cell (i,j,k) a V1 cell of colour c?
__device__ __forceinline__ bool across_is_v1_of_colour(const Lev &L, int cellw, int a, int c) {
    int i, j, k;
    unpack_cell(cellw, i, j, k);
    const int d = a >> 1, sg = (a & 1) ? 1 : -1;
    const int ni = i + (d == 0 ? sg : 0), nj = j + (d == 1 ? sg : 0), nk = k + (d == 2 ? sg : 0);
    if (ni < 0 || nj < 0 || nk < 0 || ni >= L.nx || nj >= L.ny || nk >= L.nz) return false;
    const int col = (ni & 1) | ((nj & 1) << 1) | ((nk & 1) << 2);
    if (col != c) return false;
    if (L.flags) {
        const uint8_t f = L.flags[pidx(L, 3, ni, nj, nk)];
        return (f & kFlagActive) && !(f & kFlagV2);
    }
    return !v2_cell_at(L, ni, nj, nk);
}

template <class T, class TB, class IDX>
__global__ void __launch_bounds__(256) k_vanka_step(Lev L, const T *__restrict__ R, T *__restrict__ W,
                                                    const TB *__restrict__ b, const int *__restrict__ cells,
                                                    const int *__restrict__ tab, int ncell,
                                                    const int *__restrict__ pcells, int npcell, int colour,
                                                    const T *__restrict__ kinv, Coef<T> K) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = t >> 3, a = t & 7;
    // lane a of slot s also carries DOF a of the previous colour's s-th patch over from R, unless a colour-c
    // patch writes it (static: which entry, and whether it is carried)
    long long qc = 0;
    bool carry = false;
    if (slot < npcell && a != 7) {
        const int pw = pcells[slot];
        int dc;
        carry = vanka_dof<T>(L, pw, a, qc, dc) && !(dc >= 0 && across_is_v1_of_colour(L, pw, a, colour));
    }
    if (slot < ncell) {
        // the patch correction, as vanka_compute_lane, written as R + correction into W; the static part
        // (cell, configuration, inverse table entry, target entry) before the wait for the previous kernel
        const int cellw = cells[slot];
        VankaLane<T> v;
        vanka_lane_setup<T>(L, cellw, a, kinv, tab, slot, v);
        long long q;
        int d;
        const bool wr = a < 7 && vanka_dof<T>(L, cellw, a, q, d);
        pdl_enter();
        const T cval = carry ? R[qc] : T(0);
        T r = T(0);
        if (a == 6 || (a < 6 && ((v.cfg >> a) & 1))) r = vanka_residual_idx<T, TB, IDX>(L, R, b, a, v.i, v.j, v.k, K);
        const unsigned gmask = 0xffu << (threadIdx.x & 24);
        T sacc = T(0);
#pragma unroll
        for (int bb = 0; bb < 7; ++bb) sacc += v.Ki[bb] * __shfl_sync(gmask, r, bb, 8);
        if (wr) W[q] = R[q] + T(1) * sacc;
        if (carry) W[qc] = cval;
        return;
    }
    if (!carry) return;
    pdl_enter();
    W[qc] = R[qc];
}

// the second copy takes the level's current values on every DOF a Vanka patch reads or writes
template <class T>
__global__ void __launch_bounds__(256) k_vanka_shell_copy(const T *__restrict__ x, T *__restrict__ x2,
                                                          const int *__restrict__ list, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const int q = list[t];  // static list: read before the wait
        pdl_enter();
        x2[q] = x[q];
    }
}

template <class T, class TB>
void launch_vanka_pingpong(const Lev &L, T *x, T *x2, const TB *b, const VankaLists &lists, const int *shell,
                           int nshell, const T *kinv, int sweeps, cudaStream_t s) {
    const Coef<T> K = coef<T>(L, L.gamma);
    for (int sw = 0; sw < sweeps; ++sw) {
        if (nshell > 0)
            launch_k(k_vanka_shell_copy<T>, dim3(cdiv(nshell, 256)), dim3(256), 0, s, (const T *)x, x2, shell, nshell);
        int prev = -1;
        for (int t = 0; t < 16; ++t) {
            const int c = t < 8 ? t : 15 - t;
            const T *R = (t & 1) ? x2 : x;
            T *W = (t & 1) ? x : x2;
            const int nc = lists.count[c];
            const int np = (prev >= 0 && prev != c) ? lists.count[prev] : 0;
            const int *pc = prev >= 0 ? lists.cells[prev] : nullptr;
            const int ns = nc > np ? nc : np;  // slot s: patch s of colour c and patch s of the previous colour
            if (ns > 0) {
                if (idx32(L))
                    launch_k(k_vanka_step<T, TB, int>, dim3(cdiv(8LL * ns, 256)), dim3(256), 0, s, L, R, W, b,
                             lists.cells[c], lists.tab[c], nc, pc, np, c, kinv, K);
                else
                    launch_k(k_vanka_step<T, TB, long long>, dim3(cdiv(8LL * ns, 256)), dim3(256), 0, s, L, R, W, b,
                             lists.cells[c], lists.tab[c], nc, pc, np, c, kinv, K);
            }
            prev = c;
        }
    }
}

// ---- one cooperative launch per symmetric Vanka sweep ----
// grid-wide barrier: generation counter in global memory, bounded spin (see kernels.h)
__device__ __forceinline__ void grid_sync(GridBarrier *bar, unsigned nblocks, unsigned spin_limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &bar->gen;
        volatile int *verr = &bar->err;
        if (!*verr) {
            unsigned g = *vgen;
            __threadfence();
            if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
                atomicExch(&bar->count, 0u);
                __threadfence();
                atomicAdd(&bar->gen, 1u);
            } else {
                unsigned spins = 0;
                while (*vgen == g && !*verr) {
                    if (++spins > spin_limit) {
                        atomicExch(&bar->err, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
}

template <class T, class TB>
__global__ void __launch_bounds__(256) k_vanka_sweep(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                     VankaLists lists, const T *__restrict__ kinv,
                                                     T *__restrict__ corr, int cap, Coef<T> K, int sweeps,
                                                     GridBarrier *bar, unsigned expect, unsigned spin_limit) {
    pdl_enter();
    // blocks the barrier waits for: the grid, or more in the bounded-wait self-test (never completes)
    const unsigned nb = expect ? expect : gridDim.x;
    const long long stride = (long long)gridDim.x * blockDim.x;  // a multiple of 8: lanes keep their group
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int ph = 0; ph < 16; ++ph) {
            int col = ph < 8 ? ph : 15 - ph;
            int n = lists.count[col];
            if (n == 0) continue;
            const int *cells = lists.cells[col];
            for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; (t >> 3) < n; t += stride)
                vanka_compute_lane(L, x, b, cells[t >> 3], (int)(t & 7), gmask, kinv, corr, cap, (int)(t >> 3), K, T(1),
                                   lists.tab[col]);
            grid_sync(bar, nb, spin_limit);
            for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; (t >> 3) < n; t += stride)
                vanka_apply_lane(L, x, cells[t >> 3], (int)(t & 7), corr, cap, (int)(t >> 3));
            grid_sync(bar, nb, spin_limit);
        }
}

template <class T, class TB> int vanka_sweep_blocks_per_sm() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_vanka_sweep<T, TB>, 256, 0);
    return nb;
}

template <class T, class TB>
void launch_vanka_sweep(const Lev &L, T *x, const TB *b, const VankaLists &lists, const T *kinv, T *corr, int cap,
                        int sweeps, GridBarrier *bar, int max_blocks, cudaStream_t s, int missing_blocks,
                        unsigned spin_limit) {
    int mx = 0;
    for (int c = 0; c < 8; ++c) mx = lists.count[c] > mx ? lists.count[c] : mx;
    if (mx == 0 || sweeps <= 0) return;
    int need = cdiv(8LL * mx, 256);
    int nb = need < max_blocks ? need : max_blocks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const unsigned expect = missing_blocks > 0 ? (unsigned)(nb + missing_blocks) : 0u;
    cudaLaunchKernelEx(&cfg, k_vanka_sweep<T, TB>, L, x, b, lists, kinv, corr, cap, coef<T>(L, L.gamma), sweeps, bar,
                       expect, spin_limit);
}

// ---- one symmetric Vanka sweep in one thread block with the level in shared memory ----
// Small levels only (x, b and the corrections must fit in shared memory): the level's x and b are
// copied in, the 16 colour steps run on the shared copies with __syncthreads() between the compute
// and apply steps, and x is copied back.  The per-lane arithmetic is the same code as the global
// version (generic pointers), so the result is bit-identical.
// shared-memory layout: x [n] | b [n] | corrections [7 cap] | local inverses [64 x 49] | cell lists [8 cap]
template <class T, class TB> struct VankaSmem {
    size_t xo, bo, co, ko, lo, bytes;
    __host__ __device__ VankaSmem(long long n, int cap) {
        auto up = [](size_t v) { return (v + 15) / 16 * 16; };
        xo = 0;
        bo = up((size_t)n * sizeof(T));
        co = bo + up((size_t)n * sizeof(TB));
        ko = co + up((size_t)7 * cap * sizeof(T));
        lo = ko + up((size_t)64 * 49 * sizeof(T));
        bytes = lo + (size_t)8 * cap * sizeof(int);
    }
};
template <class T, class TB> size_t vanka_smem_bytes(const Lev &L, int cap) { return VankaSmem<T, TB>(L.n, cap).bytes; }

template <class T, class TB>
__global__ void __launch_bounds__(1024) k_vanka_smem(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                     VankaLists lists, const T *__restrict__ kinv, int cap, Coef<T> K,
                                                     int sweeps) {
    extern __shared__ __align__(16) unsigned char vsm[];
    const VankaSmem<T, TB> lay(L.n, cap);
    T *xs = reinterpret_cast<T *>(vsm + lay.xo);
    TB *bs = reinterpret_cast<TB *>(vsm + lay.bo);
    T *cs = reinterpret_cast<T *>(vsm + lay.co);
    T *ks = reinterpret_cast<T *>(vsm + lay.ko);
    int *cl = reinterpret_cast<int *>(vsm + lay.lo);
    pdl_enter();
    const int n = (int)L.n;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        xs[e] = x[e];
        bs[e] = b[e];
    }
    for (int e = threadIdx.x; e < 64 * 49; e += blockDim.x) ks[e] = kinv[e];
    for (int col = 0; col < 8; ++col)
        for (int e = threadIdx.x; e < lists.count[col]; e += blockDim.x) cl[col * cap + e] = lists.cells[col][e];
    __syncthreads();
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int ph = 0; ph < 16; ++ph) {
            const int col = ph < 8 ? ph : 15 - ph;
            const int nc = lists.count[col];
            if (nc == 0) continue;  // uniform across the block
            const int *cells = cl + col * cap;
            for (int t = threadIdx.x; (t >> 3) < nc; t += blockDim.x)
                vanka_compute_lane(L, (const T *)xs, (const TB *)bs, cells[t >> 3], t & 7, gmask, (const T *)ks, cs, cap,
                                   t >> 3, K);
            __syncthreads();
            for (int t = threadIdx.x; (t >> 3) < nc; t += blockDim.x)
                vanka_apply_lane(L, xs, cells[t >> 3], t & 7, (const T *)cs, cap, t >> 3);
            __syncthreads();
        }
    for (int e = threadIdx.x; e < n; e += blockDim.x) x[e] = xs[e];
}

// the dynamic shared-memory opt-in, set once outside any capture; false if the level does not fit
template <class T, class TB> bool vanka_smem_prepare(const Lev &L, int cap) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t need = vanka_smem_bytes<T, TB>(L, cap);
    if (need > (size_t)optin || L.n >= (1LL << 31)) return false;
    // the attribute is per kernel, shared by every handle: always the device maximum
    return cudaFuncSetAttribute(k_vanka_smem<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) ==
           cudaSuccess;
}

template <class T, class TB>
void launch_vanka_smem(const Lev &L, T *x, const TB *b, const VankaLists &lists, const T *kinv, int cap, int sweeps,
                       cudaStream_t s) {
    if (sweeps <= 0) return;
    launch_k(k_vanka_smem<T, TB>, dim3(1), dim3(1024), vanka_smem_bytes<T, TB>(L, cap), s, L, x, b, lists, kinv, cap,
             coef<T>(L, L.gamma), sweeps);
}

// ---- one symmetric Vanka sweep in one thread-block cluster (small levels) ----
// The cluster's CTAs stride over the cells of a colour; hardware cluster barriers (release/acquire
// at cluster scope) separate the compute and apply steps, so no launch and no software spin sits
// between colours.  Every thread executes every barrier (no early exit), the colour counts are
// uniform, and the result is bit-identical to the per-colour launches.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

template <class T, class TB>
__global__ void __launch_bounds__(1024) k_vanka_cluster(Lev L, T *__restrict__ x, const TB *__restrict__ b,
                                                        VankaLists lists, const T *__restrict__ kinv,
                                                        T *__restrict__ corr, int cap, Coef<T> K, int sweeps) {
    pdl_enter();
    const long long stride = (long long)cluster_size() * blockDim.x;  // a multiple of 8: lanes keep their group
    const long long t0 = (long long)cluster_rank() * blockDim.x + threadIdx.x;
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int ph = 0; ph < 16; ++ph) {
            const int col = ph < 8 ? ph : 15 - ph;
            const int n = lists.count[col];
            if (n == 0) continue;  // uniform across the cluster
            const int *cells = lists.cells[col];
            for (long long t = t0; (t >> 3) < n; t += stride)
                vanka_compute_lane(L, x, b, cells[t >> 3], (int)(t & 7), gmask, kinv, corr, cap, (int)(t >> 3), K, T(1),
                                   lists.tab[col]);
            cluster_sync_all();
            for (long long t = t0; (t >> 3) < n; t += stride)
                vanka_apply_lane(L, x, cells[t >> 3], (int)(t & 7), corr, cap, (int)(t >> 3));
            cluster_sync_all();
        }
}

// clusters above the portable size of 8 need the kernel attribute, set once (outside any capture)
template <class T, class TB> cudaError_t vanka_cluster_prepare() {
    return cudaFuncSetAttribute(k_vanka_cluster<T, TB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <class T, class TB>
cudaError_t launch_vanka_cluster(const Lev &L, T *x, const TB *b, const VankaLists &lists, const T *kinv, T *corr,
                                 int cap, int sweeps, int cluster, cudaStream_t s) {
    if (sweeps <= 0) return cudaSuccess;
    if (cluster < 1 || cluster > 16) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_vanka_cluster<T, TB>, L, x, b, lists, kinv, corr, cap, coef<T>(L, L.gamma), sweeps);
}

// ------------------------------------------------------------------------------------------
// Sec. 3.1 distributive weighted Jacobi (symmetric, block by block; see launch order in the host
// code): every step computes its updates from one state into a buffer, then adds them.
__device__ __forceinline__ bool v2_face(const Lev &L, int c, int i, int j, int k) {
    const int n[3] = {L.nx, L.ny, L.nz}, q[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int lo = d == c ? 2 : 1, hi = d == c ? n[d] - 2 : n[d] - 2;
        if (q[d] < lo || q[d] > hi) return false;
    }
    return !L.flags || (L.flags[pidx(L, c, i, j, k)] & kFlagV2);
}

// velocity block: t_f = w (b - L~x)_f / (6 eta/h^2) on the V2 faces, 0 on every other face entry
template <class T, class TB, int C, class IDX>
__device__ __forceinline__ void dwj_face_entry(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                               T *__restrict__ t, const Coef<T> &K, T w, int i, int j, int k) {
    if (!entry_exists<C>(L, i, j, k)) return;
    const long long q = entry_index<C, IDX>(L, i, j, k);
    T v = T(0);
    if (v2_face(L, C, i, j, k)) v = w * (T(ldv(b[q])) - row_at<T, C, true, IDX>(x, L, i, j, k, K)) / (T(6) * K.eh2);
    t[q] = v;
}
template <class T, class TB, class IDX>
__global__ void __launch_bounds__(256, 8) k_dwj_face(Lev L, const T *__restrict__ x, const TB *__restrict__ b,
                                                     T *__restrict__ t, Coef<T> K, T w) {
    pdl_enter();
    const int c = blockIdx.z % 3, k = blockIdx.z / 3;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: dwj_face_entry<T, TB, 0, IDX>(L, x, b, t, K, w, i, j, k); break;
    case 1: dwj_face_entry<T, TB, 1, IDX>(L, x, b, t, K, w, i, j, k); break;
    default: dwj_face_entry<T, TB, 2, IDX>(L, x, b, t, K, w, i, j, k);
    }
}
// x_f += t_f on the face entries
template <class T>
__global__ void __launch_bounds__(256) k_add_faces(long long nf, T *__restrict__ x, const T *__restrict__ t) {
    pdl_enter();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += (long long)gridDim.x * blockDim.x)
        x[q] += t[q];
}
// pressure block, right-preconditioned: delta_c = (b - L~x)_c / d on the V2 cells, 0 elsewhere
template <class T, class TB>
__global__ void __launch_bounds__(256) k_dwj_pdelta(Lev L, const T *__restrict__ x, const TB *__restrict__ b,
                                                    T *__restrict__ delta, Coef<T> K, T dP) {
    pdl_enter();
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    if (i >= L.nx || j >= L.ny || k >= L.nz) return;
    const long long cl = cell_lin(L, i, j, k);
    T v = T(0);
    if (in_v2_cell(L, i, j, k)) v = (T(ldv(b[L.off[3] + cl])) - row_at<T, 3, true, long long>(x, L, i, j, k, K)) / dP;
    delta[cl] = v;
}
// x += w sum_c delta_c M_{.c}: faces -= w (delta_plus - delta_minus)/h, cells += w eta/h^2 (6 delta_c -
// sum of the 6 neighbours); delta is 0 outside V2, so every neighbour a nonzero delta needs exists
template <class T, int C>
__device__ __forceinline__ void dwj_dist_entry(const Lev &L, T *__restrict__ x, const T *__restrict__ delta,
                                               const Coef<T> &K, T w, int i, int j, int k) {
    if (!entry_exists<C>(L, i, j, k)) return;
    const long long q = entry_index<C, long long>(L, i, j, k);
    if (!entry_unknown<C>(L, i, j, k, q)) return;
    const long long sy = L.nx, sz = (long long)L.nx * L.ny;
    if constexpr (C < 3) {
        const long long plus = cell_lin(L, i, j, k), ps = C == 0 ? 1 : (C == 1 ? sy : sz);
        x[q] -= w * K.ih * (delta[plus] - delta[plus - ps]);
    } else {
        const long long t = cell_lin(L, i, j, k);
        T g = T(6) * delta[t];
        g -= (i > 0 ? delta[t - 1] : T(0)) + (i < L.nx - 1 ? delta[t + 1] : T(0));
        g -= (j > 0 ? delta[t - sy] : T(0)) + (j < L.ny - 1 ? delta[t + sy] : T(0));
        g -= (k > 0 ? delta[t - sz] : T(0)) + (k < L.nz - 1 ? delta[t + sz] : T(0));
        x[q] += w * K.eh2 * g;
    }
}
template <class T>
__global__ void __launch_bounds__(256, 8) k_dwj_pdist(Lev L, T *__restrict__ x, const T *__restrict__ delta, Coef<T> K,
                                                      T w) {
    pdl_enter();
    const int c = blockIdx.z & 3, k = blockIdx.z >> 2;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: dwj_dist_entry<T, 0>(L, x, delta, K, w, i, j, k); break;
    case 1: dwj_dist_entry<T, 1>(L, x, delta, K, w, i, j, k); break;
    case 2: dwj_dist_entry<T, 2>(L, x, delta, K, w, i, j, k); break;
    default: dwj_dist_entry<T, 3>(L, x, delta, K, w, i, j, k);
    }
}
// r = b - L~x into a buffer of the arithmetic type (every packed entry)
template <class T, class TB, int C>
__device__ __forceinline__ void resid_entry(const Lev &L, const T *__restrict__ x, const TB *__restrict__ b,
                                            T *__restrict__ r, const Coef<T> &K, int i, int j, int k) {
    if (!entry_exists<C>(L, i, j, k)) return;
    const long long q = entry_index<C, long long>(L, i, j, k);
    r[q] = entry_unknown<C>(L, i, j, k, q) ? T(ldv(b[q])) - row_at<T, C, true, long long>(x, L, i, j, k, K) : T(0);
}
template <class T, class TB>
__global__ void __launch_bounds__(256, 8) k_resid_t(Lev L, const T *__restrict__ x, const TB *__restrict__ b,
                                                    T *__restrict__ r, Coef<T> K) {
    pdl_enter();
    const int c = blockIdx.z & 3, k = blockIdx.z >> 2;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    switch (c) {
    case 0: resid_entry<T, TB, 0>(L, x, b, r, K, i, j, k); break;
    case 1: resid_entry<T, TB, 1>(L, x, b, r, K, i, j, k); break;
    case 2: resid_entry<T, TB, 2>(L, x, b, r, K, i, j, k); break;
    default: resid_entry<T, TB, 3>(L, x, b, r, K, i, j, k);
    }
}
// pressure block, left-preconditioned: p_c += w M_{.c}^T r / d on the V2 cells
template <class T>
__global__ void __launch_bounds__(256) k_dwj_pleft(Lev L, T *__restrict__ x, const T *__restrict__ r, Coef<T> K, T w,
                                                   T dP) {
    pdl_enter();
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    if (i >= L.nx || j >= L.ny || k >= L.nz || !in_v2_cell(L, i, j, k)) return;
    const long long nx = L.nx, ny = L.ny, sy = nx, sz = nx * ny;
    const long long cl = cell_lin(L, i, j, k);
    const T *rc = r + L.off[3] + cl;
    const T *ru = r + L.off[0] + (i + (nx + 1) * (j + ny * k));
    const T *rv = r + L.off[1] + (i + nx * (j + (ny + 1) * k));
    const T *rw = r + L.off[2] + (i + nx * (j + ny * k));
    const T s = K.ih * ((ru[1] - ru[0]) + (rv[sy] - rv[0]) + (rw[sz] - rw[0])) +
                K.eh2 * (T(6) * rc[0] - (rc[-1] + rc[1] + rc[-sy] + rc[sy] + rc[-sz] + rc[sz]));
    x[L.off[3] + cl] += w * s / dP;
}

template <class T, class TB>
void launch_dwj_sym(const Lev &L, T *x, const TB *b, T *t, T *delta, double w, cudaStream_t s) {
    const Coef<T> K = coef<T>(L, L.gamma);
    const T W = T(w), dP = dgs_pressure_diag<T>(L);
    const long long nf = L.off[3];
    const dim3 fgrid(cdiv(L.nx + 1, BX), cdiv(L.ny + 1, BY), 3 * (L.nz + 1));
    const dim3 cgrid(cdiv(L.nx, BX), cdiv(L.ny, BY), L.nz);
    const int ab = (int)std::min<long long>(4736, (nf + 255) / 256);
    auto vel = [&]() {
        if (idx32(L)) launch_k(k_dwj_face<T, TB, int>, fgrid, dim3(kBlock3), 0, s, L, (const T *)x, b, t, K, W);
        else launch_k(k_dwj_face<T, TB, long long>, fgrid, dim3(kBlock3), 0, s, L, (const T *)x, b, t, K, W);
        launch_k(k_add_faces<T>, dim3(ab), dim3(256), 0, s, nf, x, (const T *)t);
    };
    vel();
    launch_k(k_dwj_pdelta<T, TB>, cgrid, dim3(kBlock3), 0, s, L, (const T *)x, b, delta, K, dP);
    launch_k(k_dwj_pdist<T>, dim3(entry_grid(L)), dim3(kBlock3), 0, s, L, x, (const T *)delta, K, W);
    launch_k(k_resid_t<T, TB>, dim3(entry_grid(L)), dim3(kBlock3), 0, s, L, (const T *)x, b, t, K);
    launch_k(k_dwj_pleft<T>, cgrid, dim3(kBlock3), 0, s, L, x, (const T *)t, K, W, dP);
    vel();
}

// ------------------------------------------------------------------------------------------
// Sec. 2 transfers.  P (coarse -> fine): pressure constant per coarse cell; a face value takes
// weight 1 from a coincident coarse face or 1/2 + 1/2 from the two coarse faces around it along
// its normal, and 3/4 (coarse row containing it) + 1/4 (next coarse row on the far side) along
// each tangential axis; coarse entries that are not unknowns contribute 0.  R = P^T / 8.
// component C of the face transfers, with every index known at compile time; offsets are strides
// from one base address.  Along the normal axis every referenced fine/coarse face lies inside the
// array (walls hold 0); along a tangential axis the rows outside the box are skipped.
template <class T, int C, class TF>
__device__ __forceinline__ T restrict_face(const Lev &F, const Lev &Cl, const TF *__restrict__ rf, int I, int J,
                                           int Kk) {
    const long long sy = F.nx + (C == 0), sz = sy * (F.ny + (C == 1));
    const long long st[3] = {1, sy, sz};
    const TF *fb = rf + comp_base(F, C) + 2 * I + sy * (2 * J) + sz * (2LL * Kk);
    const int t1 = C == 0 ? 1 : 0, t2 = C == 2 ? 1 : 2;  // tangential axes
    const int T1 = t1 == 0 ? I : (t1 == 1 ? J : Kk), T2 = t2 == 1 ? J : Kk;
    const int n1 = t1 == 0 ? Cl.nx : (t1 == 1 ? Cl.ny : Cl.nz), n2 = t2 == 1 ? Cl.ny : Cl.nz;
    const T nw[3] = {T(0.5), T(1), T(0.5)};
    const T tw[4] = {T(0.25), T(0.75), T(0.75), T(0.25)};
    T s = T(0);
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
        if ((bb == 0 && T1 == 0) || (bb == 3 && T1 == n1 - 1)) continue;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            if ((g == 0 && T2 == 0) || (g == 3 && T2 == n2 - 1)) continue;
            const TF *row = fb + (bb - 1) * st[t1] + (g - 1) * st[t2];
            T sn = nw[0] * T(ldv(row[-st[C]])) + nw[1] * T(ldv(row[0])) + nw[2] * T(ldv(row[st[C]]));
            s += tw[bb] * tw[g] * sn;
        }
    }
    return s * T(0.125);
}

// thread_entry with the launch's own tile: block (blockDim.x, blockDim.y) over (x, y), kz planes per thread
__device__ __forceinline__ bool thread_entry_tile(const Lev &L, int gy, int kz, int zb, int &c, int &i, int &j, int &k0,
                                                  int &k1) {
    c = blockIdx.y / gy;
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = (blockIdx.y - c * gy) * blockDim.y + threadIdx.y;
    k0 = zb * kz;
    int ez = ext(L, c, 2);
    k1 = k0 + kz < ez ? k0 + kz : ez;
    return i < ext(L, c, 0) && j < ext(L, c, 1) && k0 < ez;
}

template <class T, class TF, class TC, bool BATCH>
__global__ void __launch_bounds__(256) k_restrict(Lev F, Lev C, int gy, int kz, const TF *__restrict__ rf,
                                                  TC *__restrict__ bc) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(C) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) rf = bslot(rf, F.bstride, zs.p);
    if constexpr (BATCH) bc = bslot(bc, C.bstride, zs.p);
    int c, I, J, k0, k1;
    if (!thread_entry_tile(C, gy, kz, zs.z, c, I, J, k0, k1)) return;
    for (int Kk = k0; Kk < k1; ++Kk) {
    long long q = pidx(C, c, I, J, Kk);
    if (!unknown(C, c, I, J, Kk)) {
        bc[q] = cvt<TC>(T(0));
        continue;
    }
    T v;
    switch (c) {
    case 0: v = restrict_face<T, 0, TF>(F, C, rf, I, J, Kk); break;
    case 1: v = restrict_face<T, 1, TF>(F, C, rf, I, J, Kk); break;
    case 2: v = restrict_face<T, 2, TF>(F, C, rf, I, J, Kk); break;
    default: {
        T s = T(0);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            s += T(ldv(rf[pidx(F, 3, 2 * I + (m & 1), 2 * J + ((m >> 1) & 1), 2 * Kk + ((m >> 2) & 1))]));
        v = s * T(0.125);
    }
    }
    bc[q] = cvt<TC>(v);
    }
}

// Coarse-cell-centric prolongation: the thread of coarse cell (I,J,K) adds P e to the 8 fine cells
// and to the fine faces (2I+a, 2J+b, 2K+c), a,b,c in {0,1}, of each velocity component.  For
// component C it loads the coarse faces at normal index {I, I+1} and tangential rows {T-1, T, T+1}
// once (18 values; rows outside the box are 0).
template <class T, int C>
__device__ __forceinline__ void prolong_comp(const Lev &F, const Lev &Cl, const T *__restrict__ ec, T *__restrict__ xf,
                                             int I, int J, int Kk) {
    const long long csy = Cl.nx + (C == 0), csz = csy * (Cl.ny + (C == 1));
    const long long fsy = F.nx + (C == 0), fsz = fsy * (F.ny + (C == 1));
    const int cn[3] = {Cl.nx, Cl.ny, Cl.nz};
    const int ci[3] = {I, J, Kk};
    // axes: n = normal (C), t1, t2 = tangential
    const int t1 = C == 0 ? 1 : 0, t2 = C == 2 ? 1 : 2;
    const long long cst[3] = {1, csy, csz}, fst[3] = {1, fsy, fsz};
    const T *cb = ec + comp_base(Cl, C) + I + csy * J + csz * Kk;
    T c[2][3][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                int r1 = ci[t1] + p - 1, r2 = ci[t2] + q - 1;
                bool ok = r1 >= 0 && r1 < cn[t1] && r2 >= 0 && r2 < cn[t2];
                c[a][p][q] = ok ? cb[a * cst[C] + (p - 1) * cst[t1] + (q - 1) * cst[t2]] : T(0);
            }
    const int fn = C == 0 ? F.nx : (C == 1 ? F.ny : F.nz);
    T *fb = xf + comp_base(F, C) + 2 * I + fsy * (2LL * J) + fsz * (2LL * Kk);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        int fidx = 2 * ci[C] + a;
        if (fidx < 1 || fidx > fn - 1) continue;  // wall-normal fine faces are not unknowns
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                // tangential: 3/4 from row T, 1/4 from row T-1 (even fine index) or T+1 (odd)
                const T w1[3] = {bb == 0 ? T(0.25) : T(0), T(0.75), bb == 1 ? T(0.25) : T(0)};
                const T w2[3] = {g == 0 ? T(0.25) : T(0), T(0.75), g == 1 ? T(0.25) : T(0)};
                T s = T(0);
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        T tv = a == 0 ? c[0][p][q] : T(0.5) * (c[0][p][q] + c[1][p][q]);
                        s += w1[p] * w2[q] * tv;
                    }
                const long long o = a * fst[C] + bb * fst[t1] + g * fst[t2];
                // label domains: fine faces that are not unknowns keep their 0
                if (!F.flags || (F.flags[(fb - xf) + o] & kFlagActive)) fb[o] += s;
            }
    }
}

template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_prolong(Lev F, Lev Cl, int kz, const T *__restrict__ ec, T *__restrict__ xf) {
    pdl_enter();
    const ZSlot zs = BATCH ? zslot(Cl) : ZSlot{0, (int)blockIdx.z};
    if constexpr (BATCH) ec = bslot(ec, Cl.bstride, zs.p);
    if constexpr (BATCH) xf = bslot(xf, F.bstride, zs.p);
    int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= Cl.nx || J >= Cl.ny) return;
    int k0 = zs.z * kz, k1 = k0 + kz < Cl.nz ? k0 + kz : Cl.nz;
    const long long fy = F.nx, fz = (long long)F.nx * F.ny;
    for (int Kk = k0; Kk < k1; ++Kk) {
        T pcv = ec[pidx(Cl, 3, I, J, Kk)];
        T *pf = xf + F.off[3] + 2 * I + fy * (2 * J) + fz * (2LL * Kk);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const long long o = (m & 1) + fy * ((m >> 1) & 1) + fz * ((m >> 2) & 1);
            if (!F.flags || (F.flags[(pf - xf) + o] & kFlagActive)) pf[o] += pcv;
        }
        prolong_comp<T, 0>(F, Cl, ec, xf, I, J, Kk);
        prolong_comp<T, 1>(F, Cl, ec, xf, I, J, Kk);
        prolong_comp<T, 2>(F, Cl, ec, xf, I, J, Kk);
    }
}

// Transfers take a tile (block bx x by over the coarse (x, y) positions, kz coarse z-planes per
// thread): every output entry is produced by one thread with the same arithmetic whatever the tile,
// so all tiles give the same bits; the handle picks one per level by timing (coarse levels want
// small tiles and one plane per thread: few entries, latency-bound).
template <class T, class TF, class TC>
void launch_restrict(const Lev &F, const Lev &C, const TF *rf, TC *bc, cudaStream_t s, Tile t) {
    const int mx = C.nx + 1, my = C.ny + 1, mz = C.nz + 1;
    const int gy = cdiv(my, t.by);
    launch_k(BSEL(C.nb, k_restrict<T, TF, TC), dim3(cdiv(mx, t.bx), gy * 4, cdiv(mz, t.kz) * C.nb), dim3(t.bx, t.by, 1), 0, s, F, C,
             gy, t.kz, rf, bc);
}
template <class T> void launch_prolong(const Lev &F, const Lev &C, const T *ec, T *xf, cudaStream_t s, Tile t) {
    dim3 grid(cdiv(C.nx, t.bx), cdiv(C.ny, t.by), cdiv(C.nz, t.kz) * C.nb);
    launch_k(BSEL(C.nb, k_prolong<T), dim3(grid), dim3(t.bx, t.by, 1), 0, s, F, C, t.kz, ec, xf);
}

// ------------------------------------------------------------------------------------------
// Alg. 1 exact coarsest solve: x[cidx[r]] = sum_k Kinv[r][k] b[cidx[k]] (FP64, one warp per row,
// deterministic lane-strided sums then a fixed shuffle tree)
template <class T, bool BATCH>
__global__ void __launch_bounds__(256) k_coarse(const int *__restrict__ cidx, int nc, const double *__restrict__ kinv,
                                                const T *__restrict__ b, T *__restrict__ x, long long bstride) {
    pdl_enter();
    if constexpr (BATCH) b = bslot(b, bstride, (int)blockIdx.y);
    if constexpr (BATCH) x = bslot(x, bstride, (int)blockIdx.y);
    extern __shared__ double sb[];
    for (int m = threadIdx.x; m < nc; m += blockDim.x) sb[m] = (double)b[cidx[m]];
    __syncthreads();
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= nc) return;
    const double *row = kinv + (long long)r * nc;
    double s = 0.0;
    for (int m = lane; m < nc; m += 32) s += row[m] * sb[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[cidx[r]] = (T)s;
}

template <class T>
void launch_coarse(const Lev &C, const int *cidx, int nc, const double *kinv, const T *b, T *x, cudaStream_t s) {
    int rows_per_block = 256 / 32;
    launch_k(BSEL(C.nb, k_coarse<T), dim3((nc + rows_per_block - 1) / rows_per_block, C.nb), dim3(256), nc * sizeof(double), s, cidx,
             nc, kinv, b, x, C.bstride);
}

// ------------------------------------------------------------------------------------------
template <class T> __global__ void __launch_bounds__(256) k_mask(Lev L, int gy, T *__restrict__ x) {
    pdl_enter();
    int c, i, j, k0, k1;
    if (!thread_entry(L, gy, c, i, j, k0, k1)) return;
    for (int k = k0; k < k1; ++k)
        if (!unknown(L, c, i, j, k)) x[pidx(L, c, i, j, k)] = cvt<T>(0.0f);
}
template <class T> void launch_mask(const Lev &L, T *x, cudaStream_t s) {
    Geo g = geo_components(L, 4);
    launch_k(k_mask<T>, dim3(g.grid), dim3(kBlock3), 0, s, L, g.gy, x);
}
template void launch_mask<float>(const Lev &, float *, cudaStream_t);
template void launch_mask<double>(const Lev &, double *, cudaStream_t);
template void launch_mask<bf16>(const Lev &, bf16 *, cudaStream_t);

template <class A, class B> __global__ void k_convert(long long n, const A *__restrict__ in, B *__restrict__ out) {
    pdl_enter();
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = cvt<B>(in[t]);
}
template <class A, class B> void launch_convert(long long n, const A *in, B *out, cudaStream_t s) {
    long long nb = (n + 255) / 256;
    launch_k(k_convert<A, B>, dim3((unsigned)(nb < 4736 ? nb : 4736)), dim3(256), 0, s, n, in, out);
}

// explicit instantiations: T the arithmetic precision, TB the storage of the level operands
// (right-hand side, residual, pressure-sweep residual parts)
#define SMG_INST_TB(T, TB)                                                                                          \
    template void launch_apply<T, TB>(const Lev &, const T *, const TB *, TB *, double, cudaStream_t);             \
    template void launch_dgs_u<T, TB>(const Lev &, T *, const TB *, int, cudaStream_t);                           \
    template void launch_dgs_u_fused<T, TB>(const Lev &, const T *, T *, const TB *, int, cudaStream_t);           \
    template bool dgs_u_fused_prepare<T, TB>();                                                                   \
    template void launch_dgs_p_fwd<T, TB>(const Lev &, T *, const TB *, T *, int, cudaStream_t);                  \
    template void launch_dgs_p_bwd_prep<T, TB>(const Lev &, T *, const TB *, TB *, const T *, cudaStream_t);      \
    template void launch_dgs_p_bwd<T, TB>(const Lev &, T *, const TB *, int, cudaStream_t);                       \
    template bool launch_dgs_p_fwd_pair<T, TB>(const Lev &, T *, const TB *, T *, int, cudaStream_t);              \
    template bool launch_dgs_p_bwd_pair<T, TB>(const Lev &, T *, const TB *, int, cudaStream_t);                   \
    template void launch_vanka_compute<T, TB>(const Lev &, const T *, const TB *, const int *, const int *, int,   \
                                              const T *, T *, int, double, cudaStream_t);                           \
    template void launch_vanka_pingpong<T, TB>(const Lev &, T *, T *, const TB *, const VankaLists &, const int *, \
                                               int, const T *, int, cudaStream_t);                                \
    template void launch_vanka_sweep<T, TB>(const Lev &, T *, const TB *, const VankaLists &, const T *, T *, int,  \
                                            int, GridBarrier *, int, cudaStream_t, int, unsigned);                  \
    template cudaError_t vanka_cluster_prepare<T, TB>();                                                          \
    template bool vanka_smem_prepare<T, TB>(const Lev &, int);                                                     \
    template void launch_vanka_smem<T, TB>(const Lev &, T *, const TB *, const VankaLists &, const T *, int, int,   \
                                           cudaStream_t);                                                          \
    template cudaError_t launch_vanka_cluster<T, TB>(const Lev &, T *, const TB *, const VankaLists &, const T *,   \
                                                     T *, int, int, int, cudaStream_t);                             \
    template int vanka_sweep_blocks_per_sm<T, TB>();
#define SMG_INST(T)                                                                                               \
    SMG_INST_TB(T, T)                                                                                             \
    template void launch_dgs_p_gather<T>(const Lev &, T *, const T *, cudaStream_t);                              \
    template void launch_vanka_apply<T>(const Lev &, T *, const int *, int, const T *, int, cudaStream_t);        \
    template void launch_restrict<T, T, T>(const Lev &, const Lev &, const T *, T *, cudaStream_t, Tile);               \
    template void launch_prolong<T>(const Lev &, const Lev &, const T *, T *, cudaStream_t, Tile);                      \
    template void launch_coarse<T>(const Lev &, const int *, int, const double *, const T *, T *, cudaStream_t);
SMG_INST(float)
SMG_INST(double)
SMG_INST_TB(float, bf16)
template void launch_dwj_sym<float, float>(const Lev &, float *, const float *, float *, float *, double, cudaStream_t);
template void launch_dwj_sym<double, double>(const Lev &, double *, const double *, double *, double *, double,
                                             cudaStream_t);
template void launch_dwj_sym<float, bf16>(const Lev &, float *, const bf16 *, float *, float *, double, cudaStream_t);
template void launch_restrict<float, bf16, bf16>(const Lev &, const Lev &, const bf16 *, bf16 *, cudaStream_t, Tile);
template void launch_restrict<float, bf16, float>(const Lev &, const Lev &, const bf16 *, float *, cudaStream_t, Tile);
template void launch_restrict<float, float, bf16>(const Lev &, const Lev &, const float *, bf16 *, cudaStream_t, Tile);
template void launch_convert<double, float>(long long, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(long long, const float *, double *, cudaStream_t);
template void launch_convert<double, double>(long long, const double *, double *, cudaStream_t);
template void launch_convert<double, bf16>(long long, const double *, bf16 *, cudaStream_t);
template void launch_convert<bf16, double>(long long, const bf16 *, double *, cudaStream_t);

}  // namespace smg
