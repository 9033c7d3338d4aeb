// kernels_level.cu -- per-level CUDA kernels of the symmetric multigrid V-cycle (sm_103a):
// operator apply / residual (Eq. 2, Sec. 4), Dirichlet folding (Sec. 5), symmetric distributive
// Gauss-Seidel (Alg. 2, Eq. ldist, App. A), 8-colour multiplicative Vanka (Sec. 3.2, App. C,
// Sec. 6), restriction / prolongation (Sec. 2) and the exact coarsest solve (Alg. 1).
//
// Every kernel is bandwidth-shaped: one thread per unknown (or per cell of a colour), coalesced
// along x, stencil neighbours served by L1/L2.  No tensor cores: nothing here is a contraction.
#include "kernels.h"

namespace smg {

namespace {
constexpr int kBlock = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

inline long long comp_box(const Lev &L, int c) {
    return (long long)ext(L, c, 0) * ext(L, c, 1) * ext(L, c, 2);
}
inline long long max_box(const Lev &L, int ncomp) {
    long long m = 0;
    for (int c = 0; c < ncomp; ++c) m = comp_box(L, c) > m ? comp_box(L, c) : m;
    return m;
}

// V2 index ranges of the box problem: faces of component c with normal index in [2, n-2] and
// tangential indices in [1, n-2]; cells with every index in [1, n-2].
__host__ __device__ inline void v2_face_range(const Lev &L, int c, int lo[3], int cnt[3]) {
    int n[3] = {L.nx, L.ny, L.nz};
    for (int d = 0; d < 3; ++d) {
        lo[d] = d == c ? 2 : 1;
        cnt[d] = d == c ? n[d] - 3 : n[d] - 2;
        if (cnt[d] < 0) cnt[d] = 0;
    }
}

// cells of colour (bx, by, bz) inside the V2 cell range [1, n-2]
__host__ __device__ inline void v2_colour_range(const Lev &L, int colour, int lo[3], int cnt[3]) {
    int n[3] = {L.nx, L.ny, L.nz};
    for (int d = 0; d < 3; ++d) {
        int bit = (colour >> d) & 1;
        lo[d] = bit ? 1 : 2;
        cnt[d] = (n[d] - 2 >= lo[d]) ? (n[d] - 2 - lo[d]) / 2 + 1 : 0;
    }
}

__device__ __forceinline__ bool in_v2_cell(const Lev &L, int i, int j, int k) {
    return i >= 1 && j >= 1 && k >= 1 && i <= L.nx - 2 && j <= L.ny - 2 && k <= L.nz - 2;
}

__device__ __forceinline__ long long cell_lin(const Lev &L, int i, int j, int k) {
    return i + (long long)L.nx * (j + (long long)L.ny * k);
}
}  // namespace

// ------------------------------------------------------------------------------------------
// y = L~x or b - L~x on every packed entry (0 off the unknowns); blockIdx.y = component
template <class T>
__global__ void __launch_bounds__(256) k_apply(Lev L, const T *__restrict__ x, const T *__restrict__ b,
                                               T *__restrict__ y, Coef<T> K) {
    int c = blockIdx.y;
    int ex = ext(L, c, 0), ey = ext(L, c, 1), ez = ext(L, c, 2);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ex * ey * ez) return;
    int i, j, k;
    decode3(t, ex, ey, i, j, k);
    long long q = L.off[c] + t;
    if (!active(L, c, i, j, k)) {
        y[q] = T(0);
        return;
    }
    T v = c < 3 ? face_Lx(x, L, c, i, j, k, K) : cell_Lx(x, L, i, j, k, K);
    y[q] = b ? b[q] - v : v;
}

template <class T> void launch_apply(const Lev &L, const T *x, const T *b, T *y, double gam, cudaStream_t s) {
    dim3 grid(blocks_for(max_box(L, 4)), 4);
    k_apply<T><<<grid, kBlock, 0, s>>>(L, x, b, y, coef<T>(L, gam));
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

__global__ void __launch_bounds__(256) k_rhs(Lev L, const double *__restrict__ f, const double *__restrict__ g,
                                             double *__restrict__ b, Coef<double> K) {
    int c = blockIdx.y;
    int ex = ext(L, c, 0), ey = ext(L, c, 1), ez = ext(L, c, 2);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ex * ey * ez) return;
    int i, j, k;
    decode3(t, ex, ey, i, j, k);
    long long q = L.off[c] + t;
    if (!active(L, c, i, j, k)) {
        b[q] = 0.0;
        return;
    }
    double v = f ? f[q] : 0.0;
    if (g) {
        if (c < 3) {
            const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
            for (int m = 0; m < 6; ++m) {
                int a = i + di[m], bb = j + dj[m], cc = k + dk[m];
                if (!active(L, c, a, bb, cc)) v += K.eh2 * g[gidx(L, c, a, bb, cc)];
            }
        } else {
            for (int d = 0; d < 3; ++d) {
                int hi = i + (d == 0), hj = j + (d == 1), hk = k + (d == 2);
                if (!active(L, d, hi, hj, hk)) v += K.ih * g[gidx(L, d, hi, hj, hk)];
                if (!active(L, d, i, j, k)) v -= K.ih * g[gidx(L, d, i, j, k)];
            }
        }
    }
    b[q] = v;
}

void launch_rhs(const Lev &L, const double *f, const double *g, double *b, cudaStream_t s) {
    dim3 grid(blocks_for(max_box(L, 4)), 4);
    k_rhs<<<grid, kBlock, 0, s>>>(L, f, g, b, coef<double>(L, 0.0));
}

// ------------------------------------------------------------------------------------------
// Alg. 2 velocity block: V2 faces of one parity (i+j+k), u, v, w together (A does not couple
// components; same-parity faces are not A-neighbours, pressures are not written) -- in place.
template <class T>
__global__ void __launch_bounds__(256) k_dgs_u(Lev L, T *__restrict__ x, const T *__restrict__ b, int parity,
                                               Coef<T> K) {
    int c = blockIdx.y;
    int lo[3], cnt[3];
    v2_face_range(L, c, lo, cnt);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)cnt[0] * cnt[1] * cnt[2]) return;
    int i, j, k;
    decode3(t, cnt[0], cnt[1], i, j, k);
    i += lo[0];
    j += lo[1];
    k += lo[2];
    if (((i + j + k) & 1) != parity) return;
    long long q = pidx(L, c, i, j, k);
    T r = b[q] - face_Lx(x, L, c, i, j, k, K);
    x[q] += r / (T(6) * K.eh2);
}

template <class T> void launch_dgs_u(const Lev &L, T *x, const T *b, int parity, cudaStream_t s) {
    long long m = 0;
    for (int c = 0; c < 3; ++c) {
        int lo[3], cnt[3];
        v2_face_range(L, c, lo, cnt);
        long long v = (long long)cnt[0] * cnt[1] * cnt[2];
        m = v > m ? v : m;
    }
    if (m == 0) return;
    dim3 grid(blocks_for(m), 3);
    k_dgs_u<T><<<grid, kBlock, 0, s>>>(L, x, b, parity, coef<T>(L, L.gamma));
}

// Alg. 2 pressure block, one colour (i mod 2, j mod 2, k mod 2):
//   r = b_c - (L~x)_c,  delta = r / d,  d = L~_c . M_{.c} = -6 (1 + gamma eta)/h^2,
//   x += delta M_{.c}:  low faces -= delta/h, high faces += delta/h, p_c += 6 eta/h^2 delta,
//                       p of the 6 neighbours -= eta/h^2 delta.
// The neighbour-pressure part is applied in gather form: a cell first collects the deltas of
// neighbours whose colour came earlier in this sweep (pre-gather); k_dgs_p_gather applies the rest
// after the last colour.  delta is stored per cell and stays 0 outside V2.
template <class T>
__global__ void __launch_bounds__(256) k_dgs_p_fwd(Lev L, T *__restrict__ x, const T *__restrict__ b,
                                                   T *__restrict__ delta, int colour, Coef<T> K, T dP) {
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)cnt[0] * cnt[1] * cnt[2]) return;
    int i, j, k;
    decode3(t, cnt[0], cnt[1], i, j, k);
    i = lo[0] + 2 * i;
    j = lo[1] + 2 * j;
    k = lo[2] + 2 * k;
    long long cl = cell_lin(L, i, j, k);
    long long qp = L.off[3] + cl;
    T p = x[qp];
    long long sy = L.nx, sz = (long long)L.nx * L.ny;
    T g = T(0);
    if (colour & 1) g += delta[cl - 1] + delta[cl + 1];
    if (colour & 2) g += delta[cl - sy] + delta[cl + sy];
    if (colour & 4) g += delta[cl - sz] + delta[cl + sz];
    p -= K.eh2 * g;
    long long u0 = pidx(L, 0, i, j, k), v0 = pidx(L, 1, i, j, k), w0 = pidx(L, 2, i, j, k);
    long long vs = L.nx, ws = (long long)L.nx * L.ny;
    T div = (x[u0 + 1] - x[u0]) + (x[v0 + vs] - x[v0]) + (x[w0 + ws] - x[w0]);
    T r = b[qp] + K.ih * div + K.gam * p;
    T dl = r / dP;
    T fd = dl * K.ih;
    x[u0] -= fd;
    x[u0 + 1] += fd;
    x[v0] -= fd;
    x[v0 + vs] += fd;
    x[w0] -= fd;
    x[w0 + ws] += fd;
    x[qp] = p + T(6) * K.eh2 * dl;
    delta[cl] = dl;
}

template <class T>
__global__ void __launch_bounds__(256) k_dgs_p_gather(Lev L, T *__restrict__ x, const T *__restrict__ delta,
                                                      Coef<T> K) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)L.nx * L.ny * L.nz) return;
    int i, j, k;
    decode3(t, L.nx, L.ny, i, j, k);
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

// Eq. (ldist) backward sweep, one pressure colour: p_c += M_{.c}^T (b - L~x) / d with
//   M_{.c}^T r = sum_axes (r_high_face - r_low_face)/h + eta/h^2 (6 r_c - sum of the 6 neighbour r)
// Only p_c changes; same-colour cells read none of each other's values.
template <class T>
__global__ void __launch_bounds__(256) k_dgs_p_bwd(Lev L, T *__restrict__ x, const T *__restrict__ b, int colour,
                                                   Coef<T> K, T dP) {
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)cnt[0] * cnt[1] * cnt[2]) return;
    int i, j, k;
    decode3(t, cnt[0], cnt[1], i, j, k);
    i = lo[0] + 2 * i;
    j = lo[1] + 2 * j;
    k = lo[2] + 2 * k;
    T sf = T(0);
    sf += b[pidx(L, 0, i + 1, j, k)] - face_Lx(x, L, 0, i + 1, j, k, K);
    sf -= b[pidx(L, 0, i, j, k)] - face_Lx(x, L, 0, i, j, k, K);
    sf += b[pidx(L, 1, i, j + 1, k)] - face_Lx(x, L, 1, i, j + 1, k, K);
    sf -= b[pidx(L, 1, i, j, k)] - face_Lx(x, L, 1, i, j, k, K);
    sf += b[pidx(L, 2, i, j, k + 1)] - face_Lx(x, L, 2, i, j, k + 1, K);
    sf -= b[pidx(L, 2, i, j, k)] - face_Lx(x, L, 2, i, j, k, K);
    T rc = b[pidx(L, 3, i, j, k)] - cell_Lx(x, L, i, j, k, K);
    T rn = T(0);
    rn += b[pidx(L, 3, i - 1, j, k)] - cell_Lx(x, L, i - 1, j, k, K);
    rn += b[pidx(L, 3, i + 1, j, k)] - cell_Lx(x, L, i + 1, j, k, K);
    rn += b[pidx(L, 3, i, j - 1, k)] - cell_Lx(x, L, i, j - 1, k, K);
    rn += b[pidx(L, 3, i, j + 1, k)] - cell_Lx(x, L, i, j + 1, k, K);
    rn += b[pidx(L, 3, i, j, k - 1)] - cell_Lx(x, L, i, j, k - 1, K);
    rn += b[pidx(L, 3, i, j, k + 1)] - cell_Lx(x, L, i, j, k + 1, K);
    T s = K.ih * sf + K.eh2 * (T(6) * rc - rn);
    x[pidx(L, 3, i, j, k)] += s / dP;
}

template <class T> static T dgs_pressure_diag(const Lev &L) {
    return T(-6.0 * (1.0 + L.gamma * L.eta) / (L.h * L.h));
}

template <class T> void launch_dgs_p_fwd(const Lev &L, T *x, const T *b, T *delta, int colour, cudaStream_t s) {
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    long long m = (long long)cnt[0] * cnt[1] * cnt[2];
    if (m == 0) return;
    k_dgs_p_fwd<T><<<blocks_for(m), kBlock, 0, s>>>(L, x, b, delta, colour, coef<T>(L, L.gamma),
                                                     dgs_pressure_diag<T>(L));
}
template <class T> void launch_dgs_p_gather(const Lev &L, T *x, const T *delta, cudaStream_t s) {
    long long m = (long long)L.nx * L.ny * L.nz;
    k_dgs_p_gather<T><<<blocks_for(m), kBlock, 0, s>>>(L, x, delta, coef<T>(L, L.gamma));
}
template <class T> void launch_dgs_p_bwd(const Lev &L, T *x, const T *b, int colour, cudaStream_t s) {
    int lo[3], cnt[3];
    v2_colour_range(L, colour, lo, cnt);
    long long m = (long long)cnt[0] * cnt[1] * cnt[2];
    if (m == 0) return;
    k_dgs_p_bwd<T><<<blocks_for(m), kBlock, 0, s>>>(L, x, b, colour, coef<T>(L, L.gamma), dgs_pressure_diag<T>(L));
}

// ------------------------------------------------------------------------------------------
// Vanka (Sec. 3.2): patch of cell c = its active faces [u_lo, u_hi, v_lo, v_hi, w_lo, w_hi] and
// p_c; correction = (C L~ C^T)^{-1} C (b - L~x) with the inverse of the cell's configuration
// (which faces are unknowns: 6-bit mask, 64 pre-factorised 7x7 inverses per level, Sec. 6).
// Corrections of one colour are computed from the pre-colour state, stored, then added.
template <class T>
__global__ void __launch_bounds__(256) k_vanka_compute(Lev L, const T *__restrict__ x, const T *__restrict__ b,
                                                       const int *__restrict__ cells, int ncell,
                                                       const T *__restrict__ kinv, T *__restrict__ corr, int cap,
                                                       Coef<T> K) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    int cl = cells[t];
    int i, j, k;
    decode3(cl, L.nx, L.ny, i, j, k);
    T r[7];
    int cfg = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        int d = a >> 1, side = a & 1;
        int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
        bool act = active(L, d, fi, fj, fk);
        cfg |= act ? (1 << a) : 0;
        r[a] = act ? b[pidx(L, d, fi, fj, fk)] - face_Lx(x, L, d, fi, fj, fk, K) : T(0);
    }
    r[6] = b[pidx(L, 3, i, j, k)] - cell_Lx(x, L, i, j, k, K);
    const T *Ki = kinv + cfg * 49;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        T s = T(0);
#pragma unroll
        for (int bb = 0; bb < 7; ++bb) s += Ki[a * 7 + bb] * r[bb];
        corr[(long long)a * cap + t] = s;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_vanka_apply(Lev L, T *__restrict__ x, const int *__restrict__ cells,
                                                     int ncell, const T *__restrict__ corr, int cap) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    int cl = cells[t];
    int i, j, k;
    decode3(cl, L.nx, L.ny, i, j, k);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        int d = a >> 1, side = a & 1;
        int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
        if (active(L, d, fi, fj, fk)) x[pidx(L, d, fi, fj, fk)] += corr[(long long)a * cap + t];
    }
    x[pidx(L, 3, i, j, k)] += corr[6LL * cap + t];
}

template <class T>
void launch_vanka_compute(const Lev &L, const T *x, const T *b, const int *cells, int ncell, const T *kinv, T *corr,
                          int cap, cudaStream_t s) {
    if (ncell <= 0) return;
    k_vanka_compute<T><<<blocks_for(ncell), kBlock, 0, s>>>(L, x, b, cells, ncell, kinv, corr, cap,
                                                             coef<T>(L, L.gamma));
}
template <class T>
void launch_vanka_apply(const Lev &L, T *x, const int *cells, int ncell, const T *corr, int cap, cudaStream_t s) {
    if (ncell <= 0) return;
    k_vanka_apply<T><<<blocks_for(ncell), kBlock, 0, s>>>(L, x, cells, ncell, corr, cap);
}

// ------------------------------------------------------------------------------------------
// Sec. 2 transfers.  P (coarse -> fine): pressure constant per coarse cell; a face value takes
// weight 1 from a coincident coarse face or 1/2 + 1/2 from the two coarse faces around it along
// its normal, and 3/4 (coarse row containing it) + 1/4 (next coarse row on the far side) along
// each tangential axis; coarse entries that are not unknowns contribute 0.  R = P^T / 8.
template <class T>
__global__ void __launch_bounds__(256) k_restrict(Lev F, Lev C, const T *__restrict__ rf, T *__restrict__ bc) {
    int c = blockIdx.y;
    int ex = ext(C, c, 0), ey = ext(C, c, 1), ez = ext(C, c, 2);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ex * ey * ez) return;
    int I, J, Kk;
    decode3(t, ex, ey, I, J, Kk);
    long long q = C.off[c] + t;
    if (!active(C, c, I, J, Kk)) {
        bc[q] = T(0);
        return;
    }
    if (c == 3) {
        T s = T(0);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            s += rf[pidx(F, 3, 2 * I + (m & 1), 2 * J + ((m >> 1) & 1), 2 * Kk + ((m >> 2) & 1))];
        bc[q] = s * T(0.125);
        return;
    }
    const int no[3] = {-1, 0, 1};
    const T nw[3] = {T(0.5), T(1), T(0.5)};
    const int to[4] = {-1, 0, 1, 2};
    const T tw[4] = {T(0.25), T(0.75), T(0.75), T(0.25)};
    int base[3] = {2 * I, 2 * J, 2 * Kk};
    int t1 = c == 0 ? 1 : 0, t2 = c == 2 ? 1 : 2;  // the two tangential axes
    T s = T(0);
    for (int a = 0; a < 3; ++a)
        for (int bb = 0; bb < 4; ++bb)
            for (int g = 0; g < 4; ++g) {
                int f[3];
                f[c] = base[c] + no[a];
                f[t1] = base[t1] + to[bb];
                f[t2] = base[t2] + to[g];
                s += nw[a] * tw[bb] * tw[g] * xget(rf, F, c, f[0], f[1], f[2]);
            }
    bc[q] = s * T(0.125);
}

template <class T>
__global__ void __launch_bounds__(256) k_prolong(Lev F, Lev C, const T *__restrict__ ec, T *__restrict__ xf) {
    int c = blockIdx.y;
    int ex = ext(F, c, 0), ey = ext(F, c, 1), ez = ext(F, c, 2);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ex * ey * ez) return;
    int fi[3];
    decode3(t, ex, ey, fi[0], fi[1], fi[2]);
    if (!active(F, c, fi[0], fi[1], fi[2])) return;
    long long q = F.off[c] + t;
    if (c == 3) {
        xf[q] += ec[pidx(C, 3, fi[0] / 2, fi[1] / 2, fi[2] / 2)];
        return;
    }
    int ci[3][2];
    T cw[3][2];
    int cn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d == c) {
            if ((fi[d] & 1) == 0) {
                cn[d] = 1; ci[d][0] = fi[d] / 2; cw[d][0] = T(1);
            } else {
                cn[d] = 2; ci[d][0] = (fi[d] - 1) / 2; ci[d][1] = (fi[d] + 1) / 2; cw[d][0] = cw[d][1] = T(0.5);
            }
        } else {
            cn[d] = 2;
            ci[d][0] = fi[d] / 2; cw[d][0] = T(0.75);
            ci[d][1] = (fi[d] & 1) == 0 ? fi[d] / 2 - 1 : fi[d] / 2 + 1; cw[d][1] = T(0.25);
        }
    }
    T s = T(0);
    for (int a = 0; a < cn[0]; ++a)
        for (int bb = 0; bb < cn[1]; ++bb)
            for (int g = 0; g < cn[2]; ++g)
                s += cw[0][a] * cw[1][bb] * cw[2][g] * xget(ec, C, c, ci[0][a], ci[1][bb], ci[2][g]);
    xf[q] += s;
}

template <class T> void launch_restrict(const Lev &F, const Lev &C, const T *rf, T *bc, cudaStream_t s) {
    dim3 grid(blocks_for(max_box(C, 4)), 4);
    k_restrict<T><<<grid, kBlock, 0, s>>>(F, C, rf, bc);
}
template <class T> void launch_prolong(const Lev &F, const Lev &C, const T *ec, T *xf, cudaStream_t s) {
    dim3 grid(blocks_for(max_box(F, 4)), 4);
    k_prolong<T><<<grid, kBlock, 0, s>>>(F, C, ec, xf);
}

// ------------------------------------------------------------------------------------------
// Alg. 1 exact coarsest solve: x[cidx[r]] = sum_k Kinv[r][k] b[cidx[k]] (FP64, one warp per row,
// deterministic lane-strided sums then a fixed shuffle tree)
template <class T>
__global__ void __launch_bounds__(256) k_coarse(const int *__restrict__ cidx, int nc, const double *__restrict__ kinv,
                                                const T *__restrict__ b, T *__restrict__ x) {
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
    (void)C;
    int rows_per_block = kBlock / 32;
    k_coarse<T><<<(nc + rows_per_block - 1) / rows_per_block, kBlock, nc * sizeof(double), s>>>(cidx, nc, kinv, b, x);
}

// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mask(Lev L, double *__restrict__ x) {
    int c = blockIdx.y;
    int ex = ext(L, c, 0), ey = ext(L, c, 1), ez = ext(L, c, 2);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ex * ey * ez) return;
    int i, j, k;
    decode3(t, ex, ey, i, j, k);
    if (!active(L, c, i, j, k)) x[L.off[c] + t] = 0.0;
}
void launch_mask(const Lev &L, double *x, cudaStream_t s) {
    dim3 grid(blocks_for(max_box(L, 4)), 4);
    k_mask<<<grid, kBlock, 0, s>>>(L, x);
}

template <class A, class B> __global__ void k_convert(long long n, const A *__restrict__ in, B *__restrict__ out) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = (B)in[t];
}
template <class A, class B> void launch_convert(long long n, const A *in, B *out, cudaStream_t s) {
    long long nb = (n + kBlock - 1) / kBlock;
    k_convert<A, B><<<(unsigned)(nb < 4736 ? nb : 4736), kBlock, 0, s>>>(n, in, out);
}

// explicit instantiations
#define SMG_INST(T)                                                                                               \
    template void launch_apply<T>(const Lev &, const T *, const T *, T *, double, cudaStream_t);                  \
    template void launch_dgs_u<T>(const Lev &, T *, const T *, int, cudaStream_t);                                \
    template void launch_dgs_p_fwd<T>(const Lev &, T *, const T *, T *, int, cudaStream_t);                       \
    template void launch_dgs_p_gather<T>(const Lev &, T *, const T *, cudaStream_t);                              \
    template void launch_dgs_p_bwd<T>(const Lev &, T *, const T *, int, cudaStream_t);                            \
    template void launch_vanka_compute<T>(const Lev &, const T *, const T *, const int *, int, const T *, T *, int, \
                                          cudaStream_t);                                                          \
    template void launch_vanka_apply<T>(const Lev &, T *, const int *, int, const T *, int, cudaStream_t);        \
    template void launch_restrict<T>(const Lev &, const Lev &, const T *, T *, cudaStream_t);                     \
    template void launch_prolong<T>(const Lev &, const Lev &, const T *, T *, cudaStream_t);                      \
    template void launch_coarse<T>(const Lev &, const int *, int, const double *, const T *, T *, cudaStream_t);
SMG_INST(float)
SMG_INST(double)
template void launch_convert<double, float>(long long, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(long long, const float *, double *, cudaStream_t);
template void launch_convert<double, double>(long long, const double *, double *, cudaStream_t);

}  // namespace smg
