// stokes_internal.cuh -- level descriptor, index math and stencil device functions shared by the
// CUDA kernels of the MAC Stokes multigrid-preconditioned SQMR solver (sm_103a).
//
// Discretisation (Tao & Sifakis, Sec. 2 Eq. 2 and Sec. 4):  for an active face f of component c
//   (L~x)_f = eta/h^2 (6 x_f - sum of its 6 same-component neighbours) + (p_plus - p_minus)/h
// and for a cell
//   (L~x)_c = -(sum over axes of (u_high - u_low))/h - gamma p_c      (gamma = 0 gives L).
// Box domain: a face is an unknown when its normal index lies in [1, n-1] and its tangential
// indices in [0, n-1]; every other referenced face (walls, ghost rows) contributes 0.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace smg {

// ---- storage vs arithmetic precision: level operands may be stored narrower (BF16) than the
// precision T a kernel computes in; ldv() widens a stored value, cvt<D>() rounds to storage type D
typedef __nv_bfloat16 bf16;
__device__ __forceinline__ float ldv(float v) { return v; }
__device__ __forceinline__ double ldv(double v) { return v; }
__device__ __forceinline__ float ldv(bf16 v) { return __bfloat162float(v); }
template <class D, class S> __device__ __forceinline__ D cvt(S v) { return (D)v; }
template <> __device__ __forceinline__ bf16 cvt<bf16, float>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ bf16 cvt<bf16, double>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ float cvt<float, bf16>(bf16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double cvt<double, bf16>(bf16 v) { return (double)__bfloat162float(v); }

// ---- programmatic dependent launch: every kernel is launched with programmatic stream
// serialisation, so its launch and block scheduling overlap the tail of the previous kernel in the
// stream; pdl_wait() (griddepcontrol.wait, a hardware dependency wait) holds the kernel until the
// previous kernel has completed and its memory is visible.  Every kernel calls it before touching
// global memory.
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
// griddepcontrol.launch_dependents: the next kernel in the stream may be scheduled once every block of
// this one has passed this point (or exited), so its blocks are resident and waiting in pdl_wait() when
// this kernel's last blocks finish.  It orders nothing: the next kernel still sees this one's writes only
// after its own pdl_wait(), which waits for this kernel's completion.
__device__ __forceinline__ void pdl_trigger() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.launch_dependents;" :::);
#endif
}
// the solver kernels' entry: wait for the previous kernel, then let the next one be scheduled
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

// set on a thread while it captures launches into a graph that must not carry programmatic edges
inline thread_local bool t_plain_launches = false;

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = t_plain_launches ? 0 : 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

struct Lev {
    int nx, ny, nz;
    long long off[4];  // offsets of the u, v, w, p blocks in the packed vector
    long long n;       // packed length
    double h, eta, gamma;
    // domains given by cell labels (Sec. 5): per packed entry, bit 0 = unknown, bit 1 = V2 DOF (the
    // Vanka set V1 is the rest of the unknowns), bit 2 = face of a Dirichlet cell (its value is data;
    // other faces that are not unknowns lie between two exterior cells and are 0); on an unknown
    // face bits 3-5 = how many viscous terms of its row drop out (do-nothing outflow condition next
    // to exterior cells), bit 6 / bit 7 = the low / high neighbour along the face normal is one of
    // them (its term crosses an exterior cell).  nullptr = the plain box, where all of this follows
    // from the indices
    const uint8_t *flags = nullptr;
    // batched handles: nb problems of this same level, problem p's buffers at byte offset p * bstride from
    // problem 0's (one stride per level for every per-problem buffer); a launch covers all of them, the
    // problem index taken from the grid (blockIdx.z = p * zpp + z-block for the 3D launches, blockIdx.y
    // for the 1D ones)
    int nb = 1;
    long long bstride = 0;
};
// problem slot of a batched 3D launch (gridDim.z = nb x the z blocks of one problem)
struct ZSlot {
    int p, z;
};
__device__ __forceinline__ ZSlot zslot(const Lev &L) {
    if (L.nb == 1) return {0, (int)blockIdx.z};
    const int zpp = (int)gridDim.z / L.nb, p = (int)blockIdx.z / zpp;
    return {p, (int)blockIdx.z - p * zpp};
}
// problem p's copy of a per-problem buffer
template <class P> __host__ __device__ __forceinline__ P *bslot(P *ptr, long long bstride, int p) {
    return ptr ? (P *)((char *)ptr + (long long)p * bstride) : ptr;
}
constexpr uint8_t kFlagActive = 1, kFlagV2 = 2, kFlagDirichlet = 4, kFlagDropLo = 64, kFlagDropHi = 128;
constexpr int kFlagDropShift = 3;
constexpr uint8_t kFlagDropMask = 0xf8;  // any dropped term
// diagonal weight of a face row: 6 minus the dropped terms
template <class T> __device__ __forceinline__ T diag_weight(uint8_t f) { return T(6 - ((f >> kFlagDropShift) & 7)); }

__host__ __device__ inline int ext(const Lev &L, int c, int d) {
    int n = d == 0 ? L.nx : (d == 1 ? L.ny : L.nz);
    return n + (c == d ? 1 : 0);
}

// linear index of entry (i,j,k) of component c (0 u, 1 v, 2 w, 3 p) in the packed vector
__host__ __device__ inline long long pidx(const Lev &L, int c, int i, int j, int k) {
    long long ex = ext(L, c, 0), ey = ext(L, c, 1);
    // select chain instead of L.off[c]: a runtime index into the parameter struct would spill it
    long long base = c == 0 ? L.off[0] : (c == 1 ? L.off[1] : (c == 2 ? L.off[2] : L.off[3]));
    return base + i + ex * (j + ey * (long long)k);
}

// is (c,i,j,k) an unknown of the box problem?  (normal index in [1, n-1], tangential in [0, n-1])
__host__ __device__ inline bool active(const Lev &L, int c, int i, int j, int k) {
    return i >= (c == 0) && j >= (c == 1) && k >= (c == 2) && i <= L.nx - 1 && j <= L.ny - 1 && k <= L.nz - 1;
}
// is (c,i,j,k) an unknown of the level's domain (box, or the cell labels' flags)?
__device__ __forceinline__ bool unknown(const Lev &L, int c, int i, int j, int k) {
    if (!active(L, c, i, j, k)) return false;
    return !L.flags || (L.flags[pidx(L, c, i, j, k)] & kFlagActive);
}
// does face (c,i,j,k) (any index, ghost faces included) carry Dirichlet data?  Faces outside the packed
// arrays touch the ghost shell, which is Dirichlet
__device__ __forceinline__ bool dirichlet_face(const Lev &L, int c, int i, int j, int k) {
    if (!L.flags) return true;
    const bool in = i >= 0 && j >= 0 && k >= 0 && i <= L.nx - 1 + (c == 0) && j <= L.ny - 1 + (c == 1) &&
                    k <= L.nz - 1 + (c == 2);
    return !in || (L.flags[pidx(L, c, i, j, k)] & kFlagDirichlet);
}
// is cell (i,j,k) a V2 cell (an interior cell none of whose six neighbours is a Dirichlet cell)?
__device__ __forceinline__ bool v2_cell_at(const Lev &L, int i, int j, int k) {
    if (!(i >= 1 && j >= 1 && k >= 1 && i <= L.nx - 2 && j <= L.ny - 2 && k <= L.nz - 2)) return false;
    return !L.flags || (L.flags[pidx(L, 3, i, j, k)] & kFlagV2);
}

template <class T>
__device__ __forceinline__ T xget(const T *__restrict__ x, const Lev &L, int c, int i, int j, int k) {
    return active(L, c, i, j, k) ? x[pidx(L, c, i, j, k)] : T(0);
}

template <class T> struct Coef {
    T eh2, ih, gam;  // eta/h^2, 1/h, gamma
};
template <class T> __host__ __device__ inline Coef<T> coef(const Lev &L, double gam) {
    Coef<T> k;
    k.eh2 = T(L.eta / (L.h * L.h));
    k.ih = T(1.0 / L.h);
    k.gam = T(gam);
    return k;
}

// (L~x) on an active face of component c at (i,j,k); neighbours that are not unknowns count 0
template <class T>
__device__ __forceinline__ T face_Lx(const T *__restrict__ x, const Lev &L, int c, int i, int j, int k,
                                     const Coef<T> &K) {
    T s = T(6) * x[pidx(L, c, i, j, k)];
    s -= xget(x, L, c, i - 1, j, k);
    s -= xget(x, L, c, i + 1, j, k);
    s -= xget(x, L, c, i, j - 1, k);
    s -= xget(x, L, c, i, j + 1, k);
    s -= xget(x, L, c, i, j, k - 1);
    s -= xget(x, L, c, i, j, k + 1);
    T pp = x[pidx(L, 3, i, j, k)];
    T pm = x[pidx(L, 3, i - (c == 0), j - (c == 1), k - (c == 2))];
    return K.eh2 * s + K.ih * (pp - pm);
}

// (L~x) on cell (i,j,k)
template <class T>
__device__ __forceinline__ T cell_Lx(const T *__restrict__ x, const Lev &L, int i, int j, int k, const Coef<T> &K) {
    T div = xget(x, L, 0, i + 1, j, k) - xget(x, L, 0, i, j, k) + xget(x, L, 1, i, j + 1, k) - xget(x, L, 1, i, j, k) +
            xget(x, L, 2, i, j, k + 1) - xget(x, L, 2, i, j, k);
    return -K.ih * div - K.gam * x[pidx(L, 3, i, j, k)];
}

// ---- fast stencils.  They rely on the invariant kept by every internal vector: entries that are
// not unknowns (wall-normal faces) hold 0.  A face stencil then needs a guard only for tangential
// neighbours outside the box (no array entry exists there); a cell stencil needs none.  All
// neighbour addresses are constant strides from one base address.
__host__ __device__ inline long long comp_base(const Lev &L, int c) {
    return c == 0 ? L.off[0] : (c == 1 ? L.off[1] : (c == 2 ? L.off[2] : L.off[3]));
}

// (L~x)_f on the active face (i,j,k) of component C (WITHP = false: the A part alone, no pressure loads)
template <class T, int C, bool WITHP = true>
__device__ __forceinline__ T face_Lx_fast(const T *__restrict__ x, const Lev &L, int i, int j, int k,
                                          const Coef<T> &K) {
    const long long sy = L.nx + (C == 0), sz = sy * (L.ny + (C == 1));
    const T *xc = x + comp_base(L, C) + i + sy * j + sz * k;
    T s = T(6) * xc[0];
    if (C == 0) s -= xc[-1] + xc[1];
    else s -= (i > 0 ? xc[-1] : T(0)) + (i < L.nx - 1 ? xc[1] : T(0));
    if (C == 1) s -= xc[-sy] + xc[sy];
    else s -= (j > 0 ? xc[-sy] : T(0)) + (j < L.ny - 1 ? xc[sy] : T(0));
    if (C == 2) s -= xc[-sz] + xc[sz];
    else s -= (k > 0 ? xc[-sz] : T(0)) + (k < L.nz - 1 ? xc[sz] : T(0));
    if (!WITHP) return K.eh2 * s;
    const long long cy = L.nx, cz = (long long)L.nx * L.ny;
    const T *pc = x + L.off[3] + i + cy * j + cz * k;
    const long long ps = C == 0 ? 1 : (C == 1 ? cy : cz);
    return K.eh2 * s + K.ih * (pc[0] - pc[-ps]);
}

// (L~x)_c on cell (i,j,k) (WITHG = false: -div u alone, no pressure load)
template <class T, bool WITHG = true>
__device__ __forceinline__ T cell_Lx_fast(const T *__restrict__ x, const Lev &L, int i, int j, int k,
                                          const Coef<T> &K) {
    const long long nx = L.nx, ny = L.ny;
    const T *u = x + L.off[0] + i + (nx + 1) * (j + ny * k);
    const T *v = x + L.off[1] + i + nx * (j + (ny + 1) * k);
    const T *w = x + L.off[2] + i + nx * (j + ny * k);
    T div = (u[1] - u[0]) + (v[nx] - v[0]) + (w[nx * ny] - w[0]);
    if (!WITHG) return -K.ih * div;
    return -K.ih * div - K.gam * x[L.off[3] + i + nx * (j + ny * k)];
}

// runtime component dispatch (the component is uniform across a thread block)
template <class T>
__device__ __forceinline__ T face_Lx_any(const T *__restrict__ x, const Lev &L, int c, int i, int j, int k,
                                         const Coef<T> &K) {
    return c == 0 ? face_Lx_fast<T, 0>(x, L, i, j, k, K)
                  : (c == 1 ? face_Lx_fast<T, 1>(x, L, i, j, k, K) : face_Lx_fast<T, 2>(x, L, i, j, k, K));
}

// ---- cell-centric evaluation: the thread that owns cell position (i,j,k), 0 <= i <= nx, ... ,
// produces the four packed entries sharing that index -- u(i,j,k), v(i,j,k), w(i,j,k), p(i,j,k) --
// as far as they exist, in one pass (shared index math, p(i,j,k) and the low faces loaded once).
// OP_APPLY: L~x  (faces eta/h^2 (6x - sum nbrs) + grad p, cells -div u - gamma p)
// OP_A_B:   faces eta/h^2 (6x - sum nbrs) only, cells -div u only (the p-free parts)
enum { OP_APPLY = 0, OP_A_B = 1 };
struct Quad {
    long long q[4];  // packed indices (valid where ex[c])
    bool ex[4];      // entry exists in the packed array
    bool act[4];     // entry is an unknown
};
__device__ __forceinline__ Quad quad_at(const Lev &L, int i, int j, int k) {
    Quad Q;
    const long long nx = L.nx, ny = L.ny;
    Q.ex[0] = j < L.ny && k < L.nz;
    Q.ex[1] = i < L.nx && k < L.nz;
    Q.ex[2] = i < L.nx && j < L.ny;
    Q.ex[3] = i < L.nx && j < L.ny && k < L.nz;
    Q.q[0] = L.off[0] + i + (nx + 1) * (j + ny * k);
    Q.q[1] = L.off[1] + i + nx * (j + (ny + 1) * k);
    Q.q[2] = L.off[2] + i + nx * (j + ny * k);
    Q.q[3] = L.off[3] + i + nx * (j + ny * k);
    Q.act[0] = Q.ex[0] && i >= 1 && i <= L.nx - 1;
    Q.act[1] = Q.ex[1] && j >= 1 && j <= L.ny - 1;
    Q.act[2] = Q.ex[2] && k >= 1 && k <= L.nz - 1;
    Q.act[3] = Q.ex[3];
    if (L.flags)
        for (int c = 0; c < 4; ++c) Q.act[c] = Q.act[c] && (L.flags[Q.q[c]] & kFlagActive);
    return Q;
}
// values of the four operator rows at (i,j,k) (0 for entries that are not unknowns); x holds 0
// off the unknowns.  A face row is formed as (w eta/h^2) x_f - (eta/h^2) (sum of its six neighbours),
// w = 6 on the box: one FP64 operation fewer per face than eta/h^2 (w x_f - neighbours), and the FP64
// operator apply is bound by the FP64 issue rate on this GPU
// LAB = true: a label domain (L.flags set), whose faces next to exterior cells drop viscous terms
template <class T, int OP, bool LAB = false>
__device__ __forceinline__ void quad_eval(const T *__restrict__ x, const Lev &L, int i, int j, int k, const Quad &Q,
                                          const Coef<T> &K, T out[4]) {
    const long long nx = L.nx, ny = L.ny;
    const long long uy = nx + 1, uz = (nx + 1) * ny, vy = nx, vz = nx * (ny + 1), wy = nx, wz = nx * ny;
    const long long py = nx, pz = nx * ny;
    T pc = Q.ex[3] ? x[Q.q[3]] : T(0);
    const bool gxm = i > 0, gxp = i < L.nx - 1, gym = j > 0, gyp = j < L.ny - 1, gzm = k > 0, gzp = k < L.nz - 1;
    out[0] = out[1] = out[2] = out[3] = T(0);
    // label domains: diagonal weight and the two normal neighbours of a face next to exterior cells
    // (the dropped viscous terms of the do-nothing outflow reading, Sec. 5); the box has none
    uint8_t f0 = 0, f1 = 0, f2 = 0;
    if (LAB) {
        if (Q.act[0]) f0 = L.flags[Q.q[0]];
        if (Q.act[1]) f1 = L.flags[Q.q[1]];
        if (Q.act[2]) f2 = L.flags[Q.q[2]];
    }
    if (Q.act[0]) {
        const T *u = x + Q.q[0];
        const T ul = (f0 & kFlagDropLo) ? T(0) : u[-1], uh = (f0 & kFlagDropHi) ? T(0) : u[1];
        const T ns = ((ul + uh) + ((gym ? u[-uy] : T(0)) + (gyp ? u[uy] : T(0)))) +
                     ((gzm ? u[-uz] : T(0)) + (gzp ? u[uz] : T(0)));
        out[0] = ((LAB ? diag_weight<T>(f0) : T(6)) * K.eh2) * u[0] - K.eh2 * ns;
        if (OP == OP_APPLY) out[0] += K.ih * (pc - x[Q.q[3] - 1]);
    }
    if (Q.act[1]) {
        const T *v = x + Q.q[1];
        const T vl = (f1 & kFlagDropLo) ? T(0) : v[-vy], vh = (f1 & kFlagDropHi) ? T(0) : v[vy];
        const T ns = (((gxm ? v[-1] : T(0)) + (gxp ? v[1] : T(0))) + (vl + vh)) +
                     ((gzm ? v[-vz] : T(0)) + (gzp ? v[vz] : T(0)));
        out[1] = ((LAB ? diag_weight<T>(f1) : T(6)) * K.eh2) * v[0] - K.eh2 * ns;
        if (OP == OP_APPLY) out[1] += K.ih * (pc - x[Q.q[3] - py]);
    }
    if (Q.act[2]) {
        const T *w = x + Q.q[2];
        const T wl = (f2 & kFlagDropLo) ? T(0) : w[-wz], wh = (f2 & kFlagDropHi) ? T(0) : w[wz];
        const T ns = (((gxm ? w[-1] : T(0)) + (gxp ? w[1] : T(0))) + ((gym ? w[-wy] : T(0)) + (gyp ? w[wy] : T(0)))) +
                     (wl + wh);
        out[2] = ((LAB ? diag_weight<T>(f2) : T(6)) * K.eh2) * w[0] - K.eh2 * ns;
        if (OP == OP_APPLY) out[2] += K.ih * (pc - x[Q.q[3] - pz]);
    }
    if (Q.act[3]) {
        const T *u = x + Q.q[0], *v = x + Q.q[1], *w = x + Q.q[2];
        T div = (u[1] - u[0]) + (v[vy] - v[0]) + (w[wz] - w[0]);
        out[3] = -K.ih * div;
        if (OP == OP_APPLY) out[3] -= K.gam * pc;
    }
}

// decode a per-component thread index t (< ex*ey*ez) into (i,j,k)
__device__ __forceinline__ void decode3(long long t, int ex, int ey, int &i, int &j, int &k) {
    i = (int)(t % ex);
    long long r = t / ex;
    j = (int)(r % ey);
    k = (int)(r / ey);
}

}  // namespace smg
