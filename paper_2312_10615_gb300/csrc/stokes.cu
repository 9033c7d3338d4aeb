// stokes.cu -- host orchestration and C ABI of the GB300 symmetric multigrid-preconditioned SQMR
// solver for the MAC Stokes system (Tao & Sifakis, arXiv 2312.10615).
//
//   stokes_create ...... Sec. 5 DOF classes, Alg. 1 re-discretised hierarchy, Sec. 6 Vanka tables,
//                        exact coarsest solve (symmetrised dense FP64 inverse)
//   mg_precondition .... Alg. 1 V-cycle with the Alg. 3 smoother, zero initial guess (Sec. 3)
//   sqmr_solve ......... Alg. 4
// Every numerical step runs in the CUDA kernels of kernels_level.cu / kernels_sqmr.cu; this file
// only schedules them, captures them in CUDA graphs and moves data across the C ABI.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <functional>
#include <map>

#include <nvtx3/nvToolsExt.h>
#include <memory>
#include <mutex>
#include <algorithm>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "setup_host.h"
#include "stokesmg.h"

using namespace smg;

namespace {

struct LevelBuf {
    Lev L;
    void *x = nullptr, *b = nullptr, *r = nullptr, *delta = nullptr, *kinv = nullptr, *corr = nullptr;
    void *t = nullptr;  // level-size scratch of the arithmetic type (distributive weighted Jacobi)
    int *vcells[8] = {};
    int *vtab[8] = {};  // per-cell entries of the inverse table (label domains with exterior cells only)
    int vcount[8] = {};
    int ntab = 64;      // local inverses in kinv (64 configurations of unknown faces, plus exterior variants)
    void *x2 = nullptr;  // second copy of the level's state (one-launch-per-colour Vanka, fused velocity DGS),
                         // 0 off the unknowns
    int ufused = 0;      // symmetric DGS with the fused out-of-place velocity passes
    float ums[2] = {0.f, 0.f};  // autotuner's time per symmetric DGS: in-place launches, fused passes
    int *shell = nullptr;  // the DOFs a Vanka patch reads or writes (copied into x2 at each sweep's start)
    int nshell = 0;
    int vcap = 0;
    VankaLists lists;
    int vmode = 0, vblocks = 0;  // Vanka schedule: 0 per-colour launches, 1 cooperative sweep of vblocks blocks,
                                 // 2 one-cluster sweep of vblocks CTAs, 3 one block on a shared-memory copy,
                                 // 4 one launch per colour step on two copies of the state
    float vms = 0.f;             // autotuner's time per symmetric sweep
    Tile rtile, ptile;           // tiles of the restriction from / prolongation into this level
    float rms = 0.f, pms = 0.f;  // autotuner's time per launch of each
};

int cuda_status(cudaError_t e) {
    cudaGetLastError();  // clear a non-sticky error so the context stays usable
    return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_status(e_);    \
    } while (0)

#define CKLAUNCH()                                        \
    do {                                                  \
        cudaError_t e_ = cudaGetLastError();              \
        if (e_ != cudaSuccess) return cuda_status(e_);    \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else if (prev == dev) prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

Lev make_level(int nx, int ny, int nz, double h, double eta, double gamma) {
    Lev L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    long long nu = (long long)(nx + 1) * ny * nz, nv = (long long)nx * (ny + 1) * nz, nw = (long long)nx * ny * (nz + 1);
    L.off[0] = 0; L.off[1] = nu; L.off[2] = nu + nv; L.off[3] = nu + nv + nw;
    L.n = L.off[3] + (long long)nx * ny * nz;
    L.h = h; L.eta = eta; L.gamma = gamma;
    return L;
}

// ---- domains given by cell labels (Sec. 5) on the ghost-extended cell grid, x fastest ----
struct Labels {
    int nx = 0, ny = 0, nz = 0;
    std::vector<uint8_t> lab;  // (nx+2)(ny+2)(nz+2); 0 interior, 1 Dirichlet, 2 exterior
    std::vector<uint8_t> prox;  // same grid: 1 where an interior cell is proximal (V1 cell), from finish()
    size_t lin(int i, int j, int k) const {
        return (size_t)(i + 1) + (size_t)(nx + 2) * ((j + 1) + (size_t)(ny + 2) * (k + 1));
    }
    uint8_t at(int i, int j, int k) const {  // i in -1..nx; beyond the ghost shell: Dirichlet
        if (i < -1 || j < -1 || k < -1 || i > nx || j > ny || k > nz) return 1;
        return lab[lin(i, j, k)];
    }
    bool interior(int i, int j, int k) const { return at(i, j, k) == 0; }
    bool dirichlet(int i, int j, int k) const { return at(i, j, k) == 1; }
    bool exterior(int i, int j, int k) const { return at(i, j, k) == 2; }
    // V1 cells (Sec. 5, "proximal"): interior cells with a Dirichlet cell among their 26 neighbours or an
    // exterior cell within Chebyshev distance 2.  Separable dilations of the two indicator fields.
    void finish() {
        const int ex = nx + 2, ey = ny + 2, ez = nz + 2;
        auto dilate = [&](std::vector<uint8_t> f, int r) {
            std::vector<uint8_t> g(f.size());
            const int ext[3] = {ex, ey, ez};
            const long long str[3] = {1, (long long)ex, (long long)ex * ey};
            for (int d = 0; d < 3; ++d) {
                for (int k = 0; k < ez; ++k)
                    for (int j = 0; j < ey; ++j)
                        for (int i = 0; i < ex; ++i) {
                            const int pos[3] = {i, j, k};
                            const long long q = i + (long long)ex * (j + (long long)ey * k);
                            uint8_t v = 0;
                            for (int o = -r; o <= r && !v; ++o) {
                                const int t = pos[d] + o;
                                if (t >= 0 && t < ext[d]) v = f[(size_t)(q + o * str[d])];
                            }
                            g[(size_t)q] = v;
                        }
                f.swap(g);
            }
            return f;
        };
        std::vector<uint8_t> dir(lab.size()), ext2(lab.size());
        for (size_t q = 0; q < lab.size(); ++q) {
            dir[q] = lab[q] == 1;
            ext2[q] = lab[q] == 2;
        }
        dir = dilate(dir, 1);
        ext2 = dilate(ext2, 2);
        prox.assign(lab.size(), 0);
        for (size_t q = 0; q < lab.size(); ++q) prox[q] = lab[q] == 0 && (dir[q] || ext2[q]);
    }
    bool v1(int i, int j, int k) const { return interior(i, j, k) && prox[lin(i, j, k)]; }
    bool any_exterior() const {
        for (uint8_t v : lab)
            if (v == 2) return true;
        return false;
    }
};
// Sec. 5 coarsening: Dirichlet if any child is Dirichlet, else interior if any child is interior, else
// exterior
Labels coarsen(const Labels &F) {
    Labels C;
    C.nx = F.nx / 2; C.ny = F.ny / 2; C.nz = F.nz / 2;
    C.lab.assign((size_t)(C.nx + 2) * (C.ny + 2) * (C.nz + 2), 1);
    for (int k = 0; k < C.nz; ++k)
        for (int j = 0; j < C.ny; ++j)
            for (int i = 0; i < C.nx; ++i) {
                bool anyd = false, anyi = false;
                for (int m = 0; m < 8; ++m) {
                    const uint8_t l = F.at(2 * i + (m & 1), 2 * j + ((m >> 1) & 1), 2 * k + ((m >> 2) & 1));
                    anyd |= l == 1;
                    anyi |= l == 0;
                }
                const uint8_t v = anyd ? 1 : (anyi ? 0 : 2);
                C.lab[(size_t)(i + 1) + (size_t)(C.nx + 2) * ((j + 1) + (size_t)(C.ny + 2) * (k + 1))] = v;
            }
    C.finish();
    return C;
}
// per packed entry (Sec. 5): kFlagActive -- an unknown: an interior cell, or a face with no Dirichlet
// cell beside it and an interior cell on at least one side (between two interior cells, or a Neumann
// face between an interior and an exterior cell); kFlagV2 -- a face between two V2 cells, or a V2 cell;
// kFlagDirichlet -- a face of a Dirichlet cell (its value is data).  Faces that are none of these lie
// between two exterior cells (inactive).  For an unknown face, the viscous terms of its row that drop
// out (the do-nothing condition): bits 3-5 count them, kFlagDropLo / kFlagDropHi mark the two neighbours
// along the face normal whose term crosses an exterior cell (tangential drops are inactive faces,
// which hold 0, so the count alone fixes the row).
std::vector<uint8_t> level_flags(const Lev &L, const Labels &B) {
    std::vector<uint8_t> f((size_t)L.n, 0);
    auto face_dir = [&](int c, int i, int j, int k) {
        return B.dirichlet(i, j, k) || B.dirichlet(i - (c == 0), j - (c == 1), k - (c == 2));
    };
    auto face_unk = [&](int c, int i, int j, int k) {
        return !face_dir(c, i, j, k) && (B.interior(i, j, k) || B.interior(i - (c == 0), j - (c == 1), k - (c == 2)));
    };
    for (int c = 0; c < 4; ++c)
        for (int k = 0; k < ext(L, c, 2); ++k)
            for (int j = 0; j < ext(L, c, 1); ++j)
                for (int i = 0; i < ext(L, c, 0); ++i) {
                    uint8_t v = 0;
                    if (c == 3) {
                        if (B.interior(i, j, k)) v = kFlagActive | (B.v1(i, j, k) ? 0 : kFlagV2);
                    } else {
                        const int mi = i - (c == 0), mj = j - (c == 1), mk = k - (c == 2);
                        if (face_unk(c, i, j, k)) {
                            v = kFlagActive;
                            if (B.interior(i, j, k) && B.interior(mi, mj, mk) && !B.v1(i, j, k) && !B.v1(mi, mj, mk))
                                v |= kFlagV2;
                            int drops = 0;
                            if (B.exterior(mi, mj, mk)) { v |= kFlagDropLo; ++drops; }
                            if (B.exterior(i, j, k)) { v |= kFlagDropHi; ++drops; }
                            for (int d = 0; d < 3; ++d) {
                                if (d == c) continue;
                                for (int sg = -1; sg <= 1; sg += 2) {
                                    const int a = i + sg * (d == 0), b = j + sg * (d == 1), cc = k + sg * (d == 2);
                                    if (!face_dir(c, a, b, cc) && !face_unk(c, a, b, cc)) ++drops;
                                }
                            }
                            v |= (uint8_t)(drops << kFlagDropShift);
                        }
                        if (face_dir(c, i, j, k)) v |= kFlagDirichlet;
                    }
                    f[(size_t)pidx(L, c, i, j, k)] = v;
                }
    return f;
}

// process-wide cache of coarsest-level inverses (set-up cost grows as n^3)
std::mutex g_cache_mu;
std::map<std::tuple<int, int, int, double, double, double>, std::shared_ptr<std::vector<double>>> g_coarse_cache;

// dense L~ on the unknowns of level C (written from the stencil of Eq. 2 / Sec. 4), inverted
// and symmetrised: K^{-1} <- (K^{-1} + K^{-T}) / 2
int coarse_inverse(const Lev &C, const std::vector<uint8_t> *hflags, std::vector<int> &cidx,
                   std::shared_ptr<std::vector<double>> &out) {
    auto unk = [&](int c, int i, int j, int k) {
        return active(C, c, i, j, k) && (!hflags || ((*hflags)[(size_t)pidx(C, c, i, j, k)] & kFlagActive));
    };
    std::vector<long long> comp(C.n, -1);
    cidx.clear();
    for (int c = 0; c < 4; ++c)
        for (int k = 0; k < ext(C, c, 2); ++k)
            for (int j = 0; j < ext(C, c, 1); ++j)
                for (int i = 0; i < ext(C, c, 0); ++i)
                    if (unk(c, i, j, k)) {
                        long long q = pidx(C, c, i, j, k);
                        comp[q] = (long long)cidx.size();
                        cidx.push_back((int)q);
                    }
    int nc = (int)cidx.size();
    auto key = std::make_tuple(C.nx * 1000003 + C.ny, C.nz, nc, C.h, C.eta, C.gamma);
    if (!hflags) {  // box levels only: a label domain's coarse matrix depends on its labels
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_coarse_cache.find(key);
        if (it != g_coarse_cache.end()) { out = it->second; return 0; }
    }
    auto K = std::make_shared<std::vector<double>>((size_t)nc * nc, 0.0);
    double e2 = C.eta / (C.h * C.h), ih = 1.0 / C.h;
    auto put = [&](long long r, int c, int i, int j, int k, double v) {
        if (!unk(c, i, j, k)) return;
        (*K)[(size_t)comp[r] * nc + comp[pidx(C, c, i, j, k)]] += v;
    };
    for (int a = 0; a < nc; ++a) {
        long long q = cidx[a];
        int c = q < C.off[1] ? 0 : (q < C.off[2] ? 1 : (q < C.off[3] ? 2 : 3));
        long long t = q - C.off[c];
        int i = (int)(t % ext(C, c, 0)), j = (int)((t / ext(C, c, 0)) % ext(C, c, 1)),
            k = (int)(t / ((long long)ext(C, c, 0) * ext(C, c, 1)));
        if (c < 3) {
            // label domains: a face next to exterior cells drops viscous terms (bits 3-5 count them, the
            // two normal neighbours carry their own bits); inactive tangential neighbours are not unknowns
            const uint8_t f = hflags ? (*hflags)[(size_t)q] : (uint8_t)0;
            const int dlo = (f & kFlagDropLo) ? 0 : 1, dhi = (f & kFlagDropHi) ? 0 : 1;
            put(q, c, i, j, k, (6.0 - ((f >> kFlagDropShift) & 7)) * e2);
            put(q, c, i - 1, j, k, -e2 * (c == 0 ? dlo : 1)); put(q, c, i + 1, j, k, -e2 * (c == 0 ? dhi : 1));
            put(q, c, i, j - 1, k, -e2 * (c == 1 ? dlo : 1)); put(q, c, i, j + 1, k, -e2 * (c == 1 ? dhi : 1));
            put(q, c, i, j, k - 1, -e2 * (c == 2 ? dlo : 1)); put(q, c, i, j, k + 1, -e2 * (c == 2 ? dhi : 1));
            put(q, 3, i, j, k, ih);
            put(q, 3, i - (c == 0), j - (c == 1), k - (c == 2), -ih);
        } else {
            put(q, 0, i + 1, j, k, -ih); put(q, 0, i, j, k, ih);
            put(q, 1, i, j + 1, k, -ih); put(q, 1, i, j, k, ih);
            put(q, 2, i, j, k + 1, -ih); put(q, 2, i, j, k, ih);
            put(q, 3, i, j, k, -C.gamma);
        }
    }
    if (dense_inverse(nc, K->data())) return STOKES_ERR_INVALID_ARG;
    std::vector<double> &A = *K;
    for (int r = 0; r < nc; ++r)
        for (int c = r + 1; c < nc; ++c) {
            double v = 0.5 * (A[(size_t)r * nc + c] + A[(size_t)c * nc + r]);
            A[(size_t)r * nc + c] = v;
            A[(size_t)c * nc + r] = v;
        }
    if (!hflags) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_coarse_cache[key] = K;
    }
    out = K;
    return 0;
}

}  // namespace

struct stokes_s {
    int dev = 0;
    int prec = STOKES_PREC_FP64;
    int kb = 1;
    int use_graphs = 1;
    int vanka_persistent = 1;
    int vanka_max_blocks = 0;  // co-resident blocks of the cooperative Vanka sweep
    int nbf = 0;               // finest levels whose b, r are stored as BF16 (STOKES_PREC_MIXED_BF16)
    int additive = 0;          // Vanka variant: 0 symmetric multiplicative sweep, 1 damped additive (Eq. av)
    int cycle = 1;             // coarse-grid visits per level: 1 V-cycle, 2 W-cycle
    int dwj = 0;               // 1: symmetric distributive weighted Jacobi in place of the symmetric DGS
    long long ncell_active = 0;  // interior cells of the finest level (pressure-mean removal)
    bool neumann = false;        // some unknown face borders an exterior cell: no pressure null space
    // batched handle (stokes_create_batch): nb problems of this grid; every per-problem buffer of level l
    // lies in one allocation, problem p's at byte offset p * lev[l].L.bstride (level 0 also holds the SQMR
    // vectors, the reduction partials and the scalar state); one launch per step covers all problems
    int nb = 1;
    Bat bat() const { return Bat{nb, nb > 1 ? lev[0].L.bstride : 0LL}; }
    GridBarrier *bar = nullptr;
    double eta = 1.0, gamma = 1e-3;
    std::vector<LevelBuf> lev;
    int nc = 0;
    int *cidx = nullptr;
    double *ckinv = nullptr;
    // FP64 vectors of the finest level used by SQMR (s aliases lev[0].b in FP64 precision)
    double *x = nullptr, *s = nullptr, *q = nullptr, *d = nullptr, *r = nullptr, *w = nullptr, *bvec = nullptr;
    double *stage_in = nullptr, *stage_out = nullptr;
    double *partials = nullptr;
    SqmrState *st = nullptr;
    double *hout = nullptr;  // mapped pinned host memory written by the scalar kernel
    cudaStream_t cs = nullptr;
    cudaStream_t zs = nullptr;  // zero-fills new buffers (alloc)
    cudaGraphExec_t g_vcycle = nullptr, g_iter[2] = {nullptr, nullptr}, g_iter_id[2] = {nullptr, nullptr};
    // the SQMR loop as one graph (a while node around the iteration; [preconditioned][parity of its first
    // iteration]); loop_mode 0 = not built yet, 1 = built with the kernels' programmatic launch edges,
    // 2 = built without them, -1 = this driver refused it (the host drives the loop one iteration graph at
    // a time); device_loop = 0 keeps the host loop
    cudaGraphExec_t g_loop[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int loop_mode = 0;
    int device_loop = 1;
    LoopCtl *lctl = nullptr;  // device copy of the loop's stopping test
    double *q2 = nullptr;  // second SQMR direction buffer: iteration j writes q_j into (j odd ? q2 : q)
    int dx_blocks = 0;     // grid of the deferred iterate update beside the V-cycle (4 blocks per SM)
    // the deferred iterate update (d_j, x_j) runs on a side stream beside the next iteration's V-cycle
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::function<void(cudaStream_t)> fork;  // one-shot hook called by the V-cycle after the finest restriction
    std::function<void(cudaStream_t)> join;  // one-shot hook called by the V-cycle before the finest prolongation
    double *mgr = nullptr;  // FP64 residual of the pure-multigrid solver (FP32 V-cycles), on first use
    std::vector<void *> allocs;

    ~stokes_s() {
        if (g_vcycle) cudaGraphExecDestroy(g_vcycle);
        for (int p = 0; p < 2; ++p) {
            if (g_iter[p]) cudaGraphExecDestroy(g_iter[p]);
            if (g_iter_id[p]) cudaGraphExecDestroy(g_iter_id[p]);
        }
        for (auto &row : g_loop)
            for (cudaGraphExec_t g : row)
                if (g) cudaGraphExecDestroy(g);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        if (zs) cudaStreamDestroy(zs);
        for (void *p : allocs) cudaFree(p);
        if (hout) cudaFreeHost(hout);
        if (cs) cudaStreamDestroy(cs);
    }
    // zero-filled device buffer, complete before the call returns: the zeroing runs on the handle's own
    // non-blocking stream and is waited for, so work the caller then issues on any stream (buffers the
    // first solve allocates, on the caller's stream) sees the zeros
    template <class P> int alloc(P **p, size_t bytes) {
        void *v = nullptr;
        cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
        if (e != cudaSuccess) return cuda_status(e);
        allocs.push_back(v);
        if (!zs && (e = cudaStreamCreateWithFlags(&zs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_status(e);
        e = cudaMemsetAsync(v, 0, bytes ? bytes : 16, zs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(zs);
        if (e != cudaSuccess) return cuda_status(e);
        *p = (P *)v;
        return 0;
    }
    long long n0() const { return lev[0].L.n; }
    int nlev() const { return (int)lev.size(); }
};

namespace {

// ---- optional per-launch timing (stokes_profile_iteration): an event pair around every launch ----
struct Prof {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind, level;
};
thread_local Prof *g_prof = nullptr;
template <class F> inline void prof(int kind, int level, cudaStream_t s, F f) {
    if (!g_prof || 2 * g_prof->kind.size() + 1 >= g_prof->ev.size()) {
        f();
        return;
    }
    size_t i = g_prof->kind.size();
    g_prof->kind.push_back(kind);
    g_prof->level.push_back(level);
    cudaEventRecord(g_prof->ev[2 * i], s);
    f();
    cudaEventRecord(g_prof->ev[2 * i + 1], s);
}

// ---- the V-cycle schedule (Alg. 1 with the Alg. 3 smoother) ----
// T: arithmetic precision of the V-cycle; TB: storage of level l's b and r (T, or BF16 on the
// finest levels of the mixed-precision V-cycle); with_tb calls f(T(), TB()) for level l
template <class T, class F> void with_tb(const stokes_s *h, int l, F &&f) {
    if constexpr (std::is_same<T, float>::value) {
        if (l < h->nbf) {
            f(float(), bf16());
            return;
        }
    }
    f(T(), T());
}

template <class T, class TB> void vanka_colour(stokes_s *h, int l, int col, cudaStream_t s) {
    LevelBuf &B = h->lev[l];
    if (B.vcount[col] == 0) return;
    prof(STOKES_K_VANKA_COMPUTE, l, s, [&] {
        launch_vanka_compute<T, TB>(B.L, (const T *)B.x, (const TB *)B.b, B.vcells[col], B.vtab[col], B.vcount[col],
                                    (const T *)B.kinv, (T *)B.corr, B.vcap, 1.0, s);
    });
    prof(STOKES_K_VANKA_APPLY, l, s,
         [&] { launch_vanka_apply<T>(B.L, (T *)B.x, B.vcells[col], B.vcount[col], (const T *)B.corr, B.vcap, s); });
}
// Eq. (av), damped by 1/2 (a face lies in two patches): every colour's corrections from the same
// state into its own slice of the correction buffer, then added colour by colour
template <class T, class TB> void vanka_additive(stokes_s *h, int l, cudaStream_t s) {
    LevelBuf &B = h->lev[l];
    const size_t slice = (size_t)7 * B.vcap;
    for (int c = 0; c < 8; ++c) {
        if (B.vcount[c] == 0) continue;
        prof(STOKES_K_VANKA_COMPUTE, l, s, [&] {
            launch_vanka_compute<T, TB>(B.L, (const T *)B.x, (const TB *)B.b, B.vcells[c], B.vtab[c], B.vcount[c],
                                        (const T *)B.kinv, (T *)B.corr + c * slice, B.vcap, 0.5, s);
        });
    }
    for (int c = 0; c < 8; ++c) {
        if (B.vcount[c] == 0) continue;
        prof(STOKES_K_VANKA_APPLY, l, s, [&] {
            launch_vanka_apply<T>(B.L, (T *)B.x, B.vcells[c], B.vcount[c], (const T *)B.corr + c * slice, B.vcap, s);
        });
    }
}
// `sweeps` symmetric Vanka sweeps (App. C: colours 0..7 then 7..0)
template <class T, class TB> void vanka_sym(stokes_s *h, int l, cudaStream_t s, int sweeps = 1) {
    LevelBuf &B = h->lev[l];
    if (h->additive) {
        for (int k = 0; k < sweeps; ++k) vanka_additive<T, TB>(h, l, s);
        return;
    }
    if (B.vmode == 4 && !h->vanka_persistent && B.x2 && B.shell) {
        prof(STOKES_K_VANKA_COMPUTE, l, s, [&] {
            launch_vanka_pingpong<T, TB>(B.L, (T *)B.x, (T *)B.x2, (const TB *)B.b, B.lists, B.shell, B.nshell,
                                         (const T *)B.kinv, sweeps, s);
        });
        return;
    }
    if (B.vmode == 3 && !h->vanka_persistent) {
        prof(STOKES_K_VANKA_COMPUTE, l, s, [&] {
            launch_vanka_smem<T, TB>(B.L, (T *)B.x, (const TB *)B.b, B.lists, (const T *)B.kinv, B.vcap, sweeps, s);
        });
        return;
    }
    if (B.vmode == 2 && !h->vanka_persistent) {
        prof(STOKES_K_VANKA_COMPUTE, l, s, [&] {
            launch_vanka_cluster<T, TB>(B.L, (T *)B.x, (const TB *)B.b, B.lists, (const T *)B.kinv, (T *)B.corr, B.vcap,
                                        sweeps, B.vblocks, s);
        });
        return;
    }
    if (h->vanka_persistent || B.vmode == 1) {
        const int nb = B.vblocks > 0 && !h->vanka_persistent ? B.vblocks : h->vanka_max_blocks;
        prof(STOKES_K_VANKA_COMPUTE, l, s, [&] {
            launch_vanka_sweep<T, TB>(B.L, (T *)B.x, (const TB *)B.b, B.lists, (const T *)B.kinv, (T *)B.corr, B.vcap,
                                      sweeps, h->bar, nb, s);
        });
        return;
    }
    for (int k = 0; k < sweeps; ++k) {
        for (int c = 0; c < 8; ++c) vanka_colour<T, TB>(h, l, c, s);
        for (int c = 7; c >= 0; --c) vanka_colour<T, TB>(h, l, c, s);
    }
}
// fused: both velocity parities in one out-of-place pass from the level's x into its second buffer x2,
// the pressure colours then run on x2, and dgs_backward's fused velocity pass brings the state back
// into x (the symmetric DGS only; the same bits as the in-place launches)
template <class T, class TB> void dgs_forward(stokes_s *h, int l, cudaStream_t s, bool fused = false) {
    LevelBuf &B = h->lev[l];
    T *x = (T *)B.x;
    const TB *b = (const TB *)B.b;
    if (fused) {
        prof(STOKES_K_DGS_U, l, s, [&] { launch_dgs_u_fused<T, TB>(B.L, (const T *)B.x, (T *)B.x2, b, 0, s); });
        x = (T *)B.x2;
    } else {
        prof(STOKES_K_DGS_U, l, s, [&] { launch_dgs_u<T, TB>(B.L, x, b, 0, s); });
        prof(STOKES_K_DGS_U, l, s, [&] { launch_dgs_u<T, TB>(B.L, x, b, 1, s); });
    }
    for (int c = 0; c < 8; c += 2)
        prof(STOKES_K_DGS_P_FWD, l, s, [&] {
            if (!launch_dgs_p_fwd_pair<T, TB>(B.L, x, b, (T *)B.delta, c, s)) {
                launch_dgs_p_fwd<T, TB>(B.L, x, b, (T *)B.delta, c, s);
                launch_dgs_p_fwd<T, TB>(B.L, x, b, (T *)B.delta, c + 1, s);
            }
        });
}
// the forward sweep's pending neighbour-pressure part is applied by the first launch after it
template <class T> void dgs_finish_forward(stokes_s *h, int l, cudaStream_t s) {
    LevelBuf &B = h->lev[l];
    prof(STOKES_K_DGS_P_GATHER, l, s, [&] { launch_dgs_p_gather<T>(B.L, (T *)B.x, (const T *)B.delta, s); });
}
template <class T, class TB>
void dgs_backward(stokes_s *h, int l, cudaStream_t s, bool forward_pending, bool fused = false) {
    LevelBuf &B = h->lev[l];
    T *x = fused ? (T *)B.x2 : (T *)B.x;
    const TB *b = (const TB *)B.b;
    prof(STOKES_K_DGS_P_BWD_PREP, l, s, [&] {
        launch_dgs_p_bwd_prep<T, TB>(B.L, x, b, (TB *)B.r, forward_pending ? (const T *)B.delta : nullptr, s);
    });
    for (int c = 7; c >= 0; c -= 2)
        prof(STOKES_K_DGS_P_BWD, l, s, [&] {
            if (!launch_dgs_p_bwd_pair<T, TB>(B.L, x, (const TB *)B.r, c, s)) {
                launch_dgs_p_bwd<T, TB>(B.L, x, (const TB *)B.r, c, s);
                launch_dgs_p_bwd<T, TB>(B.L, x, (const TB *)B.r, c - 1, s);
            }
        });
    if (fused) {
        prof(STOKES_K_DGS_U, l, s, [&] { launch_dgs_u_fused<T, TB>(B.L, (const T *)B.x2, (T *)B.x, b, 1, s); });
    } else {
        prof(STOKES_K_DGS_U, l, s, [&] { launch_dgs_u<T, TB>(B.L, x, b, 1, s); });
        prof(STOKES_K_DGS_U, l, s, [&] { launch_dgs_u<T, TB>(B.L, x, b, 0, s); });
    }
}
// Sec. 3.1 variant: symmetric distributive weighted Jacobi, weight 6/7 (the paper gives none; the
// classical pointwise-Jacobi smoothing weight of the 7-point Laplacian)
constexpr double kDwjOmega = 6.0 / 7.0;
template <class T, class TB> void dist_sym(stokes_s *h, int l, cudaStream_t s) {
    LevelBuf &B = h->lev[l];
    if (h->dwj) {
        prof(STOKES_K_DGS_U, l, s, [&] {
            launch_dwj_sym<T, TB>(B.L, (T *)B.x, (const TB *)B.b, (T *)B.t, (T *)B.delta, kDwjOmega, s);
        });
        return;
    }
    const bool fused = B.ufused && B.x2;
    dgs_forward<T, TB>(h, l, s, fused);
    dgs_backward<T, TB>(h, l, s, true, fused);
}
template <class T, class TB> void smooth(stokes_s *h, int l, cudaStream_t s) {
    vanka_sym<T, TB>(h, l, s, h->kb);
    dist_sym<T, TB>(h, l, s);
    vanka_sym<T, TB>(h, l, s, h->kb);
}
template <class T> void smooth_level(stokes_s *h, int l, cudaStream_t s) {
    with_tb<T>(h, l, [&](auto t, auto tb) { smooth<decltype(t), decltype(tb)>(h, l, s); });
}
// NVTX range for the host-side trace (the work a call issues per multigrid level and per SQMR
// iteration; in eager mode the ranges bracket the launches, under graph capture the capture)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
const char *level_range_name(int l) {
    static const char *names[] = {"mg level 0", "mg level 1", "mg level 2", "mg level 3", "mg level 4",
                                  "mg level 5", "mg level 6", "mg level 7", "mg level 8", "mg level 9"};
    return l < 10 ? names[l] : "mg level >9";
}

// Alg. 1 from level l; first: x_l starts at 0 (else from its current value, the second coarse visit
// of a W-cycle); h->cycle coarse visits per level (1 V-cycle, 2 W-cycle, Sec. 8.2)
template <class T> void cycle_level(stokes_s *h, int l, bool first, cudaStream_t s) {
    NvtxRange range(level_range_name(l));
    const int n = h->nlev();
    if (l == n - 1) {
        LevelBuf &C = h->lev[n - 1];
        prof(STOKES_K_COARSE, n - 1, s,
             [&] { launch_coarse<T>(C.L, h->cidx, h->nc, h->ckinv, (const T *)C.b, (T *)C.x, s); });
        return;
    }
    LevelBuf &B = h->lev[l];
    if (first)
        prof(STOKES_K_MEMSET, l, s, [&] {
            if (B.L.nb > 1) cudaMemset2DAsync(B.x, (size_t)B.L.bstride, 0, sizeof(T) * B.L.n, B.L.nb, s);
            else cudaMemsetAsync(B.x, 0, sizeof(T) * B.L.n, s);
        });
    smooth_level<T>(h, l, s);
    with_tb<T>(h, l, [&](auto t, auto tf) {
        using TT = decltype(t);
        using TF = decltype(tf);
        prof(STOKES_K_RESIDUAL, l, s,
             [&] { launch_apply<TT, TF>(B.L, (const TT *)B.x, (const TF *)B.b, (TF *)B.r, B.L.gamma, s); });
        with_tb<T>(h, l + 1, [&](auto, auto tc) {
            using TC = decltype(tc);
            prof(STOKES_K_RESTRICT, l, s,
                 [&] { launch_restrict<TT, TF, TC>(B.L, h->lev[l + 1].L, (const TF *)B.r, (TC *)h->lev[l + 1].b, s,
                                                   B.rtile); });
        });
    });
    if (l == 0 && h->fork) {  // the coarse levels leave the finest level's bandwidth mostly idle
        auto f = h->fork;
        h->fork = nullptr;
        f(s);
    }
    for (int g = 0; g < h->cycle; ++g) cycle_level<T>(h, l + 1, g == 0, s);
    if (l == 0 && h->join) {  // back on the finest level: the side work has had the coarse levels
        auto f = h->join;
        h->join = nullptr;
        f(s);
    }
    prof(STOKES_K_PROLONG, l, s,
         [&] { launch_prolong<T>(B.L, h->lev[l + 1].L, (const T *)h->lev[l + 1].x, (T *)B.x, s, B.ptile); });
    smooth_level<T>(h, l, s);
}
template <class T> void vcycle(stokes_s *h, cudaStream_t s) { cycle_level<T>(h, 0, true, s); }
void vcycle_any(stokes_s *h, cudaStream_t s) {
    if (h->prec == STOKES_PREC_FP64) vcycle<double>(h, s);
    else vcycle<float>(h, s);
}

// t <- s_j unchanged: the identity in place of the preconditioner (plain SQMR, Alg. 4 with M = I)
template <class T> void identity_precond(stokes_s *h, cudaStream_t s) {
    const long long n = h->lev[0].L.n;
    if (h->prec == STOKES_PREC_FP64) cudaMemcpyAsync(h->lev[0].x, h->s, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    else launch_convert<double, float>(n, h->s, (float *)h->lev[0].x, s);
}

// one SQMR iteration (Alg. 4, loop body) on the finest level; precond = false: plain SQMR.  parity = j & 1
// of the iteration j: q_{j-1} is read from one of the two direction buffers and q_j written into the other
// (qbuf), and the previous iteration's deferred iterate update (d_{j-1}, x_{j-1}, which reads q_{j-2}) runs
// on the side stream beside this iteration's coarse levels, joined before anything overwrites its inputs
double *qbuf(stokes_s *h, int parity) { return parity ? h->q2 : h->q; }
template <class T> void sqmr_iteration(stokes_s *h, cudaStream_t s, bool precond, int parity) {
    const Lev &L = h->lev[0].L;
    long long n = L.n;
    T *t = (T *)h->lev[0].x;
    double *qprev = qbuf(h, parity ^ 1), *qnext = qbuf(h, parity);
    // t <- L q_{j-1}, sigma = q^T t ; alpha = rho / sigma
    int np = reduce_parts(L);
    const Bat bt = h->bat();
    prof(STOKES_K_APPLY_DOT, 0, s, [&] { launch_apply_dot(L, qprev, h->w, h->partials, s); });
    prof(STOKES_K_SCALARS, 0, s, [&] { launch_scalars(0, h->partials, np, h->st, h->hout, s, bt); });
    // s_j = s_{j-1} - alpha t
    with_tb<T>(h, 0, [&](auto, auto tb) {
        using TB = decltype(tb);
        prof(STOKES_K_UPDATE_S, 0, s, [&] {
            launch_update_s<TB>(n, h->s, h->w, h->st, h->prec == STOKES_PREC_FP64 ? nullptr : (TB *)h->lev[0].b, s, bt);
        });
    });
    // the previous iteration's d and x (pending flag on the device), on the side stream
    bool forked = false;
    auto lazy = [&](cudaStream_t ms) {
        cudaEventRecord(h->ev_fork, ms);
        cudaStreamWaitEvent(h->side, h->ev_fork, 0);
        prof(STOKES_K_UPDATE_X, 0, h->side,
             [&] { launch_update_dx(n, h->x, h->d, qnext, h->st, h->side, h->dx_blocks, bt); });
        cudaEventRecord(h->ev_join, h->side);
        forked = true;
    };
    bool joined = false;
    auto rejoin = [&](cudaStream_t ms) {
        cudaStreamWaitEvent(ms, h->ev_join, 0);
        joined = true;
    };
    if (precond) {
        h->fork = lazy;
        h->join = rejoin;
        vcycle<T>(h, s);  // t <- V-cycle(L~, s_j, 0, n)
        h->fork = nullptr;
        h->join = nullptr;
    } else {
        lazy(s);
        identity_precond<T>(h, s);
    }
    if (!forked) lazy(s);
    if (!joined) rejoin(s);
    // |t|^2, rho_j = s_j^T t ; nu, c, tau, beta
    prof(STOKES_K_DOT2, 0, s, [&] { launch_dot2<T>(n, t, h->s, h->partials, s, bt); });
    prof(STOKES_K_SCALARS, 0, s, [&] { launch_scalars(1, h->partials, kRedBlocks, h->st, h->hout, s, bt); });
    // recursive true residual r_j, q_j ; |r_j|^2 to the host ; d_j, x_j pending
    prof(STOKES_K_UPDATE_X, 0, s,
         [&] { launch_update_rq<T>(n, qprev, qnext, t, h->r, h->s, h->st, h->partials, s, bt); });
    prof(STOKES_K_SCALARS, 0, s, [&] { launch_scalars(2, h->partials, kRedBlocks, h->st, h->hout, s, bt); });
}
// apply the deferred d_j, x_j of the last completed iteration j (reads q_{j-1}) and clear the flag
void flush_iterate(stokes_s *h, int last_iter, cudaStream_t s) {
    launch_update_dx(h->n0(), h->x, h->d, qbuf(h, (last_iter - 1) & 1), h->st, s);
    cudaMemsetAsync(&h->st->dx_pending, 0, sizeof(int), s);
}
void sqmr_iteration_any(stokes_s *h, cudaStream_t s, int parity) {
    if (h->prec == STOKES_PREC_FP64) sqmr_iteration<double>(h, s, true, parity);
    else sqmr_iteration<float>(h, s, true, parity);
}
void sqmr_iteration_plain(stokes_s *h, cudaStream_t s, int parity) {
    if (h->prec == STOKES_PREC_FP64) sqmr_iteration<double>(h, s, false, parity);
    else sqmr_iteration<float>(h, s, false, parity);
}
void drop_graphs(stokes_s *h) {
    if (h->g_vcycle) { cudaGraphExecDestroy(h->g_vcycle); h->g_vcycle = nullptr; }
    for (auto &row : h->g_loop)
        for (cudaGraphExec_t &g : row)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (h->loop_mode > 0) h->loop_mode = 0;
    for (int p = 0; p < 2; ++p) {
        if (h->g_iter[p]) { cudaGraphExecDestroy(h->g_iter[p]); h->g_iter[p] = nullptr; }
        if (h->g_iter_id[p]) { cudaGraphExecDestroy(h->g_iter_id[p]); h->g_iter_id[p] = nullptr; }
    }
}

template <class F> int capture(stokes_s *h, F body, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cs, cudaStreamCaptureModeThreadLocal));
    body(h, h->cs);
    cudaError_t e = cudaStreamEndCapture(h->cs, &g);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e);
    return 0;
}

int run_vcycle(stokes_s *h, cudaStream_t s) {
    if (h->use_graphs) {
        if (!h->g_vcycle) {
            int rc = capture(h, vcycle_any, &h->g_vcycle);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(h->g_vcycle, s));
    } else {
        vcycle_any(h, s);
        CKLAUNCH();
    }
    return 0;
}

int run_iteration(stokes_s *h, cudaStream_t s, bool precond, int parity) {
    cudaGraphExec_t &g = precond ? h->g_iter[parity] : h->g_iter_id[parity];
    void (*fn)(stokes_s *, cudaStream_t, int) = precond ? sqmr_iteration_any : sqmr_iteration_plain;
    if (h->use_graphs) {
        if (!g) {
            int rc = capture(h, [&](stokes_s *hh, cudaStream_t cs) { fn(hh, cs, parity); }, &g);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(g, s));
    } else {
        fn(h, s, parity);
        CKLAUNCH();
    }
    return 0;
}

// The SQMR loop in one graph: while (go) { iteration p; test; if (go) { iteration 1 - p; test } }.  The
// test kernel (launch_loop_check) sets the while node's handle and the if node's, so consecutive
// iterations run without the host; the graph returns when an iteration stops the loop, and the host then
// does what it does after every iteration of its own loop (explicit residual, flush, restart).
int build_loop(stokes_s *h, bool precond, int p0, cudaGraphExec_t *out) {
    void (*fn)(stokes_s *, cudaStream_t, int) = precond ? sqmr_iteration_any : sqmr_iteration_plain;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle hw = 0, hi = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, g, 0, cudaGraphCondAssignDefault);
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp);
    // capture one iteration and its test into a body graph
    auto capture_into = [&](cudaGraph_t body, int parity, int set_if) {
        cudaError_t ce = cudaStreamBeginCaptureToGraph(h->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return ce;
        fn(h, h->cs, parity);
        launch_loop_check(h->st, h->lctl, hw, hi, set_if, h->hout, h->cs);
        cudaGraph_t got = nullptr;
        ce = cudaStreamEndCapture(h->cs, &got);
        return ce;
    };
    cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess) e = capture_into(body, p0, 1);
    // the body's last node (the test) carries the if node
    cudaGraphNode_t sink = nullptr;
    if (e == cudaSuccess) {
        size_t nn = 0;
        e = cudaGraphGetNodes(body, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(body, nodes.data(), &nn);
        int nsink = 0;
        for (size_t k = 0; e == cudaSuccess && k < nn; ++k) {
            size_t nd = 0;
            e = cudaGraphNodeGetDependentNodes(nodes[k], nullptr, nullptr, &nd);
            if (e == cudaSuccess && nd == 0) {
                sink = nodes[k];
                ++nsink;
            }
        }
        if (e == cudaSuccess && nsink != 1) e = cudaErrorInvalidValue;
    }
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t in = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&in, body, &sink, nullptr, 1, &ip);
    if (e == cudaSuccess) e = capture_into(ip.conditional.phGraph_out[0], p0 ^ 1, 0);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(h->cs, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(h->cs, &junk);
            if (junk) cudaGraphDestroy(junk);
        }
        cudaGetLastError();
        return cuda_status(e);
    }
    *out = ex;
    return 0;
}
// the loop graphs of this solve kind, built on first use; false: use the host-driven loop
bool ensure_loop(stokes_s *h, bool precond) {
    if (!h->use_graphs || h->nb > 1 || h->loop_mode < 0 || !h->device_loop) return false;
    if (!h->lctl && h->alloc(&h->lctl, sizeof(LoopCtl))) return false;
    cudaGraphExec_t *g = h->g_loop[precond ? 1 : 0];
    if (g[0] && g[1]) return true;
    // first with the kernels' programmatic launch edges, then without them
    for (int plain = 0; plain < 2; ++plain) {
        t_plain_launches = plain != 0;
        int rc = 0;
        for (int p = 0; p < 2 && !rc; ++p)
            if (!g[p]) rc = build_loop(h, precond, p, &g[p]);
        t_plain_launches = false;
        if (!rc) {
            h->loop_mode = 1 + plain;
            return true;
        }
        for (int p = 0; p < 2; ++p)
            if (g[p]) { cudaGraphExecDestroy(g[p]); g[p] = nullptr; }
    }
    h->loop_mode = -1;
    return false;
}

// ---- autotuner: per smoothed level, time the Vanka schedule candidates on the level's own buffers
// (their contents do not matter for the timing and are zero at creation) and keep the fastest.
// Every candidate computes the same bits, so the choice changes speed only.
template <class T, class TB> float time_vanka(stokes_s *h, int l, int mode, int blocks, cudaStream_t s) {
    LevelBuf &B = h->lev[l];
    B.vmode = mode;
    B.vblocks = blocks;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s);
    for (int r = 0; r < 2; ++r) vanka_sym<T, TB>(h, l, s, 1);
    cudaEventRecord(e0, s);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) vanka_sym<T, TB>(h, l, s, 1);
    cudaEventRecord(e1, s);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        GridBarrier hb;
        if (cudaMemcpy(&hb, h->bar, sizeof(hb), cudaMemcpyDeviceToHost) != cudaSuccess || hb.err) ms = -1.f;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}
int autotune_vanka(stokes_s *h, int nsm) {
    cudaStream_t s = h->cs;
    // cluster sizes above 8 need the non-portable attribute; without it those candidates just fail
    if (h->prec == STOKES_PREC_FP64) vanka_cluster_prepare<double, double>();
    else {
        vanka_cluster_prepare<float, float>();
        vanka_cluster_prepare<float, bf16>();
    }
    cudaGetLastError();
    for (int l = 0; l < h->nlev() - 1; ++l) {
        LevelBuf &B = h->lev[l];
        int mx = 0;
        for (int c = 0; c < 8; ++c) mx = std::max(mx, B.vcount[c]);
        const int need = (int)((8LL * mx + 255) / 256);
        int best_mode = 0, best_blocks = 0;
        float best = -1.f;
        auto run = [&](auto t, auto tb) {
            using T = decltype(t);
            using TB = decltype(tb);
            best = time_vanka<T, TB>(h, l, 0, 0, s);
            const int cand[5] = {h->vanka_max_blocks, h->vanka_max_blocks / 2, nsm, nsm / 2, nsm / 4};
            for (int c = 0; c < 5; ++c) {
                const int nb = std::min(cand[c], need);
                if (nb < 1 || (c > 0 && nb == std::min(cand[c - 1], need))) continue;
                const float ms = time_vanka<T, TB>(h, l, 1, nb, s);
                if (ms > 0.f && (best < 0.f || ms < best)) {
                    best = ms;
                    best_mode = 1;
                    best_blocks = nb;
                }
            }
            // one launch per colour step on two copies of the state
            if (B.x2 && B.shell) {
                const float ms = time_vanka<T, TB>(h, l, 4, 0, s);
                if (ms > 0.f && (best < 0.f || ms < best)) {
                    best = ms;
                    best_mode = 4;
                    best_blocks = 0;
                }
            }
            // one block on a shared-memory copy of the level, where it fits
            if (B.ntab == 64 && vanka_smem_prepare<T, TB>(B.L, B.vcap)) {
                const float ms = time_vanka<T, TB>(h, l, 3, 1, s);
                if (ms > 0.f && (best < 0.f || ms < best)) {
                    best = ms;
                    best_mode = 3;
                    best_blocks = 1;
                }
            }
            cudaGetLastError();
            // one cluster of 4, 8 or 16 CTAs: worth it only where a colour fits in a few passes
            const int cl_need = (int)((8LL * mx + 1023) / 1024);
            for (int cl : {4, 8, 16}) {
                if (cl_need > 8 * cl || (cl > 4 && cl_need <= cl / 2)) continue;
                const float ms = time_vanka<T, TB>(h, l, 2, cl, s);
                if (ms > 0.f && (best < 0.f || ms < best)) {
                    best = ms;
                    best_mode = 2;
                    best_blocks = cl;
                }
            }
        };
        if (h->prec == STOKES_PREC_FP64) with_tb<double>(h, l, run);
        else with_tb<float>(h, l, run);
        B.vmode = best_mode;
        B.vblocks = best_blocks;
        B.vms = best > 0.f ? best : 0.f;
    }
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    CK(cudaStreamSynchronize(s));
    return 0;
}

// ---- autotuner: per level, the tile (block shape, z-planes per thread) of the restriction and the
// prolongation, timed on the level's own buffers; every candidate computes the same bits
const Tile kTileCand[] = {{32, 8, 8}, {32, 8, 4}, {32, 8, 2}, {32, 8, 1}, {32, 4, 1}, {16, 8, 1}, {8, 8, 1}, {8, 4, 1}};
constexpr int kNumTileCand = sizeof(kTileCand) / sizeof(kTileCand[0]);
template <class Fn> float time_launches(Fn fn, cudaStream_t s, int reps = 8) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int r = 0; r < 2; ++r) fn();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(e1, s);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}
int autotune_tiles(stokes_s *h) {
    cudaStream_t s = h->cs;
    for (int l = 0; l < h->nlev() - 1; ++l) {
        LevelBuf &F = h->lev[l];
        LevelBuf &C = h->lev[l + 1];
        auto run = [&](auto t, auto tf) {
            using T = decltype(t);
            using TF = decltype(tf);
            with_tb<T>(h, l + 1, [&](auto, auto tc) {
                using TC = decltype(tc);
                float best = -1.f;
                for (int c = 0; c < kNumTileCand; ++c) {
                    const Tile tl = kTileCand[c];
                    const float ms = time_launches(
                        [&] { launch_restrict<T, TF, TC>(F.L, C.L, (const TF *)F.r, (TC *)C.b, s, tl); }, s);
                    if (ms > 0.f && (best < 0.f || ms < best)) { best = ms; F.rtile = tl; F.rms = ms; }
                }
            });
            float best = -1.f;
            for (int c = 0; c < kNumTileCand; ++c) {
                const Tile tl = kTileCand[c];
                const float ms =
                    time_launches([&] { launch_prolong<T>(F.L, C.L, (const T *)C.x, (T *)F.x, s, tl); }, s);
                if (ms > 0.f && (best < 0.f || ms < best)) { best = ms; F.ptile = tl; F.pms = ms; }
            }
        };
        if (h->prec == STOKES_PREC_FP64) with_tb<double>(h, l, run);
        else with_tb<float>(h, l, run);
        // the timing runs leave arbitrary values in the level's work vectors: clear them
        const size_t es = h->prec == STOKES_PREC_FP64 ? sizeof(double) : sizeof(float);
        CK(cudaMemsetAsync(F.x, 0, es * F.L.n, s));
        CK(cudaMemsetAsync(C.x, 0, es * C.L.n, s));
    }
    CK(cudaStreamSynchronize(s));
    return 0;
}

// ---- the velocity passes of the symmetric DGS: two in-place launches per stage, or one fused
// out-of-place pass (x -> x2 -> x); with autotune the faster per level, timed on the level's buffers
int setup_dgs_fused(stokes_s *h, bool tune) {
    cudaStream_t s = h->cs;
    bool ok = true;
    if (h->prec == STOKES_PREC_FP64) ok = dgs_u_fused_prepare<double, double>();
    else ok = dgs_u_fused_prepare<float, float>() && dgs_u_fused_prepare<float, bf16>();
    cudaGetLastError();
    for (int l = 0; l < h->nlev() - 1; ++l) {
        LevelBuf &B = h->lev[l];
        B.ufused = 0;
        if (!ok || !B.x2 || h->dwj || !tune) continue;
        float t[2] = {-1.f, -1.f};
        for (int f = 0; f < 2; ++f) {
            B.ufused = f;
            auto run = [&](auto tt, auto tb) {
                using T = decltype(tt);
                using TB = decltype(tb);
                t[f] = time_launches([&] { dist_sym<T, TB>(h, l, s); }, s, 5);
            };
            if (h->prec == STOKES_PREC_FP64) with_tb<double>(h, l, run);
            else with_tb<float>(h, l, run);
        }
        B.ufused = (t[1] > 0.f && t[0] > 0.f && t[1] < t[0]) ? 1 : 0;
        B.ums[0] = t[0];
        B.ums[1] = t[1];
        // the timing runs leave arbitrary values in the level's buffers: both copies back to 0
        const size_t es = h->prec == STOKES_PREC_FP64 ? sizeof(double) : sizeof(float);
        CK(cudaMemsetAsync(B.x, 0, es * B.L.n, s));
        CK(cudaMemsetAsync(B.x2, 0, es * B.L.n, s));
    }
    CK(cudaStreamSynchronize(s));
    return 0;
}

// copy a caller vector (host or device) of n doubles into a device buffer the call may read
int stage_in(stokes_s *h, const double *p, long long n, double *dst_if_host, const double **out, cudaStream_t s) {
    if (is_device_ptr(p)) {
        *out = p;
        return 0;
    }
    CK(cudaMemcpyAsync(dst_if_host, p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    *out = dst_if_host;
    return 0;
}
int ensure_stage(stokes_s *h) {
    if (!h->stage_in) {
        int rc = h->alloc(&h->stage_in, sizeof(double) * h->n0());
        if (rc) return rc;
        rc = h->alloc(&h->stage_out, sizeof(double) * h->n0());
        if (rc) return rc;
    }
    return 0;
}

// level vector in/out (FP64 caller layout <-> precision T of the level buffers); entries off the
// unknowns are zeroed on the way in
// bf: the destination is a BF16 operand buffer (b or r of a level below h->nbf)
int to_level(stokes_s *h, const Lev &L, const double *src_dev, void *dst, cudaStream_t s, bool bf = false) {
    long long n = L.n;
    if (bf) {
        launch_convert<double, bf16>(n, src_dev, (bf16 *)dst, s);
        launch_mask<bf16>(L, (bf16 *)dst, s);
    } else if (h->prec == STOKES_PREC_FP64) {
        CK(cudaMemcpyAsync(dst, src_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        launch_mask<double>(L, (double *)dst, s);
    } else {
        launch_convert<double, float>(n, src_dev, (float *)dst, s);
        launch_mask<float>(L, (float *)dst, s);
    }
    CKLAUNCH();
    return 0;
}
// a caller vector copied into a handle buffer with the entries off the unknowns zeroed
int stage_masked(stokes_s *h, const double *p, double *dst, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, p, sizeof(double) * h->n0(), is_device_ptr(p) ? cudaMemcpyDeviceToDevice
                                                                           : cudaMemcpyHostToDevice, s));
    launch_mask<double>(h->lev[0].L, dst, s);
    CKLAUNCH();
    return 0;
}
int from_level(stokes_s *h, const void *src, double *dst_dev, long long n, cudaStream_t s, bool bf = false) {
    if (bf) launch_convert<bf16, double>(n, (const bf16 *)src, dst_dev, s);
    else if (h->prec == STOKES_PREC_FP64) CK(cudaMemcpyAsync(dst_dev, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else launch_convert<float, double>(n, (const float *)src, dst_dev, s);
    CKLAUNCH();
    return 0;
}

// read the two doubles the scalar kernel wrote to mapped host memory
int sync_read(stokes_s *h, cudaStream_t s, double *a, double *b) {
    CK(cudaStreamSynchronize(s));
    if (a) *a = h->hout[0];
    if (b) *b = h->hout[1];
    return 0;
}

int residual_norm2(stokes_s *h, const double *b, const double *x, double *w, double *out, cudaStream_t s) {
    int np = launch_residual_dot(h->lev[0].L, b, x, w, h->partials, s);
    launch_scalars(4, h->partials, np, h->st, h->hout, s);
    CKLAUNCH();
    return sync_read(h, s, out, nullptr);
}

}  // namespace

// ======================================================================================== C ABI

extern "C" {

void stokes_opts_default(stokes_opts_t *o) {
    if (!o) return;
    o->gamma = 1e-3;
    o->kb_vanka = 1;
    o->precision = STOKES_PREC_FP64;
    o->use_graphs = 1;
    o->vanka_persistent = 0;
    o->autotune = 1;
    o->vanka_additive = 0;
    o->cycle = 1;
    o->distributive_jacobi = 0;
}

const char *stokes_strerror(int st) {
    switch (st) {
    case STOKES_OK: return "ok";
    case STOKES_ERR_INVALID_ARG: return "invalid argument";
    case STOKES_ERR_OOM: return "out of memory";
    case STOKES_ERR_CUDA: return "CUDA runtime error";
    case STOKES_ERR_BREAKDOWN: return "SQMR breakdown (q^T L q = 0 or s^T t = 0)";
    case STOKES_ERR_NOT_CONVERGED: return "SQMR did not reach the tolerance within max_iter";
    case STOKES_ERR_NAN: return "non-finite value in the SQMR recurrences";
    case STOKES_ERR_TIMEOUT: return "device wait timed out";
    case STOKES_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

// host-side classification of a labelled domain on one level (no CUDA call): the per-entry flags the
// kernels read, for checking against an independent classification without a GPU
int stokes_label_flags(const stokes_grid_t *grid, const stokes_bc_t *bc, int level, uint8_t *flags, long long n) {
    if (!grid || !bc || !bc->cell_labels || !flags || level < 0) return STOKES_ERR_INVALID_ARG;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || grid->nx > 2047 || grid->ny > 2047 || grid->nz > 1023)
        return STOKES_ERR_INVALID_ARG;
    Labels lab;
    lab.nx = grid->nx; lab.ny = grid->ny; lab.nz = grid->nz;
    lab.lab.assign(bc->cell_labels, bc->cell_labels + (size_t)(grid->nx + 2) * (grid->ny + 2) * (grid->nz + 2));
    for (int k = -1; k <= grid->nz; ++k)
        for (int j = -1; j <= grid->ny; ++j)
            for (int i = -1; i <= grid->nx; ++i) {
                const uint8_t v = lab.at(i, j, k);
                const bool ghost = i < 0 || j < 0 || k < 0 || i >= grid->nx || j >= grid->ny || k >= grid->nz;
                if (v > 2 || (ghost && v != 1)) return STOKES_ERR_INVALID_ARG;
            }
    lab.finish();
    for (int l = 0; l < level; ++l) {
        if (lab.nx % 2 || lab.ny % 2 || lab.nz % 2 || lab.nx < 4 || lab.ny < 4 || lab.nz < 4) return STOKES_ERR_INVALID_ARG;
        lab = coarsen(lab);
    }
    const Lev L = make_level(lab.nx, lab.ny, lab.nz, 1.0, 1.0, 0.0);
    if (n != L.n) return STOKES_ERR_INVALID_ARG;
    const std::vector<uint8_t> f = level_flags(L, lab);
    std::memcpy(flags, f.data(), f.size());
    return STOKES_OK;
}

int stokes_create(const stokes_grid_t *grid, const stokes_bc_t *bc, double viscosity, const stokes_opts_t *opts,
                  stokes_t *out) {
    if (!grid || !out) return STOKES_ERR_INVALID_ARG;
    *out = nullptr;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || !(viscosity > 0.0)) return STOKES_ERR_INVALID_ARG;
    // packed Vanka cell coordinates hold 11 + 11 + 10 bits; the z extent folds into gridDim.z
    if (grid->nx > 2047 || grid->ny > 2047 || grid->nz > 1023) return STOKES_ERR_INVALID_ARG;
    // cell labels (Sec. 5): ghost shell Dirichlet (1), inner cells interior (0), Dirichlet (1) or exterior
    // (2).  A label array that describes the plain box is treated as the box.
    Labels lab0;
    bool labelled = false;
    if (bc && bc->cell_labels) {
        lab0.nx = grid->nx; lab0.ny = grid->ny; lab0.nz = grid->nz;
        lab0.lab.assign(bc->cell_labels, bc->cell_labels + (size_t)(grid->nx + 2) * (grid->ny + 2) * (grid->nz + 2));
        lab0.finish();
        for (int k = -1; k <= grid->nz; ++k)
            for (int j = -1; j <= grid->ny; ++j)
                for (int i = -1; i <= grid->nx; ++i) {
                    const uint8_t v = lab0.at(i, j, k);
                    const bool ghost = i < 0 || j < 0 || k < 0 || i >= grid->nx || j >= grid->ny || k >= grid->nz;
                    if (v > 2 || (ghost && v != 1)) return STOKES_ERR_INVALID_ARG;
                    if (!ghost && v != 0) labelled = true;
                }
    }
    stokes_opts_t o;
    stokes_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.gamma >= 0.0) || o.kb_vanka < 0 ||
        (o.precision != STOKES_PREC_FP64 && o.precision != STOKES_PREC_FP32 && o.precision != STOKES_PREC_MIXED_BF16) ||
        (o.vanka_additive != 0 && o.vanka_additive != 1) || o.cycle < 1 || o.cycle > 2 ||
        (o.distributive_jacobi != 0 && o.distributive_jacobi != 1))
        return STOKES_ERR_INVALID_ARG;
    int cmax = grid->coarsest_max > 0 ? grid->coarsest_max : 8;
    int nlev = grid->levels;
    if (nlev <= 0) {
        nlev = 1;
        int a = grid->nx, b = grid->ny, c = grid->nz;
        while (a % 2 == 0 && b % 2 == 0 && c % 2 == 0 && (a > cmax || b > cmax || c > cmax) && a >= 4 && b >= 4 &&
               c >= 4) {
            a /= 2; b /= 2; c /= 2; ++nlev;
        }
    } else {
        int a = grid->nx, b = grid->ny, c = grid->nz;
        for (int l = 1; l < nlev; ++l) {
            if (a % 2 || b % 2 || c % 2 || a < 4 || b < 4 || c < 4) return STOKES_ERR_INVALID_ARG;
            a /= 2; b /= 2; c /= 2;
        }
    }
    std::unique_ptr<stokes_s> h(new stokes_s());
    CK(cudaGetDevice(&h->dev));
    h->prec = o.precision;
    h->kb = o.kb_vanka;
    h->use_graphs = o.use_graphs;
    h->vanka_persistent = o.vanka_persistent;
    h->additive = o.vanka_additive;
    h->cycle = o.cycle;
    h->dwj = o.distributive_jacobi;
    h->eta = viscosity;
    h->gamma = o.gamma;
    double hh = grid->h > 0 ? grid->h : 1.0 / grid->nx;
    size_t es = h->prec == STOKES_PREC_FP64 ? sizeof(double) : sizeof(float);
    // mixed precision: the two finest levels (never the coarsest) keep b and r as BF16
    h->nbf = h->prec == STOKES_PREC_MIXED_BF16 ? std::min(2, nlev - 1) : 0;
    int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    std::vector<Labels> labs;
    std::vector<std::vector<uint8_t>> hflags;
    for (int l = 0; l < nlev; ++l) {
        LevelBuf B;
        B.L = make_level(nx, ny, nz, hh, viscosity, o.gamma);
        if (labelled) {
            labs.push_back(l == 0 ? lab0 : coarsen(labs.back()));
            hflags.push_back(level_flags(B.L, labs.back()));
        }
        h->lev.push_back(B);
        nx /= 2; ny /= 2; nz /= 2; hh *= 2.0;
    }
    h->ncell_active = (long long)grid->nx * grid->ny * grid->nz;
    if (labelled) {
        h->ncell_active = 0;
        for (int k = 0; k < grid->nz; ++k)
            for (int j = 0; j < grid->ny; ++j)
                for (int i = 0; i < grid->nx; ++i) h->ncell_active += lab0.interior(i, j, k) ? 1 : 0;
        if (h->ncell_active == 0) return STOKES_ERR_INVALID_ARG;
        for (uint8_t f : hflags[0])
            if ((f & kFlagActive) && (f & (kFlagDropLo | kFlagDropHi))) h->neumann = true;
        for (int l = 0; l < nlev; ++l) {
            uint8_t *fd = nullptr;
            int rc = h->alloc(&fd, hflags[l].size());
            if (rc) return rc;
            CK(cudaMemcpy(fd, hflags[l].data(), hflags[l].size(), cudaMemcpyHostToDevice));
            h->lev[l].L.flags = fd;
        }
    }
    // coarsest level: exact solve
    {
        LevelBuf &C = h->lev[nlev - 1];
        std::vector<int> cidx;
        long long nact = 0;
        for (int c = 0; c < 4; ++c) {
            long long cnt = 1;
            for (int d = 0; d < 3; ++d) {
                int n = d == 0 ? C.L.nx : (d == 1 ? C.L.ny : C.L.nz);
                cnt *= (c == d) ? (n - 1) : n;
            }
            nact += cnt;
        }
        if (nact > 6000) return STOKES_ERR_INVALID_ARG;  // dense inverse would not fit the design
        std::shared_ptr<std::vector<double>> K;
        int rc = coarse_inverse(C.L, labelled ? &hflags[nlev - 1] : nullptr, cidx, K);
        if (rc) return rc;
        h->nc = (int)cidx.size();
        if ((rc = h->alloc(&h->cidx, sizeof(int) * h->nc))) return rc;
        if ((rc = h->alloc(&h->ckinv, sizeof(double) * (size_t)h->nc * h->nc))) return rc;
        CK(cudaMemcpy(h->cidx, cidx.data(), sizeof(int) * h->nc, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ckinv, K->data(), sizeof(double) * (size_t)h->nc * h->nc, cudaMemcpyHostToDevice));
        if ((rc = h->alloc(&C.x, es * C.L.n))) return rc;
        if ((rc = h->alloc(&C.b, es * C.L.n))) return rc;
    }
    // smoothed levels
    for (int l = 0; l < nlev - 1; ++l) {
        LevelBuf &B = h->lev[l];
        const Lev &L = B.L;
        int rc;
        if ((rc = h->alloc(&B.x, es * L.n))) return rc;
        const size_t esb = l < h->nbf ? sizeof(bf16) : es;
        if ((rc = h->alloc(&B.b, esb * L.n))) return rc;
        if ((rc = h->alloc(&B.r, esb * L.n))) return rc;
        if ((rc = h->alloc(&B.delta, es * (size_t)L.nx * L.ny * L.nz))) return rc;
        if (h->dwj && (rc = h->alloc(&B.t, es * L.n))) return rc;
        // V1 cells (interior cells with a face on a Dirichlet cell, the ghost shell included) by colour
        std::vector<int> cells[8];
        for (int k = 0; k < L.nz; ++k)
            for (int j = 0; j < L.ny; ++j)
                for (int i = 0; i < L.nx; ++i) {
                    bool v1 = labelled ? labs[l].v1(i, j, k)
                                       : (i == 0 || j == 0 || k == 0 || i == L.nx - 1 || j == L.ny - 1 || k == L.nz - 1);
                    if (!v1) continue;
                    int col = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
                    cells[col].push_back(i | (j << 11) | (k << 22));  // packed coordinates
                }
        B.vcap = 1;
        for (int c = 0; c < 8; ++c) {
            B.vcount[c] = (int)cells[c].size();
            B.vcap = B.vcount[c] > B.vcap ? B.vcount[c] : B.vcap;
            if ((rc = h->alloc(&B.vcells[c], sizeof(int) * (cells[c].size() + 1)))) return rc;
            if (!cells[c].empty())
                CK(cudaMemcpy(B.vcells[c], cells[c].data(), sizeof(int) * cells[c].size(), cudaMemcpyHostToDevice));
        }
        if ((rc = h->alloc(&B.corr, es * 8 * 7 * (size_t)B.vcap))) return rc;  // 8 slices: additive Vanka
        // Sec. 6: pre-factorised local problems, one per configuration of unknown faces (entries 0..63).
        // Next to exterior cells a face's row drops viscous terms (Sec. 5 reading), which changes the
        // local matrix: each such cell gets the entry of its (configuration, dropped counts), appended
        // after the 64 and shared by every cell with the same key
        std::vector<int> keys;  // per table entry: cfg | drops of face a << (6 + 3a)
        for (int cfg = 0; cfg < 64; ++cfg) keys.push_back(cfg);
        bool ext_tab = false;
        std::vector<int> tabs[8];
        if (labelled && labs[l].any_exterior()) {
            std::map<int, int> id;
            for (int cfg = 0; cfg < 64; ++cfg) id[cfg] = cfg;
            const std::vector<uint8_t> &fl = hflags[l];
            for (int c = 0; c < 8; ++c)
                for (int w : cells[c]) {
                    const int i = w & 2047, j = (w >> 11) & 2047, k = (w >> 22) & 1023;
                    int key = 0;
                    for (int a = 0; a < 6; ++a) {
                        const int d = a >> 1, side = a & 1;
                        const int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
                        if (!active(L, d, fi, fj, fk)) continue;
                        const uint8_t f = fl[(size_t)pidx(L, d, fi, fj, fk)];
                        if (!(f & kFlagActive)) continue;
                        key |= 1 << a;
                        key |= ((f >> kFlagDropShift) & 7) << (6 + 3 * a);
                    }
                    auto it = id.find(key);
                    if (it == id.end()) {
                        it = id.emplace(key, (int)keys.size()).first;
                        keys.push_back(key);
                        ext_tab = true;
                    }
                    tabs[c].push_back(it->second);
                }
        }
        B.ntab = (int)keys.size();
        for (int c = 0; c < 8; ++c) {
            B.lists.cells[c] = B.vcells[c];
            B.lists.count[c] = B.vcount[c];
            B.lists.tab[c] = nullptr;
            if (ext_tab) {
                if ((rc = h->alloc(&B.vtab[c], sizeof(int) * (tabs[c].size() + 1)))) return rc;
                if (!tabs[c].empty())
                    CK(cudaMemcpy(B.vtab[c], tabs[c].data(), sizeof(int) * tabs[c].size(), cudaMemcpyHostToDevice));
                B.lists.tab[c] = B.vtab[c];
            }
        }
        std::vector<double> kd((size_t)B.ntab * 49, 0.0);
        for (int t = 0; t < B.ntab; ++t) {
            int drops[6];
            for (int a = 0; a < 6; ++a) drops[a] = (keys[t] >> (6 + 3 * a)) & 7;
            if (vanka_local_inverse(L.h, L.eta, L.gamma, keys[t] & 63, drops, &kd[(size_t)t * 49]))
                std::fill(&kd[(size_t)t * 49], &kd[(size_t)t * 49] + 49, 0.0);
        }
        if ((rc = h->alloc(&B.kinv, es * 49 * (size_t)B.ntab))) return rc;
        if (h->prec == STOKES_PREC_FP64) {
            CK(cudaMemcpy(B.kinv, kd.data(), sizeof(double) * 49 * B.ntab, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> kf(kd.begin(), kd.end());
            CK(cudaMemcpy(B.kinv, kf.data(), sizeof(float) * 49 * B.ntab, cudaMemcpyHostToDevice));
        }
        // the one-launch-per-colour Vanka schedule: a second copy of the state and the list of DOFs the
        // patches read or write (patch unknowns, their same-component neighbours and the pressures beside
        // each patch face)
        if (L.n < (1LL << 31)) {
            if ((rc = h->alloc(&B.x2, es * L.n))) return rc;
            CK(cudaMemset(B.x2, 0, es * L.n));
        }
        if (B.x2 && !h->additive && !h->vanka_persistent) {
            const std::vector<uint8_t> *fl = labelled ? &hflags[l] : nullptr;
            auto unk = [&](int c, int i, int j, int k) {
                return i >= 0 && j >= 0 && k >= 0 && i < ext(L, c, 0) && j < ext(L, c, 1) && k < ext(L, c, 2) &&
                       active(L, c, i, j, k) && (!fl || ((*fl)[(size_t)pidx(L, c, i, j, k)] & kFlagActive));
            };
            std::vector<uint8_t> mark((size_t)L.n, 0);
            auto put = [&](int c, int i, int j, int k) {
                if (unk(c, i, j, k)) mark[(size_t)pidx(L, c, i, j, k)] = 1;
            };
            for (int c = 0; c < 8; ++c)
                for (int w : cells[c]) {
                    const int i = w & 2047, j = (w >> 11) & 2047, k = (w >> 22) & 1023;
                    put(3, i, j, k);
                    for (int a = 0; a < 6; ++a) {
                        const int d = a >> 1, side = a & 1;
                        const int fi = i + (d == 0 ? side : 0), fj = j + (d == 1 ? side : 0), fk = k + (d == 2 ? side : 0);
                        if (!unk(d, fi, fj, fk)) continue;
                        put(d, fi, fj, fk);
                        for (int e = 0; e < 3; ++e)
                            for (int sg = -1; sg <= 1; sg += 2)
                                put(d, fi + sg * (e == 0), fj + sg * (e == 1), fk + sg * (e == 2));
                        put(3, fi, fj, fk);
                        put(3, fi - (d == 0), fj - (d == 1), fk - (d == 2));
                    }
                }
            std::vector<int> shell;
            for (size_t q = 0; q < mark.size(); ++q)
                if (mark[q]) shell.push_back((int)q);
            B.nshell = (int)shell.size();
            if ((rc = h->alloc(&B.shell, sizeof(int) * (shell.size() + 1)))) return rc;
            if (!shell.empty())
                CK(cudaMemcpy(B.shell, shell.data(), sizeof(int) * shell.size(), cudaMemcpyHostToDevice));
        }
    }
    // reduction scratch and scalar state (the SQMR vectors are allocated by the first sqmr_solve)
    {
        int rc;
        int nparts = reduce_parts(h->lev[0].L) > kRedBlocks ? reduce_parts(h->lev[0].L) : kRedBlocks;
        if ((rc = h->alloc(&h->partials, sizeof(double) * nparts * kRedParts))) return rc;
        if ((rc = h->alloc(&h->st, sizeof(SqmrState)))) return rc;
        CK(cudaHostAlloc((void **)&h->hout, 4 * sizeof(double), cudaHostAllocMapped));
        std::memset(h->hout, 0, 4 * sizeof(double));
    }
    CK(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
    {
        int rc, nsm = 0, coop = 0;
        if ((rc = h->alloc(&h->bar, sizeof(GridBarrier)))) return rc;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev));
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev));
        int per_sm = h->prec == STOKES_PREC_FP64 ? vanka_sweep_blocks_per_sm<double, double>()
                                                 : std::min(vanka_sweep_blocks_per_sm<float, float>(),
                                                            vanka_sweep_blocks_per_sm<float, bf16>());
        h->vanka_max_blocks = per_sm * nsm;
        if (!coop || h->vanka_max_blocks <= 0) h->vanka_persistent = 0;
        if (coop && h->vanka_max_blocks > 0 && !h->vanka_persistent && o.autotune && !h->additive) {
            if ((rc = autotune_vanka(h.get(), nsm))) return rc;
        }
        if (o.autotune && (rc = autotune_tiles(h.get()))) return rc;
        if ((rc = setup_dgs_fused(h.get(), o.autotune != 0))) return rc;
    }
    CK(cudaDeviceSynchronize());
    *out = h.release();
    return STOKES_OK;
}

int stokes_destroy(stokes_t h) {
    if (!h) return STOKES_OK;
    DeviceGuard g(h->dev);
    cudaDeviceSynchronize();
    delete h;
    return STOKES_OK;
}

long long stokes_vector_length(stokes_t h, int level) {
    if (!h || level < 0 || level >= h->nlev()) return 0;
    return h->lev[level].L.n;
}
long long stokes_ghost_length(stokes_t h) {
    if (!h) return 0;
    const Lev &L = h->lev[0].L;
    return (long long)(L.nx + 1) * (L.ny + 2) * (L.nz + 2) + (long long)(L.nx + 2) * (L.ny + 1) * (L.nz + 2) +
           (long long)(L.nx + 2) * (L.ny + 2) * (L.nz + 1);
}
int stokes_num_levels(stokes_t h) { return h ? h->nlev() : 0; }

int stokes_rhs(stokes_t h, const double *f, const double *g, double *b, void *stream) {
    if (!h || !b) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    const double *fd = nullptr, *gd = nullptr;
    double *gbuf = nullptr;
    if (f && (rc = stage_in(h, f, h->n0(), h->stage_in, &fd, s))) return rc;
    if (g) {
        if (is_device_ptr(g)) gd = g;
        else {
            long long ng = stokes_ghost_length(h);
            CK(cudaMallocAsync((void **)&gbuf, sizeof(double) * ng, s));
            CK(cudaMemcpyAsync(gbuf, g, sizeof(double) * ng, cudaMemcpyHostToDevice, s));
            gd = gbuf;
        }
    }
    bool bdev = is_device_ptr(b);
    double *bd = bdev ? b : h->stage_out;
    launch_rhs(h->lev[0].L, fd, gd, bd, s);
    CKLAUNCH();
    if (gbuf) CK(cudaFreeAsync(gbuf, s));
    if (!bdev) {
        CK(cudaMemcpyAsync(b, bd, sizeof(double) * h->n0(), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return STOKES_OK;
}

int stokes_apply(stokes_t h, const double *x, double *y, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !x || !y) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    if ((rc = stage_masked(h, x, h->stage_in, s))) return rc;
    bool ydev = is_device_ptr(y);
    double *yd = ydev ? y : h->stage_out;
    launch_apply<double, double>(h->lev[0].L, h->stage_in, nullptr, yd, 0.0, s);
    CKLAUNCH();
    if (!ydev) {
        CK(cudaMemcpyAsync(y, yd, sizeof(double) * h->n0(), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return STOKES_OK;
}

int mg_precondition(stokes_t h, const double *sv, double *tv, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !sv || !tv || (const double *)tv == sv) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    long long n = h->n0();
    if (!is_device_ptr(sv) || !is_device_ptr(tv))
        if ((rc = ensure_stage(h))) return rc;
    const double *sd;
    if ((rc = stage_in(h, sv, n, h->stage_in, &sd, s))) return rc;
    if ((rc = to_level(h, h->lev[0].L, sd, h->lev[0].b, s, h->nbf > 0))) return rc;
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    if ((rc = run_vcycle(h, s))) return rc;
    bool tdev = is_device_ptr(tv);
    double *td = tdev ? tv : h->stage_out;
    if ((rc = from_level(h, h->lev[0].x, td, n, s))) return rc;
    if (!tdev) {
        CK(cudaMemcpyAsync(tv, td, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return STOKES_OK;
}

int stokes_residual_norm(stokes_t h, const double *b, const double *x, double *out, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !b || !x || !out) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    const double *bd;
    if ((rc = ensure_stage(h))) return rc;
    if ((rc = stage_in(h, b, h->n0(), h->stage_in, &bd, s))) return rc;
    if ((rc = stage_masked(h, x, h->stage_out, s))) return rc;
    double r2 = 0.0;
    if ((rc = residual_norm2(h, bd, h->stage_out, nullptr, &r2, s))) return rc;
    *out = std::sqrt(r2);
    return STOKES_OK;
}

namespace {
// FP64 vectors of Alg. 4 on the finest level, allocated on first use
int ensure_side(stokes_s *h) {
    if (h->side) return 0;
    CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev));
    h->dx_blocks = 4 * nsm;
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    return 0;
}
int ensure_sqmr(stokes_s *h) {
    int rc = ensure_side(h);
    if (rc || h->x) return rc;
    long long n = h->n0();
    if ((rc = h->alloc(&h->x, sizeof(double) * n))) return rc;
    if ((rc = h->alloc(&h->q, sizeof(double) * n))) return rc;
    if ((rc = h->alloc(&h->q2, sizeof(double) * n))) return rc;
    if ((rc = h->alloc(&h->d, sizeof(double) * n))) return rc;
    if ((rc = h->alloc(&h->r, sizeof(double) * n))) return rc;
    if ((rc = h->alloc(&h->w, sizeof(double) * n))) return rc;
    if ((rc = h->alloc(&h->bvec, sizeof(double) * n))) return rc;
    if (h->prec == STOKES_PREC_FP64) h->s = (double *)h->lev[0].b;
    else if ((rc = h->alloc(&h->s, sizeof(double) * n))) return rc;
    return 0;
}

// Turn a freshly created handle into a batch of nb problems of its grid: every per-problem buffer of level l
// (x, b, r, the DGS deltas, the Vanka corrections; on level 0 also the SQMR vectors, reduction partials and
// scalar state) is re-laid in one allocation of nb slots of P_l bytes, problem p's copy at offset p P_l, and
// every level's Lev carries (nb, P_l) so that one launch covers all problems.  The schedule is the one that
// has a batched form: per-colour Vanka launches and in-place DGS (every schedule gives the same bits).
int make_batched(stokes_s *h, int nb) {
    const size_t es = h->prec == STOKES_PREC_FP64 ? sizeof(double) : sizeof(float);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const int nl = h->nlev();
    for (int l = 0; l < nl; ++l) {
        LevelBuf &B = h->lev[l];
        const Lev &L = B.L;
        const bool coarsest = l == nl - 1;
        const size_t esb = l < h->nbf ? sizeof(bf16) : es;
        std::vector<std::pair<void **, size_t>> bufs;
        bufs.push_back({&B.x, es * L.n});
        bufs.push_back({&B.b, (coarsest ? es : esb) * L.n});
        if (!coarsest) {
            bufs.push_back({&B.r, esb * L.n});
            bufs.push_back({&B.delta, es * (size_t)L.nx * L.ny * L.nz});
            bufs.push_back({&B.corr, es * 8 * 7 * (size_t)B.vcap});
        }
        void *partials = nullptr, *st = nullptr, *sv = nullptr;
        if (l == 0) {
            const size_t nv = sizeof(double) * L.n;
            for (double **v : {&h->x, &h->q, &h->q2, &h->d, &h->r, &h->w, &h->bvec})
                bufs.push_back({(void **)v, nv});
            if (h->prec != STOKES_PREC_FP64) bufs.push_back({&sv, nv});
            const int nparts = std::max(reduce_parts(L), kRedBlocks);
            bufs.push_back({&partials, sizeof(double) * nparts * kRedParts});
            bufs.push_back({&st, sizeof(SqmrState)});
        }
        size_t P = 0;
        std::vector<size_t> off;
        for (auto &b : bufs) {
            off.push_back(P);
            P += up(b.second);
        }
        uint8_t *arena = nullptr;
        int rc = h->alloc(&arena, P * (size_t)nb);
        if (rc) return rc;
        for (size_t k = 0; k < bufs.size(); ++k) *bufs[k].first = arena + off[k];
        if (l == 0) {
            h->partials = (double *)partials;
            h->st = (SqmrState *)st;
            h->s = h->prec == STOKES_PREC_FP64 ? (double *)B.b : (double *)sv;
        }
        B.L.nb = nb;
        B.L.bstride = (long long)P;
        B.x2 = nullptr;
        B.vmode = 0;
        B.vblocks = 0;
        B.ufused = 0;
        B.rtile = Tile();
        B.ptile = Tile();
    }
    h->nb = nb;
    // two host-visible values per problem
    if (h->hout) cudaFreeHost(h->hout);
    h->hout = nullptr;
    CK(cudaHostAlloc((void **)&h->hout, (2 * (size_t)nb + 2) * sizeof(double), cudaHostAllocMapped));
    std::memset(h->hout, 0, (2 * (size_t)nb + 2) * sizeof(double));
    drop_graphs(h);
    return ensure_side(h);
}
}  // namespace

namespace {
int sqmr_impl(stokes_t h, const double *rhs, double *xv, double tol, int max_iter, sqmr_info_t *info, void *stream,
              bool precond) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!h || !rhs || !xv || !(tol > 0.0) || max_iter < 0 || h->nb > 1) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const Lev &L = h->lev[0].L;
    long long n = L.n;
    int rc = ensure_sqmr(h);
    if (rc) return rc;
    // inputs
    if (is_device_ptr(rhs)) CK(cudaMemcpyAsync(h->bvec, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else CK(cudaMemcpyAsync(h->bvec, rhs, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    bool xdev = is_device_ptr(xv);
    CK(cudaMemcpyAsync(h->x, xv, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    launch_mask<double>(L, h->bvec, s);
    launch_mask<double>(L, h->x, s);
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    // |b|
    double bb = 0.0, ss = 0.0, rr = 0.0, flags = 0.0;
    launch_dot2<double>(n, h->bvec, nullptr, h->partials, s);
    launch_scalars(4, h->partials, kRedBlocks, h->st, h->hout, s);
    CKLAUNCH();
    if ((rc = sync_read(h, s, &bb, nullptr))) return rc;
    double nb = std::sqrt(bb);
    int it = 0, status = STOKES_OK;
    double rel = 0.0;
    bool rel_confirmed = false;  // rel holds the explicit FP64 residual of the returned x (up to the pressure shift)
    bool use_loop = false;       // the SQMR loop runs as one graph (g_loop)
    int pending = 0;             // iteration whose deferred d / x update has not been applied yet (0: none)
    if (!std::isfinite(nb)) {
        status = STOKES_ERR_NAN;
        goto finish;
    }
    if (nb == 0.0) {
        CK(cudaMemsetAsync(h->x, 0, sizeof(double) * n, s));
        goto finish;
    }
    // s_0 = b - L x_0 ; r_0 = s_0
    if ((rc = residual_norm2(h, h->bvec, h->x, h->s, &ss, s))) return rc;
    CK(cudaMemcpyAsync(h->r, h->s, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    rel = std::sqrt(ss) / nb;
    if (rel < tol) goto finish;
    // t = V-cycle(L~, s_0, 0, n) (or t = s_0); q_0 = t; tau_0 = |t|; rho_0 = s_0^T q_0; d = 0
    if (!precond) {
        if (h->prec == STOKES_PREC_FP64) identity_precond<double>(h, s);
        else identity_precond<float>(h, s);
    } else {
        if (h->nbf > 0) launch_convert<double, bf16>(n, h->s, (bf16 *)h->lev[0].b, s);
        else if (h->prec != STOKES_PREC_FP64) launch_convert<double, float>(n, h->s, (float *)h->lev[0].b, s);
        if ((rc = run_vcycle(h, s))) return rc;
    }
    if (h->prec == STOKES_PREC_FP64) {
        launch_dot2<double>(n, (const double *)h->lev[0].x, h->s, h->partials, s);
        launch_init_q<double>(n, (const double *)h->lev[0].x, h->q, h->d, s);
    } else {
        launch_dot2<float>(n, (const float *)h->lev[0].x, h->s, h->partials, s);
        launch_init_q<float>(n, (const float *)h->lev[0].x, h->q, h->d, s);
    }
    launch_scalars(3, h->partials, kRedBlocks, h->st, h->hout, s);
    CKLAUNCH();
    {
        double tt = 0.0, st0 = 0.0;
        if ((rc = sync_read(h, s, &tt, &st0))) return rc;
        if (!std::isfinite(tt) || !std::isfinite(st0)) { status = STOKES_ERR_NAN; goto finish; }
        if (tt == 0.0 || st0 == 0.0) { status = STOKES_ERR_BREAKDOWN; goto finish; }
    }
    status = STOKES_ERR_NOT_CONVERGED;
    if (max_iter > 0 && ensure_loop(h, precond)) {
        const LoopCtl lc = {nb, tol, max_iter, 0};
        CK(cudaMemcpyAsync(h->lctl, &lc, sizeof(lc), cudaMemcpyHostToDevice, s));
        use_loop = true;
    }
    for (it = 1; it <= max_iter; ++it) {
        NvtxRange range("sqmr iteration");
        if (use_loop) {
            // iterations it, it + 1, ... on the device until one stops the loop
            CK(cudaGraphLaunch(h->g_loop[precond ? 1 : 0][it & 1], s));
            if ((rc = sync_read(h, s, &rr, &flags))) return rc;
            it = (int)h->hout[2];
        } else {
            if ((rc = run_iteration(h, s, precond, it & 1))) return rc;
            if ((rc = sync_read(h, s, &rr, &flags))) return rc;
        }
        pending = it;
        int fl = (int)flags;
        if (fl & 2 || !std::isfinite(rr)) { status = STOKES_ERR_NAN; break; }
        if (fl & 1) { status = STOKES_ERR_BREAKDOWN; break; }
        if (std::sqrt(rr) / nb < tol) {
            // confirm with the explicit FP64 residual b - L x_j (x_j first takes its deferred update);
            // keep iterating from it otherwise
            flush_iterate(h, it, s);
            pending = 0;
            double r2 = 0.0;
            if ((rc = residual_norm2(h, h->bvec, h->x, h->w, &r2, s))) return rc;
            rel = std::sqrt(r2) / nb;
            if (rel < tol) {
                status = STOKES_OK;
                rel_confirmed = true;
                break;
            }
            CK(cudaMemcpyAsync(h->r, h->w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
    }
    if (it > max_iter) it = max_iter;
    if (pending) {  // the last iteration's d and x
        flush_iterate(h, pending, s);
        pending = 0;
    }
finish:
    // pressure fixed to zero mean (constant p lies in ker L) -- unless Neumann faces next to exterior
    // cells fix the pressure level (the exterior pressure is 0), where L has no null space
    if (!h->neumann) {
        launch_psum(L, h->x, h->partials, s);
        launch_scalars_aux(5, h->partials, kRedBlocks, h->st, h->hout, (double)h->ncell_active, s);
        launch_psub(L, h->x, h->st, s);
        CKLAUNCH();
    }
    // the residual reported: after a converged confirmation it is the one just computed (subtracting a
    // constant from the interior pressures changes L x only by rounding: the constant lies in ker L);
    // otherwise the explicit FP64 residual of the returned x
    if (!rel_confirmed) {
        double r2 = 0.0;
        if ((rc = residual_norm2(h, h->bvec, h->x, nullptr, &r2, s))) return rc;
        rel = nb > 0 ? std::sqrt(r2) / nb : 0.0;
    }
    CK(cudaMemcpyAsync(xv, h->x, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    {
        GridBarrier hb;
        CK(cudaMemcpyAsync(&hb, h->bar, sizeof(hb), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hb.err) status = STOKES_ERR_TIMEOUT;
    }
    if (info) {
        info->iterations = it;
        info->rel_residual = rel;
        info->status = status;
        info->vcycles = precond ? it + (it > 0 ? 1 : 0) : 0;
    }
    return status;
}
}  // namespace

namespace {
// Alg. 4 for every problem of a batched handle.  Each step of an iteration is one launch for all problems
// (the captured iteration graph); the host reads every problem's recursive residual after each iteration
// and confirms a converged problem with its own explicit FP64 residual, as the single solve does.  A
// problem that has converged (or stopped on an error) is frozen on the device: its SQMR kernels return,
// so its iterate keeps the bits of the single solve while the others go on.
int sqmr_batched_impl(stokes_t h, const double *const *rhs, double *const *xv, double tol, int max_iter,
                      sqmr_info_t *infos, void *stream) {
    if (!h || h->nb < 2 || !rhs || !xv || !(tol > 0.0) || max_iter < 0) return STOKES_ERR_INVALID_ARG;
    const int nb = h->nb;
    if (infos) std::memset(infos, 0, sizeof(sqmr_info_t) * nb);
    for (int p = 0; p < nb; ++p)
        if (!rhs[p] || !xv[p]) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    Lev L1 = h->lev[0].L;  // one problem's slice of the finest level
    L1.nb = 1;
    L1.bstride = 0;
    const long long n = L1.n, P = h->lev[0].L.bstride;
    auto S = [&](auto *ptr, int p) { return bslot(ptr, P, p); };
    static const int kZero = 0, kOne = 1;
    auto freeze = [&](int p, const int *v) {
        return cudaMemcpyAsync(&S(h->st, p)->frozen, v, sizeof(int), cudaMemcpyHostToDevice, s);
    };
    auto host = [&](int p, int k) { return h->hout[2 * p + k]; };
    const int np1 = reduce_parts(L1);
    std::vector<double> nbv(nb, 0.0), rel(nb, 0.0);
    std::vector<int> status(nb, STOKES_ERR_NOT_CONVERGED), its(nb, 0), confirmed(nb, 0), active(nb, 1), pending(nb, 0);
    // inputs
    for (int p = 0; p < nb; ++p) {
        CK(freeze(p, &kZero));
        CK(cudaMemcpyAsync(S(h->bvec, p), rhs[p], sizeof(double) * n,
                           is_device_ptr(rhs[p]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(S(h->x, p), xv[p], sizeof(double) * n,
                           is_device_ptr(xv[p]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        launch_mask<double>(L1, S(h->bvec, p), s);
        launch_mask<double>(L1, S(h->x, p), s);
        launch_dot2<double>(n, S(h->bvec, p), nullptr, S(h->partials, p), s);
        launch_scalars(4, S(h->partials, p), kRedBlocks, S(h->st, p), h->hout + 2 * p, s);
    }
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    for (int p = 0; p < nb; ++p) {
        nbv[p] = std::sqrt(host(p, 0));
        if (!std::isfinite(nbv[p])) {
            status[p] = STOKES_ERR_NAN;
            active[p] = 0;
        } else if (nbv[p] == 0.0) {
            CK(cudaMemsetAsync(S(h->x, p), 0, sizeof(double) * n, s));
            status[p] = STOKES_OK;
            active[p] = 0;
        }
    }
    // s_0 = b - L x_0 ; r_0 = s_0
    for (int p = 0; p < nb; ++p) {
        if (!active[p]) continue;
        launch_residual_dot(L1, S(h->bvec, p), S(h->x, p), S(h->s, p), S(h->partials, p), s);
        launch_scalars(4, S(h->partials, p), np1, S(h->st, p), h->hout + 2 * p, s);
        CK(cudaMemcpyAsync(S(h->r, p), S(h->s, p), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    for (int p = 0; p < nb; ++p) {
        if (!active[p]) continue;
        rel[p] = std::sqrt(host(p, 0)) / nbv[p];
        if (rel[p] < tol) {
            status[p] = STOKES_OK;
            active[p] = 0;
        }
    }
    auto any_active = [&] {
        for (int p = 0; p < nb; ++p)
            if (active[p]) return true;
        return false;
    };
    int rc = 0;
    if (any_active()) {
        // t = V-cycle(s_0) for all problems; q_0 = t ; tau_0, rho_0
        for (int p = 0; p < nb; ++p) {
            if (h->nbf > 0) launch_convert<double, bf16>(n, S(h->s, p), S((bf16 *)h->lev[0].b, p), s);
            else if (h->prec != STOKES_PREC_FP64)
                launch_convert<double, float>(n, S(h->s, p), S((float *)h->lev[0].b, p), s);
        }
        if ((rc = run_vcycle(h, s))) return rc;
        for (int p = 0; p < nb; ++p) {
            if (!active[p]) continue;
            if (h->prec == STOKES_PREC_FP64) {
                launch_dot2<double>(n, S((const double *)h->lev[0].x, p), S(h->s, p), S(h->partials, p), s);
                launch_init_q<double>(n, S((const double *)h->lev[0].x, p), S(h->q, p), S(h->d, p), s);
            } else {
                launch_dot2<float>(n, S((const float *)h->lev[0].x, p), S(h->s, p), S(h->partials, p), s);
                launch_init_q<float>(n, S((const float *)h->lev[0].x, p), S(h->q, p), S(h->d, p), s);
            }
            launch_scalars(3, S(h->partials, p), kRedBlocks, S(h->st, p), h->hout + 2 * p, s);
        }
        CKLAUNCH();
        CK(cudaStreamSynchronize(s));
        for (int p = 0; p < nb; ++p) {
            if (!active[p]) continue;
            const double tt = host(p, 0), st0 = host(p, 1);
            if (!std::isfinite(tt) || !std::isfinite(st0)) status[p] = STOKES_ERR_NAN;
            else if (tt == 0.0 || st0 == 0.0) status[p] = STOKES_ERR_BREAKDOWN;
            else continue;
            active[p] = 0;
        }
    }
    for (int p = 0; p < nb; ++p)
        if (!active[p]) CK(freeze(p, &kOne));
    // the deferred d, x update of problem p's last iteration (as flush_iterate, on p's slice)
    auto flush = [&](int p) -> int {
        if (!pending[p]) return 0;
        launch_update_dx(n, S(h->x, p), S(h->d, p), S(qbuf(h, (pending[p] - 1) & 1), p), S(h->st, p), s);
        CK(cudaMemsetAsync(&S(h->st, p)->dx_pending, 0, sizeof(int), s));
        pending[p] = 0;
        return 0;
    };
    for (int it = 1; it <= max_iter && any_active(); ++it) {
        NvtxRange range("sqmr batched iteration");
        if ((rc = run_iteration(h, s, true, it & 1))) return rc;
        for (int p = 0; p < nb; ++p)
            if (active[p]) {
                pending[p] = it;
                its[p] = it;
            }
        CK(cudaStreamSynchronize(s));
        for (int p = 0; p < nb; ++p) {
            if (!active[p]) continue;
            const double rr = host(p, 0);
            const int fl = (int)host(p, 1);
            if (fl & 2 || !std::isfinite(rr)) {
                status[p] = STOKES_ERR_NAN;
            } else if (fl & 1) {
                status[p] = STOKES_ERR_BREAKDOWN;
            } else if (std::sqrt(rr) / nbv[p] < tol) {
                // confirm with the explicit FP64 residual of x_j (its deferred update first)
                if ((rc = flush(p))) return rc;
                launch_residual_dot(L1, S(h->bvec, p), S(h->x, p), S(h->w, p), S(h->partials, p), s);
                launch_scalars(4, S(h->partials, p), np1, S(h->st, p), h->hout + 2 * p, s);
                CKLAUNCH();
                CK(cudaStreamSynchronize(s));
                rel[p] = std::sqrt(host(p, 0)) / nbv[p];
                if (rel[p] < tol) {
                    status[p] = STOKES_OK;
                    confirmed[p] = 1;
                } else {
                    CK(cudaMemcpyAsync(S(h->r, p), S(h->w, p), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                    continue;
                }
            } else {
                continue;
            }
            if ((rc = flush(p))) return rc;
            CK(freeze(p, &kOne));
            active[p] = 0;
        }
    }
    // problems still running used every iteration; then every problem's pressure level and reported residual
    for (int p = 0; p < nb; ++p) {
        if ((rc = flush(p))) return rc;
        if (!h->neumann) {
            launch_psum(L1, S(h->x, p), S(h->partials, p), s);
            launch_scalars_aux(5, S(h->partials, p), kRedBlocks, S(h->st, p), h->hout + 2 * p,
                               (double)h->ncell_active, s);
            launch_psub(L1, S(h->x, p), S(h->st, p), s);
        }
        if (!confirmed[p] && nbv[p] > 0.0 && std::isfinite(nbv[p])) {
            launch_residual_dot(L1, S(h->bvec, p), S(h->x, p), nullptr, S(h->partials, p), s);
            launch_scalars(4, S(h->partials, p), np1, S(h->st, p), h->hout + 2 * p, s);
            CKLAUNCH();
            CK(cudaStreamSynchronize(s));
            rel[p] = std::sqrt(host(p, 0)) / nbv[p];
        }
        CK(cudaMemcpyAsync(xv[p], S(h->x, p), sizeof(double) * n,
                           is_device_ptr(xv[p]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        CK(freeze(p, &kZero));
    }
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    int first_bad = STOKES_OK;
    for (int p = 0; p < nb; ++p) {
        if (infos) {
            infos[p].iterations = its[p];
            infos[p].rel_residual = rel[p];
            infos[p].status = status[p];
            infos[p].vcycles = its[p] + (its[p] > 0 ? 1 : 0);
        }
        if (status[p] != STOKES_OK && first_bad == STOKES_OK) first_bad = status[p];
    }
    return first_bad;
}
}  // namespace

extern "C" int sqmr_solve_batched(stokes_t h, const double *const *rhs, double *const *x, double tol, int max_iter,
                                  sqmr_info_t *infos, void *stream) {
    return sqmr_batched_impl(h, rhs, x, tol, max_iter, infos, stream);
}

extern "C" int sqmr_solve(stokes_t h, const double *rhs, double *xv, double tol, int max_iter, sqmr_info_t *info,
                          void *stream) {
    return sqmr_impl(h, rhs, xv, tol, max_iter, info, stream, true);
}

extern "C" int sqmr_solve_unpreconditioned(stokes_t h, const double *rhs, double *xv, double tol, int max_iter,
                                           sqmr_info_t *info, void *stream) {
    return sqmr_impl(h, rhs, xv, tol, max_iter, info, stream, false);
}

// Alg. 1 iterated as the solver on L~ x = b: x_{k+1} = x_k + V-cycle(L~, b - L~ x_k, 0, n), which equals
// the cycle started at x_k (every smoother step and the coarse correction are linear).  The residual
// b - L~ x_k and its norm are FP64; the cycle runs in the handle's precision.
extern "C" int mg_solve(stokes_t h, const double *rhs, double *xv, double tol, int max_iter, sqmr_info_t *info,
                        void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (info) std::memset(info, 0, sizeof(*info));
    if (!h || !rhs || !xv || !(tol > 0.0) || max_iter < 0) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const Lev &L = h->lev[0].L;
    long long n = L.n;
    int rc = ensure_sqmr(h);
    if (rc) return rc;
    const bool f64 = h->prec == STOKES_PREC_FP64;
    if (!f64 && !h->mgr && (rc = h->alloc(&h->mgr, sizeof(double) * n))) return rc;
    double *r = f64 ? (double *)h->lev[0].b : h->mgr;
    if (is_device_ptr(rhs)) CK(cudaMemcpyAsync(h->bvec, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else CK(cudaMemcpyAsync(h->bvec, rhs, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    bool xdev = is_device_ptr(xv);
    CK(cudaMemcpyAsync(h->x, xv, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    launch_mask<double>(L, h->bvec, s);
    launch_mask<double>(L, h->x, s);
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    double bb = 0.0, rr = 0.0;
    launch_dot2<double>(n, h->bvec, nullptr, h->partials, s);
    launch_scalars(4, h->partials, kRedBlocks, h->st, h->hout, s);
    CKLAUNCH();
    if ((rc = sync_read(h, s, &bb, nullptr))) return rc;
    const double nb = std::sqrt(bb);
    int k = 0, status = STOKES_ERR_NOT_CONVERGED;
    double rel = 0.0;
    if (!std::isfinite(nb)) status = STOKES_ERR_NAN;
    else if (nb == 0.0) {
        CK(cudaMemsetAsync(h->x, 0, sizeof(double) * n, s));
        status = STOKES_OK;
    } else
        for (k = 0;; ++k) {
            // r = b - L~ x_k and |r|^2 (FP64)
            launch_apply<double, double>(L, h->x, h->bvec, r, L.gamma, s);
            launch_dot2<double>(n, r, nullptr, h->partials, s);
            launch_scalars(4, h->partials, kRedBlocks, h->st, h->hout, s);
            CKLAUNCH();
            if ((rc = sync_read(h, s, &rr, nullptr))) return rc;
            rel = std::sqrt(rr) / nb;
            if (!std::isfinite(rel)) { status = STOKES_ERR_NAN; break; }
            if (rel < tol) { status = STOKES_OK; break; }
            if (k == max_iter) break;
            // x_{k+1} = x_k + V-cycle(L~, r, 0, n)
            if (h->nbf > 0) launch_convert<double, bf16>(n, r, (bf16 *)h->lev[0].b, s);
            else if (!f64) launch_convert<double, float>(n, r, (float *)h->lev[0].b, s);
            if ((rc = run_vcycle(h, s))) return rc;
            if (f64) launch_add_to<double>(n, (const double *)h->lev[0].x, h->x, s);
            else launch_add_to<float>(n, (const float *)h->lev[0].x, h->x, s);
            CKLAUNCH();
        }
    CK(cudaMemcpyAsync(xv, h->x, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    {
        GridBarrier hb;
        CK(cudaMemcpyAsync(&hb, h->bar, sizeof(hb), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hb.err) status = STOKES_ERR_TIMEOUT;
    }
    if (info) {
        info->iterations = k;
        info->rel_residual = rel;
        info->status = status;
        info->vcycles = k;
    }
    return status;
}

int stokes_profile_iteration(stokes_t h, int nkinds, double *ms_all, int *launches_all, double *ms_level0,
                             int *launches_level0, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || nkinds < STOKES_K_COUNT || !ms_all || !launches_all || !ms_level0 || !launches_level0)
        return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = ensure_sqmr(h);
    if (rc0) return rc0;
    Prof P;
    P.ev.resize(8192);
    for (auto &e : P.ev) CK(cudaEventCreate(&e));
    g_prof = &P;
    sqmr_iteration_any(h, s, 1);
    g_prof = nullptr;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int k = 0; k < nkinds; ++k) ms_all[k] = ms_level0[k] = 0.0, launches_all[k] = launches_level0[k] = 0;
    if (e == cudaSuccess)
        for (size_t i = 0; i < P.kind.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]);
            ms_all[P.kind[i]] += ms;
            launches_all[P.kind[i]] += 1;
            if (P.level[i] == 0) {
                ms_level0[P.kind[i]] += ms;
                launches_level0[P.kind[i]] += 1;
            }
        }
    for (auto &ev : P.ev) cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_status(e);
    return STOKES_OK;
}

int stokes_create_batch(int nprob, const stokes_grid_t *grid, const stokes_bc_t *bc, double viscosity,
                        const stokes_opts_t *opts, stokes_t *out) {
    if (!out) return STOKES_ERR_INVALID_ARG;
    *out = nullptr;
    if (nprob < 2 || nprob > 4096 || !grid) return STOKES_ERR_INVALID_ARG;
    stokes_opts_t o;
    stokes_opts_default(&o);
    if (opts) o = *opts;
    if (o.distributive_jacobi || !o.use_graphs) return STOKES_ERR_INVALID_ARG;
    o.autotune = 0;  // the batched schedule is fixed: per-colour Vanka launches, in-place DGS
    o.vanka_persistent = 0;
    // the problems fold into gridDim.z of the 3D launches (at most 4 (nz + 1) z blocks per problem)
    if ((long long)nprob * 4 * (grid->nz + 1) > 65535) return STOKES_ERR_INVALID_ARG;
    stokes_t h = nullptr;
    int rc = stokes_create(grid, bc, viscosity, &o, &h);
    if (rc) return rc;
    {
        DeviceGuard dg(h->dev);
        rc = make_batched(h, nprob);
        const cudaError_t e = cudaDeviceSynchronize();
        if (!rc && e != cudaSuccess) rc = cuda_status(e);
    }
    if (rc) {
        stokes_destroy(h);
        return rc;
    }
    *out = h;
    return STOKES_OK;
}

int stokes_batch_size(stokes_t h) { return h ? h->nb : 0; }

int stokes_device_loop(stokes_t h) { return h && h->loop_mode > 0 && h->device_loop ? h->loop_mode : 0; }

int stokes_set_device_loop(stokes_t h, int enable) {
    if (!h || (enable != 0 && enable != 1)) return STOKES_ERR_INVALID_ARG;
    h->device_loop = enable;
    return STOKES_OK;
}

int sqmr_solve_batch(int nprob, const stokes_t *handles, const double *const *rhs, double *const *x, double tol,
                     int max_iter, sqmr_info_t *infos, double *done_ms, int nstreams) {
    if (nprob <= 0 || !handles || !rhs || !x) return STOKES_ERR_INVALID_ARG;
    int dev = -1;
    for (int i = 0; i < nprob; ++i) {
        if (!handles[i] || !rhs[i] || !x[i] || handles[i]->nb > 1) return STOKES_ERR_INVALID_ARG;
        if (dev < 0) dev = handles[i]->dev;
        if (handles[i]->dev != dev) return STOKES_ERR_INVALID_ARG;  // one device per batch
    }
    int nt = nstreams < 1 ? 1 : (nstreams > nprob ? nprob : (nstreams > 64 ? 64 : nstreams));
    std::vector<int> status(nprob, STOKES_OK);
    std::atomic<int> next(0);
    std::atomic<int> setup_err(0);
    auto t0 = std::chrono::steady_clock::now();
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&]() {
            if (cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); setup_err = STOKES_ERR_CUDA; return; }
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                setup_err = STOKES_ERR_CUDA;
                return;
            }
            for (int i = next++; i < nprob; i = next++) {
                status[i] = sqmr_solve(handles[i], rhs[i], x[i], tol, max_iter, infos ? &infos[i] : nullptr, st);
                if (done_ms)
                    done_ms[i] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            }
            cudaStreamDestroy(st);
        });
    for (auto &th : pool) th.join();
    if (setup_err) return setup_err;
    for (int i = 0; i < nprob; ++i)
        if (status[i] != STOKES_OK) return status[i];
    return STOKES_OK;
}

int stokes_level_schedule(stokes_t h, int level, int *mode, int *blocks, float *ms) {
    if (!h || level < 0 || level >= h->nlev() - 1) return STOKES_ERR_INVALID_ARG;
    const LevelBuf &B = h->lev[level];
    const int m = h->vanka_persistent ? 1 : B.vmode;
    if (mode) *mode = m;
    if (blocks) *blocks = m == 0 ? 0 : (m == 1 && (h->vanka_persistent || B.vblocks <= 0) ? h->vanka_max_blocks : B.vblocks);
    if (ms) *ms = B.vms;
    return STOKES_OK;
}

int stokes_level_tiles(stokes_t h, int level, int *tiles, float *ms) {
    if (!h || level < 0 || level >= h->nlev() - 1 || !tiles) return STOKES_ERR_INVALID_ARG;
    const LevelBuf &B = h->lev[level];
    const Tile t[2] = {B.rtile, B.ptile};
    for (int k = 0; k < 2; ++k) {
        tiles[3 * k] = t[k].bx;
        tiles[3 * k + 1] = t[k].by;
        tiles[3 * k + 2] = t[k].kz;
    }
    if (ms) {
        ms[0] = B.rms;
        ms[1] = B.pms;
    }
    return STOKES_OK;
}

int stokes_set_level_tiles(stokes_t h, int level, const int *tiles) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || level < 0 || level >= h->nlev() - 1 || !tiles) return STOKES_ERR_INVALID_ARG;
    for (int k = 0; k < 2; ++k) {
        const int bx = tiles[3 * k], by = tiles[3 * k + 1], kz = tiles[3 * k + 2];
        if (bx < 1 || by < 1 || bx * by > 1024 || bx * by % 32 != 0 || kz < 1 || kz > 64) return STOKES_ERR_INVALID_ARG;
    }
    LevelBuf &B = h->lev[level];
    B.rtile = Tile{tiles[0], tiles[1], tiles[2]};
    B.ptile = Tile{tiles[3], tiles[4], tiles[5]};
    B.rms = B.pms = 0.f;
    // the captured graphs hold the old tiles
    drop_graphs(h);
    return STOKES_OK;
}

int stokes_level_dgs(stokes_t h, int level, int *fused, float *ms) {
    if (!h || level < 0 || level >= h->nlev() - 1) return STOKES_ERR_INVALID_ARG;
    const LevelBuf &B = h->lev[level];
    if (fused) *fused = B.ufused;
    if (ms) {
        ms[0] = B.ums[0];
        ms[1] = B.ums[1];
    }
    return STOKES_OK;
}

int stokes_set_level_dgs(stokes_t h, int level, int fused) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || level < 0 || level >= h->nlev() - 1 || (fused != 0 && fused != 1)) return STOKES_ERR_INVALID_ARG;
    LevelBuf &B = h->lev[level];
    if (fused && (!B.x2 || h->dwj)) return STOKES_ERR_UNSUPPORTED;
    B.ufused = fused;
    drop_graphs(h);
    return STOKES_OK;
}

int stokes_set_level_schedule(stokes_t h, int level, int mode, int blocks) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || level < 0 || level >= h->nlev() - 1 || mode < 0 || mode > 4) return STOKES_ERR_INVALID_ARG;
    if (mode == 4 && !h->lev[level].shell) return STOKES_ERR_UNSUPPORTED;
    if (mode == 1 && (h->vanka_max_blocks <= 0 || blocks < 1 || blocks > h->vanka_max_blocks)) return STOKES_ERR_INVALID_ARG;
    if (mode == 2 && (blocks < 1 || blocks > 16)) return STOKES_ERR_INVALID_ARG;
    if (mode == 3) {
        DeviceGuard dg(h->dev);
        const LevelBuf &B = h->lev[level];
        bool fits = false;
        if (h->prec == STOKES_PREC_FP64) fits = vanka_smem_prepare<double, double>(B.L, B.vcap);
        else if (level < h->nbf) fits = vanka_smem_prepare<float, bf16>(B.L, B.vcap);
        else fits = vanka_smem_prepare<float, float>(B.L, B.vcap);
        cudaGetLastError();
        if (!fits) return STOKES_ERR_UNSUPPORTED;
        blocks = 1;
    }
    if (mode == 2 && blocks > 8) {
        DeviceGuard dg(h->dev);
        if (h->prec == STOKES_PREC_FP64) vanka_cluster_prepare<double, double>();
        else {
            vanka_cluster_prepare<float, float>();
            vanka_cluster_prepare<float, bf16>();
        }
        cudaGetLastError();
    }
    LevelBuf &B = h->lev[level];
    B.vmode = mode;
    B.vblocks = (mode == 0 || mode == 4) ? 0 : blocks;
    B.vms = 0.f;
    // the captured graphs hold the old schedule
    drop_graphs(h);
    return STOKES_OK;
}

int stokes_smooth(stokes_t h, int level, int which, double *x, const double *b, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !x || !b || level < 0 || level >= h->nlev() - 1) return STOKES_ERR_INVALID_ARG;
    if (!(which >= 0 && which <= 4) && !(which >= 10 && which <= 17)) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf &B = h->lev[level];
    long long n = B.L.n;
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    const double *xd, *bd;
    bool xdev = is_device_ptr(x);
    if ((rc = stage_in(h, x, n, h->stage_in, &xd, s))) return rc;
    if ((rc = to_level(h, B.L, xd, B.x, s))) return rc;
    if ((rc = stage_in(h, b, n, h->stage_in, &bd, s))) return rc;
    if ((rc = to_level(h, B.L, bd, B.b, s, level < h->nbf))) return rc;
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    auto body = [&](auto t, auto tb) {
        using T = decltype(t);
        using TB = decltype(tb);
        switch (which) {
        case 0: smooth<T, TB>(h, level, s); break;
        case 1: dist_sym<T, TB>(h, level, s); break;
        case 2: vanka_sym<T, TB>(h, level, s); break;
        case 3: dgs_forward<T, TB>(h, level, s); dgs_finish_forward<T>(h, level, s); break;
        case 4: dgs_backward<T, TB>(h, level, s, false); break;
        default: vanka_colour<T, TB>(h, level, which - 10, s); break;
        }
    };
    if (h->prec == STOKES_PREC_FP64) with_tb<double>(h, level, body);
    else with_tb<float>(h, level, body);
    CKLAUNCH();
    double *out = xdev ? x : h->stage_out;
    if ((rc = from_level(h, B.x, out, n, s))) return rc;
    launch_mask<double>(B.L, out, s);
    if (!xdev) CK(cudaMemcpyAsync(x, out, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return STOKES_OK;
}

int stokes_test_grid_barrier(stokes_t h, int level, int missing_blocks, int spin_limit, void *stream) {
    if (!h || level < 0 || level >= h->nlev() - 1 || missing_blocks < 0 || spin_limit < 1 ||
        spin_limit > (int)kBarrierSpinLimit)
        return STOKES_ERR_INVALID_ARG;
    if (h->vanka_max_blocks <= 0) return STOKES_ERR_UNSUPPORTED;  // no cooperative launch on this device
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf &B = h->lev[level];
    const size_t es = h->prec == STOKES_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t esb = level < h->nbf ? sizeof(bf16) : es;
    CK(cudaMemsetAsync(B.x, 0, es * B.L.n, s));
    CK(cudaMemsetAsync(B.b, 0, esb * B.L.n, s));
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    auto body = [&](auto t, auto tb) {
        using T = decltype(t);
        using TB = decltype(tb);
        launch_vanka_sweep<T, TB>(B.L, (T *)B.x, (const TB *)B.b, B.lists, (const T *)B.kinv, (T *)B.corr, B.vcap, 1,
                                  h->bar, h->vanka_max_blocks, s, missing_blocks, (unsigned)spin_limit);
    };
    if (h->prec == STOKES_PREC_FP64) with_tb<double>(h, level, body);
    else with_tb<float>(h, level, body);
    CKLAUNCH();
    GridBarrier hb;
    CK(cudaMemcpyAsync(&hb, h->bar, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // leave the barrier and the level's buffers as every other call expects them
    CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), s));
    CK(cudaMemsetAsync(B.x, 0, es * B.L.n, s));
    CK(cudaStreamSynchronize(s));
    return hb.err ? STOKES_ERR_TIMEOUT : STOKES_OK;
}

int stokes_restrict(stokes_t h, int level, const double *rf, double *bc, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !rf || !bc || level < 0 || level >= h->nlev() - 1) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf &F = h->lev[level], &C = h->lev[level + 1];
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    const double *rd;
    if ((rc = stage_in(h, rf, F.L.n, h->stage_in, &rd, s))) return rc;
    if ((rc = to_level(h, F.L, rd, F.r, s, level < h->nbf))) return rc;
    auto run = [&](auto t, auto tf) {
        using T = decltype(t);
        using TF = decltype(tf);
        auto inner = [&](auto, auto tc) {
            using TC = decltype(tc);
            launch_restrict<T, TF, TC>(F.L, C.L, (const TF *)F.r, (TC *)C.b, s, F.rtile);
        };
        with_tb<T>(h, level + 1, inner);
    };
    if (h->prec == STOKES_PREC_FP64) with_tb<double>(h, level, run);
    else with_tb<float>(h, level, run);
    CKLAUNCH();
    bool dev = is_device_ptr(bc);
    double *out = dev ? bc : h->stage_out;
    if ((rc = from_level(h, C.b, out, C.L.n, s, level + 1 < h->nbf))) return rc;
    if (!dev) CK(cudaMemcpyAsync(bc, out, sizeof(double) * C.L.n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return STOKES_OK;
}

int stokes_prolong_add(stokes_t h, int level, const double *ec, double *xf, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !ec || !xf || level < 0 || level >= h->nlev() - 1) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf &F = h->lev[level], &C = h->lev[level + 1];
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    const double *ed, *xd;
    if ((rc = stage_in(h, ec, C.L.n, h->stage_in, &ed, s))) return rc;
    if ((rc = to_level(h, C.L, ed, C.x, s))) return rc;
    bool xdev = is_device_ptr(xf);
    if ((rc = stage_in(h, xf, F.L.n, h->stage_in, &xd, s))) return rc;
    if ((rc = to_level(h, F.L, xd, F.x, s))) return rc;
    auto run = [&](auto tag) {
        using T = decltype(tag);
        launch_prolong<T>(F.L, C.L, (const T *)C.x, (T *)F.x, s, F.ptile);
    };
    if (h->prec == STOKES_PREC_FP64) run(double());
    else run(float());
    CKLAUNCH();
    // the coarse x buffer must hold zeros off the unknowns for later V-cycles
    CK(cudaMemsetAsync(C.x, 0, (h->prec == STOKES_PREC_FP64 ? 8 : 4) * C.L.n, s));
    double *out = xdev ? xf : h->stage_out;
    if ((rc = from_level(h, F.x, out, F.L.n, s))) return rc;
    launch_mask<double>(F.L, out, s);
    if (!xdev) CK(cudaMemcpyAsync(xf, out, sizeof(double) * F.L.n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return STOKES_OK;
}

int stokes_coarse_solve(stokes_t h, const double *b, double *x, void *stream) {
    if (h && h->nb > 1) return STOKES_ERR_INVALID_ARG;  // batched handles: sqmr_solve_batched only
    if (!h || !b || !x) return STOKES_ERR_INVALID_ARG;
    DeviceGuard dg(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf &C = h->lev[h->nlev() - 1];
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    const double *bd;
    if ((rc = stage_in(h, b, C.L.n, h->stage_in, &bd, s))) return rc;
    if ((rc = to_level(h, C.L, bd, C.b, s))) return rc;
    CK(cudaMemsetAsync(C.x, 0, (h->prec == STOKES_PREC_FP64 ? 8 : 4) * C.L.n, s));
    auto run = [&](auto tag) {
        using T = decltype(tag);
        launch_coarse<T>(C.L, h->cidx, h->nc, h->ckinv, (const T *)C.b, (T *)C.x, s);
    };
    if (h->prec == STOKES_PREC_FP64) run(double());
    else run(float());
    CKLAUNCH();
    bool dev = is_device_ptr(x);
    double *out = dev ? x : h->stage_out;
    if ((rc = from_level(h, C.x, out, C.L.n, s))) return rc;
    if (!dev) CK(cudaMemcpyAsync(x, out, sizeof(double) * C.L.n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return STOKES_OK;
}

}  // extern "C"
