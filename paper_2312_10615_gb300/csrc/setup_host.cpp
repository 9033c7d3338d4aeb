// setup_host.cpp -- host-side set-up arithmetic of the multigrid hierarchy (FP64):
// dense inverse by Gauss-Jordan elimination with partial pivoting (the exact coarsest solve of
// Alg. 1 is stored as an explicit symmetrised inverse) and the pre-factorised Vanka local
// saddle-point problems of Sec. 6 (one per configuration of unknown faces around a cell).
#include <cmath>
#include <cstring>
#include <vector>

#include "setup_host.h"

namespace smg {

// In place: A (n x n, row-major) -> A^{-1}.  Returns 0, or -1 if a pivot is exactly zero.
int dense_inverse(int n, double *A) {
    std::vector<double> W((size_t)n * 2 * n, 0.0);
    const size_t w = (size_t)2 * n;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) {
        std::memcpy(&W[r * w], &A[(size_t)r * n], sizeof(double) * n);
        W[r * w + n + r] = 1.0;
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = std::fabs(W[col * w + col]);
        for (int r = col + 1; r < n; ++r) {
            double v = std::fabs(W[r * w + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return -1;
        if (piv != col)
            for (size_t t = 0; t < w; ++t) std::swap(W[col * w + t], W[piv * w + t]);
        double inv = 1.0 / W[col * w + col];
        for (size_t t = 0; t < w; ++t) W[col * w + t] *= inv;
        const double *prow = &W[col * w];
#pragma omp parallel for schedule(static)
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = W[r * w + col];
            if (f == 0.0) continue;
            double *row = &W[r * w];
            for (size_t t = 0; t < w; ++t) row[t] -= f * prow[t];
        }
    }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) std::memcpy(&A[(size_t)r * n], &W[r * w + n], sizeof(double) * n);
    return 0;
}

// Local matrix C_c L~ C_c^T of one cell for configuration cfg (bit a set = face a is an unknown;
// faces ordered u_low, u_high, v_low, v_high, w_low, w_high, then p_c), inverted and embedded
// into a 7x7 block with zero rows/columns for the faces that are not unknowns.  drops[a] (NULL: all
// 0) = viscous terms that drop out of face a's row next to exterior cells: its diagonal is
// (6 - drops[a]) eta/h^2 (the two faces of one axis are never separated by an exterior cell: the
// cell between them is interior).
int vanka_local_inverse(double h, double eta, double gamma, int cfg, const int *drops, double out[49]) {
    int idx[7], m = 0;
    for (int a = 0; a < 6; ++a)
        if (cfg & (1 << a)) idx[m++] = a;
    idx[m++] = 6;
    double K[49] = {0};
    auto entry = [&](int a, int b) -> double {
        double e2 = eta / (h * h), ih = 1.0 / h;
        if (a == 6 && b == 6) return -gamma;
        if (a == 6 || b == 6) {
            int f = a == 6 ? b : a;
            return (f & 1) ? -ih : ih;  // B_{c,f}: +1/h on the low face, -1/h on the high face
        }
        if (a == b) return (6.0 - (drops ? drops[a] : 0)) * e2;
        if ((a >> 1) == (b >> 1)) return -e2;  // the two faces of one axis are A-neighbours
        return 0.0;
    };
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) K[r * m + c] = entry(idx[r], idx[c]);
    if (dense_inverse(m, K)) return -1;
    std::memset(out, 0, sizeof(double) * 49);
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) out[idx[r] * 7 + idx[c]] = K[r * m + c];
    return 0;
}

}  // namespace smg
