/*
 * stokes_oracle.c -- plain FP64 CPU oracle of the symmetric multigrid-preconditioned
 * SQMR solver for the 3D MAC Stokes system (Tao & Sifakis, arXiv 2312.10615).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  It shares no code, header,
 * table or helper with the CUDA path and is never called by the product.
 *
 * Everything here is written to be checked against the paper by eye: one degree of
 * freedom (DOF) at a time, one row of the operator at a time, sequential loops, no
 * blocking, fusion or reordering beyond what the paper's algorithms state.  Loops whose
 * iterations are independent (operator rows, prolongation rows, the patch corrections of one
 * Vanka colour, computed from the pre-colour state) may run on several OpenMP threads
 * (og_set_threads); every result is the same, bit for bit, for any thread count.  The DGS
 * sweeps, scatters and every reduction stay sequential.
 *
 *   discretisation ............ Sec. 2, Eq. (2); penalised operator L~ in Sec. 4
 *   cell labels / DOF classes . Sec. 5
 *   distributive Gauss-Seidel . Sec. 3.1, Alg. 2, Eq. (dist), Eq. (ldist), App. A Eq. (SDGS)
 *   multiplicative Vanka ...... Sec. 3.2, Eq. (mv), App. C; 8-colour scheme Sec. 6
 *   combined smoother ......... Sec. 3.3, Alg. 3, App. D
 *   transfers ................. Sec. 2 (P = c R^T, c = 8 in 3D; trilinear velocity, constant pressure)
 *   V-cycle ................... Alg. 1
 *   SQMR ...................... Sec. 4, Alg. 4
 *   pure multigrid solver ..... Alg. 1 iterated on L~ (Sec. 3, Sec. 6 comparisons)
 *
 * Readings of places where the paper is silent or ambiguous:
 *  - scaling: A = (eta/h^2)(7-point stencil), B^T = gradient/h, B = -divergence/h.
 *  - a Dirichlet face neighbour keeps its value (grid-cell precision), the diagonal
 *    stays 6 eta/h^2; inside the preconditioner the Dirichlet values are zero.
 *  - V1 = all active DOFs of interior cells that lie within one cell (26-neighbourhood) of a
 *    Dirichlet cell or within two cells (Chebyshev distance) of an exterior cell.  With exterior
 *    cells absent this is the face-neighbour set on the box; the rule as a whole reproduces the
 *    total and boundary DOF counts of Table 1 for the box and for every cylinder row.
 *  - DGS traversal order: V2 velocities with (i+j+k) even, then odd, then V2 pressures in
 *    8 colours (i mod 2, j mod 2, k mod 2); the backward sweep is the exact reverse.  DGS relaxes the V2 rows and
 *    distributes along the full column M_{.j} (Alg. 2), which for a V2 pressure next to the
 *    V1/V2 interface also updates V1 DOFs; with it L~M stays block lower triangular on
 *    every V2 row (Eq. disc).
 *  - Vanka patch = active DOFs of {p_c, the 6 faces of c}; 8 colours by
 *    (i mod 2, j mod 2, k mod 2); within a colour every patch correction is computed
 *    from the state before the colour and then added; colours 0..7 then 7..0.
 *  - prolongation of a face value: weight 1 (coincident) or 1/2,1/2 along the normal,
 *    3/4,1/4 along each tangential axis; coarse DOFs that are not active contribute 0.
 *  - convergence: true relative residual ||b - L x||_2 / ||b||_2 < tol.
 *  - exterior cells (Sec. 5): the velocity on a face between an interior and an exterior cell is an
 *    unknown (Table 1 counts it) whose equation carries the homogeneous Neumann condition as a
 *    natural (do-nothing) outflow condition: the pressure of an exterior cell is the known value 0,
 *    and a viscous difference term of the velocity stencil drops out (diagonal and neighbour alike)
 *    when it crosses an exterior cell along the face normal, or when the tangential neighbour face
 *    has no interior cell beside it (an inactive face).  Dropped terms are symmetric pairs, so L stays
 *    symmetric; nonzero Neumann data would enter the right-hand side only.  Faces with no interior
 *    cell beside them that are not faces of a Dirichlet cell are inactive.  When some unknown face
 *    borders an exterior cell the pressure has no null space and is not shifted to zero mean.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LAB_INTERIOR 0
#define LAB_DIRICHLET 1
#define LAB_EXTERIOR 2

#define OG_OK 0
#define OG_ERR_ARG -1
#define OG_ERR_OOM -2
#define OG_ERR_BREAKDOWN -4
#define OG_ERR_NOT_CONVERGED -5
#define OG_ERR_UNSUPPORTED -8
#define OG_ERR_SINGULAR -9

typedef struct {
    int nx, ny, nz;
    double h, eta, gamma;
    long nu, nv, nw, np, n; /* packed sizes: [u | v | w | p] */
    long ov, ow, op;        /* offsets of v, w, p */
    uint8_t *lab;           /* (nx+2)(ny+2)(nz+2) cell labels including the ghost shell */
    uint8_t *active;        /* per packed entry */
    uint8_t *v1;            /* per packed entry: active DOF of a cell proximal to a non-interior cell */
    int neumann;            /* some unknown face borders an exterior cell (no pressure null space) */
    long *order;            /* DGS traversal order of the V2 DOFs */
    long norder;
    long gstart[11];        /* order[gstart[g] .. gstart[g+1]) = group g: velocity parities 0, 1, pressure colours 0..7 */
    double *dgs_d;          /* d_j = L~_j . M_{.j} per packed entry (V2 entries only) */
    long *vcell[8];         /* V1 cells (linear cell index) per colour */
    long nvcell[8];
    double *scratch;        /* zero vector, used to evaluate single matrix entries */
    double **tzero;         /* per-thread zero vectors of the threaded Vanka loops (thread >= 1) */
    double *x, *b, *r;      /* per-level work vectors */
    /* coarsest level only: dense LU of L~ on the active DOFs */
    long nc;
    long *cidx;
    double *lu;
    long *piv;
} og_level;

typedef struct {
    int nlev, kb;
    int additive; /* Sec. 3.2 variant: additive Vanka (Eq. av) in place of the symmetric multiplicative sweep */
    int dwj;      /* Sec. 3.1 variant: symmetric distributive weighted Jacobi in place of the symmetric DGS */
    int cycle;    /* coarse-grid visits per level: 1 V-cycle (Alg. 1), 2 W-cycle (Sec. 8.2) */
    og_level *lev;
} og_hier;

/* threads of the order-free loops (1 = sequential) */
static int og_threads = 1;
static inline int nthreads(void) { return og_threads; }

/* ------------------------------------------------------------------------------------ */
/* index helpers                                                                         */

static inline int lab_at(const og_level *L, int i, int j, int k) {
    if (i < -1 || j < -1 || k < -1 || i > L->nx || j > L->ny || k > L->nz) return LAB_DIRICHLET;
    return L->lab[(long)(i + 1) + (long)(L->nx + 2) * ((j + 1) + (long)(L->ny + 2) * (k + 1))];
}

/* does face (c,i,j,k) of component c exist in the packed array? (c = 3: cell) */
static inline int in_array(const og_level *L, int c, int i, int j, int k) {
    int ex = L->nx + (c == 0), ey = L->ny + (c == 1), ez = L->nz + (c == 2);
    return i >= 0 && j >= 0 && k >= 0 && i < ex && j < ey && k < ez;
}

static inline long pidx(const og_level *L, int c, int i, int j, int k) {
    long nx = L->nx, ny = L->ny;
    switch (c) {
    case 0: return i + (nx + 1) * (j + ny * (long)k);
    case 1: return L->ov + i + nx * (j + (ny + 1) * (long)k);
    case 2: return L->ow + i + nx * (j + ny * (long)k);
    default: return L->op + i + nx * (j + ny * (long)k);
    }
}

static void decode(const og_level *L, long q, int *c, int *i, int *j, int *k) {
    long nx = L->nx, ny = L->ny, r;
    if (q < L->ov) { *c = 0; r = q; *i = (int)(r % (nx + 1)); r /= (nx + 1); *j = (int)(r % ny); *k = (int)(r / ny); }
    else if (q < L->ow) { *c = 1; r = q - L->ov; *i = (int)(r % nx); r /= nx; *j = (int)(r % (ny + 1)); *k = (int)(r / (ny + 1)); }
    else if (q < L->op) { *c = 2; r = q - L->ow; *i = (int)(r % nx); r /= nx; *j = (int)(r % ny); *k = (int)(r / ny); }
    else { *c = 3; r = q - L->op; *i = (int)(r % nx); r /= nx; *j = (int)(r % ny); *k = (int)(r / ny); }
}

static inline void unit(int d, int *e) { e[0] = d == 0; e[1] = d == 1; e[2] = d == 2; }

/* Sec. 5: a face of a Dirichlet cell is Dirichlet; otherwise a face with an interior cell beside it
 * is an unknown (between two interior cells, or a Neumann face between an interior and an exterior
 * cell); a face between two exterior cells is inactive. */
static inline int face_dirichlet(const og_level *L, int c, int i, int j, int k) {
    int e[3]; unit(c, e);
    return lab_at(L, i - e[0], j - e[1], k - e[2]) == LAB_DIRICHLET || lab_at(L, i, j, k) == LAB_DIRICHLET;
}
static inline int face_active(const og_level *L, int c, int i, int j, int k) {
    int e[3]; unit(c, e);
    if (face_dirichlet(L, c, i, j, k)) return 0;
    return lab_at(L, i - e[0], j - e[1], k - e[2]) == LAB_INTERIOR || lab_at(L, i, j, k) == LAB_INTERIOR;
}
static inline int face_inactive(const og_level *L, int c, int i, int j, int k) {
    return !face_dirichlet(L, c, i, j, k) && !face_active(L, c, i, j, k);
}

/* does the viscous term between face (c,i,j,k) and its same-component neighbour one cell away along
 * axis d (sgn = +1 or -1) drop out?  Along the normal (d = c) the term crosses the cell between the
 * two faces, and drops when that cell is exterior (the zero-normal-derivative condition of a Neumann
 * face); along a tangential axis it drops when the neighbour face is inactive. */
static inline int nbr_dropped(const og_level *L, int c, int i, int j, int k, int d, int sgn) {
    int e[3]; unit(d, e);
    if (d == c) {
        int a = i - (sgn < 0) * e[0], b = j - (sgn < 0) * e[1], cc = k - (sgn < 0) * e[2];
        return lab_at(L, a, b, cc) == LAB_EXTERIOR;
    }
    return face_inactive(L, c, i + sgn * e[0], j + sgn * e[1], k + sgn * e[2]);
}

/* value of an unknown in x; entries that are not active DOFs count as zero */
static inline double xval(const og_level *L, const double *x, int c, int i, int j, int k) {
    if (!in_array(L, c, i, j, k)) return 0.0;
    long q = pidx(L, c, i, j, k);
    return L->active[q] ? x[q] : 0.0;
}

/* ------------------------------------------------------------------------------------ */
/* Eq. (2): one row of L (gam = 0) or of L~ (gam = gamma, Sec. 4) applied to x.           */
/* velocity row:  eta/h^2 (sum over the 6 same-component neighbours g of (u_f - u_g))        */
/*                + (p_+ - p_-)/h; terms that drop out (nbr_dropped) are left out of the sum,  */
/*                Dirichlet neighbours and exterior pressures count zero                      */
/* pressure row: -(sum over axes of (u_hi - u_lo))/h - gam p_c                            */
static double og_row(const og_level *L, long q, const double *x, double gam) {
    int c, i, j, k, e[3];
    decode(L, q, &c, &i, &j, &k);
    double h = L->h;
    if (c < 3) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            unit(d, e);
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                if (nbr_dropped(L, c, i, j, k, d, sgn)) continue;
                s += x[q] - xval(L, x, c, i + sgn * e[0], j + sgn * e[1], k + sgn * e[2]);
            }
        }
        unit(c, e);
        double pp = xval(L, x, 3, i, j, k);
        double pm = xval(L, x, 3, i - e[0], j - e[1], k - e[2]);
        return L->eta / (h * h) * s + (pp - pm) / h;
    }
    double div = 0.0;
    for (int d = 0; d < 3; ++d) {
        unit(d, e);
        div += xval(L, x, d, i + e[0], j + e[1], k + e[2]) - xval(L, x, d, i, j, k);
    }
    return -div / h - gam * x[q];
}

/* y = L x (gam = 0) or L~ x on the active rows; every other entry of y is 0 */
static void og_apply_level(const og_level *L, const double *x, double *y, double gam) {
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (long q = 0; q < L->n; ++q) y[q] = L->active[q] ? og_row(L, q, x, gam) : 0.0;
}

/* single matrix entry L~_{a,b}, evaluated as row a applied to the unit vector e_b held in a zero
 * vector z (the level's own, or one per thread) */
static double og_entry_z(const og_level *L, double *z, long a, long b, double gam) {
    z[b] = 1.0;
    double v = og_row(L, a, z, gam);
    z[b] = 0.0;
    return v;
}
static double og_entry(og_level *L, long a, long b, double gam) { return og_entry_z(L, L->scratch, a, b, gam); }

/* zero vector of the level for thread t (t = 0: the level's own scratch), allocated on first use */
static double *thread_zero(og_level *L, int t) {
    if (t == 0) return L->scratch;
    if (!L->tzero) L->tzero = (double **)calloc(64, sizeof(double *));
    if (!L->tzero[t]) L->tzero[t] = (double *)calloc(L->n, sizeof(double));
    return L->tzero[t];
}

/* ------------------------------------------------------------------------------------ */
/* dense Gaussian elimination with partial pivoting (textbook), row-major n x n            */
static int og_lu(long n, double *A, long *piv) {
    for (long col = 0; col < n; ++col) {
        long p = col;
        double best = fabs(A[col * n + col]);
        for (long r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > best) { best = fabs(A[r * n + col]); p = r; }
        piv[col] = p;
        if (best == 0.0) return OG_ERR_SINGULAR;
        if (p != col)
            for (long t = 0; t < n; ++t) { double s = A[col * n + t]; A[col * n + t] = A[p * n + t]; A[p * n + t] = s; }
        double inv = 1.0 / A[col * n + col];
        for (long r = col + 1; r < n; ++r) {
            double f = A[r * n + col] * inv;
            A[r * n + col] = f;
            if (f != 0.0)
                for (long t = col + 1; t < n; ++t) A[r * n + t] -= f * A[col * n + t];
        }
    }
    return OG_OK;
}

/* solve with the factors of og_lu: og_lu swaps whole rows (multipliers included), so LU holds the
 * factors of P A with P the product of all its swaps; apply P to y first, then L and U */
static void og_lu_solve(long n, const double *LU, const long *piv, double *y) {
    for (long col = 0; col < n; ++col) {
        long p = piv[col];
        if (p != col) { double s = y[col]; y[col] = y[p]; y[p] = s; }
    }
    for (long col = 0; col < n; ++col)
        for (long r = col + 1; r < n; ++r) y[r] -= LU[r * n + col] * y[col];
    for (long r = n - 1; r >= 0; --r) {
        double s = y[r];
        for (long t = r + 1; t < n; ++t) s -= LU[r * n + t] * y[t];
        y[r] = s / LU[r * n + r];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Sec. 3.1: column j of the distribution matrix M = [[I, -B^T], [0, eta B B^T]] (Alg. 2    */
/* distributes along the whole column; for a V2 pressure it reaches active DOFs of V1      */
/* cells next to the V1/V2 interface, never a Dirichlet face).                             */
static int og_mcol(const og_level *L, long q, long *idx, double *val) {
    int c, i, j, k, e[3];
    decode(L, q, &c, &i, &j, &k);
    if (c < 3) { idx[0] = q; val[0] = 1.0; return 1; }
    double h = L->h;
    /* B^T e_c: faces of cell c; c is the plus cell of its low face (+1/h), the minus cell of its high face (-1/h) */
    long fidx[6]; double fbt[6]; int fc[6], fi[6], fj[6], fk[6]; int nf = 0;
    for (int d = 0; d < 3; ++d) {
        unit(d, e);
        for (int side = 0; side < 2; ++side) {
            int a = i + side * e[0], b = j + side * e[1], cc = k + side * e[2];
            if (!in_array(L, d, a, b, cc) || !face_active(L, d, a, b, cc)) continue;
            fidx[nf] = pidx(L, d, a, b, cc); fbt[nf] = side == 0 ? 1.0 / h : -1.0 / h;
            fc[nf] = d; fi[nf] = a; fj[nf] = b; fk[nf] = cc; ++nf;
        }
    }
    int m = 0;
    for (int t = 0; t < nf; ++t) { idx[m] = fidx[t]; val[m] = -fbt[t]; ++m; }
    /* eta B B^T e_c: for each active face f of c, B_{c',f} (B^T e_c)_f for both cells c' beside f */
    long cidx[7]; double cval[7]; int ncl = 0;
    for (int t = 0; t < nf; ++t) {
        unit(fc[t], e);
        for (int side = 0; side < 2; ++side) { /* side 0: minus cell, side 1: plus cell */
            int a = fi[t] - (side == 0) * e[0], b = fj[t] - (side == 0) * e[1], cc = fk[t] - (side == 0) * e[2];
            double bcf = side == 1 ? 1.0 / h : -1.0 / h; /* B_{c',f} = B^T_{f,c'} */
            long pc = pidx(L, 3, a, b, cc);
            int u = 0;
            while (u < ncl && cidx[u] != pc) ++u;
            if (u == ncl) { cidx[ncl] = pc; cval[ncl] = 0.0; ++ncl; }
            cval[u] += bcf * fbt[t];
        }
    }
    for (int u = 0; u < ncl; ++u)
        if (L->active[cidx[u]]) { idx[m] = cidx[u]; val[m] = L->eta * cval[u]; ++m; }
    return m;
}

/* Alg. 2, forward sweep over the V2 rows: x <- x + (b_j - L~_j x)/d_j M_{.j} in traversal order.
 * The order is a sequence of groups (V2 velocities of one parity of i+j+k, then V2 pressures of one
 * colour); the DOFs of one group are decoupled in L~M, so a DOF's residual does not read what the
 * updates of its own group write.  With several threads the residuals of a group are therefore
 * computed first, in parallel, and the updates then applied in traversal order: the same numbers, in
 * the same order, as the one-DOF-at-a-time loop. */
static void og_dgs_forward(og_level *L, double *x, const double *b) {
    long idx[16]; double val[16];
    if (nthreads() == 1) {
        for (long t = 0; t < L->norder; ++t) {
            long q = L->order[t];
            double r = b[q] - og_row(L, q, x, L->gamma);
            double delta = r / L->dgs_d[q];
            int m = og_mcol(L, q, idx, val);
            for (int u = 0; u < m; ++u) x[idx[u]] += delta * val[u];
        }
        return;
    }
    double *delta = (double *)malloc(sizeof(double) * (L->norder + 1));
    for (int g = 0; g < 10; ++g) {
        long t0 = L->gstart[g], t1 = L->gstart[g + 1];
#pragma omp parallel for schedule(static) num_threads(nthreads())
        for (long t = t0; t < t1; ++t) {
            long q = L->order[t];
            delta[t] = (b[q] - og_row(L, q, x, L->gamma)) / L->dgs_d[q];
        }
        for (long t = t0; t < t1; ++t) {
            int m = og_mcol(L, L->order[t], idx, val);
            for (int u = 0; u < m; ++u) x[idx[u]] += delta[t] * val[u];
        }
    }
    free(delta);
}

/* Eq. (ldist) / Eq. (SDGS), backward sweep: Gauss-Seidel on M^T L~ x = M^T b in exactly the
 * reverse order, x_j <- x_j + M_{.j}^T (b - L~ x) / d_j  (the update x + G~^{-T} M^T (b - L~ x)).
 * Each update changes x_j alone, and within a group no DOF reads another's x_j: a group's updates
 * are independent and may run in parallel. */
static void og_dgs_backward(og_level *L, double *x, const double *b) {
    for (int g = 9; g >= 0; --g) {
        long t0 = L->gstart[g], t1 = L->gstart[g + 1];
#pragma omp parallel for schedule(static) num_threads(nthreads())
        for (long t = t1 - 1; t >= t0; --t) {
            long idx[16]; double val[16];
            long q = L->order[t];
            int m = og_mcol(L, q, idx, val);
            double s = 0.0;
            for (int u = 0; u < m; ++u) s += val[u] * (b[idx[u]] - og_row(L, idx[u], x, L->gamma));
            x[q] += s / L->dgs_d[q];
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Sec. 3.2: Vanka patch of cell c = active DOFs among {6 faces of c, p_c}                */
static int og_patch(const og_level *L, int i, int j, int k, long *dofs) {
    int m = 0, e[3];
    for (int d = 0; d < 3; ++d) {
        unit(d, e);
        for (int side = 0; side < 2; ++side) {
            int a = i + side * e[0], b = j + side * e[1], cc = k + side * e[2];
            if (in_array(L, d, a, b, cc) && face_active(L, d, a, b, cc)) dofs[m++] = pidx(L, d, a, b, cc);
        }
    }
    dofs[m++] = pidx(L, 3, i, j, k);
    return m;
}

/* Sec. 3.2: correction of the patch of V1 cell cl, (C L~ C^T)^{-1} C (b - L~ x), from the state x;
 * the local matrix is built entry by entry (z: a zero vector) and solved by Gaussian elimination.
 * D receives the patch's DOFs; returns their number. */
static int og_patch_correction(const og_level *L, double *z, const double *x, const double *b, long cl, long *D,
                               double *corr) {
    int i = (int)(cl % L->nx), j = (int)((cl / L->nx) % L->ny), k = (int)(cl / ((long)L->nx * L->ny));
    int m = og_patch(L, i, j, k, D);
    double K[49], rl[7];
    long piv[7];
    for (int a = 0; a < m; ++a) {
        rl[a] = b[D[a]] - og_row(L, D[a], x, L->gamma);
        for (int bb = 0; bb < m; ++bb) K[a * m + bb] = og_entry_z(L, z, D[a], D[bb], L->gamma);
    }
    og_lu(m, K, piv);
    og_lu_solve(m, K, piv, rl);
    for (int a = 0; a < m; ++a) corr[a] = rl[a];
    return m;
}

/* patch corrections of cells[0..ncell) from the same state x (independent: threads may share them) */
static void og_patch_corrections(og_level *L, const double *x, const double *b, const long *cells, long ncell,
                                 long *dofs, int *nd, double *corr) {
    int nt = nthreads();
    for (int t = 1; t < nt; ++t) thread_zero(L, t);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (long t = 0; t < ncell; ++t) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        nd[t] = og_patch_correction(L, tid == 0 ? L->scratch : L->tzero[tid], x, b, cells[t], dofs + 7 * t,
                                    corr + 7 * t);
    }
}

/* one colour of the multiplicative Vanka sweep: every patch correction
 * x_D += (C_D L~ C_D^T)^{-1} C_D (b - L~ x) is computed from the state before the colour */
static void og_vanka_colour(og_level *L, double *x, const double *b, int col) {
    long ncell = L->nvcell[col];
    if (ncell == 0) return;
    long *dofs = (long *)malloc(sizeof(long) * 7 * ncell);
    int *nd = (int *)malloc(sizeof(int) * ncell);
    double *corr = (double *)malloc(sizeof(double) * 7 * ncell);
    og_patch_corrections(L, x, b, L->vcell[col], ncell, dofs, nd, corr);
    for (long t = 0; t < ncell; ++t)
        for (int a = 0; a < nd[t]; ++a) x[dofs[7 * t + a]] += corr[7 * t + a];
    free(dofs); free(nd); free(corr);
}

/* Eq. (av): additive Vanka, x += w sum_i C_i^T (C_i L~ C_i^T)^{-1} C_i (b - L~ x) over every V1 patch,
 * every correction computed from the same state, then added (colours 0..7, cells in list order).
 * Reading: Eq. (av) states no damping; a face lies in the patches of its two cells, and the undamped
 * sum over-corrects it (SQMR then stagnates near 3e-2 at 16^3), so w = 1/2, the reciprocal of that
 * overlap, as for additive Schwarz smoothers.  A scalar multiple keeps S_AV symmetric. */
#define OG_ADDITIVE_DAMPING 0.5
static void og_vanka_additive(og_level *L, double *x, const double *b) {
    long ntot = 0;
    for (int col = 0; col < 8; ++col) ntot += L->nvcell[col];
    if (ntot == 0) return;
    long *dofs = (long *)malloc(sizeof(long) * 7 * ntot);
    int *nd = (int *)malloc(sizeof(int) * ntot);
    double *corr = (double *)malloc(sizeof(double) * 7 * ntot);
    long t = 0;
    for (int col = 0; col < 8; ++col) {
        og_patch_corrections(L, x, b, L->vcell[col], L->nvcell[col], dofs + 7 * t, nd + t, corr + 7 * t);
        t += L->nvcell[col];
    }
    for (t = 0; t < ntot; ++t)
        for (int a = 0; a < nd[t]; ++a) x[dofs[7 * t + a]] += OG_ADDITIVE_DAMPING * corr[7 * t + a];
    free(dofs); free(nd); free(corr);
}

/* App. C: symmetric multiplicative Vanka = colours 0..7 followed by 7..0 */
static void og_vanka_sym(og_level *L, double *x, const double *b) {
    for (int col = 0; col < 8; ++col) og_vanka_colour(L, x, b, col);
    for (int col = 7; col >= 0; --col) og_vanka_colour(L, x, b, col);
}

static void og_dgs_sym(og_level *L, double *x, const double *b) {
    og_dgs_forward(L, x, b);
    og_dgs_backward(L, x, b);
}

/* Sec. 3.1, distributive weighted Jacobi (S_DWJ = w M D~^{-1}, D~ the diagonal of L~M) made symmetric
 * like the DGS.  As the DGS applies its smoother block by block (velocities, then pressures, Sec. 3.1),
 * each block here gets one weighted Jacobi step, every update of a step from the same state:
 * right-preconditioned velocities, x_j += w r_j / d_j; right-preconditioned pressures,
 * x += w sum_j M_{.j} r_j / d_j; then in reverse block order the left-preconditioned steps,
 * pressures x_j += w M_{.j}^T r / d_j and velocities x_j += w r_j / d_j (r = b - L~x before each step).
 * Reading: the paper gives no w; w = 6/7, the classical smoothing weight of pointwise Jacobi for the
 * 7-point Laplacian that both diagonal blocks of L~M carry. */
#define OG_DWJ_OMEGA (6.0 / 7.0)
static void og_dwj_step(og_level *L, double *x, const double *b, int pressure, int left) {
    long idx[16]; double val[16];
    double *r = (double *)malloc(sizeof(double) * L->n);
    double *dx = (double *)calloc(L->n, sizeof(double));
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (long q = 0; q < L->n; ++q) r[q] = L->active[q] ? b[q] - og_row(L, q, x, L->gamma) : 0.0;
    for (long t = 0; t < L->norder; ++t) {
        long q = L->order[t];
        if ((q >= L->op) != pressure) continue;
        int m = og_mcol(L, q, idx, val);
        if (left) {
            double s = 0.0;
            for (int u = 0; u < m; ++u) s += val[u] * r[idx[u]];
            dx[q] = s / L->dgs_d[q];
        } else {
            double delta = r[q] / L->dgs_d[q];
            for (int u = 0; u < m; ++u) dx[idx[u]] += delta * val[u];
        }
    }
    for (long q = 0; q < L->n; ++q) x[q] += OG_DWJ_OMEGA * dx[q];
    free(r); free(dx);
}
static void og_dwj_sym(og_level *L, double *x, const double *b) {
    og_dwj_step(L, x, b, 0, 0);
    og_dwj_step(L, x, b, 1, 0);
    og_dwj_step(L, x, b, 1, 1);
    og_dwj_step(L, x, b, 0, 1);
}

/* Alg. 3 (x threaded through the three calls, as in App. D); additive: Eq. (av) in place of the
 * symmetric multiplicative Vanka sweep */
static void og_smooth(og_level *L, double *x, const double *b, int kb, int additive, int dwj) {
    for (int s = 0; s < kb; ++s) (additive ? og_vanka_additive : og_vanka_sym)(L, x, b);
    (dwj ? og_dwj_sym : og_dgs_sym)(L, x, b);
    for (int s = 0; s < kb; ++s) (additive ? og_vanka_additive : og_vanka_sym)(L, x, b);
}

/* ------------------------------------------------------------------------------------ */
/* Sec. 2: prolongation weights of fine DOF q of level F onto the coarse level C.          */
/* pressure: constant per coarse cell.  face velocity: along the normal weight 1 on a      */
/* coincident coarse face, 1/2 + 1/2 between two; along each tangential axis 3/4 to the    */
/* coarse cell containing the fine face and 1/4 to its neighbour on the far side.          */
static int og_pweights(const og_level *F, const og_level *C, long q, long *cq, double *w) {
    int c, i, j, k;
    decode(F, q, &c, &i, &j, &k);
    int fi[3] = {i, j, k};
    if (c == 3) {
        int a = i / 2, b = j / 2, cc = k / 2;
        long t = pidx(C, 3, a, b, cc);
        if (!C->active[t]) return 0;
        cq[0] = t; w[0] = 1.0;
        return 1;
    }
    int ci[3][2]; double cw[3][2]; int cn[3];
    for (int d = 0; d < 3; ++d) {
        if (d == c) {
            if (fi[d] % 2 == 0) { cn[d] = 1; ci[d][0] = fi[d] / 2; cw[d][0] = 1.0; }
            else { cn[d] = 2; ci[d][0] = (fi[d] - 1) / 2; ci[d][1] = (fi[d] + 1) / 2; cw[d][0] = cw[d][1] = 0.5; }
        } else {
            cn[d] = 2;
            ci[d][0] = fi[d] / 2; cw[d][0] = 0.75;
            ci[d][1] = (fi[d] % 2 == 0) ? fi[d] / 2 - 1 : fi[d] / 2 + 1; cw[d][1] = 0.25;
        }
    }
    int m = 0;
    for (int a = 0; a < cn[0]; ++a)
        for (int b = 0; b < cn[1]; ++b)
            for (int g = 0; g < cn[2]; ++g) {
                int I = ci[0][a], J = ci[1][b], K = ci[2][g];
                if (!in_array(C, c, I, J, K)) continue;
                long t = pidx(C, c, I, J, K);
                if (!C->active[t]) continue; /* coarse Dirichlet neighbours carry zero error */
                cq[m] = t; w[m] = cw[0][a] * cw[1][b] * cw[2][g]; ++m;
            }
    return m;
}

/* R = P^T / 8 : bc = R rf (bc overwritten) */
static void og_restrict(const og_level *F, const og_level *C, const double *rf, double *bc) {
    long cq[8]; double w[8];
    memset(bc, 0, sizeof(double) * C->n);
    for (long q = 0; q < F->n; ++q) {
        if (!F->active[q]) continue;
        int m = og_pweights(F, C, q, cq, w);
        for (int u = 0; u < m; ++u) bc[cq[u]] += w[u] / 8.0 * rf[q];
    }
}

/* xf += P ec (rows independent) */
static void og_prolong_add(const og_level *F, const og_level *C, const double *ec, double *xf) {
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (long q = 0; q < F->n; ++q) {
        long cq[8]; double w[8];
        if (!F->active[q]) continue;
        int m = og_pweights(F, C, q, cq, w);
        double s = 0.0;
        for (int u = 0; u < m; ++u) s += w[u] * ec[cq[u]];
        xf[q] += s;
    }
}

/* Alg. 1, "solve exactly" on the coarsest level: dense LU of L~ over the active DOFs */
static void og_coarse_solve(const og_level *L, const double *b, double *x) {
    double *y = (double *)malloc(sizeof(double) * L->nc);
    for (long a = 0; a < L->nc; ++a) y[a] = b[L->cidx[a]];
    og_lu_solve(L->nc, L->lu, L->piv, y);
    memset(x, 0, sizeof(double) * L->n);
    for (long a = 0; a < L->nc; ++a) x[L->cidx[a]] = y[a];
    free(y);
}

/* Alg. 1: V-cycle(L~, b, x0, n) starting at level l (x0 = 0 if zero_init, else the given x); result
 * in x.  H->cycle = 2 visits the coarse problem twice (W-cycle, Sec. 8.2): the second visit starts
 * from the first one's coarse iterate. */
static void og_cycle_level(og_hier *H, int l, const double *b, double *x, int zero_init) {
    og_level *L = &H->lev[l];
    if (l == H->nlev - 1) { og_coarse_solve(L, b, x); return; }
    og_level *C = &H->lev[l + 1];
    if (zero_init) memset(x, 0, sizeof(double) * L->n);
    og_smooth(L, x, b, H->kb, H->additive, H->dwj);
    og_apply_level(L, x, L->r, L->gamma);
    for (long q = 0; q < L->n; ++q) L->r[q] = L->active[q] ? b[q] - L->r[q] : 0.0;
    og_restrict(L, C, L->r, C->b);
    for (int g = 0; g < H->cycle; ++g) og_cycle_level(H, l + 1, C->b, C->x, g == 0);
    og_prolong_add(L, C, C->x, x);
    og_smooth(L, x, b, H->kb, H->additive, H->dwj);
}
static void og_vcycle_level(og_hier *H, int l, const double *b, double *x) { og_cycle_level(H, l, b, x, 1); }

/* ------------------------------------------------------------------------------------ */
/* level construction                                                                    */

static void level_free(og_level *L) {
    free(L->lab); free(L->active); free(L->v1); free(L->order); free(L->dgs_d);
    for (int c = 0; c < 8; ++c) free(L->vcell[c]);
    if (L->tzero) {
        for (int t = 0; t < 64; ++t) free(L->tzero[t]);
        free(L->tzero);
    }
    free(L->scratch); free(L->x); free(L->b); free(L->r);
    free(L->cidx); free(L->lu); free(L->piv);
    memset(L, 0, sizeof(*L));
}

static int level_init(og_level *L, int nx, int ny, int nz, double h, double eta, double gamma,
                      const uint8_t *lab /* (nx+2)(ny+2)(nz+2) or NULL for the box */) {
    memset(L, 0, sizeof(*L));
    L->nx = nx; L->ny = ny; L->nz = nz; L->h = h; L->eta = eta; L->gamma = gamma;
    L->nu = (long)(nx + 1) * ny * nz; L->nv = (long)nx * (ny + 1) * nz; L->nw = (long)nx * ny * (nz + 1);
    L->np = (long)nx * ny * nz;
    L->ov = L->nu; L->ow = L->nu + L->nv; L->op = L->ow + L->nw; L->n = L->op + L->np;
    long nlab = (long)(nx + 2) * (ny + 2) * (nz + 2);
    L->lab = (uint8_t *)malloc(nlab);
    if (!L->lab) return OG_ERR_OOM;
    if (lab) memcpy(L->lab, lab, nlab);
    else
        for (int k = -1; k <= nz; ++k)
            for (int j = -1; j <= ny; ++j)
                for (int i = -1; i <= nx; ++i) {
                    int ghost = i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz;
                    L->lab[(long)(i + 1) + (long)(nx + 2) * ((j + 1) + (long)(ny + 2) * (k + 1))] = ghost ? LAB_DIRICHLET : LAB_INTERIOR;
                }
    /* labels are 0, 1 or 2; the ghost shell is always Dirichlet */
    for (long t = 0; t < nlab; ++t)
        if (L->lab[t] > LAB_EXTERIOR) return OG_ERR_ARG;
    for (int k = -1; k <= nz; ++k)
        for (int j = -1; j <= ny; ++j)
            for (int i = -1; i <= nx; ++i) {
                int ghost = i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz;
                if (ghost && L->lab[(long)(i + 1) + (long)(nx + 2) * ((j + 1) + (long)(ny + 2) * (k + 1))] != LAB_DIRICHLET)
                    return OG_ERR_ARG;
            }
    L->active = (uint8_t *)calloc(L->n, 1);
    L->v1 = (uint8_t *)calloc(L->n, 1);
    L->scratch = (double *)calloc(L->n, sizeof(double));
    L->x = (double *)calloc(L->n, sizeof(double));
    L->b = (double *)calloc(L->n, sizeof(double));
    L->r = (double *)calloc(L->n, sizeof(double));
    L->dgs_d = (double *)calloc(L->n, sizeof(double));
    L->order = (long *)malloc(sizeof(long) * (L->n + 1));
    if (!L->active || !L->v1 || !L->scratch || !L->x || !L->b || !L->r || !L->dgs_d || !L->order) return OG_ERR_OOM;
    /* Sec. 5: active DOFs */
    for (long q = 0; q < L->n; ++q) {
        int c, i, j, k;
        decode(L, q, &c, &i, &j, &k);
        L->active[q] = c < 3 ? (uint8_t)face_active(L, c, i, j, k) : (uint8_t)(lab_at(L, i, j, k) == LAB_INTERIOR);
        if (c < 3 && L->active[q]) {
            int e0[3]; unit(c, e0);
            if (lab_at(L, i, j, k) == LAB_EXTERIOR || lab_at(L, i - e0[0], j - e0[1], k - e0[2]) == LAB_EXTERIOR)
                L->neumann = 1;
        }
    }
    /* Sec. 5: V1 = every active DOF of an interior cell "proximal" to a Dirichlet or an exterior cell:
     * a Dirichlet cell within Chebyshev distance 1 (the 26 neighbours) or an exterior cell within
     * Chebyshev distance 2 */
    int e[3];
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (lab_at(L, i, j, k) != LAB_INTERIOR) continue;
                int prox = 0;
                for (int dk = -2; dk <= 2; ++dk)
                    for (int dj = -2; dj <= 2; ++dj)
                        for (int di = -2; di <= 2; ++di) {
                            int l = lab_at(L, i + di, j + dj, k + dk);
                            int near1 = di >= -1 && di <= 1 && dj >= -1 && dj <= 1 && dk >= -1 && dk <= 1;
                            if ((l == LAB_DIRICHLET && near1) || l == LAB_EXTERIOR) prox = 1;
                        }
                if (!prox) continue;
                long D[7];
                int m = og_patch(L, i, j, k, D);
                for (int a = 0; a < m; ++a) L->v1[D[a]] = 1;
                int col = (i & 1) + 2 * (j & 1) + 4 * (k & 1);
                L->nvcell[col]++;
            }
    for (int c = 0; c < 8; ++c) { L->vcell[c] = (long *)malloc(sizeof(long) * (L->nvcell[c] + 1)); L->nvcell[c] = 0; }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long q = pidx(L, 3, i, j, k);
                if (!L->v1[q]) continue;
                int col = (i & 1) + 2 * (j & 1) + 4 * (k & 1);
                L->vcell[col][L->nvcell[col]++] = q - L->op;
            }
    /* DGS traversal order (Sec. 3.1 leaves it open): the V2 velocities first (block forward
     * substitution on L~M), those with i+j+k even, then odd; then the V2 pressures by colour
     * (i mod 2) + 2 (j mod 2) + 4 (k mod 2), colours 0..7.  Inside a group the order is the
     * packed order; DOFs of one group are decoupled in L~M. */
    L->norder = 0;
    for (int par = 0; par < 2; ++par) {
        L->gstart[par] = L->norder;
        for (long q = 0; q < L->op; ++q) {
            int c, i, j, k;
            decode(L, q, &c, &i, &j, &k);
            if (L->active[q] && !L->v1[q] && ((i + j + k) & 1) == par) L->order[L->norder++] = q;
        }
    }
    for (int col = 0; col < 8; ++col) {
        L->gstart[2 + col] = L->norder;
        for (long q = L->op; q < L->n; ++q) {
            int c, i, j, k;
            decode(L, q, &c, &i, &j, &k);
            if (L->active[q] && !L->v1[q] && (i & 1) + 2 * (j & 1) + 4 * (k & 1) == col) L->order[L->norder++] = q;
        }
    }
    L->gstart[10] = L->norder;
    /* Alg. 2: d_j = L~_{j,} . M_{,j} (row j of L~ applied to column j of M) */
    long idx[16]; double val[16];
    for (long t = 0; t < L->norder; ++t) {
        long q = L->order[t];
        int m = og_mcol(L, q, idx, val);
        for (int u = 0; u < m; ++u) L->scratch[idx[u]] = val[u];
        L->dgs_d[q] = og_row(L, q, L->scratch, L->gamma);
        for (int u = 0; u < m; ++u) L->scratch[idx[u]] = 0.0;
    }
    return OG_OK;
}

static int level_coarse_factor(og_level *L) {
    L->nc = 0;
    for (long q = 0; q < L->n; ++q) L->nc += L->active[q];
    L->cidx = (long *)malloc(sizeof(long) * (L->nc + 1));
    L->piv = (long *)malloc(sizeof(long) * (L->nc + 1));
    L->lu = (double *)malloc(sizeof(double) * L->nc * L->nc);
    if (!L->cidx || !L->piv || !L->lu) return OG_ERR_OOM;
    long a = 0;
    for (long q = 0; q < L->n; ++q) if (L->active[q]) L->cidx[a++] = q;
    for (long r = 0; r < L->nc; ++r)
        for (long c = 0; c < L->nc; ++c) L->lu[r * L->nc + c] = og_entry(L, L->cidx[r], L->cidx[c], L->gamma);
    return og_lu(L->nc, L->lu, L->piv);
}

/* Sec. 5 label coarsening: Dirichlet if any child is Dirichlet, else interior if any child is interior */
static void coarsen_labels(const og_level *F, uint8_t *out) {
    int nx = F->nx / 2, ny = F->ny / 2, nz = F->nz / 2;
    for (int k = -1; k <= nz; ++k)
        for (int j = -1; j <= ny; ++j)
            for (int i = -1; i <= nx; ++i) {
                int lab;
                if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) lab = LAB_DIRICHLET;
                else {
                    int anyd = 0, anyi = 0;
                    for (int c = 0; c < 8; ++c) {
                        int l = lab_at(F, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1));
                        anyd |= l == LAB_DIRICHLET; anyi |= l == LAB_INTERIOR;
                    }
                    lab = anyd ? LAB_DIRICHLET : (anyi ? LAB_INTERIOR : LAB_EXTERIOR);
                }
                out[(long)(i + 1) + (long)(nx + 2) * ((j + 1) + (long)(ny + 2) * (k + 1))] = (uint8_t)lab;
            }
}

/* ------------------------------------------------------------------------------------ */
/* exported API (ctypes)                                                                 */

int og_auto_levels(int nx, int ny, int nz, int coarsest_max) {
    int l = 1;
    while (nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && (nx > coarsest_max || ny > coarsest_max || nz > coarsest_max)) {
        nx /= 2; ny /= 2; nz /= 2; ++l;
    }
    return l;
}

void og_destroy(og_hier *H) {
    if (!H) return;
    for (int l = 0; l < H->nlev; ++l) level_free(&H->lev[l]);
    free(H->lev);
    free(H);
}

/* levels <= 0 selects the automatic depth (halve while every dimension is even and some
 * dimension exceeds coarsest_max).  lab may be NULL (box: one Dirichlet ghost shell). */
int og_create(int nx, int ny, int nz, double h, double eta, double gamma, int levels, int coarsest_max, int kb,
              const uint8_t *lab, og_hier **out) {
    if (nx < 1 || ny < 1 || nz < 1 || h <= 0 || eta <= 0 || gamma < 0 || kb < 0 || !out) return OG_ERR_ARG;
    if (levels <= 0) levels = og_auto_levels(nx, ny, nz, coarsest_max > 0 ? coarsest_max : 8);
    og_hier *H = (og_hier *)calloc(1, sizeof(og_hier));
    if (!H) return OG_ERR_OOM;
    H->kb = kb;
    H->additive = 0;
    H->cycle = 1;
    H->dwj = 0;
    H->lev = (og_level *)calloc(levels, sizeof(og_level));
    int rc = OG_OK;
    uint8_t *clab = NULL;
    for (int l = 0; l < levels; ++l) {
        if (l > 0) {
            og_level *F = &H->lev[l - 1];
            if (F->nx % 2 || F->ny % 2 || F->nz % 2) { rc = OG_ERR_ARG; break; }
            clab = (uint8_t *)malloc((long)(F->nx / 2 + 2) * (F->ny / 2 + 2) * (F->nz / 2 + 2));
            coarsen_labels(F, clab);
            rc = level_init(&H->lev[l], F->nx / 2, F->ny / 2, F->nz / 2, 2 * F->h, eta, gamma, clab);
            free(clab);
        } else {
            rc = level_init(&H->lev[0], nx, ny, nz, h, eta, gamma, lab);
        }
        H->nlev = l + 1;
        if (rc) break;
    }
    if (!rc) rc = level_coarse_factor(&H->lev[H->nlev - 1]);
    if (rc) { og_destroy(H); return rc; }
    *out = H;
    return OG_OK;
}

int og_nlevels(const og_hier *H) { return H->nlev; }
/* threads of the order-free loops (1..64; the result does not depend on it); returns the count set */
int og_set_threads(int n) {
    if (n < 1) n = 1;
    if (n > 64) n = 64;
#ifndef _OPENMP
    n = 1;
#endif
    og_threads = n;
    return n;
}
int og_has_neumann(const og_hier *H) { return H->lev[0].neumann; }
long og_level_n(const og_hier *H, int l) { return H->lev[l].n; }
void og_level_dims(const og_hier *H, int l, int *dims) { dims[0] = H->lev[l].nx; dims[1] = H->lev[l].ny; dims[2] = H->lev[l].nz; }
void og_level_masks(const og_hier *H, int l, uint8_t *active, uint8_t *v1) {
    memcpy(active, H->lev[l].active, H->lev[l].n);
    memcpy(v1, H->lev[l].v1, H->lev[l].n);
}
void og_level_order(const og_hier *H, int l, long *order, long *norder) {
    memcpy(order, H->lev[l].order, sizeof(long) * H->lev[l].norder);
    *norder = H->lev[l].norder;
}

/* DOF counts of Table 1 without building a hierarchy: active DOFs and V1 DOFs */
int og_count_dofs(int nx, int ny, int nz, const uint8_t *lab, long *n_active, long *n_v1) {
    og_level L;
    int rc = level_init(&L, nx, ny, nz, 1.0, 1.0, 0.0, lab);
    if (!rc) {
        long a = 0, v = 0;
        for (long q = 0; q < L.n; ++q) { a += L.active[q]; v += L.v1[q]; }
        *n_active = a; *n_v1 = v;
    }
    level_free(&L);
    return rc;
}

/* y = L x (penalised = 0) or L~ x (penalised = 1) on level l */
void og_apply(og_hier *H, int l, int penalised, const double *x, double *y) {
    og_level *L = &H->lev[l];
    og_apply_level(L, x, y, penalised ? L->gamma : 0.0);
}

/* Sec. 5: b = f on the active rows with the Dirichlet values g moved to the right-hand side.
 * f: packed layout (only active entries read).  g: ghost-extended face arrays
 * [u (nx+1)(ny+2)(nz+2) | v (nx+2)(ny+1)(nz+2) | w (nx+2)(ny+2)(nz+1)], index -1..n per tangential axis. */
static double gval(const og_level *L, const double *g, int c, int i, int j, int k) {
    long nx = L->nx, ny = L->ny, nz = L->nz;
    long gu = (nx + 1) * (ny + 2) * (nz + 2), gv = (nx + 2) * (ny + 1) * (nz + 2);
    if (c == 0) return g[i + (nx + 1) * ((j + 1) + (ny + 2) * (long)(k + 1))];
    if (c == 1) return g[gu + (i + 1) + (nx + 2) * (j + (ny + 1) * (long)(k + 1))];
    return g[gu + gv + (i + 1) + (nx + 2) * ((j + 1) + (ny + 2) * (long)k)];
}

void og_rhs(og_hier *H, const double *f, const double *g, double *b) {
    og_level *L = &H->lev[0];
    double h = L->h;
    int e[3];
    for (long q = 0; q < L->n; ++q) {
        if (!L->active[q]) { b[q] = 0.0; continue; }
        int c, i, j, k;
        decode(L, q, &c, &i, &j, &k);
        double v = f ? f[q] : 0.0;
        if (c < 3) {
            for (int d = 0; d < 3; ++d) {
                unit(d, e);
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    int a = i + sgn * e[0], bb = j + sgn * e[1], cc = k + sgn * e[2];
                    if (nbr_dropped(L, c, i, j, k, d, sgn)) continue;
                    if (face_dirichlet(L, c, a, bb, cc) && g) v += L->eta / (h * h) * gval(L, g, c, a, bb, cc);
                }
            }
        } else {
            for (int d = 0; d < 3; ++d) {
                unit(d, e);
                if (g && face_dirichlet(L, d, i + e[0], j + e[1], k + e[2])) v += gval(L, g, d, i + e[0], j + e[1], k + e[2]) / h;
                if (g && face_dirichlet(L, d, i, j, k)) v -= gval(L, g, d, i, j, k) / h;
            }
        }
        b[q] = v;
    }
}

void og_dgs(og_hier *H, int l, int direction /* +1 forward, -1 backward, 0 symmetric */, double *x, const double *b) {
    og_level *L = &H->lev[l];
    if (direction == 0 && H->dwj) { og_dwj_sym(L, x, b); return; }
    if (direction >= 0) og_dgs_forward(L, x, b);
    if (direction <= 0) og_dgs_backward(L, x, b);
}
void og_vanka(og_hier *H, int l, int colour /* 0..7 one colour, -1 symmetric sweep (additive step if set) */,
              double *x, const double *b) {
    og_level *L = &H->lev[l];
    if (colour >= 0) og_vanka_colour(L, x, b, colour);
    else if (H->additive) og_vanka_additive(L, x, b);
    else og_vanka_sym(L, x, b);
}
void og_smooth_level(og_hier *H, int l, double *x, const double *b) {
    og_smooth(&H->lev[l], x, b, H->kb, H->additive, H->dwj);
}
/* smoother and cycle variants (Sec. 3.2 additive Vanka; Sec. 8.2 W-cycle) */
int og_set_variant(og_hier *H, int additive, int cycle, int dwj) {
    if (!H || (additive != 0 && additive != 1) || cycle < 1 || cycle > 2 || (dwj != 0 && dwj != 1)) return OG_ERR_ARG;
    H->additive = additive;
    H->cycle = cycle;
    H->dwj = dwj;
    return OG_OK;
}
void og_restrict_level(og_hier *H, int l, const double *rf, double *bc) { og_restrict(&H->lev[l], &H->lev[l + 1], rf, bc); }
void og_prolong_level(og_hier *H, int l, const double *ec, double *xf) { og_prolong_add(&H->lev[l], &H->lev[l + 1], ec, xf); }
void og_coarse(og_hier *H, const double *b, double *x) { og_coarse_solve(&H->lev[H->nlev - 1], b, x); }
void og_dgs_diag(const og_hier *H, int l, double *d) { memcpy(d, H->lev[l].dgs_d, sizeof(double) * H->lev[l].n); }

/* t = V-cycle(L~, s, 0, n) on the finest level (Sec. 3: W^dagger s) */
void og_vcycle(og_hier *H, const double *s, double *t) { og_vcycle_level(H, 0, s, t); }

static double dot(long n, const double *a, const double *b) {
    double s = 0.0;
    for (long q = 0; q < n; ++q) s += a[q] * b[q];
    return s;
}

/* one V-cycle of Alg. 1 on L~ with a given initial guess: x holds x0 on entry, the cycle's result on exit */
void og_vcycle_x0(og_hier *H, const double *b, double *x) {
    og_level *L = &H->lev[0];
    for (long a = 0; a < L->n; ++a) if (!L->active[a]) x[a] = 0.0;
    og_cycle_level(H, 0, b, x, 0);
}

/* Alg. 1 used outright as the solver (Sec. 3: iterating the cycle instead of preconditioning with it),
 * on the penalised system L~ x = b, as in the paper's pure-multigrid comparisons (Sec. 6):
 * x_{k+1} = V-cycle(L~, b, x_k, n) until ||b - L~ x_k||_2 / ||b||_2 < tol.
 * x holds x0 on entry.  hist (optional, maxit+1 entries): that relative residual for k = 0, 1, ... */
int og_mg_solve(og_hier *H, const double *b, double *x, double tol, int maxit, int *iters, double *relres,
                double *hist) {
    og_level *L = &H->lev[0];
    long n = L->n;
    double *r = (double *)calloc(n, sizeof(double));
    if (!r) return OG_ERR_OOM;
    int rc = OG_ERR_NOT_CONVERGED, k = 0;
    double nb = sqrt(dot(n, b, b)), rel = 0.0;
    for (long a = 0; a < n; ++a) if (!L->active[a]) x[a] = 0.0;
    for (k = 0;; ++k) {
        og_apply_level(L, x, r, L->gamma);
        for (long a = 0; a < n; ++a) r[a] = L->active[a] ? b[a] - r[a] : 0.0;
        rel = nb > 0 ? sqrt(dot(n, r, r)) / nb : 0.0;
        if (hist) hist[k] = rel;
        if (rel < tol || nb == 0.0) { rc = OG_OK; break; }
        if (k == maxit) break;
        og_cycle_level(H, 0, b, x, 0);
    }
    if (iters) *iters = k;
    if (relres) *relres = rel;
    free(r);
    return rc;
}

/* Alg. 4: MG-preconditioned SQMR on L (precond = 1) or plain SQMR (precond = 0).
 * x holds x0 on entry and the solution on exit (pressure mean removed).
 * hist (optional, maxit+1 entries): true relative residual after each iteration.
 * If fixed_iters > 0 the loop runs exactly that many iterations (no convergence test). */
int og_sqmr(og_hier *H, const double *b, double *x, double tol, int maxit, int precond, int fixed_iters,
            int *iters, double *relres, double *hist) {
    og_level *L = &H->lev[0];
    long n = L->n;
    double *s = (double *)calloc(n, sizeof(double)), *t = (double *)calloc(n, sizeof(double));
    double *q = (double *)calloc(n, sizeof(double)), *d = (double *)calloc(n, sizeof(double));
    double *w = (double *)calloc(n, sizeof(double));
    int rc = OG_ERR_NOT_CONVERGED, j = 0;
    double nb = sqrt(dot(n, b, b)), rr = 0.0;
    for (long a = 0; a < n; ++a) if (!L->active[a]) x[a] = 0.0;
    og_apply_level(L, x, w, 0.0);
    for (long a = 0; a < n; ++a) s[a] = L->active[a] ? b[a] - w[a] : 0.0;
    rr = nb > 0 ? sqrt(dot(n, s, s)) / nb : 0.0;
    if (hist) hist[0] = rr;
    if (nb == 0.0) { memset(x, 0, sizeof(double) * n); rc = OG_OK; goto done; }
    if (precond) og_vcycle(H, s, t); else memcpy(t, s, sizeof(double) * n);
    memcpy(q, t, sizeof(double) * n);
    double tau = sqrt(dot(n, t, t)), nu_prev = 0.0, rho = dot(n, s, q);
    for (j = 1; j <= maxit; ++j) {
        og_apply_level(L, q, t, 0.0);
        double sigma = dot(n, q, t);
        if (sigma == 0.0) { rc = OG_ERR_BREAKDOWN; --j; break; }
        double alpha = rho / sigma;
        for (long a = 0; a < n; ++a) s[a] -= alpha * t[a];
        if (precond) og_vcycle(H, s, t); else memcpy(t, s, sizeof(double) * n);
        double nu = sqrt(dot(n, t, t)) / tau;
        double c = 1.0 / sqrt(1.0 + nu * nu);
        tau = tau * nu * c;
        for (long a = 0; a < n; ++a) { d[a] = c * c * nu_prev * nu_prev * d[a] + c * c * alpha * q[a]; x[a] += d[a]; }
        nu_prev = nu;
        og_apply_level(L, x, w, 0.0);
        for (long a = 0; a < n; ++a) w[a] = L->active[a] ? b[a] - w[a] : 0.0;
        rr = sqrt(dot(n, w, w)) / nb;
        if (hist) hist[j] = rr;
        if (fixed_iters > 0 ? j >= fixed_iters : rr < tol) { rc = OG_OK; break; }
        if (rho == 0.0) { rc = OG_ERR_BREAKDOWN; break; }
        double rho_new = dot(n, s, t);
        double beta = rho_new / rho;
        for (long a = 0; a < n; ++a) q[a] = t[a] + beta * q[a];
        rho = rho_new;
    }
    if (j > maxit) j = maxit;
done:
    /* pressure fixed to zero mean (only where constant pressures form a null space: no Neumann face) */
    if (!L->neumann) {
        double sum = 0.0; long cnt = 0;
        for (long a = L->op; a < n; ++a) if (L->active[a]) { sum += x[a]; ++cnt; }
        if (cnt) for (long a = L->op; a < n; ++a) if (L->active[a]) x[a] -= sum / cnt;
    }
    if (iters) *iters = j;
    if (relres) *relres = rr;
    free(s); free(t); free(q); free(d); free(w);
    return rc;
}
