"""Independent dense construction of the paper's matrices for small box grids (test helper).

Built from Kronecker products of 1D difference matrices -- a different construction from the
oracle's per-row stencil loops -- so that agreement pins the oracle's operator, distribution
matrix and DOF classes.  Everything is in the packed numbering [u | v | w | p] (x fastest);
rows/columns of entries that are not active unknowns are zero.

Eq. 2:  L = [[A, B^T], [B, 0]],  A = -eta Lap_h,  B^T = grad_h,  B = -div_h
Sec. 4: L~ = [[A, B^T], [B, -gamma I]]
Eq. dist: M = [[I, -B^T], [0, eta B B^T]]
"""
import numpy as np
import scipy.sparse as sp


def _shift(m):
    return sp.diags([np.ones(m - 1), np.ones(m - 1)], [-1, 1], shape=(m, m))


def _grad1d(m):
    """(m+1) x m: face i gets cell i minus cell i-1 (cells outside the range absent)."""
    G = sp.lil_matrix((m + 1, m))
    for i in range(m + 1):
        if i < m:
            G[i, i] = 1.0
        if i >= 1:
            G[i, i - 1] = -1.0
    return G.tocsr()


def _kron3(z, y, x):
    return sp.kron(z, sp.kron(y, x))


class DenseBox:
    def __init__(self, nx, ny=None, nz=None, h=None, eta=1.0, gamma=1e-3):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        h = 1.0 / nx if h is None else h
        self.nx, self.ny, self.nz, self.h, self.eta, self.gamma = nx, ny, nz, h, eta, gamma
        dims = [(nx + 1, ny, nz), (nx, ny + 1, nz), (nx, ny, nz + 1)]
        I = sp.identity
        lap, grad = [], []
        for c in range(3):
            mx, my, mz = dims[c]
            S = _kron3(I(mz), I(my), _shift(mx)) + _kron3(I(mz), _shift(my), I(mx)) + _kron3(_shift(mz), I(my), I(mx))
            lap.append(6.0 * sp.identity(mx * my * mz) - S)
            G = [_kron3(I(nz), I(ny), _grad1d(nx)), _kron3(I(nz), _grad1d(ny), I(nx)),
                 _kron3(_grad1d(nz), I(ny), I(nx))][c]
            grad.append(G)
        sizes = [a * b * c for (a, b, c) in dims] + [nx * ny * nz]
        self.sizes = sizes
        self.n = sum(sizes)
        self.offsets = np.cumsum([0] + sizes)
        # active: faces whose normal index lies strictly inside (both cells interior); all pressures
        act = []
        for c in range(3):
            mx, my, mz = dims[c]
            k, j, i = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
            idx = [i, j, k][c]
            nmax = [nx, ny, nz][c]
            act.append(((idx >= 1) & (idx <= nmax - 1)).reshape(-1))
        act.append(np.ones(nx * ny * nz, bool))
        self.active = np.concatenate(act)
        A = sp.block_diag(lap) * (eta / h ** 2)
        BT = sp.vstack(grad) / h
        Dm = sp.diags(self.active.astype(float))
        nf = sum(sizes[:3])
        Df = sp.diags(self.active[:nf].astype(float))
        A = Df @ A @ Df
        BT = Df @ BT
        self.A, self.BT = A.tocsr(), BT.tocsr()
        self.L = sp.bmat([[A, BT], [BT.T, None]], format="csr")
        self.Lt = sp.bmat([[A, BT], [BT.T, -gamma * sp.identity(nx * ny * nz)]], format="csr")
        self.M = sp.bmat([[sp.identity(nf), -BT], [None, eta * (BT.T @ BT)]], format="csr")
        self.L = (Dm @ self.L @ Dm).tocsr()
        self.Lt = (Dm @ self.Lt @ Dm).tocsr()
        self.M = (Dm @ self.M @ Dm).tocsr()
        # V1: active DOFs of the cells in the outer layer of the box (face-adjacent to the ghost shell)
        v1 = np.zeros(self.n, bool)
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        outer = ((ii == 0) | (ii == nx - 1) | (jj == 0) | (jj == ny - 1) | (kk == 0) | (kk == nz - 1)).reshape(-1)
        v1[self.offsets[3]:] = outer
        for c in range(3):
            mx, my, mz = dims[c]
            k, j, i = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
            idx = [i, j, k]
            # the two cells beside the face: index along c minus 1 and the index itself
            lo = [a.copy() for a in idx]
            lo[c] = lo[c] - 1
            hi = [a.copy() for a in idx]
            n3 = (nx, ny, nz)

            def outer_cell(t):
                inside = np.all([(t[d] >= 0) & (t[d] < n3[d]) for d in range(3)], axis=0)
                edge = np.any([(t[d] == 0) | (t[d] == n3[d] - 1) for d in range(3)], axis=0)
                return inside & edge

            f = (outer_cell(lo) | outer_cell(hi)).reshape(-1)
            v1[self.offsets[c]:self.offsets[c + 1]] = f
        self.v1 = v1 & self.active
        self.v2 = self.active & ~self.v1
        # parity of the own (i+j+k) index of every packed entry
        par = []
        for c in range(4):
            mx, my, mz = (dims[c] if c < 3 else (nx, ny, nz))
            k, j, i = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
            par.append(((i + j + k) % 2).reshape(-1))
        self.parity = np.concatenate(par)
        self.is_p = np.zeros(self.n, bool)
        self.is_p[self.offsets[3]:] = True

    def dgs_order(self):
        # velocities by parity of i+j+k, then pressures by colour (i%2)+2(j%2)+4(k%2)
        out = []
        for par in (0, 1):
            out.append(np.nonzero(self.v2 & ~self.is_p & (self.parity == par))[0])
        nx, ny, nz = self.nx, self.ny, self.nz
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        col = ((i % 2) + 2 * (j % 2) + 4 * (k % 2)).reshape(-1)
        for c in range(8):
            sel = np.nonzero(col == c)[0] + self.offsets[3]
            out.append(sel[self.v2[sel]])
        return np.concatenate(out)
