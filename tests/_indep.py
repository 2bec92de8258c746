"""Independent constructions used to pin the oracle (test-side only).

The operator is rebuilt here from its definition as products of sparse difference
matrices, not from the oracle's loops:  A = -(L5 + Lcross) with
  L5     = -(Gx^T Mx Gx)/hx^2 - (Gy^T My Gy)/hy^2   (face differences, face means of eps)
  Lcross = Dx E Dy + Dy E Dx                         (central differences, E = diag(eps_xy))
restricted to the rows of the unknowns.  Bilinear prolongation is built as a sparse
matrix from its weights.
"""
import numpy as np
import scipy.sparse as sp


def node_index(grid):
    return np.arange(grid.nyr * grid.nx).reshape(grid.shape)


def _shift(grid, di, dj):
    """Sparse S with (S u)(i,j) = u(i+di, j+dj); rows whose neighbour is missing are 0."""
    nx, nyr = grid.nx, grid.nyr
    idx = node_index(grid)
    rows, cols = [], []
    for j in range(nyr):
        jj = j + dj
        if grid.periodic_y:
            jj %= nyr
        elif not 0 <= jj < nyr:
            continue
        for i in range(nx):
            ii = i + di
            if 0 <= ii < nx:
                rows.append(idx[j, i])
                cols.append(idx[jj, ii])
    n = nx * nyr
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))


def full_operator(grid, exx, exy, eyy):
    """Sparse A (all nodes x all nodes); only unknown rows are meaningful."""
    hx, hy = grid.hx, grid.hy
    n = grid.nx * grid.nyr
    I = sp.identity(n, format="csr")
    Sxp, Sxm = _shift(grid, 1, 0), _shift(grid, -1, 0)
    Syp, Sym = _shift(grid, 0, 1), _shift(grid, 0, -1)
    ex, ey, e = exx.ravel(), exy.ravel(), eyy.ravel()
    # face means at (i+1/2, j) and (i, j+1/2)
    mx = 0.5 * (ex + Sxp @ ex)
    my = 0.5 * (e + Syp @ e)
    # u -> (u(i+1)-u(i)) Mx, then the backward difference of that flux
    fx = sp.diags(mx) @ (Sxp - I)
    fy = sp.diags(my) @ (Syp - I)
    L5 = (fx - Sxm @ fx) / (hx * hx) + (fy - Sym @ fy) / (hy * hy)
    Dx = (Sxp - Sxm) / (2 * hx)
    Dy = (Syp - Sym) / (2 * hy)
    E = sp.diags(ey)
    Lc = Dx @ E @ Dy + Dy @ E @ Dx
    return -(L5 + Lc).tocsr()


def unknown_ids(grid):
    return node_index(grid)[grid.interior_mask()]


def system(grid, exx, exy, eyy, b_nodes, phi_bc):
    """(A_uu, rhs) of the unknowns with the Dirichlet data moved to the right-hand side."""
    A = full_operator(grid, exx, exy, eyy)
    u = unknown_ids(grid)
    mask = np.ones(grid.nx * grid.nyr, dtype=bool)
    mask[u] = False
    d = np.nonzero(mask)[0]
    Auu = A[u][:, u]
    rhs = b_nodes.ravel()[u] - A[u][:, d] @ phi_bc.ravel()[d]
    return Auu, rhs


def prolongation(grid_f, grid_c):
    """Sparse bilinear P from coarse unknowns to fine unknowns."""
    uf, uc = unknown_ids(grid_f), unknown_ids(grid_c)
    posf = {int(k): p for p, k in enumerate(uf)}
    posc = {int(k): p for p, k in enumerate(uc)}
    idxf, idxc = node_index(grid_f), node_index(grid_c)
    rows, cols, vals = [], [], []
    for J in range(grid_c.nyr):
        for Ic in range(grid_c.nx):
            kc = int(idxc[J, Ic])
            if kc not in posc:
                continue
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    w = (1.0 if di == 0 else 0.5) * (1.0 if dj == 0 else 0.5)
                    fi, fj = 2 * Ic + di, 2 * J + dj
                    if grid_f.periodic_y:
                        fj %= grid_f.nyr
                    if not (0 <= fi < grid_f.nx and 0 <= fj < grid_f.nyr):
                        continue
                    kf = int(idxf[fj, fi])
                    if kf in posf:
                        rows.append(posf[kf])
                        cols.append(posc[kc])
                        vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(uf), len(uc)))


def coupling_matrix(grid, op):
    """Sparse matrix of the unknowns assembled from an oracle Operator's stored couplings."""
    idx = node_index(grid)
    u = unknown_ids(grid)
    pos = {int(k): p for p, k in enumerate(u)}
    rows, cols, vals = [], [], []
    nyr = grid.nyr
    for j in range(nyr):
        for i in range(grid.nx):
            k = int(idx[j, i])
            if k not in pos:
                continue
            jd, ju = (j - 1) % nyr, (j + 1) % nyr
            ent = {(0, 0): op.diag[j, i], (1, 0): op.cE[j, i], (-1, 0): op.cE[j, i - 1],
                   (0, 1): op.cN[j, i], (0, -1): op.cN[jd, i], (1, 1): op.cNE[j, i],
                   (-1, -1): op.cNE[jd, i - 1], (-1, 1): op.cNW[j, i], (1, -1): op.cNW[jd, i + 1]}
            for (di, dj), v in ent.items():
                jj = j + dj
                if grid.periodic_y:
                    jj %= nyr
                elif not 0 <= jj < nyr:
                    continue
                q = int(idx[jj, i + di])
                if q in pos:
                    rows.append(pos[k])
                    cols.append(pos[q])
                    vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(u), len(u)))
