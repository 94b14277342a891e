"""In-mask voxel graph for the UGL spatial prior (Section 2, after Eq. 5; Section 3.1, Eq. 6-7)
and its weighted form, the WGL prior of the Discussion.

D_w has, for every in-mask voxel, its number of in-mask face neighbours on the diagonal
and -1 for every adjacent in-mask pair. G_w has one row per adjacent pair (i, j) with +1 in
column i and -1 in column j, so that D_w = G_w' G_w (Eq. 6-7).

Weighted graph Laplacian (Discussion: D_w = G_w' C G_w for a diagonal edge-weight matrix C
chosen from the distances between neighbouring voxels; in Algorithm 2 row e of G_w is
multiplied by sqrt(C_ee)). Here C_ee = weights[d] for an edge along direction d (x, y, z), the
form that anisotropic voxel sizes call for; weights = (1, 1, 1) is the UGL prior. D() then has
the weighted degree sum_d c_d on the diagonal and -c_d per adjacent pair.

Conventions (shared with the CUDA library by specification only, not by code):
* the mask is an (nz, ny, nx) array, x fastest; in-mask voxels are numbered in raster order;
* neighbourhood 6 links +-x, +-y, +-z; neighbourhood 4 links +-x, +-y only (slice-wise 2D);
* an edge is oriented from its lower lattice-linear endpoint i to j = i + stride(d),
  d in {0:+x, 1:+y, 2:+z}; edges are ordered by (lattice-linear index of i, d).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Lattice:
    def __init__(self, mask: np.ndarray, neighbourhood: int, weights=(1.0, 1.0, 1.0),
                 edge_factors=None):
        """edge_factors: optional per-edge factors of C, shape (3, nz, ny, nx) (or (3, sites)):
        entry [d, site] multiplies the weight of the edge from that site along +d, so that
        C_ee = weights[d] * edge_factors[d, lattice-linear(i)] for the edge (i, i + stride(d)),
        a general diagonal C; None is all ones."""
        self.weights = np.asarray(weights, dtype=np.float64)
        if self.weights.shape != (3,) or not np.all(self.weights > 0):
            raise ValueError("weights: three positive edge weights (x, y, z)")
        self.edge_factors = None
        if edge_factors is not None:
            f = np.asarray(edge_factors, dtype=np.float64).reshape(3, -1)
            if not np.all(f > 0):
                raise ValueError("edge_factors must be positive")
            self.edge_factors = f
        mask = np.asarray(mask)
        if mask.ndim == 2:
            mask = mask[None]
        self.mask = (mask != 0)
        self.nz, self.ny, self.nx = self.mask.shape
        if neighbourhood not in (4, 6):
            raise ValueError("neighbourhood must be 4 or 6")
        self.neighbourhood = neighbourhood
        flat = self.mask.reshape(-1)
        self.lin = np.flatnonzero(flat).astype(np.int64)       # compact -> lattice-linear
        self.N = len(self.lin)
        self.index_of = np.full(flat.size, -1, dtype=np.int64)  # lattice-linear -> compact
        self.index_of[self.lin] = np.arange(self.N)

    @property
    def dims(self):
        return (self.nx, self.ny, self.nz)

    def coords(self):
        """(x, y, z) lattice coordinates of each in-mask voxel."""
        l = self.lin
        x = l % self.nx
        y = (l // self.nx) % self.ny
        z = l // (self.nx * self.ny)
        return x, y, z

    def n_dirs(self):
        return 3 if self.neighbourhood == 6 else 2

    def forward_neighbour(self, d):
        """Compact index of the +d neighbour of each voxel (-1 if outside lattice or mask)."""
        x, y, z = self.coords()
        if d == 0:
            ok, step = x + 1 < self.nx, 1
        elif d == 1:
            ok, step = y + 1 < self.ny, self.nx
        else:
            ok, step = z + 1 < self.nz, self.nx * self.ny
        out = np.full(self.N, -1, dtype=np.int64)
        out[ok] = self.index_of[self.lin[ok] + step]
        return out

    def edges(self):
        """Edge list (i, j, d), ordered by (lattice-linear index of i, d)."""
        rows = []
        for d in range(self.n_dirs()):
            j = self.forward_neighbour(d)
            i = np.flatnonzero(j >= 0)
            rows.append(np.stack([i, j[i], np.full(len(i), d)], axis=1))
        e = np.concatenate(rows, axis=0) if rows else np.zeros((0, 3), np.int64)
        order = np.lexsort((e[:, 2], self.lin[e[:, 0]]))
        return e[order]

    def edge_weights(self):
        """C_ee for the edges in edges() order."""
        e = self.edges()
        c = self.weights[e[:, 2]]
        if self.edge_factors is not None:
            c = c * self.edge_factors[e[:, 2], self.lin[e[:, 0]]]
        return c

    def Gw(self):
        """C^(1/2) G_w: row e of G_w times sqrt(C_ee) (the form Algorithm 2 uses)."""
        return (sp.diags(np.sqrt(self.edge_weights())) @ self.G()).tocsr()

    def G(self):
        """G_w (Eq. 7): one row per edge, +1 at the lower endpoint i, -1 at j."""
        e = self.edges()
        m = len(e)
        r = np.concatenate([np.arange(m), np.arange(m)])
        c = np.concatenate([e[:, 0], e[:, 1]])
        v = np.concatenate([np.ones(m), -np.ones(m)])
        return sp.csr_matrix((v, (r, c)), shape=(m, self.N))

    def D(self):
        """D_w, the graph Laplacian (Section 2; weighted as in the Discussion), built from
        adjacency lookups: weighted degree on the diagonal, -c_d per adjacent in-mask pair along
        direction d. Built independently of G()."""
        x, y, z = self.coords()
        offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
        if self.neighbourhood == 6:
            offs += [(0, 0, 1), (0, 0, -1)]
        rows, cols, vals = [], [], []
        for idx, (dx, dy, dz) in enumerate(offs):
            xx, yy, zz = x + dx, y + dy, z + dz
            ok = (xx >= 0) & (xx < self.nx) & (yy >= 0) & (yy < self.ny) & (zz >= 0) & (zz < self.nz)
            lin = zz * self.nx * self.ny + yy * self.nx + xx
            nb = np.full(self.N, -1)
            nb[ok] = self.index_of[lin[ok]]
            keep = nb >= 0
            rows.append(np.flatnonzero(keep))
            cols.append(nb[keep])
            c = np.full(int(keep.sum()), self.weights[idx // 2])
            if self.edge_factors is not None:
                # the +d edge of voxel i is stored at i, the -d edge at the neighbour
                low = self.lin[keep] if idx % 2 == 0 else self.lin[nb[keep]]
                c = c * self.edge_factors[idx // 2, low]
            vals.append(c)
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        adj = sp.csr_matrix((np.concatenate(vals), (rows, cols)), shape=(self.N, self.N))
        deg = np.asarray(adj.sum(axis=1)).ravel()
        return (sp.diags(deg) - adj).tocsr()

    def degree(self):
        return np.asarray(np.diag(self.D().toarray())) if self.N <= 4000 else self.D().diagonal()
