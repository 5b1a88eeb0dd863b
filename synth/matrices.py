"""Seeded sparse symmetric matrices in CSR form, shaped like the paper's workloads.

The paper measures on PARSEC real-space Hamiltonians (Section 4, Table 1):
high-order finite-difference Laplacians plus potentials, n ~ 1e5-3e5. Those
files are not available here, so these generators build synthetic stand-ins of
the same structure (stencil Laplacians plus seeded potentials, and graph
Laplacians for irregular sparsity).

All matrices are returned as :class:`CSR` with int32 row pointers and column
indices and float64 values, both triangles stored, columns sorted within each
row (the layout Section 3.2.1 describes: general CSR, symmetry not exploited).
"""

from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray     # int32[nnz]
    val: np.ndarray     # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        out[rows, self.col] = self.val
        return out


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _stencil_csr(dims, offsets, weights, diag) -> CSR:
    """Assemble a Dirichlet-truncated stencil operator on a box grid.

    ``dims`` are the grid extents (x fastest). ``offsets`` are integer grid
    displacements (tuples), ``weights`` their constant coefficients, and
    ``diag`` the diagonal (scalar or per-point array). Rows are grid points
    in x-fastest order; neighbours outside the box are dropped.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]  # coords[a][p]
    entries = [(tuple(0 for _ in dims), None)] + list(zip(offsets, weights))
    lin = [sum(o[a] * strides[a] for a in range(len(dims))) for o, _ in entries]
    order = np.argsort(lin, kind="stable")
    masks = []
    for o, _ in entries:
        m = np.ones(n, dtype=bool)
        for a, oa in enumerate(o):
            if oa:
                c = coords[a] + oa
                m &= (c >= 0) & (c < dims[a])
        masks.append(m)
    counts = np.zeros(n, dtype=np.int64)
    for m in masks:
        counts += m
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    fill = rowptr[:-1].copy()
    diag_arr = np.broadcast_to(np.asarray(diag, dtype=np.float64), (n,))
    for k in order:
        o, w = entries[k]
        rows = np.nonzero(masks[k])[0]
        pos = fill[rows]
        col[pos] = rows + lin[k]
        val[pos] = diag_arr[rows] if w is None else w
        fill[rows] += 1
    return CSR(n, rowptr.astype(np.int32), col, val)


def laplacian_2d(nx: int, ny: int, potential=None) -> CSR:
    """5-point Dirichlet Laplacian (4 on the diagonal, -1 to each neighbour)."""
    diag = 4.0 if potential is None else 4.0 + np.asarray(potential, dtype=np.float64)
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    return _stencil_csr((nx, ny), offs, [-1.0] * 4, diag)


def laplacian_3d_7pt(nx: int, ny: int, nz: int, potential=None) -> CSR:
    """7-point Dirichlet Laplacian (6 on the diagonal) plus an optional diagonal potential."""
    diag = 6.0 if potential is None else 6.0 + np.asarray(potential, dtype=np.float64)
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return _stencil_csr((nx, ny, nz), offs, [-1.0] * 6, diag)


def fd4_laplacian_3d(N: int, potential=None) -> CSR:
    """Fourth-order 13-point finite-difference -Laplacian on an N^3 grid, h = 1.

    Per axis the second-derivative stencil is (-1, 16, -30, 16, -1)/12, so -d2/dx2
    contributes 30/12 to the diagonal, -16/12 to the +-1 neighbours and 1/12 to
    the +-2 neighbours. Dirichlet truncation at the box faces.
    """
    diag = 7.5 if potential is None else 7.5 + np.asarray(potential, dtype=np.float64)
    offs, ws = [], []
    for a in range(3):
        for d, w in ((-2, 1.0 / 12.0), (-1, -4.0 / 3.0), (1, -4.0 / 3.0), (2, 1.0 / 12.0)):
            o = [0, 0, 0]
            o[a] = d
            offs.append(tuple(o))
            ws.append(w)
    return _stencil_csr((N, N, N), offs, ws, diag)


def gaussian_wells_potential(N: int, count: int = 64, seed: int = 0) -> np.ndarray:
    """Sum of ``count`` negative Gaussians on an N^3 grid (x fastest).

    depth ~ U(1, 5), width ~ U(0.5, 1.5) grid units, centres ~ U(0, N-1) per axis.
    """
    g = _rng(seed)
    depth = 1.0 + 4.0 * g.random(count)
    width = 0.5 + 1.0 * g.random(count)
    centre = (N - 1) * g.random((count, 3))
    ax = np.arange(N, dtype=np.float64)
    V = np.zeros((N, N, N))  # indexed [z, y, x]
    for k in range(count):
        s = 1.0 / (2.0 * width[k] ** 2)
        ex = np.exp(-s * (ax - centre[k, 0]) ** 2)
        ey = np.exp(-s * (ax - centre[k, 1]) ** 2)
        ez = np.exp(-s * (ax - centre[k, 2]) ** 2)
        V -= depth[k] * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return V.reshape(-1)


def diagonal_csr(d) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.copy())


def powerlaw_graph_laplacian(n: int, exponent: float = 2.5, mean_degree: float = 15.0,
                             seed: int = 0, i0: int = 50) -> CSR:
    """Weighted graph Laplacian L = D - W of a Chung-Lu power-law graph plus a ring.

    Expected degrees follow w_i ~ (i + i0)^(-1/(exponent-1)). Edge endpoints are
    drawn proportionally to w; self loops are dropped and duplicates merged. A
    ring i -- i+1 (mod n) keeps the graph connected, so 0 is a simple eigenvalue
    with eigenvector 1/sqrt(n). Edge weights ~ U(0.1, 1).
    """
    g = _rng(seed)
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (exponent - 1.0))
    cw = np.cumsum(w)
    draws = int(round(n * (mean_degree / 2.0 - 1.0)))
    u = g.random((draws, 2)) * cw[-1]
    a = np.minimum(np.searchsorted(cw, u[:, 0], side="right"), n - 1).astype(np.int64)
    b = np.minimum(np.searchsorted(cw, u[:, 1], side="right"), n - 1).astype(np.int64)
    ring_a = np.arange(n, dtype=np.int64)
    ring_b = (ring_a + 1) % n
    a = np.concatenate([a, ring_a])
    b = np.concatenate([b, ring_b])
    keep = a != b
    lo = np.minimum(a[keep], b[keep])
    hi = np.maximum(a[keep], b[keep])
    key = np.unique(lo * n + hi)
    lo = key // n
    hi = key % n
    wt = 0.1 + 0.9 * g.random(key.shape[0])
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    vals = np.concatenate([-wt, -wt])
    deg = np.zeros(n)
    np.add.at(deg, lo, wt)
    np.add.at(deg, hi, wt)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, deg])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


def uneven_batch(count: int = 64, seed: int = 0, n_lo: float = 1e4, n_hi: float = 2e5):
    """Independent 2D/3D Laplacians with U(0,1) diagonal potentials, n log-uniform.

    Returns a list of (CSR, kind, dims). The grid is the integer grid nearest
    the drawn n (square for 2D, cube for 3D); 2D vs 3D by a fair coin.
    """
    g = _rng(seed)
    out = []
    for _ in range(count):
        n_target = float(np.exp(np.log(n_lo) + (np.log(n_hi) - np.log(n_lo)) * g.random()))
        three_d = g.random() < 0.5
        if three_d:
            s = max(2, int(round(n_target ** (1.0 / 3.0))))
            pot = g.random(s ** 3)
            out.append((laplacian_3d_7pt(s, s, s, pot), "3d", (s, s, s)))
        else:
            s = max(2, int(round(n_target ** 0.5)))
            pot = g.random(s * s)
            out.append((laplacian_2d(s, s, pot), "2d", (s, s)))
    return out


def random_normal_block(n: int, r: int, seed: int) -> np.ndarray:
    """n x r row-major block of N(0,1) samples (Box-Muller on PCG64 uniforms)."""
    g = _rng(seed)
    cnt = n * r
    half = (cnt + 1) // 2
    u1 = g.random(half)
    u2 = g.random(half)
    rad = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0,1]
    z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])[:cnt]
    return z.reshape(n, r)


def csr_checksum(A: CSR) -> str:
    h = hashlib.sha256()
    for arr in (A.rowptr, A.col, A.val):
        h.update(np.ascontiguousarray(arr).tobytes())
    return h.hexdigest()[:16]


def fd_second_derivative_weights(half_order: int) -> np.ndarray:
    """Central-difference weights c_0..c_N of f'' of order 2N on a unit grid.

    c_k = 2 (-1)^(k+1) (N!)^2 / (k^2 (N-k)! (N+k)!) for k >= 1 and
    c_0 = -2 sum_k c_k, so f''(x) ~ c_0 f(x) + sum_k c_k (f(x+k) + f(x-k)).
    """
    from math import factorial
    N = int(half_order)
    c = np.zeros(N + 1)
    for k in range(1, N + 1):
        c[k] = 2.0 * (-1) ** (k + 1) * factorial(N) ** 2 / (k * k * factorial(N - k) * factorial(N + k))
    c[0] = -2.0 * c[1:].sum()
    return c


def parsec_like_hamiltonian(radius: float = 30.0, h: float = 0.563, half_order: int = 6, heavy: int = 87,
                            light: int = 76, nl_radius: float = 3.8, seed: int = 0,
                            heavy_depth: float = 0.9, heavy_width: float = 3.0, light_depth: float = 0.55,
                            light_width: float = 2.0, nl_strength: float = 0.6, cluster: float = 0.85) -> CSR:
    """A real-space Hamiltonian stand-in shaped like the PARSEC matrices of Table 1.

    Grid points of a cubic lattice (spacing h) inside a sphere of ``radius``
    grid units; kinetic term -1/2 Laplacian by central differences of order
    2 * half_order (Dirichlet outside the sphere); a local potential that is a
    sum of Gaussian wells at ``heavy`` + ``light`` atom sites (depths and
    widths per species, widths in grid units); and for every heavy atom a
    rank-one non-local term s p p^T, p the Gaussian of width nl_radius / 2
    truncated to the ball of radius nl_radius around the atom (these dense
    blocks carry most of the stored entries, as the paper's non-local term
    does). Atom sites are drawn uniformly in the ball of radius
    ``cluster`` * radius.

    The defaults give the shape of Ge87H76 (Table 1: n = 112,985, nnz/n = 69.9,
    spectrum [-1.21, 32.8]; Table 2: 212 eigenvalues in [-0.645, -0.0053]):
    n = 113,081, nnz = 7,955,253 (70.4 per row), spectrum about [-1.25, 33.1]
    and about 214 eigenvalues in that interval (a Chebyshev-moment estimate).
    """
    g = _rng(seed)
    R = float(radius)
    m = int(np.ceil(R))
    ax = np.arange(-m, m + 1)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    inside = (X * X + Y * Y + Z * Z) <= R * R
    pts = np.stack([Z[inside], Y[inside], X[inside]], axis=1)  # sorted lexicographically (z, y, x)
    order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0]))
    pts = pts[order]
    n = pts.shape[0]
    side = 2 * m + 1
    index = -np.ones(side ** 3, dtype=np.int64)
    key = ((pts[:, 0] + m) * side + (pts[:, 1] + m)) * side + (pts[:, 2] + m)
    index[key] = np.arange(n)
    c = fd_second_derivative_weights(half_order)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.full(n, -0.5 * 3.0 * c[0] / (h * h))]
    for a in range(3):
        for k in range(1, half_order + 1):
            for sgn in (-1, 1):
                q = pts.copy()
                q[:, a] += sgn * k
                ok = np.all(np.abs(q) <= m, axis=1)
                kk = ((q[:, 0] + m) * side + (q[:, 1] + m)) * side + (q[:, 2] + m)
                tgt = np.where(ok, index[np.where(ok, kk, 0)], -1)
                sel = tgt >= 0
                rows.append(np.nonzero(sel)[0])
                cols.append(tgt[sel])
                vals.append(np.full(int(sel.sum()), -0.5 * c[k] / (h * h)))
    # atoms: uniform in the inner ball (rejection sampling on the cube)
    def sites(count):
        out = []
        while len(out) < count:
            u = (2.0 * g.random(3) - 1.0) * cluster * R
            if u @ u <= (cluster * R) ** 2:
                out.append(u)
        return np.array(out).reshape(-1, 3)
    heavy_xyz = sites(heavy)
    light_xyz = sites(light)
    fp = pts.astype(np.float64)
    pot = np.zeros(n)
    for xyz, depth, width in ((heavy_xyz, heavy_depth, heavy_width), (light_xyz, light_depth, light_width)):
        for a in xyz:
            d2 = np.sum((fp - a) ** 2, axis=1)
            pot -= depth * np.exp(-d2 / (2.0 * width * width))
    vals[0] = vals[0] + pot
    for a in heavy_xyz:
        d2 = np.sum((fp - a) ** 2, axis=1)
        ball = np.nonzero(d2 <= nl_radius * nl_radius)[0]
        p = np.exp(-d2[ball] / (2.0 * (0.5 * nl_radius) ** 2))
        p /= np.linalg.norm(p)
        rows.append(np.repeat(ball, ball.shape[0]))
        cols.append(np.tile(ball, ball.shape[0]))
        vals.append(nl_strength * np.outer(p, p).ravel())
    import scipy.sparse as sp
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    A = (A + A.T) * 0.5  # exact symmetry of the assembled sum
    A = A.tocsr()
    A.sort_indices()
    return CSR(n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))
