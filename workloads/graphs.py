"""Seeded synthetic matrices shaped like the paper's workloads.

The paper (Sec. 5.1) measures on graph Laplacians of a collaboration network
with many connected components, and on sparse cohomology matrices from a public
collection.  Neither dataset is available here; the generators below build
matrices with the same structure (disjoint-component Laplacians, +-1 incidence
matrices, rectangular sparse matrices with an exactly known null space), at the
sizes of the five benchmark configurations.

Every generator is a pure function of its integer seed (numpy's PCG64), so the
same matrix is produced on any host.  Node labels are shuffled by one global
random permutation, so components are not contiguous index ranges.

Readings of underspecified points (recorded in the design notes as well):
* Erdos-Renyi components are rejection-sampled until connected.
* "random graph of mean degree k" components are the union of k/2 independent
  random Hamiltonian cycles on the component's nodes (connected, expander-like),
  duplicate edges merged at unit weight for Laplacians and kept as parallel rows
  for incidence matrices.
* Power-law / uniform component sizes are affinely rescaled so that they sum to
  the requested total while keeping the minimum, then rounded by the largest
  remainder.
* The copied-column matrix tops every random column up to at least 8 nonzeros,
  so that no random column is (nearly) zero and the only null vectors are the
  planted ones.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

BASE_SEED = 0x2407046340


def config_seed(c: int) -> int:
    """Generator seed of benchmark configuration c (0-based)."""
    return BASE_SEED + c


def solver_seed(c: int) -> int:
    """Seed passed to the solver (random diagonal D and start block) for config c."""
    return 1000 + c


@dataclass
class CSR:
    rowptr: np.ndarray  # int64, m + 1
    colind: np.ndarray  # int32, nnz
    vals: np.ndarray  # float64 (values are exactly representable in float32)
    m: int
    n: int

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.vals, self.colind, self.rowptr), shape=(self.m, self.n))

    @staticmethod
    def from_scipy(M) -> "CSR":
        M = sp.csr_matrix(M)
        M.sum_duplicates()
        M.sort_indices()
        return CSR(
            rowptr=np.ascontiguousarray(M.indptr, dtype=np.int64),
            colind=np.ascontiguousarray(M.indices, dtype=np.int32),
            vals=np.ascontiguousarray(M.data, dtype=np.float64),
            m=M.shape[0],
            n=M.shape[1],
        )


@dataclass
class Workload:
    name: str
    A: CSR
    mode: str  # "spd": B = A + eps*D ; "normal": B = A^T A + eps*D
    nullity: int  # planted nullity
    labels: np.ndarray | None = None  # connected-component label of every column
    copy_pairs: np.ndarray | None = None  # (k, 2) int64: (source column, copied column)
    params: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _rescaled_sizes(raw: np.ndarray, total: int, minimum: int) -> np.ndarray:
    """Affine rescale of raw sizes (all >= minimum) to sum to total, integer by largest remainder."""
    k = raw.size
    assert total >= minimum * k
    excess = raw - minimum
    if excess.sum() <= 0:
        excess = np.ones_like(raw)
    target = excess * ((total - minimum * k) / excess.sum())
    base = np.floor(target).astype(np.int64)
    rem = int(total - minimum * k - base.sum())
    order = np.argsort(-(target - base), kind="stable")
    base[order[:rem]] += 1
    sizes = base + minimum
    assert sizes.sum() == total and sizes.min() >= minimum
    return sizes


def _cycle_edges(rng: np.random.Generator, offsets: np.ndarray, sizes: np.ndarray, ncycles: int):
    """Union of `ncycles` random Hamiltonian cycles on each block of contiguous nodes."""
    us, vs = [], []
    for off, s in zip(offsets, sizes):
        for _ in range(ncycles):
            p = rng.permutation(int(s)) + off
            us.append(p)
            vs.append(np.roll(p, -1))
    return np.concatenate(us), np.concatenate(vs)


def _laplacian(u: np.ndarray, v: np.ndarray, n: int) -> CSR:
    """Unit-weight graph Laplacian; duplicate edges merged, self loops dropped."""
    a = np.minimum(u, v).astype(np.int64)
    b = np.maximum(u, v).astype(np.int64)
    keep = a != b
    key = np.unique(a[keep] * n + b[keep])
    a, b = key // n, key % n
    deg = (np.bincount(a, minlength=n) + np.bincount(b, minlength=n)).astype(np.float64)
    rows = np.concatenate([a, b, np.arange(n)])
    cols = np.concatenate([b, a, np.arange(n)])
    vals = np.concatenate([-np.ones(2 * a.size), deg])
    return CSR.from_scipy(sp.coo_matrix((vals, (rows, cols)), shape=(n, n)))


def _labels_from_sizes(sizes: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(sizes.size, dtype=np.int64), sizes)


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------

def laplacian_er_components(seed: int, ncomp: int = 20, size: int = 100, p: float = 0.05) -> Workload:
    """Laplacian of `ncomp` disjoint connected Erdos-Renyi G(size, p) graphs."""
    rng = np.random.default_rng(seed)
    n = ncomp * size
    us, vs = [], []
    iu = np.triu_indices(size, 1)
    for c in range(ncomp):
        while True:
            mask = rng.random(iu[0].size) < p
            a, b = iu[0][mask], iu[1][mask]
            g = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(size, size))
            ncc, _ = sp.csgraph.connected_components(g, directed=False)
            if ncc == 1:
                break
        us.append(a + c * size)
        vs.append(b + c * size)
    perm = rng.permutation(n)
    u = perm[np.concatenate(us)]
    v = perm[np.concatenate(vs)]
    labels = np.empty(n, dtype=np.int64)
    labels[perm] = _labels_from_sizes(np.full(ncomp, size))
    return Workload("laplacian_er", _laplacian(u, v, n), "spd", ncomp, labels=labels)


def laplacian_cycle_components(seed: int, n: int, ncomp: int, mean_degree: int = 8,
                               sizes: str = "powerlaw", min_size: int = 50,
                               max_uniform: int | None = None) -> Workload:
    """Laplacian of `ncomp` disjoint components, each a union of mean_degree/2 random cycles.

    sizes="powerlaw": Pareto(alpha=1, x_min=min_size) draws rescaled to sum n.
    sizes="uniform": U{min_size, max_uniform} draws rescaled to sum n.
    """
    rng = np.random.default_rng(seed)
    if sizes == "powerlaw":
        raw = min_size / (1.0 - rng.random(ncomp))
    else:
        hi = max_uniform if max_uniform is not None else 39 * min_size
        raw = rng.integers(min_size, hi + 1, size=ncomp).astype(np.float64)
    sz = _rescaled_sizes(raw, n, max(3, min_size))
    offsets = np.concatenate([[0], np.cumsum(sz)[:-1]])
    u, v = _cycle_edges(rng, offsets, sz, mean_degree // 2)
    perm = rng.permutation(n)
    labels = np.empty(n, dtype=np.int64)
    labels[perm] = _labels_from_sizes(sz)
    return Workload("laplacian_cycles", _laplacian(perm[u], perm[v], n), "spd", ncomp, labels=labels)


def laplacian_grid_components(seed: int, ncomp: int, side_min: int = 10, side_max: int = 40) -> Workload:
    """Laplacian of `ncomp` disjoint 2-D grid graphs (4-neighbour, unit weights), side
    lengths uniform in [side_min, side_max] per axis.  A grid's smallest nonzero
    eigenvalue falls like 1/side^2, so these components are badly conditioned: a
    stand-in for the real-world Laplacians whose condition numbers outer
    preconditioning is meant to reduce (Sec. 5.1)."""
    rng = np.random.default_rng(seed)
    shapes = rng.integers(side_min, side_max + 1, size=(ncomp, 2))
    sz = shapes[:, 0] * shapes[:, 1]
    offsets = np.concatenate([[0], np.cumsum(sz)[:-1]])
    us, vs = [], []
    for (a, b), o in zip(shapes, offsets):
        idx = o + np.arange(a * b).reshape(a, b)
        us += [idx[:, :-1].ravel(), idx[:-1, :].ravel()]
        vs += [idx[:, 1:].ravel(), idx[1:, :].ravel()]
    n = int(sz.sum())
    perm = rng.permutation(n)
    u = perm[np.concatenate(us)]
    v = perm[np.concatenate(vs)]
    labels = np.empty(n, dtype=np.int64)
    labels[perm] = _labels_from_sizes(sz)
    return Workload("laplacian_grid", _laplacian(u, v, n), "spd", ncomp, labels=labels)


def incidence_cycle_components(seed: int, n: int, ncomp: int, mean_degree: int = 8,
                               min_size: int = 100, max_size: int = 3900) -> Workload:
    """Oriented edge-vertex incidence matrix (+1 at the lower, -1 at the higher endpoint).

    Each component is a union of mean_degree/2 random Hamiltonian cycles; parallel
    edges are kept as separate rows, so m = (mean_degree/2) * n exactly.  Rows are
    sorted by (lower endpoint, higher endpoint).  A^T A is the multigraph Laplacian,
    so the null space is spanned by the component indicators.
    """
    rng = np.random.default_rng(seed)
    raw = rng.integers(min_size, max_size + 1, size=ncomp).astype(np.float64)
    sz = _rescaled_sizes(raw, n, min_size)
    offsets = np.concatenate([[0], np.cumsum(sz)[:-1]])
    u, v = _cycle_edges(rng, offsets, sz, mean_degree // 2)
    perm = rng.permutation(n)
    u, v = perm[u], perm[v]
    lo, hi = np.minimum(u, v).astype(np.int64), np.maximum(u, v).astype(np.int64)
    order = np.lexsort((hi, lo))
    lo, hi = lo[order], hi[order]
    m = lo.size
    rowptr = np.arange(0, 2 * m + 1, 2, dtype=np.int64)
    colind = np.empty(2 * m, dtype=np.int32)
    colind[0::2] = lo
    colind[1::2] = hi
    vals = np.empty(2 * m, dtype=np.float64)
    vals[0::2] = 1.0
    vals[1::2] = -1.0
    labels = np.empty(n, dtype=np.int64)
    labels[perm] = _labels_from_sizes(sz)
    A = CSR(rowptr, colind, vals, m, n)
    return Workload("incidence_cycles", A, "normal", ncomp, labels=labels)


def rectangular_copies(seed: int, m: int, n: int, ncopies: int, nnz_per_row: int = 12,
                       min_col_nnz: int = 8) -> Workload:
    """m x n sparse matrix with N(0,1) float32-valued entries and `ncopies` planted
    sign-flipped column copies.

    The n - ncopies random columns receive `nnz_per_row` distinct uniform columns per
    row; columns with fewer than `min_col_nnz` entries are topped up at random rows.
    Copy j equals minus its (distinct) source column, so (e_src + e_copy)/sqrt(2)
    spans the planted null space.
    """
    rng = np.random.default_rng(seed)
    nr = n - ncopies
    cols = rng.integers(0, nr, size=(m, nnz_per_row), dtype=np.int64)
    while True:  # make the columns of every row distinct
        cols.sort(axis=1)
        dup = np.zeros(cols.shape, dtype=bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        if not dup.any():
            break
        cols[dup] = rng.integers(0, nr, size=int(dup.sum()))
    rows = np.repeat(np.arange(m, dtype=np.int64), nnz_per_row)
    cols = cols.ravel()
    cnt = np.bincount(cols, minlength=nr)
    low = np.nonzero(cnt < min_col_nnz)[0]
    if low.size:  # top up sparse columns; skip (row, col) pairs that already exist
        existing = set(zip(rows[np.isin(cols, low)].tolist(), cols[np.isin(cols, low)].tolist()))
        add_r, add_c = [], []
        for c in low.tolist():
            need = min_col_nnz - int(cnt[c])
            while need > 0:
                r = int(rng.integers(0, m))
                if (r, c) not in existing:
                    existing.add((r, c))
                    add_r.append(r)
                    add_c.append(c)
                    need -= 1
        rows = np.concatenate([rows, np.array(add_r, dtype=np.int64)])
        cols = np.concatenate([cols, np.array(add_c, dtype=np.int64)])
    vals = rng.standard_normal(rows.size).astype(np.float32).astype(np.float64)
    # sources of the copies: distinct random columns
    src = rng.choice(nr, size=ncopies, replace=False)
    order = np.argsort(cols, kind="stable")
    starts = np.searchsorted(cols[order], src)
    ends = np.searchsorted(cols[order], src, side="right")
    cr, cc, cv = [], [], []
    for j, (s0, s1) in enumerate(zip(starts, ends)):
        idx = order[s0:s1]
        cr.append(rows[idx])
        cc.append(np.full(idx.size, nr + j, dtype=np.int64))
        cv.append(-vals[idx])
    rows = np.concatenate([rows] + cr)
    cols = np.concatenate([cols] + cc)
    vals = np.concatenate([vals] + cv)
    # shuffle column labels so the copies are not the trailing columns
    perm = rng.permutation(n)
    M = sp.coo_matrix((vals, (rows, perm[cols])), shape=(m, n)).tocsr()
    assert M.nnz == rows.size, "duplicate (row, col) entry in generator"
    pairs = np.stack([perm[src], perm[nr + np.arange(ncopies)]], axis=1).astype(np.int64)
    return Workload("rectangular_copies", CSR.from_scipy(M), "normal", ncopies, copy_pairs=pairs)


def rectangular_copies_scaled(seed: int, m: int, n: int, ncopies: int, decades: float = 3.0) -> Workload:
    """rectangular_copies with every row multiplied by 10^u, u uniform in
    [-decades/2, decades/2]: a copied column stays a copy (both entries of a row get
    the same factor), so the planted null space is unchanged while A^T A becomes
    badly scaled -- the case inner preconditioning with diag(A A^T) is meant for."""
    w = rectangular_copies(seed, m, n, ncopies)
    rng = np.random.default_rng(seed + 7919)
    f = 10.0 ** rng.uniform(-decades / 2, decades / 2, size=w.A.m)
    A = w.A.to_scipy()
    w.A = CSR.from_scipy(sp.coo_matrix(sp.diags(f) @ A))
    w.name = "copies_scaled"
    return w


def batched_laplacians(seed: int, count: int, n_min: int = 200, n_max: int = 20000,
                       mean_degree: int = 6, max_comp: int = 8) -> list[Workload]:
    """Independent cycle-union Laplacians, n log-uniform in [n_min, n_max], 1..max_comp components."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        k = int(rng.integers(1, max_comp + 1))
        mmin = max(3, n // (4 * k))
        sz = _rescaled_sizes(rng.dirichlet(np.ones(k)) * n + mmin, n, mmin)
        offsets = np.concatenate([[0], np.cumsum(sz)[:-1]])
        u, v = _cycle_edges(rng, offsets, sz, mean_degree // 2)
        perm = rng.permutation(n)
        labels = np.empty(n, dtype=np.int64)
        labels[perm] = _labels_from_sizes(sz)
        out.append(Workload("batched_laplacian", _laplacian(perm[u], perm[v], n), "spd", k, labels=labels))
    return out


def diag_example() -> Workload:
    """Diagonal 10064 x 10064 matrix: 64 zeros, then 1 + k/10000 for k = 1..10000 (Sec. 1, eq. matrixA)."""
    n = 10064
    d = np.concatenate([np.zeros(64), 1.0 + np.arange(1, 10001) / 10000.0])
    nz = np.nonzero(d)[0]
    M = sp.csr_matrix((d[nz], (nz, nz)), shape=(n, n))
    labels = None
    return Workload("diag_example", CSR.from_scipy(M), "spd", 64, labels=labels)


def tiny_planted(seed: int, m: int, n: int, nullity: int, density: float = 0.15) -> Workload:
    """Small random sparse m x n matrix whose last `nullity` columns are random
    combinations of two earlier columns (nullity exactly `nullity` when the rest
    has full column rank, which the tests confirm with a dense SVD)."""
    rng = np.random.default_rng(seed)
    base = n - nullity
    Md = (rng.random((m, base)) < density) * rng.standard_normal((m, base))
    for j in range(base):  # no empty columns
        if not Md[:, j].any():
            Md[rng.integers(0, m), j] = 1.0
    extra = np.zeros((m, nullity))
    for j in range(nullity):
        a, b = rng.choice(base, size=2, replace=False)
        extra[:, j] = rng.choice([-2.0, -1.0, 1.0, 2.0]) * Md[:, a] + rng.choice([-1.0, 0.5, 1.0]) * Md[:, b]
    perm = rng.permutation(n)
    full = np.concatenate([Md, extra], axis=1)
    Ad = np.empty_like(full)
    Ad[:, perm] = full
    return Workload("tiny_planted", CSR.from_scipy(sp.csr_matrix(Ad)), "normal", nullity)


# ----------------------------------------------------------------------------
# the five benchmark configurations (full size) and their reduced-size twins
# ----------------------------------------------------------------------------

CONFIGS = {
    1: dict(d=1, restart=60, tol=1e-10, precision="fp64"),
    2: dict(d=1, restart=120, tol=1e-10, precision="fp64"),
    3: dict(d=4, restart=160, tol=1e-10, precision="mixed"),
    4: dict(d=2, restart=150, tol=1e-10, precision="mixed"),
    5: dict(d=1, restart=40, tol=1e-5, precision="mixed"),
    # not one of the five benchmark configurations: badly conditioned grid Laplacians
    # for the outer preconditioning (Sec. 4.4.2, Sec. 5.1)
    6: dict(d=1, restart=120, tol=1e-10, precision="fp64"),
}


def make_config(c: int, scale: float = 1.0):
    """Benchmark configuration c (1..5; 6 = 500 grid Laplacians, sides 15-30).  scale < 1 shrinks sizes and component
    counts proportionally (reduced-size twins used by the parity tests)."""
    seed = config_seed(c - 1)
    p = dict(CONFIGS[c])
    if c == 1:
        w = laplacian_er_components(seed)
    elif c == 2:
        n = int(1_000_000 * scale)
        k = max(2, int(500 * scale))
        w = laplacian_cycle_components(seed, n, k, 8, "powerlaw", 50)
    elif c == 3:
        k = max(2, int(1000 * scale))
        n = int(2_000_000 * scale)
        w = incidence_cycle_components(seed, n, k, 8, 100, 3900)
    elif c == 4:
        m, n = int(3_000_000 * scale), int(2_000_000 * scale)
        w = rectangular_copies(seed, m, n, max(2, int(300 * scale)))
    elif c == 5:
        return batched_laplacians(seed, max(1, int(4096 * scale))), p
    elif c == 6:
        w = laplacian_grid_components(seed, max(2, int(500 * scale)), 15, 30)
    else:
        raise ValueError(c)
    w.params = p
    return w, p
