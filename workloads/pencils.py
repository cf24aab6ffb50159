"""Seeded synthetic pencils (A, B): the inputs both the oracle and the CUDA path consume.

This module only *builds inputs*: it holds none of the slicing method's arithmetic
(no factorisation, no eigensolver, no shift placement).  Every generator is
deterministic for a given seed and returns a symmetric CSR pattern with two value
arrays aligned to it.

Pencils provided
----------------
* ``gaussian_pencil``: s-type Gaussian-orbital pencils on a cubic atom lattice, the
  stand-in for the paper's DFT pencils (problem statement, Eq. 1: A symmetric, B SPD).
  S_ij = N_a N_b (pi/(a+b))^{3/2} exp(-mu r^2) with normalised primitives, so
  S_ij = (2 sqrt(ab)/(a+b))^{3/2} exp(-mu r^2), mu = ab/(a+b), S_ii = 1;
  kinetic T_ij = mu (3 - 2 mu r^2) S_ij; potential V_ij = (v_I + v_J)/2 S_ij with
  v_I ~ U(-1, 0) per atom.  A = T + V, B = S.  Entries with |.| < drop are dropped
  from S and from A separately; the stored pattern is the union, where an entry
  dropped from one matrix is an explicit zero in that matrix.
* ``laplacian_1d``: K = tridiag(-1, 2, -1) with B = I (``mass=False``) or the
  linear-FEM mass matrix M = tridiag(1, 4, 1)/6 (``mass=True``).
* ``scf_sequence_perturbation``: a seeded symmetric U(-1,1) matrix R on A's own
  nonzero pattern, for pencils A_k = A_0 + 0.1 * 2^-k * R.
* ``random_sparse_pencil``: small random symmetric pencils (B diagonally dominant SPD)
  for edge-case tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BOHR_SPACING = 2.0
EXPONENTS_4 = (0.3, 0.8, 2.0, 5.0)
EXPONENTS_2 = (0.3, 2.0)


def exponents_8() -> tuple:
    """Eight exponents log-spaced over [0.2, 8.0]: a_i = 0.2 * 40^(i/7)."""
    return tuple(float(0.2 * 40.0 ** (i / 7.0)) for i in range(8))


@dataclass
class Pencil:
    """A symmetric pencil stored on one full (both triangles) CSR pattern."""
    n: int
    rowptr: np.ndarray          # int64[n+1]
    colind: np.ndarray          # int32[nnz], sorted within each row
    a: np.ndarray               # float64[nnz]
    b: np.ndarray               # float64[nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def rows(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))

    def dense(self, which: str = "a") -> np.ndarray:
        m = np.zeros((self.n, self.n))
        v = self.a if which == "a" else self.b
        m[self.rows(), self.colind] = v
        return m

    def with_a(self, a_new: np.ndarray) -> "Pencil":
        return Pencil(self.n, self.rowptr, self.colind, a_new, self.b, dict(self.meta))


def _lattice_offsets(rmax_sites: float):
    """Integer lattice offsets (dz, dy, dx) with |d| <= rmax, in lexicographic order."""
    r = int(np.floor(rmax_sites))
    d = np.arange(-r, r + 1)
    dz, dy, dx = np.meshgrid(d, d, d, indexing="ij")
    dz, dy, dx = dz.ravel(), dy.ravel(), dx.ravel()
    keep = (dx * dx + dy * dy + dz * dz) <= rmax_sites * rmax_sites + 1e-9
    return dz[keep], dy[keep], dx[keep]


def _pair_cutoff(exps, drop):
    """Largest distance (bohr) at which any function pair can still reach |.| >= drop."""
    rmax = 0.0
    r = np.linspace(0.0, 60.0, 60001)
    for a in exps:
        for b in exps:
            mu = a * b / (a + b)
            s = (2.0 * np.sqrt(a * b) / (a + b)) ** 1.5 * np.exp(-mu * r * r)
            t = mu * (3.0 - 2.0 * mu * r * r) * s
            alive = (s >= drop) | (np.abs(t) + s >= drop)
            rmax = max(rmax, float(r[alive].max()))
    return rmax + 0.05


def gaussian_pencil(dims, exps=EXPONENTS_4, seed: int = 1, spacing: float = BOHR_SPACING,
                    drop: float = 1e-6, chunk_atoms: int = 1024, compensate_drop: bool = False) -> Pencil:
    """s-type Gaussian-orbital pencil on a dims[0] x dims[1] x dims[2] atom lattice.

    Basis ordering: atom-major (atom = x + Lx*(y + Ly*z)), then function index in
    ``exps`` order.  The per-atom potentials are drawn as
    ``np.random.default_rng(seed).uniform(-1, 0, n_atoms)``.

    compensate_drop: add to each diagonal entry of S the overlap mass its row loses to
    the drop rule, sum_j (S_exact)_ij - sum_j (S_kept)_ij over the whole lattice.  Every
    S entry is positive, so S_kept + D - S_exact is diagonally dominant and S_kept + D is
    at least as positive definite as the exact overlap -- needed where the drop alone
    leaves S indefinite (a nearly linearly dependent basis).
    """
    lx, ly, lz = (int(d) for d in dims)
    exps = np.asarray(exps, dtype=np.float64)
    nf = exps.size
    n_atoms = lx * ly * lz
    n = n_atoms * nf
    rng = np.random.default_rng(seed)
    v_atom = rng.uniform(-1.0, 0.0, n_atoms)

    rcut = _pair_cutoff(exps, drop)
    odz, ody, odx = _lattice_offsets(rcut / spacing)
    r2_off = (odx * odx + ody * ody + odz * odz).astype(np.float64) * spacing * spacing

    # function-pair constants, shape (nf, nf)
    ea, eb = np.meshgrid(exps, exps, indexing="ij")
    mu = ea * eb / (ea + eb)
    pref = (2.0 * np.sqrt(ea * eb) / (ea + eb)) ** 1.5

    ax = np.arange(n_atoms)
    x_of = ax % lx
    y_of = (ax // lx) % ly
    z_of = ax // (lx * ly)

    rowptr_counts = np.zeros(n, dtype=np.int64)
    col_parts, a_parts, b_parts = [], [], []
    for i0 in range(0, n_atoms, chunk_atoms):
        i1 = min(n_atoms, i0 + chunk_atoms)
        I = np.arange(i0, i1)
        xi, yi, zi = x_of[I], y_of[I], z_of[I]
        # atom pairs (I, J) within the cutoff, ordered by I then J (offsets are
        # lexicographic in (dz, dy, dx), so J increases with the offset index)
        jx = xi[:, None] + odx[None, :]
        jy = yi[:, None] + ody[None, :]
        jz = zi[:, None] + odz[None, :]
        ok = (jx >= 0) & (jx < lx) & (jy >= 0) & (jy < ly) & (jz >= 0) & (jz < lz)
        pi, po = np.nonzero(ok)                      # row-major: sorted by I, then offset
        J = jx[pi, po] + lx * (jy[pi, po] + ly * jz[pi, po])
        Ig = I[pi]
        r2 = r2_off[po]
        npair = pi.size
        # values for every function pair: shape (npair, nf, nf)
        e = np.exp(-mu[None, :, :] * r2[:, None, None])
        s = pref[None, :, :] * e
        t = mu[None, :, :] * (3.0 - 2.0 * mu[None, :, :] * r2[:, None, None]) * s
        vv = 0.5 * (v_atom[Ig] + v_atom[J])
        a = t + vv[:, None, None] * s
        s = np.where(np.abs(s) < drop, 0.0, s)
        a = np.where(np.abs(a) < drop, 0.0, a)
        # reorder (pair, fa, fb) -> row-major CSR order (I, fa, J, fb)
        cnt = np.bincount(pi, minlength=i1 - i0)          # pairs per atom in chunk
        p0 = np.concatenate(([0], np.cumsum(cnt)[:-1]))
        q = np.arange(npair) - p0[pi]                       # local pair index
        fa = np.arange(nf)
        fb = np.arange(nf)
        dest = (p0[pi][:, None, None] * nf * nf
                + fa[None, :, None] * (cnt[pi][:, None, None] * nf)
                + q[:, None, None] * nf + fb[None, None, :])
        col = np.broadcast_to(J[:, None, None] * nf + fb[None, None, :], (npair, nf, nf))
        tot = npair * nf * nf
        col_o = np.empty(tot, dtype=np.int64)
        a_o = np.empty(tot)
        s_o = np.empty(tot)
        col_o[dest.ravel()] = col.ravel()
        a_o[dest.ravel()] = a.ravel()
        s_o[dest.ravel()] = s.ravel()
        keep = (a_o != 0.0) | (s_o != 0.0)
        # row of each kept entry: rows run (I, fa) with cnt[I]*nf entries each
        per_row = np.repeat(cnt, nf) * nf
        row_local = np.repeat(np.arange((i1 - i0) * nf), per_row)
        rowptr_counts[i0 * nf:i1 * nf] = np.bincount(row_local[keep], minlength=(i1 - i0) * nf)
        col_parts.append(col_o[keep].astype(np.int32))
        a_parts.append(a_o[keep])
        b_parts.append(s_o[keep])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(rowptr_counts, out=rowptr[1:])
    colind = np.concatenate(col_parts)
    b_vals = np.concatenate(b_parts)
    if compensate_drop:
        # full-lattice row sums of S: the Gaussian factorises over the three axes, so the
        # sum over all atoms J is a product of three one-dimensional sums
        def axis_sums(L):
            d = np.arange(L)[:, None] - np.arange(L)[None, :]            # (coordinate, other)
            g = np.exp(-mu[:, :, None, None] * (spacing * d[None, None, :, :]) ** 2)
            return g.sum(axis=3)                                        # (nf, nf, L)
        gx, gy, gz = axis_sums(lx), axis_sums(ly), axis_sums(lz)
        tot = np.einsum("ab,abn->nab", pref, gx[:, :, x_of] * gy[:, :, y_of] * gz[:, :, z_of])
        total = tot.sum(axis=2).reshape(n)                              # row (atom, fa)
        kept = np.add.reduceat(b_vals, rowptr[:-1]) if n else np.zeros(0)
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
        diag = np.flatnonzero(colind == rows)
        b_vals = b_vals.copy()
        b_vals[diag] += np.maximum(total - kept, 0.0)
    meta = dict(kind="gaussian", dims=(lx, ly, lz), exps=tuple(float(x) for x in exps),
                seed=seed, spacing=spacing, drop=drop, compensate_drop=compensate_drop)
    return Pencil(n, rowptr, colind, np.concatenate(a_parts), b_vals, meta)


def laplacian_1d(n: int, mass: bool = False) -> Pencil:
    """K = tridiag(-1, 2, -1); B = I, or the linear-FEM mass matrix tridiag(1,4,1)/6."""
    rows, cols, a, b = [], [], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                a.append(2.0 if i == j else -1.0)
                if mass:
                    b.append(4.0 / 6.0 if i == j else 1.0 / 6.0)
                else:
                    b.append(1.0 if i == j else 0.0)
    rows = np.asarray(rows)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Pencil(n, rowptr, np.asarray(cols, dtype=np.int32), np.asarray(a, dtype=np.float64),
                  np.asarray(b, dtype=np.float64), dict(kind="laplacian_1d", mass=mass))


def scf_sequence_perturbation(p: Pencil, seed: int = 33) -> np.ndarray:
    """Symmetric R with U(-1,1) values on A's own nonzero pattern, aligned to p's CSR."""
    rows = p.rows()
    cols = p.colind.astype(np.int64)
    upper = (cols >= rows) & (p.a != 0.0)
    rng = np.random.default_rng(seed)
    r_up = rng.uniform(-1.0, 1.0, int(upper.sum()))
    key_up = rows[upper] * p.n + cols[upper]
    # mirror entries: (c, r) for each stored (r, c) in the upper triangle
    key_all = np.minimum(rows, cols) * p.n + np.maximum(rows, cols)
    pos = np.searchsorted(key_up, key_all)
    pos = np.clip(pos, 0, max(0, key_up.size - 1))
    hit = (key_up.size > 0) & (key_up[pos] == key_all) & (p.a != 0.0)
    r = np.zeros(p.nnz)
    r[hit] = r_up[pos[hit]]
    return r


def scf_pencil(p: Pencil, r: np.ndarray, k: int) -> Pencil:
    """A_k = A_0 + 0.1 * 2^-k * R (config of the 10-pencil SCF-like sequence)."""
    return p.with_a(p.a + 0.1 * 2.0 ** (-k) * r)


def random_sparse_pencil(n: int, density: float, seed: int) -> Pencil:
    """Random symmetric A (indefinite) and diagonally dominant SPD B on one pattern."""
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < density
    m = m | m.T
    np.fill_diagonal(m, True)
    rows, cols = np.nonzero(m)
    a_full = rng.uniform(-1.0, 1.0, (n, n))
    a_full = 0.5 * (a_full + a_full.T)
    b_full = rng.uniform(-0.5, 0.5, (n, n))
    b_full = 0.5 * (b_full + b_full.T) * m
    np.fill_diagonal(b_full, 0.0)
    np.fill_diagonal(b_full, np.abs(b_full).sum(axis=1) + 1.0)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Pencil(n, rowptr, cols.astype(np.int32), a_full[rows, cols], b_full[rows, cols],
                  dict(kind="random", seed=seed, density=density))


def config_pencil(config: int) -> Pencil:
    """The benchmark pencils: 1 = 6^3 lattice, 4 functions (N=864, seed 1);
    2 = 16^3, 4 functions (N=16,384, seed 2); 3 = 24^3, 8 functions (N=110,592, seed 3,
    dropped overlap mass compensated on the diagonal)."""
    if config == 1:
        return gaussian_pencil((6, 6, 6), EXPONENTS_4, seed=1)
    if config == 2:
        return gaussian_pencil((16, 16, 16), EXPONENTS_4, seed=2)
    if config == 3:
        # the eight-exponent basis is nearly linearly dependent (lambda_min of the exact
        # overlap ~ 1e-7): the 1e-6 drop alone leaves S indefinite, so the dropped overlap
        # mass is moved to the diagonal (compensate_drop)
        return gaussian_pencil((24, 24, 24), exponents_8(), seed=3, compensate_drop=True)
    raise ValueError(f"unknown config {config}")


def uneven_batch_specs(count: int = 256, seed: int = 44):
    """The uneven batch of independent pencils: for each, lattice dims drawn uniformly from
    8..18 per axis and 2 or 4 functions per atom (EXPONENTS_2 / EXPONENTS_4, equally
    likely), with its own potential seed.  Returns a list of (dims, exps, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dims = tuple(int(d) for d in rng.integers(8, 19, size=3))
        exps = EXPONENTS_4 if rng.random() < 0.5 else EXPONENTS_2
        out.append((dims, exps, 1000 + i))
    return out


def batch_pencils(specs):
    return [gaussian_pencil(d, e, seed=s_) for d, e, s_ in specs]


def stack_pencils(pencils):
    """Block-diagonal stack of independent pencils on one pattern: pencil p's rows and
    columns follow those of pencils 0..p-1.  Returns (stacked Pencil, pencil of each row,
    row offset of each pencil)."""
    offs = np.cumsum([0] + [q.n for q in pencils]).astype(np.int64)
    nnz_off = np.cumsum([0] + [q.nnz for q in pencils]).astype(np.int64)
    rowptr = np.concatenate([[0]] + [q.rowptr[1:] + nnz_off[i] for i, q in enumerate(pencils)]).astype(np.int64)
    colind = np.concatenate([q.colind.astype(np.int64) + offs[i] for i, q in enumerate(pencils)]).astype(np.int32)
    a = np.concatenate([q.a for q in pencils])
    b = np.concatenate([q.b for q in pencils])
    seg = np.concatenate([np.full(q.n, i, dtype=np.int32) for i, q in enumerate(pencils)])
    st = Pencil(int(offs[-1]), rowptr, colind, a, b, dict(kind="stack", count=len(pencils)))
    return st, seg, offs


def normal_block(n: int, k: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) start block, N x k row-major (used as V0 / Lanczos start vectors)."""
    return np.random.default_rng(seed).standard_normal((n, k))
