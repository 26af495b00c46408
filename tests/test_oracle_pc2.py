"""PC2 (Sec. 3.1) on the conduction Backward Euler system: how many PCG iterations an
incomplete-factorisation preconditioner saves against point-Jacobi (PC1), and how much of that
saving the GPU-parallel form keeps.

The system is the oracle's S x = b (S = M - dt A, b = M u^n) on a 24 x 24 x 48 dipole shell at
dt = 1e3 dt_E, solved to rtol 1e-10 from x0 = u^n.  S is assembled as a sparse matrix from the
oracle's 27-point row entries (checked against its matrix-free product).  Preconditioners:
  - point-Jacobi, D = diag(S) (the library's PC1);
  - IC0, the zero-fill incomplete Cholesky factor of S in the natural (r fastest) ordering: the
    symmetric form of the ILU0 that PC2 is;
  - symmetric Gauss-Seidel, (D + L) D^-1 (D + U), in the natural ordering;
  - the same two in the 8-colour ordering (colour = parity of (k, j, i)): with the 27-point
    stencil no two cells of one colour are coupled, so each triangular solve becomes 8 parallel
    colour steps -- the form a GPU can run;
  - block-local IC0 (PC2 as a distributed code applies it, ILU0 inside each subdomain): IC0 of S
    without the couplings between blocks, for GPU-tile-sized 8 x 8 x 8 blocks and for blocks of
    a third of the grid (16 phi x 24 theta x 24 r, a rank's subdomain).
Run with -s to print the iteration counts.  The checks pin that every preconditioned solve
reaches the same solution, that the factorisations save iterations in the natural order, that
the 8-colour order keeps less than a tenth of that saving, and that block-local IC0 keeps it
only with blocks far larger than a GPU tile."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from gpu_common import tc_problem


def _assemble(op):
    """A as a CSR matrix from the oracle's row entries A[cell, cell + o] (entries across the r
    and theta ends are zero, so a periodic index map in all three directions is exact)."""
    idx = np.arange(op.n).reshape(op.shape)
    I, J, V = [], [], []
    for (ok, oj, oi), a in op.row_entries().items():
        col = np.roll(idx, (-ok, -oj, -oi), axis=(0, 1, 2))
        m = a != 0.0
        I.append(idx[m])
        J.append(col[m])
        V.append(a[m])
    return sp.csr_matrix((np.concatenate(V), (np.concatenate(I), np.concatenate(J))), shape=(op.n, op.n))


def _pcg(S, b, x0, prec, rtol, max_iter=20000):
    """Textbook PCG with the stopping test r.r <= rtol^2 b.b (as the library's)."""
    x = x0.copy()
    r = b - S @ x
    tol2 = rtol * rtol * float(b @ b)
    z = prec(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, max_iter + 1):
        q = S @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        if float(r @ r) <= tol2:
            return x, it
        z = prec(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise AssertionError("PCG did not converge")


class _Breakdown(Exception):
    pass


def _ic0(S):
    """Zero-fill incomplete Cholesky S ~ L L^T on the lower pattern of S (row by row); raises
    _Breakdown at a non-positive pivot."""
    S = sp.csr_matrix(S)
    S.sort_indices()
    n = S.shape[0]
    rows = [dict() for _ in range(n)]
    for i in range(n):
        lo, hi = S.indptr[i], S.indptr[i + 1]
        Li = rows[i]
        for jj in range(lo, hi):
            j = int(S.indices[jj])
            if j > i:
                break
            Lj = rows[j]
            small, big = (Li, Lj) if len(Li) < len(Lj) else (Lj, Li)
            s = float(S.data[jj]) - sum(v * big.get(k, 0.0) for k, v in small.items() if k < j)
            if j < i:
                Li[j] = s / Lj[j]
            else:
                if not s > 0.0:
                    raise _Breakdown(i)
                Li[i] = np.sqrt(s)
    I = [i for i in range(n) for _ in rows[i]]
    J = [j for i in range(n) for j in rows[i]]
    V = [v for i in range(n) for v in rows[i].values()]
    return sp.csr_matrix((V, (I, J)), shape=(n, n))


SHIFTS = (0.0, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3, 1.0)


def _ic0_prec(S):
    """IC0 of S + alpha diag(S) with the smallest alpha of SHIFTS that has no breakdown (the
    corner scheme's S is SPD but not an M-matrix: it has positive off-diagonal entries, and
    plain IC0 need not exist)."""
    D = sp.diags(S.diagonal())
    for alpha in SHIFTS:
        try:
            L = _ic0(S + alpha * D)
            break
        except _Breakdown:
            continue
    Lt = sp.csr_matrix(L.T)
    f = lambda r: spla.spsolve_triangular(Lt, spla.spsolve_triangular(L, r, lower=True), lower=False)
    f.alpha = alpha
    return f


def _sgs_prec(S):
    D = S.diagonal()
    lower = sp.csr_matrix(sp.tril(S, 0))
    upper = sp.csr_matrix(sp.triu(S, 0))
    return lambda r: spla.spsolve_triangular(upper, D * spla.spsolve_triangular(lower, r, lower=True), lower=False)


def _block_local(S, shape, block):
    """S without the entries that couple different blocks of size block = (bk, bj, bi)."""
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    nb = [-(-n // b) for n, b in zip(shape, block)]
    blk = (((k // block[0]) * nb[1] + j // block[1]) * nb[2] + i // block[2]).reshape(-1)
    C = sp.coo_matrix(S)
    keep = blk[C.row] == blk[C.col]
    return sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=S.shape)


@pytest.fixture(scope="module")
def system():
    g, inp, op, u = tc_problem(24, 24, 48)
    A = _assemble(op)
    return op, A, u


def test_assembled_matrix_is_the_operator(system):
    op, A, u = system
    x = np.random.default_rng(3).standard_normal(op.n)
    ref = op.apply_A(x)
    assert np.abs(A @ x - ref).max() <= 1e-13 * np.abs(ref).max()
    assert abs(A - A.T).max() == 0.0


def test_pc2_iteration_counts(system):
    op, A, u = system
    dt = 1000.0 * op.dt_explicit()
    M = 1.0 / op.w
    S = sp.csr_matrix(sp.diags(M) - dt * A)
    b = M * u
    D = S.diagonal()
    k, j, i = np.meshgrid(*[np.arange(s) for s in op.shape], indexing="ij")
    colour = ((k % 2) * 4 + (j % 2) * 2 + (i % 2)).reshape(-1)
    perm = np.argsort(colour, kind="stable")
    Sp = sp.csr_matrix(S[perm][:, perm])
    # no two cells of one colour are coupled: each colour's diagonal block is diagonal
    for c in range(8):
        sel = np.nonzero(colour[perm] == c)[0]
        blk = Sp[sel][:, sel]
        assert blk.nnz == len(sel)
    runs = {}
    x_j, runs["point-Jacobi (PC1)"] = _pcg(S, b, u, lambda r: r / D, 1e-10)
    shifts = {}
    for name, mat, make in (("IC0, natural order", S, _ic0_prec), ("SGS, natural order", S, _sgs_prec),
                            ("IC0, 8 colours", Sp, _ic0_prec), ("SGS, 8 colours", Sp, _sgs_prec)):
        p = perm if mat is Sp else np.arange(op.n)
        pre = make(mat)
        shifts[name] = getattr(pre, "alpha", None)
        x, runs[name] = _pcg(mat, b[p], u[p], pre, 1e-10)
        xs = np.empty_like(x)
        xs[p] = x
        # the same system solved: true residual at the tolerance, and x within cond(S) times it
        assert np.linalg.norm(b - S @ xs) <= 2e-10 * np.linalg.norm(b), name
        assert np.linalg.norm(xs - x_j) <= 1e-6 * np.linalg.norm(x_j), name
    for name, block in (("block IC0, 8x8x8", (8, 8, 8)), ("block IC0, 16x24x24", (16, 24, 24))):
        pre = _ic0_prec(_block_local(S, op.shape, block))
        shifts[name] = pre.alpha
        x, runs[name] = _pcg(S, b, u, pre, 1e-10)
        assert np.linalg.norm(b - S @ x) <= 2e-10 * np.linalg.norm(b), name
    print()
    for name, it in runs.items():
        extra = f"  (IC0 of S + {shifts[name]:g} diag S)" if shifts.get(name) is not None else ""
        print(f"  {name:22s} {it:5d} iterations{extra}")
    # the factorisations save iterations in the natural (sequential) order ...
    assert runs["IC0, natural order"] < runs["SGS, natural order"] < runs["point-Jacobi (PC1)"]
    # ... and the parallel 8-colour order keeps less than a tenth of that saving
    for name in ("IC0, 8 colours", "SGS, 8 colours"):
        assert runs[name] >= 0.9 * runs["point-Jacobi (PC1)"], name
    # block-local IC0 keeps the saving only with blocks far larger than a GPU tile
    assert runs["block IC0, 8x8x8"] >= 0.75 * runs["point-Jacobi (PC1)"]
    assert runs["block IC0, 16x24x24"] <= 0.5 * runs["point-Jacobi (PC1)"]
