"""Smoothed-aggregation AMG setup (oracle, FP64, test use only).

Follows the construction the paper uses (Sec. 3.2 and the AMG setup paragraph of Sec. 4,
smoothed aggregation after Vanek, Mandel & Brezina 1996):

1. block strength of connection, one value per node: nodes i != j are strongly connected when
   ||A_ij||_F^2 > beta ||A_ii||_F ||A_jj||_F with beta = 0.003 (Eq. 10; the Frobenius norm of
   the nodal blocks is the reading adopted for "one value per node");
2. aggregation of strongly connected nodes.  The paper names smoothed aggregation only; the
   aggregates here come from a distance-2 maximal independent set computed in synchronous
   rounds with splitmix64 priorities (the parallel scheme of Bell, Dalton & Olson 2012),
   so the CUDA path can reproduce them exactly:
     round:  v_j = TOP if j is IN, key_j if undecided, 0 if OUT;
             m1_i = max of v over {i} + strong neighbours; m2_i = max of m1 likewise;
             undecided i becomes OUT if m2_i = TOP, IN if m2_i = key_i.
   Nodes without strong neighbours start OUT and stay unaggregated.
   Phase 1: each IN node (root) takes its strong neighbours.  Phase 2: every node still
   unaggregated joins the phase-1 aggregate of its strong neighbour with the largest key.
   Aggregates are numbered in increasing root index.
3. tentative prolongator T from the near-nullspace B (rigid-body modes, Sec. 4): per
   aggregate, modified Gram-Schmidt QR of the aggregate's rows of B with a positive R
   diagonal; a column whose remainder falls below 1e-8 of its norm (rank-deficient aggregate)
   becomes a zero column.  Coarse candidates B_c = R.
4. P = (I - omega D^-1 A) T with D the point-block diagonal and omega = 4 / (3 rho(D^-1 A)),
   rho from 20 power iterations started at a splitmix64 vector ("improved with a weighted
   Jacobi smoother", Sec. 4; the weight is the reading adopted).
5. A_c = P^T A P (Eq. 9); a coarse DOF whose row is entirely zero (zero column of T) gets a
   unit diagonal so the coarse operator stays nonsingular; its correction is always 0.

Parity: pinned (tests/test_oracle_amg.py: brute-force distance-2 independence and maximality,
strength on E / 10E and E / 2E interfaces, T^T T = I, T B_c = B, P interpolates B up to the
smoothing step, SPD coarse operator).  Aggregate shapes differ from the paper's PETSc/PyAMG
(parity unpinned against the paper's own iteration counts, whose figures are lost).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .hashing import mis_keys, unit_uniform, SALT_POWER

TOP = np.uint64(np.iinfo(np.uint64).max)


def block_norms(A, b):
    """Nodal block Frobenius norms: returns (row_node, col_node, ||A_IJ||_F) for every stored
    block of A viewed with b x b blocks."""
    Ab = sp.bsr_matrix(A, blocksize=(b, b))
    Ab.sort_indices()
    nbr = Ab.shape[0] // b
    rows = np.repeat(np.arange(nbr), np.diff(Ab.indptr))
    cols = Ab.indices.astype(np.int64)
    fro = np.sqrt((Ab.data.reshape(len(cols), -1) ** 2).sum(axis=1))
    return rows, cols, fro


def strength(A, b, beta=0.003):
    """Symmetric nodal strength graph S (CSR, boolean pattern, no self loops) (Eq. 10)."""
    rows, cols, fro = block_norms(A, b)
    nn = A.shape[0] // b
    diag = np.zeros(nn)
    on = rows == cols
    diag[rows[on]] = fro[on]
    strong = (rows != cols) & (fro * fro > beta * diag[rows] * diag[cols])
    S = sp.csr_matrix((np.ones(int(strong.sum())), (rows[strong], cols[strong])), shape=(nn, nn))
    S.sort_indices()
    return S


def _neigh_max(S, v):
    """m_i = max(v_i, max_{j in N(i)} v_j) for uint64 v."""
    out = v.copy()
    rows = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    np.maximum.at(out, rows, v[S.indices])
    return out


def mis2(S, level):
    """Distance-2 maximal independent set by synchronous rounds (see module docstring).
    Returns (is_root bool array, keys uint64 array, isolated bool array)."""
    n = S.shape[0]
    keys = mis_keys(n, level)
    deg = np.diff(S.indptr)
    isolated = deg == 0
    UND, IN, OUT = 0, 1, 2
    state = np.where(isolated, OUT, UND)
    while (state == UND).any():
        v = np.where(state == IN, TOP, np.where(state == UND, keys, np.uint64(0))).astype(np.uint64)
        m2 = _neigh_max(S, _neigh_max(S, v))
        und = state == UND
        new = state.copy()
        new[und & (m2 == TOP)] = OUT
        new[und & (m2 == keys)] = IN
        state = new
    return state == IN, keys, isolated


def aggregate(S, level):
    """Aggregate id per node (-1 = unaggregated) and the number of aggregates."""
    is_root, keys, isolated = mis2(S, level)
    n = S.shape[0]
    agg = np.full(n, -1, dtype=np.int64)
    roots = np.flatnonzero(is_root)
    agg[roots] = np.arange(len(roots))
    # phase 1: neighbours of a root (the root is unique: roots are > 2 apart)
    agg1 = agg.copy()
    for i in range(n):
        if agg[i] >= 0 or isolated[i]:
            continue
        nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
        r = nb[is_root[nb]]
        if len(r):
            agg1[i] = agg[r[0]]
    # phase 2: join the phase-1 aggregate of the strong neighbour with the largest key
    agg2 = agg1.copy()
    for i in range(n):
        if agg1[i] >= 0 or isolated[i]:
            continue
        nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
        nb = nb[agg1[nb] >= 0]
        if len(nb) == 0:
            raise RuntimeError("node %d left unaggregated" % i)
        agg2[i] = agg1[nb[np.argmax(keys[nb])]]
    return agg2, len(roots)


def mgs_qr(Bm, tol=1e-8):
    """Modified Gram-Schmidt QR with positive R diagonal; columns whose remainder is below
    tol * (column norm) become zero columns of Q (and zero rows/diagonal of R)."""
    m, k = Bm.shape
    Q = np.zeros((m, k))
    R = np.zeros((k, k))
    for c in range(k):
        v = Bm[:, c].copy()
        n0 = np.sqrt(v @ v)
        for j in range(c):
            R[j, c] = Q[:, j] @ v
            v = v - R[j, c] * Q[:, j]
        nr = np.sqrt(v @ v)
        if n0 > 0.0 and nr > tol * n0:
            Q[:, c] = v / nr
            R[c, c] = nr
    return Q, R


def tentative(agg, n_agg, B, b):
    """Tentative prolongator T (n x n_agg*k) and coarse candidates B_c (n_agg*k x k)."""
    n, k = B.shape
    rows, cols, vals = [], [], []
    Bc = np.zeros((n_agg * k, k))
    order = np.argsort(agg, kind="stable")
    aggs = agg[order]
    starts = np.searchsorted(aggs, np.arange(n_agg))
    ends = np.searchsorted(aggs, np.arange(n_agg), side="right")
    for a in range(n_agg):
        nodes = order[starts[a]:ends[a]]  # ascending node index (stable sort)
        dofs = (b * nodes[:, None] + np.arange(b)[None, :]).ravel()
        Q, R = mgs_qr(B[dofs])
        Bc[a * k:(a + 1) * k] = R
        rr, cc = np.meshgrid(dofs, a * k + np.arange(k), indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(Q.ravel())
    T = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n_agg * k))
    T.eliminate_zeros()
    T.sort_indices()
    return T, Bc


def block_diag_inv(A, b):
    """Inverse nodal diagonal blocks, array (n/b, b, b)."""
    nn = A.shape[0] // b
    Ab = sp.bsr_matrix(A, blocksize=(b, b))
    Ab.sort_indices()
    rows = np.repeat(np.arange(nn), np.diff(Ab.indptr))
    on = Ab.indices == rows
    D = np.zeros((nn, b, b))
    D[rows[on]] = Ab.data[on]
    return np.linalg.inv(D)


def apply_block_diag(Dinv, x):
    nn, b, _ = Dinv.shape
    return np.einsum("nij,nj->ni", Dinv, x.reshape(nn, b)).ravel()


def block_diag_matrix(Dinv):
    nn, b, _ = Dinv.shape
    return sp.bsr_matrix((Dinv, np.arange(nn), np.arange(nn + 1)), shape=(nn * b, nn * b)).tocsr()


def spectral_radius_DinvA(A, Dinv, level, iters=20):
    """rho(D^-1 A) estimated by ``iters`` power iterations from a splitmix64 start vector."""
    v = unit_uniform(A.shape[0], SALT_POWER + level)
    v = v / np.linalg.norm(v)
    rho = 0.0
    for _ in range(iters):
        w = apply_block_diag(Dinv, A @ v)
        rho = np.linalg.norm(w)
        v = w / rho
    return rho


def smooth_prolongator(A, T, Dinv, level):
    """P = (I - omega D^-1 A) T, omega = 4 / (3 rho(D^-1 A))."""
    rho = spectral_radius_DinvA(A, Dinv, level)
    omega = 4.0 / (3.0 * rho)
    AT = (A @ T).tocsr()
    P = (T - omega * (block_diag_matrix(Dinv) @ AT)).tocsr()
    P.sort_indices()
    return P, omega


def fix_zero_rows(Ac):
    """Unit diagonal on coarse DOFs whose row is entirely zero."""
    Ac = Ac.tocsr()
    absrow = np.asarray(abs(Ac).sum(axis=1)).ravel()
    dead = absrow == 0.0
    if dead.any():
        Ac = (Ac + sp.diags(dead.astype(np.float64))).tocsr()
    return Ac


def sa_level(A, B, b, level, beta=0.003):
    """One smoothed-aggregation coarsening step.  Returns dict with S, agg, T, P, Ac, Bc."""
    S = strength(A, b, beta)
    agg, n_agg = aggregate(S, level)
    k = B.shape[1]
    T, Bc = tentative(agg, n_agg, B, b)
    Dinv = block_diag_inv(A, b)
    P, omega = smooth_prolongator(A, T, Dinv, level)
    Ac = fix_zero_rows(P.T @ A @ P)
    Ac.sort_indices()
    return dict(S=S, agg=agg, n_agg=n_agg, T=T, P=P, Ac=Ac, Bc=Bc, omega=omega, k=k)
