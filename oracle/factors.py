"""Oracle of the integral factorisations of Sec. II.C: density fitting (DF) in
the MO basis, and the Cholesky decomposition (CD) of the two-electron integrals.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy, FP64.

DF (Sec. II.C): B^Q_pq = sum_P (pq|P) [J^{-1/2}]_PQ with the MO three-centre
integrals (pq|P) = sum_{mu nu} C_{mu p} C_{nu q} (mu nu|P) and the two-centre
metric J. The factorised integrals are then (pq|rs) = sum_Q B^Q_pq B^Q_rs =
sum_{PQ} (pq|P) [J^{-1}]_PQ (Q|rs) for any square root of J^{-1}; this oracle
takes the symmetric one, J^{-1/2} = V diag(w^{-1/2}) V^T from the eigenvectors
of J.

CD (Sec. II.C): the integral matrix M[(pq),(rs)] = (pq|rs) is positive
semi-definite; its pivoted incomplete Cholesky decomposition (Golub & Van
Loan, Matrix Computations, "outer product" Cholesky with diagonal pivoting)
stops when the largest remaining diagonal element falls below the threshold
tau (1e-5 Eh in Table 3). Step k: pick the pair p with the largest remaining
diagonal d_p; L[:, k] = (M[:, p] - sum_{j<k} L[:, j] L[p, j]) / sqrt(d_p);
d -= L[:, k]^2. The factors are B^k_pq = L[(pq), k], and the error of every
integral is bounded by the largest remaining diagonal (M - L L^T is PSD).
"""
from __future__ import annotations

import numpy as np


def mo_three_centre(ao3, C, rows=None, cols=None):
    """(pq|P) = sum_{mu nu} C_{mu p} C_{nu q} (mu nu|P), layout [naux, p, q];
    ``rows`` / ``cols``: optional MO index ranges (slices) of p and q."""
    ao3 = np.asarray(ao3, float)
    C = np.asarray(C, float)
    Cp = C[:, rows] if rows is not None else C
    Cq = C[:, cols] if cols is not None else C
    return np.einsum("mp,Pmn,nq->Ppq", Cp, ao3, Cq, optimize=True)


def inverse_sqrt(Jm):
    """J^{-1/2} of a symmetric positive-definite metric (eigendecomposition)."""
    w, V = np.linalg.eigh(np.asarray(Jm, float))
    return (V * w ** -0.5) @ V.T


def df_factors(ao3, C, Jm, rows=None, cols=None):
    """B^Q_pq = sum_P (pq|P) [J^{-1/2}]_PQ, layout [naux, p, q]."""
    mo = mo_three_centre(ao3, C, rows, cols)
    return np.einsum("Ppq,PQ->Qpq", mo, inverse_sqrt(Jm), optimize=True)


def df_integrals(ao3, C, Jm, rows=None, cols=None):
    """(pq|rs) = sum_{PQ} (pq|P) [J^{-1}]_PQ (Q|rs): the DF integrals without any
    choice of square root, for the pins; [p, q, r, s] over the given ranges."""
    mo = mo_three_centre(ao3, C, rows, cols)
    Jinv = np.linalg.inv(np.asarray(Jm, float))
    return np.einsum("Ppq,PQ,Qrs->pqrs", mo, Jinv, mo, optimize=True)


def pivoted_cholesky(column, diag, tau, max_rank=None):
    """Pivoted incomplete Cholesky of a PSD matrix given by its diagonal and a
    function returning column p. Returns (L [N, k], pivots)."""
    d = np.array(diag, dtype=float)
    N = d.size
    max_rank = N if max_rank is None else max_rank
    cols, piv = [], []
    while len(cols) < max_rank:
        p = int(np.argmax(d))
        if d[p] < tau:
            break
        col = np.array(column(p), dtype=float)
        for Lj in cols:
            col -= Lj * Lj[p]
        col /= np.sqrt(d[p])
        cols.append(col)
        piv.append(p)
        d -= col * col
        d[p] = 0.0
    L = np.stack(cols, axis=1) if cols else np.zeros((N, 0))
    return L, piv


def cd_factors_from_eri(eri, tau):
    """CD factors of (pq|rs) given as a dense [n, n, n, n] array (tiny inputs):
    B [k, n, n] with (pq|rs) - sum_k B^k_pq B^k_rs below tau on the diagonal."""
    n = eri.shape[0]
    M = eri.reshape(n * n, n * n)
    L, _ = pivoted_cholesky(lambda p: M[:, p], np.diag(M), tau)
    return L.T.reshape(-1, n, n)
