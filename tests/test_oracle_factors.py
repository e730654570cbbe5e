"""Pins of the factorisation oracle (Sec. II.C): the DF factors reproduce the
DF integrals sum_PQ (pq|P) [J^{-1}]_PQ (Q|rs) whatever square root of J^{-1}
is used; with an identity metric B is the MO three-centre tensor; the MO
transformation is exact against explicit AO -> MO products; the pivoted
Cholesky decomposition reproduces a PSD matrix to its threshold and recovers
an exactly low-rank one in as many steps as its rank."""
import numpy as np
import pytest

from dsrg_synth import make_ao_problem, make_eri_factors
from oracle import factors


@pytest.mark.parametrize("nbf,nmo,naux,seed", [(6, 6, 10, 0), (8, 5, 12, 1)])
def test_df_factors_reproduce_df_integrals(nbf, nmo, naux, seed):
    p = make_ao_problem(nbf, nmo, naux, seed=seed)
    B = factors.df_factors(p.ao3, p.C, p.metric)
    lhs = np.einsum("Qpq,Qrs->pqrs", B, B)
    rhs = factors.df_integrals(p.ao3, p.C, p.metric)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_identity_metric_gives_the_three_centre_integrals():
    p = make_ao_problem(5, 5, 7, seed=2)
    B = factors.df_factors(p.ao3, p.C, np.eye(7))
    mo = np.zeros((7, 5, 5))
    for P in range(7):
        for a in range(5):
            for b in range(5):
                mo[P, a, b] = sum(p.C[m, a] * p.ao3[P, m, n] * p.C[n, b]
                                  for m in range(5) for n in range(5))
    assert np.abs(B - mo).max() <= 1e-13 * np.abs(mo).max()


def test_df_integrals_invariant_under_metric_square_root():
    """Any W with W W^T = J^{-1} gives the same integrals: the inverse
    Cholesky factor and the symmetric inverse square root."""
    p = make_ao_problem(6, 6, 9, seed=3)
    mo = factors.mo_three_centre(p.ao3, p.C)
    Linv = np.linalg.inv(np.linalg.cholesky(p.metric))          # J = L L^T
    Bc = np.einsum("Ppq,QP->Qpq", mo, Linv)                      # L^{-1} (pq|.)
    Bs = factors.df_factors(p.ao3, p.C, p.metric)
    a = np.einsum("Qpq,Qrs->pqrs", Bc, Bc)
    b = np.einsum("Qpq,Qrs->pqrs", Bs, Bs)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("n,rank,seed", [(5, 8, 0), (6, 20, 1)])
def test_cholesky_recovers_low_rank_integrals(n, rank, seed):
    F = make_eri_factors(n, rank, seed=seed)
    eri = np.einsum("kpq,krs->pqrs", F, F)
    B = factors.cd_factors_from_eri(eri, 1e-12)
    # the matrix has rank <= min(rank, n (n+1) / 2): CD needs no more vectors
    assert B.shape[0] <= min(rank, n * (n + 1) // 2)
    rec = np.einsum("kpq,krs->pqrs", B, B)
    assert np.abs(rec - eri).max() <= 1e-10 * np.abs(eri).max()


def test_cholesky_threshold_bounds_the_error():
    """M - L L^T is PSD with diagonal below tau, so every element of it is
    below tau in magnitude (|M_ij| <= sqrt(M_ii M_jj) for a PSD matrix)."""
    F = make_eri_factors(6, 30, seed=4)
    eri = np.einsum("kpq,krs->pqrs", F, F)
    for tau in (1e-3, 1e-5):
        B = factors.cd_factors_from_eri(eri, tau)
        R = (eri - np.einsum("kpq,krs->pqrs", B, B)).reshape(36, 36)
        assert np.diag(R).max() < tau
        assert np.abs(R).max() < tau
        assert np.linalg.eigvalsh(R).min() > -1e-12
