"""The integral factorisations of Sec. II.C on the GPU against the oracle
(oracle/factors.py): DF factors in the MO basis and the pivoted Cholesky
decomposition of the integrals, then the energy computed from them.

The GPU's DF factors use the Cholesky factor of the metric as its inverse
square root, the oracle the symmetric one; the two differ by a rotation of
the auxiliary index, so the comparison is on the integrals sum_Q B^Q_pq B^Q_rs
(and, for the identity metric, on the factors themselves). Bars: 1e-11 of the
largest integral (FP64 GEMMs over a few hundred terms); energies 1e-10
relative (the FP64 bar).
"""
import numpy as np
import pytest

from dsrg_synth import make_ao_problem, make_eri_factors, make_problem
from oracle import dsrg as odsrg
from oracle import factors as ofac

pytestmark = pytest.mark.gpu

BLOCKS = ["ccvv", "cavv", "ccav", "active", "total"]


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64).cuda()


@pytest.mark.parametrize("nbf,nmo,naux,seed", [(20, 20, 50, 0), (24, 18, 70, 1), (9, 9, 257, 2)])
def test_df_factors_give_the_df_integrals(pk, nbf, nmo, naux, seed):
    p = make_ao_problem(nbf, nmo, naux, seed=seed)
    B = pk.df_mo_transform(_dev(p.ao3), _dev(p.C), _dev(p.metric)).cpu().numpy()
    lhs = np.einsum("Qpq,Qrs->pqrs", B, B)
    rhs = ofac.df_integrals(p.ao3, p.C, p.metric)
    assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(rhs).max()


def test_df_identity_metric_and_sub_blocks(pk):
    """With J = I the factors are the MO three-centre integrals; a hole x
    particle sub-block of rows and columns equals that block of the full result."""
    p = make_ao_problem(16, 14, 40, seed=3)
    I = np.eye(40)
    B = pk.df_mo_transform(_dev(p.ao3), _dev(p.C), _dev(I)).cpu().numpy()
    mo = ofac.mo_three_centre(p.ao3, p.C)
    assert np.abs(B - mo).max() <= 1e-12 * np.abs(mo).max()
    Bs = pk.df_mo_transform(_dev(p.ao3), _dev(p.C), _dev(p.metric), 0, 5, 3, 11).cpu().numpy()
    Bf = pk.df_mo_transform(_dev(p.ao3), _dev(p.C), _dev(p.metric)).cpu().numpy()
    assert np.abs(Bs - Bf[:, :5, 3:]).max() <= 1e-13 * np.abs(Bf).max()


def test_df_rejects_an_indefinite_metric(pk):
    p = make_ao_problem(6, 6, 8, seed=4)
    M = p.metric.copy()
    M[3, 3] = -1.0
    with pytest.raises(pk.DSRGError):
        pk.df_mo_transform(_dev(p.ao3), _dev(p.C), _dev(M))


def test_energy_from_df_factors(pk):
    """The DSRG-MRPT2 energy from the GPU's DF factors (hole x particle block)
    equals the oracle's energy from its J^{-1/2} factors: same integrals."""
    nC, nA, nV = 4, 2, 30
    n = nC + nA + nV
    p = make_ao_problem(n, n, 90, seed=5)
    q = make_problem(nC, nA, nV, 1, s=0.5, seed=5)
    B = pk.df_mo_transform(_dev(p.ao3), _dev(p.C), _dev(p.metric), 0, nC + nA, nC, nA + nV)
    plan = pk.Plan(nC, nA, nV, 90, precision="fp64")
    e = plan.energy(B, _dev(q.eps), _dev(q.gamma1), _dev(q.lambda2), q.s).cpu().numpy()
    Bo = ofac.df_factors(p.ao3, p.C, p.metric, slice(0, nC + nA), slice(nC, n))
    ref = odsrg.energy(Bo, q.eps, q.gamma1, q.lambda2, q.s, nC, nA, nV)
    for k, v in zip(BLOCKS, e):
        assert abs(v - ref[k]) <= 1e-10 * abs(ref[k]), (k, v, ref[k])


@pytest.mark.parametrize("n,rank,tau,seed", [(8, 30, 1e-5, 0), (12, 60, 1e-5, 1), (10, 200, 1e-8, 2)])
def test_cholesky_factors_against_the_oracle(pk, n, rank, tau, seed):
    F = make_eri_factors(n, rank, seed=seed)
    L = pk.cd_factors(_dev(F), tau).cpu().numpy()
    M = np.einsum("kpq,krs->pqrs", F, F).reshape(n * n, n * n)
    Lo, piv = ofac.pivoted_cholesky(lambda p: M[:, p], np.diag(M), tau)
    print(n, rank, tau, "rank gpu", L.shape[0], "oracle", Lo.shape[1])
    assert L.shape[0] == Lo.shape[1]
    assert np.abs(L.reshape(L.shape[0], -1) - Lo.T).max() <= 1e-10 * np.abs(Lo).max()
    R = M - L.reshape(L.shape[0], -1).T @ L.reshape(L.shape[0], -1)
    assert np.diag(R).max() < tau
    assert np.abs(R).max() < tau


def test_energy_from_cholesky_factors(pk):
    """CD factors of exact integrals (threshold 1e-5 Eh, the paper's value) as
    the source of B: the energy from the GPU's vectors equals the oracle's
    energy from its own decomposition, and both stay within the decomposition
    error of the energy from the exact factors."""
    nC, nA, nV = 3, 2, 20
    n = nC + nA + nV
    F = make_eri_factors(n, 120, seed=6)
    q = make_problem(nC, nA, nV, 1, s=0.5, seed=6)
    L = pk.cd_factors(_dev(F), 1e-5)
    rank = L.shape[0]
    Bhp = L[:, : nC + nA, nC:].contiguous()
    plan = pk.Plan(nC, nA, nV, rank, precision="fp64")
    e = plan.energy(Bhp, _dev(q.eps), _dev(q.gamma1), _dev(q.lambda2), q.s).cpu().numpy()
    M = np.einsum("kpq,krs->pqrs", F, F).reshape(n * n, n * n)
    Lo, _ = ofac.pivoted_cholesky(lambda p: M[:, p], np.diag(M), 1e-5)
    Bo = Lo.T.reshape(-1, n, n)[:, : nC + nA, nC:]
    ref = odsrg.energy(Bo, q.eps, q.gamma1, q.lambda2, q.s, nC, nA, nV)
    exact = odsrg.energy(F[:, : nC + nA, nC:], q.eps, q.gamma1, q.lambda2, q.s, nC, nA, nV)
    for k, v in zip(BLOCKS, e):
        assert abs(v - ref[k]) <= 1e-10 * abs(ref[k]), (k, v, ref[k])
    print("CD rank", rank, "total", e[4], "exact", exact["total"])
    assert abs(e[4] - exact["total"]) <= 1e-3 * abs(exact["total"])
