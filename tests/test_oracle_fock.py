"""Pins of the Fock / semicanonicalisation oracle (Sec. II.B Eq. (8); Sec. III
steps 2-3) against what the mathematics fixes: Eq. (8) written literally in
spin orbitals from explicit four-index integrals, the defining property of the
semicanonical basis, exact transformation of the integrals, and invariance of
the whole pipeline under rotations of the input orbitals within each space."""
import numpy as np
import pytest

from dsrg_synth import make_fock_problem
from oracle import dsrg, fock

SIZES = [(2, 2, 4, 9, 1), (3, 0, 5, 7, 2), (1, 3, 3, 8, 3), (2, 1, 6, 10, 4)]


@pytest.mark.parametrize("nC,nA,nV,Q,seed", SIZES)
def test_spatial_fock_equals_eq8_in_spin_orbitals(nC, nA, nV, Q, seed):
    """f_p^q = h_p^q + sum_rs <pr||qs> gamma_s^r over spin orbitals (Eq. (8)),
    from the explicit four-index integrals, equals the spatial DF form for both
    spins and vanishes between spins."""
    p = make_fock_problem(nC, nA, nV, Q, seed=seed)
    f = fock.fock_spatial(p.h, p.Bfull, nC, nA, nV, p.gamma1)
    fso = fock.fock_spin_orbital(p.h, p.Bfull, nC, nA, nV, p.gamma1)
    assert np.abs(fso[0::2, 0::2] - f).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(fso[1::2, 1::2] - f).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(fso[0::2, 1::2]).max() == 0.0
    assert np.abs(f - f.T).max() <= 1e-14 * np.abs(f).max()


def test_fock_without_electrons_is_h():
    """No occupied orbitals (the density vanishes): f = h."""
    p = make_fock_problem(0, 2, 4, 6, seed=5)
    f = fock.fock_spatial(p.h, p.Bfull, 0, 2, 4, np.zeros((2, 2)))
    assert np.array_equal(f, p.h)


@pytest.mark.parametrize("nC,nA,nV,Q,seed", SIZES)
def test_semicanonical_basis(nC, nA, nV, Q, seed):
    """U is orthogonal and block diagonal; U^T f U is diagonal inside the core,
    active and virtual blocks with the orbital energies on the diagonal; each
    block's trace is unchanged."""
    p = make_fock_problem(nC, nA, nV, Q, seed=seed)
    r = fock.semicanonicalize(p.h, p.Bfull, p.gamma1, p.lambda2, nC, nA, nV)
    U, fs, eps, f = r["U"], r["fs"], r["eps"], r["f"]
    n = nC + nA + nV
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-13
    for lo, hi in ((0, nC), (nC, nC + nA), (nC + nA, n)):
        if hi == lo:
            continue
        blk = fs[lo:hi, lo:hi]
        assert np.abs(blk - np.diag(eps[lo:hi])).max() <= 1e-12 * np.abs(f).max()
        assert abs(np.trace(f[lo:hi, lo:hi]) - eps[lo:hi].sum()) <= 1e-12 * np.abs(f).max()
        off = np.ones((n, n), bool)
        off[lo:hi, lo:hi] = False
        assert np.abs(U[lo:hi][:, off[lo]]).max() == 0.0


def test_transformed_integrals_brute_force():
    """(ia|jb) from the transformed hole x particle factors equals the four-index
    transformation of the explicit integrals with U."""
    nC, nA, nV, Q = 2, 2, 4, 9
    p = make_fock_problem(nC, nA, nV, Q, seed=6)
    r = fock.semicanonicalize(p.h, p.Bfull, p.gamma1, p.lambda2, nC, nA, nV)
    U = r["U"]
    eri = np.einsum("Qpq,Qrs->pqrs", p.Bfull, p.Bfull)
    eri_u = np.einsum("pi,qa,rj,sb,pqrs->iajb", U, U, U, U, eri)
    nH = nC + nA
    lhs = np.einsum("Qia,Qjb->iajb", r["B"], r["B"])
    rhs = eri_u[:nH, nC:, :nH, nC:]
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


@pytest.mark.parametrize("nC,nA,nV,Q,seed", [(2, 2, 4, 9, 7), (3, 3, 3, 8, 8)])
def test_semicanonical_energy_invariant_to_input_rotations(nC, nA, nV, Q, seed):
    """The semicanonical orbitals are fixed by f up to signs (non-degenerate
    spectra): rotating the input orbitals within the core, active and virtual
    spaces (h, B, G, lambda2, lambda3 transformed with them) leaves the orbital
    energies and the DSRG-MRPT2 energy of the semicanonicalised problem
    (with its f^(1) and lambda3) unchanged."""
    p = make_fock_problem(nC, nA, nV, Q, seed=seed, with_lambda3=True)
    rng = np.random.default_rng(seed)
    n = nC + nA + nV
    W = np.zeros((n, n))
    for lo, hi in ((0, nC), (nC, nC + nA), (nC + nA, n)):
        q, _ = np.linalg.qr(rng.standard_normal((hi - lo, hi - lo)))
        W[lo:hi, lo:hi] = q
    WA = W[nC:nC + nA, nC:nC + nA]
    h2 = W.T @ p.h @ W
    B2 = np.einsum("pi,Qpq,qj->Qij", W, p.Bfull, W)
    G2 = WA.T @ p.gamma1 @ WA
    L2 = np.einsum("au,bv,cx,dy,abcd->uvxy", WA, WA, WA, WA, p.lambda2)
    Ws = np.kron(WA, np.eye(2))
    L3 = np.einsum("aU,bV,cW,dX,eY,gZ,abcdeg->UVWXYZ", Ws, Ws, Ws, Ws, Ws, Ws, p.lambda3,
                   optimize="optimal")

    def energy(h, B, G, L, L3_):
        r = fock.semicanonicalize(h, B, G, L, nC, nA, nV, L3_)
        e = dsrg.energy(r["B"], r["eps"], r["gamma1"], r["lambda2"], p.s, nC, nA, nV,
                        lambda3=r["lambda3"], f1=r["f1"])
        return r["eps"], e
    eps1, e1 = energy(p.h, p.Bfull, p.gamma1, p.lambda2, p.lambda3)
    eps2, e2 = energy(h2, B2, G2, L2, L3)
    assert np.abs(eps1 - eps2).max() <= 1e-12
    for k in ("ccvv", "cavv", "ccav", "active", "total"):
        assert abs(e1[k] - e2[k]) <= 1e-11 * max(abs(e1[k]), 1.0), k
