"""Oracle of the generalized Fock build and the semicanonical basis.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy, FP64.

What it computes (Sec. II.B, Eq. (8); Sec. III, steps 2-3 of the procedure):

* the generalized Fock matrix in spin orbitals, f_p^q = h_p^q + sum_{rs}
  v_{pr}^{qs} gamma_s^r, with v_{pr}^{qs} = <pr||qs> and the one-particle
  density of the reference (1 on core spin orbitals, G/2 per spin on the
  active block, 0 on virtuals). For a spin-free density this is the spatial
  matrix f_pq = h_pq + sum_{rs} D_rs [(pq|rs) - 1/2 (ps|rq)], D = 2 on the
  core diagonal and G on the active block; (pq|rs) = sum_Q B^Q_pq B^Q_rs
  (Eq. (19));
* the semicanonical orbitals: the core, active and virtual diagonal blocks of
  f are diagonalised separately, U = blockdiag(U_C, U_A, U_V); the orbital
  energies eps are their eigenvalues (ascending within each block) and the
  off-diagonal blocks of U^T f U form f^(1);
* the inputs of the energy in that basis: the hole x particle block of
  B'^Q = U^T B^Q U, the active density G' = U_A^T G U_A, the cumulant
  L'[u,v,x,y] = sum U_A L U_A U_A U_A over every index, the spin-orbital
  three-body cumulant rotated by U_A on each spatial index, and f^(1) on the
  hole x particle block.

Inputs: h [n, n] (symmetric), Bfull [naux, n, n] (symmetric in the orbital
pair), orbitals ordered [core | active | virtual].
"""
from __future__ import annotations

import numpy as np


def density(ncore: int, nactive: int, nvirt: int, gamma1) -> np.ndarray:
    """Spin-summed one-particle density D over all orbitals (Fig. 1 block structure)."""
    n = ncore + nactive + nvirt
    D = np.zeros((n, n))
    D[np.arange(ncore), np.arange(ncore)] = 2.0
    D[ncore:ncore + nactive, ncore:ncore + nactive] = np.asarray(gamma1, float)
    return D


def fock_spatial(h, Bfull, ncore, nactive, nvirt, gamma1) -> np.ndarray:
    """f_pq = h_pq + sum_rs D_rs [(pq|rs) - 1/2 (ps|rq)] with (pq|rs) from the DF
    factors; D vanishes outside the hole block, so the sums over r, s run over
    the holes only."""
    B = np.asarray(Bfull, float)
    nH = ncore + nactive
    D = density(ncore, nactive, nvirt, gamma1)[:nH, :nH]
    w = np.einsum("Qrs,rs->Q", B[:, :nH, :nH], D)        # sum_rs B^Q_rs D_rs
    J = np.einsum("Qpq,Q->pq", B, w)
    K = np.einsum("Qps,sr,Qrq->pq", B[:, :, :nH], D, B[:, :nH, :], optimize=True)
    return np.asarray(h, float) + J - 0.5 * K


def fock_spin_orbital(h, Bfull, ncore, nactive, nvirt, gamma1) -> np.ndarray:
    """Eq. (8) literally in spin orbitals (spin orbital 2p + sigma), from the
    explicit four-index integrals; tiny inputs only. Returns the spin-orbital
    matrix [2n, 2n]."""
    B = np.asarray(Bfull, float)
    n = B.shape[1]
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)               # (pq|rs)
    sp = np.repeat(np.arange(n), 2)
    sg = np.tile([0, 1], n)
    same = (sg[:, None] == sg[None, :]).astype(float)
    # <PR|QS> = (PQ|RS) d(sP,sQ) d(sR,sS)
    phys = eri[sp][:, sp][:, :, sp][:, :, :, sp].transpose(0, 2, 1, 3)  # [P,R,Q,S] = (pq|rs)
    phys = phys * same[:, None, :, None] * same[None, :, None, :]
    anti = phys - phys.transpose(0, 1, 3, 2)                            # <PR||QS>
    g = np.zeros((2 * n, 2 * n))
    D = density(ncore, nactive, nvirt, gamma1) / 2.0
    g[:, :] = np.kron(D, np.eye(2))                                     # gamma_S^R (symmetric)
    hs = np.kron(np.asarray(h, float), np.eye(2))
    return hs + np.einsum("prqs,rs->pq", anti, g)


def semicanonical_rotation(f, ncore, nactive, nvirt):
    """U = blockdiag(U_C, U_A, U_V) diagonalising the three diagonal blocks of f;
    eps the eigenvalues (ascending per block). Eigenvector signs: the largest
    component of each column is made positive."""
    n = ncore + nactive + nvirt
    U = np.zeros((n, n))
    eps = np.zeros(n)
    for lo, hi in ((0, ncore), (ncore, ncore + nactive), (ncore + nactive, n)):
        if hi == lo:
            continue
        w, V = np.linalg.eigh(f[lo:hi, lo:hi])
        k = np.argmax(np.abs(V), axis=0)
        V = V * np.sign(V[k, np.arange(hi - lo)])[None, :]
        U[lo:hi, lo:hi] = V
        eps[lo:hi] = w
    return U, eps


def semicanonicalize(h, Bfull, gamma1, lambda2, ncore, nactive, nvirt, lambda3=None) -> dict:
    """The energy's inputs in the semicanonical basis (module docstring)."""
    nC, nA, nV = ncore, nactive, nvirt
    f = fock_spatial(h, Bfull, nC, nA, nV, gamma1)
    U, eps = semicanonical_rotation(f, nC, nA, nV)
    B = np.asarray(Bfull, float)
    nH = nC + nA
    # U is block diagonal: the hole rows mix only holes, the particle columns only particles
    Bhp = np.einsum("pi,Qpq,qa->Qia", U[:nH, :nH], B[:, :nH, nC:], U[nC:, nC:], optimize=True)
    fs = U.T @ f @ U
    f1 = fs[:nH, nC:].copy()
    f1[nC:, :nA] = 0.0                                   # the active x active block is diagonal
    UA = U[nC:nH, nC:nH]
    G = UA.T @ np.asarray(gamma1, float) @ UA
    L = np.einsum("au,bv,cx,dy,abcd->uvxy", UA, UA, UA, UA, np.asarray(lambda2, float))
    out = dict(f=f, U=U, eps=eps, B=np.ascontiguousarray(Bhp), f1=f1, gamma1=G, lambda2=L,
               fs=fs)
    if lambda3 is not None:
        # spin-orbital rotation: U_A on the spatial part, identity on spin
        Us = np.kron(UA, np.eye(2))
        out["lambda3"] = np.einsum("aU,bV,cW,dX,eY,gZ,abcdeg->UVWXYZ", Us, Us, Us, Us, Us, Us,
                                   np.asarray(lambda3, float), optimize="optimal")
    return out
