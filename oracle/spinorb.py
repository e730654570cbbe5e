"""Tier-0 oracle: the DSRG-MRPT2 energy of Table 1, literally, in spin orbitals.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy, FP64,
dense tensors over the full spin-orbital hole space H = C+A and particle
space P = A+V. Meant for tiny inputs (a few orbitals per space).

Conventions (Sec. II):
* spin orbital ``2*p + sigma`` for spatial orbital ``p`` of a space, sigma in
  {0 (alpha), 1 (beta)};
* ``V[i, j, a, b] = <ij||ab> = (ia|jb) d(si,sa) d(sj,sb) - (ib|ja) d(si,sb) d(sj,sa)``
  with ``(ia|jb) = sum_Q B[Q,i,a] B[Q,j,b]`` (Eq. (19)); holes first, so this
  array stands for both v_{ij}^{ab} and v_{ab}^{ij} (real orbitals);
* Delta = (sum of hole energies) - (sum of particle energies) (Sec. II.B);
* T2 amplitude, Eq. (13): ``t_{ab}^{ij} = v (1 - exp(-s D^2)) / D``, zero when
  all four indices are active (internal amplitudes are excluded, Sec. II.A);
* modified integrals, Eq. (15): ``vt = v (1 + exp(-s D^2))``;
* T1 amplitude, Eq. (12):
  ``t_a^i = [f_a^i + sum_{ux} D_u^x t_{ax}^{iu} gamma_u^x] (1 - exp(-s D_a^i^2)) / D_a^i``
  with ``D_u^x = eps_x - eps_u``; zero when i and a are both active. The
  off-diagonal Fock block f^(1) is an optional spatial input ``f1[i, a]``
  (hole i, particle a; the same for both spins, none between spins; its
  active x active entries belong to the diagonal block F^(0) and are not
  read); absent, it is 0;
* modified Fock, Eq. (14): ``ft_a^i = f_a^i (1 + exp(-s D_a^i^2)) + [sum ...] exp(-s D_a^i^2)``;
  Table 1's ``ft_j^b`` is read as the same (Hermitian) element ``ft_b^j``;
* densities (Fig. 1): gamma = 1 on core, G/2 per spin on the active block
  (G = spin-summed input), 0 on virtuals; eta = 1 - gamma;
* cumulant: input ``L[u,v,x,y] = lambda_{u a, v b}^{x a, y b}`` (alpha, beta);
  same-spin blocks ``L[u,v,x,y] - L[u,v,y,x]``; the other opposite-spin
  orderings follow from antisymmetry;
* three-body cumulant (terms J and K): optional spin-orbital input
  ``lam3[U,V,W,X,Y,Z] = lambda_{UVW}^{XYZ}`` over the active spin orbitals
  (index ``2u + sigma``); absent, it is 0 and so are J and K.
* the regulated denominators use ``-expm1(-x)`` for ``1 - exp(-x)`` and are 0
  when D == 0 (the limit of Sec. II.B's Maclaurin expansion).
"""
from __future__ import annotations

import numpy as np


def _reg_t(D, s):
    """(1 - exp(-s D^2)) / D, with the D -> 0 limit 0."""
    out = np.zeros_like(D)
    nz = D != 0
    out[nz] = -np.expm1(-s * D[nz] ** 2) / D[nz]
    return out


class SpinOrbitalSystem:
    """Spin-orbital tensors over the full hole and particle spaces."""

    def __init__(self, B, eps, gamma1, lambda2, s, ncore, nactive, nvirt, lambda3=None, f1=None):
        nC, nA, nV = ncore, nactive, nvirt
        nH, nP = nC + nA, nA + nV
        B = np.asarray(B, dtype=float)
        assert B.shape[1:] == (nH, nP)
        self.nC, self.nA, self.nV, self.s = nC, nA, nV, float(s)
        self.nH2, self.nP2, self.nA2 = 2 * nH, 2 * nP, 2 * nA
        eps = np.asarray(eps, dtype=float)
        eH = eps[:nH]
        eP = eps[nC:]
        # spin-orbital energies and spins
        self.eH = np.repeat(eH, 2)
        self.eP = np.repeat(eP, 2)
        sH = np.tile([0, 1], nH)
        sP = np.tile([0, 1], nP)
        hsp = np.repeat(np.arange(nH), 2)   # spatial index of each hole spin orbital
        psp = np.repeat(np.arange(nP), 2)
        # active flags
        self.actH = np.repeat(np.arange(nH) >= nC, 2)
        self.actP = np.repeat(np.arange(nP) < nA, 2)

        # chemist integrals (ia|jb) over spatial hole/particle orbitals
        K = np.einsum("Qia,Qjb->iajb", B, B)
        Ks = K[hsp][:, psp][:, :, hsp][:, :, :, psp]          # [I, A, J, B]
        d = lambda x, y: (x[:, None] == y[None, :]).astype(float)
        dHP = d(sH, sP)                                      # [I, A]
        # <IJ|AB> = (IA|JB) d(sI,sA) d(sJ,sB)
        coul = np.einsum("iajb,ia,jb->ijab", Ks, dHP, dHP)
        self.V = coul - coul.transpose(0, 1, 3, 2)            # antisymmetrise in a,b

        D2 = (self.eH[:, None, None, None] + self.eH[None, :, None, None]
              - self.eP[None, None, :, None] - self.eP[None, None, None, :])
        internal = (self.actH[:, None, None, None] & self.actH[None, :, None, None]
                    & self.actP[None, None, :, None] & self.actP[None, None, None, :])
        self.D2 = D2
        self.T2 = self.V * _reg_t(D2, self.s)
        self.T2[internal] = 0.0
        self.Vt = self.V * (1.0 + np.exp(-self.s * D2 ** 2))

        # densities
        G = np.asarray(gamma1, dtype=float)
        gH = np.zeros((self.nH2, self.nH2))
        gH[: 2 * nC, : 2 * nC] = np.eye(2 * nC)
        gA = np.kron(G / 2.0, np.eye(2))                      # spin orbital active block
        gH[2 * nC:, 2 * nC:] = gA
        eP_ = np.eye(self.nP2)
        eP_[: 2 * nA, : 2 * nA] = np.eye(2 * nA) - gA
        self.gamma = gH                                       # gamma[k, i] = gamma_i^k
        self.eta = eP_                                        # eta[a, c] = eta_c^a
        self.gA = gA
        self.lam = self._lambda_so(np.asarray(lambda2, dtype=float), nA)

        # T1 and modified Fock (f^(1) read as 0)
        D1 = self.eH[:, None] - self.eP[None, :]
        # index maps of the active spin orbitals inside H and P
        aH = np.arange(2 * nC, self.nH2)
        aP = np.arange(0, 2 * nA)
        eA = self.eH[aH]
        DUX = eA[None, :] - eA[:, None]                      # DUX[u, x] = eps_x - eps_u
        # sum_{ux} D_u^x t_{ax}^{iu} gamma_u^x ; t_{ax}^{iu} = T2[i, u, a, x]
        T2_iuax = self.T2[:, aH][:, :, :, aP]                 # [i, u, a, x]
        S = np.einsum("ux,iuax,ux->ia", DUX, T2_iuax, gA)
        internal1 = self.actH[:, None] & self.actP[None, :]
        F1 = np.zeros_like(S)
        if f1 is not None:
            F1 = np.asarray(f1, dtype=float)[hsp][:, psp] * (sH[:, None] == sP[None, :])
            F1[internal1] = 0.0
        self.F1 = F1
        self.T1 = (F1 + S) * _reg_t(D1, self.s)
        self.T1[internal1] = 0.0
        g1 = np.exp(-self.s * D1 ** 2)
        self.Ft = F1 * (1.0 + g1) + S * g1
        self.lam3 = None if lambda3 is None else np.asarray(lambda3, dtype=float)

    @staticmethod
    def _lambda_so(L, nA):
        """Spin-orbital cumulant lam[u, v, x, y] = lambda_{uv}^{xy} over active spin orbitals."""
        n2 = 2 * nA
        lam = np.zeros((n2,) * 4)
        for U in range(n2):
            for V in range(n2):
                for X in range(n2):
                    for Y in range(n2):
                        u, su = divmod(U, 2)
                        v, sv = divmod(V, 2)
                        x, sx = divmod(X, 2)
                        y, sy = divmod(Y, 2)
                        if su == sv == sx == sy:
                            val = L[u, v, x, y] - L[u, v, y, x]
                        elif su == sx and sv == sy:           # (a b | a b) or (b a | b a)
                            val = L[u, v, x, y] if su == 0 else L[v, u, y, x]
                        elif su == sy and sv == sx:           # (a b | b a) or (b a | a b)
                            val = -L[u, v, y, x] if su == 0 else -L[v, u, x, y]
                        else:
                            val = 0.0
                        lam[U, V, X, Y] = val
        return lam

    # ----- Table 1 (Sec. II.B), every term over the full H and P spaces -----
    def terms(self) -> dict:
        nC2, nA2 = 2 * self.nC, 2 * self.nA
        g, et, lam = self.gamma, self.eta, self.lam
        V, Vt, T = self.V, self.Vt, self.T2
        aH = slice(nC2, self.nH2)       # active holes
        aP = slice(0, nA2)              # active particles
        cH = slice(0, nC2)              # core
        vP = slice(nA2, self.nP2)       # virtuals
        t1, ft = self.T1, self.Ft
        out = {}
        # A: + ft_j^b t_a^i gamma_i^j eta_b^a
        out["A"] = np.einsum("jb,ia,ji,ab->", ft, t1, g, et)
        # B: + 1/2 vt_{xy}^{ev} t_e^u lambda_{uv}^{xy}
        out["B"] = 0.5 * np.einsum("xyev,ue,uvxy->", Vt[aH, aH, vP, aP], t1[aH, vP], lam)
        # C: - 1/2 vt_{my}^{uv} t_x^m lambda_{uv}^{xy}
        out["C"] = -0.5 * np.einsum("myuv,mx,uvxy->", Vt[cH, aH, aP, aP], t1[cH, aP], lam)
        # D: + 1/2 ft_x^e t_{ey}^{uv} lambda_{uv}^{xy}
        out["D"] = 0.5 * np.einsum("xe,uvey,uvxy->", ft[aH, vP], T[aH, aH, vP, aP], lam)
        # E: - 1/2 ft_m^v t_{xy}^{um} lambda_{uv}^{xy}
        out["E"] = -0.5 * np.einsum("mv,umxy,uvxy->", ft[cH, aP], T[aH, cH, aP, aP], lam)
        # F: + 1/4 vt_{kl}^{cd} t_{ab}^{ij} gamma_i^k gamma_j^l eta_c^a eta_d^b
        out["F"] = 0.25 * np.einsum("klcd,ijab,ki,lj,ac,bd->", Vt, T, g, g, et, et,
                                    optimize="optimal")
        # G: + 1/8 vt_{xy}^{cd} t_{ab}^{uv} eta_c^a eta_d^b lambda_{uv}^{xy}
        out["G"] = 0.125 * np.einsum("xycd,uvab,ac,bd,uvxy->", Vt[aH, aH], T[aH, aH], et, et,
                                     lam, optimize="optimal")
        # H: + 1/8 vt_{kl}^{uv} t_{xy}^{ij} gamma_i^k gamma_j^l lambda_{uv}^{xy}
        out["H"] = 0.125 * np.einsum("kluv,ijxy,ki,lj,uvxy->", Vt[:, :, aP, aP], T[:, :, aP, aP],
                                     g, g, lam, optimize="optimal")
        # I: + vt_{jx}^{bu} t_{ay}^{iv} gamma_i^j eta_b^a lambda_{uv}^{xy}
        out["I"] = np.einsum("jxbu,ivay,ji,ab,uvxy->", Vt[:, aH, :, aP], T[:, aH, :, aP],
                             g, et, lam, optimize="optimal")
        # J: + 1/4 vt_{mz}^{uv} t_{xy}^{mw} lambda_{uvw}^{xyz}
        # K: + 1/4 vt_{xy}^{we} t_{ez}^{uv} lambda_{uvw}^{xyz}
        if self.lam3 is None:
            out["J"] = 0.0
            out["K"] = 0.0
        else:
            l3 = self.lam3
            out["J"] = 0.25 * np.einsum("mzuv,mwxy,uvwxyz->", Vt[cH, aH, aP, aP],
                                        T[cH, aH, aP, aP], l3, optimize="optimal")
            out["K"] = 0.25 * np.einsum("xywe,uvez,uvwxyz->", Vt[aH, aH, aP, vP],
                                        T[aH, aH, vP, aP], l3, optimize="optimal")
        return out

    # ----- Table 2: the eight pieces of term F -----
    def f_pieces(self) -> dict:
        nC2, nA2 = 2 * self.nC, 2 * self.nA
        Vt, T = self.Vt, self.T2
        gA = self.gA
        eA = np.eye(nA2) - gA
        c = slice(0, nC2)
        aH = slice(nC2, self.nH2)
        aP = slice(0, nA2)
        v = slice(nA2, self.nP2)
        out = {}
        out["F1"] = 0.25 * np.einsum("mnef,mnef->", Vt[c, c, v, v], T[c, c, v, v])
        out["F2"] = 0.5 * np.einsum("muef,mvef,uv->", Vt[c, aH, v, v], T[c, aH, v, v], gA)
        out["F3"] = 0.5 * np.einsum("mnev,mneu,uv->", Vt[c, c, v, aP], T[c, c, v, aP], eA)
        out["F4"] = 0.25 * np.einsum("xuef,yvef,xy,uv->", Vt[aH, aH, v, v], T[aH, aH, v, v],
                                     gA, gA)
        out["F5"] = 0.25 * np.einsum("mnvy,mnux,uv,xy->", Vt[c, c, aP, aP], T[c, c, aP, aP],
                                     eA, eA)
        out["F6"] = np.einsum("mxve,myue,xy,uv->", Vt[c, aH, aP, v], T[c, aH, aP, v], gA, eA)
        out["F7"] = 0.5 * np.einsum("yzve,wxue,yw,zx,uv->", Vt[aH, aH, aP, v], T[aH, aH, aP, v],
                                    gA, gA, eA)
        out["F8"] = 0.5 * np.einsum("mwvy,mzux,wz,uv,xy->", Vt[c, aH, aP, aP], T[c, aH, aP, aP],
                                    gA, eA, eA)
        return out


def energy(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt, lambda3=None, f1=None) -> dict:
    """Literal Table 1 energy and its Table 2 split.

    Returns the terms A-K, F1-F8, and the four reported blocks: ``ccvv`` = F1,
    ``cavv`` = F2, ``ccav`` = F3, ``active`` = everything else (total minus
    F1-F3), plus ``total``.
    """
    so = SpinOrbitalSystem(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt, lambda3, f1)
    t = so.terms()
    f = so.f_pieces()
    total = sum(t.values())
    res = dict(t)
    res.update(f)
    res["total"] = total
    res["ccvv"] = f["F1"]
    res["cavv"] = f["F2"]
    res["ccav"] = f["F3"]
    res["active"] = total - f["F1"] - f["F2"] - f["F3"]
    return res


def mp2_spin_orbital(B, eps, ncore, nvirt, nactive=0):
    """Textbook spin-orbital MP2 correlation energy over core -> virtual:
    1/4 sum |<mn||ef>|^2 / (e_m + e_n - e_e - e_f), built from explicit
    antisymmetrised spin-orbital integrals (no spin summation)."""
    nC, nV, nA = ncore, nvirt, nactive
    B = np.asarray(B, float)
    Bcv = B[:, :nC, nA:]
    eC = np.repeat(np.asarray(eps)[:nC], 2)
    eV = np.repeat(np.asarray(eps)[nC + nA:], 2)
    K = np.einsum("Qme,Qnf->menf", Bcv, Bcv)
    hs = np.repeat(np.arange(nC), 2)
    ps = np.repeat(np.arange(nV), 2)
    sh = np.tile([0, 1], nC)
    sp = np.tile([0, 1], nV)
    Ks = K[hs][:, ps][:, :, hs][:, :, :, ps]
    dd = (sh[:, None] == sp[None, :]).astype(float)
    coul = np.einsum("menf,me,nf->mnef", Ks, dd, dd)
    anti = coul - coul.transpose(0, 1, 3, 2)
    D = eC[:, None, None, None] + eC[None, :, None, None] - eV[None, None, :, None] - eV[None, None, None, :]
    return 0.25 * np.sum(anti ** 2 / D)
