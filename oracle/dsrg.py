"""Tier-1 oracle: the DF/CD DSRG-MRPT2 energy by the paper's algorithm.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain PyTorch CPU
operations in FP64, no blocking beyond what the paper describes; gradients by
autograd on this same code.

Inputs (Sec. II.A, Eq. (19)):
  B        [naux, nH, nP]  hole x particle block of the DF/CD factors B^Q_{pq}
                           (H = core+active, P = active+virtual, in that order)
  eps      [n]             semicanonical orbital energies, [core|active|virtual]
  gamma1   [nA, nA]        spin-summed active 1-RDM G (spin orbital: G/2 per spin)
  lambda2  [nA]^4          L[u,v,x,y] = lambda_{u alpha, v beta}^{x alpha, y beta}
  s        flow parameter (Eh^-2)

Optional inputs:
  lambda3  [2nA]^6         spin-orbital three-body cumulant lam3[U,V,W,X,Y,Z] =
                           lambda_{UVW}^{XYZ} over the active spin orbitals 2u + sigma
                           (terms J and K of Table 1); absent: 0
  f1       [nH, nP]        off-diagonal Fock block f^(1) (Eqs. (12), (14)), spatial,
                           the same for both spins; its active x active entries are
                           not read (they belong to the diagonal block); absent: 0

Blocks reported (Table 2): ``ccvv`` = F1, ``cavv`` = F2, ``ccav`` = F3,
``active`` = A-E + G-K + F4-F8, ``total`` = their sum.

Readings shared with tier 0 (restated here so this file stands alone):
Delta = hole energies minus particle energies; Table 1's ft_j^b is the
Hermitian element ft_b^j; internal (all active) amplitudes are zero; in
Eq. (12) D_u^x = eps_x - eps_u; the regulated denominators use -expm1 and
vanish at D = 0.

Spin adaptation of F1-F3 (closed-shell spin sums of the spin-orbital Table 2
expressions, since every regulator depends only on spatial energies):
  F1 = sum_{mn} sum_{ef} v_ef (2 v_ef - v_fe) (1 - e^{-2 s D^2}) / D,
       v_ef = (me|nf), D = e_m + e_n - e_e - e_f                   (Eq. (23))
  F2 = sum_{m,u,v} G_uv sum_{ef} X_u[e,f] (2 X_v[e,f] - X_v[f,e])
       (1 + e^{-s D_u^2}) (1 - e^{-s D_v^2}) / D_v,
       X_u[e,f] = (me|uf), D_u = e_m + e_u - e_e - e_f
  F3 = sum_{u,v} Hh_uv sum_{m,n,e} Z_v[m,n,e] (2 Z_u[m,n,e] - Z_u[n,m,e])
       (1 + e^{-s D'_v^2}) (1 - e^{-s D'_u^2}) / D'_u,
       Z_u[m,n,e] = (me|nu), D'_u = e_m + e_n - e_e - e_u, Hh = 2 I - G
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def _t(x):
    if isinstance(x, torch.Tensor):
        return x.to(DT)
    return torch.as_tensor(np.asarray(x), dtype=DT)


def reg_t(D, s):
    """(1 - exp(-s D^2)) / D (Eq. (13)). At D == 0 it takes the leading Maclaurin
    term s D of Sec. II.B: the value there is 0, and autograd sees the slope s
    of this analytic function (the quotient form has no derivative at 0)."""
    nz = D != 0
    Ds = torch.where(nz, D, torch.ones_like(D))
    return torch.where(nz, -torch.expm1(-s * D * D) / Ds, s * D)


def reg_v(D, s):
    """1 + exp(-s D^2) (Eq. (15))."""
    return 1.0 + torch.exp(-s * D * D)


def reg_f1(D, s):
    """(1 - exp(-2 s D^2)) / D: the product of Eq. (13) and Eq. (15) (Eq. (23)).
    At D == 0 the leading Maclaurin term 2 s D (value 0, slope 2 s), as in reg_t."""
    nz = D != 0
    Ds = torch.where(nz, D, torch.ones_like(D))
    return torch.where(nz, -torch.expm1(-2.0 * s * D * D) / Ds, 2.0 * s * D)


# --------------------------------------------------------------------------
# F1 (CCVV): outer loop over core pairs (m, n), one DF product per pair, then a
# dot product with the renormalised denominators (Sec. III, Eq. (23)).
# --------------------------------------------------------------------------
def ccvv_pair_energies(B, eps, s, ncore, nactive, nvirt, pairs=None):
    """Pair energies e[m, n] of diagram F1; e.sum() is E_CCVV.

    ``pairs``: optional list of (m, n); only those entries are computed (the
    rest stay 0)."""
    B, eps = _t(B), _t(eps)
    s = _t(s)
    nC, nA = ncore, nactive
    Bcv = B[:, :nC, nA:]                        # [Q, nC, nV]
    eC = eps[:nC]
    eV = eps[nC + nA:]
    A = Bcv.permute(1, 2, 0)                    # [nC, nV, Q]: row m is B[:, m, :]^T
    if pairs is None:
        pairs = [(m, n) for m in range(nC) for n in range(nC)]
    rows = []
    for (m, n) in pairs:
        v = A[m] @ A[n].T                       # v[e, f] = (me|nf)
        D = eC[m] + eC[n] - eV[:, None] - eV[None, :]
        rows.append(((m, n), torch.sum(v * (2.0 * v - v.T) * reg_f1(D, s))))
    e = torch.zeros((nC, nC), dtype=DT)
    for (m, n), val in rows:
        e = e.index_put((torch.tensor([m]), torch.tensor([n])), val.reshape(1))
    return e


def cavv(B, eps, gamma1, s, ncore, nactive, nvirt):
    """Diagram F2 of Table 2 in spin-adapted form (module docstring)."""
    B, eps, G, s = _t(B), _t(eps), _t(gamma1), _t(s)
    nC, nA = ncore, nactive
    if nA == 0 or nC == 0:
        return torch.zeros((), dtype=DT)
    Bc = B[:, :nC, nA:].permute(1, 2, 0)        # [nC, nV, Q]
    Ba = B[:, nC:, nA:].permute(1, 2, 0)        # [nA, nV, Q]
    eC, eA, eV = eps[:nC], eps[nC:nC + nA], eps[nC + nA:]
    tot = torch.zeros((), dtype=DT)
    for m in range(nC):
        X = torch.einsum("eQ,ufQ->uef", Bc[m], Ba)              # X_u[e,f] = (me|uf)
        D = eC[m] + eA[:, None, None] - eV[None, :, None] - eV[None, None, :]
        Rv = reg_v(D, s)                                        # with X_u (vt)
        Rt = reg_t(D, s)                                        # with X_v (t)
        for u in range(nA):
            for v in range(nA):
                tot = tot + G[u, v] * torch.sum(
                    X[u] * (2.0 * X[v] - X[v].T) * Rv[u] * Rt[v])
    return tot


def ccav(B, eps, gamma1, s, ncore, nactive, nvirt):
    """Diagram F3 of Table 2 in spin-adapted form (module docstring)."""
    B, eps, G, s = _t(B), _t(eps), _t(gamma1), _t(s)
    nC, nA = ncore, nactive
    if nA == 0 or nC == 0:
        return torch.zeros((), dtype=DT)
    Hh = 2.0 * torch.eye(nA, dtype=DT) - G
    Bce = B[:, :nC, nA:]                        # [Q, m, e]
    Bcu = B[:, :nC, :nA]                        # [Q, n, u]
    Z = torch.einsum("Qme,Qnu->umne", Bce, Bcu)  # Z_u[m,n,e] = (me|nu)
    eC, eA, eV = eps[:nC], eps[nC:nC + nA], eps[nC + nA:]
    D = (eC[None, :, None, None] + eC[None, None, :, None]
         - eV[None, None, None, :] - eA[:, None, None, None])  # D'_u[m,n,e]
    Rv = reg_v(D, s)
    Rt = reg_t(D, s)
    tot = torch.zeros((), dtype=DT)
    for u in range(nA):
        for v in range(nA):
            tot = tot + Hh[u, v] * torch.sum(
                Z[v] * (2.0 * Z[u] - Z[u].transpose(0, 1)) * Rv[v] * Rt[u])
    return tot


# --------------------------------------------------------------------------
# Active block: Table 1 terms A-E, G-I and Table 2 F4-F8 in spin orbitals, on
# the blocks with at least two active indices (Sec. III, step 6).
# --------------------------------------------------------------------------
class _SpinBlocks:
    """Spin-orbital integrals <ij||ab> (holes first) on three blocks:
    W1 = (H, A | P, A), W2 = (H, H | A, A), W3 = (A, A | P, P), where the
    A entries of a hole slot are active holes and of a particle slot active
    particles. Spin orbital 2p + sigma."""

    def __init__(self, B, eps, s, nC, nA, nV):
        self.nC, self.nA, self.nV = nC, nA, nV
        nH, nP = nC + nA, nA + nV
        self.s = s
        eH = eps[:nH].repeat_interleave(2)
        eP = eps[nC:].repeat_interleave(2)
        self.eH, self.eP = eH, eP
        self.eAh = eH[2 * nC:]                  # active spin orbitals as holes
        self.eAp = eP[: 2 * nA]                 # ... and as particles (same energies)
        sH = torch.arange(2 * nH) % 2
        sP = torch.arange(2 * nP) % 2
        hsp = torch.arange(2 * nH) // 2
        psp = torch.arange(2 * nP) // 2
        self.sH, self.sP, self.hsp, self.psp = sH, sP, hsp, psp
        self.B = B
        aH = torch.arange(2 * nC, 2 * nH)       # active hole spin orbitals (indices into H)
        aP = torch.arange(0, 2 * nA)            # active particle spin orbitals (into P)
        allH = torch.arange(2 * nH)
        allP = torch.arange(2 * nP)
        self.aH, self.aP, self.allH, self.allP = aH, aP, allH, allP
        self.W1 = self._block(allH, aH, allP, aP)
        self.W2 = self._block(allH, allH, aP, aP)
        self.W3 = self._block(aH, aH, allP, allP)

    def _block(self, I, J, A, Bb):
        """<IJ||AB> for spin-orbital index lists I, J (holes) and A, Bb (particles)."""
        Bt = self.B
        hi, hj = self.hsp[I], self.hsp[J]
        pa, pb = self.psp[A], self.psp[Bb]
        # (ia|jb) and (ib|ja) over the spatial orbitals of the lists
        Bia = Bt[:, hi][:, :, pa]               # [Q, I, A]
        Bjb = Bt[:, hj][:, :, pb]               # [Q, J, B]
        Bib = Bt[:, hi][:, :, pb]               # [Q, I, B]
        Bja = Bt[:, hj][:, :, pa]               # [Q, J, A]
        coul = torch.einsum("Qia,Qjb->ijab", Bia, Bjb)
        exch = torch.einsum("Qib,Qja->ijab", Bib, Bja)
        si, sj = self.sH[I], self.sH[J]
        sa, sb = self.sP[A], self.sP[Bb]
        dc = ((si[:, None, None, None] == sa[None, None, :, None])
              & (sj[None, :, None, None] == sb[None, None, None, :])).to(DT)
        dx = ((si[:, None, None, None] == sb[None, None, None, :])
              & (sj[None, :, None, None] == sa[None, None, :, None])).to(DT)
        V = coul * dc - exch * dx
        D = (self.eH[I][:, None, None, None] + self.eH[J][None, :, None, None]
             - self.eP[A][None, None, :, None] - self.eP[Bb][None, None, None, :])
        actI = (I >= 2 * self.nC)
        actJ = (J >= 2 * self.nC)
        actA = (A < 2 * self.nA)
        actB = (Bb < 2 * self.nA)
        internal = (actI[:, None, None, None] & actJ[None, :, None, None]
                    & actA[None, None, :, None] & actB[None, None, None, :])
        T = torch.where(internal, torch.zeros_like(V), V * reg_t(D, self.s))
        Vt = V * reg_v(D, self.s)
        return dict(V=V, T=T, Vt=Vt)


def _lambda_so(L, nA):
    """Spin-orbital cumulant lam[U,V,X,Y] = lambda_{UV}^{XY} from the opposite-spin
    spatial input: same spin L[u,v,x,y] - L[u,v,y,x]; (a b|a b) L[u,v,x,y];
    (b a|b a) L[v,u,y,x]; (a b|b a) -L[u,v,y,x]; (b a|a b) -L[v,u,x,y]."""
    n2 = 2 * nA
    idx = torch.arange(n2)
    sp, sg = idx // 2, idx % 2
    u = sp[:, None, None, None]; su = sg[:, None, None, None]
    v = sp[None, :, None, None]; sv = sg[None, :, None, None]
    x = sp[None, None, :, None]; sx = sg[None, None, :, None]
    y = sp[None, None, None, :]; sy = sg[None, None, None, :]
    same = (su == sv) & (sv == sx) & (sx == sy)
    direct = (~same) & (su == sx) & (sv == sy)
    cross = (~same) & (su == sy) & (sv == sx)
    Luvxy = L[u, v, x, y]
    Luvyx = L[u, v, y, x]
    Lvuyx = L[v, u, y, x]
    Lvuxy = L[v, u, x, y]
    alpha_first = (su == 0)
    lam = torch.zeros((n2,) * 4, dtype=DT)
    lam = lam + torch.where(same, Luvxy - Luvyx, torch.zeros_like(lam))
    lam = lam + torch.where(direct & alpha_first, Luvxy, torch.zeros_like(lam))
    lam = lam + torch.where(direct & ~alpha_first, Lvuyx, torch.zeros_like(lam))
    lam = lam + torch.where(cross & alpha_first, -Luvyx, torch.zeros_like(lam))
    lam = lam + torch.where(cross & ~alpha_first, -Lvuxy, torch.zeros_like(lam))
    return lam


def active_block(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt, return_terms=False,
                 lambda3=None, f1=None):
    """Terms A-E, G-K (Table 1) and F4-F8 (Table 2), spin-orbital."""
    B, eps, G, L, s = _t(B), _t(eps), _t(gamma1), _t(lambda2), _t(s)
    nC, nA, nV = ncore, nactive, nvirt
    if nA == 0:
        # no active orbitals: only term A survives, from f^(1) (gamma = 1 on the
        # core, eta = 1 on the virtuals, the sum over u x of Eq. (12) is empty)
        if f1 is None:
            z = torch.zeros((), dtype=DT)
            return (z, {}) if return_terms else z
        D1 = eps[:nC, None] - eps[None, nC:]
        F = _t(f1)
        termA = 2.0 * torch.sum(F * (1.0 + torch.exp(-s * D1 * D1)) * F * reg_t(D1, s))
        return (termA, {"A": termA}) if return_terms else termA
    sb = _SpinBlocks(B, eps, s, nC, nA, nV)
    nH2, nP2, nA2, nC2 = 2 * (nC + nA), 2 * (nA + nV), 2 * nA, 2 * nC
    gA = torch.kron(G / 2.0, torch.eye(2, dtype=DT))          # gamma on active spin orbitals
    eA = torch.eye(nA2, dtype=DT) - gA                        # eta on active spin orbitals
    lam = _lambda_so(L, nA)
    W1, W2, W3 = sb.W1, sb.W2, sb.W3
    c = slice(0, nC2)                 # core rows of an H axis
    ah = slice(nC2, nH2)              # active rows of an H axis
    ap = slice(0, nA2)                # active rows of a P axis
    vv = slice(nA2, nP2)              # virtual rows of a P axis

    def gam(X, ax):
        """Contract gamma_i^k over a full H axis: core part identity, active part gA."""
        Xc = X.narrow(ax, 0, nC2)
        Xa = torch.movedim(torch.tensordot(gA, torch.movedim(X.narrow(ax, nC2, nA2), ax, 0),
                                           dims=([1], [0])), 0, ax)
        return torch.cat([Xc, Xa], dim=ax)

    def eta(X, ax):
        """Contract eta over a full P axis: active part eA, virtual part identity."""
        Xa = torch.movedim(torch.tensordot(eA, torch.movedim(X.narrow(ax, 0, nA2), ax, 0),
                                           dims=([1], [0])), 0, ax)
        Xv = X.narrow(ax, nA2, nP2 - nA2)
        return torch.cat([Xa, Xv], dim=ax)

    # T1 and ft (Eqs. (12), (14)) from t_{ax}^{iu} = W1.T[i, u, a, x]
    DUX = sb.eAh[None, :] - sb.eAh[:, None]                   # D_u^x = e_x - e_u
    S = torch.einsum("ux,iuax,ux->ia", DUX, W1["T"], gA)
    D1 = sb.eH[:, None] - sb.eP[None, :]
    actI = torch.arange(nH2) >= nC2
    actA = torch.arange(nP2) < nA2
    internal1 = actI[:, None] & actA[None, :]
    if f1 is None:
        F1 = torch.zeros_like(S)
    else:
        same = (sb.sH[:, None] == sb.sP[None, :]).to(DT)
        F1 = _t(f1)[sb.hsp][:, sb.psp] * same
        F1 = torch.where(internal1, torch.zeros_like(F1), F1)
    t1 = torch.where(internal1, torch.zeros_like(S), (F1 + S) * reg_t(D1, s))
    g1 = torch.exp(-s * D1 * D1)
    ft = F1 * (1.0 + g1) + S * g1

    terms = {}
    # A: ft_j^b t_a^i gamma_i^j eta_b^a
    terms["A"] = torch.sum(gam(ft, 0) * eta(t1, 1))
    # B: 1/2 vt_{xy}^{ev} t_e^u lambda_{uv}^{xy}      [W3: x,y | e in V, v in A]
    terms["B"] = 0.5 * torch.einsum("xyev,ue,uvxy->", W3["Vt"][:, :, vv, ap], t1[ah, vv], lam)
    # C: -1/2 vt_{my}^{uv} t_x^m lambda_{uv}^{xy}     [W1: m in C, y | u in A, v]
    terms["C"] = -0.5 * torch.einsum("myuv,mx,uvxy->", W1["Vt"][c, :, ap, :], t1[c, ap], lam)
    # D: 1/2 ft_x^e t_{ey}^{uv} lambda_{uv}^{xy}      [W3: u,v | e in V, y in A]
    terms["D"] = 0.5 * torch.einsum("xe,uvey,uvxy->", ft[ah, vv], W3["T"][:, :, vv, ap], lam)
    # E: -1/2 ft_m^v t_{xy}^{um} lambda_{uv}^{xy}     [W2: u in A, m in C | x, y]
    terms["E"] = -0.5 * torch.einsum("mv,umxy,uvxy->", ft[c, ap], W2["T"][ah, c], lam)
    # G: 1/8 vt_{xy}^{cd} t_{ab}^{uv} eta_c^a eta_d^b lambda_{uv}^{xy}   [W3]
    Tg = eta(eta(W3["T"], 2), 3)
    terms["G"] = 0.125 * torch.einsum("xycd,uvcd,uvxy->", W3["Vt"], Tg, lam)
    # H: 1/8 vt_{kl}^{uv} t_{xy}^{ij} gamma_i^k gamma_j^l lambda_{uv}^{xy}   [W2]
    Th = gam(gam(W2["T"], 0), 1)
    terms["H"] = 0.125 * torch.einsum("kluv,klxy,uvxy->", W2["Vt"], Th, lam)
    # I: vt_{jx}^{bu} t_{ay}^{iv} gamma_i^j eta_b^a lambda_{uv}^{xy}   [W1 both]
    Ti = eta(gam(W1["T"], 0), 2)                              # [j, v, b, y]
    terms["I"] = torch.einsum("jxbu,jvby,uvxy->", W1["Vt"], Ti, lam)
    # F4: 1/4 vt_{xu}^{ef} t_{ef}^{yv} gamma_y^x gamma_v^u      [W3: V V]
    terms["F4"] = 0.25 * torch.einsum("xuef,yvef,xy,uv->", W3["Vt"][:, :, vv, vv],
                                      W3["T"][:, :, vv, vv], gA, gA)
    # F5: 1/4 vt_{mn}^{vy} t_{ux}^{mn} eta_v^u eta_y^x          [W2: C C]
    terms["F5"] = 0.25 * torch.einsum("mnvy,mnux,uv,xy->", W2["Vt"][c, c], W2["T"][c, c], eA, eA)
    # F6: vt_{mx}^{ve} t_{ue}^{my} gamma_y^x eta_v^u   [W1 (C,A|V,A) with particles swapped]
    V6 = W1["Vt"][c, :, vv, :]                                # [m, x, e, v] = -vt_{mx}^{ve}
    T6 = W1["T"][c, :, vv, :]                                 # [m, y, e, u] = -t_{ue}^{my}
    terms["F6"] = torch.einsum("mxev,myeu,xy,uv->", V6, T6, gA, eA)
    # F7: 1/2 vt_{yz}^{ve} t_{ue}^{wx} gamma_w^y gamma_x^z eta_v^u   [W3: A V]
    terms["F7"] = 0.5 * torch.einsum("yzve,wxue,yw,zx,uv->", W3["Vt"][:, :, ap, vv],
                                     W3["T"][:, :, ap, vv], gA, gA, eA)
    # F8: 1/2 vt_{mw}^{vy} t_{ux}^{mz} gamma_z^w eta_v^u eta_y^x   [W1: m in C | A A]
    terms["F8"] = 0.5 * torch.einsum("mwvy,mzux,wz,uv,xy->", W1["Vt"][c, :, ap, :],
                                     W1["T"][c, :, ap, :], gA, eA, eA)
    if lambda3 is not None:
        l3 = _t(lambda3)
        # J: 1/4 vt_{mz}^{uv} t_{xy}^{mw} lambda_{uvw}^{xyz}   [W1: m in C, z | u in A, v]
        terms["J"] = 0.25 * torch.einsum("mzuv,mwxy,uvwxyz->", W1["Vt"][c, :, ap, :],
                                         W1["T"][c, :, ap, :], l3)
        # K: 1/4 vt_{xy}^{we} t_{ez}^{uv} lambda_{uvw}^{xyz}   [W3: w in A, e in V]
        terms["K"] = 0.25 * torch.einsum("xywe,uvez,uvwxyz->", W3["Vt"][:, :, ap, vv],
                                         W3["T"][:, :, vv, ap], l3)
    tot = sum(terms.values())
    return (tot, terms) if return_terms else tot


def energy(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt, with_pairs=False,
           with_terms=False, lambda3=None, f1=None) -> dict:
    """All four blocks and the total, as Python floats (pair energies as numpy)."""
    with torch.no_grad():
        e = ccvv_pair_energies(B, eps, s, ncore, nactive, nvirt)
        f2 = cavv(B, eps, gamma1, s, ncore, nactive, nvirt)
        f3 = ccav(B, eps, gamma1, s, ncore, nactive, nvirt)
        act, terms = active_block(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt,
                                  return_terms=True, lambda3=lambda3, f1=f1)
    out = dict(ccvv=float(e.sum()), cavv=float(f2), ccav=float(f3), active=float(act))
    out["total"] = out["ccvv"] + out["cavv"] + out["ccav"] + out["active"]
    if with_pairs:
        out["pairs"] = e.numpy()
    if with_terms:
        out["terms"] = {k: float(v) for k, v in terms.items()}
    return out


def energy_and_grad(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt, lambda3=None,
                    f1=None) -> dict:
    """Energy blocks plus dE_total/dB, dE_total/deps and dE_total/ds by autograd."""
    Bt = _t(B).clone().requires_grad_(True)
    et = _t(eps).clone().requires_grad_(True)
    st = _t(s).clone().requires_grad_(True)
    e = ccvv_pair_energies(Bt, et, st, ncore, nactive, nvirt).sum()
    f2 = cavv(Bt, et, gamma1, st, ncore, nactive, nvirt)
    f3 = ccav(Bt, et, gamma1, st, ncore, nactive, nvirt)
    act = active_block(Bt, et, gamma1, lambda2, st, ncore, nactive, nvirt, lambda3=lambda3, f1=f1)
    tot = e + f2 + f3 + act
    dB, de, ds = torch.autograd.grad(tot, (Bt, et, st))
    return dict(ccvv=float(e.detach()), cavv=float(f2.detach()), ccav=float(f3.detach()),
                active=float(act.detach()), total=float(tot.detach()), dB=dB.numpy(),
                deps=de.numpy(), ds=float(ds))


def block_grads(B, eps, gamma1, lambda2, s, ncore, nactive, nvirt) -> dict:
    """Per-block gradients (dB, deps, ds) for each of ccvv, cavv, ccav, active."""
    out = {}
    fns = {
        "ccvv": lambda Bt, et, st: ccvv_pair_energies(Bt, et, st, ncore, nactive, nvirt).sum(),
        "cavv": lambda Bt, et, st: cavv(Bt, et, gamma1, st, ncore, nactive, nvirt),
        "ccav": lambda Bt, et, st: ccav(Bt, et, gamma1, st, ncore, nactive, nvirt),
        "active": lambda Bt, et, st: active_block(Bt, et, gamma1, lambda2, st, ncore, nactive,
                                                  nvirt),
    }
    for k, fn in fns.items():
        Bt = _t(B).clone().requires_grad_(True)
        et = _t(eps).clone().requires_grad_(True)
        st = _t(s).clone().requires_grad_(True)
        val = fn(Bt, et, st)
        if not val.requires_grad:
            out[k] = dict(value=float(val), dB=np.zeros(Bt.shape), deps=np.zeros(et.shape), ds=0.0)
            continue
        dB, de, ds = torch.autograd.grad(val, (Bt, et, st), allow_unused=True)
        out[k] = dict(value=float(val),
                      dB=np.zeros(Bt.shape) if dB is None else dB.numpy(),
                      deps=np.zeros(et.shape) if de is None else de.numpy(),
                      ds=0.0 if ds is None else float(ds))
    return out
