"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows. None of them re-types the oracle's
own formula: the comparisons are between the two oracle tiers (literal
spin-orbital Table 1 vs the spin-adapted pair-loop algorithm), against a
textbook limit, against exact invariances, or against a brute-force
second-quantised wavefunction.
"""
import itertools

import numpy as np
import pytest
import torch

from dsrg_synth import make_problem
from oracle import dsrg, spinorb

BLOCKS = ["ccvv", "cavv", "ccav", "active", "total"]


def _args(p):
    return (p.B, p.eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt)


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


TINY = [(3, 2, 4, 9, 0.37, 0), (2, 3, 3, 7, 0.8, 1), (3, 1, 5, 11, 0.1, 2), (1, 2, 2, 5, 1.3, 3)]


def _extra(p):
    return dict(lambda3=p.lambda3, f1=p.f1)


@pytest.mark.parametrize("extra", [False, True], ids=["lam2", "lam3_f1"])
@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", TINY)
def test_tiers_agree_per_block(nC, nA, nV, Q, s, seed, extra):
    """Table 1 (literal, spin orbitals) == tier-1 (Table 2 split, Eq. (23) pair
    loop, spin-adapted F1-F3), for every block and the total, lambda2 != 0;
    with the three-body cumulant (terms J, K) and the off-diagonal Fock block
    f^(1) (Eqs. (12), (14)) as well."""
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed, with_lambda3=extra, with_f1=extra)
    r0 = spinorb.energy(*_args(p), **_extra(p))
    r1 = dsrg.energy(*_args(p), with_terms=True, **_extra(p))
    for k in BLOCKS:
        assert _rel(r0[k], r1[k]) < 1e-12, (k, r0[k], r1[k])
    for k, v in r1["terms"].items():
        assert abs(v - r0[k]) <= 1e-12 * max(1.0, abs(r0[k])), k
    if extra and nA >= 2:
        assert r0["J"] != 0.0 and r0["K"] != 0.0


@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", TINY)
def test_table2_splits_term_F(nC, nA, nV, Q, s, seed):
    """Table 2: F1 + ... + F8 equals the eight-index term F of Eq. (22)."""
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed)
    r0 = spinorb.energy(*_args(p))
    fs = sum(r0["F%d" % i] for i in range(1, 9))
    assert _rel(r0["F"], fs) < 1e-12


def test_large_s_limit_is_df_mp2():
    """s -> infinity removes the regulator (Sec. II.B): F1 becomes the
    spin-orbital MP2 energy 1/4 sum |<mn||ef>|^2 / D (textbook MP2)."""
    p = make_problem(4, 2, 7, 13, s=1.0e6, seed=5)
    e1 = dsrg.energy(*_args(p))["ccvv"]
    mp2 = spinorb.mp2_spin_orbital(p.B, p.eps, p.ncore, p.nvirt, p.nactive)
    assert _rel(e1, mp2) < 1e-12


def test_s_zero_gives_zero_energy():
    """Every amplitude carries 1 - exp(-s D^2) (Eqs. (12), (13)): E(s=0) = 0 exactly."""
    p = make_problem(3, 2, 5, 9, s=0.0, seed=4)
    r1 = dsrg.energy(*_args(p))
    r0 = spinorb.energy(*_args(p))
    for k in BLOCKS:
        assert r1[k] == 0.0 and r0[k] == 0.0, k


def test_small_s_slope_of_ccvv():
    """Maclaurin form of Sec. II.B: t = v (s D + O(s^{3/2} D^3)) and vt -> 2v, so
    dF1/ds at s = 0 is 1/4 sum |<mn||ef>|^2 2D, taken here from the literal
    spin-orbital tensors; the oracle side is autograd of the pair loop."""
    p = make_problem(3, 1, 5, 8, s=0.0, seed=6)
    so = spinorb.SpinOrbitalSystem(*_args(p))
    c = slice(0, 2 * p.ncore)
    v = slice(2 * p.nactive, 2 * (p.nactive + p.nvirt))
    V = so.V[c, c, v, v]
    D = so.D2[c, c, v, v]
    slope = 0.25 * np.sum(V ** 2 * 2.0 * D)
    st = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    e = dsrg.ccvv_pair_energies(p.B, p.eps, st, p.ncore, p.nactive, p.nvirt).sum()
    (g,) = torch.autograd.grad(e, st)
    assert _rel(float(g), slope) < 1e-12


def test_pair_symmetry():
    """Pair energies of Eq. (23) are symmetric: e_mn = e_nm."""
    p = make_problem(6, 2, 9, 15, s=0.5, seed=7)
    e = dsrg.energy(*_args(p), with_pairs=True)["pairs"]
    assert np.max(np.abs(e - e.T)) <= 1e-14 * np.max(np.abs(e))


@pytest.mark.parametrize("occ", ["full", "empty"])
def test_one_determinant_limits(occ):
    """Fig. 1 block structure: with lambda2 = 0, a doubly occupied active space
    (G = 2I) behaves as core, an empty one (G = 0) as virtual. Then T1 = 0
    (Eq. (12): sum_u D_u^u = 0 or gamma = 0) and the whole energy is the F1
    formula on the enlarged core (or virtual) space."""
    p = make_problem(3, 2, 4, 10, s=0.6, seed=8, occupation=occ)
    p.lambda2[...] = 0.0
    r1 = dsrg.energy(*_args(p))
    r0 = spinorb.energy(*_args(p))
    nC, nA, nV = p.ncore, p.nactive, p.nvirt
    if occ == "full":
        Bp = p.B[:, :, nA:]                       # holes C+A, particles V
        ref = dsrg.energy(Bp, p.eps, np.zeros((0, 0)), np.zeros((0,) * 4), p.s, nC + nA, 0, nV)
    else:
        Bp = p.B[:, :nC, :]                       # holes C, particles A+V
        ref = dsrg.energy(Bp, p.eps, np.zeros((0, 0)), np.zeros((0,) * 4), p.s, nC, 0, nA + nV)
    assert ref["total"] == ref["ccvv"]
    assert _rel(r1["total"], ref["ccvv"]) < 1e-12
    assert _rel(r0["total"], ref["ccvv"]) < 1e-12


def test_size_consistency():
    """Size consistency (Sec. I): two non-interacting fragments (disjoint
    auxiliary sets, block-diagonal densities, separable cumulant) give
    E(A+B) = E(A) + E(B) for every block."""
    pa = make_problem(2, 2, 3, 6, s=0.5, seed=11)
    pb = make_problem(2, 1, 4, 5, s=0.5, seed=12)
    nC = pa.ncore + pb.ncore
    nA = pa.nactive + pb.nactive
    nV = pa.nvirt + pb.nvirt
    Q = pa.naux + pb.naux
    # orbital maps into the combined [core | active | virtual] order
    hA = list(range(pa.ncore)) + [nC + u for u in range(pa.nactive)]
    hB = list(range(pa.ncore, nC)) + [nC + pa.nactive + u for u in range(pb.nactive)]
    pA = list(range(pa.nactive)) + [nA + e for e in range(pa.nvirt)]
    pB = [pa.nactive + u for u in range(pb.nactive)] + [nA + pa.nvirt + e for e in range(pb.nvirt)]
    B = np.zeros((Q, nC + nA, nA + nV))
    B[np.ix_(range(pa.naux), hA, pA)] = pa.B
    B[np.ix_(range(pa.naux, Q), hB, pB)] = pb.B
    eps = np.zeros(nC + nA + nV)
    eps[hA] = pa.eps[: pa.nhole]
    eps[hB] = pb.eps[: pb.nhole]
    eps[[nC + x for x in pA]] = pa.eps[pa.ncore:]
    eps[[nC + x for x in pB]] = pb.eps[pb.ncore:]
    G = np.zeros((nA, nA))
    G[: pa.nactive, : pa.nactive] = pa.gamma1
    G[pa.nactive:, pa.nactive:] = pb.gamma1
    L = np.zeros((nA,) * 4)
    a, b = slice(0, pa.nactive), slice(pa.nactive, nA)
    L[a, a, a, a] = pa.lambda2
    L[b, b, b, b] = pb.lambda2
    rab = dsrg.energy(B, eps, G, L, 0.5, nC, nA, nV)
    ra = dsrg.energy(*_args(pa))
    rb = dsrg.energy(*_args(pb))
    for k in BLOCKS:
        assert abs(rab[k] - ra[k] - rb[k]) <= 1e-12 * max(1.0, abs(rab[k])), k
    r0 = spinorb.energy(B, eps, G, L, 0.5, nC, nA, nV)
    assert _rel(r0["total"], ra["total"] + rb["total"]) < 1e-12
    # with three-body cumulants and off-diagonal Fock blocks of each fragment
    # (nothing between the fragments)
    pa = make_problem(2, 2, 3, 6, s=0.5, seed=11, with_lambda3=True, with_f1=True)
    pb = make_problem(2, 1, 4, 5, s=0.5, seed=12, with_lambda3=True, with_f1=True)
    F = np.zeros((nC + nA, nA + nV))
    F[np.ix_(hA, pA)] = pa.f1
    F[np.ix_(hB, pB)] = pb.f1
    soA = [2 * u + sg for u in range(pa.nactive) for sg in (0, 1)]
    soB = [2 * (pa.nactive + u) + sg for u in range(pb.nactive) for sg in (0, 1)]
    L3 = np.zeros((2 * nA,) * 6)
    L3[np.ix_(soA, soA, soA, soA, soA, soA)] = pa.lambda3
    L3[np.ix_(soB, soB, soB, soB, soB, soB)] = pb.lambda3
    rab = dsrg.energy(B, eps, G, L, 0.5, nC, nA, nV, lambda3=L3, f1=F)
    ra = dsrg.energy(*_args(pa), **_extra(pa))
    rb = dsrg.energy(*_args(pb), **_extra(pb))
    for k in BLOCKS:
        assert abs(rab[k] - ra[k] - rb[k]) <= 1e-12 * max(1.0, abs(rab[k])), k
    r0 = spinorb.energy(B, eps, G, L, 0.5, nC, nA, nV, lambda3=L3, f1=F)
    assert _rel(r0["total"], ra["total"] + rb["total"]) < 1e-12


@pytest.mark.parametrize("spectrum,seed", [("overlap", 20), ("degenerate", 21), ("negative", 22)])
def test_tiers_agree_on_unusual_spectra(spectrum, seed):
    """Neither Table 1 nor Table 2 assumes an order of the orbital energies or a
    sign of the denominators: with virtual energies below core and active ones
    (denominators of both signs, unsorted blocks), with exactly zero
    denominators, and with every virtual energy negative, the literal
    spin-orbital tier and the pair-loop tier agree per block."""
    p = make_problem(2, 2, 5, 9, s=0.7, seed=seed, spectrum=spectrum)
    r0 = spinorb.energy(*_args(p))
    r1 = dsrg.energy(*_args(p))
    for k in BLOCKS:
        assert abs(r0[k] - r1[k]) <= 1e-12 * max(abs(r0[k]), 1.0), (k, r0[k], r1[k])


def test_zero_denominator_is_the_removable_limit():
    """Sec. II.B, Maclaurin form: the regulated amplitude behaves as t ~ v s D
    for small D, so each term is continuous through D = 0 with value 0 there.
    With exactly zero denominators planted in F1, F2 and F3, moving one of the
    planted virtual energies by delta changes the energy linearly in delta:
    E(2 delta) - E(0) = 2 (E(delta) - E(0)) + O(delta^2). A regulator with any
    other value at D = 0 would leave a jump that does not shrink with delta."""
    p = make_problem(2, 1, 5, 8, s=0.6, seed=23, spectrum="degenerate")
    ve = p.ncore + p.nactive

    def e_at(delta, tier):
        eps = p.eps.copy()
        eps[ve + 1] += delta   # virtual 1: the D = 0 quadruple of F1
        eps[ve + 2] += delta   # virtual 2: the D = 0 position of F2
        eps[ve + 3] += delta   # virtual 3: the D = 0 position of F3
        args = list(_args(p))
        args[1] = eps
        return tier.energy(*args)
    for tier in (dsrg, spinorb):
        r0, r1, r2 = e_at(0.0, tier), e_at(1e-5, tier), e_at(2e-5, tier)
        for k in ("ccvv", "cavv", "ccav", "total"):
            d1, d2 = r1[k] - r0[k], r2[k] - r0[k]
            assert np.isfinite(r0[k])
            assert abs(d2 - 2.0 * d1) <= 1e-3 * abs(d1) + 1e-12 * abs(r0[k]), (tier.__name__, k, d1, d2)


def test_power_of_two_scaling_is_exact():
    """E is homogeneous of degree 4 in B (Eqs. (12)-(15) with f^(1) = 0, Eq. (19)):
    B -> 2B multiplies every block by 16 exactly, bit for bit."""
    p = make_problem(4, 2, 6, 12, s=0.5, seed=9)
    r = dsrg.energy(*_args(p))
    r2 = dsrg.energy(*_args(p.scaled(2.0)))
    for k in BLOCKS:
        assert r2[k] == 16.0 * r[k], k


def test_orbital_permutation_invariance():
    """Nothing in Table 1 depends on the order of orbitals inside a space:
    permuting core, active (with G and lambda2) and virtual orbitals together
    with their energies and factor rows leaves every block unchanged."""
    p = make_problem(4, 3, 6, 12, s=0.5, seed=10)
    rng = np.random.default_rng(0)
    nC, nA, nV = p.ncore, p.nactive, p.nvirt
    pc, pa_, pv = rng.permutation(nC), rng.permutation(nA), rng.permutation(nV)
    hole = np.concatenate([pc, nC + pa_])
    part = np.concatenate([pa_, nA + pv])
    B = p.B[:, hole][:, :, part]
    eps = np.concatenate([p.eps[:nC][pc], p.eps[nC:nC + nA][pa_], p.eps[nC + nA:][pv]])
    G = p.gamma1[np.ix_(pa_, pa_)]
    L = p.lambda2[np.ix_(pa_, pa_, pa_, pa_)]
    r = dsrg.energy(*_args(p))
    rp = dsrg.energy(B, eps, G, L, p.s, nC, nA, nV)
    for k in BLOCKS:
        assert _rel(r[k], rp[k]) < 1e-13, k


def test_linear_in_lambda3():
    """The three-body cumulant enters only terms J and K of Table 1, linearly:
    E(2 L3) - E(0) = 2 (E(L3) - E(0)), and with L3 absent J = K = 0."""
    p = make_problem(2, 3, 4, 8, s=0.5, seed=15, with_lambda3=True)
    e = lambda l3: dsrg.energy(*_args(p), lambda3=l3)["total"]
    e0, e1, e2 = e(None), e(p.lambda3), e(2.0 * p.lambda3)
    assert e1 != e0
    assert abs((e2 - e0) - 2.0 * (e1 - e0)) <= 1e-13 * abs(e1)
    assert e(0.0 * p.lambda3) == e0


@pytest.mark.parametrize("occ", ["full", "empty"])
def test_singles_limit_is_mp2_with_singles(occ):
    """One-determinant limits (lambda = 0, G = 2I or 0) with an off-diagonal
    Fock block: T1 is f^(1) regulated (Eq. (12): the sum over u x vanishes),
    the modified Fock is f (1 + e^{-sD^2}) (Eq. (14)), and term A becomes
    sum_{ia} f_ia^2 (1 - e^{-2sD^2}) / D per spin. For s -> infinity the total is
    the textbook spin-orbital MP2 energy with the non-Brillouin singles term,
    1/4 sum |<ij||ab>|^2 / D_ij^ab + sum |f_ia|^2 / D_ia over the occupied (core,
    and active when G = 2I) and unoccupied spin orbitals."""
    p = make_problem(3, 2, 4, 10, s=1.0e6, seed=16, occupation=occ, with_f1=True)
    p.lambda2[...] = 0.0
    nC, nA, nV = p.ncore, p.nactive, p.nvirt
    r1 = dsrg.energy(*_args(p), f1=p.f1)
    r0 = spinorb.energy(*_args(p), f1=p.f1)
    if occ == "full":
        occ_idx, vir_idx = list(range(nC + nA)), list(range(nA, nA + nV))
        Bp, e_occ = p.B[:, :, nA:], p.eps[: nC + nA]
        mp2 = spinorb.mp2_spin_orbital(Bp, p.eps, nC + nA, nV, 0)
    else:
        occ_idx, vir_idx = list(range(nC)), list(range(nA + nV))
        Bp, e_occ = p.B[:, :nC, :], p.eps[:nC]
        mp2 = spinorb.mp2_spin_orbital(Bp, p.eps, nC, nA + nV, 0)
    e_vir = p.eps[nC:][vir_idx]
    f = p.f1[np.ix_(occ_idx, vir_idx)]
    singles = 2.0 * np.sum(f ** 2 / (e_occ[:, None] - e_vir[None, :]))
    assert singles != 0.0
    assert _rel(r1["total"], mp2 + singles) < 1e-12
    assert _rel(r0["total"], mp2 + singles) < 1e-12


def test_affine_in_lambda2():
    """Every Table 1 term is linear in lambda2 or independent of it (J, K absent):
    E(2L) - E(0) = 2 (E(L) - E(0))."""
    p = make_problem(3, 3, 5, 10, s=0.5, seed=13)
    args = list(_args(p))
    e1 = dsrg.energy(*args)["total"]
    args[3] = 2.0 * p.lambda2
    e2 = dsrg.energy(*args)["total"]
    args[3] = 0.0 * p.lambda2
    e0 = dsrg.energy(*args)["total"]
    assert abs((e2 - e0) - 2.0 * (e1 - e0)) <= 1e-13 * abs(e1)


@pytest.mark.parametrize("extra", [False, True], ids=["lam2", "lam3_f1"])
def test_gradient_matches_finite_differences_of_tier0(extra):
    """Autograd of tier 1 against central differences of the independent
    literal Table 1 (tier 0), on B entries in every block, on eps and on s
    (also with the three-body cumulant and f^(1))."""
    p = make_problem(3, 2, 4, 7, s=0.45, seed=14, with_lambda3=extra, with_f1=extra)
    g = dsrg.energy_and_grad(*_args(p), **_extra(p))
    rng = np.random.default_rng(1)
    h = 1e-5

    def e0(B=p.B, eps=p.eps, s=p.s):
        return spinorb.energy(B, eps, p.gamma1, p.lambda2, s, p.ncore, p.nactive, p.nvirt,
                              **_extra(p))["total"]

    idx = [tuple(rng.integers(0, n) for n in p.B.shape) for _ in range(12)]
    idx += [(0, 0, 0), (1, p.ncore, 0), (2, p.ncore + 1, p.nactive + 1), (3, 0, 1)]
    for ix in idx:
        Bp = p.B.copy(); Bp[ix] += h
        Bm = p.B.copy(); Bm[ix] -= h
        fd = (e0(B=Bp) - e0(B=Bm)) / (2 * h)
        assert abs(fd - g["dB"][ix]) <= 1e-7 * max(1.0, abs(fd)), (ix, fd, g["dB"][ix])
    for k in range(p.norb):
        ep = p.eps.copy(); ep[k] += h
        em = p.eps.copy(); em[k] -= h
        fd = (e0(eps=ep) - e0(eps=em)) / (2 * h)
        assert abs(fd - g["deps"][k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g["deps"][k])
    fd = (e0(s=p.s + h) - e0(s=p.s - h)) / (2 * h)
    assert abs(fd - g["ds"]) <= 1e-7 * max(1.0, abs(fd))


def test_gradient_at_zero_denominators():
    """With denominators exactly 0 in F1, F2 and F3 (planted degenerate orbital
    energies), the energy is still an analytic function of eps (Sec. II.B:
    t ~ v s D near D = 0). Autograd of tier 1 at that point equals central
    differences of tier 0, for the energies of the planted orbitals and for B
    entries of the orbitals involved."""
    p = make_problem(2, 1, 5, 8, s=0.6, seed=23, spectrum="degenerate")
    g = dsrg.energy_and_grad(*_args(p))
    h = 1e-6

    def e0(B=p.B, eps=p.eps):
        return spinorb.energy(B, eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt)["total"]

    for k in range(p.norb):
        ep = p.eps.copy(); ep[k] += h
        em = p.eps.copy(); em[k] -= h
        fd = (e0(eps=ep) - e0(eps=em)) / (2 * h)
        assert abs(fd - g["deps"][k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g["deps"][k])
    A = p.nactive
    for ix in [(0, 0, A + 0), (1, 1, A + 1), (2, 0, A + 2), (0, 1, A + 3), (3, p.ncore, A + 2)]:
        Bp = p.B.copy(); Bp[ix] += h
        Bm = p.B.copy(); Bm[ix] -= h
        fd = (e0(B=Bp) - e0(B=Bm)) / (2 * h)
        assert abs(fd - g["dB"][ix]) <= 1e-6 * max(1.0, abs(fd)), (ix, fd, g["dB"][ix])


# ---------------------------------------------------------------------------
# The cumulant reading, pinned by a brute-force CAS wavefunction: for a real
# singlet state, the spin-orbital lambda2 built from its opposite-spin block
# equals the one computed from the state's 1- and 2-RDMs (Sec. II.A, Eqs. (2)-(3)).
# ---------------------------------------------------------------------------
def _fock_ops(norb_spin):
    """Annihilation operators as dense matrices over all 2^n determinants
    (Jordan-Wigner ordering: spin orbital k = 2*p + sigma)."""
    n = norb_spin
    dim = 1 << n
    ops = []
    for k in range(n):
        a = np.zeros((dim, dim))
        for det in range(dim):
            if det >> k & 1:
                sign = (-1) ** bin(det & ((1 << k) - 1)).count("1")
                a[det ^ (1 << k), det] = sign
        ops.append(a)
    return ops


def _singlet_state(nspat, nelec, rng):
    n = 2 * nspat
    a = _fock_ops(n)
    ad = [x.T for x in a]
    dim = 1 << n
    Nop = sum(ad[k] @ a[k] for k in range(n))
    Sz = sum((0.5 if k % 2 == 0 else -0.5) * ad[k] @ a[k] for k in range(n))
    Sp = sum(ad[2 * p] @ a[2 * p + 1] for p in range(nspat))
    S2 = Sp.T @ Sp + Sz @ Sz + Sz                      # S^2 = S- S+ + Sz^2 + Sz
    sector = [d for d in range(dim) if abs(Nop[d, d] - nelec) < 1e-12 and abs(Sz[d, d]) < 1e-12]
    M = S2[np.ix_(sector, sector)]
    w, U = np.linalg.eigh(M)
    sing = U[:, np.abs(w) < 1e-9]
    c = sing @ rng.standard_normal(sing.shape[1])
    c /= np.linalg.norm(c)
    psi = np.zeros(dim)
    psi[sector] = c
    return psi, a, ad


@pytest.mark.parametrize("nspat,nelec,seed", [(2, 2, 0), (3, 2, 1), (3, 4, 2), (4, 4, 3)])
def test_cumulant_reading_against_wavefunction(nspat, nelec, seed):
    rng = np.random.default_rng(seed)
    psi, a, ad = _singlet_state(nspat, nelec, rng)
    n = 2 * nspat
    # gamma_q^p = <a^+_p a_q>, gamma_{uv}^{xy} = <a^+_x a^+_y a_v a_u>
    g1 = np.array([[psi @ ad[p] @ a[q] @ psi for q in range(n)] for p in range(n)])
    g2 = np.zeros((n,) * 4)
    for u, v, x, y in itertools.product(range(n), repeat=4):
        g2[u, v, x, y] = psi @ ad[x] @ ad[y] @ a[v] @ a[u] @ psi
    # lambda_{uv}^{xy} = gamma_{uv}^{xy} - gamma_u^x gamma_v^y + gamma_u^y gamma_v^x
    # with gamma_u^x = g1[x, u]
    lam = g2 - np.einsum("xu,yv->uvxy", g1, g1) + np.einsum("yu,xv->uvxy", g1, g1)
    # spatial inputs: G (spin summed) and L (alpha, beta; alpha, beta)
    G = g1[0::2, 0::2] + g1[1::2, 1::2]
    assert np.allclose(g1[0::2, 0::2], g1[1::2, 1::2])          # singlet: equal spins
    assert np.allclose(g1[0::2, 1::2], 0.0)
    L = lam[0::2, 1::2, 0::2, 1::2]
    rebuilt_t0 = spinorb.SpinOrbitalSystem._lambda_so(L, nspat)
    rebuilt_t1 = dsrg._lambda_so(torch.as_tensor(L), nspat).numpy()
    assert np.max(np.abs(rebuilt_t0 - lam)) < 1e-12
    assert np.max(np.abs(rebuilt_t1 - lam)) < 1e-12
    # and the 1-RDM reading: spin orbital gamma = G / 2 on each spin
    assert np.allclose(np.kron(G / 2.0, np.eye(2)), g1)
