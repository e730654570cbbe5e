"""Seeded synthetic inputs for the DF/CD DSRG-MRPT2 energy.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic. Both the CPU oracle and the CUDA library are fed from it.

What is generated (sizes follow the orbital partition of Sec. II.A: core C,
active A, virtual V; hole space H = C+A, particle space P = A+V; orbital order
[core | active | virtual]):

* ``B`` -- the hole x particle block of the three-index factors of Eq. (19),
  ``B[Q, i, a]`` for ``i`` in H and ``a`` in P, shape ``[naux, nH, nP]``, FP64,
  row-major. Entries are ``b_scale * N(0,1) * exp(-b_decay * Q)``. The factors
  are symmetric in their two orbital indices, so the active x active sub-block
  (hole index active, particle index active) is symmetrised: the entry for the
  orbital pair (u, x) equals the one for (x, u).
* ``eps`` -- semicanonical orbital energies (diagonal of the generalized Fock
  matrix, Eq. (8)), shape ``[n]``: core ~ U[-2.0, -0.3], active ~ U[-0.2, 0.1],
  virtual ~ U[0.05, 5.0] Eh, each block sorted ascending.
* ``gamma1`` -- spin-summed active one-particle density matrix, ``[nA, nA]``,
  symmetric, eigenvalues ``1 + d_k`` in [0, 2] with trace nA (half filling),
  rotated by a seeded Haar-random orthogonal matrix.
* ``lambda2`` -- the opposite-spin active two-body cumulant
  ``lambda2[u, v, x, y]`` (u, x alpha; v, y beta), entries ~ U(-0.05, 0.05),
  averaged over the 8 index permutations of a real (ux|vy)-type tensor.
* optional ``lambda3`` (``with_lambda3=True``) -- a spin-orbital three-body
  cumulant over the active spin orbitals ``2u + sigma``,
  ``lambda3[U,V,W,X,Y,Z]`` for lambda_{UVW}^{XYZ}: entries ~ U(-0.02, 0.02),
  zero unless the lower and upper triples hold the same number of alpha spin
  orbitals, antisymmetrised over the lower triple and over the upper triple,
  and symmetrised under the exchange of the two triples (a real Hermitian
  cumulant).
* optional ``f1`` (``with_f1=True``) -- the off-diagonal Fock block,
  ``f1[i, a]`` for hole i and particle a, entries ~ U(-0.05, 0.05), zero on the
  active x active sub-block (which belongs to the diagonal block).

Random streams come from numpy's PCG64 seeded with ``SeedSequence(seed)``,
one child stream per tensor, so each tensor is independent of the others'
sizes only through its own shape.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["Problem", "make_problem", "CONFIGS", "batch_sizes", "FockProblem", "make_fock_problem",
           "AOProblem", "make_ao_problem", "make_eri_factors"]


@dataclasses.dataclass
class Problem:
    ncore: int
    nactive: int
    nvirt: int
    naux: int
    s: float
    B: np.ndarray        # [naux, nH, nP] float64
    eps: np.ndarray      # [n] float64, order [core | active | virtual]
    gamma1: np.ndarray   # [nA, nA] float64
    lambda2: np.ndarray  # [nA, nA, nA, nA] float64
    lambda3: np.ndarray | None = None  # [2nA]^6 float64, spin orbitals
    f1: np.ndarray | None = None       # [nH, nP] float64

    @property
    def nhole(self) -> int:
        return self.ncore + self.nactive

    @property
    def npart(self) -> int:
        return self.nactive + self.nvirt

    @property
    def norb(self) -> int:
        return self.ncore + self.nactive + self.nvirt

    def scaled(self, factor: float) -> "Problem":
        """Same problem with B multiplied by ``factor``."""
        return dataclasses.replace(self, B=self.B * factor)


def _haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    if n == 0:
        return np.zeros((0, 0))
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    q = q * np.sign(np.diag(r))[None, :]
    return q


# Planted orbital energies of the "degenerate" spectrum (dyadic, so every sum
# and difference below is exact in binary floating point):
#   core 0, 1 = -1/2, -1/4; active 0 = 1/8; virtual 0..3 = -1/2, -1/4, 1/8, -7/8,
# which make one denominator of each kind exactly zero: core pair (0, 1) with
# virtuals (0, 1); core 0, active 0 with virtuals (0, 2); core pair (0, 1) with
# virtual 3 and active 0.
DEGENERATE = dict(core=(-0.5, -0.25), active=(0.125,), virt=(-0.5, -0.25, 0.125, -0.875))


def _antisym3(t: np.ndarray, axes) -> np.ndarray:
    """Antisymmetrise a tensor over three of its axes (sum over the 6 orders with signs, / 6)."""
    a, b, c = axes
    out = np.zeros_like(t)
    for perm, sign in (((a, b, c), 1), ((b, c, a), 1), ((c, a, b), 1),
                       ((b, a, c), -1), ((a, c, b), -1), ((c, b, a), -1)):
        order = list(range(t.ndim))
        order[a], order[b], order[c] = perm
        out += sign * t.transpose(order)
    return out / 6.0


def make_lambda3(nactive: int, rng: np.random.Generator, scale: float = 0.02) -> np.ndarray:
    """Random real Hermitian spin-orbital three-body cumulant (see module docstring)."""
    n2 = 2 * nactive
    R = rng.uniform(-scale, scale, (n2,) * 6)
    alpha = (np.arange(n2) % 2 == 0).astype(int)
    na_low = alpha[:, None, None] + alpha[None, :, None] + alpha[None, None, :]
    mask = na_low[:, :, :, None, None, None] == na_low[None, None, None, :, :, :]
    R = R * mask
    R = _antisym3(_antisym3(R, (0, 1, 2)), (3, 4, 5))
    return 0.5 * (R + R.transpose(3, 4, 5, 0, 1, 2))


def make_problem(ncore: int, nactive: int, nvirt: int, naux: int, s: float = 0.5,
                 seed: int = 0, b_scale: float = 0.3, b_decay: float = 0.02,
                 occupation: str = "random", spectrum: str = "sorted",
                 with_lambda3: bool = False, with_f1: bool = False) -> Problem:
    """Draw one synthetic problem.

    ``occupation`` selects gamma1: ``"random"`` (the recipe above), ``"full"``
    (gamma1 = 2 I: the active orbitals doubly occupied) or ``"empty"``
    (gamma1 = 0). ``lambda2`` is drawn in all cases; callers zero it when a
    test needs a one-determinant reference.

    ``spectrum`` selects the orbital energies: ``"sorted"`` (the recipe above);
    ``"overlap"`` (core ~ U[-2.0, -0.3], active ~ U[-0.2, 0.1], virtual ~
    U[-1.2, 5.0], none of the blocks sorted, so virtual energies fall below core
    and active ones and the denominators of every block cross zero);
    ``"degenerate"`` (``"overlap"`` with the energies of ``DEGENERATE`` planted
    at the start of each block, so that some denominators are exactly zero;
    needs ncore >= 2, nactive >= 1, nvirt >= 4); ``"negative"`` (virtual ~
    U[-1.9, -0.4], sorted, core and active as in the recipe: every virtual
    energy negative).
    """
    if min(ncore, nactive, nvirt) < 0 or naux < 1:
        raise ValueError("sizes must be >= 0 and naux >= 1")
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(5)
    rB, re, rg, rl, rx = (np.random.Generator(np.random.PCG64(k)) for k in kids)
    nH, nP = ncore + nactive, nactive + nvirt

    B = rB.standard_normal((naux, nH, nP))
    if nactive > 0:
        # active-active sub-block: hole index ncore+u, particle index x.
        aa = B[:, ncore:, :nactive]
        iu = np.triu_indices(nactive, 1)
        # copy the upper triangle over the lower one so (u, x) == (x, u)
        aa[:, iu[1], iu[0]] = aa[:, iu[0], iu[1]]
        B[:, ncore:, :nactive] = aa
    B *= b_scale * np.exp(-b_decay * np.arange(naux, dtype=np.float64))[:, None, None]

    if spectrum == "sorted":
        eC = np.sort(re.uniform(-2.0, -0.3, ncore))
        eA = np.sort(re.uniform(-0.2, 0.1, nactive))
        eV = np.sort(re.uniform(0.05, 5.0, nvirt))
    elif spectrum in ("overlap", "degenerate"):
        eC = re.uniform(-2.0, -0.3, ncore)
        eA = re.uniform(-0.2, 0.1, nactive)
        eV = re.uniform(-1.2, 5.0, nvirt)
        if spectrum == "degenerate":
            if ncore < 2 or nactive < 1 or nvirt < 4:
                raise ValueError("the degenerate spectrum needs ncore >= 2, nactive >= 1, nvirt >= 4")
            eC[:2] = DEGENERATE["core"]
            eA[:1] = DEGENERATE["active"]
            eV[:4] = DEGENERATE["virt"]
    elif spectrum == "negative":
        eC = np.sort(re.uniform(-2.0, -0.3, ncore))
        eA = np.sort(re.uniform(-0.2, 0.1, nactive))
        eV = np.sort(re.uniform(-1.9, -0.4, nvirt))
    else:
        raise ValueError(spectrum)
    eps = np.concatenate([eC, eA, eV])

    if occupation == "random":
        d = rg.uniform(-1.0, 1.0, nactive)
        if nactive > 0:
            d = d - d.mean()
            m = np.abs(d).max()
            if m > 1.0:
                d = d / m
        U = _haar_orthogonal(rg, nactive)
        gamma1 = (U * (1.0 + d)[None, :]) @ U.T
        gamma1 = 0.5 * (gamma1 + gamma1.T)
    elif occupation == "full":
        gamma1 = 2.0 * np.eye(nactive)
    elif occupation == "empty":
        gamma1 = np.zeros((nactive, nactive))
    else:
        raise ValueError(occupation)

    L = rl.uniform(-0.05, 0.05, (nactive,) * 4)
    # (ux|vy)-type 8-fold symmetry of L[u, v, x, y]: u<->x, v<->y, (u,x)<->(v,y)
    perms = []
    for t in (L, L.transpose(2, 1, 0, 3)):             # u<->x
        for t2 in (t, t.transpose(0, 3, 2, 1)):         # v<->y
            perms.append(t2)
            perms.append(t2.transpose(1, 0, 3, 2))      # (u,x)<->(v,y)
    lambda2 = sum(perms) / 8.0

    lambda3 = make_lambda3(nactive, rx) if with_lambda3 else None
    f1 = None
    if with_f1:
        f1 = rx.uniform(-0.05, 0.05, (nH, nP))
        f1[ncore:, :nactive] = 0.0
    return Problem(ncore, nactive, nvirt, naux, float(s), B, eps, gamma1, lambda2, lambda3, f1)


@dataclasses.dataclass
class FockProblem:
    """Inputs of the generalized Fock build and semicanonicalisation: the
    one-electron integrals and the DF factors over ALL orbital pairs (not only
    hole x particle), plus the active density and cumulants (non-semicanonical
    orbitals: the Fock matrix has off-diagonal elements inside each block)."""
    ncore: int
    nactive: int
    nvirt: int
    naux: int
    s: float
    h: np.ndarray        # [n, n] symmetric
    Bfull: np.ndarray    # [naux, n, n] symmetric in the orbital pair
    gamma1: np.ndarray   # [nA, nA]
    lambda2: np.ndarray  # [nA]^4
    lambda3: np.ndarray | None = None


def make_fock_problem(ncore: int, nactive: int, nvirt: int, naux: int, s: float = 0.5,
                      seed: int = 0, b_scale: float = 0.05, b_decay: float = 0.02,
                      with_lambda3: bool = False) -> FockProblem:
    """Draw one problem for the Fock build: ``Bfull[Q, p, q]`` = b_scale *
    N(0,1) * exp(-b_decay Q), symmetrised in (p, q) (b_scale 0.05 keeps the
    two-electron part of the Fock matrix a perturbation of h at these sizes,
    so that core, active and virtual orbital energies stay apart); ``h`` = diag(h0) + a
    symmetric matrix with entries ~ U(-0.05, 0.05), h0 drawn like the orbital
    energies of the recipe (core ~ U[-2.0, -0.3], active ~ U[-0.2, 0.1],
    virtual ~ U[0.05, 5.0], unsorted); gamma1, lambda2 (and lambda3) as in
    ``make_problem`` with the same seed."""
    n = ncore + nactive + nvirt
    base = make_problem(ncore, nactive, nvirt, 1, s=s, seed=seed, with_lambda3=with_lambda3)
    ss = np.random.SeedSequence([seed, 4242])
    rB, rh = (np.random.Generator(np.random.PCG64(k)) for k in ss.spawn(2))
    B = rB.standard_normal((naux, n, n))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    B *= b_scale * np.exp(-b_decay * np.arange(naux, dtype=np.float64))[:, None, None]
    h0 = np.concatenate([rh.uniform(-2.0, -0.3, ncore), rh.uniform(-0.2, 0.1, nactive),
                         rh.uniform(0.05, 5.0, nvirt)])
    R = rh.uniform(-0.05, 0.05, (n, n))
    h = np.diag(h0) + 0.5 * (R + R.T)
    return FockProblem(ncore, nactive, nvirt, naux, float(s), h, B, base.gamma1, base.lambda2,
                       base.lambda3)


@dataclasses.dataclass
class AOProblem:
    """Inputs of the DF integral transformation (Sec. II.C): AO three-centre
    integrals, the two-centre metric and MO coefficients."""
    nbf: int
    naux: int
    ao3: np.ndarray    # [naux, nbf, nbf] (mu nu|P), symmetric in (mu, nu)
    metric: np.ndarray  # [naux, naux] J_PQ, symmetric positive definite
    C: np.ndarray      # [nbf, nmo] MO coefficients


def make_ao_problem(nbf: int, nmo: int, naux: int, seed: int = 0) -> AOProblem:
    """``ao3[P, mu, nu]`` = 0.3 N(0,1) exp(-0.02 P), symmetrised in (mu, nu);
    ``metric`` = W diag(w) W^T with a Haar-random orthogonal W and w log-uniform
    in [0.1, 10]; ``C`` = the first nmo columns of a Haar-random orthogonal matrix."""
    ss = np.random.SeedSequence([seed, 1603])
    ra, rm, rc = (np.random.Generator(np.random.PCG64(k)) for k in ss.spawn(3))
    ao3 = ra.standard_normal((naux, nbf, nbf))
    ao3 = 0.5 * (ao3 + ao3.transpose(0, 2, 1))
    ao3 *= 0.3 * np.exp(-0.02 * np.arange(naux, dtype=np.float64))[:, None, None]
    W = _haar_orthogonal(rm, naux)
    w = np.exp(rm.uniform(np.log(0.1), np.log(10.0), naux))
    metric = (W * w[None, :]) @ W.T
    metric = 0.5 * (metric + metric.T)
    C = _haar_orthogonal(rc, nbf)[:, :nmo]
    return AOProblem(nbf, naux, ao3, metric, np.ascontiguousarray(C))


def make_eri_factors(n: int, rank: int, seed: int = 0, scale: float = 0.3,
                     decay: float = 0.02) -> np.ndarray:
    """Exact low-rank factors of a synthetic two-electron integral matrix for
    the Cholesky decomposition: ``F[k, p, q]`` = scale N(0,1) exp(-decay k),
    symmetric in (p, q); the integrals are (pq|rs) = sum_k F[k,p,q] F[k,r,s]."""
    r = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 315])))
    F = r.standard_normal((rank, n, n))
    F = 0.5 * (F + F.transpose(0, 2, 1))
    return F * scale * np.exp(-decay * np.arange(rank, dtype=np.float64))[:, None, None]


# The synthetic workloads, by what they stand for (sizes nC/nA/nV/naux, s).
CONFIGS = {
    "tiny-74": dict(ncore=10, nactive=4, nvirt=60, naux=200, s=0.5, seed=0),
    "naphthyne-vtz-398": dict(ncore=24, nactive=2, nvirt=372, naux=1200, s=0.5, seed=0),
    "naphthyne-v5z-1240": dict(ncore=24, nactive=2, nvirt=1214, naux=3400, s=0.5, seed=0),
}


def batch_sizes(seed: int) -> dict:
    """Sizes of molecule ``seed`` of the uneven 64-molecule batch: nC ~ U{8..40},
    nA ~ U{2..6}, nV ~ U{100..600}, naux = round(3.2 * (nC + nA + nV))."""
    r = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7919])))
    nC = int(r.integers(8, 41))
    nA = int(r.integers(2, 7))
    nV = int(r.integers(100, 601))
    return dict(ncore=nC, nactive=nA, nvirt=nV, naux=int(round(3.2 * (nC + nA + nV))))
