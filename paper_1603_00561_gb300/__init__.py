"""GB300-native DF/CD DSRG-MRPT2 second-order energy (arXiv:1603.00561).

Thin Python layer over the C ABI of ``libdsrg.so`` (``include/dsrg.h``): it
passes device pointers of FP64 CUDA tensors and the current CUDA stream, and
nothing else. Every step of the energy runs in the library's kernels; there
is no CPU path. Importing the package does not load the library; the first
``Plan`` does, and fails loudly if it is missing or no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import ctypes as C_

import torch

from . import _native
from ._native import DSRGError, PREC

__all__ = ["Plan", "Batch", "DSRGError", "PREC", "BLOCKS", "build", "DSRGEnergy", "energy_total",
           "SemicanonicalPlan", "df_mo_transform", "cd_factors", "shard_pairs"]

BLOCKS = ("ccvv", "cavv", "ccav", "active", "total")


def build(verbose: bool = False, force: bool = False) -> str:
    from ._buildlib import build as _b
    return _b(verbose=verbose, force=force)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("arrays must be contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


class Plan:
    """A problem size + precision with its device workspace (``dsrg_df_plan``).

    ``precision``: ``"fp64"``, ``"tf32x3"`` or ``"bf16x3"``.
    """

    def __init__(self, ncore: int, nactive: int, nvirt: int, naux: int,
                 precision: str = "fp64", host_io: bool = False, grad: bool = False, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the DSRG-MRPT2 library needs a CUDA GPU")
        self.lib = _native.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.sizes = (int(ncore), int(nactive), int(nvirt), int(naux))
        self.precision = precision
        sz = _native.Sizes(*self.sizes)
        h = C.c_void_p()
        flags = (_native.PLAN_HOST_IO if host_io else 0) | (_native.PLAN_GRAD if grad else 0)
        with torch.cuda.device(self.device):
            st = self.lib.dsrg_df_plan(C.byref(h), C.byref(sz), PREC[precision],
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream), flags)
        if st != _native.OK:
            raise DSRGError(st, f"dsrg_df_plan{self.sizes} {precision}")
        self.h = h

    # -- helpers ---------------------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != _native.OK:
            raise DSRGError(st, f"{what}: {self.lib.dsrg_plan_last_error(self.h).decode()}")

    def _stream(self):
        self.lib.dsrg_plan_set_stream(self.h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    @property
    def ncore(self):
        return self.sizes[0]

    @property
    def nactive(self):
        return self.sizes[1]

    def last_launch_count(self) -> int:
        return int(self.lib.dsrg_plan_last_launch_count(self.h))

    def workspace_bytes(self) -> int:
        return int(self.lib.dsrg_plan_workspace_bytes(self.h))

    # -- entry points ------------------------------------------------------------------------
    def energy(self, B, eps, gamma1, lambda2, s: float, out=None, lambda3=None, f1=None):
        """Block energies [E_CCVV, E_CAVV, E_CCAV, E_active, E_total] as a device tensor.
        ``lambda3`` (spin-orbital three-body cumulant, [2nA]^6) and ``f1`` (off-diagonal
        Fock block, [nH, nP]) are optional (``dsrg_mrpt2_energy_ext``)."""
        if out is None:
            out = torch.empty(5, dtype=torch.float64, device=self.device)
        self._stream()
        if lambda3 is None and f1 is None:
            st = self.lib.dsrg_mrpt2_energy(self.h, _ptr(B), _ptr(eps), _ptr(gamma1),
                                            _ptr(lambda2), float(s), _ptr(out))
            self._check(st, "dsrg_mrpt2_energy")
        else:
            st = self.lib.dsrg_mrpt2_energy_ext(self.h, _ptr(B), _ptr(eps), _ptr(gamma1),
                                                _ptr(lambda2), _ptr(lambda3), _ptr(f1), float(s),
                                                _ptr(out))
            self._check(st, "dsrg_mrpt2_energy_ext")
        return out

    def pair_energies(self, B, eps, s: float, out=None):
        """Pair energies e[m, n] of diagram F1 as an [nC, nC] device tensor."""
        nC = self.ncore
        if out is None:
            out = torch.empty((nC, nC), dtype=torch.float64, device=self.device)
        self._stream()
        st = self.lib.dsrg_ccvv_pair_energies(self.h, _ptr(B), _ptr(eps), float(s), _ptr(out))
        self._check(st, "dsrg_ccvv_pair_energies")
        return out

    def energy_grad(self, B, eps, gamma1, lambda2, s: float, lambda3=None, f1=None):
        """Energies plus dE_total/dB, dE_total/deps, dE_total/ds (device tensors);
        optional ``lambda3`` and ``f1`` as for ``energy``."""
        out = torch.empty(5, dtype=torch.float64, device=self.device)
        dB = torch.empty_like(B)
        de = torch.empty_like(eps)
        ds = torch.empty(1, dtype=torch.float64, device=self.device)
        self._stream()
        st = self.lib.dsrg_mrpt2_energy_grad_ext(self.h, _ptr(B), _ptr(eps), _ptr(gamma1),
                                                 _ptr(lambda2), _ptr(lambda3), _ptr(f1), float(s),
                                                 _ptr(out), _ptr(dB), _ptr(de), _ptr(ds))
        self._check(st, "dsrg_mrpt2_energy_grad_ext")
        return out, dB, de, ds

    def energy_host(self, B, eps, gamma1, lambda2, s: float, out=None):
        """Host-buffer entry: numpy/pinned-tensor inputs, host out[5]; synchronises."""
        import numpy as np

        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                assert a.device.type == "cpu" and a.dtype == torch.float64 and a.is_contiguous()
                return C.c_void_p(a.data_ptr())
            a = np.ascontiguousarray(a, dtype=np.float64)
            return a.ctypes.data_as(C.c_void_p)

        keep = [np.ascontiguousarray(x, dtype=np.float64) if not isinstance(x, torch.Tensor)
                and x is not None else x for x in (B, eps, gamma1, lambda2)]
        if out is None:
            out = np.zeros(5)
        outp = out.ctypes.data_as(C.c_void_p) if isinstance(out, np.ndarray) else C.c_void_p(out.data_ptr())
        self._stream()
        st = self.lib.dsrg_mrpt2_energy_host(self.h, *[hp(x) for x in keep], float(s), outp)
        self._check(st, "dsrg_mrpt2_energy_host")
        return out

    def autotune(self, B, eps, s: float, reps: int = 3) -> int:
        """Time the candidate work-item orders of the CCVV launch on these inputs
        and keep the fastest (``dsrg_plan_autotune``); returns its code."""
        chosen = C.c_int32(-1)
        self._stream()
        st = self.lib.dsrg_plan_autotune(self.h, _ptr(B), _ptr(eps), float(s), int(reps), C.byref(chosen))
        self._check(st, "dsrg_plan_autotune")
        return int(chosen.value)

    @property
    def item_order(self) -> int:
        return int(self.lib.dsrg_plan_item_order(self.h))

    @item_order.setter
    def item_order(self, order: int):
        self._check(self.lib.dsrg_plan_set_item_order(self.h, int(order)), "dsrg_plan_set_item_order")

    def time_ccvv(self, B, eps, s: float, reps: int = 5) -> float:
        """Average device milliseconds of the CCVV kernel alone (``dsrg_plan_time_ccvv``)."""
        ms = C.c_float(0.0)
        self._stream()
        st = self.lib.dsrg_plan_time_ccvv(self.h, _ptr(B), _ptr(eps), float(s), int(reps), C.byref(ms))
        self._check(st, "dsrg_plan_time_ccvv")
        return float(ms.value)

    def sync(self):
        self._check(self.lib.dsrg_plan_sync(self.h), "dsrg_plan_sync")

    def set_shard(self, rank: int, world: int):
        """Compute only this rank's share of the molecule (``dsrg_plan_set_shard``):
        energies and gradients become partial sums over ranks."""
        self._check(self.lib.dsrg_plan_set_shard(self.h, int(rank), int(world)),
                    "dsrg_plan_set_shard")

    def branch_counts(self, reset: bool = False) -> dict:
        """Epilogue branch counters of the split kernels (``dsrg_plan_branch_counts``)."""
        arr = (C.c_uint64 * _native.NCOUNTERS)()
        self._check(self.lib.dsrg_plan_branch_counts(self.h, arr, 1 if reset else 0),
                    "dsrg_plan_branch_counts")
        return {k: int(arr[i]) for k, i in _native.COUNTERS.items()}

    def close(self):
        if getattr(self, "h", None):
            self.lib.dsrg_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many molecules of uneven size in one call (``dsrg_batch_plan``): one
    persistent tensor-core CCVV launch over all molecules, the whole call
    captured in a CUDA graph and replayed while inputs stay the same."""

    def __init__(self, sizes, precision: str = "bf16x3", device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the DSRG-MRPT2 library needs a CUDA GPU")
        self.lib = _native.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.sizes = [tuple(int(v) for v in sz) for sz in sizes]
        arr = (_native.Sizes * len(self.sizes))(*[_native.Sizes(*sz) for sz in self.sizes])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.dsrg_batch_plan(C.byref(h), len(self.sizes), arr, PREC[precision],
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream), 0)
        if st != _native.OK:
            raise DSRGError(st, f"dsrg_batch_plan({len(self.sizes)} molecules) {precision}")
        self.h = h
        self.n = len(self.sizes)

    def energy(self, inputs, s, out=None):
        """``inputs``: list of (B, eps, gamma1, lambda2) device tensors per molecule;
        ``s``: list of flow parameters. Returns [nmol, 5] block energies (device)."""
        if out is None:
            out = torch.empty((self.n, 5), dtype=torch.float64, device=self.device)
        P = C.c_void_p * self.n
        cols = list(zip(*inputs))
        ptrs = [P(*[_ptr(t) for t in col]) for col in cols]
        svals = (C.c_double * self.n)(*[float(x) for x in s])
        st = self.lib.dsrg_mrpt2_energy_batched(self.h, *ptrs, svals, _ptr(out))
        if st != _native.OK:
            raise DSRGError(st, self.lib.dsrg_batch_last_error(self.h).decode())
        return out

    def autotune(self, inputs, s, reps: int = 2) -> int:
        """Time the candidate work-item orders of the batched CCVV launch and keep
        the fastest (``dsrg_batch_autotune``); returns its code."""
        P = C.c_void_p * self.n
        Bs = P(*[_ptr(t[0]) for t in inputs])
        es = P(*[_ptr(t[1]) for t in inputs])
        svals = (C.c_double * self.n)(*[float(x) for x in s])
        chosen = C.c_int32(-1)
        st = self.lib.dsrg_batch_autotune(self.h, Bs, es, svals, int(reps), C.byref(chosen))
        if st != _native.OK:
            raise DSRGError(st, self.lib.dsrg_batch_last_error(self.h).decode())
        return int(chosen.value)

    @property
    def item_order(self) -> int:
        return int(self.lib.dsrg_batch_item_order(self.h))

    @item_order.setter
    def item_order(self, order: int):
        st = self.lib.dsrg_batch_set_item_order(self.h, int(order))
        if st != _native.OK:
            raise DSRGError(st, self.lib.dsrg_batch_last_error(self.h).decode())

    @property
    def branches(self) -> int:
        """Concurrent branches of the per-molecule blocks in the batched graph."""
        return int(self.lib.dsrg_batch_branches(self.h))

    @branches.setter
    def branches(self, k: int):
        st = self.lib.dsrg_batch_set_branches(self.h, int(k))
        if st != _native.OK:
            raise DSRGError(st, f"dsrg_batch_set_branches({k})")

    def autotune_branches(self, inputs, s, reps: int = 2, out=None) -> int:
        """Time the whole batched call for every allowed branch count and keep the
        fastest (``dsrg_batch_autotune_branches``); returns it."""
        if out is None:
            out = torch.empty((self.n, 5), dtype=torch.float64, device=self.device)
        P = C.c_void_p * self.n
        cols = list(zip(*inputs))
        ptrs = [P(*[_ptr(t) for t in col]) for col in cols]
        svals = (C.c_double * self.n)(*[float(x) for x in s])
        chosen = C.c_int32(-1)
        st = self.lib.dsrg_batch_autotune_branches(self.h, *ptrs, svals, _ptr(out), int(reps),
                                                   C.byref(chosen))
        if st != _native.OK:
            raise DSRGError(st, self.lib.dsrg_batch_last_error(self.h).decode())
        return int(chosen.value)

    def sync(self):
        st = self.lib.dsrg_batch_sync(self.h)
        if st != _native.OK:
            raise DSRGError(st, self.lib.dsrg_batch_last_error(self.h).decode())

    def launch_count(self) -> int:
        return int(self.lib.dsrg_batch_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dsrg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_cache_get(path, key):
    """The value stored under ``key`` in the autotuners' cache file, or None
    (``dsrg_tune_cache_get``; no GPU needed). A malformed file raises."""
    lib = _native.load()
    v = C.c_int64(0)
    r = lib.dsrg_tune_cache_get(str(path).encode(), key.encode(), C.byref(v))
    if r < 0:
        raise ValueError(f"{path} is not an autotune cache file")
    return int(v.value) if r == 1 else None


def tune_cache_put(path, key, value):
    """Store ``value`` under ``key`` in the autotuners' cache file
    (``dsrg_tune_cache_put``; no GPU needed)."""
    lib = _native.load()
    st = lib.dsrg_tune_cache_put(str(path).encode(), key.encode(), int(value))
    if st != _native.OK:
        raise DSRGError(st, f"dsrg_tune_cache_put({path}, {key})")


class SemicanonicalPlan:
    """Generalized Fock matrix (Eq. (8)) and the semicanonical basis
    (``dsrg_sc_plan_create``, ``dsrg_generalized_fock``, ``dsrg_semicanonicalize``):
    from h [n, n], the full DF factors Bfull [naux, n, n] and the active density,
    the inputs of the energy in the semicanonical orbitals."""

    def __init__(self, ncore: int, nactive: int, nvirt: int, naux: int, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the DSRG-MRPT2 library needs a CUDA GPU")
        self.lib = _native.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.sizes = (int(ncore), int(nactive), int(nvirt), int(naux))
        sz = _native.Sizes(*self.sizes)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.dsrg_sc_plan_create(C.byref(h), C.byref(sz),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != _native.OK:
            raise DSRGError(st, f"dsrg_sc_plan_create{self.sizes}")
        self.h = h

    def _check(self, st, what):
        if st != _native.OK:
            raise DSRGError(st, f"{what}: {self.lib.dsrg_sc_last_error(self.h).decode()}")

    def fock(self, h, Bfull, gamma1):
        n = sum(self.sizes[:3])
        f = torch.empty((n, n), dtype=torch.float64, device=self.device)
        self._check(self.lib.dsrg_generalized_fock(self.h, _ptr(h), _ptr(Bfull), _ptr(gamma1), _ptr(f)),
                    "dsrg_generalized_fock")
        return f

    def semicanonicalize(self, h, Bfull, gamma1, lambda2, lambda3=None) -> dict:
        nC, nA, nV, Q = self.sizes
        n, nH, nP = nC + nA + nV, nC + nA, nA + nV
        z = lambda *shape: torch.empty(shape, dtype=torch.float64, device=self.device)
        out = dict(eps=z(n), B=z(Q, nH, nP), f1=z(nH, nP), U=z(n, n),
                   gamma1=z(nA, nA) if nA else None, lambda2=z(nA, nA, nA, nA) if nA else None,
                   lambda3=z(*(2 * nA,) * 6) if (nA and lambda3 is not None) else None)
        st = self.lib.dsrg_semicanonicalize(
            self.h, _ptr(h), _ptr(Bfull), _ptr(gamma1), _ptr(lambda2), _ptr(lambda3),
            _ptr(out["eps"]), _ptr(out["B"]), _ptr(out["f1"]), _ptr(out["gamma1"]),
            _ptr(out["lambda2"]), _ptr(out["lambda3"]), _ptr(out["U"]))
        self._check(st, "dsrg_semicanonicalize")
        return out

    def last_sweeps(self) -> int:
        return int(self.lib.dsrg_sc_last_sweeps(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dsrg_sc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_pairs(ncore: int, rank: int, world: int):
    """The (i, j) core pairs of one rank's share (``dsrg_shard_pairs``; host only,
    needs the library but no GPU)."""
    lib = _native.load()
    n = int(lib.dsrg_shard_pairs(int(ncore), int(rank), int(world), None))
    if n < 0:
        raise ValueError("bad shard arguments")
    buf = (C_.c_int32 * (2 * max(n, 1)))()
    lib.dsrg_shard_pairs(int(ncore), int(rank), int(world), buf)
    return [(buf[2 * k], buf[2 * k + 1]) for k in range(n)]


def df_mo_transform(ao3, C, metric, p0: int = 0, np_: int | None = None, q0: int = 0,
                    nq: int | None = None):
    """DF factors B^Q_pq of the MO three-centre integrals for p in [p0, p0+np_),
    q in [q0, q0+nq) (``dsrg_df_mo_transform``; metric square root from its
    Cholesky factor). Device tensors in, [naux, np_, nq] device tensor out."""
    lib = _native.load()
    naux, nbf, _ = ao3.shape
    nmo = C.shape[1]
    np_ = nmo - p0 if np_ is None else np_
    nq = nmo - q0 if nq is None else nq
    out = torch.empty((naux, np_, nq), dtype=torch.float64, device=ao3.device)
    wb = int(lib.dsrg_df_mo_transform_work_bytes(nbf, naux, np_, nq))
    work = torch.empty((wb + 7) // 8, dtype=torch.float64, device=ao3.device)
    st = lib.dsrg_df_mo_transform(_ptr(ao3), _ptr(C), _ptr(metric), nbf, nmo, naux, p0, np_, q0, nq,
                                  _ptr(out), _ptr(work), wb,
                                  C_.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != _native.OK:
        raise DSRGError(st, "dsrg_df_mo_transform")
    return out


def cd_factors(F, tau: float = 1e-5, max_rank: int | None = None):
    """Pivoted Cholesky vectors of the integral matrix sum_k F^k (F^k)^T
    (``dsrg_cd_factors``): F [nfac, n, n] device tensor; returns [rank, n, n]."""
    lib = _native.load()
    nfac, n, _ = F.shape
    max_rank = n * n if max_rank is None else max_rank
    L = torch.empty((max_rank, n, n), dtype=torch.float64, device=F.device)
    wb = int(lib.dsrg_cd_factors_work_bytes(n))
    work = torch.empty((wb + 7) // 8, dtype=torch.float64, device=F.device)
    rank = C_.c_int32(0)
    st = lib.dsrg_cd_factors(_ptr(F), nfac, n, float(tau), max_rank, _ptr(L), C_.byref(rank),
                             _ptr(work), wb, C_.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != _native.OK:
        raise DSRGError(st, "dsrg_cd_factors")
    return L[: rank.value]


class DSRGEnergy(torch.autograd.Function):
    """E_total(B, eps, s) as a differentiable scalar. The backward pass calls the
    library's adjoint (``dsrg_mrpt2_energy_grad``), which recomputes the pair
    integrals per core row instead of storing anything from the forward pass.
    gamma1 and lambda2 are treated as constants."""

    @staticmethod
    def forward(ctx, B, eps, s, gamma1, lambda2, plan):
        sval = float(s)
        out = plan.energy(B, eps, gamma1, lambda2, sval)
        ctx.save_for_backward(B, eps)
        ctx.extra = (gamma1, lambda2, sval, plan)
        return out[4].clone()

    @staticmethod
    def backward(ctx, g):
        B, eps = ctx.saved_tensors
        gamma1, lambda2, sval, plan = ctx.extra
        _, dB, de, ds = plan.energy_grad(B, eps, gamma1, lambda2, sval)
        return g * dB, g * de, (g * ds[0]).reshape(()), None, None, None


def energy_total(plan, B, eps, s, gamma1=None, lambda2=None):
    """Differentiable E_total (see ``DSRGEnergy``); ``s`` may be a tensor."""
    if not isinstance(s, torch.Tensor):
        s = torch.tensor(float(s), dtype=torch.float64, device=B.device)
    return DSRGEnergy.apply(B, eps, s, gamma1, lambda2, plan)


def extra_to_device(problem, device="cuda"):
    """The optional (lambda3, f1) of a ``dsrg_synth.Problem`` as FP64 device tensors (or None)."""
    f = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float64).contiguous().to(device)
    return f(problem.lambda3), f(problem.f1)


def to_device(problem, device="cuda"):
    """Copy a ``dsrg_synth.Problem``'s arrays to FP64 device tensors (B, eps, gamma1, lambda2)."""
    f = lambda a: torch.as_tensor(a, dtype=torch.float64).contiguous().to(device)
    g = problem.gamma1 if problem.nactive else None
    lam = problem.lambda2 if problem.nactive else None
    return f(problem.B), f(problem.eps), (f(g) if g is not None else None), \
        (f(lam) if lam is not None else None)
