"""The allocation-free CCVV entry point (dsrg_ccvv_energy_noalloc).

It is meant for callers that cannot allocate device memory (code running
inside someone else's memory pool, hosts that forbid allocation on their hot
path). It must give the same E_CCVV as the plan-based FP64 path, call after
call, with its scratch held in a fixed device array inside the library.
This file is collected last so that a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from dsrg_synth import make_problem

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 bar of the parity tests (relative)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    from paper_1603_00561_gb300 import _native
    pk.build()
    return pk, _native, _native.load(), torch


def _noalloc(native, lib, torch, p, B, eps, out):
    sz = native.Sizes(p.ncore, p.nactive, p.nvirt, p.naux)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.dsrg_ccvv_energy_noalloc(ctypes.byref(sz), ctypes.c_void_p(B.data_ptr()),
                                        ctypes.c_void_p(eps.data_ptr()), p.s,
                                        ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_plan_path_twice(env):
    pk, native, lib, torch = env
    # two problems of different size, each called twice in a row: the second
    # call reuses the scratch left behind by the first
    for (nC, nA, nV, Q, s, seed) in [(6, 2, 130, 90, 0.5, 21), (3, 1, 70, 41, 0.8, 22)]:
        p = make_problem(nC, nA, nV, Q, s=s, seed=seed)
        B, eps, g, l = pk.to_device(p)
        plan = pk.Plan(nC, nA, nV, Q, precision="fp64")
        ref = float(plan.energy(B, eps, g, l, p.s)[0])
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):
            assert _noalloc(native, lib, torch, p, B, eps, out) == native.OK
            torch.cuda.synchronize()
            val = float(out[0])
            assert abs(val - ref) <= TOL * abs(ref), (val, ref)
            out.fill_(float("nan"))


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    pk, native, lib, torch = env
    p = make_problem(200, 0, 10, 4, s=0.5, seed=23)   # 20100 core pairs > 8192
    B, eps, _, _ = pk.to_device(p)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(native, lib, torch, p, B, eps, out) == native.ERR_UNSUPPORTED
