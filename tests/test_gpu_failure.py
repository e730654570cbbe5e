"""The timeout path of the tensor-core kernels' bounded waits.

Every wait in those kernels (on TMA copies, MMAs and TMEM buffers) gives up after
about 2 s, records a status word and lets the kernel return, so that a lost
arrival shows up as DSRG_ERR_TIMEOUT on the host instead of a hung GPU. Here one
such wait is made to run out on purpose: the self-test entry point queues it on
a barrier that nothing completes. The host must read the timeout, the status
must clear, and the same plan must still compute the same energy afterwards.
"""
import time

import numpy as np
import pytest

from dsrg_synth import make_problem

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_timeout():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    from paper_1603_00561_gb300 import _native
    p = make_problem(3, 2, 70, 40, s=0.5, seed=50)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="bf16x3")
    dev = pk.to_device(p)
    before = plan.energy(*dev, p.s).cpu().numpy()
    lib = _native.load()
    assert lib.dsrg_plan_sync(plan.h) == _native.OK
    assert lib.dsrg_plan_selftest_wait_timeout(plan.h) == _native.OK
    t0 = time.time()
    assert lib.dsrg_plan_sync(plan.h) == _native.ERR_TIMEOUT
    assert time.time() - t0 >= 1.0  # the wait ran to its bound before giving up
    assert lib.dsrg_plan_sync(plan.h) == _native.OK  # the status was cleared
    after = plan.energy(*dev, p.s).cpu().numpy()
    assert np.array_equal(before, after)  # the context and the plan still work
    plan.close()
