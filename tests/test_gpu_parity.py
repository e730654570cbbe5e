"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar (FP64 path): every block within 1e-10 relative of the oracle. The energy
scale of the synthetic inputs is 1e3-1e7 Eh, so the 1e-10 Eh figure is read
as a relative bound; the absolute difference is printed too.
"""
import numpy as np
import pytest

from dsrg_synth import CONFIGS, make_problem
from oracle import dsrg as odsrg

pytestmark = pytest.mark.gpu

BLOCKS = ["ccvv", "cavv", "ccav", "active", "total"]
FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


def _gpu_blocks(pk, p, precision="fp64"):
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=precision)
    B, eps, g, l = pk.to_device(p)
    out = plan.energy(B, eps, g, l, p.s).cpu().numpy()
    assert plan.last_launch_count() > 0
    return dict(zip(BLOCKS, out)), plan, (B, eps, g, l)


def _oracle(p):
    return odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt,
                        with_pairs=True)


def _cmp(gpu, ref, tol, label=""):
    for k in BLOCKS:
        a, b = gpu[k], ref[k]
        err = abs(a - b)
        rel = err / max(abs(b), 1e-300)
        print(f"{label} {k:7s} gpu={a:+.15e} oracle={b:+.15e} |d|={err:.2e} rel={rel:.2e}")
        if b == 0.0:
            assert a == 0.0, k
        else:
            assert rel <= tol, (k, a, b, rel)


SMALL = [
    # (nC, nA, nV, Q, s, seed): ragged virtual tails (not multiples of 32/64), several tiles,
    # no active orbitals, one active orbital, the largest active space, a single core orbital
    (10, 4, 60, 200, 0.5, 0),
    (5, 2, 130, 77, 0.37, 1),
    (3, 0, 70, 41, 0.5, 2),
    (4, 1, 33, 50, 1.0, 3),
    (2, 8, 20, 30, 0.2, 4),
    (1, 3, 65, 17, 0.8, 5),
]


@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", SMALL)
def test_fp64_blocks_small(pkg, nC, nA, nV, Q, s, seed):
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed)
    gpu, plan, dev = _gpu_blocks(pkg, p)
    ref = _oracle(p)
    _cmp(gpu, ref, FP64_TOL, f"{nC}/{nA}/{nV}/{Q}")
    pairs = plan.pair_energies(dev[0], dev[1], p.s).cpu().numpy()
    np.testing.assert_allclose(pairs, ref["pairs"], rtol=1e-11, atol=1e-12 * np.abs(ref["pairs"]).max())


def test_fp64_tiny74_config(pkg):
    p = make_problem(**CONFIGS["tiny-74"])
    gpu, _, _ = _gpu_blocks(pkg, p)
    _cmp(gpu, _oracle(p), FP64_TOL, "tiny-74")


def test_fp64_naphthyne_vtz_config(pkg):
    """The cc-pVTZ-sized instance (nC=24, nA=2, nV=372, naux=1200), all blocks."""
    p = make_problem(**CONFIGS["naphthyne-vtz-398"])
    gpu, _, _ = _gpu_blocks(pkg, p)
    _cmp(gpu, _oracle(p), FP64_TOL, "vtz")


def test_fp64_v5z_sampled_pairs(pkg):
    """Quintuple-zeta size (nV=1214, naux=3400): pair energies the oracle computes
    one by one, including the first/last pairs and a diagonal pair."""
    p = make_problem(**CONFIGS["naphthyne-v5z-1240"])
    import paper_1603_00561_gb300 as pk
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux)
    B, eps, g, l = pk.to_device(p)
    pairs = plan.pair_energies(B, eps, p.s).cpu().numpy()
    sample = [(0, 0), (0, 23), (23, 23), (5, 17), (17, 5), (11, 12)]
    ref = odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt, pairs=sample).numpy()
    for (m, n) in sample:
        rel = abs(pairs[m, n] - ref[m, n]) / abs(ref[m, n])
        print(m, n, pairs[m, n], ref[m, n], rel)
        assert rel <= FP64_TOL


def test_s_zero_is_exactly_zero(pkg):
    p = make_problem(4, 2, 40, 30, s=0.0, seed=7)
    gpu, _, _ = _gpu_blocks(pkg, p)
    for k in BLOCKS:
        assert gpu[k] == 0.0, k


def test_power_of_two_scaling_bitwise(pkg):
    p = make_problem(5, 2, 70, 40, s=0.5, seed=8)
    g1, _, _ = _gpu_blocks(pkg, p)
    g2, _, _ = _gpu_blocks(pkg, p.scaled(2.0))
    for k in BLOCKS:
        assert g2[k] == 16.0 * g1[k], k


def test_deterministic_repeat(pkg):
    p = make_problem(6, 3, 90, 50, s=0.5, seed=9)
    plan = pkg.Plan(p.ncore, p.nactive, p.nvirt, p.naux)
    dev = pkg.to_device(p)
    a = plan.energy(*dev, p.s).cpu().numpy()
    b = plan.energy(*dev, p.s).cpu().numpy()
    assert np.array_equal(a, b)


def test_host_io_entry_matches_device_entry(pkg):
    p = make_problem(4, 2, 50, 40, s=0.5, seed=10)
    plan = pkg.Plan(p.ncore, p.nactive, p.nvirt, p.naux, host_io=True)
    dev = pkg.to_device(p)
    a = plan.energy(*dev, p.s).cpu().numpy()
    b = plan.energy_host(p.B, p.eps, p.gamma1, p.lambda2, p.s)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec,nC,nV,Q", [("bf16x3", 5, 140, 70), ("bf16x3", 12, 298, 4000),
                                          ("tf32x3", 24, 600, 2000), ("fp64", 5, 140, 70)])
def test_host_io_entry_pinned_matches_device_entry(pkg, prec, nC, nV, Q):
    """Page-locked host inputs: split plans copy B in groups of core rows while
    the CCVV work of the groups already copied runs (one group for the small
    case; three and five for the larger two, whose copy time is comparable to
    their CCVV time); FP64 plans copy it whole. Either way the result equals the
    device entry's bit for bit, call after call."""
    import torch
    p = make_problem(nC, 2, nV, Q, s=0.5, seed=12)
    plan = pkg.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, host_io=True)
    dev = pkg.to_device(p)
    a = plan.energy(*dev, p.s).cpu().numpy()
    pinned = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
              for x in (p.B, p.eps, p.gamma1, p.lambda2)]
    out = torch.zeros(5, dtype=torch.float64).pin_memory()
    for _ in range(2):
        out.zero_()
        plan.energy_host(*pinned, p.s, out=out)
        assert np.array_equal(a, out.numpy())


def test_error_statuses(pkg):
    import torch
    from paper_1603_00561_gb300 import _native
    p = make_problem(3, 2, 20, 10, s=0.5, seed=11)
    plan = pkg.Plan(p.ncore, p.nactive, p.nvirt, p.naux)
    B, eps, g, l = pkg.to_device(p)
    with pytest.raises(pkg.DSRGError) as ei:
        plan.energy(B, eps, g, l, float("nan"))
    assert ei.value.status == _native.ERR_NONFINITE
    with pytest.raises(pkg.DSRGError) as ei:
        plan.energy(B, eps, g, l, -1.0)
    assert ei.value.status == _native.ERR_INVALID_ARG
    with pytest.raises(pkg.DSRGError) as ei:
        plan.energy(B, eps, None, None, 0.5)
    assert ei.value.status == _native.ERR_INVALID_ARG
    # host-IO entry on a plan without staging
    with pytest.raises(pkg.DSRGError):
        plan.energy_host(p.B, p.eps, p.gamma1, p.lambda2, 0.5)
    plan.sync()


def test_allocation_failure_is_reported(pkg, monkeypatch):
    from paper_1603_00561_gb300 import _native
    monkeypatch.setenv("DSRG_FAIL_ALLOC_AFTER", "3")
    with pytest.raises(pkg.DSRGError) as ei:
        pkg.Plan(3, 2, 20, 10)
    assert ei.value.status == _native.ERR_OOM


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_energy_call_captures_into_a_cuda_graph(pkg, prec):
    """An energy call neither allocates nor synchronises, so it can be captured
    into a CUDA graph by the caller and replayed: the replay gives the same
    numbers bit for bit."""
    import torch
    p = make_problem(6, 2, 150, 90, s=0.5, seed=40)
    plan = pkg.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec)
    dev = pkg.to_device(p)
    out = plan.energy(*dev, p.s)          # first call outside the capture
    torch.cuda.synchronize()
    ref = out.clone()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.energy(*dev, p.s, out=out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.sync()
