"""CPU oracle for the DF/CD DSRG-MRPT2 second-order energy.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg use it. It shares no code with the CUDA library.

Two tiers, which share only the synthetic input generator:

* ``oracle.spinorb`` (tier 0, numpy): the spin-orbital energy of Table 1 taken
  literally, every term as one dense contraction over the full hole and
  particle spaces, with term F as the eight-index sum of Eq. (22); Table 2's
  F1-F8 taken literally as well. Tiny inputs only.
* ``oracle.dsrg`` (tier 1, PyTorch CPU FP64): the paper's algorithm. Diagram
  F1 by the pair loop of Eq. (23), F2 and F3 in spin-adapted form, the
  remaining terms (A-E, G-I, F4-F8) in spin orbitals on the small blocks that
  carry at least two active indices. Gradients come from autograd on the same
  code.

Readings of the paper that both tiers share are listed in the design notes
and restated in the module docstrings.
"""
