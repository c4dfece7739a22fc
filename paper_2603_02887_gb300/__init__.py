"""GB300 (sm_103a) library for generalized non-exponential Gaussian splatting.

* ``paper_2603_02887_gb300.render`` -- ``Renderer`` and the differentiable ``render`` (torch autograd),
  over the C ABI of ``include/ngs.h`` implemented in ``csrc/`` (hand-written CUDA).
* ``paper_2603_02887_gb300.synth`` -- seeded synthetic scenes and cameras.
* ``paper_2603_02887_gb300.build`` -- in-tree build of ``_build/libngs.so``.

Importing the package does not load the CUDA library; ``render`` does, and fails loudly if it was not built.
"""
__all__ = ["build", "synth", "render"]
