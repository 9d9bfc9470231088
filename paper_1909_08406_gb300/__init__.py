"""GB300-native RD3Q41 energy-conserving lattice Boltzmann solver (arXiv:1909.08406).

The compute path is the CUDA library ``libgblb.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/gblb.h``; ``lb`` is its thin Python
binding.  Importing the package does not load the library; the first call
into ``lb`` does, and raises if the library is missing.
"""
__all__ = ["lb", "workloads"]
