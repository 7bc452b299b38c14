"""GB300-native executor for tensor-network contraction trees (arXiv 2002.01935).

Submodules:
  inputs   -- seeded synthetic networks (random circuits, Ising models)
  planner  -- host-side greedy tree, greedy slicer and cost model
  binding  -- ctypes binding of the C-ABI library ``libtn.so`` (CUDA, sm_103a)
  autograd -- torch.autograd.Function around the forward/backward calls

Importing the package does not load the CUDA library; ``binding`` does, and
raises if the library is missing.
"""
__all__ = ["inputs", "planner"]
