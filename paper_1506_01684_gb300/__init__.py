"""GB300 (sm_103a) implementation of the explicit time step of the grand-potential
phase-field model for ternary eutectic directional solidification (arXiv:1506.01684).

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/pf.h``);
``pf`` is its Python binding.  ``workloads`` holds the seeded synthetic inputs.
Attribute access such as ``paper_1506_01684_gb300.pf_create`` is forwarded to ``pf``.
"""
from importlib import import_module as _imp


def __getattr__(name):
    if name.startswith("pf_") or name in ("Simulation", "PfError", "params_from_dict", "use_torch_allocator"):
        return getattr(_imp(".pf", __name__), name)
    raise AttributeError(name)
