"""GB300-native (sm_103a) domain-decomposition parabolic Monge-Ampere mesh
generator (Sulman, Nguyen, Haynes & Huang).

The compute path is the CUDA library ``libpma`` behind the C ABI declared in
``include/pma.h``; ``paper_2006_14602_gb300.pma`` is its thin ctypes binding.
Importing the package itself loads nothing, so the seeded input module
(``workloads``) can be used without a GPU.
"""
__all__ = ["workloads", "pma"]
