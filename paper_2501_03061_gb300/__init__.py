"""GB300 (sm_103a) library for the hot path of finite-temperature PT-IM rt-TDDFT with a hybrid
functional: occupation-weighted screened Fock exchange, its ACE compression, H·Psi and one
PT-IM(-ACE) time step.  The compute runs in libptim.so (C ABI in include/ptim.h); `api`
is its thin PyTorch binding and `synth` draws the seeded synthetic workloads.
"""
from __future__ import annotations

import importlib

__all__ = ["api", "synth", "build", "Context"]


def __getattr__(name):
    if name in ("api", "synth", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    if name == "Context":
        return importlib.import_module(f"{__name__}.api").Context
    raise AttributeError(name)
