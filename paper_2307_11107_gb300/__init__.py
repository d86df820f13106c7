"""GB300 (sm_103a) implementation of the APIC particle-in-cell step
(Smirnov & Krasheninnikov, arXiv:2307.11107) behind the C ABI of include/apic.h.

`Sim` is the thin Python binding; `build()` compiles libapic.so in-tree.
"""
from ._abi import (EXPLICIT, FLUX_SURFACE, FP32_REFINED, FP64, LOAD_VOLUME, NH, NO_FIELD, NO_INJECT, NT,
                   SYMBOLS, load)
from .build import build
from .sim import ApicError, Sim, make_config, probe_fp32_fma


def __getattr__(name):
    # the torch.autograd binding is loaded on first use
    if name == "AdjointWindow":
        from .autograd import AdjointWindow
        return AdjointWindow
    raise AttributeError(name)


__all__ = ["Sim", "ApicError", "make_config", "probe_fp32_fma", "AdjointWindow", "build", "load", "SYMBOLS", "FP64", "FP32_REFINED",
           "LOAD_VOLUME", "FLUX_SURFACE", "EXPLICIT", "NO_INJECT", "NO_FIELD", "NT", "NH"]
