"""GB300-native PPPM for the long-range Gaussian-charge electrostatics of DPLR
(arXiv 2504.15508).

The computation lives in ``libpppm.so`` (CUDA, sm_103a), built in-tree by
``paper_2504_15508_gb300.build.build()``; this package is a thin binding.
"""
from ._native import PPPMError, lib  # noqa: F401


def __getattr__(name):
    if name == "Plan":
        from .pppm import Plan
        return Plan
    raise AttributeError(name)
