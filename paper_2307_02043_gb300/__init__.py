"""GB300-native hot path of the mini-batch quasi-Newton proximal method (BQNPM)
for constrained-TV optical diffraction tomography.

The computation lives in libmqnpm (hand-written sm_103a CUDA behind a C ABI,
declared in include/mqnpm.h); :class:`MQNPM` is a thin ctypes binding and
:class:`LSGradient` wraps the data-term gradient as a torch.autograd.Function.
"""

__all__ = ["MQNPM", "MQNPMError", "NotConverged", "LSGradient", "build"]


def __getattr__(name):
    if name in ("MQNPM", "MQNPMError", "NotConverged"):
        from . import binding
        return getattr(binding, name)
    if name == "LSGradient":
        from .autograd import LSGradient
        return LSGradient
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
