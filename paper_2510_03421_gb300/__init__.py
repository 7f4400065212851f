"""GB300 permanent library: Glynn / Ryser Gray-code sweeps, the combinatoric
algorithm, a batched launcher and a learned dispatcher, behind the C ABI of
``include/perm.h``.  ``capi`` is the ctypes binding; ``inputs`` holds the seeded
workload generators."""

__all__ = ["capi", "inputs", "perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto", "perm_batched",
           "perm_glynn_partial"]


def __getattr__(name):
    if name in ("perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto", "perm_batched",
                "perm_glynn_partial"):
        from . import capi
        return getattr(capi, name)
    raise AttributeError(name)
