"""KPA grouping path of StreamBox-HBM on B300 (sm_103a).

The kernels and the C ABI live in libsbh.so (sources in csrc/, header in
include/sbh.h); ``sbh`` is the Python binding (argument marshalling only).
Importing ``sbh`` (or any name it defines, from this package) loads
libsbh.so and raises ImportError when it is missing: there is no CPU
fallback.  ``build`` compiles it and does not load it.
"""


_SUBMODULES = ("build", "sbh", "pipeline", "serve", "autotune")


def __getattr__(name):
    import importlib

    if name.startswith("__") or (name in _SUBMODULES and name != "sbh"):
        # let the import system load submodules (build must work without the library)
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
    sbh = importlib.import_module(__name__ + ".sbh")  # raises ImportError when libsbh.so is missing
    if name == "sbh":
        return sbh
    try:
        return getattr(sbh, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
