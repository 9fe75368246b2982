"""GB300-native Nystrom solver for boundary integral equations with the
generalized Neumann kernel (Nasser's fast method, re-designed for sm_103a).

Submodules:
  domains  - seeded synthetic boundaries and right-hand sides (inputs only)
  gnk      - the Python binding of the C-ABI library libgnk (loaded lazily)
"""
__all__ = ["domains", "gnk"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
