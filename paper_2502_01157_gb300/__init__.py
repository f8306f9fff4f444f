"""GB300-native differentiable ray tracing through a 3D Voronoi foam
(Radiant Foam, arXiv 2502.01157).

Submodules are imported lazily so that the input generators
(:mod:`.scenes`) can be used without the CUDA library.
"""
__all__ = ["scenes", "rf"]


def __getattr__(name):
    import importlib
    if name in ("scenes", "rf", "serve"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
