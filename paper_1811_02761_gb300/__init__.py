"""GB300 (sm_103a) gravitational octree force library.

The compute path is the CUDA library libnbody.so (csrc/, C ABI in
include/nbody.h); ``nbody`` is its thin ctypes binding.
"""
from . import nbody  # noqa: F401
from .nbody import *  # noqa: F401,F403

__all__ = [n for n in dir(nbody) if n.startswith("nbody_")] + [
    "Config", "Stats", "NbodyError", "load", "library_path"]


def build(force: bool = False) -> str:
    """Compile libnbody.so for sm_103a (nvcc) and return its path."""
    from . import _build
    return _build.build(force=force)
