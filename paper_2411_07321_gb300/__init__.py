"""GB300 (sm_103a) w-stacking imaging: the hot path of RICK (De Rubeis et al.).

``rick``     -- ctypes binding of librick.so (the C ABI of include/rick.h)
``imager``   -- torch-facing resident state and stage order
``autograd`` -- torch.autograd.Functions (gridding <-> degridding adjoints)
``serve``    -- continuous-batching imaging server
``build``    -- compiles librick.so (importing it does not load the library)

Attributes load on first use, so ``paper_2411_07321_gb300.build`` works before
the library exists; every other use raises ImportError if librick.so is not
built -- there is no fallback path.
"""
import importlib

_LAZY = {"Imager": "imager", "IMAGE_FLAGS": "imager", "PREDICT_FLAGS": "imager",
         "grid_sparse_batch": "imager",
         "GridFn": "autograd", "DegridFn": "autograd", "Server": "serve"}
_SUBMODULES = ("rick", "imager", "autograd", "serve", "build")


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    if name in _LAZY:
        return getattr(importlib.import_module(f"{__name__}.{_LAZY[name]}"), name)
    raise AttributeError(name)
