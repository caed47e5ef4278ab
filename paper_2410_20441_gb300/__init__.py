"""GB300-native solver for the effective elastic stiffness of voxel images
(accelerated pseudo-transient method on a staggered grid).

* ``ce``        -- ctypes binding of the C-ABI library libce (include/ce.h)
* ``autograd``  -- torch.autograd.Function giving dJ/dK, dJ/dG per voxel
* ``images``    -- seeded synthetic images (inputs only)
* ``build``     -- nvcc build of libce.so for sm_103a

Submodules load lazily so that importing the input generators does not load
the CUDA library.
"""
import importlib

__all__ = ["ce", "autograd", "images", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
