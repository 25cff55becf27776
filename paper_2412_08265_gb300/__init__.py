"""GB300-native (sm_103a) particle -> IFU data-cube forward model of RUBIX
(arXiv 2412.08265): C-ABI CUDA library + thin Python binding.

Submodules:
  capi   -- ctypes binding with the C names of include/rubix.h
  model  -- CubeModel (torch device memory/streams) and RubixCube (autograd)
  synth  -- seeded synthetic galaxies, SSP grids and telescopes
  build  -- nvcc build of the in-tree shared library
"""
__all__ = ["capi", "model", "synth", "build"]


def __getattr__(name):
    if name in ("CubeModel", "RubixCube"):
        from . import model
        return getattr(model, name)
    raise AttributeError(name)
