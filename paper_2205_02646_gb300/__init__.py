"""GB300-native (sm_103a) RL-JSDE: reconstruction of three-quarter sampling
measurements with recurrent local joint sparse deconvolution and
extrapolation.

``rljsde`` binds the C ABI of ``include/rljsde.h`` (CUDA library
``librljsde.so``, built by ``build.py``); ``synth`` draws seeded synthetic
inputs.  Importing the package does not load the library.
"""
__all__ = ["rljsde", "synth", "build"]
