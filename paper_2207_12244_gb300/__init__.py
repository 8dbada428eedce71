"""GB300-native (sm_103a) keyframe depth optimiser of DeepFusion (Section II-C).

The compute path is the CUDA library ``libdeepfusion.so`` (C ABI in
``include/deepfusion.h``); ``deepfusion`` is its thin Python binding and
``synth`` the seeded synthetic-input generator. Importing the package does not
load the library; the first call does, and fails loudly if it is missing.
"""
from . import deepfusion  # noqa: F401
from .deepfusion import *  # noqa: F401,F403
