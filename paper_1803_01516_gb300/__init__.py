"""GB300-native exact min-cut for the gaze-line / depth-number stereo
formulation (Oguri & Shibata, "A new stereo formulation not using pixel and
disparity models").

The compute path is the C-ABI library ``libgazecut.so`` (CUDA, sm_103a),
bound by :mod:`paper_1803_01516_gb300.gazecut`.  Importing this package does
not load the library; the first call into :mod:`.gazecut` does, and fails
loudly if it has not been built.
"""
__version__ = "0.1.0"
