"""GB300-native (sm_103a) augmentation hot path of arXiv 1809.06839.

Importing the package loads nothing native; ``paper_1809_06839_gb300.alb``
loads the CUDA library (and fails loudly when it is missing).
"""
