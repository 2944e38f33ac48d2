"""Exact Smith-Waterman/Gotoh protein database search on one GB300 (sm_103a).

Importing the package loads nothing native.  The CUDA library is loaded by
``paper_2309_09609_gb300.swgb`` on first use and fails loudly if it is missing.
"""
__version__ = "0.1.0"
