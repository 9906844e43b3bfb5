"""Buffered fork-processing of many single-source graph queries on one GB300.

Importing the package loads nothing native; :mod:`paper_2103_14915_gb300.fg`
loads the CUDA library on first use and raises if it is missing.
"""
