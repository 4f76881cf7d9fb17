"""Experiment drivers that run the paper's simulations through the library (not part of the
importable library itself)."""
