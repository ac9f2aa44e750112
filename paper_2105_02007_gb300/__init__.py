"""GB300-native multilevel quadrature for the stochastic monodomain equation.

The compute path lives in the CUDA library ``libmlq`` (``csrc/``), reached
through the thin ctypes binding in :mod:`paper_2105_02007_gb300.mlq`.  This
package file imports nothing heavy so that the seeded input generators in
:mod:`paper_2105_02007_gb300.inputs` can be used without a GPU.
"""
__all__ = ["inputs", "mlq"]
