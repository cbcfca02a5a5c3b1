"""GB300-native overlap-save variable-bandwidth filtering (HFSO coefficients).

The compute path is ``csrc/`` (CUDA for sm_103a plus the C-ABI host library ``libvbw.so``);
``vbw`` is the thin ctypes binding with the same names as the C entry points. Importing the
package loads nothing: the CUDA library is opened on first use and its absence is an error.
"""
__all__ = ["vbw", "workloads"]
