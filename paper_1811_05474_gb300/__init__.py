"""GB300-native mass-transfer particle tracking (arXiv 1811.05474).

The compute path is the CUDA library ``libmt`` (C ABI in ``include/mt.h``);
``paper_1811_05474_gb300.mt`` is its thin ctypes binding.  Importing this
package loads nothing; the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["mt", "synth"]
