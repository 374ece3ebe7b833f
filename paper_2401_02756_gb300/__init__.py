"""GB300-native A-Bruijn graph build from sequencing reads.

The compute path is the CUDA library ``libdbg.so`` (sm_103a) behind the C ABI
declared in ``include/dbg.h``; :mod:`.dbg` is its thin ctypes binding and
:mod:`.synth` makes seeded synthetic read sets.
"""
