"""GB300-native peptide database search hot path (HiCOPS, superstep 3).

The compute path lives in the CUDA library ``libhicops.so`` (built in-tree by
``__graft_entry__.build()``); :mod:`.hicops` is its ctypes binding.
"""
