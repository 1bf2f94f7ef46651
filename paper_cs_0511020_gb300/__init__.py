"""GB300-native Pbit: stable MSD bucket sort of singly-linked lists on the GPU.

The compute path is the C-ABI library ``libpbit.so`` (hand-written sm_103a
CUDA, built by ``__graft_entry__.build()``); ``paper_cs_0511020_gb300.pbit``
is a thin ctypes binding over it that takes torch device tensors and streams.
"""
__all__ = ["pbit", "inputs"]
