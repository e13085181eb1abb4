"""GB300-native batched word-RASP engine.

The compute path is the C-ABI library ``librasp_gb300.so`` built from
``csrc/`` (CUDA for sm_103a); ``rasp`` is its thin ctypes binding. Importing
this package loads nothing: the library is opened on first use, and every
call fails loudly if it has not been built.
"""
__all__ = ["rasp", "workloads", "dsl", "serving"]
