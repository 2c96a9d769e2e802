"""GB300-native Acc-Sinkhorn: hand-written sm_103a CUDA kernels behind a C-ABI.

Import is lightweight: the CUDA library is loaded by ``binding`` on first use
and a missing library raises an error (there is no CPU fallback).
"""
__all__ = ["binding", "workloads"]
