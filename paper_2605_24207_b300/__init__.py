"""relnn-b300: B300-native evaluation of RelaNN rules over embedded relations.

The compute path is the C-ABI library ``librelnn.so`` (hand-written sm_103a CUDA kernels);
``relnn`` is its thin Python binding. PyTorch is used for device memory and streams only.
"""
__all__ = ["relnn", "workloads"]
