"""CMRS (Compressed Multi-Row Storage) sparse matrix-vector product for GB300.

The compute path is the C-ABI library libcmrs.so (hand-written CUDA for
sm_103a, declared in include/cmrs.h).  `paper_1203_2946_gb300.binding` holds
the thin ctypes binding with the same entry-point names; it is imported lazily
so that the input generators (`paper_1203_2946_gb300.inputs`) load without a
GPU or a built library.
"""
import importlib

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name in ("binding", "inputs"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
