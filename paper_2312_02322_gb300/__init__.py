"""GB300-native MQCT trajectory library (arXiv 2312.02322 hot path).

The compute lives in the CUDA library built from ``csrc/`` (C ABI: include/mqct.h);
``api`` is its Python binding, ``inputs`` the seeded synthetic workloads.  The binding
is imported lazily so that the workload generator needs no built library.
"""
from importlib import import_module

__all__ = ["api", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        return import_module(f".{name}", __name__)
    raise AttributeError(name)
