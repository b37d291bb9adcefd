"""GB300-native Cuckoo++ flow tables (Le Scouarnec, "Cuckoo++ Hash Tables:
High-Performance Hash Tables for Networking Applications", 2017).

``libckpp.so`` (CUDA, sm_103a) implements bulk lookup, insert, delete and the
expiration scan behind the C ABI of ``include/ckpp.h``; ``_ckpp`` binds it with
ctypes under the same names and ``FlowTable`` wraps one table. Importing
``FlowTable`` (or ``_ckpp``) loads the library and fails loudly if it is not
built. ``workload`` (synthetic 5-tuple traffic) needs neither CUDA nor the
library.
"""

__all__ = ["FlowTable", "workload", "build"]


def __getattr__(name):
    if name == "FlowTable":
        from .table import FlowTable
        return FlowTable
    raise AttributeError(name)
