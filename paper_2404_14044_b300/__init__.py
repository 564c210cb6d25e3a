"""B300-native (sm_103a) HashPoint point-search-and-sample hot path.

Submodules are imported lazily: ``scenes`` (seeded input generators) needs no
GPU and no compiled code; ``hashpoint`` binds the C-ABI library
``libhashpoint.so`` and fails loudly if it is missing.
"""
__all__ = ["scenes", "hashpoint"]
