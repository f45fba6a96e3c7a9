"""GB300-native bulk-parallel incremental graph connectivity.

Bulk-Update folds a minibatch of edges into a device-resident union-find
forest; Bulk-Query answers a minibatch of vertex-pair connectivity queries on
all edges seen so far (Section 1, "Model"; Algorithms 1 and 2). The work runs
in hand-written sm_103a kernels behind the C-ABI of ``include/cc.h``; the
Python classes here only marshal arguments (see ``cc.py``).

Importing the package loads nothing native; ``cc.load()`` (or the first use
of a ``Forest``) loads ``libcc.so`` and raises if it is missing.
"""
__all__ = ["Forest", "SegmentedForest", "CCError", "load"]


def __getattr__(name):
    if name in __all__:
        from . import cc
        return getattr(cc, name)
    raise AttributeError(name)
