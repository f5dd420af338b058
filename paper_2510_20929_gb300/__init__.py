"""GB300-native LSQML ptychography hot path (Pty-Chi, arXiv 2510.20929).

The compute path lives in the C-ABI library ``libptycho.so`` (sm_103a CUDA,
built by ``__graft_entry__.build()``); :mod:`.api` is a thin ctypes binding to
it and :mod:`.synth` makes seeded synthetic inputs. Importing this package does
not load the library; the first call into :mod:`.api` does, and fails loudly if
the library is missing.
"""
__all__ = ["api", "synth"]
