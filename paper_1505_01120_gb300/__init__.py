"""GB300-native SparkCL per-partition offload (Segal et al. 2015).

A partition's primitive arrays become device buffers, a catalogue kernel runs
over every element, and a reduction or keyed reduction folds the result
(MapCL / MapCLPartition / ReduceCL, Sec. 3.1.3).  The compute path is the
C-ABI library ``_lib/libscl.so`` (hand-written sm_103a CUDA + C++ runtime);
``scl`` is its ctypes binding and ``context`` a small helper that gives it a
PyTorch-owned arena.  ``synth`` draws the seeded synthetic partitions.

Importing the package does not load the library; ``import
paper_1505_01120_gb300.scl`` does, and fails loudly if it is not built.
"""

__all__ = ["scl", "context", "synth", "build"]
