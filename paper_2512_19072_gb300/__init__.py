"""FOT on GB300: the separable entropic dual-potential iteration of Torchylo et al.
("A fast, large-scale optimal transport algorithm for holographic beam shaping"),
as hand-written sm_103a CUDA kernels behind a C ABI (include/fot.h).

Importing the package loads nothing; `paper_2512_19072_gb300.binding` loads the
compiled library and fails loudly when it is missing.
"""
__all__ = ["binding", "inputs"]
