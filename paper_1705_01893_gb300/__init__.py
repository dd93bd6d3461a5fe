"""GB300-native messenger-field CMB mapmaker (Huffenberger & Naess, arXiv:1705.01893).

The solver runs in hand-written sm_103a CUDA kernels behind a C ABI (``include/mm.h``);
``paper_1705_01893_gb300.binding`` marshals torch tensors into it.  ``synth`` generates
seeded synthetic inputs.  Importing the package does not load the CUDA library.
"""
__all__ = ["binding", "synth"]
