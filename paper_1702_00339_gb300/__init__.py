"""GB300-native lattice core-Hamiltonian eigensolver (libfock).

`paper_1702_00339_gb300.fock` is the Python binding of the C ABI in
include/fock.h; `paper_1702_00339_gb300.build` compiles the CUDA library
in-tree for sm_103a.
"""
