"""GB300-native real-space grid integration for numeric atom-centred orbitals.

Hamiltonian integration h_ij = sum_p w_p [phi_i v phi_j + 1/2 grad phi_i . grad phi_j] and
density update n_p = sum_ij phi_i P_ij phi_j (arXiv:1912.06636, Eq. H_int_aims and
Eq. Density) in hand-written sm_103a CUDA behind the C ABI of include/nao.h.
``nao`` is the thin binding, ``synth`` the seeded input generator.
"""
from . import nao  # noqa: F401
from .nao import Grid  # noqa: F401
