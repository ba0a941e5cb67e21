"""Plain FP64 CPU oracle for the lattice Boltzmann model in generalized metrics.

Source: J.-D. Debus, M. Mendoza, H. J. Herrmann, "Dean Instability in
Double-Curved Channels" (arXiv:1411.3133), Sec. II (the LB method), Sec. III
(cylindrical channel) and Sec. IV (double-curved channel, ellipsoidal
coordinates).

This package is TEST INFRASTRUCTURE. It is slow on purpose and written to be
checked against the paper by eye: separate stream and collide passes, two
arrays, explicit tensor-index sums (numpy ``einsum`` over the Hermite tensors),
exact rational arithmetic for the wall rule, and Christoffel symbols computed
from their defining formula by automatic differentiation of the embedding.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and reference legs) may import it. It shares no code, table or
constant with the CUDA library, and it never imports it.

Modules
-------
lattice      D3Q41 velocity set and weights (Table I), Hermite tensors.
geometry     embeddings, metric, Christoffel symbols (Sec. III-IV).
lbm          streaming with walls, equilibrium, forcing, BGK step (Sec. II);
             the half-force velocity variant of the collision as a flag (not
             the paper's printed scheme).
diagnostics  Dean number, mean velocity, vorticity, mass (Sec. III-IV).
"""
