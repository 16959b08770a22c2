"""Plain, slow, obviously-correct FP64 CPU oracle for tree-level |M|^2.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and this package imports nothing from
the product.

What it computes (Hagiwara et al., arXiv:1305.0708, Sect. 2, Eqs. 4-6): for
every phase-space point the spin- and colour-summed squared amplitude,
averaged over the initial helicities (1/4) and colours (1/(n_a n_b)),

    |M|^2_avg = 1/(4 n_a n_b) * sum_lambda sum_c | sum_diagrams M |^2 .

How: textbook Feynman rules written with explicit 4x4 chiral-basis gamma
matrices (numpy, vectorised over events), helicity spinors and polarisation
vectors from their definitions, and colour summed by brute force over
explicit SU(3) generator components.  The six-gluon process uses the
colour-ordered Berends-Giele recursion for the partial amplitudes and a
colour matrix summed by brute force over explicit generators.  Phase space:
Philox4x64-10 (Salmon et al., SC'11), RAMBO (Kleiss, Stirling, Ellis 1986),
two-body decay chains with the Breit-Wigner mapping of Eq. 16 / App. A.2.
Adaptive integration: VEGAS (Lepage 1978) grids over the generators' uniform
variables (vegas.py), the role of the BASES / gBASES integrator of Sect. 6.

Parity status per function is given in each module header.
"""
