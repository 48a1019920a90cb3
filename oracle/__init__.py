"""FP64 CPU oracle for LO matrix-element parameter reweighting.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (the CUDA library and its Python binding) never imports,
links or executes anything here, and nothing here imports the product.

What it computes (paper Sec. 3, the weight factorisation w' = w |M'|^2/|M|^2,
and the teaRex normaliser convention that maps 1/0 to 0): for every event and
every parameter point, the spin- and colour-summed, initial-state averaged
tree-level |M|^2, evaluated from Feynman rules in the most literal way:

* ``lorentz``: explicit 4x4 Dirac matrices in the chiral basis, helicity
  spinors u, v built as sqrt(p.sigma) xi, polarisation vectors of definite
  helicity (Peskin & Schroeder, Ch. 3 and 5).
* ``colour``: explicit Gell-Mann matrices and structure constants.
* ``qcd``: every tree-level Feynman diagram of g g -> t t~ + n g (n = 0, 1, 2)
  is enumerated, each diagram is evaluated with the textbook QCD vertices and
  propagators, and the colour sum is taken over explicit colour indices
  through the diagram-level colour matrix  G_{dd'} = sum_colours K_d^* K_d'.
* ``ee``: e+ e- -> mu+ mu- through photon and Z exchange.
* ``reweight``: the ratio epilogue.

Parity status: every function here is pinned by the tests in
``tests/test_oracle_*.py`` (closed forms, Parke-Taylor amplitudes, gauge,
Lorentz and Bose invariance, exact coupling scaling, diagram counts).
"""
