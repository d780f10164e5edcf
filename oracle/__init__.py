"""Plain, slow, dense FP64 CPU oracle for the symmetric CTMRG hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this code; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
path: the two meet only in the seeded input recipes of ``workloads``.

What it computes is the plain definition of the method (Sec. 2, Eqs. 1-2 and
the contraction rule that follows them): every symmetric tensor is expanded
to a dense array whose entries outside the symmetry-allowed blocks are
exactly zero; contractions are dense ``numpy.einsum`` in FP64; the projector
SVD runs per conserved-charge sector of the dense half-system product.

Modules
  u1   -- U(1) legs, canonical block layout, dense expansion, leg fusion,
          double layer and remover (Sec. 2, Sec. 3.1, Sec. 3.2)
  ctm  -- the directional CTMRG move with SVD projectors (Sec. 3) and the
          four-direction move
  su2  -- exact Clebsch-Gordan coefficients and SU(2) dense expansion
"""
