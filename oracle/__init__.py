"""Plain FP64 CPU oracle for the layered-media Helmholtz FMM (Wang, Zhang & Cai).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.  It shares no
code with the CUDA library; the two meet only through the seeded input
generators, which hold none of the method's arithmetic.

Modules
-------
specfun   normalized associated Legendre functions on C with the branch of
          Sec. 2.2 (eq. branch), spherical harmonics, spherical Bessel and
          cylindrical Bessel functions (thin wrappers of scipy).
media     layered medium, layer classification, reaction densities sigma
          obtained by imposing the transmission conditions (Sec. 3.1).
green     Sommerfeld-integral evaluation of the layered Green's function on
          the oracle's own contour (semi-ellipse + real tail), reaction
          components, equivalent polarization sources, direct sum.
gaunt     Wigner 3-j symbols (Racah's formula, exact integers) and Gaunt
          coefficients (Sec. 2.1).
fmm       adaptive octree and interaction lists, free-space and reaction
          expansions/translations and the full FMM of Algorithm 1.

Every function with no independent pin says "parity unpinned" in its
docstring; all others are pinned by tests under ``tests/test_oracle_*.py``.
"""
