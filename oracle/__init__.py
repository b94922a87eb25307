"""FP64 CPU oracle of the HOPU convection hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything
in this package.  The GPU library never calls it and shares no code with it.

It is a plain, slow, vectorised-numpy restatement of the paper's convection
operator (Section 2.2 eq. "upwind"; Section 3.2 eq. "hopudefinition") on affine
simplices, written in FP64:

* ``fe``         reference element: collapsed Gauss-Jacobi quadrature, the
                 orthonormal Dubiner basis, facet bases, the interior moment space.
* ``mesh``       topology and affine geometry of a periodic simplicial mesh.
* ``hdiv``       the normal-continuous velocity space V_h (its degrees of freedom,
                 V_h -> L2 embedding, the averaging back-projection R of
                 Section 2.3, the transpose map, the canonical interpolant).
* ``convection`` the HOPU convection form in conservative and in the paper's
                 non-conservative form, the inverse mass, energy functionals.
* ``rk``         SSP-RK3 substeps (Shu-Osher) with the two wind rules.
* ``sampled``    the apply on sampled elements of a large mesh, evaluated on the
                 sub-mesh of their facet neighbourhood (pinned: equal to the full
                 apply on the sampled elements, bit for bit).

Parity status of every function is listed in its module docstring; functions
without an independent pin say "parity unpinned".
"""
