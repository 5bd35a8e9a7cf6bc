"""Plain FP64 CPU oracle for the HHO elasto-acoustic ERK scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never imports, links or calls it, and it imports
nothing from the GPU library.

What it computes (Mottier, Ern, Guillot, "Elasto-acoustic wave propagation in
geophysical media using hybrid high-order methods on general meshes"):

* ``mesh``      -- the mesh description of Sec. 3.1 (faces, face sets, normals)
                   plus the canonical numbering/colouring/class conventions.
* ``quadrature``-- exact polygon integrals of monomials (Green's theorem with
                   Gauss-Legendre on the edges) and a triangle-fan rule for
                   non-polynomial integrands.
* ``spaces``    -- the local scaled-monomial bases of Sec. 3.3.
* ``assemble``  -- the full non-condensed algebraic system (the block system
                   "algebraic_system" / compact form "compact_AR" of Sec. 3.3)
                   assembled from the defining integrals: mass (Eq. mass),
                   gradient reconstruction (Eq. rec), least-squares
                   stabilisation (Eq. stab), coupling and sources (Eq. rhs).
* ``erk``       -- the ERK tableaux (Eq. ERK) and the time step of Sec. 4.2
                   ("ERK_compact" with the face elimination "ex_solve"), done
                   with generic global sparse solves.
* ``sdirk``     -- the SDIRK tableaux (Eq. SDIRK) and the implicit step of
                   Sec. 4.1 (Eq. SDIRK_compact, Eq. cp_dirk) on the full
                   non-condensed system with a generic sparse LU.
* ``diagnostics`` -- discrete energy (Sec. 5.1), stabilisation dissipation,
                   sensor evaluation.

Everything is FP64.  Loops are plain Python over cells and faces; the only
library steps are numpy/scipy linear algebra (sparse LU, dense solves).

Parity status of each function is listed in the module docstrings; every
function is pinned by a ``-m "not gpu"`` test against a closed form, an
identity or a value printed in the paper.
"""
