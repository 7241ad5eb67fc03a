"""Plain FP64 CPU oracle for the deflated-CG hot path (test infrastructure).

This package is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the CUDA library and its Python binding) never imports,
links or calls anything here, and this package imports nothing from the
product path.

It follows the paper step by step, in numpy/scipy float64, with no blocking,
fusion or reordering beyond what the paper's definitions state:

* ``fem``     -- Q1 nodal discretisation of the pseudo-stress forms
                 (Section 2.3, Eq. component_form; Section 3.1 block structure;
                 Section 3.2.1 conforming forms), BSR pattern and values.
* ``mg``      -- multigrid for the inner Laplacian: Galerkin hierarchy
                 (Algorithm 2), RAS smoother (Section 4.2), W-cycle and the
                 multigrid driver (Algorithms 3 and 4).
* ``solvers`` -- plain CG and the flexible deflated CG (Section 4.1,
                 Eqs. x_defl / defl_sys / inner / fixed_tol / tol, Algorithms 1
                 and 2; truncation rule of the FCG remark in Section 5.1).
* ``timestep`` -- implicit Euler, Crank-Nicolson and BDF2 steps of Eq.
                 weak_IE (Section 2.3) and the pressure / velocity
                 reconstruction of Section 5.2.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, textbook identities, the matrices the paper prints for
d = 2 and d = 3, brute force on tiny meshes and dense direct solves. None is
"parity unpinned".
"""
from . import fem, mg, solvers, timestep  # noqa: F401
