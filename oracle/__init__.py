"""Plain FP64 CPU oracle of the HEVI 1D-IMEX step (Abdi, Giraldo et al., arXiv:1702.04316).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct reference that
the CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_1702_04316_gb300``) never imports it and shares no code with it.

Every function follows one passage of the paper, cited by section, equation label,
algorithm or table:

* ``lgl``        -- LGL nodes/weights and the nodal derivative matrix sD
                    (Sec. "Volume kernels", Algorithms 1-2).
* ``mesh``       -- box mesh, element-to-global map, direct stiffness summation
                    (Sec. "Direct stiffness summation"; column numbering of
                    Sec. "1D-IMEX kernels").
* ``reference``  -- constants, equation of state and hydrostatic reference state
                    (Sec. "Equation Set2NC"; sound speed of Sec. "Acoustic wave problem").
* ``rhs``        -- explicit right-hand side R(q) of the Set2NC perturbation equations,
                    element by element, then DSS (Sec. "Equation Set2NC",
                    Sec. "Spatial discretization", Algorithm 2).
* ``column``     -- the vertical operator L_V, the Schur-complement column operator,
                    its Jacobian by probing (Algorithm 7), banded LU without pivoting
                    (Algorithm 9), the solve and the extraction (Eqs. imex2nc, 2ncp,
                    utteqn, helm2nc; Algorithms 4-5).
* ``ark2``       -- the ARK2 double Butcher tableau (Table 1) and the SDIRK
                    predictor-corrector stage form (Sec. "Linear multi-stage methods").
* ``ark3``, ``ark4``, ``ark5`` -- the ARK3(2)4L[2]SA, ARK4(3)6L[2]SA and ARK5(4)8L[2]SA
                    tableaux for the paper's ARK3 - ARK5 runs, whose tableaux the paper
                    does not print (readings stated there); ``derive_ark5_row8`` re-derives
                    two entries of ARK5 from its order conditions.
* ``ark_order``  -- the bicoloured-tree order conditions of ARK pairs, exact arithmetic.
* ``rk35``       -- the explicit five-stage third-order SSP comparator
                    (Sec. "Performance of IMEX on manycore processors").
* ``schur3d``    -- 3D-IMEX in the Schur form: the 3D Schur operator and right-hand side,
                    the extraction (Eqs. utteqn, helm2nc with the full gradient), BiCGstab
                    with a polynomial preconditioner (Algorithm "BiCGstabPBNO"; Chebyshev
                    coefficients as the reading of PBNO) and the 3D-IMEX ARK2 integrator.
* ``tangent``    -- tangent-linear and adjoint models of R, of the column solve
                    (transposed stored LU of Algorithm 9) and of the ARK2 step, and the
                    gradient of a quadratic misfit of the final theta' (differentiation
                    form: the chain rule applied to the steps above).

Parity pins for every function live in ``tests/test_oracle_*.py``.  Four tableaux are
pinned only as methods of their order, not as the schemes the paper ran (which it does not
print): see the ``PARITY UNPINNED`` notes in ``rk35``, ``ark3``, ``ark4`` and ``ark5``.
"""
