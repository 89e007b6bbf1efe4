"""Plain, slow FP64 CPU oracle for the Riesz-map solvers of Brubeck & Farrell,
"Multigrid solvers for the de Rham complex with optimal complexity in
polynomial degree" (arXiv 2211.14284).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only tests/, __graft_entry__.smoke() and the bench's
CPU-baseline leg use it.  It shares no code with the CUDA path; the two meet
only through the seeded input generators in paper_2211_14284_gb300/inputs.py.

Modules
-------
basis          1D FDM basis (Sec. 2.2-2.3, Eqs. fdmbasis, fdmdualbasis, eigs)
discretization tensor-product spaces, lattice numbering, element matrices by
               full-tensor quadrature, assembly (Sec. 2.4, 3.1, Eq.
               common_weak_formulation)
auxiliary      sparse auxiliary operator P (Sec. 3.2, Eq.
               sum-factorization_approx)
relaxation     stars, patches, static condensation, Cholesky / ICC(0),
               coarse space, additive and hybrid compositions (Sec. 4)
krylov         PCG and flexible CG (Sec. 5.1)

Every function cites the passage it follows.  Parity status of each function
is listed in the module docstrings; functions without an independent pin say
"parity unpinned".
"""
