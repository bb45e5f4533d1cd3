"""Plain FP64 CPU oracle for the stochastic Galerkin (SG) finite-difference
Helmholtz system of Pulch & Sete, "The Helmholtz equation with uncertainties
in the wavenumber" (2022).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run it.  The CUDA product path never calls
into it, and it never calls into the product path: the two share no code.

What it computes, and where the paper defines it:

* ``pc``      -- orthonormal Legendre chaos basis, multi-indices of total degree
                 <= r (Sec. 2.3), Galerkin triple products <xi_l phi_i phi_j>,
                 <xi_l xi_l' phi_i phi_j> (Lemma 3.2, Lemma A.3).
* ``fd``      -- finite-difference matrices of Theorems A.1, A.2, A.5, A.6,
                 point sources (App. A.3) and the mesh rule of Sec. 6.
* ``sg``      -- the explicit Kronecker SG matrix A = I (x) L - i[B_ij] - [C_ij]
                 (Theorem 3.4 with Theorems A.2/A.6), the right-hand side
                 b = e_0 (x) b_0, the mean-value matrix A_0 = I (x) S(xi_bar)
                 (Sec. 5), the CSL matrices M = A - i beta K and M_0 (Sec. 4,
                 Sec. 6.3).
* ``krylov``  -- restarted GMRES with right or left preconditioning, classical
                 Gram-Schmidt applied twice and complex Givens rotations
                 (Sec. 6.3), the stationary iteration of Sec. 5, direct
                 sparse solves (SuperLU), block preconditioners applied to all
                 P modes with one factorisation (Sec. 6.3 reshape).

Everything is FP64 / complex128.  Nothing here is blocked, fused or
reordered beyond what the paper's definitions state.

Parity status per function is recorded in each module header; functions
without an external pin say "parity unpinned".
"""
