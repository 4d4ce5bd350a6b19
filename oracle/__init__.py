"""CPU oracle for the lattice core-Hamiltonian eigenproblem (FP64, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this
package.  The product path (the C-ABI library and its Python binding) never
imports, calls or links anything here, and nothing here imports the
product.  The two share only the seeded input module `lattice_inputs`.

What it computes is the plain definition of the grid-discretised Galerkin
problem of Sec. 2 of the paper:

* `sinc`    - the R-term Gaussian-sum rule for 1/z (Sec. 2.2, Eqs. 2.6-2.7);
* `grid`    - nodes, nodal GTO vectors (Sec. 2.4), the P0 cell integrals
              of the shifted Gaussians and the lattice-summed potential
              tensor (Eqs. 2.8-2.13, Eq. 3.6), for a box either replicated
              from the central cell (reading R1, what the library computes)
              or the plain sum over the box's cells (reading R2, Sec. 2.3
              case (B));
* `dense`   - the dense N_b x N_b matrices H = A/2 - V and S (Eqs. 2.4-2.5,
              2.15-2.17, Lemma 2.1) by direct contractions over the 3D grid,
              and their dense generalized eigensolve;
* `blocks`  - generator blocks read off the dense matrices, the direct
              (non-FFT) DFT over the lattice index and per-block eigensolves
              (Lemma 3.1, Prop. A.1), the back-transform of block
              eigenvectors to the lattice and the real-space orbitals on the
              grid, the dense Toeplitz/box matvec;
* `closed_forms` - textbook Gaussian integrals and the exact cell integral
              of 1/|x|, used only to pin the grid quantities.

Every function is pinned by `tests/test_oracle_*.py` against closed forms,
invariants, brute force on tiny inputs or library routines.  The defect
kernel `dense.defect_matrix` is pinned through three independent routes:
a substituted single molecule equals a charge change, substituting every
cell of an odd periodic chain equals a charge change of the window-summed
lattice potential, and vacating every nucleus of a box cancels the box's
lattice-sum potential (itself pinned by brute force and the Boys-function
closed form).  What a defect means physically is a reading (R-DEF), not a
parity question.
"""
