"""CPU oracle for the Nekbone AX solve path (plain FP64; numpy + plain C).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call or link anything in this
package.  It shares no code with the CUDA library, and the CUDA library never
imports it.

Parity status of each function (what pins it, beyond itself, lives in
``tests/test_oracle_*.py``):

* ``gll``              pinned: weight sum, quadrature exactness, derivative of monomials, textbook nx=2,3
* ``geom``             pinned: axis-aligned closed form, energy identity on affine elements
* ``ax``               pinned: constants in the kernel, symmetry, energy identity, dense brute force,
                       Kronecker form on boxes, paper's operation counts
* ``gs_build``/``dssum`` pinned: pure-Python grouping, multiplicity counts of the lattice
* ``jacobi_minv``      pinned: diagonal of the dense assembled matrix
* ``pcg``              pinned: dense direct solve, one-unknown and no-unknown special cases
"""
