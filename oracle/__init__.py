"""FP64 CPU oracle for the reduced-order Newton / FETI-DP lattice solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of the method in numpy/scipy, FP64
throughout, written from the paper's equations in the paper's order and notation:

  fe.py        Q1 shape functions and Gauss-Legendre rules on the reference cell
               (Section 3.1.5, Eq. fullquadraturerule; reduced rule of Eq. snapshots)
  material.py  neo-Hookean Cauchy stress (Eq. sig_eq), spatial elasticity tensor
               (Eq. const_eq) and the tensor D of Section 3.1.4
  cell.py      per-cell internal force (Eq. internalloadvec) and tangent K^s
               (Section 3.1.4, Eq. stiffmatPulledback), snapshot data() (Eq. snapshots)
  assembly.py  global residual (Eq. residualvector) and tangent (Section 3.1.4), Dirichlet split
  newton.py    Newton-Raphson with Armijo backtracking (Section 2.2.5, Eq. linsys), load stepping
  greedy.py    Algorithm 1 (principal cells) and the RB coefficients alpha (Section 3.2.2)
  rom.py       reduced local tangents and their action (Eq. romstiffnessmatrix)
  fetidp.py    the FETI-DP saddle-point system of Section 3.3.1, solved directly
  adjoint.py   adjoint gradient of end compliance w.r.t. per-cell shear-modulus factors
               (not in the paper: derived from the discrete equilibrium r_F(u, theta) = 0)

It shares no code with the GPU library; both read their inputs from ``latgen``.
Pins that tie each function to something other than itself live in ``tests/test_oracle_*.py``.
"""
