"""CPU oracle for the TT-SFFT Carr-Madan pricer -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the pricing path computes, written
from the paper (Hauck & Turkalj, "Classical Tensor Train and Quantum Fourier
Transform Approaches for Large-Scale Carr-Madan Option Pricing"):

  cf.py            characteristic functions of log(S_T/S0) and psi (Eq. psi)
  carr_madan.py    the discrete Carr-Madan sum: grids, integrand x_j (Eq. x and
                   the Simpson variant the paper allows after Eq.
                   discretization_dft), unitary DFT (Eq. dft) by three
                   independent routes, prices (Eq. discretization_dft), NRMSE
                   (Eq. error_measure), the QFT amplitude readout
                   (Eq. qft_observable_price)
  closed_forms.py  Black-Scholes (Eq. analytic_BS) and Merton's series
  tt.py            tensor-train toolkit on dense numpy arrays (Sec. 3.1):
                   TT-SVD, rounding, contraction, the bit-reversed DFT operator
                   Q_n of Sec. 3.2 written out densely
  mlp.py           the price surrogate's network (not in the paper): forward,
                   mean squared error, backpropagation, Adam, bfloat16 rounding

Only tests, the smoke check and the bench's CPU-baseline leg may import this
package. It shares no code with the CUDA path: the product never imports it and
it never imports the product. Inputs (problem parameters) come from the
separate seeded generator module; the oracle reads them by attribute name only.

Parity status: every function here is pinned by a CPU test against values the
paper prints, closed forms, library routines, invariants or brute force
(tests/test_oracle_*.py). There is no "parity unpinned" function.
"""
