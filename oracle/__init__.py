"""Plain FP64 CPU oracle for the free-space Poisson method of Exl, arXiv:1612.01799.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The library's solve path never
imports, links or runs anything here, and nothing here imports the library: the two
share no code.  Inputs reach both sides as plain arrays from the seeded generators in
``paper_1612_01799_gb300.densities``, a module without any of the method's arithmetic.

The oracle takes the method's steps in the paper's order, slowly and in FP64:

* ``gauss_sum``  -- the Gaussian-sum approximation of 1/(4 pi r) by sinc quadrature
  (Sec. 2, eq. approx) and the near-zone radius delta (Sec. 3 heuristic).
* ``gtensor``    -- the per-axis factors of the G-tensor by adaptive Gauss-Kronrod
  quadrature (Sec. 2, G-tensor formula), the Taylor near-field constants C0 and C2
  (Sec. 2, correction integral I_delta) and the full padded symbol.
* ``fft``        -- the oracle's own FP64 mixed-radix Cooley-Tukey FFT (fft.c), used by
  every transform below; no library FFT is called.
* ``solver``     -- zero padding to (2N)^3, forward FFT, product with the symbol,
  inverse FFT, crop to N^3 (Sec. 2 and Sec. 3), with the correction either folded into
  the symbol or applied the paper's literal way through an N^3 FFT pair.
* ``direct``     -- the same discrete convolution evaluated in real space one output
  line at a time, for sampled outputs of grids too large for the FFT oracle and for
  brute force on tiny grids.
* ``box``        -- the same steps on a general rectangular box with n_q points per axis
  (Sec. 2 standardised form: lambda, l_q and the per-axis G-tensor factors), with the
  correction folded into the symbol or in the paper's literal order.
* ``exact``      -- closed-form potentials of the paper's test densities (Sec. 5) and of
  Gaussian sums, used to pin the oracle to something other than itself.

Readings of points the paper leaves open (grid offset, delta's units, the GS range,
the GS construction, epsilon from the tolerance, the normalisation) are stated in the
module that uses them.
"""
from . import box, direct, exact, fft, gauss_sum, gtensor, solver  # noqa: F401
