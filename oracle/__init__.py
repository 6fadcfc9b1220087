"""FP64 CPU oracle for spectral Gaussian-random-field synthesis.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes anything in this directory; only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use it.  It shares
no code with the CUDA library: it has its own counter-based generator, its own
mode drawing, its own field sum, maps and adjoint.

What it computes (Icardi et al., arXiv 2212.10961):

* Sec. 4.1, Eq. (DiscreteFT): the field is a finite sum of N cosine modes
  evaluated directly at every cell centre, with no FFT.
* Sec. 4.1 (anisotropic rescaling): per-axis correlation lengths rescale the
  frequency space.
* Appendix A, Eqs. (gauSpe), (expSpe), (matSpe): covariance functions and
  their spectral densities, from which the wave-vectors are drawn.
* Sec. 3.1 and Appendix B: lognormal scaling and the single truncation rule
  (facies thresholds).

The readings taken where the paper is silent or garbled are written at the
top of each module.  Modules:

``philox``   Philox4x32-10 counter-based generator, uniforms, Box-Muller.
``spectra``  Covariance functions and spectral densities of Appendix A.
``modes``    Drawing the mode set (wave-vectors, amplitudes, phases).
``field``    The field sum, property maps, loss and adjoint (numpy, FP64).
``native``   The same field sum and adjoint as plain C + OpenMP (FP64), for
             sizes numpy cannot finish quickly and for the CPU baseline.
"""
