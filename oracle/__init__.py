"""Plain CPU oracle for the NDSGLFT of Wuelker, arXiv:1809.10786.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA implementation and never calls it.

* :mod:`oracle.direct` (C, ``sgl_oracle.c``): the definition of the transform,
  ``f = Lambda fhat`` (Def. of the NDSGLFT, Sect. 1), its adjoint and its point
  gradient, by direct summation of ``H_nlm`` from three-term recurrences.
* :mod:`oracle.factorization` (numpy): the paper's exact factorization of
  ``Lambda`` (Sect. 6, Thm. on the factorization) up to the trigonometric
  coefficients ``eta``, plus the NDFT that evaluates them (Sect. 2).
* :mod:`oracle.nfft` (numpy): the NFFT of Sect. 2 (deconvolution, oversampled
  inverse FFT, windowed sum) and the Gaussian error bound of its Thm. on the
  d-dimensional error.
"""
