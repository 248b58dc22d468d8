"""Reference oracle for the sector-decomposition Monte-Carlo hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, independently written
CPU restatement of what the GPU path computes.  Only the test suite, the smoke
check in ``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  The product package never imports it and must
not fall back to it.

Contents, each module citing the part of the paper (A.V. Smirnov, "FIESTA 4:
optimized Feynman integral calculations with GPU support", arXiv:1511.03614)
it restates:

* ``uf``        Symanzik polynomials U, F from propagators (Eq. 2 "Alpha"; Sec. 4.3 ``UF``)
* ``sectors``   primary and iterated sector decomposition, pole subtraction and
                epsilon expansion (Sec. 1 and the program summary's "sector
                decomposition / pole resolution and epsilon expansion")
* ``prefactor`` Gamma-function prefactor series with (i pi^{d/2})^l e^{-l gamma eps}
                pulled out (Eq. 2; Sec. 4.3)
* ``philox``    Philox4x32-10 counter-based generator (Salmon et al., SC'11)
* ``sobol``     Sobol sequence from primitive polynomials (Bratley-Fox construction)
* ``vegas``     Lepage's VEGAS adaptive Monte Carlo (the default integrator, Sec. 4.4)
* ``quadrature`` tensor tanh-sinh rule for low-dimensional exact checks
* ``cuhre``     deterministic adaptive cubature (Genz-Malik rule, passes of region
                splitting): the Cuhre alternative among the integrators of Sec. 4.4
* ``pipeline``  end-to-end: units, integration, error combination (Sec. 4.3) and
                assembly with the prefactor.

Everything is float64 (numpy) or arbitrary precision (mpmath / exact rationals).
"""
