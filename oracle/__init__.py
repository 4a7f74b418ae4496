"""FP64 CPU oracle for the Dirac quantum walk (D'Ariano, Mosco, Perinotti, Tosini,
"Discrete Time Dirac Quantum Walk in 3+1 Dimensions", Entropy 2016, arXiv:1603.06442).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, table or
constant with the CUDA library: every transition matrix here is re-derived
numerically from the paper's Fourier symbols.

Plain, slow, obviously correct numpy in complex128:

* ``walk``        -- symbols (Eqs. weyl1d/weyl2d/weyl3d, the Dirac coupling of
                     Sec. 3.2), transition matrices as Fourier coefficients of the
                     symbol (Eq. walk-K), the update rule (Eq. upd-rule), layouts.
* ``spectral``    -- naive DFT, and U^t psi through the DFT with a per-k matrix
                     power (Sec. 4; the plain definition, no closed form).
* ``observables`` -- norm, mean position (Sec. 5.2, operator X), position
                     covariance, probability projections (Sec. 5.2), particle and
                     antiparticle weights (spectral projector of U_k).
* ``kinematics``  -- drift v = grad omega and diffusion D = grad grad omega of
                     particle states (Sec. 5.1, second-order dispersive equation).
* ``states``      -- the paper's eigenvector formulas (Eqs. evecs-W, evecs-D) and
                     particle-state packets (Definition 1, Eq. state-zitter).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
facts the paper and the mathematics fix (unitarity, dense spectra, special
cases, closed forms, small-k limit, Zitterbewegung).  No function is unpinned.
"""

from . import walk, spectral, observables, states, kinematics  # noqa: F401
