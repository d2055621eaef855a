"""FP64 CPU oracle for the batched time-domain LISA log-likelihood.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
numpy restatement of what the GPU library computes, written from the paper
(arXiv:2501.08261, "GPU-accelerated LISA parameter estimation with full time
domain response").  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2501_08261_gb300``) never imports, links or runs
anything here, and this package shares no code, tables or constants with the
CUDA sources.

Module map (paper section / equation each follows):

* ``consts``     physical constants and the declared stand-in constants.
* ``orbits``     spacecraft positions and link light times (Sec. II.B, text
                 before Eq. (yslr)); rigid equal-arm and Keplerian models.
* ``waveform``   declared stand-in for the IMRPhenomT(HM) modes (Sec. II.A)
                 and the two-step twist-up of the precessing sector (Sec. II.A,
                 the three displayed equations before Eq. (newtwistup)).
* ``wigner``     Wigner small-d / D matrices and spin-weighted spherical
                 harmonics (textbook definitions used by the two-step form).
* ``response``   Lagrange fractional-delay interpolation, the link response
                 y_slr (Eq. yslr), TDI X 1.5 / 2.0, Y/Z by cyclic permutation,
                 A,E,T (Sec. II.B).
* ``likelihood`` DFT, Sangria PSD, matched-filter inner product and logL
                 (Sec. II.B, end).
* ``pipeline``   parameters -> A,E,T -> logL for one walker.
* ``heterodyne`` the heterodyned time-domain likelihood (the speed-up route
                 the paper names in Sec. I and Sec. IV, defined in the module):
                 analytic mode polarisations, the continuous-time response at
                 nodes, fiducial carriers and the interpolated model.
* ``sampler``    Fisher matrix by central differences of logL, the
                 Fisher-Gaussian proposal, the Metropolis-Hastings step and
                 tempered replica exchange (Sec. II.C).
* ``flow``       the affine-coupling flow of the learned proposal (forward,
                 inverse, log q, gradients, Adam), with the kernels' bf16
                 operand rounding as an option.
* ``noise``      coloured Gaussian noise with the likelihood's PSDs (the
                 signal-plus-noise data of the paper's next step, Sec. IV).

Parity status: everything here is pinned by ``tests/test_oracle_*.py`` to
closed forms, invariants, brute force or special cases, EXCEPT the absolute
agreement of the stand-in waveform / precession angles with the real
IMRPhenomT / NNLO models and of the Keplerian orbits with ESA's orbit file:
parity unpinned (the paper defers those formulas to earlier work).
"""
