"""Plain FP64 CPU oracle for CRBM-aided Monte Carlo (arXiv:2008.05401).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA path; the only common module is ``crbm_workloads`` (seeded inputs and
the packed-bit format, no arithmetic of the method).

Modules and what pins each (pins are tests under ``tests/test_oracle_*.py``):

* ``philox``  Philox4x32-10 counter RNG (Salmon et al., SC'11).  Pinned against
  an independent library implementation (Triton's ``tl.philox`` run by its CPU
  interpreter) and by uniformity checks.  The paper does not name a generator.
* ``crbm``    CRBM joint energy (Eq. 12), free energy (Eq. 13), conditionals
  (Eqs. B1-B3) and the block-Gibbs step (Eq. B4).  Pinned by brute-force
  marginalisation of the joint energy, exact conditionals of the joint
  distribution, exact detailed balance of the Gibbs kernel, and the analytic
  Ising CRBM of App. C.
* ``ising``   Ising energy (Eq. 14) and magnetisation.  Pinned by brute-force
  enumeration against Kaufman's closed-form finite-torus partition function.
* ``kitaev``  Majorana hopping matrix of Eq. (16) and the configuration
  log-weight sum_l log 2cosh(beta eps_l / 2).  Pinned by the Bloch closed
  form at uniform eta, the Frobenius sum rule, lattice symmetries and the full
  2N x 2N Majorana spectrum.
* ``chain``   Gibbs proposal + exact Metropolis-Hastings correction
  (Eq. B5 read with (pi, P_CRBM) as the two distributions).  Pinned by exact
  stationary distributions (Ising L=4, Kitaev L=2) and by acceptance == 1 for
  the analytic Ising CRBM.
* ``lcrbm``      Locally connected CRBM with unshared edge kernels for the
  open-boundary Kitaev model (Sec. IV); ``kitaev`` takes ``open_cols`` for the
  lattice open along j.  Pinned by brute-force marginalisation, conditionals
  read off the joint energy, the 1x1-kernel reduction to the CRBM, closed-form
  open spectra, the sum rule and exact stationarity of the chain.
* ``tempering``  Parallel-tempering exchange correction (App. B.2, Fig. 8b).
  Pinned by exact stationarity at every temperature of a ladder (Ising L=4)
  and by planted mistakes that break it.
* ``metropolis`` Local-update Metropolis baselines (Sec. III, Sec. IV):
  checkerboard single-spin flips (Ising), sequential single-eta flips (Kitaev),
  optionally with temperature exchange.  Pinned by exact stationarity and a
  deterministic zero-temperature sweep.
* ``train``      The paper's trainer: energy-matching loss with the optimal
  constant C, its gradient, ADAM, epochs of minibatches and the outer loop of
  Algorithm 1.  Pinned by finite differences, the zero loss of the analytic
  CRBM of App. C, closed-form ADAM properties and the L = 3 Ising protocol.
* ``autocorr``   Integrated autocorrelation time (Sokal's windowed
  estimator).  Pinned by the AR(1) closed form and exact small cases.
"""
