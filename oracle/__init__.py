"""FP64 CPU oracle for the differentiable forward model and its gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

The oracle computes every step of the method by its definition in the paper,
in float64, with torch CPU ops used as an array library (library FFT
``torch.fft``, library ``torch.linalg.eigvalsh``, ``index_add_`` for the
mass assignment).  Gradients come from torch autograd of that forward
function, which is independent of the hand-written adjoint in the CUDA path.

Modules:
  cosmo  - linear power spectrum and its sigma(R) normalisation (App. A, Sect. 2.1)
  model  - white noise -> ALPT -> CIC -> cosmic web -> bias -> NB log posterior
  mock   - gamma-Poisson (negative binomial) mock counts (Sect. 2.6, Sect. 3)
  hmc    - leapfrog integrator (Sect. 2.2)

Pins: every function is checked by ``tests/test_oracle_pins.py`` against
closed forms, limits, library distributions and brute force.  The composed
end-to-end values have no printed worked example in the paper; they are pinned
only through those composed invariants and finite differences.
"""
from . import cosmo, model, mock, hmc  # noqa: F401
