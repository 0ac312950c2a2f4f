"""CPU oracle for the boundary-MPS sampler of 2D tensor-network states (arXiv 2507.11424).

TEST INFRASTRUCTURE ONLY.  Plain, slow, complex128 numpy/LAPACK code written
from the paper, used by tests/, the smoke check and bench.py's CPU-baseline
leg to check the GB300 library.  The product path never imports it, and it
shares no code with the library (only the seeded inputs in ``workloads``).

Modules:
* philox      -- Philox4x32-10 counter RNG (Salmon et al., SC'11).
* statevector -- exact circuit simulation that pins the TNS oracle.
* tns         -- grid TNS, belief propagation, BP-gauged simple update.
* bmps        -- boundary-MPS compression, norm environments, sampler, amplitudes.
* metrics     -- p/q ratios, sample KLD, sector fraction, marginals.
"""
