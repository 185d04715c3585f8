"""Plain, slow FP64 CPU oracle for the PauliNet VMC hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes this package; only the test-suite, the smoke check and the CPU
baseline leg of the benchmark do.  It shares no code with the CUDA library:
its one shared input is the seeded generator module
``paper_1909_08423_gb300.synth``, which holds none of the method's arithmetic.

Modules
  ansatz      psi of Eq. (ansatz), orbitals with the Ma et al. nuclear cusp
              splice, the SchNet-style network (Methods, "PauliNet extension
              of SchNet"), determinants, gamma, Coulomb potential, local
              energy (Eq. monte-carlo) and the parameter gradient of ln|psi|
              (Eq. trainig).  Exact derivatives come from torch.autograd in
              float64 -- a different algorithm from the GPU's forward jet.
  cusp        host-side coefficients of the nuclear cusp correction.
  philox      Philox4x32-10 counter-based generator (Salmon et al., SC'11)
              and Box-Muller normals.
  sampling    Metropolis walker update and walker initialisation.
  clip        smooth logarithmic clipping of local energies (Methods,
              "Ansatz optimization").

Pins (tests/test_oracle_pins.py) cover every function: closed forms of the
local energy (hydrogen-like atoms, a Gaussian, a two-electron product, an
electron beside bare nuclei for the nucleus-nucleus terms of V), Leibniz
determinants, finite differences, symmetries and cusps, Philox4x32-10
known-answer vectors, a hand-worked table of the distance features e_k and a
hand-worked two-layer map with the shifted softplus.  The network's message
passing and heads are also pinned by a special case: with constant filters
every message is a partner count times a spin-class row, which fixes the
channel assignment, the partner sums, the layer recursion and both heads.
"""
