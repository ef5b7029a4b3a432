"""FP64 CPU oracle of the differentiable ray-wave DOE step (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct restatement of the
method, used only to check the CUDA path.  Only the tests, the smoke check
and the benchmark's CPU-baseline / reference leg may import it; the product
library never does, and shares no code with it.

Everything is float64 PyTorch CPU arithmetic, vectorised over rays, so
torch.autograd gives the exact derivative of the oracle's forward model
(the "oracle gradient").  Each function cites the passage of the paper it
follows:

  Section "Ray-Wave Simulator Formalism": rays are plane-wave wavelets that
  are traced with conventional (Snell) ray tracing between surfaces; at a
  DOE a tangent frame is built at the hit point, a square patch of the
  transmission U = A exp(i phi) centred there is Fourier transformed into
  its angular spectrum, evanescent components are dropped and secondary
  rays carry weight U~/p (Eq. 1); sampling uses Gumbel noise with a softmax
  relaxation; the sensor field is a coherent sum of plane wavelets (Eq. 2).
  Section "Benchmark and Inverse Design Demonstrations": Eq. 3 loss.

Readings of points the paper leaves open (normalisation of the spectrum,
the k-grid, patch centring, how the incident tilt enters, obliquity) are
stated where they are used; every function in this package is pinned by a
CPU test against closed forms (grating equation, thick-lens focus,
Parseval, angular-spectrum propagation, finite differences).
"""
