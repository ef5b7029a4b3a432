"""GB300-native ray-wave DOE library: Python binding of librw.so.

    from paper_2605_15418_gb300 import raywave, autograd
    sim = raywave.Simulator(workload)          # rays generated on the GPU (A0)
    psf = sim.forward()                        # A1..A7 in one fused kernel

The compiled library is required; there is no CPU fallback.
"""
__all__ = ["raywave", "autograd", "build"]
