"""GB300-native differentiable Monte Carlo ray-traced face rendering.

Dib et al., "Practical Face Reconstruction via Differentiable Ray Tracing"
(Eurographics 2021): a morphable face (Sec. 3.1) with Cook-Torrance reflectance
(Sec. 3.2, App. A) lit by a virtual light stage of area lights (Sec. 3.3), rendered
by a Monte Carlo estimator with shadow rays and differentiated with edge sampling
(Sec. 4).  The compute path is a C-ABI CUDA library (``libfacert.so``); this
package holds the thin ctypes binding, the autograd wrapper, the optimiser and
the serving loop.  Submodules are imported lazily so that the synthetic input
generators can be used without the CUDA library.
"""
__all__ = ["synth"]
