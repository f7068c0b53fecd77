"""GB300 fast forward of gravity and gravity-gradient data on a right-prism
mesh: translation-equivalent BTTB kernels, circulant embedding and FFT
(Cao, "Rapid forward of gravity and tensor gravity data", Secs. 2.2.2-2.2.3).

The compute path is ``libgravfft.so`` (hand-written sm_103a CUDA behind the C
ABI of ``include/grav.h``).  ``capi`` binds it with ctypes; ``plan.Plan``
wraps it for CUDA tensors.  Importing this package loads nothing; the
library is opened on first use and its absence is an error.
"""

__all__ = ["capi", "plan", "workloads", "build"]
