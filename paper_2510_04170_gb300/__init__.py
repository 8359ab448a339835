"""GB300-native (sm_103a) random-feature-method nonlinear solvers IPN / AMIPN
(arXiv 2510.04170).  The numerical path is the CUDA library librfm.so behind a
C ABI (include/rfm.h); this package only marshals arguments to it."""
from .rfm import *  # noqa: F401,F403
