"""GB300 (sm_103a) multilevel fast multipole product y = Z x for the Galerkin
EFIE with RWG basis functions (Dai, Wu, Meng, Chew, Sha: "Multilevel Fast
Multipole Algorithm for Characteristic Mode Analysis").

The compute path is the C-ABI library built from ``csrc/`` (declared in
``include/mlfma.h``); ``mlfma`` is its ctypes binding."""
from .mlfma import FP32, FP64, MIXED_3XTF32, MIXED_TF32, MlfmaError, MlfmaPlan, load  # noqa: F401
from ._build import build  # noqa: F401
