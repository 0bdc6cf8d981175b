"""GB300 (sm_103a) implementation of the IFEM fluid-structure coupling step
(Saadat, Guido, Iaccarino & Shaqfeh, arXiv:1807.08219): element forces,
spreading and interpolation as hand-written CUDA kernels behind the C ABI of
include/ifem.h (libifem.so), with a thin ctypes binding (``ifem``) and
torch.autograd adjoints (``autograd``)."""
from . import ifem  # noqa: F401
