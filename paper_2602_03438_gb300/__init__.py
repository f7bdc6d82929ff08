"""GB300-native batched RGF selected inversion for atomistic NEGF (arXiv:2602.03438).

The compute path is libnegf.so (CUDA, sm_103a) behind the C ABI declared in
include/negf.h; ``negf`` is its thin ctypes binding.
"""
from . import negf  # noqa: F401
from . import tuning  # noqa: F401
from .negf import (FP64, MIXED, MIXED_TF32, Context, NegfError, Scattering, System, allocate_outputs,  # noqa: F401
                   negf_obc, negf_observables, negf_rgf_keldysh, negf_rgf_lesser, negf_rgf_partitioned,
                   negf_rgf_retarded,
                   system_layout, upload)
