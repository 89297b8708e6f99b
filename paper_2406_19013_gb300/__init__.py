"""GB300 (sm_103a) X-engine of an FX radio correlator: per-channel conjugate
multiply-accumulate of 4+4-bit complex voltages on the tensor cores, int64
integration and full-Stokes output, behind the C ABI of include/corr.h."""
from .corr import (Batch, Correlator, CorrError, FEngine, Server, load,  # noqa: F401
                   strerror)
