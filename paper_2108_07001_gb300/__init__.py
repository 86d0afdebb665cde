"""GB300-native data-parallel hot path of a dual-polarisation coherent
optical receiver (overlap-save CD compensation, timing and frequency-offset
recovery, 2x2 block-LMS MIMO, blind phase search, demapping, BER), after
the GPU receiver of arXiv 2108.07001.  The compute path is librx.so
(hand-written sm_103a CUDA kernels behind the C ABI in include/rx.h);
``rx`` is its ctypes binding."""
from . import rx  # noqa: F401
from .rx import Receiver, default_config, load  # noqa: F401
