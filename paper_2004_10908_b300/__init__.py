"""Device-resident Taskflow-style task-graph executor for B300 (sm_103a).

Static and condition tasks, strong/weak edges, join counters and work
stealing all run inside one persistent CUDA kernel (libtg.so, C-ABI in
include/tg.h).  `binding` mirrors the C names; `Executor` is a thin
convenience layer whose device memory and stream come from PyTorch."""
from . import binding
from .binding import TgError, STATUS_NAMES
from .executor import Executor, GraphHandle, Batch

__all__ = ["binding", "TgError", "STATUS_NAMES", "Executor", "GraphHandle", "Batch"]
