"""GB300-native labeling of discrete abstractions for LTL planning
(arXiv 1810.02612): CUDA kernels for sm_103a behind the C ABI in
``include/lbl.h``, with a thin Python binding in :mod:`.lbl`."""
from . import lbl  # noqa: F401
from .lbl import *  # noqa: F401,F403

__all__ = list(lbl.EXPORTS) + ["LblError", "lbl_grid", "lbl_pose", "lbl_config", "packed_word_bytes",
                               "packed_word_dtype"]
