"""GB300 (sm_103a) symmetric-deletion Levenshtein neighbour search.

The search (Appendix A of arXiv 2403.09010, XTNeighbor steps 0-7) runs in
hand-written CUDA kernels behind the C ABI of include/xtn.h; this package is
its thin Python binding.  ``build()`` compiles the library.
"""
from .buildlib import build  # noqa: F401
from .native import XtnError, LIB_PATH  # noqa: F401
from .native import (XTN_TUNE_FILTER_SEGMENT, XTN_TUNE_GROUPING,  # noqa: F401
                     XTN_TUNE_RECORD_HISTOGRAM, XTN_TUNE_SORT_PAIRS, XTN_TUNE_SORT_RECORDS)
from .xtn import (Index, Plan, index_build, profile_enable, profile_only, profile_report,  # noqa: F401
                  scratch_trim, search_between, search_paired, search_query, search_self,
                  search_self_streaming,
                  set_wait_limit, tcrdist_filter, tune_count, tune_get, tune_set)
