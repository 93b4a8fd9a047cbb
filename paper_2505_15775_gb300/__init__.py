"""GB300 (sm_103a) ALM-BM hot path: the inner loop of rank-adaptive ALM-BM
(ALORA, arXiv 2505.15775) behind the C ABI of ``include/alm.h``.

``paper_2505_15775_gb300.alm`` is the Python binding (argument marshalling only);
``paper_2505_15775_gb300.build`` compiles the CUDA library.  Importing this
package loads nothing: the library is loaded on the first binding call, and a
missing library is an error, never a fallback.
"""
__all__ = ["alm", "build"]
