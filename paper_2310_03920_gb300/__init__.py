"""GB300 (sm_103a) two-site DMRG hot path: C-ABI library ``libb2.so`` and its binding.

``paper_2310_03920_gb300.b2`` exposes the library calls by their C names.  Build the
library with ``python -m paper_2310_03920_gb300.build`` (``__graft_entry__.build()``).
"""
