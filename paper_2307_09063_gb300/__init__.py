"""Radar-STDA on GB300: CUDA kernels for sm_103a behind the C-ABI library
libstda, with a thin Python binding (``paper_2307_09063_gb300.stda``)."""
