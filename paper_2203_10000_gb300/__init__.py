"""GB300-native solid-angle labeling (arXiv:2203.10000, Sec. 2.1-2.1.3).

`paper_2203_10000_gb300.zef` is the ctypes binding of the C-ABI library
`libzef.so` (include/zef.h); `paper_2203_10000_gb300.build` compiles it.
"""
__all__ = ["build", "zef"]
