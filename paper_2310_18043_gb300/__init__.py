"""GB300 (sm_103a) interior eigensolver on the composite-rule rational filter
(Chen & Li, arXiv 2310.18043). The compute path is the C-ABI library libie.so
(include/ie.h); `paper_2310_18043_gb300.ie` is its ctypes binding."""
