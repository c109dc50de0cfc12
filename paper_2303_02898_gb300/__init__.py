"""GB300-native (sm_103a) hot path of the 35-moment maximal-entropy moment
method of arXiv 2303.02898.  The CUDA library sits behind a C ABI
(include/mem.h); `paper_2303_02898_gb300.mem` is its thin Python binding."""
