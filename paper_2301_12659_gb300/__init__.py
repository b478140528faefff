"""GB300-native Newton's method on truncated power series in multiple double
precision (arXiv 2301.12659): CUDA kernels for sm_103a behind the C-ABI
library libmdnewton, with a thin Python binding (``mdnewton``)."""
