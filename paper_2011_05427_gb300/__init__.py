"""GB300-native MLQD / multigrid-in-frequency TRT solver (arXiv 2011.05427).

The compute path is the CUDA library built from csrc/ behind the C ABI in
include/trt.h; `paper_2011_05427_gb300.trt` is the Python binding.  Importing the
package does not load the library; the binding does, and fails loudly if the shared
library is missing.
"""
