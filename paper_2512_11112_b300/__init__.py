"""B300-native SPDZ online phase: C-ABI CUDA library (libspdz.so) and its
thin Python binding.

``spdz`` is the binding (same names as ``include/spdz.h``); ``shares`` holds
helpers that allocate party-major share tensors with torch.  Importing the
package does not load the CUDA library; importing ``spdz`` does, and fails if
it is not built.
"""
