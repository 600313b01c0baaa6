"""GB300 (sm_103a) Vanka-smoothed shifted-Laplacian multigrid / FGMRES solver
for the finite-difference Helmholtz equation (arXiv 2511.16808).

The compute path is the C-ABI CUDA library libhz.so (include/hz.h, sources in
csrc/); `hz` is its Python binding and `solver` a convenience layer that
fills the ABI's structs from problem parameters.  Import `hz` explicitly:
importing the package itself loads nothing.
"""
