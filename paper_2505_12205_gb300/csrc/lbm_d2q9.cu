// Kernels of the D2Q9 lattice (explicit instantiation).
#include "lbm_kernels.cuh"
template struct lbm::Launch<lbm::D2Q9>;
