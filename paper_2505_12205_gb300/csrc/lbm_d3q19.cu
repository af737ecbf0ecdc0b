// Kernels of the D3Q19 lattice with float32 storage (explicit instantiation).
#include "lbm_kernels.cuh"
template struct lbm::Launch<lbm::D3Q19, lbm::StoreF32>;
