// Batched step kernels of the D3Q19 lattice (explicit instantiation): 32 x 8
// tiles, float32 and float16 storage.
#include "lbm_kernels.cuh"
template struct lbm::BatchLaunch<lbm::D3Q19, lbm::StoreF32, 32, 8>;
template struct lbm::BatchLaunch<lbm::D3Q19, lbm::StoreF16, 32, 8>;
