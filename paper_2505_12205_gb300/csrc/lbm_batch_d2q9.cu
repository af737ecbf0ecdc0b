// Batched step kernels of the D2Q9 lattice (explicit instantiation): tile
// widths 32, 64 and 128, float32 and float16 storage.
#include "lbm_kernels.cuh"
template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF32, 32, 1>;
template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF32, 64, 1>;
template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF32, 128, 1>;
template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF16, 32, 1>;
template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF16, 64, 1>;
template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF16, 128, 1>;
