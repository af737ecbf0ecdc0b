// Kernels of the D2Q9 lattice (explicit instantiation), every storage format.
#include "lbm_kernels.cuh"
template struct lbm::Launch<lbm::D2Q9, lbm::StoreF32>;
template struct lbm::Launch<lbm::D2Q9, lbm::StoreF16>;
template struct lbm::Launch<lbm::D2Q9, lbm::StoreBF16>;
