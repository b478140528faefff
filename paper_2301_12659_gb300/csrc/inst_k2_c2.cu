// Kernels of libmdnewton for K = 2 limbs, C = 2 (one translation unit per
// instantiation so the library builds in parallel).
#include "batch.cuh"
namespace mdn {
const KernelTable* kernels_k2_c2() { return make_table<2, 2>(); }
}  // namespace mdn
