// Kernels of libmdnewton for K = 4 limbs, C = 2 (one translation unit per
// instantiation so the library builds in parallel).
#include "batch.cuh"
namespace mdn {
const KernelTable* kernels_k4_c2() { return make_table<4, 2>(); }
}  // namespace mdn
