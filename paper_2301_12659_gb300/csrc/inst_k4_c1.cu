// Kernels of libmdnewton for K = 4 limbs, C = 1 (one translation unit per
// instantiation so the library builds in parallel).
#include "batch.cuh"
namespace mdn {
const KernelTable* kernels_k4_c1() { return make_table<4, 1>(); }
}  // namespace mdn
