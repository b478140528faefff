// Kernels of libmdnewton for K = 8 limbs, C = 1 (one translation unit per
// instantiation so the library builds in parallel).
#include "batch.cuh"
namespace mdn {
const KernelTable* kernels_k8_c1() { return make_table<8, 1>(); }
}  // namespace mdn
