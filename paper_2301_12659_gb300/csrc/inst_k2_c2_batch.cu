// The batched solver's kernel for K = 2 limbs, C = 2 (a translation unit of
// its own so that it compiles beside the other kernels of this instantiation).
#include "batch.cuh"
namespace mdn {
template cudaError_t launch_batch<2, 2>(const BatchParams&, int, int, cudaStream_t);
template int batch_occupancy<2, 2>(int);
}  // namespace mdn
