// The batched solver's kernel for K = 1 limbs, C = 1 (a translation unit of
// its own so that it compiles beside the other kernels of this instantiation).
#include "batch.cuh"
namespace mdn {
template cudaError_t launch_batch<1, 1>(const BatchParams&, int, int, cudaStream_t);
template int batch_occupancy<1, 1>(int);
}  // namespace mdn
