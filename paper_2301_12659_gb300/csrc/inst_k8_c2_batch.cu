// The batched solver's kernel for K = 8 limbs, C = 2 (a translation unit of
// its own so that it compiles beside the other kernels of this instantiation).
#include "batch.cuh"
namespace mdn {
template cudaError_t launch_batch<8, 2>(const BatchParams&, int, int, cudaStream_t);
template int batch_occupancy<8, 2>(int);
}  // namespace mdn
