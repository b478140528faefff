// The QR of A_0 (qr_kernel, w_kernel) for K = 2 limbs, C = 1.
#include "batch.cuh"
namespace mdn {
template cudaError_t launch_qr<2, 1>(const QrParams&, cudaStream_t);
}  // namespace mdn
