// The QR of A_0 (qr_kernel, w_kernel) for K = 4 limbs, C = 1.
#include "batch.cuh"
namespace mdn {
template cudaError_t launch_qr<4, 1>(const QrParams&, cudaStream_t);
}  // namespace mdn
