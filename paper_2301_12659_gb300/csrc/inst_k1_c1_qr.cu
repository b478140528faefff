// The QR of A_0 (qr_kernel, w_kernel) for K = 1 limbs, C = 1.
#include "batch.cuh"
namespace mdn {
template cudaError_t launch_qr<1, 1>(const QrParams&, cudaStream_t);
}  // namespace mdn
