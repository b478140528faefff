// Kernels of libmdnewton for K = 4 limbs, C = 2.  Each instantiation is
// split over three translation units that build in parallel: this one (the
// table, evaluation, forward substitution and the rest), the QR of A_0 in
// inst_k4_c2_qr.cu and the batched solver in inst_k4_c2_batch.cu.
#include "batch.cuh"
namespace mdn {
extern template cudaError_t launch_qr<4, 2>(const QrParams&, cudaStream_t);
extern template cudaError_t launch_batch<4, 2>(const BatchParams&, int, int, cudaStream_t);
extern template int batch_occupancy<4, 2>(int);
const KernelTable* kernels_k4_c2() { return make_table<4, 2>(); }
}  // namespace mdn
