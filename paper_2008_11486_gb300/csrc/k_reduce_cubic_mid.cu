// k_reduce_cubic_mid.cu -- fused reduction kernels, Keys' cubic convolution,
// register buckets 16 to 32.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(cubic_mid, ST_CUBIC, SRC_RAW, IRP_BUCKETS_MID)

}  // namespace irp
