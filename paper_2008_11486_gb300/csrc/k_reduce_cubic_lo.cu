// k_reduce_cubic_lo.cu -- fused reduction kernels, Keys' cubic convolution,
// register buckets 4 to 12.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(cubic_lo, ST_CUBIC, SRC_RAW, IRP_BUCKETS_LO)

}  // namespace irp
