// k_reduce_cubic_hi.cu -- fused reduction kernels, Keys' cubic convolution,
// register buckets 40 to 64.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(cubic_hi, ST_CUBIC, SRC_RAW, IRP_BUCKETS_HI)

}  // namespace irp
