// k_reduce_nearest_hi.cu -- fused reduction kernels, nearest stencil,
// register buckets 40 to 64.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(nearest_hi, ST_NEAREST, SRC_RAW, IRP_BUCKETS_HI)

}  // namespace irp
