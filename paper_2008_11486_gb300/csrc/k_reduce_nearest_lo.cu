// k_reduce_nearest_lo.cu -- fused reduction kernels, nearest stencil,
// register buckets 4 to 12.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(nearest_lo, ST_NEAREST, SRC_RAW, IRP_BUCKETS_LO)

}  // namespace irp
