// k_reduce_nearest_mid.cu -- fused reduction kernels, nearest stencil,
// register buckets 16 to 32.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(nearest_mid, ST_NEAREST, SRC_RAW, IRP_BUCKETS_MID)

}  // namespace irp
