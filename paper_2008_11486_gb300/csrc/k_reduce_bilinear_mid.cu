// k_reduce_bilinear_mid.cu -- fused reduction kernels, bilinear stencil,
// register buckets 16 to 32.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bilinear_mid, ST_BILINEAR, SRC_RAW, IRP_BUCKETS_MID)

}  // namespace irp
