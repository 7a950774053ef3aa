// k_reduce_bilinear_lo.cu -- fused reduction kernels, bilinear stencil,
// register buckets 4 to 12.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bilinear_lo, ST_BILINEAR, SRC_RAW, IRP_BUCKETS_LO)

}  // namespace irp
