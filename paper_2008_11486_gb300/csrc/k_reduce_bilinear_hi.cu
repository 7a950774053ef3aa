// k_reduce_bilinear_hi.cu -- fused reduction kernels, bilinear stencil,
// register buckets 40 to 64.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bilinear_hi, ST_BILINEAR, SRC_RAW, IRP_BUCKETS_HI)

}  // namespace irp
