// k_reduce_bspline_mid.cu -- fused reduction kernels, cubic-spline stencil,
// register buckets 16 to 32.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bspline_mid, ST_BSPLINE, SRC_F32, IRP_BUCKETS_MID)

}  // namespace irp
