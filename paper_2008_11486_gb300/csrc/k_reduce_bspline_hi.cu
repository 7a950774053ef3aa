// k_reduce_bspline_hi.cu -- fused reduction kernels, cubic-spline stencil,
// register buckets 40 to 64.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bspline_hi, ST_BSPLINE, SRC_F32, IRP_BUCKETS_HI)

}  // namespace irp
