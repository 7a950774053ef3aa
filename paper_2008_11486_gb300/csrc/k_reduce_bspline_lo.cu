// k_reduce_bspline_lo.cu -- fused reduction kernels, cubic-spline stencil,
// register buckets 4 to 12.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bspline_lo, ST_BSPLINE, SRC_F32, IRP_BUCKETS_LO)

}  // namespace irp
