// k_reduce_bsplinev_lo.cu -- fused reduction kernels, vertical cubic-spline taps on
// horizontally filtered frames, register buckets 4 to 12.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bsplinev_lo, ST_BSPLINE_V, SRC_F32, IRP_BUCKETS_LO)

}  // namespace irp
