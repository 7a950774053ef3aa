// k_reduce_bsplinev_hi.cu -- fused reduction kernels, vertical cubic-spline taps on
// horizontally filtered frames, register buckets 40 to 64.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bsplinev_hi, ST_BSPLINE_V, SRC_F32, IRP_BUCKETS_HI)

}  // namespace irp
