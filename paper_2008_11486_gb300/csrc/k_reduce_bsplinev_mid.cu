// k_reduce_bsplinev_mid.cu -- fused reduction kernels, vertical cubic-spline taps on
// horizontally filtered frames, register buckets 16 to 32.
#include "reduce_kernels.cuh"

namespace irp {

IRP_REDUCE_PART(bsplinev_mid, ST_BSPLINE_V, SRC_F32, IRP_BUCKETS_MID)

}  // namespace irp
