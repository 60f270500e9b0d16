// The grid product (Eq. 8 / Eq. 10) compiled for complex64 (mixed precision) grid arithmetic. One translation unit per
// element type keeps the build parallel.
#include "matvec_kernels.cuh"

namespace aim {

template aim_status grid_pass<float2>(aim_ctx*, const PassSpec&, int, const double2*, double2*, cudaStream_t);
template aim_status grid_product_dense<float2>(aim_ctx*, bool, int, const double2*, double2*, void*, size_t,
                                          cudaStream_t);
template aim_status grid_pass_multi<float2>(const MultiPassSpec*, int, unsigned*, int*, cudaStream_t);

}  // namespace aim
