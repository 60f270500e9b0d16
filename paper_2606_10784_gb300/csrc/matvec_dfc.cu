// The grid product (Eq. 8 / Eq. 10) compiled for double-float complex (FP64 mode) grid arithmetic. One translation unit per
// element type keeps the build parallel.
#include "matvec_kernels.cuh"

namespace aim {

template aim_status grid_pass<dfc>(aim_ctx*, const PassSpec&, int, const double2*, double2*, cudaStream_t);
template aim_status grid_product_dense<dfc>(aim_ctx*, bool, int, const double2*, double2*, void*, size_t,
                                          cudaStream_t);
template aim_status grid_pass_multi<dfc>(const MultiPassSpec*, int, unsigned*, int*, cudaStream_t);

}  // namespace aim
