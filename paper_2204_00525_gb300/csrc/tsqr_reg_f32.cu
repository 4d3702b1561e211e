// Instantiation of the register-path TSQR kernels for float tiles.
#include "tsqr_reg.cuh"

namespace fig {

template <>
void launch_reg_n<float>(const TsqrBlock& b, const double* tri_in, double* tri_out, int64_t div_in, int64_t tiles,
                       cudaStream_t st) {
  launch_reg_dispatch<float>(b, tri_in, tri_out, div_in, tiles, st);
}

}  // namespace fig
