// tcgen05 split-precision GEMM (placeholder until the tensor-core kernel lands).
#include "kernels.h"

namespace rcc {
int launch_gemm_tc(int, const void*, const void*, const void*, const void*, int, const EpiArgs&, int*, long long,
                   cudaStream_t) {
  return 1;
}
}  // namespace rcc
