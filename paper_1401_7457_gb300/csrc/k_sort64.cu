// Instantiations of the onesweep digit pass for 64-bit suffix ids
// (collections with n * 2^shift >= 2^32): one tile shape.  See onesweep.cuh.
#include "onesweep.cuh"

namespace cxbwt {

template <>
cudaError_t launch_onesweep_t<uint64_t>(const PassArgs& a, int mode, bool wk, bool filter, const TileShape& /*s*/,
                                        cudaStream_t st) {
  if (a.n_tiles == 0) return cudaSuccess;
  return onesweep::launch_shape<uint64_t, onesweep::ShapeMid>(a, mode, wk, filter, st);
}

}  // namespace cxbwt
