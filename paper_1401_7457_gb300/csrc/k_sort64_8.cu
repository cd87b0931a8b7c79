// Onesweep digit pass, 64-bit suffix ids, tiles of 256 threads x 8 items.
#include "onesweep.cuh"
#include "sort64.cuh"

namespace cxbwt {

cudaError_t launch_onesweep64_8(const PassArgs& a, int mode, bool wk, bool filter, cudaStream_t st) {
  return onesweep::launch_shape<uint64_t, onesweep::Shape64x8>(a, mode, wk, filter, st);
}

}  // namespace cxbwt
