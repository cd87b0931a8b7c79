// Instantiations of the onesweep digit pass for 64-bit suffix ids
// (collections with n * 2^shift >= 2^32), and the choice among their tile
// shapes.  See onesweep.cuh.  With 64-bit ids a tile of 4096 items stages
// 48 KB in shared memory, which holds a GB300 SM to three CTAs; the smaller
// tiles (k_sort64_small.cu) trade more look-back words per item for more
// resident CTAs.
#include "onesweep.cuh"
#include "sort64.cuh"

namespace cxbwt {

cudaError_t launch_onesweep64_mid(const PassArgs& a, int mode, bool wk, bool filter, cudaStream_t st) {
  return onesweep::launch_shape<uint64_t, onesweep::Shape64x16>(a, mode, wk, filter, st);
}

template <>
cudaError_t launch_onesweep_t<uint64_t>(const PassArgs& a, int mode, bool wk, bool filter, const TileShape& s,
                                        cudaStream_t st) {
  if (a.n_tiles == 0) return cudaSuccess;
  if (s.threads == onesweep::Shape64x12::threads && s.items_per_thread == onesweep::Shape64x12::ipt)
    return launch_onesweep64_12(a, mode, wk, filter, st);
  if (s.threads == onesweep::Shape64x8::threads && s.items_per_thread == onesweep::Shape64x8::ipt)
    return launch_onesweep64_8(a, mode, wk, filter, st);
  return launch_onesweep64_mid(a, mode, wk, filter, st);
}

}  // namespace cxbwt
