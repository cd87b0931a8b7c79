// Instantiations of the onesweep digit pass for 32-bit suffix ids
// (n * 2^shift < 2^32): two tile shapes.  See onesweep.cuh.
#include "onesweep.cuh"

namespace cxbwt {

TileShape onesweep_shape(int tile_items_hint, int id_bytes) {
  if (id_bytes == 4 && tile_items_hint == 8192)
    return TileShape{onesweep::ShapeLarge::threads, onesweep::ShapeLarge::ipt};
  if (id_bytes == 8 && tile_items_hint == 2048)
    return TileShape{onesweep::Shape64x8::threads, onesweep::Shape64x8::ipt};
  if (id_bytes == 8 && tile_items_hint == 3072)
    return TileShape{onesweep::Shape64x12::threads, onesweep::Shape64x12::ipt};
  // Everything else: 4096-item tiles (for 64-bit ids the instantiation whose
  // registers are sized for the three CTAs its shared memory allows).
  return TileShape{onesweep::ShapeMid::threads, onesweep::ShapeMid::ipt};
}

template <>
cudaError_t launch_onesweep_t<uint32_t>(const PassArgs& a, int mode, bool wk, bool filter, const TileShape& s,
                                        cudaStream_t st) {
  if (a.n_tiles == 0) return cudaSuccess;
  if (s.threads == onesweep::ShapeLarge::threads && s.items_per_thread == onesweep::ShapeLarge::ipt)
    return onesweep::launch_shape<uint32_t, onesweep::ShapeLarge>(a, mode, wk, filter, st);
  return onesweep::launch_shape<uint32_t, onesweep::ShapeMid>(a, mode, wk, filter, st);
}

cudaError_t launch_onesweep(const PassArgs& a, int mode, bool write_key, bool filter, int id_bytes,
                            const TileShape& shape, cudaStream_t st) {
  return id_bytes == 8 ? launch_onesweep_t<uint64_t>(a, mode, write_key, filter, shape, st)
                       : launch_onesweep_t<uint32_t>(a, mode, write_key, filter, shape, st);
}

}  // namespace cxbwt
