// Launchers of the 64-bit-id onesweep instantiations, one translation unit
// per tile shape (compiled in parallel).
#pragma once
#include "kernels.cuh"

namespace cxbwt {

cudaError_t launch_onesweep64_mid(const PassArgs& a, int mode, bool wk, bool filter, cudaStream_t st);
cudaError_t launch_onesweep64_12(const PassArgs& a, int mode, bool wk, bool filter, cudaStream_t st);
cudaError_t launch_onesweep64_8(const PassArgs& a, int mode, bool wk, bool filter, cudaStream_t st);

}  // namespace cxbwt
