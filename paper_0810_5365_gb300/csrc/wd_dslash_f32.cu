// Instances of the hopping kernel for WD_F32 fields (one translation unit per
// precision so that the library builds in parallel).
#include "wd_dslash.cuh"

namespace wd {

cudaError_t launch_dslash_f32(const DslashArgs& a, int recon, bool dagger, cudaStream_t st) {
  return launch_dslash_prec<WD_F32>(a, recon, dagger, st);
}

}  // namespace wd
