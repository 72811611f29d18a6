// Instances of the multi-right-hand-side hopping kernel for WD_F32 fields.
#include "wd_mrhs.cuh"

namespace wd {

cudaError_t launch_mrhs_f32(const MrhsBatch& bt, int recon, bool dagger, const int* active,
                            RedScratch rs, bool norm, int lanes, cudaStream_t st) {
  return launch_mrhs_prec<WD_F32>(bt, recon, dagger, active, rs, norm, lanes, st);
}

}  // namespace wd
