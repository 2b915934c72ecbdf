#include "stf_internal.h"
namespace stf {
stf_status build_sparse(stf_texture_s*, const stf_texture_desc*, cudaStream_t) {
  return fail(STF_ERR_UNSUPPORTED, "sparse grids not built yet");
}
cudaError_t launch_sparse3d(Op, int, int, const SparseDev&, const LookupArgs&, cudaStream_t) {
  return cudaErrorNotSupported;
}
}
