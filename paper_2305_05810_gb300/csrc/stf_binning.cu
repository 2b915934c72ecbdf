#include "stf_internal.h"
namespace stf {
stf_status lookup_binned(stf_texture, int, const LookupArgs&, cudaStream_t) {
  return fail(STF_ERR_UNSUPPORTED, "binning not built yet");
}
}
