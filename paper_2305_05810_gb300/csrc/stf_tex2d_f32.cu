// 2D lookups of float32 textures: the kernels of stf_tex2d.cuh for that format (one
// translation unit per format keeps the build parallel).
#include "stf_tex2d.cuh"

namespace stf {

cudaError_t launch_tex2d_f32(Op op, int filter, int channels, const Tex2DView& t, const LookupArgs& a,
                             cudaStream_t s) {
  return launch_tex2d_format<STF_FMT_F32>(op, filter, channels, t, a, s);
}

}  // namespace stf
