// Launchers implemented by the kernel translation units, called by stf_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "stf_device.cuh"

namespace stf {

enum Op { OP_STOCHASTIC = 0, OP_DETERMINISTIC = 1, OP_ACCUMULATE = 2 };

int grid_blocks(int64_t n, int threads);   // grid size for a grid-stride launch

cudaError_t launch_tex2d(Op op, int filter, int fmt, int channels, const Tex2DView& t,
                         const LookupArgs& a, cudaStream_t s);
cudaError_t launch_dense3d(Op op, int filter, int fmt, const Dense3DView& g,
                           const LookupArgs& a, cudaStream_t s);
cudaError_t launch_sparse3d(Op op, int filter, int fmt, const SparseDev& g,
                            const LookupArgs& a, cudaStream_t s);

// Create-time kernels.
cudaError_t launch_convert_f32(const float* src, void* dst, int fmt, int64_t n, cudaStream_t s);
cudaError_t launch_box_mip(const float* src, float* dst, int w, int h, int c, cudaStream_t s);

}  // namespace stf
