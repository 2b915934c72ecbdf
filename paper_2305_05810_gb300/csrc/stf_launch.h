// Launchers implemented by the kernel translation units, called by stf_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "stf_device.cuh"

namespace stf {

enum Op { OP_STOCHASTIC = 0, OP_DETERMINISTIC = 1, OP_ACCUMULATE = 2 };

// Grid size for a grid-stride launch: enough blocks for n, capped at `waves` full waves
// of 2048 threads per SM.
int grid_blocks(int64_t n, int threads, int waves = 4);
// The stochastic dense and sparse kernels launch up to 8 waves of 256-thread blocks.
// With four queries per thread and the miss shortcut, 8 waves finished the dense
// benchmark call 3% sooner than 16 and 6% sooner than 32 (2: 11% later; 4 and 6 within
// 1% of 8, sparse 1-5% slower).  The 2D kernels keep 4 waves (no gain at 16.8M queries,
// 3% slower at 5.3M with 16).
constexpr int kStochasticWaves = 8;

cudaError_t launch_tex2d(Op op, int filter, int fmt, int channels, const Tex2DView& t,
                         const LookupArgs& a, cudaStream_t s);
cudaError_t launch_tex2d_f32(Op op, int filter, int channels, const Tex2DView& t,
                             const LookupArgs& a, cudaStream_t s);
cudaError_t launch_tex2d_f16(Op op, int filter, int channels, const Tex2DView& t,
                             const LookupArgs& a, cudaStream_t s);
cudaError_t launch_tex2d_dct(Op op, int filter, int channels, const Tex2DView& t,
                             const LookupArgs& a, cudaStream_t s);
cudaError_t launch_dense3d(Op op, int filter, int fmt, const Dense3DView& g,
                           const LookupArgs& a, cudaStream_t s);
cudaError_t launch_sparse3d(Op op, int filter, int fmt, const SparseDev& g,
                            const LookupArgs& a, cudaStream_t s);

// Create-time kernels.
cudaError_t launch_convert_f32(const float* src, void* dst, int fmt, int64_t n, cudaStream_t s);
cudaError_t launch_box_mip(const float* src, float* dst, int w, int h, int c, cudaStream_t s);
// DCT6 encoding of a float32 pyramid (levels at level_off texels of src, C channels):
// codes at code_off words of dst, per-channel AC ranges R_c (float64, host) out.
cudaError_t launch_dct_encode(const float* src, const int64_t* level_off, const int32_t* w,
                              const int32_t* h, int levels, int C, uint32_t* dst,
                              const int64_t* code_off, double* scratch, double* h_range, cudaStream_t s);

}  // namespace stf
