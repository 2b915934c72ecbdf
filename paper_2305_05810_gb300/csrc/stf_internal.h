// Internal declarations shared by the host-side translation units.
#pragma once
#include <cuda_runtime.h>

#include "stf_launch.h"

namespace stf {

stf_status fail(stf_status code, const char* fmt, ...);
stf_status fail_cuda(cudaError_t e, const char* what);
cudaError_t dev_alloc(void** p, size_t bytes);
// Failure-injection hook: counts one device allocation and says whether it must fail
// (stf_debug_fail_allocation); allocates nothing.
bool alloc_should_fail();
bool handle_ok(stf_texture t);
stf_status dispatch(Op op, stf_texture t, int filter, const LookupArgs& a, cudaStream_t s);
stf_status triplanar(Op op, stf_texture t, const stf_lookup_params* p, const float* pos,
                     const float* normal, const float* lod, int64_t n, float scale, float* out,
                     int32_t* taps, cudaStream_t s);
stf_status check_lookup(stf_texture t, const stf_lookup_params* p, const float* coords,
                        const float* lod, int64_t n, const void* out);
Tex2DView view2d(const stf_texture_s* t);
LookupArgs make_args(const stf_lookup_params* p, const float* coords, const float* lod, int64_t n,
                     float* out, int32_t* taps);

// Sparse grid construction (stf_sparse.cu).
stf_status build_sparse(stf_texture_s* t, const stf_texture_desc* d, cudaStream_t s);

// Neural textures (stf_neural.cu).
stf_status build_neural(stf_texture_s* t, const stf_neural_desc* d, cudaStream_t s);
cudaError_t launch_neural(Op op, int filter, const NeuralDev& nd, const LookupArgs& a, cudaStream_t s);

// Morton-binned stochastic lookup (stf_binning.cu).
stf_status lookup_binned(stf_texture t, int filter, const LookupArgs& a, cudaStream_t s);

}  // namespace stf
