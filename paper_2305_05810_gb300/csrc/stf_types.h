// Internal types shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/stf.h"

#define STF_MAX_LEVELS 16
#define STF_TEX_MAGIC 0x53544654u  // "STFT"

// Device status word bits (set by kernels with atomicOr, read by stf_synchronize).
#define STF_DEV_BAD_NODE 1u        // sparse traversal met an index outside its arrays
#define STF_DEV_MMA_TIMEOUT 2u     // a tensor-core completion wait gave up

namespace stf {

struct SparseDev {
  // Root: a short list of upper nodes (each covers 4096^3 voxels).
  int32_t n_upper;
  const int32_t* upper_origin;     // n_upper x 3
  const uint64_t* upper_mask;      // n_upper x 512 words (32^3 child bits)
  const uint32_t* upper_prefix;    // n_upper x 512: index of the lower node of the first
                                   // set bit of each word (node base + set bits before it)
  // Lower nodes (each covers 128^3 voxels, 16^3 leaves): one 16-byte record per mask
  // word, {mask low, mask high, index of the leaf of the word's first set bit, 0}.
  int32_t n_lower;
  const uint4* lower_rec;          // n_lower x 64
  // Leaves: 512 values each, [x&7][y&7][z&7].
  int64_t n_leaves;
  const float* leaf_f32;           // FP32 format
  const uint8_t* leaf_e4m3;        // E4M3 format
  const float* leaf_scale;         // E4M3 format: one scale per leaf
  float background;
  unsigned* status;
  // Bounding box [bb_lo, bb_hi) of the active leaves in voxels (clamped to +-2^30;
  // empty for a grid without leaves): outside it every voxel reads the background.
  int32_t bb_lo[3], bb_hi[3];
};

// Device view of a neural texture (stf_neural.cu).
struct NeuralDev {
  const __half* lat16;        // [texel][8], latent levels
  float* lat32;               // float32 master latents (training)
  float* m_lat;
  float* v_lat;
  const __half* fb16;         // [texel][8] (7 + pad), fallback levels
  const __half* wimg;         // weight images
  const float* bias;          // nn::NBIAS floats
  int64_t lvl_off[STF_MAX_LEVELS];   // texel offset within lat16 (latent) or fb16 (fallback)
  int32_t lvl_w[STF_MAX_LEVELS];
  int32_t lvl_h[STF_MAX_LEVELS];
  int32_t nlat, nlev;
  int64_t n_lat_texels;
  unsigned* status;           // device status word
};

}  // namespace stf

struct stf_texture_s {
  uint32_t magic;
  int32_t kind, format, channels, levels;
  int32_t dims[3];
  float background;
  // 2D / dense texels in storage format
  void* d_texels;
  int64_t level_off[STF_MAX_LEVELS];   // texels, or code words for DCT6
  int32_t level_w[STF_MAX_LEVELS];
  int32_t level_h[STF_MAX_LEVELS];
  // DCT6: blocks per row, AC step per channel (R_c / 15), basis constants
  int32_t blocks_w[STF_MAX_LEVELS];
  float ac_step[8];
  float dct_k[7];
  // sparse tree (one allocation, views into it)
  void* d_tree;
  stf::SparseDev sparse;
  // neural texture: one allocation holding latents, optimizer state and weights
  void* d_neural;
  stf::NeuralDev neural;
  float* n_params;    // float32 parameters
  float* n_m;         // Adam moments of the parameters
  float* n_v;
  float* n_grads;
  float* n_loss;      // one float
  int64_t n_step;     // training steps taken
  // device status word
  unsigned* d_status;
  // binning scratch, grown on demand
  void* d_scratch;
  int64_t scratch_bytes;
  int64_t bytes;
};
