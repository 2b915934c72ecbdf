/*
 * stf.h -- C ABI of the GB300 stochastic texture filtering library (libstf.so).
 *
 * The library performs batched filtered lookups into 2D MIP-mapped textures (plain
 * or DCT-compressed), dense or sparse 3D voxel grids and neural textures, following
 * "Stochastic Texture Filtering" (Fajardo, Wronski, Salvi, Pharr; arXiv 2305.05810):
 *
 *   stochastic form   -- one tap per axis is drawn with probability |w| / sum|w|
 *                        from the separable filter weights (sampling arrays,
 *                        Section 2.2; Eq. 7-9 in Section 4) and the single texel
 *                        is returned, times sign(w) * sum|w| per axis for kernels
 *                        with negative lobes (Section 2.2, "Positivization", first
 *                        sentence), or two taps by positivization, or one texel by
 *                        filter importance sampling (Section 4.4).  Its expectation
 *                        is the filtered value (Eq. 3).
 *   deterministic form -- the full weighted sum over every tap (Eq. 2, Eq. 9), the
 *                        same-GPU baseline.
 * Further entry points: anisotropic level of detail and EWA filtering, triplanar
 * mapping, validation accumulators, neural-texture training, an allocation-free
 * binned lookup.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an stf_status.  On failure stf_last_error() returns a
 *     message for the calling thread.  Argument errors are reported before any
 *     work is queued.
 *   - Device pointers ("d_" prefix) are memory the device can address, owned by the
 *     caller: CUDA device or managed memory, or page-locked host memory mapped into
 *     the device's address space (cudaHostAlloc; cudaHostRegister with
 *     cudaHostRegisterMapped), whose host address is its device address under
 *     unified addressing.  The kernels then read coordinates and write results across
 *     the host link with no staging copy (stf_device_accessible checks a pointer).
 *     Host pointers ("h_" prefix) are ordinary host memory.
 *   - Work is queued on the given CUDA stream (cudaStream_t passed as void*; NULL
 *     is the legacy default stream) and is asynchronous unless stated otherwise.
 *   - n == 0 is a no-op that returns STF_OK.
 *   - Coordinates: 2D lookups take texture coordinates (u, v); the raster position
 *     on level L is x = u * W_L - 1/2 (texel centres at i + 1/2).  3D lookups take
 *     index-space positions; voxel values sit at integer coordinates.  A NaN or
 *     infinite coordinate (or level of detail) yields the background value.
 *   - Addressing: 2D clamps to the edge; dense and sparse 3D read the background
 *     value outside the grid / outside active leaves.
 *   - Random variates: the i-th query of a call draws its variates from
 *     Philox4x32-10 with key = seed and counter = (q, q >> 32, sample_index, 0),
 *     q = query_offset + i (counter word 3, the stream, is 0; the positivized filter
 *     also draws stream 1, the cubic B-spline FIS filter streams 1 and 2).
 *     Results therefore do not depend on how a batch is
 *     split into calls, on launch shape, or on what else runs on the GPU.
 */
#ifndef STF_H_
#define STF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stf_texture_s* stf_texture; /* opaque handle owned by the library */

typedef enum {
  STF_OK = 0,
  STF_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, enum value or descriptor */
  STF_ERR_INVALID_HANDLE = 2,   /* handle never created or already destroyed */
  STF_ERR_OUT_OF_MEMORY = 3,    /* a device or host allocation failed */
  STF_ERR_UNSUPPORTED = 4,      /* valid request this texture kind cannot serve */
  STF_ERR_CUDA = 5,             /* a CUDA runtime call failed (message has details) */
  STF_ERR_DEVICE_ASSERT = 6,    /* a kernel found an inconsistent data structure */
  STF_ERR_BUDGET = 7            /* a memory budget would be exceeded */
} stf_status;

typedef enum {
  STF_KIND_TEX2D = 0,    /* 2D texture, optional MIP pyramid */
  STF_KIND_DENSE3D = 1,  /* dense voxel grid */
  STF_KIND_SPARSE3D = 2, /* sparse grid: root -> upper (32^3) -> lower (16^3) -> 8^3 leaves */
  STF_KIND_NEURAL2D = 3  /* neural 2D texture (stf_create_neural_texture) */
} stf_kind;

typedef enum {
  STF_FMT_F32 = 0,        /* IEEE binary32 texels */
  STF_FMT_F16 = 1,        /* IEEE binary16 texels (round-to-nearest-even at create) */
  STF_FMT_E4M3_SCALED = 2, /* sparse only: OCP FP8 E4M3 codes with one float32 scale
                             per leaf, scale = max|v| / 448 */
  STF_FMT_DCT6 = 3        /* 2D only: DCT-compressed 8x8 blocks (Section 5.2, "Texture
                             compression"), 32 bits per block and channel: the six
                             coefficients (u, v) = (0,0), (1,0), (0,1), (2,0), (1,1), (0,2)
                             of the orthonormal 8-point DCT-II (u along x), DC code
                             round(DC 127 / 8) in [0, 127] (bits 0-6; texel values in
                             [0, 1], DC = 8 x block mean), AC code j round(AC 15 / R_c)
                             in [-15, 15] (bits 7+5j .. 11+5j, two's complement), R_c =
                             largest |AC| of channel c over the whole pyramid (0 below
                             2^-20), rounding half away from zero.  Each level is
                             ceil(W_L/8) x ceil(H_L/8) blocks, edge texels repeated
                             past the level's edge, and is encoded in float64 from the
                             float32 level at creation.  Lookups decode the texels they
                             fetch (one per stochastic lookup) in float32. */
} stf_format;

typedef enum {
  STF_FILTER_LINEAR = 0,     /* tent kernel K1: bilinear / trilinear (Eq. 7, Eq. 8) */
  STF_FILTER_BSPLINE3 = 1,   /* cubic B-spline K_bs, 4 taps per axis (Eq. 9) */
  STF_FILTER_CATMULL_ROM = 2, /* cubic K3 with a = -1/2 (Appendix A), 4 taps per axis;
                                 stochastic form: one tap by |w| with scale sign * sum|w| */
  STF_FILTER_CATMULL_ROM_POSITIVIZED = 3, /* the same filter, stochastic form with
                                 positivization (Section 2.2; Appendix B): one tap from
                                 the positive and one from the negative weights,
                                 W+ t(j+) - W- t(j-); two texel fetches, lower variance.
                                 The deterministic form equals STF_FILTER_CATMULL_ROM.
                                 reuse_xi is ignored.  Not offered for neural textures. */
  /* Filter importance sampling (Section 4.4, "Filter Importance Sampling"): a
   * continuous offset s is drawn from a density and the texel nearest to x + s,
   * floor(x + s + 1/2), is returned unscaled.  The nearest-texel step convolves the
   * density with a unit box, which gives the filter each entry names.  reuse_xi is
   * ignored; not offered for neural textures. */
  STF_FILTER_FIS_LINEAR = 4,   /* s uniform on [-1/2, 1/2) per axis (one variate): the
                                  tent filter K1.  Deterministic form: STF_FILTER_LINEAR */
  STF_FILTER_FIS_BSPLINE3 = 5, /* s = sum of three uniforms on [-1/2, 1/2) per axis
                                  (the quadratic B-spline density): the cubic B-spline.
                                  Draws Philox streams 0, 1 and 2.  Deterministic form:
                                  STF_FILTER_BSPLINE3 */
  STF_FILTER_FIS_GAUSSIAN = 6  /* s = sigma * normal (Box-Muller on stream 0 words
                                  (0, 1), and (2, 3) for the z axis), sigma =
                                  params->filter_width in texels of the chosen level,
                                  0 < sigma <= STF_FIS_MAX_WIDTH.  The filter is the
                                  Gaussian convolved with the box; the deterministic
                                  form sums it over every tap within 5.77 sigma (the
                                  largest offset a 24-bit draw can make) */
} stf_filter;

#define STF_FIS_MAX_WIDTH 8.0f

typedef enum {
  STF_LEVEL_NEAREST = 0,   /* level floor(lod + 1/2) in both forms */
  STF_LEVEL_STOCHASTIC = 1 /* stochastic: floor(lod + u); deterministic: blend of
                              floor(lod) and the next level by frac(lod)
                              (trilinear MIP mapping, Section 2.1) */
} stf_level_mode;

/* Texture description for stf_create_texture.
 *   TEX2D:    dims = {W, H, 1}; channels in {1, 2, 4, 8}; format F32 or F16;
 *             mip_levels >= 1.  h_data/d_data holds float32 texels
 *             [level][y][x][channel]; all levels concatenated, level L being
 *             max(1, W >> L) x max(1, H >> L), unless generate_mips != 0, in which
 *             case it holds level 0 only and the library builds the other levels
 *             with a 2x2 box filter (power-of-two W and H required).
 *   DENSE3D:  dims = {X, Y, Z}; channels 1; format F32 or F16; float32 values
 *             [z][y][x].
 *   SPARSE3D: leaf_origins = num_leaves x 3 int32 (x, y, z), each a multiple of 8
 *             and distinct; data holds num_leaves x 512 float32 values, laid out
 *             [leaf][x & 7][y & 7][z & 7]; format F32 or E4M3_SCALED; dims ignored.
 *   data points to host memory if data_on_device == 0, else to device memory.
 *   The library copies (and quantises) the data; the caller keeps ownership.
 */
typedef struct {
  int32_t kind;           /* stf_kind */
  int32_t format;         /* stf_format */
  int32_t dims[3];
  int32_t channels;
  int32_t mip_levels;
  int32_t generate_mips;
  int32_t data_on_device;
  int32_t reserved0;
  const void* data;               /* float32 values, see above */
  const int32_t* leaf_origins;    /* sparse only; host or device per data_on_device */
  int64_t num_leaves;             /* sparse only */
  float background;               /* value outside the grid / in inactive regions */
  int32_t reserved1;
} stf_texture_desc;

/* Per-call lookup parameters. */
typedef struct {
  int32_t filter;         /* stf_filter */
  int32_t level_mode;     /* stf_level_mode; used only when d_lod != NULL */
  uint64_t seed;          /* Philox key */
  uint64_t query_offset;  /* q of the first query of this call */
  uint32_t sample_index;  /* third Philox counter word */
  int32_t bin_queries;    /* 1: counting-sort queries by spatial tile first
                             (same results, better gather locality) */
  int32_t reuse_xi;       /* 1: one variate carried across axes by the remapping
                             of Eq. 4 instead of one variate per axis */
  float filter_width;     /* STF_FILTER_FIS_GAUSSIAN: sigma in texels; ignored by the
                             other filters */
} stf_lookup_params;

/* Create a device-resident texture from desc: the texel function t of Section 2.1
 * (Eq. 1), non-zero at the discrete texel positions, whose filtered values the
 * lookups below return (the filter implementations of Appendix B take a texture and a
 * lookup position).  Queued on `stream`, and the call synchronises that stream before
 * returning so that the caller may free its data.  Returns STF_ERR_INVALID_ARGUMENT
 * for an inconsistent descriptor, STF_ERR_OUT_OF_MEMORY if device memory runs out
 * (nothing is leaked). */
stf_status stf_create_texture(const stf_texture_desc* desc, void* stream, stf_texture* out);

/* Release a texture created by stf_create_texture (the texel function of Section 2.1)
 * and everything it owns.  Waits for work queued on it. */
stf_status stf_destroy(stf_texture tex);

/* Stochastic filtered lookups (one texel per query; Eq. 3 with the sampling-arrays
 * rule of Section 2.2 applied per axis, Section 4.2).
 *   d_coords: n x 2 float32 (u, v) for TEX2D, n x 3 float32 (x, y, z) otherwise.
 *   d_lod:    NULL (level 0) or n float32 levels of detail (log2 footprint in level-0
 *             texels), TEX2D only.
 *   d_out:    n x channels float32, query-major.
 *   d_taps:   NULL or n x 4 int32 receiving the chosen texel (x, y, z, level) before
 *             clamping; level = -1 when nothing was fetched (non-finite input). */
stf_status stf_lookup_batch(stf_texture tex, const stf_lookup_params* params,
                            const float* d_coords, const float* d_lod, int64_t n,
                            float* d_out, int32_t* d_taps, void* stream);

/* Deterministic filtered lookups: the full 2^d or 4^d tap weighted sum (Eq. 2,
 * Eq. 9) with float32 accumulation; arguments as for stf_lookup_batch. */
stf_status stf_lookup_batch_deterministic(stf_texture tex, const stf_lookup_params* params,
                                          const float* d_coords, const float* d_lod,
                                          int64_t n, float* d_out, void* stream);

/* Validation accumulators for unbiasedness checks: for each query, n_samples
 * stochastic lookups with sample_index = params->sample_index + s, summed in
 * float64.  d_sum and d_sumsq are n x channels float64 (overwritten). */
stf_status stf_lookup_accumulate(stf_texture tex, const stf_lookup_params* params,
                                 const float* d_coords, const float* d_lod, int64_t n,
                                 int32_t n_samples, double* d_sum, double* d_sumsq,
                                 void* stream);

/* ---------------------------------------------------------------- anisotropic filtering
 *
 * 2D textures only.  d_grad holds, per query, the texture-coordinate derivatives
 * along the two screen axes (du/dx, dv/dx, du/dy, dv/dy) in uv units, float32,
 * 16-byte aligned.  In level-0 texels the footprint's axes are (du/dx W, dv/dx H) and
 * (du/dy W, dv/dy H); the longer is the major axis.  If the major axis is more than
 * max_anisotropy times the minor one, the minor axis is lengthened to
 * major / max_anisotropy (Section 5.2: the ratio is limited, 64 in the paper; pbrt
 * uses 8); lod = log2(minor length).  1 <= max_anisotropy <= STF_EWA_MAX_ANISOTROPY.
 * Derivatives that are not finite, or whose squared lengths in texels overflow
 * float32, give a NaN lod (stf_anisotropic_lod) or the background 0 with tap level -1
 * (the EWA lookups).  Every float32 step of the level and tap decisions is rounded
 * individually in a fixed order, so the choices are reproducible by any float32
 * implementation of the same steps. */
#define STF_EWA_MAX_ANISOTROPY 64.0f

/* Level of detail of each query's footprint (the anisotropic LOD of Section 5.2 and
 * Appendix B), clamped to [0, levels - 1]; d_lod (n floats, caller-owned) can be passed
 * to stf_lookup_batch, whose stochastic level choice floor(lod + u) is the listing's
 * jitter by u - 1/2 followed by rounding. */
stf_status stf_anisotropic_lod(stf_texture tex, const float* d_grad, int64_t n,
                               float max_anisotropy, float* d_lod, void* stream);

/* Elliptically weighted average (EWA; Section 4.2 and Appendix B, pbrt's filter).
 * The level is chosen from the footprint's lod as params->level_mode says (stochastic:
 * floor(lod + u) with word 3 of the query's Philox stream 0; nearest: floor(lod + 1/2)).
 * At level L (W_L x H_L texels) the axes are scaled to that level's texels (a minor
 * axis longer than 2 texels, possible only above the coarsest level, shrinks both
 * axes so that it is 2) and the filter is the Gaussian table
 * w = LUT[min(floor(Q * 128), 127)], LUT[i] = exp(-2 i/127) - exp(-2), over the
 * ellipse Q(s, t) = A s^2 + B s t + C t^2 < 1 centred on (u W_L - 1/2, v H_L - 1/2),
 * where (A, B, C) / F is the inverse of d0 d0^T + d1 d1^T + I; taps are clamped to the
 * edge.  stf_lookup_batch_ewa returns one texel of the ellipse's bounding box drawn
 * with probability w / sum(w): the smallest k, in row-major order (t, then s,
 * ascending), with u S < C_k (u = word 0 of stream 0).  d_taps (nullable) receives
 * (s, t, 0, L) of the drawn texel.  The deterministic form returns sum(w t) / sum(w)
 * at one level (nearest) or two levels blended by frac(lod) (stochastic level mode),
 * as pbrt does.  params->filter, reuse_xi and filter_width are ignored; bin_queries
 * is STF_ERR_UNSUPPORTED.  d_uv: n x 2 floats (8-byte aligned); d_out: n x channels
 * floats. */
stf_status stf_lookup_batch_ewa(stf_texture tex, const stf_lookup_params* params,
                                const float* d_uv, const float* d_grad, int64_t n,
                                float max_anisotropy, float* d_out, int32_t* d_taps,
                                void* stream);
stf_status stf_lookup_batch_ewa_deterministic(stf_texture tex, const stf_lookup_params* params,
                                              const float* d_uv, const float* d_grad, int64_t n,
                                              float max_anisotropy, float* d_out, void* stream);

/* The 128 float32 entries of the EWA weight table the library uses (host memory). */
stf_status stf_ewa_weight_table(float* h_out);

/* Triplanar mapping (Section 5.2, "Triplanar mapping"; Eq. 3) over a 2D texture (plain
 * or DCT6).  d_pos and d_normal: n x 3 floats each (4-byte aligned); the three planes
 * YZ, XZ and XY look the texture up at uv = scale (p_y, p_z), scale (p_x, p_z),
 * scale (p_x, p_y) with weights |n_x|, |n_y|, |n_z| / (|n_x| + |n_y| + |n_z|).  The
 * stochastic form draws one plane with probability equal to its weight (the smallest
 * k with u S < C_k over the planes in that order, float32, u = word 2 of the query's
 * Philox stream 0) and filters that plane's lookup stochastically with
 * params->filter (taps and level as stf_lookup_batch, words 0, 1 and 3); d_taps
 * (nullable) receives (x, y, plane, level).  The deterministic form blends the three
 * deterministic lookups.  d_lod (nullable) is one lod per query, used by every plane.
 * A non-finite position or normal, or a zero normal, gives 0 and tap level -1.
 * STF_FILTER_CATMULL_ROM_POSITIVIZED and bin_queries are STF_ERR_UNSUPPORTED. */
stf_status stf_lookup_batch_triplanar(stf_texture tex, const stf_lookup_params* params,
                                      const float* d_pos, const float* d_normal, const float* d_lod,
                                      int64_t n, float scale, float* d_out, int32_t* d_taps,
                                      void* stream);
stf_status stf_lookup_batch_triplanar_deterministic(stf_texture tex, const stf_lookup_params* params,
                                                    const float* d_pos, const float* d_normal,
                                                    const float* d_lod, int64_t n, float scale,
                                                    float* d_out, void* stream);

/* ---------------------------------------------------------------- neural textures
 *
 * A neural texture stores, for MIP levels 0 .. latent_levels-1, one latent texel
 * of STF_NEURAL_LATENT channels per texel, and a small decoder MLP that maps a
 * latent texel to the STF_NEURAL_OUT channels of the texel it stands for:
 *     H1 = relu(z W1 + b1), H2 = relu(H1 W2 + b2), y = H2 W3 + b3
 * with W1: 8x64, W2: 64x64, W3: 64x7 (row-major [in][out]).  Levels from
 * latent_levels up to levels-1 hold stored texels (the fallback).  The paper
 * motivates stochastic filtering for such expensive decoders (Section 1,
 * Section 5.2): the stochastic lookup decodes the one latent texel it picks, the
 * deterministic lookup decodes every tap and filters the decoded values.  Latents
 * and weights are used in binary16 by the tensor-core kernels (float32 masters are
 * kept for training); biases and accumulation are float32.
 * stf_lookup_batch / stf_lookup_batch_deterministic take (u, v) coordinates and an
 * optional level of detail as for 2D textures and write n x 7 floats. */
#define STF_NEURAL_LATENT 8
#define STF_NEURAL_HIDDEN 64
#define STF_NEURAL_OUT 7
#define STF_NEURAL_PARAMS (8 * 64 + 64 + 64 * 64 + 64 + 64 * 7 + 7) /* 5191 */

typedef struct {
  int32_t width, height;       /* level-0 size, powers of two */
  int32_t latent_levels;       /* 1 .. 4 */
  int32_t levels;              /* total levels >= latent_levels (<= log2(max(w,h)) + 1) */
  int32_t data_on_device;      /* pointers below are device (1) or host (0) memory */
  int32_t reserved;
  const float* latents;        /* [level][y][x][8] for the latent levels, concatenated */
  const float* params;         /* STF_NEURAL_PARAMS floats: W1, b1, W2, b2, W3, b3 */
  const float* fallback;       /* [level][y][x][7] for levels latent_levels .. levels-1,
                                  concatenated; NULL when levels == latent_levels */
} stf_neural_desc;

/* Create a neural texture (copies the data; synchronises `stream`). */
stf_status stf_create_neural_texture(const stf_neural_desc* desc, void* stream, stf_texture* out);

/* Loss and gradients of one batch, without changing the texture: texels given as
 * flat indices over the latent levels (level 0 texels first, row-major), targets as
 * batch x 7 floats.  d_param_grads (STF_NEURAL_PARAMS floats), d_latent_grads
 * (batch x 8) and d_loss (one float) may each be NULL; all are overwritten.  The
 * loss is (1 / batch) * sum over rows and channels of (y - target)^2.  batch must be
 * a multiple of 32. */
stf_status stf_neural_gradients(stf_texture tex, const int64_t* d_texels, int64_t batch,
                                const float* d_target_rows, float* d_param_grads,
                                float* d_latent_grads, float* d_loss, void* stream);

typedef struct {
  float lr_latent;   /* Adam step size for the latents */
  float lr_params;   /* Adam step size for the MLP parameters */
  float beta1, beta2, eps;
  int32_t batch;     /* texels per step (multiple of 32, at most the latent texel count) */
  uint64_t seed;     /* keys the permutation that orders texels into batches */
} stf_train_config;

/* Run `steps` Adam steps on the loss above.  Step s (counted from the texture's
 * creation) trains on texels perm((s * batch + i) mod N), i < batch, where perm is a
 * seeded bijection of the N latent texels, so every texel is visited once per epoch
 * and a batch holds distinct texels.  d_target holds the target texels of the
 * latent levels, [level][y][x][7] concatenated (float32, device).  d_loss_per_step,
 * if not NULL, receives one float per step. */
stf_status stf_neural_train(stf_texture tex, const float* d_target, const stf_train_config* cfg,
                            int32_t steps, float* d_loss_per_step, void* stream);

/* Copy the current float32 parameters (STF_NEURAL_PARAMS floats) and, if
 * d_latents is not NULL, the float32 latents ([level][y][x][8]) to device memory. */
stf_status stf_neural_read(stf_texture tex, float* d_params, float* d_latents, void* stream);

/* Largest n accepted by stf_lookup_batch_binned_noalloc. */
#define STF_NOALLOC_MAX_QUERIES (1 << 20)

/* Allocation-free Morton-binned stochastic lookup.  Same arguments and results as
 * stf_lookup_batch with params->bin_queries = 1 (bin_queries itself is ignored),
 * but the binning scratch lives in a fixed array inside the library's device
 * image (16 MiB plus 8 KiB, held by every GPU that loads the library until the process
 * exits) instead of device memory allocated per call.  It is meant for callers
 * that must not have the library allocate device memory: processes that reserve
 * their whole device-memory budget up front with their own allocator, and
 * callers that cannot accept the synchronisation an allocation may imply.  The
 * paper has no counterpart; this is an integration entry point.
 *   - n above STF_NOALLOC_MAX_QUERIES returns STF_ERR_INVALID_ARGUMENT.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any stream
 *     capture.
 *   - Every call shares the one array, which keeps the last call's contents (the
 *     bin counts are cleared at the start of each call).  Calls whose work
 *     overlaps on the GPU (different streams, or different host threads) race on
 *     it: serialise them, e.g. on one stream.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine. */
stf_status stf_lookup_batch_binned_noalloc(stf_texture tex, const stf_lookup_params* params,
                                           const float* d_coords, const float* d_lod, int64_t n,
                                           float* d_out, int32_t* d_taps, void* stream);

/* Bytes of device memory the texture holds (texels, tree nodes, scratch). */
stf_status stf_texture_bytes(stf_texture tex, int64_t* out_bytes);

/* Wait for `stream`, then report and clear the texture's device status word:
 * STF_ERR_DEVICE_ASSERT if a kernel flagged an inconsistent structure since the
 * last check, STF_ERR_CUDA if the stream reported an error, else STF_OK. */
stf_status stf_synchronize(stf_texture tex, void* stream);

/* Whether the current device can address `ptr` at that same address (*out = 1):
 * device or managed memory, or page-locked host memory mapped at its host address;
 * *out = 0 for other memory (pageable host memory, another process's memory).  With
 * host memory this lets a caller pass its host buffers to the lookups directly: the
 * kernels read the coordinates and write the results over the host link, which on
 * a Grace host moves them faster than staging copies for one pass (it is no
 * operation of the paper).  Errors: STF_ERR_INVALID_ARGUMENT for a NULL out,
 * STF_ERR_CUDA if the runtime cannot be queried (no device). */
stf_status stf_device_accessible(const void* ptr, int32_t* out);

/* Message of the last failed call on this thread ("" if none). */
const char* stf_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int32_t stf_version(void);

/* Failure-injection hook for tests of the error paths: the k-th device allocation
 * the library makes from now on fails as if the device were out of memory, and the
 * call that made it returns STF_ERR_OUT_OF_MEMORY with nothing leaked.  k <= 0
 * disables the hook.  Not thread-safe; meant for single-threaded tests. */
void stf_debug_fail_allocation(int64_t k);

#ifdef __cplusplus
}
#endif
#endif /* STF_H_ */
