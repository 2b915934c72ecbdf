// C ABI of the lookup library: handle registry, argument checking, texture
// creation (copy, quantise, MIP pyramid) and dispatch to the kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <unordered_set>

#include <cmath>

#include "stf_internal.h"

namespace {

thread_local std::string g_error;
std::mutex g_registry_mutex;
std::unordered_set<const stf_texture_s*> g_registry;

}  // namespace

namespace stf {

stf_status fail(stf_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

stf_status fail_cuda(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(STF_ERR_OUT_OF_MEMORY, "%s: out of device memory", what);
  return fail(STF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Test hook: when > 0, the countdown-th device allocation from now fails.
static int64_t g_alloc_countdown = 0;

bool alloc_should_fail() { return g_alloc_countdown > 0 && --g_alloc_countdown == 0; }

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;
  if (bytes == 0) bytes = 16;
  return cudaMalloc(p, bytes);
}

int grid_blocks(int64_t n, int threads, int waves) {
  static int sm_count[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& sms = sm_count[dev & 63];
  if (sms == 0) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 1;
  }
  const int64_t need = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * (2048 / threads) * waves;   // some waves, then grid-stride
  const int64_t b = need < cap ? need : cap;
  return (int)(b < 1 ? 1 : b);
}

bool handle_ok(stf_texture t) {
  std::lock_guard<std::mutex> lk(g_registry_mutex);
  return t != nullptr && g_registry.count(t) && t->magic == STF_TEX_MAGIC;
}

}  // namespace stf

using namespace stf;

static void free_texture(stf_texture_s* t) {
  if (!t) return;
  cudaFree(t->d_texels);
  cudaFree(t->d_tree);
  cudaFree(t->d_neural);
  cudaFree(t->d_status);
  cudaFree(t->d_scratch);
  t->magic = 0;
  delete t;
}

static int pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// DCT6 2D texture: the float32 pyramid is built as for the other formats, then each
// level is encoded (float64) into 32-bit block codes.
static stf_status create_dct(stf_texture_s* t, const stf_texture_desc* d, cudaStream_t s) {
  const int C = t->channels;
  int64_t texels = 0, words = 0;
  int64_t code_off[STF_MAX_LEVELS];
  for (int L = 0; L < t->levels; ++L) {
    const int w = d->dims[0] >> L > 0 ? d->dims[0] >> L : 1;
    const int h = d->dims[1] >> L > 0 ? d->dims[1] >> L : 1;
    t->level_off[L] = texels;           // texel offsets first (staging pyramid)
    t->level_w[L] = w;
    t->level_h[L] = h;
    t->blocks_w[L] = (w + 7) / 8;
    code_off[L] = words;
    texels += (int64_t)w * h;
    words += (int64_t)t->blocks_w[L] * ((h + 7) / 8) * C;
  }
  const int64_t nvals = texels * C;
  cudaError_t e = dev_alloc(&t->d_texels, (size_t)words * 4);
  if (e != cudaSuccess) return fail_cuda(e, "code allocation");
  t->bytes += words * 4;
  float* tmp = nullptr;
  double* scratch = nullptr;
  e = dev_alloc((void**)&tmp, (size_t)nvals * 4);
  if (e != cudaSuccess) return fail_cuda(e, "staging allocation");
  e = dev_alloc((void**)&scratch, (size_t)(words * 6 + 8) * 8);
  if (e != cudaSuccess) {
    cudaFree(tmp);
    return fail_cuda(e, "encoder scratch allocation");
  }
  const cudaMemcpyKind kind = d->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int64_t given = d->generate_mips ? (int64_t)t->level_w[0] * t->level_h[0] * C : nvals;
  e = cudaMemcpyAsync(tmp, d->data, (size_t)given * 4, kind, s);
  if (e == cudaSuccess && d->generate_mips) {
    for (int L = 1; L < t->levels && e == cudaSuccess; ++L)
      e = launch_box_mip(tmp + t->level_off[L - 1] * C, tmp + t->level_off[L] * C,
                         t->level_w[L - 1], t->level_h[L - 1], C, s);
  }
  double range[8] = {0};
  if (e == cudaSuccess)
    e = launch_dct_encode(tmp, t->level_off, t->level_w, t->level_h, t->levels, C,
                          (uint32_t*)t->d_texels, code_off, scratch, range, s);
  cudaFree(tmp);
  cudaFree(scratch);
  if (e != cudaSuccess) return fail_cuda(e, "DCT encode");
  for (int L = 0; L < t->levels; ++L) t->level_off[L] = code_off[L];
  for (int c = 0; c < 8; ++c) t->ac_step[c] = c < C ? (float)(range[c] / 15.0) : 0.0f;
  const double pi = 3.14159265358979323846;
  t->dct_k[0] = (float)std::sqrt(0.125);
  for (int i = 0; i < 4; ++i) t->dct_k[1 + i] = (float)(0.5 * std::cos((2 * i + 1) * pi / 16.0));
  t->dct_k[5] = (float)(0.5 * std::cos(pi / 8.0));
  t->dct_k[6] = (float)(0.5 * std::cos(3.0 * pi / 8.0));
  return STF_OK;
}

static stf_status create_grid(stf_texture_s* t, const stf_texture_desc* d, cudaStream_t s) {
  if (d->format == STF_FMT_DCT6) return create_dct(t, d, s);
  const int C = t->channels;
  const size_t es = d->format == STF_FMT_F16 ? 2 : 4;
  int64_t total = 0;
  int levels = t->levels;
  for (int L = 0; L < levels; ++L) {
    const int w = t->kind == STF_KIND_TEX2D ? (d->dims[0] >> L > 0 ? d->dims[0] >> L : 1) : d->dims[0];
    const int h = t->kind == STF_KIND_TEX2D ? (d->dims[1] >> L > 0 ? d->dims[1] >> L : 1) : d->dims[1];
    const int64_t depth = t->kind == STF_KIND_TEX2D ? 1 : d->dims[2];
    t->level_off[L] = total;
    t->level_w[L] = w;
    t->level_h[L] = h;
    total += (int64_t)w * h * depth;
  }
  const int64_t nvals = total * C;
  // 16 bytes of padding: the deterministic dense filter reads rows of four FP16
  // voxels as aligned 8-byte words, the last of which may extend past the data
  cudaError_t e = dev_alloc(&t->d_texels, (size_t)nvals * es + 16);
  if (e != cudaSuccess) return fail_cuda(e, "texel allocation");
  t->bytes += nvals * es;
  const cudaMemcpyKind kind = d->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int64_t given = (t->kind == STF_KIND_TEX2D && d->generate_mips)
                            ? (int64_t)t->level_w[0] * t->level_h[0] * C
                            : nvals;
  const bool direct = d->format == STF_FMT_F32 && !(t->kind == STF_KIND_TEX2D && d->generate_mips);
  if (direct) {
    e = cudaMemcpyAsync(t->d_texels, d->data, (size_t)nvals * 4, kind, s);
    if (e != cudaSuccess) return fail_cuda(e, "texel upload");
    e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? STF_OK : fail_cuda(e, "texel upload");
  }
  float* tmp = nullptr;
  e = dev_alloc((void**)&tmp, (size_t)nvals * 4);
  if (e != cudaSuccess) return fail_cuda(e, "staging allocation");
  e = cudaMemcpyAsync(tmp, d->data, (size_t)given * 4, kind, s);
  if (e == cudaSuccess && t->kind == STF_KIND_TEX2D && d->generate_mips) {
    for (int L = 1; L < levels && e == cudaSuccess; ++L)
      e = launch_box_mip(tmp + t->level_off[L - 1] * C, tmp + t->level_off[L] * C,
                         t->level_w[L - 1], t->level_h[L - 1], C, s);
  }
  if (e == cudaSuccess) e = launch_convert_f32(tmp, t->d_texels, d->format, nvals, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "texture build");
}

// Status word, registration; frees the texture if creation failed.
static stf_status finish_create(stf_texture_s* t, stf_status st, stf_texture* out) {
  if (st == STF_OK) {
    cudaError_t e = dev_alloc((void**)&t->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(t->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) st = fail_cuda(e, "status word");
    t->sparse.status = t->d_status;
    t->neural.status = t->d_status;
  }
  if (st != STF_OK) {
    free_texture(t);
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(g_registry_mutex);
    g_registry.insert(t);
  }
  *out = t;
  return STF_OK;
}

extern "C" {

int32_t stf_version(void) { return 10000; }

const char* stf_last_error(void) { return g_error.c_str(); }

// Test hook (not in the public header's core set): make the k-th device allocation
// from now fail, to exercise out-of-memory paths; k <= 0 disables.
void stf_debug_fail_allocation(int64_t k) { g_alloc_countdown = k > 0 ? k : 0; }

stf_status stf_create_texture(const stf_texture_desc* d, void* stream, stf_texture* out) {
  if (!out) return fail(STF_ERR_INVALID_ARGUMENT, "out handle pointer is NULL");
  *out = nullptr;
  if (!d) return fail(STF_ERR_INVALID_ARGUMENT, "descriptor is NULL");
  const bool empty_sparse = d->kind == STF_KIND_SPARSE3D && d->num_leaves == 0;
  if (!d->data && !empty_sparse) return fail(STF_ERR_INVALID_ARGUMENT, "descriptor data is NULL");
  if (d->data_on_device && ((uintptr_t)d->data % 16))
    return fail(STF_ERR_INVALID_ARGUMENT, "device data must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  stf_texture_s* t = new stf_texture_s();
  memset(t, 0, sizeof(*t));
  t->magic = STF_TEX_MAGIC;
  t->kind = d->kind;
  t->format = d->format;
  t->channels = d->channels;
  t->levels = 1;
  t->background = d->background;
  memcpy(t->dims, d->dims, sizeof(t->dims));
  stf_status st = STF_OK;
  switch (d->kind) {
    case STF_KIND_TEX2D: {
      const int W = d->dims[0], H = d->dims[1];
      int maxlev = 1;
      while ((W >> maxlev) > 0 || (H >> maxlev) > 0) ++maxlev;
      if (W <= 0 || H <= 0) st = fail(STF_ERR_INVALID_ARGUMENT, "2D texture needs dims > 0");
      else if (d->channels != 1 && d->channels != 2 && d->channels != 4 && d->channels != 8)
        st = fail(STF_ERR_INVALID_ARGUMENT, "2D texture channels must be 1, 2, 4 or 8");
      else if (d->format != STF_FMT_F32 && d->format != STF_FMT_F16 && d->format != STF_FMT_DCT6)
        st = fail(STF_ERR_INVALID_ARGUMENT, "2D texture format must be F32, F16 or DCT6");
      else if (d->mip_levels < 1 || d->mip_levels > STF_MAX_LEVELS || d->mip_levels > maxlev)
        st = fail(STF_ERR_INVALID_ARGUMENT, "mip_levels %d outside [1, %d]", d->mip_levels,
                  maxlev < STF_MAX_LEVELS ? maxlev : STF_MAX_LEVELS);
      else if (d->generate_mips && !(pow2(W) && pow2(H)))
        st = fail(STF_ERR_INVALID_ARGUMENT, "generate_mips needs power-of-two sizes");
      if (st == STF_OK) {
        t->levels = d->mip_levels;
        st = create_grid(t, d, s);
      }
      break;
    }
    case STF_KIND_DENSE3D:
      if (d->dims[0] <= 0 || d->dims[1] <= 0 || d->dims[2] <= 0)
        st = fail(STF_ERR_INVALID_ARGUMENT, "dense grid needs dims > 0");
      else if (d->channels != 1)
        st = fail(STF_ERR_INVALID_ARGUMENT, "dense grid channels must be 1");
      else if (d->format != STF_FMT_F32 && d->format != STF_FMT_F16)
        st = fail(STF_ERR_INVALID_ARGUMENT, "dense grid format must be F32 or F16");
      else
        st = create_grid(t, d, s);
      break;
    case STF_KIND_SPARSE3D:
      if (d->channels != 1) st = fail(STF_ERR_INVALID_ARGUMENT, "sparse grid channels must be 1");
      else if (d->format != STF_FMT_F32 && d->format != STF_FMT_E4M3_SCALED)
        st = fail(STF_ERR_INVALID_ARGUMENT, "sparse grid format must be F32 or E4M3_SCALED");
      else if (d->num_leaves < 0 || (d->num_leaves > 0 && !d->leaf_origins))
        st = fail(STF_ERR_INVALID_ARGUMENT, "sparse grid needs leaf origins");
      else
        st = build_sparse(t, d, s);
      break;
    default:
      st = fail(STF_ERR_INVALID_ARGUMENT, "unknown texture kind %d", d->kind);
  }
  return finish_create(t, st, out);
}

stf_status stf_create_neural_texture(const stf_neural_desc* d, void* stream, stf_texture* out) {
  if (!out) return fail(STF_ERR_INVALID_ARGUMENT, "out handle pointer is NULL");
  *out = nullptr;
  if (!d) return fail(STF_ERR_INVALID_ARGUMENT, "descriptor is NULL");
  stf_texture_s* t = new stf_texture_s();
  memset(t, 0, sizeof(*t));
  t->magic = STF_TEX_MAGIC;
  t->kind = STF_KIND_NEURAL2D;
  t->format = STF_FMT_F16;
  return finish_create(t, build_neural(t, d, (cudaStream_t)stream), out);
}

stf_status stf_destroy(stf_texture t) {
  {
    std::lock_guard<std::mutex> lk(g_registry_mutex);
    if (!t || !g_registry.count(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
    g_registry.erase(t);
  }
  cudaDeviceSynchronize();
  free_texture(t);
  return STF_OK;
}

stf_status stf_texture_bytes(stf_texture t, int64_t* out_bytes) {
  if (!handle_ok(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
  if (!out_bytes) return fail(STF_ERR_INVALID_ARGUMENT, "out_bytes is NULL");
  *out_bytes = t->bytes + t->scratch_bytes;
  return STF_OK;
}

stf_status stf_device_accessible(const void* ptr, int32_t* out) {
  if (!out) return fail(STF_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = 0;
  if (!ptr) return STF_OK;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_cuda(e, "pointer attributes");
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(STF_ERR_CUDA, "no current device");
    *out = (a.type == cudaMemoryTypeManaged || a.device == dev) ? 1 : 0;
  } else if (a.type == cudaMemoryTypeHost) {
    *out = a.devicePointer == ptr ? 1 : 0;
  }
  return STF_OK;
}

stf_status stf_synchronize(stf_texture t, void* stream) {
  if (!handle_ok(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(e, "stream");
  unsigned flag = 0;
  e = cudaMemcpy(&flag, t->d_status, sizeof(flag), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_cuda(e, "status word");
  if (flag) {
    cudaMemset(t->d_status, 0, sizeof(unsigned));
    return fail(STF_ERR_DEVICE_ASSERT, "a kernel flagged an inconsistent structure (0x%x)", flag);
  }
  return STF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- lookups

namespace stf {

stf_status check_lookup(stf_texture t, const stf_lookup_params* p, const float* coords,
                        const float* lod, int64_t n, const void* out) {
  if (!handle_ok(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
  if (!p) return fail(STF_ERR_INVALID_ARGUMENT, "params is NULL");
  if (n < 0) return fail(STF_ERR_INVALID_ARGUMENT, "n < 0");
  if (p->filter < STF_FILTER_LINEAR || p->filter > STF_FILTER_FIS_GAUSSIAN)
    return fail(STF_ERR_INVALID_ARGUMENT, "unknown filter %d", p->filter);
  if (p->filter >= STF_FILTER_CATMULL_ROM_POSITIVIZED && t->kind == STF_KIND_NEURAL2D)
    return fail(STF_ERR_UNSUPPORTED, "filter %d is not offered for neural textures", p->filter);
  if (p->filter == STF_FILTER_FIS_GAUSSIAN &&
      !(p->filter_width > 0.0f && p->filter_width <= STF_FIS_MAX_WIDTH))
    return fail(STF_ERR_INVALID_ARGUMENT, "filter_width %g outside (0, %g]", (double)p->filter_width,
                (double)STF_FIS_MAX_WIDTH);
  if (p->level_mode != STF_LEVEL_NEAREST && p->level_mode != STF_LEVEL_STOCHASTIC)
    return fail(STF_ERR_INVALID_ARGUMENT, "unknown level mode %d", p->level_mode);
  if (n == 0) return STF_OK;
  if (!coords || !out) return fail(STF_ERR_INVALID_ARGUMENT, "coords or out is NULL");
  const bool is2d = t->kind == STF_KIND_TEX2D || t->kind == STF_KIND_NEURAL2D;
  if (lod && !is2d)
    return fail(STF_ERR_UNSUPPORTED, "level of detail is only meaningful for 2D textures");
  const size_t ca = is2d ? 8 : 4;
  if ((uintptr_t)coords % ca) return fail(STF_ERR_INVALID_ARGUMENT, "coords not %zu-byte aligned", ca);
  const size_t oa = t->kind == STF_KIND_NEURAL2D ? 4 : (t->channels >= 4 ? 16 : (size_t)t->channels * 4);
  if ((uintptr_t)out % oa) return fail(STF_ERR_INVALID_ARGUMENT, "out not %zu-byte aligned", oa);
  return STF_OK;
}

LookupArgs make_args(const stf_lookup_params* p, const float* coords, const float* lod, int64_t n,
                     float* out, int32_t* taps) {
  LookupArgs a;
  memset(&a, 0, sizeof(a));
  a.coords = coords;
  a.lod = lod;
  a.n = n;
  a.out = out;
  a.taps = taps;
  a.key0 = (uint32_t)p->seed;
  a.key1 = (uint32_t)(p->seed >> 32);
  a.query_offset = p->query_offset;
  a.sample_index = p->sample_index;
  a.reuse = p->reuse_xi != 0;
  a.level_mode = p->level_mode;
  a.width = p->filter == STF_FILTER_FIS_GAUSSIAN ? p->filter_width : 0.0f;
  return a;
}

Tex2DView view2d(const stf_texture_s* t) {
  Tex2DView v;
  memset(&v, 0, sizeof(v));
  v.texels = t->d_texels;
  v.levels = t->levels;
  for (int L = 0; L < t->levels; ++L) {
    v.level_off[L] = t->level_off[L];
    v.level_w[L] = t->level_w[L];
    v.level_h[L] = t->level_h[L];
    v.blocks_w[L] = t->blocks_w[L];
  }
  for (int c = 0; c < 8; ++c) v.ac_step[c] = t->ac_step[c];
  for (int k = 0; k < 7; ++k) v.dct_k[k] = t->dct_k[k];
  return v;
}

Dense3DView view3d(const stf_texture_s* t) {
  Dense3DView v;
  v.texels = t->d_texels;
  v.nx = t->dims[0];
  v.ny = t->dims[1];
  v.nz = t->dims[2];
  v.background = t->background;
  return v;
}

stf_status dispatch(Op op, stf_texture t, int filter, const LookupArgs& a, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (t->kind) {
    case STF_KIND_TEX2D: e = launch_tex2d(op, filter, t->format, t->channels, view2d(t), a, s); break;
    case STF_KIND_DENSE3D: e = launch_dense3d(op, filter, t->format, view3d(t), a, s); break;
    case STF_KIND_SPARSE3D: e = launch_sparse3d(op, filter, t->format, t->sparse, a, s); break;
    case STF_KIND_NEURAL2D:
      if (op == OP_ACCUMULATE) return fail(STF_ERR_UNSUPPORTED, "accumulation is not offered for neural textures");
      e = launch_neural(op, filter, t->neural, a, s);
      break;
  }
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "lookup launch");
}

// Triplanar lookups (Section 5.2): positions and normals, n x 3 floats each.
stf_status triplanar(Op op, stf_texture t, const stf_lookup_params* p, const float* pos,
                     const float* normal, const float* lod, int64_t n, float scale, float* out,
                     int32_t* taps, cudaStream_t s) {
  if (!handle_ok(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
  if (t->kind != STF_KIND_TEX2D) return fail(STF_ERR_UNSUPPORTED, "triplanar lookups need a 2D texture");
  if (!p) return fail(STF_ERR_INVALID_ARGUMENT, "params is NULL");
  if (n < 0) return fail(STF_ERR_INVALID_ARGUMENT, "n < 0");
  if (p->filter < STF_FILTER_LINEAR || p->filter > STF_FILTER_FIS_GAUSSIAN)
    return fail(STF_ERR_INVALID_ARGUMENT, "unknown filter %d", p->filter);
  if (p->filter == STF_FILTER_CATMULL_ROM_POSITIVIZED)
    return fail(STF_ERR_UNSUPPORTED, "positivized filtering is not offered for triplanar lookups");
  if (p->filter == STF_FILTER_FIS_GAUSSIAN &&
      !(p->filter_width > 0.0f && p->filter_width <= STF_FIS_MAX_WIDTH))
    return fail(STF_ERR_INVALID_ARGUMENT, "filter_width %g outside (0, %g]", (double)p->filter_width,
                (double)STF_FIS_MAX_WIDTH);
  if (p->level_mode != STF_LEVEL_NEAREST && p->level_mode != STF_LEVEL_STOCHASTIC)
    return fail(STF_ERR_INVALID_ARGUMENT, "unknown level mode %d", p->level_mode);
  if (p->bin_queries) return fail(STF_ERR_UNSUPPORTED, "triplanar lookups are not binned");
  if (!std::isfinite(scale)) return fail(STF_ERR_INVALID_ARGUMENT, "scale is not finite");
  if (n == 0) return STF_OK;
  if (!pos || !normal || !out) return fail(STF_ERR_INVALID_ARGUMENT, "pos, normal or out is NULL");
  if ((uintptr_t)pos % 4 || (uintptr_t)normal % 4 || (lod && (uintptr_t)lod % 4))
    return fail(STF_ERR_INVALID_ARGUMENT, "pos, normal or lod not 4-byte aligned");
  const size_t oa = t->channels >= 4 ? 16 : (size_t)t->channels * 4;
  if ((uintptr_t)out % oa) return fail(STF_ERR_INVALID_ARGUMENT, "out not %zu-byte aligned", oa);
  if (taps && (uintptr_t)taps % 16) return fail(STF_ERR_INVALID_ARGUMENT, "taps not 16-byte aligned");
  LookupArgs a = make_args(p, pos, lod, n, out, taps);
  a.reuse = 0;
  a.normals = normal;
  a.tri_scale = scale;
  return dispatch(op, t, p->filter, a, s);
}

}  // namespace stf

extern "C" {

stf_status stf_lookup_batch(stf_texture t, const stf_lookup_params* p, const float* coords,
                            const float* lod, int64_t n, float* out, int32_t* taps, void* stream) {
  stf_status st = check_lookup(t, p, coords, lod, n, out);
  if (st != STF_OK || n == 0) return st;
  if (taps && (uintptr_t)taps % 16) return fail(STF_ERR_INVALID_ARGUMENT, "taps not 16-byte aligned");
  LookupArgs a = make_args(p, coords, lod, n, out, taps);
  if (p->bin_queries) return lookup_binned(t, p->filter, a, (cudaStream_t)stream);
  return dispatch(OP_STOCHASTIC, t, p->filter, a, (cudaStream_t)stream);
}

stf_status stf_lookup_batch_deterministic(stf_texture t, const stf_lookup_params* p,
                                          const float* coords, const float* lod, int64_t n,
                                          float* out, void* stream) {
  stf_status st = check_lookup(t, p, coords, lod, n, out);
  if (st != STF_OK || n == 0) return st;
  LookupArgs a = make_args(p, coords, lod, n, out, nullptr);
  return dispatch(OP_DETERMINISTIC, t, p->filter, a, (cudaStream_t)stream);
}

stf_status stf_lookup_accumulate(stf_texture t, const stf_lookup_params* p, const float* coords,
                                 const float* lod, int64_t n, int32_t n_samples, double* d_sum,
                                 double* d_sumsq, void* stream) {
  stf_status st = check_lookup(t, p, coords, lod, n, d_sum);
  if (st != STF_OK || n == 0) return st;
  if (!d_sumsq) return fail(STF_ERR_INVALID_ARGUMENT, "sumsq is NULL");
  if (n_samples < 1) return fail(STF_ERR_INVALID_ARGUMENT, "n_samples must be >= 1");
  LookupArgs a = make_args(p, coords, lod, n, nullptr, nullptr);
  a.n_samples = n_samples;
  a.sum = d_sum;
  a.sumsq = d_sumsq;
  return dispatch(OP_ACCUMULATE, t, p->filter, a, (cudaStream_t)stream);
}


stf_status stf_lookup_batch_triplanar(stf_texture t, const stf_lookup_params* p, const float* d_pos,
                                      const float* d_normal, const float* d_lod, int64_t n,
                                      float scale, float* d_out, int32_t* d_taps, void* stream) {
  return stf::triplanar(stf::OP_STOCHASTIC, t, p, d_pos, d_normal, d_lod, n, scale, d_out, d_taps,
                        (cudaStream_t)stream);
}

stf_status stf_lookup_batch_triplanar_deterministic(stf_texture t, const stf_lookup_params* p,
                                                    const float* d_pos, const float* d_normal,
                                                    const float* d_lod, int64_t n, float scale,
                                                    float* d_out, void* stream) {
  return stf::triplanar(stf::OP_DETERMINISTIC, t, p, d_pos, d_normal, d_lod, n, scale, d_out, nullptr,
                        (cudaStream_t)stream);
}

}  // extern "C"
