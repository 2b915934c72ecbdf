// Anisotropic level of detail and EWA filtering of 2D textures.
//
// Level of detail (Section 5.2, "Anisotropic filtering and minification"; the
// anisotropic LOD listing of Appendix B): the footprint's axes are the texture-space
// derivatives along the two screen axes, in level-0 texels; the shorter is the minor
// axis, lengthened to major / max_anisotropy when the ratio exceeds the limit, and
// lod = log2(minor).
//
// EWA (Section 4.2 and the stochastic EWA listing of Appendix B, which samples
// pbrt's elliptically weighted average): at level L the filter is a Gaussian table
// over the ellipse Q(s, t) = A s^2 + B s t + C t^2 < 1, (A, B, C) / F being the
// inverse of d0 d0^T + d1 d1^T + I.  The stochastic form draws one texel of the
// ellipse's bounding box with probability w / sum(w) by inverse CDF over the texels
// in row-major order (two passes: the sum, then the search), the deterministic form
// returns sum(w t) / sum(w).  Every step of the tap decision is a float32 operation
// in a fixed order (no contraction), so any float32 implementation of the same steps
// makes the same choice.
#include <climits>
#include <cmath>
#include <cstring>

#include "stf_internal.h"

namespace stf {

constexpr int kEwaLut = 128;
constexpr int kEwaMaxSpan = 4096;   // bounding boxes are far smaller (see ewa_ellipse)
constexpr int kEwaRows = 48;        // rows whose running sums the stochastic search caches

// Gaussian weight table exp(-2 r) - exp(-2), r = i / 127, rounded to float32.  It is
// passed by value and staged in shared memory by every block.
struct EwaTable {
  float w[kEwaLut];
};

static const EwaTable& ewa_table() {
  static const EwaTable tab = [] {
    EwaTable t;
    for (int i = 0; i < kEwaLut; ++i) {
      const double r = (double)i / (double)(kEwaLut - 1);
      t.w[i] = (float)(std::exp(-2.0 * r) - std::exp(-2.0));
    }
    return t;
  }();
  return tab;
}

struct Footprint {
  float Mx, My;   // major axis, uv units
  float mx, my;   // minor axis after the anisotropy limit, uv units
  float lod;      // log2(minor length in level-0 texels); -inf for a zero footprint
  bool ok;        // finite uv, derivatives and squared lengths
};

__device__ __forceinline__ Footprint ewa_footprint(float4 g, float W, float H, float max_aniso) {
  Footprint f;
  const float axW = __fmul_rn(g.x, W), ayH = __fmul_rn(g.y, H);
  const float bxW = __fmul_rn(g.z, W), byH = __fmul_rn(g.w, H);
  const float la = __fadd_rn(__fmul_rn(axW, axW), __fmul_rn(ayH, ayH));
  const float lb = __fadd_rn(__fmul_rn(bxW, bxW), __fmul_rn(byH, byH));
  f.ok = isfinite(la) && isfinite(lb);
  const bool swap = la < lb;
  f.Mx = swap ? g.z : g.x;
  f.My = swap ? g.w : g.y;
  f.mx = swap ? g.x : g.z;
  f.my = swap ? g.y : g.w;
  const float major = __fsqrt_rn(swap ? lb : la);
  float minor = __fsqrt_rn(swap ? la : lb);
  if (minor > 0.0f && __fmul_rn(minor, max_aniso) < major) {
    const float scale = __fdiv_rn(major, __fmul_rn(minor, max_aniso));
    f.mx = __fmul_rn(f.mx, scale);
    f.my = __fmul_rn(f.my, scale);
    minor = __fmul_rn(minor, scale);
  }
  f.lod = log2f(minor);
  return f;
}

struct Ellipse {
  float A, B, C;
  int s0, s1, t0, t1;
  float st_s, st_t;
};

// Axes at level L in that level's texels; a minor axis longer than 2 texels (only
// when lod lies above the coarsest level) shrinks both axes so that it is 2.  The
// major axis is then at most 2 * max_anisotropy texels of the level (times the
// texture's aspect ratio at the clamped 1-texel levels), which bounds the box.
__device__ __forceinline__ Ellipse ewa_ellipse(const Footprint& f, float2 uv, float WL, float HL) {
  float d0u = __fmul_rn(f.Mx, WL), d0v = __fmul_rn(f.My, HL);
  float d1u = __fmul_rn(f.mx, WL), d1v = __fmul_rn(f.my, HL);
  const float m = __fsqrt_rn(__fadd_rn(__fmul_rn(d1u, d1u), __fmul_rn(d1v, d1v)));
  if (m > 2.0f) {
    const float k = __fdiv_rn(2.0f, m);
    d0u = __fmul_rn(d0u, k);
    d0v = __fmul_rn(d0v, k);
    d1u = __fmul_rn(d1u, k);
    d1v = __fmul_rn(d1v, k);
  }
  Ellipse e;
  float A = __fadd_rn(__fadd_rn(__fmul_rn(d0v, d0v), __fmul_rn(d1v, d1v)), 1.0f);
  float B = __fmul_rn(-2.0f, __fadd_rn(__fmul_rn(d0u, d0v), __fmul_rn(d1u, d1v)));
  float C = __fadd_rn(__fadd_rn(__fmul_rn(d0u, d0u), __fmul_rn(d1u, d1u)), 1.0f);
  const float F = __fsub_rn(__fmul_rn(A, C), __fmul_rn(__fmul_rn(B, B), 0.25f));
  const float inv = __fdiv_rn(1.0f, F);
  A = __fmul_rn(A, inv);
  B = __fmul_rn(B, inv);
  C = __fmul_rn(C, inv);
  const float det = __fsub_rn(__fmul_rn(__fmul_rn(4.0f, A), C), __fmul_rn(B, B));
  const float inv_det = __fdiv_rn(1.0f, det);
  const float hs = __fmul_rn(__fmul_rn(2.0f, inv_det), __fsqrt_rn(__fmul_rn(det, C)));
  const float ht = __fmul_rn(__fmul_rn(2.0f, inv_det), __fsqrt_rn(__fmul_rn(A, det)));
  e.A = A;
  e.B = B;
  e.C = C;
  // raster position, clamped to +-2^24 texels like the other 2D lookups (the taps are
  // clamped to the edge anyway), which keeps every loop index far from overflow
  e.st_s = fminf(fmaxf(__fsub_rn(__fmul_rn(uv.x, WL), 0.5f), -16777216.0f), 16777216.0f);
  e.st_t = fminf(fmaxf(__fsub_rn(__fmul_rn(uv.y, HL), 0.5f), -16777216.0f), 16777216.0f);
  e.s0 = (int)ceilf(__fsub_rn(e.st_s, hs));
  e.s1 = (int)floorf(__fadd_rn(e.st_s, hs));
  e.t0 = (int)ceilf(__fsub_rn(e.st_t, ht));
  e.t1 = (int)floorf(__fadd_rn(e.st_t, ht));
  return e;
}

__device__ __forceinline__ bool ewa_span_ok(const Ellipse& e) {
  return e.s1 - e.s0 < kEwaMaxSpan && e.t1 - e.t0 < kEwaMaxSpan;
}

// Terms of Q that are constant along row it: tt = it - st_t, B tt and C tt^2.
struct EwaRow {
  float tt, Btt, Ctt2;
};

__device__ __forceinline__ EwaRow ewa_row(const Ellipse& e, int it) {
  EwaRow r;
  r.tt = __fsub_rn((float)it, e.st_t);
  r.Btt = __fmul_rn(e.B, r.tt);
  r.Ctt2 = __fmul_rn(e.C, __fmul_rn(r.tt, r.tt));
  return r;
}

// Weight of texel (is, it); 0 outside the ellipse.  Q = (A ss + B tt) ss + C tt^2 in
// that order.  Q < 1 keeps the table index at most kEwaLut - 1; the lower clamp only
// guards a rounding-negative Q near the centre (index 0 either way).
__device__ __forceinline__ float ewa_weight(const Ellipse& e, const float* lut, int is, const EwaRow& row) {
  const float ss = __fsub_rn((float)is, e.st_s);
  const float r2 = __fadd_rn(__fmul_rn(__fadd_rn(__fmul_rn(e.A, ss), row.Btt), ss), row.Ctt2);
  if (!(r2 < 1.0f)) return 0.0f;
  return lut[max((int)__fmul_rn(r2, (float)kEwaLut), 0)];
}

struct EwaArgs {
  const float* uv;      // n x 2
  const float4* grad;   // n x (du/dx, dv/dx, du/dy, dv/dy)
  int64_t n;
  float* out;
  int32_t* taps;
  float* lod_out;       // stf_anisotropic_lod
  uint32_t key0, key1;
  uint64_t query_offset;
  uint32_t sample_index;
  int32_t level_mode;
  float max_aniso;
  unsigned* status;
};

// Per query: stochastic (one texel) or deterministic (weighted average, two levels
// blended by frac(lod) in the stochastic level mode).
template <int FMT, int C, bool STOCH>
__global__ void __launch_bounds__(256) k_ewa(Tex2DView t, EwaArgs a, EwaTable tab) {
  __shared__ float lut[kEwaLut];
  for (int k = threadIdx.x; k < kEwaLut; k += blockDim.x) lut[k] = tab.w[k];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float W0 = (float)t.level_w[0], H0 = (float)t.level_h[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float2 uv = reinterpret_cast<const float2*>(a.uv)[i];
    const float4 g = a.grad[i];
    float v[C];
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = 0.0f;
    int4 tap = make_int4(0, 0, 0, -1);
    const Footprint f = ewa_footprint(g, W0, H0, a.max_aniso);
    const bool finite_in = isfinite(uv.x) && isfinite(uv.y) && isfinite(g.x) && isfinite(g.y) &&
                           isfinite(g.z) && isfinite(g.w) && f.ok;
    if (finite_in) {
      const float lc = fminf(fmaxf(f.lod, 0.0f), (float)(t.levels - 1));
      int L0, L1 = 0;
      float frac = 0.0f;
      if (STOCH) {
        const uint64_t q = a.query_offset + (uint64_t)i;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), a.sample_index, 0u),
                                      a.key0, a.key1);
        const float u_level = a.level_mode == STF_LEVEL_NEAREST ? 0.5f : unit24(r.w);
        L0 = t.levels <= 1 ? 0 : min((int)floorf(__fadd_rn(lc, u_level)), t.levels - 1);
        const int WL = t.level_w[L0], HL = t.level_h[L0];
        const Ellipse e = ewa_ellipse(f, uv, (float)WL, (float)HL);
        if (!ewa_span_ok(e)) {
          atomicOr(a.status, STF_DEV_BAD_NODE);
        } else {
          // Pass 1: the running float32 sum, recorded at the end of each of the first
          // kEwaRows rows.  Pass 2 resumes from the last recorded value below u S, so it
          // rescans one row in the common case and repeats exactly the same additions.
          float S = 0.0f;
          float row_end[kEwaRows];
          // (adding a zero weight leaves a float32 sum unchanged, so texels outside
          // the ellipse are summed without a test)
          for (int it = e.t0; it <= e.t1; ++it) {
            const EwaRow row = ewa_row(e, it);
            for (int is = e.s0; is <= e.s1; ++is) S = __fadd_rn(S, ewa_weight(e, lut, is, row));
            if (it - e.t0 < kEwaRows) row_end[it - e.t0] = S;
          }
          const float us = __fmul_rn(unit24(r.x), S);
          float Cs = 0.0f;
          int start = e.t0;
          const int cached = min(e.t1 - e.t0 + 1, kEwaRows);
          for (int k = 0; k < cached && row_end[k] <= us; ++k) {
            Cs = row_end[k];
            start = e.t0 + k + 1;
          }
          int cs = INT_MIN, ct = 0;
          for (int it = start; it <= e.t1 && cs == INT_MIN; ++it) {
            const EwaRow row = ewa_row(e, it);
            for (int is = e.s0; is <= e.s1; ++is) {
              Cs = __fadd_rn(Cs, ewa_weight(e, lut, is, row));
              if (us < Cs) {   // never true right after a zero weight
                cs = is;
                ct = it;
                break;
              }
            }
          }
          if (cs == INT_MIN) {
            atomicOr(a.status, STF_DEV_BAD_NODE);   // cannot happen: us < S
          } else {
            tap = make_int4(cs, ct, 0, L0);
            fetch2d<FMT, C>(t, L0, min(max(cs, 0), WL - 1), min(max(ct, 0), HL - 1), v);
          }
        }
      } else {
        if (t.levels <= 1) {
          L0 = 0;
        } else if (a.level_mode == STF_LEVEL_NEAREST) {
          L0 = min((int)floorf(__fadd_rn(lc, 0.5f)), t.levels - 1);
        } else {
          L0 = (int)floorf(lc);
          frac = __fsub_rn(lc, (float)L0);
          L1 = min(L0 + 1, t.levels - 1);
        }
        for (int part = 0; part < (frac > 0.0f ? 2 : 1); ++part) {
          const int L = part ? L1 : L0;
          const float wl = part ? frac : 1.0f - frac;
          const int WL = t.level_w[L], HL = t.level_h[L];
          const Ellipse e = ewa_ellipse(f, uv, (float)WL, (float)HL);
          if (!ewa_span_ok(e)) {
            atomicOr(a.status, STF_DEV_BAD_NODE);
            continue;
          }
          float S = 0.0f, acc[C];
#pragma unroll
          for (int c = 0; c < C; ++c) acc[c] = 0.0f;
          for (int it = e.t0; it <= e.t1; ++it) {
            const EwaRow row = ewa_row(e, it);
            const int cy = min(max(it, 0), HL - 1);
            for (int is = e.s0; is <= e.s1; ++is) {
              const float w = ewa_weight(e, lut, is, row);
              if (w > 0.0f) {
                float tv[C];
                fetch2d<FMT, C>(t, L, min(max(is, 0), WL - 1), cy, tv);
                S = __fadd_rn(S, w);
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] = fmaf(w, tv[c], acc[c]);
              }
            }
          }
          const float k = __fdiv_rn(wl, S);
#pragma unroll
          for (int c = 0; c < C; ++c) v[c] = fmaf(k, acc[c], v[c]);
        }
      }
    }
    store_out<C>(a.out, i, v);
    if (STOCH && a.taps) reinterpret_cast<int4*>(a.taps)[i] = tap;
  }
}

__global__ void k_aniso_lod(EwaArgs a, float W0, float H0, int levels) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float4 g = a.grad[i];
    const Footprint f = ewa_footprint(g, W0, H0, a.max_aniso);
    const bool fin = isfinite(g.x) && isfinite(g.y) && isfinite(g.z) && isfinite(g.w) && f.ok;
    a.lod_out[i] = fin ? fminf(fmaxf(f.lod, 0.0f), (float)(levels - 1)) : __int_as_float(0x7fc00000);
  }
}

template <int FMT, int C>
static cudaError_t run_ewa(bool stoch, const Tex2DView& t, const EwaArgs& a, cudaStream_t s) {
  const int blocks = grid_blocks(a.n, 256);
  if (stoch) k_ewa<FMT, C, true><<<blocks, 256, 0, s>>>(t, a, ewa_table());
  else k_ewa<FMT, C, false><<<blocks, 256, 0, s>>>(t, a, ewa_table());
  return cudaGetLastError();
}

static cudaError_t launch_ewa(bool stoch, int fmt, int c, const Tex2DView& t, const EwaArgs& a,
                              cudaStream_t s) {
  if (fmt == STF_FMT_F32) {
    switch (c) {
      case 1: return run_ewa<STF_FMT_F32, 1>(stoch, t, a, s);
      case 2: return run_ewa<STF_FMT_F32, 2>(stoch, t, a, s);
      case 4: return run_ewa<STF_FMT_F32, 4>(stoch, t, a, s);
      case 8: return run_ewa<STF_FMT_F32, 8>(stoch, t, a, s);
    }
  } else if (fmt == STF_FMT_F16) {
    switch (c) {
      case 1: return run_ewa<STF_FMT_F16, 1>(stoch, t, a, s);
      case 2: return run_ewa<STF_FMT_F16, 2>(stoch, t, a, s);
      case 4: return run_ewa<STF_FMT_F16, 4>(stoch, t, a, s);
      case 8: return run_ewa<STF_FMT_F16, 8>(stoch, t, a, s);
    }
  } else if (fmt == STF_FMT_DCT6) {
    switch (c) {
      case 1: return run_ewa<STF_FMT_DCT6, 1>(stoch, t, a, s);
      case 2: return run_ewa<STF_FMT_DCT6, 2>(stoch, t, a, s);
      case 4: return run_ewa<STF_FMT_DCT6, 4>(stoch, t, a, s);
      case 8: return run_ewa<STF_FMT_DCT6, 8>(stoch, t, a, s);
    }
  }
  return cudaErrorInvalidValue;
}

static stf_status check_ewa(stf_texture t, const float* grad, int64_t n, float max_aniso) {
  if (!handle_ok(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
  if (t->kind != STF_KIND_TEX2D)
    return fail(STF_ERR_UNSUPPORTED, "anisotropic filtering is offered for 2D textures only");
  if (n < 0) return fail(STF_ERR_INVALID_ARGUMENT, "n < 0");
  if (!(max_aniso >= 1.0f && max_aniso <= STF_EWA_MAX_ANISOTROPY))
    return fail(STF_ERR_INVALID_ARGUMENT, "max_anisotropy %g outside [1, %g]", (double)max_aniso,
                (double)STF_EWA_MAX_ANISOTROPY);
  if (n > 0 && (!grad || (uintptr_t)grad % 16))
    return fail(STF_ERR_INVALID_ARGUMENT, "grad is NULL or not 16-byte aligned");
  return STF_OK;
}

static stf_status ewa_lookup(bool stoch, stf_texture t, const stf_lookup_params* p, const float* uv,
                             const float* grad, int64_t n, float max_aniso, float* out, int32_t* taps,
                             cudaStream_t s) {
  stf_status st = check_ewa(t, grad, n, max_aniso);
  if (st != STF_OK) return st;
  if (!p) return fail(STF_ERR_INVALID_ARGUMENT, "params is NULL");
  if (p->level_mode != STF_LEVEL_NEAREST && p->level_mode != STF_LEVEL_STOCHASTIC)
    return fail(STF_ERR_INVALID_ARGUMENT, "unknown level mode %d", p->level_mode);
  if (p->bin_queries) return fail(STF_ERR_UNSUPPORTED, "EWA lookups are not binned");
  if (n == 0) return STF_OK;
  if (!uv || (uintptr_t)uv % 8) return fail(STF_ERR_INVALID_ARGUMENT, "uv is NULL or not 8-byte aligned");
  const size_t oa = t->channels >= 4 ? 16 : (size_t)t->channels * 4;
  if (!out || (uintptr_t)out % oa) return fail(STF_ERR_INVALID_ARGUMENT, "out is NULL or not %zu-byte aligned", oa);
  if (taps && (uintptr_t)taps % 16) return fail(STF_ERR_INVALID_ARGUMENT, "taps not 16-byte aligned");
  EwaArgs a;
  memset(&a, 0, sizeof(a));
  a.uv = uv;
  a.grad = reinterpret_cast<const float4*>(grad);
  a.n = n;
  a.out = out;
  a.taps = taps;
  a.key0 = (uint32_t)p->seed;
  a.key1 = (uint32_t)(p->seed >> 32);
  a.query_offset = p->query_offset;
  a.sample_index = p->sample_index;
  a.level_mode = p->level_mode;
  a.max_aniso = max_aniso;
  a.status = t->d_status;
  const cudaError_t e = launch_ewa(stoch, t->format, t->channels, view2d(t), a, s);
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "EWA launch");
}

}  // namespace stf

using namespace stf;

extern "C" {

stf_status stf_anisotropic_lod(stf_texture t, const float* d_grad, int64_t n, float max_anisotropy,
                               float* d_lod, void* stream) {
  stf_status st = check_ewa(t, d_grad, n, max_anisotropy);
  if (st != STF_OK || n == 0) return st;
  if (!d_lod || (uintptr_t)d_lod % 4) return fail(STF_ERR_INVALID_ARGUMENT, "lod is NULL or misaligned");
  EwaArgs a;
  memset(&a, 0, sizeof(a));
  a.grad = reinterpret_cast<const float4*>(d_grad);
  a.n = n;
  a.lod_out = d_lod;
  a.max_aniso = max_anisotropy;
  k_aniso_lod<<<grid_blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(a, (float)t->level_w[0],
                                                                        (float)t->level_h[0], t->levels);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "anisotropic LOD launch");
}

stf_status stf_lookup_batch_ewa(stf_texture t, const stf_lookup_params* p, const float* d_uv,
                                const float* d_grad, int64_t n, float max_anisotropy, float* d_out,
                                int32_t* d_taps, void* stream) {
  return ewa_lookup(true, t, p, d_uv, d_grad, n, max_anisotropy, d_out, d_taps, (cudaStream_t)stream);
}

stf_status stf_lookup_batch_ewa_deterministic(stf_texture t, const stf_lookup_params* p,
                                              const float* d_uv, const float* d_grad, int64_t n,
                                              float max_anisotropy, float* d_out, void* stream) {
  return ewa_lookup(false, t, p, d_uv, d_grad, n, max_anisotropy, d_out, nullptr, (cudaStream_t)stream);
}

stf_status stf_ewa_weight_table(float* h_out) {
  if (!h_out) return fail(STF_ERR_INVALID_ARGUMENT, "out is NULL");
  memcpy(h_out, ewa_table().w, sizeof(float) * kEwaLut);
  return STF_OK;
}

}  // extern "C"
