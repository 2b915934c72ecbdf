// Lookup kernels for 2D MIP-mapped textures, shared by the translation units that
// instantiate them for the plain (FP32 / FP16) and the DCT-compressed formats.
//
// One thread per query (grid-stride).  The stochastic kernels pick a level and one
// tap per axis by inverse CDF over |w| (sampling arrays, Section 2.2; separable
// sampling, Section 4.2), by positivization or by filter importance sampling, and
// fetch one texel (Eq. 3); the deterministic kernels sum every tap (Eq. 2, Eq. 9)
// over one level or two blended by frac(lod); the accumulate kernels repeat the
// stochastic form over many sample indices in float64 (validation only).
//
// Triplanar mapping (Section 5.2, "Triplanar mapping"): the query is a position p
// and a normal n; the three planes YZ, XZ, XY (uv = scale (p_y, p_z), scale (p_x, p_z),
// scale (p_x, p_y)) carry weights |n_x|, |n_y|, |n_z|.  Stochastically one plane is
// drawn with probability equal to its normalised weight (Eq. 3; inverse CDF in float32
// on word 2 of the query's stream 0) and its lookup is filtered stochastically; the
// deterministic form blends the three deterministic lookups.
#pragma once
#include "stf_launch.h"

namespace stf {

// Level choice: floor(lod + 1/2) (nearest) or floor(lod + u) (stochastic), lod
// clamped to [0, levels - 1].
__device__ __forceinline__ int level_stochastic(const Tex2DView& t, const LookupArgs& a,
                                                float lod, float u) {
  if (a.lod == nullptr || t.levels <= 1) return 0;
  const float lc = fminf(fmaxf(lod, 0.0f), (float)(t.levels - 1));
  const float s = __fadd_rn(lc, a.level_mode == STF_LEVEL_NEAREST ? 0.5f : u);
  return min((int)floorf(s), t.levels - 1);
}

template <int FMT, int C>
__device__ __forceinline__ void fetch_clamped(const Tex2DView& t, int L, int ix, int iy, float* v) {
  fetch2d<FMT, C>(t, L, min(max(ix, 0), t.level_w[L] - 1), min(max(iy, 0), t.level_h[L] - 1), v);
}

// One stochastic lookup at (uv, lod) with the variates r of caller query j.
template <int F, int FMT, int C, bool REUSE>
__device__ __forceinline__ void tex2d_stochastic_at(const Tex2DView& t, const LookupArgs& a,
                                                    float2 uv, float lod, int64_t j, uint32_t sample,
                                                    const uint4& r, float* v, int4& tap) {
  const int L = level_stochastic(t, a, lod, unit24(r.w));
  const int W = t.level_w[L], H = t.level_h[L];
  float x[2] = {__fsub_rn(__fmul_rn(uv.x, (float)W), 0.5f),
                __fsub_rn(__fmul_rn(uv.y, (float)H), 0.5f)};
  if (!(prepare_coords<2>(x) && isfinite(lod))) {
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = 0.0f;
    tap = make_int4(0, 0, 0, -1);
    return;
  }
  if constexpr (IsFis<F>::value) {
    int idx[2];
    pick_fis<F, 2>(x, a, j, sample, r, idx);
    tap = make_int4(idx[0], idx[1], 0, L);
    fetch_clamped<FMT, C>(t, L, idx[0], idx[1], v);
  } else if constexpr (F == STF_FILTER_CATMULL_ROM_POSITIVIZED) {
    const uint4 r1 = query_variates(a, j, sample, 1u);
    const float up[3] = {unit24(r.x), unit24(r.y), unit24(r.z)};
    const float un[3] = {unit24(r1.x), unit24(r1.y), unit24(r1.z)};
    int ip[2], in[2];
    float Wp, Wn;
    pick_positivized<2>(x, up, un, ip, in, Wp, Wn);
    tap = make_int4(ip[0], ip[1], 0, L);
    fetch_clamped<FMT, C>(t, L, ip[0], ip[1], v);
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] *= Wp;
    if (Wn > 0.0f) {
      float tn[C];
      fetch_clamped<FMT, C>(t, L, in[0], in[1], tn);
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = fmaf(-Wn, tn[c], v[c]);
    }
  } else {
    int idx[2];
    const float sigma = pick_taps_r<F, 2, REUSE>(x, r, idx);
    tap = make_int4(idx[0], idx[1], 0, L);
    fetch_clamped<FMT, C>(t, L, idx[0], idx[1], v);
    if constexpr (!Filter<F>::NONNEG) {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] *= sigma;
    }
  }
}

// One stochastic lookup of query i (caller's index j); I is int64_t, or uint32_t in the
// fast loop.
template <int F, int FMT, int C, bool REUSE, typename I>
__device__ __forceinline__ void tex2d_stochastic_one(const Tex2DView& t, const LookupArgs& a,
                                                     I i, I j, uint32_t sample,
                                                     float* v, int4& tap) {
  const float2 uv = reinterpret_cast<const float2*>(a.coords)[i];
  const float lod = a.lod ? a.lod[i] : 0.0f;
  const uint4 r = query_variates(a, j, sample);
  tex2d_stochastic_at<F, FMT, C, REUSE>(t, a, uv, lod, j, sample, r, v, tap);
}

// Deterministic filter at one level, weighted by `scale`, added to acc.
template <int F, int FMT, int C>
__device__ __forceinline__ void tex2d_det_level(const Tex2DView& t, int L, float2 uv, float scale,
                                                float width, float* acc) {
  using Fl = Filter<F>;
  const int W = t.level_w[L], H = t.level_h[L];
  float x[2] = {__fsub_rn(__fmul_rn(uv.x, (float)W), 0.5f),
                __fsub_rn(__fmul_rn(uv.y, (float)H), 0.5f)};
  if (!prepare_coords<2>(x)) return;
  if constexpr (F == STF_FILTER_FIS_GAUSSIAN) {
    const GaussAxis gx = gauss_axis(x[0], width), gy = gauss_axis(x[1], width);
    float ey0 = gauss_edge(gy, gy.lo);
    for (int iy = gy.lo; iy <= gy.hi; ++iy) {
      const float ey1 = gauss_edge(gy, iy + 1);
      const float wy = 0.5f * (ey1 - ey0) * scale;
      ey0 = ey1;
      const int cy = min(max(iy, 0), H - 1);
      float ex0 = gauss_edge(gx, gx.lo);
      for (int ix = gx.lo; ix <= gx.hi; ++ix) {
        const float ex1 = gauss_edge(gx, ix + 1);
        const float w = 0.5f * (ex1 - ex0) * wy;
        ex0 = ex1;
        float tv[C];
        fetch2d<FMT, C>(t, L, min(max(ix, 0), W - 1), cy, tv);
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(w, tv[c], acc[c]);
      }
    }
  } else {
    float fx, fy;
    const int bx = axis_base(x[0], fx) + Fl::OFF0, by = axis_base(x[1], fy) + Fl::OFF0;
    float wx[Fl::T], wy[Fl::T];
    Fl::weights(fx, wx);
    Fl::weights(fy, wy);
    int cxs[Fl::T];
#pragma unroll
    for (int k = 0; k < Fl::T; ++k) cxs[k] = min(max(bx + k, 0), W - 1);
#pragma unroll
    for (int ky = 0; ky < Fl::T; ++ky) {
      const int cy = min(max(by + ky, 0), H - 1);
      const float wyk = wy[ky] * scale;
#pragma unroll
      for (int kx = 0; kx < Fl::T; ++kx) {
        float tv[C];
        fetch2d<FMT, C>(t, L, cxs[kx], cy, tv);
        const float w = wx[kx] * wyk;
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(w, tv[c], acc[c]);
      }
    }
  }
}

// Deterministic lookup at (uv, lod) weighted by `scale`, added to acc: one level
// (nearest mode or no lod) or floor(lod) and the next blended by frac(lod).
template <int F, int FMT, int C>
__device__ __forceinline__ void tex2d_det_at(const Tex2DView& t, const LookupArgs& a, float2 uv,
                                             float lod, float scale, float* acc) {
  if (!isfinite(lod)) return;
  if (a.lod == nullptr || t.levels <= 1) {
    tex2d_det_level<F, FMT, C>(t, 0, uv, scale, a.width, acc);
    return;
  }
  const float lc = fminf(fmaxf(lod, 0.0f), (float)(t.levels - 1));
  if (a.level_mode == STF_LEVEL_NEAREST) {
    tex2d_det_level<F, FMT, C>(t, min((int)floorf(__fadd_rn(lc, 0.5f)), t.levels - 1), uv, scale,
                               a.width, acc);
  } else {
    const float fl = floorf(lc);
    const float frac = __fsub_rn(lc, fl);
    const int L0 = (int)fl, L1 = min(L0 + 1, t.levels - 1);
    tex2d_det_level<F, FMT, C>(t, L0, uv, scale * (1.0f - frac), a.width, acc);
    if (frac > 0.0f) tex2d_det_level<F, FMT, C>(t, L1, uv, scale * frac, a.width, acc);
  }
}

template <int F, int FMT, int C, bool REUSE>
__global__ void __launch_bounds__(256) k_tex2d_stochastic(Tex2DView t, LookupArgs a) {
  if (fast_loop(a)) {
    const uint32_t n = (uint32_t)a.n, stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float v[C];
      int4 tap;
      tex2d_stochastic_one<F, FMT, C, REUSE>(t, a, i, i, a.sample_index, v, tap);
      store_out<C>(a.out, i, v);
    }
    return;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    float v[C];
    int4 tap;
    const int64_t j = query_slot(a, i);
    tex2d_stochastic_one<F, FMT, C, REUSE>(t, a, i, j, a.sample_index, v, tap);
    store_out<C>(a.out, j, v);
    if (a.taps) reinterpret_cast<int4*>(a.taps)[j] = tap;
  }
}

template <int F, int FMT, int C>
__global__ void __launch_bounds__(256) k_tex2d_deterministic(Tex2DView t, LookupArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float2 uv = reinterpret_cast<const float2*>(a.coords)[i];
    const float lod = a.lod ? a.lod[i] : 0.0f;
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.0f;
    tex2d_det_at<F, FMT, C>(t, a, uv, lod, 1.0f, acc);
    store_out<C>(a.out, i, acc);
  }
}

template <int F, int FMT, int C, bool REUSE>
__global__ void __launch_bounds__(256) k_tex2d_accumulate(Tex2DView t, LookupArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double s[C], s2[C];
#pragma unroll
    for (int c = 0; c < C; ++c) s[c] = s2[c] = 0.0;
    for (int k = 0; k < a.n_samples; ++k) {
      float v[C];
      int4 tap;
      tex2d_stochastic_one<F, FMT, C, REUSE>(t, a, i, i, a.sample_index + (uint32_t)k, v, tap);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        s[c] += (double)v[c];
        s2[c] += (double)v[c] * (double)v[c];
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      a.sum[i * C + c] = s[c];
      a.sumsq[i * C + c] = s2[c];
    }
  }
}

// ---------------------------------------------------------------- triplanar

struct Planes {
  float2 uv[3];
  float a[3];       // |n_x|, |n_y|, |n_z|
  bool ok;          // finite position and normal, non-zero normal
};

__device__ __forceinline__ Planes triplanar_planes(const LookupArgs& a, int64_t i) {
  Planes P;
  const float px = __ldg(a.coords + 3 * i), py = __ldg(a.coords + 3 * i + 1), pz = __ldg(a.coords + 3 * i + 2);
  const float nx = __ldg(a.normals + 3 * i), ny = __ldg(a.normals + 3 * i + 1), nz = __ldg(a.normals + 3 * i + 2);
  const float s = a.tri_scale;
  P.uv[0] = make_float2(__fmul_rn(py, s), __fmul_rn(pz, s));
  P.uv[1] = make_float2(__fmul_rn(px, s), __fmul_rn(pz, s));
  P.uv[2] = make_float2(__fmul_rn(px, s), __fmul_rn(py, s));
  P.a[0] = fabsf(nx);
  P.a[1] = fabsf(ny);
  P.a[2] = fabsf(nz);
  P.ok = finite3(px, py, pz) && finite3(nx, ny, nz) && (P.a[0] > 0.0f || P.a[1] > 0.0f || P.a[2] > 0.0f);
  return P;
}

template <int F, int FMT, int C>
__device__ __forceinline__ void triplanar_stochastic_one(const Tex2DView& t, const LookupArgs& a,
                                                         int64_t i, int64_t j, uint32_t sample,
                                                         float* v, int4& tap) {
  const Planes P = triplanar_planes(a, i);
  if (!P.ok) {
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = 0.0f;
    tap = make_int4(0, 0, 0, -1);
    return;
  }
  const uint4 r = query_variates(a, j, sample);
  const float c0 = P.a[0], c1 = __fadd_rn(P.a[0], P.a[1]), S = __fadd_rn(c1, P.a[2]);
  const float us = __fmul_rn(unit24(r.z), S);
  const int k = (us >= c0 ? 1 : 0) + (us >= c1 ? 1 : 0);
  const float lod = a.lod ? a.lod[i] : 0.0f;
  tex2d_stochastic_at<F, FMT, C, false>(t, a, P.uv[k], lod, j, sample, r, v, tap);
  if (tap.w >= 0) tap.z = k;
}

template <int F, int FMT, int C>
__global__ void __launch_bounds__(256) k_triplanar_stochastic(Tex2DView t, LookupArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    float v[C];
    int4 tap;
    triplanar_stochastic_one<F, FMT, C>(t, a, i, i, a.sample_index, v, tap);
    store_out<C>(a.out, i, v);
    if (a.taps) reinterpret_cast<int4*>(a.taps)[i] = tap;
  }
}

template <int F, int FMT, int C>
__global__ void __launch_bounds__(256) k_triplanar_deterministic(Tex2DView t, LookupArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const Planes P = triplanar_planes(a, i);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.0f;
    if (P.ok) {
      const float S = __fadd_rn(__fadd_rn(P.a[0], P.a[1]), P.a[2]);
      const float lod = a.lod ? a.lod[i] : 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (P.a[k] > 0.0f) tex2d_det_at<F, FMT, C>(t, a, P.uv[k], lod, __fdiv_rn(P.a[k], S), acc);
    }
    store_out<C>(a.out, i, acc);
  }
}

// ---------------------------------------------------------------- launchers

template <int F, int FMT, int C>
static cudaError_t run_tex2d(Op op, const Tex2DView& t, const LookupArgs& a, cudaStream_t s) {
  const int threads = 256;
  const int blocks = grid_blocks(a.n, threads);
  if (a.normals) {                                    // triplanar queries
    if constexpr (F == STF_FILTER_CATMULL_ROM_POSITIVIZED) {
      return cudaErrorInvalidValue;                   // rejected by the argument checks
    } else {
      if (op == OP_STOCHASTIC) k_triplanar_stochastic<F, FMT, C><<<blocks, threads, 0, s>>>(t, a);
      else if (op == OP_DETERMINISTIC) k_triplanar_deterministic<F, FMT, C><<<blocks, threads, 0, s>>>(t, a);
      else return cudaErrorInvalidValue;              // no triplanar accumulation
      return cudaGetLastError();
    }
  }
  if (op == OP_STOCHASTIC) {
    if constexpr (UsesReuse<F>::value) {
      if (a.reuse) k_tex2d_stochastic<F, FMT, C, true><<<blocks, threads, 0, s>>>(t, a);
      else k_tex2d_stochastic<F, FMT, C, false><<<blocks, threads, 0, s>>>(t, a);
    } else {
      k_tex2d_stochastic<F, FMT, C, false><<<blocks, threads, 0, s>>>(t, a);
    }
  } else if (op == OP_DETERMINISTIC) {
    k_tex2d_deterministic<F, FMT, C><<<blocks, threads, 0, s>>>(t, a);
  } else {
    if constexpr (UsesReuse<F>::value) {
      if (a.reuse) k_tex2d_accumulate<F, FMT, C, true><<<blocks, threads, 0, s>>>(t, a);
      else k_tex2d_accumulate<F, FMT, C, false><<<blocks, threads, 0, s>>>(t, a);
    } else {
      k_tex2d_accumulate<F, FMT, C, false><<<blocks, threads, 0, s>>>(t, a);
    }
  }
  return cudaGetLastError();
}

template <int F, int FMT>
static cudaError_t run_tex2d_c(Op op, int c, const Tex2DView& t, const LookupArgs& a, cudaStream_t s) {
  switch (c) {
    case 1: return run_tex2d<F, FMT, 1>(op, t, a, s);
    case 2: return run_tex2d<F, FMT, 2>(op, t, a, s);
    case 4: return run_tex2d<F, FMT, 4>(op, t, a, s);
    case 8: return run_tex2d<F, FMT, 8>(op, t, a, s);
  }
  return cudaErrorInvalidValue;
}

// All filters for one storage format.
template <int FMT>
static cudaError_t launch_tex2d_format(Op op, int filter, int channels, const Tex2DView& t,
                                      const LookupArgs& a, cudaStream_t s) {
  switch (filter) {
    case STF_FILTER_LINEAR: return run_tex2d_c<STF_FILTER_LINEAR, FMT>(op, channels, t, a, s);
    case STF_FILTER_BSPLINE3: return run_tex2d_c<STF_FILTER_BSPLINE3, FMT>(op, channels, t, a, s);
    case STF_FILTER_CATMULL_ROM: return run_tex2d_c<STF_FILTER_CATMULL_ROM, FMT>(op, channels, t, a, s);
    case STF_FILTER_CATMULL_ROM_POSITIVIZED:
      return run_tex2d_c<STF_FILTER_CATMULL_ROM_POSITIVIZED, FMT>(op, channels, t, a, s);
    case STF_FILTER_FIS_LINEAR: return run_tex2d_c<STF_FILTER_FIS_LINEAR, FMT>(op, channels, t, a, s);
    case STF_FILTER_FIS_BSPLINE3: return run_tex2d_c<STF_FILTER_FIS_BSPLINE3, FMT>(op, channels, t, a, s);
    case STF_FILTER_FIS_GAUSSIAN: return run_tex2d_c<STF_FILTER_FIS_GAUSSIAN, FMT>(op, channels, t, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stf
