// Lookup kernels for regular grids: 2D MIP-mapped textures and dense 3D voxel grids.
//
// One thread per query (grid-stride).  The stochastic kernels draw one tap per axis
// by inverse CDF over |w| (sampling arrays, Section 2.2; separable sampling,
// Section 4.2) and fetch a single texel (Eq. 3); the deterministic kernels sum all
// 2^d / 4^d taps (Eq. 2, Eq. 9); the accumulate kernels repeat the stochastic form
// over many sample indices and sum in float64 (validation only).
#include "stf_launch.h"

namespace stf {

// ---------------------------------------------------------------- 2D

// Level choice: floor(lod + 1/2) (nearest) or floor(lod + u) (stochastic), lod
// clamped to [0, levels - 1].
__device__ __forceinline__ int level_stochastic(const Tex2DView& t, const LookupArgs& a,
                                                float lod, float u) {
  if (a.lod == nullptr || t.levels <= 1) return 0;
  const float lc = fminf(fmaxf(lod, 0.0f), (float)(t.levels - 1));
  const float s = __fadd_rn(lc, a.level_mode == STF_LEVEL_NEAREST ? 0.5f : u);
  return min((int)floorf(s), t.levels - 1);
}

template <int F, int FMT, int C, bool REUSE>
__device__ __forceinline__ void tex2d_stochastic_one(const Tex2DView& t, const LookupArgs& a,
                                                     int64_t i, int64_t j, uint32_t sample,
                                                     float* v, int4& tap) {
  const float2 uv = reinterpret_cast<const float2*>(a.coords)[i];
  const float lod = a.lod ? a.lod[i] : 0.0f;
  const uint4 r = query_variates(a, j, sample);
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
    TexelIO<FMT, C>::load(t.texels, t.level_off[L] + (int64_t)min(max(idx[1], 0), H - 1) * W +
                                        min(max(idx[0], 0), W - 1), v);
  } else if constexpr (F == STF_FILTER_CATMULL_ROM_POSITIVIZED) {
    const uint4 r1 = query_variates(a, j, sample, 1u);
    const float up[3] = {unit24(r.x), unit24(r.y), unit24(r.z)};
    const float un[3] = {unit24(r1.x), unit24(r1.y), unit24(r1.z)};
    int ip[2], in[2];
    float Wp, Wn;
    pick_positivized<2>(x, up, un, ip, in, Wp, Wn);
    tap = make_int4(ip[0], ip[1], 0, L);
    TexelIO<FMT, C>::load(t.texels, t.level_off[L] + (int64_t)min(max(ip[1], 0), H - 1) * W +
                                        min(max(ip[0], 0), W - 1), v);
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] *= Wp;
    if (Wn > 0.0f) {
      float tn[C];
      TexelIO<FMT, C>::load(t.texels, t.level_off[L] + (int64_t)min(max(in[1], 0), H - 1) * W +
                                          min(max(in[0], 0), W - 1), tn);
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = fmaf(-Wn, tn[c], v[c]);
    }
  } else {
    const float u[2] = {unit24(r.x), unit24(r.y)};
    int idx[2];
    const float sigma = pick_taps<F, 2, REUSE>(x, u, idx);
    tap = make_int4(idx[0], idx[1], 0, L);
    const int cx = min(max(idx[0], 0), W - 1), cy = min(max(idx[1], 0), H - 1);
    TexelIO<FMT, C>::load(t.texels, t.level_off[L] + (int64_t)cy * W + cx, v);
    if constexpr (!Filter<F>::NONNEG) {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] *= sigma;
    }
  }
}

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
      const int64_t row = t.level_off[L] + (int64_t)min(max(iy, 0), H - 1) * W;
      float ex0 = gauss_edge(gx, gx.lo);
      for (int ix = gx.lo; ix <= gx.hi; ++ix) {
        const float ex1 = gauss_edge(gx, ix + 1);
        const float w = 0.5f * (ex1 - ex0) * wy;
        ex0 = ex1;
        float tv[C];
        TexelIO<FMT, C>::load(t.texels, row + min(max(ix, 0), W - 1), tv);
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(w, tv[c], acc[c]);
      }
    }
    return;
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
    const int64_t row = t.level_off[L] + (int64_t)cy * W;
    const float wyk = wy[ky] * scale;
#pragma unroll
    for (int kx = 0; kx < Fl::T; ++kx) {
      float tv[C];
      TexelIO<FMT, C>::load(t.texels, row + cxs[kx], tv);
      const float w = wx[kx] * wyk;
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaf(w, tv[c], acc[c]);
    }
  }
  }
}

template <int F, int FMT, int C, bool REUSE>
__global__ void __launch_bounds__(256) k_tex2d_stochastic(Tex2DView t, LookupArgs a) {
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
    if (isfinite(lod)) {
      if (a.lod == nullptr || t.levels <= 1) {
        tex2d_det_level<F, FMT, C>(t, 0, uv, 1.0f, a.width, acc);
      } else {
        const float lc = fminf(fmaxf(lod, 0.0f), (float)(t.levels - 1));
        if (a.level_mode == STF_LEVEL_NEAREST) {
          tex2d_det_level<F, FMT, C>(t, min((int)floorf(__fadd_rn(lc, 0.5f)), t.levels - 1), uv,
                                     1.0f, a.width, acc);
        } else {
          const float fl = floorf(lc);
          const float frac = __fsub_rn(lc, fl);
          const int L0 = (int)fl, L1 = min(L0 + 1, t.levels - 1);
          tex2d_det_level<F, FMT, C>(t, L0, uv, 1.0f - frac, a.width, acc);
          if (frac > 0.0f) tex2d_det_level<F, FMT, C>(t, L1, uv, frac, a.width, acc);
        }
      }
    }
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

// ---------------------------------------------------------------- dense 3D

template <int FMT>
__device__ __forceinline__ float dense_fetch(const Dense3DView& g, int ix, int iy, int iz) {
  if ((unsigned)ix >= (unsigned)g.nx || (unsigned)iy >= (unsigned)g.ny ||
      (unsigned)iz >= (unsigned)g.nz)
    return g.background;
  const int64_t e = ((int64_t)iz * g.ny + iy) * g.nx + ix;
  if constexpr (FMT == STF_FMT_F16)
    return __half2float(__ldg(reinterpret_cast<const __half*>(g.texels) + e));
  else
    return __ldg(reinterpret_cast<const float*>(g.texels) + e);
}

template <int F, int FMT, bool REUSE>
__device__ __forceinline__ float dense_stochastic_one(const Dense3DView& g, const LookupArgs& a,
                                                      int64_t i, int64_t j, uint32_t sample,
                                                      int4& tap) {
  float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
  if (!prepare_coords<3>(x)) {
    tap = make_int4(0, 0, 0, -1);
    return g.background;
  }
  const uint4 r = query_variates(a, j, sample);
  if constexpr (IsFis<F>::value) {
    int idx[3];
    pick_fis<F, 3>(x, a, j, sample, r, idx);
    tap = make_int4(idx[0], idx[1], idx[2], 0);
    return dense_fetch<FMT>(g, idx[0], idx[1], idx[2]);
  } else if constexpr (F == STF_FILTER_CATMULL_ROM_POSITIVIZED) {
    const uint4 r1 = query_variates(a, j, sample, 1u);
    const float up[4] = {unit24(r.x), unit24(r.y), unit24(r.z), unit24(r.w)};
    const float un[4] = {unit24(r1.x), unit24(r1.y), unit24(r1.z), unit24(r1.w)};
    int ip[3], in[3];
    float Wp, Wn;
    pick_positivized<3>(x, up, un, ip, in, Wp, Wn);
    tap = make_int4(ip[0], ip[1], ip[2], 0);
    float t = Wp * dense_fetch<FMT>(g, ip[0], ip[1], ip[2]);
    if (Wn > 0.0f) t = fmaf(-Wn, dense_fetch<FMT>(g, in[0], in[1], in[2]), t);
    return t;
  } else {
    const float u[3] = {unit24(r.x), unit24(r.y), unit24(r.z)};
    int idx[3];
    const float sigma = pick_taps<F, 3, REUSE>(x, u, idx);
    tap = make_int4(idx[0], idx[1], idx[2], 0);
    float t = dense_fetch<FMT>(g, idx[0], idx[1], idx[2]);
    if constexpr (!Filter<F>::NONNEG) t *= sigma;
    return t;
  }
}

template <int F, int FMT, bool REUSE>
__global__ void __launch_bounds__(256) k_dense_stochastic(Dense3DView g, LookupArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    int4 tap;
    const int64_t j = query_slot(a, i);
    a.out[j] = dense_stochastic_one<F, FMT, REUSE>(g, a, i, j, a.sample_index, tap);
    if (a.taps) reinterpret_cast<int4*>(a.taps)[j] = tap;
  }
}

template <int F, int FMT>
__global__ void __launch_bounds__(256) k_dense_deterministic(Dense3DView g, LookupArgs a) {
  using Fl = Filter<F>;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
    float acc = g.background;
    if (prepare_coords<3>(x)) {
      if constexpr (F == STF_FILTER_FIS_GAUSSIAN) {
        acc = gauss_window_sum3(x, a.width, [&](int ix, int iy, int iz) {
          return dense_fetch<FMT>(g, ix, iy, iz);
        });
      } else {
        float fx, fy, fz;
        const int bx = axis_base(x[0], fx) + Fl::OFF0, by = axis_base(x[1], fy) + Fl::OFF0,
                  bz = axis_base(x[2], fz) + Fl::OFF0;
        float wx[Fl::T], wy[Fl::T], wz[Fl::T];
        Fl::weights(fx, wx);
        Fl::weights(fy, wy);
        Fl::weights(fz, wz);
        acc = 0.0f;
#pragma unroll
        for (int kz = 0; kz < Fl::T; ++kz) {
#pragma unroll
          for (int ky = 0; ky < Fl::T; ++ky) {
            const float wyz = wy[ky] * wz[kz];
#pragma unroll
            for (int kx = 0; kx < Fl::T; ++kx)
              acc = fmaf(wx[kx] * wyz, dense_fetch<FMT>(g, bx + kx, by + ky, bz + kz), acc);
          }
        }
      }
    }
    a.out[i] = acc;
  }
}

template <int F, int FMT, bool REUSE>
__global__ void __launch_bounds__(256) k_dense_accumulate(Dense3DView g, LookupArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double s = 0.0, s2 = 0.0;
    for (int k = 0; k < a.n_samples; ++k) {
      int4 tap;
      const double v = dense_stochastic_one<F, FMT, REUSE>(g, a, i, i, a.sample_index + (uint32_t)k, tap);
      s += v;
      s2 += v * v;
    }
    a.sum[i] = s;
    a.sumsq[i] = s2;
  }
}

// ---------------------------------------------------------------- launchers

template <int F, int FMT, int C>
static cudaError_t run_tex2d(Op op, const Tex2DView& t, const LookupArgs& a, cudaStream_t s) {
  const int threads = 256;
  const int blocks = grid_blocks(a.n, threads);
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

template <int F>
static cudaError_t run_tex2d_f(Op op, int fmt, int c, const Tex2DView& t, const LookupArgs& a,
                               cudaStream_t s) {
  if (fmt == STF_FMT_F32) {
    switch (c) {
      case 1: return run_tex2d<F, STF_FMT_F32, 1>(op, t, a, s);
      case 2: return run_tex2d<F, STF_FMT_F32, 2>(op, t, a, s);
      case 4: return run_tex2d<F, STF_FMT_F32, 4>(op, t, a, s);
      case 8: return run_tex2d<F, STF_FMT_F32, 8>(op, t, a, s);
    }
  } else if (fmt == STF_FMT_F16) {
    switch (c) {
      case 1: return run_tex2d<F, STF_FMT_F16, 1>(op, t, a, s);
      case 2: return run_tex2d<F, STF_FMT_F16, 2>(op, t, a, s);
      case 4: return run_tex2d<F, STF_FMT_F16, 4>(op, t, a, s);
      case 8: return run_tex2d<F, STF_FMT_F16, 8>(op, t, a, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tex2d(Op op, int filter, int fmt, int channels, const Tex2DView& t,
                         const LookupArgs& a, cudaStream_t s) {
  switch (filter) {
    case STF_FILTER_LINEAR: return run_tex2d_f<STF_FILTER_LINEAR>(op, fmt, channels, t, a, s);
    case STF_FILTER_BSPLINE3: return run_tex2d_f<STF_FILTER_BSPLINE3>(op, fmt, channels, t, a, s);
    case STF_FILTER_CATMULL_ROM:
      return run_tex2d_f<STF_FILTER_CATMULL_ROM>(op, fmt, channels, t, a, s);
    case STF_FILTER_CATMULL_ROM_POSITIVIZED:
      return run_tex2d_f<STF_FILTER_CATMULL_ROM_POSITIVIZED>(op, fmt, channels, t, a, s);
    case STF_FILTER_FIS_LINEAR: return run_tex2d_f<STF_FILTER_FIS_LINEAR>(op, fmt, channels, t, a, s);
    case STF_FILTER_FIS_BSPLINE3:
      return run_tex2d_f<STF_FILTER_FIS_BSPLINE3>(op, fmt, channels, t, a, s);
    case STF_FILTER_FIS_GAUSSIAN:
      return run_tex2d_f<STF_FILTER_FIS_GAUSSIAN>(op, fmt, channels, t, a, s);
  }
  return cudaErrorInvalidValue;
}

template <int F, int FMT>
static cudaError_t run_dense(Op op, const Dense3DView& g, const LookupArgs& a, cudaStream_t s) {
  const int threads = 256;
  const int blocks = grid_blocks(a.n, threads);
  if (op == OP_STOCHASTIC) {
    if constexpr (UsesReuse<F>::value) {
      if (a.reuse) k_dense_stochastic<F, FMT, true><<<blocks, threads, 0, s>>>(g, a);
      else k_dense_stochastic<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    } else {
      k_dense_stochastic<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    }
  } else if (op == OP_DETERMINISTIC) {
    k_dense_deterministic<F, FMT><<<blocks, threads, 0, s>>>(g, a);
  } else {
    if constexpr (UsesReuse<F>::value) {
      if (a.reuse) k_dense_accumulate<F, FMT, true><<<blocks, threads, 0, s>>>(g, a);
      else k_dense_accumulate<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    } else {
      k_dense_accumulate<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    }
  }
  return cudaGetLastError();
}

template <int F>
static cudaError_t run_dense_f(Op op, int fmt, const Dense3DView& g, const LookupArgs& a,
                               cudaStream_t s) {
  if (fmt == STF_FMT_F32) return run_dense<F, STF_FMT_F32>(op, g, a, s);
  if (fmt == STF_FMT_F16) return run_dense<F, STF_FMT_F16>(op, g, a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_dense3d(Op op, int filter, int fmt, const Dense3DView& g, const LookupArgs& a,
                           cudaStream_t s) {
  switch (filter) {
    case STF_FILTER_LINEAR: return run_dense_f<STF_FILTER_LINEAR>(op, fmt, g, a, s);
    case STF_FILTER_BSPLINE3: return run_dense_f<STF_FILTER_BSPLINE3>(op, fmt, g, a, s);
    case STF_FILTER_CATMULL_ROM: return run_dense_f<STF_FILTER_CATMULL_ROM>(op, fmt, g, a, s);
    case STF_FILTER_CATMULL_ROM_POSITIVIZED:
      return run_dense_f<STF_FILTER_CATMULL_ROM_POSITIVIZED>(op, fmt, g, a, s);
    case STF_FILTER_FIS_LINEAR: return run_dense_f<STF_FILTER_FIS_LINEAR>(op, fmt, g, a, s);
    case STF_FILTER_FIS_BSPLINE3: return run_dense_f<STF_FILTER_FIS_BSPLINE3>(op, fmt, g, a, s);
    case STF_FILTER_FIS_GAUSSIAN: return run_dense_f<STF_FILTER_FIS_GAUSSIAN>(op, fmt, g, a, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- create-time kernels

__global__ void k_convert_f32(const float* __restrict__ src, void* __restrict__ dst, int fmt,
                              int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = src[i];
    if (fmt == STF_FMT_F16) reinterpret_cast<__half*>(dst)[i] = __float2half_rn(v);
    else reinterpret_cast<float*>(dst)[i] = v;
  }
}

cudaError_t launch_convert_f32(const float* src, void* dst, int fmt, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_convert_f32<<<grid_blocks(n, 256), 256, 0, s>>>(src, dst, fmt, n);
  return cudaGetLastError();
}

// One level of a 2x2 box pyramid from the level above it (w x h x c floats):
// ((a + b) + (c + d)) / 4, or the mean of 2 where one dimension is already 1.
__global__ void k_box_mip(const float* __restrict__ src, float* __restrict__ dst, int w, int h,
                          int c) {
  const int w2 = max(1, w >> 1), h2 = max(1, h >> 1);
  const int64_t n = (int64_t)w2 * h2 * c;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int ch = (int)(i % c);
    const int64_t p = i / c;
    const int x = (int)(p % w2), y = (int)(p / w2);
    const int x0 = (w > 1) ? 2 * x : x, x1 = (w > 1) ? 2 * x + 1 : x;
    const int y0 = (h > 1) ? 2 * y : y, y1 = (h > 1) ? 2 * y + 1 : y;
    const float a = src[((int64_t)y0 * w + x0) * c + ch], b = src[((int64_t)y0 * w + x1) * c + ch];
    const float d = src[((int64_t)y1 * w + x0) * c + ch], e = src[((int64_t)y1 * w + x1) * c + ch];
    dst[i] = __fmul_rn(__fadd_rn(__fadd_rn(a, b), __fadd_rn(d, e)), 0.25f);
  }
}

cudaError_t launch_box_mip(const float* src, float* dst, int w, int h, int c, cudaStream_t s) {
  const int64_t n = (int64_t)max(1, w >> 1) * max(1, h >> 1) * c;
  k_box_mip<<<grid_blocks(n, 256), 256, 0, s>>>(src, dst, w, h, c);
  return cudaGetLastError();
}

}  // namespace stf
