// Lookup kernels for dense 3D voxel grids, the 2D launcher's format dispatch (the 2D
// kernels are in stf_tex2d.cuh, one translation unit per storage format), and the
// create-time kernels of regular grids.
//
// One thread per query (grid-stride).  The stochastic kernels draw one tap per axis
// by inverse CDF over |w| (sampling arrays, Section 2.2; separable sampling,
// Section 4.2) and fetch a single texel (Eq. 3); the deterministic kernels sum all
// 2^d / 4^d taps (Eq. 2, Eq. 9); the accumulate kernels repeat the stochastic form
// over many sample indices and sum in float64 (validation only).
#include "stf_launch.h"

namespace stf {

// ---------------------------------------------------------------- dense 3D

// Voxel (ix, iy, iz), or the background outside the grid.  OFF32: the grid has at
// most 2^32 voxels, so the element offset is computed in 32 bits.
template <int FMT, bool OFF32 = false>
__device__ __forceinline__ float dense_fetch(const Dense3DView& g, int ix, int iy, int iz) {
  if ((unsigned)ix >= (unsigned)g.nx || (unsigned)iy >= (unsigned)g.ny ||
      (unsigned)iz >= (unsigned)g.nz)
    return g.background;
  int64_t e;
  if constexpr (OFF32)
    e = (uint32_t)(((uint32_t)iz * (uint32_t)g.ny + (uint32_t)iy) * (uint32_t)g.nx + (uint32_t)ix);
  else
    e = ((int64_t)iz * g.ny + iy) * g.nx + ix;
  if constexpr (FMT == STF_FMT_F16)
    return __half2float(__ldg(reinterpret_cast<const __half*>(g.texels) + e));
  else
    return __ldg(reinterpret_cast<const float*>(g.texels) + e);
}

// One stochastic lookup at coordinates x (caller's query index j).  J is int64_t, or
// uint32_t in the fast loops.  With a miss box (the fast loops, which write no tap
// output), a fixed-window filter whose window lies outside the grid returns the
// background without drawing.
template <int F, int FMT, bool REUSE, bool OFF32 = false, typename J>
__device__ __forceinline__ float dense_stochastic_at(const Dense3DView& g, const LookupArgs& a,
                                                     float* x, J j, uint32_t sample, int4& tap,
                                                     const MissBox* miss = nullptr) {
  if (!prepare_coords<3>(x)) {
    tap = make_int4(0, 0, 0, -1);
    return g.background;
  }
  if constexpr (FixedWindow<F>::value) {
    if (miss && misses(*miss, x)) return g.background;
  }
  const uint4 r = query_variates(a, j, sample);
  if constexpr (IsFis<F>::value) {
    int idx[3];
    pick_fis<F, 3>(x, a, j, sample, r, idx);
    tap = make_int4(idx[0], idx[1], idx[2], 0);
    return dense_fetch<FMT, OFF32>(g, idx[0], idx[1], idx[2]);
  } else if constexpr (F == STF_FILTER_CATMULL_ROM_POSITIVIZED) {
    const uint4 r1 = query_variates(a, j, sample, 1u);
    const float up[4] = {unit24(r.x), unit24(r.y), unit24(r.z), unit24(r.w)};
    const float un[4] = {unit24(r1.x), unit24(r1.y), unit24(r1.z), unit24(r1.w)};
    int ip[3], in[3];
    float Wp, Wn;
    pick_positivized<3>(x, up, un, ip, in, Wp, Wn);
    tap = make_int4(ip[0], ip[1], ip[2], 0);
    float t = Wp * dense_fetch<FMT, OFF32>(g, ip[0], ip[1], ip[2]);
    if (Wn > 0.0f) t = fmaf(-Wn, dense_fetch<FMT, OFF32>(g, in[0], in[1], in[2]), t);
    return t;
  } else {
    int idx[3];
    const float sigma = pick_taps_r<F, 3, REUSE>(x, r, idx);
    tap = make_int4(idx[0], idx[1], idx[2], 0);
    float t = dense_fetch<FMT, OFF32>(g, idx[0], idx[1], idx[2]);
    if constexpr (!Filter<F>::NONNEG) t *= sigma;
    return t;
  }
}

// One stochastic lookup of query i (caller's index j).  I is int64_t, or uint32_t in
// the fast loop (3 i + 2 < 2^32 there).
template <int F, int FMT, bool REUSE, bool OFF32 = false, typename I>
__device__ __forceinline__ float dense_stochastic_one(const Dense3DView& g, const LookupArgs& a,
                                                      I i, I j, uint32_t sample, int4& tap) {
  float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
  return dense_stochastic_at<F, FMT, REUSE, OFF32>(g, a, x, j, sample, tap);
}

// Packed form of the four-query loop for the fixed-window filters (tent, B-spline, and
// their FIS forms): a warp's 128 queries are tested against the miss box, each lane
// writes the background over its four results, and the warp's live queries are then
// packed onto its lanes, lane t taking the live queries of rank t, t + 32, ... in
// (query-in-group, lane) order, R = ceil(live / 32) per lane, drawn, chosen and gathered
// side by side.  A warp with at most 64 live queries thus runs one or two draws per lane
// instead of four; a warp with more keeps each lane's own four (joint_one_tap4).  The
// packed lanes reload their queries' coordinates (from L1: the warp has just read them)
// and store each result over the background its owner wrote.
// Position of the set bit of rank n (0-based) in m, for n < popc(m): a binary search on
// the population counts of the low halves.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t n) {
  uint32_t pos = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const uint32_t low = __popc(m & ((1u << w) - 1u));
    if (n >= low) {
      n -= low;
      m >>= w;
      pos += (uint32_t)w;
    }
  }
  return pos;
}

template <int F, int FMT, int R>
__device__ __forceinline__ void dense_packed_rounds(const Dense3DView& g, const LookupArgs& a, uint32_t q0,
                                                    const uint32_t (&b)[4], uint32_t live_count, uint32_t lane,
                                                    uint32_t groups) {
  const uint32_t c0 = __popc(b[0]), c1 = c0 + __popc(b[1]), c2 = c1 + __popc(b[2]);
  uint32_t qi[R];
  bool ok[R];
  float x[R][3];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const uint32_t r = lane + 32u * (uint32_t)q;
    ok[q] = r < live_count;
    const int k = r < c0 ? 0 : r < c1 ? 1 : r < c2 ? 2 : 3;
    const uint32_t before = k == 0 ? 0u : k == 1 ? c0 : k == 2 ? c1 : c2;
    const uint32_t bk = k == 0 ? b[0] : k == 1 ? b[1] : k == 2 ? b[2] : b[3];
    const uint32_t src = ok[q] ? nth_set_bit(bk, r - before) : 0u;
    qi[q] = 4u * (q0 + src) + (uint32_t)k;
    ok[q] = ok[q] && qi[q] < 4u * groups;    // a live query lies in an active lane's group
    x[q][0] = x[q][1] = x[q][2] = 0.0f;
    if (ok[q]) {
      x[q][0] = __ldg(a.coords + 3 * qi[q]);
      x[q][1] = __ldg(a.coords + 3 * qi[q] + 1);
      x[q][2] = __ldg(a.coords + 3 * qi[q] + 2);
    }
    prepare_coords<3>(x[q]);            // the owner's clamp of huge coordinates, again
  }
  uint4 rv[R];
#pragma unroll
  for (int q = 0; q < R; ++q) rv[q] = query_variates(a, qi[q], a.sample_index);
  int t[R][3];
#pragma unroll
  for (int q = 0; q < R; ++q) draw_one_tap3<F>(a, x[q], qi[q], rv[q], t[q]);
#pragma unroll
  for (int q = 0; q < R; ++q)
    if (ok[q]) a.out[qi[q]] = dense_fetch<FMT, true>(g, t[q][0], t[q][1], t[q][2]);
}

template <int F, int FMT>
__device__ __forceinline__ void dense_packed_loop(const Dense3DView& g, const LookupArgs& a, const MissBox& mb) {
  const uint32_t n = (uint32_t)a.n, groups = n >> 2, stride = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31u;
  const float4* c4 = reinterpret_cast<const float4*>(a.coords);
  float4* o4 = reinterpret_cast<float4*>(a.out);
  const float bg = g.background;
  // every lane of a warp runs the same iterations (the loop bound is the warp's first
  // group), so the warp-wide votes below see all 32 lanes
  for (uint32_t w0 = tid - lane; w0 < groups; w0 += stride) {
    const uint32_t gq = w0 + lane;
    const bool act = gq < groups;
    float x[4][3] = {};
    bool live[4] = {false, false, false, false};
    if (act) {
      const float4 p = __ldg(c4 + 3 * gq), q = __ldg(c4 + 3 * gq + 1), r = __ldg(c4 + 3 * gq + 2);
      x[0][0] = p.x; x[0][1] = p.y; x[0][2] = p.z;
      x[1][0] = p.w; x[1][1] = q.x; x[1][2] = q.y;
      x[2][0] = q.z; x[2][1] = q.w; x[2][2] = r.x;
      x[3][0] = r.y; x[3][1] = r.z; x[3][2] = r.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) live[k] = prepare_coords<3>(x[k]) && !misses(mb, x[k]);
    }
    uint32_t b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = __ballot_sync(0xffffffffu, live[k]);
    const uint32_t live_count = __popc(b[0]) + __popc(b[1]) + __popc(b[2]) + __popc(b[3]);
    // (every branch below is the same for all lanes)
    if (live_count > 64) {
      // mostly live: each lane its own four queries, side by side
      if (act) o4[gq] = joint_one_tap4<F>(a, x, 4 * gq, mb, bg, [&](const int* t) {
        return dense_fetch<FMT, true>(g, t[0], t[1], t[2]);
      });
      continue;
    }
    if (act) o4[gq] = make_float4(bg, bg, bg, bg);
    if (live_count == 0) continue;
    __syncwarp();                        // the owners' background stores come first
    if (live_count <= 32) dense_packed_rounds<F, FMT, 1>(g, a, w0, b, live_count, lane, groups);
    else dense_packed_rounds<F, FMT, 2>(g, a, w0, b, live_count, lane, groups);
    __syncwarp();
  }
  for (uint32_t i = 4 * groups + tid; i < n; i += stride) {
    float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
    int4 tap;
    a.out[i] = dense_stochastic_at<F, FMT, false, true>(g, a, x, i, a.sample_index, tap, &mb);
  }
}

// Resident 256-thread blocks per SM: six (at most 40 registers a thread) for the tent
// and B-spline filters, 1.4% sooner than five on the dense benchmark call without
// spills; five for Catmull-Rom and the Gaussian, which would spill at 40; four for
// the two-tap positivized Catmull-Rom (at 84 registers and three blocks it ran 17%
// slower).
template <int F>
constexpr int dense_stochastic_min_blocks() {
  return F == STF_FILTER_CATMULL_ROM_POSITIVIZED ? 4
         : (F == STF_FILTER_CATMULL_ROM || F == STF_FILTER_FIS_GAUSSIAN) ? 5 : 6;
}

template <int F, int FMT, bool REUSE>
__global__ void __launch_bounds__(256, dense_stochastic_min_blocks<F>()) k_dense_stochastic(Dense3DView g,
                                                                                         LookupArgs a) {
  const bool off32 = (uint64_t)g.nx * (uint64_t)g.ny * (uint64_t)g.nz <= (uint64_t(1) << 32);
  const MissBox mb = miss_box<F>(0, 0, 0, g.nx, g.ny, g.nz);
  if constexpr (FixedWindow<F>::value && F != STF_FILTER_FIS_BSPLINE3 && !REUSE) {
    if (off32 && quad_loop3_ok(a)) {
      dense_packed_loop<F, FMT>(g, a, mb);
      return;
    }
  }
  if constexpr (JointOneTap<F, REUSE>::value) {
    if (off32 && quad_loop3_ok(a)) {
      quad_loop3_joint(a, [&](float (&x)[4][3], uint32_t i) {
        return joint_one_tap4<F>(a, x, i, mb, g.background,
                                 [&](const int* t) { return dense_fetch<FMT, true>(g, t[0], t[1], t[2]); });
      }, [&](float x0, float x1, float x2, uint32_t j) {
        float x[3] = {x0, x1, x2};
        int4 tap;
        return dense_stochastic_at<F, FMT, REUSE, true>(g, a, x, j, a.sample_index, tap, &mb);
      });
      return;
    }
  }
  if (off32 && quad_loop3_ok(a)) {
    quad_loop3(a, [&](float x0, float x1, float x2, uint32_t j) {
      float x[3] = {x0, x1, x2};
      int4 tap;
      return dense_stochastic_at<F, FMT, REUSE, true>(g, a, x, j, a.sample_index, tap, &mb);
    });
    return;
  }
  if (fast_loop(a) && off32) {
    const uint32_t n = (uint32_t)a.n, stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
      int4 tap;
      a.out[i] = dense_stochastic_at<F, FMT, REUSE, true>(g, a, x, i, a.sample_index, tap, &mb);
    }
    return;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    int4 tap;
    const int64_t j = query_slot(a, i);
    a.out[j] = dense_stochastic_one<F, FMT, REUSE>(g, a, i, j, a.sample_index, tap);
    if (a.taps) reinterpret_cast<int4*>(a.taps)[j] = tap;
  }
}

// The T consecutive voxels e .. e + T - 1 of one grid row.  FP16 rows of
// four come from aligned 8-byte words: one word when e is a multiple of 4, else two
// (the texel allocation is padded by 16 bytes, so the second word never leaves it),
// shifted into place.  Other rows are read voxel by voxel.
template <int FMT, int T>
__device__ __forceinline__ void dense_row(const void* texels, uint32_t e, float* v) {
  if constexpr (FMT == STF_FMT_F16 && T == 4) {
    const uint2* w = reinterpret_cast<const uint2*>(texels) + (e >> 2);
    const uint32_t s = e & 3;
    const uint2 a = __ldg(w);
    uint32_t lo = a.x, hi = a.y;
    if (s != 0) {
      const uint2 b = __ldg(w + 1);
      const uint32_t x0 = s >= 2 ? a.y : a.x, x1 = s >= 2 ? b.x : a.y, x2 = s >= 2 ? b.y : b.x;
      const uint32_t sh = (s & 1) * 16;
      lo = __funnelshift_r(x0, x1, sh);
      hi = __funnelshift_r(x1, x2, sh);
    }
    const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&lo));
    const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
  } else {
#pragma unroll
    for (int k = 0; k < T; ++k) {
      if constexpr (FMT == STF_FMT_F16)
        v[k] = __half2float(__ldg(reinterpret_cast<const __half*>(texels) + e + k));
      else
        v[k] = __ldg(reinterpret_cast<const float*>(texels) + e + k);
    }
  }
}

template <int F, int FMT>
__global__ void __launch_bounds__(256) k_dense_deterministic(Dense3DView g, LookupArgs a) {
  using Fl = Filter<F>;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // grids of at most 2^32 voxels take 32-bit row offsets in the interior path
  const bool off32 = (uint64_t)g.nx * (uint64_t)g.ny * (uint64_t)g.nz <= (uint64_t(1) << 32);
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
        // a window entirely outside the grid on some axis reads only the background,
        // and the weights sum to one (partition of unity)
        const bool outside = bx + Fl::T <= 0 || by + Fl::T <= 0 || bz + Fl::T <= 0 || bx >= g.nx ||
                             by >= g.ny || bz >= g.nz;
        // (the two-tap filters keep the checked loop: eight scattered voxels gain
        // nothing from row loads, and measured slower with the extra path)
        const bool interior = Fl::T == 4 && off32 && bx >= 0 && by >= 0 && bz >= 0 &&
                              bx + Fl::T <= g.nx && by + Fl::T <= g.ny && bz + Fl::T <= g.nz;
        if (outside) {
          acc = g.background;
        } else if (interior) {
          // the whole window inside the grid: rows of T voxels along x, no bounds tests;
          // each row's weighted sum, then the rows weighted by wy * wz
          const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
          const uint32_t e0 = ((uint32_t)bz * ny + (uint32_t)by) * nx + (uint32_t)bx;
#pragma unroll
          for (int kz = 0; kz < Fl::T; ++kz) {
#pragma unroll
            for (int ky = 0; ky < Fl::T; ++ky) {
              float v[Fl::T];
              dense_row<FMT, Fl::T>(g.texels, e0 + ((uint32_t)kz * ny + (uint32_t)ky) * nx, v);
              float r = wx[0] * v[0];
#pragma unroll
              for (int kx = 1; kx < Fl::T; ++kx) r = fmaf(wx[kx], v[kx], r);
              acc = fmaf(wy[ky] * wz[kz], r, acc);
            }
          }
        } else {
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

cudaError_t launch_tex2d(Op op, int filter, int fmt, int channels, const Tex2DView& t,
                         const LookupArgs& a, cudaStream_t s) {
  if (fmt == STF_FMT_F32) return launch_tex2d_f32(op, filter, channels, t, a, s);
  if (fmt == STF_FMT_F16) return launch_tex2d_f16(op, filter, channels, t, a, s);
  if (fmt == STF_FMT_DCT6) return launch_tex2d_dct(op, filter, channels, t, a, s);
  return cudaErrorInvalidValue;
}

template <int F, int FMT>
static cudaError_t run_dense(Op op, const Dense3DView& g, const LookupArgs& a, cudaStream_t s) {
  const int threads = 256;
  // the four-query loop needs a quarter of the threads
  const int64_t units = (op == OP_STOCHASTIC && quad_loop3_ok(a)) ? (a.n + 3) / 4 : a.n;
  const int blocks = grid_blocks(units, threads, op == OP_STOCHASTIC ? kStochasticWaves : 4);
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
