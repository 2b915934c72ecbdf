// Device-side building blocks of the lookup kernels: the counter-based generator,
// the separable filter weights, the inverse-CDF tap choice and the texture views.
// Written for sm_103a; every function here is inlined into the kernels.
#pragma once
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "stf_types.h"

namespace stf {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 32x32->64 multiplies; the key is bumped by the Weyl
// constants between rounds.  The key is a kernel argument, so its schedule is the
// same for every thread.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Top 24 bits as a float in [0, 1): exact in float32.
__device__ __forceinline__ float unit24(uint32_t r) { return (float)(r >> 8) * 0x1p-24f; }

// ---------------------------------------------------------------- filter weights
// Weights of the taps floor(x) + OFF0 + k, k = 0..T-1, at fraction f = x - floor(x).
template <int F> struct Filter;

// Tent K1 (Appendix A): taps floor(x), floor(x)+1.  CDF boundary (the weights sum to
// exactly 1): C_0 = 1 - f.
template <> struct Filter<STF_FILTER_LINEAR> {
  static constexpr int T = 2, OFF0 = 0;
  static constexpr bool NONNEG = true, UNIT_SUM = true;
  __device__ __forceinline__ static void weights(float f, float* w) {
    w[0] = 1.0f - f;
    w[1] = f;
  }
  __device__ __forceinline__ static void cdf(float f, float* c) { c[0] = 1.0f - f; }
  // The same boundary times 2^24, for comparison with the 24-bit integer variate:
  // a power-of-two scale, so every rounding is the scaled one and the choice is equal.
  __device__ __forceinline__ static void cdf24(float f, float* c) { c[0] = fmaf(f, -16777216.0f, 16777216.0f); }
};

// Cubic B-spline K_bs (Appendix A, "Convolutional"): with g = 1 - f the four taps
// floor(x)-1 .. floor(x)+2 carry g^3/6, f^2(f/2 - 1) + 2/3, g^2(g/2 - 1) + 2/3, f^3/6.
// The weights sum to exactly 1, so the interior CDF boundaries have closed forms:
// C_0 = g^3/6, C_1 = w_0 + w_1 = (5 - 3f - 3f^2 + 2f^3)/6, C_2 = 1 - f^3/6.
template <> struct Filter<STF_FILTER_BSPLINE3> {
  static constexpr int T = 4, OFF0 = -1;
  static constexpr bool NONNEG = true, UNIT_SUM = true;
  __device__ __forceinline__ static void weights(float f, float* w) {
    const float g = 1.0f - f;
    w[0] = g * g * g * (1.0f / 6.0f);
    w[1] = fmaf(f * f, fmaf(0.5f, f, -1.0f), 2.0f / 3.0f);
    w[2] = fmaf(g * g, fmaf(0.5f, g, -1.0f), 2.0f / 3.0f);
    w[3] = f * f * f * (1.0f / 6.0f);
  }
  __device__ __forceinline__ static void cdf(float f, float* c) {
    const float g = 1.0f - f, f2 = f * f;
    c[0] = g * g * (g * (1.0f / 6.0f));
    c[1] = fmaf(fmaf(fmaf(f, 1.0f / 3.0f, -0.5f), f, -0.5f), f, 5.0f / 6.0f);
    c[2] = fmaf(f2, f * (-1.0f / 6.0f), 1.0f);
  }
  // cdf() times 2^24 (every constant scaled by the power of two: the same roundings).
  __device__ __forceinline__ static void cdf24(float f, float* c) {
    const float g = 1.0f - f, f2 = f * f;
    c[0] = g * g * (g * (16777216.0f / 6.0f));
    c[1] = fmaf(fmaf(fmaf(f, 16777216.0f / 3.0f, -8388608.0f), f, -8388608.0f), f, 16777216.0f * 5.0f / 6.0f);
    c[2] = fmaf(f2, f * (-16777216.0f / 6.0f), 16777216.0f);
  }
};

// Cubic K3 with a = -1/2 (Appendix A), Catmull-Rom.  The inner piece
// 1 - 5/2 t^2 + 3/2 t^3 is factored as (1 - t)(1 + t(1 - 3t/2)) so that the taps at
// t = f and t = 1 - f carry no cancellation near f = 0 or 1 (1 - t is then the exact
// g or f):  -f g^2/2,  g(1 + f(1 - 3f/2)),  f(1 + g(1 - 3g/2)),  -g f^2/2.
template <> struct Filter<STF_FILTER_CATMULL_ROM> {
  static constexpr int T = 4, OFF0 = -1;
  static constexpr bool NONNEG = false, UNIT_SUM = false;
  __device__ __forceinline__ static void weights(float f, float* w) {
    const float g = 1.0f - f;
    w[0] = -0.5f * f * g * g;
    w[1] = g * fmaf(f, fmaf(-1.5f, f, 1.0f), 1.0f);
    w[2] = f * fmaf(g, fmaf(-1.5f, g, 1.0f), 1.0f);
    w[3] = -0.5f * g * f * f;
  }
};

// Positivized Catmull-Rom: the same weights, a different stochastic estimator.
template <> struct Filter<STF_FILTER_CATMULL_ROM_POSITIVIZED> : Filter<STF_FILTER_CATMULL_ROM> {};

// ---------------------------------------------------------------- tap choice
// Inverse CDF over |w| (sampling arrays, Section 2.2): tap k is the smallest k with
// u*S < C_k, C_k = running float32 sum of |w_j|, S = C_{T-1}.  Because u <= 1 - 2^-24
// and S >= 1, the float32 product u*S is always below S, so that k equals the
// number of interior boundaries C_0 .. C_{T-2} that are <= u*S; zero-weight taps
// (C_k == C_{k-1}) are skipped by construction.
// Number of the boundaries c[0] <= c[1] <= ... <= c[T-2] that are <= v.  Every caller's
// boundaries are non-decreasing (running sums of |w|, or the closed forms, whose
// neighbours differ by a weight of at least 1/6), so for four taps the comparison with
// the middle boundary picks the half and one more comparison the tap: the same count
// with two comparisons instead of three.
template <int T>
__device__ __forceinline__ int boundaries_below(float v, const float* c) {
  if constexpr (T == 4) {
    const bool upper = v >= c[1];
    return (upper ? 2 : 0) + ((v >= (upper ? c[2] : c[0])) ? 1 : 0);
  } else {
    int k = 0;
#pragma unroll
    for (int j = 0; j < T - 1; ++j) k += (v >= c[j]) ? 1 : 0;
    return k;
  }
}

template <int T>
struct TapPick {
  int k;
  float S;     // sum |w|
  float us;    // u * S
  float c[T];  // running sums
};

template <int T>
__device__ __forceinline__ TapPick<T> choose_tap(float u, const float* w) {
  TapPick<T> p;
  p.c[0] = fabsf(w[0]);
#pragma unroll
  for (int k = 1; k < T; ++k) p.c[k] = __fadd_rn(p.c[k - 1], fabsf(w[k]));
  p.S = p.c[T - 1];
  p.us = __fmul_rn(u, p.S);
  p.k = boundaries_below<T>(p.us, p.c);
  return p;
}

// Sign of the chosen weight for the Catmull-Rom window, whose taps carry the signs
// (-, +, +, -); a zero weight is never chosen.
__device__ __forceinline__ float cr_sign(int k) { return ((k + 1) & 2) ? 1.0f : -1.0f; }

// Eq. 4 generalised to T taps: u' = (u*S - C_{k-1}) / |w_k|, kept in [0, 1).
template <int T>
__device__ __forceinline__ float remap_variate(const TapPick<T>& p, const float* w) {
  float cprev = 0.0f, wk = 1.0f;
#pragma unroll
  for (int j = 0; j < T; ++j) {
    if (j == p.k) wk = fabsf(w[j]);
    if (j + 1 == p.k) cprev = p.c[j];
  }
  return fminf(fmaxf(__fdiv_rn(__fsub_rn(p.us, cprev), wk), 0.0f), 0x1.fffffep-1f);
}

// Integer tap base floor(x) and fraction x - floor(x); |x| < 2^24 here.
__device__ __forceinline__ int axis_base(float x, float& f) {
  const float fl = floorf(x);
  f = __fsub_rn(x, fl);
  return (int)fl;
}

// Coordinates are used as is when every |x| < 2^24.  Otherwise: a NaN or infinity
// makes the query return the background value (false); finite values beyond 2^24
// (all integers in float32) are clamped to +-2^24, which leaves floor(x) = +-2^24
// and fraction 0, the same as clamping floor(x).
template <int D>
__device__ __forceinline__ bool prepare_coords(float* x) {
  bool small = true;
#pragma unroll
  for (int a = 0; a < D; ++a) small = small && fabsf(x[a]) < 16777216.0f;
  if (small) return true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (!isfinite(x[a])) return false;
    x[a] = fminf(fmaxf(x[a], -16777216.0f), 16777216.0f);
  }
  return true;
}

// One tap per axis for a D-dimensional separable filter.  u[a] is axis a's own
// variate; with REUSE only u[0] is used and carried across axes by Eq. 4.
// Returns the tap coordinates and the estimator's scale sigma (prod sign * S for
// Catmull-Rom, exactly 1 for the non-negative kernels).
// With independent variates and a kernel whose weights sum to exactly 1 (tent, cubic
// B-spline) the tap is the number of closed-form CDF boundaries C_0 .. C_{T-2} that are
// <= u (S = 1): the same rule, without summing the weights.  Its float32 boundaries
// differ from the summed ones by a few 1e-8, inside the 1e-6 band in which the tap is
// allowed to differ from the float64 reference.
template <int F, int D, bool REUSE>
__device__ __forceinline__ float pick_taps(const float* x, const float* u, int* idx) {
  using Fl = Filter<F>;
  if constexpr (!REUSE && Fl::UNIT_SUM) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float f;
      const int b = axis_base(x[a], f);
      float c[Fl::T - 1];
      Fl::cdf(f, c);
      idx[a] = b + Fl::OFF0 + boundaries_below<Fl::T>(u[a], c);
    }
    return 1.0f;
  }
  float sigma = 1.0f;
  float uc = u[0];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float f;
    const int b = axis_base(x[a], f);
    float w[Fl::T];
    Fl::weights(f, w);
    const TapPick<Fl::T> p = choose_tap<Fl::T>(REUSE ? uc : u[a], w);
    if constexpr (REUSE) uc = remap_variate<Fl::T>(p, w);
    if constexpr (!Fl::NONNEG) sigma *= cr_sign(p.k) * p.S;
    idx[a] = b + Fl::OFF0 + p.k;
  }
  return sigma;
}

// pick_taps from the raw Philox words r (word a for axis a).  For the closed-form
// kernels the 24-bit integer variate is compared with the boundaries scaled by 2^24,
// which skips the conversion of the variate to [0, 1) and decides identically.
template <int F, int D, bool REUSE>
__device__ __forceinline__ float pick_taps_r(const float* x, const uint4& r, int* idx) {
  using Fl = Filter<F>;
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
  if constexpr (!REUSE && Fl::UNIT_SUM) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float f;
      const int b = axis_base(x[a], f);
      float c[Fl::T - 1];
      Fl::cdf24(f, c);
      idx[a] = b + Fl::OFF0 + boundaries_below<Fl::T>((float)(w[a] >> 8), c);
    }
    return 1.0f;
  } else {
    float u[D];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = unit24(w[a]);
    return pick_taps<F, D, REUSE>(x, u, idx);
  }
}

// ---------------------------------------------------------------- misses
// Filters whose estimate is the fetched texel itself, drawn from the fixed window
// floor(x) + LO .. floor(x) + HI on every axis: the tent and the cubic B-spline, as
// discrete taps or by filter importance sampling (a sum of 1 or 3 uniforms on
// [-1/2, 1/2) keeps floor(x + s + 1/2) in the same window).  When that window lies
// outside the region that holds texels on some axis, every tap the draw can reach reads
// the background, so the lookup returns it without drawing (the same value).
template <int F> struct FixedWindow { static constexpr bool value = false; static constexpr int LO = 0, HI = 0; };
template <> struct FixedWindow<STF_FILTER_LINEAR> { static constexpr bool value = true; static constexpr int LO = 0, HI = 1; };
template <> struct FixedWindow<STF_FILTER_BSPLINE3> { static constexpr bool value = true; static constexpr int LO = -1, HI = 2; };
template <> struct FixedWindow<STF_FILTER_FIS_LINEAR> { static constexpr bool value = true; static constexpr int LO = 0, HI = 1; };
template <> struct FixedWindow<STF_FILTER_FIS_BSPLINE3> { static constexpr bool value = true; static constexpr int LO = -1, HI = 2; };

// The window misses [lo, hi) on an axis iff floor(x) + HI < lo or floor(x) + LO >= hi,
// that is x < lo - HI or x >= hi - LO for the integers lo - HI and hi - LO; compared
// with these integers rounded up to float32 both tests stay exact.
struct MissBox {
  float lo[3], hi[3];
};

template <int F>
__device__ __forceinline__ MissBox miss_box(int lx, int ly, int lz, int hx, int hy, int hz) {
  using W = FixedWindow<F>;
  MissBox m;
  m.lo[0] = __int2float_ru(lx - W::HI); m.lo[1] = __int2float_ru(ly - W::HI); m.lo[2] = __int2float_ru(lz - W::HI);
  m.hi[0] = __int2float_ru(hx - W::LO); m.hi[1] = __int2float_ru(hy - W::LO); m.hi[2] = __int2float_ru(hz - W::LO);
  return m;
}

__device__ __forceinline__ bool misses(const MissBox& m, const float* x) {
  return x[0] < m.lo[0] || x[0] >= m.hi[0] || x[1] < m.lo[1] || x[1] >= m.hi[1] || x[2] < m.lo[2] ||
         x[2] >= m.hi[2];
}

// ---------------------------------------------------------------- views
struct Tex2DView {
  const void* texels;     // storage format, [level][y][x][c]; DCT6: [level][by][bx][c] words
  int64_t level_off[STF_MAX_LEVELS];   // offset of each level: texels, or DCT6 code words
  int32_t level_w[STF_MAX_LEVELS];
  int32_t level_h[STF_MAX_LEVELS];
  int32_t levels;
  // DCT6 only
  int32_t blocks_w[STF_MAX_LEVELS];    // blocks per row of each level
  float ac_step[8];                    // value of one AC code step per channel, R_c / 15
  // a(0) = sqrt(1/8); (1/2) cos((2i+1) pi/16), i = 0..3; (1/2) cos(pi/8), (1/2) cos(3 pi/8)
  float dct_k[7];
};

struct Dense3DView {
  const void* texels;     // [z][y][x]
  int32_t nx, ny, nz;
  float background;
};

struct LookupArgs {
  const float* coords;
  const float* lod;
  int64_t n;
  float* out;
  int32_t* taps;
  uint32_t key0, key1;
  uint64_t query_offset;
  uint32_t sample_index;
  int32_t reuse;
  int32_t level_mode;
  float width;            // Gaussian FIS: sigma in texels
  int32_t n_samples;      // accumulate kernels
  double* sum;
  double* sumsq;
  // Binned calls: coords/lod are in binned order and perm[i] is the caller's index
  // of binned query i (it keys the generator and picks the output slot).
  const uint32_t* perm;
  // Triplanar calls: coords are positions (n x 3), normals n x 3, uv = scale * p.
  const float* normals;
  float tri_scale;
};

// Calls without a binning permutation or tap output and with at most 2^30 queries
// run the stochastic kernels' loops on 32-bit indices, without the per-query pointer
// tests (3 i + 2 then stays below 2^32); other calls take the general 64-bit loop.
constexpr int64_t kFastLoopMaxQueries = int64_t(1) << 30;

__device__ __forceinline__ bool fast_loop(const LookupArgs& a) {
  return a.perm == nullptr && a.taps == nullptr && a.n <= kFastLoopMaxQueries;
}

// The 3D fast loop takes four consecutive queries per thread when the coordinates and
// results are 16-byte aligned: its coordinates are then three aligned 16-byte loads
// and its four results one 16-byte store.  Host and device test the same condition
// (the host sizes the grid by it).
__host__ __device__ __forceinline__ bool quad_loop3_ok(const LookupArgs& a) {
  return a.perm == nullptr && a.taps == nullptr && a.n <= kFastLoopMaxQueries &&
         (((uintptr_t)a.coords | (uintptr_t)a.out) & 15) == 0;
}

// Queries 4g .. 4g + 3 for g = thread, thread + stride, ...; the last n mod 4 queries
// one per thread.  one(x, y, z, j) filters the query with caller's index j.
template <class One>
__device__ __forceinline__ void quad_loop3(const LookupArgs& a, One one) {
  const uint32_t n = (uint32_t)a.n, groups = n >> 2, stride = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const float4* c4 = reinterpret_cast<const float4*>(a.coords);
  float4* o4 = reinterpret_cast<float4*>(a.out);
  for (uint32_t g = tid; g < groups; g += stride) {
    const float4 p = __ldg(c4 + 3 * g), q = __ldg(c4 + 3 * g + 1), r = __ldg(c4 + 3 * g + 2);
    const uint32_t i = 4 * g;
    float4 o;
    o.x = one(p.x, p.y, p.z, i);
    o.y = one(p.w, q.x, q.y, i + 1);
    o.z = one(q.z, q.w, r.x, i + 2);
    o.w = one(r.y, r.z, r.w, i + 3);
    o4[g] = o;
  }
  for (uint32_t i = 4 * groups + tid; i < n; i += stride)
    a.out[i] = one(__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2), i);
}

// quad_loop3 with a thread's four queries handed over together, so that their
// independent work (generator chains, gathers) can overlap: quad(x, i) returns the
// results of queries i .. i + 3 from their coordinates x[4][3]; the tail as one().
template <class Quad, class One>
__device__ __forceinline__ void quad_loop3_joint(const LookupArgs& a, Quad quad, One one) {
  const uint32_t n = (uint32_t)a.n, groups = n >> 2, stride = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const float4* c4 = reinterpret_cast<const float4*>(a.coords);
  float4* o4 = reinterpret_cast<float4*>(a.out);
  for (uint32_t g = tid; g < groups; g += stride) {
    const float4 p = __ldg(c4 + 3 * g), q = __ldg(c4 + 3 * g + 1), r = __ldg(c4 + 3 * g + 2);
    float x[4][3] = {{p.x, p.y, p.z}, {p.w, q.x, q.y}, {q.z, q.w, r.x}, {r.y, r.z, r.w}};
    o4[g] = quad(x, 4 * g);
  }
  for (uint32_t i = 4 * groups + tid; i < n; i += stride)
    a.out[i] = one(__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2), i);
}

__device__ __forceinline__ int64_t query_slot(const LookupArgs& a, int64_t i) {
  return a.perm ? (int64_t)__ldg(a.perm + i) : i;
}

// Philox variates of the caller's query j for one sample index (and stream).
__device__ __forceinline__ uint4 query_variates(const LookupArgs& a, int64_t j, uint32_t sample,
                                                uint32_t stream = 0u) {
  const uint64_t q = a.query_offset + (uint64_t)j;
  return philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), sample, stream), a.key0, a.key1);
}

// Positivization (Section 2.2): with the Catmull-Rom signs (-, +, +, -) on every
// axis, the 2^D blocks "inner taps (1, 2) or outer taps (0, 3) on each axis"
// partition the taps by sign (an even number of outer axes is positive).  Each set
// is sampled once: a block with probability proportional to its mass (variate
// u[D]; blocks in increasing order, float32 running sums), then on each axis one tap
// of the block's pair with probability proportional to |w| (variate u[a]).  Returns
// the positive and negative tap coordinates and W+, W- (sums of |w| in each set).
template <int D>
__device__ __forceinline__ void pick_positivized(const float* x, const float* up, const float* un,
                                                 int* ip, int* in, float& Wp, float& Wn) {
  using Fl = Filter<STF_FILTER_CATMULL_ROM>;
  float aw[D][4], ain[D], aout[D];
  int base[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float f, w[4];
    base[a] = axis_base(x[a], f) + Fl::OFF0;
    Fl::weights(f, w);
#pragma unroll
    for (int k = 0; k < 4; ++k) aw[a][k] = fabsf(w[k]);
    ain[a] = __fadd_rn(aw[a][1], aw[a][2]);
    aout[a] = __fadd_rn(aw[a][0], aw[a][3]);
  }
  float m[1 << D];
#pragma unroll
  for (int b = 0; b < (1 << D); ++b) {
    float p = 1.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) p = __fmul_rn(p, ((b >> a) & 1) ? aout[a] : ain[a]);
    m[b] = p;
  }
#pragma unroll
  for (int set = 0; set < 2; ++set) {               // 0: positive (even), 1: negative (odd)
    const float* u = set ? un : up;
    float C[(1 << D) / 2];
    int blk[(1 << D) / 2];
    float acc = 0.0f;
    int nb = 0;
#pragma unroll
    for (int b = 0; b < (1 << D); ++b)
      if ((__popc(b) & 1) == set) {
        acc = __fadd_rn(acc, m[b]);
        C[nb] = acc;
        blk[nb] = b;
        ++nb;
      }
    const float us = __fmul_rn(u[D], acc);
    int chosen = blk[0];
#pragma unroll
    for (int j = 0; j < (1 << D) / 2 - 1; ++j)
      if (us >= C[j]) chosen = blk[j + 1];
    int* idx = set ? in : ip;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool outer = (chosen >> a) & 1;
      const float w0 = outer ? aw[a][0] : aw[a][1], w1 = outer ? aw[a][3] : aw[a][2];
      const float s2 = __fadd_rn(w0, w1);
      const bool second = __fmul_rn(u[a], s2) >= w0;
      idx[a] = base[a] + (outer ? (second ? 3 : 0) : (second ? 2 : 1));
    }
    if (set) Wn = acc; else Wp = acc;
  }
}

// ---------------------------------------------------------------- filter importance sampling
// Section 4.4, "Filter Importance Sampling": an offset s is drawn from a density and
// the texel nearest to x + s, floor(x + s + 1/2), is fetched unscaled.  Taking the
// nearest texel convolves the density with a unit box; that convolution is the
// filter applied (a B-spline of one degree higher, or the box-blurred Gaussian).
template <int F>
struct IsFis {
  static constexpr bool value = F == STF_FILTER_FIS_LINEAR || F == STF_FILTER_FIS_BSPLINE3 ||
                                F == STF_FILTER_FIS_GAUSSIAN;
};

// Filters whose stochastic form can carry one variate across axes (Eq. 4).
template <int F>
struct UsesReuse {
  static constexpr bool value = !IsFis<F>::value && F != STF_FILTER_CATMULL_ROM_POSITIVIZED;
};

// Deterministic forms of the B-spline FIS filters: the filters they apply.
template <> struct Filter<STF_FILTER_FIS_LINEAR> : Filter<STF_FILTER_LINEAR> {};
template <> struct Filter<STF_FILTER_FIS_BSPLINE3> : Filter<STF_FILTER_BSPLINE3> {};

// B-splines: s is the sum of n uniforms on [-1/2, 1/2), so the index is
// floor(x + sum u - (n - 1)/2).  With u = k 2^-24 (24-bit integers k) and x 2^24 exact
// in float32 (|x| <= 2^24), it is formed exactly in 64-bit integers as
// (floor(x 2^24) + sum k - (n - 1) 2^23) >> 24 (arithmetic shift = floor division).
__device__ __forceinline__ int fis_bspline_index(float x, uint32_t ksum, int n) {
  const long long X = __float2ll_rd(__fmul_rn(x, 16777216.0f));
  return (int)((X + (long long)ksum - (long long)(n - 1) * 8388608LL) >> 24);
}

// Gaussian: Box-Muller radius sigma sqrt(-2 ln(1 - u)); 1 - u is exact and positive
// for a 24-bit u, so the largest radius is sigma sqrt(48 ln 2) = 5.7683 sigma.
__device__ __forceinline__ float bm_radius(float u, float sigma) {
  return sigma * sqrtf(-2.0f * logf(1.0f - u));
}

// floor(x + s + 1/2) as floor(x) + floor(frac(x) + s + 1/2), which keeps the float32
// sum small.
__device__ __forceinline__ int fis_nearest(float x, float s) {
  float f;
  const int b = axis_base(x, f);
  return b + (int)floorf(__fadd_rn(__fadd_rn(f, s), 0.5f));
}

// Tap of each axis for the FIS filters.  Variates: B-spline uniform j of axis a is
// word a of Philox stream j; the Gaussian takes the Box-Muller pair (word 0, word 1)
// of stream 0 for x and y, and (word 2, word 3) for z.  r0 is stream 0.
template <int F, int D>
__device__ __forceinline__ void pick_fis(const float* x, const LookupArgs& a, int64_t j,
                                         uint32_t sample, const uint4& r0, int* idx) {
  const uint32_t w0[4] = {r0.x, r0.y, r0.z, r0.w};
  if constexpr (F == STF_FILTER_FIS_GAUSSIAN) {
    const float r = bm_radius(unit24(r0.x), a.width);
    float sn, cs;
    sincospif(2.0f * unit24(r0.y), &sn, &cs);
    idx[0] = fis_nearest(x[0], r * cs);
    idx[1] = fis_nearest(x[1], r * sn);
    if constexpr (D == 3) idx[2] = fis_nearest(x[2], bm_radius(unit24(r0.z), a.width) *
                                                         cospif(2.0f * unit24(r0.w)));
  } else if constexpr (F == STF_FILTER_FIS_LINEAR) {
#pragma unroll
    for (int d = 0; d < D; ++d) idx[d] = fis_bspline_index(x[d], w0[d] >> 8, 1);
  } else {
    const uint4 r1 = query_variates(a, j, sample, 1u), r2 = query_variates(a, j, sample, 2u);
    const uint32_t w1[4] = {r1.x, r1.y, r1.z, r1.w}, w2[4] = {r2.x, r2.y, r2.z, r2.w};
#pragma unroll
    for (int d = 0; d < D; ++d)
      idx[d] = fis_bspline_index(x[d], (w0[d] >> 8) + (w1[d] >> 8) + (w2[d] >> 8), 3);
  }
}

// Filters whose dense 3D stochastic lookups take the joint four-query form: one tap
// from one set of draws per query, independent variates per axis, and a gain measured
// on the dense benchmark rays (tent +14%, B-spline +6%, FIS tent +8%, FIS B-spline +5%,
// FIS Gaussian +3%).  Catmull-Rom measured 4% slower in it and keeps the one-query
// form; so do the two-tap positivized estimator and the sparse grids, whose traversal
// per tap measured 7% slower joint.
template <int F, bool REUSE>
struct JointOneTap {
  static constexpr bool value = (F == STF_FILTER_LINEAR || F == STF_FILTER_BSPLINE3 || IsFis<F>::value) && !REUSE;
};

// The tap of one such lookup at coordinates x (checked by prepare_coords) from its
// stream-0 variates r; returns the estimator's scale (sign * S for Catmull-Rom, else 1).
template <int F>
__device__ __forceinline__ float draw_one_tap3(const LookupArgs& a, const float* x, uint32_t j,
                                               const uint4& r, int* idx) {
  if constexpr (IsFis<F>::value) {
    pick_fis<F, 3>(x, a, j, a.sample_index, r, idx);
    return 1.0f;
  } else {
    return pick_taps_r<F, 3, false>(x, r, idx);
  }
}

// Four queries i .. i + 3 of quad_loop3_joint through a one-tap filter.  Each query's
// coordinates are checked and, for a fixed-window filter, tested against the miss box
// (a miss returns the background without drawing, as in the one-query form); when any
// of the four is live, all four draw (a dead query's draw is discarded), then the live
// ones fetch.  The four generator chains and the four gathers are independent, so
// they overlap; the results equal the one-query form's.  fetch(idx) returns the texel
// at idx, or the background outside the stored region.
template <int F, class Fetch>
__device__ __forceinline__ float4 joint_one_tap4(const LookupArgs& a, float (&x)[4][3], uint32_t i,
                                                 const MissBox& mb, float background, Fetch fetch) {
  bool live[4];
  bool any = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    live[k] = prepare_coords<3>(x[k]);
    if constexpr (FixedWindow<F>::value) live[k] = live[k] && !misses(mb, x[k]);
    any = any || live[k];
  }
  float v[4] = {background, background, background, background};
  if (any) {
    uint4 r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = query_variates(a, i + k, a.sample_index);
    int idx[4][3];
    float sigma[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) sigma[k] = draw_one_tap3<F>(a, x[k], i + k, r[k], idx[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (live[k]) {
        float t = fetch(idx[k]);
        if constexpr (F == STF_FILTER_CATMULL_ROM) t *= sigma[k];
        v[k] = t;
      }
    }
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

// Deterministic form of the Gaussian FIS filter, one axis: taps lo..hi, the nearest
// texels of x -+ 5.7683 sigma (every tap a 24-bit draw can reach), with weights
// (erf((i + 1/2 - x) k) - erf((i - 1/2 - x) k)) / 2, k = 1 / (sigma sqrt 2): the
// Gaussian convolved with the unit box.  The mass beyond the window is below 1e-8.
struct GaussAxis {
  int lo, hi;
  float x, k;
};

__device__ __forceinline__ GaussAxis gauss_axis(float x, float sigma) {
  GaussAxis g;
  const float R = 5.7683466f * sigma;
  g.lo = (int)floorf(__fadd_rn(__fsub_rn(x, R), 0.5f));
  g.hi = (int)floorf(__fadd_rn(__fadd_rn(x, R), 0.5f));
  g.x = x;
  g.k = 0.70710678f / sigma;
  return g;
}

// Edge value erf((e - x) k) at e = i - 1/2; consecutive taps share their edges.
__device__ __forceinline__ float gauss_edge(const GaussAxis& g, int i) {
  return erff(__fsub_rn((float)i - 0.5f, g.x) * g.k);
}

// Sum over the D-dimensional Gaussian window of prod_a w_a(i_a) * fetch(i).  Each
// axis walks its taps carrying the shared edge value, so a tap costs one erf per
// axis.
template <class Fetch>
__device__ __forceinline__ float gauss_window_sum3(const float* x, float sigma, Fetch fetch) {
  const GaussAxis gx = gauss_axis(x[0], sigma), gy = gauss_axis(x[1], sigma),
                  gz = gauss_axis(x[2], sigma);
  float acc = 0.0f;
  float ez0 = gauss_edge(gz, gz.lo);
  for (int iz = gz.lo; iz <= gz.hi; ++iz) {
    const float ez1 = gauss_edge(gz, iz + 1);
    const float wz = 0.5f * (ez1 - ez0);
    ez0 = ez1;
    float ey0 = gauss_edge(gy, gy.lo);
    for (int iy = gy.lo; iy <= gy.hi; ++iy) {
      const float ey1 = gauss_edge(gy, iy + 1);
      const float wyz = 0.5f * (ey1 - ey0) * wz;
      ey0 = ey1;
      float ex0 = gauss_edge(gx, gx.lo);
      for (int ix = gx.lo; ix <= gx.hi; ++ix) {
        const float ex1 = gauss_edge(gx, ix + 1);
        acc = fmaf(0.5f * (ex1 - ex0) * wyz, fetch(ix, iy, iz), acc);
        ex0 = ex1;
      }
    }
  }
  return acc;
}

template <int FMT, int C> struct TexelIO;

template <int C> struct TexelIO<STF_FMT_F32, C> {
  __device__ __forceinline__ static void load(const void* base, int64_t texel, float* v) {
    const float* p = reinterpret_cast<const float*>(base) + texel * C;
    if constexpr (C == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (C == 2) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(p));
      v[0] = q.x; v[1] = q.y;
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = __ldg(p + c);
    }
  }
};

template <int C> struct TexelIO<STF_FMT_F16, C> {
  __device__ __forceinline__ static void load(const void* base, int64_t texel, float* v) {
    const __half* p = reinterpret_cast<const __half*>(base) + texel * C;
    if constexpr (C == 8) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
      const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f2 = __half22float2(h[j]);
        v[2 * j] = f2.x; v[2 * j + 1] = f2.y;
      }
    } else if constexpr (C == 4) {
      const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
      const __half2* h = reinterpret_cast<const __half2*>(&q);
      const float2 a = __half22float2(h[0]), b = __half22float2(h[1]);
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = __half2float(__ldg(p + c));
    }
  }
};

// ---------------------------------------------------------------- DCT6 texels
// a(u) cos((2x+1) u pi / 16) for u = 0, 1, 2 from the seven stored constants, using
// c1(7 - x) = -c1(x) and c2(7 - x) = c2(x) (only compile-time indices into the view).
__device__ __forceinline__ void dct_basis(const Tex2DView& t, int x, float& c0, float& c1, float& c2) {
  const bool lo = x < 4;
  const int i = lo ? x : 7 - x;
  const float m1 = i == 0 ? t.dct_k[1] : i == 1 ? t.dct_k[2] : i == 2 ? t.dct_k[3] : t.dct_k[4];
  c0 = t.dct_k[0];
  c1 = lo ? m1 : -m1;
  const float m2 = (i == 0 || i == 3) ? t.dct_k[5] : t.dct_k[6];
  c2 = i < 2 ? m2 : -m2;
}

__device__ __forceinline__ float dct_ac(uint32_t w, int j) {
  return (float)(((int32_t)(w << (20 - 5 * j))) >> 27);     // 5-bit field, sign-extended
}

// Texel (x, y) of level L, clamped to the level: f = sum over the six coefficients of
// value * basis(x) * basis(y), float32.
template <int C>
__device__ __forceinline__ void dct_texel(const Tex2DView& t, int L, int x, int y, float* v) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(t.texels) + t.level_off[L] +
                      ((int64_t)(y >> 3) * t.blocks_w[L] + (x >> 3)) * C;
  uint32_t w[C];
  if constexpr (C % 4 == 0) {
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p) + k);
      w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
    }
  } else if constexpr (C == 2) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = q.x; w[1] = q.y;
  } else {
    w[0] = __ldg(p);
  }
  float x0, x1, x2, y0, y1, y2;
  dct_basis(t, x & 7, x0, x1, x2);
  dct_basis(t, y & 7, y0, y1, y2);
  // DC code step folded into its basis product; each channel's AC step multiplies the
  // sum of its five integer codes times their basis products
  const float b[6] = {x0 * y0 * (8.0f / 127.0f), x1 * y0, x0 * y1, x2 * y0, x1 * y1, x0 * y2};
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float ac = dct_ac(w[c], 0) * b[1];
#pragma unroll
    for (int j = 1; j < 5; ++j) ac = fmaf(dct_ac(w[c], j), b[j + 1], ac);
    v[c] = fmaf(t.ac_step[c], ac, (float)(w[c] & 127u) * b[0]);
  }
}

// Texel (cx, cy) of level L, already clamped to the level, in any 2D storage format.
template <int FMT, int C>
__device__ __forceinline__ void fetch2d(const Tex2DView& t, int L, int cx, int cy, float* v) {
  if constexpr (FMT == STF_FMT_DCT6) dct_texel<C>(t, L, cx, cy, v);
  else TexelIO<FMT, C>::load(t.texels, t.level_off[L] + (int64_t)cy * t.level_w[L] + cx, v);
}

template <int C>
__device__ __forceinline__ void store_out(float* out, int64_t i, const float* v) {
  float* p = out + i * C;
  if constexpr (C == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (C == 8) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else if constexpr (C == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) p[c] = v[c];
  }
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

}  // namespace stf
