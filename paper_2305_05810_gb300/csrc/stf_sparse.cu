// Sparse voxel grids in a NanoVDB-style hierarchy: a root list of upper nodes
// (32^3 children, 4096^3 voxels each), lower nodes (16^3 children, 128^3 voxels)
// and 8^3-voxel leaves; children are located through bit masks plus per-word
// popcount prefixes, so a lookup is a fixed-depth walk with no loops that depend
// on the data (except the short root list).
//
// The paper names NanoVDB as the sparse format it filters (Section 5.3) but gives
// no layout; this one keeps the NanoVDB fan-outs and voxel order
// (x & 7) << 6 | (y & 7) << 3 | (z & 7) within a leaf.
#include <algorithm>
#include <climits>
#include <vector>

#include "stf_internal.h"

namespace stf {

// ---------------------------------------------------------------- builder

static inline int lower_bit(int x, int y, int z) {
  return (((x >> 7) & 31) << 10) | (((y >> 7) & 31) << 5) | ((z >> 7) & 31);
}
static inline int leaf_bit(int x, int y, int z) {
  return (((x >> 3) & 15) << 8) | (((y >> 3) & 15) << 4) | ((z >> 3) & 15);
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Leaves in tree order: dst leaf l takes source leaf perm[l]; FP32 copy or E4M3 with
// scale = max|v| / 448 (1 for an all-zero leaf), codes = E4M3(v / scale), RNE,
// saturating.  One 128-thread block per leaf.
__global__ void __launch_bounds__(128) k_leaf_place(const float* __restrict__ src,
                                                    const int32_t* __restrict__ perm,
                                                    int64_t n_leaves, int fmt, float* dst_f32,
                                                    uint8_t* dst_e4m3, float* dst_scale) {
  __shared__ float red[4];
  for (int64_t l = blockIdx.x; l < n_leaves; l += gridDim.x) {
    const float4 v =
        reinterpret_cast<const float4*>(src + (int64_t)perm[l] * 512)[threadIdx.x];
    if (fmt == STF_FMT_F32) {
      reinterpret_cast<float4*>(dst_f32 + l * 512)[threadIdx.x] = v;
      continue;
    }
    float m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
    __syncthreads();
    float scale = __fdiv_rn(m, 448.0f);
    if (!(scale > 0.0f)) scale = 1.0f;
    const float q[4] = {v.x, v.y, v.z, v.w};
    uint32_t packed = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_fp8_storage_t c =
          __nv_cvt_float_to_fp8(__fdiv_rn(q[k], scale), __NV_SATFINITE, __NV_E4M3);
      packed |= (uint32_t)c << (8 * k);
    }
    reinterpret_cast<uint32_t*>(dst_e4m3 + l * 512)[threadIdx.x] = packed;
    if (threadIdx.x == 0) dst_scale[l] = scale;
  }
}

stf_status build_sparse(stf_texture_s* t, const stf_texture_desc* d, cudaStream_t s) {
  const int64_t nl = d->num_leaves;
  if (nl > (int64_t)INT32_MAX) return fail(STF_ERR_INVALID_ARGUMENT, "too many leaves");
  std::vector<int32_t> org((size_t)(3 * nl));
  cudaError_t e = cudaSuccess;
  if (nl > 0) {
    e = cudaMemcpy(org.data(), d->leaf_origins, sizeof(int32_t) * 3 * nl,
                   d->data_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return fail_cuda(e, "leaf origin read");
  }
  // Upper nodes: distinct origin & ~4095, sorted.
  struct Key3 {
    int32_t x, y, z;
    bool operator<(const Key3& o) const {
      return x != o.x ? x < o.x : (y != o.y ? y < o.y : z < o.z);
    }
    bool operator==(const Key3& o) const { return x == o.x && y == o.y && z == o.z; }
  };
  std::vector<Key3> uppers;
  for (int64_t l = 0; l < nl; ++l) {
    const int32_t x = org[3 * l], y = org[3 * l + 1], z = org[3 * l + 2];
    if ((x & 7) || (y & 7) || (z & 7))
      return fail(STF_ERR_INVALID_ARGUMENT, "leaf origin %lld is not a multiple of 8", (long long)l);
    uppers.push_back({x & ~4095, y & ~4095, z & ~4095});
  }
  std::sort(uppers.begin(), uppers.end());
  uppers.erase(std::unique(uppers.begin(), uppers.end()), uppers.end());
  const int n_upper = (int)uppers.size();
  if (n_upper > 4096) return fail(STF_ERR_UNSUPPORTED, "more than 4096 upper nodes");
  // Sort leaves by (upper, lower slot, leaf slot).
  std::vector<std::pair<uint64_t, int32_t>> rec((size_t)nl);
  for (int64_t l = 0; l < nl; ++l) {
    const int32_t x = org[3 * l], y = org[3 * l + 1], z = org[3 * l + 2];
    const Key3 k{x & ~4095, y & ~4095, z & ~4095};
    const uint64_t u = (uint64_t)(std::lower_bound(uppers.begin(), uppers.end(), k) - uppers.begin());
    rec[l] = {(u << 27) | ((uint64_t)lower_bit(x, y, z) << 12) | (uint64_t)leaf_bit(x, y, z),
              (int32_t)l};
  }
  std::sort(rec.begin(), rec.end());
  for (int64_t l = 1; l < nl; ++l)
    if (rec[l].first == rec[l - 1].first)
      return fail(STF_ERR_INVALID_ARGUMENT, "duplicate leaf origin (leaf %d)", rec[l].second);
  // Masks and prefixes.
  std::vector<uint64_t> umask((size_t)n_upper * 512, 0);
  std::vector<uint32_t> uprefix((size_t)n_upper * 512, 0);
  std::vector<int32_t> ubase((size_t)n_upper, 0), uorigin((size_t)n_upper * 3);
  std::vector<uint64_t> lmask;
  std::vector<int32_t> lbase, perm((size_t)nl);
  int64_t prev_lower_key = -1;
  int prev_upper = -1;
  for (int64_t l = 0; l < nl; ++l) {
    const uint64_t key = rec[l].first;
    const int u = (int)(key >> 27);
    const int lb = (int)((key >> 12) & 32767), fb = (int)(key & 4095);
    perm[l] = rec[l].second;
    if (u != prev_upper) {
      ubase[u] = (int32_t)lbase.size();
      prev_upper = u;
    }
    if ((int64_t)(key >> 12) != prev_lower_key) {
      prev_lower_key = (int64_t)(key >> 12);
      umask[(size_t)u * 512 + (lb >> 6)] |= 1ull << (lb & 63);
      lbase.push_back((int32_t)l);
      lmask.resize(lmask.size() + 64, 0);
    }
    lmask[(lbase.size() - 1) * 64 + (fb >> 6)] |= 1ull << (fb & 63);
  }
  const int n_lower = (int)lbase.size();
  // Absolute prefixes: the node or leaf index of each word's first set bit, so a
  // lookup adds only the popcount below its bit.
  for (int u = 0; u < n_upper; ++u) {
    uint32_t acc = (uint32_t)ubase[u];
    for (int w = 0; w < 512; ++w) {
      uprefix[(size_t)u * 512 + w] = acc;
      acc += (uint32_t)__builtin_popcountll(umask[(size_t)u * 512 + w]);
    }
    uorigin[3 * u] = uppers[u].x;
    uorigin[3 * u + 1] = uppers[u].y;
    uorigin[3 * u + 2] = uppers[u].z;
  }
  std::vector<uint32_t> lrec((size_t)n_lower * 64 * 4, 0);
  for (int lo = 0; lo < n_lower; ++lo) {
    uint32_t acc = (uint32_t)lbase[lo];
    for (int w = 0; w < 64; ++w) {
      const uint64_t m = lmask[(size_t)lo * 64 + w];
      uint32_t* r = lrec.data() + ((size_t)lo * 64 + w) * 4;
      r[0] = (uint32_t)m;
      r[1] = (uint32_t)(m >> 32);
      r[2] = acc;
      acc += (uint32_t)__builtin_popcountll(m);
    }
  }
  // One device allocation: nodes, then leaves.
  const size_t b_uo = align256(sizeof(int32_t) * 3 * (size_t)std::max(n_upper, 1));
  const size_t b_um = align256(sizeof(uint64_t) * umask.size() + 8);
  const size_t b_up = align256(sizeof(uint32_t) * uprefix.size() + 4);
  const size_t b_lr = align256(sizeof(uint32_t) * lrec.size() + 16);
  const bool e4 = d->format == STF_FMT_E4M3_SCALED;
  const size_t b_leaf = align256((size_t)nl * 512 * (e4 ? 1 : 4) + 16);
  const size_t b_scale = e4 ? align256(sizeof(float) * (size_t)nl + 4) : 0;
  const size_t total = b_uo + b_um + b_up + b_lr + b_leaf + b_scale;
  e = dev_alloc(&t->d_tree, total);
  if (e != cudaSuccess) return fail_cuda(e, "sparse tree allocation");
  t->bytes += (int64_t)total;
  char* p = (char*)t->d_tree;
  SparseDev& g = t->sparse;
  // bounding box of the active leaves, clamped to +-2^30 (coordinates beyond 2^24 are
  // clamped by the lookups, so the clamp changes no answer)
  for (int a = 0; a < 3; ++a) {
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (int64_t l = 0; l < nl; ++l) {
      lo = std::min<int64_t>(lo, org[3 * l + a]);
      hi = std::max<int64_t>(hi, (int64_t)org[3 * l + a] + 8);
    }
    if (nl == 0) lo = hi = 0;
    g.bb_lo[a] = (int32_t)std::max<int64_t>(std::min<int64_t>(lo, 1 << 30), -(1 << 30));
    g.bb_hi[a] = (int32_t)std::max<int64_t>(std::min<int64_t>(hi, 1 << 30), -(1 << 30));
  }
  g.n_upper = n_upper;
  g.n_lower = n_lower;
  g.n_leaves = nl;
  g.background = d->background;
  g.upper_origin = (const int32_t*)p;     p += b_uo;
  g.upper_mask = (const uint64_t*)p;      p += b_um;
  g.upper_prefix = (const uint32_t*)p;    p += b_up;
  g.lower_rec = (const uint4*)p;          p += b_lr;
  if (e4) {
    g.leaf_e4m3 = (const uint8_t*)p;      p += b_leaf;
    g.leaf_scale = (const float*)p;       p += b_scale;
  } else {
    g.leaf_f32 = (const float*)p;         p += b_leaf;
  }
  struct Up { const void* dst; const void* src; size_t bytes; } ups[] = {
      {g.upper_origin, uorigin.data(), sizeof(int32_t) * uorigin.size()},
      {g.upper_mask, umask.data(), sizeof(uint64_t) * umask.size()},
      {g.upper_prefix, uprefix.data(), sizeof(uint32_t) * uprefix.size()},
      {g.lower_rec, lrec.data(), sizeof(uint32_t) * lrec.size()}};
  for (const Up& u : ups)
    if (u.bytes && e == cudaSuccess) e = cudaMemcpy((void*)u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_cuda(e, "sparse tree upload");
  if (nl == 0) return STF_OK;
  // Leaf values: stage (if on the host) and place in tree order.
  float* staged = nullptr;
  int32_t* d_perm = nullptr;
  const float* src = (const float*)d->data;
  e = dev_alloc((void**)&d_perm, sizeof(int32_t) * (size_t)nl);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_perm, perm.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !d->data_on_device) {
    e = dev_alloc((void**)&staged, sizeof(float) * 512 * (size_t)nl);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(staged, d->data, sizeof(float) * 512 * nl, cudaMemcpyHostToDevice, s);
    src = staged;
  }
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>(nl, 1 << 20);
    k_leaf_place<<<blocks, 128, 0, s>>>(src, d_perm, nl, d->format, (float*)g.leaf_f32,
                                        (uint8_t*)g.leaf_e4m3, (float*)g.leaf_scale);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(staged);
  cudaFree(d_perm);
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "sparse leaf placement");
}

// ---------------------------------------------------------------- traversal

struct UpperSmem {
  uint64_t mask[512];
  uint32_t prefix[512];
  int32_t origin[3];       // upper node 0 (origin[0] = INT_MIN without upper nodes)
};

// Leaf index holding voxel (x, y, z), or -1 if the voxel lies in no active leaf.
// Upper node 0 (origin, mask and prefixes) is read from shared memory.
__device__ __forceinline__ int64_t sparse_leaf(const SparseDev& g, const UpperSmem& su, int x,
                                               int y, int z) {
  const int ox = x & ~4095, oy = y & ~4095, oz = z & ~4095;
  int u = -1;
  if (su.origin[0] == ox && su.origin[1] == oy && su.origin[2] == oz) {
    u = 0;
  } else {
    for (int j = 1; j < g.n_upper; ++j) {
      const int32_t* o = g.upper_origin + 3 * j;
      if (__ldg(o) == ox && __ldg(o + 1) == oy && __ldg(o + 2) == oz) {
        u = j;
        break;
      }
    }
  }
  if (u < 0) return -1;
  const int lb = (((x >> 7) & 31) << 10) | (((y >> 7) & 31) << 5) | ((z >> 7) & 31);
  const uint64_t bit = 1ull << (lb & 63);
  uint64_t m;
  uint32_t pre;
  if (u == 0) {
    m = su.mask[lb >> 6];
    pre = su.prefix[lb >> 6];
  } else {
    m = __ldg(g.upper_mask + (int64_t)u * 512 + (lb >> 6));
    pre = __ldg(g.upper_prefix + (int64_t)u * 512 + (lb >> 6));
  }
  if (!(m & bit)) return -1;
  const int lower = (int)pre + __popcll(m & (bit - 1));
  if ((unsigned)lower >= (unsigned)g.n_lower) {
    atomicOr(g.status, STF_DEV_BAD_NODE);
    return -1;
  }
  const int fb = (((x >> 3) & 15) << 8) | (((y >> 3) & 15) << 4) | ((z >> 3) & 15);
  const uint64_t bit2 = 1ull << (fb & 63);
  const uint4 rec = __ldg(g.lower_rec + (int64_t)lower * 64 + (fb >> 6));
  const uint64_t m2 = (uint64_t)rec.x | ((uint64_t)rec.y << 32);
  if (!(m2 & bit2)) return -1;
  const int64_t leaf = (int64_t)rec.z + __popcll(m2 & (bit2 - 1));
  if (leaf >= g.n_leaves) {
    atomicOr(g.status, STF_DEV_BAD_NODE);
    return -1;
  }
  return leaf;
}

template <int FMT>
__device__ __forceinline__ float sparse_value(const SparseDev& g, int64_t leaf, int x, int y, int z) {
  if (leaf < 0) return g.background;
  const int v = ((x & 7) << 6) | ((y & 7) << 3) | (z & 7);
  if constexpr (FMT == STF_FMT_F32) {
    return __ldg(g.leaf_f32 + leaf * 512 + v);
  } else {
    const __nv_fp8_storage_t c = __ldg(g.leaf_e4m3 + leaf * 512 + v);
    const __half h(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3));
    return __half2float(h) * __ldg(g.leaf_scale + leaf);
  }
}

__device__ __forceinline__ void stage_upper(const SparseDev& g, UpperSmem& su) {
  if (g.n_upper > 0) {
    for (int k = threadIdx.x; k < 512; k += blockDim.x) {
      su.mask[k] = __ldg(g.upper_mask + k);
      su.prefix[k] = __ldg(g.upper_prefix + k);
    }
  }
  if (threadIdx.x < 3) su.origin[threadIdx.x] = g.n_upper > 0 ? __ldg(g.upper_origin + threadIdx.x) : INT_MIN;
  __syncthreads();
}

// One stochastic lookup at coordinates x (caller's query index j).  J is int64_t, or
// uint32_t in the fast loops.
// With a miss box (the fast loops, which write no tap output), a fixed-window filter
// whose window lies outside the active leaves' bounding box returns the background
// without drawing.
template <int F, int FMT, bool REUSE, typename J>
__device__ __forceinline__ float sparse_stochastic_at(const SparseDev& g, const UpperSmem& su,
                                                      const LookupArgs& a, float* x, J j,
                                                      uint32_t sample, int4& tap,
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
    return sparse_value<FMT>(g, sparse_leaf(g, su, idx[0], idx[1], idx[2]), idx[0], idx[1], idx[2]);
  } else if constexpr (F == STF_FILTER_CATMULL_ROM_POSITIVIZED) {
    const uint4 r1 = query_variates(a, j, sample, 1u);
    const float up[4] = {unit24(r.x), unit24(r.y), unit24(r.z), unit24(r.w)};
    const float un[4] = {unit24(r1.x), unit24(r1.y), unit24(r1.z), unit24(r1.w)};
    int ip[3], in[3];
    float Wp, Wn;
    pick_positivized<3>(x, up, un, ip, in, Wp, Wn);
    tap = make_int4(ip[0], ip[1], ip[2], 0);
    float t = Wp * sparse_value<FMT>(g, sparse_leaf(g, su, ip[0], ip[1], ip[2]), ip[0], ip[1], ip[2]);
    if (Wn > 0.0f)
      t = fmaf(-Wn, sparse_value<FMT>(g, sparse_leaf(g, su, in[0], in[1], in[2]), in[0], in[1], in[2]), t);
    return t;
  } else {
    int idx[3];
    const float sigma = pick_taps_r<F, 3, REUSE>(x, r, idx);
    tap = make_int4(idx[0], idx[1], idx[2], 0);
    float t = sparse_value<FMT>(g, sparse_leaf(g, su, idx[0], idx[1], idx[2]), idx[0], idx[1], idx[2]);
    if constexpr (!Filter<F>::NONNEG) t *= sigma;
    return t;
  }
}

// One stochastic lookup of query i (caller's index j).  I is int64_t, or uint32_t in
// the fast loop (3 i + 2 < 2^32 there).
template <int F, int FMT, bool REUSE, typename I>
__device__ __forceinline__ float sparse_stochastic_one(const SparseDev& g, const UpperSmem& su,
                                                       const LookupArgs& a, I i, I j,
                                                       uint32_t sample, int4& tap) {
  float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
  return sparse_stochastic_at<F, FMT, REUSE>(g, su, a, x, j, sample, tap);
}

template <int F, int FMT, bool REUSE>
__global__ void __launch_bounds__(256) k_sparse_stochastic(SparseDev g, LookupArgs a) {
  __shared__ UpperSmem su;
  stage_upper(g, su);
  const MissBox mb = miss_box<F>(g.bb_lo[0], g.bb_lo[1], g.bb_lo[2], g.bb_hi[0], g.bb_hi[1], g.bb_hi[2]);
  if (quad_loop3_ok(a)) {
    quad_loop3(a, [&](float x0, float x1, float x2, uint32_t j) {
      float x[3] = {x0, x1, x2};
      int4 tap;
      return sparse_stochastic_at<F, FMT, REUSE>(g, su, a, x, j, a.sample_index, tap, &mb);
    });
    return;
  }
  if (fast_loop(a)) {
    const uint32_t n = (uint32_t)a.n, stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
      int4 tap;
      a.out[i] = sparse_stochastic_at<F, FMT, REUSE>(g, su, a, x, i, a.sample_index, tap, &mb);
    }
    return;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    int4 tap;
    const int64_t j = query_slot(a, i);
    a.out[j] = sparse_stochastic_one<F, FMT, REUSE>(g, su, a, i, j, a.sample_index, tap);
    if (a.taps) reinterpret_cast<int4*>(a.taps)[j] = tap;
  }
}

// Deterministic: the tap window spans at most two leaves per axis, so the (up to 8)
// leaves are resolved once and every tap reads from the one that holds it.
template <int F, int FMT>
__global__ void __launch_bounds__(256) k_sparse_deterministic(SparseDev g, LookupArgs a) {
  using Fl = Filter<F>;
  __shared__ UpperSmem su;
  stage_upper(g, su);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    float x[3] = {__ldg(a.coords + 3 * i), __ldg(a.coords + 3 * i + 1), __ldg(a.coords + 3 * i + 2)};
    float acc = g.background;
    if constexpr (F == STF_FILTER_FIS_GAUSSIAN) {
      // Every tap of the window is resolved on its own (root to leaf).
      if (prepare_coords<3>(x))
        acc = gauss_window_sum3(x, a.width, [&](int ix, int iy, int iz) {
          return sparse_value<FMT>(g, sparse_leaf(g, su, ix, iy, iz), ix, iy, iz);
        });
    } else if (prepare_coords<3>(x)) {
      float fx, fy, fz;
      const int bx = axis_base(x[0], fx) + Fl::OFF0, by = axis_base(x[1], fy) + Fl::OFF0,
                bz = axis_base(x[2], fz) + Fl::OFF0;
      float wx[Fl::T], wy[Fl::T], wz[Fl::T];
      Fl::weights(fx, wx);
      Fl::weights(fy, wy);
      Fl::weights(fz, wz);
      // a window outside the active leaves' bounding box on some axis reads only the
      // background, and the weights sum to one (partition of unity)
      if (bx + Fl::T <= g.bb_lo[0] || by + Fl::T <= g.bb_lo[1] || bz + Fl::T <= g.bb_lo[2] ||
          bx >= g.bb_hi[0] || by >= g.bb_hi[1] || bz >= g.bb_hi[2]) {
        a.out[i] = g.background;
        continue;
      }
      const int lx[2] = {bx >> 3, (bx + Fl::T - 1) >> 3};
      const int ly[2] = {by >> 3, (by + Fl::T - 1) >> 3};
      const int lz[2] = {bz >> 3, (bz + Fl::T - 1) >> 3};
      int64_t leaf[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const bool need = (dx == 0 || lx[1] != lx[0]) && (dy == 0 || ly[1] != ly[0]) &&
                          (dz == 0 || lz[1] != lz[0]);
        leaf[c] = need ? sparse_leaf(g, su, lx[dx] << 3, ly[dy] << 3, lz[dz] << 3) : -1;
      }
      acc = 0.0f;
#pragma unroll
      for (int kz = 0; kz < Fl::T; ++kz) {
        const int z = bz + kz, sz = (z >> 3) != lz[0];
#pragma unroll
        for (int ky = 0; ky < Fl::T; ++ky) {
          const int y = by + ky, sy = (y >> 3) != ly[0];
          const float wyz = wy[ky] * wz[kz];
#pragma unroll
          for (int kx = 0; kx < Fl::T; ++kx) {
            const int x = bx + kx, sx = (x >> 3) != lx[0];
            const float t = sparse_value<FMT>(g, leaf[(sz << 2) | (sy << 1) | sx], x, y, z);
            acc = fmaf(wx[kx] * wyz, t, acc);
          }
        }
      }
    }
    a.out[i] = acc;
  }
}

template <int F, int FMT, bool REUSE>
__global__ void __launch_bounds__(256) k_sparse_accumulate(SparseDev g, LookupArgs a) {
  __shared__ UpperSmem su;
  stage_upper(g, su);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double s = 0.0, s2 = 0.0;
    for (int k = 0; k < a.n_samples; ++k) {
      int4 tap;
      const double v = sparse_stochastic_one<F, FMT, REUSE>(g, su, a, i, i, a.sample_index + (uint32_t)k, tap);
      s += v;
      s2 += v * v;
    }
    a.sum[i] = s;
    a.sumsq[i] = s2;
  }
}

template <int F, int FMT>
static cudaError_t run_sparse(Op op, const SparseDev& g, const LookupArgs& a, cudaStream_t s) {
  const int threads = 256;
  // the four-query loop needs a quarter of the threads
  const int64_t units = (op == OP_STOCHASTIC && quad_loop3_ok(a)) ? (a.n + 3) / 4 : a.n;
  const int blocks = grid_blocks(units, threads, op == OP_STOCHASTIC ? kStochasticWaves : 4);
  if (op == OP_STOCHASTIC) {
    if constexpr (UsesReuse<F>::value) {
      if (a.reuse) k_sparse_stochastic<F, FMT, true><<<blocks, threads, 0, s>>>(g, a);
      else k_sparse_stochastic<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    } else {
      k_sparse_stochastic<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    }
  } else if (op == OP_DETERMINISTIC) {
    k_sparse_deterministic<F, FMT><<<blocks, threads, 0, s>>>(g, a);
  } else {
    if constexpr (UsesReuse<F>::value) {
      if (a.reuse) k_sparse_accumulate<F, FMT, true><<<blocks, threads, 0, s>>>(g, a);
      else k_sparse_accumulate<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    } else {
      k_sparse_accumulate<F, FMT, false><<<blocks, threads, 0, s>>>(g, a);
    }
  }
  return cudaGetLastError();
}

template <int F>
static cudaError_t run_sparse_f(Op op, int fmt, const SparseDev& g, const LookupArgs& a,
                                cudaStream_t s) {
  if (fmt == STF_FMT_F32) return run_sparse<F, STF_FMT_F32>(op, g, a, s);
  if (fmt == STF_FMT_E4M3_SCALED) return run_sparse<F, STF_FMT_E4M3_SCALED>(op, g, a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sparse3d(Op op, int filter, int fmt, const SparseDev& g, const LookupArgs& a,
                            cudaStream_t s) {
  switch (filter) {
    case STF_FILTER_LINEAR: return run_sparse_f<STF_FILTER_LINEAR>(op, fmt, g, a, s);
    case STF_FILTER_BSPLINE3: return run_sparse_f<STF_FILTER_BSPLINE3>(op, fmt, g, a, s);
    case STF_FILTER_CATMULL_ROM: return run_sparse_f<STF_FILTER_CATMULL_ROM>(op, fmt, g, a, s);
    case STF_FILTER_CATMULL_ROM_POSITIVIZED:
      return run_sparse_f<STF_FILTER_CATMULL_ROM_POSITIVIZED>(op, fmt, g, a, s);
    case STF_FILTER_FIS_LINEAR: return run_sparse_f<STF_FILTER_FIS_LINEAR>(op, fmt, g, a, s);
    case STF_FILTER_FIS_BSPLINE3: return run_sparse_f<STF_FILTER_FIS_BSPLINE3>(op, fmt, g, a, s);
    case STF_FILTER_FIS_GAUSSIAN: return run_sparse_f<STF_FILTER_FIS_GAUSSIAN>(op, fmt, g, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stf
