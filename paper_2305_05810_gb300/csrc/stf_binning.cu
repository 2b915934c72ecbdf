// Morton-tile binning of queries before a stochastic lookup.
//
// Queries are counting-sorted by the Morton code of the spatial tile that holds
// them, so that the threads of a warp (and the warps of a CTA) gather from nearby
// texels and the texel traffic hits L2.  The variates stay keyed on the caller's
// query index and results are written back to the caller's slots, so a binned call
// returns exactly what the unbinned call returns.
//
// Tiles: 3D cubes of 2^shift voxels, 8 per axis (512 bins, coordinates wrap),
// shift = max(3, ceil(log2(extent / 8))) for dense grids and 8 for sparse grids;
// 2D squares of 2^shift level-0 texels, 32 per axis (1024 bins),
// shift = max(2, ceil(log2(extent / 32))).  A tile's texels fit in L2, which is
// the locality binning is for; finer tiles only shorten the contiguous runs the
// placement pass writes.
//
// Counting sort in chunks of 4096 queries per CTA: keys are counted in shared
// memory with warp-aggregated atomics, and a global atomic is issued once per
// (chunk, bin) rather than per query, so hot bins do not serialise on one address.
//
// Scratch (histogram, cursors, permutation, binned coordinates) comes from a
// library-owned stream-ordered pool and is released on the same stream after the
// lookup, so concurrent binned calls on different streams do not share memory.
#include <mutex>

#include "stf_internal.h"

namespace stf {

static constexpr int kBins = 1024;
static constexpr int kChunk = 4096;
static constexpr int kBinThreads = 256;

__device__ __forceinline__ uint32_t spread3_3(uint32_t v) {  // 3 bits -> every third bit
  v &= 7u;
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}

__device__ __forceinline__ uint32_t spread2_5(uint32_t v) {  // 5 bits -> every second bit
  v &= 31u;
  v = (v | (v << 4)) & 0x10Fu;
  v = (v | (v << 2)) & 0x133u;
  v = (v | (v << 1)) & 0x155u;
  return v;
}

struct BinSpec {
  int dims;        // 2 or 3
  int shift;       // tile edge = 2^shift texels / voxels
  float scale_x;   // 2D: level-0 width and height
  float scale_y;
};

__device__ __forceinline__ int clamp_floor(float v) {
  return (int)floorf(fminf(fmaxf(v, -1.0e9f), 1.0e9f));   // NaN converts to 0
}

__device__ __forceinline__ uint32_t bin_key(const BinSpec& b, const float* coords, int64_t i) {
  if (b.dims == 2) {
    const float2 uv = reinterpret_cast<const float2*>(coords)[i];
    const int tx = clamp_floor(uv.x * b.scale_x) >> b.shift;
    const int ty = clamp_floor(uv.y * b.scale_y) >> b.shift;
    return spread2_5((uint32_t)tx) | (spread2_5((uint32_t)ty) << 1);
  }
  const float* p = coords + 3 * i;
  const int x = clamp_floor(__ldg(p)) >> b.shift;
  const int y = clamp_floor(__ldg(p + 1)) >> b.shift;
  const int z = clamp_floor(__ldg(p + 2)) >> b.shift;
  return spread3_3((uint32_t)x) | (spread3_3((uint32_t)y) << 1) | (spread3_3((uint32_t)z) << 2);
}

// Pass 1: per-chunk counts in shared memory, added to the global histogram.
__global__ void __launch_bounds__(kBinThreads) k_bin_count(BinSpec b, const float* coords,
                                                           int64_t n, uint32_t* hist) {
  __shared__ uint32_t cnt[kBins];
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < n; c0 += (int64_t)gridDim.x * kChunk) {
    for (int k = threadIdx.x; k < kBins; k += kBinThreads) cnt[k] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < kChunk; k += kBinThreads) {
      const int64_t i = c0 + k;
      const uint32_t key = i < n ? bin_key(b, coords, i) : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
      if (i < n && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + key, (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kBins; k += kBinThreads)
      if (cnt[k]) atomicAdd(hist + k, cnt[k]);
    __syncthreads();
  }
}

// Exclusive scan of nbins counts into cursors, one 1024-thread block.
__global__ void __launch_bounds__(1024) k_bin_scan(const uint32_t* hist, uint32_t* cursor,
                                                   int nbins) {
  __shared__ uint32_t part[1024];
  const int per = (nbins + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(lo + per, nbins);
  uint32_t s = 0;
  for (int k = lo; k < hi; ++k) s += hist[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {   // Hillis-Steele inclusive scan
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int k = lo; k < hi; ++k) {
    cursor[k] = run;
    run += hist[k];
  }
}

// Pass 2: local ranks in shared memory, one global reservation per (chunk, bin),
// then each query is written to its slot: perm[pos] = i and its coordinates (lod).
__global__ void __launch_bounds__(kBinThreads) k_bin_place(BinSpec b, const float* coords,
                                                           const float* lod, int64_t n,
                                                           uint32_t* cursor, uint32_t* perm,
                                                           float* coords_out, float* lod_out) {
  __shared__ uint32_t cnt[kBins];
  __shared__ uint32_t base[kBins];
  __shared__ uint16_t keys[kChunk];
  __shared__ uint16_t rank[kChunk];
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < n; c0 += (int64_t)gridDim.x * kChunk) {
    for (int k = threadIdx.x; k < kBins; k += kBinThreads) cnt[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < kChunk; k += kBinThreads) {
      const int64_t i = c0 + k;
      const uint32_t key = i < n ? bin_key(b, coords, i) : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
      const int leader = __ffs(peers) - 1;
      uint32_t first = 0;
      if (i < n && lane == leader) first = atomicAdd(cnt + key, (uint32_t)__popc(peers));
      first = __shfl_sync(0xFFFFFFFFu, first, leader);
      if (i < n) {
        keys[k] = (uint16_t)key;
        rank[k] = (uint16_t)(first + __popc(peers & ((1u << lane) - 1u)));
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kBins; k += kBinThreads)
      if (cnt[k]) base[k] = atomicAdd(cursor + k, cnt[k]);
    __syncthreads();
    for (int k = threadIdx.x; k < kChunk; k += kBinThreads) {
      const int64_t i = c0 + k;
      if (i >= n) continue;
      const uint32_t pos = base[keys[k]] + rank[k];
      perm[pos] = (uint32_t)i;
      if (b.dims == 2) {
        reinterpret_cast<float2*>(coords_out)[pos] = reinterpret_cast<const float2*>(coords)[i];
        if (lod) lod_out[pos] = lod[i];
      } else {
        coords_out[3 * (int64_t)pos] = coords[3 * i];
        coords_out[3 * (int64_t)pos + 1] = coords[3 * i + 1];
        coords_out[3 * (int64_t)pos + 2] = coords[3 * i + 2];
      }
    }
    __syncthreads();
  }
}

static int bin_blocks(int64_t n) {
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  const int64_t cap = (int64_t)grid_blocks(1LL << 40, kBinThreads);
  return (int)(chunks < cap ? (chunks < 1 ? 1 : chunks) : cap);
}

// Histogram, scan and placement on stream s with the given scratch pointers.
static cudaError_t bin_queries(const BinSpec& b, const float* coords, const float* lod, int64_t n,
                               uint32_t* hist, uint32_t* cursor, uint32_t* perm, float* bcoords,
                               float* blod, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kBins, s);   // counts start at zero
  if (e != cudaSuccess) return e;
  const int blocks = bin_blocks(n);
  k_bin_count<<<blocks, kBinThreads, 0, s>>>(b, coords, n, hist);
  k_bin_scan<<<1, 1024, 0, s>>>(hist, cursor, kBins);
  k_bin_place<<<blocks, kBinThreads, 0, s>>>(b, coords, lod, n, cursor, perm, bcoords, blod);
  return cudaGetLastError();
}

static std::mutex g_pool_mutex;
static cudaMemPool_t g_pool[64];

static cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pool[dev & 63]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pool[dev & 63], &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;   // keep freed blocks for reuse by later calls
      cudaMemPoolSetAttribute(g_pool[dev & 63], cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;   // the failure-injection hook
  return cudaMallocFromPoolAsync(p, bytes, g_pool[dev & 63], s);
}

BinSpec bin_spec(const stf_texture_s* t) {
  BinSpec b;
  b.dims = (t->kind == STF_KIND_TEX2D || t->kind == STF_KIND_NEURAL2D) ? 2 : 3;
  b.scale_x = (float)t->dims[0];
  b.scale_y = (float)t->dims[1];
  if (t->kind == STF_KIND_SPARSE3D) {
    b.shift = 8;
  } else if (b.dims == 2) {
    const int ext = t->dims[0] > t->dims[1] ? t->dims[0] : t->dims[1];
    int sh = 2;
    while ((ext >> sh) > 32) ++sh;
    b.shift = sh;
  } else {
    int ext = t->dims[0] > t->dims[1] ? t->dims[0] : t->dims[1];
    if (t->dims[2] > ext) ext = t->dims[2];
    int sh = 3;
    while ((ext >> sh) > 8) ++sh;
    b.shift = sh;
  }
  return b;
}

stf_status lookup_binned(stf_texture t, int filter, const LookupArgs& a0, cudaStream_t s) {
  const BinSpec b = bin_spec(t);
  const int64_t n = a0.n;
  if (n > (int64_t)UINT32_MAX) return fail(STF_ERR_INVALID_ARGUMENT, "binned calls take < 2^32 queries");
  const size_t b_hist = sizeof(uint32_t) * 2 * kBins;
  const size_t b_perm = (sizeof(uint32_t) * n + 255) & ~(size_t)255;
  const size_t b_coords = (sizeof(float) * b.dims * n + 255) & ~(size_t)255;
  const size_t b_lod = a0.lod ? sizeof(float) * n : 0;
  void* scratch = nullptr;
  cudaError_t e = pool_alloc(&scratch, b_hist + b_perm + b_coords + b_lod, s);
  if (e != cudaSuccess) return fail_cuda(e, "binning scratch");
  char* p = (char*)scratch;
  uint32_t* hist = (uint32_t*)p;
  uint32_t* cursor = hist + kBins;
  uint32_t* perm = (uint32_t*)(p + b_hist);
  float* coords = (float*)(p + b_hist + b_perm);
  float* lod = a0.lod ? (float*)(p + b_hist + b_perm + b_coords) : nullptr;
  e = bin_queries(b, a0.coords, a0.lod, n, hist, cursor, perm, coords, lod, s);
  stf_status st = STF_OK;
  if (e != cudaSuccess) {
    st = fail_cuda(e, "binning launch");
  } else {
    LookupArgs a = a0;
    a.coords = coords;
    a.lod = lod;
    a.perm = perm;
    st = dispatch(OP_STOCHASTIC, t, filter, a, s);
  }
  cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace stf

// ---------------------------------------------------------------- allocation-free variant
//
// stf_lookup_batch_binned_noalloc: the binned stochastic lookup above, with its
// scratch in a fixed device array that is part of the library image instead of
// the stream-ordered pool.  For callers that must not allocate device memory from
// inside the library: processes that reserve their whole device-memory budget up
// front with their own allocator (render engines, serving processes), where a
// library-side allocation could fail or fragment that budget, and callers that
// cannot afford the device-wide synchronisation cudaMalloc/cudaFree may imply.

namespace {

constexpr int64_t kNoAllocMaxQueries = STF_NOALLOC_MAX_QUERIES;
// [histogram | cursors] (2 x kBins = 2 x 1024 words) | permutation (max queries words) |
// binned coordinates, 3 floats per query for 3D, or 2 floats + lod for 2D.
constexpr size_t kNoAllocHistBytes = sizeof(uint32_t) * 2 * stf::kBins;
constexpr size_t kNoAllocPermBytes = sizeof(uint32_t) * kNoAllocMaxQueries;
constexpr size_t kNoAllocCoordBytes = sizeof(float) * 3 * kNoAllocMaxQueries;
constexpr size_t kNoAllocBytes = kNoAllocHistBytes + kNoAllocPermBytes + kNoAllocCoordBytes;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64];   // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device (looked up once per
// device; the host-side name of the array is not a device address).
stf_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return stf::fail_cuda(e, "current device");
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev & 63]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return stf::fail_cuda(e, "static scratch address");
    g_noalloc_ptr[dev & 63] = p;
  }
  *out = g_noalloc_ptr[dev & 63];
  return STF_OK;
}

}  // namespace

extern "C" stf_status stf_lookup_batch_binned_noalloc(stf_texture t, const stf_lookup_params* p,
                                                      const float* coords, const float* lod,
                                                      int64_t n, float* out, int32_t* taps,
                                                      void* stream) {
  using namespace stf;
  stf_status st = check_lookup(t, p, coords, lod, n, out);
  if (st != STF_OK || n == 0) return st;
  if (n > kNoAllocMaxQueries)
    return fail(STF_ERR_INVALID_ARGUMENT,
                "n = %lld exceeds the allocation-free limit of %lld queries per call",
                (long long)n, (long long)kNoAllocMaxQueries);
  if (taps && (uintptr_t)taps % 16) return fail(STF_ERR_INVALID_ARGUMENT, "taps not 16-byte aligned");
  void* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != STF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const BinSpec b = bin_spec(t);
  char* base = (char*)scratch;
  uint32_t* hist = (uint32_t*)base;
  uint32_t* cursor = hist + kBins;
  uint32_t* perm = (uint32_t*)(base + kNoAllocHistBytes);
  float* bcoords = (float*)(base + kNoAllocHistBytes + kNoAllocPermBytes);
  float* blod = (b.dims == 2 && lod) ? bcoords + 2 * kNoAllocMaxQueries : nullptr;
  const cudaError_t e = bin_queries(b, coords, lod, n, hist, cursor, perm, bcoords, blod, s);
  if (e != cudaSuccess) return fail_cuda(e, "binning launch");
  LookupArgs a = make_args(p, bcoords, blod, n, out, taps);
  a.perm = perm;
  return dispatch(OP_STOCHASTIC, t, p->filter, a, s);
}
