// DCT-compressed 2D textures (Section 5.2, "Texture compression"): the lookup kernels
// of stf_tex2d.cuh instantiated for the DCT6 format (texels decoded where fetched),
// and the create-time encoder.
//
// Encoding, per level, 8x8 block and channel (float64): the six coefficients with
// u + v <= 2 of the orthonormal 8-point DCT-II, F(u, v) = a(u) a(v) sum_{x,y} f(x, y)
// cos((2x+1) u pi/16) cos((2y+1) v pi/16), a(0) = sqrt(1/8), a(k) = 1/2, over the block's
// texels (edge texels repeated past the level's edge).  DC code round(DC 127 / 8) in
// [0, 127]; AC code round(AC 15 / R_c) in [-15, 15], R_c = the channel's largest |AC|
// over the pyramid (0 below 2^-20); rounding half away from zero; 7 + 5 x 5 bits.
#include <cmath>
#include <vector>

#include "stf_tex2d.cuh"

namespace stf {

cudaError_t launch_tex2d_dct(Op op, int filter, int channels, const Tex2DView& t, const LookupArgs& a,
                             cudaStream_t s) {
  return launch_tex2d_format<STF_FMT_DCT6>(op, filter, channels, t, a, s);
}

struct DctPyramid {
  const float* src;                       // float32 levels, [y][x][c]
  int64_t level_off[STF_MAX_LEVELS];      // texels
  int64_t code_off[STF_MAX_LEVELS];       // code words
  int64_t block_base[STF_MAX_LEVELS + 1]; // first global block index of each level
  int32_t w[STF_MAX_LEVELS], h[STF_MAX_LEVELS], bw[STF_MAX_LEVELS];
  int32_t levels, C;
};

__device__ constexpr int kDctKept[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};

__device__ __forceinline__ double dct_basis64(int u, int x) {
  return u == 0 ? sqrt(0.125) : 0.5 * cospi((double)((2 * x + 1) * u) / 16.0);
}

// Block b (global index) of its level: level, block row and column.
__device__ __forceinline__ int dct_locate(const DctPyramid& P, int64_t b, int& by, int& bx) {
  int L = 0;
  while (L + 1 < P.levels && b >= P.block_base[L + 1]) ++L;
  const int64_t k = b - P.block_base[L];
  by = (int)(k / P.bw[L]);
  bx = (int)(k % P.bw[L]);
  return L;
}

// Coefficients (float64) of every (block, channel) and the channel ranges, as the
// order-preserving bit patterns of non-negative doubles (atomicMax).
__global__ void k_dct_forward(DctPyramid P, double* coef, unsigned long long* range_bits) {
  const int64_t total = P.block_base[P.levels] * P.C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int c = (int)(i % P.C);
    int by, bx;
    const int L = dct_locate(P, i / P.C, by, bx);
    double rows[3][8];                          // sum over x of f(x, y) c_u(x), per row y
    for (int y = 0; y < 8; ++y) {
      const int yy = min(by * 8 + y, P.h[L] - 1);
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int x = 0; x < 8; ++x) {
        const int xx = min(bx * 8 + x, P.w[L] - 1);
        const double f = (double)P.src[(P.level_off[L] + (int64_t)yy * P.w[L] + xx) * P.C + c];
        s0 = fma(f, dct_basis64(0, x), s0);
        s1 = fma(f, dct_basis64(1, x), s1);
        s2 = fma(f, dct_basis64(2, x), s2);
      }
      rows[0][y] = s0;
      rows[1][y] = s1;
      rows[2][y] = s2;
    }
    double amax = 0.0;
    for (int k = 0; k < 6; ++k) {
      const int u = kDctKept[k][0], v = kDctKept[k][1];
      double F = 0.0;
      for (int y = 0; y < 8; ++y) F = fma(rows[u][y], dct_basis64(v, y), F);
      coef[i * 6 + k] = F;
      if (k > 0) amax = fmax(amax, fabs(F));
    }
    atomicMax(range_bits + c, (unsigned long long)__double_as_longlong(amax));
  }
}

__device__ __forceinline__ double round_half_away(double x) { return copysign(floor(fabs(x) + 0.5), x); }

__global__ void k_dct_pack(DctPyramid P, const double* coef, const unsigned long long* range_bits,
                           uint32_t* dst) {
  const int64_t total = P.block_base[P.levels] * P.C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int c = (int)(i % P.C);
    int by, bx;
    const int L = dct_locate(P, i / P.C, by, bx);
    double R = __longlong_as_double((long long)range_bits[c]);
    if (R < 0x1p-20) R = 0.0;
    const double dc = fmin(fmax(round_half_away(coef[i * 6] * 127.0 / 8.0), 0.0), 127.0);
    uint32_t w = (uint32_t)dc;
    for (int j = 0; j < 5; ++j) {
      const double q = R > 0.0 ? fmin(fmax(round_half_away(coef[i * 6 + 1 + j] * 15.0 / R), -15.0), 15.0) : 0.0;
      w |= ((uint32_t)((int)q & 31)) << (7 + 5 * j);
    }
    dst[P.code_off[L] + ((int64_t)by * P.bw[L] + bx) * P.C + c] = w;
  }
}

cudaError_t launch_dct_encode(const float* src, const int64_t* level_off, const int32_t* w,
                              const int32_t* h, int levels, int C, uint32_t* dst,
                              const int64_t* code_off, double* scratch, double* h_range,
                              cudaStream_t s) {
  DctPyramid P;
  memset(&P, 0, sizeof(P));
  P.src = src;
  P.levels = levels;
  P.C = C;
  int64_t nb = 0;
  for (int L = 0; L < levels; ++L) {
    P.level_off[L] = level_off[L];
    P.code_off[L] = code_off[L];
    P.w[L] = w[L];
    P.h[L] = h[L];
    P.bw[L] = (w[L] + 7) / 8;
    P.block_base[L] = nb;
    nb += (int64_t)P.bw[L] * ((h[L] + 7) / 8);
  }
  P.block_base[levels] = nb;
  double* coef = scratch;
  unsigned long long* range_bits = reinterpret_cast<unsigned long long*>(scratch + nb * C * 6);
  cudaError_t e = cudaMemsetAsync(range_bits, 0, sizeof(unsigned long long) * C, s);
  if (e != cudaSuccess) return e;
  const int blocks = grid_blocks(nb * C, 128);
  k_dct_forward<<<blocks, 128, 0, s>>>(P, coef, range_bits);
  k_dct_pack<<<blocks, 128, 0, s>>>(P, coef, range_bits, dst);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  std::vector<unsigned long long> bits(C);
  e = cudaMemcpyAsync(bits.data(), range_bits, sizeof(unsigned long long) * C, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < C; ++c) {
    double r;
    memcpy(&r, &bits[c], sizeof(r));
    h_range[c] = r < 0x1p-20 ? 0.0 : r;
  }
  return cudaSuccess;
}

}  // namespace stf
