// Neural textures: latent MIP levels decoded by an 8 -> 64 -> 64 -> 7 ReLU MLP on
// the tensor cores (mma.sync m16n8k16, binary16 operands, float32 accumulation).
//
// The paper motivates stochastic filtering for decoders that are expensive to run
// per texel, neural texture representations among them (Section 1; Section 5.2,
// "Texture compression"): the stochastic lookup picks one latent texel with the same
// inverse-CDF tap choice as a plain 2D texture and decodes it once; the
// deterministic lookup decodes every tap and filters the decoded values.
//
// MMA data flow: a warp owns 16-row tiles (queries or training texels).  The float32
// accumulator fragment of two adjacent 8-column output tiles has exactly the
// register layout of a 16-wide binary16 A fragment, so each layer's ReLU output is
// packed in registers and fed to the next layer without a trip through shared
// memory.  Weight B fragments are read from shared-memory images laid out so that
// every fragment register is one aligned 32-bit word (rows padded to avoid bank
// conflicts).  The weight gradients H^T G reduce over the batch, which is the K
// dimension of that product; their fragments come from row-major activation tiles
// through ldmatrix.trans.
#include <cstddef>
#include <math.h>

#include "stf_internal.h"

namespace stf {

namespace nn {

constexpr int P_W1 = 0, P_B1 = 512, P_W2 = 576, P_B2 = 4672, P_W3 = 4736, P_B3 = 5184;
constexpr int NPARAM = STF_NEURAL_PARAMS;
static_assert(NPARAM == 5191, "parameter count");

// binary16 weight images (halves): w1t[64][24] = W1^T (k >= 8 zero), w2t[64][72] = W2^T,
// w3t[8][72] = W3^T (row 7 zero); backward: w2r[64][72] = W2, w3r[64][8] = W3 (col 7
// zero), w1r[8][72] = W1.
constexpr int I_W1T = 0, I_W2T = 1536, I_W3T = 6144, I_W2R = 6720, I_W3R = 11328, I_W1R = 11840;
constexpr int IMG_FWD = 6720, IMG_ALL = 12416;
constexpr int NBIAS = 136;   // b1[64], b2[64], b3[8] (b3[7] = 0)
constexpr int S24 = 12, S72 = 36, S8 = 4;   // row strides in 32-bit words

}  // namespace nn

// ---------------------------------------------------------------- MMA helpers

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float2 unpack_h2(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x2_trans(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}

// Copy the weight images and biases into shared memory (whole CTA).
__device__ __forceinline__ void stage_weights(const NeuralDev& nd, uint32_t* sW, float* sB, int words) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(nd.wimg);
  for (int k = threadIdx.x; k < words; k += blockDim.x) sW[k] = __ldg(src + k);
  for (int k = threadIdx.x; k < nn::NBIAS; k += blockDim.x) sB[k] = __ldg(nd.bias + k);
  __syncthreads();
}

// Forward pass of MT 16-row tiles.  sA: the warp's 32 input rows, 4 words (8 halves)
// per row; rows 16*mt .. 16*mt + 15 form tile mt.  Y rows go to sY (8 floats per
// row, column 7 is padding).  When H1/H2 pointers are given the tiles' hidden
// activations (binary16) are kept for the caller in a2/a3.
template <int MT>
__device__ __forceinline__ void mlp_forward(const uint32_t* sW, const float* sB, const uint32_t* sA,
                                            int row0, float (*sY)[8], uint32_t (*a2)[4][4],
                                            uint32_t (*a3)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a1[MT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    a1[m][0] = sA[(row0 + 16 * m + g) * 4 + t];
    a1[m][1] = sA[(row0 + 16 * m + g + 8) * 4 + t];
    a1[m][2] = 0u;
    a1[m][3] = 0u;
  }
  const uint32_t* w1t = sW + nn::I_W1T / 2;
  const uint32_t* w2t = sW + nn::I_W2T / 2;
  const uint32_t* w3t = sW + nn::I_W3T / 2;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t b0 = w1t[(8 * j + g) * nn::S24 + t];
    const float bl = sB[8 * j + 2 * t], bh = sB[8 * j + 2 * t + 1];
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      float c[4] = {bl, bh, bl, bh};
      mma16816(c, a1[m], b0, 0u);
      a2[m][j >> 1][(j & 1) * 2 + 0] = pack_h2(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f));
      a2[m][j >> 1][(j & 1) * 2 + 1] = pack_h2(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f));
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = sB[64 + 8 * j + 2 * t], bh = sB[64 + 8 * j + 2 * t + 1];
    float c[MT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      c[m][0] = bl; c[m][1] = bh; c[m][2] = bl; c[m][3] = bh;
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const uint32_t b0 = w2t[(8 * j + g) * nn::S72 + 8 * kc + t];
      const uint32_t b1 = w2t[(8 * j + g) * nn::S72 + 8 * kc + 4 + t];
#pragma unroll
      for (int m = 0; m < MT; ++m) mma16816(c[m], a2[m][kc], b0, b1);
    }
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      a3[m][j >> 1][(j & 1) * 2 + 0] = pack_h2(fmaxf(c[m][0], 0.f), fmaxf(c[m][1], 0.f));
      a3[m][j >> 1][(j & 1) * 2 + 1] = pack_h2(fmaxf(c[m][2], 0.f), fmaxf(c[m][3], 0.f));
    }
  }
  float c[MT][4];
  const float bl = sB[128 + 2 * t], bh = sB[128 + 2 * t + 1];
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    c[m][0] = bl; c[m][1] = bh; c[m][2] = bl; c[m][3] = bh;
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    const uint32_t b0 = w3t[g * nn::S72 + 8 * kc + t];
    const uint32_t b1 = w3t[g * nn::S72 + 8 * kc + 4 + t];
#pragma unroll
    for (int m = 0; m < MT; ++m) mma16816(c[m], a3[m][kc], b0, b1);
  }
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    sY[row0 + 16 * m + g][2 * t] = c[m][0];
    sY[row0 + 16 * m + g][2 * t + 1] = c[m][1];
    sY[row0 + 16 * m + g + 8][2 * t] = c[m][2];
    sY[row0 + 16 * m + g + 8][2 * t + 1] = c[m][3];
  }
}

// ---------------------------------------------------------------- lookups

// Level of texel storage: returns a pointer to 8 binary16 values of texel (x, y) at
// level L (latent or fallback; clamp-to-edge).
__device__ __forceinline__ uint4 neural_texel(const NeuralDev& nd, int L, int x, int y) {
  const int w = nd.lvl_w[L], h = nd.lvl_h[L];
  const int cx = min(max(x, 0), w - 1), cy = min(max(y, 0), h - 1);
  const __half* base = L < nd.nlat ? nd.lat16 : nd.fb16;
  return __ldg(reinterpret_cast<const uint4*>(base + (nd.lvl_off[L] + (int64_t)cy * w + cx) * 8));
}

struct NeuralSmem {
  uint32_t w[nn::IMG_ALL / 2];
  float b[nn::NBIAS];
  uint32_t a[4][32 * 4];   // per warp: 32 rows x 8 halves
  float y[4][32][8];       // per warp: 32 rows x 8 floats
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Per-lane state of one 32-query chunk between tap choice and output.
struct NeuralPick {
  int64_t j;      // caller's query slot
  float sigma;    // estimator scale (Catmull-Rom)
  int4 tap;
  int mode;       // 0: no texel (background), 1: decode the latent, 2: stored fallback texel
};

// Tap choice for query i of the chunk; starts the 16-byte gather of the chosen texel
// (latent or fallback) into the lane's shared-memory row.
template <int F>
__device__ __forceinline__ NeuralPick neural_pick(const NeuralDev& nd, const LookupArgs& a, int64_t i,
                                                  uint4* row) {
  NeuralPick pk;
  pk.j = 0;
  pk.sigma = 1.0f;
  pk.tap = make_int4(0, 0, 0, -1);
  pk.mode = 0;
  if (i >= a.n) return pk;
  pk.j = query_slot(a, i);
  const float2 uv = reinterpret_cast<const float2*>(a.coords)[i];
  const float lod = a.lod ? a.lod[i] : 0.0f;
  const uint4 r = query_variates(a, pk.j, a.sample_index);
  int L = 0;
  if (a.lod != nullptr && nd.nlev > 1) {
    const float lc = fminf(fmaxf(lod, 0.0f), (float)(nd.nlev - 1));
    L = min((int)floorf(__fadd_rn(lc, a.level_mode == STF_LEVEL_NEAREST ? 0.5f : unit24(r.w))), nd.nlev - 1);
  }
  const int w = nd.lvl_w[L], h = nd.lvl_h[L];
  float x[2] = {__fsub_rn(__fmul_rn(uv.x, (float)w), 0.5f), __fsub_rn(__fmul_rn(uv.y, (float)h), 0.5f)};
  if (!(prepare_coords<2>(x) && isfinite(lod))) return pk;
  int idx[2];
  pk.sigma = pick_taps_r<F, 2, false>(x, r, idx);
  pk.tap = make_int4(idx[0], idx[1], 0, L);
  const int cx = min(max(idx[0], 0), w - 1), cy = min(max(idx[1], 0), h - 1);
  const __half* base = L < nd.nlat ? nd.lat16 : nd.fb16;
  cp_async16(row, base + (nd.lvl_off[L] + (int64_t)cy * w + cx) * 8);
  pk.mode = L < nd.nlat ? 1 : 2;
  return pk;
}

// ---------------------------------------------------------------- tcgen05 decode
//
// The stochastic decode on the fifth-generation tensor cores: for a tile of 128
// queries (one per thread) the chosen latent texels are gathered into a shared-memory
// A tile; one elected thread issues the three layers as tcgen05.mma (M = 128, binary16
// operands from shared memory, float32 accumulators in tensor memory); after each
// layer every thread loads its own accumulator row with tcgen05.ld, adds the bias,
// applies ReLU, rounds to binary16 and writes the next layer's A tile.  Operand tiles
// use the no-swizzle K-major layout: 8-row x 16-byte core matrices, core matrices
// along K 128 bytes apart (LBO), 8-row groups K/8 * 128 bytes apart (SBO).

namespace tc {

constexpr int ROWS = 128;            // queries per tile = threads per group
constexpr int TMEM_COLS = 128;       // 64 columns per group: D1/D2 in 0..63, D3 in 0..15
constexpr int A1_BYTES = ROWS * 16 * 2, A2_BYTES = ROWS * 64 * 2;
constexpr int B1_BYTES = 64 * 16 * 2, B2_BYTES = 64 * 64 * 2, B3_BYTES = 16 * 64 * 2;

// byte offset of element (r, k) in an R x K tile (K = 16 or 64)
__host__ __device__ constexpr int off(int r, int k, int K) {
  return (r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t desc(const void* p, int K) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;                 // LBO: next core matrix along K
  d |= (uint64_t)(((K / 8) * 128) >> 4) << 32;     // SBO: next 8-row group
  d |= (uint64_t)1 << 46;                           // descriptor version; no swizzle
  return d;
}

// The same with the 8-row-group stride set to 0: every group of 8 rows reads the same
// two core matrices, so one 8-row tile stands for a 128-row operand whose rows are
// all equal.
__device__ __forceinline__ uint64_t desc_rows_repeated(const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: F32 accumulate, F16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      (uint32_t)__cvta_generic_to_shared(bar)));
}

// Wait for phase `parity` of the mbarrier; false on timeout.  Each try_wait may suspend
// the thread for up to 20 us, waking it when the phase completes, so the waiting lane
// does not spin on the issue slots its warp shares with the computing warps; at most
// 2^16 tries (about 1.3 s).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  uint32_t done = 0;
  for (int it = 0; it < (1 << 16) && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(a), "r"(parity), "r"(20000u));
  }
  return done != 0;
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* r);

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

struct Group {                       // one tile in flight
  unsigned char a1[A1_BYTES];
  unsigned char a2[A2_BYTES];          // H1, then H2, then the staged output rows
  uint64_t bar;
  int abort;
};

struct Smem {
  unsigned char b1[B1_BYTES];          // W1^T in k 0..7, (b1_hi, b1_lo) in k 8, 9
  unsigned char b2[B2_BYTES];
  unsigned char b3[B3_BYTES];
  unsigned char b2x[64 * 16 * 2];      // (b2_hi, b2_lo) in k 0, 1
  unsigned char b3x[16 * 16 * 2];      // (b3_hi, b3_lo) in k 0, 1
  unsigned char ones[8 * 16 * 2];      // one 8-row group: 1 in columns 0, 1
  Group grp[2];
  uint32_t tmem;
};
// A2 doubles as the 16-byte-aligned staging area of the output rows
static_assert(offsetof(Smem, grp) % 16 == 0 && offsetof(Group, a2) % 16 == 0 && sizeof(Group) % 16 == 0,
              "A2 tiles are 16-byte aligned");

}  // namespace tc

// Hidden layer epilogue: D (64 float32 per row, tensor memory, bias included by the
// MMA) -> ReLU -> binary16 row of the next A tile.
__device__ __forceinline__ void tc_hidden(uint32_t taddr, unsigned char* a2, int row) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t r[32];
    tc::tmem_ld<32>(taddr + 32 * half, r);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = 8 * q + 2 * e;
        const float lo = __uint_as_float(r[c]);
        const float hi = __uint_as_float(r[c + 1]);
        // ReLU and round to binary16 in one instruction (the first source goes to the
        // upper half)
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(w[e]) : "f"(hi), "f"(lo));
      }
      *reinterpret_cast<uint4*>(a2 + tc::off(row, 32 * half + 8 * q, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Named barrier of one 128-thread group.
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

// Two groups of 128 threads per CTA decode two tiles concurrently: each group owns an
// A1/A2 tile pair, 64 tensor-memory columns (D1, D2, then D3 over the first 16 once D2
// has been read), an mbarrier and a named barrier, and walks its own tile sequence;
// while one group waits on its MMAs or its gathers the other computes.  The weights
// are shared.  A group's A1 is refilled with the next tile's gather as soon as layer 1
// has consumed it.
template <int F>
__global__ void __launch_bounds__(256, 4) k_neural_stochastic_tc(NeuralDev nd, LookupArgs a) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  tc::Smem& s = *reinterpret_cast<tc::Smem*>(dyn);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid >> 7, row = tid & 127;          // group, row of the group's tile
  tc::Group& G = s.grp[g];
  // weights: binary16 images -> K-major no-swizzle B tiles (16-byte rows)
  {
    const uint4* img = reinterpret_cast<const uint4*>(nd.wimg);
    // Biases enter the MMAs as an extra K chunk: a bias b is split into binary16
    // b_hi = fp16(b) and b_lo = fp16(b - b_hi), multiplied by two columns of ones, so
    // the float32 accumulator receives b to about 2^-22 |b|.
    auto split = [](float b) -> uint32_t {
      const __half hi = __float2half_rn(b);
      const __half lo = __float2half_rn(b - __half2float(hi));
      return (uint32_t)__half_as_ushort(hi) | ((uint32_t)__half_as_ushort(lo) << 16);
    };
    for (int n = tid; n < 64; n += 256) {             // W1^T: n < 64, k 0..7; bias in k 8, 9
      *reinterpret_cast<uint4*>(s.b1 + tc::off(n, 0, 16)) = __ldg(img + (nn::I_W1T + n * 24) / 8);
      *reinterpret_cast<uint4*>(s.b1 + tc::off(n, 8, 16)) = make_uint4(split(__ldg(nd.bias + n)), 0, 0, 0);
      *reinterpret_cast<uint4*>(s.b2x + tc::off(n, 0, 16)) = make_uint4(split(__ldg(nd.bias + 64 + n)), 0, 0, 0);
      *reinterpret_cast<uint4*>(s.b2x + tc::off(n, 8, 16)) = make_uint4(0, 0, 0, 0);
    }
    for (int n = tid; n < 16; n += 256) {
      const uint32_t b = n < 7 ? split(__ldg(nd.bias + 128 + n)) : 0u;
      *reinterpret_cast<uint4*>(s.b3x + tc::off(n, 0, 16)) = make_uint4(b, 0, 0, 0);
      *reinterpret_cast<uint4*>(s.b3x + tc::off(n, 8, 16)) = make_uint4(0, 0, 0, 0);
    }
    for (int r = tid; r < 8; r += 256) {
      *reinterpret_cast<uint4*>(s.ones + tc::off(r, 0, 16)) = make_uint4(0x3C003C00u, 0, 0, 0);
      *reinterpret_cast<uint4*>(s.ones + tc::off(r, 8, 16)) = make_uint4(0, 0, 0, 0);
    }
    for (int e = tid; e < 64 * 8; e += 256) {        // W2^T: n < 64, k chunks of 8 (< 64)
      const int n = e >> 3, kc = e & 7;
      *reinterpret_cast<uint4*>(s.b2 + tc::off(n, 8 * kc, 64)) = __ldg(img + (nn::I_W2T + n * 72 + 8 * kc) / 8);
    }
    for (int e = tid; e < 16 * 8; e += 256) {        // W3^T: n < 16 (rows >= 8 zero)
      const int n = e >> 3, kc = e & 7;
      *reinterpret_cast<uint4*>(s.b3 + tc::off(n, 8 * kc, 64)) =
          n < 8 ? __ldg(img + (nn::I_W3T + n * 72 + 8 * kc) / 8) : make_uint4(0, 0, 0, 0);
    }
    // columns 8..15 of A1: the ones that multiply W1's bias rows, then zeros (the
    // gathers write columns 0..7 only)
    *reinterpret_cast<uint4*>(G.a1 + tc::off(row, 8, 16)) = make_uint4(0x3C003C00u, 0, 0, 0);
  }
  if (row == 0) {
    G.abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&G.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&s.tmem)), "n"(tc::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s.tmem + 64 * g;                          // this group's columns
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
  uint32_t parity = 0;
  const int64_t ntiles = (a.n + tc::ROWS - 1) / tc::ROWS;
  const int64_t step = 2 * (int64_t)gridDim.x;
  int64_t tile = 2 * (int64_t)blockIdx.x + g;
  uint4* arow = reinterpret_cast<uint4*>(G.a1 + tc::off(row, 0, 16));
  NeuralPick cur;
  if (tile < ntiles) cur = neural_pick<F>(nd, a, tile * tc::ROWS + row, arow);
  cp_async_commit();
  for (; tile < ntiles; tile += step) {
    cp_async_wait<0>();
    uint4 fb = make_uint4(0, 0, 0, 0);
    if (cur.mode == 2) fb = *arow;                   // stored fallback texel (own row)
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    group_sync(g);
    // layer 1: D[0, 64) = A1 (128 x 16) * W1 (16 x 64); one thread issues and waits
    if (row == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      tc::mma(tmem, tc::desc(G.a1, 16), tc::desc(s.b1, 16), tc::idesc(128, 64), 0);
      tc::commit(&G.bar);
      if (!tc::wait_bar(&G.bar, parity)) G.abort = 1;
    }
    parity ^= 1;
    group_sync(g);
    if (G.abort) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // A1 is free: start the next tile's gather
    const int64_t next = tile + step;
    NeuralPick nxt;
    if (next < ntiles) nxt = neural_pick<F>(nd, a, next * tc::ROWS + row, arow);
    cp_async_commit();
    tc_hidden(trow, G.a2, row);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    group_sync(g);
    // layer 2: D[0, 64) = H1 (128 x 64) * W2 (64 x 64)
    if (row == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma(tmem, tc::desc(G.a2 + kk * 256, 64), tc::desc(s.b2 + kk * 256, 64), tc::idesc(128, 64), kk);
      tc::mma(tmem, tc::desc_rows_repeated(s.ones), tc::desc(s.b2x, 16), tc::idesc(128, 64), 1);   // + b2
      tc::commit(&G.bar);
      if (!tc::wait_bar(&G.bar, parity)) G.abort = 1;
    }
    parity ^= 1;
    group_sync(g);
    if (G.abort) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    tc_hidden(trow, G.a2, row);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    group_sync(g);
    // layer 3: D[0, 16) = H2 (128 x 64) * W3 (64 x 16); D2 has been read
    if (row == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma(tmem, tc::desc(G.a2 + kk * 256, 64), tc::desc(s.b3 + kk * 256, 64), tc::idesc(128, 16), kk);
      tc::mma(tmem, tc::desc_rows_repeated(s.ones), tc::desc(s.b3x, 16), tc::idesc(128, 16), 1);   // + b3
      tc::commit(&G.bar);
      if (!tc::wait_bar(&G.bar, parity)) G.abort = 1;
    }
    parity ^= 1;
    group_sync(g);
    if (G.abort) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float v[8];
    {
      uint32_t r[8];
      tc::tmem_ld<8>(trow, r);
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] = __uint_as_float(r[k]);
    }
    if (cur.mode == 2) {
      const uint32_t* tw = reinterpret_cast<const uint32_t*>(&fb);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = unpack_h2(tw[k]);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
      }
    } else if (cur.mode == 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] *= cur.sigma;
    const int64_t i = tile * tc::ROWS + row;
    const bool live = i < a.n;
    if (a.perm == nullptr) {
      // stage the tile's rows in A2 (free now) and store them coalesced
      float* stage = reinterpret_cast<float*>(G.a2);
#pragma unroll
      for (int k = 0; k < 7; ++k) stage[row * 7 + k] = v[k];
      group_sync(g);
      const int nrows = (int)min((int64_t)tc::ROWS, a.n - tile * tc::ROWS);
      float* dst = a.out + tile * tc::ROWS * 7;
      if (nrows == tc::ROWS && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        // a full tile: 896 floats as 224 16-byte copies
        const float4* src4 = reinterpret_cast<const float4*>(stage);
        float4* dst4 = reinterpret_cast<float4*>(dst);
        for (int e = row; e < tc::ROWS * 7 / 4; e += 128) dst4[e] = src4[e];
      } else {
        for (int e = row; e < nrows * 7; e += 128) dst[e] = stage[e];
      }
    } else if (live) {
#pragma unroll
      for (int k = 0; k < 7; ++k) a.out[cur.j * 7 + k] = v[k];
    }
    if (live && a.taps) reinterpret_cast<int4*>(a.taps)[cur.j] = cur.tap;
    cur = nxt;
    // the next iteration's first group barrier orders these reads of A2 before the
    // next tile writes it
  }
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (row == 0 && G.abort) atomicOr(nd.status, STF_DEV_MMA_TIMEOUT);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "n"(tc::TMEM_COLS));
}

// Deterministic: every tap of the filter window (at one level, or two blended by
// frac(lod)) is decoded and the decoded values are weighted and summed.
template <int F>
__global__ void __launch_bounds__(128) k_neural_deterministic(NeuralDev nd, LookupArgs a) {
  using Fl = Filter<F>;
  __shared__ __align__(16) NeuralSmem s;
  stage_weights(nd, s.w, s.b, nn::IMG_FWD / 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t a2[2][4][4], a3[2][4][4];
  const int64_t nwarps = (int64_t)gridDim.x * 4;
  for (int64_t c = (int64_t)blockIdx.x * 4 + warp; c * 32 < a.n; c += nwarps) {
    const int64_t i = c * 32 + lane;
    const bool live = i < a.n;
    float acc[7] = {0, 0, 0, 0, 0, 0, 0};
    int lv[2] = {0, 0};
    float lw[2] = {0.0f, 0.0f};
    float2 uv = make_float2(0.f, 0.f);
    if (live) {
      uv = reinterpret_cast<const float2*>(a.coords)[i];
      const float lod = a.lod ? a.lod[i] : 0.0f;
      if (isfinite(lod) && isfinite(uv.x) && isfinite(uv.y)) {
        lw[0] = 1.0f;
        if (a.lod != nullptr && nd.nlev > 1) {
          const float lc = fminf(fmaxf(lod, 0.0f), (float)(nd.nlev - 1));
          if (a.level_mode == STF_LEVEL_NEAREST) {
            lv[0] = min((int)floorf(__fadd_rn(lc, 0.5f)), nd.nlev - 1);
          } else {
            const float fl = floorf(lc), fr = __fsub_rn(lc, fl);
            lv[0] = (int)fl;
            lv[1] = min(lv[0] + 1, nd.nlev - 1);
            lw[0] = 1.0f - fr;
            lw[1] = fr;
          }
        }
      }
    }
#pragma unroll 1
    for (int p = 0; p < 2; ++p) {
      if (!__any_sync(0xffffffffu, lw[p] > 0.0f)) continue;
      const int L = lv[p];
      float x[2] = {__fsub_rn(__fmul_rn(uv.x, (float)nd.lvl_w[L]), 0.5f),
                    __fsub_rn(__fmul_rn(uv.y, (float)nd.lvl_h[L]), 0.5f)};
      const bool ok = lw[p] > 0.0f && prepare_coords<2>(x);
      float fx = 0.f, fy = 0.f;
      int bx = 0, by = 0;
      if (ok) {
        bx = axis_base(x[0], fx) + Fl::OFF0;
        by = axis_base(x[1], fy) + Fl::OFF0;
      }
      float wx[Fl::T], wy[Fl::T];
      Fl::weights(fx, wx);
      Fl::weights(fy, wy);
#pragma unroll 1
      for (int ty = 0; ty < Fl::T; ++ty) {
#pragma unroll 1
        for (int tx = 0; tx < Fl::T; ++tx) {
          const float w = ok ? wx[tx] * wy[ty] * lw[p] : 0.0f;
          uint4 texel = make_uint4(0, 0, 0, 0);
          if (ok) texel = neural_texel(nd, L, bx + tx, by + ty);
          const bool decode = ok && L < nd.nlat;
          reinterpret_cast<uint4*>(s.a[warp])[lane] = decode ? texel : make_uint4(0, 0, 0, 0);
          __syncwarp();
          mlp_forward<2>(s.w, s.b, s.a[warp], 0, s.y[warp], a2, a3);
          __syncwarp();
          if (decode) {
#pragma unroll
            for (int k = 0; k < 7; ++k) acc[k] = fmaf(w, s.y[warp][lane][k], acc[k]);
          } else if (ok) {
            const uint32_t* tw = reinterpret_cast<const uint32_t*>(&texel);
#pragma unroll
            for (int k = 0; k < 7; ++k) {
              const float2 f = unpack_h2(tw[k >> 1]);
              acc[k] = fmaf(w, (k & 1) ? f.y : f.x, acc[k]);
            }
          }
          __syncwarp();
        }
      }
    }
    if (live) {
#pragma unroll
      for (int k = 0; k < 7; ++k) a.out[i * 7 + k] = acc[k];
    }
  }
}

// ---------------------------------------------------------------- training

struct ActBuffers {   // binary16 activations of one batch, row-major
  __half* x;    // [B][8]
  __half* h1;   // [B][64]
  __half* h2;   // [B][64]
  __half* dy;   // [B][8]
  __half* da2;  // [B][64]
  __half* da1;  // [B][64]
};

struct TrainArgs {
  const int64_t* ids;          // explicit texel ids (gradient check) or NULL
  const float* target_rows;    // explicit targets [B][7] or NULL
  const float* target_levels;  // targets [texel][7] (training)
  int64_t batch;
  float inv_batch;
  uint64_t seed;
  int64_t step;                // training step (permutation position and Adam t)
  float lr, beta1, beta2, eps;
  float* loss;                 // accumulated sum of squared errors / batch
  float* dx_out;               // [B][8] latent gradients (gradient check) or NULL
  int train;                   // 1: Adam update of the latents in place
};

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// Seeded bijection of [0, n): a 4-round Feistel network on the smallest even-width
// power-of-two domain covering n, with cycle walking back into [0, n).
__device__ __forceinline__ int64_t permute_index(int64_t x, int64_t n, uint64_t seed) {
  int bits = 2;
  while ((1LL << bits) < n) bits += 2;
  const int h = bits / 2;
  const uint64_t mask = (1ull << h) - 1;
  uint64_t v = (uint64_t)x;
  for (int walk = 0; walk < 4096; ++walk) {
    uint64_t L = v >> h, R = v & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint64_t f = mix32((uint32_t)R ^ (uint32_t)(seed >> (16 * r)) ^ (0x9E3779B9u * (r + 1))) & mask;
      const uint64_t nl = R;
      R = L ^ f;
      L = nl;
    }
    v = (L << h) | R;
    if ((int64_t)v < n) return (int64_t)v;
  }
  return x % n;   // unreachable in practice: cycles return to [0, n) within a few steps
}

struct TrainSmem {
  uint32_t w[nn::IMG_ALL / 2];
  float b[nn::NBIAS];
  uint32_t a[4][32 * 4];    // latent rows (binary16)
  uint32_t d[4][32 * 4];    // dY rows (binary16)
  float y[4][32][8];        // Y rows, then dX rows
};

// Forward and backward of 32 texels per warp iteration: stores the batch's
// activations for the weight gradients, accumulates the loss and either applies
// Adam to the latents (training) or returns their gradients.
__global__ void __launch_bounds__(128) k_neural_fwd_bwd(NeuralDev nd, TrainArgs ta, ActBuffers act) {
  __shared__ __align__(16) TrainSmem s;
  stage_weights(nd, s.w, s.b, nn::IMG_ALL / 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* w3r = s.w + nn::I_W3R / 2;
  const uint32_t* w2r = s.w + nn::I_W2R / 2;
  const uint32_t* w1r = s.w + nn::I_W1R / 2;
  float loss_part = 0.0f;
  const int64_t nwarps = (int64_t)gridDim.x * 4;
  for (int64_t c = (int64_t)blockIdx.x * 4 + warp; c * 32 < ta.batch; c += nwarps) {
    const int64_t r = c * 32 + lane;
    const bool live = r < ta.batch;
    int64_t id = 0, epoch = 0;
    float T[7] = {0, 0, 0, 0, 0, 0, 0};
    float X[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (live) {
      if (ta.ids) {
        id = ta.ids[r];
      } else {
        const int64_t gp = ta.step * ta.batch + r;
        epoch = gp / nd.n_lat_texels;
        id = permute_index(gp % nd.n_lat_texels, nd.n_lat_texels, ta.seed);
      }
      const float4 x0 = reinterpret_cast<const float4*>(nd.lat32 + id * 8)[0];
      const float4 x1 = reinterpret_cast<const float4*>(nd.lat32 + id * 8)[1];
      X[0] = x0.x; X[1] = x0.y; X[2] = x0.z; X[3] = x0.w;
      X[4] = x1.x; X[5] = x1.y; X[6] = x1.z; X[7] = x1.w;
      const float* tp = ta.target_rows ? ta.target_rows + r * 7 : ta.target_levels + id * 7;
#pragma unroll
      for (int k = 0; k < 7; ++k) T[k] = tp[k];
    }
    const uint4 xh = make_uint4(pack_h2(X[0], X[1]), pack_h2(X[2], X[3]), pack_h2(X[4], X[5]),
                                pack_h2(X[6], X[7]));
    reinterpret_cast<uint4*>(s.a[warp])[lane] = xh;
    if (live) reinterpret_cast<uint4*>(act.x)[r] = xh;
    __syncwarp();
#pragma unroll 1
    for (int m = 0; m < 2; ++m) {
      uint32_t a2[1][4][4], a3[1][4][4];
      mlp_forward<1>(s.w, s.b, s.a[warp], 16 * m, s.y[warp], a2, a3);
      const int64_t rg = c * 32 + 16 * m + g, rh = rg + 8;   // batch rows of this lane's fragments
      const bool lg = rg < ta.batch, lh = rh < ta.batch;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col2 = 8 * kc + 4 * q + t;   // 32-bit word column of hidden pair
          if (lg) reinterpret_cast<uint32_t*>(act.h1)[rg * 32 + col2] = a2[0][kc][2 * q];
          if (lh) reinterpret_cast<uint32_t*>(act.h1)[rh * 32 + col2] = a2[0][kc][2 * q + 1];
          if (lg) reinterpret_cast<uint32_t*>(act.h2)[rg * 32 + col2] = a3[0][kc][2 * q];
          if (lh) reinterpret_cast<uint32_t*>(act.h2)[rh * 32 + col2] = a3[0][kc][2 * q + 1];
        }
      }
      __syncwarp();
      // dY = 2 (Y - T) / B for the rows of this tile (lanes 16m .. 16m + 15)
      if ((lane >> 4) == m) {
        float d[8];
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          const float e = live ? s.y[warp][lane][k] - T[k] : 0.0f;
          loss_part = fmaf(e, e, loss_part);
          d[k] = 2.0f * ta.inv_batch * e;
        }
        d[7] = 0.0f;
        const uint4 dh = make_uint4(pack_h2(d[0], d[1]), pack_h2(d[2], d[3]), pack_h2(d[4], d[5]),
                                    pack_h2(d[6], d[7]));
        reinterpret_cast<uint4*>(s.d[warp])[lane] = dh;
        if (live) reinterpret_cast<uint4*>(act.dy)[r] = dh;
      }
      __syncwarp();
      uint32_t ady[4] = {s.d[warp][(16 * m + g) * 4 + t], s.d[warp][(16 * m + g + 8) * 4 + t], 0u, 0u};
      // dA2 = (dY W3^T) * [H2 > 0]
      uint32_t da2[4][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float cc[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(cc, ady, w3r[(8 * j + g) * nn::S8 + t], 0u);
        const float2 hl = unpack_h2(a3[0][j >> 1][(j & 1) * 2]);
        const float2 hh = unpack_h2(a3[0][j >> 1][(j & 1) * 2 + 1]);
        const uint32_t lo = pack_h2(hl.x > 0.f ? cc[0] : 0.f, hl.y > 0.f ? cc[1] : 0.f);
        const uint32_t hi = pack_h2(hh.x > 0.f ? cc[2] : 0.f, hh.y > 0.f ? cc[3] : 0.f);
        da2[j >> 1][(j & 1) * 2] = lo;
        da2[j >> 1][(j & 1) * 2 + 1] = hi;
        const int col2 = 4 * j + t;
        if (lg) reinterpret_cast<uint32_t*>(act.da2)[rg * 32 + col2] = lo;
        if (lh) reinterpret_cast<uint32_t*>(act.da2)[rh * 32 + col2] = hi;
      }
      // dA1 = (dA2 W2^T) * [H1 > 0]
      uint32_t da1[4][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float cc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
          mma16816(cc, da2[kc], w2r[(8 * j + g) * nn::S72 + 8 * kc + t],
                   w2r[(8 * j + g) * nn::S72 + 8 * kc + 4 + t]);
        const float2 hl = unpack_h2(a2[0][j >> 1][(j & 1) * 2]);
        const float2 hh = unpack_h2(a2[0][j >> 1][(j & 1) * 2 + 1]);
        const uint32_t lo = pack_h2(hl.x > 0.f ? cc[0] : 0.f, hl.y > 0.f ? cc[1] : 0.f);
        const uint32_t hi = pack_h2(hh.x > 0.f ? cc[2] : 0.f, hh.y > 0.f ? cc[3] : 0.f);
        da1[j >> 1][(j & 1) * 2] = lo;
        da1[j >> 1][(j & 1) * 2 + 1] = hi;
        const int col2 = 4 * j + t;
        if (lg) reinterpret_cast<uint32_t*>(act.da1)[rg * 32 + col2] = lo;
        if (lh) reinterpret_cast<uint32_t*>(act.da1)[rh * 32 + col2] = hi;
      }
      // dX = dA1 W1^T
      float cx[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        mma16816(cx, da1[kc], w1r[g * nn::S72 + 8 * kc + t], w1r[g * nn::S72 + 8 * kc + 4 + t]);
      __syncwarp();
      s.y[warp][16 * m + g][2 * t] = cx[0];
      s.y[warp][16 * m + g][2 * t + 1] = cx[1];
      s.y[warp][16 * m + g + 8][2 * t] = cx[2];
      s.y[warp][16 * m + g + 8][2 * t + 1] = cx[3];
      __syncwarp();
    }
    if (live) {
      float dx[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) dx[k] = s.y[warp][lane][k];
      if (ta.dx_out) {
#pragma unroll
        for (int k = 0; k < 8; ++k) ta.dx_out[r * 8 + k] = dx[k];
      }
      if (ta.train) {
        // Adam on this latent row; its update count is its epoch + 1 (one visit per epoch)
        const float tt = (float)(epoch + 1);
        const float c1 = 1.0f - powf(ta.beta1, tt), c2 = 1.0f - powf(ta.beta2, tt);
        float xn[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t e = id * 8 + k;
          const float mm = ta.beta1 * nd.m_lat[e] + (1.0f - ta.beta1) * dx[k];
          const float vv = ta.beta2 * nd.v_lat[e] + (1.0f - ta.beta2) * dx[k] * dx[k];
          nd.m_lat[e] = mm;
          nd.v_lat[e] = vv;
          xn[k] = X[k] - ta.lr * (mm / c1) / (sqrtf(vv / c2) + ta.eps);
          nd.lat32[e] = xn[k];
        }
        reinterpret_cast<uint4*>(const_cast<__half*>(nd.lat16))[id] =
            make_uint4(pack_h2(xn[0], xn[1]), pack_h2(xn[2], xn[3]), pack_h2(xn[4], xn[5]),
                       pack_h2(xn[6], xn[7]));
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
  if (lane == 0) atomicAdd(ta.loss, loss_part * ta.inv_batch);
}

// Weight and bias gradients of one batch: dW1 = X^T dA1, dW2 = H1^T dA2, dW3 = H2^T dY,
// db = column sums.  Each CTA reduces 64-row chunks; warp w owns rows 16w..16w+15 of
// dW2 and dW3 and columns 16w..16w+15 of dW1.  Partial sums are added atomically.
struct WgradSmem {
  __half x[64][24];
  __half h1[64][72];
  __half h2[64][72];
  __half dy[64][8];
  __half da2[64][72];
  __half da1[64][72];
};

__global__ void __launch_bounds__(128) k_neural_wgrad(ActBuffers act, int64_t batch, float* grads) {
  __shared__ __align__(16) WgradSmem s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mi = lane >> 3, mr = lane & 7;   // ldmatrix: matrix index, row within it
  float w2acc[8][4], w3acc[4], w1acc[2][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) w2acc[j][0] = w2acc[j][1] = w2acc[j][2] = w2acc[j][3] = 0.f;
  w3acc[0] = w3acc[1] = w3acc[2] = w3acc[3] = 0.f;
  w1acc[0][0] = w1acc[0][1] = w1acc[0][2] = w1acc[0][3] = 0.f;
  w1acc[1][0] = w1acc[1][1] = w1acc[1][2] = w1acc[1][3] = 0.f;
  float bsum[2] = {0.f, 0.f};   // bias columns threadIdx.x and threadIdx.x + 128 (< 136)
  for (int64_t c0 = (int64_t)blockIdx.x * 64; c0 < batch; c0 += (int64_t)gridDim.x * 64) {
    // stage 64 rows (zero beyond the batch), 16-byte copies
    for (int k = threadIdx.x; k < 64 * 8; k += 128) {
      const int row = k >> 3, q = k & 7;
      const int64_t gr = c0 + row;
      const bool in = gr < batch;
      const uint4 z = make_uint4(0, 0, 0, 0);
      reinterpret_cast<uint4*>(&s.h1[row][0])[q] = in ? reinterpret_cast<const uint4*>(act.h1 + gr * 64)[q] : z;
      reinterpret_cast<uint4*>(&s.h2[row][0])[q] = in ? reinterpret_cast<const uint4*>(act.h2 + gr * 64)[q] : z;
      reinterpret_cast<uint4*>(&s.da2[row][0])[q] = in ? reinterpret_cast<const uint4*>(act.da2 + gr * 64)[q] : z;
      reinterpret_cast<uint4*>(&s.da1[row][0])[q] = in ? reinterpret_cast<const uint4*>(act.da1 + gr * 64)[q] : z;
      if (q == 0) {
        reinterpret_cast<uint4*>(&s.x[row][0])[0] = in ? reinterpret_cast<const uint4*>(act.x + gr * 8)[0] : z;
        reinterpret_cast<uint4*>(&s.x[row][0])[1] = z;
        reinterpret_cast<uint4*>(&s.dy[row][0])[0] = in ? reinterpret_cast<const uint4*>(act.dy + gr * 8)[0] : z;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int kc = 0; kc < 4; ++kc) {
      const int k0 = 16 * kc;
      // A = H1^T tile (hidden 16w.., batch k0..): matrix mi covers rows k0 + 8*(mi/2), cols 16w + 8*(mi%2)
      uint32_t ah1[4], ah2[4], ax[4];
      ldsm_x4_trans(ah1, &s.h1[k0 + mr + 8 * (mi >> 1)][16 * warp + 8 * (mi & 1)]);
      ldsm_x4_trans(ah2, &s.h2[k0 + mr + 8 * (mi >> 1)][16 * warp + 8 * (mi & 1)]);
      ldsm_x4_trans(ax, &s.x[k0 + mr + 8 * (mi >> 1)][8 * (mi & 1)]);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        // B = dA2 columns 16p .. 16p+15: matrices (k lo, n 16p), (k hi, n 16p), (k lo, n 16p+8), (k hi, n 16p+8)
        uint32_t b[4];
        ldsm_x4_trans(b, &s.da2[k0 + mr + 8 * (mi & 1)][16 * p + 8 * (mi >> 1)]);
        mma16816(w2acc[2 * p], ah1, b[0], b[1]);
        mma16816(w2acc[2 * p + 1], ah1, b[2], b[3]);
      }
      {
        uint32_t b[2];
        ldsm_x2_trans(b, &s.dy[k0 + mr + 8 * (mi & 1)][0]);
        mma16816(w3acc, ah2, b[0], b[1]);
      }
      {
        uint32_t b[4];
        ldsm_x4_trans(b, &s.da1[k0 + mr + 8 * (mi & 1)][16 * warp + 8 * (mi >> 1)]);
        mma16816(w1acc[0], ax, b[0], b[1]);
        mma16816(w1acc[1], ax, b[2], b[3]);
      }
    }
    for (int q = 0; q < 2; ++q) {
      const int k = threadIdx.x + 128 * q;
      if (k >= nn::NBIAS) break;
      for (int row = 0; row < 64; ++row) {
        if (k < 64) bsum[q] += __half2float(s.da1[row][k]);
        else if (k < 128) bsum[q] += __half2float(s.da2[row][k - 64]);
        else bsum[q] += __half2float(s.dy[row][k - 128]);
      }
    }
    __syncthreads();
  }
  // dW2[m][n]: m = 16w + g (+8), n = 8j + 2t (+1)
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int n = 8 * j + 2 * t, m = 16 * warp + g;
    atomicAdd(grads + nn::P_W2 + m * 64 + n, w2acc[j][0]);
    atomicAdd(grads + nn::P_W2 + m * 64 + n + 1, w2acc[j][1]);
    atomicAdd(grads + nn::P_W2 + (m + 8) * 64 + n, w2acc[j][2]);
    atomicAdd(grads + nn::P_W2 + (m + 8) * 64 + n + 1, w2acc[j][3]);
  }
  {
    const int o = 2 * t, m = 16 * warp + g;
    if (o < 7) {
      atomicAdd(grads + nn::P_W3 + m * 7 + o, w3acc[0]);
      atomicAdd(grads + nn::P_W3 + (m + 8) * 7 + o, w3acc[2]);
    }
    if (o + 1 < 7) {
      atomicAdd(grads + nn::P_W3 + m * 7 + o + 1, w3acc[1]);
      atomicAdd(grads + nn::P_W3 + (m + 8) * 7 + o + 1, w3acc[3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {   // dW1[ch = g][hidden n]; rows g + 8 are the zero padding
    const int n = 16 * warp + 8 * q + 2 * t;
    atomicAdd(grads + nn::P_W1 + g * 64 + n, w1acc[q][0]);
    atomicAdd(grads + nn::P_W1 + g * 64 + n + 1, w1acc[q][1]);
  }
  for (int q = 0; q < 2; ++q) {
    const int k = threadIdx.x + 128 * q;
    if (k >= nn::NBIAS) break;
    if (k < 64) atomicAdd(grads + nn::P_B1 + k, bsum[q]);
    else if (k < 128) atomicAdd(grads + nn::P_B2 + (k - 64), bsum[q]);
    else if (k - 128 < 7) atomicAdd(grads + nn::P_B3 + (k - 128), bsum[q]);
  }
}

// Binary16 weight images and padded biases from the float32 parameters.
__device__ void build_images(const float* p, __half* img, float* bias) {
  for (int k = threadIdx.x; k < nn::IMG_ALL; k += blockDim.x) img[k] = __float2half_rn(0.0f);
  __syncthreads();
  for (int e = threadIdx.x; e < 8 * 64; e += blockDim.x) {   // W1[c][h]
    const int c = e / 64, h = e % 64;
    const __half v = __float2half_rn(p[nn::P_W1 + e]);
    img[nn::I_W1T + h * 24 + c] = v;
    img[nn::I_W1R + c * 72 + h] = v;
  }
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {  // W2[i][o]
    const int i = e / 64, o = e % 64;
    const __half v = __float2half_rn(p[nn::P_W2 + e]);
    img[nn::I_W2T + o * 72 + i] = v;
    img[nn::I_W2R + i * 72 + o] = v;
  }
  for (int e = threadIdx.x; e < 64 * 7; e += blockDim.x) {   // W3[h][o]
    const int h = e / 7, o = e % 7;
    const __half v = __float2half_rn(p[nn::P_W3 + e]);
    img[nn::I_W3T + o * 72 + h] = v;
    img[nn::I_W3R + h * 8 + o] = v;
  }
  for (int k = threadIdx.x; k < nn::NBIAS; k += blockDim.x) {
    float v = 0.0f;
    if (k < 64) v = p[nn::P_B1 + k];
    else if (k < 128) v = p[nn::P_B2 + k - 64];
    else if (k - 128 < 7) v = p[nn::P_B3 + k - 128];
    bias[k] = v;
  }
}

__global__ void k_neural_images(const float* params, __half* img, float* bias) {
  build_images(params, img, bias);
}

// Adam on the MLP parameters (step t >= 1), then fresh binary16 images; the batch
// loss is copied out.
__global__ void __launch_bounds__(256) k_neural_adam(float* params, float* m, float* v, const float* grads,
                                                     float t, float lr, float beta1, float beta2,
                                                     float eps, __half* img, float* bias,
                                                     const float* loss, float* loss_out) {
  const float c1 = 1.0f - powf(beta1, t), c2 = 1.0f - powf(beta2, t);
  for (int k = threadIdx.x; k < nn::NPARAM; k += blockDim.x) {
    const float gk = grads[k];
    const float mm = beta1 * m[k] + (1.0f - beta1) * gk;
    const float vv = beta2 * v[k] + (1.0f - beta2) * gk * gk;
    m[k] = mm;
    v[k] = vv;
    params[k] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
  __syncthreads();
  build_images(params, img, bias);
  if (threadIdx.x == 0 && loss_out) *loss_out = *loss;
}

// Float32 -> binary16 rows: dst[r][0..7] from src[r][0..cin-1] (zero beyond cin).
__global__ void k_rows_to_h8(const float* src, int cin, __half* dst, int64_t rows) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = k < cin ? src[r * cin + k] : 0.0f;
    reinterpret_cast<uint4*>(dst)[r] = make_uint4(pack_h2(v[0], v[1]), pack_h2(v[2], v[3]),
                                                  pack_h2(v[4], v[5]), pack_h2(v[6], v[7]));
  }
}

// ---------------------------------------------------------------- launchers

template <int F>
static cudaError_t run_neural(Op op, const NeuralDev& nd, const LookupArgs& a, cudaStream_t s) {
  const int blocks = grid_blocks(a.n, 128);
  if (op == OP_STOCHASTIC) {
    // at least 46 KiB of shared memory per CTA keeps at most 4 CTAs on an SM (228 KiB),
    // so their 4 x 128 tensor-memory columns fit in the SM's 512 and no allocation waits
    const int need = (int)sizeof(tc::Smem) + 1024;
    const int smem = need > 46 * 1024 ? need : 46 * 1024;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_neural_stochastic_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr = true;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t pairs = ((a.n + tc::ROWS - 1) / tc::ROWS + 1) / 2;   // two tiles per CTA pass
    const int grid = (int)(pairs < (int64_t)sms * 4 ? pairs : (int64_t)sms * 4);
    k_neural_stochastic_tc<F><<<grid, 256, smem, s>>>(nd, a);
    return cudaGetLastError();
  }
  else if (op == OP_DETERMINISTIC) k_neural_deterministic<F><<<blocks, 128, 0, s>>>(nd, a);
  else return cudaErrorNotSupported;
  return cudaGetLastError();
}

cudaError_t launch_neural(Op op, int filter, const NeuralDev& nd, const LookupArgs& a, cudaStream_t s) {
  switch (filter) {
    case STF_FILTER_LINEAR: return run_neural<STF_FILTER_LINEAR>(op, nd, a, s);
    case STF_FILTER_BSPLINE3: return run_neural<STF_FILTER_BSPLINE3>(op, nd, a, s);
    case STF_FILTER_CATMULL_ROM: return run_neural<STF_FILTER_CATMULL_ROM>(op, nd, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stf

// ---------------------------------------------------------------- host side

namespace stf {

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

stf_status build_neural(stf_texture_s* t, const stf_neural_desc* d, cudaStream_t s) {
  const int W = d->width, H = d->height;
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!pow2(W) || !pow2(H)) return fail(STF_ERR_INVALID_ARGUMENT, "neural texture sizes must be powers of two");
  int maxlev = 1;
  while ((W >> maxlev) > 0 || (H >> maxlev) > 0) ++maxlev;
  if (d->latent_levels < 1 || d->latent_levels > 4)
    return fail(STF_ERR_INVALID_ARGUMENT, "latent_levels must be 1 .. 4");
  if (d->levels < d->latent_levels || d->levels > maxlev || d->levels > STF_MAX_LEVELS)
    return fail(STF_ERR_INVALID_ARGUMENT, "levels %d outside [latent_levels, %d]", d->levels, maxlev);
  if (!d->latents || !d->params) return fail(STF_ERR_INVALID_ARGUMENT, "latents or params is NULL");
  if (d->levels > d->latent_levels && !d->fallback)
    return fail(STF_ERR_INVALID_ARGUMENT, "fallback texels are NULL");
  NeuralDev& nd = t->neural;
  memset(&nd, 0, sizeof(nd));
  nd.nlat = d->latent_levels;
  nd.nlev = d->levels;
  int64_t n_lat = 0, n_fb = 0;
  for (int L = 0; L < d->levels; ++L) {
    nd.lvl_w[L] = (W >> L) > 0 ? (W >> L) : 1;
    nd.lvl_h[L] = (H >> L) > 0 ? (H >> L) : 1;
    const int64_t cnt = (int64_t)nd.lvl_w[L] * nd.lvl_h[L];
    if (L < nd.nlat) {
      nd.lvl_off[L] = n_lat;
      n_lat += cnt;
    } else {
      nd.lvl_off[L] = n_fb;
      n_fb += cnt;
    }
  }
  nd.n_lat_texels = n_lat;
  const size_t b_lat = al256(sizeof(float) * 8 * n_lat), b_lat16 = al256(2 * 8 * n_lat);
  const size_t b_fb16 = al256(2 * 8 * (n_fb > 0 ? n_fb : 1));
  const size_t b_p = al256(sizeof(float) * nn::NPARAM);
  const size_t b_img = al256(2 * nn::IMG_ALL), b_bias = al256(sizeof(float) * nn::NBIAS);
  const size_t total = 3 * b_lat + b_lat16 + b_fb16 + 4 * b_p + 256 + b_img + b_bias;
  cudaError_t e = dev_alloc(&t->d_neural, total);
  if (e != cudaSuccess) return fail_cuda(e, "neural texture allocation");
  t->bytes += (int64_t)total;
  char* p = (char*)t->d_neural;
  nd.lat32 = (float*)p;  p += b_lat;
  nd.m_lat = (float*)p;  p += b_lat;
  nd.v_lat = (float*)p;  p += b_lat;
  nd.lat16 = (const __half*)p; p += b_lat16;
  nd.fb16 = (const __half*)p;  p += b_fb16;
  t->n_params = (float*)p; p += b_p;
  t->n_m = (float*)p;      p += b_p;
  t->n_v = (float*)p;      p += b_p;
  t->n_grads = (float*)p;  p += b_p;
  t->n_loss = (float*)p;   p += 256;
  nd.wimg = (const __half*)p; p += b_img;
  nd.bias = (const float*)p;
  const cudaMemcpyKind kind = d->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  e = cudaMemcpyAsync(nd.lat32, d->latents, sizeof(float) * 8 * n_lat, kind, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(nd.m_lat, 0, 2 * b_lat, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->n_params, d->params, sizeof(float) * nn::NPARAM, kind, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->n_m, 0, 2 * b_p, s);
  if (e == cudaSuccess) {
    k_rows_to_h8<<<grid_blocks(n_lat, 256), 256, 0, s>>>(nd.lat32, 8, (__half*)nd.lat16, n_lat);
    k_neural_images<<<1, 256, 0, s>>>(t->n_params, (__half*)nd.wimg, (float*)nd.bias);
    e = cudaGetLastError();
  }
  float* tmp = nullptr;
  if (e == cudaSuccess && n_fb > 0) {
    e = dev_alloc((void**)&tmp, sizeof(float) * 7 * n_fb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, d->fallback, sizeof(float) * 7 * n_fb, kind, s);
    if (e == cudaSuccess) {
      k_rows_to_h8<<<grid_blocks(n_fb, 256), 256, 0, s>>>(tmp, 7, (__half*)nd.fb16, n_fb);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail_cuda(e, "neural texture upload");
  t->kind = STF_KIND_NEURAL2D;
  t->channels = STF_NEURAL_OUT;
  t->levels = d->levels;
  t->dims[0] = W;
  t->dims[1] = H;
  t->dims[2] = 1;
  t->n_step = 0;
  return STF_OK;
}

static cudaError_t alloc_acts(ActBuffers& act, void** block, int64_t batch) {
  const size_t rows = (size_t)batch;
  cudaError_t e = dev_alloc(block, 2 * rows * (8 + 64 + 64 + 8 + 64 + 64));
  if (e != cudaSuccess) return e;
  __half* p = (__half*)*block;
  act.x = p;   p += rows * 8;
  act.h1 = p;  p += rows * 64;
  act.h2 = p;  p += rows * 64;
  act.dy = p;  p += rows * 8;
  act.da2 = p; p += rows * 64;
  act.da1 = p;
  return cudaSuccess;
}

static int train_blocks(int64_t rows, int per_block) {
  const int64_t need = (rows + per_block - 1) / per_block;
  const int64_t cap = (int64_t)grid_blocks(1LL << 40, 128);
  return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

static stf_status neural_handle(stf_texture t) {
  if (!handle_ok(t)) return fail(STF_ERR_INVALID_HANDLE, "unknown texture handle");
  if (t->kind != STF_KIND_NEURAL2D) return fail(STF_ERR_UNSUPPORTED, "not a neural texture");
  return STF_OK;
}

}  // namespace stf

using namespace stf;

extern "C" stf_status stf_neural_gradients(stf_texture t, const int64_t* ids, int64_t batch,
                                           const float* target_rows, float* d_param_grads,
                                           float* d_latent_grads, float* d_loss, void* stream) {
  stf_status st = neural_handle(t);
  if (st != STF_OK) return st;
  if (batch < 1 || !ids || !target_rows) return fail(STF_ERR_INVALID_ARGUMENT, "need batch >= 1, ids and targets");
  cudaStream_t s = (cudaStream_t)stream;
  ActBuffers act;
  void* block = nullptr;
  cudaError_t e = alloc_acts(act, &block, batch);
  if (e != cudaSuccess) return fail_cuda(e, "activation buffers");
  TrainArgs ta;
  memset(&ta, 0, sizeof(ta));
  ta.ids = ids;
  ta.target_rows = target_rows;
  ta.batch = batch;
  ta.inv_batch = 1.0f / (float)batch;
  ta.loss = t->n_loss;
  ta.dx_out = d_latent_grads;
  e = cudaMemsetAsync(t->n_grads, 0, sizeof(float) * nn::NPARAM, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->n_loss, 0, sizeof(float), s);
  if (e == cudaSuccess) {
    k_neural_fwd_bwd<<<train_blocks(batch, 128), 128, 0, s>>>(t->neural, ta, act);
    k_neural_wgrad<<<train_blocks(batch, 64), 128, 0, s>>>(act, batch, t->n_grads);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && d_param_grads)
    e = cudaMemcpyAsync(d_param_grads, t->n_grads, sizeof(float) * nn::NPARAM, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_loss) e = cudaMemcpyAsync(d_loss, t->n_loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(block);
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "neural gradients");
}

extern "C" stf_status stf_neural_train(stf_texture t, const float* d_target, const stf_train_config* cfg,
                                       int32_t steps, float* d_loss_per_step, void* stream) {
  stf_status st = neural_handle(t);
  if (st != STF_OK) return st;
  if (!cfg || !d_target) return fail(STF_ERR_INVALID_ARGUMENT, "config or target is NULL");
  if (cfg->batch < 1 || cfg->batch > t->neural.n_lat_texels)
    return fail(STF_ERR_INVALID_ARGUMENT, "batch must be in [1, %lld]", (long long)t->neural.n_lat_texels);
  if (!(cfg->lr_latent >= 0.f) || !(cfg->lr_params >= 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
    return fail(STF_ERR_INVALID_ARGUMENT, "invalid optimizer settings");
  if (steps < 0) return fail(STF_ERR_INVALID_ARGUMENT, "steps < 0");
  if (steps == 0) return STF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ActBuffers act;
  void* block = nullptr;
  cudaError_t e = alloc_acts(act, &block, cfg->batch);
  if (e != cudaSuccess) return fail_cuda(e, "activation buffers");
  for (int k = 0; k < steps && e == cudaSuccess; ++k) {
    TrainArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.target_levels = d_target;
    ta.batch = cfg->batch;
    ta.inv_batch = 1.0f / (float)cfg->batch;
    ta.seed = cfg->seed;
    ta.step = t->n_step;
    ta.lr = cfg->lr_latent;
    ta.beta1 = cfg->beta1;
    ta.beta2 = cfg->beta2;
    ta.eps = cfg->eps;
    ta.loss = t->n_loss;
    ta.train = 1;
    e = cudaMemsetAsync(t->n_grads, 0, sizeof(float) * nn::NPARAM, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->n_loss, 0, sizeof(float), s);
    if (e != cudaSuccess) break;
    k_neural_fwd_bwd<<<train_blocks(cfg->batch, 128), 128, 0, s>>>(t->neural, ta, act);
    k_neural_wgrad<<<train_blocks(cfg->batch, 64), 128, 0, s>>>(act, cfg->batch, t->n_grads);
    k_neural_adam<<<1, 256, 0, s>>>(t->n_params, t->n_m, t->n_v, t->n_grads, (float)(t->n_step + 1),
                                    cfg->lr_params, cfg->beta1, cfg->beta2, cfg->eps,
                                    (__half*)t->neural.wimg, (float*)t->neural.bias, t->n_loss,
                                    d_loss_per_step ? d_loss_per_step + k : nullptr);
    e = cudaGetLastError();
    t->n_step += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(block);
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "neural training");
}

extern "C" stf_status stf_neural_read(stf_texture t, float* d_params, float* d_latents, void* stream) {
  stf_status st = neural_handle(t);
  if (st != STF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (d_params) e = cudaMemcpyAsync(d_params, t->n_params, sizeof(float) * nn::NPARAM, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_latents)
    e = cudaMemcpyAsync(d_latents, t->neural.lat32, sizeof(float) * 8 * t->neural.n_lat_texels,
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? STF_OK : fail_cuda(e, "neural read");
}
