// Neural textures: latent MIP levels decoded by an 8 -> 64 -> 64 -> 7 ReLU MLP on
// the tensor cores (binary16 operands, float32 accumulation).
//
// The paper motivates stochastic filtering for decoders that are expensive to run
// per texel, neural texture representations among them (Section 1; Section 5.2,
// "Texture compression"): the stochastic lookup picks one latent texel with the same
// inverse-CDF tap choice as a plain 2D texture and decodes it once; the
// deterministic lookup decodes every tap and filters the decoded values.
//
// The stochastic and the deterministic decode and the training (forward, backward and
// weight gradients) run on the fifth-generation tensor cores: tcgen05.mma on 128-row
// tiles, operands in shared memory, accumulators in tensor memory (see the tcgen05
// sections below).
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
constexpr int IMG_ALL = 12416;
constexpr int NBIAS = 136;   // b1[64], b2[64], b3[8] (b3[7] = 0)

}  // namespace nn

// ---------------------------------------------------------------- binary16 pairs

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float2 unpack_h2(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
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
// (latent or fallback) into the lane's shared-memory row.  SLIM: the call has no
// binning permutation and no tap output, so the caller's index is i.
// uv and lod of query i (zeros past the end).
struct QueryCoords {
  float2 uv;
  float lod;
};
__device__ __forceinline__ QueryCoords load_coords(const LookupArgs& a, int64_t i) {
  QueryCoords q;
  q.uv = make_float2(0.0f, 0.0f);
  q.lod = 0.0f;
  if (i < a.n) {
    q.uv = reinterpret_cast<const float2*>(a.coords)[i];
    q.lod = a.lod ? a.lod[i] : 0.0f;
  }
  return q;
}

template <int F, bool SLIM = false>
__device__ __forceinline__ NeuralPick neural_pick(const NeuralDev& nd, const LookupArgs& a, int64_t i,
                                                  uint4* row, const QueryCoords* pre = nullptr) {
  NeuralPick pk;
  pk.j = 0;
  pk.sigma = 1.0f;
  pk.tap = make_int4(0, 0, 0, -1);
  pk.mode = 0;
  if (i >= a.n) return pk;
  pk.j = SLIM ? i : query_slot(a, i);
  const QueryCoords qc = pre ? *pre : load_coords(a, i);
  const float2 uv = qc.uv;
  const float lod = qc.lod;
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
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
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

// The forward weights as K-major no-swizzle B tiles (threads tid, tid + nt, ...):
// W1^T (64 x 16) with its bias split into binary16 (hi, lo) in k 8, 9; W2^T (64 x 64);
// W3^T (16 x 64, rows >= 7 zero); the b2 and b3 bias chunks (64 x 16, 16 x 16) with
// (hi, lo) in k 0, 1; and one 8-row group of ones in columns 0, 1.  A bias b enters the
// accumulator as b_hi + b_lo, b_hi = fp16(b), b_lo = fp16(b - b_hi): to about 2^-22 |b|.
__device__ __forceinline__ void stage_fwd_weights(const NeuralDev& nd, unsigned char* b1, unsigned char* b2,
                                                  unsigned char* b3, unsigned char* b2x, unsigned char* b3x,
                                                  unsigned char* ones, int tid, int nt) {
  const uint4* img = reinterpret_cast<const uint4*>(nd.wimg);
  auto split = [](float b) -> uint32_t {
    const __half hi = __float2half_rn(b);
    const __half lo = __float2half_rn(b - __half2float(hi));
    return (uint32_t)__half_as_ushort(hi) | ((uint32_t)__half_as_ushort(lo) << 16);
  };
  const uint4 z = make_uint4(0, 0, 0, 0);
  for (int n = tid; n < 64; n += nt) {
    *reinterpret_cast<uint4*>(b1 + off(n, 0, 16)) = __ldg(img + (nn::I_W1T + n * 24) / 8);
    *reinterpret_cast<uint4*>(b1 + off(n, 8, 16)) = make_uint4(split(__ldg(nd.bias + n)), 0, 0, 0);
    *reinterpret_cast<uint4*>(b2x + off(n, 0, 16)) = make_uint4(split(__ldg(nd.bias + 64 + n)), 0, 0, 0);
    *reinterpret_cast<uint4*>(b2x + off(n, 8, 16)) = z;
  }
  for (int n = tid; n < 16; n += nt) {
    const uint32_t b = n < 7 ? split(__ldg(nd.bias + 128 + n)) : 0u;
    *reinterpret_cast<uint4*>(b3x + off(n, 0, 16)) = make_uint4(b, 0, 0, 0);
    *reinterpret_cast<uint4*>(b3x + off(n, 8, 16)) = z;
  }
  for (int r = tid; r < 8; r += nt) {
    *reinterpret_cast<uint4*>(ones + off(r, 0, 16)) = make_uint4(0x3C003C00u, 0, 0, 0);
    *reinterpret_cast<uint4*>(ones + off(r, 8, 16)) = z;
  }
  for (int e = tid; e < 64 * 8; e += nt) {
    const int n = e >> 3, kc = e & 7;
    *reinterpret_cast<uint4*>(b2 + off(n, 8 * kc, 64)) = __ldg(img + (nn::I_W2T + n * 72 + 8 * kc) / 8);
  }
  for (int e = tid; e < 16 * 8; e += nt) {
    const int n = e >> 3, kc = e & 7;
    *reinterpret_cast<uint4*>(b3 + off(n, 8 * kc, 64)) = n < 8 ? __ldg(img + (nn::I_W3T + n * 72 + 8 * kc) / 8) : z;
  }
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
// MMA) -> ReLU -> binary16 row of the next A tile, 16 columns per tensor-memory load:
// 32-column loads left the stochastic decode spilling at its 64-register cap and made
// it 26% slower.
__device__ __forceinline__ void tc_hidden(uint32_t taddr, unsigned char* a2, int row) {
#pragma unroll
  for (int half = 0; half < 4; ++half) {
    uint32_t r[16];
    tc::tmem_ld<16>(taddr + 16 * half, r);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
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
      *reinterpret_cast<uint4*>(a2 + tc::off(row, 16 * half + 8 * q, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
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
// has consumed it, and the coordinates of the tile after that are loaded right then, a
// whole tile ahead of its tap choice (6% sooner than loading them at the choice).
//
// SLIM (calls without a binning permutation or tap output) compiles out the per-query
// caller index and tap, which leaves the registers the epilogues need at the
// 64-register cap of four CTAs per SM.
template <int F, bool SLIM>
__global__ void __launch_bounds__(256, 4) k_neural_stochastic_tc(NeuralDev nd, LookupArgs a) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  tc::Smem& s = *reinterpret_cast<tc::Smem*>(dyn);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid >> 7, row = tid & 127;          // group, row of the group's tile
  tc::Group& G = s.grp[g];
  // weights: binary16 images -> K-major no-swizzle B tiles (16-byte rows)
  {
    tc::stage_fwd_weights(nd, s.b1, s.b2, s.b3, s.b2x, s.b3x, s.ones, tid, 256);
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
  if (tile < ntiles) cur = neural_pick<F, SLIM>(nd, a, tile * tc::ROWS + row, arow);
  cp_async_commit();
  // coordinates of the next tile, loaded a whole tile ahead of its tap choice
  QueryCoords qn = load_coords(a, (tile + step) * tc::ROWS + row);
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
    if (next < ntiles) nxt = neural_pick<F, SLIM>(nd, a, next * tc::ROWS + row, arow, &qn);
    cp_async_commit();
    qn = load_coords(a, (next + step) * tc::ROWS + row);
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
    if (SLIM || a.perm == nullptr) {
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
    if (!SLIM && live && a.taps) reinterpret_cast<int4*>(a.taps)[cur.j] = cur.tap;
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

// Deterministic decode on the tensor cores: every tap of the filter window (at one
// level, or at two blended by frac(lod)) is a row of a 128-row tile; a query takes R =
// parts x T^2 consecutive rows (parts = 2 when the level is blended, else 1), so a tile
// holds 128 / R queries.  Each thread gathers its tap's latent texel into the A tile
// (zeros for fallback levels and for taps of queries without a texture value), the
// three layers run as in the stochastic decode, and each row's output times its
// weight (the tap weights wx wy times the level weight) is staged in shared memory;
// the query's first row then sums its R rows.  Fallback levels use the stored texel.
namespace tcd {

struct Smem {
  unsigned char b1[tc::B1_BYTES];
  unsigned char b2[tc::B2_BYTES];
  unsigned char b3[tc::B3_BYTES];
  unsigned char b2x[64 * 16 * 2];
  unsigned char b3x[16 * 16 * 2];
  unsigned char ones[8 * 16 * 2];
  unsigned char a1[tc::A1_BYTES];
  unsigned char a2[tc::A2_BYTES];      // H1, then H2, then the weighted output rows
  uint64_t bar;
  uint32_t tmem;
  int abort;
};

constexpr int TMEM_COLS = 64;

}  // namespace tcd

// One row of a deterministic tile: its query, weight and texel kind.  The texel (latent
// or stored fallback) is gathered into the row of the A tile by cp.async.
struct DetRow {
  int64_t i;     // query
  float w;       // tap weight times level weight (0: the row adds nothing)
  int mode;      // 0: nothing, 1: decode the latent, 2: stored fallback texel
};

template <int F>
__device__ __forceinline__ DetRow det_row(const NeuralDev& nd, const LookupArgs& a, int64_t i, int p, int tx,
                                          int ty, uint4* arow, const QueryCoords* pre = nullptr) {
  using Fl = Filter<F>;
  DetRow d;
  d.i = i;
  d.w = 0.0f;
  d.mode = 0;
  if (i >= a.n) return d;
  const QueryCoords qc = pre ? *pre : load_coords(a, i);
  const float2 uv = qc.uv;
  const float lod = qc.lod;
  if (!(isfinite(lod) && isfinite(uv.x) && isfinite(uv.y))) return d;
  float lw = p == 0 ? 1.0f : 0.0f;
  int L = 0;
  if (a.lod != nullptr && nd.nlev > 1) {
    const float lc = fminf(fmaxf(lod, 0.0f), (float)(nd.nlev - 1));
    if (a.level_mode == STF_LEVEL_NEAREST) {
      L = min((int)floorf(__fadd_rn(lc, 0.5f)), nd.nlev - 1);
    } else {
      const float fl = floorf(lc), fr = __fsub_rn(lc, fl);
      L = p == 0 ? (int)fl : min((int)fl + 1, nd.nlev - 1);
      lw = p == 0 ? 1.0f - fr : fr;
    }
  }
  const int w = nd.lvl_w[L], h = nd.lvl_h[L];
  float x[2] = {__fsub_rn(__fmul_rn(uv.x, (float)w), 0.5f), __fsub_rn(__fmul_rn(uv.y, (float)h), 0.5f)};
  if (!(lw > 0.0f) || !prepare_coords<2>(x)) return d;
  float fx, fy;
  const int bx = axis_base(x[0], fx) + Fl::OFF0, by = axis_base(x[1], fy) + Fl::OFF0;
  float wx[Fl::T], wy[Fl::T];
  Fl::weights(fx, wx);
  Fl::weights(fy, wy);
  float wxs = wx[0], wys = wy[0];
#pragma unroll
  for (int k = 1; k < Fl::T; ++k) {
    if (tx == k) wxs = wx[k];
    if (ty == k) wys = wy[k];
  }
  d.w = wxs * wys * lw;
  const int cx = min(max(bx + tx, 0), w - 1), cy = min(max(by + ty, 0), h - 1);
  const __half* base = L < nd.nlat ? nd.lat16 : nd.fb16;
  cp_async16(arow, base + (nd.lvl_off[L] + (int64_t)cy * w + cx) * 8);
  d.mode = L < nd.nlat ? 1 : 2;
  return d;
}

template <int F>
__global__ void __launch_bounds__(128, 6) k_neural_deterministic_tc(NeuralDev nd, LookupArgs a) {
  using Fl = Filter<F>;
  extern __shared__ __align__(1024) unsigned char dyn[];
  tcd::Smem& s = *reinterpret_cast<tcd::Smem*>(dyn);
  const int tid = threadIdx.x, warp = tid >> 5;
  tc::stage_fwd_weights(nd, s.b1, s.b2, s.b3, s.b2x, s.b3x, s.ones, tid, 128);
  uint4* arow = reinterpret_cast<uint4*>(s.a1 + tc::off(tid, 0, 16));
  *reinterpret_cast<uint4*>(s.a1 + tc::off(tid, 8, 16)) = make_uint4(0x3C003C00u, 0, 0, 0);
  if (tid == 0) {
    s.abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&s.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&s.tmem)), "n"(tcd::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s.tmem;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  uint32_t parity = 0;
  auto run = [&](auto issue) -> bool {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue();
      tc::commit(&s.bar);
      if (!tc::wait_bar(&s.bar, parity)) s.abort = 1;
    }
    parity ^= 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    return s.abort == 0;
  };
  constexpr int T2 = Fl::T * Fl::T;
  const int parts = (a.lod != nullptr && nd.nlev > 1 && a.level_mode != STF_LEVEL_NEAREST) ? 2 : 1;
  const int R = parts * T2;                    // rows per query: 4, 8, 16 or 32
  const int Q = 128 / R;                       // queries per tile
  const int qi = tid / R, sub = tid % R, p = sub / T2, tap = sub % T2;
  const int tx = tap % Fl::T, ty = tap / Fl::T;
  float* stage = reinterpret_cast<float*>(s.a2);
  const int64_t ntiles = (a.n + Q - 1) / Q;
  int64_t tile = blockIdx.x;
  DetRow cur;
  if (tile < ntiles) cur = det_row<F>(nd, a, tile * Q + qi, p, tx, ty, arow);
  cp_async_commit();
  QueryCoords qn = load_coords(a, (tile + gridDim.x) * Q + qi);   // a tile ahead
  for (; tile < ntiles; tile += gridDim.x) {
    cp_async_wait<0>();
    uint4 fb = make_uint4(0, 0, 0, 0);
    if (cur.mode == 2) fb = *arow;               // stored fallback texel (own row)
    if (cur.mode != 1) *arow = make_uint4(0, 0, 0, 0);
    if (!run([&] { tc::mma(tmem, tc::desc(s.a1, 16), tc::desc(s.b1, 16), tc::idesc(128, 64), 0); })) break;
    // A1 is free: gather the next tile's texels while this tile's layers run
    const int64_t next = tile + gridDim.x;
    DetRow nxt;
    if (next < ntiles) nxt = det_row<F>(nd, a, next * Q + qi, p, tx, ty, arow, &qn);
    cp_async_commit();
    qn = load_coords(a, (next + gridDim.x) * Q + qi);
    tc_hidden(trow, s.a2, tid);
    if (!run([&] {
          for (int kk = 0; kk < 4; ++kk)
            tc::mma(tmem, tc::desc(s.a2 + kk * 256, 64), tc::desc(s.b2 + kk * 256, 64), tc::idesc(128, 64), kk);
          tc::mma(tmem, tc::desc_rows_repeated(s.ones), tc::desc(s.b2x, 16), tc::idesc(128, 64), 1);
        }))
      break;
    tc_hidden(trow, s.a2, tid);
    if (!run([&] {
          for (int kk = 0; kk < 4; ++kk)
            tc::mma(tmem, tc::desc(s.a2 + kk * 256, 64), tc::desc(s.b3 + kk * 256, 64), tc::idesc(128, 16), kk);
          tc::mma(tmem, tc::desc_rows_repeated(s.ones), tc::desc(s.b3x, 16), tc::idesc(128, 16), 1);
        }))
      break;
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
    }
    // A2 (H2) has been consumed by layer 3: it now stages the weighted rows
#pragma unroll
    for (int k = 0; k < 7; ++k) stage[tid * 8 + k] = cur.mode ? cur.w * v[k] : 0.0f;
    __syncthreads();
    if (sub == 0 && cur.i < a.n) {
      float acc[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int rr = 0; rr < R; ++rr)
#pragma unroll
        for (int k = 0; k < 7; ++k) acc[k] += stage[(tid + rr) * 8 + k];
#pragma unroll
      for (int k = 0; k < 7; ++k) a.out[cur.i * 7 + k] = acc[k];
    }
    cur = nxt;
    // the next tile's first barrier orders these reads before A2 is rewritten
  }
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && s.abort) atomicOr(nd.status, STF_DEV_MMA_TIMEOUT);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "n"(tcd::TMEM_COLS));
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

// ---------------------------------------------------------------- tcgen05 training
//
// Forward and backward of the decoder for tiles of 128 training texels on the
// fifth-generation tensor cores: six tcgen05.mma round trips per tile (M = 128,
// binary16 operands in shared memory, float32 accumulators in tensor memory), issued
// by one thread, each followed by an epilogue in which every thread reads its row:
//   H1 = ReLU(X W1 + b1), H2 = ReLU(H1 W2 + b2), Y = H2 W3 + b3       (forward)
//   dY = 2 (Y - T) / B, dA2 = (dY W3^T) [H2 > 0], dA1 = (dA2 W2^T) [H1 > 0],
//   dX = dA1 W1^T                                                      (backward)
// The biases enter the forward MMAs as an extra K chunk against columns of ones, as in
// the decode.  The activations of the batch go to global memory for the weight
// gradients; the latents take an Adam step (training) or their gradients are returned.

namespace tct {

struct Smem {
  unsigned char b1[tc::B1_BYTES];      // W1^T (64 x 16): k 0..7, biases (hi, lo) in k 8, 9
  unsigned char b2[tc::B2_BYTES];      // W2^T (64 x 64)
  unsigned char b3[tc::B3_BYTES];      // W3^T (16 x 64), rows >= 7 zero
  unsigned char b2x[64 * 16 * 2];      // (b2_hi, b2_lo) in k 0, 1
  unsigned char b3x[16 * 16 * 2];      // (b3_hi, b3_lo) in k 0, 1
  unsigned char ones[8 * 16 * 2];      // one 8-row group: 1 in columns 0, 1
  unsigned char r3[64 * 16 * 2];       // W3 (64 x 16): B of dY W3^T (k = output, < 7)
  unsigned char r2[64 * 64 * 2];       // W2 (64 x 64): B of dA2 W2^T
  unsigned char r1[16 * 64 * 2];       // W1 (16 x 64), rows >= 8 zero: B of dA1 W1^T
  unsigned char x[128 * 16 * 2];       // latents in k 0..7, ones in k 8, 9
  unsigned char h1[128 * 64 * 2];
  unsigned char h2[128 * 64 * 2];
  unsigned char dy[128 * 16 * 2];      // dY in k 0..6, zeros beyond
  unsigned char da2[128 * 64 * 2];
  unsigned char da1[128 * 64 * 2];
  uint64_t bar;
  uint32_t tmem;
  int abort;
};

constexpr int TMEM_COLS = 64;

}  // namespace tct

// Forward hidden epilogue with the row also written to global memory (the batch's
// activations for the weight gradients): D -> ReLU -> binary16 -> A tile row, grow.
__device__ __forceinline__ void tc_hidden_keep(uint32_t taddr, unsigned char* tile, int row, uint4* grow) {
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
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(w[e]) : "f"(__uint_as_float(r[c + 1])), "f"(__uint_as_float(r[c])));
      }
      const uint4 v = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(tile + tc::off(row, 32 * half + 8 * q, 64)) = v;
      if (grow) grow[4 * half + q] = v;
    }
  }
}

// Backward epilogue: D (64 float32) masked by the row of the forward activation tile
// (kept where the activation is > 0, the ReLU derivative) -> binary16 -> A tile row,
// and to global memory.
__device__ __forceinline__ void tc_masked_keep(uint32_t taddr, const unsigned char* mask, unsigned char* tile,
                                               int row, uint4* grow) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t r[32];
    tc::tmem_ld<32>(taddr + 32 * half, r);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 m = *reinterpret_cast<const uint4*>(mask + tc::off(row, 32 * half + 8 * q, 64));
      const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = 8 * q + 2 * e;
        const float2 h = unpack_h2(mw[e]);
        w[e] = pack_h2(h.x > 0.f ? __uint_as_float(r[c]) : 0.f, h.y > 0.f ? __uint_as_float(r[c + 1]) : 0.f);
      }
      const uint4 v = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(tile + tc::off(row, 32 * half + 8 * q, 64)) = v;
      if (grow) grow[4 * half + q] = v;
    }
  }
}

__global__ void __launch_bounds__(128, 2) k_neural_fwd_bwd_tc(NeuralDev nd, TrainArgs ta, ActBuffers act) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  tct::Smem& s = *reinterpret_cast<tct::Smem*>(dyn);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const uint4* img = reinterpret_cast<const uint4*>(nd.wimg);
    const uint4 z = make_uint4(0, 0, 0, 0);
    tc::stage_fwd_weights(nd, s.b1, s.b2, s.b3, s.b2x, s.b3x, s.ones, tid, 128);
    for (int n = tid; n < 64; n += 128) {      // W3 rows (k = output) for dY W3^T
      *reinterpret_cast<uint4*>(s.r3 + tc::off(n, 0, 16)) = __ldg(img + (nn::I_W3R + n * 8) / 8);
      *reinterpret_cast<uint4*>(s.r3 + tc::off(n, 8, 16)) = z;
    }
    for (int e = tid; e < 64 * 8; e += 128) {  // W2 rows for dA2 W2^T
      const int n = e >> 3, kc = e & 7;
      *reinterpret_cast<uint4*>(s.r2 + tc::off(n, 8 * kc, 64)) = __ldg(img + (nn::I_W2R + n * 72 + 8 * kc) / 8);
    }
    for (int e = tid; e < 16 * 8; e += 128) {  // W1 rows (rows >= 8 zero) for dA1 W1^T
      const int n = e >> 3, kc = e & 7;
      *reinterpret_cast<uint4*>(s.r1 + tc::off(n, 8 * kc, 64)) =
          n < 8 ? __ldg(img + (nn::I_W1R + n * 72 + 8 * kc) / 8) : z;
    }
    *reinterpret_cast<uint4*>(s.x + tc::off(tid, 8, 16)) = make_uint4(0x3C003C00u, 0, 0, 0);
    *reinterpret_cast<uint4*>(s.dy + tc::off(tid, 8, 16)) = z;
  }
  if (tid == 0) {
    s.abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&s.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&s.tmem)), "n"(tct::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s.tmem;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's lanes
  uint32_t parity = 0;
  // make the tiles written so far visible to the tensor cores, let one thread issue
  // the MMAs, wait for them (bounded), and release every thread to read the result
  auto run = [&](auto issue) -> bool {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue();
      tc::commit(&s.bar);
      if (!tc::wait_bar(&s.bar, parity)) s.abort = 1;
    }
    parity ^= 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    return s.abort == 0;
  };
  float loss_part = 0.0f;
  const int64_t ntiles = (ta.batch + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r = tile * 128 + tid;
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
    *reinterpret_cast<uint4*>(s.x + tc::off(tid, 0, 16)) = xh;
    if (live) reinterpret_cast<uint4*>(act.x)[r] = xh;
    // forward
    if (!run([&] { tc::mma(tmem, tc::desc(s.x, 16), tc::desc(s.b1, 16), tc::idesc(128, 64), 0); })) break;
    tc_hidden_keep(trow, s.h1, tid, live ? reinterpret_cast<uint4*>(act.h1) + r * 8 : nullptr);
    if (!run([&] {
          for (int kk = 0; kk < 4; ++kk)
            tc::mma(tmem, tc::desc(s.h1 + kk * 256, 64), tc::desc(s.b2 + kk * 256, 64), tc::idesc(128, 64), kk);
          tc::mma(tmem, tc::desc_rows_repeated(s.ones), tc::desc(s.b2x, 16), tc::idesc(128, 64), 1);
        }))
      break;
    tc_hidden_keep(trow, s.h2, tid, live ? reinterpret_cast<uint4*>(act.h2) + r * 8 : nullptr);
    if (!run([&] {
          for (int kk = 0; kk < 4; ++kk)
            tc::mma(tmem, tc::desc(s.h2 + kk * 256, 64), tc::desc(s.b3 + kk * 256, 64), tc::idesc(128, 16), kk);
          tc::mma(tmem, tc::desc_rows_repeated(s.ones), tc::desc(s.b3x, 16), tc::idesc(128, 16), 1);
        }))
      break;
    {
      uint32_t y[8];
      tc::tmem_ld<8>(trow, y);
      float d[8];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const float e = live ? __uint_as_float(y[k]) - T[k] : 0.0f;
        loss_part = fmaf(e, e, loss_part);
        d[k] = 2.0f * ta.inv_batch * e;
      }
      d[7] = 0.0f;
      const uint4 dh = make_uint4(pack_h2(d[0], d[1]), pack_h2(d[2], d[3]), pack_h2(d[4], d[5]),
                                  pack_h2(d[6], d[7]));
      *reinterpret_cast<uint4*>(s.dy + tc::off(tid, 0, 16)) = dh;
      if (live) reinterpret_cast<uint4*>(act.dy)[r] = dh;
    }
    // backward
    if (!run([&] { tc::mma(tmem, tc::desc(s.dy, 16), tc::desc(s.r3, 16), tc::idesc(128, 64), 0); })) break;
    tc_masked_keep(trow, s.h2, s.da2, tid, live ? reinterpret_cast<uint4*>(act.da2) + r * 8 : nullptr);
    if (!run([&] {
          for (int kk = 0; kk < 4; ++kk)
            tc::mma(tmem, tc::desc(s.da2 + kk * 256, 64), tc::desc(s.r2 + kk * 256, 64), tc::idesc(128, 64), kk);
        }))
      break;
    tc_masked_keep(trow, s.h1, s.da1, tid, live ? reinterpret_cast<uint4*>(act.da1) + r * 8 : nullptr);
    if (!run([&] {
          for (int kk = 0; kk < 4; ++kk)
            tc::mma(tmem, tc::desc(s.da1 + kk * 256, 64), tc::desc(s.r1 + kk * 256, 64), tc::idesc(128, 16), kk);
        }))
      break;
    float dx[8];
    {
      uint32_t q[8];
      tc::tmem_ld<8>(trow, q);
#pragma unroll
      for (int k = 0; k < 8; ++k) dx[k] = __uint_as_float(q[k]);
    }
    if (live) {
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
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
  if (lane == 0) atomicAdd(ta.loss, loss_part * ta.inv_batch);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && s.abort) atomicOr(nd.status, STF_DEV_MMA_TIMEOUT);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "n"(tct::TMEM_COLS));
}

// Weight and bias gradients on the tensor cores.  The batch is the reduction (K)
// dimension, so each chunk of 128 batch rows is staged transposed (feature-major, K
// = batch row) into K-major operand tiles, and two accumulating tcgen05.mma chains per
// chunk sum over the CTA's chunks in tensor memory:
//   D1 (128 x 80)  = [H1^T; H2^T] [dA2^T; dY^T]^T : dW2 = rows 0..63 x cols 0..63,
//                                                    dW3 = rows 64..127 x cols 64..70
//   D2 (128 x 144) = [X^T; 1; 0] [dA1^T; dA2^T; dY^T]^T : dW1 = rows 0..7 x cols 0..63,
//                                                    db1, db2, db3 = row 8
// (the other blocks of the products are not used).  One CTA-wide atomic add per
// gradient entry at the end.
namespace tcw {

struct Smem {
  unsigned char a1[128 * 128 * 2];   // H1^T (rows 0..63), H2^T (rows 64..127)
  unsigned char a2[128 * 128 * 2];   // X^T (rows 0..7), ones (row 8), zeros
  unsigned char b[144 * 128 * 2];    // dA1^T (rows 0..63), dA2^T (64..127), dY^T (128..143)
  uint64_t bar;
  uint32_t tmem;
  int abort;
};

constexpr int TMEM_COLS = 256;   // D1 in columns 0..79, D2 in 96..239

}  // namespace tcw

// Element (m, k) of a K-major operand tile with K = 128.
__device__ __forceinline__ __half* t128(unsigned char* tile, int m, int k) {
  return reinterpret_cast<__half*>(tile + tc::off(m, k, 128));
}

__device__ __forceinline__ void scatter_row(unsigned char* tile, int m0, int k, uint4 v) {
  const __half* h = reinterpret_cast<const __half*>(&v);
#pragma unroll
  for (int e = 0; e < 8; ++e) *t128(tile, m0 + e, k) = h[e];
}

__global__ void __launch_bounds__(128, 2) k_neural_wgrad_tc(ActBuffers act, int64_t batch, float* grads,
                                                            unsigned* status) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  tcw::Smem& s = *reinterpret_cast<tcw::Smem*>(dyn);
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int e = tid; e < 128 * 128 * 2 / 16; e += 128) reinterpret_cast<uint4*>(s.a2)[e] = z;
  }
  __syncthreads();
  *t128(s.a2, 8, tid) = __float2half_rn(1.0f);
  if (tid == 0) {
    s.abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&s.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&s.tmem)), "n"(tcw::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t d1 = s.tmem, d2 = s.tmem + 96;
  uint32_t parity = 0;
  int chunks_done = 0;
  const int64_t nchunks = (batch + 127) / 128;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    // stage this thread's batch row (zeros beyond the batch) as column k = tid
    const int64_t r = c * 128 + tid;
    const bool live = r < batch;
    const uint4 z = make_uint4(0, 0, 0, 0);
    const uint4* h1 = reinterpret_cast<const uint4*>(act.h1) + r * 8;
    const uint4* h2 = reinterpret_cast<const uint4*>(act.h2) + r * 8;
    const uint4* a2 = reinterpret_cast<const uint4*>(act.da2) + r * 8;
    const uint4* a1 = reinterpret_cast<const uint4*>(act.da1) + r * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      scatter_row(s.a1, 8 * q, tid, live ? h1[q] : z);
      scatter_row(s.a1, 64 + 8 * q, tid, live ? h2[q] : z);
      scatter_row(s.b, 8 * q, tid, live ? a1[q] : z);
      scatter_row(s.b, 64 + 8 * q, tid, live ? a2[q] : z);
    }
    scatter_row(s.a2, 0, tid, live ? reinterpret_cast<const uint4*>(act.x)[r] : z);
    scatter_row(s.b, 128, tid, live ? reinterpret_cast<const uint4*>(act.dy)[r] : z);
    scatter_row(s.b, 136, tid, z);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t acc = (chunks_done > 0 || kk > 0) ? 1u : 0u;
        // B rows 64..143 start at the 8th 8-row group (2048 bytes per group at K = 128)
        tc::mma(d1, tc::desc(s.a1 + kk * 256, 128), tc::desc(s.b + 8 * 2048 + kk * 256, 128),
                tc::idesc(128, 80), acc);
        tc::mma(d2, tc::desc(s.a2 + kk * 256, 128), tc::desc(s.b + kk * 256, 128), tc::idesc(128, 144), acc);
      }
      tc::commit(&s.bar);
      if (!tc::wait_bar(&s.bar, parity)) s.abort = 1;   // the tiles are restaged only after this
    }
    parity ^= 1;
    ++chunks_done;
    __syncthreads();
    if (s.abort) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (chunks_done > 0 && !s.abort) {
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    const int m = tid;                      // accumulator row = thread
    uint32_t v[32];
    // D1 columns 0..63: dW2 (rows < 64); columns 64..79: dW3 (rows >= 64)
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      tc::tmem_ld<32>(d1 + lane_off + 32 * cb, v);
      if (m < 64)
        for (int n = 0; n < 32; ++n) atomicAdd(grads + nn::P_W2 + m * 64 + 32 * cb + n, __uint_as_float(v[n]));
    }
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      tc::tmem_ld<8>(d1 + lane_off + 64 + 8 * cb, v);
      if (m >= 64)
        for (int o = 0; o < 8 && 8 * cb + o < 7; ++o)
          atomicAdd(grads + nn::P_W3 + (m - 64) * 7 + 8 * cb + o, __uint_as_float(v[o]));
    }
    // D2 columns 0..63: dW1 (rows < 8), db1 (row 8); 64..127: db2 (row 8); 128..134: db3
#pragma unroll
    for (int cb = 0; cb < 4; ++cb) {
      tc::tmem_ld<32>(d2 + lane_off + 32 * cb, v);
      for (int n = 0; n < 32; ++n) {
        const int col = 32 * cb + n;
        if (m < 8 && col < 64) atomicAdd(grads + nn::P_W1 + m * 64 + col, __uint_as_float(v[n]));
        if (m == 8) atomicAdd(grads + (col < 64 ? nn::P_B1 + col : nn::P_B2 + col - 64), __uint_as_float(v[n]));
      }
    }
    tc::tmem_ld<8>(d2 + lane_off + 128, v);
    if (m == 8)
      for (int o = 0; o < 7; ++o) atomicAdd(grads + nn::P_B3 + o, __uint_as_float(v[o]));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && s.abort) atomicOr(status, STF_DEV_MMA_TIMEOUT);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "n"(tcw::TMEM_COLS));
}

static cudaError_t launch_wgrad_tc(const ActBuffers& act, int64_t batch, float* grads, unsigned* status,
                                   cudaStream_t s) {
  const int smem = (int)sizeof(tcw::Smem) + 1024;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_neural_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = (batch + 127) / 128;
  // a few chunks per CTA, so that the accumulators' atomic flush is amortised
  const int64_t want = (nchunks + 3) / 4;
  const int grid = (int)(want < (int64_t)sms ? (want < 1 ? 1 : want) : (int64_t)sms);
  k_neural_wgrad_tc<<<grid, 128, smem, s>>>(act, batch, grads, status);
  return cudaGetLastError();
}

// Launch of the tcgen05 forward and backward over a batch.
static cudaError_t launch_fwd_bwd_tc(const NeuralDev& nd, const TrainArgs& ta, const ActBuffers& act,
                                     cudaStream_t s) {
  const int smem = (int)sizeof(tct::Smem) + 1024;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_neural_fwd_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (ta.batch + 127) / 128;
  const int grid = (int)(ntiles < (int64_t)sms * 2 ? ntiles : (int64_t)sms * 2);
  k_neural_fwd_bwd_tc<<<grid, 128, smem, s>>>(nd, ta, act);
  return cudaGetLastError();
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
      cudaFuncSetAttribute(k_neural_stochastic_tc<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      cudaFuncSetAttribute(k_neural_stochastic_tc<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr = true;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t pairs = ((a.n + tc::ROWS - 1) / tc::ROWS + 1) / 2;   // two tiles per CTA pass
    const int grid = (int)(pairs < (int64_t)sms * 4 ? pairs : (int64_t)sms * 4);
    if (a.perm == nullptr && a.taps == nullptr) k_neural_stochastic_tc<F, true><<<grid, 256, smem, s>>>(nd, a);
    else k_neural_stochastic_tc<F, false><<<grid, 256, smem, s>>>(nd, a);
    return cudaGetLastError();
  }
  else if (op == OP_DETERMINISTIC) {
    const int smem = (int)sizeof(tcd::Smem) + 1024;
    static bool attr_d = false;
    if (!attr_d) {
      cudaFuncSetAttribute(k_neural_deterministic_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr_d = true;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int parts = (a.lod != nullptr && nd.nlev > 1 && a.level_mode != STF_LEVEL_NEAREST) ? 2 : 1;
    const int q = 128 / (parts * Filter<F>::T * Filter<F>::T);
    const int64_t ntiles = (a.n + q - 1) / q;
    const int grid = (int)(ntiles < (int64_t)sms * 6 ? ntiles : (int64_t)sms * 6);
    k_neural_deterministic_tc<F><<<grid, 128, smem, s>>>(nd, a);
  }
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
    e = launch_fwd_bwd_tc(t->neural, ta, act, s);
    if (e == cudaSuccess) e = launch_wgrad_tc(act, batch, t->n_grads, t->d_status, s);
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
    e = launch_fwd_bwd_tc(t->neural, ta, act, s);
    if (e == cudaSuccess) e = launch_wgrad_tc(act, cfg->batch, t->n_grads, t->d_status, s);
    if (e != cudaSuccess) break;
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
