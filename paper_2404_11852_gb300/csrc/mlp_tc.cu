// Feature Gathering + Feature Computation on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One persistent CTA per SM holds the MLP weights in shared memory (BF16, ~48 KB) and runs G
// independent tile pipelines ("groups" of 4 warps = 128 threads, one thread per sample row), so
// that while one group gathers features or runs its epilogue on CUDA cores, another group's MMAs
// keep the tensor pipe busy.  Per 128-sample tile a group runs
//   gather   : staged brick (TMA, one copy per brick visit) -> trilinear -> BF16 row of A
//   layer 1  : D = A[128x48] W1^T      (tcgen05.mma kind::f16, FP32 accumulators in TMEM)
//   epilogue : +b1, ReLU, BF16 (cvt.rn.relu.bf16x2)  -> A[128x128]   (A reused in place)
//   layer 2  : D = A W2^T  -> +b2, ReLU, BF16 -> A3 in TMEM (tcgen05.st)
//   layer 3  : D = A3 W3^T (A from TMEM, N padded 3 -> 16) -> +b3, sigmoid -> (c, w) record
// Each group owns 128 TMEM columns (D of layers 1 and 2 reuses them: every accumulator is read
// back before the next MMA is issued; the layer-2 epilogue writes its BF16 output back into the
// first 64 of them, where layer 3 reads its A operand, so that activation never touches shared
// memory) and synchronises on its own named barrier.  The elected
// thread of a group issues the MMAs and commits them to the group's mbarrier.
// Operands use the canonical K-major, no-swizzle layout: 8-row x 16-byte core matrices stored as
// 128 contiguous bytes, K-adjacent core matrices 128 B apart (leading byte offset) and 8-row groups
// K*16 bytes apart (stride byte offset).  A group's activation buffer keeps the K = 144 stride for
// both layers that read it, so layer 1's 48 input columns and the constant columns 128..143 of
// layer 2 never overlap and the constants are written once per CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace cicero {

namespace tc {

constexpr int kK1 = kMaxIn;            // 48: layer-1 K (input padded; column in_dim carries a 1 for b1)
constexpr int kK2 = kHidden + 16;      // 144: layer-2 K (column 128 carries a 1 for b2)
constexpr int kN3 = 16;                // layer-3 N padded to the smallest M=128 MMA width
constexpr int kGT = 128;               // threads per group
constexpr int kMaxGroups = 4;
constexpr uint32_t kTmemCols = 512;    // all of an SM's tensor memory; 128 columns per group
constexpr uint32_t kL3Col = 64;        // layer-3 accumulator columns [64, 80) of a group (A sits in [0, 64))
constexpr int kActBytes = kTile * kK2 * 2;

struct Smem {
  static constexpr int w1 = 0;                                 // [128][48]  bf16
  static constexpr int w2 = w1 + kHidden * kK1 * 2;            // [128][144] bf16 (column 128 = b2)
  static constexpr int w3 = w2 + kHidden * kK2 * 2;            // [16][128]  bf16
  static constexpr int b1 = w3 + kN3 * kHidden * 2;            // [128] f32
  static constexpr int b2 = b1 + kHidden * 4;                  // [128] f32
  static constexpr int b3 = b2 + kHidden * 4;                  // [4] f32
  static constexpr int bars = ((b3 + 16 + 127) / 128) * 128;   // per group 2 mbarriers; TMEM address at +96
  static constexpr int geo = bars + 128;                       // batch: geometry of the current job
  static constexpr int groups = geo + 128;                     // per group: activations, then brick tile
  static_assert(sizeof(GridGeo) <= 128, "job geometry slot");
  static_assert(groups % 128 == 0 && w2 % 16 == 0 && w3 % 16 == 0, "alignment");
};

__host__ __device__ constexpr int align128(int x) { return (x + 127) / 128 * 128; }
__host__ __device__ constexpr int group_bytes(int box_bytes) { return kActBytes + align128(box_bytes); }

// named barrier of one group (ids 1..4; id 0 is __syncthreads)
__device__ __forceinline__ void gsync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kGT) : "memory");
}
__device__ __forceinline__ bool gsync_and(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(g + 1), "r"(kGT)
      : "memory");
  return r != 0;
}

__device__ void load_weights(char* sm, const MlpPtrs& m) {
  for (int i = threadIdx.x; i < kHidden * (kK1 / 8); i += blockDim.x) {
    const int n = i / (kK1 / 8), k0 = (i % (kK1 / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = k0 + j;
      v[j] = k < m.in_dim ? m.w1[n * m.in_dim + k] : (k == m.in_dim ? m.b1[n] : 0.0f);  // b1 rides on x[in_dim] = 1
    }
    store_chunk(sm + Smem::w1, n, k0, kK1, v);
  }
  for (int i = threadIdx.x; i < kHidden * (kK2 / 8); i += blockDim.x) {
    const int n = i / (kK2 / 8), k0 = (i % (kK2 / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = k0 + j;
      v[j] = k < kHidden ? m.w2[n * kHidden + k] : (k == kHidden ? m.b2[n] : 0.0f);  // b2 rides on a 1 column
    }
    store_chunk(sm + Smem::w2, n, k0, kK2, v);
  }
  for (int i = threadIdx.x; i < kN3 * (kHidden / 8); i += blockDim.x) {
    const int n = i / (kHidden / 8), k0 = (i % (kHidden / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = n < 3 ? m.w3[n * kHidden + k0 + j] : 0.0f;
    store_chunk(sm + Smem::w3, n, k0, kHidden, v);
  }
  float* b1 = (float*)(sm + Smem::b1);
  float* b2 = (float*)(sm + Smem::b2);
  float* b3 = (float*)(sm + Smem::b3);
  for (int i = threadIdx.x; i < kHidden; i += blockDim.x) {
    b1[i] = m.in_dim < kK1 ? 0.0f : m.b1[i];  // folded into W1 unless the input fills all 48 columns
    b2[i] = 0.0f;                             // folded into W2 (column 128)
  }
  if (threadIdx.x < 4) b3[threadIdx.x] = threadIdx.x < 3 ? m.b3[threadIdx.x] : 0.0f;
}

struct Group {
  int g;            // group index
  int m;            // row (thread) inside the group
  char* act;        // activation operand (A), 32 KB
  char* tile;       // staged brick
  uint64_t* bar_tma;
  uint64_t* bar_mma;
  uint32_t tmem;    // first of the group's 128 TMEM columns
  uint32_t ph_tma, ph_mma;
};

// Issue one layer (elected thread) and wait for it (whole group).  False on timeout.
// Layers 0 and 1 read A from shared memory and accumulate into the group's columns [0, 128);
// layer 2 reads A from the group's TMEM columns [0, 64) and accumulates into [64, 80).
__device__ __forceinline__ bool run_layer(char* sm, Group& G, int layer, uint32_t* err) {
  gsync(G.g);
  if (G.m == 0) {
    fence_after();
    if (layer < 2) {
      // descriptors built once; the next K step of 16 is 256 bytes on, +16 in the address field.
      // A always has the K = 144 row-group stride (layer 1's A fills its first 48 columns).
      const uint64_t da = smem_desc(smem_u32(G.act), 128u, kK2 * 16);
      const uint64_t db = smem_desc(smem_u32(sm + (layer == 0 ? Smem::w1 : Smem::w2)), 128u,
                                    (uint32_t)(layer == 0 ? kK1 : kK2) * 16);
      const uint32_t idesc = idesc_bf16(kHidden);
      if (layer == 0) {
#pragma unroll
        for (int s = 0; s < kK1 / 16; s++) mma_bf16(G.tmem, da + 16u * s, db + 16u * s, idesc, s > 0 ? 1u : 0u);
      } else {
#pragma unroll
        for (int s = 0; s < kK2 / 16; s++) mma_bf16(G.tmem, da + 16u * s, db + 16u * s, idesc, s > 0 ? 1u : 0u);
      }
    } else {
      const uint64_t db = smem_desc(smem_u32(sm + Smem::w3), 128u, kHidden * 16);
#pragma unroll
      for (int s = 0; s < kHidden / 16; s++)
        mma_bf16_ta(G.tmem + kL3Col, G.tmem + 8u * s, db + 16u * s, idesc_bf16(kN3), s > 0 ? 1u : 0u);
    }
    mma_commit(G.bar_mma);
  }
  const bool ok = gsync_and(G.g, mbar_wait(G.bar_mma, G.ph_mma, err));
  if (ok) G.ph_mma ^= 1u;  // on a timeout the phase stays, so a final bounded wait watches the right one
  fence_after();
  return ok;
}

// ReLU of the 128 accumulator columns (+ bias when it could not be folded into the MMA) -> BF16
// K-major rows of A (K = 144: column 128 is the constant 1 that multiplies b2 and 129..143 are
// zero; the CTA prologue writes those once, and no other store reaches them).
__device__ __forceinline__ void epilogue_hidden(const Group& G, const float* bias) {
  const uint32_t taddr = G.tmem + ((uint32_t)((G.m >> 5) * 32) << 16);
#pragma unroll 1
  for (int cc = 0; cc < kHidden / 64; cc++) {
    float v[64];
    tmem_ld<64>(taddr + cc * 64, v);  // one TMEM round trip per 64 columns
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const float* x = v + q * 8;
      float y[8];
      if (bias) {
        const float4* b4 = reinterpret_cast<const float4*>(bias + cc * 64 + q * 8);
        add2(x, b4[0], y);
        add2(x + 4, b4[1], y + 4);
      } else {
#pragma unroll
        for (int j = 0; j < 8; j++) y[j] = x[j];
      }
      uint4 o;
      o.x = pack_bf16_relu(y[0], y[1]);
      o.y = pack_bf16_relu(y[2], y[3]);
      o.z = pack_bf16_relu(y[4], y[5]);
      o.w = pack_bf16_relu(y[6], y[7]);
      *reinterpret_cast<uint4*>(G.act + kmaj_off(G.m, cc * 64 + q * 8, kK2)) = o;
    }
  }
  fence_proxy_async();
  fence_before();
}

// Layer-2 epilogue: ReLU of the 128 accumulator columns -> BF16, written back into the group's
// TMEM columns [0, 64) as the A operand of layer 3 (b2 rides on the MMA).  Chunk c of 64 FP32
// columns becomes BF16 columns [32c, 32c + 32), which chunk 0 has already read.
__device__ __forceinline__ void epilogue_to_tmem(const Group& G) {
  const uint32_t taddr = G.tmem + ((uint32_t)((G.m >> 5) * 32) << 16);
#pragma unroll 1
  for (int cc = 0; cc < kHidden / 64; cc++) {
    float v[64];
    tmem_ld<64>(taddr + cc * 64, v);
    uint32_t o[32];
#pragma unroll
    for (int j = 0; j < 32; j++) o[j] = pack_bf16_relu(v[2 * j], v[2 * j + 1]);
    tmem_st32(taddr + cc * 32, o);
  }
  tmem_wait_st();
  fence_before();
}

// The three layers of a tile whose A (K = 48 layout) has been written and proxy-fenced by every
// thread of the group.  c receives this thread's colour.  False on timeout.
__device__ __forceinline__ float sigmoid_fast(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

__device__ __forceinline__ bool mlp_tile(char* sm, Group& G, uint32_t* err, float c[3], bool folded_b1) {
  if (!run_layer(sm, G, 0, err)) return false;
  epilogue_hidden(G, folded_b1 ? nullptr : (const float*)(sm + Smem::b1));
  if (!run_layer(sm, G, 1, err)) return false;
  epilogue_to_tmem(G);
  if (!run_layer(sm, G, 2, err)) return false;
  float v[16];
  tmem_ld<16>(G.tmem + kL3Col + ((uint32_t)((G.m >> 5) * 32) << 16), v);
  const float* b3 = (const float*)(sm + Smem::b3);
  c[0] = sigmoid_fast(v[0] + b3[0]);
  c[1] = sigmoid_fast(v[1] + b3[1]);
  c[2] = sigmoid_fast(v[2] + b3[2]);
  fence_before();
  return true;
}

// View-direction encoding with the fast hardware sine/cosine (|d| <= 1, error ~1e-6, far below
// the BF16 rounding of the MLP input) and the double-angle recurrence.
template <int NF>
__device__ __forceinline__ void encode_dir_fast(const float d[3], int n_freq_rt, float* x) {
  const int n_freq = NF ? NF : n_freq_rt;
  float s[3], c[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    x[a] = d[a];
    __sincosf(d[a], &s[a], &c[a]);
  }
#pragma unroll
  for (int k = 0; k < n_freq; k++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      x[3 + 6 * k + a] = s[a];
      x[3 + 6 * k + 3 + a] = c[a];
      const float s2 = 2.0f * s[a] * c[a];
      c[a] = 1.0f - 2.0f * s[a] * s[a];
      s[a] = s2;
    }
  }
}

template <typename T, int CC>
__device__ __forceinline__ void tri_tile(const T* tile, int vb, int vx, int Cr, const int l[3], const float f[3],
                                         float* out) {
  const int C = CC ? CC : Cr;
  const float fx = f[0], fy = f[1], fz = f[2];
  for (int c = 0; c < C; c++) out[c] = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int x = l[0] + (q & 1), y = l[1] + ((q >> 1) & 1), z = l[2] + (q >> 2);
    const float wq = ((q & 1) ? fx : 1.f - fx) * (((q >> 1) & 1) ? fy : 1.f - fy) * ((q >> 2) ? fz : 1.f - fz);
    const T* v = tile + ((size_t)(z * vb + y) * vx + x) * C;
    if constexpr (CC == 12 && sizeof(T) == 2) {
      continue;  // handled by tri_tile_h2
    } else if constexpr (CC == 12 && sizeof(T) == 4) {
      const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
      for (int u = 0; u < 3; u++) {
        float4 a = v4[u];
        out[4 * u + 0] += wq * a.x;
        out[4 * u + 1] += wq * a.y;
        out[4 * u + 2] += wq * a.z;
        out[4 * u + 3] += wq * a.w;
      }
    } else {
      for (int c = 0; c < C; c++) {
        float vv;
        if constexpr (sizeof(T) == 4) vv = v[c];
        else vv = __half2float(v[c]);
        out[c] += wq * vv;
      }
    }
  }
}

// FP16 grids, 12 channels: the eight corners accumulated in half2 (6 HFMA2 per corner).  The
// accumulation error (~1e-3 worst case, features |f| <= 1) stays below the BF16 rounding of the
// MLP input that follows.
__device__ __forceinline__ void tri_tile_h2(const __half* tile, int vb, int vx, const int l[3], const float f[3],
                                            float* out) {
  __half2 acc[6];
#pragma unroll
  for (int u = 0; u < 6; u++) acc[u] = __float2half2_rn(0.0f);
  const float fx = f[0], fy = f[1], fz = f[2];
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int x = l[0] + (q & 1), y = l[1] + ((q >> 1) & 1), z = l[2] + (q >> 2);
    const float wq = ((q & 1) ? fx : 1.f - fx) * (((q >> 1) & 1) ? fy : 1.f - fy) * ((q >> 2) ? fz : 1.f - fz);
    const __half2 w2 = __float2half2_rn(wq);
    const uint2* v2 = reinterpret_cast<const uint2*>(tile + ((size_t)(z * vb + y) * vx + x) * 12);
#pragma unroll
    for (int u = 0; u < 3; u++) {
      uint2 a = v2[u];
      acc[2 * u] = __hfma2(w2, *reinterpret_cast<__half2*>(&a.x), acc[2 * u]);
      acc[2 * u + 1] = __hfma2(w2, *reinterpret_cast<__half2*>(&a.y), acc[2 * u + 1]);
    }
  }
#pragma unroll
  for (int u = 0; u < 6; u++) {
    const float2 fv = __half22float2(acc[u]);
    out[2 * u] = fv.x;
    out[2 * u + 1] = fv.y;
  }
}

__device__ __forceinline__ void tmem_alloc_all(uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

__device__ __forceinline__ void tmem_free_all(uint32_t tmem) {
  fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// CTA prologue shared by the kernels: weights (unless NULL), barriers, TMEM; returns the group handle.
__device__ __forceinline__ Group setup(char* sm, const MlpPtrs* mlp, int groups, int box_bytes) {
  uint64_t* bars = (uint64_t*)(sm + Smem::bars);
  uint32_t* tslot = (uint32_t*)(sm + Smem::bars + 96);
  if (mlp) load_weights(sm, *mlp);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * groups; i++) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  fence_proxy_async();
  tmem_alloc_all(tslot);
  fence_before();
  __syncthreads();
  fence_after();
  Group G;
  G.g = threadIdx.x / kGT;
  G.m = threadIdx.x % kGT;
  G.act = sm + Smem::groups + G.g * group_bytes(box_bytes);
  G.tile = G.act + kActBytes;
  G.bar_tma = &bars[2 * G.g];
  G.bar_mma = &bars[2 * G.g + 1];
  G.tmem = *tslot + (uint32_t)(G.g * 128);
  G.ph_tma = 0;
  G.ph_mma = 0;
  // the constant columns 128..143 of this row of A: 1 (times b2), then zeros
  *reinterpret_cast<uint4*>(G.act + kmaj_off(G.m, kHidden, kK2)) = make_uint4(0x3f80u, 0u, 0u, 0u);  // bf16 1.0
  *reinterpret_cast<uint4*>(G.act + kmaj_off(G.m, kHidden + 8, kK2)) = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async();
  return G;
}

}  // namespace tc

// Features of the multiresolution hash encoding at world position p: per level, the box mapped
// onto res cells per axis, the 8 corner entries (dense index where the level's vertices fit the
// table, else the spatial hash (x * 1 xor y * 2654435761 xor z * 805459861) mod T) interpolated
// trilinearly; two features per level, levels concatenated.  The tables are read straight from
// global memory (they fit in L2).
template <int LL, typename T>
__device__ __forceinline__ void hash_features(const HashGeo& h, const float p[3], float* x) {
  const int L = LL ? LL : h.levels;
  float pn[3];
#pragma unroll
  for (int a = 0; a < 3; a++) pn[a] = __saturatef(__fmul_rn(__fsub_rn(p[a], h.amin[a]), h.inv_ext[a]));
#pragma unroll
  for (int l = 0; l < (LL ? LL : kMaxHashLevels); l++) {
    if (!LL && l >= L) break;
    const int N = h.res[l];
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float gx = pn[a] * (float)N;
      const int i = min((int)gx, N - 1);
      i0[a] = i;
      f[a] = gx - (float)i;
    }
    const uint32_t s1 = (uint32_t)N + 1u;
    const bool dense = (h.dense >> l) & 1u;
    const size_t base = (size_t)l * (h.mask + 1u);
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const uint32_t cx = (uint32_t)i0[0] + (q & 1), cy = (uint32_t)i0[1] + ((q >> 1) & 1),
                     cz = (uint32_t)i0[2] + (q >> 2);
      const uint32_t idx = dense ? cx + s1 * (cy + s1 * cz) : ((cx ^ (cy * 2654435761u) ^ (cz * 805459861u)) & h.mask);
      const float w = ((q & 1) ? f[0] : 1.f - f[0]) * (((q >> 1) & 1) ? f[1] : 1.f - f[1]) *
                      ((q >> 2) ? f[2] : 1.f - f[2]);
      float2 v;
      if constexpr (sizeof(T) == 2) v = __half22float2(__ldg((const __half2*)h.table + base + idx));
      else v = __ldg((const float2*)h.table + base + idx);
      a0 += w * v.x;
      a1 += w * v.y;
    }
    x[2 * l] = a0;
    x[2 * l + 1] = a1;
  }
}

// One group's tiles [t_begin, t_end) through gather + MLP, software-pipelined: while layer 3 of
// tile t runs on the tensor cores (its A operand is in TMEM, so shared memory is free), the group
// gathers tile t + 1 into its A buffer.  `loaded` is the brick held in the group's tile buffer
// (global brick ids, so it stays valid across calls).  Returns false if a bounded wait ran out;
// with alive false on entry it does nothing.
// The grid's geometry `g` and the MLP dimensions are read where they live (kernel parameters for
// one grid, the job table for a batch); `map` is the generic address of the feature grid's tensor map.
// With HASH, the features come from the hash encoding `hg` instead of staged bricks (no TMA).
template <typename T, int CC, int NF, bool HASH = false>
__device__ __forceinline__ bool gather_tiles(char* sm, tc::Group& G, const GridGeo& g, const CUtensorMap* map,
                                             int in_dim, int n_freq, int vb, int vx, int box_bytes, const RenderWs& w,
                                             long long t_begin, long long t_end, int& loaded, bool alive,
                                             const HashGeo* hg = nullptr) {
  using namespace tc;
  if (!alive) return false;
  const int B = g.brick, C = CC ? CC : g.C, m = G.m;
  const T* tile = (const T*)G.tile;
  // Tile descriptors run two tiles ahead of the gather and record payloads one tile ahead, and a
  // payload load is never conditional on loaded data (rows past a tile's count re-read its last
  // record), so no load of this pipeline waits on another.
  const uint4 none = make_uint4(0u, 0u, 0u, 0u);
  auto payload = [&](const uint4& d, float4& a, float4& q) {
    const uint32_t row = d.x + min((uint32_t)m, (d.y & 0xFFu) - 1u);  // every listed tile has >= 1 record
    a = w.srt[row].pw;
    q = w.srt[row].qd;
  };
  auto tma_brick = [&](const uint4& d) {
    mbar_expect_tx(G.bar_tma, (uint32_t)box_bytes);
    tma_load_3d(G.tile, map, (int)(d.w & 0xFFFFu) * B * C, (int)(d.w >> 16) * B, (int)((d.y >> 8) & 0x1FFFu) * B,
                G.bar_tma);
  };
  // tg: the tile gathered in iteration ti (= tile ti + 1), tg1 the one after it
  uint4 tg = t_begin < t_end ? w.tile[t_begin] : none;
  uint4 tg1 = t_begin + 1 < t_end ? w.tile[t_begin + 1] : none;
  float4 gpw = make_float4(0.f, 0.f, 0.f, 0.f), gdir = make_float4(0.f, 0.f, 0.f, 1.f);
  if (t_begin < t_end) payload(tg, gpw, gdir);
  // the tile whose MLP runs in iteration ti: this row's record (kNoRecord past the tile's count)
  // and weight; then the same for the previous tile with its layer-3 output, written out once the
  // next tile's layer 1 is issued
  constexpr uint32_t kNoRecord = 0xFFFFFFFFu;
  uint32_t csid = kNoRecord, osid = kNoRecord;
  float cw = 0.0f, ow = 0.0f;
  float o3[3] = {0.f, 0.f, 0.f};
  const float* b3 = (const float*)(sm + Smem::b3);
  auto write_out = [&]() {
    if (osid != kNoRecord)
      w.rec_c[osid] = make_float4(sigmoid_fast(o3[0] + b3[0]), sigmoid_fast(o3[1] + b3[1]),
                                  sigmoid_fast(o3[2] + b3[2]), ow);
    osid = kNoRecord;
  };
  bool tma_pending = false, mma_pending = false;
  if (!HASH && t_begin < t_end) {
    if (m == 0) tma_brick(tg);
    loaded = (int)tg.z;
    tma_pending = true;
  }
  for (long long ti = t_begin - 1; ti < t_end; ti++) {
    const bool run = ti >= t_begin, gather = ti + 1 < t_end;
    if (run) {
      // layer 1 of tile ti (its A was gathered in the previous iteration)
      gsync(G.g);
      if (m == 0) {
        fence_after();
        const uint64_t da = smem_desc(smem_u32(G.act), 128u, kK2 * 16);
        const uint64_t db = smem_desc(smem_u32(sm + Smem::w1), 128u, kK1 * 16);
#pragma unroll
        for (int s2 = 0; s2 < kK1 / 16; s2++)
          mma_bf16(G.tmem, da + 16u * s2, db + 16u * s2, idesc_bf16(kHidden), s2 > 0 ? 1u : 0u);
        mma_commit(G.bar_mma);
      }
      mma_pending = true;
      // every thread is done with the staged brick: copy the next tile's brick if it differs
      if (!HASH && gather && (int)tg.z != loaded) {
        if (m == 0) tma_brick(tg);
        loaded = (int)tg.z;
        tma_pending = true;
      }
      write_out();  // the previous tile's colours, while layer 1 runs
      alive = gsync_and(G.g, mbar_wait(G.bar_mma, G.ph_mma, &w.hdr[0]));
      fence_after();
      if (!alive) break;
      G.ph_mma ^= 1u;
      mma_pending = false;
      epilogue_hidden(G, in_dim < kK1 ? nullptr : (const float*)(sm + Smem::b1));
      mma_pending = true;
      if (!(alive = run_layer(sm, G, 1, &w.hdr[0]))) break;
      mma_pending = false;
      epilogue_to_tmem(G);
      // layer 3 of tile ti, not waited for yet
      gsync(G.g);
      if (m == 0) {
        fence_after();
        const uint64_t db = smem_desc(smem_u32(sm + Smem::w3), 128u, kHidden * 16);
#pragma unroll
        for (int s2 = 0; s2 < kHidden / 16; s2++)
          mma_bf16_ta(G.tmem + kL3Col, G.tmem + 8u * s2, db + 16u * s2, idesc_bf16(kN3), s2 > 0 ? 1u : 0u);
        mma_commit(G.bar_mma);
      }
      mma_pending = true;
    }
    // payload of the tile after the one gathered now, and the descriptor after that
    float4 npw = gpw, ndir = gdir;
    uint4 tg2 = none;
    if (ti + 2 < t_end) payload(tg1, npw, ndir);
    if (ti + 3 < t_end) tg2 = w.tile[ti + 3];
    if (gather) {
      if (tma_pending) {
        alive = gsync_and(G.g, mbar_wait(G.bar_tma, G.ph_tma, &w.hdr[0]));
        if (!alive) break;
        G.ph_tma ^= 1u;
        tma_pending = false;
      }
      const int mcnt = (int)(tg.y & 0xFFu);
      const int bx = (int)(tg.w & 0xFFFFu), by = (int)(tg.w >> 16), bz = (int)((tg.y >> 8) & 0x1FFFu);
      float x[kK1];
#pragma unroll
      for (int j = 0; j < kK1; j++) x[j] = 0.0f;
      if (m < mcnt) {
        const float p[3] = {gpw.x, gpw.y, gpw.z};
        if constexpr (HASH) {
          hash_features<CC / 2, T>(*hg, p, x);
        } else {
          int l[3];
          float f[3];
          bool ok = true;
#pragma unroll
          for (int a = 0; a < 3; a++) {
            const float ga = __fmul_rn(__fsub_rn(p[a], g.amin[a]), g.inv_h[a]);
            int i = (int)floorf(ga);
            if (i > g.n[a] - 2) i = g.n[a] - 2;
            f[a] = __fsub_rn(ga, (float)i);
            l[a] = i - (a == 0 ? bx : a == 1 ? by : bz) * B;
            ok = ok && l[a] >= 0 && l[a] < B;
          }
          if (!ok)
            set_err(&w.hdr[0], kErrInternal);
          else if constexpr (CC == 12 && sizeof(T) == 2)
            tri_tile_h2((const __half*)tile, vb, vx, l, f, x);
          else
            tri_tile<T, CC>(tile, vb, vx, C, l, f, x);
        }
        const float d[3] = {gdir.y, gdir.z, gdir.w};
        encode_dir_fast<NF>(d, n_freq, x + C);
        if (in_dim < kK1) x[CC && NF ? (CC + 3 + 6 * NF) % kK1 : in_dim % kK1] = 1.0f;  // folded layer-1 bias
      }
#pragma unroll
      for (int k0 = 0; k0 < kK1; k0 += 8) store_chunk(G.act, m, k0, kK2, x + k0);
      fence_proxy_async();
    }
    if (run) {
      alive = gsync_and(G.g, mbar_wait(G.bar_mma, G.ph_mma, &w.hdr[0]));
      fence_after();
      if (!alive) break;
      G.ph_mma ^= 1u;
      mma_pending = false;
      float v[16];
      tmem_ld<16>(G.tmem + kL3Col + ((uint32_t)((m >> 5) * 32) << 16), v);
      fence_before();
      o3[0] = v[0];
      o3[1] = v[1];
      o3[2] = v[2];
      osid = csid;
      ow = cw;
    }
    // the gathered tile is the next one through the MLP
    csid = m < (int)(tg.y & 0xFFu) ? __float_as_uint(gdir.x) : kNoRecord;
    cw = gpw.w;
    tg = tg1;
    tg1 = tg2;
    gpw = npw;
    gdir = ndir;
  }
  if (alive) write_out();
  if (tma_pending) mbar_wait(G.bar_tma, G.ph_tma, &w.hdr[0]);  // a copy may still be landing (bounded)
  if (mma_pending) mbar_wait(G.bar_mma, G.ph_mma, &w.hdr[0]);  // MMAs may still be running (bounded)
  return alive;
}

// The persistent gather + MLP kernel of the BF16 path for one grid (launched with 128 * groups
// threads): each CTA takes a contiguous range of tiles, split evenly among its groups.
template <typename T, int CC, int NF>
__global__ void __launch_bounds__(512, 1) k_gather_mlp_bf16(GridGeo g, int S, MlpPtrs mlp, RenderWs w,
                                                            const __grid_constant__ CUtensorMap fmap, int vb, int vx,
                                                            int box_bytes, int groups) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  Group G = setup(sm, &mlp, groups, box_bytes);
  const uint32_t tmem_base = G.tmem - (uint32_t)(G.g * 128);
  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t c_begin = blockIdx.x * per, c_end = min(n_tiles, c_begin + per);
  const uint32_t span = c_end > c_begin ? c_end - c_begin : 0;
  const long long t_begin = c_begin + (span * G.g) / groups, t_end = c_begin + (span * (G.g + 1)) / groups;
  int loaded = -1;
  gather_tiles<T, CC, NF>(sm, G, g, &fmap, mlp.in_dim, mlp.n_freq, vb, vx, box_bytes, w, t_begin, t_end, loaded, true);
  tmem_free_all(tmem_base);
}

// The hash-grid workload: the single-grid kernel with features from the hash encoding (every level
// gathered from global memory / L2; no brick staging).
template <typename T, int CC, int NF>
__global__ void __launch_bounds__(512, 1) k_gather_mlp_bf16_hash(GridGeo g, MlpPtrs mlp, RenderWs w,
                                                                 const __grid_constant__ HashGeo hg, int groups) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  Group G = setup(sm, &mlp, groups, 0);
  const uint32_t tmem_base = G.tmem - (uint32_t)(G.g * 128);
  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t c_begin = blockIdx.x * per, c_end = min(n_tiles, c_begin + per);
  const uint32_t span = c_end > c_begin ? c_end - c_begin : 0;
  const long long t_begin = c_begin + (span * G.g) / groups, t_end = c_begin + (span * (G.g + 1)) / groups;
  int loaded = -1;
  gather_tiles<T, CC, NF, true>(sm, G, g, nullptr, mlp.in_dim, mlp.n_freq, 0, 0, 0, w, t_begin, t_end, loaded, true,
                                &hg);
  tmem_free_all(tmem_base);
}

// The batched version, job-major: the jobs are taken one after the other (in table order, where
// jobs that share MLP weights are adjacent), and every CTA takes its contiguous share of each job's
// tiles, split evenly among its groups, as a launch per job would; so at any moment the GPU works on
// one or two jobs' grids, which keeps their bricks in L2.  The CTA stages each job's geometry in
// shared memory and loads the job's MLP weights when they differ from the ones there.
template <typename T, int CC, int NF>
__global__ void __launch_bounds__(512, 1) k_gather_mlp_bf16_batch(const JobDesc* __restrict__ jobs, int n_jobs,
                                                                  RenderWs w, int vb, int vx, int box_bytes,
                                                                  int groups) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  Group G = setup(sm, nullptr, groups, box_bytes);
  const uint32_t tmem_base = G.tmem - (uint32_t)(G.g * 128);
  GridGeo& geo = *(GridGeo*)(sm + Smem::geo);  // the current job's geometry, read by every group
  const MlpPtrs* cur = nullptr;
  int loaded = -1;
  bool alive = true;
  for (int j = 0; j < n_jobs; j++) {
    const JobDesc& J = jobs[j];
    const long long j0 = w.tile_off[J.brick_base], j1 = w.tile_off[J.brick_base + J.nb];
    const long long per = (j1 - j0 + gridDim.x - 1) / gridDim.x;
    const long long a = min(j1, j0 + (long long)blockIdx.x * per), b = min(j1, a + per);
    if (b <= a) continue;
    __syncthreads();  // every group is done with the previous job's geometry (and weights)
    if (threadIdx.x == 0) geo = J.geo;
    if (!cur || !same_mlp(*cur, J.mlp)) {
      load_weights(sm, J.mlp);
      fence_proxy_async();
      cur = &J.mlp;
    }
    __syncthreads();
    const long long span = b - a;
    const long long t0 = a + (span * G.g) / groups, t1 = a + (span * (G.g + 1)) / groups;
    alive = gather_tiles<T, CC, NF>(sm, G, geo, &J.map, J.mlp.in_dim, J.mlp.n_freq, vb, vx, box_bytes, w, t0, t1,
                                    loaded, alive);
  }
  tmem_free_all(tmem_base);
}

// Feature Computation alone on tensor cores: c = MLP(x), x [M][in_dim] FP32.
__global__ void __launch_bounds__(512, 1) k_mlp_eval_bf16(MlpPtrs mlp, const float* x, int M, float* c, uint32_t* err) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  Group G = setup(sm, &mlp, kMaxGroups, 0);
  const uint32_t tmem_base = G.tmem - (uint32_t)(G.g * 128);
  const int ntile = (M + kTile - 1) / kTile;
  bool alive = true;
  for (int t = blockIdx.x * kMaxGroups + G.g; alive && t < ntile; t += gridDim.x * kMaxGroups) {
    const int row = t * kTile + G.m;
    float v[kK1];
#pragma unroll
    for (int j = 0; j < kK1; j++)
      v[j] = (row < M && j < mlp.in_dim) ? x[(size_t)row * mlp.in_dim + j] : (j == mlp.in_dim ? 1.0f : 0.0f);
#pragma unroll
    for (int k0 = 0; k0 < kK1; k0 += 8) store_chunk(G.act, G.m, k0, kK2, v + k0);
    fence_proxy_async();
    float cc[3];
    alive = mlp_tile(sm, G, err, cc, mlp.in_dim < kK1);
    if (alive && row < M) {
      c[3 * row + 0] = cc[0];
      c[3 * row + 1] = cc[1];
      c[3 * row + 2] = cc[2];
    }
  }
  if (!alive) mbar_wait(G.bar_mma, G.ph_mma, err);
  tmem_free_all(tmem_base);
}

// -------------------------------------------------------------------------------------------

// Tile pipelines per CTA: as many as fit the shared memory, at most `requested` (0 = no limit).
static int tc_groups(int box_bytes, int requested) {
  using namespace tc;
  int groups = kMaxGroups;
  while (groups > 1 && Smem::groups + groups * group_bytes(box_bytes) > 227 * 1024) groups--;
  return requested > 0 && requested < groups ? requested : groups;
}

template <typename T, int CC, int NF>
static cicero_status launch_tc(const GridGeo& geo, int S, const MlpPtrs& mlp, const RenderWs& ws,
                               const CUtensorMap& map, const BrickBox& box, int mlp_groups, cudaStream_t st) {
  using namespace tc;
  const int groups = tc_groups(box.box_bytes, mlp_groups);
  int smem = Smem::groups + groups * group_bytes(box.box_bytes);
  if (smem > 227 * 1024) return fail(CICERO_ERR_UNSUPPORTED, "brick too large for the tensor-core kernel");
  smem = std::max(smem, 120 * 1024);  // one CTA per SM: it owns all 512 TMEM columns
  auto kern = k_gather_mlp_bf16<T, CC, NF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gather_mlp_bf16)");
  {
    ProfScope ps(kStGatherMlp, st);
    kern<<<num_sms(), 128 * groups, smem, st>>>(geo, S, mlp, ws, map, box.vb, box.vx, box.box_bytes, groups);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_gather_mlp_bf16");
}

cicero_status launch_gather_mlp_bf16(const cicero_grid* grid, const GridGeo& geo, int mlp_groups,
                                     const MlpPtrs& mlp, const RenderWs& ws, const CUtensorMap& map,
                                     const BrickBox& box, cudaStream_t st) {
  const bool f16 = grid->dtype == CICERO_F16;
  if (geo.C == 12 && mlp.n_freq == 4)
    return f16 ? launch_tc<__half, 12, 4>(geo, ws.S, mlp, ws, map, box, mlp_groups, st)
               : launch_tc<float, 12, 4>(geo, ws.S, mlp, ws, map, box, mlp_groups, st);
  return f16 ? launch_tc<__half, 0, 0>(geo, ws.S, mlp, ws, map, box, mlp_groups, st)
             : launch_tc<float, 0, 0>(geo, ws.S, mlp, ws, map, box, mlp_groups, st);
}

template <typename T, int CC, int NF>
static cicero_status launch_tc_hash(const GridGeo& geo, const MlpPtrs& mlp, const RenderWs& ws, const HashGeo& hg,
                                    cudaStream_t st) {
  using namespace tc;
  const int groups = kMaxGroups;
  const int smem = std::max(Smem::groups + groups * group_bytes(0), 120 * 1024);
  auto kern = k_gather_mlp_bf16_hash<T, CC, NF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gather_mlp_bf16_hash)");
  {
    ProfScope ps(kStGatherMlp, st);
    kern<<<num_sms(), 128 * groups, smem, st>>>(geo, mlp, ws, hg, groups);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_gather_mlp_bf16_hash");
}

cicero_status launch_gather_mlp_bf16_hash(const GridGeo& geo, const MlpPtrs& mlp, const RenderWs& ws,
                                          const HashGeo& hg, cudaStream_t st) {
  // the kernel's type is the table's element type; 8 levels x 2 features with 4 frequencies is specialised
  if (hg.levels == 8 && mlp.n_freq == 4)
    return hg.f16 ? launch_tc_hash<__half, 16, 4>(geo, mlp, ws, hg, st) : launch_tc_hash<float, 16, 4>(geo, mlp, ws, hg, st);
  return hg.f16 ? launch_tc_hash<__half, 0, 0>(geo, mlp, ws, hg, st) : launch_tc_hash<float, 0, 0>(geo, mlp, ws, hg, st);
}

template <typename T, int CC, int NF>
static cicero_status launch_tc_batch(const BatchPlan& b, cudaStream_t st) {
  using namespace tc;
  const int groups = tc_groups(b.box.box_bytes, b.mlp_groups);
  int smem = Smem::groups + groups * group_bytes(b.box.box_bytes);
  if (smem > 227 * 1024) return fail(CICERO_ERR_UNSUPPORTED, "brick too large for the tensor-core kernel");
  smem = std::max(smem, 120 * 1024);  // one CTA per SM: it owns all 512 TMEM columns
  auto kern = k_gather_mlp_bf16_batch<T, CC, NF>;
  // set once per size, so that a launch after the first one is pure kernel launches (graph capture)
  static std::atomic<int> smem_set{0};
  cudaError_t e = cudaSuccess;
  if (smem > smem_set.load()) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gather_mlp_bf16_batch)");
    smem_set.store(smem);
  }
  {
    ProfScope ps(kStGatherMlp, st);
    kern<<<num_sms(), 128 * groups, smem, st>>>(b.jobs, b.n_jobs, b.ws, b.box.vb, b.box.vx, b.box.box_bytes, groups);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_gather_mlp_bf16_batch");
}

cicero_status launch_gather_mlp_bf16_batch(const BatchPlan& b, cudaStream_t st) {
  if (b.C == 12 && b.n_freq == 4)
    return b.f16 ? launch_tc_batch<__half, 12, 4>(b, st) : launch_tc_batch<float, 12, 4>(b, st);
  return b.f16 ? launch_tc_batch<__half, 0, 0>(b, st) : launch_tc_batch<float, 0, 0>(b, st);
}

cicero_status launch_mlp_eval_bf16(const MlpPtrs& mlp, const float* x, int M, float* c, uint32_t* err,
                                   cudaStream_t st) {
  using namespace tc;
  const int smem = std::max(Smem::groups + kMaxGroups * group_bytes(0), 120 * 1024);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_eval_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_eval_bf16)");
  const int ntile = (M + kTile - 1) / kTile;
  const int grid = std::max(1, std::min((ntile + kMaxGroups - 1) / kMaxGroups, num_sms()));
  {
    ProfScope ps(kStMlpEval, st);
    k_mlp_eval_bf16<<<grid, 128 * kMaxGroups, smem, st>>>(mlp, x, M, c, err);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_mlp_eval_bf16");
}

}  // namespace cicero
