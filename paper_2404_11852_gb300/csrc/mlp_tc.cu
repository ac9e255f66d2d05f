// Feature Computation on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One CTA of 128 threads owns a 128-sample tile at a time:
//   A1 [128 x 48]  BF16  gathered features + view encoding (written by the threads)
//   D1 = A1 W1^T   FP32 in tensor memory (columns 0..127)    -> bias, ReLU, BF16 -> A2
//   D2 = A2 W2^T   FP32 in tensor memory (columns 128..255)  -> bias, ReLU, BF16 -> A2
//   D3 = A2 W3^T   FP32 in tensor memory (columns 0..15, N padded 3 -> 16) -> bias, sigmoid
// One elected thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) and commits to an
// mbarrier; the four warps read their 32 accumulator rows back with tcgen05.ld.
// Operands use the canonical K-major, no-swizzle shared-memory layout: 8-row x 16-byte core
// matrices stored contiguously (128 B), consecutive K core matrices 128 B apart (LBO) and
// consecutive 8-row groups K*2*8 bytes apart (SBO).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace cicero {

namespace tc {

constexpr int kK1 = kMaxIn;           // 48
constexpr int kN3 = 16;               // layer-3 N padded to the smallest M=128 MMA width
constexpr uint32_t kTmemCols = 256;

struct Smem {
  static constexpr int w1 = 0;                                 // [128][48]  bf16
  static constexpr int w2 = w1 + kHidden * kK1 * 2;            // [128][128] bf16
  static constexpr int w3 = w2 + kHidden * kHidden * 2;        // [16][128]  bf16
  static constexpr int a1 = w3 + kN3 * kHidden * 2;            // [128][48]  bf16
  static constexpr int a2 = a1 + kTile * kK1 * 2;              // [128][128] bf16
  static constexpr int b1 = a2 + kTile * kHidden * 2;          // [128] f32
  static constexpr int b2 = b1 + kHidden * 4;                  // [128] f32
  static constexpr int b3 = b2 + kHidden * 4;                  // [4] f32
  static constexpr int bars = ((b3 + 16 + 127) / 128) * 128;   // 2 mbarriers + TMEM address
  static constexpr int tile = bars + 128;                      // brick box
  static_assert(tile % 128 == 0 && a1 % 16 == 0 && a2 % 16 == 0 && w2 % 16 == 0 && w3 % 16 == 0, "alignment");
};

// byte offset of element (row, k) in a K-major no-swizzle operand with K columns
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 8 consecutive K values of one row -> one 16-byte chunk of a K-major operand
__device__ __forceinline__ void store_chunk(char* base, int row, int k0, int K, const float* v) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(base + kmaj_off(row, k0, K)) = q;
}

__device__ void load_weights(char* sm, const MlpPtrs& m) {
  // W1: rows n, K padded to 48
  for (int i = threadIdx.x; i < kHidden * (kK1 / 8); i += blockDim.x) {
    const int n = i / (kK1 / 8), k0 = (i % (kK1 / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = (k0 + j < m.in_dim) ? m.w1[n * m.in_dim + k0 + j] : 0.0f;
    store_chunk(sm + Smem::w1, n, k0, kK1, v);
  }
  for (int i = threadIdx.x; i < kHidden * (kHidden / 8); i += blockDim.x) {
    const int n = i / (kHidden / 8), k0 = (i % (kHidden / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = m.w2[n * kHidden + k0 + j];
    store_chunk(sm + Smem::w2, n, k0, kHidden, v);
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
    b1[i] = m.b1[i];
    b2[i] = m.b2[i];
  }
  if (threadIdx.x < 4) b3[threadIdx.x] = threadIdx.x < 3 ? m.b3[threadIdx.x] : 0.0f;
}

struct TcState {
  uint32_t tmem;
  uint32_t phase;
  uint64_t* bar_mma;
};

// Issue layer `L` (single thread) and wait for it (all threads).  Returns false on timeout.
__device__ __forceinline__ bool run_layer(char* sm, TcState& st, int layer, uint32_t* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_after();
    const uint32_t a_base = smem_u32(sm + (layer == 0 ? Smem::a1 : Smem::a2));
    const uint32_t b_base = smem_u32(sm + (layer == 0 ? Smem::w1 : layer == 1 ? Smem::w2 : Smem::w3));
    const int K = layer == 0 ? kK1 : kHidden;
    const uint32_t sbo_a = (uint32_t)K * 16, sbo_b = (uint32_t)K * 16;
    const uint32_t idesc = idesc_bf16(layer == 2 ? kN3 : kHidden);
    const uint32_t d = st.tmem + (layer == 1 ? 128u : 0u);
    for (int s = 0; s < K / 16; s++) {
      const uint64_t ad = smem_desc(a_base + 256u * s, 128u, sbo_a);
      const uint64_t bd = smem_desc(b_base + 256u * s, 128u, sbo_b);
      mma_bf16(d, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    mma_commit(st.bar_mma);
  }
  const bool ok = __syncthreads_and(mbar_wait(st.bar_mma, st.phase, err));
  st.phase ^= 1u;
  fence_after();
  return ok;
}

// bias + ReLU of accumulator columns [col0, col0 + 128) -> BF16 into A2 (row = this thread)
__device__ __forceinline__ void epilogue_hidden(char* sm, const TcState& st, uint32_t col0, const float* bias) {
  const int warp = threadIdx.x >> 5, row = threadIdx.x;
  const uint32_t taddr = st.tmem + ((uint32_t)(warp * 32) << 16) + col0;
#pragma unroll 1
  for (int cc = 0; cc < kHidden / 16; cc++) {
    float v[16];
    tmem_ld16(taddr + cc * 16, v);
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = fmaxf(v[j] + bias[cc * 16 + j], 0.0f);
    store_chunk(sm + Smem::a2, row, cc * 16, kHidden, v);
    store_chunk(sm + Smem::a2, row, cc * 16 + 8, kHidden, v + 8);
  }
  fence_proxy_async();
  fence_before();
}

// The three layers of the tile whose A1 is already written (and fenced) by every thread.
// Returns false on a timeout; c receives this thread's row.
__device__ __forceinline__ bool mlp_tile(char* sm, TcState& st, uint32_t* err, float c[3]) {
  if (!run_layer(sm, st, 0, err)) return false;
  epilogue_hidden(sm, st, 0, (const float*)(sm + Smem::b1));
  if (!run_layer(sm, st, 1, err)) return false;
  epilogue_hidden(sm, st, 128, (const float*)(sm + Smem::b2));
  if (!run_layer(sm, st, 2, err)) return false;
  const int warp = threadIdx.x >> 5;
  float v[16];
  tmem_ld16(st.tmem + ((uint32_t)(warp * 32) << 16), v);
  const float* b3 = (const float*)(sm + Smem::b3);
  c[0] = sigmoid_f(v[0] + b3[0]);
  c[1] = sigmoid_f(v[1] + b3[1]);
  c[2] = sigmoid_f(v[2] + b3[2]);
  fence_before();
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

__device__ __forceinline__ void tmem_free(uint32_t tmem) {
  fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <typename T>
__device__ __forceinline__ void tri_smem_tc(const T* tile, int vb, int vx, int C, const int l[3], const float f[3],
                                            float* out) {
  const float fx = f[0], fy = f[1], fz = f[2];
  for (int c = 0; c < C; c++) out[c] = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int x = l[0] + (q & 1), y = l[1] + ((q >> 1) & 1), z = l[2] + (q >> 2);
    const float wq = ((q & 1) ? fx : 1.f - fx) * (((q >> 1) & 1) ? fy : 1.f - fy) * ((q >> 2) ? fz : 1.f - fz);
    const T* v = tile + ((size_t)(z * vb + y) * vx + x) * C;
    if constexpr (sizeof(T) == 2) {
      if (C == 12) {
        const uint2* v2 = reinterpret_cast<const uint2*>(v);
#pragma unroll
        for (int u = 0; u < 3; u++) {
          uint2 a = v2[u];
          float2 lo = __half22float2(*reinterpret_cast<__half2*>(&a.x));
          float2 hi = __half22float2(*reinterpret_cast<__half2*>(&a.y));
          out[4 * u + 0] += wq * lo.x;
          out[4 * u + 1] += wq * lo.y;
          out[4 * u + 2] += wq * hi.x;
          out[4 * u + 3] += wq * hi.y;
        }
        continue;
      }
    } else {
      if (C == 12) {
        const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
        for (int u = 0; u < 3; u++) {
          float4 a = v4[u];
          out[4 * u + 0] += wq * a.x;
          out[4 * u + 1] += wq * a.y;
          out[4 * u + 2] += wq * a.z;
          out[4 * u + 3] += wq * a.w;
        }
        continue;
      }
    }
    for (int c = 0; c < C; c++) {
      float vv;
      if constexpr (sizeof(T) == 4) vv = v[c];
      else vv = __half2float(v[c]);
      out[c] += wq * vv;
    }
  }
}

}  // namespace tc

template <typename T>
__global__ void __launch_bounds__(128) k_gather_mlp_bf16(GridGeo g, RaySrc src, int S, MlpPtrs mlp, RenderWs w,
                                                         const __grid_constant__ CUtensorMap fmap, int vb, int vx,
                                                         int box_bytes) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  uint64_t* bar_tma = (uint64_t*)(sm + Smem::bars);
  uint64_t* bar_mma = bar_tma + 1;
  uint32_t* tslot = (uint32_t*)(bar_tma + 2);
  T* tile = (T*)(sm + Smem::tile);
  load_weights(sm, mlp);
  if (threadIdx.x == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    fence_mbar_init();
  }
  fence_proxy_async();  // weights written by the threads are read by the tensor cores
  tmem_alloc(tslot);
  fence_before();
  __syncthreads();
  fence_after();
  TcState st;
  st.tmem = *tslot;
  st.phase = 0;
  st.bar_mma = bar_mma;

  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * per, t_end = min(n_tiles, t_begin + per);
  const int B = g.brick, C = g.C, m = threadIdx.x;
  int loaded = -1;
  uint32_t tphase = 0;
  bool alive = true;
  for (uint32_t ti = t_begin; ti < t_end; ti++) {
    const int b = (int)w.tile_brick[ti];
    const uint32_t start = w.tile_start[ti];
    const uint32_t end = min(start + (uint32_t)kTile, w.brick_off[b + 1]);
    const int mcnt = (int)(end - start);
    const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
    if (b != loaded) {
      __syncthreads();
      if (threadIdx.x == 0) {
        mbar_expect_tx(bar_tma, (uint32_t)box_bytes);
        tma_load_3d(tile, &fmap, bx * B * C, by * B, bz * B, bar_tma);
      }
      alive = mbar_wait(bar_tma, tphase, &w.hdr[0]);
      tphase ^= 1u;
      loaded = b;
    }
    if (!__syncthreads_and(alive)) break;
    uint32_t sid = 0;
    float x[kK1];
#pragma unroll
    for (int j = 0; j < kK1; j++) x[j] = 0.0f;
    if (m < mcnt) {
      sid = w.sorted[start + m];
      const int r = (int)(sid / (uint32_t)S);
      float o[3], d[3], p[3], f[3];
      int i0[3];
      ray_gen(src, r, o, d);
      sample_pos(o, d, w.rec_t[sid], p);
      const bool ok = index_sample(g, p, i0, f);
      const int l[3] = {i0[0] - bx * B, i0[1] - by * B, i0[2] - bz * B};
      if (!ok || l[0] < 0 || l[0] >= B || l[1] < 0 || l[1] >= B || l[2] < 0 || l[2] >= B)
        set_err(&w.hdr[0], kErrInternal);
      else
        tri_smem_tc<T>(tile, vb, vx, C, l, f, x);
      encode_dir(d, mlp.n_freq, x + C);
    }
#pragma unroll
    for (int k0 = 0; k0 < kK1; k0 += 8) store_chunk(sm + Smem::a1, m, k0, kK1, x + k0);
    fence_proxy_async();
    float c[3];
    if (!mlp_tile(sm, st, &w.hdr[0], c)) {
      alive = false;
      break;
    }
    if (m < mcnt) {
      w.rec_c[sid] = make_float4(c[0], c[1], c[2], w.rec_w[sid]);
    }
  }
  if (!alive) {
    // a bounded wait ran out: give in-flight copies and MMAs one more bounded wait
    mbar_wait(bar_tma, tphase, &w.hdr[0]);
    mbar_wait(bar_mma, st.phase, &w.hdr[0]);
  }
  tmem_free(st.tmem);
}

// Feature Computation alone on tensor cores: c = MLP(x), x [M][in_dim] FP32.
__global__ void __launch_bounds__(128) k_mlp_eval_bf16(MlpPtrs mlp, const float* x, int M, float* c, uint32_t* err) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  uint64_t* bar_mma = (uint64_t*)(sm + Smem::bars) + 1;
  uint32_t* tslot = (uint32_t*)(bar_mma + 1);
  load_weights(sm, mlp);
  if (threadIdx.x == 0) {
    mbar_init(bar_mma, 1);
    fence_mbar_init();
  }
  fence_proxy_async();
  tmem_alloc(tslot);
  fence_before();
  __syncthreads();
  fence_after();
  TcState st;
  st.tmem = *tslot;
  st.phase = 0;
  st.bar_mma = bar_mma;
  const int ntile = (M + kTile - 1) / kTile;
  bool alive = true;
  for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
    const int row = t * kTile + threadIdx.x;
    float v[kK1];
#pragma unroll
    for (int j = 0; j < kK1; j++) v[j] = (row < M && j < mlp.in_dim) ? x[(size_t)row * mlp.in_dim + j] : 0.0f;
#pragma unroll
    for (int k0 = 0; k0 < kK1; k0 += 8) store_chunk(sm + Smem::a1, threadIdx.x, k0, kK1, v + k0);
    fence_proxy_async();
    float cc[3];
    if (!mlp_tile(sm, st, err, cc)) {
      alive = false;
      break;
    }
    if (row < M) {
      c[3 * row + 0] = cc[0];
      c[3 * row + 1] = cc[1];
      c[3 * row + 2] = cc[2];
    }
  }
  if (!alive) mbar_wait(bar_mma, st.phase, err);
  tmem_free(st.tmem);
}

// -------------------------------------------------------------------------------------------

template <typename T>
static cicero_status launch_tc(const GridGeo& geo, const RaySrc& src, int S, const MlpPtrs& mlp, const RenderWs& ws,
                               const CUtensorMap& map, const BrickBox& box, cudaStream_t st) {
  const int smem = tc::Smem::tile + box.box_bytes;
  if (smem > 227 * 1024) return fail(CICERO_ERR_UNSUPPORTED, "brick too large for the tensor-core kernel");
  auto kern = k_gather_mlp_bf16<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gather_mlp_bf16)");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  per_sm = std::max(1, std::min(per_sm, 2));  // 2 x 256 TMEM columns fit in one SM's 512
  {
    ProfScope ps(kStGatherMlp, st);
    kern<<<num_sms() * per_sm, 128, smem, st>>>(geo, src, S, mlp, ws, map, box.vb, box.vx, box.box_bytes);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_gather_mlp_bf16");
}

cicero_status launch_gather_mlp_bf16(const cicero_grid* grid, const GridGeo& geo, const Samp& samp, const RaySrc& src,
                                     const MlpPtrs& mlp, const RenderWs& ws, const CUtensorMap& map,
                                     const BrickBox& box, cudaStream_t st) {
  (void)samp;
  if (grid->dtype == CICERO_F16) return launch_tc<__half>(geo, src, ws.S, mlp, ws, map, box, st);
  return launch_tc<float>(geo, src, ws.S, mlp, ws, map, box, st);
}

cicero_status launch_mlp_eval_bf16(const MlpPtrs& mlp, const float* x, int M, float* c, uint32_t* err,
                                   cudaStream_t st) {
  const int smem = tc::Smem::tile;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_eval_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_eval_bf16)");
  const int ntile = (M + kTile - 1) / kTile;
  {
    ProfScope ps(kStMlpEval, st);
    k_mlp_eval_bf16<<<std::max(1, std::min(ntile, num_sms() * 2)), 128, smem, st>>>(mlp, x, M, c, err);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_mlp_eval_bf16");
}

}  // namespace cicero
