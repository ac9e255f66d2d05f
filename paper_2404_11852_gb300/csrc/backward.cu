// Backward of the FP32 renderer: gradient of a loss L(rgb) with respect to the density and
// feature grids.  Nothing is stored by the forward pass; the backward recomputes it:
//
//   forward recompute  K1-K4 of render.cu (march, Ray Index Table), then per brick the features
//                      and the MLP: k_fwd_x3 (tensor cores, split-BF16 products) and k_fwd_fix
//                      (FP32, the samples with a ReLU pre-activation within k_fwd_x3's error
//                      estimate of zero); this
//                      leaves per composited sample (c, w, T, raw density) and the ReLU masks
//   B1 k_bwd_ray       per ray (warp), in slot order: R_k = sum_{j>k} w_j c_j + T_end bg by a
//                      warp scan, dL/dsigma_k = delta (T_{k+1} g.c_k - g.R_k) and
//                      dL/draw_k = dL/dsigma_k * sigmoid(raw_k + shift); each record's colour
//                      is replaced by what the brick pass needs of it: dL/dz3 (the gradient at
//                      the sigmoid's input, w_k g c_k (1 - c_k)) and dL/draw_k
//   B2 k_bwd_brick_tc  grid gradients: per brick (Ray Index Table order), 128 samples at a time,
//                      the MLP backward down to dL/dfeatures on the tensor cores, with the ReLU
//                      masks the recompute recorded (no forward layer is evaluated again), then
//                      the trilinear adjoint added straight into d_features and d_density with
//                      global atomics, 16-byte vector atomics where the channels allow.
//                      With d_mlp and a workspace that holds the staging, B0 and B2 also store
//                      each sample's weight-gradient operands (x, h1, h2; dL/dh2, dL/dh1, dL/dz3)
//                      as split-BF16 rows in the layout the tensor cores read, and
//   B3 k_dw            forms the MLP weight gradients from them as tensor-core GEMMs over the
//                      samples (bulk copies straight into MMA operands).
//   B2 k_bwd_brick     with d_mlp and no room for the staging, or above 16 channels: the same
//                      per brick, 64 samples at a time, MLP forward and backward on CUDA cores, the
//                      weight gradients summed over the CTA's tiles in registers and added to
//                      d_mlp once per CTA; the trilinear adjoint as in k_bwd_brick_tc.
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace cicero {

constexpr int kBT = 64;  // samples per backward tile

__device__ __forceinline__ float warp_sum_b(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// B1: per composited sample, (dL/dz3, dL/draw) written over its colour record (rec_c).
__global__ void __launch_bounds__(256) k_bwd_ray(RaySrc src, Samp s, RenderWs w, const float* __restrict__ d_rgb,
                                                 float act_shift) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int R = ray_count(src);
  const float dt = s.step > 0.0f ? s.step : __fdiv_rn(__fsub_rn(s.far_t, s.near_t), (float)s.n_samples);
  for (int r = warp; r < R; r += nwarps) {
    const uint32_t n = w.ray_n[r];
    const size_t rec0 = w.ray_start[r];
    const float g0 = d_rgb[3 * r], g1 = d_rgb[3 * r + 1], g2 = d_rgb[3 * r + 2];
    float tot = 0.0f;
    for (uint32_t j = lane; j < n; j += 32) {
      const float4 c = w.rec_c[rec0 + j];
      tot += c.w * (g0 * c.x + g1 * c.y + g2 * c.z);
    }
    tot = warp_sum_b(tot);
    const float gbg = w.ray_T[r] * (g0 * s.bg[0] + g1 * s.bg[1] + g2 * s.bg[2]);
    float run = 0.0f;  // sum of e_j over earlier chunks
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
      const uint32_t j = j0 + lane;
      float e = 0.0f, gc = 0.0f, wk = 0.0f;
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < n) {
        c = w.rec_c[rec0 + j];
        gc = g0 * c.x + g1 * c.y + g2 * c.z;
        wk = c.w;
        e = wk * gc;
      }
      float incl = e;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (j < n) {
        const float gR = (tot - (run + incl)) + gbg;
        const float Tn = w.rec_T[rec0 + j] - wk;
        const float dsig = dt * (Tn * gc - gR);
        w.rec_c[rec0 + j] = make_float4(wk * g0 * c.x * (1.0f - c.x), wk * g1 * c.y * (1.0f - c.y),
                                        wk * g2 * c.z * (1.0f - c.z),
                                        dsig * sigmoid_f(w.rec_raw[rec0 + j] + act_shift));
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// Tiles are stored feature-major, [feature][sample], with a row stride of kLD = 68 floats: 64
// samples plus 4 of padding, so that 8 threads reading one float4 each from 8 consecutive
// feature rows at the same samples hit 8 different bank quads (68 = 4 mod 32).
constexpr int kLD = 68;

struct BwdSmem {
  static constexpr int w1t = 0;                          // [48][128]
  static constexpr int w2t = w1t + kMaxIn * kHidden * 4; // [128][128]
  static constexpr int w3 = w2t + kHidden * kHidden * 4; // [3][128]
  static constexpr int b1 = w3 + 3 * kHidden * 4;
  static constexpr int b2 = b1 + kHidden * 4;
  static constexpr int x = b2 + kHidden * 4;             // [48][kLD]  inputs
  static constexpr int h1 = x + kMaxIn * kLD * 4;        // [128][kLD] h1, later dL/dh1
  static constexpr int h2 = h1 + kHidden * kLD * 4;      // [128][kLD] h2, later dL/dh2, then dL/dfeatures
  static constexpr int dz = h2 + kHidden * kLD * 4;      // [3][kLD]
  static constexpr int meta = dz + 3 * kLD * 4;          // per sample: i0[3] (int), f[3], draw, valid
  static constexpr int bytes = meta + 8 * kBT * 4;
};

// acc[i][j]: rows tm*4+i (i < 4), cols {tn*4+j, 64+tn*4+(j-4)}; A [K][kLD], B [K][128] k-major
__device__ __forceinline__ void gemm64(const float* A, const float* Bw, int K, int tm, int tn, float acc[4][8]) {
#pragma unroll 2
  for (int k = 0; k < K; k++) {
    const float4 a = *reinterpret_cast<const float4*>(&A[k * kLD + tm * 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&Bw[k * kHidden + tn * 4]);
    const float4 b1 = *reinterpret_cast<const float4*>(&Bw[k * kHidden + 64 + tn * 4]);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

__device__ __forceinline__ int col8(int tn, int j) { return j < 4 ? tn * 4 + j : 64 + tn * 4 + (j - 4); }

// same with B read transposed from Bt [128][128]: B[k][n] = Bt[n][k], four k at a time (one
// float4 of Bt per column); K is a multiple of 4
__device__ __forceinline__ void gemm64_bt(const float* A, const float* Bt, int K, int tm, int tn, float acc[4][8]) {
#pragma unroll 1
  for (int k = 0; k < K; k += 4) {
    float4 bq[8];
#pragma unroll
    for (int j = 0; j < 8; j++) bq[j] = *reinterpret_cast<const float4*>(&Bt[col8(tn, j) * kHidden + k]);
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
      const float4 a = *reinterpret_cast<const float4*>(&A[(k + kk) * kLD + tm * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const float b = kk == 0 ? bq[j].x : kk == 1 ? bq[j].y : kk == 2 ? bq[j].z : bq[j].w;
#pragma unroll
        for (int i = 0; i < 4; i++) acc[i][j] = fmaf(av[i], b, acc[i][j]);
      }
    }
  }
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// corners q0 and q0 + 1 of the trilinear interpolation of the features at (i0, f), weighted,
// into out[0, C) (the caller sums the four corner pairs)
template <typename T>
__device__ __forceinline__ void feat_corner_pair(const GridGeo& g, const T* feat, const int i0[3], const float f[3],
                                                 int q0, float* out) {
  const int C = g.C;
#pragma unroll
  for (int u = 0; u < 2; u++) {
    const int q = q0 + u;
    const int x = i0[0] + (q & 1), y = i0[1] + ((q >> 1) & 1), z = i0[2] + (q >> 2);
    const float wq = ((q & 1) ? f[0] : 1.f - f[0]) * (((q >> 1) & 1) ? f[1] : 1.f - f[1]) * ((q >> 2) ? f[2] : 1.f - f[2]);
    const T* v = feat + (((size_t)z * g.n[1] + y) * g.n[0] + x) * C;
    for (int c = 0; c < C; c++) out[c] += wq * ldf(v + c);
  }
}

// One corner of the trilinear adjoint, added straight into the gradients of vertex v:
// d_feat[v][c] += wq df(c) for c < C and d_dens[v] += wq dr.  Samples reach a vertex from many
// CTAs, so the adds are global atomics (their results unused); with vec (C % 4 == 0 and d_feat
// 16-byte aligned) the channels go as 16-byte vector atomics (sm_90 and later), four channels per
// operation.  (Explicit red.global.add.v4.f32 reductions measured 6% slower.)
// Measured against a shared-memory copy of the brick flushed once per brick: 2.45 -> 0.90 ms on
// the 8192-ray backward (the shared-memory atomics conflicted on the vertices that neighbouring
// samples share, and the flush touched every entry of the brick).
// CMAX > 0: C <= CMAX, loops unrolled (df indexes a register array).
template <int CMAX, typename DF>
__device__ __forceinline__ void scatter_corner(int C, bool vec, size_t v, float wq, DF df, float dr, float* d_dens,
                                               float* d_feat) {
  float* gf = d_feat + v * (size_t)C;
  if constexpr (CMAX > 0) {
    if (vec) {
#pragma unroll
      for (int c = 0; c < CMAX; c += 4)
        if (c < C)
          atomicAdd(reinterpret_cast<float4*>(gf + c),
                    make_float4(wq * df(c), wq * df(c + 1), wq * df(c + 2), wq * df(c + 3)));
    } else {
#pragma unroll
      for (int c = 0; c < CMAX; c++)
        if (c < C) atomicAdd(gf + c, wq * df(c));
    }
  } else {
    if (vec) {
      for (int c = 0; c < C; c += 4)
        atomicAdd(reinterpret_cast<float4*>(gf + c),
                  make_float4(wq * df(c), wq * df(c + 1), wq * df(c + 2), wq * df(c + 3)));
    } else {
      for (int c = 0; c < C; c++) atomicAdd(gf + c, wq * df(c));
    }
  }
  atomicAdd(d_dens + v, wq * dr);
}

__device__ __forceinline__ size_t corner_vertex(const GridGeo& g, int x, int y, int z, int q) {
  return ((size_t)(z + (q >> 2)) * g.n[1] + (y + ((q >> 1) & 1))) * g.n[0] + (x + (q & 1));
}

__device__ __forceinline__ float corner_weight(const float f0, const float f1, const float f2, int q) {
  return ((q & 1) ? f0 : 1.f - f0) * (((q >> 1) & 1) ? f1 : 1.f - f1) * ((q >> 2) ? f2 : 1.f - f2);
}

// WG: also accumulate the MLP weight gradients.  Each thread keeps its share in registers for the
// whole launch and adds it to d_mlp once at the end:
//   dW2[o][i] (o = tn + 16a, i = tm + 16b, a, b < 8)   dW1[o][k] (k = tm + 16b, b < 3)   db1[o]
//   dW3[j][o], db2[o] (o = tid mod 128, one half of the tile's samples each)   db3[j]
template <typename T, bool WG>
__global__ void __launch_bounds__(256, 1) k_bwd_brick(GridGeo g, RaySrc src, MlpPtrs mlp, RenderWs w,
                                                      const T* __restrict__ feat, float* d_dens, float* d_feat,
                                                      float* d_mlp) {
  extern __shared__ __align__(1024) char sm[];
  float* w1t = (float*)(sm + BwdSmem::w1t);
  float* w2t = (float*)(sm + BwdSmem::w2t);
  float* w3 = (float*)(sm + BwdSmem::w3);
  float* b1 = (float*)(sm + BwdSmem::b1);
  float* b2 = (float*)(sm + BwdSmem::b2);
  float* X = (float*)(sm + BwdSmem::x);
  float* H1 = (float*)(sm + BwdSmem::h1);
  float* H2 = (float*)(sm + BwdSmem::h2);
  float* DZ = (float*)(sm + BwdSmem::dz);
  int* ml = (int*)(sm + BwdSmem::meta);              // [3][64]
  float* mf = (float*)(sm + BwdSmem::meta) + 3 * kBT; // [3][64]
  float* mdraw = mf + 3 * kBT;                        // [64]
  int* mval = (int*)(mdraw + kBT);                    // [64]
  const int C = g.C, B = g.brick;
  const bool vec = (C & 3) == 0 && (reinterpret_cast<uintptr_t>(d_feat) & 15u) == 0;
  for (int i = threadIdx.x; i < kMaxIn * kHidden; i += blockDim.x) {
    const int k = i / kHidden, n = i % kHidden;
    w1t[i] = k < mlp.in_dim ? mlp.w1[n * mlp.in_dim + k] : 0.0f;
  }
  for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) w2t[i] = mlp.w2[(i % kHidden) * kHidden + i / kHidden];
  for (int i = threadIdx.x; i < 3 * kHidden; i += blockDim.x) w3[i] = mlp.w3[i];
  for (int i = threadIdx.x; i < kHidden; i += blockDim.x) {
    b1[i] = mlp.b1[i];
    b2[i] = mlp.b2[i];
  }
  __syncthreads();

  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * per, t_end = min(n_tiles, t_begin + per);
  const int tm = threadIdx.x & 15, tn = threadIdx.x >> 4;
  const int ro = threadIdx.x & (kHidden - 1), rs0 = (threadIdx.x >> 7) * (kBT / 2);  // dh2 phase: row, samples
  float gw2[8][8], gw1[8][3], gb1[8], gw3[3], gb3[3], gb2 = 0.0f;
  if constexpr (WG) {
#pragma unroll
    for (int a = 0; a < 8; a++) {
#pragma unroll
      for (int b = 0; b < 8; b++) gw2[a][b] = 0.0f;
#pragma unroll
      for (int b = 0; b < 3; b++) gw1[a][b] = 0.0f;
      gb1[a] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 3; j++) gw3[j] = gb3[j] = 0.0f;
  }
  for (uint32_t ti = t_begin; ti < t_end; ti++) {
    const uint4 td = w.tile[ti];
    const uint32_t start0 = td.x;
    const uint32_t end = start0 + (td.y & 0xFFu);
    const int bx = (int)(td.w & 0xFFFFu), by = (int)(td.w >> 16), bz = (int)((td.y >> 8) & 0x1FFFu);
    for (uint32_t start = start0; start < end; start += kBT) {
      const int mcnt = (int)min((uint32_t)kBT, end - start);
      // gather: four threads per sample (m = tid / 4), each interpolating two of the eight corners;
      // the quad's partial sums are added with shuffles, then the first thread writes the features
      // and the per-sample data and the second the direction encoding.  Samples past mcnt and
      // rejected samples get x = 0 and dL/dz = 0, so they add nothing to any gradient.
      {
        const int m = threadIdx.x >> 2, qp = threadIdx.x & 3;
        const bool valid = m < mcnt;
        const float4 qd = valid ? w.srt[start + m].qd : make_float4(0.f, 0.f, 0.f, 1.f);
        const uint32_t sid = __float_as_uint(qd.x);
        float f[3] = {0.f, 0.f, 0.f}, fv[24];
        int i0[3] = {0, 0, 0}, l[3] = {0, 0, 0};
        bool ok = false;
        if (valid) {
          const float4 pw = w.srt[start + m].pw;
          const float p[3] = {pw.x, pw.y, pw.z};
          const bool in = index_sample(g, p, i0, f);
          l[0] = i0[0] - bx * B;
          l[1] = i0[1] - by * B;
          l[2] = i0[2] - bz * B;
          ok = in && l[0] >= 0 && l[0] < B && l[1] >= 0 && l[1] < B && l[2] >= 0 && l[2] < B;
          if (!ok && qp == 0) set_err(&w.hdr[0], kErrInternal);
        }
        for (int c = 0; c < C; c++) fv[c] = 0.0f;
        if (ok) feat_corner_pair<T>(g, feat, i0, f, 2 * qp, fv);
        for (int c = 0; c < C; c++) {
          fv[c] += __shfl_xor_sync(0xffffffffu, fv[c], 1);
          fv[c] += __shfl_xor_sync(0xffffffffu, fv[c], 2);
        }
        if (qp == 0) {
          for (int c = 0; c < C; c++) X[c * kLD + m] = fv[c];
          if (ok) {
            for (int a = 0; a < 3; a++) {
              ml[a * kBT + m] = i0[a];
              mf[a * kBT + m] = f[a];
            }
            const float4 dz = w.rec_c[sid];  // (dL/dz3, dL/draw) from B1
            mdraw[m] = dz.w;
            DZ[m] = dz.x;
            DZ[kLD + m] = dz.y;
            DZ[2 * kLD + m] = dz.z;
          } else {
            for (int j = 0; j < 3; j++) DZ[j * kLD + m] = 0.0f;
          }
          mval[m] = ok ? 1 : 0;
        } else if (qp == 1) {
          float e[3 + 6 * 7];
          const int ne = 3 + 6 * mlp.n_freq;
          const float d[3] = {qd.y, qd.z, qd.w};
          if (valid) encode_dir(d, mlp.n_freq, e);
          for (int j = 0; j < ne; j++) X[(C + j) * kLD + m] = valid ? e[j] : 0.0f;
          for (int j = C + ne; j < kMaxIn; j++) X[j * kLD + m] = 0.0f;
        }
      }
      __syncthreads();
      float acc[4][8];
      // layer 1
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
      gemm64(X, w1t, (mlp.in_dim + 3) & ~3, tm, tn, acc);  // rows in_dim.. of X and W1^T are zero
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int n = col8(tn, j);
        float4 v;
        v.x = fmaxf(acc[0][j] + b1[n], 0.f);
        v.y = fmaxf(acc[1][j] + b1[n], 0.f);
        v.z = fmaxf(acc[2][j] + b1[n], 0.f);
        v.w = fmaxf(acc[3][j] + b1[n], 0.f);
        *reinterpret_cast<float4*>(&H1[n * kLD + tm * 4]) = v;
      }
      __syncthreads();
      // layer 2
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
      gemm64(H1, w2t, kHidden, tm, tn, acc);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int n = col8(tn, j);
        float4 v;
        v.x = fmaxf(acc[0][j] + b2[n], 0.f);
        v.y = fmaxf(acc[1][j] + b2[n], 0.f);
        v.z = fmaxf(acc[2][j] + b2[n], 0.f);
        v.w = fmaxf(acc[3][j] + b2[n], 0.f);
        *reinterpret_cast<float4*>(&H2[n * kLD + tm * 4]) = v;
      }
      __syncthreads();
      // dL/dh2 = W3^T dz masked by relu'(pre2), in place over h2 (each element read and written by
      // the same thread); dW3 += dz h2^T, db3 += dz, db2 += dL/dh2 on the way
      {
        const float wa = w3[ro], wb = w3[kHidden + ro], wc = w3[2 * kHidden + ro];
        float* hr = H2 + ro * kLD;
#pragma unroll 2
        for (int s = rs0; s < rs0 + kBT / 2; s += 4) {
          const float4 h = *reinterpret_cast<const float4*>(&hr[s]);
          const float4 z0 = *reinterpret_cast<const float4*>(&DZ[s]);
          const float4 z1 = *reinterpret_cast<const float4*>(&DZ[kLD + s]);
          const float4 z2 = *reinterpret_cast<const float4*>(&DZ[2 * kLD + s]);
          float4 v;
          v.x = h.x > 0.0f ? wa * z0.x + wb * z1.x + wc * z2.x : 0.0f;
          v.y = h.y > 0.0f ? wa * z0.y + wb * z1.y + wc * z2.y : 0.0f;
          v.z = h.z > 0.0f ? wa * z0.z + wb * z1.z + wc * z2.z : 0.0f;
          v.w = h.w > 0.0f ? wa * z0.w + wb * z1.w + wc * z2.w : 0.0f;
          if constexpr (WG) {
            gw3[0] += dot4(z0, h);
            gw3[1] += dot4(z1, h);
            gw3[2] += dot4(z2, h);
            gb3[0] += (z0.x + z0.y) + (z0.z + z0.w);
            gb3[1] += (z1.x + z1.y) + (z1.z + z1.w);
            gb3[2] += (z2.x + z2.y) + (z2.z + z2.w);
            gb2 += (v.x + v.y) + (v.z + v.w);
          }
          *reinterpret_cast<float4*>(&hr[s]) = v;
        }
      }
      __syncthreads();
      // dW2 += dL/dh2 h1^T, while H1 still holds h1
      if constexpr (WG) {
#pragma unroll 1
        for (int s = 0; s < kBT; s += 4) {
          float4 hv[8];
#pragma unroll
          for (int bb = 0; bb < 8; bb++) hv[bb] = *reinterpret_cast<const float4*>(&H1[(tm + 16 * bb) * kLD + s]);
#pragma unroll
          for (int a = 0; a < 8; a++) {
            const float4 dv = *reinterpret_cast<const float4*>(&H2[(tn + 16 * a) * kLD + s]);
#pragma unroll
            for (int bb = 0; bb < 8; bb++) gw2[a][bb] += dot4(dv, hv[bb]);
          }
        }
      }
      // dL/dh1 = W2^T dh2, masked by relu'(pre1)
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
      gemm64_bt(H2, w2t, kHidden, tm, tn, acc);
      if constexpr (WG) __syncthreads();  // every thread's dW2 reads of h1 are done
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int n = col8(tn, j);
        float4 h = *reinterpret_cast<float4*>(&H1[n * kLD + tm * 4]);
        h.x = h.x > 0.f ? acc[0][j] : 0.f;
        h.y = h.y > 0.f ? acc[1][j] : 0.f;
        h.z = h.z > 0.f ? acc[2][j] : 0.f;
        h.w = h.w > 0.f ? acc[3][j] : 0.f;
        *reinterpret_cast<float4*>(&H1[n * kLD + tm * 4]) = h;
      }
      __syncthreads();
      // dW1 += dL/dh1 x^T, db1 += dL/dh1
      if constexpr (WG) {
#pragma unroll 1
        for (int s = 0; s < kBT; s += 4) {
          float4 xv[3];
#pragma unroll
          for (int bb = 0; bb < 3; bb++) xv[bb] = *reinterpret_cast<const float4*>(&X[(tm + 16 * bb) * kLD + s]);
#pragma unroll
          for (int a = 0; a < 8; a++) {
            const float4 dv = *reinterpret_cast<const float4*>(&H1[(tn + 16 * a) * kLD + s]);
            gb1[a] += (dv.x + dv.y) + (dv.z + dv.w);
#pragma unroll
            for (int bb = 0; bb < 3; bb++) gw1[a][bb] += dot4(dv, xv[bb]);
          }
        }
      }
      // dL/dfeatures = W1[:, :C]^T dh1, into H2 (dL/dh2 is no longer read): thread (mm = tid mod 64,
      // cg = tid / 64) takes channels cg, cg + 4, cg + 8 (then + 12, ...) of sample mm, four hidden
      // units at a time
      {
        const int mm = threadIdx.x & (kBT - 1), cg = threadIdx.x >> 6;
        for (int c0 = cg; c0 < C; c0 += 12) {
          const bool v1 = c0 + 4 < C, v2 = c0 + 8 < C;
          float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll 2
          for (int n = 0; n < kHidden; n += 4) {
            const float4 h = make_float4(H1[n * kLD + mm], H1[(n + 1) * kLD + mm], H1[(n + 2) * kLD + mm],
                                         H1[(n + 3) * kLD + mm]);
            s0 += dot4(*reinterpret_cast<const float4*>(&w1t[c0 * kHidden + n]), h);
            if (v1) s1 += dot4(*reinterpret_cast<const float4*>(&w1t[(c0 + 4) * kHidden + n]), h);
            if (v2) s2 += dot4(*reinterpret_cast<const float4*>(&w1t[(c0 + 8) * kHidden + n]), h);
          }
          H2[c0 * kLD + mm] = s0;
          if (v1) H2[(c0 + 4) * kLD + mm] = s1;
          if (v2) H2[(c0 + 8) * kLD + mm] = s2;
        }
      }
      __syncthreads();
      // trilinear adjoint: 4 threads per sample, 2 corners each
      {
        const int mm = threadIdx.x >> 2, qp = threadIdx.x & 3;
        if (mm < mcnt && mval[mm]) {
          const float f0 = mf[mm], f1 = mf[kBT + mm], f2 = mf[2 * kBT + mm];
          const int x0 = ml[mm], y0 = ml[kBT + mm], z0 = ml[2 * kBT + mm];
          const float dr = mdraw[mm];
          const float* dfm = H2 + mm;
#pragma unroll
          for (int u = 0; u < 2; u++) {
            const int q = 2 * qp + u;
            scatter_corner<0>(C, vec, corner_vertex(g, x0, y0, z0, q), corner_weight(f0, f1, f2, q),
                           [&](int c) { return dfm[c * kLD]; }, dr, d_dens, d_feat);
          }
        }
      }
      __syncthreads();
    }
  }
  if (WG && t_begin < t_end) {
    // d_mlp = [W1 [128][in_dim], b1 [128], W2 [128][128], b2 [128], W3 [3][128], b3 [3]]
    const int I = mlp.in_dim;
    float* dW1 = d_mlp;
    float* db1 = dW1 + kHidden * I;
    float* dW2 = db1 + kHidden;
    float* db2 = dW2 + kHidden * kHidden;
    float* dW3 = db2 + kHidden;
    float* db3 = dW3 + 3 * kHidden;
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int o = tn + 16 * a;
#pragma unroll
      for (int bb = 0; bb < 8; bb++) atomicAdd(&dW2[o * kHidden + tm + 16 * bb], gw2[a][bb]);
#pragma unroll
      for (int bb = 0; bb < 3; bb++)
        if (tm + 16 * bb < I) atomicAdd(&dW1[o * I + tm + 16 * bb], gw1[a][bb]);
      if (tm == 0) atomicAdd(&db1[o], gb1[a]);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) atomicAdd(&dW3[j * kHidden + ro], gw3[j]);
    atomicAdd(&db2[ro], gb2);
    if (ro == 0)
#pragma unroll
      for (int j = 0; j < 3; j++) atomicAdd(&db3[j], gb3[j]);
  }
}

// ---------------------------------------------------------------------------------------------
// B2 on the tensor cores (grid gradients).  Two independent groups of 128 threads per CTA, each
// with its own tiles (alternate tiles of the CTA's range), operand buffers, TMEM columns and
// mbarrier, so that one group's MMA waits and loads overlap the other's CUDA-core work.  Per tile
// of <= 128 samples of one brick, one thread per sample:
//   dh2 = (dz3 W3) masked by relu'(z2)           CUDA cores (K = 3)
//   dh1 = (dh2 W2) masked by relu'(z1)           tcgen05 kind::f16, M = 128, N = 128, K = 128
//   dL/dfeatures = dh1 W1[:, :C]                 tcgen05, N = 16 (channels padded), K = 128
// Near-FP32 accuracy from BF16 operands: every operand x is split into hi = bf16(x) and
// lo = bf16(x - hi) and each product is hi hi' + hi lo' + lo hi' (the bf16x3 scheme of Henry, Tang
// and Heinecke, ARITH 2019: the dropped lo lo' term and the residuals of the split are each ~2^-18
// of the product, so a product keeps ~16 significant bits), accumulated in FP32 in tensor memory.
// The ReLU masks are the recompute's (rec_mask): every decision whose pre-activation the split-BF16
// recompute found within its error estimate of zero was taken again by the FP32 MLP.

namespace bt {
constexpr int kGroups = 2;
constexpr int kThreads = kGroups * kTile;  // one thread per sample of each group's 128-sample tile
constexpr int kN1 = 16;                    // channels of dL/dfeatures, padded to the smallest MMA width
struct Smem {
  static constexpr int w2t_hi = 0;                                  // [128][128] bf16: row i, K = o: W2[o][i]
  static constexpr int w2t_lo = w2t_hi + kHidden * kHidden * 2;
  static constexpr int w1t_hi = w2t_lo + kHidden * kHidden * 2;     // [16][128] bf16: row c, K = i: W1[i][c]
  static constexpr int w1t_lo = w1t_hi + kN1 * kHidden * 2;
  static constexpr int a = w1t_lo + kN1 * kHidden * 2;              // per group: [128][128] bf16 hi, then lo:
  static constexpr int a_group = 2 * kTile * kHidden * 2;           // dh2, then dh1
  static constexpr int w3 = a + kGroups * a_group;                  // [3][128] f32
  static constexpr int bars = w3 + 3 * kHidden * 4;                 // one mbarrier per group; TMEM address at +16
  static constexpr int bytes = bars + 128;
  static_assert(a % 16 == 0 && w1t_hi % 16 == 0 && bars % 16 == 0, "operand alignment");
};
constexpr uint32_t kTmemCols = kGroups * 128;  // 128 columns per group
}  // namespace bt

// Barriers of one group of 128 threads (named barriers 1 and 2; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(kTile) : "memory");
}
__device__ __forceinline__ bool group_sync_and(int grp, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + grp), "r"(kTile)
      : "memory");
  return r != 0;
}

// 8 consecutive K values of one row, split into the hi and lo operands (hi exactly representable in
// BF16, so its packing rounds nothing)
__device__ __forceinline__ void store_chunk_split(char* hi_base, char* lo_base, int row, int k0, int K,
                                                  const float* v) {
  float h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    h[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
    l[j] = v[j] - h[j];
  }
  tc::store_chunk(hi_base, row, k0, K, h);
  tc::store_chunk(lo_base, row, k0, K, l);
}

// the same split of 8 values, packed as the two 16-byte rows (hi, lo) of a BF16 operand
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  float h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    h[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
    l[j] = v[j] - h[j];
  }
  hi = make_uint4(tc::pack_bf16(h[0], h[1]), tc::pack_bf16(h[2], h[3]), tc::pack_bf16(h[4], h[5]),
                  tc::pack_bf16(h[6], h[7]));
  lo = make_uint4(tc::pack_bf16(l[0], l[1]), tc::pack_bf16(l[2], l[3]), tc::pack_bf16(l[4], l[5]),
                  tc::pack_bf16(l[6], l[7]));
}

// row (k0 .. k0 + 7) of a K-major operand in shared memory, from packed hi and lo rows
__device__ __forceinline__ void store_rows(char* hi_base, char* lo_base, int row, int k0, int K, const uint4& hi,
                                           const uint4& lo) {
  *reinterpret_cast<uint4*>(hi_base + tc::kmaj_off(row, k0, K)) = hi;
  *reinterpret_cast<uint4*>(lo_base + tc::kmaj_off(row, k0, K)) = lo;
}

// row group g of the staged operand at offset op (R rows) of one sample, whose rows start at col
// (stage_col of the sample)
__device__ __forceinline__ void stage_put(char* col, int op, int R, int g, const uint4& hi, const uint4& lo) {
  *reinterpret_cast<uint4*>(col + op + 256 * g) = hi;
  *reinterpret_cast<uint4*>(col + op + 32 * R + 256 * g) = lo;
}

// ReLU mask of the half h of the hidden units (h = 0: units 0..63, 1: 64..127), in the layout the
// recompute writes (unit n < 64 is bit n % 4 of byte n / 4, unit 64 + n bit 4 + n % 4): the
// words shifted so that unit 64 h + i is bit (i / 4 % 4) * 8 + i % 4 of word i / 16.
struct HalfMask {
  uint32_t w[4];
  __device__ __forceinline__ HalfMask(const uint4& mk, int h) {
    const uint32_t sh = 4u * (uint32_t)h;
    w[0] = mk.x >> sh;
    w[1] = mk.y >> sh;
    w[2] = mk.z >> sh;
    w[3] = mk.w >> sh;
  }
  __device__ __forceinline__ bool operator[](int i) const {  // i = 0..63, a compile-time constant in use
    return (w[i >> 4] >> (((i >> 2) & 3) * 8 + (i & 3))) & 1u;
  }
};

// A (hi, lo) x B (hi, lo) over K = 16 KSTEPS into the accumulator at d: three products per K step
template <int KSTEPS = kHidden / 16>
__device__ __forceinline__ void mma_split(uint32_t d, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl,
                                          uint32_t idesc) {
#pragma unroll
  for (int s = 0; s < KSTEPS; s++) {
    tc::mma_bf16(d, ah + 16u * s, bh + 16u * s, idesc, s > 0 ? 1u : 0u);
    tc::mma_bf16(d, ah + 16u * s, bl + 16u * s, idesc, 1u);
    tc::mma_bf16(d, al + 16u * s, bh + 16u * s, idesc, 1u);
  }
}

// Group grp = tid / 128 takes tiles t_begin + grp, t_begin + grp + 2, ...; thread m = tid mod 128
// takes sample m of each (TMEM lane m of the group's columns [128 grp, 128 grp + 128)), its 128
// hidden units 64 at a time and its eight trilinear corners.  The group's barriers are named
// barriers of 128 threads, so the two groups never wait for each other until the kernel ends.
template <bool WG>
__global__ void __launch_bounds__(bt::kThreads, 1) k_bwd_brick_tc(GridGeo g, MlpPtrs mlp, RenderWs w, float* d_dens,
                                                                  float* d_feat) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  const int C = g.C, B = g.brick;
  const bool vec = (C & 3) == 0 && (reinterpret_cast<uintptr_t>(d_feat) & 15u) == 0;
  const int m = threadIdx.x & (kTile - 1), grp = threadIdx.x / kTile;
  char* a_hi = sm + bt::Smem::a + grp * bt::Smem::a_group;
  char* a_lo = a_hi + kTile * kHidden * 2;
  float* w3s = (float*)(sm + bt::Smem::w3);
  uint64_t* bar = (uint64_t*)(sm + bt::Smem::bars) + grp;
  uint32_t* tslot = (uint32_t*)(sm + bt::Smem::bars + 16);
  // the weights, transposed into the B operands and split
  for (int i = threadIdx.x; i < kHidden * (kHidden / 8); i += bt::kThreads) {
    const int n = i / (kHidden / 8), k0 = (i % (kHidden / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = mlp.w2[(k0 + j) * kHidden + n];
    store_chunk_split(sm + bt::Smem::w2t_hi, sm + bt::Smem::w2t_lo, n, k0, kHidden, v);
  }
  for (int i = threadIdx.x; i < bt::kN1 * (kHidden / 8); i += bt::kThreads) {
    const int n = i / (kHidden / 8), k0 = (i % (kHidden / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = n < C ? mlp.w1[(k0 + j) * mlp.in_dim + n] : 0.0f;
    store_chunk_split(sm + bt::Smem::w1t_hi, sm + bt::Smem::w1t_lo, n, k0, kHidden, v);
  }
  for (int i = threadIdx.x; i < 3 * kHidden; i += bt::kThreads) w3s[i] = mlp.w3[i];
  if (threadIdx.x == 0) {
    for (int j = 0; j < bt::kGroups; j++) mbar_init((uint64_t*)(sm + bt::Smem::bars) + j, 1);
    fence_mbar_init();
  }
  fence_proxy_async();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(bt::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tslot;
  const uint32_t tmem = tmem_base + 128u * (uint32_t)grp;                             // this group's columns
  const uint32_t taddr = tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16);  // this warp's lanes
  const uint64_t ah = smem_desc(smem_u32(a_hi), 128u, kHidden * 16), al = smem_desc(smem_u32(a_lo), 128u, kHidden * 16);
  const uint64_t b2h = smem_desc(smem_u32(sm + bt::Smem::w2t_hi), 128u, kHidden * 16);
  const uint64_t b2l = smem_desc(smem_u32(sm + bt::Smem::w2t_lo), 128u, kHidden * 16);
  const uint64_t b1h = smem_desc(smem_u32(sm + bt::Smem::w1t_hi), 128u, kHidden * 16);
  const uint64_t b1l = smem_desc(smem_u32(sm + bt::Smem::w1t_lo), 128u, kHidden * 16);
  uint32_t phase = 0;
  bool alive = true;

  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * per, t_end = min(n_tiles, t_begin + per);
  // This thread's sample of the next tile, loaded in two dependent levels: the sorted record
  // (position, record index), then the record's (dL/dz3, dL/draw) and ReLU masks.  The first level
  // of tile t + 1 is issued when tile t starts, the second after its first MMA wait, so the loads
  // run behind tile t's work.
  uint4 n_td = make_uint4(0u, 0u, 0u, 0u), n_m1 = n_td, n_m2 = n_td;
  float4 n_pw = make_float4(0.f, 0.f, 0.f, 0.f), n_dz = n_pw;
  uint32_t n_rid = 0;
  auto level_a = [&](uint32_t t) {
    n_td = w.tile[t];
    if (m < (int)(n_td.y & 0xFFu)) {
      n_pw = w.srt[n_td.x + m].pw;
      n_rid = __float_as_uint(w.srt[n_td.x + m].qd.x);
    }
  };
  auto level_b = [&]() {
    if (m < (int)(n_td.y & 0xFFu)) {
      n_dz = w.rec_c[n_rid];
      n_m1 = w.rec_mask[2 * (size_t)n_rid];
      n_m2 = w.rec_mask[2 * (size_t)n_rid + 1];
    }
  };
  if (t_begin + grp < t_end) {
    level_a(t_begin + grp);
    level_b();
  }
  for (uint32_t ti = t_begin + grp; ti < t_end && alive; ti += bt::kGroups) {
    const uint4 td = n_td;
    const float4 pw = n_pw, dzw = n_dz;
    const uint4 m1 = n_m1, m2 = n_m2;
    const float draw = dzw.w;
    const bool more = ti + bt::kGroups < t_end;
    if (more) level_a(ti + bt::kGroups);
    const int mcnt = (int)(td.y & 0xFFu);
    const int bx = (int)(td.w & 0xFFFFu), by = (int)(td.w >> 16), bz = (int)((td.y >> 8) & 0x1FFFu);
    // the weight gradients' operands of this sample (with d_mlp): column td.x + m of the staging
    char* stg = (WG && m < mcnt) ? w.stage + stage_col(td.x + m) : nullptr;
    // this thread's sample: its voxel, weights of the colour gradient
    bool ok = false;
    float dz0 = 0.f, dz1 = 0.f, dz2 = 0.f, f[3] = {0.f, 0.f, 0.f};
    int i0[3] = {0, 0, 0};
    if (m < mcnt) {
      const float p[3] = {pw.x, pw.y, pw.z};
      const bool in = index_sample(g, p, i0, f);
      const int l[3] = {i0[0] - bx * B, i0[1] - by * B, i0[2] - bz * B};
      ok = in && l[0] >= 0 && l[0] < B && l[1] >= 0 && l[1] < B && l[2] >= 0 && l[2] < B;
      if (!ok) {
        set_err(&w.hdr[0], kErrInternal);
      } else {
        dz0 = dzw.x;
        dz1 = dzw.y;
        dz2 = dzw.z;
      }
    }
    // dh2 = (dz3 W3) masked by relu'(z2): row m of A, one half of the hidden units at a time
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
      const HalfMask mk(m2, h);
      const float4* w30 = reinterpret_cast<const float4*>(w3s + 64 * h);
      const float4* w31 = reinterpret_cast<const float4*>(w3s + kHidden + 64 * h);
      const float4* w32 = reinterpret_cast<const float4*>(w3s + 2 * kHidden + 64 * h);
#pragma unroll
      for (int k0 = 0; k0 < kHidden / 2; k0 += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const float4 a = w30[(k0 >> 2) + q], b = w31[(k0 >> 2) + q], c = w32[(k0 >> 2) + q];
          const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int j = 0; j < 4; j++)
            v[4 * q + j] = mk[k0 + 4 * q + j] ? av[j] * dz0 + bv[j] * dz1 + cv[j] * dz2 : 0.0f;
        }
        uint4 hi, lo;
        split8(v, hi, lo);
        store_rows(a_hi, a_lo, m, 64 * h + k0, kHidden, hi, lo);
        if (WG && stg) stage_put(stg, WgStage::dh2, kHidden, (64 * h + k0) / 8, hi, lo);
      }
    }
    if (WG && stg) {
      const float v[8] = {dz0, dz1, dz2, 0.f, 0.f, 0.f, 0.f, 0.f};
      uint4 hi, lo;
      split8(v, hi, lo);
      stage_put(stg, WgStage::dz, 8, 0, hi, lo);
    }
    fence_proxy_async();
    fence_before();
    group_sync(grp);
    // dh1 = dh2 W2 into the group's columns [0, 128)
    if (m == 0) {
      fence_after();
      mma_split(tmem, ah, al, b2h, b2l, idesc_bf16(kHidden));
      mma_commit(bar);
    }
    alive = group_sync_and(grp, mbar_wait(bar, phase, &w.hdr[0]));
    fence_after();
    if (!alive) break;
    phase ^= 1u;
    if (more) level_b();
    // dh1 masked by relu'(z1) -> row m of A (dh2 is no longer read), one half at a time
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
      const HalfMask mk(m1, h);
      float v[64];
      tmem_ld<64>(taddr + 64 * h, v);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = mk[q * 8 + j] ? v[q * 8 + j] : 0.0f;
        uint4 hi, lo;
        split8(x, hi, lo);
        store_rows(a_hi, a_lo, m, 64 * h + q * 8, kHidden, hi, lo);
        if (WG && stg) stage_put(stg, WgStage::dh1, kHidden, 8 * h + q, hi, lo);
      }
    }
    fence_proxy_async();
    fence_before();
    group_sync(grp);
    // dL/dfeatures = dh1 W1[:, :C] into the group's columns [0, 16)
    if (m == 0) {
      fence_after();
      mma_split(tmem, ah, al, b1h, b1l, idesc_bf16(bt::kN1));
      mma_commit(bar);
    }
    alive = group_sync_and(grp, mbar_wait(bar, phase, &w.hdr[0]));
    fence_after();
    if (!alive) break;
    phase ^= 1u;
    float dft[16];
    tmem_ld<16>(taddr, dft);
    fence_before();
    // trilinear adjoint, the eight corners (the next tile's first group barrier also orders these
    // TMEM reads before the next MMA into the same columns)
    if (ok) {
#pragma unroll
      for (int q = 0; q < 8; q++)
        scatter_corner<bt::kN1>(C, vec, corner_vertex(g, i0[0], i0[1], i0[2], q), corner_weight(f[0], f[1], f[2], q),
                                [&](int c) { return dft[c]; }, draw, d_dens, d_feat);
    }
  }
  if (!alive) mbar_wait(bar, phase, &w.hdr[0]);  // MMAs may still be running (bounded)
  fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(bt::kTmemCols)
                 : "memory");
  }
}


// ------------------------------------------------------------------------------------------------
// The backward's forward recompute on the tensor cores.  Per tile of 128 samples of one brick:
// x -> h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> c = sigmoid(W3 h2 + b3), layers 1 and 2 as
// tcgen05 MMAs on split-BF16 operands (hi + lo, three products per K step as in k_bwd_brick_tc,
// FP32 accumulation in TMEM), the biases, layer 3 and the sigmoid in FP32 on the CUDA cores.  It
// writes what the backward reads: (c, w) into rec_c and the ReLU masks of layers 1 and 2 into
// rec_mask.  Two independent groups of 128 threads per CTA (alternate tiles, each its own operand
// region, TMEM columns and mbarrier), one thread per sample: the thread interpolates its sample's
// eight corners, stages its FP32 input row in shared memory (the row then read back in chunks), and
// takes all 128 hidden units in the epilogues, 64 at a time.
//
// A ReLU decision taken on a split-BF16 pre-activation can differ from the FP32 one where the
// pre-activation is within the products' error of zero, and one flipped mask moves that sample's
// whole gradient through the unit.  So each decision is checked against an estimate of that
// error: unit n of layer 1 is uncertain when |z1_n| <= eps ||W1_n|| ||x||, unit n of layer 2 when
// |z2_n| <= eps ||W2_n|| (||h1|| + ||x|| ||W1||_F) (its own products plus layer 1's errors carried
// through W2).  Each split product drops terms of at most ~3 2^-18 |w x|, and the rounding errors
// of a K-term sum add up like a random walk, to ~2^-17 ||w o x||_2, while ||w|| ||x|| is about
// sqrt(K) ||w o x||_2: eps = 2^-17 leaves a margin of 7 to 11 times the typical error (K = 48,
// 128).  The samples with an uncertain decision are listed (their sorted record index, in rec_key,
// which the Ray Index Table no longer needs; count in hdr[4]) and recomputed by the FP32 MLP
// afterwards (k_fwd_fix), so their masks are the FP32 path's.  On the 8192-ray workload 8.6% of
// the samples are listed (16.5% with eps = 2^-16, 4.4% with 2^-18; the gradients of the three
// parity scenes agree with the FP64 oracle to ~5e-6 in all three cases, and to 2e-3 without the
// fix-up).
namespace xt {
constexpr int kGroups = 2;
constexpr int kThreads = kGroups * kTile;  // one thread per sample of each group's 128-sample tile
constexpr int kK1 = 48;                    // layer-1 K: in_dim padded to a multiple of 16
constexpr int kMaxC = 16;                  // feature channels
constexpr int kXS = kK1 + 1;               // FP32 row stride of the staged inputs (odd: rows in distinct banks)
constexpr float kEps = 7.62939453125e-06f;  // 2^-17
// A group's operand region (64 KB).  While x is built: the FP32 rows at [0, 128 kXS 4) and the
// layer-1 operand x (hi, lo; K = 48) at [40 KB, 64 KB).  From layer 1's epilogue on: h1 hi at
// [0, 32 KB), lo at [32 KB, 64 KB), written once layer 1's MMA has read x and every row was read.
struct Region {
  static constexpr int xs = 0;
  static constexpr int x_hi = 40 * 1024;
  static constexpr int x_lo = x_hi + kTile * kK1 * 2;
  static constexpr int h_hi = 0;
  static constexpr int h_lo = kTile * kHidden * 2;
  static constexpr int bytes = 2 * kTile * kHidden * 2;
  static_assert(xs + kTile * kXS * 4 <= x_hi && x_lo + kTile * kK1 * 2 == bytes, "region layout");
};
struct Smem {
  static constexpr int w1_hi = 0;                             // [128][48] bf16: row n, K = k: W1[n][k]
  static constexpr int w1_lo = w1_hi + kHidden * kK1 * 2;
  static constexpr int w2_hi = w1_lo + kHidden * kK1 * 2;     // [128][128] bf16: row n, K = k: W2[n][k]
  static constexpr int w2_lo = w2_hi + kHidden * kHidden * 2;
  static constexpr int region = w2_lo + kHidden * kHidden * 2;  // kGroups operand regions
  static constexpr int prm = region + kGroups * Region::bytes;  // b1 [128], b2 [128], w3 [3][128], b3 [4] f32
  static constexpr int nrm = prm + (5 * kHidden + 4) * 4;     // ||W1_n|| [128], ||W2_n|| [128], ||W1||_F f32
  static constexpr int bars = nrm + (2 * kHidden + 4) * 4;    // one mbarrier per group; TMEM address at +16
  static constexpr int bytes = bars + 128;
  static_assert(region % 16 == 0 && w2_hi % 16 == 0 && bars % 16 == 0, "alignment");
};
constexpr uint32_t kTmemCols = kGroups * 128;  // 128 columns per group
}  // namespace xt

bool fwd_x3_supported(const GridGeo& g, const MlpPtrs& mlp) {
  return g.C <= xt::kMaxC && mlp.in_dim <= xt::kK1 && mlp.in_dim == g.C + 3 + 6 * mlp.n_freq;
}

// Bits of this thread's ReLU decisions: unit 64 h + n (n < 64) is bit ((n / 4) % 4) * 8 + 4 h + n % 4
// of word n / 16 (the rec_mask layout)
__device__ __forceinline__ void relu_bit(uint32_t mw[4], int n, int h, bool on) {
  mw[n >> 4] |= (on ? 1u : 0u) << (((n >> 2) & 3) * 8 + 4 * h + (n & 3));
}

// BWD: the backward's recompute (masks, uncertain samples listed); otherwise a forward render's
// Feature Computation (colours only).  WG (with BWD): also stage x, h1 and h2 for the weight gradients.
template <typename T, bool BWD, bool WG = false>
__global__ void __launch_bounds__(xt::kThreads, 1) k_fwd_x3(GridGeo g, MlpPtrs mlp, RenderWs w,
                                                            const T* __restrict__ feat) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  const int C = g.C, B = g.brick;
  const int m = threadIdx.x & (kTile - 1), grp = threadIdx.x / kTile;
  char* region = sm + xt::Smem::region + grp * xt::Region::bytes;
  char* h_hi = region + xt::Region::h_hi;
  char* h_lo = region + xt::Region::h_lo;
  float* xs = (float*)(region + xt::Region::xs) + m * xt::kXS;  // this sample's FP32 row
  float* b1s = (float*)(sm + xt::Smem::prm);
  float* b2s = b1s + kHidden;
  float* w3s = b2s + kHidden;
  float* b3s = w3s + 3 * kHidden;
  float* nw1 = (float*)(sm + xt::Smem::nrm);
  float* nw2 = nw1 + kHidden;
  float* fro1 = nw2 + kHidden;
  uint64_t* bar = (uint64_t*)(sm + xt::Smem::bars) + grp;
  uint32_t* tslot = (uint32_t*)(sm + xt::Smem::bars + 16);
  // the weights, split into the hi and lo B operands; the other parameters in FP32
  for (int i = threadIdx.x; i < kHidden * (xt::kK1 / 8); i += xt::kThreads) {
    const int n = i / (xt::kK1 / 8), k0 = (i % (xt::kK1 / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = k0 + j < mlp.in_dim ? mlp.w1[n * mlp.in_dim + k0 + j] : 0.0f;
    store_chunk_split(sm + xt::Smem::w1_hi, sm + xt::Smem::w1_lo, n, k0, xt::kK1, v);
  }
  for (int i = threadIdx.x; i < kHidden * (kHidden / 8); i += xt::kThreads) {
    const int n = i / (kHidden / 8), k0 = (i % (kHidden / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = mlp.w2[n * kHidden + k0 + j];
    store_chunk_split(sm + xt::Smem::w2_hi, sm + xt::Smem::w2_lo, n, k0, kHidden, v);
  }
  for (int i = threadIdx.x; i < kHidden; i += xt::kThreads) {
    b1s[i] = mlp.b1[i];
    b2s[i] = mlp.b2[i];
  }
  for (int i = threadIdx.x; i < 3 * kHidden; i += xt::kThreads) w3s[i] = mlp.w3[i];
  if (threadIdx.x < 4) b3s[threadIdx.x] = threadIdx.x < 3 ? mlp.b3[threadIdx.x] : 0.0f;
  if constexpr (BWD) {  // row norms of W1 (threads < 128) and W2 (the others)
    const int n = threadIdx.x & (kHidden - 1);
    float s2 = 0.0f;
    if (threadIdx.x < kHidden)
      for (int k = 0; k < mlp.in_dim; k++) s2 = fmaf(mlp.w1[n * mlp.in_dim + k], mlp.w1[n * mlp.in_dim + k], s2);
    else
      for (int k = 0; k < kHidden; k++) s2 = fmaf(mlp.w2[n * kHidden + k], mlp.w2[n * kHidden + k], s2);
    (threadIdx.x < kHidden ? nw1 : nw2)[n] = sqrtf(s2);
  }
  if (threadIdx.x == 0) {
    for (int j = 0; j < xt::kGroups; j++) mbar_init((uint64_t*)(sm + xt::Smem::bars) + j, 1);
    fence_mbar_init();
  }
  fence_proxy_async();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(xt::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (BWD && threadIdx.x == 0) {  // read after the first tile's first group barrier
    float f2 = 0.0f;
    for (int n = 0; n < kHidden; n++) f2 = fmaf(nw1[n], nw1[n], f2);
    *fro1 = sqrtf(f2);
  }
  __syncthreads();
  const uint32_t tmem_base = *tslot;
  const uint32_t tmem = tmem_base + 128u * (uint32_t)grp;                             // this group's columns
  const uint32_t taddr = tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16);  // this warp's lanes
  const uint64_t ax_h = smem_desc(smem_u32(region + xt::Region::x_hi), 128u, xt::kK1 * 16);
  const uint64_t ax_l = smem_desc(smem_u32(region + xt::Region::x_lo), 128u, xt::kK1 * 16);
  const uint64_t ah_h = smem_desc(smem_u32(h_hi), 128u, kHidden * 16), ah_l = smem_desc(smem_u32(h_lo), 128u, kHidden * 16);
  const uint64_t b1h = smem_desc(smem_u32(sm + xt::Smem::w1_hi), 128u, xt::kK1 * 16);
  const uint64_t b1l = smem_desc(smem_u32(sm + xt::Smem::w1_lo), 128u, xt::kK1 * 16);
  const uint64_t b2h = smem_desc(smem_u32(sm + xt::Smem::w2_hi), 128u, kHidden * 16);
  const uint64_t b2l = smem_desc(smem_u32(sm + xt::Smem::w2_lo), 128u, kHidden * 16);
  const int ne = 3 + 6 * mlp.n_freq;
  uint32_t phase = 0;
  bool alive = true;

  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * per, t_end = min(n_tiles, t_begin + per);
  // this thread's sorted record of the group's next tile, loaded when the current tile starts
  uint4 n_td = make_uint4(0u, 0u, 0u, 0u);
  float4 n_pw = make_float4(0.f, 0.f, 0.f, 0.f), n_qd = n_pw;
  auto prefetch = [&](uint32_t t) {
    n_td = w.tile[t];
    if (m < (int)(n_td.y & 0xFFu)) {
      n_pw = w.srt[n_td.x + m].pw;
      n_qd = w.srt[n_td.x + m].qd;
    }
  };
  if (t_begin + grp < t_end) prefetch(t_begin + grp);
  for (uint32_t ti = t_begin + grp; ti < t_end && alive; ti += xt::kGroups) {
    const uint4 td = n_td;
    const float4 pw = n_pw, qd = n_qd;
    if (ti + xt::kGroups < t_end) prefetch(ti + xt::kGroups);
    const uint32_t start = td.x;
    const int mcnt = (int)(td.y & 0xFFu);
    const int bx = (int)(td.w & 0xFFFFu), by = (int)(td.w >> 16), bz = (int)((td.y >> 8) & 0x1FFFu);
    const bool valid = m < mcnt;
    // the weight gradients' operands of this sample (backward with d_mlp): column start + m
    char* stg = (BWD && WG && valid) ? w.stage + stage_col(start + m) : nullptr;
    uint32_t rid = 0;
    float wgt = 0.0f, fx[xt::kMaxC];
#pragma unroll
    for (int c = 0; c < xt::kMaxC; c++) fx[c] = 0.0f;
    if (valid) {
      rid = __float_as_uint(qd.x);
      wgt = pw.w;
      const float p[3] = {pw.x, pw.y, pw.z};
      int i0[3];
      float f[3];
      const bool in = index_sample(g, p, i0, f);
      const int l[3] = {i0[0] - bx * B, i0[1] - by * B, i0[2] - bz * B};
      if (!(in && l[0] >= 0 && l[0] < B && l[1] >= 0 && l[1] < B && l[2] >= 0 && l[2] < B)) {
        set_err(&w.hdr[0], kErrInternal);
      } else {
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const float wq = corner_weight(f[0], f[1], f[2], q);
          const T* v = feat + corner_vertex(g, i0[0], i0[1], i0[2], q) * (size_t)C;
#pragma unroll
          for (int c = 0; c < xt::kMaxC; c++)
            if (c < C) fx[c] = fmaf(wq, ldf(v + c), fx[c]);
        }
      }
    }
    // this sample's FP32 row of x (features, direction encoding, zeros), staged, then split into
    // the layer-1 operand 8 K values at a time
#pragma unroll
    for (int c = 0; c < xt::kMaxC; c++)
      if (c < C) xs[c] = fx[c];
    if (valid) {
      const float d[3] = {qd.y, qd.z, qd.w};
      encode_dir(d, mlp.n_freq, xs + C);
    } else {
      for (int j = 0; j < ne; j++) xs[C + j] = 0.0f;
    }
    for (int k = C + ne; k < xt::kK1; k++) xs[k] = 0.0f;
    float x2 = 0.0f;
#pragma unroll
    for (int j = 0; j < xt::kK1 / 8; j++) {
      float v[8];
#pragma unroll
      for (int t = 0; t < 8; t++) {
        v[t] = xs[8 * j + t];
        x2 = fmaf(v[t], v[t], x2);
      }
      uint4 hi, lo;
      split8(v, hi, lo);
      store_rows(region + xt::Region::x_hi, region + xt::Region::x_lo, m, 8 * j, xt::kK1, hi, lo);
      if (WG && stg) stage_put(stg, WgStage::x, xt::kK1, j, hi, lo);
    }
    fence_proxy_async();
    fence_before();
    group_sync(grp);
    // layer 1: W1 x into the group's columns [0, 128)
    if (m == 0) {
      fence_after();
      mma_split<xt::kK1 / 16>(tmem, ax_h, ax_l, b1h, b1l, idesc_bf16(kHidden));
      mma_commit(bar);
    }
    alive = group_sync_and(grp, mbar_wait(bar, phase, &w.hdr[0]));
    fence_after();
    if (!alive) break;
    phase ^= 1u;
    uint32_t mw1[4] = {0u, 0u, 0u, 0u}, mw2[4] = {0u, 0u, 0u, 0u};
    const float tx = xt::kEps * sqrtf(x2);
    bool unsure = false;
    float h2s = 0.0f;  // ||h1||^2
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
      float v[64];
      tmem_ld<64>(taddr + 64 * h, v);
      const float4* b4 = reinterpret_cast<const float4*>(b1s + 64 * h);  // per-unit constants, 4 at a time
      const float4* n4 = reinterpret_cast<const float4*>(nw1 + 64 * h);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        float x[8];
#pragma unroll
        for (int t4 = 0; t4 < 2; t4++) {
          const float4 bq = b4[2 * q + t4];
          const float bv[4] = {bq.x, bq.y, bq.z, bq.w};
          float nv[4] = {0.f, 0.f, 0.f, 0.f};
          if constexpr (BWD) {
            const float4 nq = n4[2 * q + t4];
            nv[0] = nq.x;
            nv[1] = nq.y;
            nv[2] = nq.z;
            nv[3] = nq.w;
          }
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const int t = 4 * t4 + j, n = 8 * q + t;
            const float z = v[n] + bv[j];
            if constexpr (BWD) {
              relu_bit(mw1, n, h, z > 0.0f);
              unsure |= fabsf(z) <= tx * nv[j];
            }
            x[t] = fmaxf(z, 0.0f);
            h2s = fmaf(x[t], x[t], h2s);
          }
        }
        uint4 hi, lo;
        split8(x, hi, lo);
        store_rows(h_hi, h_lo, m, 64 * h + 8 * q, kHidden, hi, lo);
        if (WG && stg) stage_put(stg, WgStage::h1, kHidden, 8 * h + q, hi, lo);
      }
    }
    fence_proxy_async();
    fence_before();
    group_sync(grp);
    // layer 2: W2 h1 into the group's columns [0, 128)
    if (m == 0) {
      fence_after();
      mma_split(tmem, ah_h, ah_l, b2h, b2l, idesc_bf16(kHidden));
      mma_commit(bar);
    }
    alive = group_sync_and(grp, mbar_wait(bar, phase, &w.hdr[0]));
    fence_after();
    if (!alive) break;
    phase ^= 1u;
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;
    float h2v[8];  // h2 of 8 consecutive units, staged once complete (WG)
    const float th = BWD ? xt::kEps * (sqrtf(h2s) + sqrtf(x2) * *fro1) : 0.0f;
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
      float v[64];
      tmem_ld<64>(taddr + 64 * h, v);
      const float4* b4 = reinterpret_cast<const float4*>(b2s + 64 * h);  // per-unit constants, 4 at a time
      const float4* n4 = reinterpret_cast<const float4*>(nw2 + 64 * h);
      const float4* w0 = reinterpret_cast<const float4*>(w3s + 64 * h);
      const float4* w1 = reinterpret_cast<const float4*>(w3s + kHidden + 64 * h);
      const float4* w2 = reinterpret_cast<const float4*>(w3s + 2 * kHidden + 64 * h);
#pragma unroll
      for (int n4i = 0; n4i < 16; n4i++) {
        const float4 bq = b4[n4i], c0 = w0[n4i], c1 = w1[n4i], c2 = w2[n4i];
        const float bv[4] = {bq.x, bq.y, bq.z, bq.w};
        const float u0[4] = {c0.x, c0.y, c0.z, c0.w}, u1[4] = {c1.x, c1.y, c1.z, c1.w}, u2[4] = {c2.x, c2.y, c2.z, c2.w};
        float nv[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (BWD) {
          const float4 nq = n4[n4i];
          nv[0] = nq.x;
          nv[1] = nq.y;
          nv[2] = nq.z;
          nv[3] = nq.w;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int n = 4 * n4i + j;
          const float z = v[n] + bv[j];
          if constexpr (BWD) {
            relu_bit(mw2, n, h, z > 0.0f);
            unsure |= fabsf(z) <= th * nv[j];
          }
          const float a2 = fmaxf(z, 0.0f);
          if constexpr (WG) h2v[4 * (n4i & 1) + j] = a2;
          z0 = fmaf(u0[j], a2, z0);
          z1 = fmaf(u1[j], a2, z1);
          z2 = fmaf(u2[j], a2, z2);
        }
        if (WG && stg && (n4i & 1)) {  // units 64 h + 8 (n4i / 2) .. + 7 complete
          uint4 hi, lo;
          split8(h2v, hi, lo);
          stage_put(stg, WgStage::h2, kHidden, 8 * h + n4i / 2, hi, lo);
        }
      }
    }
    fence_before();
    if constexpr (BWD) {  // list the uncertain samples (one atomic per warp)
      const bool fix = valid && unsure;
      const uint32_t bal = __ballot_sync(0xffffffffu, fix);
      uint32_t base = 0;
      if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(&w.hdr[4], (uint32_t)__popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (fix) w.rec_key[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = start + m;
    }
    if (valid) {
      w.rec_c[rid] = make_float4(sigmoid_f(z0 + b3s[0]), sigmoid_f(z1 + b3s[1]), sigmoid_f(z2 + b3s[2]), wgt);
      if constexpr (BWD) {
        w.rec_mask[2 * (size_t)rid] = make_uint4(mw1[0], mw1[1], mw1[2], mw1[3]);
        w.rec_mask[2 * (size_t)rid + 1] = make_uint4(mw2[0], mw2[1], mw2[2], mw2[3]);
      }
    }
  }
  if (!alive) mbar_wait(bar, phase, &w.hdr[0]);  // MMAs may still be running (bounded)
  fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(xt::kTmemCols)
                 : "memory");
  }
}

cicero_status launch_fwd_x3(const cicero_grid* grid, const GridGeo& geo, const MlpPtrs& mlp, const RenderWs& ws,
                            cudaStream_t st) {
  const bool f16 = grid->dtype == CICERO_F16, bwd = ws.rec_mask != nullptr;
  cudaError_t e = cudaSuccess;
  const int sb = xt::Smem::bytes;
  const dim3 grid_dim(num_sms()), block(xt::kThreads);
  {
    ProfScope ps(kStGatherMlp, st);
    if (bwd && ws.stage) {  // the backward with the weight gradients' staging
      if (f16) {
        e = cudaFuncSetAttribute(k_fwd_x3<__half, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess)
          k_fwd_x3<__half, true, true><<<grid_dim, block, sb, st>>>(geo, mlp, ws, (const __half*)grid->features);
      } else {
        e = cudaFuncSetAttribute(k_fwd_x3<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess)
          k_fwd_x3<float, true, true><<<grid_dim, block, sb, st>>>(geo, mlp, ws, (const float*)grid->features);
      }
    } else if (f16) {
      const __half* feat = (const __half*)grid->features;
      if (bwd) {
        e = cudaFuncSetAttribute(k_fwd_x3<__half, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess) k_fwd_x3<__half, true><<<grid_dim, block, sb, st>>>(geo, mlp, ws, feat);
      } else {
        e = cudaFuncSetAttribute(k_fwd_x3<__half, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess) k_fwd_x3<__half, false><<<grid_dim, block, sb, st>>>(geo, mlp, ws, feat);
      }
    } else {
      const float* feat = (const float*)grid->features;
      if (bwd) {
        e = cudaFuncSetAttribute(k_fwd_x3<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess) k_fwd_x3<float, true><<<grid_dim, block, sb, st>>>(geo, mlp, ws, feat);
      } else {
        e = cudaFuncSetAttribute(k_fwd_x3<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess) k_fwd_x3<float, false><<<grid_dim, block, sb, st>>>(geo, mlp, ws, feat);
      }
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fwd_x3)");
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_fwd_x3");
}

// ------------------------------------------------------------------------------------------------
// The MLP weight gradients on the tensor cores, from the operands that the recompute (x, h1, h2)
// and B2 (dL/dh2, dL/dh1, dL/dz3) staged per composited sample, already split into BF16 hi and lo
// in the MN-major layout the MMAs read (WgStage; K = the block's 16 samples, in sorted order).
// They are sums over the samples s of outer products,
//   dW2 = sum_s dh2_s h1_s^T    M = 128, N = 128     db2 = sum_s dh2_s    (against a ones operand)
//   dW1 = sum_s dh1_s x_s^T     M = 128, N = 48      db1 = sum_s dh1_s
//   dW3^T = sum_s h2_s dz3_s^T  M = 128, N = 16 (3 used)   db3 = sum_s dz3_s (A = ones)
// taken as tcgen05 MMAs with K = 16 samples per step on split-BF16 operands (three products as in
// k_bwd_brick_tc; the biases two: hi and lo against exact ones), each CTA accumulating its range of
// samples in TMEM and adding the sums to d_mlp once.  Staged blocks (36 KB each) stream in by bulk
// copies into a ring of kRing buffers, kRing - 1 of them in flight, and feed the MMAs as they are:
// the kernel converts nothing.
namespace dw {
constexpr int kThreads = 128;                  // thread 0 runs the pipeline; all four warps read TMEM out
constexpr int kRing = 6;                       // staged blocks in shared memory (copies in flight)
constexpr int kBuf = WgStage::bytes + 256;     // a staged block and a zero row group (dL/dz3 rows 8..15)
struct Smem {
  static constexpr int ring = 0;                     // [kRing][kBuf]
  static constexpr int ones = ring + kRing * kBuf;   // [128][16] BF16 ones: A of db3, B of db1 and db2
  static constexpr int bars = ones + 4096;           // full [kRing], free [kRing]; TMEM address after
  static constexpr int bytes = bars + 16 * kRing + 16;
  static_assert(kBuf % 16 == 0 && ones % 16 == 0 && bars % 16 == 0, "alignment");
};
// tensor memory: dW2 [0, 128), db2 [128, 144), dW1 [160, 208), db1 [208, 224), dW3^T [224, 240), db3 [240, 256)
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColB2 = 128, kColW1 = 160, kColB1 = 208, kColW3 = 224, kColB3 = 240;
}  // namespace dw

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// MLP weight gradients over all composited samples, from the staged operands (WgStage): per block
// of 16 samples, D += A B^T with K = the samples, split-BF16 products (hi hi + hi lo + lo hi):
//   [dW2 | db2] = dL/dh2^T [h1 | 1],  [dW1 | db1] = dL/dh1^T [x | 1],  dW3^T = h2^T dL/dz3,
//   db3 = 1^T dL/dz3,
// both operands MN-major (the staged rows), accumulated in TMEM over the CTA's blocks and added to
// d_mlp once per CTA.  Thread 0 streams the blocks through a ring of kRing buffers with bulk copies
// (one mbarrier per buffer for the copy, one for the MMAs that read it) and issues the MMAs.
__global__ void __launch_bounds__(dw::kThreads, 1) k_dw(MlpPtrs mlp, RenderWs w, float* d_mlp) {
  using namespace tc;
  extern __shared__ __align__(1024) char sm[];
  const int I = mlp.in_dim;
  const uint32_t n = w.hdr[2];  // composited samples: staged columns [0, n)
  const uint32_t nblk = (n + kStageBlock - 1) / kStageBlock;
  const uint32_t per = (nblk + gridDim.x - 1) / gridDim.x;
  const uint32_t b0 = blockIdx.x * per, b1 = min(nblk, b0 + per);
  if (b0 >= b1) return;  // nothing to add (uniform per CTA, before any barrier or TMEM use)
  uint64_t* full = (uint64_t*)(sm + dw::Smem::bars);  // [kRing]: the buffer's copy landed
  uint64_t* fre = full + dw::kRing;                   // [kRing]: the MMAs reading the buffer are done
  uint32_t* tslot = (uint32_t*)(fre + dw::kRing);
  // the last block's columns from n on are written by no producer: zero them in global memory
  // (every row group of every operand) before a copy reads them
  const uint32_t kt = n % kStageBlock;
  if (b1 == nblk && kt != 0) {
    char* blk = w.stage + (size_t)(nblk - 1) * WgStage::bytes;
    const int nk = kStageBlock - (int)kt;
    for (int i = threadIdx.x; i < (WgStage::bytes / 256) * nk; i += dw::kThreads)
      *reinterpret_cast<uint4*>(blk + 256 * (i / nk) + 16 * ((int)kt + i % nk)) = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.global;" ::: "memory");  // before the async proxy's copies
  }
  // constants: the ones operand, each buffer's zero row group
  for (int i = threadIdx.x; i < 4096 / 16; i += dw::kThreads)
    *reinterpret_cast<uint4*>(sm + dw::Smem::ones + 16 * i) = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  for (int i = threadIdx.x; i < dw::kRing * 16; i += dw::kThreads)
    *reinterpret_cast<uint4*>(sm + dw::Smem::ring + (i / 16) * dw::kBuf + WgStage::bytes + 16 * (i % 16)) =
        make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    for (int j = 0; j < dw::kRing; j++) {
      mbar_init(full + j, 1);
      mbar_init(fre + j, 1);
    }
    fence_mbar_init();
  }
  fence_proxy_async();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(dw::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  bool alive = true;
  if (threadIdx.x == 0) {
    // block b into buffer p: the byte count expected, then one bulk copy
    auto issue = [&](uint32_t b, int p) {
      static_assert(WgStage::bytes % 16 == 0, "bulk copy sizes must be multiples of 16 bytes");
      mbar_expect_tx(full + p, WgStage::bytes);
      bulk_load(sm + dw::Smem::ring + p * dw::kBuf, w.stage + (size_t)b * WgStage::bytes, WgStage::bytes, full + p);
    };
    // descriptors of buffer 0 (buffer p lies p kBuf further; the address field counts 16 bytes):
    // MN-major, K-adjacent core matrices (8 samples) 128 bytes apart, row groups 256 bytes apart;
    // dL/dz3's hi half with its row groups 512 bytes apart, so that rows 8..15 are the zero group
    const uint32_t r0 = smem_u32(sm + dw::Smem::ring);
    auto op = [&](int off, int R, int half) { return smem_desc(r0 + off + half * 32 * R, 128u, 256u); };
    const uint64_t dh2h = op(WgStage::dh2, kHidden, 0), dh2l = op(WgStage::dh2, kHidden, 1);
    const uint64_t h1h = op(WgStage::h1, kHidden, 0), h1l = op(WgStage::h1, kHidden, 1);
    const uint64_t dh1h = op(WgStage::dh1, kHidden, 0), dh1l = op(WgStage::dh1, kHidden, 1);
    const uint64_t h2h = op(WgStage::h2, kHidden, 0), h2l = op(WgStage::h2, kHidden, 1);
    const uint64_t xh = op(WgStage::x, kMaxIn, 0), xl = op(WgStage::x, kMaxIn, 1);
    const uint64_t dzh = smem_desc(r0 + WgStage::dz, 128u, 512u), dzl = op(WgStage::dz, 8, 1);
    const uint64_t one = smem_desc(smem_u32(sm + dw::Smem::ones), 128u, 256u);
    constexpr uint32_t iw2 = idesc_bf16_mn(kHidden), ib = idesc_bf16_mn(16), iw1 = idesc_bf16_mn(kMaxIn);
    uint32_t fph = 0u, eph = 0u;  // parity of each buffer's next copy and next MMA completion
    uint32_t issued = b0, landed = b0, mma_from = b0, mma_to = b0;  // copies [landed, issued) and MMA
                                                                     // commits [mma_from, mma_to) pending
    for (; issued < min(b1, b0 + (uint32_t)dw::kRing); issued++) issue(issued, (int)(issued - b0));
    for (uint32_t b = b0; b < b1 && alive; b++) {
      const int p = (int)((b - b0) % dw::kRing);
      alive = mbar_wait(full + p, (fph >> p) & 1u, &w.hdr[0]);
      if (!alive) break;
      fph ^= 1u << p;
      landed = b + 1;
      fence_after();
      const uint64_t o = (uint64_t)(p * dw::kBuf) >> 4;
      const uint32_t acc = b == b0 ? 0u : 1u;
      mma_bf16(tmem, dh2h + o, h1h + o, iw2, acc);
      mma_bf16(tmem, dh2h + o, h1l + o, iw2, 1u);
      mma_bf16(tmem, dh2l + o, h1h + o, iw2, 1u);
      mma_bf16(tmem + dw::kColB2, dh2h + o, one, ib, acc);
      mma_bf16(tmem + dw::kColB2, dh2l + o, one, ib, 1u);
      mma_bf16(tmem + dw::kColW1, dh1h + o, xh + o, iw1, acc);
      mma_bf16(tmem + dw::kColW1, dh1h + o, xl + o, iw1, 1u);
      mma_bf16(tmem + dw::kColW1, dh1l + o, xh + o, iw1, 1u);
      mma_bf16(tmem + dw::kColB1, dh1h + o, one, ib, acc);
      mma_bf16(tmem + dw::kColB1, dh1l + o, one, ib, 1u);
      mma_bf16(tmem + dw::kColW3, h2h + o, dzh + o, ib, acc);
      mma_bf16(tmem + dw::kColW3, h2h + o, dzl + o, ib, 1u);
      mma_bf16(tmem + dw::kColW3, h2l + o, dzh + o, ib, 1u);
      mma_bf16(tmem + dw::kColB3, one, dzh + o, ib, acc);
      mma_bf16(tmem + dw::kColB3, one, dzl + o, ib, 1u);
      mma_commit(fre + p);
      mma_to = b + 1;
      // block b - 1's MMAs done: its buffer takes the next copy
      if (b > b0) {
        const int pp = (int)((b - 1 - b0) % dw::kRing);
        alive = mbar_wait(fre + pp, (eph >> pp) & 1u, &w.hdr[0]);
        if (!alive) break;
        eph ^= 1u << pp;
        mma_from = b;
        if (issued < b1) {
          issue(issued, pp);
          issued++;
        }
      }
    }
    // the last MMAs; after a timeout, also the MMAs and the copies still in flight (bounded waits)
    for (uint32_t b = mma_from; b < mma_to; b++) {
      const int pp = (int)((b - b0) % dw::kRing);
      if (mbar_wait(fre + pp, (eph >> pp) & 1u, &w.hdr[0])) eph ^= 1u << pp;
      else alive = false;
    }
    for (uint32_t b = landed; b < issued; b++) {
      const int pp = (int)((b - b0) % dw::kRing);
      if (mbar_wait(full + pp, (fph >> pp) & 1u, &w.hdr[0])) fph ^= 1u << pp;
      alive = false;
    }
  }
  fence_before();
  alive = __syncthreads_and(alive);
  fence_after();
  if (alive) {
    // d_mlp = [W1 [128][I], b1 [128], W2 [128][128], b2 [128], W3 [3][128], b3 [3]]
    float* dW1 = d_mlp;
    float* db1 = dW1 + kHidden * I;
    float* dW2 = db1 + kHidden;
    float* db2 = dW2 + kHidden * kHidden;
    float* dW3 = db2 + kHidden;
    float* db3 = dW3 + 3 * kHidden;
    const int un = threadIdx.x;  // this thread's hidden unit: TMEM lane (warp w reads lanes 32 w ..)
    const uint32_t taddr = tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
    float v[64];
    tmem_ld<64>(taddr, v);
#pragma unroll
    for (int k = 0; k < 64; k++) atomicAdd(&dW2[un * kHidden + k], v[k]);
    tmem_ld<64>(taddr + 64, v);
#pragma unroll
    for (int k = 0; k < 64; k++) atomicAdd(&dW2[un * kHidden + 64 + k], v[k]);
    tmem_ld<32>(taddr + dw::kColW1, v);
#pragma unroll
    for (int k = 0; k < 32; k++)
      if (k < I) atomicAdd(&dW1[un * I + k], v[k]);
    tmem_ld<16>(taddr + dw::kColW1 + 32, v);
#pragma unroll
    for (int k = 0; k < 16; k++)
      if (32 + k < I) atomicAdd(&dW1[un * I + 32 + k], v[k]);
    tmem_ld<16>(taddr + dw::kColB2, v);
    atomicAdd(&db2[un], v[0]);
    tmem_ld<16>(taddr + dw::kColB1, v);
    atomicAdd(&db1[un], v[0]);
    tmem_ld<16>(taddr + dw::kColW3, v);
#pragma unroll
    for (int j = 0; j < 3; j++) atomicAdd(&dW3[j * kHidden + un], v[j]);
    tmem_ld<16>(taddr + dw::kColB3, v);  // every lane holds db3
    if (un == 0)
#pragma unroll
      for (int j = 0; j < 3; j++) atomicAdd(&db3[j], v[j]);
  }
  fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(dw::kTmemCols) : "memory");
  }
}

cicero_status launch_dw(const MlpPtrs& mlp, const RenderWs& ws, float* d_mlp, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, dw::Smem::bytes);
  if (e == cudaSuccess) {
    k_dw<<<num_sms(), dw::kThreads, dw::Smem::bytes, st>>>(mlp, ws, d_mlp);
    e = cudaGetLastError();
  }
  count_launches(1);
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_dw");
}

template <typename T, bool WG>
static cudaError_t launch_bwd_brick(const RenderPlan& plan, const RaySrc& src, const MlpPtrs& mlp, const RenderWs& ws,
                                    const void* feat, float* d_dens, float* d_feat, float* d_mlp,
                                    int smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_bwd_brick<T, WG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_bwd_brick<T, WG><<<num_sms(), 256, smem, st>>>(plan.geo, src, mlp, ws, (const T*)feat, d_dens, d_feat, d_mlp);
  return cudaGetLastError();
}

cicero_status run_backward(const cicero_grid* grid, const MlpPtrs& mlp, const RenderPlan& plan, const RaySrc& src,
                           const RenderWs& ws, const float* d_rgb, float* d_dens, float* d_feat, float* d_mlp,
                           cudaStream_t st) {
  OutBufs none;
  memset(&none, 0, sizeof none);
  cicero_status s = run_render(grid, mlp, plan, src, ws, none, false, st);
  if (s != CICERO_OK) return s;
  const int nw = src.n_max;
  int blocks = (nw + 7) / 8;
  blocks = std::max(1, std::min(blocks, num_sms() * 16));
  {
    ProfScope ps(kStBwdRay, st);
    k_bwd_ray<<<blocks, 256, 0, st>>>(src, plan.samp, ws, d_rgb, plan.geo.act_shift);
  }
  count_launches(2);
  const int smem = BwdSmem::bytes;
  const bool f16 = grid->dtype == CICERO_F16;
  cudaError_t e;
  const int smem_tc = bt::Smem::bytes;
  if (ws.rec_mask && plan.geo.C <= bt::kN1 && (!d_mlp || ws.stage)) {
    // grid gradients on the tensor cores, with the recompute's ReLU masks; with d_mlp, the weight
    // gradients' operands staged on the way and the weight gradients as tensor-core GEMMs after
    {
      ProfScope ps(kStBwdBrick, st);
      if (ws.stage) {
        e = cudaFuncSetAttribute(k_bwd_brick_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tc);
        if (e == cudaSuccess)
          k_bwd_brick_tc<true><<<num_sms(), bt::kThreads, smem_tc, st>>>(plan.geo, mlp, ws, d_dens, d_feat);
      } else {
        e = cudaFuncSetAttribute(k_bwd_brick_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tc);
        if (e == cudaSuccess)
          k_bwd_brick_tc<false><<<num_sms(), bt::kThreads, smem_tc, st>>>(plan.geo, mlp, ws, d_dens, d_feat);
      }
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "backward kernels");
    }
    if (!d_mlp) return CICERO_OK;
    ProfScope ps(kStBwdWeights, st);
    return launch_dw(mlp, ws, d_mlp, st);
  }
  ProfScope ps(kStBwdBrick, st);
  if (d_mlp)
    e = f16 ? launch_bwd_brick<__half, true>(plan, src, mlp, ws, grid->features, d_dens, d_feat, d_mlp, smem, st)
            : launch_bwd_brick<float, true>(plan, src, mlp, ws, grid->features, d_dens, d_feat, d_mlp, smem, st);
  else
    e = f16 ? launch_bwd_brick<__half, false>(plan, src, mlp, ws, grid->features, d_dens, d_feat, nullptr, smem,
                                              st)
            : launch_bwd_brick<float, false>(plan, src, mlp, ws, grid->features, d_dens, d_feat, nullptr, smem,
                                             st);
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "backward kernels");
}

}  // namespace cicero
