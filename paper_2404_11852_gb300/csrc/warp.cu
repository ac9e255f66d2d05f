// SpaRW target-frame warping (Sec. III-B, steps 1-3 and the hole/void handling of step 4).
//
//   W1 k_zclear    depth buffer <- all ones
//   W2 k_splat     per reference pixel: Eq. 1 (point from depth), Eq. 2 (rigid transform),
//                  Eq. 3 (projection) and the depth test as one 64-bit atomicMin of
//                  (float bits of Z') << 32 | reference index
//   W3 k_resolve   per target pixel: copy the winner's colour, or classify the hole (void when
//                  its ray has no sample in the grid box / occupied cells)
//   W4 k_hole_*    stream compaction of the holes in ascending pixel order (block scans)
// All decision arithmetic uses explicit round-to-nearest intrinsics (no FMA contraction).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace cicero {

struct Splat {
  bool ok;
  int px, py;
  float X, Y, Z;
  bool inf;
};

__device__ __forceinline__ Splat splat_point(const WarpArgs& a, const float* ref_depth, int q) {
  Splat s;
  s.ok = false;
  const int i = q % a.wr, j = q / a.wr;
  const float u = __fadd_rn((float)i, 0.5f), v = __fadd_rn((float)j, 0.5f);
  const float dx = __fdiv_rn(__fsub_rn(u, a.cxr), a.fr);
  const float dy = __fdiv_rn(__fsub_rn(v, a.cyr), a.fr);
  const float D = ref_depth[q];
  float P[3];
  const bool at_inf = isinf(D) && D > 0.0f;
  if (at_inf) {
    P[0] = dx;
    P[1] = dy;
    P[2] = 1.0f;
  } else {
    if (!(D > 0.0f)) return s;
    const float nrm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), 1.0f));
    const float Z = __fdiv_rn(D, nrm);
    P[0] = __fmul_rn(dx, Z);
    P[1] = __fmul_rn(dy, Z);
    P[2] = Z;
  }
  float Q[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float acc =
        __fadd_rn(__fadd_rn(__fmul_rn(a.R[3 * k], P[0]), __fmul_rn(a.R[3 * k + 1], P[1])), __fmul_rn(a.R[3 * k + 2], P[2]));
    Q[k] = at_inf ? acc : __fadd_rn(acc, a.t[k]);
  }
  if (!(Q[2] > 1e-6f)) return s;
  const float up = __fadd_rn(__fdiv_rn(__fmul_rn(a.ft, Q[0]), Q[2]), a.cxt);
  const float vp = __fadd_rn(__fdiv_rn(__fmul_rn(a.ft, Q[1]), Q[2]), a.cyt);
  if (!(up >= 0.0f && up < (float)a.wt && vp >= 0.0f && vp < (float)a.ht)) return s;
  if (a.use_phi && !at_inf) {
    const float A0 = __fsub_rn(Q[0], a.t[0]), A1 = __fsub_rn(Q[1], a.t[1]), A2 = __fsub_rn(Q[2], a.t[2]);
    const float dot = __fadd_rn(__fadd_rn(__fmul_rn(A0, Q[0]), __fmul_rn(A1, Q[1])), __fmul_rn(A2, Q[2]));
    const float na = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(A0, A0), __fmul_rn(A1, A1)), __fmul_rn(A2, A2)));
    const float nq = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(Q[0], Q[0]), __fmul_rn(Q[1], Q[1])), __fmul_rn(Q[2], Q[2])));
    if (!(dot > __fmul_rn(a.cos_phi, __fmul_rn(na, nq)))) return s;
  }
  s.ok = true;
  s.px = (int)floorf(up);
  s.py = (int)floorf(vp);
  s.X = Q[0];
  s.Y = Q[1];
  s.Z = Q[2];
  s.inf = at_inf;
  return s;
}

__global__ void k_zclear(unsigned long long* z, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) z[i] = ~0ull;
}

__global__ void __launch_bounds__(256) k_splat(WarpArgs a, const float* __restrict__ ref_depth, unsigned long long* z) {
  const int n = a.wr * a.hr;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const Splat s = splat_point(a, ref_depth, q);
    if (!s.ok) continue;
    const float zk = s.inf ? __int_as_float(0x7f800000) : s.Z;
    const unsigned long long key = ((unsigned long long)__float_as_uint(zk) << 32) | (unsigned int)q;
    atomicMin(&z[s.py * a.wt + s.px], key);
  }
}

// Void depth test of pixel p by a whole warp: 32 slots per step, stop at the first slot that
// is inside the box (and in an occupied cell).  Same FP32 slot placement and indexing as rendering.
__device__ __forceinline__ bool warp_ray_has_sample(const VoidTest& vt, int p) {
  const int lane = threadIdx.x & 31;
  float o[3], d[3];
  RayRef rr;
  rr.view = 0;
  rr.pix = p;
  ray_gen(vt.src, rr, o, d);
  const Slots sl = place_slots(vt.g, vt.s, o, d);
  for (int k0 = 0; k0 < sl.n; k0 += 32) {
    const int k = k0 + lane;
    const float t = slot_t(sl, k);
    const bool valid = slot_valid(sl, k, t);
    bool in = false;
    if (valid) {
      float pp[3], f[3];
      int i0[3];
      sample_pos(o, d, t, pp);
      in = index_sample(vt.g, pp, i0, f);
    }
    if (__any_sync(0xffffffffu, in)) return true;
    if (!__all_sync(0xffffffffu, valid)) return false;
  }
  return false;
}

// One warp per 32 consecutive target pixels.
__global__ void __launch_bounds__(256) k_resolve(WarpArgs a, VoidTest vt, const float* __restrict__ ref_rgb,
                                                 const float* __restrict__ ref_depth, const unsigned long long* z,
                                                 float* wrgb, float* wdepth, uint8_t* mask) {
  const int n = a.wt * a.ht;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int p0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; p0 < n; p0 += nwarps * 32) {
    const int p = p0 + lane;
    const bool px = p < n;
    const unsigned long long key = px ? z[p] : 0ull;
    const bool hole = px && key == ~0ull;
    if (px && !hole) {
      const int q = (int)(key & 0xffffffffull);
      wrgb[3 * p + 0] = ref_rgb[3 * q + 0];
      wrgb[3 * p + 1] = ref_rgb[3 * q + 1];
      wrgb[3 * p + 2] = ref_rgb[3 * q + 2];
      if (wdepth) {
        const Splat s = splat_point(a, ref_depth, q);
        wdepth[p] = s.inf ? __int_as_float(0x7f800000)
                          : __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(s.X, s.X), __fmul_rn(s.Y, s.Y)), __fmul_rn(s.Z, s.Z)));
      }
      mask[p] = 0;
    }
    if (hole) {
      wrgb[3 * p + 0] = 0.0f;
      wrgb[3 * p + 1] = 0.0f;
      wrgb[3 * p + 2] = 0.0f;
      if (wdepth) wdepth[p] = 0.0f;
      mask[p] = vt.enabled ? 3 : 1;  // 3: hole still to be tested for void
    }
  }
}

// Void depth test of the listed candidates, one warp each (candidates cluster in the image, so
// testing them where they lie would serialise a warp's worth of marches).
__global__ void __launch_bounds__(256) k_void(VoidTest vt, const int32_t* cand, const int32_t* n_cand, float* wrgb,
                                              float* wdepth, uint8_t* mask) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = *n_cand;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const int p = cand[i];
    const bool v = !warp_ray_has_sample(vt, p);
    if (lane == 0) {
      if (v) {
        wrgb[3 * p + 0] = vt.s.bg[0];
        wrgb[3 * p + 1] = vt.s.bg[1];
        wrgb[3 * p + 2] = vt.s.bg[2];
        if (wdepth) wdepth[p] = __int_as_float(0x7f800000);
        mask[p] = 2;
      } else {
        mask[p] = 1;
      }
    }
  }
}

// Hole compaction: each block of 1024 threads owns kHoleChunk consecutive pixels.
constexpr int kHoleChunk = 4096;

__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t* tot, uint32_t* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const uint32_t r = (wid ? sh[wid - 1] : 0) + x - v;
  *tot = sh[nw - 1];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_hole_count(const uint8_t* mask, int n, uint8_t val, uint32_t* block_sums) {
  __shared__ uint32_t sh[32];
  const int base = blockIdx.x * kHoleChunk + threadIdx.x * 4;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) c += (base + k < n && mask[base + k] == val) ? 1u : 0u;
  uint32_t tot;
  block_exscan(c, &tot, sh);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_hole_blocks(uint32_t* block_sums, int nblocks, int32_t* n_holes) {
  __shared__ uint32_t sh[32];
  uint32_t run = 0;
  for (int b0 = 0; b0 < nblocks; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < nblocks ? block_sums[i] : 0;
    uint32_t tot;
    const uint32_t e = block_exscan(v, &tot, sh);
    if (i < nblocks) block_sums[i] = run + e;
    run += tot;
  }
  if (threadIdx.x == 0) *n_holes = (int32_t)run;
}

__global__ void __launch_bounds__(1024) k_hole_write(const uint8_t* mask, int n, uint8_t val, const uint32_t* block_off,
                                                     int32_t* hole_idx) {
  __shared__ uint32_t sh[32];
  const int base = blockIdx.x * kHoleChunk + threadIdx.x * 4;
  uint32_t c = 0;
  bool h[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    h[k] = base + k < n && mask[base + k] == val;
    c += h[k] ? 1u : 0u;
  }
  uint32_t tot;
  uint32_t pos = block_off[blockIdx.x] + block_exscan(c, &tot, sh);
#pragma unroll
  for (int k = 0; k < 4; k++)
    if (h[k]) hole_idx[pos++] = base + k;
}

// workspace: [256-byte header (error word)] [depth buffer, 8 B per target pixel] [block sums]
size_t warp_ws_bytes(int wt, int ht) {
  const size_t n = (size_t)wt * ht;
  const size_t nb = (n + kHoleChunk - 1) / kHoleChunk;
  return 256 + ((8 * n + 255) & ~size_t(255)) + ((4 * nb + 255) & ~size_t(255));
}

cicero_status run_warp(const WarpArgs& a, const VoidTest& vt, const float* ref_rgb, const float* ref_depth,
                       float* wrgb, float* wdepth, uint8_t* mask, int32_t* hole_idx, int32_t* n_holes, void* ws,
                       cudaStream_t st) {
  const int nt = a.wt * a.ht, nr = a.wr * a.hr;
  unsigned long long* z = (unsigned long long*)((char*)ws + 256);
  uint32_t* bsum = (uint32_t*)((char*)ws + 256 + ((8 * (size_t)nt + 255) & ~size_t(255)));
  const int nblk = (nt + kHoleChunk - 1) / kHoleChunk;
  const int g = num_sms() * 8;
  {
    ProfScope ps(kStWarpSplat, st);
    k_zclear<<<std::min(g, (nt + 255) / 256), 256, 0, st>>>(z, nt);
    k_splat<<<std::min(g, (nr + 255) / 256), 256, 0, st>>>(a, ref_depth, z);
  }
  {
    ProfScope ps(kStWarpResolve, st);
    k_resolve<<<std::min(g, (nt + 255) / 256), 256, 0, st>>>(a, vt, ref_rgb, ref_depth, z, wrgb, wdepth, mask);
    if (vt.enabled) {  // list the candidates, test them, then list the holes that remain
      k_hole_count<<<nblk, 1024, 0, st>>>(mask, nt, 3, bsum);
      k_hole_blocks<<<1, 1024, 0, st>>>(bsum, nblk, n_holes);
      k_hole_write<<<nblk, 1024, 0, st>>>(mask, nt, 3, bsum, hole_idx);
      k_void<<<g, 256, 0, st>>>(vt, hole_idx, n_holes, wrgb, wdepth, mask);
      count_launches(4);
    }
    k_hole_count<<<nblk, 1024, 0, st>>>(mask, nt, 1, bsum);
    k_hole_blocks<<<1, 1024, 0, st>>>(bsum, nblk, n_holes);
    k_hole_write<<<nblk, 1024, 0, st>>>(mask, nt, 1, bsum, hole_idx);
  }
  count_launches(6);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "warp kernels");
}

// -------------------------------------------------------------------------------------------
// Allocation-free warp.  Some callers cannot allocate device memory: code running while a stream
// is being captured into a CUDA graph (cudaMalloc is not allowed there), real-time loops that must
// not enter the allocator, or host programs linking this library without a device allocator of
// their own.  For them cicero_warp_noalloc uses a scratch array that is part of the library's
// device image instead of a caller-provided workspace.

namespace {

constexpr int kNoAllocMaxPixels = 1024 * 1024;  // largest target image (width * height)
constexpr size_t kNoAllocBytes = 256 + ((8 * (size_t)kNoAllocMaxPixels + 255) & ~size_t(255)) +
                                 ((4 * (size_t)((kNoAllocMaxPixels + kHoleChunk - 1) / kHoleChunk) + 255) & ~size_t(255));

// Depth buffer and scan sums of the allocation-free warp (~8 MiB on every device that loads the
// library, held until the process exits).  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cicero_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(CICERO_ERR_UNSUPPORTED, "device index out of range");
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CICERO_OK;
}

}  // namespace

}  // namespace cicero

extern "C" cicero_status cicero_warp_noalloc(const float* ref_rgb, const float* ref_depth,
                                             const cicero_camera* ref_cam, const cicero_camera* tgt_cam,
                                             float max_angle_deg, const cicero_grid* void_grid,
                                             const cicero_sampling* void_sampling, float* warped_rgb,
                                             float* warped_depth, uint8_t* hole_mask, int32_t* hole_idx,
                                             int32_t* n_holes, void* stream) {
  using namespace cicero;
  if (!tgt_cam) return fail(CICERO_ERR_INVALID_ARG, "tgt_cam is NULL");
  if ((long long)tgt_cam->width * tgt_cam->height > kNoAllocMaxPixels)
    return fail(CICERO_ERR_UNSUPPORTED, "cicero_warp_noalloc: the target image exceeds 1048576 pixels "
                                        "(the size of its built-in scratch); use cicero_warp with a workspace");
  void* scratch = nullptr;
  cicero_status st = noalloc_scratch(&scratch);
  if (st != CICERO_OK) return st;
  return cicero_warp(ref_rgb, ref_depth, ref_cam, tgt_cam, max_angle_deg, void_grid, void_sampling, warped_rgb,
                     warped_depth, hole_mask, hole_idx, n_holes, scratch, kNoAllocBytes, stream);
}

