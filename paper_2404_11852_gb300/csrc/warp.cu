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

#include <atomic>

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

// Kernels take the whole batch of target views as a __grid_constant__ parameter; blockIdx.y is
// the view.
__global__ void k_zclear(const __grid_constant__ WarpBatch B) {
  const WarpView& V = B.v[blockIdx.y];
  const int n = V.a.wt * V.a.ht;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) V.z[i] = ~0ull;
}

__global__ void __launch_bounds__(256) k_splat(const __grid_constant__ WarpBatch B, const float* __restrict__ ref_depth) {
  const WarpView& V = B.v[blockIdx.y];
  const int n = V.a.wr * V.a.hr;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const Splat s = splat_point(V.a, ref_depth, q);
    if (!s.ok) continue;
    const float zk = s.inf ? __int_as_float(0x7f800000) : s.Z;
    const unsigned long long key = ((unsigned long long)__float_as_uint(zk) << 32) | (unsigned int)q;
    atomicMin(&V.z[s.py * V.a.wt + s.px], key);
  }
}

// Void depth test of pixel p of view v by a whole warp: 32 slots per step, stop at the first slot
// that is inside the box (and in an occupied cell).  Same FP32 slot placement and indexing as
// rendering.
__device__ __forceinline__ bool warp_ray_has_sample(const VoidTest& vt, const float o[3], const float d[3],
                                                    const Slots& sl) {
  const int lane = threadIdx.x & 31;
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

// One warp per 32 consecutive target pixels: copy the winners, mark the holes (3 = still to be
// tested for void when the void test is on, else 1).
__global__ void __launch_bounds__(256) k_resolve(const __grid_constant__ WarpBatch B, int void_on,
                                                 const float* __restrict__ ref_rgb, const float* __restrict__ ref_depth) {
  const WarpView& V = B.v[blockIdx.y];
  const int n = V.a.wt * V.a.ht;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int p0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; p0 < n; p0 += nwarps * 32) {
    const int p = p0 + lane;
    if (p >= n) continue;
    const unsigned long long key = V.z[p];
    if (key != ~0ull) {
      const int q = (int)(key & 0xffffffffull);
      V.wrgb[3 * p + 0] = ref_rgb[3 * q + 0];
      V.wrgb[3 * p + 1] = ref_rgb[3 * q + 1];
      V.wrgb[3 * p + 2] = ref_rgb[3 * q + 2];
      if (V.wdepth) {
        const Splat s = splat_point(V.a, ref_depth, q);
        V.wdepth[p] = s.inf ? __int_as_float(0x7f800000)
                            : __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(s.X, s.X), __fmul_rn(s.Y, s.Y)), __fmul_rn(s.Z, s.Z)));
      }
      V.mask[p] = 0;
    } else {
      V.wrgb[3 * p + 0] = 0.0f;
      V.wrgb[3 * p + 1] = 0.0f;
      V.wrgb[3 * p + 2] = 0.0f;
      if (V.wdepth) V.wdepth[p] = 0.0f;
      V.mask[p] = void_on ? 3 : 1;
    }
  }
}

// Per-candidate setup shared by a warp: the target ray and its slots.
struct VoidSetup {
  float o[3], d[3];
  float t0, dt, tout;
  int n, march, p;
};

// Void depth test of the listed candidates, one warp each (candidates cluster in the image, so
// testing them where they lie would serialise a warp's worth of marches).  A warp's candidates are
// i = warp + k nwarps; lane j prepares the ray and slots of the j-th of each group of 32 of them,
// which the whole warp then reads from shared memory candidate by candidate.
__global__ void __launch_bounds__(256) k_void(const __grid_constant__ WarpBatch B, const __grid_constant__ VoidTest vt) {
  const int v = blockIdx.y;
  const WarpView& V = B.v[v];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = *V.n_holes;
  __shared__ VoidSetup setup[8][32];
  const int wb = threadIdx.x >> 5;
  for (long long i0 = 0;; i0 += 32) {
    const long long il = (long long)warp + (i0 + lane) * nwarps;
    const unsigned have = __ballot_sync(0xffffffffu, il < n);
    if (!have) break;
    if (il < n) {
      VoidSetup& q = setup[wb][lane];
      RayRef rr;
      rr.view = v;
      rr.pix = V.hole_idx[il];
      float o[3], d[3];
      ray_gen(vt.src, rr, o, d);
      const Slots sl = place_slots(vt.g, vt.s, o, d);
#pragma unroll
      for (int a = 0; a < 3; a++) {
        q.o[a] = o[a];
        q.d[a] = d[a];
      }
      q.t0 = sl.t0;
      q.dt = sl.dt;
      q.tout = sl.tout;
      q.n = sl.n;
      q.march = sl.march ? 1 : 0;
      q.p = rr.pix;
    }
    __syncwarp();
    const int nq = __popc(have);  // il grows with the lane: the candidates present are lanes 0 .. nq-1
    for (int j = 0; j < nq; j++) {
      const VoidSetup& q = setup[wb][j];
      const float o[3] = {q.o[0], q.o[1], q.o[2]}, d[3] = {q.d[0], q.d[1], q.d[2]};
      Slots sl;
      sl.t0 = q.t0;
      sl.dt = q.dt;
      sl.tout = q.tout;
      sl.n = q.n;
      sl.march = q.march != 0;
      const int p = q.p;
      const bool is_void = !warp_ray_has_sample(vt, o, d, sl);
      if (lane == 0) {
        if (is_void) {
          V.wrgb[3 * p + 0] = vt.s.bg[0];
          V.wrgb[3 * p + 1] = vt.s.bg[1];
          V.wrgb[3 * p + 2] = vt.s.bg[2];
          if (V.wdepth) V.wdepth[p] = __int_as_float(0x7f800000);
          V.mask[p] = 2;
        } else {
          V.mask[p] = 1;
        }
      }
    }
    __syncwarp();  // the setup slots are free for the next group
  }
}

// Hole compaction: each block of 1024 threads owns kHoleChunk consecutive pixels of its view.
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

__global__ void __launch_bounds__(1024) k_hole_count(const __grid_constant__ WarpBatch B, uint8_t val) {
  __shared__ uint32_t sh[32];
  const WarpView& V = B.v[blockIdx.y];
  if ((int)blockIdx.x >= V.nblk) return;  // uniform per block
  const int n = V.a.wt * V.a.ht;
  const int base = blockIdx.x * kHoleChunk + threadIdx.x * 4;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) c += (base + k < n && V.mask[base + k] == val) ? 1u : 0u;
  uint32_t tot;
  block_exscan(c, &tot, sh);
  if (threadIdx.x == 0) V.bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_hole_blocks(const __grid_constant__ WarpBatch B) {
  __shared__ uint32_t sh[32];
  const WarpView& V = B.v[blockIdx.y];
  uint32_t run = 0;
  for (int b0 = 0; b0 < V.nblk; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const uint32_t x = i < V.nblk ? V.bsum[i] : 0;
    uint32_t tot;
    const uint32_t e = block_exscan(x, &tot, sh);
    if (i < V.nblk) V.bsum[i] = run + e;
    run += tot;
  }
  if (threadIdx.x == 0) *V.n_holes = (int32_t)run;
}

__global__ void __launch_bounds__(1024) k_hole_write(const __grid_constant__ WarpBatch B, uint8_t val) {
  __shared__ uint32_t sh[32];
  const WarpView& V = B.v[blockIdx.y];
  if ((int)blockIdx.x >= V.nblk) return;
  const int n = V.a.wt * V.a.ht;
  const int base = blockIdx.x * kHoleChunk + threadIdx.x * 4;
  uint32_t c = 0;
  bool h[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    h[k] = base + k < n && V.mask[base + k] == val;
    c += h[k] ? 1u : 0u;
  }
  uint32_t tot;
  uint32_t pos = V.bsum[blockIdx.x] + block_exscan(c, &tot, sh);
#pragma unroll
  for (int k = 0; k < 4; k++)
    if (h[k]) V.hole_idx[pos++] = base + k;
}

// Bilinear resampling of an image (the DS-2 comparator of the evaluation: render at half resolution,
// then upsample).  Pixel centres align: output pixel i samples the source at u = (i + 1/2) w / W - 1/2,
// interpolating the two nearest source pixel centres per axis, clamped to the image.
__global__ void __launch_bounds__(256) k_upsample(const float* __restrict__ src, int w, int h, int C,
                                                  float* __restrict__ dst, int W, int H) {
  const long long n = (long long)W * H;
  const float sx = (float)w / (float)W, sy = (float)h / (float)H;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % W), j = (int)(q / W);
    const float u = fmaxf(((float)i + 0.5f) * sx - 0.5f, 0.0f), v = fmaxf(((float)j + 0.5f) * sy - 0.5f, 0.0f);
    const int x0 = min((int)u, w - 1), y0 = min((int)v, h - 1);
    const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const float fx = fminf(u - (float)x0, 1.0f), fy = fminf(v - (float)y0, 1.0f);
    const float* a = src + ((size_t)y0 * w + x0) * C;
    const float* b = src + ((size_t)y0 * w + x1) * C;
    const float* c = src + ((size_t)y1 * w + x0) * C;
    const float* d = src + ((size_t)y1 * w + x1) * C;
    float* o = dst + (size_t)q * C;
    for (int k = 0; k < C; k++) {
      const float top = a[k] + fx * (b[k] - a[k]), bot = c[k] + fx * (d[k] - c[k]);
      o[k] = top + fy * (bot - top);
    }
  }
}

cicero_status run_upsample(const float* src, int w, int h, int C, float* dst, int W, int H, cudaStream_t st) {
  const long long n = (long long)W * H;
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
  k_upsample<<<blocks, 256, 0, st>>>(src, w, h, C, dst, W, H);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_upsample");
}

static size_t al256w(size_t x) { return (x + 255) & ~size_t(255); }

// workspace: [256-byte header] then per view [depth buffer, 8 B per target pixel] [block sums]
size_t warp_ws_bytes(int wt, int ht) {
  const size_t n = (size_t)wt * ht;
  const size_t nb = (n + kHoleChunk - 1) / kHoleChunk;
  return 256 + al256w(8 * n) + al256w(4 * nb);
}

size_t warp_batch_ws_bytes(const int* wt, const int* ht, int n_views) {
  size_t b = 256;
  for (int v = 0; v < n_views; v++) b += warp_ws_bytes(wt[v], ht[v]) - 256;
  return b;
}

void carve_warp_ws(WarpBatch& B, void* ws) {
  char* q = (char*)ws + 256;
  for (int v = 0; v < B.n_views; v++) {
    const size_t n = (size_t)B.v[v].a.wt * B.v[v].a.ht;
    B.v[v].nblk = (int)((n + kHoleChunk - 1) / kHoleChunk);
    B.v[v].z = (unsigned long long*)q;
    q += al256w(8 * n);
    B.v[v].bsum = (uint32_t*)q;
    q += al256w(4 * (size_t)B.v[v].nblk);
  }
}

cicero_status run_warp(const WarpBatch& B, const VoidTest& vt, const float* ref_rgb, const float* ref_depth,
                       cudaStream_t st) {
  int max_nt = 1, max_blk = 1;
  for (int v = 0; v < B.n_views; v++) {
    max_nt = std::max(max_nt, B.v[v].a.wt * B.v[v].a.ht);
    max_blk = std::max(max_blk, B.v[v].nblk);
  }
  const int nr = B.v[0].a.wr * B.v[0].a.hr;
  const int g = std::max(1, num_sms() * 8 / B.n_views);
  const dim3 gz(std::min(g, (max_nt + 255) / 256), B.n_views), gs(std::min(g, (nr + 255) / 256), B.n_views);
  const dim3 gb(max_blk, B.n_views), g1(1, B.n_views), gv(g, B.n_views);
  {
    ProfScope ps(kStWarpSplat, st);
    k_zclear<<<gz, 256, 0, st>>>(B);
    k_splat<<<gs, 256, 0, st>>>(B, ref_depth);
  }
  {
    ProfScope ps(kStWarpResolve, st);
    k_resolve<<<gz, 256, 0, st>>>(B, vt.enabled, ref_rgb, ref_depth);
    if (vt.enabled) {  // list the candidates, test them, then list the holes that remain
      k_hole_count<<<gb, 1024, 0, st>>>(B, 3);
      k_hole_blocks<<<g1, 1024, 0, st>>>(B);
      k_hole_write<<<gb, 1024, 0, st>>>(B, 3);
      k_void<<<gv, 256, 0, st>>>(B, vt);
      count_launches(4);
    }
    k_hole_count<<<gb, 1024, 0, st>>>(B, 1);
    k_hole_blocks<<<g1, 1024, 0, st>>>(B);
    k_hole_write<<<gb, 1024, 0, st>>>(B, 1);
  }
  count_launches(6);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "warp kernels");
}

// -------------------------------------------------------------------------------------------
// Allocation-free warp.  Some callers cannot allocate device memory: real-time loops that must
// not enter an allocator (an allocation can block for an unbounded time), host programs that link
// this library without any device allocator of their own, and plugins whose host framework owns
// every byte of device memory.  For them cicero_warp_noalloc uses a scratch array that is part of
// the library's device image instead of a caller-provided workspace.

namespace {

constexpr int kNoAllocMaxPixels = 1024 * 1024;  // largest target image (width * height)
constexpr size_t kNoAllocBytes = 256 + ((8 * (size_t)kNoAllocMaxPixels + 255) & ~size_t(255)) +
                                 ((4 * (size_t)((kNoAllocMaxPixels + kHoleChunk - 1) / kHoleChunk) + 255) & ~size_t(255));

// Depth buffer and scan sums of the allocation-free warp (~8 MiB on every device that loads the
// library, held until the process exits).  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
// Per-device address of the scratch array, looked up on the first call on that device.  Atomic
// entries: host threads driving different devices may make their first calls at the same time
// (two threads on one device both look it up and store the same address).  The cache lives as
// long as the process; after cudaDeviceReset on a device its entry is stale.
std::atomic<void*> g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once per device).
cicero_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(CICERO_ERR_UNSUPPORTED, "device index out of range");
  void* p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
  if (!p) {
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev].store(p, std::memory_order_relaxed);
  }
  *out = p;
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

