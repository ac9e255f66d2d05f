// Device-side building blocks shared by the kernels of libcicero (sm_103a).
//
// The "decision" helpers (ray generation, slot placement, voxel and cell indexing, brick ids)
// use explicit round-to-nearest intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn), which
// the compiler never contracts into FMAs, so every kernel that recomputes a sample position gets
// the same bits as the kernel that bucketed it.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cicero {

constexpr int kWarp = 32;
constexpr int kTile = 128;          // samples per Feature-Computation tile (MMA M)
constexpr int kHidden = 128;
constexpr int kMaxIn = 48;          // MLP input padded to 48 (3 x K16 MMA steps)

// error bits recorded in the workspace header
constexpr uint32_t kErrInternal = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrCapacity = 4u;   // the record capacity of the workspace was exceeded
constexpr long long kWaitCycles = 4ll << 30;  // bounded mbarrier waits: ~2 s of SM clock

// -------------------------------------------------------------------------------------------
// descriptors passed by value to kernels

struct GridGeo {
  int n[3];
  int C;
  float amin[3], amax[3];
  float inv_h[3];      // (n - 1) / (amax - amin), rounded to FP32 on the host
  float occ_scale[3];  // R / (n - 1), rounded to FP32 on the host
  float act_shift;
  int occ_res;
  const uint8_t* occ;
  int brick;           // voxels per brick edge (a power of two)
  int brick_shift;     // log2(brick)
  int nb[3];           // bricks per axis
  int idx32;           // 1 when every vertex index fits in 31 bits (32-bit address arithmetic)
};

struct Samp {
  float near_t, far_t;
  int n_samples;
  float step;
  float t_stop;
  float bg[3];
  float void_acc;
};

constexpr int kMaxViews = 32;

struct ViewCam {
  float c2w[12];
  float f, cx, cy;
  int width;
};

// Where the rays of a call come from.
//   kind 0: pixels of cam[0] (all of them, or the list pix[0] of *n_dev / n_max entries)
//   kind 1: explicit rays o, d [n_max][3]
//   kind 2: the pixel lists pix[v] of n_views cameras, n_dev[v] entries each (device counts)
struct RaySrc {
  int kind;
  int n_views;
  int n_max;              // host bound on the total ray count
  const int32_t* n_dev;   // device ray count(s) or NULL
  const float* o;
  const float* d;
  const int32_t* pix[kMaxViews];
  ViewCam cam[kMaxViews];
};

__device__ __forceinline__ int ray_count(const RaySrc& s) {
  long long n = s.n_max;
  if (s.kind == 2) {
    long long t = 0;
    for (int v = 0; v < s.n_views; v++) t += max(0, s.n_dev[v]);
    n = t < n ? t : n;
  } else if (s.n_dev) {
    const int c = *s.n_dev;
    n = c < n ? (c < 0 ? 0 : c) : n;
  }
  return (int)n;
}

// Which view and which pixel (ray index for explicit rays) ray r is.
struct RayRef {
  int view;
  int pix;
};

__device__ __forceinline__ RayRef ray_ref(const RaySrc& s, int r) {
  RayRef q;
  q.view = 0;
  q.pix = r;
  if (s.kind == 0) {
    if (s.pix[0]) q.pix = s.pix[0][r];
  } else if (s.kind == 2) {
    int base = 0;
    for (int v = 0; v < s.n_views; v++) {
      const int n = max(0, s.n_dev[v]);
      if (r < base + n) {
        q.view = v;
        q.pix = s.pix[v][r - base];
        return q;
      }
      base += n;
    }
  }
  return q;
}

// Ray through pixel `pix` of camera c: pinhole model of Eq. 1 / Eq. 3 (centre (i + 1/2, j + 1/2)).
__device__ __forceinline__ void ray_gen_cam(const ViewCam& c, int pix, float o[3], float d[3]) {
  const int i = pix % c.width, j = pix / c.width;
  const float u = __fadd_rn((float)i, 0.5f), v = __fadd_rn((float)j, 0.5f);
  const float dx = __fdiv_rn(__fsub_rn(u, c.cx), c.f);
  const float dy = __fdiv_rn(__fsub_rn(v, c.cy), c.f);
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; a++)
    w[a] = __fadd_rn(__fadd_rn(__fmul_rn(c.c2w[4 * a], dx), __fmul_rn(c.c2w[4 * a + 1], dy)), c.c2w[4 * a + 2]);
  const float nn =
      __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(w[0], w[0]), __fmul_rn(w[1], w[1])), __fmul_rn(w[2], w[2])));
#pragma unroll
  for (int a = 0; a < 3; a++) {
    d[a] = __fdiv_rn(w[a], nn);
    o[a] = c.c2w[4 * a + 3];
  }
}

// Ray of pixel/ray r of a ray source.
__device__ __forceinline__ void ray_gen(const RaySrc& s, const RayRef& q, float o[3], float d[3]) {
  if (s.kind == 1) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      o[a] = s.o[3 * q.pix + a];
      d[a] = s.d[3 * q.pix + a];
    }
    return;
  }
  ray_gen_cam(s.cam[q.view], q.pix, o, d);
}

// Slot placement: t_k = t0 + (k + 1/2) dt for k < n (and t_k < t_out in box-march mode).
struct Slots {
  int n;
  float t0, dt, tout;
  bool march;
};

__device__ __forceinline__ Slots place_slots(const GridGeo& g, const Samp& s, const float o[3], const float d[3]) {
  Slots r;
  r.march = s.step > 0.0f;
  if (!r.march) {
    r.n = s.n_samples;
    r.t0 = s.near_t;
    r.dt = __fdiv_rn(__fsub_rn(s.far_t, s.near_t), (float)s.n_samples);
    r.tout = 0.0f;
    return r;
  }
  r.dt = s.step;
  r.t0 = 0.0f;
  r.tout = 0.0f;
  r.n = 0;
  float lo = s.near_t, hi = s.far_t;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (d[a] == 0.0f) {
      if (o[a] < g.amin[a] || o[a] > g.amax[a]) return r;
      continue;
    }
    float t0 = __fdiv_rn(__fsub_rn(g.amin[a], o[a]), d[a]);
    float t1 = __fdiv_rn(__fsub_rn(g.amax[a], o[a]), d[a]);
    if (t0 > t1) {
      float q = t0;
      t0 = t1;
      t1 = q;
    }
    if (t0 > lo) lo = t0;
    if (t1 < hi) hi = t1;
  }
  if (!(lo < hi)) return r;
  r.t0 = lo;
  r.tout = hi;
  r.n = s.n_samples;
  return r;
}

__device__ __forceinline__ float slot_t(const Slots& sl, int k) {
  return __fadd_rn(sl.t0, __fmul_rn(__fadd_rn((float)k, 0.5f), sl.dt));
}

__device__ __forceinline__ bool slot_valid(const Slots& sl, int k, float t) {
  return k < sl.n && (!sl.march || t < sl.tout);
}

__device__ __forceinline__ void sample_pos(const float o[3], const float d[3], float t, float p[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) p[a] = __fadd_rn(o[a], __fmul_rn(t, d[a]));
}

// Position p and ray direction d of slot k of a ray whose geometry is ot = (origin, t0) and
// dd = (direction, dt): the march's own operations (slot_t, sample_pos), so the bits are the
// march's.
__device__ __forceinline__ void sample_of(const float4& ot, const float4& dd, uint32_t k, float p[3], float d[3]) {
  Slots sl;
  sl.t0 = ot.w;
  sl.dt = dd.w;
  const float t = slot_t(sl, (int)k);
  const float o[3] = {ot.x, ot.y, ot.z};
  d[0] = dd.x;
  d[1] = dd.y;
  d[2] = dd.z;
  sample_pos(o, d, t, p);
}

// Indexing (Sec. II-B): continuous vertex coordinate g, voxel i0 = min(floor g, n - 2) and the
// fraction inside the voxel; false when the sample is outside the box or in an empty cell.
__device__ __forceinline__ bool index_sample(const GridGeo& g, const float p[3], int i0[3], float f[3]) {
  int cell[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float ga = __fmul_rn(__fsub_rn(p[a], g.amin[a]), g.inv_h[a]);
    if (!(ga >= 0.0f && ga <= (float)(g.n[a] - 1))) return false;
    int i = (int)floorf(ga);
    if (i > g.n[a] - 2) i = g.n[a] - 2;
    i0[a] = i;
    f[a] = __fsub_rn(ga, (float)i);
    if (g.occ) {
      int c = (int)floorf(__fmul_rn(ga, g.occ_scale[a]));
      if (c > g.occ_res - 1) c = g.occ_res - 1;
      cell[a] = c;
    }
  }
  if (g.occ) {
    int R = g.occ_res;
    if (!__ldg(&g.occ[((size_t)cell[2] * R + cell[1]) * R + cell[0]])) return false;
  }
  return true;
}

__device__ __forceinline__ uint32_t brick_id(const GridGeo& g, const int i0[3]) {
  const int sh = g.brick_shift;
  return (uint32_t)(((i0[2] >> sh) * g.nb[1] + (i0[1] >> sh)) * g.nb[0] + (i0[0] >> sh));
}

// Sort key of a sample in the Ray Index Table: its brick (offset by the job's first brick in a
// batch) times kOctants plus the octant of the brick its voxel lies in (x, y, z halves).  Keys of
// one brick are consecutive, so the table groups samples by brick exactly as the paper's RIT and,
// inside a brick, by octant.  For bricks of 4 voxels an octant is a 2x2x2 block of voxels whose
// 8 voxels (24 B each, rows of 5 in the staged box) sit in 8 distinct pairs of shared-memory
// banks, so the trilinear loads of samples from one octant never conflict.
constexpr int kOctants = 8;
__device__ __forceinline__ uint32_t brick_key(const GridGeo& g, const int i0[3], uint32_t brick_base) {
  const int h = g.brick_shift - 1;
  const uint32_t oct = (uint32_t)(((i0[0] >> h) & 1) | (((i0[1] >> h) & 1) << 1) | (((i0[2] >> h) & 1) << 2));
  return (brick_base + brick_id(g, i0)) * kOctants + oct;
}

template <typename T>
__device__ __forceinline__ float ldf(const T* p);
template <>
__device__ __forceinline__ float ldf<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldf<__half>(const __half* p) { return __half2float(__ldg(p)); }

// Trilinear density from the global grid (read through the read-only path).
template <typename T>
__device__ __forceinline__ float density_trilinear(const GridGeo& g, const T* dens, const int i0[3], const float f[3]) {
  const T *p00, *p01, *p10, *p11;  // the four x-pairs of corners: (y, z) = (0,0), (1,0), (0,1), (1,1)
  if (g.idx32) {
    const int nx = g.n[0], nxy = g.n[0] * g.n[1];
    const int b = (i0[2] * g.n[1] + i0[1]) * nx + i0[0];
    p00 = dens + b;
    p01 = dens + (b + nx);
    p10 = dens + (b + nxy);
    p11 = dens + (b + nxy + nx);
  } else {
    const size_t nx = g.n[0], nxy = (size_t)g.n[0] * g.n[1];
    const size_t b = (size_t)i0[2] * nxy + (size_t)i0[1] * nx + i0[0];
    p00 = dens + b;
    p01 = dens + b + nx;
    p10 = dens + b + nxy;
    p11 = dens + b + nxy + nx;
  }
  float v000 = ldf(p00), v001 = ldf(p00 + 1);
  float v010 = ldf(p01), v011 = ldf(p01 + 1);
  float v100 = ldf(p10), v101 = ldf(p10 + 1);
  float v110 = ldf(p11), v111 = ldf(p11 + 1);
  float fx = f[0], fy = f[1], fz = f[2];
  float c00 = v000 + fx * (v001 - v000), c01 = v010 + fx * (v011 - v010);
  float c10 = v100 + fx * (v101 - v100), c11 = v110 + fx * (v111 - v110);
  float c0 = c00 + fy * (c01 - c00), c1 = c10 + fy * (c11 - c10);
  return c0 + fz * (c1 - c0);
}

__device__ __forceinline__ float softplus_f(float x) { return x > 20.0f ? x : log1pf(expf(x)); }
// softplus with the hardware exp/log (relative error ~1e-6; for x < -16 it returns 0 instead of ~e^x)
__device__ __forceinline__ float softplus_fast(float x) { return x > 15.0f ? x : __logf(1.0f + __expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// View-direction encoding: d, then sin/cos(2^k d) by the double-angle recurrence
// sin 2a = 2 sin a cos a, cos 2a = 1 - 2 sin^2 a (exact identities; error < 1e-6 for |d| <= 1).
__device__ __forceinline__ void encode_dir(const float d[3], int n_freq, float* x /* 3 + 6 n_freq */) {
  float s[3], c[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    x[a] = d[a];
    sincosf(d[a], &s[a], &c[a]);
  }
  for (int k = 0; k < n_freq; k++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      x[3 + 6 * k + a] = s[a];
      x[3 + 6 * k + 3 + a] = c[a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      float s2 = 2.0f * s[a] * c[a];
      float c2 = 1.0f - 2.0f * s[a] * s[a];
      s[a] = s2;
      c[a] = c2;
    }
  }
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bits) { atomicOr(err, bits); }

// -------------------------------------------------------------------------------------------
// PTX wrappers: shared-memory addresses, mbarrier, TMA, tcgen05

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Waits for the phase with the given parity; the warp may sleep for a system-chosen time per try
// (an explicit 10 us suspend hint measured ~1% slower on the tensor-core gather).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: returns false (after recording a timeout) if the phase
// did not complete within kWaitCycles SM clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 < kWaitCycles)
    if (mbar_try_wait(bar, parity)) return true;
  set_err(err, kErrTimeout);
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace cicero
