// Memory-centric voxel-grid NeRF rendering (Sec. II-B stages, reordered as in Sec. IV-A).
//
//   K1 k_march        one warp per ray, 32 slots per step: Indexing, density gathering,
//                     alpha, transmittance by a warp scan of sigma*delta, early stop; reserves an
//                     upper bound of its records, emits one record (position, w, RIT key =
//                     brick x 8 + octant) per composited sample and counts them into the key
//                     histogram
//   K2 k_brick_*      key offsets (3-phase exclusive scan of the histogram, one brick of 8 keys
//                     per thread), tile offsets per brick and the tile list
//   K3 k_scatter      counting sort of the records by key, moving their payload into (brick,
//                     octant) order as 32-byte records: the Ray Index Table
//   K5 k_gather_mlp_f32 / mlp_tc.cu
//                     per brick: one TMA copy of the brick (+1 vertex halo) into shared memory,
//                     trilinear feature gathering from there, view encoding and the MLP
//   K6 k_composite    per ray, in slot order: rgb = sum w c + T_end bg
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace cicero {

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kScanChunk = 1024;  // bricks per block of the RIT offset scan (one per thread)
constexpr size_t kRaySetupBytes = 84;  // sizeof(RaySetup), checked where it is defined

size_t render_ws_bytes(const RenderPlan& p) {
  const size_t Q = p.Q, R = (size_t)p.R;
  size_t b = al256(64);
  b += 3 * al256(4 * R) + al256(16 * R) + al256(32 * R);
  b += 2 * al256(4 * Q) + al256(2 * Q) + al256(16 * Q);
  if (p.want_bwd) b += 2 * al256(4 * Q) + al256(32 * Q);
  if (p.want_k) b += al256(4 * Q);
  if (p.want_wg) b += al256(stage_bytes(p.Q));
  const size_t nk = (size_t)p.nb * kOctants;  // RIT keys: (brick, octant)
  b += 2 * al256(4 * nk) + al256(4 * (nk + 1)) + al256(4 * ((size_t)p.nb + 1));
  b += al256(8 * ((size_t)p.nb / kScanChunk + 2));
  b += al256(16 * (size_t)p.max_tiles);
  b += al256(32 * Q);
  b += al256(kRaySetupBytes * R);
  return b;
}

bool carve_render_ws(void* ws, size_t bytes, const RenderPlan& p, RenderWs* w) {
  if (render_ws_bytes(p) > bytes) return false;
  char* q = (char*)ws;
  const size_t Q = p.Q, R = (size_t)p.R;
  auto take = [&](size_t n) {
    char* r = q;
    q += al256(n);
    return (void*)r;
  };
  w->hdr = (uint32_t*)take(64);
  w->ray_n = (uint32_t*)take(4 * R);
  w->ray_start = (uint32_t*)take(4 * R);
  w->ray_T = (float*)take(4 * R);
  w->ray_dir = (float4*)take(16 * R);
  w->ray_geo = (RayGeo*)take(32 * R);
  w->rec_key = (uint32_t*)take(4 * Q);
  w->rec_w = (float*)take(4 * Q);
  w->rec_slot = (uint16_t*)take(2 * Q);
  w->rec_c = (float4*)take(16 * Q);
  w->rec_T = p.want_bwd ? (float*)take(4 * Q) : nullptr;
  w->rec_raw = p.want_bwd ? (float*)take(4 * Q) : nullptr;
  w->rec_ray = p.want_k ? (uint32_t*)take(4 * Q) : nullptr;
  w->stage = p.want_wg ? (char*)take(stage_bytes(p.Q)) : nullptr;
  w->rec_mask = p.want_bwd ? (uint4*)take(32 * Q) : nullptr;
  const size_t nk = (size_t)p.nb * kOctants;
  w->brick_cnt = (uint32_t*)take(4 * nk);
  w->brick_cur = (uint32_t*)take(4 * nk);
  w->brick_off = (uint32_t*)take(4 * (nk + 1));
  w->tile_off = (uint32_t*)take(4 * ((size_t)p.nb + 1));
  w->blk_sums = (uint32_t*)take(8 * ((size_t)p.nb / kScanChunk + 2));
  w->tile = (uint4*)take(16 * (size_t)p.max_tiles);
  w->srt = (SrtRec*)take(32 * Q);
  w->setup = (RaySetup*)take(kRaySetupBytes * R);
  w->R = p.R;
  w->S = p.S;
  w->nb = p.nb;
  w->max_tiles = p.max_tiles;
  w->Q = p.Q;
  return true;
}

// -------------------------------------------------------------------------------------------

__global__ void k_clear(uint32_t* a, size_t na, uint32_t* b, size_t nb) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x, s = (size_t)gridDim.x * blockDim.x;
  for (size_t k = i; k < na; k += s) a[k] = 0;
  for (size_t k = i; k < nb; k += s) b[k] = 0;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// -------------------------------------------------------------------------------------------
// Exact active-slot masks.  Along one axis, a slot's position p = o + t_k d, its vertex coordinate
// g = (p - min) / h and its occupancy cell floor(g R / (n - 1)) are each a monotone function of
// the slot index k (t_k grows with k and every FP32 operation on the way rounds monotonically), so
// the slots of a ray fall into runs of constant (inside/outside, cell) per axis.  The setup lane of
// a ray walks these runs: it estimates where the next cell boundary is crossed and then finds the
// exact slot by evaluating the same FP32 expressions as index_sample at a few slots, so the mask it
// builds holds exactly the slots index_sample accepts (inside the box, in an occupied cell), while
// evaluating only ~2 slots per cell boundary instead of every slot.

constexpr int kMaskWords = 8;                   // slots covered by the mask: 256
constexpr int kMaskSlots = 32 * kMaskWords;
constexpr int kStateHigh = 0x7fffffff;          // past the box along an axis
constexpr uint32_t kNoRoom = 0xffffffffu;       // a ray whose records found no room

// One axis of a ray and of the grid, as the index test sees it.
struct AxisP {
  float o, d, inv_d;       // ray origin and direction along the axis, 1/d (0 when d = 0)
  float amin, inv_h, top;  // box minimum, vertices per unit length, n - 1
  float occ_scale;         // occupancy cells per vertex step
};

__device__ __forceinline__ AxisP axis_p(const GridGeo& g, const float o[3], const float d[3], const float inv_d[3],
                                        int a) {
  auto pick = [a](float x0, float x1, float x2) { return a == 0 ? x0 : (a == 1 ? x1 : x2); };
  AxisP A;
  A.o = pick(o[0], o[1], o[2]);
  A.d = pick(d[0], d[1], d[2]);
  A.inv_d = pick(inv_d[0], inv_d[1], inv_d[2]);
  A.amin = pick(g.amin[0], g.amin[1], g.amin[2]);
  A.inv_h = pick(g.inv_h[0], g.inv_h[1], g.inv_h[2]);
  A.top = pick((float)(g.n[0] - 1), (float)(g.n[1] - 1), (float)(g.n[2] - 1));
  A.occ_scale = pick(g.occ_scale[0], g.occ_scale[1], g.occ_scale[2]);
  return A;
}

// State of slot k along an axis: -1 before the box, kStateHigh past it, otherwise the occupancy
// cell (0 when the grid has no mask, R = 0).  The operations are those of index_sample, in the
// same order.
__device__ __forceinline__ int axis_state(const AxisP& A, int R, const Slots& sl, int k) {
  const float t = slot_t(sl, k);
  const float p = __fadd_rn(A.o, __fmul_rn(t, A.d));
  const float ga = __fmul_rn(__fsub_rn(p, A.amin), A.inv_h);
  if (!(ga >= 0.0f)) return -1;
  if (!(ga <= A.top)) return kStateHigh;
  if (!R) return 0;
  const int c = (int)floorf(__fmul_rn(ga, A.occ_scale));
  return c > R - 1 ? R - 1 : c;
}

// Smallest k in (lo, hi] with P(k), for a predicate that is false up to some slot and true after
// it, given P(lo) false and P(hi) true (neither is evaluated).  `est` is a guess: the search walks
// from it in doubling steps and bisects, so a guess off by one costs two or three evaluations.
template <typename Pred>
__device__ __forceinline__ int first_true(int lo, int hi, float est, Pred P) {
  int e = !(est > (float)lo) ? lo + 1 : (!(est < (float)hi) ? hi : (int)est);
  if (e == hi || P(e)) {
    hi = e;
    for (int step = 1;; step <<= 1) {
      const int m = hi - step;
      if (m <= lo) break;
      if (P(m)) {
        hi = m;
      } else {
        lo = m;
        break;
      }
    }
  } else {
    lo = e;
    for (int step = 1;; step <<= 1) {
      const int m = lo + step;
      if (m >= hi) break;
      if (P(m)) {
        hi = m;
        break;
      }
      lo = m;
    }
  }
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (P(m)) hi = m;
    else lo = m;
  }
  return hi;
}

// First slot after k whose state along the axis differs from s = axis_state(k); kend if none before it.
__device__ __forceinline__ int next_change(const AxisP& A, int R, const Slots& sl, float inv_dt, int k, int s,
                                           int kend) {
  if (A.d == 0.0f) return kend;  // the coordinate does not change along the ray
  const int Rc = R ? R : 1;
  float B;  // the vertex coordinate where the state changes
  if (A.d > 0.0f) {
    if (s == kStateHigh) return kend;
    B = s < 0 ? 0.0f : (s < Rc - 1 ? __fdividef((float)(s + 1), A.occ_scale) : A.top);
  } else {
    if (s < 0) return kend;
    B = s == kStateHigh ? A.top : (s > 0 ? __fdividef((float)s, A.occ_scale) : 0.0f);
  }
  const float tb = (A.amin + __fdividef(B, A.inv_h) - A.o) * A.inv_d;
  const float est = ceilf((tb - sl.t0) * inv_dt - 0.5f);
  return first_true(k, kend, est, [&](int kk) { return axis_state(A, R, sl, kk) != s; });
}

__device__ __forceinline__ void set_bits(uint32_t* mask, int k, int e) {
  for (int w = k >> 5; w <= (e - 1) >> 5; w++) {
    const int lo = max(k - 32 * w, 0), hi = min(e - 32 * w, 32);
    const uint32_t upto = hi == 32 ? 0xffffffffu : ((1u << hi) - 1u);
    mask[w] |= upto & ~((1u << lo) - 1u);
  }
}

// Mask of the active slots among the first kend (<= kMaskSlots) slots of a ray; returns their
// count.  Each pass takes the segment of slots up to the next state change on any axis, then moves
// the one axis that changes there (ties take one pass each, the later ones with empty segments), so
// every lane of a warp runs the same instructions whichever axis its ray crosses.
__device__ __forceinline__ int active_mask(const GridGeo& g, const Slots& sl, const float o[3], const float d[3],
                                           int kend, uint32_t* mask) {
#pragma unroll
  for (int w = 0; w < kMaskWords; w++) mask[w] = 0u;
  if (kend <= 0) return 0;
  const int R = g.occ ? g.occ_res : 0;
  const float inv_dt = __fdividef(1.0f, sl.dt);
  float inv_d[3];
#pragma unroll
  for (int a = 0; a < 3; a++) inv_d[a] = d[a] != 0.0f ? __fdividef(1.0f, d[a]) : 0.0f;
  int st[3], nx[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const AxisP A = axis_p(g, o, d, inv_d, a);
    st[a] = axis_state(A, R, sl, 0);
    nx[a] = next_change(A, R, sl, inv_dt, 0, st[a], kend);
  }
  int k = 0, count = 0;
  for (;;) {  // every pass moves k forward or settles one of the axes that change at k
    const int e = min(nx[0], min(nx[1], nx[2]));
    bool on = e > k;
#pragma unroll
    for (int a = 0; a < 3; a++) on = on && st[a] >= 0 && st[a] != kStateHigh;
    if (on && R) on = __ldg(&g.occ[((size_t)st[2] * R + st[1]) * R + st[0]]) != 0;
    if (on) {
      set_bits(mask, k, e);
      count += e - k;
    }
    if (e >= kend) break;
    k = e;
    const int a = nx[0] == e ? 0 : (nx[1] == e ? 1 : 2);
    const AxisP A = axis_p(g, o, d, inv_d, a);
    const int sa = axis_state(A, R, sl, e);
    const int na = next_change(A, R, sl, inv_dt, e, sa, kend);
    st[0] = a == 0 ? sa : st[0];
    st[1] = a == 1 ? sa : st[1];
    st[2] = a == 2 ? sa : st[2];
    nx[0] = a == 0 ? na : nx[0];
    nx[1] = a == 1 ? na : nx[1];
    nx[2] = a == 2 ? na : nx[2];
  }
  return count;
}

// Per-ray setup, prepared by one lane for the warp that marches the ray.
struct RaySetup {
  float o[3], d[3];
  float t0, dt;
  int nv;        // valid slots: before the box exit (box-march mode) and within the slot budget
  int nact;      // slots that reach Feature Gathering at most: the mask's count plus every valid slot past it
  uint32_t base; // first record reserved for the ray (nact of them), or kNoRoom
  int view, pix;
  uint32_t mask[kMaskWords];  // bit k: slot k is inside the box and in an occupied cell
};
static_assert(sizeof(RaySetup) == kRaySetupBytes, "RaySetup layout");
constexpr int kSetupWords = (int)(sizeof(RaySetup) / 4);

__device__ __forceinline__ void prepare_ray(const GridGeo& g, const Samp& s, const float o[3], const float d[3],
                                            RaySetup& q) {
  const Slots sl = place_slots(g, s, o, d);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    q.o[a] = o[a];
    q.d[a] = d[a];
  }
  q.t0 = sl.t0;
  q.dt = sl.dt;
  int nv = sl.n;
  if (sl.march && nv > 0) {  // slots run while t_k < t_out: the first slot past the exit, exactly
    const float est = ceilf(__fdividef(sl.tout - sl.t0, sl.dt) - 0.5f);
    nv = first_true(-1, nv, est, [&](int k) { return !(slot_t(sl, k) < sl.tout); });
  }
  q.nv = nv;
  const int kend = min(nv, kMaskSlots);
  q.nact = active_mask(g, sl, o, d, kend, q.mask) + (nv - kend);
}

// Reserves the records of the warp's (up to) 32 prepared rays with one atomic: lane j's ray gets
// nact records from its base, or kNoRoom (and an error) when they pass the capacity.
__device__ __forceinline__ void reserve_records(const RenderWs& w, RaySetup* q, bool have) {
  const int lane = threadIdx.x & 31;
  const uint32_t n = have ? (uint32_t)q[lane].nact : 0u;
  uint32_t incl = n;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  uint32_t base = 0;
  if (lane == 31 && incl) base = atomicAdd(&w.hdr[3], incl);
  base = __shfl_sync(0xffffffffu, base, 31) + (incl - n);
  if (have) {
    const bool room = (unsigned long long)base + n <= (unsigned long long)w.Q;
    if (!room) set_err(&w.hdr[0], kErrCapacity);
    q[lane].base = room ? base : kNoRoom;
  }
}

// 1 - e^{-x} for x >= 0 without cancellation: the Taylor series x (1 - x/2 (1 - x/3 (1 - x/4 (1 - x/5))))
// below 1/32 (truncation < x^6/720, ~1e-12 relative), the hardware exponential above it (absolute
// error ~1e-7, relative < 4e-6 there).
__device__ __forceinline__ float one_minus_exp_neg(float x) {
  const float series = x * (1.0f - 0.5f * x * (1.0f - (1.0f / 3.0f) * x * (1.0f - 0.25f * x * (1.0f - 0.2f * x))));
  return x < 0.03125f ? series : 1.0f - __expf(-x);
}

// Voxel and fraction of a sample that index_sample accepted (the same operations, without the tests).
__device__ __forceinline__ void index_voxel(const GridGeo& g, const float p[3], int i0[3], float f[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const float ga = __fmul_rn(__fsub_rn(p[a], g.amin[a]), g.inv_h[a]);
    int i = (int)floorf(ga);
    if (i > g.n[a] - 2) i = g.n[a] - 2;
    if (i < 0) i = 0;  // never taken for an accepted sample (g >= 0); keeps every load inside the grid
    i0[a] = i;
    f[a] = __fsub_rn(ga, (float)i);
  }
}

// K1 per ray (one warp), from the ray's prepared setup q.  The ray's active slots inside the mask
// are listed in slot order (list: the warp's kMaskSlots bytes of shared memory) and composited 32
// at a time, lane j taking the j-th active slot of the chunk; slots past the mask (rays of more
// than kMaskSlots slots) follow in chunks of 32 consecutive slots, each tested with index_sample.
// Inactive slots add nothing to the transmittance, so the early stop falls on the slot after the
// last active slot processed before the transmittance dropped below t_stop, as in a plain
// slot-by-slot march.  Records carry the RIT key of their brick, offset by key_base (the job's first
// brick in a batch), and octant; dep/acc/steps point at the ray's outputs (or are NULL).
// A record is the sample's RIT key, weight and slot (the scatter recomputes its position from the
// ray's geometry).  EXTRA: the records also carry their ray, transmittance and raw density (the
// backward and the Ray Index Table export); a compile-time flag, so that the forward march tests
// nothing for them.
template <typename T, bool EXTRA>
__device__ __forceinline__ void march_ray_core(const GridGeo& g, const Samp& s, const T* __restrict__ dens,
                                               const RenderWs& w, int r, const RaySetup& q, uint32_t key_base,
                                               float* dep, float* acc_out, int32_t* steps_out, uint8_t* list,
                                               int tag = 0) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const unsigned lt_mask = (1u << lane) - 1u;
  const unsigned le_mask = (2u << lane) - 1u;  // lanes <= this one (all ones for lane 31)
  const float o[3] = {q.o[0], q.o[1], q.o[2]}, d[3] = {q.d[0], q.d[1], q.d[2]};
  Slots sl;
  sl.t0 = q.t0;
  sl.dt = q.dt;
  sl.n = q.nv;
  sl.tout = 0.0f;
  sl.march = false;
  const int nv = q.nv;
  const bool room = q.base != kNoRoom;
  const uint32_t base = room ? q.base : 0u;
  float Ssum = 0.0f, acc_l = 0.0f, dsum_l = 0.0f;
  uint32_t cnt = 0;
  // One chunk of up to 32 samples, lane by lane in slot order: density, the scan of sigma delta,
  // the stop test (lanes with `elig`), weights, records and the brick histogram.  Returns the first
  // lane whose transmittance is below t_stop (32: none); Ssum then holds the sum up to that lane.
  auto chunk = [&](bool act, bool elig, int k, float t, const float p[3], const int i0[3], const float f[3]) -> int {
    float sd = 0.0f, raw = 0.0f;
    if (act) {
      raw = density_trilinear(g, dens, i0, f);
      sd = softplus_fast(raw + g.act_shift) * sl.dt;
    }
    float incl = sd;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float v = __shfl_up_sync(full, incl, off);
      if (lane >= off) incl += v;
    }
    float excl = __shfl_up_sync(full, incl, 1);
    if (lane == 0) excl = 0.0f;
    const float Tk = __expf(-(Ssum + excl));
    const bool stop = elig && s.t_stop > 0.0f && Tk < s.t_stop;
    const unsigned smask = __ballot_sync(full, stop);
    const int first = smask ? __ffs(smask) - 1 : 32;
    const bool contrib = act && lane < first && room;
    const float wk = (act && lane < first) ? Tk * one_minus_exp_neg(sd) : 0.0f;
    const unsigned cmask = __ballot_sync(full, contrib);
    const uint32_t key = contrib ? brick_key(g, i0, key_base) : 0xffffffffu;
    if (contrib) {
      const size_t qi = (size_t)base + cnt + __popc(cmask & lt_mask);
      w.rec_key[qi] = key;
      w.rec_w[qi] = wk;
      w.rec_slot[qi] = (uint16_t)k;
      if constexpr (EXTRA) {
        if (w.rec_ray) w.rec_ray[qi] = (uint32_t)r;
        if (w.rec_T) {
          w.rec_T[qi] = Tk;
          w.rec_raw[qi] = raw;
        }
      }
    }
    // brick histogram: one atomic per run of consecutive lanes with the same key
    const uint32_t prev = __shfl_up_sync(full, key, 1);
    const bool head = contrib && (lane == 0 || prev != key);
    const unsigned heads = __ballot_sync(full, head);
    if (head) {
      const unsigned after = heads & ~le_mask;
      const int end = after ? __ffs(after) - 1 : 32;
      const unsigned run = cmask & ~lt_mask & (end == 32 ? full : ((1u << end) - 1u));
      atomicAdd(&w.brick_cnt[key], (uint32_t)__popc(run));
    }
    acc_l += wk;
    dsum_l += wk * t;
    cnt += __popc(cmask);
    const int last = first == 32 ? 31 : first - 1;
    const float tot = __shfl_sync(full, incl, last < 0 ? 0 : last);
    if (first > 0) Ssum += tot;
    return first;
  };

  // the active slots of the mask, in slot order: lane j lists those of slots 8 j .. 8 j + 7
  int n_act;
  {
    uint32_t bits = (q.mask[lane >> 2] >> ((lane & 3) * 8)) & 0xffu;
    const int c = __popc(bits);
    int incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(full, incl, off);
      if (lane >= off) incl += v;
    }
    n_act = __shfl_sync(full, incl, 31);
    int pos = incl - c;
    while (bits) {
      list[pos++] = (uint8_t)(8 * lane + __ffs(bits) - 1);
      bits &= bits - 1u;
    }
    __syncwarp();
  }
  int steps = nv, last = -1;  // last: slot of the last active sample composited so far
  bool stopped = false;
  for (int j0 = 0; j0 < n_act; j0 += 32) {
    const int j = j0 + lane;
    const bool has = j < n_act;
    const int k = has ? (int)list[j] : 0;
    const float t = slot_t(sl, k);
    int i0[3] = {0, 0, 0};
    float f[3] = {0.0f, 0.0f, 0.0f}, p[3] = {0.0f, 0.0f, 0.0f};
    if (has) {
      sample_pos(o, d, t, p);
      index_voxel(g, p, i0, f);
    }
    const int first = chunk(has, has, k, t, p, i0, f);
    const int prev_k = __shfl_sync(full, k, first > 0 && first < 32 ? first - 1 : 0);
    if (first < 32) {  // the stop falls right after the previous active slot
      steps = (first > 0 ? prev_k : last) + 1;
      stopped = true;
      break;
    }
    last = __shfl_sync(full, k, min(n_act - j0, 32) - 1);
  }
  __syncwarp();  // the list is free for the warp's next ray
  if (!stopped && s.t_stop > 0.0f && __expf(-(Ssum + 0.0f)) < s.t_stop) {
    // the transmittance fell below the threshold at the last active slot: the next slot stops
    steps = last + 1;
    stopped = true;
  }
  if (!stopped) {
    for (int k0 = kMaskSlots; k0 < nv; k0 += 32) {  // slots past the mask, tested one by one
      const int k = k0 + lane;
      const bool valid = k < nv;
      const float t = slot_t(sl, k);
      int i0[3] = {0, 0, 0};
      float f[3] = {0.0f, 0.0f, 0.0f}, p[3] = {0.0f, 0.0f, 0.0f};
      bool act = false;
      if (valid) {
        sample_pos(o, d, t, p);
        act = index_sample(g, p, i0, f);
      }
      if (!__any_sync(full, act)) {  // nothing to composite in these slots: only the stop test
        if (s.t_stop > 0.0f && __expf(-(Ssum + 0.0f)) < s.t_stop) {
          steps = k0;
          break;
        }
        continue;
      }
      const int first = chunk(act, valid, k, t, p, i0, f);
      if (first < 32) {
        steps = k0 + first;
        break;
      }
    }
  }
  const float acc = warp_sum(acc_l), dsum = warp_sum(dsum_l);
  if (lane == 0) {
    w.ray_n[r] = cnt;
    w.ray_start[r] = base;
    w.ray_T[r] = __expf(-Ssum);
    w.ray_dir[r] = make_float4(d[0], d[1], d[2], __int_as_float(tag));  // tag: the ray's job in a batch
    if (dep) *dep = acc >= s.void_acc ? dsum / acc : __int_as_float(0x7f800000);
    if (acc_out) *acc_out = acc;
    if (steps_out) *steps_out = steps;
  }
}

// The job whose first ray (or first brick) is the largest one <= x, from the contiguous array of
// the jobs' first rays (or bricks).
__device__ __forceinline__ int job_of(const int* __restrict__ base, int n_jobs, int x) {
  int lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&base[mid]) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// K0: the setup of every ray, one thread per ray (ray generation, slot placement, the exact mask
// of active slots), with the records reserved by one atomic per 32 rays.  A separate kernel keeps
// all 32 lanes of a warp busy on the mask walk however many rays a launch has, while the march
// keeps one warp per ray.  With BATCH, ray r belongs to the job found among the jobs' first rays.
template <bool BATCH>
__global__ void __launch_bounds__(256) k_ray_setup(GridGeo g, Samp s, RaySrc src, const JobDesc* __restrict__ jobs,
                                                   const int* __restrict__ bases, int n_jobs, int R_batch, RenderWs w) {
  __shared__ RaySetup sq[256];
  const int R = BATCH ? R_batch : ray_count(src);
  for (long long r0 = (long long)blockIdx.x * 256; r0 < R; r0 += (long long)gridDim.x * 256) {
    const long long r = r0 + threadIdx.x;
    const bool have = r < R;
    if (have) {
      RaySetup& q = sq[threadIdx.x];
      float o[3], d[3];
      if constexpr (BATCH) {
        const int j = job_of(bases, n_jobs, (int)r);
        const JobDesc& J = jobs[j];
        const int pix = (int)r - J.ray_base;
        ray_gen_cam(J.cam, pix, o, d);
        prepare_ray(J.geo, J.samp, o, d, q);
        q.view = j;
        q.pix = pix;
      } else {
        const RayRef rr = ray_ref(src, (int)r);
        ray_gen(src, rr, o, d);
        prepare_ray(g, s, o, d, q);
        q.view = rr.view;
        q.pix = rr.pix;
      }
    }
    reserve_records(w, sq + (threadIdx.x & ~31), have);
    if (have) {
      const RaySetup& q = sq[threadIdx.x];
      RayGeo rg;
      rg.ot = make_float4(q.o[0], q.o[1], q.o[2], q.t0);
      rg.dd = make_float4(q.d[0], q.d[1], q.d[2], q.dt);
      w.ray_geo[r] = rg;
    }
    __syncthreads();
    const int n = (int)min((long long)256, (long long)R - r0);
    const uint32_t* from = reinterpret_cast<const uint32_t*>(sq);
    uint32_t* to = reinterpret_cast<uint32_t*>(w.setup + r0);
    for (int i = threadIdx.x; i < n * kSetupWords; i += 256) to[i] = from[i];
    __syncthreads();
  }
}

// The warp's copy of ray r's setup: lane i < kSetupWords holds word i (loaded ahead of time).
__device__ __forceinline__ uint32_t setup_word(const RenderWs& w, long long r, int lane) {
  return lane < kSetupWords ? __ldg(reinterpret_cast<const uint32_t*>(w.setup + r) + lane) : 0u;
}

// K1: one warp per ray, rays r = warp + i nwarps; each ray's setup (from K0) is staged in shared
// memory, the next ray's loaded while the current one marches.
template <typename T, bool EXTRA>
__global__ void __launch_bounds__(256, 4) k_march(GridGeo g, Samp s, RaySrc src, const T* __restrict__ dens,
                                               RenderWs w, OutBufs out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int R = ray_count(src);
  __shared__ RaySetup setup[8];
  __shared__ uint8_t slot_list[8][kMaskSlots];
  const int wb = threadIdx.x >> 5;
  uint32_t next = warp < R ? setup_word(w, warp, lane) : 0u;
  for (long long r = warp; r < R; r += nwarps) {
    if (lane < kSetupWords) reinterpret_cast<uint32_t*>(&setup[wb])[lane] = next;
    __syncwarp();
    if (r + nwarps < R) next = setup_word(w, r + nwarps, lane);
    const RaySetup& q = setup[wb];
    float* dep = out.depth[q.view];
    march_ray_core<T, EXTRA>(g, s, dens, w, (int)r, q, 0u, dep ? dep + q.pix : nullptr,
                             out.acc ? out.acc + q.pix : nullptr, out.n_steps ? out.n_steps + q.pix : nullptr,
                             slot_list[wb]);
    __syncwarp();  // the setup slot is free for the next ray
  }
}

// K2: exclusive scan of the brick histogram and the list of tiles (<= kTile samples of one brick).
__device__ __forceinline__ void block_exscan2(uint32_t a, uint32_t b, uint32_t* ea, uint32_t* eb, uint32_t* ta,
                                              uint32_t* tb, uint32_t* sh /* 64 words */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t va = __shfl_up_sync(0xffffffffu, ia, o), vb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += va;
      ib += vb;
    }
  }
  if (lane == 31) {
    sh[wid] = ia;
    sh[32 + wid] = ib;
  }
  __syncthreads();
  if (wid == 0) {
    uint32_t xa = lane < nw ? sh[lane] : 0, xb = lane < nw ? sh[32 + lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t va = __shfl_up_sync(0xffffffffu, xa, o), vb = __shfl_up_sync(0xffffffffu, xb, o);
      if (lane >= o) {
        xa += va;
        xb += vb;
      }
    }
    sh[lane] = xa;
    sh[32 + lane] = xb;
  }
  __syncthreads();
  const uint32_t pa = wid ? sh[wid - 1] : 0, pb = wid ? sh[32 + wid - 1] : 0;
  *ea = pa + ia - a;
  *eb = pb + ib - b;
  *ta = sh[nw - 1];
  *tb = sh[32 + nw - 1];
  __syncthreads();
}

// The kOctants counters of brick b (zeros past the last brick).
__device__ __forceinline__ uint32_t brick_counts(const RenderWs& w, int b, uint32_t v[kOctants]) {
  static_assert(kOctants == 8, "two 16-byte loads per brick");
  uint4 a = make_uint4(0u, 0u, 0u, 0u), c = a;
  if (b < w.nb) {
    const uint4* p = reinterpret_cast<const uint4*>(w.brick_cnt + (size_t)b * kOctants);
    a = p[0];
    c = p[1];
  }
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = c.x, v[5] = c.y, v[6] = c.z, v[7] = c.w;
  return a.x + a.y + a.z + a.w + c.x + c.y + c.z + c.w;
}

// K2a: per block of kScanChunk bricks (one per thread), the sums of sample counts and tile counts.
__global__ void __launch_bounds__(1024) k_brick_sums(RenderWs w) {
  __shared__ uint32_t sh[64];
  uint32_t v[kOctants];
  const uint32_t c = brick_counts(w, blockIdx.x * kScanChunk + threadIdx.x, v);
  const uint32_t t = (c + kTile - 1) / kTile;
  uint32_t ec, et, tc, tt;
  block_exscan2(c, t, &ec, &et, &tc, &tt, sh);
  if (threadIdx.x == 0) {
    w.blk_sums[2 * blockIdx.x] = tc;
    w.blk_sums[2 * blockIdx.x + 1] = tt;
  }
}

// K2b: exclusive scan of the block sums (one block); totals into the header.
__global__ void __launch_bounds__(1024) k_brick_blocks(RenderWs w, int nblk) {
  __shared__ uint32_t sh[64];
  uint32_t run_c = 0, run_t = 0;
  for (int b0 = 0; b0 < nblk; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const uint32_t c = i < nblk ? w.blk_sums[2 * i] : 0, t = i < nblk ? w.blk_sums[2 * i + 1] : 0;
    uint32_t ec, et, tc, tt;
    block_exscan2(c, t, &ec, &et, &tc, &tt, sh);
    if (i < nblk) {
      w.blk_sums[2 * i] = run_c + ec;
      w.blk_sums[2 * i + 1] = run_t + et;
    }
    run_c += tc;
    run_t += tt;
  }
  if (threadIdx.x == 0) {
    w.brick_off[(size_t)w.nb * kOctants] = run_c;
    w.tile_off[w.nb] = run_t;
    if (run_t > (uint32_t)w.max_tiles) {
      set_err(&w.hdr[0], kErrInternal);
      run_t = w.max_tiles;
    }
    w.hdr[1] = run_t;
    w.hdr[2] = run_c;
  }
}

// K2c: the offset of every (brick, octant) key and of every brick's first tile; the scatter's
// cursors start at the keys' offsets.
__global__ void __launch_bounds__(1024) k_brick_offsets(RenderWs w) {
  __shared__ uint32_t sh[64];
  const int b = blockIdx.x * kScanChunk + threadIdx.x;
  uint32_t v[kOctants];
  const uint32_t c = brick_counts(w, b, v);
  const uint32_t t = (c + kTile - 1) / kTile;
  uint32_t ec, et, tc, tt;
  block_exscan2(c, t, &ec, &et, &tc, &tt, sh);
  if (b < w.nb) {
    uint32_t o[kOctants], run = w.blk_sums[2 * blockIdx.x] + ec;
#pragma unroll
    for (int k = 0; k < kOctants; k++) {
      o[k] = run;
      run += v[k];
    }
    uint4* off = reinterpret_cast<uint4*>(w.brick_off + (size_t)b * kOctants);
    off[0] = make_uint4(o[0], o[1], o[2], o[3]);
    off[1] = make_uint4(o[4], o[5], o[6], o[7]);
    uint4* cur = reinterpret_cast<uint4*>(w.brick_cur + (size_t)b * kOctants);  // cursors start at the offsets
    cur[0] = make_uint4(o[0], o[1], o[2], o[3]);
    cur[1] = make_uint4(o[4], o[5], o[6], o[7]);
    w.tile_off[b] = w.blk_sums[2 * blockIdx.x + 1] + et;
  }
}

// K2d: the tile list, one entry per tile: its brick (binary search over tile offsets) and start.
__global__ void __launch_bounds__(256) k_tiles(GridGeo g, RenderWs w) {
  const uint32_t n = w.hdr[1];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int lo = 0, hi = w.nb;  // largest b with tile_off[b] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w.tile_off[mid] <= t) lo = mid;
      else hi = mid;
    }
    const uint32_t start = w.brick_off[(size_t)lo * kOctants] + (t - w.tile_off[lo]) * kTile;
    const uint32_t cnt = min(start + (uint32_t)kTile, w.brick_off[(size_t)(lo + 1) * kOctants]) - start;
    const uint32_t bx = lo % g.nb[0], by = (lo / g.nb[0]) % g.nb[1], bz = lo / (g.nb[0] * g.nb[1]);
    w.tile[t] = make_uint4(start, cnt | (bz << 8), (uint32_t)lo, bx | (by << 16));
  }
}

// K3: counting sort of the records by (brick, octant) key; the payload moves into brick order so
// that the gather kernels stream it, octant by octant inside a brick (order inside an octant is
// unspecified).  A warp takes one ray at a time in chunks of 32 records.  The cursors start at
// their keys' offsets, so the atomic of a run of equal keys returns the run's destination.  A
// chunk's records are written one step later, while the next chunk's atomics are in flight, and
// the next ray's header and first chunk are loaded ahead too.
__global__ void __launch_bounds__(256, 4) k_scatter(RaySrc src, RenderWs w) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int R = ray_count(src);
  const unsigned full = 0xffffffffu;
  const unsigned lt_mask = (1u << lane) - 1u;
  const unsigned le_mask = (2u << lane) - 1u;
  struct Chunk {
    uint32_t key, slot;
    float wk;
  };
  auto load_chunk = [&](uint32_t start, uint32_t n, uint32_t j0, Chunk& c) {
    const uint32_t j = j0 + lane;
    const bool valid = j < n;
    c.key = valid ? w.rec_key[start + j] : 0xffffffffu;
    c.slot = valid ? w.rec_slot[start + j] : 0u;
    c.wk = valid ? w.rec_w[start + j] : 0.0f;
  };
  // the chunk whose atomics were issued in the previous step: written once their results are
  // back (every lane takes the base of its run's head), one step later
  bool p_any = false, p_valid = false;
  uint32_t p_off = 0, p_q = 0;
  int p_hl = 0;
  float4 p_pw = make_float4(0.f, 0.f, 0.f, 0.f), p_dir = p_pw;
  auto flush = [&]() {
    if (!p_any) return;
    const uint32_t base = __shfl_sync(full, p_off, p_hl < 0 ? 0 : p_hl);
    if (p_valid) {
      const uint32_t dst = base + (uint32_t)(lane - p_hl);
      w.srt[dst].pw = p_pw;
      w.srt[dst].qd = make_float4(__uint_as_float(p_q), p_dir.x, p_dir.y, p_dir.z);
    }
    p_any = false;
  };
  // the warp's current ray (its header and geometry) and its first chunk
  int r = warp;
  uint32_t n = 0, start = 0;
  RayGeo geo;
  geo.ot = geo.dd = make_float4(0.f, 0.f, 0.f, 0.f);
  Chunk cur;
  if (r < R) {
    n = w.ray_n[r];
    start = w.ray_start[r];
    geo = w.ray_geo[r];
    load_chunk(start, n, 0, cur);
  }
  for (; r < R; r += nwarps) {
    // the next ray's header, geometry and first chunk
    const int rn = r + nwarps;
    uint32_t nn = 0, nstart = 0;
    RayGeo ngeo = geo;
    Chunk nxt;
    nxt.key = 0xffffffffu;
    nxt.slot = 0u;
    nxt.wk = 0.0f;
    if (rn < R) {
      nn = w.ray_n[rn];
      nstart = w.ray_start[rn];
      ngeo = w.ray_geo[rn];
    }
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
      Chunk c = cur;
      if (j0 + 32 < n) load_chunk(start, n, j0 + 32, cur);  // this ray's next chunk
      else if (rn < R) load_chunk(nstart, nn, 0, nxt);        // or the next ray's first
      const uint32_t j = j0 + lane;
      const bool valid = j < n;
      const uint32_t q = start + j;
      const unsigned vmask = __ballot_sync(full, valid);
      const uint32_t prev = __shfl_up_sync(full, c.key, 1);
      const bool head = valid && (lane == 0 || prev != c.key);
      const unsigned heads = __ballot_sync(full, head);
      uint32_t off = 0;
      if (head) {
        const unsigned after = heads & ~le_mask;
        const int end = after ? __ffs(after) - 1 : 32;
        const unsigned run = vmask & ~lt_mask & (end == 32 ? full : ((1u << end) - 1u));
        off = atomicAdd(&w.brick_cur[c.key], (uint32_t)__popc(run));
      }
      // the previous chunk is written while this chunk's atomics are in flight
      flush();
      // the sample's position, recomputed from its ray and slot as the march computed it
      float p[3], d[3];
      sample_of(geo.ot, geo.dd, c.slot, p, d);
      p_any = true;
      p_valid = valid;
      p_off = off;
      p_hl = 31 - __clz(heads & le_mask);  // this lane's run head
      p_q = q;
      p_pw = make_float4(p[0], p[1], p[2], c.wk);
      p_dir = make_float4(d[0], d[1], d[2], 0.0f);
    }
    if (n == 0 && rn < R) load_chunk(nstart, nn, 0, nxt);
    n = nn;
    start = nstart;
    geo = ngeo;
    cur = nxt;
  }
  flush();
}

// -------------------------------------------------------------------------------------------
// K5 (FP32): Feature Gathering from the staged brick and an FP32 SIMT MLP over 128-sample tiles.

template <typename T>
__device__ __forceinline__ void tri_smem(const T* tile, int vb, int vx, int C, const int l[3], const float f[3],
                                         float* out) {
  const float fx = f[0], fy = f[1], fz = f[2];
  float wc[8];
  wc[0] = (1.f - fx) * (1.f - fy) * (1.f - fz);
  wc[1] = fx * (1.f - fy) * (1.f - fz);
  wc[2] = (1.f - fx) * fy * (1.f - fz);
  wc[3] = fx * fy * (1.f - fz);
  wc[4] = (1.f - fx) * (1.f - fy) * fz;
  wc[5] = fx * (1.f - fy) * fz;
  wc[6] = (1.f - fx) * fy * fz;
  wc[7] = fx * fy * fz;
  for (int c = 0; c < C; c++) out[c] = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int x = l[0] + (q & 1), y = l[1] + ((q >> 1) & 1), z = l[2] + (q >> 2);
    const T* v = tile + ((size_t)(z * vb + y) * vx + x) * C;
    if constexpr (sizeof(T) == 4) {
      if (C == 12) {
        const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
        for (int u = 0; u < 3; u++) {
          float4 a = v4[u];
          out[4 * u + 0] += wc[q] * a.x;
          out[4 * u + 1] += wc[q] * a.y;
          out[4 * u + 2] += wc[q] * a.z;
          out[4 * u + 3] += wc[q] * a.w;
        }
        continue;
      }
    } else {
      if (C == 12) {
        const uint2* v2 = reinterpret_cast<const uint2*>(v);
#pragma unroll
        for (int u = 0; u < 3; u++) {
          uint2 a = v2[u];
          float2 lo = __half22float2(*reinterpret_cast<__half2*>(&a.x));
          float2 hi = __half22float2(*reinterpret_cast<__half2*>(&a.y));
          out[4 * u + 0] += wc[q] * lo.x;
          out[4 * u + 1] += wc[q] * lo.y;
          out[4 * u + 2] += wc[q] * hi.x;
          out[4 * u + 3] += wc[q] * hi.y;
        }
        continue;
      }
    }
    for (int c = 0; c < C; c++) {
      float vv;
      if constexpr (sizeof(T) == 4) vv = v[c];
      else vv = __half2float(v[c]);
      out[c] += wc[q] * vv;
    }
  }
}

constexpr int kK1 = kMaxIn;  // padded input width of layer 1

struct F32Smem {
  // byte offsets inside dynamic shared memory
  static constexpr int w1t = 0;                                  // [48][128]
  static constexpr int w2t = w1t + kK1 * kHidden * 4;            // [128][128]
  static constexpr int w3 = w2t + kHidden * kHidden * 4;         // [3][128]
  static constexpr int b1 = w3 + 3 * kHidden * 4;                // [128]
  static constexpr int b2 = b1 + kHidden * 4;                    // [128]
  static constexpr int b3 = b2 + kHidden * 4;                    // [4]
  static constexpr int x = b3 + 16;                              // [48][128] inputs, buffer 0
  static constexpr int h = x + kK1 * kTile * 4;                  // [128][128]
  static constexpr int bar = ((h + kHidden * kTile * 4 + 127) / 128) * 128;  // mbarrier (8 B, pad 128)
  static constexpr int x2 = bar + 128;                           // [48][128] inputs, buffer 1
  // brick tile (TMA destination, 128-B aligned): after buffer 1, or in its place with one buffer
  static constexpr int tile = x2 + kK1 * kTile * 4;
  static constexpr int tile1 = x2;
  static_assert(tile % 128 == 0 && tile1 % 128 == 0, "TMA destination must be 128-byte aligned");
};

// acc[i][j]: rows {tm*4+i, 64+tm*4+(i-4)}, cols {tn*4+j, 64+tn*4+(j-4)}; A, B k-major [K][128].
// The operands of step k + 1 are loaded before the 64 FMAs of step k.
__device__ __forceinline__ void simt_gemm(const float* __restrict__ A, const float* __restrict__ Bw, int K, int tm,
                                          int tn, float acc[8][8]) {
  float4 a0 = *reinterpret_cast<const float4*>(&A[tm * 4]);
  float4 a1 = *reinterpret_cast<const float4*>(&A[64 + tm * 4]);
  float4 b0 = *reinterpret_cast<const float4*>(&Bw[tn * 4]);
  float4 b1 = *reinterpret_cast<const float4*>(&Bw[64 + tn * 4]);
#pragma unroll 2
  for (int k = 0; k < K; k++) {
    const int kn = k + 1 < K ? k + 1 : k;
    const float4 na0 = *reinterpret_cast<const float4*>(&A[kn * kTile + tm * 4]);
    const float4 na1 = *reinterpret_cast<const float4*>(&A[kn * kTile + 64 + tm * 4]);
    const float4 nb0 = *reinterpret_cast<const float4*>(&Bw[kn * kHidden + tn * 4]);
    const float4 nb1 = *reinterpret_cast<const float4*>(&Bw[kn * kHidden + 64 + tn * 4]);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
      for (int j = 0; j < 8; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    a0 = na0;
    a1 = na1;
    b0 = nb0;
    b1 = nb1;
  }
}

__device__ __forceinline__ int gemm_row(int tm, int i) { return i < 4 ? tm * 4 + i : 64 + tm * 4 + (i - 4); }

// bias + relu, then store transposed as the next layer's k-major input H[n][m]
__device__ __forceinline__ void simt_epilogue(float acc[8][8], const float* bias, float* H, int tm, int tn) {
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n = gemm_row(tn, j);
    const float bj = bias[n];
    float4 lo, hi;
    lo.x = fmaxf(acc[0][j] + bj, 0.f);
    lo.y = fmaxf(acc[1][j] + bj, 0.f);
    lo.z = fmaxf(acc[2][j] + bj, 0.f);
    lo.w = fmaxf(acc[3][j] + bj, 0.f);
    hi.x = fmaxf(acc[4][j] + bj, 0.f);
    hi.y = fmaxf(acc[5][j] + bj, 0.f);
    hi.z = fmaxf(acc[6][j] + bj, 0.f);
    hi.w = fmaxf(acc[7][j] + bj, 0.f);
    *reinterpret_cast<float4*>(&H[n * kTile + tm * 4]) = lo;
    *reinterpret_cast<float4*>(&H[n * kTile + 64 + tm * 4]) = hi;
  }
}

__device__ void load_mlp_f32_smem(char* sm, const MlpPtrs& m) {
  float* w1t = (float*)(sm + F32Smem::w1t);
  float* w2t = (float*)(sm + F32Smem::w2t);
  float* w3 = (float*)(sm + F32Smem::w3);
  float* b1 = (float*)(sm + F32Smem::b1);
  float* b2 = (float*)(sm + F32Smem::b2);
  float* b3 = (float*)(sm + F32Smem::b3);
  for (int i = threadIdx.x; i < kK1 * kHidden; i += blockDim.x) {
    const int k = i / kHidden, n = i % kHidden;
    w1t[i] = k < m.in_dim ? m.w1[n * m.in_dim + k] : 0.0f;
  }
  for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) {
    const int k = i / kHidden, n = i % kHidden;
    w2t[i] = m.w2[n * kHidden + k];
  }
  for (int i = threadIdx.x; i < 3 * kHidden; i += blockDim.x) w3[i] = m.w3[i];
  for (int i = threadIdx.x; i < kHidden; i += blockDim.x) {
    b1[i] = m.b1[i];
    b2[i] = m.b2[i];
  }
  if (threadIdx.x < 4) b3[threadIdx.x] = threadIdx.x < 3 ? m.b3[threadIdx.x] : 0.0f;
}

// Named barriers of the FP32 kernels: the 256 MLP threads among themselves, and the hand-off of
// the two input buffers between the producer warps and the MLP threads (full: the producers
// arrive, the MLP threads wait; empty: the reverse).
constexpr int kBarMlp = 1, kBarProd = 2, kBarFull0 = 3, kBarEmpty0 = 5;
constexpr int kMlpThreads = 256, kProdThreads = 128;
__device__ __forceinline__ void nbar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ bool nbar_sync_and(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void nbar_arrive(int id, int n) {
  __threadfence_block();  // this thread's shared-memory accesses before the arrival
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Three-layer MLP of the 128 samples whose inputs are in X [48][128] (rows in_dim.. zero);
// threads < 128 return c of sample m = threadIdx.x.  Run by the 256 MLP threads (threadIdx.x < 256), which synchronise on
// their own named barrier; with empty_id > 0 they also arrive on that barrier (with the producers,
// kMlpThreads + kProdThreads) once layer 1 has read X.
// This thread's ReLU bits of one layer into msk [16][128] bytes: byte (tn, m) holds units
// tn * 4 + j (bit j) and 64 + tn * 4 + j (bit 4 + j) of sample m, as relu(acc + bias) > 0 decides.
__device__ __forceinline__ void store_relu_bits(const float acc[8][8], const float* bias, uint8_t* msk, int tm,
                                                int tn) {
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint32_t byte = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) byte |= (acc[i][j] + bias[gemm_row(tn, j)] > 0.f ? 1u : 0u) << j;
    msk[tn * kTile + gemm_row(tm, i)] = (uint8_t)byte;
  }
}

// msk (may be NULL): [2][16][128] bytes receiving the ReLU masks of layers 1 and 2 (store_relu_bits).
__device__ __forceinline__ void mlp_f32_tile(char* sm, const float* X, float c[3], int in_dim, int empty_id = 0,
                                             uint8_t* msk = nullptr) {
  const float* w1t = (const float*)(sm + F32Smem::w1t);
  const float* w2t = (const float*)(sm + F32Smem::w2t);
  const float* w3 = (const float*)(sm + F32Smem::w3);
  const float* b1 = (const float*)(sm + F32Smem::b1);
  const float* b2 = (const float*)(sm + F32Smem::b2);
  const float* b3 = (const float*)(sm + F32Smem::b3);
  float* H = (float*)(sm + F32Smem::h);
  const int tm = threadIdx.x & 15, tn = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
  simt_gemm(X, w1t, (in_dim + 3) & ~3, tm, tn, acc);  // rows in_dim.. of X and W1^T are zero
  if (msk) store_relu_bits(acc, b1, msk, tm, tn);
  simt_epilogue(acc, b1, H, tm, tn);
  nbar_sync(kBarMlp, kMlpThreads);
  if (empty_id) nbar_arrive(empty_id, kMlpThreads + kProdThreads);  // X may be refilled
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
  simt_gemm(H, w2t, kHidden, tm, tn, acc);
  if (msk) store_relu_bits(acc, b2, msk + 16 * kTile, tm, tn);
  // layer-2 epilogue fused with layer 3: h2 = relu(acc + b2) stays in registers; this thread's 8
  // hidden units give partial sums z[i][o] = sum_j w3[o][n_j] h2[i][j] for its 8 samples, and the
  // 16 threads that share the samples add theirs through shared memory (P [16][3][128], over H)
  float z[8][3];
#pragma unroll
  for (int i = 0; i < 8; i++) z[i][0] = z[i][1] = z[i][2] = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int n = gemm_row(tn, j);
    const float bj = b2[n], u0 = w3[n], u1 = w3[kHidden + n], u2 = w3[2 * kHidden + n];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const float h = fmaxf(acc[i][j] + bj, 0.f);
      z[i][0] = fmaf(u0, h, z[i][0]);
      z[i][1] = fmaf(u1, h, z[i][1]);
      z[i][2] = fmaf(u2, h, z[i][2]);
    }
  }
  nbar_sync(kBarMlp, kMlpThreads);  // every thread is done reading H (h1)
  float* P = H;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int m = gemm_row(tm, i);
#pragma unroll
    for (int o = 0; o < 3; o++) P[(tn * 3 + o) * kTile + m] = z[i][o];
  }
  nbar_sync(kBarMlp, kMlpThreads);
  if (threadIdx.x < kTile) {
    const int m = threadIdx.x;
    float z0 = b3[0], z1 = b3[1], z2 = b3[2];
#pragma unroll
    for (int t = 0; t < 16; t++) {
      z0 += P[(t * 3 + 0) * kTile + m];
      z1 += P[(t * 3 + 1) * kTile + m];
      z2 += P[(t * 3 + 2) * kTile + m];
    }
    c[0] = sigmoid_f(z0);
    c[1] = sigmoid_f(z1);
    c[2] = sigmoid_f(z2);
  }
}

// K5f: FP32 Feature Gathering + Computation.  Warps 0-7 run the MLP of tile t while warps 8-11
// (producers, one thread per sample row) gather tile t + 1 into the other input buffer: staged
// brick (TMA, reloaded when the brick changes) -> trilinear features + direction encoding.  With
// nbuf = 1 (a brick too large for two buffers) the producers wait until layer 1 of tile t has read
// the single buffer.  The buffers are handed over with named barriers (full / empty, alternating
// between two ids per tile so that consecutive generations never mix); a producer that runs into
// a timeout keeps taking part in them (with zero inputs), so the MLP threads never wait on a
// barrier that cannot complete.
template <typename T>
__global__ void __launch_bounds__(kMlpThreads + kProdThreads, 1)
    k_gather_mlp_f32(GridGeo g, int S, MlpPtrs mlp, RenderWs w, const __grid_constant__ CUtensorMap fmap, int vb,
                     int vx, int box_bytes, int nbuf) {
  extern __shared__ __align__(128) char sm[];
  uint64_t* bar = (uint64_t*)(sm + F32Smem::bar);
  T* tile = (T*)(sm + (nbuf == 2 ? F32Smem::tile : F32Smem::tile1));
  // the ReLU masks of two tiles, after the brick tile (present only when the launch records masks)
  uint8_t* mask_smem = (uint8_t*)tile + ((box_bytes + 127) & ~127);
  load_mlp_f32_smem(sm, mlp);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t n_tiles = w.hdr[1];
  const uint32_t per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * per, t_end = min(n_tiles, t_begin + per);
  const uint32_t n = t_end > t_begin ? t_end - t_begin : 0;
  if (threadIdx.x >= kMlpThreads) {
    // ------------------------------------------------------------------ producers
    const int m = threadIdx.x - kMlpThreads;
    const int B = g.brick, C = g.C;
    int loaded = -1;
    uint32_t phase = 0;
    bool alive = true;
    for (uint32_t i = 0; i < n; i++) {
      const int b = i & 1;
      float* X = (float*)(sm + ((i % nbuf) ? F32Smem::x2 : F32Smem::x));
      // layer 1 of tile i - nbuf, the buffer's last user, is done with it
      if (i >= (uint32_t)nbuf) nbar_sync(kBarEmpty0 + ((i - nbuf) & 1), kMlpThreads + kProdThreads);
      const uint4 td = w.tile[t_begin + i];
      const uint32_t start = td.x;
      const int mcnt = (int)(td.y & 0xFFu);
      const int bx = (int)(td.w & 0xFFFFu), by = (int)(td.w >> 16), bz = (int)((td.y >> 8) & 0x1FFFu);
      if (alive && (int)td.z != loaded) {
        nbar_sync(kBarProd, kProdThreads);  // every producer is done with the staged brick
        if (m == 0) {
          mbar_expect_tx(bar, (uint32_t)box_bytes);
          tma_load_3d(tile, &fmap, bx * B * C, by * B, bz * B, bar);
        }
        alive = nbar_sync_and(kBarProd, kProdThreads, mbar_wait(bar, phase, &w.hdr[0]));
        if (alive) phase ^= 1u;
        loaded = (int)td.z;
      }
      if (alive && m < mcnt) {
        const float4 pw = w.srt[start + m].pw;
        const float4 dd = w.srt[start + m].qd;
        const float p[3] = {pw.x, pw.y, pw.z}, d[3] = {dd.y, dd.z, dd.w};
        float f[3], feat[24], e[3 + 6 * 7];
        int i0[3];
        const bool ok = index_sample(g, p, i0, f);
        const int l[3] = {i0[0] - bx * B, i0[1] - by * B, i0[2] - bz * B};
        if (!ok || l[0] < 0 || l[0] >= B || l[1] < 0 || l[1] >= B || l[2] < 0 || l[2] >= B) {
          set_err(&w.hdr[0], kErrInternal);
          for (int c = 0; c < C; c++) X[c * kTile + m] = 0.0f;
        } else {
          tri_smem<T>(tile, vb, vx, C, l, f, feat);
          for (int c = 0; c < C; c++) X[c * kTile + m] = feat[c];
        }
        encode_dir(d, mlp.n_freq, e);
        const int ne = 3 + 6 * mlp.n_freq;
        for (int j = 0; j < ne; j++) X[(C + j) * kTile + m] = e[j];
        for (int j = C + ne; j < kK1; j++) X[j * kTile + m] = 0.0f;
      } else {
        for (int j = 0; j < kK1; j++) X[j * kTile + m] = 0.0f;
      }
      nbar_arrive(kBarFull0 + b, kMlpThreads + kProdThreads);
    }
    // the MLP threads' last releases of each buffer, so that every barrier is left balanced
    for (uint32_t i = n >= (uint32_t)nbuf ? n - nbuf : 0; i < n; i++)
      nbar_sync(kBarEmpty0 + (i & 1), kMlpThreads + kProdThreads);
    return;
  }
  // -------------------------------------------------------------------- MLP threads
  for (uint32_t i = 0; i < n; i++) {
    const int b = i & 1;
    const float* X = (const float*)(sm + ((i % nbuf) ? F32Smem::x2 : F32Smem::x));
    const uint4 td = w.tile[t_begin + i];
    const uint32_t start = td.x;
    const int mcnt = (int)(td.y & 0xFFu);
    nbar_sync(kBarFull0 + b, kMlpThreads + kProdThreads);  // the producers have filled X
    float c[3];
    // with a backward to follow, the layers' ReLU masks too (two buffers by tile parity: a thread
    // cannot write tile i + 2's masks before every thread has passed tile i + 1's first barrier,
    // which follows its reads of tile i's)
    uint8_t* msk = w.rec_mask ? mask_smem + (i & 1) * 32 * kTile : nullptr;
    mlp_f32_tile(sm, X, c, mlp.in_dim, kBarEmpty0 + b, msk);
    const int m = threadIdx.x;
    if (m < kTile && m < mcnt) {
      const uint32_t rid = __float_as_uint(w.srt[start + m].qd.x);
      w.rec_c[rid] = make_float4(c[0], c[1], c[2], w.srt[start + m].pw.w);
      if (msk) {
        uint32_t v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {  // word q: bytes tn = 4 q' .. of layer q / 4
          const uint8_t* src = msk + (q >> 2) * 16 * kTile + (q & 3) * 4 * kTile + m;
          v[q] = (uint32_t)src[0] | ((uint32_t)src[kTile] << 8) | ((uint32_t)src[2 * kTile] << 16) |
                 ((uint32_t)src[3 * kTile] << 24);
        }
        w.rec_mask[2 * (size_t)rid] = make_uint4(v[0], v[1], v[2], v[3]);
        w.rec_mask[2 * (size_t)rid + 1] = make_uint4(v[4], v[5], v[6], v[7]);
      }
    }
  }
}

// The samples that the backward's tensor-core forward recompute (k_fwd_x3) listed (a ReLU
// pre-activation within its error estimate of zero for the split-BF16 products), recomputed with the FP32
// MLP of K5f: (c, w) and both ReLU masks overwritten.  The list holds sorted record indices
// (rec_key, count in hdr[4]); 128 samples per step, features interpolated from global memory.
// Launched only after k_fwd_x3, so C <= 16.
template <typename T>
__global__ void __launch_bounds__(kMlpThreads, 1) k_fwd_fix(GridGeo g, MlpPtrs mlp, RenderWs w,
                                                           const T* __restrict__ feat) {
  extern __shared__ __align__(128) char sm[];
  float* X = (float*)(sm + F32Smem::x);
  uint8_t* msk = (uint8_t*)(sm + F32Smem::x2);  // [2][16][128] ReLU bytes (store_relu_bits)
  load_mlp_f32_smem(sm, mlp);
  const uint32_t n = w.hdr[4];
  const int C = g.C, m = threadIdx.x;
  const int ne = 3 + 6 * mlp.n_freq;
  const int ms = m & (kTile - 1);  // the step's sample of this thread: threads < 128 interpolate its
                                   // features, the others encode its direction, side by side
  for (uint32_t base = blockIdx.x * kTile; base < n; base += gridDim.x * kTile) {
    const bool valid = m < kTile && base + m < n;
    const bool has = base + ms < n;
    uint32_t si = 0;
    __syncthreads();  // the weights, or the previous step's reads of X and the masks
    if (has) si = w.rec_key[base + ms];
    if (m < kTile) {
      float fx[16];
#pragma unroll
      for (int c = 0; c < 16; c++) fx[c] = 0.0f;
      if (has) {
        const float4 pw = w.srt[si].pw;
        const float p[3] = {pw.x, pw.y, pw.z};
        int i0[3];
        float f[3];
        if (index_sample(g, p, i0, f)) {
#pragma unroll
          for (int q = 0; q < 8; q++) {  // corners outer, channels inner: every load in flight at once
            const float wq = ((q & 1) ? f[0] : 1.f - f[0]) * (((q >> 1) & 1) ? f[1] : 1.f - f[1]) *
                             ((q >> 2) ? f[2] : 1.f - f[2]);
            const size_t vx = ((size_t)(i0[2] + (q >> 2)) * g.n[1] + (i0[1] + ((q >> 1) & 1))) * g.n[0] +
                              (i0[0] + (q & 1));
            const T* v = feat + vx * C;
#pragma unroll
            for (int c = 0; c < 16; c++)
              if (c < C) fx[c] = fmaf(wq, ldf(v + c), fx[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 16; c++)
        if (c < C) X[c * kTile + m] = fx[c];
    } else {
      float e[3 + 6 * 7];
      if (has) {
        const float4 qd = w.srt[si].qd;
        const float d[3] = {qd.y, qd.z, qd.w};
        encode_dir(d, mlp.n_freq, e);
        for (int j = 0; j < ne; j++) X[(C + j) * kTile + ms] = e[j];
      } else {
        for (int j = 0; j < ne; j++) X[(C + j) * kTile + ms] = 0.0f;
      }
      for (int j = C + ne; j < kK1; j++) X[j * kTile + ms] = 0.0f;
    }
    __syncthreads();
    float c[3];
    mlp_f32_tile(sm, X, c, mlp.in_dim, 0, msk);
    if (valid) {
      const uint32_t rid = __float_as_uint(w.srt[si].qd.x);
      w.rec_c[rid] = make_float4(c[0], c[1], c[2], w.srt[si].pw.w);
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const uint8_t* src = msk + (q >> 2) * 16 * kTile + (q & 3) * 4 * kTile + m;
        v[q] = (uint32_t)src[0] | ((uint32_t)src[kTile] << 8) | ((uint32_t)src[2 * kTile] << 16) |
               ((uint32_t)src[3 * kTile] << 24);
      }
      w.rec_mask[2 * (size_t)rid] = make_uint4(v[0], v[1], v[2], v[3]);
      w.rec_mask[2 * (size_t)rid + 1] = make_uint4(v[4], v[5], v[6], v[7]);
    }
  }
}

template <typename T>
static cicero_status launch_fwd_fix(const GridGeo& geo, const MlpPtrs& mlp, const RenderWs& ws, const void* feat,
                                    cudaStream_t st) {
  const int smem = F32Smem::x2 + 2 * 16 * kTile;
  cudaError_t e = cudaFuncSetAttribute(k_fwd_fix<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fwd_fix)");
  {
    ProfScope ps(kStGatherMlp, st);
    k_fwd_fix<T><<<num_sms(), kMlpThreads, smem, st>>>(geo, mlp, ws, (const T*)feat);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_fwd_fix");
}

// K6: per ray, in slot order.
// Sum over one ray's n records of w c: lane l takes records l, l + 32, l + 64, ... in that order
// (so every caller sums identically), with the loads of four of them issued before their sums.
__device__ __forceinline__ void ray_color_sum(const RenderWs& w, uint32_t start, uint32_t n, float& a0, float& a1,
                                              float& a2) {
  const uint32_t lane = threadIdx.x & 31u;
  a0 = a1 = a2 = 0.f;
  for (uint32_t j0 = 0; j0 < n; j0 += 128) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t j = j0 + 32u * u + lane;
      v[u] = j < n ? w.rec_c[start + j] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      if (j0 + 32u * u + lane < n) {
        a0 += v[u].w * v[u].x;
        a1 += v[u].w * v[u].y;
        a2 += v[u].w * v[u].z;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_composite(RaySrc src, Samp s, RenderWs w, OutBufs out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int R = ray_count(src);
  const unsigned full = 0xffffffffu;
  // lane j reads the header and output pixel of the j-th of each group of 32 of the warp's rays
  // (r = warp + i nwarps); the warp then composites them one by one
  for (long long i0 = 0;; i0 += 32) {
    const long long rl = (long long)warp + (i0 + lane) * nwarps;
    const unsigned have = __ballot_sync(full, rl < R);
    if (!have) break;
    uint32_t n_l = 0, start_l = 0;
    float T_l = 0.0f;
    RayRef rr;
    rr.view = 0;
    rr.pix = 0;
    if (rl < R) {
      n_l = w.ray_n[rl];
      start_l = w.ray_start[rl];
      T_l = w.ray_T[rl];
      rr = ray_ref(src, (int)rl);
    }
    const int nq = __popc(have);
    for (int jj = 0; jj < nq; jj++) {
      const uint32_t n = __shfl_sync(full, n_l, jj), start = __shfl_sync(full, start_l, jj);
      const float T = __shfl_sync(full, T_l, jj);
      const int view = __shfl_sync(full, rr.view, jj), pix = __shfl_sync(full, rr.pix, jj);
      float a0, a1, a2;
      ray_color_sum(w, start, n, a0, a1, a2);
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      if (lane == 0) {
        float* rgb = out.rgb[view];
        rgb[3 * pix + 0] = a0 + T * s.bg[0];
        rgb[3 * pix + 1] = a1 + T * s.bg[1];
        rgb[3 * pix + 2] = a2 + T * s.bg[2];
      }
    }
  }
}

// -------------------------------------------------------------------------------------------
// Batched render: every ray of every job in one launch per stage.  Rays are numbered job after
// job, and so are bricks, so bucketing, scan and scatter run unchanged on the batch.

// Per-warp copy of the current job's geometry and sampling in shared memory, refreshed when the
// warp's ray belongs to another job (the march reads them there, not from registers).
struct JobCache {
  GridGeo g;
  Samp s;
  int job;
};

template <typename T>
__global__ void __launch_bounds__(256, 4) k_march_batch(const JobDesc* __restrict__ jobs, int R, RenderWs w) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  __shared__ JobCache cache[8];
  __shared__ RaySetup setup[8];
  __shared__ uint8_t slot_list[8][kMaskSlots];
  const int wb = threadIdx.x >> 5;
  JobCache& C = cache[wb];
  if (lane == 0) C.job = -1;
  __syncwarp();
  // as in k_march: the rays' setups (with their jobs) come from K0
  uint32_t next = warp < R ? setup_word(w, warp, lane) : 0u;
  for (long long r = warp; r < R; r += nwarps) {
    if (lane < kSetupWords) reinterpret_cast<uint32_t*>(&setup[wb])[lane] = next;
    __syncwarp();
    if (r + nwarps < R) next = setup_word(w, r + nwarps, lane);
    const RaySetup& q = setup[wb];
    const int j = q.view;
    const JobDesc& J = jobs[j];
    if (C.job != j) {
      constexpr int kWords = (int)((sizeof(GridGeo) + sizeof(Samp)) / 4);
      static_assert(offsetof(JobCache, s) == sizeof(GridGeo), "cache layout");
      static_assert(offsetof(JobDesc, samp) == offsetof(JobDesc, geo) + sizeof(GridGeo), "job layout");
      const uint32_t* src = (const uint32_t*)&J.geo;
      uint32_t* dst = (uint32_t*)&C.g;
      for (int k = lane; k < kWords; k += 32) dst[k] = src[k];
      if (lane == 0) C.job = j;
      __syncwarp();
    }
    // a batch's records carry no extras (no backward, no export)
    march_ray_core<T, false>(C.g, C.s, (const T*)J.density, w, (int)r, q, (uint32_t)J.brick_base,
                             J.depth ? J.depth + q.pix : nullptr, nullptr, nullptr, slot_list[wb], j);
    __syncwarp();  // the setup slot is free for the next ray
  }
}

__global__ void __launch_bounds__(256) k_tiles_batch(const JobDesc* __restrict__ jobs, const int* __restrict__ bases,
                                                     int n_jobs, RenderWs w) {
  const uint32_t n = w.hdr[1];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int lo = 0, hi = w.nb;  // largest b with tile_off[b] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w.tile_off[mid] <= t) lo = mid;
      else hi = mid;
    }
    const uint32_t start = w.brick_off[(size_t)lo * kOctants] + (t - w.tile_off[lo]) * kTile;
    const uint32_t cnt = min(start + (uint32_t)kTile, w.brick_off[(size_t)(lo + 1) * kOctants]) - start;
    const int j = job_of(bases + n_jobs, n_jobs, lo);
    const int* nb = jobs[j].geo.nb;
    const uint32_t b = (uint32_t)(lo - jobs[j].brick_base);
    const uint32_t bx = b % nb[0], by = (b / nb[0]) % nb[1], bz = b / (nb[0] * nb[1]);
    w.tile[t] = make_uint4(start, cnt | (bz << 8) | ((uint32_t)j << 21), (uint32_t)lo, bx | (by << 16));
  }
}

__global__ void __launch_bounds__(256) k_composite_batch(const JobDesc* __restrict__ jobs, int n_jobs, int R,
                                                         RenderWs w) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned full = 0xffffffffu;
  // as in k_composite: lane j reads the header of the j-th of each group of 32 of the warp's rays,
  // with its job (the tag the march left), output pixel and background; the warp then composites
  // them one by one
  for (long long i0 = 0;; i0 += 32) {
    const long long rl = (long long)warp + (i0 + lane) * nwarps;
    const unsigned have = __ballot_sync(full, rl < R);
    if (!have) break;
    uint32_t n_l = 0, start_l = 0;
    float T_l = 0.0f, bg0 = 0.0f, bg1 = 0.0f, bg2 = 0.0f;
    float* px_l = nullptr;
    if (rl < R) {
      n_l = w.ray_n[rl];
      start_l = w.ray_start[rl];
      T_l = w.ray_T[rl];
      const JobDesc& J = jobs[__float_as_int(w.ray_dir[rl].w)];
      px_l = J.rgb + 3 * ((int)rl - J.ray_base);
      bg0 = J.samp.bg[0];
      bg1 = J.samp.bg[1];
      bg2 = J.samp.bg[2];
    }
    const int nq = __popc(have);
    for (int jj = 0; jj < nq; jj++) {
      const uint32_t n = __shfl_sync(full, n_l, jj), start = __shfl_sync(full, start_l, jj);
      const float T = __shfl_sync(full, T_l, jj);
      float a0, a1, a2;
      ray_color_sum(w, start, n, a0, a1, a2);
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      if (lane == jj) {  // the lane that holds the ray's pixel writes it
        px_l[0] = a0 + T * bg0;
        px_l[1] = a1 + T * bg1;
        px_l[2] = a2 + T * bg2;
      }
    }
  }
  (void)n_jobs;
}

// Ray Index Table export: sample id = ray * S + slot.
__global__ void k_rit_export(RenderWs w, int n_bricks, int32_t* offs, int32_t* samples) {
  const uint32_t total = w.hdr[2];
  const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  for (size_t i = i0; i <= (size_t)n_bricks; i += st) offs[i] = (int32_t)w.brick_off[i * kOctants];
  for (size_t i = i0; i < total; i += st) {
    const uint32_t q = __float_as_uint(w.srt[i].qd.x);
    samples[i] = (int32_t)(w.rec_ray[q] * (uint32_t)w.S + w.rec_slot[q]);
  }
}

// -------------------------------------------------------------------------------------------
// host side

BrickBox brick_box(const GridGeo& geo, int elem) {
  BrickBox b;
  b.vb = geo.brick + 1;
  int vx = b.vb;
  while ((vx * geo.C * elem) % 16) vx++;
  b.vx = vx;
  b.row_bytes = vx * geo.C * elem;
  b.box_bytes = b.vb * b.vb * b.row_bytes;
  return b;
}

// blocks of K0 (256 rays each, grid-stride beyond 8 blocks per SM)
static int setup_blocks(long long rays) {
  return (int)std::max(1ll, std::min((rays + 255) / 256, (long long)num_sms() * 8));
}

static int blocks_for_warps(long long warps, int per_sm) {
  long long blocks = (warps + 7) / 8;
  long long cap = (long long)num_sms() * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <typename T>
static cicero_status launch_f32(const GridGeo& geo, int S, const MlpPtrs& mlp, const RenderWs& ws,
                                const CUtensorMap& map, const BrickBox& box, cudaStream_t st) {
  const int masks = ws.rec_mask ? 2 * 32 * kTile : 0;  // ReLU masks of two tiles for the backward
  const int boxa = (box.box_bytes + 127) & ~127;
  const int nbuf = F32Smem::tile + boxa + masks <= 227 * 1024 ? 2 : 1;  // two input buffers when they fit
  const int smem = (nbuf == 2 ? F32Smem::tile : F32Smem::tile1) + boxa + masks;
  if (smem > 227 * 1024) return fail(CICERO_ERR_UNSUPPORTED, "brick too large for the FP32 feature-computation kernel");
  auto kern = k_gather_mlp_f32<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gather_mlp_f32)");
  {
    ProfScope ps(kStGatherMlp, st);
    kern<<<num_sms(), kMlpThreads + kProdThreads, smem, st>>>(geo, S, mlp, ws, map, box.vb, box.vx, box.box_bytes,
                                                                   nbuf);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_gather_mlp_f32");
}

cicero_status run_render(const cicero_grid* grid, const MlpPtrs& mlp, const RenderPlan& plan, const RaySrc& src,
                         const RenderWs& ws, const OutBufs& out, bool stop_after_bucketing, cudaStream_t st,
                         const HashGeo* hash) {
  const GridGeo& geo = plan.geo;
  const bool f16 = grid->dtype == CICERO_F16;
  const int mb = blocks_for_warps(src.n_max, 16);
  {
    ProfScope ps(kStMarch, st);
    k_clear<<<std::min(num_sms() * 4, (plan.nb * kOctants + 255) / 256 + 1), 256, 0, st>>>(ws.hdr, 16, ws.brick_cnt,
                                                                                  (size_t)plan.nb * kOctants);
    const bool extra = ws.rec_ray || ws.rec_T;
    k_ray_setup<false><<<setup_blocks(src.n_max), 256, 0, st>>>(geo, plan.samp, src, nullptr, nullptr, 0, 0, ws);
    if (f16 && extra)
      k_march<__half, true><<<mb, 256, 0, st>>>(geo, plan.samp, src, (const __half*)grid->density, ws, out);
    else if (f16)
      k_march<__half, false><<<mb, 256, 0, st>>>(geo, plan.samp, src, (const __half*)grid->density, ws, out);
    else if (extra)
      k_march<float, true><<<mb, 256, 0, st>>>(geo, plan.samp, src, (const float*)grid->density, ws, out);
    else
      k_march<float, false><<<mb, 256, 0, st>>>(geo, plan.samp, src, (const float*)grid->density, ws, out);
  }
  {
    ProfScope ps(kStBucket, st);
    const int nblk = (plan.nb + kScanChunk - 1) / kScanChunk;
    k_brick_sums<<<nblk, 1024, 0, st>>>(ws);
    k_brick_blocks<<<1, 1024, 0, st>>>(ws, nblk);
    k_brick_offsets<<<nblk, 1024, 0, st>>>(ws);
    k_tiles<<<num_sms() * 4, 256, 0, st>>>(geo, ws);
    k_scatter<<<mb, 256, 0, st>>>(src, ws);
  }
  count_launches(8);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "march/bucket kernels");
  if (stop_after_bucketing) return CICERO_OK;

  cicero_status s;
  const BrickBox box = brick_box(geo, f16 ? 2 : 4);
  CUtensorMap map;
  if (hash) {
    s = launch_gather_mlp_bf16_hash(geo, mlp, ws, *hash, st);  // features from the hash encoding
  } else if (plan.precision == CICERO_MLP_FP32_SPLIT) {
    // split-BF16 tensor-core MLP, features read from global memory (no staged brick)
    if (!fwd_x3_supported(geo, mlp))
      return fail(CICERO_ERR_UNSUPPORTED, "the split-BF16 MLP takes at most 16 feature channels");
    s = launch_fwd_x3(grid, geo, mlp, ws, st);  // colours only (no masks: rec_mask is NULL)
  } else if (ws.rec_mask && fwd_x3_supported(geo, mlp)) {
    // a backward follows: colours and ReLU masks only, on the tensor cores, then the uncertain
    // samples again in FP32
    s = launch_fwd_x3(grid, geo, mlp, ws, st);
    if (s == CICERO_OK)
      s = f16 ? launch_fwd_fix<__half>(geo, mlp, ws, grid->features, st)
              : launch_fwd_fix<float>(geo, mlp, ws, grid->features, st);
  } else if ((s = encode_brick_map(grid, geo, box, &map)) != CICERO_OK) {
    return s;
  } else if (plan.precision == CICERO_MLP_BF16) {
    s = launch_gather_mlp_bf16(grid, geo, plan.mlp_groups, mlp, ws, map, box, st);
  } else {
    s = f16 ? launch_f32<__half>(geo, plan.S, mlp, ws, map, box, st)
            : launch_f32<float>(geo, plan.S, mlp, ws, map, box, st);
  }
  if (s != CICERO_OK) return s;
  if (!out.rgb[0]) return CICERO_OK;  // the backward only needs the per-sample records
  {
    ProfScope ps(kStComposite, st);
    k_composite<<<mb, 256, 0, st>>>(src, plan.samp, ws, out);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_composite");
}

cicero_status run_render_batch(const BatchPlan& b, cudaStream_t st) {
  const RenderPlan& plan = b.plan;
  const RenderWs& ws = b.ws;
  const int R = plan.R;
  if (R == 0) return CICERO_OK;
  RaySrc src;
  memset(&src, 0, sizeof src);
  src.n_max = R;
  const int mb = blocks_for_warps(R, 16);
  {
    ProfScope ps(kStMarch, st);
    k_clear<<<std::min(num_sms() * 4, (plan.nb * kOctants + 255) / 256 + 1), 256, 0, st>>>(ws.hdr, 16, ws.brick_cnt,
                                                                                  (size_t)plan.nb * kOctants);
    k_ray_setup<true><<<setup_blocks(R), 256, 0, st>>>(plan.geo, plan.samp, src, b.jobs, b.bases, b.n_jobs, R, ws);
    if (b.f16)
      k_march_batch<__half><<<mb, 256, 0, st>>>(b.jobs, R, ws);
    else
      k_march_batch<float><<<mb, 256, 0, st>>>(b.jobs, R, ws);
  }
  {
    ProfScope ps(kStBucket, st);
    const int nblk = (plan.nb + kScanChunk - 1) / kScanChunk;
    k_brick_sums<<<nblk, 1024, 0, st>>>(ws);
    k_brick_blocks<<<1, 1024, 0, st>>>(ws, nblk);
    k_brick_offsets<<<nblk, 1024, 0, st>>>(ws);
    k_tiles_batch<<<num_sms() * 4, 256, 0, st>>>(b.jobs, b.bases, b.n_jobs, ws);
    k_scatter<<<mb, 256, 0, st>>>(src, ws);
  }
  count_launches(8);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batched march/bucket kernels");
  cicero_status s = launch_gather_mlp_bf16_batch(b, st);
  if (s != CICERO_OK) return s;
  {
    ProfScope ps(kStComposite, st);
    k_composite_batch<<<mb, 256, 0, st>>>(b.jobs, b.n_jobs, R, ws);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_composite_batch");
}

cicero_status run_rit_export(const RenderWs& ws, int n_bricks, int S, int32_t* brick_offsets, int32_t* samples,
                             cudaStream_t st) {
  (void)S;
  k_rit_export<<<num_sms() * 4, 256, 0, st>>>(ws, n_bricks, brick_offsets, samples);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_rit_export");
}

// Feature Computation alone (FP32): c = MLP(x) for M inputs, 128 per tile.
__global__ void __launch_bounds__(256, 1) k_mlp_eval_f32(MlpPtrs mlp, const float* x, int M, float* c) {
  extern __shared__ __align__(128) char sm[];
  float* X = (float*)(sm + F32Smem::x);
  load_mlp_f32_smem(sm, mlp);
  __syncthreads();
  const int ntile = (M + kTile - 1) / kTile;
  for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
    for (int i = threadIdx.x; i < kK1 * kTile; i += blockDim.x) {
      const int k = i / kTile, m = i % kTile, row = t * kTile + m;
      X[i] = (k < mlp.in_dim && row < M) ? x[(size_t)row * mlp.in_dim + k] : 0.0f;
    }
    __syncthreads();
    float cc[3];
    mlp_f32_tile(sm, X, cc, mlp.in_dim);
    const int row = t * kTile + threadIdx.x;
    if (threadIdx.x < kTile && row < M) {
      c[3 * row + 0] = cc[0];
      c[3 * row + 1] = cc[1];
      c[3 * row + 2] = cc[2];
    }
    __syncthreads();
  }
}

cicero_status launch_mlp_eval_f32(const MlpPtrs& mlp, const float* x, int M, float* c, cudaStream_t st) {
  const int smem = F32Smem::bar;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_eval_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_eval_f32)");
  const int ntile = (M + kTile - 1) / kTile;
  {
    ProfScope ps(kStMlpEval, st);
    k_mlp_eval_f32<<<std::max(1, std::min(ntile, num_sms())), 256, smem, st>>>(mlp, x, M, c);
  }
  count_launches(1);
  e = cudaGetLastError();
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "k_mlp_eval_f32");
}

}  // namespace cicero
