// Host-side declarations shared by the translation units of libcicero.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/cicero.h"
#include "common.cuh"

namespace cicero {

void set_error(const std::string& msg);
cicero_status fail(cicero_status st, const std::string& msg);
cicero_status cuda_fail(cudaError_t e, const char* where);

int num_sms();

// Stage timing with CUDA events on the launching stream (off unless cicero_profile_begin was
// called) and a count of the kernels the library launches.
enum Stage { kStMarch = 0, kStBucket, kStGatherMlp, kStComposite, kStWarpSplat, kStWarpResolve, kStBwdRay,
             kStBwdBrick, kStMlpEval, kStBwdWeights, kNumStages };
void count_launches(int n);
struct ProfScope {
  ProfScope(int stage, cudaStream_t st);
  ~ProfScope();
  int stage;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  bool on;
};

// Workspace of one rendering call (all device pointers, carved from the caller's buffer).
// Records (one per composited sample) are allocated per ray from a capacity of Q records: each ray
// reserves an upper bound of its sample count (from the slab test) and fills a prefix of it.
// One record of the sorted Ray Index Table payload: (position, weight) and (record index as
// bits, ray direction).  32 bytes, so that every record the scatter writes is one whole DRAM
// sector (no partial-sector writes when neighbouring records land from different rays).
struct __align__(32) SrtRec {
  float4 pw, qd;
};

// Per-ray geometry of the samples: (origin, first slot's t0) and (unit direction, slot step dt);
// slot k sits at o + (t0 + (k + 1/2) dt) d.
struct __align__(16) RayGeo {
  float4 ot, dd;
};

struct RenderWs {
  uint32_t* hdr;        // [0] error bits, [1] tile count, [2] composited samples, [3] records reserved,
                        // [4] samples listed for the FP32 fix-up of the backward's forward recompute
  uint32_t* ray_n;      // [R] composited samples of each ray
  uint32_t* ray_start;  // [R] first record of each ray
  float* ray_T;         // [R] transmittance after the last composited slot
  float4* ray_dir;      // [R] unit direction of each ray
  uint32_t* rec_key;    // [Q] RIT key: brick id * kOctants + octant; once the RIT is built, the backward's
                        // forward recompute lists its uncertain samples here (sorted record indices)
  float* rec_w;         // [Q] weight T_k alpha_k
  uint16_t* rec_slot;   // [Q] slot index
  float4* rec_c;        // [Q] (c_r, c_g, c_b, w) of each record (written by the gather, in record order); in
                        // the backward, B1 replaces it by (dL/dz3 [3], dL/draw)
  float* rec_T;         // [Q] transmittance before the slot (backward only; may be null)
  float* rec_raw;       // [Q] interpolated raw density (backward only; may be null)
  uint32_t* rec_ray;    // [Q] ray of each record (RIT export only; may be null)
  uint4* rec_mask;      // [Q][2] ReLU masks of MLP layers 1 and 2 from the FP32 forward (backward only; may be
                        // null): hidden unit n < 64 is bit n % 4 of byte n / 4, unit 64 + n is bit 4 + n % 4
  uint32_t* brick_cnt;  // [nb * kOctants] records per RIT key
  uint32_t* brick_off;  // [nb * kOctants + 1] first record of each key (brick b starts at key b * kOctants)
  uint32_t* brick_cur;  // [nb * kOctants] scatter cursors
  uint32_t* tile_off;   // [nb + 1] first tile of each brick
  uint32_t* blk_sums;   // [2 * scan blocks] per-block sums of the brick scan
  uint4* tile;          // [max_tiles] (first record, count | bz << 8 | job << 21, brick id, bx | by << 16)
  SrtRec* srt;          // [Q] the Ray Index Table payload in brick order
  RayGeo* ray_geo;      // [R] geometry of each ray's samples
  struct RaySetup* setup;  // [R] per-ray setup of the march (ray, slots, active-slot mask, records)
  char* stage;          // per-sample operands of the MLP weight gradients (backward with d_mlp only; may be
                        // null): blocks of kStageBlock sorted samples, WgStage::bytes each (stage_col)
  int R, S, nb, max_tiles;
  uint32_t Q;
};

// Weight-gradient staging: per block of kStageBlock sorted samples, the split-BF16 operands of the
// weight-gradient GEMMs over the samples, in the MN-major no-swizzle layout that the tensor cores
// read (K = the block's samples): an operand of R rows (hidden units, inputs or outputs) is R / 8
// row groups of 256 bytes for the hi halves, then as many for the lo halves; in row group g, the
// 16 bytes at 16 k hold rows 8 g .. 8 g + 7 of sample k (two 128-byte core matrices of 8 samples).
// Operands: dL/dh2, h1, dL/dh1, h2 (128 rows each), x (48 rows: the input, zero from in_dim),
// dL/dz3 (8 rows: 3 used).
constexpr int kStageBlock = 16;
struct WgStage {
  static constexpr int dh2 = 0, h1 = 8192, dh1 = 16384, h2 = 24576, x = 32768, dz = 35840, bytes = 36352;
};
// bytes of the staging for a capacity of Q samples, and where sample s's 16-byte rows start (row
// group g of an operand of R rows at offset op: + op + 256 g for hi, + op + 32 R + 256 g for lo)
__host__ __device__ inline size_t stage_bytes(uint32_t Q) {
  return (((size_t)Q + kStageBlock - 1) / kStageBlock) * WgStage::bytes;
}
__host__ __device__ inline size_t stage_col(uint32_t s) {
  return (size_t)(s / kStageBlock) * WgStage::bytes + (size_t)(s % kStageBlock) * 16;
}

struct RenderPlan {
  GridGeo geo;
  Samp samp;
  int R, S, nb;
  int max_tiles;
  uint32_t Q;
  bool want_k;
  bool want_bwd;
  bool want_wg;  // the backward stages the MLP weight gradients' operands (RenderWs::stage)
  cicero_precision precision;
  int mlp_groups;  // BF16 tensor-core MLP tiles in flight per SM (0 = as many as fit)
};

// Output buffers of a rendering call, per view (rgb/depth indexed by pixel, or by ray for explicit
// rays); acc and n_steps only for single-view calls.
struct OutBufs {
  float* rgb[kMaxViews];
  float* depth[kMaxViews];
  float* acc;
  int32_t* n_steps;
};

size_t render_ws_bytes(const RenderPlan& p);
bool carve_render_ws(void* ws, size_t bytes, const RenderPlan& p, RenderWs* out);

// grid/sampling validation and geometry (api.cu)
cicero_status make_geo(const cicero_grid* g, int brick, GridGeo* geo, bool with_features = true);
cicero_status make_samp(const cicero_sampling* s, Samp* out);
cicero_status check_mlp(const cicero_mlp* m, const cicero_grid* g);

// the stages (render.cu)
struct MlpPtrs {
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  int in_dim, n_freq;
};

// Two jobs whose MLPs are the same tensors (so their weights need loading once).
__host__ __device__ inline bool same_mlp(const MlpPtrs& a, const MlpPtrs& b) {
  return a.w1 == b.w1 && a.b1 == b.b1 && a.w2 == b.w2 && a.b2 == b.b2 && a.w3 == b.w3 && a.b3 == b.b3 &&
         a.in_dim == b.in_dim && a.n_freq == b.n_freq;
}

struct HashGeo;
cicero_status run_render(const cicero_grid* grid, const MlpPtrs& mlp, const RenderPlan& plan, const RaySrc& src,
                         const RenderWs& ws, const OutBufs& out, bool stop_after_bucketing, cudaStream_t st,
                         const HashGeo* hash = nullptr);

cicero_status run_rit_export(const RenderWs& ws, int n_bricks, int S, int32_t* brick_offsets, int32_t* samples,
                             cudaStream_t st);

// tensor map of the feature grid viewed as [n2][n1][n0 * C] (box: brick + halo)
struct BrickBox {
  int vb;          // vertices per brick edge staged (brick + 1)
  int vx;          // vertices along x in the box (>= vb, box row a multiple of 16 bytes)
  int row_bytes;   // vx * C * elem
  int box_bytes;   // vb * vb * row_bytes
};
BrickBox brick_box(const GridGeo& geo, int elem_bytes);
cicero_status encode_brick_map(const cicero_grid* grid, const GridGeo& geo, const BrickBox& box, CUtensorMap* map);

// One job of a batched render as the kernels read it from the workspace.  Aligned like its first
// member, so the tensor map at its start is a valid TMA descriptor in global memory.
struct JobDesc {  // aligned as CUtensorMap (64 bytes or more)
  CUtensorMap map;   // the job's feature grid, viewed as for a single render
  GridGeo geo;
  Samp samp;
  ViewCam cam;
  MlpPtrs mlp;
  const void* density;
  float* rgb;        // [H*W][3]
  float* depth;      // [H*W] or NULL
  int ray_base;      // first ray of the job in the batch's ray numbering
  int brick_base;    // first brick of the job in the batch's brick numbering
  int n_rays, nb;
};
constexpr int kMaxBatchJobs = 2048;  // the job index rides in 11 bits of a tile descriptor

// Host side of a planned batch (the public cicero_batch handle wraps it).
struct BatchPlan {
  int n_jobs;
  const JobDesc* jobs;  // device copy, in the workspace
  const int* bases;     // device: first ray of each job [n_jobs], then first brick of each job [n_jobs]
  RenderPlan plan;      // totals: rays, records, bricks, tiles
  RenderWs ws;
  BrickBox box;
  bool f16;
  int C, n_freq;
  int mlp_groups;       // tiles in flight per SM requested (0 = as many as fit)
  void* workspace;
  size_t ws_bytes;
};
size_t batch_table_bytes(int n_jobs);
cicero_status run_render_batch(const BatchPlan& b, cudaStream_t st);
cicero_status launch_gather_mlp_bf16_batch(const BatchPlan& b, cudaStream_t st);

cicero_status run_upsample(const float* src, int w, int h, int C, float* dst, int W, int H, cudaStream_t st);

// Multiresolution hash encoding of the hash-grid workload, as the kernels read it.
constexpr int kMaxHashLevels = 16;
struct HashGeo {
  const void* table;            // [levels][T][2], FP16 or FP32
  int levels;
  bool f16;
  uint32_t mask;                // T - 1
  uint32_t dense;               // bit l: level l stored densely
  int res[kMaxHashLevels];      // cells per axis
  float amin[3], inv_ext[3];    // the box: p -> (p - amin) * inv_ext in [0, 1]
};
cicero_status launch_gather_mlp_bf16_hash(const GridGeo& geo, const MlpPtrs& mlp, const RenderWs& ws,
                                          const HashGeo& hg, cudaStream_t st);

// BF16 tensor-core Feature Computation (mlp_tc.cu)
cicero_status launch_gather_mlp_bf16(const cicero_grid* grid, const GridGeo& geo, int mlp_groups,
                                     const MlpPtrs& mlp, const RenderWs& ws, const CUtensorMap& map, const BrickBox& box,
                                     cudaStream_t st);
cicero_status launch_mlp_eval_bf16(const MlpPtrs& mlp, const float* x, int M, float* c, uint32_t* err,
                                   cudaStream_t st);

// SpaRW warp (warp.cu)
struct WarpArgs {
  int wr, hr;          // reference image
  float fr, cxr, cyr;
  int wt, ht;          // target image
  float ft, cxt, cyt;
  float R[9];          // [R_rel | t_rel] = inverse(c2w_tgt) c2w_ref, rounded to FP32
  float t[3];
  float cos_phi;
  int use_phi;
};

struct VoidTest {
  int enabled;
  GridGeo g;
  Samp s;
  RaySrc src;  // target camera pixels
};

constexpr int kMaxWarpViews = kMaxViews;

struct WarpView {
  WarpArgs a;
  float* wrgb;
  float* wdepth;
  uint8_t* mask;
  int32_t* hole_idx;
  int32_t* n_holes;
  unsigned long long* z;  // depth buffer (workspace)
  uint32_t* bsum;         // scan block sums (workspace)
  int nblk;
};

struct WarpBatch {
  int n_views;
  WarpView v[kMaxWarpViews];
};

size_t warp_ws_bytes(int wt, int ht);
size_t warp_batch_ws_bytes(const int* wt, const int* ht, int n_views);
void carve_warp_ws(WarpBatch& B, void* ws);
cicero_status run_warp(const WarpBatch& B, const VoidTest& vt, const float* ref_rgb, const float* ref_depth,
                       cudaStream_t st);
cicero_status run_backward(const cicero_grid* grid, const MlpPtrs& mlp, const RenderPlan& plan, const RaySrc& src,
                           const RenderWs& ws, const float* d_rgb, float* d_dens, float* d_feat, float* d_mlp,
                           cudaStream_t st);
cicero_status launch_mlp_eval_f32(const MlpPtrs& mlp, const float* x, int M, float* c, cudaStream_t st);

// The backward's forward recompute on the tensor cores (split-BF16 products, FP32 accumulation):
// (c, w) into rec_c and the ReLU masks into rec_mask for every composited sample (backward.cu)
bool fwd_x3_supported(const GridGeo& g, const MlpPtrs& mlp);
// dW1 | db1, dW2 | db2, dW3 (and db3) from the staged operands, added to d_mlp (backward.cu)
cicero_status launch_dw(const MlpPtrs& mlp, const RenderWs& ws, float* d_mlp, cudaStream_t st);
cicero_status launch_fwd_x3(const cicero_grid* grid, const GridGeo& geo, const MlpPtrs& mlp, const RenderWs& ws,
                            cudaStream_t st);

}  // namespace cicero
