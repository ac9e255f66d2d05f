// C ABI of libcicero: argument validation, workspace carving and stage launches.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cicero.h"
#include "common.cuh"
#include "internal.h"

namespace cicero {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

cicero_status fail(cicero_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

cicero_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return CICERO_ERR_CUDA;
}

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches += n; }

struct ProfState {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int stage;
    cudaEvent_t e0, e1;
  };
  std::vector<Rec> recs;
  double ms[kNumStages] = {0};
  long long n[kNumStages] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
static ProfState g_prof;

ProfScope::ProfScope(int s, cudaStream_t stream) : stage(s), st(stream), e0(nullptr), e1(nullptr), on(false) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on) return;
  on = true;
  e0 = g_prof.get();
  e1 = g_prof.get();
  cudaEventRecord(e0, st);
}

ProfScope::~ProfScope() {
  if (!on) return;
  cudaEventRecord(e1, st);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.recs.push_back({stage, e0, e1});
}

static void prof_drain() {
  for (auto& r : g_prof.recs) {
    float ms = 0.0f;
    if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      g_prof.ms[r.stage] += ms;
      g_prof.n[r.stage] += 1;
    }
    g_prof.pool.push_back(r.e0);
    g_prof.pool.push_back(r.e1);
  }
  g_prof.recs.clear();
}

static int elem_bytes(cicero_dtype t) { return t == CICERO_F16 ? 2 : 4; }

cicero_status make_geo(const cicero_grid* g, int brick, GridGeo* geo, bool with_features) {
  if (!g) return fail(CICERO_ERR_INVALID_ARG, "grid is NULL");
  if (!g->density || (with_features && !g->features))
    return fail(CICERO_ERR_INVALID_ARG, "grid density/features is NULL");
  if (g->dtype != CICERO_F32 && g->dtype != CICERO_F16) return fail(CICERO_ERR_INVALID_ARG, "grid dtype");
  if (g->C < 1 || g->C > 21) return fail(CICERO_ERR_UNSUPPORTED, "feature channels must be 1..21");
  if (brick != 4 && brick != 8 && brick != 16) return fail(CICERO_ERR_INVALID_ARG, "brick must be 4, 8 or 16");
  memset(geo, 0, sizeof *geo);
  for (int a = 0; a < 3; a++) {
    if (g->n[a] < 2 || g->n[a] > (1 << 15)) return fail(CICERO_ERR_INVALID_ARG, "grid size must be 2..32768");
    if (!(g->aabb_max[a] > g->aabb_min[a])) return fail(CICERO_ERR_INVALID_ARG, "empty grid box");
    geo->n[a] = g->n[a];
    geo->amin[a] = g->aabb_min[a];
    geo->amax[a] = g->aabb_max[a];
    const float ext = g->aabb_max[a] - g->aabb_min[a];
    geo->inv_h[a] = (float)(g->n[a] - 1) / ext;
    geo->nb[a] = (g->n[a] - 2) / brick + 1;
  }
  if (g->occ) {
    if (g->occ_res < 1) return fail(CICERO_ERR_INVALID_ARG, "occupancy mask needs occ_res >= 1");
    for (int a = 0; a < 3; a++) geo->occ_scale[a] = (float)g->occ_res / (float)(g->n[a] - 1);
  }
  geo->C = g->C;
  geo->act_shift = g->act_shift;
  geo->occ = g->occ;
  geo->occ_res = g->occ ? g->occ_res : 0;
  geo->brick = brick;
  geo->brick_shift = brick == 4 ? 2 : brick == 8 ? 3 : 4;
  geo->idx32 = (unsigned long long)g->n[0] * g->n[1] * g->n[2] <= 0x7FFFFFFFull ? 1 : 0;
  const size_t row = (size_t)g->n[0] * g->C * elem_bytes(g->dtype);
  if (with_features && (((uintptr_t)g->features & 15) || (row & 15)))
    return fail(CICERO_ERR_ALIGNMENT, "features must be 16-byte aligned with n0*C*elem a multiple of 16 (TMA)");
  const long long nbr = (long long)geo->nb[0] * geo->nb[1] * geo->nb[2];
  if (nbr > (1ll << 26)) return fail(CICERO_ERR_UNSUPPORTED, "too many bricks");
  return CICERO_OK;
}

cicero_status make_samp(const cicero_sampling* s, Samp* out) {
  if (!s) return fail(CICERO_ERR_INVALID_ARG, "sampling is NULL");
  if (s->n_samples < 1 || s->n_samples > 65535) return fail(CICERO_ERR_INVALID_ARG, "n_samples must be 1..65535");
  if (!(s->step >= 0.0f)) return fail(CICERO_ERR_INVALID_ARG, "step must be >= 0");
  if (s->step == 0.0f && !(s->far_t > s->near_t)) return fail(CICERO_ERR_INVALID_ARG, "far must exceed near");
  if (!(s->t_stop >= 0.0f)) return fail(CICERO_ERR_INVALID_ARG, "t_stop must be >= 0");
  out->near_t = s->near_t;
  out->far_t = s->far_t;
  out->n_samples = s->n_samples;
  out->step = s->step;
  out->t_stop = s->t_stop;
  for (int c = 0; c < 3; c++) out->bg[c] = s->bg[c];
  out->void_acc = s->void_acc;
  return CICERO_OK;
}

cicero_status check_mlp(const cicero_mlp* m, const cicero_grid* g) {
  if (!m) return fail(CICERO_ERR_INVALID_ARG, "mlp is NULL");
  if (!m->w1 || !m->b1 || !m->w2 || !m->b2 || !m->w3 || !m->b3) return fail(CICERO_ERR_INVALID_ARG, "mlp weight is NULL");
  if (m->hidden != kHidden) return fail(CICERO_ERR_UNSUPPORTED, "hidden width must be 128");
  if (m->n_freq < 0) return fail(CICERO_ERR_INVALID_ARG, "n_freq must be >= 0");
  if (g && m->in_dim != g->C + 3 + 6 * m->n_freq) return fail(CICERO_ERR_INVALID_ARG, "in_dim != C + 3 + 6 n_freq");
  if (m->in_dim > kMaxIn || m->in_dim < 1) return fail(CICERO_ERR_UNSUPPORTED, "in_dim must be 1..48");
  return CICERO_OK;
}

static MlpPtrs mlp_ptrs(const cicero_mlp* m) {
  MlpPtrs p;
  p.w1 = m->w1;
  p.b1 = m->b1;
  p.w2 = m->w2;
  p.b2 = m->b2;
  p.w3 = m->w3;
  p.b3 = m->b3;
  p.in_dim = m->in_dim;
  p.n_freq = m->n_freq;
  return p;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

cicero_status encode_brick_map(const cicero_grid* grid, const GridGeo& geo, const BrickBox& box, CUtensorMap* map) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(CICERO_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const int es = elem_bytes(grid->dtype);
  if (box.vx * geo.C > 256 || box.vb > 256) return fail(CICERO_ERR_UNSUPPORTED, "brick box exceeds 256 elements");
  if (box.box_bytes > 227 * 1024) return fail(CICERO_ERR_UNSUPPORTED, "brick box does not fit in shared memory");
  cuuint64_t dims[3] = {(cuuint64_t)geo.n[0] * geo.C, (cuuint64_t)geo.n[1], (cuuint64_t)geo.n[2]};
  cuuint64_t strides[2] = {(cuuint64_t)geo.n[0] * geo.C * es, (cuuint64_t)geo.n[0] * geo.n[1] * geo.C * es};
  cuuint32_t boxd[3] = {(cuuint32_t)(box.vx * geo.C), (cuuint32_t)box.vb, (cuuint32_t)box.vb};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, grid->dtype == CICERO_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  (void*)grid->features, dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CICERO_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return CICERO_OK;
}

static bool ws_ok(const void* ws) { return ws && (((uintptr_t)ws) & 255) == 0; }

static cicero_status plan_render(const cicero_grid* grid, const cicero_mlp* mlp, int n_rays, const cicero_sampling* s,
                                 const cicero_options* opt, RenderPlan* p, bool need_mlp, bool with_features = true) {
  const int brick = (opt && opt->brick) ? opt->brick : 8;
  cicero_status st = make_geo(grid, brick, &p->geo, with_features);
  if (st != CICERO_OK) return st;
  st = make_samp(s, &p->samp);
  if (st != CICERO_OK) return st;
  if (need_mlp) {
    st = check_mlp(mlp, grid);
    if (st != CICERO_OK) return st;
  }
  if (n_rays < 0) return fail(CICERO_ERR_INVALID_ARG, "negative ray count");
  const unsigned long long RS = (unsigned long long)n_rays * (unsigned long long)s->n_samples;
  unsigned long long Q = RS;
  if (opt && opt->max_records > 0 && (unsigned long long)opt->max_records < Q) Q = (unsigned long long)opt->max_records;
  if (Q >= 0xffffffffull) return fail(CICERO_ERR_UNSUPPORTED, "record capacity must be below 2^32 (set max_records)");
  p->R = n_rays;
  p->S = s->n_samples;
  p->Q = (uint32_t)Q;
  p->nb = p->geo.nb[0] * p->geo.nb[1] * p->geo.nb[2];
  p->max_tiles = (int)((Q + kTile - 1) / kTile) + p->nb;
  p->want_k = false;
  p->want_bwd = false;
  p->want_wg = false;
  p->precision = opt ? opt->precision : CICERO_MLP_FP32;
  if (p->precision != CICERO_MLP_FP32 && p->precision != CICERO_MLP_BF16 && p->precision != CICERO_MLP_FP32_SPLIT)
    return fail(CICERO_ERR_INVALID_ARG, "precision");
  p->mlp_groups = opt ? opt->mlp_groups : 0;
  if (p->mlp_groups < 0 || p->mlp_groups > 4) return fail(CICERO_ERR_INVALID_ARG, "mlp_groups must be 0..4");
  return CICERO_OK;
}

static ViewCam view_of(const cicero_camera* cam) {
  ViewCam v;
  for (int i = 0; i < 12; i++) v.c2w[i] = cam->c2w[i];
  v.f = cam->f;
  v.cx = cam->cx;
  v.cy = cam->cy;
  v.width = cam->width;
  return v;
}

static RaySrc camera_src(const cicero_camera* cam) {
  RaySrc s;
  memset(&s, 0, sizeof s);
  s.kind = 0;
  s.n_views = 1;
  s.cam[0] = view_of(cam);
  s.n_max = cam->width * cam->height;
  return s;
}

static OutBufs single_out(float* rgb, float* depth, float* acc, int32_t* n_steps) {
  OutBufs o;
  memset(&o, 0, sizeof o);
  o.rgb[0] = rgb;
  o.depth[0] = depth;
  o.acc = acc;
  o.n_steps = n_steps;
  return o;
}

static cicero_status check_cam(const cicero_camera* c) {
  if (!c) return fail(CICERO_ERR_INVALID_ARG, "camera is NULL");
  if (c->width < 1 || c->height < 1 || (long long)c->width * c->height > (1ll << 30))
    return fail(CICERO_ERR_INVALID_ARG, "camera size");
  if (!(c->f > 0.0f)) return fail(CICERO_ERR_INVALID_ARG, "focal length must be > 0");
  for (int i = 0; i < 12; i++)
    if (!isfinite(c->c2w[i])) return fail(CICERO_ERR_INVALID_ARG, "camera pose is not finite");
  return CICERO_OK;
}

// A call with no rays queues no kernel; it still clears the workspace's status word (on the
// caller's stream), so that cicero_workspace_status after it reports CICERO_OK whatever the
// workspace held before.
static cicero_status no_rays(const RenderWs& w, void* stream) {
  const cudaError_t e = cudaMemsetAsync(w.hdr, 0, 4, (cudaStream_t)stream);
  return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "cudaMemsetAsync(status word)");
}

static cicero_status render_common(const cicero_grid* grid, const cicero_mlp* mlp, const cicero_sampling* s,
                                   const cicero_options* opt, const RaySrc& src, int n_rays, float* rgb, float* depth,
                                   float* acc, int32_t* n_steps, void* ws, size_t ws_bytes, void* stream) {
  RenderPlan plan;
  cicero_status st = plan_render(grid, mlp, n_rays, s, opt, &plan, true);
  if (st != CICERO_OK) return st;
  if (!rgb && n_rays > 0) return fail(CICERO_ERR_INVALID_ARG, "rgb is NULL");
  if (!ws_ok(ws)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  RenderWs w;
  if (!carve_render_ws(ws, ws_bytes, plan, &w)) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  if (n_rays == 0) return no_rays(w, stream);
  return run_render(grid, mlp_ptrs(mlp), plan, src, w, single_out(rgb, depth, acc, n_steps), false,
                    (cudaStream_t)stream);
}

// relative pose [R | t] = inverse(c2w_tgt) c2w_ref in FP64, rounded once to FP32
static void relative_pose(const cicero_camera* ref, const cicero_camera* tgt, float R[9], float t[3]) {
  double Ra[9], Rb[9], ta[3], tb[3];
  for (int a = 0; a < 3; a++) {
    for (int b = 0; b < 3; b++) {
      Ra[3 * a + b] = ref->c2w[4 * a + b];
      Rb[3 * a + b] = tgt->c2w[4 * a + b];
    }
    ta[a] = ref->c2w[4 * a + 3];
    tb[a] = tgt->c2w[4 * a + 3];
  }
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) {
      double acc = Rb[i] * Ra[j];
      acc = acc + Rb[3 + i] * Ra[3 + j];
      acc = acc + Rb[6 + i] * Ra[6 + j];
      R[3 * i + j] = (float)acc;
    }
    double acc = Rb[i] * (ta[0] - tb[0]);
    acc = acc + Rb[3 + i] * (ta[1] - tb[1]);
    acc = acc + Rb[6 + i] * (ta[2] - tb[2]);
    t[i] = (float)acc;
  }
}

static cicero_status warp_common(const float* ref_rgb, const float* ref_depth, const cicero_camera* ref_cam,
                                 const cicero_camera* tgt_cams, int n_views, float max_angle_deg,
                                 const cicero_grid* void_grid, const cicero_sampling* void_sampling,
                                 float* const* warped_rgb, float* const* warped_depth, uint8_t* const* hole_mask,
                                 int32_t* const* hole_idx, int32_t* n_holes, void* workspace, size_t ws_bytes,
                                 void* stream) {
  cicero_status st = check_cam(ref_cam);
  if (st != CICERO_OK) return st;
  if (n_views < 1 || n_views > kMaxWarpViews) return fail(CICERO_ERR_INVALID_ARG, "n_views must be 1..32");
  if (!ref_rgb || !ref_depth || !tgt_cams || !warped_rgb || !hole_mask || !hole_idx || !n_holes)
    return fail(CICERO_ERR_INVALID_ARG, "a warp buffer is NULL");
  if (!ws_ok(workspace)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  if (!(max_angle_deg > 0.0f)) return fail(CICERO_ERR_INVALID_ARG, "max_angle_deg must be > 0");
  static thread_local WarpBatch B;
  memset(&B, 0, sizeof B);
  B.n_views = n_views;
  int wt[kMaxWarpViews], ht[kMaxWarpViews];
  VoidTest vt;
  memset(&vt, 0, sizeof vt);
  for (int v = 0; v < n_views; v++) {
    const cicero_camera* tgt = &tgt_cams[v];
    st = check_cam(tgt);
    if (st != CICERO_OK) return st;
    if (!warped_rgb[v] || !hole_mask[v] || !hole_idx[v]) return fail(CICERO_ERR_INVALID_ARG, "a warp output is NULL");
    WarpArgs& a = B.v[v].a;
    a.wr = ref_cam->width;
    a.hr = ref_cam->height;
    a.fr = ref_cam->f;
    a.cxr = ref_cam->cx;
    a.cyr = ref_cam->cy;
    a.wt = tgt->width;
    a.ht = tgt->height;
    a.ft = tgt->f;
    a.cxt = tgt->cx;
    a.cyt = tgt->cy;
    relative_pose(ref_cam, tgt, a.R, a.t);
    a.use_phi = max_angle_deg < 180.0f;
    a.cos_phi = a.use_phi ? (float)cos((double)max_angle_deg * 3.14159265358979323846 / 180.0) : -1.0f;
    B.v[v].wrgb = warped_rgb[v];
    B.v[v].wdepth = warped_depth ? warped_depth[v] : nullptr;
    B.v[v].mask = hole_mask[v];
    B.v[v].hole_idx = hole_idx[v];
    B.v[v].n_holes = n_holes + v;
    wt[v] = tgt->width;
    ht[v] = tgt->height;
    vt.src.cam[v] = view_of(tgt);
  }
  if (ws_bytes < warp_batch_ws_bytes(wt, ht, n_views)) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  carve_warp_ws(B, workspace);
  if (void_grid) {
    if (!void_sampling) return fail(CICERO_ERR_INVALID_ARG, "void_sampling is NULL");
    // the void test needs only the box, the occupancy mask and the sampling; features are unused
    cicero_grid gg = *void_grid;
    if (!gg.density) gg.density = (const void*)16;
    if (!gg.features) gg.features = (const void*)16;
    st = make_geo(&gg, 8, &vt.g);
    if (st != CICERO_OK) return st;
    st = make_samp(void_sampling, &vt.s);
    if (st != CICERO_OK) return st;
    vt.enabled = 1;
    vt.src.kind = 0;
    vt.src.n_views = n_views;
  } else if (void_sampling) {
    st = make_samp(void_sampling, &vt.s);  // unused without a grid, but validated like everywhere else
    if (st != CICERO_OK) return st;
  }
  return run_warp(B, vt, ref_rgb, ref_depth, (cudaStream_t)stream);
}

// -------------------------------------------------------------------------------------------
// batched render: validation, totals and the job table

static size_t al256h(size_t x) { return (x + 255) & ~size_t(255); }

// job descriptors, then the jobs' first rays and first bricks as two contiguous int arrays
size_t batch_table_bytes(int n_jobs) {
  return al256h(sizeof(JobDesc) * (size_t)n_jobs) + al256h(sizeof(int) * 2 * (size_t)n_jobs);
}

// Validates the jobs and fills the totals of the batch; with `table`, also each job's descriptor.
static cicero_status plan_batch(const cicero_job* jobs, int n_jobs, const cicero_options* opt, BatchPlan* b,
                                JobDesc* table) {
  if (!jobs || n_jobs < 1 || n_jobs > kMaxBatchJobs) return fail(CICERO_ERR_INVALID_ARG, "n_jobs must be 1..2048");
  if (!opt || opt->precision != CICERO_MLP_BF16)
    return fail(CICERO_ERR_UNSUPPORTED, "batched rendering runs the BF16 tensor-core MLP only");
  const int brick = opt->brick ? opt->brick : 8;
  if (opt->mlp_groups < 0 || opt->mlp_groups > 4) return fail(CICERO_ERR_INVALID_ARG, "mlp_groups must be 0..4");
  memset(b, 0, sizeof *b);
  b->mlp_groups = opt->mlp_groups;
  unsigned long long R = 0, Q = 0, nb = 0;
  int S = 0;
  // table order: jobs that share MLP weights side by side (in the caller's order otherwise), so the
  // persistent gather loads each set of weights once per CTA range; every job still writes its own
  // outputs, so the order is not visible to the caller
  std::vector<int> order((size_t)n_jobs);
  {
    std::vector<char> taken((size_t)n_jobs, 0);
    int k = 0;
    for (int j = 0; j < n_jobs; j++) {
      if (taken[j]) continue;
      if (!jobs[j].mlp) return fail(CICERO_ERR_INVALID_ARG, "a job field is NULL");
      for (int i = j; i < n_jobs; i++)
        if (!taken[i] && jobs[i].mlp && same_mlp(mlp_ptrs(jobs[i].mlp), mlp_ptrs(jobs[j].mlp))) {
          order[k++] = i;
          taken[i] = 1;
        }
    }
  }
  for (int jt = 0; jt < n_jobs; jt++) {
    const int j = order[jt];
    const cicero_job& J = jobs[j];
    if (!J.grid || !J.mlp || !J.cam || !J.sampling || !J.rgb) return fail(CICERO_ERR_INVALID_ARG, "a job field is NULL");
    GridGeo geo;
    Samp samp;
    cicero_status st = make_geo(J.grid, brick, &geo);
    if (st == CICERO_OK) st = make_samp(J.sampling, &samp);
    if (st == CICERO_OK) st = check_cam(J.cam);
    if (st == CICERO_OK) st = check_mlp(J.mlp, J.grid);
    if (st != CICERO_OK) return st;
    if (jt == 0) {
      b->f16 = J.grid->dtype == CICERO_F16;
      b->C = J.grid->C;
      b->n_freq = J.mlp->n_freq;
    } else if ((J.grid->dtype == CICERO_F16) != b->f16 || J.grid->C != b->C || J.mlp->n_freq != b->n_freq) {
      return fail(CICERO_ERR_UNSUPPORTED, "all jobs of a batch need the same grid dtype, channels and encoding");
    }
    const unsigned long long rj = (unsigned long long)J.cam->width * J.cam->height;
    const unsigned long long nbj = (unsigned long long)geo.nb[0] * geo.nb[1] * geo.nb[2];
    if (table) {
      JobDesc& D = table[jt];
      memset(&D, 0, sizeof D);
      D.geo = geo;
      D.samp = samp;
      D.cam = view_of(J.cam);
      D.mlp = mlp_ptrs(J.mlp);
      D.density = J.grid->density;
      D.rgb = J.rgb;
      D.depth = J.depth;
      D.ray_base = (int)R;
      D.brick_base = (int)nb;
      D.n_rays = (int)rj;
      D.nb = (int)nbj;
      st = encode_brick_map(J.grid, geo, brick_box(geo, elem_bytes(J.grid->dtype)), &D.map);
      if (st != CICERO_OK) return st;
    }
    R += rj;
    Q += rj * (unsigned long long)J.sampling->n_samples;
    nb += nbj;
    S = std::max(S, J.sampling->n_samples);
    if (jt == 0) b->box = brick_box(geo, elem_bytes(J.grid->dtype));
    if (jt == 0) b->plan.geo = geo;
  }
  if (R >= (1ull << 31) || nb >= (1ull << 31)) return fail(CICERO_ERR_UNSUPPORTED, "batch has too many rays or bricks");
  if (opt->max_records > 0 && (unsigned long long)opt->max_records < Q) Q = (unsigned long long)opt->max_records;
  if (Q >= 0xffffffffull) return fail(CICERO_ERR_UNSUPPORTED, "batch records must stay below 2^32 (set max_records)");
  b->n_jobs = n_jobs;
  RenderPlan& p = b->plan;
  p.R = (int)R;
  p.S = S;
  p.Q = (uint32_t)Q;
  p.nb = (int)nb;
  p.max_tiles = (int)((Q + kTile - 1) / kTile) + p.nb;
  p.want_k = false;
  p.want_bwd = false;
  p.want_wg = false;
  p.precision = CICERO_MLP_BF16;
  return CICERO_OK;
}

}  // namespace cicero

struct cicero_batch {
  cicero::BatchPlan plan;
};

namespace cicero {

static size_t batch_ws_bytes(const BatchPlan& b) { return batch_table_bytes(b.n_jobs) + render_ws_bytes(b.plan); }

}  // namespace cicero

using namespace cicero;

extern "C" {

cicero_status cicero_render(const cicero_grid* grid, const cicero_mlp* mlp, const cicero_camera* cam,
                            const cicero_sampling* sampling, const cicero_options* opt, float* rgb, float* depth,
                            float* acc, int32_t* n_steps, void* workspace, size_t ws_bytes, void* stream) {
  cicero_status st = check_cam(cam);
  if (st != CICERO_OK) return st;
  return render_common(grid, mlp, sampling, opt, camera_src(cam), cam->width * cam->height, rgb, depth, acc, n_steps,
                       workspace, ws_bytes, stream);
}

cicero_status cicero_render_rays(const cicero_grid* grid, const cicero_mlp* mlp, const float* ray_o, const float* ray_d,
                                 int n_rays, const cicero_sampling* sampling, const cicero_options* opt, float* rgb,
                                 float* depth, float* acc, int32_t* n_steps, void* workspace, size_t ws_bytes,
                                 void* stream) {
  if (n_rays > 0 && (!ray_o || !ray_d)) return fail(CICERO_ERR_INVALID_ARG, "ray_o/ray_d is NULL");
  RaySrc src;
  memset(&src, 0, sizeof src);
  src.kind = 1;
  src.n_views = 1;
  src.o = ray_o;
  src.d = ray_d;
  src.n_max = n_rays;
  return render_common(grid, mlp, sampling, opt, src, n_rays, rgb, depth, acc, n_steps, workspace, ws_bytes, stream);
}

cicero_status cicero_render_holes(const cicero_grid* grid, const cicero_mlp* mlp, const cicero_camera* cam,
                                  const cicero_sampling* sampling, const cicero_options* opt, const int32_t* hole_idx,
                                  const int32_t* n_holes, int max_holes, float* rgb_inout, float* depth_inout,
                                  void* workspace, size_t ws_bytes, void* stream) {
  cicero_status st = check_cam(cam);
  if (st != CICERO_OK) return st;
  if (!hole_idx || !n_holes) return fail(CICERO_ERR_INVALID_ARG, "hole_idx/n_holes is NULL");
  if (max_holes < 0 || max_holes > cam->width * cam->height) return fail(CICERO_ERR_INVALID_ARG, "max_holes");
  RaySrc src = camera_src(cam);
  src.pix[0] = hole_idx;
  src.n_dev = n_holes;
  src.n_max = max_holes;
  return render_common(grid, mlp, sampling, opt, src, max_holes, rgb_inout, depth_inout, nullptr, nullptr, workspace,
                       ws_bytes, stream);
}

cicero_status cicero_render_holes_batch(const cicero_grid* grid, const cicero_mlp* mlp, const cicero_camera* cams,
                                        int n_views, const cicero_sampling* sampling, const cicero_options* opt,
                                        const int32_t* const* hole_idx, const int32_t* n_holes, int max_rays,
                                        float* const* rgb_inout, float* const* depth_inout, void* workspace,
                                        size_t ws_bytes, void* stream) {
  if (n_views < 1 || n_views > kMaxViews) return fail(CICERO_ERR_INVALID_ARG, "n_views must be 1..32");
  if (!cams || !hole_idx || !n_holes || !rgb_inout) return fail(CICERO_ERR_INVALID_ARG, "a batch argument is NULL");
  RaySrc src;
  memset(&src, 0, sizeof src);
  src.kind = 2;
  src.n_views = n_views;
  src.n_dev = n_holes;
  src.n_max = max_rays;
  OutBufs out;
  memset(&out, 0, sizeof out);
  long long total = 0;
  for (int v = 0; v < n_views; v++) {
    cicero_status st = check_cam(&cams[v]);
    if (st != CICERO_OK) return st;
    if (!hole_idx[v] || !rgb_inout[v]) return fail(CICERO_ERR_INVALID_ARG, "hole_idx/rgb_inout entry is NULL");
    src.cam[v] = view_of(&cams[v]);
    src.pix[v] = hole_idx[v];
    out.rgb[v] = rgb_inout[v];
    out.depth[v] = depth_inout ? depth_inout[v] : nullptr;
    total += (long long)cams[v].width * cams[v].height;
  }
  if (max_rays < 0 || max_rays > total) return fail(CICERO_ERR_INVALID_ARG, "max_rays must be 0..sum of pixels");
  RenderPlan plan;
  cicero_status st = plan_render(grid, mlp, max_rays, sampling, opt, &plan, true);
  if (st != CICERO_OK) return st;
  if (!ws_ok(workspace)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  RenderWs w;
  if (!carve_render_ws(workspace, ws_bytes, plan, &w)) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  if (max_rays == 0) return no_rays(w, stream);
  return run_render(grid, mlp_ptrs(mlp), plan, src, w, out, false, (cudaStream_t)stream);
}

size_t cicero_render_workspace_size(const cicero_grid* grid, int n_rays, const cicero_sampling* sampling,
                                    const cicero_options* opt) {
  RenderPlan plan;
  if (plan_render(grid, nullptr, n_rays, sampling, opt, &plan, false) != CICERO_OK) return 0;
  return render_ws_bytes(plan);
}

size_t cicero_build_rit_workspace_size(const cicero_grid* grid, const cicero_camera* cam,
                                       const cicero_sampling* sampling, const cicero_options* opt) {
  if (!cam) return 0;
  RenderPlan plan;
  if (plan_render(grid, nullptr, cam->width * cam->height, sampling, opt, &plan, false) != CICERO_OK) return 0;
  plan.want_k = true;
  return render_ws_bytes(plan);
}

cicero_status cicero_build_rit(const cicero_grid* grid, const cicero_camera* cam, const cicero_sampling* sampling,
                               const cicero_options* opt, int32_t* brick_offsets, int32_t* samples, int* n_bricks_out,
                               void* workspace, size_t ws_bytes, void* stream) {
  cicero_status st = check_cam(cam);
  if (st != CICERO_OK) return st;
  if (!brick_offsets || !samples) return fail(CICERO_ERR_INVALID_ARG, "brick_offsets/samples is NULL");
  RenderPlan plan;
  const int R = cam->width * cam->height;
  st = plan_render(grid, nullptr, R, sampling, opt, &plan, false);
  if (st != CICERO_OK) return st;
  if ((long long)R * plan.S > 0x7fffffffll)
    return fail(CICERO_ERR_UNSUPPORTED, "the RIT's sample ids (ray x n_samples + slot) must fit in 31 bits");
  plan.want_k = true;
  if (!ws_ok(workspace)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  RenderWs w;
  if (!carve_render_ws(workspace, ws_bytes, plan, &w))
    return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small (the RIT needs the slot array)");
  if (n_bricks_out) *n_bricks_out = plan.nb;
  const RaySrc src = camera_src(cam);
  MlpPtrs none;
  memset(&none, 0, sizeof none);
  st = run_render(grid, none, plan, src, w, single_out(nullptr, nullptr, nullptr, nullptr), true, (cudaStream_t)stream);
  if (st != CICERO_OK) return st;
  return run_rit_export(w, plan.nb, plan.S, brick_offsets, samples, (cudaStream_t)stream);
}

cicero_status cicero_autotune_brick(const cicero_grid* grid, const cicero_mlp* mlp, const cicero_camera* cam,
                                    const cicero_sampling* sampling, cicero_precision precision, float* rgb,
                                    float* depth, void* workspace, size_t ws_bytes, void* stream, int* best_brick,
                                    float* ms) {
  if (!best_brick) return fail(CICERO_ERR_INVALID_ARG, "best_brick is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int cand[3] = {4, 8, 16};
  float best = 1e30f;
  *best_brick = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  for (int i = 0; i < 3; i++) {
    if (ms) ms[i] = -1.0f;
    cicero_options opt = {precision, cand[i], 0};
    const size_t need = cicero_render_workspace_size(grid, cam ? cam->width * cam->height : 0, sampling, &opt);
    if (need == 0 || need > ws_bytes) continue;
    // one untimed render (first use of the kernel), then one timed render
    if (cicero_render(grid, mlp, cam, sampling, &opt, rgb, depth, nullptr, nullptr, workspace, ws_bytes, stream) !=
        CICERO_OK)
      continue;  // this brick size is not supported for this grid
    cudaEventRecord(e0, st);
    cicero_render(grid, mlp, cam, sampling, &opt, rgb, depth, nullptr, nullptr, workspace, ws_bytes, stream);
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    if (ms) ms[i] = t;
    if (t < best) {
      best = t;
      *best_brick = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune render");
  if (!*best_brick) return fail(CICERO_ERR_UNSUPPORTED, "no brick size could render this grid");
  return cicero_workspace_status(workspace, stream);
}

cicero_status cicero_warp(const float* ref_rgb, const float* ref_depth, const cicero_camera* ref_cam,
                          const cicero_camera* tgt_cam, float max_angle_deg, const cicero_grid* void_grid,
                          const cicero_sampling* void_sampling, float* warped_rgb, float* warped_depth,
                          uint8_t* hole_mask, int32_t* hole_idx, int32_t* n_holes, void* workspace, size_t ws_bytes,
                          void* stream) {
  if (!tgt_cam) return fail(CICERO_ERR_INVALID_ARG, "tgt_cam is NULL");
  return warp_common(ref_rgb, ref_depth, ref_cam, tgt_cam, 1, max_angle_deg, void_grid, void_sampling, &warped_rgb,
                     &warped_depth, &hole_mask, &hole_idx, n_holes, workspace, ws_bytes, stream);
}

cicero_status cicero_warp_batch(const float* ref_rgb, const float* ref_depth, const cicero_camera* ref_cam,
                                const cicero_camera* tgt_cams, int n_views, float max_angle_deg,
                                const cicero_grid* void_grid, const cicero_sampling* void_sampling,
                                float* const* warped_rgb, float* const* warped_depth, uint8_t* const* hole_mask,
                                int32_t* const* hole_idx, int32_t* n_holes, void* workspace, size_t ws_bytes,
                                void* stream) {
  return warp_common(ref_rgb, ref_depth, ref_cam, tgt_cams, n_views, max_angle_deg, void_grid, void_sampling,
                     warped_rgb, warped_depth, hole_mask, hole_idx, n_holes, workspace, ws_bytes, stream);
}

size_t cicero_warp_batch_workspace_size(const cicero_camera* tgt_cams, int n_views) {
  if (!tgt_cams || n_views < 1 || n_views > kMaxWarpViews) return 0;
  int wt[kMaxWarpViews], ht[kMaxWarpViews];
  for (int v = 0; v < n_views; v++) {
    if (tgt_cams[v].width < 1 || tgt_cams[v].height < 1) return 0;
    wt[v] = tgt_cams[v].width;
    ht[v] = tgt_cams[v].height;
  }
  return warp_batch_ws_bytes(wt, ht, n_views);
}

size_t cicero_warp_workspace_size(const cicero_camera* tgt_cam) {
  if (!tgt_cam || tgt_cam->width < 1 || tgt_cam->height < 1) return 0;
  return warp_ws_bytes(tgt_cam->width, tgt_cam->height);
}


// The backward's plan: FP32, bricks of 16 up to 16 channels (the tensor-core kernels and the
// CUDA-core weight-gradient kernel read features from global memory, so a brick only groups the
// samples: larger bricks give fewer, fuller 128-sample tiles); bricks of 4 above that, where the
// FP32 recompute stages each brick in shared memory beside its two input buffers.
static cicero_options backward_options(const cicero_grid* grid) {
  cicero_options o;
  memset(&o, 0, sizeof o);
  o.precision = CICERO_MLP_FP32;
  o.brick = (grid && grid->C > 16) ? 4 : 16;
  return o;
}

cicero_status cicero_render_backward(const cicero_grid* grid, const cicero_mlp* mlp, const float* ray_o,
                                     const float* ray_d, int n_rays, const cicero_sampling* sampling,
                                     const float* d_rgb, float* d_density, float* d_features, float* d_mlp,
                                     void* workspace, size_t ws_bytes, void* stream) {
  if (n_rays > 0 && (!ray_o || !ray_d || !d_rgb)) return fail(CICERO_ERR_INVALID_ARG, "ray_o/ray_d/d_rgb is NULL");
  if (!d_density || !d_features) return fail(CICERO_ERR_INVALID_ARG, "d_density/d_features is NULL");
  RenderPlan plan;
  const cicero_options opt = backward_options(grid);
  cicero_status st = plan_render(grid, mlp, n_rays, sampling, &opt, &plan, true);
  if (st != CICERO_OK) return st;
  plan.want_bwd = true;
  if (d_mlp && grid->C <= 16) {
    // the weight gradients on the tensor cores when the workspace holds their staged operands
    plan.want_wg = true;
    if (render_ws_bytes(plan) > ws_bytes) plan.want_wg = false;
  }
  if (!ws_ok(workspace)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  RenderWs w;
  if (!carve_render_ws(workspace, ws_bytes, plan, &w)) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  if (n_rays == 0) return no_rays(w, stream);
  RaySrc src;
  memset(&src, 0, sizeof src);
  src.kind = 1;
  src.n_views = 1;
  src.o = ray_o;
  src.d = ray_d;
  src.n_max = n_rays;
  return run_backward(grid, mlp_ptrs(mlp), plan, src, w, d_rgb, d_density, d_features, d_mlp, (cudaStream_t)stream);
}

size_t cicero_backward_workspace_size(const cicero_grid* grid, int n_rays, const cicero_sampling* sampling) {
  RenderPlan plan;
  const cicero_options opt = backward_options(grid);
  if (plan_render(grid, nullptr, n_rays, sampling, &opt, &plan, false) != CICERO_OK) return 0;
  plan.want_bwd = true;
  return render_ws_bytes(plan);
}

size_t cicero_backward_mlp_workspace_size(const cicero_grid* grid, int n_rays, const cicero_sampling* sampling) {
  RenderPlan plan;
  const cicero_options opt = backward_options(grid);
  if (plan_render(grid, nullptr, n_rays, sampling, &opt, &plan, false) != CICERO_OK) return 0;
  plan.want_bwd = true;
  plan.want_wg = grid->C <= 16;
  return render_ws_bytes(plan);
}

cicero_status cicero_mlp_eval(const cicero_mlp* mlp, const float* x, int M, cicero_precision precision, float* c,
                              void* workspace, size_t ws_bytes, void* stream) {
  cicero_status st = check_mlp(mlp, nullptr);
  if (st != CICERO_OK) return st;
  if (M < 0 || (M > 0 && (!x || !c))) return fail(CICERO_ERR_INVALID_ARG, "x/c is NULL or M < 0");
  if (!ws_ok(workspace) || ws_bytes < 256) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaError_t e = cudaMemsetAsync(workspace, 0, 4, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status word)");
  if (M == 0) return CICERO_OK;
  const MlpPtrs p = mlp_ptrs(mlp);
  if (precision == CICERO_MLP_BF16) return launch_mlp_eval_bf16(p, x, M, c, (uint32_t*)workspace, (cudaStream_t)stream);
  if (precision == CICERO_MLP_FP32) return launch_mlp_eval_f32(p, x, M, c, (cudaStream_t)stream);
  if (precision == CICERO_MLP_FP32_SPLIT) return fail(CICERO_ERR_UNSUPPORTED, "the split-BF16 MLP runs inside the renders only");
  return fail(CICERO_ERR_INVALID_ARG, "precision");
}

size_t cicero_mlp_eval_workspace_size(int M) {
  (void)M;
  return 256;
}

cicero_status cicero_workspace_status(void* workspace, void* stream) {
  if (!workspace) return fail(CICERO_ERR_INVALID_ARG, "workspace is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  uint32_t word = 0;
  e = cudaMemcpy(&word, workspace, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
  const uint32_t zero = 0;
  e = cudaMemcpy(workspace, &zero, 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(clear status)");
  if (word & kErrTimeout) return fail(CICERO_ERR_TIMEOUT, "a kernel's bounded wait ran out");
  if (word & kErrCapacity)
    return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "the rays composited more samples than opt->max_records allows");
  if (word & kErrInternal) return fail(CICERO_ERR_INTERNAL, "a kernel found a broken invariant");
  return CICERO_OK;
}

cicero_status cicero_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  prof_drain();
  for (int i = 0; i < kNumStages; i++) {
    g_prof.ms[i] = 0.0;
    g_prof.n[i] = 0;
  }
  g_prof.on = true;
  return CICERO_OK;
}

cicero_status cicero_profile_end(double* total_ms, long long* count, int n_stages) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = false;
  prof_drain();
  for (int i = 0; i < n_stages && i < kNumStages; i++) {
    if (total_ms) total_ms[i] = g_prof.ms[i];
    if (count) count[i] = g_prof.n[i];
  }
  return CICERO_OK;
}

long long cicero_launch_count(void) { return g_launches.load(); }

const char* cicero_last_error(void) { return g_last_error.c_str(); }

const char* cicero_version(void) { return "cicero-gb300 0.1 (sm_103a)"; }

// The grid of a hash-encoded render: the caller's density grid with C = levels * features.
static cicero_status hash_grid(const cicero_grid* grid, const cicero_hash_grid* h, const cicero_mlp* mlp,
                               cicero_grid* out, HashGeo* hg) {
  if (!grid || !h) return fail(CICERO_ERR_INVALID_ARG, "grid/hash is NULL");
  if (h->levels < 1 || h->levels > kMaxHashLevels) return fail(CICERO_ERR_INVALID_ARG, "hash levels must be 1..16");
  if (h->features != 2) return fail(CICERO_ERR_UNSUPPORTED, "hash encodings with 2 features per level only");
  if (h->log2_size < 1 || h->log2_size > 24) return fail(CICERO_ERR_INVALID_ARG, "hash log2_size must be 1..24");
  if (!h->table) return fail(CICERO_ERR_INVALID_ARG, "hash table is NULL");
  if (h->dtype != CICERO_F16 && h->dtype != CICERO_F32) return fail(CICERO_ERR_INVALID_ARG, "hash dtype");
  if (((uintptr_t)h->table) & (h->dtype == CICERO_F16 ? 3 : 7)) return fail(CICERO_ERR_ALIGNMENT, "hash table alignment");
  *out = *grid;
  out->C = h->levels * h->features;
  memset(hg, 0, sizeof *hg);
  hg->table = h->table;
  hg->levels = h->levels;
  hg->f16 = h->dtype == CICERO_F16;
  hg->mask = (uint32_t)((1ull << h->log2_size) - 1);
  for (int l = 0; l < h->levels; l++) {
    const long long N = h->res[l];
    if (N < 1 || N > (1 << 20)) return fail(CICERO_ERR_INVALID_ARG, "hash level resolution must be 1..2^20");
    hg->res[l] = (int)N;
    if ((N + 1) * (N + 1) * (N + 1) <= (1ll << h->log2_size)) hg->dense |= 1u << l;
  }
  for (int a = 0; a < 3; a++) {
    hg->amin[a] = grid->aabb_min[a];
    hg->inv_ext[a] = 1.0f / (grid->aabb_max[a] - grid->aabb_min[a]);
  }
  if (mlp && mlp->in_dim != out->C + 3 + 6 * mlp->n_freq)
    return fail(CICERO_ERR_INVALID_ARG, "mlp in_dim != 2 levels + 3 + 6 n_freq");
  return CICERO_OK;
}

cicero_status cicero_render_hash(const cicero_grid* grid, const cicero_hash_grid* hash, const cicero_mlp* mlp,
                                 const cicero_camera* cam, const cicero_sampling* sampling, const cicero_options* opt,
                                 float* rgb, float* depth, void* workspace, size_t ws_bytes, void* stream) {
  cicero_status st = check_cam(cam);
  if (st != CICERO_OK) return st;
  if (!opt || opt->precision != CICERO_MLP_BF16)
    return fail(CICERO_ERR_UNSUPPORTED, "hash-encoded rendering runs the BF16 tensor-core MLP only");
  cicero_grid g;
  HashGeo hg;
  if ((st = hash_grid(grid, hash, mlp, &g, &hg)) != CICERO_OK) return st;
  const int R = cam->width * cam->height;
  RenderPlan plan;
  if ((st = plan_render(&g, mlp, R, sampling, opt, &plan, true, false)) != CICERO_OK) return st;
  if (!rgb) return fail(CICERO_ERR_INVALID_ARG, "rgb is NULL");
  if (!ws_ok(workspace)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  RenderWs w;
  if (!carve_render_ws(workspace, ws_bytes, plan, &w)) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  return run_render(&g, mlp_ptrs(mlp), plan, camera_src(cam), w, single_out(rgb, depth, nullptr, nullptr), false,
                    (cudaStream_t)stream, &hg);
}

size_t cicero_render_hash_workspace_size(const cicero_grid* grid, const cicero_hash_grid* hash, int n_rays,
                                         const cicero_sampling* sampling, const cicero_options* opt) {
  cicero_grid g;
  HashGeo hg;
  RenderPlan plan;
  if (hash_grid(grid, hash, nullptr, &g, &hg) != CICERO_OK) return 0;
  if (plan_render(&g, nullptr, n_rays, sampling, opt, &plan, false, false) != CICERO_OK) return 0;
  return render_ws_bytes(plan);
}

cicero_status cicero_upsample_bilinear(const float* src, int w, int h, int channels, float* dst, int W, int H,
                                       void* stream) {
  if (!src || !dst) return fail(CICERO_ERR_INVALID_ARG, "src/dst is NULL");
  if (w < 1 || h < 1 || W < 1 || H < 1 || channels < 1 || channels > 16)
    return fail(CICERO_ERR_INVALID_ARG, "sizes must be >= 1 and channels 1..16");
  if ((long long)W * H > (1ll << 30) || (long long)w * h > (1ll << 30)) return fail(CICERO_ERR_UNSUPPORTED, "image too large");
  return run_upsample(src, w, h, channels, dst, W, H, (cudaStream_t)stream);
}

size_t cicero_batch_table_bytes(int n_jobs) {
  return n_jobs >= 1 && n_jobs <= kMaxBatchJobs ? batch_table_bytes(n_jobs) : 0;
}

size_t cicero_batch_workspace_size(const cicero_job* jobs, int n_jobs, const cicero_options* opt) {
  BatchPlan b;
  if (plan_batch(jobs, n_jobs, opt, &b, nullptr) != CICERO_OK) return 0;
  return batch_ws_bytes(b);
}

cicero_status cicero_batch_create(const cicero_job* jobs, int n_jobs, const cicero_options* opt, void* workspace,
                                  size_t ws_bytes, cicero_batch** out) {
  if (!out) return fail(CICERO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ws_ok(workspace)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  std::vector<JobDesc> table(n_jobs > 0 && n_jobs <= kMaxBatchJobs ? n_jobs : 1);
  BatchPlan b;
  cicero_status st = plan_batch(jobs, n_jobs, opt, &b, table.data());
  if (st != CICERO_OK) return st;
  if (batch_ws_bytes(b) > ws_bytes) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small for the batch");
  char* base = (char*)workspace;
  const size_t tb = batch_table_bytes(n_jobs);
  if (!carve_render_ws(base + tb, ws_bytes - tb, b.plan, &b.ws))
    return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small for the batch");
  const size_t jb = al256h(sizeof(JobDesc) * (size_t)n_jobs);
  std::vector<int> bases(2 * (size_t)n_jobs);
  for (int j = 0; j < n_jobs; j++) {
    bases[j] = table[j].ray_base;
    bases[n_jobs + j] = table[j].brick_base;
  }
  cudaError_t e = cudaMemcpy(base, table.data(), sizeof(JobDesc) * (size_t)n_jobs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + jb, bases.data(), sizeof(int) * bases.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "job table upload");
  b.jobs = (const JobDesc*)base;
  b.bases = (const int*)(base + jb);
  b.workspace = workspace;
  b.ws_bytes = ws_bytes;
  cicero_batch* h = new (std::nothrow) cicero_batch;
  if (!h) return fail(CICERO_ERR_INTERNAL, "out of host memory");
  h->plan = b;
  *out = h;
  return CICERO_OK;
}

cicero_status cicero_batch_launch(const cicero_batch* batch, void* stream) {
  if (!batch) return fail(CICERO_ERR_INVALID_ARG, "batch is NULL");
  return run_render_batch(batch->plan, (cudaStream_t)stream);
}

cicero_status cicero_batch_destroy(cicero_batch* batch) {
  delete batch;
  return CICERO_OK;
}

cicero_status cicero_batch_autotune(const cicero_job* jobs, int n_jobs, const cicero_options* opt, void* workspace,
                                    size_t ws_bytes, void* stream, cicero_options* best_opt, float* ms) {
  if (!best_opt || !opt) return fail(CICERO_ERR_INVALID_ARG, "best/opt is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int bricks[3] = {4, 8, 16};
  float best = 1e30f;
  bool found = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  if (ms)
    for (int i = 0; i < 12; i++) ms[i] = -1.0f;
  for (int i = 0; i < 3 && e == cudaSuccess; i++) {
    for (int g = 1; g <= 4; g++) {
      cicero_options o = *opt;
      o.brick = bricks[i];
      o.mlp_groups = g;
      cicero_batch* b = nullptr;
      if (cicero_batch_create(jobs, n_jobs, &o, workspace, ws_bytes, &b) != CICERO_OK) break;  // brick does not fit
      // one untimed launch (first use of the kernels), then one timed launch
      if (cicero_batch_launch(b, stream) != CICERO_OK) {
        cicero_batch_destroy(b);
        break;  // this brick size is not supported for these grids
      }
      cudaEventRecord(e0, st);
      cicero_batch_launch(b, stream);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      const cicero_status ws_st = cicero_workspace_status((char*)workspace + batch_table_bytes(n_jobs), stream);
      cicero_batch_destroy(b);
      if (e != cudaSuccess) break;
      if (ws_st != CICERO_OK) continue;
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (ms) ms[4 * i + (g - 1)] = t;
      if (t < best) {
        best = t;
        *best_opt = o;
        found = true;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
  if (!found) return fail(CICERO_ERR_UNSUPPORTED, "no brick size could render this batch");
  return CICERO_OK;
}

}  // extern "C"
