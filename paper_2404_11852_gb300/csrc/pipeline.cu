// SpaRW over a camera trajectory (Sec. III-C "Reference Frame Rendering"): reference poses
// extrapolated from the latest target poses (Eq. 5-6), and reference frames rendered on a second
// stream while the targets of the previous window are warped and hole-rendered (host scheduling
// of the library's own calls; no kernels of its own).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/cicero.h"
#include "internal.h"

namespace cicero {

namespace {

struct Quat {
  double w, x, y, z;
};

Quat quat_of(const double R[9]) {  // rotation matrix (row-major) -> unit quaternion
  Quat q;
  const double tr = R[0] + R[4] + R[8];
  if (tr > 0.0) {
    const double s = 2.0 * sqrt(tr + 1.0);
    q = {0.25 * s, (R[7] - R[5]) / s, (R[2] - R[6]) / s, (R[3] - R[1]) / s};
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[0] - R[4] - R[8]);
    q = {(R[7] - R[5]) / s, 0.25 * s, (R[1] + R[3]) / s, (R[2] + R[6]) / s};
  } else if (R[4] > R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[4] - R[0] - R[8]);
    q = {(R[2] - R[6]) / s, (R[1] + R[3]) / s, 0.25 * s, (R[5] + R[7]) / s};
  } else {
    const double s = 2.0 * sqrt(1.0 + R[8] - R[0] - R[4]);
    q = {(R[3] - R[1]) / s, (R[2] + R[6]) / s, (R[5] + R[7]) / s, 0.25 * s};
  }
  const double n = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  return {q.w / n, q.x / n, q.y / n, q.z / n};
}

Quat mul(const Quat& a, const Quat& b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}

void mat_of(const Quat& q, double R[9]) {
  const double w = q.w, x = q.x, y = q.y, z = q.z;
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

}  // namespace

// Device buffers of a pipeline, carved from its workspace (all 256-byte aligned).
struct PipeLayout {
  size_t ref_rgb[2], ref_depth[2], mask, hidx, nh, ws_ref[2], ws_warp, ws_holes, total;
  size_t ws_ref_bytes, ws_warp_bytes, ws_holes_bytes;
};

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

static cicero_status pipe_layout(const cicero_grid* grid, const cicero_camera* cam, const cicero_sampling* samp,
                                 const cicero_options* opt, int window, long long hole_records, PipeLayout* L) {
  if (!grid || !cam || !samp || !opt) return fail(CICERO_ERR_INVALID_ARG, "a pipeline argument is NULL");
  if (window < 1 || window > kMaxWarpViews) return fail(CICERO_ERR_INVALID_ARG, "window must be 1..32");
  if (hole_records < 0) return fail(CICERO_ERR_INVALID_ARG, "hole_records must be >= 0");
  const size_t R = (size_t)cam->width * cam->height;
  L->ws_ref_bytes = cicero_render_workspace_size(grid, (int)R, samp, opt);
  cicero_camera tc[kMaxWarpViews];
  for (int v = 0; v < window; v++) tc[v] = *cam;
  L->ws_warp_bytes = cicero_warp_batch_workspace_size(tc, window);
  cicero_options oh = *opt;
  oh.max_records = hole_records;
  if ((long long)R * window > 0x7fffffffll) return fail(CICERO_ERR_UNSUPPORTED, "window x pixels must fit 31 bits");
  L->ws_holes_bytes = cicero_render_workspace_size(grid, (int)(R * window), samp, &oh);
  if (!L->ws_ref_bytes || !L->ws_warp_bytes || !L->ws_holes_bytes) return fail(CICERO_ERR_INVALID_ARG, cicero_last_error());
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t r = o;
    o += up256(n);
    return r;
  };
  for (int b = 0; b < 2; b++) {
    L->ref_rgb[b] = take(12 * R);
    L->ref_depth[b] = take(4 * R);
  }
  L->mask = take(R * window);
  L->hidx = take(4 * R * window);
  L->nh = take(4 * (size_t)window);
  for (int b = 0; b < 2; b++) L->ws_ref[b] = take(L->ws_ref_bytes);
  L->ws_warp = take(L->ws_warp_bytes);
  L->ws_holes = take(L->ws_holes_bytes);
  L->total = o;
  return CICERO_OK;
}

}  // namespace cicero

struct cicero_pipeline {
  cicero_grid grid;
  cicero_mlp mlp;
  cicero_sampling samp;
  cicero_options opt_ref, opt_holes;
  cicero_camera cam;
  int window;
  float max_angle;
  char* ws;
  cicero::PipeLayout L;
  cudaEvent_t ref_done[2], tgt_done[2];
};

using namespace cicero;

extern "C" {

cicero_status cicero_extrapolate_pose(const cicero_camera* prev, const cicero_camera* cur, float lead,
                                      cicero_camera* out) {
  if (!prev || !cur || !out) return fail(CICERO_ERR_INVALID_ARG, "a camera is NULL");
  if (!isfinite(lead)) return fail(CICERO_ERR_INVALID_ARG, "lead must be finite");
  double Rp[9], Rc[9], pp[3], pc[3];
  for (int a = 0; a < 3; a++) {
    for (int b = 0; b < 3; b++) {
      Rp[3 * a + b] = prev->c2w[4 * a + b];
      Rc[3 * a + b] = cur->c2w[4 * a + b];
    }
    pp[a] = prev->c2w[4 * a + 3];
    pc[a] = cur->c2w[4 * a + 3];
  }
  for (int i = 0; i < 12; i++)
    if (!isfinite(prev->c2w[i]) || !isfinite(cur->c2w[i])) return fail(CICERO_ERR_INVALID_ARG, "pose not finite");
  // angular velocity: the rotation from prev to cur, d = q_cur q_prev^-1 (shortest arc)
  const Quat qp = quat_of(Rp), qc = quat_of(Rc);
  Quat d = mul(qc, {qp.w, -qp.x, -qp.y, -qp.z});
  if (d.w < 0.0) d = {-d.w, -d.x, -d.y, -d.z};
  const double vn = sqrt(d.x * d.x + d.y * d.y + d.z * d.z);
  Quat s = {1.0, 0.0, 0.0, 0.0};
  if (vn > 0.0) {
    const double half = 0.5 * (double)lead * 2.0 * atan2(vn, d.w);  // the angle, lead times, halved
    const double k = sin(half) / vn;
    s = {cos(half), d.x * k, d.y * k, d.z * k};
  }
  double R[9];
  mat_of(mul(s, qc), R);
  cicero_camera o = *cur;  // intrinsics of the latest frame
  for (int a = 0; a < 3; a++) {
    for (int b = 0; b < 3; b++) o.c2w[4 * a + b] = (float)R[3 * a + b];
    o.c2w[4 * a + 3] = (float)(pc[a] + (double)lead * (pc[a] - pp[a]));  // Eq. 5-6
  }
  *out = o;
  return CICERO_OK;
}

cicero_status cicero_reference_poses(const cicero_camera* targets, int n_frames, int window, cicero_lead lead,
                                     cicero_camera* refs) {
  if (!targets || !refs) return fail(CICERO_ERR_INVALID_ARG, "targets/refs is NULL");
  if (n_frames < 1 || window < 1) return fail(CICERO_ERR_INVALID_ARG, "n_frames and window must be >= 1");
  if (lead != CICERO_LEAD_CENTRED && lead != CICERO_LEAD_PAPER) return fail(CICERO_ERR_INVALID_ARG, "unknown lead");
  const int n_win = (n_frames + window - 1) / window;
  refs[0] = targets[0];
  for (int w = 1; w < n_win; w++) {
    // the first frame of window w - 1 (frame 1 for the first window: two poses are needed)
    const int s = (w - 1) * window > 1 ? (w - 1) * window : 1;
    const double frames = lead == CICERO_LEAD_CENTRED ? (double)w * window + window / 2.0 - s : window / 2.0;
    const cicero_status st = cicero_extrapolate_pose(&targets[s - 1], &targets[s], (float)frames, &refs[w]);
    if (st != CICERO_OK) return st;
  }
  return CICERO_OK;
}

size_t cicero_pipeline_workspace_size(const cicero_grid* grid, const cicero_camera* cam,
                                      const cicero_sampling* sampling, const cicero_options* opt, int window,
                                      long long hole_records) {
  PipeLayout L;
  return pipe_layout(grid, cam, sampling, opt, window, hole_records, &L) == CICERO_OK ? L.total : 0;
}

cicero_status cicero_pipeline_create(const cicero_grid* grid, const cicero_mlp* mlp, const cicero_camera* cam,
                                     const cicero_sampling* sampling, const cicero_options* opt, int window,
                                     long long hole_records, float max_angle_deg, void* workspace, size_t ws_bytes,
                                     cicero_pipeline** out) {
  if (!out || !mlp) return fail(CICERO_ERR_INVALID_ARG, "out/mlp is NULL");
  *out = nullptr;
  PipeLayout L;
  cicero_status st = pipe_layout(grid, cam, sampling, opt, window, hole_records, &L);
  if (st != CICERO_OK) return st;
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(CICERO_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (L.total > ws_bytes) return fail(CICERO_ERR_WORKSPACE_TOO_SMALL, "workspace too small for the pipeline");
  cicero_pipeline* p = new (std::nothrow) cicero_pipeline;
  if (!p) return fail(CICERO_ERR_INTERNAL, "out of host memory");
  p->grid = *grid;
  p->mlp = *mlp;
  p->samp = *sampling;
  p->opt_ref = *opt;
  p->opt_holes = *opt;
  p->opt_holes.max_records = hole_records;
  p->cam = *cam;
  p->window = window;
  p->max_angle = max_angle_deg;
  p->ws = (char*)workspace;
  p->L = L;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; b++) {
    e = cudaEventCreateWithFlags(&p->ref_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->tgt_done[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaEventCreate");
  }
  *out = p;
  return CICERO_OK;
}

cicero_status cicero_pipeline_run(cicero_pipeline* p, const cicero_camera* targets, int n_frames, cicero_lead lead,
                                  float* const* rgb, float* const* depth, void* stream_tgt, void* stream_ref) {
  if (!p || !targets || !rgb) return fail(CICERO_ERR_INVALID_ARG, "a pipeline argument is NULL");
  if (n_frames < 1) return fail(CICERO_ERR_INVALID_ARG, "n_frames must be >= 1");
  const int N = p->window, n_win = (n_frames + N - 1) / N;
  std::vector<cicero_camera> ref_poses;
  try {
    ref_poses.resize((size_t)n_win);
  } catch (...) {
    return fail(CICERO_ERR_INTERNAL, "out of host memory");
  }
  const cicero_camera* refs = ref_poses.data();
  if (cicero_status s0 = cicero_reference_poses(targets, n_frames, N, lead, ref_poses.data()); s0 != CICERO_OK)
    return s0;
  for (int i = 0; i < n_frames; i++)
    if (targets[i].width != p->cam.width || targets[i].height != p->cam.height || !rgb[i])
      return fail(CICERO_ERR_INVALID_ARG, "every target frame must have the pipeline's size and an rgb buffer");
  const PipeLayout& L = p->L;
  cudaStream_t st = (cudaStream_t)stream_tgt, sr = (cudaStream_t)stream_ref;
  char* ws = p->ws;
  auto ref_rgb = [&](int b) { return (float*)(ws + L.ref_rgb[b]); };
  auto ref_depth = [&](int b) { return (float*)(ws + L.ref_depth[b]); };
  auto render_ref = [&](int w) -> cicero_status {
    const int b = w & 1;
    cicero_status s = cicero_render(&p->grid, &p->mlp, &refs[w], &p->samp, &p->opt_ref, ref_rgb(b), ref_depth(b),
                                    nullptr, nullptr, ws + L.ws_ref[b], L.ws_ref_bytes, sr);
    if (s != CICERO_OK) return s;
    cudaError_t e = cudaEventRecord(p->ref_done[b], sr);
    return e == cudaSuccess ? CICERO_OK : cuda_fail(e, "cudaEventRecord");
  };
  const size_t R = (size_t)p->cam.width * p->cam.height;
  // the reference buffers may still be read by the previous run's last windows
  for (int b = 0; b < 2; b++)
    if (cudaStreamWaitEvent(sr, p->tgt_done[b], 0) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "cudaStreamWaitEvent");
  cicero_status s = render_ref(0);
  if (s != CICERO_OK) return s;
  for (int w = 0; w < n_win; w++) {
    const int b = w & 1;
    if (w + 1 < n_win) {
      // reference w + 1 on the reference stream, once window w - 1 is done with its buffer
      if (w >= 1 && cudaStreamWaitEvent(sr, p->tgt_done[(w + 1) & 1], 0) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "cudaStreamWaitEvent");
      if ((s = render_ref(w + 1)) != CICERO_OK) return s;
    }
    // window w on the target stream, from reference w
    if (cudaStreamWaitEvent(st, p->ref_done[b], 0) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "cudaStreamWaitEvent");
    const int f0 = w * N, k = n_frames - f0 < N ? n_frames - f0 : N;
    float* wr[kMaxWarpViews];
    float* wd[kMaxWarpViews];
    uint8_t* wm[kMaxWarpViews];
    int32_t* wh[kMaxWarpViews];
    const int32_t* whc[kMaxWarpViews];
    for (int v = 0; v < k; v++) {
      wr[v] = rgb[f0 + v];
      wd[v] = depth ? depth[f0 + v] : nullptr;
      wm[v] = (uint8_t*)(ws + L.mask) + R * v;
      wh[v] = (int32_t*)(ws + L.hidx) + R * v;
      whc[v] = wh[v];
    }
    int32_t* nh = (int32_t*)(ws + L.nh);
    // No separate void test: a void hole's march in the hole render finds no occupied slot and
    // writes the background with depth +inf, the result the test would give, so the test would only
    // repeat the start of every real hole's march.
    s = cicero_warp_batch(ref_rgb(b), ref_depth(b), &refs[w], &targets[f0], k, p->max_angle, nullptr, nullptr, wr,
                          depth ? wd : nullptr, wm, wh, nh, ws + L.ws_warp, L.ws_warp_bytes, st);
    if (s != CICERO_OK) return s;
    s = cicero_render_holes_batch(&p->grid, &p->mlp, &targets[f0], k, &p->samp, &p->opt_holes, whc, nh,
                                  (int)(R * k), wr, depth ? wd : nullptr, ws + L.ws_holes, L.ws_holes_bytes, st);
    if (s != CICERO_OK) return s;
    if (cudaEventRecord(p->tgt_done[b], st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventRecord");
  }
  return CICERO_OK;
}

cicero_status cicero_pipeline_status(const cicero_pipeline* p, void* stream) {
  if (!p) return fail(CICERO_ERR_INVALID_ARG, "pipeline is NULL");
  for (int b = 0; b < 2; b++) {
    cicero_status s = cicero_workspace_status(p->ws + p->L.ws_ref[b], stream);
    if (s != CICERO_OK) return s;
  }
  return cicero_workspace_status(p->ws + p->L.ws_holes, stream);
}

cicero_status cicero_pipeline_destroy(cicero_pipeline* p) {
  if (!p) return CICERO_OK;
  for (int b = 0; b < 2; b++) {
    cudaEventDestroy(p->ref_done[b]);
    cudaEventDestroy(p->tgt_done[b]);
  }
  delete p;
  return CICERO_OK;
}

}  // extern "C"
