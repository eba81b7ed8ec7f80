// C ABI of the skew-Gaussian rasterizer: argument checks, the workspace
// plan, and the kernel launches of each stage (declared in skewraster.h).
#include <atomic>
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "nvtx3/nvToolsExt.h"

using namespace sr;

namespace {
// A named range around each stage call for profilers (NVTX; a no-op unless a
// tool is attached).
struct StageRange {
  explicit StageRange(const char* name) { nvtxRangePushA(name); }
  ~StageRange() { nvtxRangePop(); }
  StageRange(const StageRange&) = delete;
  StageRange& operator=(const StageRange&) = delete;
};
}  // namespace

namespace {
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void sr::count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

namespace {

constexpr int kDefaultSpin = 1 << 20;  // look-back polls (32 ns sleeps) before giving up

int device_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) s = 152;
    cache[dev] = s;
  }
  return cache[dev];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool valid_dtype(int32_t d) { return d == SR_F32 || d == SR_BF16 || d == SR_F16; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

sr_status check_config(const sr_config* c) {
  if (!c) return SR_ERR_INVALID;
  if (c->tile_w != kTile || c->tile_h != kTile) return SR_ERR_UNSUPPORTED;
  if (!(c->alpha_min > 0.0f && c->alpha_min < 1.0f)) return SR_ERR_INVALID;
  if (!(c->alpha_max > c->alpha_min && c->alpha_max < 1.0f)) return SR_ERR_INVALID;
  if (!(c->t_stop >= 0.0f && c->t_stop < 1.0f)) return SR_ERR_INVALID;
  if (!(c->dilation >= 0.0f) || !(c->fov_clamp > 0.0f) || !(c->near_z > 0.0f)) return SR_ERR_INVALID;
  if (c->antialias_comp && !(c->dilation > 0.0f)) return SR_ERR_INVALID;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->bg[k])) return SR_ERR_INVALID;
  for (int px : {c->fwd_pixels_per_thread, c->bwd_pixels_per_thread})
    if (px != 0 && px != 1 && px != 2 && px != 4) return SR_ERR_INVALID;
  if (c->fwd_batch != 0 && c->fwd_batch != 128 && c->fwd_batch != 256 && c->fwd_batch != 512) return SR_ERR_INVALID;
  if (c->bwd_batch != 0 && c->bwd_batch != 128 && c->bwd_batch != 256) return SR_ERR_INVALID;
  if (c->recompute_keys != 0 && c->recompute_keys != 1) return SR_ERR_INVALID;
  if (c->recompute_keys && c->forward_only) return SR_ERR_INVALID;
  if (c->persistent < 0 || c->persistent > 3) return SR_ERR_INVALID;
  if (c->fwd_blocks_per_sm < 0 || c->fwd_blocks_per_sm > 32 || c->bwd_blocks_per_sm < 0 || c->bwd_blocks_per_sm > 32)
    return SR_ERR_INVALID;
  return SR_OK;
}

sr_status check_gaussians(const sr_plan* p, const sr_gaussians* g, bool need_data) {
  if (!g) return SR_ERR_INVALID;
  if (g->n != p->n || g->sh_degree != p->sh_degree) return SR_ERR_INVALID;
  if ((g->two_opacities != 0) != (p->two_opacities != 0)) return SR_ERR_INVALID;
  if ((g->split_dir != nullptr) != (p->has_split != 0)) return SR_ERR_INVALID;
  if (!valid_dtype(g->dt_sh) || !valid_dtype(g->dt_scale) || !valid_dtype(g->dt_skew)) return SR_ERR_INVALID;
  if (need_data && g->n > 0) {
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->skew || !g->sh) return SR_ERR_INVALID;
    if (!aligned16(g->quats)) return SR_ERR_INVALID;  // read as float4
  }
  return SR_OK;
}

sr_status from_cuda(cudaError_t e) { return e == cudaSuccess ? SR_OK : SR_ERR_CUDA; }

}  // namespace

extern "C" {

int32_t sr_abi_version(void) { return SR_ABI_VERSION; }

const char* sr_status_string(sr_status s) {
  switch (s) {
    case SR_OK: return "ok";
    case SR_ERR_INVALID: return "invalid argument";
    case SR_ERR_CAPACITY: return "tile-key capacity exceeded";
    case SR_ERR_CUDA: return "CUDA runtime error";
    case SR_ERR_TIMEOUT: return "bounded device wait gave up";
    case SR_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

sr_status sr_config_default(sr_config* c) {
  if (!c) return SR_ERR_INVALID;
  std::memset(c, 0, sizeof(*c));
  c->tile_w = c->tile_h = kTile;
  c->alpha_min = 1.0f / 255.0f;
  c->alpha_max = 0.99f;
  c->t_stop = 1e-4f;
  c->dilation = 0.3f;
  c->fov_clamp = 1.3f;
  c->near_z = 0.2f;
  c->antialias_comp = 1;
  return SR_OK;
}

// Alg. 3: M_cv = M_gl diag(1,-1,-1,1), W2C = M_cv^-1, K from (W, H, FoV).
sr_status sr_camera_from_gl(const double c2w_gl[16], int32_t width, int32_t height, double fovx, double fovy,
                            sr_camera* out) {
  if (!c2w_gl || !out || width < 1 || height < 1 || width > 32768 || height > 32768) return SR_ERR_INVALID;
  if (!(fovx > 0.0 && fovx < M_PI) || !(fovy > 0.0 && fovy < M_PI)) return SR_ERR_INVALID;
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(c2w_gl[k])) return SR_ERR_INVALID;
  double cv[3][4];
  for (int r = 0; r < 3; ++r) {
    cv[r][0] = c2w_gl[4 * r + 0];
    cv[r][1] = -c2w_gl[4 * r + 1];
    cv[r][2] = -c2w_gl[4 * r + 2];
    cv[r][3] = c2w_gl[4 * r + 3];
  }
  // rigid inverse: rotation transposed, translation -R^T t
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) out->w2c[4 * r + k] = (float)cv[k][r];
    const double tr = -(cv[0][r] * cv[0][3] + cv[1][r] * cv[1][3] + cv[2][r] * cv[2][3]);
    out->w2c[4 * r + 3] = (float)tr;
  }
  const double tx = std::tan(0.5 * fovx), ty = std::tan(0.5 * fovy);
  out->fx = (float)(width / (2.0 * tx));
  out->fy = (float)(height / (2.0 * ty));
  out->cx = (float)(0.5 * width);
  out->cy = (float)(0.5 * height);
  out->tan_fovx = (float)tx;
  out->tan_fovy = (float)ty;
  for (int k = 0; k < 3; ++k) out->campos[k] = (float)cv[k][3];
  out->width = width;
  out->height = height;
  return SR_OK;
}

sr_status sr_plan_init(sr_plan* p, const sr_config* cfg, const sr_gaussians* g, const sr_camera* cams_host,
                       int32_t n_views, int64_t key_capacity) {
  if (!p || !g || !cams_host) return SR_ERR_INVALID;
  sr_status s = check_config(cfg);
  if (s != SR_OK) return s;
  if (g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return SR_ERR_INVALID;
  if (n_views < 1 || n_views > SR_MAX_VIEWS) return SR_ERR_INVALID;
  if (key_capacity < 0 || key_capacity > (int64_t)0xffffffffLL) return SR_ERR_INVALID;
  if (!valid_dtype(g->dt_sh) || !valid_dtype(g->dt_scale) || !valid_dtype(g->dt_skew)) return SR_ERR_INVALID;
  const int64_t m = g->n * (int64_t)n_views;
  if (m >= (int64_t)1 << 31) return SR_ERR_INVALID;
  std::memset(p, 0, sizeof(*p));
  p->abi_version = SR_ABI_VERSION;
  p->n_views = n_views;
  p->n = g->n;
  p->sh_degree = g->sh_degree;
  p->tile_w = cfg->tile_w;
  p->tile_h = cfg->tile_h;
  p->two_opacities = g->two_opacities ? 1 : 0;
  p->has_split = g->split_dir ? 1 : 0;
  p->render_mode = !p->two_opacities ? MODE_PLAIN : (p->has_split ? MODE_SPLIT : MODE_TWO);
  p->forward_only = cfg->forward_only ? 1 : 0;
  p->recompute_keys = cfg->recompute_keys ? 1 : 0;
  p->key_capacity = key_capacity;
  int64_t tb = 0, io = 0, po = 0;
  for (int v = 0; v < n_views; ++v) {
    const int32_t w = cams_host[v].width, h = cams_host[v].height;
    if (w < 1 || h < 1 || w > 32768 || h > 32768) return SR_ERR_INVALID;
    p->width[v] = w;
    p->height[v] = h;
    p->tile_base[v] = tb;
    p->image_offset[v] = io;
    p->pixel_offset[v] = po;
    tb += (int64_t)((w + kTile - 1) / kTile) * ((h + kTile - 1) / kTile);
    io += 3 * (int64_t)w * h;
    po += (int64_t)w * h;
  }
  p->tile_base[n_views] = tb;
  p->image_offset[n_views] = io;
  p->pixel_offset[n_views] = po;
  p->total_tiles = tb;
  p->total_pixels = po;
  if (tb >= (int64_t)1 << 31) return SR_ERR_INVALID;
  int tile_bits = 0;
  while (((int64_t)1 << tile_bits) < tb) ++tile_bits;
  p->sort_bits = 32 + tile_bits;
  p->sort_passes = (tile_bits + 7) / 8;  // the depth bits are sorted once per record, not per key

  const int64_t scan_blocks = (m + kScanBlock - 1) / kScanBlock;
  const int64_t parts = (key_capacity + kSortPart - 1) / kSortPart;
  const int64_t dparts = (m + kSortPart - 1) / kSortPart;
  static_assert(WS_NUM_SLOTS <= (int)(sizeof(p->off) / sizeof(p->off[0])), "plan offset table too small");
  size_t sizes[WS_NUM_SLOTS];
  sizes[WS_STATUS] = sizeof(Status);
  sizes[WS_VIEWS] = sizeof(ViewInfo) * SR_MAX_VIEWS;
  sizes[WS_REC] = sizeof(float4) * 4 * (size_t)m;
  sizes[WS_DEPTH] = sizeof(uint32_t) * (size_t)m;
  sizes[WS_DKEY0] = sizes[WS_DKEY1] = sizeof(uint32_t) * (size_t)m;
  sizes[WS_PERM0] = sizes[WS_PERM1] = sizeof(uint32_t) * (size_t)m;
  sizes[WS_RECT] = sizeof(uint2) * (size_t)m;
  sizes[WS_NTOUCH] = sizeof(uint32_t) * (size_t)m;
  sizes[WS_OFFSETS] = sizeof(uint32_t) * (size_t)m;
  sizes[WS_SCAN_PART] = sizeof(unsigned long long) * (size_t)(scan_blocks + 1);
  sizes[WS_KEYS0] = sizes[WS_KEYS1] = sizeof(uint32_t) * (size_t)key_capacity;
  sizes[WS_VALS0] = sizes[WS_VALS1] = sizeof(uint32_t) * (size_t)key_capacity;
  sizes[WS_HIST] = sizeof(uint32_t) * 2 * kMaxPasses * 256;
  sizes[WS_LOOKBACK_D] = sizeof(unsigned long long) * 256 * kDepthPasses * (size_t)dparts;
  sizes[WS_LOOKBACK] = sizeof(unsigned long long) * 256 * (size_t)p->sort_passes * (size_t)parts;
  sizes[WS_RANGES] = sizeof(uint2) * (size_t)tb;
  sizes[WS_D2] = p->forward_only ? 0 : sizeof(float) * kD2Stride * (size_t)m;
  sizes[WS_FOOT] = sizeof(float4) * 4 * (size_t)m;
  sizes[WS_MASK] = (p->forward_only || p->recompute_keys)
                       ? 0
                       : sizeof(uint32_t) * 256 * (size_t)(key_capacity / 32 + tb + 1);
  sizes[WS_TILE_ORDER] = sizeof(uint32_t) * ((size_t)tb + kOrderWords);
  sizes[WS_SHJAC] = p->forward_only ? 0 : sizeof(float4) * 3 * (size_t)m;
  size_t off = 0;
  for (int k = 0; k < WS_NUM_SLOTS; ++k) {
    p->off[k] = off;
    off += align256(sizes[k] > 0 ? sizes[k] : 1);
  }
  p->ws_bytes = off;
  return SR_OK;
}

size_t sr_workspace_size(const sr_plan* p) { return p ? p->ws_bytes : 0; }

static sr_status check_plan(const sr_plan* p, void* ws) {
  if (!p || p->abi_version != SR_ABI_VERSION || !ws) return SR_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return SR_ERR_INVALID;
  return SR_OK;
}

sr_status sr_preprocess(const sr_plan* p, const sr_gaussians* g, const sr_camera* cams_dev, const sr_config* cfg,
                        void* ws, void* stream) {
  const StageRange range_("sr_preprocess");
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if ((s = check_config(cfg)) != SR_OK) return s;
  if ((s = check_gaussians(p, g, true)) != SR_OK) return s;
  if (!cams_dev) return SR_ERR_INVALID;
  PreArgs a;
  a.g = *g;
  a.cams = cams_dev;
  a.n_views = p->n_views;
  a.cfg = to_dev(*cfg);
  a.mode = p->render_mode;
  a.ws = ws_ptrs(*p, ws);
  a.d2 = p->forward_only ? nullptr : reinterpret_cast<float4*>(a.ws.d2);
  return from_cuda(launch_preprocess_fwd(a, static_cast<cudaStream_t>(stream), device_sms()));
}

static BinArgs bin_args(const sr_plan* p, const sr_config* cfg, void* ws) {
  BinArgs b;
  b.n = p->n;
  b.n_views = p->n_views;
  b.passes = p->sort_passes;
  b.tile_bits = p->sort_bits - 32;
  b.cap = (unsigned long long)p->key_capacity;
  b.total_tiles = p->total_tiles;
  b.spin_limit = cfg->sort_spin_limit > 0 ? cfg->sort_spin_limit : kDefaultSpin;
  b.ws = ws_ptrs(*p, ws);
  return b;
}

// One mapped pinned status buffer per host thread (portable across devices)
// for the key-count readback: a kernel writes it (no copy engine, so the
// readback never queues behind the caller's own large transfers); nullptr
// if mapped pinned memory is unavailable.
static Status* pinned_status() {
  thread_local Status* buf = nullptr;
  thread_local bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(Status), cudaHostAllocPortable | cudaHostAllocMapped) == cudaSuccess)
      buf = static_cast<Status*>(p);
    else
      cudaGetLastError();
  }
  return buf;
}

sr_status sr_bin_sort(const sr_plan* p, const sr_config* cfg, void* ws, int64_t* keys_needed, void* stream) {
  const StageRange range_("sr_bin_sort");
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if ((s = check_config(cfg)) != SR_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const BinArgs b = bin_args(p, cfg, ws);
  cudaError_t e = launch_bin_phase1(b, st, device_sms());
  if (e != cudaSuccess) return SR_ERR_CUDA;
  int run[kMaxPasses];
  for (int k = 0; k < kMaxPasses; ++k) run[k] = 1;
  if (!keys_needed) return from_cuda(launch_bin_phase2(b, run, -1, st));
  // Synchronous form.  With a mapped pinned status buffer a one-block kernel
  // writes the status into host memory while the tile passes (grids sized
  // for the capacity; blocks past the device-side key count leave at once)
  // are already queued behind it, so the GPU does not idle during the host
  // round trip; the call still returns only once the count is known.
  // Without one, the passes wait for the count and are sized by it (trivial
  // passes skipped).
  Status* h = pinned_status();
  Status* h_dev = nullptr;
  if (h && cudaHostGetDevicePointer(reinterpret_cast<void**>(&h_dev), h, 0) != cudaSuccess) {
    cudaGetLastError();
    h_dev = nullptr;
  }
  cudaEvent_t ev = nullptr;
  if (h_dev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) ev = nullptr;
  if (h_dev && ev) {
    const bool ok = launch_status_export(b.ws.status, h_dev, st) == cudaSuccess &&
                    cudaEventRecord(ev, st) == cudaSuccess && launch_bin_phase2(b, run, -1, st) == cudaSuccess &&
                    cudaEventSynchronize(ev) == cudaSuccess;
    cudaEventDestroy(ev);
    if (!ok) return SR_ERR_CUDA;
    *keys_needed = (int64_t)h->keys_needed;
    return h->keys_needed > (unsigned long long)p->key_capacity ? SR_ERR_CAPACITY : SR_OK;
  }
  Status hs;
  e = cudaMemcpyAsync(&hs, b.ws.status, sizeof(Status), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return SR_ERR_CUDA;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return SR_ERR_CUDA;
  *keys_needed = (int64_t)hs.keys_needed;
  if (hs.keys_needed > (unsigned long long)p->key_capacity) return SR_ERR_CAPACITY;
  for (int k = 0; k < p->sort_passes; ++k) run[k] = hs.pass_trivial[kMaxPasses + k] ? 0 : 1;
  return from_cuda(launch_bin_phase2(b, run, (long long)hs.keys_needed, st));
}

static RenderArgs render_args(const sr_plan* p, const sr_config* cfg, void* ws) {
  const Ws w = ws_ptrs(*p, ws);
  RenderArgs r;
  r.rec = w.rec;
  r.vals0 = w.vals[0];
  r.vals1 = w.vals[1];
  r.ranges = w.ranges;
  r.views = w.views;
  r.status = w.status;
  r.n_views = p->n_views;
  r.cfg = to_dev(*cfg);
  r.images = nullptr;
  r.t_final = nullptr;
  r.n_contrib = nullptr;
  r.d_images = nullptr;
  r.d2 = w.d2;
  r.mask = w.mask;
  r.tile_order = w.tile_order;
  r.batch_fwd = cfg->fwd_batch > 0 ? cfg->fwd_batch : 256;
  r.batch_bwd = cfg->bwd_batch > 0 ? cfg->bwd_batch : 128;
  r.px_fwd = cfg->fwd_pixels_per_thread > 0 ? cfg->fwd_pixels_per_thread : 2;
  r.px_bwd = cfg->bwd_pixels_per_thread > 0 ? cfg->bwd_pixels_per_thread : 2;
  r.n_order = (uint32_t)p->total_tiles;
  r.persistent = 0;
  r.work = w.tile_order + p->total_tiles + 2 * kOrderBuckets;  // [0]: forward counter, [1]: backward counter
  r.sms = device_sms();
  r.blocks_fwd = cfg->fwd_blocks_per_sm;
  r.blocks_bwd = cfg->bwd_blocks_per_sm;
  return r;
}

sr_status sr_render_fwd(const sr_plan* p, const sr_config* cfg, void* ws, float* images, float* t_final,
                        uint32_t* n_contrib, void* stream) {
  const StageRange range_("sr_render_fwd");
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if ((s = check_config(cfg)) != SR_OK) return s;
  if (!images || !t_final || !n_contrib) return SR_ERR_INVALID;
  RenderArgs r = render_args(p, cfg, ws);
  r.images = images;
  r.t_final = t_final;
  r.n_contrib = n_contrib;
  r.persistent = (cfg->persistent & 1) ? 1 : 0;
  return from_cuda(launch_render_fwd(r, p->render_mode, p->total_tiles, static_cast<cudaStream_t>(stream)));
}

sr_status sr_render_bwd_composite(const sr_plan* p, const sr_config* cfg, void* ws, const float* d_images,
                                  const float* t_final, const uint32_t* n_contrib, void* stream) {
  const StageRange range_("sr_render_bwd_composite");
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if ((s = check_config(cfg)) != SR_OK) return s;
  if (!d_images || !t_final || !n_contrib) return SR_ERR_INVALID;
  if (p->forward_only) return SR_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Ws w = ws_ptrs(*p, ws);
  // the 2D-gradient records start at zero: the projection zeroed this
  // frame's touched records unless a backward composite has used them since
  // (a device-side test; the clear kernel then zeroes them all)
  cudaError_t e = launch_d2_clear(w.status, reinterpret_cast<float4*>(w.d2),
                                  (int64_t)kD2Stride / 4 * p->n * p->n_views, device_sms(), st);
  if (e != cudaSuccess) return SR_ERR_CUDA;
  RenderArgs r = render_args(p, cfg, ws);
  r.t_final = const_cast<float*>(t_final);
  r.n_contrib = const_cast<uint32_t*>(n_contrib);
  r.d_images = d_images;
  r.persistent = (cfg->persistent & 2) ? 1 : 0;
  r.work += 1;
  return from_cuda(launch_render_bwd(r, p->render_mode, p->total_tiles, st));
}

sr_status sr_render_bwd_project(const sr_plan* p, const sr_gaussians* g, const sr_camera* cams_dev,
                                const sr_config* cfg, void* ws, const sr_grads* out, void* stream) {
  const StageRange range_("sr_render_bwd_project");
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if ((s = check_config(cfg)) != SR_OK) return s;
  if ((s = check_gaussians(p, g, true)) != SR_OK) return s;
  if (!cams_dev || !out) return SR_ERR_INVALID;
  if (p->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->skew || !out->sh))
    return SR_ERR_INVALID;
  if (p->has_split && p->n > 0 && !out->split_dir) return SR_ERR_INVALID;
  if (p->n > 0 && !aligned16(out->quats)) return SR_ERR_INVALID;
  BwdArgs b;
  b.g = *g;
  b.cams = cams_dev;
  b.n_views = p->n_views;
  b.cfg = to_dev(*cfg);
  b.ws = ws_ptrs(*p, ws);
  b.out = *out;
  return from_cuda(launch_preprocess_bwd(b, static_cast<cudaStream_t>(stream), device_sms()));
}

sr_status sr_render_bwd(const sr_plan* p, const sr_gaussians* g, const sr_camera* cams_dev, const sr_config* cfg,
                        void* ws, const float* d_images, const float* t_final, const uint32_t* n_contrib,
                        const sr_grads* out, void* stream) {
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if ((s = check_config(cfg)) != SR_OK) return s;
  if ((s = check_gaussians(p, g, true)) != SR_OK) return s;
  if (!cams_dev || !d_images || !t_final || !n_contrib || !out) return SR_ERR_INVALID;
  if (p->forward_only) return SR_ERR_UNSUPPORTED;
  if (p->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->skew || !out->sh))
    return SR_ERR_INVALID;
  if (p->has_split && p->n > 0 && !out->split_dir) return SR_ERR_INVALID;
  if (p->n > 0 && !aligned16(out->quats)) return SR_ERR_INVALID;
  if (p->recompute_keys) {
    // rebuild the frame's records and sorted key lists (the workspace may
    // have served other frames since the forward); no host round trip
    s = sr_preprocess(p, g, cams_dev, cfg, ws, stream);
    if (s != SR_OK) return s;
    s = sr_bin_sort(p, cfg, ws, nullptr, stream);
    if (s != SR_OK) return s;
  }
  s = sr_render_bwd_composite(p, cfg, ws, d_images, t_final, n_contrib, stream);
  if (s != SR_OK) return s;
  return sr_render_bwd_project(p, g, cams_dev, cfg, ws, out, stream);
}

sr_status sr_selftest_bounded_wait(const sr_plan* p, void* ws, int32_t spin_limit, int64_t* gave_up_partition,
                                   void* stream) {
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if (spin_limit < 1 || p->key_capacity < 2 * kSortPart || p->sort_passes < 1) return SR_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Ws w = ws_ptrs(*p, ws);
  if (launch_selftest_bounded_wait(w, (unsigned long long)p->key_capacity, spin_limit, st) != cudaSuccess)
    return SR_ERR_CUDA;
  Status h;
  if (cudaMemcpyAsync(&h, w.status, sizeof(Status), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaMemsetAsync(&w.status->flags, 0, sizeof(uint32_t), st) != cudaSuccess) return SR_ERR_CUDA;
  if (gave_up_partition) *gave_up_partition = h.timeout_where ? (int64_t)((h.timeout_where - 1) % 1000000) : -1;
  return (h.flags & kStatusTimeout) ? SR_ERR_TIMEOUT : SR_OK;
}

uint64_t sr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

sr_status sr_frame_counters(const sr_plan* p, void* ws, uint64_t* pairs_tested, uint64_t* pairs_blended,
                            void* stream) {
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Status h;
  if (cudaMemcpyAsync(&h, ws_ptrs(*p, ws).status, sizeof(Status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SR_ERR_CUDA;
  if (pairs_tested) *pairs_tested = h.pairs_tested;
  if (pairs_blended) *pairs_blended = h.pairs_blended;
  return SR_OK;
}

size_t sr_loss_scratch_size(const sr_plan* p) {
  if (!p || p->abi_version != SR_ABI_VERSION) return 0;
  return loss_scratch_bytes(p->total_pixels, p->total_tiles);
}

sr_status sr_loss_l1_dssim(const sr_plan* p, void* ws, const float* images, const float* targets, float lambda,
                           float* d_images, float* loss, float* ssim_l1, void* scratch, void* stream) {
  const StageRange range_("sr_loss_l1_dssim");
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  if (!images || !targets || !d_images || !loss || !scratch) return SR_ERR_INVALID;
  if (!(lambda >= 0.0f && lambda <= 1.0f)) return SR_ERR_INVALID;
  if (((uintptr_t)scratch & 255) != 0) return SR_ERR_INVALID;
  if (p->tile_w != kTile || p->tile_h != kTile) return SR_ERR_UNSUPPORTED;
  if (p->total_pixels == 0) return SR_OK;
  const Ws w = ws_ptrs(*p, ws);
  const cudaError_t e = launch_loss(images, targets, lambda, d_images, loss, ssim_l1, scratch, w.views, p->n_views,
                                    p->total_tiles, p->total_pixels, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SR_OK : SR_ERR_CUDA;
}

sr_status sr_adam_step(const sr_adam_group* groups, int32_t n_groups, int64_t step, float beta1, float beta2,
                       float eps, void* stream) {
  const StageRange range_("sr_adam_step");
  if (!groups || n_groups < 1 || n_groups > SR_ADAM_MAX_GROUPS || step < 1) return SR_ERR_INVALID;
  if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f)) return SR_ERR_INVALID;
  for (int i = 0; i < n_groups; ++i) {
    const sr_adam_group& g = groups[i];
    if (g.n < 0 || g.period < 0 || g.split_at < 0) return SR_ERR_INVALID;
    if (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v)) return SR_ERR_INVALID;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e = launch_adam(groups, n_groups, step, beta1, beta2, eps, sms, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SR_OK : SR_ERR_CUDA;
}

sr_status sr_densify_stats(const float* means2d_abs, const float* depth_grad, int64_t n, float* uv_sum,
                           int32_t* seen, float* z_max, void* stream) {
  const StageRange range_("sr_densify_stats");
  if (n < 0) return SR_ERR_INVALID;
  if (n > 0 && (!means2d_abs || !depth_grad || !uv_sum || !seen || !z_max)) return SR_ERR_INVALID;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e =
      launch_densify_stats(means2d_abs, depth_grad, n, uv_sum, seen, z_max, sms, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SR_OK : SR_ERR_CUDA;
}

size_t sr_densify_scratch_size(int64_t n) { return densify_scratch_bytes(n < 0 ? 0 : n); }

sr_status sr_densify(const sr_gaussians* g, const float* uv_sum, const int32_t* seen, const float* z_max,
                     const sr_densify_config* cfg, const sr_scene_arrays* out, uint32_t* src_map, int64_t* counts,
                     void* scratch, void* stream) {
  const StageRange range_("sr_densify");
  if (!g || !cfg || !out || !counts || !scratch) return SR_ERR_INVALID;
  if (g->n < 0 || g->n >= ((int64_t)1 << 30) || g->sh_degree < 0 || g->sh_degree > 3) return SR_ERR_INVALID;
  if (g->dt_sh != SR_F32 || g->dt_scale != SR_F32 || g->dt_skew != SR_F32) return SR_ERR_INVALID;
  if (g->n > 0) {
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->skew || !g->sh) return SR_ERR_INVALID;
    if (!uv_sum || !seen || !z_max) return SR_ERR_INVALID;
    if (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->skew || !out->sh)
      return SR_ERR_INVALID;
    if ((g->split_dir != nullptr) != (out->split_dir != nullptr)) return SR_ERR_INVALID;
    if (!aligned16(g->quats) || !aligned16(out->quats)) return SR_ERR_INVALID;
  }
  DensifyArgs a;
  a.means = static_cast<const float*>(g->means);
  a.log_scales = static_cast<const float*>(g->log_scales);
  a.quats = static_cast<const float*>(g->quats);
  a.opacity = static_cast<const float*>(g->opacity_logits);
  a.skew = static_cast<const float*>(g->skew);
  a.split_dir = static_cast<const float*>(g->split_dir);
  a.sh = static_cast<const float*>(g->sh);
  a.n = g->n;
  a.two = g->two_opacities ? 1 : 0;
  a.k3 = 3 * (g->sh_degree + 1) * (g->sh_degree + 1);
  a.sh_vec4 = (a.k3 % 4 == 0 && aligned16(g->sh) && aligned16(out->sh)) ? 1 : 0;
  a.uv_sum = uv_sum;
  a.seen = seen;
  a.z_max = z_max;
  a.grad_uv = cfg->grad_uv;
  a.grad_z = cfg->grad_z;
  a.log_scale_split = cfg->log_scale_split;
  a.logit_prune = cfg->logit_prune;
  a.o_means = out->means;
  a.o_log_scales = out->log_scales;
  a.o_quats = out->quats;
  a.o_opacity = out->opacity_logits;
  a.o_skew = out->skew;
  a.o_split_dir = out->split_dir;
  a.o_sh = out->sh;
  a.src_map = src_map;
  a.counts = counts;
  a.block_sums = static_cast<uint32_t*>(scratch);
  return from_cuda(launch_densify(a, static_cast<cudaStream_t>(stream)));
}

sr_status sr_densify_remap(const float* in, int32_t width, const uint32_t* src_map, const int64_t* counts,
                           int64_t cap, float* out, void* stream) {
  const StageRange range_("sr_densify_remap");
  if (width < 0 || cap < 0) return SR_ERR_INVALID;
  if (width > 0 && cap > 0 && (!in || !src_map || !counts || !out)) return SR_ERR_INVALID;
  return from_cuda(launch_densify_remap(in, width, src_map, counts, cap, out, device_sms(),
                                        static_cast<cudaStream_t>(stream)));
}

sr_status sr_read_status(const sr_plan* p, void* ws, int64_t* keys_needed, void* stream) {
  sr_status s = check_plan(p, ws);
  if (s != SR_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Ws w = ws_ptrs(*p, ws);
  Status h;
  if (cudaMemcpyAsync(&h, w.status, sizeof(Status), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SR_ERR_CUDA;
  if (keys_needed) *keys_needed = (int64_t)h.keys_needed;
  if (cudaMemsetAsync(&w.status->flags, 0, sizeof(uint32_t), st) != cudaSuccess) return SR_ERR_CUDA;
  if (h.flags & kStatusCapacity) return SR_ERR_CAPACITY;
  if (h.flags & kStatusTimeout) return SR_ERR_TIMEOUT;
  return SR_OK;
}

}  // extern "C"
