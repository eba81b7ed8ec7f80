// Argument blocks and launchers of the rasterizer's kernels (one per stage).
#pragma once

#include "common.cuh"

namespace sr {

struct PreArgs {        // preprocess forward
  sr_gaussians g;
  const sr_camera* cams;
  int n_views;
  CfgDev cfg;
  int mode;             // RenderMode
  Ws ws;
  float4* d2;           // 2D-gradient records to zero for touched records (null: forward-only plan)
};

struct BwdArgs {        // preprocess backward
  sr_gaussians g;
  const sr_camera* cams;
  int n_views;
  CfgDev cfg;
  Ws ws;
  sr_grads out;
};

struct BinArgs {        // binning and sort
  int64_t n;
  int n_views;
  int passes;
  int tile_bits;        // significant bits of the global tile ids (passes = ceil(tile_bits / 8))
  unsigned long long cap;
  int64_t total_tiles;
  int spin_limit;
  Ws ws;
};

struct RenderArgs {     // forward and backward composite
  const float4* rec;
  const uint32_t* vals0;
  const uint32_t* vals1;
  const uint2* ranges;
  const uint32_t* tile_order;  // blockIdx.x -> tile (longest key lists first)
  const ViewInfo* views;
  Status* status;
  int n_views;
  CfgDev cfg;
  float* images;
  float* t_final;
  uint32_t* n_contrib;
  const float* d_images;
  float* d2;
  uint32_t* mask;       // per-pixel blend masks, or null (forward-only or recompute-keys plan;
                        // the backward then replays with the alpha gate)
  int batch_fwd;        // records staged per batch (128, 256, 512)
  int batch_bwd;        // (128, 256)
  int px_fwd;           // pixels per thread (1, 2, 4)
  int px_bwd;
  uint32_t n_order;     // tiles in tile_order
  int persistent;       // 1: blocks take tiles from *work until none is left
  uint32_t* work;       // tile counter of a persistent launch (zeroed before it)
  int sms;
  int blocks_fwd;       // cap on resident blocks per SM (0: as many as fit)
  int blocks_bwd;
};

struct DensifyArgs {     // densification
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity;
  const float* skew;
  const float* split_dir;  // or null
  const float* sh;
  int64_t n;
  int two;                 // two opacity logits per Gaussian
  int k3;                  // SH floats per Gaussian
  int sh_vec4;             // SH rows 16-byte aligned: float4 copies
  const float* uv_sum;
  const int32_t* seen;
  const float* z_max;
  float grad_uv, grad_z, log_scale_split, logit_prune;
  float* o_means;
  float* o_log_scales;
  float* o_quats;
  float* o_opacity;
  float* o_skew;
  float* o_split_dir;
  float* o_sh;
  uint32_t* src_map;       // or null
  int64_t* counts;         // [4] kept, cloned, split, total
  uint32_t* block_sums;    // scratch [blocks][4]
};

// Launch with programmatic stream serialisation: the kernel (which calls
// pdl_entry first) may be scheduled during its predecessor's last wave.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The same launch without the programmatic attribute, for kernels that do
// not wait on their predecessor with griddepcontrol.wait.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_preprocess_fwd(const PreArgs& a, cudaStream_t st, int sms);
cudaError_t launch_preprocess_bwd(const BwdArgs& a, cudaStream_t st, int sms);
cudaError_t launch_bin_phase1(const BinArgs& a, cudaStream_t st, int sms);
cudaError_t launch_status_export(const Status* src, Status* dst_mapped, cudaStream_t st);
cudaError_t launch_bin_phase2(const BinArgs& a, const int* run, long long keys_known, cudaStream_t st);
cudaError_t launch_selftest_bounded_wait(const Ws& ws, unsigned long long cap, int spin_limit, cudaStream_t st);
cudaError_t launch_render_fwd(const RenderArgs& a, int mode, int64_t total_tiles, cudaStream_t st);
cudaError_t launch_render_bwd(const RenderArgs& a, int mode, int64_t total_tiles, cudaStream_t st);
cudaError_t launch_d2_clear(Status* status, float4* d2, int64_t n4, int sms, cudaStream_t st);
size_t loss_scratch_bytes(int64_t total_pixels, int64_t total_tiles);
cudaError_t launch_loss(const float* images, const float* targets, float lambda, float* d_images, float* loss,
                        float* ssim_l1, void* scratch, const ViewInfo* views, int n_views, int64_t total_tiles,
                        int64_t total_pixels, cudaStream_t st);
cudaError_t launch_adam(const sr_adam_group* groups, int n_groups, int64_t step, float b1, float b2, float eps,
                        int sms, cudaStream_t st);
size_t densify_scratch_bytes(int64_t n);
cudaError_t launch_densify(const DensifyArgs& a, cudaStream_t st);
cudaError_t launch_densify_remap(const float* in, int width, const uint32_t* src_map, const int64_t* counts,
                                 int64_t cap, float* out, int sms, cudaStream_t st);
cudaError_t launch_densify_stats(const float* g_uv, const float* g_z, int64_t n, float* uv_sum, int32_t* seen,
                                 float* z_max, int sms, cudaStream_t st);

}  // namespace sr
