// extern "C" entry points of libprtgs: argument checks, workspace checks, dispatch.
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

using namespace prtgs;

namespace prtgs {
std::atomic<unsigned long long>& launch_counter() {
  static std::atomic<unsigned long long> c{0};
  return c;
}
}  // namespace prtgs

namespace {

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

int check_ws(void* ws, size_t have, size_t need) {
  if (need == 0) return PRTGS_OK;
  if (!ws || have < need || !aligned256(ws)) return PRTGS_ERR_WORKSPACE;
  return PRTGS_OK;
}

int check_gaussians(const prtgs_gaussians* g) {
  if (!g || g->n < 0) return PRTGS_ERR_INVALID_ARG;
  if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacity)) return PRTGS_ERR_INVALID_ARG;
  if (g->n >= (int64_t(1) << 31)) return PRTGS_ERR_UNSUPPORTED;
  return PRTGS_OK;
}

// SH orders 1-6 (4-49 coefficients).
static int check_order_high(int32_t order) { return (order >= 1 && order <= 6) ? PRTGS_OK : PRTGS_ERR_UNSUPPORTED; }

int finish(int rc) {
  if (rc != PRTGS_OK) return rc;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return PRTGS_ERR_CUDA;
  }
  return PRTGS_OK;
}

}  // namespace

extern "C" {

int prtgs_version(void) { return 10000; }

unsigned long long prtgs_launch_count(void) { return launch_counter().load(std::memory_order_relaxed); }

const char* prtgs_strerror(int code) {
  switch (code) {
    case PRTGS_OK: return "ok";
    case PRTGS_ERR_INVALID_ARG: return "invalid argument";
    case PRTGS_ERR_SHAPE: return "inconsistent shapes";
    case PRTGS_ERR_UNSUPPORTED: return "unsupported configuration";
    case PRTGS_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case PRTGS_ERR_CUDA: return "CUDA error";
    default: return "unknown error";
  }
}

int prtgs_read_status(int32_t* status, prtgs_stream_t stream) {
  if (!status) return PRTGS_ERR_INVALID_ARG;
  int32_t h = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PRTGS_ERR_CUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return PRTGS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PRTGS_ERR_CUDA;
  return h;
}

// ---- BVH ----
size_t prtgs_bvh_bytes(int64_t n, int32_t n_scenes) {
  if (n < 0 || n_scenes < 1) return 0;
  return bvh_bytes(n, n_scenes);
}

int prtgs_bvh_init(void* buffer, size_t bytes, int64_t n, int32_t n_scenes, const int64_t* scene_offsets,
                   prtgs_bvh* out) {
  if (!out || n < 0 || n_scenes < 1 || !scene_offsets) return PRTGS_ERR_INVALID_ARG;
  if (n_scenes > kMaxScenes) return PRTGS_ERR_UNSUPPORTED;
  if (n > 0 && (!buffer || !aligned256(buffer) || bytes < bvh_bytes(n, n_scenes))) return PRTGS_ERR_WORKSPACE;
  return bvh_layout(buffer, n, n_scenes, scene_offsets, out);
}

size_t prtgs_build_bvh_workspace_size(int64_t n, int32_t n_scenes) {
  if (n < 0 || n_scenes < 1) return 0;
  return build_bvh_workspace(n, n_scenes);
}

int prtgs_build_bvh(const prtgs_gaussians* g, prtgs_bvh* bvh, int32_t* status, void* workspace,
                    size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (!bvh || bvh->n != g->n || bvh->n_scenes < 1 || !bvh->scene_offsets) return PRTGS_ERR_SHAPE;
  if (g->n > 0 && !g->normals) return PRTGS_ERR_INVALID_ARG;
  if (g->n == 0) return PRTGS_OK;
  rc = check_ws(workspace, workspace_bytes, build_bvh_workspace(g->n, bvh->n_scenes));
  if (rc) return rc;
  return finish(build_bvh(g, bvh, status, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"

namespace prtgs {
int transfer_check_dirs(int S);
}

extern "C" {

// ---- transfer ----

size_t prtgs_transfer_workspace_size(int64_t n, int64_t n_glossy, const prtgs_transfer_params* p) {
  if (!p || n < 0 || n_glossy < 0) return 0;
  return transfer_workspace(n, n_glossy, p);
}

int prtgs_precompute_transfer(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                              float* P, float* T, int32_t* idx, float* M, int64_t n_glossy, int32_t* status,
                              void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (!p || !bvh) return PRTGS_ERR_INVALID_ARG;
  if ((rc = check_order_high(p->sh_order))) return rc;
  if (prtgs::transfer_check_dirs(p->n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if ((p->flags & PRTGS_GLOSSY) && !prtgs::glossy_fits(p->n_dirs, p->sh_order)) return PRTGS_ERR_UNSUPPORTED;
  if (!p->dirs || !(p->t_min >= 0.f) || !(p->same_surface_t >= 0.f)) return PRTGS_ERR_INVALID_ARG;
  if (p->n_bounces < 0 || p->n_bounces > 64) return PRTGS_ERR_INVALID_ARG;
  if (p->walk < 0 || p->walk > 1 || p->packet_dirs < 0 || p->packet_dirs > 64) return PRTGS_ERR_INVALID_ARG;
  if (bvh->n != g->n) return PRTGS_ERR_SHAPE;
  if (g->n == 0) return PRTGS_OK;
  if (!P || !g->normals) return PRTGS_ERR_INVALID_ARG;
  if ((p->flags & PRTGS_BOUNCE) && (!T || !idx || !g->albedo)) return PRTGS_ERR_INVALID_ARG;
  if (p->flags & PRTGS_GLOSSY) {
    if (n_glossy < 0 || n_glossy > g->n) return PRTGS_ERR_SHAPE;
    if (n_glossy > 0 && (!M || !g->glossy_mask || !g->roughness || !g->metallic)) return PRTGS_ERR_INVALID_ARG;
  }
  rc = check_ws(workspace, workspace_bytes, transfer_workspace(g->n, n_glossy, p));
  if (rc) return rc;
  return finish(precompute_transfer(g, bvh, p, P, T, idx, M, n_glossy, status, workspace,
                                    reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_transfer_backward_workspace_size(int64_t n, const prtgs_transfer_params* p) {
  if (!p || n < 0) return 0;
  return transfer_backward_workspace(n, p);
}

int prtgs_precompute_transfer_backward(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                                       const float* dP, float* d_means, float* d_scales, float* d_quats,
                                       float* d_opacity, float* d_normals, int32_t* status, void* workspace,
                                       size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (!p || !bvh) return PRTGS_ERR_INVALID_ARG;
  if ((rc = check_order_high(p->sh_order))) return rc;
  if (p->flags & ~PRTGS_SHADOW) return PRTGS_ERR_UNSUPPORTED;
  if (prtgs::transfer_check_dirs(p->n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if (!p->dirs || !(p->t_min >= 0.f)) return PRTGS_ERR_INVALID_ARG;
  if (bvh->n != g->n) return PRTGS_ERR_SHAPE;
  if (g->n == 0) return PRTGS_OK;
  if (!dP || !g->normals || !d_means || !d_scales || !d_quats || !d_opacity || !d_normals)
    return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, transfer_backward_workspace(g->n, p));
  if (rc) return rc;
  return finish(precompute_transfer_backward(g, bvh, p, dP, d_means, d_scales, d_quats, d_opacity, d_normals, status,
                                             workspace, reinterpret_cast<cudaStream_t>(stream)));
}

// ---- backward of the glossy matrices, and the transfer backward with a visibility gradient ----

size_t prtgs_glossy_backward_workspace_size(int64_t n, const prtgs_transfer_params* p) {
  if (!p || n < 0 || check_order_high(p->sh_order)) return 0;
  return glossy_backward_workspace(n, p);
}

int prtgs_glossy_backward(const prtgs_gaussians* g, const prtgs_transfer_params* p, const float* V, const float* dM,
                          int64_t n_glossy, float* dV, float* d_roughness, float* d_metallic, float* d_normals,
                          int32_t* status, void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (!p) return PRTGS_ERR_INVALID_ARG;
  if ((rc = check_order_high(p->sh_order))) return rc;
  if (prtgs::transfer_check_dirs(p->n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if (!prtgs::glossy_backward_fits(p->n_dirs, p->sh_order)) return PRTGS_ERR_UNSUPPORTED;
  if (n_glossy < 0 || n_glossy > g->n) return PRTGS_ERR_SHAPE;
  if (g->n == 0) return PRTGS_OK;
  if (!p->dirs || !dV || !d_roughness || !d_metallic || !d_normals || !g->normals) return PRTGS_ERR_INVALID_ARG;
  if (n_glossy > 0 && (!V || !dM || !g->glossy_mask || !g->roughness || !g->metallic)) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, glossy_backward_workspace(g->n, p));
  if (rc) return rc;
  return finish(glossy_backward(g, p, V, dM, n_glossy, dV, d_roughness, d_metallic, d_normals, status, workspace,
                                reinterpret_cast<cudaStream_t>(stream)));
}

int prtgs_precompute_transfer_backward_v(const prtgs_gaussians* g, const prtgs_bvh* bvh,
                                         const prtgs_transfer_params* p, const float* dP, const float* dV,
                                         float* d_means, float* d_scales, float* d_quats, float* d_opacity,
                                         float* d_normals, int32_t* status, void* workspace, size_t workspace_bytes,
                                         prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (!p || !bvh) return PRTGS_ERR_INVALID_ARG;
  if ((rc = check_order_high(p->sh_order))) return rc;
  if (p->flags & ~PRTGS_SHADOW) return PRTGS_ERR_UNSUPPORTED;
  if (prtgs::transfer_check_dirs(p->n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if (!p->dirs || !(p->t_min >= 0.f)) return PRTGS_ERR_INVALID_ARG;
  if (bvh->n != g->n) return PRTGS_ERR_SHAPE;
  if (g->n == 0) return PRTGS_OK;
  if (!g->normals || !d_means || !d_scales || !d_quats || !d_opacity || !d_normals) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, transfer_backward_workspace(g->n, p));
  if (rc) return rc;
  return finish(precompute_transfer_backward(g, bvh, p, dP, d_means, d_scales, d_quats, d_opacity, d_normals, status,
                                             workspace, reinterpret_cast<cudaStream_t>(stream), dV));
}

// ---- backward of the self-transfer bounces ----

size_t prtgs_bounce_backward_workspace_size(int64_t n, int32_t sh_order, int32_t n_bounces) {
  if (n < 0 || check_order_high(sh_order) || n_bounces < 0 || n_bounces > 64) return 0;
  return bounce_backward_workspace(n, sh_order, n_bounces);
}

int prtgs_bounce_backward(int64_t n, int32_t sh_order, int32_t n_dirs, const float* dirs, const float* normals,
                          const float* albedo, const float* P, const int32_t* idx, int32_t n_bounces, const float* dT,
                          float* dP, float* d_albedo, float* d_normals, int32_t* status, void* workspace,
                          size_t workspace_bytes, prtgs_stream_t stream) {
  int rc;
  if (n < 0) return PRTGS_ERR_SHAPE;
  if ((rc = check_order_high(sh_order))) return rc;
  if (prtgs::transfer_check_dirs(n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if (n_bounces < 0 || n_bounces > 64) return PRTGS_ERR_INVALID_ARG;
  if (n == 0) return PRTGS_OK;
  if (!dirs || !normals || !albedo || !P || !idx || !dT || !dP || !d_albedo || !d_normals)
    return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, bounce_backward_workspace(n, sh_order, n_bounces));
  if (rc) return rc;
  return finish(bounce_backward(n, sh_order, n_dirs, dirs, normals, albedo, P, idx, n_bounces, dT, dP, d_albedo,
                                d_normals, status, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

// ---- visibility cache, training-stage transfer, pseudo-normal, normal loss ----

size_t prtgs_visibility_workspace_size(int64_t n, const prtgs_transfer_params* p) {
  if (!p || n < 0) return 0;
  return transfer_workspace(n, 0, p, true);
}

int prtgs_precompute_visibility(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                                float* V, float* P, int32_t* status, void* workspace, size_t workspace_bytes,
                                prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (!p || !bvh) return PRTGS_ERR_INVALID_ARG;
  if ((rc = check_order_high(p->sh_order))) return rc;
  if (p->flags != PRTGS_SHADOW) return PRTGS_ERR_UNSUPPORTED;
  if (prtgs::transfer_check_dirs(p->n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if (!p->dirs || !(p->t_min >= 0.f) || !(p->same_surface_t >= 0.f)) return PRTGS_ERR_INVALID_ARG;
  if (p->walk < 0 || p->walk > 1 || p->packet_dirs < 0 || p->packet_dirs > 64) return PRTGS_ERR_INVALID_ARG;
  if (bvh->n != g->n) return PRTGS_ERR_SHAPE;
  if (g->n == 0) return PRTGS_OK;
  if (!V || !P || !g->normals) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, transfer_workspace(g->n, 0, p, true));
  if (rc) return rc;
  return finish(precompute_transfer(g, bvh, p, P, nullptr, nullptr, nullptr, 0, status, workspace,
                                    reinterpret_cast<cudaStream_t>(stream), V));
}

size_t prtgs_training_transfer_workspace_size(int32_t sh_order, int32_t n_dirs) {
  if (check_order_high(sh_order) || prtgs::transfer_check_dirs(n_dirs)) return 0;
  return training_transfer_workspace(sh_order, n_dirs);
}

static int check_training(const prtgs_gaussians* g, int32_t sh_order, int32_t n_dirs, const float* dirs,
                          const float* V, const float* cam_pos, const void* out, void* workspace,
                          size_t workspace_bytes) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if ((rc = check_order_high(sh_order))) return rc;
  if (prtgs::transfer_check_dirs(n_dirs) != PRTGS_OK) return PRTGS_ERR_UNSUPPORTED;
  if (!cam_pos || !(cam_pos[0] == cam_pos[0] && cam_pos[1] == cam_pos[1] && cam_pos[2] == cam_pos[2]))
    return PRTGS_ERR_INVALID_ARG;
  if (g->n == 0) return PRTGS_OK;
  if (!dirs || !V || !out || !g->normals || !g->roughness || !g->metallic) return PRTGS_ERR_INVALID_ARG;
  return check_ws(workspace, workspace_bytes, training_transfer_workspace(sh_order, n_dirs));
}

int prtgs_training_transfer(const prtgs_gaussians* g, int32_t sh_order, int32_t n_dirs, const float* dirs,
                            const float* V, const float* cam_pos, float* t, void* workspace, size_t workspace_bytes,
                            prtgs_stream_t stream) {
  int rc = check_training(g, sh_order, n_dirs, dirs, V, cam_pos, t, workspace, workspace_bytes);
  if (rc || g->n == 0) return rc;
  return finish(training_transfer(g, sh_order, n_dirs, dirs, V, cam_pos, nullptr, t, nullptr, nullptr, workspace,
                                  reinterpret_cast<cudaStream_t>(stream)));
}

int prtgs_training_transfer_backward(const prtgs_gaussians* g, int32_t sh_order, int32_t n_dirs, const float* dirs,
                                     const float* V, const float* cam_pos, const float* dt, float* d_roughness,
                                     float* d_metallic, void* workspace, size_t workspace_bytes,
                                     prtgs_stream_t stream) {
  int rc = check_training(g, sh_order, n_dirs, dirs, V, cam_pos, dt, workspace, workspace_bytes);
  if (rc || g->n == 0) return rc;
  if (!d_roughness || !d_metallic) return PRTGS_ERR_INVALID_ARG;
  return finish(training_transfer(g, sh_order, n_dirs, dirs, V, cam_pos, dt, nullptr, d_roughness, d_metallic,
                                  workspace, reinterpret_cast<cudaStream_t>(stream)));
}

int prtgs_pseudo_normal(const prtgs_camera* cam, const float* depth, float* pseudo, prtgs_stream_t stream) {
  if (!cam || cam->width < 0 || cam->height < 0) return PRTGS_ERR_INVALID_ARG;
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return PRTGS_ERR_INVALID_ARG;
  if ((int64_t)cam->width * cam->height == 0) return PRTGS_OK;
  if (!depth || !pseudo) return PRTGS_ERR_INVALID_ARG;
  return finish(pseudo_normal(cam, depth, pseudo, reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_normal_loss_workspace_size(int32_t width, int32_t height) {
  if (width < 0 || height < 0) return 0;
  return normal_loss_workspace(width, height);
}

int prtgs_normal_loss(int32_t width, int32_t height, const float* normal, const float* pseudo, float* loss,
                      float* d_normal, void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  if (width < 0 || height < 0 || !loss) return PRTGS_ERR_INVALID_ARG;
  if ((int64_t)width * height > 0 && (!normal || !pseudo)) return PRTGS_ERR_INVALID_ARG;
  int rc = check_ws(workspace, workspace_bytes, normal_loss_workspace(width, height));
  if (rc) return rc;
  return finish(normal_loss(width, height, normal, pseudo, loss, d_normal, workspace,
                            reinterpret_cast<cudaStream_t>(stream)));
}

// ---- relight ----
size_t prtgs_relight_workspace_size(int64_t n, int32_t sh_order, int32_t k, int32_t precision) {
  if (n < 0 || k < 0) return 0;
  return relight_workspace(n, sh_order, k, precision);
}

int prtgs_relight(int64_t n, int32_t sh_order, const float* T, int32_t t_channels, const float* albedo,
                  int64_t n_glossy, const int32_t* glossy_ids, const float* M, const float* means,
                  const float* cam_pos, const float* L, int32_t k, int32_t precision, float* colors,
                  int32_t* status, uint32_t tc_wait_polls, void* workspace, size_t workspace_bytes,
                  prtgs_stream_t stream) {
  int rc;
  if (n < 0 || k < 0 || n_glossy < 0 || n_glossy > n) return PRTGS_ERR_SHAPE;
  if ((rc = check_order_high(sh_order))) return rc;
  if (t_channels != 1 && t_channels != 3) return PRTGS_ERR_SHAPE;
  if (precision < PRTGS_PREC_FP32 || precision > PRTGS_PREC_BF16) return PRTGS_ERR_INVALID_ARG;
  if (n == 0 || k == 0) return PRTGS_OK;
  if (precision != PRTGS_PREC_FP32 && !prtgs::relight_tc_fits(sh_order, k, t_channels, precision))
    return PRTGS_ERR_UNSUPPORTED;
  if (!T || !albedo || !L || !colors) return PRTGS_ERR_INVALID_ARG;
  if (n_glossy > 0 && (!glossy_ids || !M || !means || !cam_pos)) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, relight_workspace(n, sh_order, k, precision));
  if (rc) return rc;
  return finish(relight(n, sh_order, T, t_channels, albedo, n_glossy, glossy_ids, M, means, cam_pos, L, k, precision,
                        colors, status, tc_wait_polls, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

int prtgs_relight_batched(int64_t n, int32_t sh_order, const float* T, int32_t t_channels, const float* albedo,
                          const int64_t* scene_offsets, int32_t n_scenes, const float* L, int32_t k,
                          int32_t precision, float* colors, int32_t* status, uint32_t tc_wait_polls,
                          prtgs_stream_t stream) {
  int rc;
  if (n < 0 || k < 0 || n_scenes < 1) return PRTGS_ERR_SHAPE;
  if ((rc = check_order_high(sh_order))) return rc;
  if (t_channels != 1 && t_channels != 3) return PRTGS_ERR_SHAPE;
  if (precision < PRTGS_PREC_FP32 || precision > PRTGS_PREC_BF16) return PRTGS_ERR_INVALID_ARG;
  if (n == 0 || k == 0) return PRTGS_OK;
  if (!T || !albedo || !L || !colors || !scene_offsets) return PRTGS_ERR_INVALID_ARG;
  if (precision != PRTGS_PREC_FP32 && !prtgs::relight_tc_fits(sh_order, k, t_channels, precision))
    return PRTGS_ERR_UNSUPPORTED;
  return finish(relight_batched(n, sh_order, T, t_channels, albedo, scene_offsets, n_scenes, L, k, precision,
                                colors, status, tc_wait_polls, reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_relight_backward_workspace_size(int64_t n, int32_t sh_order, int32_t k) {
  if (n < 0 || k < 0 || check_order_high(sh_order)) return 0;
  return relight_backward_workspace(n, sh_order, k);
}

int prtgs_relight_backward(int64_t n, int32_t sh_order, const float* T, int32_t t_channels, const float* albedo,
                           const float* L, int32_t k, const float* dcolors, float* d_albedo, float* dT, float* dL,
                           void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  int rc;
  if (n < 0 || k < 0) return PRTGS_ERR_SHAPE;
  if ((rc = check_order_high(sh_order))) return rc;
  if (t_channels != 1 && t_channels != 3) return PRTGS_ERR_SHAPE;
  if (k == 0) return PRTGS_OK;
  if (!dL || (n > 0 && (!T || !albedo || !L || !dcolors || !d_albedo))) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, relight_backward_workspace(n, sh_order, k));
  if (rc) return rc;
  return finish(relight_backward(n, sh_order, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, workspace,
                                 reinterpret_cast<cudaStream_t>(stream)));
}

// ---- render ----
size_t prtgs_render_state_bytes(int64_t n, int32_t width, int32_t height, int64_t max_pairs) {
  if (n < 0 || width <= 0 || height <= 0 || max_pairs < 0) return 0;
  return render_state_bytes(n, width, height, max_pairs);
}

int prtgs_render_state_init(void* buffer, size_t bytes, int64_t n, int32_t width, int32_t height,
                            int64_t max_pairs, prtgs_render_state* out) {
  if (!out || n < 0 || width <= 0 || height <= 0 || max_pairs < 0) return PRTGS_ERR_INVALID_ARG;
  if (max_pairs >= (int64_t(1) << 32)) return PRTGS_ERR_UNSUPPORTED;
  if (!buffer || !aligned256(buffer) || bytes < render_state_bytes(n, width, height, max_pairs))
    return PRTGS_ERR_WORKSPACE;
  return render_state_layout(buffer, n, width, height, max_pairs, out);
}

size_t prtgs_render_workspace_size(int64_t n, int32_t width, int32_t height, int64_t max_pairs) {
  if (n < 0 || width <= 0 || height <= 0 || max_pairs < 0) return 0;
  return render_workspace(n, width, height, max_pairs);
}

static int check_camera(const prtgs_camera* cam) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || !(cam->fx > 0.f) || !(cam->fy > 0.f))
    return PRTGS_ERR_INVALID_ARG;
  if ((int64_t)((cam->width + 15) / 16) * ((cam->height + 15) / 16) >= (int64_t(1) << 31))
    return PRTGS_ERR_UNSUPPORTED;
  return PRTGS_OK;
}

size_t prtgs_render_relit_workspace_size(int64_t n, int32_t sh_order, int32_t width, int32_t height,
                                         int64_t max_pairs) {
  if (n < 0 || width <= 0 || height <= 0 || max_pairs < 0 || check_order_high(sh_order)) return 0;
  return render_relit_workspace(n, sh_order, width, height, max_pairs);
}

int prtgs_render_relit(const prtgs_gaussians* g, int32_t sh_order, const float* T, int32_t t_channels,
                       int64_t n_glossy, const int32_t* glossy_ids, const float* M, const float* L, int32_t k,
                       int32_t precision, const prtgs_camera* cam, const float* bg, float* image,
                       prtgs_render_state* st, int32_t* status, uint32_t tc_wait_polls, void* workspace,
                       size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if ((rc = check_camera(cam))) return rc;
  if ((rc = check_order_high(sh_order))) return rc;
  if (!st || st->n != g->n || st->n_scenes != 1 || st->width != cam->width || st->height != cam->height)
    return PRTGS_ERR_SHAPE;
  if (t_channels != 1 && t_channels != 3) return PRTGS_ERR_SHAPE;
  if (n_glossy < 0 || n_glossy > g->n) return PRTGS_ERR_SHAPE;
  if (precision < PRTGS_PREC_FP32 || precision > PRTGS_PREC_BF16) return PRTGS_ERR_INVALID_ARG;
  if (k < 1 || k > 256 || !L || !bg || !image || (g->n > 0 && (!T || !g->albedo))) return PRTGS_ERR_INVALID_ARG;
  if (n_glossy > 0 && (!glossy_ids || !M || !g->means)) return PRTGS_ERR_INVALID_ARG;
  if (precision != PRTGS_PREC_FP32 && !prtgs::relight_tc_fits(sh_order, k, 3, precision)) return PRTGS_ERR_UNSUPPORTED;
  rc = check_ws(workspace, workspace_bytes,
                render_relit_workspace(g->n, sh_order, cam->width, cam->height, st->max_pairs));
  if (rc) return rc;
  return finish(render_relit(g, sh_order, T, t_channels, n_glossy, glossy_ids, M, L, k, precision, cam, bg, image,
                             st, status, tc_wait_polls, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_render_geometry_workspace_size(int64_t n, int32_t width, int32_t height, int64_t max_pairs) {
  if (n < 0 || width <= 0 || height <= 0 || max_pairs < 0) return 0;
  return render_geometry_workspace(n, width, height, max_pairs);
}

int prtgs_render_geometry(const prtgs_gaussians* g, const prtgs_camera* cam, float* depth, float* normal,
                          prtgs_render_state* st, int32_t* status, void* workspace, size_t workspace_bytes,
                          prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if ((rc = check_camera(cam))) return rc;
  if (!st || st->n != g->n || st->n_scenes != 1 || st->width != cam->width || st->height != cam->height)
    return PRTGS_ERR_SHAPE;
  if (!depth || !normal || (g->n > 0 && !g->normals)) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, render_geometry_workspace(g->n, cam->width, cam->height, st->max_pairs));
  if (rc) return rc;
  return finish(render_geometry(g, cam, depth, normal, st, status, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

int prtgs_render(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam,
                 const float* bg, float* image, prtgs_render_state* st, int32_t* status, void* workspace,
                 size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if ((rc = check_camera(cam))) return rc;
  if (!st || st->n != g->n || st->n_scenes != 1 || st->width != cam->width || st->height != cam->height)
    return PRTGS_ERR_SHAPE;
  if (k < 1 || !bg || !image || (g->n > 0 && !colors)) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, render_workspace(g->n, cam->width, cam->height, st->max_pairs));
  if (rc) return rc;
  return finish(render(g, colors, k, cam, bg, image, st, status, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_render_backward_workspace_size(int64_t n, int32_t k) {
  if (n < 0 || k < 1) return 0;
  return render_backward_workspace(n, k);
}

int prtgs_render_backward(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam,
                          const float* bg, const prtgs_render_state* st, const float* dimage, float* d_means,
                          float* d_scales, float* d_quats, float* d_opacity, float* d_colors, void* workspace,
                          size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if ((rc = check_camera(cam))) return rc;
  if (!st || st->n != g->n || st->n_scenes != 1 || st->width != cam->width || st->height != cam->height)
    return PRTGS_ERR_SHAPE;
  if (k < 1 || !bg || !dimage) return PRTGS_ERR_INVALID_ARG;
  if (g->n == 0) return PRTGS_OK;
  if (!colors || !d_means || !d_scales || !d_quats || !d_opacity || !d_colors) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, render_backward_workspace(g->n, k));
  if (rc) return rc;
  return finish(render_backward(g, colors, k, cam, bg, st, dimage, d_means, d_scales, d_quats, d_opacity, d_colors,
                                workspace, reinterpret_cast<cudaStream_t>(stream)));
}

// ---- batched scenes: one launch per stage over every scene ----
size_t prtgs_render_state_bytes_batched(int64_t n, int32_t n_scenes, int32_t width, int32_t height,
                                        int64_t max_pairs) {
  if (n < 0 || n_scenes < 1 || width <= 0 || height <= 0 || max_pairs < 0) return 0;
  return render_state_bytes_batched(n, n_scenes, width, height, max_pairs);
}

int prtgs_render_state_init_batched(void* buffer, size_t bytes, int64_t n, int32_t n_scenes, int32_t width,
                                    int32_t height, int64_t max_pairs, prtgs_render_state* out) {
  if (!out || n < 0 || n_scenes < 1 || width <= 0 || height <= 0 || max_pairs < 0) return PRTGS_ERR_INVALID_ARG;
  if (n_scenes > kMaxScenes || max_pairs >= (int64_t(1) << 32)) return PRTGS_ERR_UNSUPPORTED;
  if (!buffer || !aligned256(buffer) || bytes < render_state_bytes_batched(n, n_scenes, width, height, max_pairs))
    return PRTGS_ERR_WORKSPACE;
  return render_state_layout_batched(buffer, n, n_scenes, width, height, max_pairs, out);
}

static int check_batch(const prtgs_gaussians* g, const int64_t* offsets, int32_t n_scenes, const prtgs_camera* cams,
                       const prtgs_render_state* st) {
  int rc = check_gaussians(g);
  if (rc) return rc;
  if (n_scenes < 1 || n_scenes > kMaxScenes) return PRTGS_ERR_UNSUPPORTED;
  if (!offsets || !cams) return PRTGS_ERR_INVALID_ARG;
  for (int b = 0; b < n_scenes; ++b) {
    if ((rc = check_camera(cams + b))) return rc;
    if (cams[b].width != cams[0].width || cams[b].height != cams[0].height) return PRTGS_ERR_SHAPE;
  }
  if (!st || st->n != g->n || st->n_scenes != n_scenes || st->width != cams[0].width ||
      st->height != cams[0].height)
    return PRTGS_ERR_SHAPE;
  if ((int64_t)n_scenes * st->tiles_x * st->tiles_y >= (int64_t(1) << 31)) return PRTGS_ERR_UNSUPPORTED;
  return PRTGS_OK;
}

size_t prtgs_render_batched_workspace_size(int64_t n, int32_t n_scenes, int32_t width, int32_t height,
                                           int64_t max_pairs) {
  if (n < 0 || n_scenes < 1 || width <= 0 || height <= 0 || max_pairs < 0) return 0;
  return render_workspace(n, width, height, max_pairs);
}

int prtgs_render_batched(const prtgs_gaussians* g, const int64_t* scene_offsets, int32_t n_scenes,
                         const float* colors, int32_t k, const prtgs_camera* cams, const float* bg, float* images,
                         prtgs_render_state* st, int32_t* status, void* workspace, size_t workspace_bytes,
                         prtgs_stream_t stream) {
  int rc = check_batch(g, scene_offsets, n_scenes, cams, st);
  if (rc) return rc;
  if (k < 1 || !bg || !images || (g->n > 0 && !colors)) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, render_workspace(g->n, cams[0].width, cams[0].height, st->max_pairs));
  if (rc) return rc;
  return finish(render_batched(g, scene_offsets, n_scenes, colors, k, cams, bg, images, st, status, workspace,
                               reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_render_backward_batched_workspace_size(int64_t n, int32_t k) {
  if (n < 0 || k < 1) return 0;
  return render_backward_workspace(n, k);
}

int prtgs_render_backward_batched(const prtgs_gaussians* g, const int64_t* scene_offsets, int32_t n_scenes,
                                  const float* colors, int32_t k, const prtgs_camera* cams, const float* bg,
                                  const prtgs_render_state* st, const float* dimages, float* d_means, float* d_scales,
                                  float* d_quats, float* d_opacity, float* d_colors, void* workspace,
                                  size_t workspace_bytes, prtgs_stream_t stream) {
  int rc = check_batch(g, scene_offsets, n_scenes, cams, st);
  if (rc) return rc;
  if (k < 1 || !bg || !dimages) return PRTGS_ERR_INVALID_ARG;
  if (g->n == 0) return PRTGS_OK;
  if (!colors || !d_means || !d_scales || !d_quats || !d_opacity || !d_colors) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, render_backward_workspace(g->n, k));
  if (rc) return rc;
  return finish(render_backward_batched(g, scene_offsets, n_scenes, colors, k, cams, bg, st, dimages, d_means,
                                        d_scales, d_quats, d_opacity, d_colors, workspace,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_l2_loss_batched_workspace_size(int64_t count, int32_t n_scenes) {
  return count > 0 && n_scenes > 0 ? l2_loss_batched_workspace(count, n_scenes) : 0;
}

int prtgs_l2_loss_batched(const float* images, const float* targets, int64_t count, int32_t n_scenes, float* losses,
                          float* dimages, void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  if (count <= 0 || n_scenes < 1 || !images || !targets || !losses || !dimages) return PRTGS_ERR_INVALID_ARG;
  if (n_scenes > 65535) return PRTGS_ERR_UNSUPPORTED;
  int rc = check_ws(workspace, workspace_bytes, l2_loss_batched_workspace(count, n_scenes));
  if (rc) return rc;
  return finish(l2_loss_batched(images, targets, count, n_scenes, losses, dimages, workspace,
                                reinterpret_cast<cudaStream_t>(stream)));
}

size_t prtgs_relight_backward_batched_workspace_size(int64_t n, int32_t n_scenes, int32_t sh_order, int32_t k) {
  if (n < 0 || k < 0 || n_scenes < 1 || check_order_high(sh_order)) return 0;
  return relight_backward_batched_workspace(n, n_scenes, sh_order, k);
}

int prtgs_relight_backward_batched(int64_t n, int32_t sh_order, const float* T, int32_t t_channels,
                                   const float* albedo, const int64_t* scene_offsets, int32_t n_scenes, const float* L,
                                   int32_t k, const float* dcolors, float* d_albedo, float* dT, float* dL,
                                   void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  int rc;
  if (n < 0 || k < 0 || n_scenes < 1) return PRTGS_ERR_SHAPE;
  if (n_scenes > 65535) return PRTGS_ERR_UNSUPPORTED;
  if ((rc = check_order_high(sh_order))) return rc;
  if (t_channels != 1 && t_channels != 3) return PRTGS_ERR_SHAPE;
  if (k == 0) return PRTGS_OK;
  if (!dL || !scene_offsets || (n > 0 && (!T || !albedo || !L || !dcolors || !d_albedo))) return PRTGS_ERR_INVALID_ARG;
  rc = check_ws(workspace, workspace_bytes, relight_backward_batched_workspace(n, n_scenes, sh_order, k));
  if (rc) return rc;
  return finish(relight_backward_batched(n, sh_order, T, t_channels, albedo, scene_offsets, n_scenes, L, k, dcolors,
                                         d_albedo, dT, dL, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

// ---- CUDA graph capture of a sequence of calls ----
int prtgs_graph_begin(prtgs_stream_t stream) {
  if (!stream) return PRTGS_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  if (cudaStreamBeginCapture(reinterpret_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return PRTGS_ERR_CUDA;
  }
  return PRTGS_OK;
}

int prtgs_graph_end(prtgs_stream_t stream, prtgs_graph_t* out) {
  if (!stream || !out) return PRTGS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture(reinterpret_cast<cudaStream_t>(stream), &graph) != cudaSuccess || !graph) {
    (void)cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return PRTGS_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess || !exec) {
    (void)cudaGetLastError();
    return PRTGS_ERR_CUDA;
  }
  *out = reinterpret_cast<prtgs_graph_t>(exec);
  return PRTGS_OK;
}

int prtgs_graph_launch(prtgs_graph_t graph, prtgs_stream_t stream) {
  if (!graph) return PRTGS_ERR_INVALID_ARG;
  if (cudaGraphLaunch(reinterpret_cast<cudaGraphExec_t>(graph), reinterpret_cast<cudaStream_t>(stream)) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return PRTGS_ERR_CUDA;
  }
  return PRTGS_OK;
}

int prtgs_graph_destroy(prtgs_graph_t graph) {
  if (!graph) return PRTGS_OK;
  return cudaGraphExecDestroy(reinterpret_cast<cudaGraphExec_t>(graph)) == cudaSuccess ? PRTGS_OK : PRTGS_ERR_CUDA;
}

size_t prtgs_l2_loss_workspace_size(int64_t count) { return count > 0 ? l2_loss_workspace(count) : 0; }

int prtgs_l2_loss(const float* image, const float* target, int64_t count, float* loss, float* dimage,
                  void* workspace, size_t workspace_bytes, prtgs_stream_t stream) {
  if (count <= 0 || !image || !target || !loss || !dimage) return PRTGS_ERR_INVALID_ARG;
  int rc = check_ws(workspace, workspace_bytes, l2_loss_workspace(count));
  if (rc) return rc;
  return finish(l2_loss(image, target, count, loss, dimage, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
