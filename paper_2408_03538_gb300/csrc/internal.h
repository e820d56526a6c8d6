// Host-side launchers shared between the translation units of libprtgs.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/prtgs.h"

namespace prtgs {

// sort.cu
size_t scan_workspace(int64_t n);
int scan_u32(const uint32_t* in, uint32_t* out, int64_t n, bool exclusive, uint32_t* total, void* ws,
             cudaStream_t stream);
size_t radix_sort_workspace(int64_t capacity);
int radix_sort_pairs(const uint64_t* keys_x, const int32_t* vals_x, uint64_t* keys_f, int32_t* vals_f,
                     uint64_t* keys_y, int32_t* vals_y, int64_t capacity, const uint32_t* d_count, int begin_bit,
                     int end_bit, void* ws, cudaStream_t stream);

// bvh.cu
size_t bvh_bytes(int64_t n, int32_t n_scenes);
int bvh_layout(void* buffer, int64_t n, int32_t n_scenes, const int64_t* scene_offsets, prtgs_bvh* out);
size_t build_bvh_workspace(int64_t n, int32_t n_scenes);
int build_bvh(const prtgs_gaussians* g, prtgs_bvh* bvh, int32_t* status, void* ws, cudaStream_t stream);

// transfer.cu
// want_V / V_out: also write every receiver's visibility row V[n,S] (not with glossy matrices)
size_t transfer_workspace(int64_t n, int64_t n_glossy, const prtgs_transfer_params* p, bool want_V = false);
int precompute_transfer(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p, float* P,
                        float* T, int32_t* idx, float* M, int64_t n_glossy, int32_t* status, void* ws,
                        cudaStream_t stream, float* V_out = nullptr);
// whether the glossy matrices of S directions at this order fit one block's shared memory
bool glossy_fits(int S, int order);
// one bounce of the self-transfer (Eq. 33-35): Tcur = B(Tprev), or B(P) when Tprev is NULL
// (Tscratch receives the forward's running sum and is not read afterwards)
int bounce_step(int64_t n, int C, int S, const float* dirs, const float* normals, const float* albedo, const float* P,
                const float* Tprev, const int32_t* idx, float* Tscratch, float* Tcur, int32_t* status,
                cudaStream_t stream);
// bounce_bwd.cu: backward of the bounces with the index matrix fixed
size_t bounce_backward_workspace(int64_t n, int32_t order, int32_t n_bounces);
int bounce_backward(int64_t n, int32_t order, int32_t S, const float* dirs, const float* normals,
                    const float* albedo, const float* P, const int32_t* idx, int32_t n_bounces, const float* dT,
                    float* dP, float* d_albedo, float* d_normals, int32_t* status, void* ws, cudaStream_t stream);
// Y[S, (order+1)^2] of the direction set, orders 1..6 (FP64, rounded once)
int sh_table(int S, int order, const float* dirs, float* Y, cudaStream_t stream);

struct TraceArgs;
// packet.cu
int launch_packet(const TraceArgs& a, float* V, bool bounce, int sms, cudaStream_t stream);

size_t transfer_backward_workspace(int64_t n, const prtgs_transfer_params* p);
// dP [n,C] and dV [n,S] (extra dLoss/dV per ray, e.g. from the glossy matrices) are both nullable
int precompute_transfer_backward(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                                 const float* dP, float* d_means, float* d_scales, float* d_quats, float* d_opacity,
                                 float* d_normals, int32_t* status, void* ws, cudaStream_t stream,
                                 const float* dV = nullptr);
// glossy-matrix backward (Eq. 40): dM -> dV [n,S] (to the transfer backward), roughness, metallic, normals
size_t glossy_backward_workspace(int64_t n, const prtgs_transfer_params* p);
int glossy_backward(const prtgs_gaussians* g, const prtgs_transfer_params* p, const float* V, const float* dM,
                    int64_t n_glossy, float* dV, float* d_roughness, float* d_metallic, float* d_normals,
                    int32_t* status, void* ws, cudaStream_t stream);
bool glossy_backward_fits(int S, int order);

// relight.cu
size_t relight_workspace(int64_t n, int32_t order, int32_t k, int32_t precision);
int relight(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo, int64_t n_glossy,
            const int32_t* glossy_ids, const float* M, const float* means, const float* cam_pos, const float* L,
            int32_t k, int32_t precision, float* colors, int32_t* status, unsigned tc_wait_polls, void* ws,
            cudaStream_t stream);
int relight_batched(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo,
                    const int64_t* offsets, int32_t n_scenes, const float* L, int32_t k, int32_t precision,
                    float* colors, int32_t* status, unsigned tc_wait_polls, cudaStream_t stream);
// relight_tc.cu
int relight_tc_shape(int32_t k, int32_t t_channels, int* n_pad, int* tmem_cols);
int relight_tc_fits(int32_t order, int32_t k, int32_t t_channels, int32_t precision);
int relight_tc(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo, const float* L,
               int32_t k, int32_t precision, const int64_t* offsets, int32_t n_scenes, float* colors,
               int32_t* status, unsigned tc_wait_polls, cudaStream_t stream);

int relight_tc_pixels(int64_t n_pix, int32_t order, const float* TI, const float* final_T, const float* bg,
                      const float* L, int32_t k, int32_t precision, float* image, int32_t* status,
                      unsigned tc_wait_polls, cudaStream_t stream);
size_t render_relit_workspace(int64_t n, int32_t order, int32_t width, int32_t height, int64_t max_pairs);
int render_relit(const prtgs_gaussians* g, int32_t order, const float* T, int32_t t_channels, int64_t n_glossy,
                 const int32_t* glossy_ids, const float* M, const float* L, int32_t k, int32_t precision,
                 const prtgs_camera* cam, const float* bg, float* image, prtgs_render_state* st, int32_t* status,
                 unsigned tc_wait_polls, void* ws, cudaStream_t stream);

size_t relight_backward_workspace(int64_t n, int32_t order, int32_t k);
size_t relight_backward_batched_workspace(int64_t n, int32_t n_scenes, int32_t order, int32_t k);
int relight_backward_batched(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo,
                             const int64_t* offsets, int32_t n_scenes, const float* L, int32_t k,
                             const float* dcolors, float* d_albedo, float* dT, float* dL, void* ws,
                             cudaStream_t stream);
int relight_backward(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo,
                     const float* L, int32_t k, const float* dcolors, float* d_albedo, float* dT, float* dL,
                     void* ws, cudaStream_t stream);

// render.cu
size_t render_state_bytes(int64_t n, int32_t width, int32_t height, int64_t max_pairs);
size_t render_state_bytes_batched(int64_t n, int32_t B, int32_t width, int32_t height, int64_t max_pairs);
int render_state_layout_batched(void* buffer, int64_t n, int32_t B, int32_t width, int32_t height,
                                int64_t max_pairs, prtgs_render_state* out);
int render_batched(const prtgs_gaussians* g, const int64_t* offsets, int32_t B, const float* colors, int32_t k,
                   const prtgs_camera* cams, const float* bg, float* images, prtgs_render_state* st, int32_t* status,
                   void* ws, cudaStream_t stream);
int render_backward_batched(const prtgs_gaussians* g, const int64_t* offsets, int32_t B, const float* colors,
                            int32_t k, const prtgs_camera* cams, const float* bg, const prtgs_render_state* st,
                            const float* dimages, float* d_means, float* d_scales, float* d_quats, float* d_opacity,
                            float* d_colors, void* ws, cudaStream_t stream);
size_t l2_loss_batched_workspace(int64_t count, int32_t n_scenes);
int l2_loss_batched(const float* images, const float* targets, int64_t count, int32_t n_scenes, float* losses,
                    float* dimages, void* ws, cudaStream_t stream);
int render_state_layout(void* buffer, int64_t n, int32_t width, int32_t height, int64_t max_pairs,
                        prtgs_render_state* out);
size_t render_workspace(int64_t n, int32_t width, int32_t height, int64_t max_pairs);
int render(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam, const float* bg,
           float* image, prtgs_render_state* st, int32_t* status, void* ws, cudaStream_t stream);
size_t render_geometry_workspace(int64_t n, int32_t width, int32_t height, int64_t max_pairs);
int render_geometry(const prtgs_gaussians* g, const prtgs_camera* cam, float* depth, float* normal,
                    prtgs_render_state* st, int32_t* status, void* ws, cudaStream_t stream);
size_t render_backward_workspace(int64_t n, int32_t k);
int render_backward(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam,
                    const float* bg, const prtgs_render_state* st, const float* dimage, float* d_means,
                    float* d_scales, float* d_quats, float* d_opacity, float* d_colors, void* ws,
                    cudaStream_t stream);
size_t l2_loss_workspace(int64_t count);
int l2_loss(const float* image, const float* target, int64_t count, float* loss, float* dimage, void* ws,
            cudaStream_t stream);

// training.cu: training-stage transfer (Eq. 28), pseudo-normal and normal loss (Eq. 24-25)
size_t training_transfer_workspace(int32_t order, int32_t n_dirs);
int training_transfer(const prtgs_gaussians* g, int32_t order, int32_t S, const float* dirs, const float* V,
                      const float* cam_pos, const float* dt, float* t, float* d_roughness, float* d_metallic,
                      void* ws, cudaStream_t stream);
int pseudo_normal(const prtgs_camera* cam, const float* depth, float* pseudo, cudaStream_t stream);
size_t normal_loss_workspace(int32_t width, int32_t height);
int normal_loss(int32_t width, int32_t height, const float* normal, const float* pseudo, float* loss,
                float* d_normal, void* ws, cudaStream_t stream);

}  // namespace prtgs
