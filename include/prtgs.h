/*
 * libprtgs -- C ABI of a GB300 (sm_103a) implementation of the data-parallel hot path of
 * "PRTGS: Precomputed Radiance Transfer of Gaussian Splats for Real-Time High-Quality
 * Relighting" (arxiv 2408.03538).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Every array argument is a caller-owned, contiguous DEVICE pointer unless a comment
 *    says "host". Floating point arrays are FP32, structure-of-arrays, row-major.
 *  * The library never allocates device memory. Calls that need scratch space take
 *    (void* workspace, size_t workspace_bytes) sized by the matching *_workspace_size()
 *    query; the workspace must be 256-byte aligned and is clobbered by the call.
 *  * All work is enqueued on the caller's stream (cudaStream_t passed as prtgs_stream_t)
 *    and the call returns without synchronising. Calls keep no state between invocations,
 *    so concurrent calls on different streams with distinct buffers are safe.
 *  * Return value: PRTGS_OK or a negative PRTGS_ERR_* code for errors detected on the host
 *    (arguments, shapes, workspace size, CUDA launch errors). Errors detected on the device
 *    (non-finite inputs, traversal stack overflow, buffer capacity) are OR-ed as bit flags
 *    into a caller-provided int32 device status word, read after synchronisation with
 *    prtgs_read_status(). No kernel traps, asserts or waits without a bound: the one device
 *    wait, for the tensor cores' completion in the tcgen05 relight paths, polls at most
 *    tc_wait_polls times (PRTGS_TC_WAIT_POLLS normally). When it gives up, the CTA sets
 *    PRTGS_STATUS_TIMEOUT, waits once more with PRTGS_TC_WAIT_POLLS polls so that the
 *    tensor cores have finished with its shared and tensor memory before either is reused or
 *    freed, writes NaN to the outputs of that tile and of every later tile it owns, and issues
 *    no further tensor-core work.
 *
 * Notation follows the paper: N Gaussians, S sphere directions, C = (order+1)^2 real SH
 * coefficients (orders 1-6, so C <= 49, on every path; the tensor-core relight pads K = C to a
 * multiple of 16), k lights, H x W image.
 */
#ifndef PRTGS_H
#define PRTGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* prtgs_stream_t; /* a cudaStream_t; NULL = legacy default stream */

/* ---- status codes (host return values) ---------------------------------------------- */
#define PRTGS_OK 0
#define PRTGS_ERR_INVALID_ARG (-1)  /* null pointer, negative size, value out of range */
#define PRTGS_ERR_SHAPE (-2)        /* inconsistent sizes */
#define PRTGS_ERR_UNSUPPORTED (-3)  /* SH order outside 1..6, too many scenes, ... */
#define PRTGS_ERR_WORKSPACE (-4)    /* workspace too small or misaligned */
#define PRTGS_ERR_CUDA (-5)         /* a CUDA launch or copy failed */

/* ---- device status bits (OR-ed into the caller's int32 status word) ------------------ */
#define PRTGS_STATUS_NONFINITE 1       /* a non-finite or out-of-range Gaussian parameter */
#define PRTGS_STATUS_STACK_OVERFLOW 2  /* BVH traversal stack exceeded (cannot happen for <= 2^27 leaves) */
#define PRTGS_STATUS_CAPACITY 4        /* render: more (Gaussian, tile) pairs than max_pairs */
#define PRTGS_STATUS_BAD_INDEX 8       /* an index outside its array was met and skipped */
#define PRTGS_STATUS_TIMEOUT 16        /* a tensor-core completion wait gave up (outputs of that tile are NaN) */

/* Default poll limit of the tensor cores' completion wait (argument tc_wait_polls below). */
#define PRTGS_TC_WAIT_POLLS (1u << 26)

/* ---- flags of prtgs_transfer_params.flags ------------------------------------------- */
#define PRTGS_SHADOW 1u  /* visibility V from the other Gaussians (else V = 1) */
#define PRTGS_BOUNCE 2u  /* index matrix + one-bounce self-transfer, T becomes [N,3,C] */
#define PRTGS_GLOSSY 4u  /* C x C transfer matrices for Gaussians with glossy_mask != 0 */

/* ---- relight precision ---------------------------------------------------------------- */
#define PRTGS_PREC_FP32 0   /* FP32 FMA on the CUDA cores */
#define PRTGS_PREC_BF16X3 1 /* tensor cores (tcgen05), operands split into 3 BF16 terms, FP32 accumulate */
#define PRTGS_PREC_BF16 2   /* tensor cores, plain BF16 operands, FP32 accumulate */

/*
 * Gaussian set (Sec. 3.1, Eq. 1-2; PBR attributes of Sec. 4.2-4.3).
 *   means[n,3], scales[n,3] (standard deviations along the local axes, > 0),
 *   quats[n,4] as (w,x,y,z) (normalised by the library), opacity[n] in [0,1),
 *   normals[n,3] (unit), albedo[n,3], roughness[n] and metallic[n] (glossy only, may be
 *   NULL otherwise), glossy_mask[n] uint8 (NULL = no glossy splats).
 */
typedef struct prtgs_gaussians {
  int64_t n;
  const float* means;
  const float* scales;
  const float* quats;
  const float* opacity;
  const float* normals;
  const float* albedo;
  const float* roughness;
  const float* metallic;
  const uint8_t* glossy_mask;
} prtgs_gaussians;

/*
 * Linear BVH over the Gaussians' 3-sigma boxes (Sec. 4.4 "constructed upon the BVH"):
 * one binary radix tree (Karras 2012) over 64-bit Morton keys, one subtree per scene.
 * All pointers lie inside one caller buffer laid out by prtgs_bvh_init().
 *   keys[n]        sorted keys: scene << 57 | morton30 << 27 | index within scene
 *   order[n]       Gaussian index at each sorted position
 *   nodes[n-1,16]  internal nodes: floats 0-5 box of child 0 (lo xyz, hi xyz), 6-11 box of
 *                  child 1, then int32 child0, child1, parent, 0. A child >= 0 is an
 *                  internal node, a child < 0 is the leaf at sorted position ~child.
 *   records[n,16]  per sorted position: mean xyz, opacity, A = diag(1/s) R^T (9, row-major),
 *                  normal xyz -- the traversal record
 *   leaf_parent[n] parent node of each leaf (sorted position); -1 for a single-leaf scene
 *   roots[n_scenes] root of each scene's subtree (same encoding as a child)
 *   scene_offsets  device int64 [n_scenes+1], offsets of the scenes in the Gaussian arrays
 */
typedef struct prtgs_bvh {
  int64_t n;
  int32_t n_scenes;
  int32_t reserved;
  uint64_t* keys;
  int32_t* order;
  float* nodes;
  float* records;
  int32_t* leaf_parent;
  int32_t* roots;
  const int64_t* scene_offsets;
} prtgs_bvh;

/* Bytes needed for a BVH over n Gaussians in n_scenes scenes (host query). */
size_t prtgs_bvh_bytes(int64_t n, int32_t n_scenes);

/*
 * Lay out a BVH in `buffer` (device, >= prtgs_bvh_bytes, 256-byte aligned). Host only;
 * no GPU work. `scene_offsets` is a device int64 array [n_scenes+1] starting at 0 and
 * ending at n; it must stay alive as long as the BVH is used. Scenes may hold at most
 * 2^27 Gaussians each and n_scenes <= 128.
 */
int prtgs_bvh_init(void* buffer, size_t bytes, int64_t n, int32_t n_scenes, const int64_t* scene_offsets,
                   prtgs_bvh* out);

size_t prtgs_build_bvh_workspace_size(int64_t n, int32_t n_scenes);

/*
 * Build the BVH (Sec. 4.4): per-scene centre bounds, 30-bit Morton codes quantised in
 * FP32 as q = min(floor((c - lo) * (1024 / (hi - lo))), 1023), an LSD radix sort, the
 * Karras split search, traversal records and a bottom-up box refit. Keys, order and
 * topology are deterministic and integer-exact. Boxes are conservative (padded 3-sigma
 * boxes: half-extent_a = 3 sqrt(Sigma_aa) from Eq. 2). `status` (device int32, may be
 * NULL) receives PRTGS_STATUS_NONFINITE for invalid Gaussians.
 */
int prtgs_build_bvh(const prtgs_gaussians* g, prtgs_bvh* bvh, int32_t* status, void* workspace,
                    size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Transfer precompute parameters (Sec. 4.4-4.5).
 *   sh_order        1..6 (C = (order+1)^2 coefficients; for 4..6 the SH of the direction set
 *                   are tabulated per call). With PRTGS_GLOSSY the block of the glossy matrices
 *                   holds 3 S + 3 S C floats and 2 S ints of shared memory: above 227 KB of
 *                   it (e.g. S > 382 at order 6) -> PRTGS_ERR_UNSUPPORTED
 *   n_dirs, dirs    S shared world-space directions [S,3] (device); weight 4 pi / S each
 *   t_min           a ray stops once its transmittance falls below t_min (bounded error
 *                   t_min per ray); 0 disables early exit. Suggested 2^-30.
 *   same_surface_t  the Sec. 4.4 filter: a hit is eligible for the index matrix only if the
 *                   transmittance in front of it is <= t; 1 disables the filter.
 *   flags           PRTGS_SHADOW | PRTGS_BOUNCE | PRTGS_GLOSSY
 *   index_buffer    tuning: candidates per index-matrix search round (1, 2, 4 or 8; 0 = default)
 *   n_bounces       self-transfer bounces with PRTGS_BOUNCE (Eq. 34-35): T = P + T^1 + ... + T^n,
 *                   T^k_i = sum_s w (n_i.w_s)^+ (rho_j/pi) T^{k-1}_j over the index matrix, T^0 = P;
 *                   0 or 1 = one bounce (Eq. 33), at most 64; more than one needs 3nC floats of
 *                   workspace per extra buffer (two at most)
 *   walk            tuning: 0 = warp packets (default: the rays that 32 receivers adjacent in
 *                   Morton order cast along one direction walk the BVH together), 1 = one ray
 *                   per lane (the plain per-ray walk); both give the same results
 *   packet_dirs     tuning: directions per work item of the packet walk (a work item is a
 *                   window of 64 receivers adjacent in Morton order x packet_dirs directions;
 *                   for each direction the window's receivers that face it are compacted into
 *                   packets of 32 lanes), 1..64; 0 = the default (1, see prtgs_autotune); the
 *                   results do not depend on it
 *   stats           optional device uint64[10] that the call ADDS its work counters to:
 *                   BVH node visits of the visibility walks, node visits of the index-matrix
 *                   search, leaf tests, ray-Gaussian hits, search rounds, traced rays, rays
 *                   queued for the first index-matrix round, rays that needed later rounds,
 *                   warp-packet walks, leaves a packet evaluated for at least one of its rays
 *                   (NULL = not gathered)
 */
typedef struct prtgs_transfer_params {
  int32_t sh_order;
  int32_t n_dirs;
  const float* dirs;
  float t_min;
  float same_surface_t;
  uint32_t flags;
  int32_t index_buffer;
  unsigned long long* stats;
  int32_t n_bounces;
  int32_t walk;
  int32_t packet_dirs;
} prtgs_transfer_params;

size_t prtgs_transfer_workspace_size(int64_t n, int64_t n_glossy, const prtgs_transfer_params* p);

/*
 * Per-Gaussian radiance transfer (Eq. 29, Eq. 33-35, Eq. 40).
 *  P[n,C]        out: P_i = sum_s (4 pi/S) V_is max(0, n_i.w_s) Y(w_s), with
 *                V_is = prod over the other Gaussians j hit by the ray from mu_i along w_s
 *                of (1 - opacity_j exp(-D_ij^2/2)); a hit is t* > 0 and D^2 <= 9, with t*
 *                and D the closest approach of the ray to j in j's Mahalanobis metric
 *                (Eq. 27 read as the Gaussian's maximum along the ray). Albedo and 1/pi are
 *                applied at relight time.
 *  T[n,3,C]      out (PRTGS_BOUNCE, else unused): T_i = P_i + sum_s (4 pi/S) max(0, n_i.w_s)
 *                (albedo_j/pi) P_j, j = idx[i,s] (Eq. 33, one bounce); with p->n_bounces > 1
 *                the further bounces of Eq. 34-35 are added (see prtgs_transfer_params).
 *  idx[n,S]      out (required with PRTGS_BOUNCE, else unused): index matrix of Sec. 4.4:
 *                the hit with the largest W_j = alpha_j prod_{before j}(1-alpha) max(0,-w.n_j)
 *                (Eq. 26), -1 when no eligible hit has W > 0 or n_i.w_s <= 0.
 *  M[n_glossy,C,C] out (PRTGS_GLOSSY): glossy transfer matrices (Eq. 40), in increasing
 *                Gaussian order of the glossy splats:
 *                M[a,b] = sum_s sum_o (4 pi/S)^2 Y_a(w_s) k(w_s,w_o) max(0,n.w_s) V_s Y_b(w_o),
 *                k = (1-metallic) + pi D F G / (4 (n.w_s)(n.w_o)), zero for n.w_o <= 0, with
 *                the unit normal n/|n| in D, F, G (GGX with alpha = roughness^2, Schlick with
 *                F0 = 0.04, Smith-Schlick with k = alpha/2).
 *  status        device int32 word for PRTGS_STATUS_* bits (may be NULL).
 * A BVH built from the same Gaussian arrays must be passed.
 */
int prtgs_precompute_transfer(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                              float* P, float* T, int32_t* idx, float* M, int64_t n_glossy, int32_t* status,
                              void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Transfer backward: gradients of a loss through P (the shadowed diffuse transfer of Eq. 29
 * projected by Eq. 9) to the Gaussians, for optimising geometry against relit images
 * (Sec. 4.4). Each traced ray is walked again twice in the forward's order -- once for
 * V_is, once pushing dL/dalpha_j = -g V_is / (1 - alpha_j) to every occluder up to the same
 * early exit -- so no per-ray hit list is stored. The hit set (t* > 0, D^2 <= 9) and the
 * hemisphere test are held fixed (non-differentiable boundaries); the gradient flows through
 * opacity_j exp(-D^2/2), D^2 at the closest approach (to mu_j, s_j, q_j and, via the ray
 * origin, mu_i) and the cosine max(0, n_i.w) (to the raw normal n_i).
 *   dP[n,C]      in (device)
 *   d_means[n,3], d_scales[n,3], d_quats[n,4], d_opacity[n], d_normals[n,3]  out (device;
 *                overwritten; accumulated with float atomics, so the last bits vary run to run)
 * p->flags must be PRTGS_SHADOW or 0 (unshadowed: only d_normals is non-zero); PRTGS_BOUNCE or
 * PRTGS_GLOSSY -> PRTGS_ERR_UNSUPPORTED. The bvh must have been built from the same g.
 * Errors: as prtgs_precompute_transfer.
 */
size_t prtgs_transfer_backward_workspace_size(int64_t n, const prtgs_transfer_params* p);
int prtgs_precompute_transfer_backward(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                                       const float* dP, float* d_means, float* d_scales, float* d_quats,
                                       float* d_opacity, float* d_normals, int32_t* status, void* workspace,
                                       size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Backward of the glossy transfer matrices (Eq. 40): from dM = dLoss/dM [n_glossy,C,C] (the glossy
 * splats in increasing Gaussian order, as prtgs_precompute_transfer returns M) to
 *   dV[n,S]         out: dLoss/dV_is of each glossy receiver's rays (0 for the others); pass it to
 *                   prtgs_precompute_transfer_backward_v to reach the occluders' geometry
 *   d_roughness[n], d_metallic[n]  out: through the BRDF kernel k (GGX with alpha = r^2; k = 1 - m + ...)
 *   d_normals[n,3]  out: through the cosine max(0, n.w_s) (raw normal) and the kernel (n / |n|)
 * With U_so = Y(w_s)^T dM Y(w_o): dLoss/dV_s = w^2 (n.w_s)^+ sum_o k(s,o) U_so, and the others as
 * the derivatives of sum_s sum_o w^2 (n.w_s)^+ V_s k(s,o) U_so. The cut-offs n.w > 0 are held
 * fixed. V[n,S] is the visibility of prtgs_precompute_visibility (same walk as the forward).
 * Outputs are overwritten (deterministic). Workspace: prtgs_glossy_backward_workspace_size;
 * PRTGS_ERR_UNSUPPORTED when the block's shared memory (3S + 2SC + C^2 floats, 2S ints) exceeds 227 KB.
 */
size_t prtgs_glossy_backward_workspace_size(int64_t n, const prtgs_transfer_params* p);
int prtgs_glossy_backward(const prtgs_gaussians* g, const prtgs_transfer_params* p, const float* V, const float* dM,
                          int64_t n_glossy, float* dV, float* d_roughness, float* d_metallic, float* d_normals,
                          int32_t* status, void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/*
 * prtgs_precompute_transfer_backward with an additional per-ray visibility gradient: dV[n,S]
 * (nullable) is added to the dLoss/dV_is that dP implies (w (n_i.w_s)^+ Y(w_s) . dP_i) before the
 * walk pushes it to the occluders; dP (nullable) as before. Receivers whose dP and dV rows are
 * zero are skipped. Same workspace and errors as prtgs_precompute_transfer_backward.
 */
int prtgs_precompute_transfer_backward_v(const prtgs_gaussians* g, const prtgs_bvh* bvh,
                                         const prtgs_transfer_params* p, const float* dP, const float* dV,
                                         float* d_means, float* d_scales, float* d_quats, float* d_opacity,
                                         float* d_normals, int32_t* status, void* workspace, size_t workspace_bytes,
                                         prtgs_stream_t stream);

/*
 * Backward of the self-transfer bounces (Eq. 33-35) with the index matrix held fixed (its argmax
 * is a discrete decision). Forward, per channel c: T = T^0 + ... + T^n, T^0_i = P_i,
 * T^k_i[c] = sum_s (4 pi/S) max(0, n_i.w_s) (albedo_j[c]/pi) T^{k-1}_j[c], j = idx[i,s]; the call
 * takes G = dLoss/dT back through it:
 *   dP[n,C]         out: dLoss/dP (feed it to prtgs_precompute_transfer_backward for the geometry)
 *   d_albedo[n,3]   out: through the hit splats' albedo in every bounce
 *   d_normals[n,3]  out: through the receivers' cosines max(0, n_i.w_s) (raw normals; add the
 *                   transfer backward's own d_normals for the total)
 * Inputs (device): dirs[S,3], normals[n,3], albedo[n,3], P[n,C] and idx[n,S] of the forward call,
 * dT[n,3,C]; n_bounces as the forward's (0 or 1 = one bounce, at most 64). The intermediate bounces
 * are recomputed. Outputs are overwritten; the scatters use float atomics, so the last bits vary
 * from run to run. sh_order 1..6. Workspace: prtgs_bounce_backward_workspace_size
 * ((max(n_bounces, 1) + 2) n 3 C floats, one fewer for one bounce). idx entries >= n set
 * PRTGS_STATUS_BAD_INDEX and are skipped.
 */
size_t prtgs_bounce_backward_workspace_size(int64_t n, int32_t sh_order, int32_t n_bounces);
int prtgs_bounce_backward(int64_t n, int32_t sh_order, int32_t n_dirs, const float* dirs, const float* normals,
                          const float* albedo, const float* P, const int32_t* idx, int32_t n_bounces, const float* dT,
                          float* dP, float* d_albedo, float* d_normals, int32_t* status, void* workspace,
                          size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Visibility cache for training (Sec. 4.4-4.5): the same walk as prtgs_precompute_transfer with
 * flags = PRTGS_SHADOW, keeping every ray's visibility.
 *  V[n,S]   out (device): V_is, the transmittance of the ray from mu_i along w_s as in P below;
 *           0 where n_i.w_s <= 0 (the ray is not traced)
 *  P[n,C]   out (device, required): the shadowed diffuse transfer of the same rays (Eq. 29)
 * Geometry is frozen after the ray tracing (Sec. 4.4), so V serves every later training step's
 * prtgs_training_transfer. p->flags must be exactly PRTGS_SHADOW (else PRTGS_ERR_UNSUPPORTED);
 * sh_order 1..6; walk and packet_dirs as for prtgs_precompute_transfer.
 * Workspace: prtgs_visibility_workspace_size. Errors: as prtgs_precompute_transfer.
 */
size_t prtgs_visibility_workspace_size(int64_t n, const prtgs_transfer_params* p);
int prtgs_precompute_visibility(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                                float* V, float* P, int32_t* status, void* workspace, size_t workspace_bytes,
                                prtgs_stream_t stream);

/*
 * Training-stage transfer for one known view (Sec. 4.5, Eq. 28):
 *   t[i,c] = sum_s (4 pi/S) k_i(w_s, v_i) max(0, n_i.w_s) V[i,s] Y_c(w_s),
 *   v_i = (cam_pos - mu_i) / |cam_pos - mu_i|,
 * k the BRDF kernel of the glossy matrices (see prtgs_precompute_transfer's M; zero when
 * n_i.v_i <= 0). Eq. 28 is printed with the cosine and visibility of v; they are read as those
 * of the incident direction w_s, the view entering through the BRDF only, so that with f_s = 0
 * and metallic 0 the vector is the diffuse P of Eq. 29. Relight it like P (t_channels = 1):
 * colors = (albedo/pi) (t . L). No bounce term (the paper trades indirect accuracy for speed here).
 *   g: n, means, normals, roughness[n], metallic[n] (device)
 *   dirs[S,3], V[n,S] (device; V from prtgs_precompute_visibility); cam_pos[3] (HOST)
 *   t[n,C] out (device)
 * sh_order 1..6, S 1..1024. Workspace: prtgs_training_transfer_workspace_size (the SH table).
 * The backward takes dt[n,C] = dLoss/dt and writes d_roughness[n], d_metallic[n] (device;
 * overwritten, no atomics: deterministic). Gradients to the normals, means and visibility are
 * not formed (the normals are guided by the normal loss, Eq. 25; geometry is frozen).
 */
size_t prtgs_training_transfer_workspace_size(int32_t sh_order, int32_t n_dirs);
int prtgs_training_transfer(const prtgs_gaussians* g, int32_t sh_order, int32_t n_dirs, const float* dirs,
                            const float* V, const float* cam_pos, float* t, void* workspace, size_t workspace_bytes,
                            prtgs_stream_t stream);
int prtgs_training_transfer_backward(const prtgs_gaussians* g, int32_t sh_order, int32_t n_dirs, const float* dirs,
                                     const float* V, const float* cam_pos, const float* dt, float* d_roughness,
                                     float* d_metallic, void* workspace, size_t workspace_bytes,
                                     prtgs_stream_t stream);

/*
 * Relight (Eq. 14; glossy Eq. 41):
 *   colors[k,n,3] = (albedo_i/pi) * (T_i[c] . L[k,c,:]) per channel c,
 * with T [n,C] (t_channels = 1) or [n,3,C] (t_channels = 3). Glossy splats (n_glossy > 0,
 * glossy_ids[n_glossy] their Gaussian indices, M[n_glossy,C,C]) use
 *   t_eff[a] = sum_b M[a,b] Y_b(v_i), v_i = normalize(cam_pos - mean_i).
 * L[k,3,C] light SH per light and channel. sh_order 1..6. precision: PRTGS_PREC_*. The
 * tensor-core paths take every row through tcgen05 (one MMA chain of N = 3k for t_channels = 1,
 * three of N = k for t_channels = 3, K = C padded to 16 per K block: one block for orders 1-3,
 * 2-4 for orders 4-6) and then rewrite the glossy rows in FP32; they need 3k <= 256
 * (t_channels 1) or k <= 160 (t_channels 3: three accumulators in the 512 TMEM columns), and the
 * lights of every K block plus one K block of the rows in one CTA's shared memory (e.g. at order
 * 6 with BF16x3: k <= 64 for t_channels 3), otherwise
 * PRTGS_ERR_UNSUPPORTED.
 * cam_pos and means may be NULL when n_glossy == 0.
 * status (device int32, may be NULL) receives PRTGS_STATUS_TIMEOUT when a tensor-core wait gave
 * up; tc_wait_polls bounds that wait (PRTGS_TC_WAIT_POLLS; 0 gives up at once, which exercises the
 * failure path). Both are ignored by PRTGS_PREC_FP32.
 */
size_t prtgs_relight_workspace_size(int64_t n, int32_t sh_order, int32_t k, int32_t precision);
int prtgs_relight(int64_t n, int32_t sh_order, const float* T, int32_t t_channels, const float* albedo,
                  int64_t n_glossy, const int32_t* glossy_ids, const float* M, const float* means,
                  const float* cam_pos, const float* L, int32_t k, int32_t precision, float* colors,
                  int32_t* status, uint32_t tc_wait_polls, void* workspace, size_t workspace_bytes,
                  prtgs_stream_t stream);

/*
 * Relight of many scenes in one launch: scene b holds Gaussians scene_offsets[b] ..
 * scene_offsets[b+1] (device int64 [n_scenes+1]) and has its own k lights
 * L[b,k,3,C] (device). colors[3 k n] holds one contiguous [k, n_b, 3] block per scene,
 * scene b's block starting at float 3 k scene_offsets[b] (the input layout of prtgs_render
 * for that scene). No workspace. Tensor-core precisions need 3k <= 256 (t_channels 1) or
 * k <= 160 (t_channels 3). status, tc_wait_polls: as prtgs_relight.
 */
int prtgs_relight_batched(int64_t n, int32_t sh_order, const float* T, int32_t t_channels, const float* albedo,
                          const int64_t* scene_offsets, int32_t n_scenes, const float* L, int32_t k,
                          int32_t precision, float* colors, int32_t* status, uint32_t tc_wait_polls,
                          prtgs_stream_t stream);

/*
 * Relight backward (diffuse splats; glossy rows of dcolors must be zero or are ignored).
 *   dcolors[k,n,3] in; d_albedo[n,3] out (overwritten); dT[n,t_channels,C] out (may be NULL);
 *   dL[k,3,C] out (overwritten; deterministic two-pass reduction over n).
 */
size_t prtgs_relight_backward_workspace_size(int64_t n, int32_t sh_order, int32_t k);
int prtgs_relight_backward(int64_t n, int32_t sh_order, const float* T, int32_t t_channels, const float* albedo,
                           const float* L, int32_t k, const float* dcolors, float* d_albedo, float* dT, float* dL,
                           void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Relight backward that allocates nothing and takes no workspace. The paper has no
 * counterpart: this is a convenience for callers that cannot give the library device
 * memory, e.g. a host application that owns every device allocation through its own fixed
 * pool, or a latency-critical loop that must not call cudaMalloc. Same arguments and results
 * as prtgs_relight_backward.
 *  * Its scratch is a fixed 1 MiB array in the library's device memory
 *    (prtgs_relight_backward_noalloc_max_bytes()), present on every GPU that loads the
 *    library until the process exits. Problems needing more scratch than that
 *    (ceil(n / 2048) * k * 3 * C floats) return PRTGS_ERR_UNSUPPORTED.
 *  * The first call on a device looks up the array's device address on the current device;
 *    make that first call before any stream capture.
 *  * Every call shares the one array and leaves its partial sums in it (the kernels
 *    overwrite all they read, so nothing needs clearing). Calls that overlap on the GPU
 *    (different streams, or different host threads) race on it.
 */
size_t prtgs_relight_backward_noalloc_max_bytes(void);
int prtgs_relight_backward_noalloc(int64_t n, int32_t sh_order, const float* T, int32_t t_channels,
                                   const float* albedo, const float* L, int32_t k, const float* dcolors,
                                   float* d_albedo, float* dT, float* dL, prtgs_stream_t stream);

/*
 * Pinhole camera. world -> camera: x_c = rot * x_w + trans (rot row-major, camera x right,
 * y down, z forward). Pixel (px,py) has its centre at (fx x_c/z_c + cx, fy y_c/z_c + cy).
 */
typedef struct prtgs_camera {
  float rot[9];
  float trans[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_plane;
  float pos[3];
} prtgs_camera;

/*
 * Render state: per-Gaussian projection results, the sorted (tile, depth) pairs and the
 * per-pixel bookkeeping that the backward pass reuses. Lives in one caller buffer laid out
 * by prtgs_render_state_init(); max_pairs bounds the number of (Gaussian, tile) pairs.
 */
typedef struct prtgs_render_state {
  int64_t n;
  int64_t max_pairs;
  int32_t width, height, tiles_x, tiles_y;
  float* mean2d;       /* [n,2] */
  float* conic_op;     /* [n,4] conic a,b,c and opacity */
  float* depth;        /* [n] */
  int32_t* radius;     /* [n] (0 = culled) */
  uint32_t* tiles_touched; /* [n] then inclusive prefix sums */
  uint64_t* pair_keys; /* [max_pairs] tile << 32 | depth bits, sorted */
  int32_t* pair_ids;   /* [max_pairs] Gaussian index per sorted pair */
  uint32_t* ranges;    /* [tiles, 2] start, end of each tile's run of pairs */
  float* final_T;      /* [H,W] */
  int32_t* n_contrib;  /* [H,W] one past the last contributing pair of each pixel's tile list */
  /* (batched states: ranges [n_scenes * tiles, 2], final_T and n_contrib [n_scenes, H, W]) */
  uint32_t* n_pairs;   /* [1] number of pairs produced */
  int32_t n_scenes;    /* scenes whose tiles, final_T and n_contrib the state holds (1 unless batched) */
} prtgs_render_state;

size_t prtgs_render_state_bytes(int64_t n, int32_t width, int32_t height, int64_t max_pairs);
int prtgs_render_state_init(void* buffer, size_t bytes, int64_t n, int32_t width, int32_t height,
                            int64_t max_pairs, prtgs_render_state* out);
size_t prtgs_render_workspace_size(int64_t n, int32_t width, int32_t height, int64_t max_pairs);

/*
 * Splat render of k relit colour sets (Eq. 3 projection, Eq. 4 front-to-back blending;
 * 3DGS rasteriser rules: near 0.2, 0.3 px^2 dilation, 3-sigma radius, 16x16 tiles,
 * alpha = min(0.99, opacity e^power), skip alpha < 1/255, stop before T < 1e-4).
 *   colors[k,n,3], bg[3] (device), image[k,3,H,W] out. The geometry is shared by the k
 *   images; each pixel's blend is evaluated once for all k colour sets.
 * status: PRTGS_STATUS_CAPACITY when max_pairs is exceeded (the image is then incomplete).
 */
int prtgs_render(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam,
                 const float* bg, float* image, prtgs_render_state* st, int32_t* status, void* workspace,
                 size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Relight of many lights in pixel space (the composite of Eq. 4 is linear in the splat colours
 * of Eq. 14): the splats' features (rho_i/pi) T_i (glossy splats: (rho_i/pi) M_i Y(v_i), Eq. 41,
 * v_i towards cam->pos) are composited once as C "lights" into a transfer image TI[C,3,H,W]
 * (this fills *st like prtgs_render), then every light's image is
 *   image[l,c,p] = sum_m TI[m,c,p] L[l,c,m] + bg[c] final_T[p]
 * one [H*W x C] x [C x k] contraction per channel: on tcgen05 (PRTGS_PREC_BF16X3 / _BF16, k <= 160)
 * or FP32 CUDA cores (k <= 256). Same result as prtgs_relight + prtgs_render up to rounding, at
 * the cost of one 3C-channel composite instead of k 3-channel ones.
 *   T[n,t_channels,C], albedo from g; glossy as prtgs_relight; L[k,3,C]; bg[3] (device);
 *   image[k,3,H,W] out. Workspace: prtgs_render_relit_workspace_size. status: as prtgs_render, plus
 *   PRTGS_STATUS_TIMEOUT from the tensor-core contraction; tc_wait_polls: as prtgs_relight.
 */
size_t prtgs_render_relit_workspace_size(int64_t n, int32_t sh_order, int32_t width, int32_t height,
                                         int64_t max_pairs);
int prtgs_render_relit(const prtgs_gaussians* g, int32_t sh_order, const float* T, int32_t t_channels,
                       int64_t n_glossy, const int32_t* glossy_ids, const float* M, const float* L, int32_t k,
                       int32_t precision, const prtgs_camera* cam, const float* bg, float* image,
                       prtgs_render_state* st, int32_t* status, uint32_t tc_wait_polls, void* workspace,
                       size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Depth and normal maps of the splats (Eq. 23 and Eq. 25): front-to-back composites, with the
 * blending weights of prtgs_render, of each splat's view-space depth d_i (the z of its mean in
 * camera space) and of its normal n_i as given. Background 0. Fills *st like prtgs_render.
 *   depth[H,W], normal[3,H,W] out (device). Workspace: prtgs_render_geometry_workspace_size.
 */
size_t prtgs_render_geometry_workspace_size(int64_t n, int32_t width, int32_t height, int64_t max_pairs);
int prtgs_render_geometry(const prtgs_gaussians* g, const prtgs_camera* cam, float* depth, float* normal,
                          prtgs_render_state* st, int32_t* status, void* workspace, size_t workspace_bytes,
                          prtgs_stream_t stream);

/*
 * Pseudo-normal map of a depth map (Sec. 4.3, Eq. 24: "computed from D"). Each pixel is
 * back-projected with the camera (pixel centre (x, y) at depth D: camera point
 * D ((x - cx)/fx, (y - cy)/fy, 1)) and N' is the unit normal of the central differences
 * (X(x,y+1) - X(x,y-1)) x (X(x+1,y) - X(x-1,y)), which faces the camera, rotated to world space.
 *   depth[H,W] in (device; e.g. from prtgs_render_geometry), pseudo[3,H,W] out (device)
 * N' = 0 on the image border and wherever the pixel or one of its four neighbours has depth <= 0
 * (no splat there). Only cam->rot, fx, fy, cx, cy, width and height are used.
 */
int prtgs_pseudo_normal(const prtgs_camera* cam, const float* depth, float* pseudo, prtgs_stream_t stream);

/*
 * Normal loss (Sec. 4.3, Eq. 25): L = ||N - N'||, the Euclidean norm of the difference of the
 * two [3,H,W] maps over the pixels where N' is defined (N' != 0), and dL/dN = (N - N') / L on
 * those pixels (0 elsewhere and when L = 0). N' is the guide and gets no gradient. The sum is a
 * fixed-order reduction, so the result is the same from run to run.
 *   normal[3,H,W], pseudo[3,H,W] in (device); loss[1] out (device); d_normal[3,H,W] out
 *   (device, may be NULL). Feed d_normal to prtgs_render_backward with the normals as the
 *   colours (k = 1, bg 0) and the state of prtgs_render_geometry to reach the splats' normals
 *   (and geometry) through Eq. 25's composite.
 * Workspace: prtgs_normal_loss_workspace_size.
 */
size_t prtgs_normal_loss_workspace_size(int32_t width, int32_t height);
int prtgs_normal_loss(int32_t width, int32_t height, const float* normal, const float* pseudo, float* loss,
                      float* d_normal, void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Render backward: dimage[k,3,H,W] in; gradients out (overwritten): d_means[n,3],
 * d_scales[n,3], d_quats[n,4], d_opacity[n], d_colors[k,n,3]. Uses the state written by the
 * matching prtgs_render call. Gradients of the discrete decisions (culling, tile binning,
 * skips, early stop) are zero; the alpha clamp at 0.99 has zero derivative.
 */
size_t prtgs_render_backward_workspace_size(int64_t n, int32_t k);
int prtgs_render_backward(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam,
                          const float* bg, const prtgs_render_state* st, const float* dimage, float* d_means,
                          float* d_scales, float* d_quats, float* d_opacity, float* d_colors, void* workspace,
                          size_t workspace_bytes, prtgs_stream_t stream);

/*
 * L2 image loss used by the differentiable relight: loss = mean((image - target)^2) and
 * dimage = 2 (image - target) / count. loss[1], dimage[count] device outputs.
 */
size_t prtgs_l2_loss_workspace_size(int64_t count);
int prtgs_l2_loss(const float* image, const float* target, int64_t count, float* loss, float* dimage,
                  void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Batched scenes (many scenes of uneven size in one launch per stage; Sec. 5's scenes relit
 * together). Scene b holds Gaussians scene_offsets[b] .. scene_offsets[b+1] (device int64
 * [n_scenes+1], n_scenes <= 128) and has its own camera cams[b] (HOST array [n_scenes]; every
 * camera has the same width and height); the cameras are passed by value to the kernels, so
 * these calls copy nothing to the device and can be captured in a CUDA graph.
 *   colors   the layout of prtgs_relight_batched: scene b's [k, n_b, 3] block at 3 k offsets[b]
 *   images   [n_scenes, k, 3, H, W]
 *   st       a state laid out by prtgs_render_state_init_batched for the same n_scenes; the
 *            single-scene calls reject it (and the batched calls reject single-scene states)
 * Tiles are numbered scene-major, so one preprocess, one duplicate, one sort, one range pass
 * and one composite launch cover every scene; the results equal prtgs_render per scene.
 */
size_t prtgs_render_state_bytes_batched(int64_t n, int32_t n_scenes, int32_t width, int32_t height,
                                        int64_t max_pairs);
int prtgs_render_state_init_batched(void* buffer, size_t bytes, int64_t n, int32_t n_scenes, int32_t width,
                                    int32_t height, int64_t max_pairs, prtgs_render_state* out);
size_t prtgs_render_batched_workspace_size(int64_t n, int32_t n_scenes, int32_t width, int32_t height,
                                           int64_t max_pairs);
int prtgs_render_batched(const prtgs_gaussians* g, const int64_t* scene_offsets, int32_t n_scenes,
                         const float* colors, int32_t k, const prtgs_camera* cams, const float* bg, float* images,
                         prtgs_render_state* st, int32_t* status, void* workspace, size_t workspace_bytes,
                         prtgs_stream_t stream);

/* Backward of prtgs_render_batched: dimages [n_scenes, k, 3, H, W] in; d_colors in the batched
 * colour layout, the other gradients per Gaussian (overwritten). As prtgs_render_backward. */
size_t prtgs_render_backward_batched_workspace_size(int64_t n, int32_t k);
int prtgs_render_backward_batched(const prtgs_gaussians* g, const int64_t* scene_offsets, int32_t n_scenes,
                                  const float* colors, int32_t k, const prtgs_camera* cams, const float* bg,
                                  const prtgs_render_state* st, const float* dimages, float* d_means, float* d_scales,
                                  float* d_quats, float* d_opacity, float* d_colors, void* workspace,
                                  size_t workspace_bytes, prtgs_stream_t stream);

/* Per-scene L2 losses of n_scenes images of `count` elements each (images and targets
 * [n_scenes, count]): losses[b] = mean over scene b, dimages = 2 (image - target) / count. */
size_t prtgs_l2_loss_batched_workspace_size(int64_t count, int32_t n_scenes);
int prtgs_l2_loss_batched(const float* images, const float* targets, int64_t count, int32_t n_scenes, float* losses,
                          float* dimages, void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/* Relight backward of prtgs_relight_batched (diffuse): dcolors in the batched colour layout,
 * L[n_scenes, k, 3, C]; d_albedo[n,3], dT[n,t_channels,C] (may be NULL) and dL[n_scenes, k, 3, C]
 * out (overwritten; dL a deterministic per-scene reduction). */
size_t prtgs_relight_backward_batched_workspace_size(int64_t n, int32_t n_scenes, int32_t sh_order, int32_t k);
int prtgs_relight_backward_batched(int64_t n, int32_t sh_order, const float* T, int32_t t_channels,
                                   const float* albedo, const int64_t* scene_offsets, int32_t n_scenes, const float* L,
                                   int32_t k, const float* dcolors, float* d_albedo, float* dT, float* dL,
                                   void* workspace, size_t workspace_bytes, prtgs_stream_t stream);

/*
 * Autotuning of launch variants (the work-tile shapes and paths that give the same results).
 * prtgs_autotune times each variant of one call on the caller's own inputs (one untimed run, then
 * `repeats` timed runs, CUDA events on `stream`; the call synchronises the stream and overwrites
 * the call's outputs), stores the fastest in *best and writes a JSON report to out_json (host,
 * json_bytes >= 512 suggested; PRTGS_ERR_INVALID_ARG if it does not fit):
 *   {"kernel": ..., "variant": ..., "shape": {...}, "ms": {"<variant>": <mean ms>, ...}, "best": ...}
 *   PRTGS_TUNE_TRANSFER   args: prtgs_tune_transfer (the arguments of prtgs_precompute_transfer);
 *                         variant: the packet walk with packet_dirs in {1, 2, 4, 8, 16, 32}, or
 *                         the per-ray walk, reported as packet_dirs 0 (use walk = 1 then); the
 *                         workspace must hold both walks' (the larger prtgs_transfer_workspace_size
 *                         of walk 0 and walk 1)
 *   PRTGS_TUNE_RELIGHT    args: prtgs_tune_relight (the arguments of prtgs_relight_batched; one
 *                         scene is scene_offsets {0, n}); variant: precision among the
 *                         FP32-accurate ones, PRTGS_PREC_FP32 and (when the shape fits the tensor
 *                         cores) PRTGS_PREC_BF16X3
 * Errors of the timed call are returned as they are.
 */
#define PRTGS_TUNE_TRANSFER 1
#define PRTGS_TUNE_RELIGHT 2

typedef struct prtgs_tune_transfer {
  const prtgs_gaussians* g;
  const prtgs_bvh* bvh;
  prtgs_transfer_params params;
  float* P;
  float* T;
  int32_t* idx;
  float* M;
  int64_t n_glossy;
  int32_t* status;
  void* workspace;
  size_t workspace_bytes;
} prtgs_tune_transfer;

typedef struct prtgs_tune_relight {
  int64_t n;
  int32_t sh_order;
  int32_t t_channels;
  const float* T;
  const float* albedo;
  const int64_t* scene_offsets;
  int32_t n_scenes;
  int32_t k;
  const float* L;
  float* colors;
  int32_t* status;
} prtgs_tune_relight;

int prtgs_autotune(int32_t kernel_id, const void* args, int32_t repeats, prtgs_stream_t stream, int32_t* best,
                   char* out_json, size_t json_bytes);

/*
 * CUDA-graph capture of a sequence of library calls (the batched step replayed with one launch
 * from the host). Between prtgs_graph_begin(stream) and prtgs_graph_end(stream, &graph), calls
 * enqueued on `stream` are recorded instead of run; prtgs_graph_launch replays them on a stream,
 * with the pointers and scalars they were recorded with (so their buffers and workspaces must
 * stay allocated), and prtgs_graph_destroy frees the graph. Every call that enqueues work can be
 * recorded, except prtgs_read_status (it synchronises) and the first call of
 * prtgs_relight_backward_noalloc on a device (it looks up its scratch address). The legacy
 * default stream (NULL) cannot be captured: PRTGS_ERR_INVALID_ARG. A CUDA error while capturing
 * or instantiating: PRTGS_ERR_CUDA. Instantiation takes driver resources, no device memory of
 * the caller.
 */
typedef struct prtgs_graph_s* prtgs_graph_t;
int prtgs_graph_begin(prtgs_stream_t stream);
int prtgs_graph_end(prtgs_stream_t stream, prtgs_graph_t* graph);
int prtgs_graph_launch(prtgs_graph_t graph, prtgs_stream_t stream);
int prtgs_graph_destroy(prtgs_graph_t graph);

/* Read and clear a device status word (synchronises `stream`). Returns the bits or a
 * negative PRTGS_ERR_* code. */
int prtgs_read_status(int32_t* status, prtgs_stream_t stream);

const char* prtgs_strerror(int code);
int prtgs_version(void);

/* Kernel launches the library has issued in this process so far (every device and thread; a
 * CUDA-graph replay relaunches captured kernels without passing through the library, so it
 * does not count). Host only; for measuring how many kernels a sequence of calls runs. */
unsigned long long prtgs_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PRTGS_H */
