/*
 * gblb surrogate — BF16 tensor-core kernels of a small 3D convolutional
 * neural operator that advances the macroscopic fields (rho, u, theta) of
 * the RD3Q41 solver many lattice Boltzmann steps at a time.  C ABI.
 *
 * The paper (arXiv:1909.08406) has no learned component; this module is the
 * project's addition: a network trained on data the solver generates, with
 * the plain lattice Boltzmann method as its fallback and as the arbiter of its
 * rollout error.
 *
 * Tensors are channels-last, periodic volumes: x[b][z][y][x][c] (NDHWC),
 * with nx = 64 and ny a multiple of 4 (a CTA owns whole 64-voxel rows), any nz.
 * Activations and weights are BF16; accumulation is FP32.  Weights are
 * w[cout][tap][cin] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1) for a 3x3x3
 * periodic ("circular") convolution
 *     z[v][co] = bias[co] + sum_{tap, ci} w[co][tap][ci] * x[v + d(tap)][ci].
 * Channel counts: cin in {16, 32}, cout in {16, 32} (zero-padded channels
 * carry zeros).  All pointers are device pointers on the current device; all
 * work is enqueued on `stream` (cudaStream_t, NULL = legacy default stream).
 * Every call returns 0 on success, -1 for a bad argument (unsupported shape or
 * null pointer) and -3 for a CUDA launch error (cudaGetLastError).  No call
 * allocates memory; scratch buffers are caller-provided and sized by the
 * *_bytes queries.
 */
#ifndef GBLB_SURROGATE_H
#define GBLB_SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int batch, nz, ny, nx;  /* volume: batch x nz x ny x nx voxels */
    int xper;               /* convolutions: the period along x, 0 (= nx, the periodic row) or 32,
                               16, 8: each row holds nx / xper independent periodic segments, the
                               d-layout of sg_relabel with xper = 64 / d; other values give -1 */
} sg_shape;

/* Activation of the forward convolution epilogue. */
#define SG_ACT_NONE 0
#define SG_ACT_GELU 1 /* GELU with the Gaussian CDF: g(z) = z * Phi(z) */

/* Forward convolution with fused epilogue:
 *   z = conv(x, w) + bias                         (FP32)
 *   y = act(z) + (res_in ? x : 0) + (add ? add : 0), stored as BF16 in y
 * res_in requires cin == cout.  z_out (FP32, [voxels][cout]) receives z when
 * non-NULL (kept for the backward pass).  add (BF16, same layout as y) may be
 * NULL.  x: [voxels][cin] BF16, w: [cout][27][cin] BF16, bias: [cout] FP32. */
int sg_conv3d_fwd(sg_shape s, int cin, int cout, const void *x, const void *w, const float *bias, int act,
                  int res_in, const void *add, float *z_out, void *y, void *stream);

/* Kernel of the two convolution entry points above and of sg_conv3d_wgrad:
 *   SG_CONV_TCGEN05  (default) 5th-generation tensor cores: tcgen05.mma with
 *                    the FP32 accumulator in tensor memory, M = 128 voxels,
 *                    K = 16 per instruction; the forward kernel puts the
 *                    three x taps of a (dz, dy) side by side in N = 3 cout
 *                    and combines them, shifted by one voxel, in its epilogue.
 *                    Persistent CTAs with the weights resident in shared
 *                    memory.  A wait for the tensor cores that runs out of
 *                    time (~1 s) ends the kernel and is reported by sg_status.
 *   SG_CONV_MMA_SYNC warp-level mma.sync.m16n8k16.
 * Returns the previous setting, or -1 for an unknown value.  Process-wide. */
#define SG_CONV_MMA_SYNC 0
#define SG_CONV_TCGEN05 1
int sg_set_conv_impl(int impl);

/* Synchronises `stream` and returns 0, or -6 if a tensor-core wait of a
 * convolution ran out of time since the last call (the flag is then
 * cleared), or -3 for a CUDA error. */
int sg_status(void *stream);

/* Input-gradient form of the convolution: y = conv(x, w) + add, with y and
 * add (may be NULL) FP32 [voxels][cout]. */
int sg_conv3d_fwd_f32(sg_shape s, int cin, int cout, const void *x, const void *w, const float *add, float *y,
                      void *stream);

/* dz = dy * act'(z) (BF16 out) for act = SG_ACT_GELU, dz = dy for SG_ACT_NONE.
 * dy: FP32 [n], z: FP32 [n], dz: BF16 [n]; n elements. */
int sg_act_backward(int64_t n, int act, const float *dy, const float *z, void *dz, void *stream);

/* Weights of the transposed convolution (the input gradient is a forward
 * convolution with these): wt[ci][tap'][co] = w[co][26 - tap'][ci]. */
int sg_transpose_weights(int cin, int cout, const void *w, void *wt, void *stream);

/* Weight and bias gradients: dw[co][tap][ci] = sum_v dz[v][co] x[v + d(tap)][ci],
 * db[co] = sum_v dz[v][co] (FP32 out, overwritten).  Deterministic: partial
 * sums per CTA (SG_CONV_TCGEN05) or per voxel partition (SG_CONV_MMA_SYNC) in
 * `scratch` (sg_wgrad_scratch_bytes, enough for either), reduced in a fixed
 * order.  SG_CONV_TCGEN05: per row of 64 voxels a tcgen05.mma GEMM over the
 * row's voxels, with A = the x rows of the 9 (dz, dy) neighbours (M = 9 cin in
 * tiles of 128) and B = the dz row in three copies shifted by dx (N =
 * 3 cout), both read by TMA in their own [voxel][channel] layout (MN-major
 * operands); the FP32 accumulators stay in tensor memory over all rows of a
 * CTA.  Its timeouts are reported by sg_status, as the forward kernel's. */
int64_t sg_wgrad_scratch_bytes(sg_shape s, int cin, int cout);
int sg_conv3d_wgrad(sg_shape s, int cin, int cout, const void *x, const void *dz, float *dw, float *db,
                    void *scratch, void *stream);

/* Mean-squared error over the first nch of c channels of [voxels][c] BF16
 * tensors pred and target: loss (FP32, device, 1 value) and
 * dpred = 2 (pred - target) / (voxels * nch) as FP32 [voxels][c] (0 for the
 * other channels).  scratch: sg_reduce_scratch_bytes. */
int64_t sg_reduce_scratch_bytes(int64_t n);
int sg_mse(int64_t voxels, int c, int nch, const void *pred, const void *target, float *loss, float *dpred,
           void *scratch, void *stream);

/* Relative L2 distance ||a - b|| / ||b|| over the first nch of c channels of
 * [voxels][c] BF16 tensors, per batch item: out[b] (FP32, device). */
int sg_rel_l2(sg_shape s, int c, int nch, const void *a, const void *b, float *out, void *scratch, void *stream);

/* Adam step on FP32 master weights p with gradient g (moments m, v, step t
 * >= 1), then p rounded to BF16 into p16 (may be NULL). */
int sg_adam(int64_t n, float *p, const float *g, float *m, float *v, void *p16, float lr, float beta1, float beta2,
            float eps, int t, void *stream);

/* Fields <-> network channels.  pack: solver fields on the A sub-lattice
 * (rho[2][nz][ny][nx], u[3][2][..], theta[2][..], float64, as lb_get_moments
 * writes them) -> x[b][z][y][x][c] BF16 with c = 16 channels
 * (rho-1)/s0, u/s1 (3), (theta/theta0-1)/s2, zeros; one batch item `item`.
 * unpack: channels 0..4 of item `item` -> float64 fields on both
 * sub-lattices; a B node (cell + (1/2,1/2,1/2)) takes the mean of its eight
 * A neighbours.  scales (3 floats: s0, s1, s2) is host memory. */
/* Dilated convolutions.  The periodic 3x3x3 convolution with taps d voxels apart (dilation d in
 * {1, 2, 4, 8}) of a volume s (nx = 64; nz, ny multiples of d) equals the plain convolution of
 * its d-layout: the volume of batch * d^2 items of (nz / d) x (ny / d) x 64 voxels with
 * xper = 64 / d, in which voxel (b, z, y, x) sits at
 *     b' = (b d + z mod d) d + y mod d,  z' = z / d,  y' = y / d,  x' = (x mod d)(64 / d) + x / d.
 * Its neighbours at +-1 along x' (inside the x segment), y' and z' are the volume's at +-d, all
 * periodic.  sg_relabel copies src, in the df-layout of s, to dst in the dt-layout (df, dt in
 * {1, 2, 4, 8}; 1 is the volume itself).  Element-wise operations commute with it, so a network
 * keeps each layer's activations in its layer's layout.  bytes_per_voxel: channels x element size,
 * 16 x a power of two up to 4096; fewer than 2^31 16-byte chunks in all; src and dst 16-byte
 * aligned, distinct.  s.xper is ignored. */
int sg_relabel(sg_shape s, int bytes_per_voxel, int df, int dt, const void *src, void *dst, void *stream);

int sg_pack_fields(sg_shape s, int item, const double *rho, const double *u, const double *theta, double theta0,
                   const float *scales, void *x, void *stream);
int sg_unpack_fields(sg_shape s, int item, const void *x, double theta0, const float *scales, double *rho, double *u,
                     double *theta, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBLB_SURROGATE_H */
