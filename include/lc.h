/*
 * lc.h -- C ABI of the learned coarse-to-fine corrector (sm_103a kernels).
 *
 * The paper resolves coastal and small-scale detail with patch-based AMR
 * (Sec. 4, Berger-Oliger-Colella).  This corrector stands in for the finest
 * refinement level: from a coarse state (eta, hu, hv, b, phi_T) it predicts the
 * fine-grid (refinement ratio r) correction of eta, hu, hv relative to the
 * piecewise-constant prolongation of the coarse state.  It is not part of the
 * paper's method; the fine solve stays available as the fallback wherever the
 * corrector's error indicator exceeds its bound.
 *
 * Network: `depth` 3x3 convolutions (padding 1), `width` channels, ReLU between
 * layers, last layer r*r*nout channels (pixel-shuffled to the fine grid).
 * Weights are kept as FP32 master copies for Adam and used as BF16 in the forward
 * and backward passes; the convolutions (forward and input gradient) are
 * implicit GEMMs on the fifth-generation tensor cores (tcgen05.mma: BF16
 * operands from shared memory, FP32 accumulators in tensor memory), the weight
 * gradients on the warp-level tensor-core instructions (mma.sync, BF16
 * operands, FP32 accumulation).
 *
 * Layouts: the network input and output are channel-major [C][H][W] float32 in
 * device memory (batch 1); hidden activations live inside the handle.  Parameters are packed per layer as weights [cout][cin][3][3]
 * then bias [cout].  Every entry point returns 0 or a negative SGN-style code
 * (-1 invalid argument, -2 allocation failure, -3 CUDA error) and issues its work
 * on the stream given to lc_create; entry points that return host values
 * synchronise that stream.
 */
#ifndef LC_H
#define LC_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lc_net lc_net;

/* Create a network with cin input channels, `width` hidden channels, `depth`
 * layers (>= 2) and cout = r*r*nout output channels (each at most 48, the
 * tensor-core kernels' limit; cout * max_hw below 2^31); He-initialised from
 * `seed`.  max_hw bounds H*W of the inputs later passed (workspace is sized for
 * it).  The convolutions multiply BF16 operands on the tensor cores with FP32
 * accumulation: the BF16 copy of the weights, and the layer inputs and
 * gradients rounded to BF16 (hidden activations and their gradients are kept
 * in BF16); biases, master weights, the output and the loss are FP32. */
int lc_create(int cin, int width, int depth, int cout, long max_hw, unsigned long long seed,
              void* cuda_stream, lc_net** out);
void lc_destroy(lc_net* n);
long lc_num_params(lc_net* n);
/* FP32 master parameters to / from host memory (n floats, packed as above). */
int lc_get_params(lc_net* n, float* host, long count);
int lc_set_params(lc_net* n, const float* host, long count);

/* y[cout][H][W] = net(x[cin][H][W]); device pointers. */
int lc_forward(lc_net* n, const float* x_dev, int H, int W, float* y_dev);

/* Wait for the work issued on the handle's stream; 0, -3 on a CUDA error, or
 * -4 when a convolution gave up waiting for its tensor-core instructions (each
 * such wait is bounded to about two seconds; the kernel then releases its
 * tensor memory and ends, leaving its output incomplete).  lc_train_step
 * returns this value too. */
int lc_sync(lc_net* n);

/* Loss and gradients for one sample.  target_dev: fine-grid target
 * [nout][r*H][r*W]; field_w: nout host weights.  Loss = sum over fields f of
 * field_w[f] * mean over fine cells of (shuffle(y)_f - target_f)^2.  With
 * lr > 0 an Adam step (beta1 0.9, beta2 0.999, eps 1e-8) follows; with lr == 0
 * the gradient is left in place and, when grad_host is not NULL, copied out
 * (lc_num_params floats).  *loss (host) receives the loss before the update. */
int lc_train_step(lc_net* n, const float* x_dev, const float* target_dev, int H, int W, int r, int nout,
                  const float* field_w, float lr, double* loss, float* grad_host);

/* Data kernels on dense double fields of the solver (row-major, x fastest). */
/* x[5][Hc][Wc] = (eta/s_eta, hu/s_q, hv/s_q, b/s_b, phi) from the coarse state's
 * first three fields (q: 3*Hc*Wc doubles), b and phi (Hc*Wc each). */
int lc_make_input(const double* q_dev, const double* b_dev, const unsigned char* phi_dev, int Hc, int Wc,
                  float s_eta, float s_q, float s_b, float* x_dev, void* cuda_stream);
/* target[3][r Hc][r Wc] = (q_fine - P q_coarse) / s, P the piecewise-constant
 * prolongation; s = (s_eta, s_q, s_q).  bf_dev (fine bathymetry, r Hc x r Wc)
 * and bc_dev (coarse bathymetry, Hc x Wc), either may be NULL: the surface
 * target is 0 on fine cells with bf >= 0 or whose coarse cell has bc >= 0 (land
 * at or above the still level, where the surface is bathymetry rather than a
 * wave), so the network is not trained to reproduce sub-grid land elevation. */
int lc_make_target(const double* qf_dev, const double* qc_dev, const double* bf_dev, const double* bc_dev, int Hc,
                   int Wc, int r, float s_eta, float s_q, float* t_dev, void* cuda_stream);
/* out[3][r Hc][r Wc] = P q_coarse + s * shuffle(y) (y = lc_forward output); with
 * use_net == 0 the plain prolongation. */
int lc_apply(const double* qc_dev, const float* y_dev, int Hc, int Wc, int r, float s_eta, float s_q,
             int use_net, double* out_dev, void* cuda_stream);
/* Fallback tiles of the learned form: the paper's refinement flag (a surface
 * jump between neighbouring cells, Sec. 6.3) evaluated on a coarse state.
 * eta_dev, b_dev: surface and bathymetry, H x W doubles on the device.  A cell
 * is flagged when it and a face neighbour are both deeper than hmin
 * (eta - b > hmin) and their surfaces differ by more than thr.  The grid is cut
 * into tiles of `tile` cells from the low corner in each direction, a one-cell
 * remainder joined to the tile before it (so nt = 1 when n < tile + 2, else
 * n / tile, plus one when n % tile >= 2); sel_dev[ty * ntx + tx] (device,
 * ntx * nty bytes, caller-owned) becomes 1 when a flagged cell lies within
 * Chebyshev distance `buffer` of tile (tx, ty) and none of the tile's cells is
 * shallower than hmin, else 0.  Asynchronous on cuda_stream; -1 for invalid
 * arguments (tile < 2, buffer < 0, thr < 0 or not finite). */
int lc_fallback_tiles(const double* eta_dev, const double* b_dev, int H, int W, double thr, double hmin, int tile,
                      int buffer, unsigned char* sel_dev, void* cuda_stream);
/* Restriction: coarse[Hc][Wc] = mean of each r x r block of fine[r Hc][r Wc]. */
int lc_restrict(const double* fine_dev, int Hc, int Wc, int r, double* coarse_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
