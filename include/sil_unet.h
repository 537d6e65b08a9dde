/*
 * sil_unet.h -- C ABI of the U-Net inference on filtered chips (libsil.so).
 *
 * Sec. III-C "U-Net Model Inferencing" of arXiv 2403.13135 cuts the scenes
 * into 256 x 256 chips, filters them and feeds them to a U-Net that labels
 * every pixel as a sea-ice class.  The paper names the model (a U-Net,
 * Sec. III-C "U-Net Model Training") but not its widths, and its trained
 * weights are not available, so this module runs the network with weights
 * the caller supplies (random ones in the tests and the benchmark) and is
 * measured for throughput.  The architecture read from the paper and fixed
 * here:
 *
 *   input    R, G, B bytes of a 256 x 256 chip, each scaled by 1/256
 *   encoder  for level l = 0..depth-1: two 3x3 convolutions (zero padding
 *            1, bias, ReLU) of width F 2^l, then 2x2 max pooling
 *   bottom   two 3x3 convolutions of width F 2^depth
 *   decoder  for l = depth-1..0: 2x2 stride-2 transposed convolution
 *            (bias, no activation) to width F 2^l, concatenation
 *            [upsampled, encoder output of level l], two 3x3 convolutions
 *   head     1x1 convolution to 3 class scores (float32); label = index of
 *            the largest score, the first on ties (0 thick ice, 1 thin ice,
 *            2 open water)
 *
 * The input may be the filtered chip (sil_unet_forward_filtered), as in the
 * paper's workflow.
 *
 * Every activation is stored as bfloat16 (round to nearest even) in
 * channels-last layout; products are bfloat16 x bfloat16 summed in float32
 * on the tensor cores.
 *
 * Conventions are those of sil.h: device pointers unless stated otherwise,
 * asynchronous on the given stream, arguments validated on the host
 * (SIL_EINVAL, nothing launched), CUDA failures SIL_ECUDA.
 */
#ifndef SIL_UNET_H_
#define SIL_UNET_H_

#include <stdint.h>

#include "sil.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sil_unet sil_unet;

typedef struct sil_unet_config {
  int32_t base_width; /* F: 16, 32 or 64 (default 32) */
  int32_t depth;      /* encoder levels: 1..5 (default 5: the paper's 28
                         convolution layers, Sec. III-C "U-Net Training") */
  int32_t max_batch;  /* chips per sil_unet_forward call: 1..4096 (default 32) */
} sil_unet_config;

/* Layer kinds of sil_unet_layer_shape. */
typedef enum sil_unet_layer_kind {
  SIL_UNET_CONV3 = 0, /* 3x3 conv + ReLU, weight [Co][Ci][3][3] */
  SIL_UNET_UP = 1,    /* 2x2 stride-2 transposed conv, weight [Ci][Co][2][2] */
  SIL_UNET_HEAD = 2   /* 1x1 conv to 3 scores, weight [3][F][1][1] */
} sil_unet_layer_kind;

/* Fills F = 32, depth = 5, max_batch = 32.  SIL_EINVAL on NULL. */
sil_status sil_unet_config_default(sil_unet_config* cfg);

/* Number of weighted layers: 5 depth + 3 (2 per encoder level, 2 at the
 * bottom, 3 per decoder level, 1 head; 28 at depth 5, the paper's count of
 * five downsampling steps, a bottleneck and five upsampling steps); -1 if
 * depth is out of range. */
int32_t sil_unet_num_layers(int32_t depth);

/* Shape of layer i in this order: enc0_0, enc0_1, enc1_0, ..., bott_0,
 * bott_1, then for l = depth-1..0: up_l, dec_l_0, dec_l_1; then head.
 * dims[4] receives the PyTorch weight shape (the first conv has Ci = 3),
 * *kind its kind; the bias has dims[0] entries (dims[1] for SIL_UNET_UP). */
sil_status sil_unet_layer_shape(const sil_unet_config* cfg, int32_t i, int64_t dims[4],
                                int32_t* kind);

/* Multiply-adds x 2 of one chip's forward pass. */
int64_t sil_unet_flops_per_chip(const sil_unet_config* cfg);

/* Creates a network on `device`: uploads the weights (HOST float32 arrays in
 * PyTorch layout, one per layer in sil_unet_layer_shape order; values are
 * rounded to bfloat16 except the head, kept in float32) and allocates the
 * activations of max_batch chips.  The caller keeps ownership of the host
 * arrays; the network owns its device memory until sil_unet_destroy.
 * SIL_EINVAL on a bad config or NULL array, SIL_ENOMEM, SIL_ECUDA. */
sil_status sil_unet_create(sil_unet** net, const sil_unet_config* cfg,
                           const float* const* weights, const float* const* biases,
                           int32_t device);
void sil_unet_destroy(sil_unet* net);

/* Forward pass of n chips (1..max_batch): chips = DEVICE uint8
 * [n][256][256][3] (R, G, B); labels = DEVICE uint8 [n][256][256] (nullable);
 * logits = DEVICE float32 [n][256][256][3] (nullable).  Asynchronous on
 * `stream`; the network's activations are reused by the next call, so calls
 * on one network must be ordered (same stream).  Waits inside the kernels
 * are bounded: a wait that runs out counts an error that
 * sil_unet_error_count reports. */
sil_status sil_unet_forward(sil_unet* net, const uint8_t* chips, int32_t n, uint8_t* labels,
                            float* logits, sil_stream stream);

/* The same on the filtered chips, as the paper's inferencing workflow does
 * (Sec. III-C): vprime = DEVICE uint8 [n][256][256], the filter's corrected
 * value V' of every pixel (sil_label_v on the scene, cut like the chips);
 * each pixel's R, G, B is first scaled by V'/V, V = max(R, G, B), rounded half
 * up: c' = floor((2 c V' + V) / (2 V)), 0 when V = 0 (HSV with V replaced by
 * V', H and S kept).  vprime = NULL is sil_unet_forward. */
sil_status sil_unet_forward_filtered(sil_unet* net, const uint8_t* chips, const uint8_t* vprime,
                                     int32_t n, uint8_t* labels, float* logits,
                                     sil_stream stream);

/* The paper's inferencing workflow on a whole scene (Sec. III-C): the
 * scene (DEVICE uint8 H x W x 3, pitch bytes per row) is cut into its
 * 256 x 256 chip grid anchored at (0, 0) (zero past the right and bottom
 * edges), the chips -- filtered by vprime (DEVICE uint8 H x W, the V' of
 * sil_label_v; NULL: unfiltered) -- run through the network max_batch at a
 * time, and each chip's labels are written back into labels (DEVICE uint8
 * H x W, label_pitch bytes per row).  Uses the network's own staging
 * buffers; asynchronous on `stream`. */
sil_status sil_unet_label_scene(sil_unet* net, const uint8_t* img, int64_t H, int64_t W,
                                int64_t pitch, const uint8_t* vprime, int64_t vprime_pitch,
                                uint8_t* labels, int64_t label_pitch, sil_stream stream);

/* Synchronises the device and returns the number of kernel waits that ran
 * out since the network was created (0 in normal operation). */
sil_status sil_unet_error_count(sil_unet* net, uint32_t* count);

/* Test hook for the bounded waits: while set, every CTA of layer `layer`'s
 * kernel leaves out the input load of its first stage, so the wait for that
 * stage runs out (about 1.3 s), the kernel counts an error, frees its tensor
 * memory and returns (that layer's output is then undefined).  layer = -1
 * clears the hook.  Only layers whose input arrives by tensor map (input
 * channels 32 or a multiple of 64) take it; others: SIL_EINVAL. */
sil_status sil_unet_set_fault(sil_unet* net, int32_t layer);

/* Output activation of layer i (sil_unet_layer_shape order) of the last
 * forward pass: dims = {n, H, W, C} (n of that pass).  i = -1: the prepared
 * input, 8 channels (R, G, B scaled by 1/256, then 5 zeros).  The head (the
 * last layer) is computed inside the last decoder convolution and keeps no
 * activation: SIL_EINVAL. */
sil_status sil_unet_tensor_shape(const sil_unet* net, int32_t i, int64_t dims[4]);

/* Copies that activation into DEVICE bfloat16 `dst`, dense [n][H][W][C]
 * (the network stores encoder outputs inside the decoder's concatenation
 * buffers, so it is strided in place).  Asynchronous on `stream`. */
sil_status sil_unet_copy_tensor(const sil_unet* net, int32_t i, void* dst, sil_stream stream);

/* ------------------------------------------------------------------------
 * Training step (Sec. III-C "U-Net Model Training": the model is trained
 * with the Adam optimizer on categorical cross-entropy; "Distributed U-Net
 * Model Training using Horovod Framework": every worker computes the
 * gradient of its own batch, the gradients are averaged across workers and
 * each worker applies the same update).
 *
 * Readings where the paper is silent: the loss is the mean over the batch's
 * pixels whose label is 0..2 (label 3, masked, is left out); the paper's
 * dropout layers (rates and positions not given) are left out, so a step is
 * deterministic up to float summation order; Adam takes TensorFlow's
 * defaults b1 0.9, b2 0.999, eps 1e-7 (the learning rate is an argument); a
 * 2x2 max pool passes its gradient to the first maximum of its window in the
 * order (0,0), (0,1), (1,0), (1,1).
 *
 * Precision: the forward pass is sil_unet_forward's (bf16 weights and
 * activations, f32 sums, f32 head); activation gradients are stored as
 * bf16, parameter gradients, Adam moments and the master weights are f32.
 * After each update the master weights are rounded to bf16 for the next
 * forward and backward pass.
 *
 * Flat parameter vector: the layers in sil_unet_layer_shape order, each its
 * weight (PyTorch layout) then its bias, f32 (offsets from
 * sil_unet_trainer_param_offset); gradients use the same layout.
 * ------------------------------------------------------------------------ */
typedef struct sil_unet_trainer sil_unet_trainer;

/* Creates a trainer and its network (the arguments of sil_unet_create; the
 * host arrays become the initial master weights).  Besides the network's
 * activations it allocates the activation gradients of max_batch chips, a
 * <= 1 GiB buffer for the 3x3 layers' tap matrices and the f32 parameters
 * and moments.  SIL_EINVAL, SIL_ENOMEM, SIL_ECUDA. */
sil_status sil_unet_trainer_create(sil_unet_trainer** tr, const sil_unet_config* cfg,
                                   const float* const* weights, const float* const* biases,
                                   int32_t device);
void sil_unet_trainer_destroy(sil_unet_trainer* tr);

/* The trainer's network (owned by the trainer): its forward pass, tensor
 * copies and error count are those of the current weights. */
sil_unet* sil_unet_trainer_net(sil_unet_trainer* tr);

/* Length of the flat parameter vector; -1 on NULL. */
int64_t sil_unet_trainer_num_params(const sil_unet_trainer* tr);

/* Offsets of layer i's weight and bias in the flat vector. */
sil_status sil_unet_trainer_param_offset(const sil_unet_trainer* tr, int32_t i, int64_t* w_off,
                                         int64_t* b_off);

/* Forward pass, loss and gradient of n chips (1..max_batch): chips = DEVICE
 * uint8 [n][256][256][3], labels = DEVICE uint8 [n][256][256] (0 thick ice,
 * 1 thin ice, 2 open water, 3 left out).  Writes every element of grads
 * (DEVICE f32 [num_params]) and the mean loss (DEVICE f32 scalar).
 * Asynchronous on `stream`; the trainer's buffers are reused by the next
 * call, so calls on one trainer must be ordered.  The weight gradients of
 * the 3x3 and transposed convolutions are cuBLAS GEMMs (bf16 in, f32 out)
 * over the batch's pixels; everything else runs in this library's kernels.
 * Every reduction runs in a fixed order: the same weights and batch give
 * the same gradient and loss bits on every call. */
sil_status sil_unet_trainer_backward(sil_unet_trainer* tr, const uint8_t* chips,
                                     const uint8_t* labels, int32_t n, float* grads, float* loss,
                                     sil_stream stream);

/* One Adam update of the master weights with grads (DEVICE f32
 * [num_params], e.g. the average of every worker's sil_unet_trainer_backward
 * output) at step t >= 1 with learning rate lr >= 0, then the network's
 * weights are re-packed.  SIL_EINVAL on t < 1 or lr < 0. */
sil_status sil_unet_trainer_adam(sil_unet_trainer* tr, const float* grads, float lr, int32_t t,
                                 sil_stream stream);

/* Copies the master weights to / from DEVICE f32 [num_params]; set also
 * clears the Adam moments (a fresh optimizer) and re-packs the network
 * (the broadcast of rank 0's initial weights). */
sil_status sil_unet_trainer_get_params(const sil_unet_trainer* tr, float* dst, sil_stream stream);
sil_status sil_unet_trainer_set_params(sil_unet_trainer* tr, const float* src, sil_stream stream);

/* Stored activation gradients of the last backward pass. */
typedef enum sil_unet_grad_kind {
  SIL_UNET_GRAD_LAYER = 0, /* index = layer i (not the head): the gradient at
                              its pre-activation (after the ReLU's mask); for
                              a transposed convolution, at its output */
  SIL_UNET_GRAD_CAT = 1,   /* index = level l: the gradient at the decoder's
                              concatenation [upsampled, encoder output] */
  SIL_UNET_GRAD_POOL = 2   /* index = level l: the gradient at level l's
                              pooled output (before it meets the skip share) */
} sil_unet_grad_kind;

/* dims = {n, H, W, C} of that gradient; the copy writes DEVICE bf16 dense
 * [n][H][W][C].  SIL_EINVAL on an unknown kind or index, or before the
 * first backward pass. */
sil_status sil_unet_trainer_grad_shape(const sil_unet_trainer* tr, int32_t kind, int32_t i,
                                       int64_t dims[4]);
sil_status sil_unet_trainer_copy_grad(const sil_unet_trainer* tr, int32_t kind, int32_t i,
                                      void* dst, sil_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* SIL_UNET_H_ */
