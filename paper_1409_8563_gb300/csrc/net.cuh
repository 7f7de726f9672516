// net.cuh -- layout constants and launchers of the learned coarse propagator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace pr {

// Linear mode (lin != 0, see net.cu): identity activations, no biases, input
// channel 2 = nu_hat * S(u).
// FP32 master parameters, in this order (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)):
//   W1[16][2][27] b1[16] W2[16][16][27] b2[16] W3[16][16][27] b3[16] W4[1][16][27] b4[1]
constexpr int NET_W1 = 0, NET_B1 = 864, NET_W2 = 880, NET_B2 = 7792, NET_W3 = 7808,
              NET_B3 = 14720, NET_W4 = 14736, NET_B4 = 15168, NET_PARAMS = 15169;
constexpr int NET_MID_PARTIAL = 27 * 256 + 16;   // dW[27][16][16] + db[16]
constexpr int NET_OUT_PARTIAL = 433;             // dW4[16][27] + db4
constexpr int NET_IN_PARTIAL = 880;              // dW1[16][2][27] + db1[16]

// LINEAR network composed into one 9x9x9 cross-correlation per slice
// (net_composed.cu): taps [ez+4][ey+4][ex+4].
constexpr int NET_K9 = 729;
size_t compose_scratch_doubles();
// keff[n] = K_0 + nu_hat[n] K_1 for n < n_slices (FP32), built in FP64 from
// the master weights; scratch: compose_scratch_doubles() doubles.
cudaError_t launch_compose_linear(const float *master, const float *nu_hat, int n_slices,
                                  double *scratch, float *keff, cudaStream_t st);
// out = S(u) + K * S(u) (S the periodic shift by s), K: NET_K9 floats on the
// device, FP32 accumulation; m a multiple of 16.
template <typename TU, typename TG>
cudaError_t launch_net_lin9(const TU *u, int m, const int s[3], const float *K, TG *out, cudaStream_t st);
// After launch_compose_linear: the two composed 9^3 kernels K_0, K_1 in FP64
// ([2][NET_K9], index (ez+4) 81 + (ey+4) 9 + (ex+4)) inside its scratch.
const double *composed_kernels(const double *scratch);

// net_poly.cu: the stencil-skip LINEAR propagator as r^3 phase kernels on the
// coarse grid.  TT taps per axis, lo_off the lowest coarse offset a tap
// reaches, win the coarse window edge of one 16^3 fine brick.
void poly_geometry(int r, int *TT, int *lo_off, int *win);
size_t poly_weights_floats(int r, int n_slices);   // per-slice FP32 phase kernels
size_t poly_scratch_doubles(int r);                 // FP64 phase kernels of K_0 and K_1
cudaError_t configure_poly_kernels(int r);
// W2 (FP64) from K2 = composed_kernels(...), then Wn (FP32, per slice).
cudaError_t launch_compose_poly(const double *K2, int r, const float *nu_hat, int n_slices, double *W2,
                                float *Wn, cudaStream_t st);
// out = (phase kernels of one slice, Wn + slice offset) applied to cnew - cold
// (cold may be null) on the coarse grid of edge n / r; out is the fine n^3
// field.  n a multiple of 16, r in {2, 4, 8, 16}.
template <typename T>
cudaError_t launch_poly_prolong(const T *cnew, const T *cold, const float *W, int n, int r, T *out,
                                cudaStream_t st);

cudaError_t configure_net_kernels();
// 16 -> 16 forward layer on the 5th-generation tensor cores (net_tc.cu);
// m a multiple of 16.  errflag (device int) is set if an MMA completion wait
// runs out.
cudaError_t configure_net_tc();
// Self-test of the bounded completion wait of the tensor-core layers: waits
// `limit` tries on an mbarrier nothing arrives on; *flag = 1 when it gave up.
cudaError_t launch_wait_selftest(long long limit, int *flag, cudaStream_t st);
bool net_tc_supported(int m);
// mode 0: forward (zout, if non-null, receives the FP32 pre-activations);
// mode 1: input gradient through the mirrored operand Bt, times gelu'(zaux).
cudaError_t launch_net_mid_tc(int mode, const __nv_bfloat16 *in, int m, int batch, const __nv_bfloat16 *Bt,
                              const float *bias, const float *zaux, float *zout, __nv_bfloat16 *out,
                              int lin, int *errflag, cudaStream_t st);
// Weight gradient of a 16 -> 16 layer on the tensor cores: the same partials
// as launch_net_mid_wgrad (nblocks slots of NET_MID_PARTIAL floats).
cudaError_t launch_net_mid_wgrad_tc(const __nv_bfloat16 *x, const __nv_bfloat16 *dz, int m, int batch,
                                    float *partials, int nblocks, int *errflag, cudaStream_t st);
template <typename TU>
cudaError_t launch_net_in_fwd(const TU *u, int m, const int s[3], const float *nu_hat, int batch,
                              const float *W1q, const float *b1, float *z1, __nv_bfloat16 *a1,
                              cudaStream_t st, int lin = 0);
cudaError_t launch_net_mid(int mode, const __nv_bfloat16 *in, int m, int batch,
                           const __nv_bfloat16 *Bt, const float *bias, const float *zaux, float *zout,
                           __nv_bfloat16 *out, cudaStream_t st, int lin = 0);
int net_partial_blocks(int m, int batch);
cudaError_t launch_net_mid_wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *dz, int m, int batch,
                                 float *partials, int nblocks, cudaStream_t st);
cudaError_t launch_net_out_dgrad(const __nv_bfloat16 *dz4, int m, int batch, const float *W4q,
                                 const float *z3, __nv_bfloat16 *dz3, cudaStream_t st, int lin = 0);
cudaError_t launch_net_out_wgrad(const __nv_bfloat16 *a3, const __nv_bfloat16 *dz4, int m, int batch,
                                 float *partials, int nblocks, cudaStream_t st);
template <typename TU>
cudaError_t launch_net_in_wgrad(const TU *u, int m, int batch, const int s[3], const float *nu_hat,
                                const __nv_bfloat16 *dz1, float *partials, int nblocks,
                                cudaStream_t st, int lin = 0);
cudaError_t launch_reduce_cols(const float *partials, int nb, int stride, int L, float *out,
                               cudaStream_t st);
cudaError_t launch_reduce_mid(const float *partials, int nb, float *W, float *b, cudaStream_t st);
cudaError_t launch_reduce_loss(const double *parts, int nb, double *out, cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *mo, float *vo, int L, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t launch_prepare_operands(const float *master, float *W1q, __nv_bfloat16 *B2f,
                                    __nv_bfloat16 *B3f, __nv_bfloat16 *B2b, __nv_bfloat16 *B3b,
                                    float *W4q, __nv_bfloat16 *B4f, cudaStream_t st);
// Last layer of training on the tensor cores: g = S(u) + z4 against the
// target, dz4 = bf16((g - tgt) * grad_scale) and the per-tile sums of
// (g - tgt)^2 in loss_partials (no G output).
cudaError_t launch_net_out_mma_train(const __nv_bfloat16 *a3, int m, int batch, const __nv_bfloat16 *B4f,
                                     const float *b4, const float *u, const int s[3], const float *tgt,
                                     float grad_scale, __nv_bfloat16 *dz4, double *loss_partials,
                                     cudaStream_t st, int lin = 0);
// Last layer for inference on the tensor cores (B4f: [27][8][16], row 0 = W4).
template <typename TU, typename TG>
cudaError_t launch_net_out_mma(const __nv_bfloat16 *a3, int m, int batch, const __nv_bfloat16 *B4f,
                               const float *b4, const TU *u, const int s[3], TG *g_out,
                               cudaStream_t st, int lin = 0);

}  // namespace pr
