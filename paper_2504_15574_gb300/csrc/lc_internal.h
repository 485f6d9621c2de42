// lc_internal.h -- shapes and launchers of the learned-correction network (lc.cu).
#pragma once

#include <cuda_bf16.h>

#include "vlbm_internal.h"

namespace vk {

constexpr int LC_LAYERS = 4;
// Input channels: 0 rho - 1, 1 u^theta, 2 u^phi, 3 T - 1, 4 cos(theta), 5 sin(theta), then the
// undivided differences 6 d6_theta rho, 7 d6_phi rho, 8 d6_theta u^theta, 9 d6_phi u^theta,
// 10 d6_theta u^phi, 11 d6_phi u^phi, 12 d4_theta u^theta, 13 d4_phi u^theta, 14 d4_theta u^phi,
// 15 d4_phi u^phi (d4 = [1 -4 6 -4 1], d6 = [1 -6 15 -20 15 -6 1] along a grid line).
constexpr int LC_IN = 16;
constexpr int LC_NSCALE = 14;   // scaled channels: 0-3 and 6-15
constexpr int LC_CIN = 16;      // input channels padded for the k = 16 tensor-core step
constexpr int LC_HID = 32;      // hidden channels
constexpr int LC_OUT = 3;       // drho, du^theta, du^phi
constexpr int LC_COUT = 8;      // output channels padded to an n = 8 tile
constexpr int LC_COUTP2 = 16;   // output-gradient channels padded for the k = 16 step (backward data)
constexpr float LC_CLAMP = 8.0f;   // bound of every scaled input feature
// input channels odd across a pole: the velocity components, their differences and sin(theta)
constexpr unsigned LC_NEGMASK = (1u << 1) | (1u << 2) | (1u << 5) | (0xFFu << 8);
struct LcInScale { float inv[LC_NSCALE]; };

// Layer `layer` on the padded input Xp: FP32 pre-activations Yf, BF16 (ReLU) outputs Yb
// [H][W][CO] and / or the next layer's padded input Ypad [H+2][W+2][CO] (any may be NULL).
// part0 (last layer only; optional): per CTA of the launch (lc_conv_ctas of them) the sum over its
// pixels of sin_t[row] times output 0.
void lc_conv(int layer, const __nv_bfloat16 *Xp, int Hp, int Wp, const __nv_bfloat16 *Wt, const float *bias,
             float *Yf, __nv_bfloat16 *Yb, __nv_bfloat16 *Ypad, int relu, cudaStream_t s,
             double *part0 = nullptr, const double *sin_t = nullptr);
int lc_conv_ctas(int H, int W);
void lc_conv_bwd(int layer, const __nv_bfloat16 *dP, int H, int W, const __nv_bfloat16 *Wb, float *dXp, cudaStream_t s);
void lc_wgrad(int layer, const __nv_bfloat16 *dPre, const __nv_bfloat16 *Xp, int H, int W, float *part, float *partb,
              cudaStream_t s);
void lc_unpad(const float *dXp, int H, int W, int C, unsigned negmask, float *dX, cudaStream_t s);
void lc_grad_pad2(const float *dY, const __nv_bfloat16 *act, int H, int W, int C, int CP, __nv_bfloat16 *dP,
                  cudaStream_t s);
void lc_grad_pre(const float *dY, const __nv_bfloat16 *act, int n, int C, int CP, __nv_bfloat16 *dPre, cudaStream_t s);
void lc_reduce_rows(const float *part, int rows, int n, float *out, cudaStream_t s);
void lc_loss(const float *Y, int CO, const double *target, const double *sin_t, int H, int W, float3 inv_scale,
             double wsum, float *dY, double *part, double *loss, cudaStream_t s);
void lc_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps, float c1,
             float c2, cudaStream_t s);
void lc_weights_bf16(const float *w, int CO, int CI, int COp, int CIp, __nv_bfloat16 *fwd, int CIp2, int COp2,
                     __nv_bfloat16 *bwd, cudaStream_t s);
void lc_wgrad_layout(const float *g9, int CO, int CI, int COp, int CIp, float *g, cudaStream_t s);
// The padded layer-0 input from the moment deviations dev = (rho - 1, u^theta, u^phi, T - 1)
// [4][H][W] (FP32).
void lc_features(const float *dev, int H, int W, const double *sin_t, const double *cos_t,
                 const LcInScale &inv_scale, __nv_bfloat16 *Xp, cudaStream_t s);
// The deviations dev [4][H][W] (FP32) of FP64 moments (rho, u^theta, u^phi, T) [4][H][W].
void lc_dev_of_moments(const double *in4, int H, int W, float *dev, cudaStream_t s);
// The deviations (rho - 1, u^theta, u^phi, T - 1) [4][H][W] of a solver's FP32 state (state scale
// ks), FP32 arithmetic on the stored deviations.
void lc_moments(const float2 *f, const Layout &L, const VelD &c, double rho_ref, const double *sin_t, double ks,
                float *dev, cudaStream_t s);
void lc_outputs(const float *Y, int CO, int H, int W, float3 scale, const double *sin_t, double *out, double *part,
                double *mean, cudaStream_t s);
void lc_nudge(float2 *f, const Layout &L, const float *dev, const double *delta, const double *mean, double wsum,
              const VelD &c, const double *sin_t, double ks, cudaStream_t s);
// The direct form's nudge from the net output Y [H][W][CO] (times scale) and the last layer's
// nparts partial sums of sin(theta) output 0 (the area mean of drho is removed).
void lc_nudge_direct(float2 *f, const Layout &L, const float *dev, const float *Y, int CO, float3 scale,
                     const double *part0, int nparts, double wsum, const VelD &c, const double *sin_t, double ks,
                     cudaStream_t s);
// Stream-function output form: output 0 times s0 is a stream function psi on the H x W cell grid
// of a sphere of radius R (dth = pi / H, dph = 2 pi / W), the correction its centred curl
// (0, d_phi psi / (R sin theta), -d_theta psi / R), psi continued across a pole as a scalar.
struct LcStream { int H, W; double s0, R, dth, dph; };
// Loss of the stream form against the velocity targets (channels 1, 2 of target [3][H][W]) scaled
// by inv_s1, inv_s2; the gradient at the net output into dY [H][W][CO] (gv: [2][H][W] scratch).
void lc_stream_loss(const float *Y, int CO, const double *target, const double *sin_t, const LcStream &g,
                    double inv_s1, double inv_s2, double wsum, double *gv, float *dY, double *part, double *loss,
                    cudaStream_t s);
// The stream form's correction (0, du^theta, du^phi) [3][H][W]; *mean (the drho area sum) = 0.
void lc_stream_outputs(const float *Y, int CO, const LcStream &g, const double *sin_t, double *out, double *part,
                       double *mean, cudaStream_t s);
// Vorticity output form: output 0 times s0 is a vorticity correction w; psi solves the
// finite-volume Poisson equation L psi = w - (area mean of w) on the sphere of radius R, and the
// correction is the curl of psi as in the stream form.  Device tables and work arrays:
struct LcPoisson {
    int H, W;
    double R, wsum;
    const float2 *tab;    // [W/2 + 1][H] Thomas factors (and the mode-0 integration's)
    const float *a;       // [H] sub-diagonal of the theta operator
    const float2 *tw;     // [2W] (cos, sin)(pi k / W)
    float2 *X;            // [W/2 + 1][H] modes
    double *w, *psi;      // [H][W]
    double *part, *sum;   // reduction scratch (>= H W / 256 + 1) and one total
};
void lc_vort_loss(const float *Y, int CO, const double *target, const double *sin_t, const LcStream &g,
                  const LcPoisson &P, double inv_s1, double inv_s2, double wsum, double *gv, float *dY, double *part,
                  double *loss, cudaStream_t s);
void lc_vort_outputs(const float *Y, int CO, const LcStream &g, const LcPoisson &P, const double *sin_t, double *out,
                     double *part, double *mean, cudaStream_t s);
// The tables of an H x W grid (R = 1): their size in floats, and a blocking fill of a device array
// of that size laid out as tab, a, tw (0 on success).
size_t lc_poisson_table_floats(int H, int W);
// Raises the mode solve's shared-memory limit where H rows need more than 48 KB (0 on success;
// call outside any stream capture).
int lc_poisson_prepare(int H);
int lc_poisson_tables(int H, int W, float *dev);

}  // namespace vk
