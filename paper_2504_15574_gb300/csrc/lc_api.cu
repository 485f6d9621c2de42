// lc_api.cu -- host side of the learned correction (vlbm_lc_* in include/vlbm.h).
//
// Owns the network's FP32 master weights and Adam state, their BF16 copies in
// the forward and backward-data layouts, and the activation / gradient buffers
// for one coarse grid.  Every step (features, padding, convolutions, ReLU masks,
// loss, weight gradients, Adam, output scaling, the nudge of a solver's
// populations) runs in the kernels of lc.cu on the handle's stream.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vlbm.h"
#include "lc_internal.h"
#include "vlbm_handle.h"

using namespace vk;

struct vlbm_lc {
    int H = 0, W = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // layer shapes: real and padded channel counts
    int ci[LC_LAYERS], co[LC_LAYERS], cip[LC_LAYERS], cop[LC_LAYERS], cop2[LC_LAYERS];
    size_t woff[LC_LAYERS], boff[LC_LAYERS];
    int nparam = 0;
    float *d_w = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    __nv_bfloat16 *d_wf[LC_LAYERS] = {}, *d_wb[LC_LAYERS] = {};
    double *d_sin = nullptr, *d_cos = nullptr, *d_in = nullptr, *d_tg = nullptr, *d_out = nullptr, *d_part = nullptr, *d_scal = nullptr;
    __nv_bfloat16 *d_xp[LC_LAYERS] = {}, *d_z[LC_LAYERS] = {};
    float *d_y = nullptr, *d_dy = nullptr, *d_dxp = nullptr, *d_dx = nullptr;
    float *d_dev = nullptr;      // the network's moment deviations (rho - 1, u^theta, u^phi, T - 1) [4][H][W]
    double *d_cpart = nullptr;   // direct-form correction: the last layer's per-CTA sums of sin(theta) output 0
    __nv_bfloat16 *d_dp = nullptr, *d_dpre = nullptr;
    float *d_wpart = nullptr, *d_bpart = nullptr, *d_g9 = nullptr;
    double wsum = 0.0;
    float in_scale[LC_NSCALE] = {1e-3f, 1e-2f, 1e-2f, 1e-3f, 1e-6f, 1e-6f, 1e-5f, 1e-5f, 1e-5f,
                                 1e-5f, 1e-5f, 1e-5f, 1e-5f, 1e-5f};
    float out_scale[3] = {1e-5f, 1e-4f, 1e-4f};
    int form = VLBM_LC_DIRECT;   // output form (vlbm_lc_set_output_form)
    double radius = 1.0;         // the stream form's sphere radius
    double *d_gv = nullptr;      // stream form: the loss's derivatives by du^theta, du^phi [2][H][W]
    // vorticity form: Poisson tables (R = 1) and work arrays
    float *d_ptabs = nullptr;    // tab, a, tw (lc_poisson_tables)
    float2 *d_pX = nullptr;
    double *d_pw = nullptr, *d_psi = nullptr, *d_ppart = nullptr, *d_psum = nullptr;
    bool vort_ok = false;        // the vorticity form's mode solve fits this grid
    long long t = 0;
    std::vector<void *> bufs;
    cudaGraphExec_t g_exec = nullptr;   // vlbm_lc_rollout: one corrected step of solver g_solver
    vlbm_t *g_solver = nullptr;
    unsigned long long g_gen = 0;       // the solver's step generation when g_exec was captured
};

namespace {

int lfail(vlbm_lc_t *n, int code, const std::string &m)
{
    if (n) n->err = m;
    return code;
}

#define LCK(n, call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return lfail((n), VLBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int lalloc(vlbm_lc_t *n, T **p, size_t count)
{
    LCK(n, cudaMalloc((void **)p, count * sizeof(T)));
    LCK(n, cudaMemset(*p, 0, count * sizeof(T)));
    n->bufs.push_back(*p);
    return VLBM_OK;
}

// splitmix64 for the initial weights
unsigned long long smix(unsigned long long &s)
{
    s += 0x9E3779B97F4A7C15ull;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int refresh_bf16(vlbm_lc_t *n)
{
    for (int l = 0; l < LC_LAYERS; ++l)
        lc_weights_bf16(n->d_w + n->woff[l], n->co[l], n->ci[l], n->cop[l], n->cip[l], n->d_wf[l], n->cip[l], n->cop2[l],
                        l > 0 ? n->d_wb[l] : nullptr, n->stream);
    LCK(n, cudaGetLastError());
    return VLBM_OK;
}

// forward pass on the moment deviations dev ([4][H][W] device, FP32), on stream s; output in d_y.
// keep: also store each hidden layer's unpadded activations (d_z) for the backward pass.
// part0: the last layer's per-CTA partial sums of sin(theta) times output 0 (optional)
int forward(vlbm_lc_t *n, const float *dev, cudaStream_t s, bool keep = true, double *part0 = nullptr)
{
    const int H = n->H, W = n->W, HW = H * W;
    LcInScale is;
    for (int q = 0; q < LC_NSCALE; ++q) is.inv[q] = 1.0f / n->in_scale[q];
    // the padded input of layer 0 (velocity channels, their differences and sin(theta) change
    // sign across a pole); each hidden layer writes the next layer's padded input itself
    (void)HW;
    lc_features(dev, H, W, n->d_sin, n->d_cos, is, n->d_xp[0], s);
    for (int l = 0; l < LC_LAYERS; ++l) {
        const bool last = (l == LC_LAYERS - 1);
        lc_conv(l, n->d_xp[l], H + 2, W + 2, n->d_wf[l], n->d_w + n->boff[l], last ? n->d_y : nullptr,
                (last || !keep) ? nullptr : n->d_z[l], last ? nullptr : n->d_xp[l + 1], last ? 0 : 1, s,
                last ? part0 : nullptr, n->d_sin);
    }
    LCK(n, cudaGetLastError());
    return VLBM_OK;
}

LcStream stream_geometry(const vlbm_lc_t *n)
{
    return LcStream{n->H, n->W, (double)n->out_scale[0], n->radius, M_PI / n->H, 2.0 * M_PI / n->W};
}

LcPoisson poisson_work(const vlbm_lc_t *n)
{
    const size_t M = (size_t)n->W / 2 + 1, H = n->H, W = n->W;
    const float *t = n->d_ptabs, *a = t + 2 * M * H, *tw = a + H + (H & 1);   // as laid out by lc_poisson_tables
    (void)W;
    return LcPoisson{n->H, n->W, n->radius, n->wsum, reinterpret_cast<const float2 *>(t), a,
                     reinterpret_cast<const float2 *>(tw), n->d_pX, n->d_pw, n->d_psi, n->d_ppart, n->d_psum};
}

// the correction in physical units into d_out ([3][H][W]) and the area sum of its drho into
// d_scal[1], from the forward pass's output d_y
void enqueue_outputs(vlbm_lc_t *n, cudaStream_t s)
{
    if (n->form == VLBM_LC_VORTICITY) {
        lc_vort_outputs(n->d_y, LC_COUT, stream_geometry(n), poisson_work(n), n->d_sin, n->d_out, n->d_part,
                        n->d_scal + 1, s);
    } else if (n->form == VLBM_LC_STREAM) {
        lc_stream_outputs(n->d_y, LC_COUT, stream_geometry(n), n->d_sin, n->d_out, n->d_part, n->d_scal + 1, s);
    } else {
        const float3 sc = make_float3(n->out_scale[0], n->out_scale[1], n->out_scale[2]);
        lc_outputs(n->d_y, LC_COUT, n->H, n->W, sc, n->d_sin, n->d_out, n->d_part, n->d_scal + 1, s);
    }
}

// loss and gradient of every parameter into d_g; loss into d_scal[0]
int backward(vlbm_lc_t *n)
{
    const int H = n->H, W = n->W, HW = H * W;
    if (n->form == VLBM_LC_VORTICITY) {
        lc_vort_loss(n->d_y, LC_COUT, n->d_tg, n->d_sin, stream_geometry(n), poisson_work(n), 1.0 / n->out_scale[1],
                     1.0 / n->out_scale[2], n->wsum, n->d_gv, n->d_dy, n->d_part, n->d_scal, n->stream);
    } else if (n->form == VLBM_LC_STREAM) {
        lc_stream_loss(n->d_y, LC_COUT, n->d_tg, n->d_sin, stream_geometry(n), 1.0 / n->out_scale[1],
                       1.0 / n->out_scale[2], n->wsum, n->d_gv, n->d_dy, n->d_part, n->d_scal, n->stream);
    } else {
        const float3 ios = make_float3(1.0f / n->out_scale[0], 1.0f / n->out_scale[1], 1.0f / n->out_scale[2]);
        lc_loss(n->d_y, LC_COUT, n->d_tg, n->d_sin, H, W, ios, n->wsum, n->d_dy, n->d_part, n->d_scal, n->stream);
    }
    // gradient at the output of layer l lives in d_dy with cop[l] channels
    for (int l = LC_LAYERS - 1; l >= 0; --l) {
        const int C = n->cop[l], CP = n->cop2[l];
        const __nv_bfloat16 *act = (l == LC_LAYERS - 1) ? nullptr : n->d_z[l];
        lc_grad_pre(n->d_dy, act, HW, C, CP, n->d_dpre, n->stream);
        lc_wgrad(l, n->d_dpre, n->d_xp[l], H, W, n->d_wpart, n->d_bpart, n->stream);
        lc_reduce_rows(n->d_wpart, H, 9 * n->cop2[l] * n->cip[l], n->d_g9, n->stream);
        lc_wgrad_layout(n->d_g9, n->co[l], n->ci[l], n->cop2[l], n->cip[l], n->d_g + n->woff[l], n->stream);
        lc_reduce_rows(n->d_bpart, H, n->cop2[l], n->d_dx, n->stream);   // bias gradient (first co entries)
        LCK(n, cudaMemcpyAsync(n->d_g + n->boff[l], n->d_dx, sizeof(float) * n->co[l], cudaMemcpyDeviceToDevice,
                               n->stream));
        if (l == 0) break;
        lc_grad_pad2(n->d_dy, act, H, W, C, CP, n->d_dp, n->stream);
        lc_conv_bwd(l, n->d_dp, H, W, n->d_wb[l], n->d_dxp, n->stream);
        lc_unpad(n->d_dxp, H, W, LC_HID, 0u, n->d_dy, n->stream);      // gradient at the output of layer l-1
    }
    LCK(n, cudaGetLastError());
    return VLBM_OK;
}

int check_solver(vlbm_lc_t *n, vlbm_t *h)
{
    if (!n || !h) return VLBM_ERR_ARG;
    if (h->prec != VLBM_FP32 || h->vd.q != 4 || h->nt != n->H || h->np != n->W)
        return lfail(n, VLBM_ERR_ARG, "the solver must be FP32 D2Q16 on the network's grid");
    if (n->form != VLBM_LC_DIRECT && n->radius != h->R)
        return lfail(n, VLBM_ERR_ARG, "the output form's radius differs from the solver's");
    return VLBM_OK;
}

// The correction of solver h's current state, enqueued on stream s without host
// synchronisation: moments, forward pass, outputs (drho area mean), nudge (which also writes each
// cell's ghost images).
int enqueue_correction(vlbm_lc_t *n, vlbm_t *h, cudaStream_t s)
{
    lc_moments((const float2 *)h->F, h->L, h->vd, h->rho_ref, h->d_sin_t, h->kscale, n->d_dev, s);
    int rc;
    if (n->form == VLBM_LC_DIRECT) {
        // the output scaling and the area mean of drho ride on the last convolution and the nudge
        if ((rc = forward(n, n->d_dev, s, false, n->d_cpart))) return rc;
        const float3 sc = make_float3(n->out_scale[0], n->out_scale[1], n->out_scale[2]);
        lc_nudge_direct((float2 *)h->F, h->L, n->d_dev, n->d_y, LC_COUT, sc, n->d_cpart, lc_conv_ctas(n->H, n->W),
                        n->wsum, h->vd, n->d_sin, h->kscale, s);
        LCK(n, cudaGetLastError());
        return VLBM_OK;
    }
    if ((rc = forward(n, n->d_dev, s, false))) return rc;
    enqueue_outputs(n, s);
    lc_nudge((float2 *)h->F, h->L, n->d_dev, n->d_out, n->d_scal + 1, n->wsum, h->vd, n->d_sin, h->kscale, s);
    LCK(n, cudaGetLastError());
    return VLBM_OK;
}

int upload_io(vlbm_lc_t *n, const double *inputs, const double *targets)
{
    const size_t HW = (size_t)n->H * n->W;
    if (inputs) {
        LCK(n, cudaMemcpyAsync(n->d_in, inputs, 4 * HW * sizeof(double), cudaMemcpyHostToDevice, n->stream));
        lc_dev_of_moments(n->d_in, n->H, n->W, n->d_dev, n->stream);
    }
    if (targets) LCK(n, cudaMemcpyAsync(n->d_tg, targets, 3 * HW * sizeof(double), cudaMemcpyHostToDevice, n->stream));
    return VLBM_OK;
}

}  // namespace

extern "C" {

int vlbm_lc_create(int n_theta, int n_phi, unsigned long long seed, vlbm_lc_t **out)
{
    if (!out) return VLBM_ERR_ARG;
    *out = nullptr;
    if (n_theta < 4 || n_phi < 2 || n_phi % 2) return VLBM_ERR_ARG;
    vlbm_lc_t *n = new vlbm_lc_t();
    n->H = n_theta;
    n->W = n_phi;
    if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete n;
        return VLBM_ERR_CUDA;
    }
    const int ci[LC_LAYERS] = {LC_IN, LC_HID, LC_HID, LC_HID}, co[LC_LAYERS] = {LC_HID, LC_HID, LC_HID, LC_OUT};
    size_t off = 0;
    for (int l = 0; l < LC_LAYERS; ++l) {
        n->ci[l] = ci[l];
        n->co[l] = co[l];
        n->cip[l] = (l == 0) ? LC_CIN : LC_HID;
        n->cop[l] = (l == LC_LAYERS - 1) ? LC_COUT : LC_HID;
        n->cop2[l] = (l == LC_LAYERS - 1) ? LC_COUTP2 : LC_HID;
        n->woff[l] = off;
        off += (size_t)co[l] * ci[l] * 9;
        n->boff[l] = off;
        off += co[l];
    }
    n->nparam = (int)off;
    // He-style uniform initialisation; the last layer starts small (a near-zero correction)
    std::vector<float> w(off, 0.0f);
    unsigned long long s = seed;
    for (int l = 0; l < LC_LAYERS; ++l) {
        const double fan = 9.0 * ci[l];
        const double a = (l == LC_LAYERS - 1 ? 0.1 : 1.0) * std::sqrt(6.0 / fan);
        for (size_t q = 0; q < (size_t)co[l] * ci[l] * 9; ++q)
            w[n->woff[l] + q] = (float)(a * (2.0 * ((smix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    }
    const size_t HW = (size_t)n_theta * n_phi, HWp = (size_t)(n_theta + 2) * (n_phi + 2),
                 HWp2 = (size_t)(n_theta + 4) * (n_phi + 4);
    int rc = 0;
    auto A = [&](auto **p, size_t c) {
        if (!rc) rc = lalloc(n, p, c);
    };
    A(&n->d_w, off);
    A(&n->d_g, off);
    A(&n->d_m, off);
    A(&n->d_v, off);
    for (int l = 0; l < LC_LAYERS; ++l) {
        A(&n->d_wf[l], (size_t)n->cop[l] * 9 * n->cip[l]);
        A(&n->d_wb[l], (size_t)n->cip[l] * 9 * n->cop2[l]);
        A(&n->d_xp[l], HWp * n->cip[l]);
        A(&n->d_z[l], HW * LC_HID);
    }
    A(&n->d_sin, (size_t)n_theta);
    A(&n->d_cos, (size_t)n_theta);
    A(&n->d_in, 4 * HW);
    A(&n->d_dev, 4 * HW);
    A(&n->d_cpart, (size_t)lc_conv_ctas(n_theta, n_phi));
    A(&n->d_tg, 3 * HW);
    A(&n->d_out, 3 * HW);
    A(&n->d_part, HW / 256 + 2);
    A(&n->d_scal, 4);
    A(&n->d_y, HW * LC_COUT);
    A(&n->d_dy, HW * LC_HID);
    A(&n->d_dxp, HWp * LC_HID);
    A(&n->d_dx, HW * LC_HID);
    A(&n->d_dp, HWp2 * LC_HID);
    A(&n->d_dpre, HW * LC_HID);
    A(&n->d_wpart, (size_t)n_theta * 9 * LC_HID * LC_HID);
    A(&n->d_bpart, (size_t)n_theta * LC_HID);
    A(&n->d_g9, (size_t)9 * LC_HID * LC_HID);
    A(&n->d_gv, 2 * HW);
    const size_t M = (size_t)n_phi / 2 + 1;
    A(&n->d_ptabs, lc_poisson_table_floats(n_theta, n_phi));
    A(&n->d_pX, (size_t)n_theta * M);
    A(&n->d_pw, HW);
    A(&n->d_psi, HW);
    A(&n->d_ppart, HW / 256 + 2);
    A(&n->d_psum, 1);
    if (rc) {
        vlbm_lc_destroy(n);
        return rc;
    }
    // cell-centre sines (north half evaluated, mirrored) and the area-weight sum
    std::vector<double> sn(n_theta), cs(n_theta);
    const double dth = M_PI / n_theta;
    for (int i = 0; i < n_theta; ++i) {
        const int m = n_theta - 1 - i;
        sn[i] = (i <= m) ? std::sin((i + 0.5) * dth) : sn[m];
        cs[i] = (i < m) ? std::cos((i + 0.5) * dth) : (i == m ? 0.0 : -cs[m]);
    }
    for (int i = 0; i < n_theta; ++i) n->wsum += sn[i] * n_phi;
    if (cudaMemcpy(n->d_sin, sn.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->d_cos, cs.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->d_w, w.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
        lc_poisson_tables(n_theta, n_phi, n->d_ptabs) != 0 ||
        refresh_bf16(n) != VLBM_OK || cudaStreamSynchronize(n->stream) != cudaSuccess) {
        vlbm_lc_destroy(n);
        return VLBM_ERR_CUDA;
    }
    // the vorticity form's mode solve needs shared memory growing with n_theta: on grids taller
    // than one CTA can stage, that form alone is unavailable
    n->vort_ok = lc_poisson_prepare(n_theta) == 0;
    if (!n->vort_ok) cudaGetLastError();
    *out = n;
    return VLBM_OK;
}

int vlbm_lc_num_params(const vlbm_lc_t *n) { return n ? n->nparam : 0; }

int vlbm_lc_get_weights(vlbm_lc_t *n, float *w)
{
    if (!n || !w) return VLBM_ERR_ARG;
    LCK(n, cudaMemcpyAsync(w, n->d_w, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
    LCK(n, cudaStreamSynchronize(n->stream));
    return VLBM_OK;
}

int vlbm_lc_set_weights(vlbm_lc_t *n, const float *w)
{
    if (!n || !w) return VLBM_ERR_ARG;
    LCK(n, cudaMemcpyAsync(n->d_w, w, sizeof(float) * n->nparam, cudaMemcpyHostToDevice, n->stream));
    LCK(n, cudaMemsetAsync(n->d_m, 0, sizeof(float) * n->nparam, n->stream));
    LCK(n, cudaMemsetAsync(n->d_v, 0, sizeof(float) * n->nparam, n->stream));
    n->t = 0;
    int rc = refresh_bf16(n);
    if (rc) return rc;
    LCK(n, cudaStreamSynchronize(n->stream));
    return VLBM_OK;
}

int vlbm_lc_set_scales(vlbm_lc_t *n, const double *in_scale, const double *out_scale)
{
    if (!n || !in_scale || !out_scale) return VLBM_ERR_ARG;
    for (int q = 0; q < LC_NSCALE; ++q)
        if (!(in_scale[q] > 0.0)) return lfail(n, VLBM_ERR_ARG, "scales must be > 0");
    for (int q = 0; q < 3; ++q)
        if (!(out_scale[q] >= 0.0) || !std::isfinite(out_scale[q]))
            return lfail(n, VLBM_ERR_ARG, "output scales must be >= 0");
    for (int q = 0; q < LC_NSCALE; ++q) n->in_scale[q] = (float)in_scale[q];
    if (n->g_exec) {   // the scales are kernel arguments of the captured rollout step
        cudaGraphExecDestroy(n->g_exec);
        n->g_exec = nullptr;
    }
    for (int q = 0; q < 3; ++q) n->out_scale[q] = (float)out_scale[q];
    return VLBM_OK;
}

int vlbm_lc_set_output_form(vlbm_lc_t *n, int form, double radius)
{
    if (!n) return VLBM_ERR_ARG;
    if (form != VLBM_LC_DIRECT && form != VLBM_LC_STREAM && form != VLBM_LC_VORTICITY)
        return lfail(n, VLBM_ERR_ARG, "unknown output form");
    if (form == VLBM_LC_VORTICITY && !n->vort_ok)
        return lfail(n, VLBM_ERR_UNSUPPORTED, "the vorticity form's mode solve does not fit this many rows");
    if (!(radius > 0.0) || !std::isfinite(radius)) return lfail(n, VLBM_ERR_ARG, "radius must be > 0");
    if (n->g_exec) {   // the form is part of the captured rollout step
        cudaGraphExecDestroy(n->g_exec);
        n->g_exec = nullptr;
    }
    n->form = form;
    n->radius = radius;
    return VLBM_OK;
}

int vlbm_lc_predict(vlbm_lc_t *n, const double *inputs, double *outputs)
{
    if (!n || !inputs || !outputs) return VLBM_ERR_ARG;
    int rc;
    if ((rc = upload_io(n, inputs, nullptr)) || (rc = forward(n, n->d_dev, n->stream))) return rc;
    enqueue_outputs(n, n->stream);
    LCK(n, cudaMemcpyAsync(outputs, n->d_out, sizeof(double) * 3 * n->H * n->W, cudaMemcpyDeviceToHost, n->stream));
    LCK(n, cudaStreamSynchronize(n->stream));
    return VLBM_OK;
}

// training needs every output scale nonzero (the loss is taken on the scaled outputs)
static int check_trainable(vlbm_lc_t *n)
{
    for (int q = 0; q < 3; ++q)
        if (!(n->out_scale[q] > 0.0f)) return lfail(n, VLBM_ERR_ARG, "an output with scale 0 cannot be trained");
    return VLBM_OK;
}

int vlbm_lc_gradients(vlbm_lc_t *n, const double *inputs, const double *targets, double *loss, float *grad)
{
    if (!n || !inputs || !targets) return VLBM_ERR_ARG;
    if (int rc0 = check_trainable(n)) return rc0;
    int rc;
    if ((rc = upload_io(n, inputs, targets)) || (rc = forward(n, n->d_dev, n->stream)) || (rc = backward(n))) return rc;
    if (loss) LCK(n, cudaMemcpyAsync(loss, n->d_scal, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    if (grad) LCK(n, cudaMemcpyAsync(grad, n->d_g, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
    LCK(n, cudaStreamSynchronize(n->stream));
    return VLBM_OK;
}

int vlbm_lc_train_step(vlbm_lc_t *n, const double *inputs, const double *targets, float lr, double *loss)
{
    if (!n || !inputs || !targets || !(lr > 0.0f)) return VLBM_ERR_ARG;
    if (int rc0 = check_trainable(n)) return rc0;
    int rc;
    if ((rc = upload_io(n, inputs, targets)) || (rc = forward(n, n->d_dev, n->stream)) || (rc = backward(n))) return rc;
    n->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)n->t), c2 = 1.0f - std::pow(b2, (float)n->t);
    lc_adam(n->d_w, n->d_g, n->d_m, n->d_v, n->nparam, lr, b1, b2, 1e-8f, c1, c2, n->stream);
    if ((rc = refresh_bf16(n))) return rc;
    if (loss) LCK(n, cudaMemcpyAsync(loss, n->d_scal, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    LCK(n, cudaStreamSynchronize(n->stream));
    return VLBM_OK;
}

int vlbm_lc_apply(vlbm_lc_t *n, vlbm_t *h)
{
    int rc;
    if ((rc = check_solver(n, h)) || (rc = enqueue_correction(n, h, h->stream))) return rc;
    LCK(n, cudaStreamSynchronize(h->stream));
    return VLBM_OK;
}

int vlbm_lc_rollout(vlbm_lc_t *n, vlbm_t *h, int steps)
{
    int rc;
    if ((rc = check_solver(n, h))) return rc;
    if (steps < 0) return lfail(n, VLBM_ERR_ARG, "negative step count");
    if (steps == 0) return VLBM_OK;
    if (!h->d_row) return lfail(n, VLBM_ERR_ARG, "FP32 state not initialised");
    // the captured step holds the solver's launch parameters (its FP32 reference density among
    // them): rebuild for another solver or once the solver has renewed them
    if (n->g_exec && (n->g_solver != h || n->g_gen != h->step_gen)) {
        cudaGraphExecDestroy(n->g_exec);
        n->g_exec = nullptr;
    }
    if (!n->g_exec) {
        // one corrected coarse step (the solver's RK3 step, then the correction) as a graph
        cudaGraph_t g = nullptr;
        LCK(n, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        solver_enqueue_step(h);
        rc = enqueue_correction(n, h, h->stream);
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return lfail(n, VLBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&n->g_exec, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return lfail(n, VLBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        n->g_solver = h;
        n->g_gen = h->step_gen;
    }
    for (int q = 0; q < steps; ++q) LCK(n, cudaGraphLaunch(n->g_exec, h->stream));
    solver_count_steps(h, steps);
    if ((rc = vlbm_sync(h))) return lfail(n, rc, vlbm_last_error(h));
    return VLBM_OK;
}

const char *vlbm_lc_last_error(const vlbm_lc_t *n) { return n ? n->err.c_str() : ""; }

void vlbm_lc_destroy(vlbm_lc_t *n)
{
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    if (n->g_exec) cudaGraphExecDestroy(n->g_exec);
    for (void *p : n->bufs) cudaFree(p);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

}  // extern "C"
