// vlbm_api.cu -- host side of libvlbm.so: the C ABI of include/vlbm.h.
//
// Owns the device state of one solver (three population arrays for the SSP-RK3
// stages of arXiv 2504.15574 Sec. 3.7, per-row geometry tables, scratch for
// read-back and diagnostics), builds the FP64 tables of the velocity space
// (App. A.2) and of the grid (Sec. 3.4), encodes the TMA descriptors of the
// FP32 path, and enqueues steps as CUDA graphs on the handle's stream.
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/vlbm.h"
#include "vlbm_internal.h"
#include "vlbm_handle.h"

using namespace vk;

namespace {

thread_local std::string g_create_error;

int fail(vlbm_t *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(h, call)                                                                                       \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail((h), VLBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

// ---- velocity space (App. A.2), FP64 --------------------------------------------
// He_l by the three-term recurrence He_{l+1} = x He_l - l He_{l-1}.
double hermite_he(int l, double x)
{
    double prev = 1.0, cur = x;
    if (l == 0) return 1.0;
    for (int m = 1; m < l; ++m) {
        double next = x * cur - (double)m * prev;
        prev = cur;
        cur = next;
    }
    return cur;
}

double fact(int l)
{
    double r = 1.0;
    for (int m = 2; m <= l; ++m) r *= (double)m;
    return r;
}

// Velocity set of order q: ascending roots of He_q (q = 4: x^4 - 6x^2 + 3, App. A.2; q = 3:
// x^3 - 3x, App. A.1), weights q!/He_{q+1}(v)^2 (Eq. GH_weights), kernels of Eqs. (KH), (KtildeH)
// row-major q x q.
void velocity_tables(VelD &c, int q)
{
    c = VelD{};
    c.q = q;
    if (q == 3) {
        c.v[0] = -std::sqrt(3.0);
        c.v[1] = 0.0;
        c.v[2] = std::sqrt(3.0);
    } else {
        const double outer = std::sqrt(3.0 + std::sqrt(6.0));
        const double inner = std::sqrt(3.0 - std::sqrt(6.0));
        c.v[0] = -outer;
        c.v[1] = -inner;
        c.v[2] = inner;
        c.v[3] = outer;
    }
    for (int a = 0; a < q; ++a) {
        const double h = hermite_he(q + 1, c.v[a]);
        c.w[a] = fact(q) / (h * h);
    }
    for (int k = 0; k < q; ++k)
        for (int kp = 0; kp < q; ++kp) {
            double sk = 0.0, skt = 0.0;
            for (int l = 0; l < q; ++l) {
                const double hk = hermite_he(l + 1, c.v[k]);
                sk += hk * hermite_he(l, c.v[kp]) / fact(l);
                double inner_l = hermite_he(l + 1, c.v[kp]);
                if (l > 0) inner_l += (double)l * hermite_he(l - 1, c.v[kp]);
                skt += hk * inner_l / fact(l);
            }
            c.K[k * q + kp] = -c.w[k] * sk;
            c.Kt[k * q + kp] = -c.w[k] * skt;
        }
}

// ---- grid (Eq. discrete_coord_sphere): north half evaluated, south half mirrored
void row_tables(int nt, std::vector<double> &s, std::vector<double> &c)
{
    s.assign(nt, 0.0);
    c.assign(nt, 0.0);
    const double dth = M_PI / (double)nt;
    for (int i = 0; i < nt; ++i) {
        const int m = nt - 1 - i;
        if (i <= m) {
            const double th = ((double)i + 0.5) * dth;
            s[i] = std::sin(th);
            c[i] = (i == m) ? 0.0 : std::cos(th);
        } else {
            s[i] = s[m];
            c[i] = -c[m];
        }
    }
}

// sin(theta) of padded row pr (row r = pr - GR); ghost rows carry the sine of their own angle
double sin_padded(const std::vector<double> &s, int nt, int pr)
{
    const int r = pr - GR;
    if (r < 0) return -s[-1 - r];
    if (r >= nt) return -s[2 * nt - 1 - r];
    return s[r];
}

// Polar ring filter block size (not in the paper): smallest power of two b with
// b sin(theta) dphi >= dtheta / 4, dividing n_phi.
int filter_block(int nt, int np, double sin_i)
{
    if (np < 2) return 1;
    const double want = (M_PI / nt) / (4.0 * sin_i * (2.0 * M_PI / np));
    int b = 1;
    while ((double)b < want && b < np) b *= 2;
    while (np % b != 0) b /= 2;
    return b;
}

template <typename T>
int upload(vlbm_t *h, T **dst, const T *src, size_t n)
{
    if (!*dst) {
        CK(h, cudaMalloc((void **)dst, n * sizeof(T)));
        h->dev_bytes += n * sizeof(T);
    }
    CK(h, cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return VLBM_OK;
}

int dalloc(vlbm_t *h, void **p, size_t bytes)
{
    CK(h, cudaMalloc(p, bytes));
    CK(h, cudaMemset(*p, 0, bytes));
    h->dev_bytes += bytes;
    return VLBM_OK;
}

// FP32 tables that depend on rho_ref: packed velocity constants, per-face sine forms,
// per-row constants and the per-row tendency of the reference state (times sin(theta)).
int build_f32_tables(vlbm_t *h)
{
    const int nt = h->nt;
    const double R = h->R, dth = M_PI / nt, dph = 2.0 * M_PI / h->np;
    const VelD &c = h->vd;
    const int q = c.q, npq = f32_pairs(q);
    const double rr = h->rho_ref, ks = h->kscale;
    RunF &run = h->run;
    if (q == 4) {
        VelC &f = h->vc;
        for (int g = 0; g < 2; ++g) f.vth[g] = make_float2((float)c.v[2 * g], (float)c.v[2 * g + 1]);
        for (int b = 0; b < 4; ++b) f.vphi2[b] = make_float2((float)c.v[b], (float)c.v[b]);
        for (int p = 0; p < 8; ++p) {
            const int g = p / 4, b = p % 4, a0 = 2 * g, a1 = 2 * g + 1;
            f.w2[p] = make_float2((float)(c.w[a0] * c.w[b]), (float)(c.w[a1] * c.w[b]));
            const double vb2 = c.v[b] * c.v[b];
            f.kf[p][0] = make_float2((float)(vb2 * c.K[a0 * 4 + 0]), (float)(vb2 * c.K[a1 * 4 + 1]));
            f.kf[p][1] = make_float2((float)(vb2 * c.K[a0 * 4 + 1]), (float)(vb2 * c.K[a1 * 4 + 0]));
            f.kf[p][2] = make_float2((float)(vb2 * c.K[a0 * 4 + 2]), (float)(vb2 * c.K[a1 * 4 + 3]));
            f.kf[p][3] = make_float2((float)(vb2 * c.K[a0 * 4 + 3]), (float)(vb2 * c.K[a1 * 4 + 2]));
            for (int m = 0; m < 4; ++m)
                f.ktf[p][m] = make_float2((float)(-c.v[a0] * c.Kt[b * 4 + m]), (float)(-c.v[a1] * c.Kt[b * 4 + m]));
        }
    } else {
        // D2Q9 in five pairs: per member its velocity and weight (0 for the empty slot), per
        // pair the common sign of the nonzero v_theta and v_phi, per slot the force bracket's
        // coefficients v_phi^2 K[a][a'] (on population (a', b)) and -v_theta Ktilde[b][b'] (on (a, b'))
        VelC3 &f = h->vc3;
        f = VelC3{};
        for (int p = 0; p < npq; ++p) {
            float vt[2], vb[2], w[2];
            int sth = 0, sph = 0;
            for (int m = 0; m < 2; ++m) {
                const int k = f32_pop_of_slot(q, 2 * p + m);
                vt[m] = vb[m] = w[m] = 0.0f;
                if (k < 0) continue;
                const int a = k / q, b = k % q;
                vt[m] = (float)c.v[a];
                vb[m] = (float)c.v[b];
                w[m] = (float)(c.w[a] * c.w[b]);
                const int st = (c.v[a] > 0) - (c.v[a] < 0), sp = (c.v[b] > 0) - (c.v[b] < 0);
                if ((st && sth && st != sth) || (sp && sph && sp != sph))
                    return fail(h, VLBM_ERR_UNSUPPORTED, "FP32 pair members with opposite velocity signs");
                if (st) sth = st;
                if (sp) sph = sp;
            }
            f.vt2[p] = make_float2(vt[0], vt[1]);
            f.vb2[p] = make_float2(vb[0], vb[1]);
            f.w2[p] = make_float2(w[0], w[1]);
            f.thdir[p] = sth;
            f.phdir[p] = sph;
        }
        for (int t = 0; t < 2 * npq; ++t) {
            const int k = f32_pop_of_slot(q, t);
            if (k < 0) continue;
            const int a = k / q, b = k % q;
            for (int m = 0; m < 3; ++m) {
                f.fcoef[t][m] = (float)(c.v[b] * c.v[b] * c.K[a * 3 + m]);
                f.fcoef[t][3 + m] = (float)(-c.v[a] * c.Kt[b * 3 + m]);
            }
        }
    }
    for (int p = 0; p < npq; ++p) {
        double wr[2];
        for (int m = 0; m < 2; ++m) {
            const int k = f32_pop_of_slot(q, 2 * p + m);
            wr[m] = (k < 0) ? 0.0 : ks * c.w[k / q] * c.w[k % q] * rr;
        }
        run.wr[p] = make_float2((float)wr[0], (float)wr[1]);
    }
    run.rho_ref = (float)rr;

    // upwind schemes (Eq. fluxes_U1-3): value = lin0 x_up2 + lin1 x_up + lin2 x_down
    double lin[3] = {0.0, 1.0, 0.0};
    if (h->scheme == VLBM_U2) {
        lin[0] = -0.5;
        lin[1] = 1.5;
    } else if (h->scheme == VLBM_U3) {
        lin[0] = -1.0 / 6.0;
        lin[1] = 5.0 / 6.0;
        lin[2] = 1.0 / 3.0;
    }
    run.lin0 = (float)lin[0];
    run.lin1 = (float)lin[1];
    run.lin2 = (float)lin[2];
    run.komissarov = h->komissarov;
    // the interface value of sin(theta) at faces fi = 0..nt (between rows fi-1 and fi) per
    // upwind direction: for WENO-5 the candidate P2 (the kernel adds the nonlinear weight terms
    // of the full g to P2 of the deviation), for the upwind schemes their linear stencil
    std::vector<double> plin(2 * (size_t)(nt + 1));
    for (int fi = 0; fi <= nt; ++fi)
        for (int dir = 0; dir < 2; ++dir) {
            double x[5];
            for (int m = 0; m < 5; ++m) {
                const int r = (dir == 0) ? (fi - 3 + m) : (fi + 2 - m);
                x[m] = sin_padded(h->sin_t, nt, r + GR);
            }
            const double b = x[1], cc = x[2], d = x[3];
            plin[2 * fi + dir] = (h->scheme == VLBM_WENO5) ? (-b + 5 * cc + 2 * d) / 6.0
                                                           : lin[0] * b + lin[1] * cc + lin[2] * d;
        }
    // the reference state's pole fluxes summed over the columns: n_phi sum_k v_theta w_k rho_ref times
    // the pole face's interface value of sin (its reconstruction per upwind direction); no flux
    // crosses a pole with the Komissarov interface sines
    h->pole_ref[0] = h->pole_ref[1] = 0.0;
    if (!h->komissarov)
        for (int k = 0; k < q * q; ++k) {
            const int a = k / q, b = k % q;
            const int dir = c.v[a] > 0 ? 0 : 1;
            const double wr = c.w[a] * c.w[b] * rr;
            h->pole_ref[0] += c.v[a] * wr * plin[2 * 0 + dir];
            h->pole_ref[1] += c.v[a] * wr * plin[2 * (size_t)nt + dir];
        }
    h->pole_ref[0] *= h->np;
    h->pole_ref[1] *= h->np;
    std::vector<RowF> row(nt);
    std::vector<float2> rref((size_t)nt * npq);
    std::vector<float> kss(nt), ikss(nt);
    for (int i = 0; i < nt; ++i) {
        kss[i] = (float)(ks * h->sin_t[i]);
        ikss[i] = (float)(1.0 / (ks * h->sin_t[i]));
    }
    for (int i = 0; i < nt; ++i) {
        const double s = h->sin_t[i], cot = h->cos_t[i] / h->sin_t[i];
        RowF rc;
        rc.s = (float)(ks * s);
        rc.inv_s = (float)(1.0 / (ks * s));
        rc.inv_dph = (float)(1.0 / (R * s * dph));
        rc.cotR = (float)(cot / R);
        rc.ephi = (float)(4.0 * h->eps * s * s * ks * ks);
        rc.kth = (float)(s / (R * (h->cos_f[i] - h->cos_f[i + 1])));
        rc.pad1 = rc.pad2 = 0.0f;
        row[i] = rc;
        double rk[NK];
        for (int k = 0; k < q * q; ++k) {
            const int a = k / q, b = k % q;
            const double va = c.v[a], vb = c.v[b];
            const double wr = c.w[a] * c.w[b] * rr;
            const int dir = va > 0 ? 0 : 1;
            // theta advection of the reference part (WENO-5: its P2; the upwind schemes are
            // linear, so theirs is exact; Komissarov: the interface sines of v_theta w rho_ref),
            // and its force
            double adv;
            if (h->komissarov)
                adv = -va * wr * (h->sin_f[i + 1] - h->sin_f[i]) / (R * (h->cos_f[i] - h->cos_f[i + 1]));
            else
                adv = -va * wr * (plin[2 * (i + 1) + dir] - plin[2 * i + dir]) / (R * s * dth);
            double kw = 0.0, ktw = 0.0;
            for (int m = 0; m < q; ++m) {
                kw += c.K[a * q + m] * c.w[m] * c.w[b] * rr;
                ktw += c.Kt[b * q + m] * c.w[a] * c.w[m] * rr;
            }
            const double force = cot / R * (vb * vb * kw - va * ktw);
            rk[k] = ks * s * (adv - force);
        }
        for (int p = 0; p < npq; ++p) {
            const int k0 = f32_pop_of_slot(q, 2 * p), k1 = f32_pop_of_slot(q, 2 * p + 1);
            rref[(size_t)i * npq + p] =
                make_float2(k0 < 0 ? 0.0f : (float)rk[k0], k1 < 0 ? 0.0f : (float)rk[k1]);
        }
    }
    // differences of sin at padded rows (pr-1, pr, pr+1 inside [0, nt + 2GR))
    const int npr = nt + 2 * GR + F32_TILE_ROWS_MAX;
    std::vector<float> ds(npr, 0.0f), d2s(npr, 0.0f);
    for (int pr = 0; pr < npr; ++pr) {
        if (pr >= 1 && pr < nt + 2 * GR)
            ds[pr] = (float)(sin_padded(h->sin_t, nt, pr) - sin_padded(h->sin_t, nt, pr - 1));
        if (pr >= 1 && pr + 1 < nt + 2 * GR)
            d2s[pr] = (float)(sin_padded(h->sin_t, nt, pr - 1) - 2.0 * sin_padded(h->sin_t, nt, pr) +
                              sin_padded(h->sin_t, nt, pr + 1));
    }
    // upwind schemes: 1/sin at padded rows (negative at ghost rows) and the interface sines
    std::vector<float> isp(npr, 0.0f), sfc(nt + 1 + F32_TILE_ROWS_MAX, 0.0f);
    for (int pr = 0; pr < nt + 2 * GR; ++pr) isp[pr] = (float)(1.0 / sin_padded(h->sin_t, nt, pr));
    for (int fi = 0; fi <= nt; ++fi) sfc[fi] = (float)h->sin_f[fi];
    int rc;
    if ((rc = upload(h, &h->d_isp, isp.data(), isp.size())) || (rc = upload(h, &h->d_sfc, sfc.data(), sfc.size())))
        return rc;
    run.isp = h->d_isp;
    run.sfc = h->d_sfc;
    if ((rc = upload(h, &h->d_dsin, ds.data(), ds.size()))) return rc;
    if ((rc = upload(h, &h->d_d2sin, d2s.data(), d2s.size()))) return rc;
    if ((rc = upload(h, &h->d_row, row.data(), row.size()))) return rc;
    if ((rc = upload(h, &h->d_rref, rref.data(), rref.size()))) return rc;
    run.F = (float2 *)h->F;
    run.A = (float2 *)h->A;
    run.B = (float2 *)h->B;
    run.row = h->d_row;
    run.rref = h->d_rref;
    run.dsin = h->d_dsin;
    run.d2sin = h->d_d2sin;
    run.L = h->L;
    run.tau_inv = (float)(1.0 / h->tau);
    run.dt = (float)h->dt;
    run.e_theta = (float)(4.0 * h->eps * ks * ks);
    run.inv_dth = (float)(1.0 / (h->R * (M_PI / h->nt)));
    run.tiles_x = (h->np + F32_TILE_COLS - 1) / F32_TILE_COLS;
    run.pole_part = h->komissarov ? nullptr : h->d_pole_part;
    run.wait_ns = h->wait_ns;
    if ((rc = upload(h, &h->d_kss, kss.data(), kss.size())) || (rc = upload(h, &h->d_ikss, ikss.data(), ikss.size())))
        return rc;
    // the persistent stage kernel's per-tile-row tables of the three stages (8-row tiles)
    if (h->ty == 8) {
        const size_t per = f32_tile_table_bytes(q), n = 3 * (size_t)((nt + 7) / 8) * per;
        std::vector<unsigned char> tabs(n);
        f32_fill_tile_tables(q, nt, run.dt, ds.data(), d2s.data(), isp.data(), sfc.data(), row.data(), rref.data(),
                             tabs.data());
        if ((rc = upload(h, &h->d_tabs, tabs.data(), tabs.size()))) return rc;
    }
    return VLBM_OK;
}

// Tensor map of an FP32 pair array: the stage input box (F32_BOX_COLS x (ty + 2 GR) x all pair
// planes, anchored GC columns and GR rows before the tile) or, with core set, the tile itself
// (F32_TILE_COLS x ty x all pair planes: 8 for D2Q16, 5 for D2Q9).
int encode_map(vlbm_t *h, CUtensorMap *m, void *base, int ty = 0, bool core = false)
{
    if (ty == 0) ty = h->ty;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        CK(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn)
            return fail(h, VLBM_ERR_CUDA, "cuTensorMapEncodeTiled not available from the driver");
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    // pair planes of float2, described as 8-byte elements
    const int npq = f32_pairs(h->vd.q);
    cuuint64_t dims[3] = {(cuuint64_t)h->L.pitch, (cuuint64_t)(h->nt + 2 * GR), (cuuint64_t)npq};
    cuuint64_t strides[2] = {(cuuint64_t)h->L.pitch * sizeof(float2), (cuuint64_t)h->L.plane * sizeof(float2)};
    cuuint32_t box[3] = {(cuuint32_t)(core ? F32_TILE_COLS : F32_BOX_COLS), (cuuint32_t)(core ? ty : ty + 2 * GR),
                         (cuuint32_t)npq};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, VLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return VLBM_OK;
}

// slot: the persistent kernel's tile counters (0: whole-grid launches, 1: polar band, 2: interior band;
// launches that may overlap take different slots)
void launch_stage_f32_any(vlbm_t *h, int st, cudaStream_t s, TileRows rows = TileRows{0, -1, 0, 0}, int slot = 0)
{
    const CUtensorMap &tm = (st == 1) ? h->tmF : (st == 2) ? h->tmA : h->tmB;
    const CUtensorMap &tmo = (st == 1) ? h->tmAc : (st == 2) ? h->tmBc : h->tmFc;
    const bool lin = h->scheme != VLBM_WENO5;
    if (h->ty == 8 && lin) {
        // the upwind schemes: the persistent kernel, whose next tile's copies are in flight during
        // the cell phase (their lighter faces leave the one-tile kernel's loads exposed; for WENO-5
        // the one-tile kernel with three resident CTAs per SM measured faster)
        unsigned *ctr = h->d_ctr + 2 * slot;
        if (h->vd.q == 3)
            launch_stage_f32_persist_q3(tm, tmo, h->tmFc, h->run, h->vc3, st, lin, h->d_tabs, h->d_flags, ctr, s,
                                        rows);
        else
            launch_stage_f32_persist(tm, tmo, h->tmFc, h->run, h->vc, st, lin, h->d_tabs, h->d_flags, ctr, s, rows);
        return;
    }
    if (h->vd.q == 3) launch_stage_f32_q3(tm, tmo, h->tmFc, h->run, h->vc3, st, h->ty, lin, h->d_flags, s, rows);
    else launch_stage_f32(tm, tmo, h->tmFc, h->run, h->vc, st, h->ty, lin, h->d_flags, s, rows);
}

// The FP32 step's pole mass-flux budget from the stage kernels' pole partials
void launch_budget_f32(vlbm_t *h, cudaStream_t s)
{
    launch_pole_budget_f32(h->d_pole_part, h->run.tiles_x, h->pole_ref[0], h->pole_ref[1], h->kscale, h->R,
                           2.0 * M_PI / h->np, h->dt, h->d_budget, s);
}

// One FP32 RK3 step with the polar filter.  The tile rows touching a filtered row and the filter
// run on stream2, created with the highest priority so that their CTAs go first; the tile rows
// clear of the filtered rows run on the handle's stream.  A stage's interior launch reads rows
// that the previous stage's filter leaves alone, so it waits for that stage's two launches only
// and runs beside the filter; the polar launch waits for the previous stage's interior launch
// and, in stream order, its polar launch and filter.  The step starts and ends joined on the
// handle's stream.
void enqueue_split_step(vlbm_t *h)
{
    cudaStream_t s = h->stream, s2 = h->stream2;
    const int tiles_y = (h->nt + h->ty - 1) / h->ty, nb = h->band_hi - h->band_lo;
    const TileRows inner{h->band_lo, nb, 1 << 30, 0};
    const TileRows polar{0, tiles_y - nb, h->band_lo, nb};
    cudaEvent_t *evP = h->evs + 1, *evI = h->evs + 4;
    cudaEventRecord(h->evs[0], s);
    cudaStreamWaitEvent(s2, h->evs[0], 0);
    for (int st = 1; st <= 3; ++st) {
        void *out = (st == 1) ? h->A : (st == 2) ? h->B : h->F;
        if (st > 1) cudaStreamWaitEvent(s2, evI[st - 2], 0);
        launch_stage_f32_any(h, st, s2, polar, 1);
        cudaEventRecord(evP[st - 1], s2);
        launch_filter_f32((float2 *)out, h->L, h->vd.q, h->d_frows, h->d_fblocks, h->nfrows, s2);
        if (st > 1) cudaStreamWaitEvent(s, evP[st - 2], 0);
        launch_stage_f32_any(h, st, s, inner, 2);
        cudaEventRecord(evI[st - 1], s);
    }
    // the step's pole budget: its partials come from the polar launches, all on stream2
    if (h->run.pole_part) launch_budget_f32(h, s2);
    cudaEventRecord(h->evs[0], s2);
    cudaStreamWaitEvent(s, h->evs[0], 0);
}

// Enqueues one RK3 step (all stages, filters, budget) on the handle's stream.  With
// stage_only = 1..3, only that stage; part 1 launches its stage kernel alone, part 2
// its polar filter alone (part 0: both).
void enqueue_step(vlbm_t *h, int stage_only = 0, int part = 0)
{
    if (h->prec == VLBM_FP32 && !stage_only && h->band_hi > h->band_lo) {
        enqueue_split_step(h);
        return;
    }
    cudaStream_t s = h->stream;
    const size_t pole_per = (size_t)2 * NK * h->np;
    for (int st = 1; st <= 3; ++st) {
        if (stage_only && stage_only != st) continue;
        void *in = (st == 1) ? h->F : (st == 2) ? h->A : h->B;
        void *out = (st == 1) ? h->A : (st == 2) ? h->B : h->F;
        if (h->prec == VLBM_FP64) {
            StageD p;
            p.in = (const double *)in;
            p.fold = (const double *)h->F;
            p.out = (double *)out;
            p.sin_ext = h->d_sin_ext;
            p.cot = h->d_cot;
            p.pole = h->d_pole + (size_t)(st - 1) * pole_per;
            p.L = h->L;
            p.dth = M_PI / h->nt;
            p.dph = 2.0 * M_PI / h->np;
            p.R = h->R;
            p.tau = h->tau;
            p.dt = h->dt;
            p.eps = h->eps;
            p.stage = st;
            p.c = h->vd;
            p.scheme = h->scheme;
            p.komissarov = h->komissarov;
            p.sin_f = h->d_sin_f;
            p.cos_f = h->d_cos_f;
            p.Ft = h->d_ft;
            p.Fp = h->d_fp;
            if (part != 2) launch_stage_f64(p, s);
            if (h->nfrows && part != 1) launch_filter_f64((double *)out, h->L, h->d_frows, h->d_fblocks, h->nfrows, s);
        } else {
            if (part != 2) launch_stage_f32_any(h, st, s);
            if (h->nfrows && part != 1)
                launch_filter_f32((float2 *)out, h->L, h->vd.q, h->d_frows, h->d_fblocks, h->nfrows, s);
        }
    }
    if (!stage_only && h->prec == VLBM_FP64)
        launch_pole_budget(h->d_pole, h->np, h->R, 2.0 * M_PI / h->np, h->dt, h->d_budget, s);
    if (!stage_only && h->prec == VLBM_FP32 && h->run.pole_part) launch_budget_f32(h, s);
}

int kernels_per_step(const vlbm_t *h)
{
    int n = 3 + (h->nfrows ? 3 : 0) + (h->band_hi > h->band_lo ? 3 : 0);
    if (h->prec == VLBM_FP64) n += 3 * 2 + 1;   // two face kernels per stage and the pole budget
    else if (h->run.pole_part) n += 1;          // the pole budget
    return n;
}

int build_graph(vlbm_t *h, int nsteps, cudaGraphExec_t *exec)
{
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < nsteps; ++q) enqueue_step(h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return fail(h, VLBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    // (node priorities: the kernels captured from the high-priority stream keep it)
    e = cudaGraphInstantiate(exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, VLBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return VLBM_OK;
}

// Generations of the captured step: unique over the process, so that a graph holding a solver's
// step (the learned correction's rollout) can tell a rebuilt step, or another solver at the same
// address, from the one it captured.
std::atomic<unsigned long long> g_step_generation{0};

void drop_graphs(vlbm_t *h)
{
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->g16) cudaGraphExecDestroy(h->g16);
    h->g1 = h->g16 = nullptr;
    h->step_gen = ++g_step_generation;
}

// After the populations changed from outside a step: ghosts, counters, mass0.
int after_reset(vlbm_t *h)
{
    if (h->prec == VLBM_FP64) launch_fill_ghosts_f64((double *)h->F, h->L, h->stream);
    else launch_fill_ghosts_f32((float2 *)h->F, h->L, h->vd.q, h->stream);
    CK(h, cudaMemsetAsync(h->d_budget, 0, sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->d_flags, 0, sizeof(unsigned) * 4, h->stream));
    CK(h, cudaGetLastError());
    h->steps = 0;
    vlbm_diag d;
    int rc = vlbm_diagnostics(h, &d);
    if (rc) return rc;
    h->mass0 = d.mass;
    return VLBM_OK;
}

// rho_ref of the FP32 deviation storage: the option, else the area-weighted mean of the density
// field d_rho (device, [nt][np]), reduced on the device in a fixed order (the same value on every
// call for the same field) and read back.
int choose_rho_ref(vlbm_t *h, const double *d_rho)
{
    if (h->rho_ref_opt > 0.0) {
        h->rho_ref = h->rho_ref_opt;
        return VLBM_OK;
    }
    launch_rho_ref(d_rho, h->nt, h->np, h->d_sin_t, h->d_part, h->d_scalar, h->stream);
    CK(h, cudaGetLastError());
    double v = 0.0;
    CK(h, cudaMemcpyAsync(&v, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->rho_ref = v;
    return VLBM_OK;
}

}  // namespace

void solver_enqueue_step(vlbm_t *h) { enqueue_step(h); }

void solver_count_steps(vlbm_t *h, int n) { h->steps += n; }

extern "C" {

void vlbm_default_options(vlbm_options *opt)
{
    if (!opt) return;
    opt->precision = VLBM_FP64;
    opt->weno_eps = 1e-6;
    opt->radius = 1.0;
    opt->polar_filter = 0;
    opt->guard = 1;
    opt->stream = nullptr;
    opt->rho_ref = 0.0;
    opt->tile_rows = 0;
    opt->scheme = VLBM_WENO5;
    opt->komissarov = 0;
    opt->velocity_set = VLBM_D2Q16;
}

int vlbm_create(int n_theta, int n_phi, int velocity_set, double tau, double dt, const vlbm_options *opt,
                vlbm_t **out)
{
    if (!out) return fail(nullptr, VLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (velocity_set != VLBM_D2Q9 && velocity_set != VLBM_D2Q16)
        return fail(nullptr, VLBM_ERR_ARG, "unknown velocity set");
    if (n_theta < 6 || n_theta > 65536) return fail(nullptr, VLBM_ERR_ARG, "n_theta must be in [6, 65536]");
    if (n_phi < 1 || n_phi > 65536 || (n_phi != 1 && n_phi % 2 != 0))
        return fail(nullptr, VLBM_ERR_ARG, "n_phi must be 1 or even, at most 65536");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(nullptr, VLBM_ERR_ARG, "tau must be > 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, VLBM_ERR_ARG, "dt must be > 0");
    vlbm_options o;
    vlbm_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != VLBM_FP64 && o.precision != VLBM_FP32) return fail(nullptr, VLBM_ERR_ARG, "bad precision");
    if (!(o.weno_eps > 0.0) || !(o.radius > 0.0)) return fail(nullptr, VLBM_ERR_ARG, "weno_eps and radius must be > 0");
    if (o.scheme < VLBM_WENO5 || o.scheme > VLBM_U3) return fail(nullptr, VLBM_ERR_ARG, "unknown advection scheme");
    if (o.tile_rows != 0 && o.tile_rows != 4 && o.tile_rows != 8)
        return fail(nullptr, VLBM_ERR_ARG, "tile_rows must be 0, 4 or 8");

    vlbm_t *h = new vlbm_t();
    h->step_gen = ++g_step_generation;
    h->nt = n_theta;
    h->np = n_phi;
    h->prec = o.precision;
    h->tau = tau;
    h->dt = dt;
    h->eps = o.weno_eps;
    h->kscale = (o.precision == VLBM_FP32) ? f32_state_scale(o.weno_eps) : 1.0;
    h->R = o.radius;
    h->filter = o.polar_filter ? 1 : 0;
    h->guard = o.guard ? 1 : 0;
    h->rho_ref_opt = o.rho_ref;
    h->ty = (o.tile_rows == 4) ? 4 : 8;
    h->scheme = o.scheme;
    h->komissarov = o.komissarov ? 1 : 0;
    h->elem = (h->prec == VLBM_FP64) ? sizeof(double) : sizeof(float);
    h->L.nt = n_theta;
    h->L.np = n_phi;
    h->L.pitch = ((n_phi + 2 * GC) + 3) / 4 * 4;
    h->L.plane = (size_t)(n_theta + 2 * GR) * (size_t)h->L.pitch;
    h->L.nk = velocity_set * velocity_set;
    // FP32: pair planes of float2 (D2Q9's fifth pair has one empty member)
    h->arr_bytes = (h->prec == VLBM_FP64) ? (size_t)h->L.nk * h->L.plane * sizeof(double)
                                          : (size_t)f32_pairs(velocity_set) * h->L.plane * sizeof(float2);
    velocity_tables(h->vd, velocity_set);
    row_tables(n_theta, h->sin_t, h->cos_t);

    auto bail = [&](int rc) {
        std::string m = h->err;
        vlbm_destroy(h);
        g_create_error = m;
        return rc;
    };
    int rc;
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        delete h;
        return fail(nullptr, VLBM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(ce));
    }
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(nullptr, VLBM_ERR_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    if ((rc = dalloc(h, &h->F, h->arr_bytes)) || (rc = dalloc(h, &h->A, h->arr_bytes)) ||
        (rc = dalloc(h, &h->B, h->arr_bytes)))
        return bail(rc);
    // geometry
    std::vector<double> sext(n_theta + 2 * GR + F32_TILE_ROWS_MAX, 0.0), cot(n_theta);
    for (int pr = 0; pr < n_theta + 2 * GR; ++pr) sext[pr] = sin_padded(h->sin_t, n_theta, pr);
    for (int i = 0; i < n_theta; ++i) cot[i] = h->cos_t[i] / h->sin_t[i];
    if ((rc = upload(h, &h->d_sin_ext, sext.data(), sext.size())) || (rc = upload(h, &h->d_cot, cot.data(), cot.size())) ||
        (rc = upload(h, &h->d_sin_t, h->sin_t.data(), h->sin_t.size())) ||
        (rc = upload(h, &h->d_cos_t, h->cos_t.data(), h->cos_t.size())))
        return bail(rc);
    // theta interfaces fi = 0..nt at theta = fi dtheta, northern half computed and mirrored (the
    // Komissarov flux; sin = 0 exactly at both poles, cos = 0 exactly at the equator)
    h->sin_f.assign(n_theta + 1, 0.0);
    h->cos_f.assign(n_theta + 1, 0.0);
    for (int fi = 0; fi <= n_theta; ++fi) {
        const int m = n_theta - fi;
        if (fi <= m) {
            h->sin_f[fi] = (fi == 0) ? 0.0 : std::sin(fi * (M_PI / n_theta));
            h->cos_f[fi] = (fi == m) ? 0.0 : std::cos(fi * (M_PI / n_theta));
        } else {
            h->sin_f[fi] = h->sin_f[m];
            h->cos_f[fi] = -h->cos_f[m];
        }
    }
    if ((rc = upload(h, &h->d_sin_f, h->sin_f.data(), h->sin_f.size())) ||
        (rc = upload(h, &h->d_cos_f, h->cos_f.data(), h->cos_f.size())))
        return bail(rc);
    if (h->prec == VLBM_FP64 &&
        ((rc = dalloc(h, (void **)&h->d_ft, sizeof(double) * h->L.nk * (size_t)(n_theta + 1) * n_phi)) ||
         (rc = dalloc(h, (void **)&h->d_fp, sizeof(double) * h->L.nk * (size_t)n_theta * (n_phi + 1)))))
        return bail(rc);
    // polar filter rows
    if (h->filter) {
        std::vector<int> rows, blocks;
        for (int i = 0; i < n_theta; ++i) {
            const int b = filter_block(n_theta, n_phi, h->sin_t[i]);
            if (b > 1) {
                rows.push_back(i);
                blocks.push_back(b);
            }
        }
        h->nfrows = (int)rows.size();
        if (h->nfrows &&
            ((rc = upload(h, &h->d_frows, rows.data(), rows.size())) || (rc = upload(h, &h->d_fblocks, blocks.data(), blocks.size()))))
            return bail(rc);
        // FP32: the tile rows whose stage input box (GR rows beyond the tile on each side)
        // touches no filtered row
        int iN = -1, iS = n_theta;
        for (int i : rows) {
            if (2 * i < n_theta) iN = std::max(iN, i);
            else iS = std::min(iS, i);
        }
        const int ty = h->ty, lo = (iN + GR + 1 + ty - 1) / ty;
        const int hi = (iS - GR - ty >= 0) ? (iS - GR - ty) / ty + 1 : 0;
        if (h->prec == VLBM_FP32 && h->nfrows && hi > lo) {
            h->band_lo = lo;
            h->band_hi = hi;
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            if (cudaStreamCreateWithPriority(&h->stream2, cudaStreamNonBlocking, greatest) != cudaSuccess) {
                h->err = "cudaStreamCreate failed";
                return bail(VLBM_ERR_CUDA);
            }
            for (cudaEvent_t &e : h->evs)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                    h->err = "cudaEventCreate failed";
                    return bail(VLBM_ERR_CUDA);
                }
        }
    }
    if ((rc = dalloc(h, (void **)&h->d_pole, sizeof(double) * 3 * 2 * NK * (size_t)n_phi)) ||
        (rc = dalloc(h, (void **)&h->d_budget, sizeof(double) * 8)) ||
        (rc = dalloc(h, (void **)&h->d_mom, sizeof(double) * 4 * (size_t)n_theta * n_phi)) ||
        (rc = dalloc(h, (void **)&h->d_part, sizeof(double) * diag_partials(h->L))) ||
        (rc = dalloc(h, (void **)&h->d_diag, sizeof(double) * 8)) ||
        (rc = dalloc(h, (void **)&h->d_flags, sizeof(unsigned) * 4)))
        return bail(rc);
    if (h->prec == VLBM_FP32) {
        // FP32 diagnostics: cos and sin of the column angles; the stage kernels' pole partials
        std::vector<double> cph(n_phi), sph(n_phi);
        const double dph = 2.0 * M_PI / n_phi;
        for (int j = 0; j < n_phi; ++j) {
            cph[j] = std::cos((j + 0.5) * dph);
            sph[j] = std::sin((j + 0.5) * dph);
        }
        const int ntx = (n_phi + F32_TILE_COLS - 1) / F32_TILE_COLS;
        if ((rc = upload(h, &h->d_cph, cph.data(), cph.size())) || (rc = upload(h, &h->d_sph, sph.data(), sph.size())) ||
            (rc = dalloc(h, (void **)&h->d_pole_part, sizeof(double) * 3 * 2 * (size_t)ntx)) ||
            (rc = dalloc(h, (void **)&h->d_ctr, sizeof(unsigned) * 6)) ||
            (rc = dalloc(h, (void **)&h->d_scalar, sizeof(double) * 8)))
            return bail(rc);
    }
    if (cudaMallocHost((void **)&h->h_flags, sizeof(unsigned) * 4) != cudaSuccess) {
        h->err = "cudaMallocHost failed";
        return bail(VLBM_ERR_CUDA);
    }
    for (int q = 0; q < 4; ++q)
        if (cudaEventCreate(&h->ev[q]) != cudaSuccess) {
            h->err = "cudaEventCreate failed";
            return bail(VLBM_ERR_CUDA);
        }
    if (h->prec == VLBM_FP32) {
        if ((rc = encode_map(h, &h->tmF, h->F)) || (rc = encode_map(h, &h->tmA, h->A)) ||
            (rc = encode_map(h, &h->tmB, h->B)) || (rc = encode_map(h, &h->tmFc, h->F, 0, true)) ||
            (rc = encode_map(h, &h->tmAc, h->A, 0, true)) || (rc = encode_map(h, &h->tmBc, h->B, 0, true)))
            return bail(rc);
        // the stage kernel needs more than the default 48 KB of dynamic shared
        // memory; set that once here, outside any graph capture
        CK(h, prepare_stage_f32());
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        h->err = "device synchronize after create failed";
        return bail(VLBM_ERR_CUDA);
    }
    *out = h;
    return VLBM_OK;
}

int vlbm_init_moments(vlbm_t *h, const double *rho, const double *u_theta, const double *u_phi, const double *T)
{
    if (!h || !rho || !u_theta || !u_phi) return fail(h, VLBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->nt * h->np;
    double *d = h->d_mom;
    CK(h, cudaMemcpyAsync(d, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(d + n, u_theta, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(d + 2 * n, u_phi, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (T) CK(h, cudaMemcpyAsync(d + 3 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (h->prec == VLBM_FP64) {
        launch_init_f64((double *)h->F, h->L, d, d + n, d + 2 * n, T ? d + 3 * n : nullptr, h->vd, h->stream);
    } else {
        const double old = h->rho_ref;
        int rc = choose_rho_ref(h, d);
        if (rc) return rc;
        if (old != h->rho_ref || !h->d_row) {
            rc = build_f32_tables(h);
            if (rc) return rc;
            drop_graphs(h);
        }
        launch_init_f32((float2 *)h->F, h->L, d, d + n, d + 2 * n, T ? d + 3 * n : nullptr, h->vd, h->rho_ref,
                        h->d_kss, h->stream);
    }
    CK(h, cudaGetLastError());
    return after_reset(h);
}

int vlbm_set_populations(vlbm_t *h, const double *f)
{
    if (!h || !f) return fail(h, VLBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->L.nk * h->nt * h->np;
    if (!h->d_dense) {
        int rc = dalloc(h, (void **)&h->d_dense, n * sizeof(double));
        if (rc) return rc;
    }
    CK(h, cudaMemcpyAsync(h->d_dense, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (h->prec == VLBM_FP64) {
        launch_unpack_f64(h->d_dense, h->L, (double *)h->F, h->stream);
    } else {
        const size_t cells = (size_t)h->nt * h->np;
        launch_density_of_populations(h->d_dense, h->L.nk, cells, h->d_mom, h->stream);
        CK(h, cudaGetLastError());
        const double old = h->rho_ref;
        int rc = choose_rho_ref(h, h->d_mom);
        if (rc) return rc;
        if (old != h->rho_ref || !h->d_row) {
            rc = build_f32_tables(h);
            if (rc) return rc;
            drop_graphs(h);
        }
        launch_unpack_f32(h->d_dense, h->L, (float2 *)h->F, h->vd, h->rho_ref, h->d_sin_t, h->kscale, h->stream);
    }
    CK(h, cudaGetLastError());
    return after_reset(h);
}

int vlbm_get_populations(vlbm_t *h, double *f)
{
    if (!h || !f) return fail(h, VLBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->L.nk * h->nt * h->np;
    if (!h->d_dense) {
        int rc = dalloc(h, (void **)&h->d_dense, n * sizeof(double));
        if (rc) return rc;
    }
    if (h->prec == VLBM_FP64) launch_pack_f64((const double *)h->F, h->L, h->d_dense, h->stream);
    else launch_pack_f32((const float2 *)h->F, h->L, h->d_dense, h->vd, h->rho_ref, h->d_sin_t, h->kscale, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(f, h->d_dense, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return VLBM_OK;
}

int vlbm_step_async(vlbm_t *h, int n)
{
    if (!h || n < 0) return fail(h, VLBM_ERR_ARG, "bad handle or step count");
    if (h->prec == VLBM_FP32 && !h->d_row) return fail(h, VLBM_ERR_ARG, "FP32 state not initialised");
    if (n == 0) return VLBM_OK;
    int rc;
    if (!h->g1 && (rc = build_graph(h, 1, &h->g1))) return rc;
    if (n >= 16 && !h->g16 && (rc = build_graph(h, 16, &h->g16))) return rc;
    int left = n;
    while (left >= 16) {
        CK(h, cudaGraphLaunch(h->g16, h->stream));
        left -= 16;
    }
    while (left-- > 0) CK(h, cudaGraphLaunch(h->g1, h->stream));
    h->steps += n;
    return VLBM_OK;
}

int vlbm_sync(vlbm_t *h)
{
    if (!h) return fail(h, VLBM_ERR_ARG, "NULL handle");
    CK(h, cudaMemcpyAsync(h->h_flags, h->d_flags, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaGetLastError());
    if (h->h_flags[0] & 1u) return fail(h, VLBM_ERR_TIMEOUT, "a tile load did not complete within its time limit");
    if (h->h_flags[1]) return fail(h, VLBM_ERR_NONFINITE, "non-finite population found by the guard");
    return VLBM_OK;
}

int vlbm_step(vlbm_t *h, int n)
{
    int rc = vlbm_step_async(h, n);
    if (rc) return rc;
    if (h->guard && n > 0) {
        if (h->prec == VLBM_FP64) launch_guard_f64((const double *)h->F, h->L.nk * h->L.plane, h->d_flags + 1, h->stream);
        else launch_guard_f32((const float *)h->F, h->arr_bytes / sizeof(float), h->d_flags + 1, h->stream);
        CK(h, cudaGetLastError());
    }
    return vlbm_sync(h);
}

int vlbm_moments(vlbm_t *h, double *rho, double *u_theta, double *u_phi, double *T)
{
    if (!h || !rho || !u_theta || !u_phi) return fail(h, VLBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->nt * h->np;
    double *d = h->d_mom;
    if (h->prec == VLBM_FP64)
        launch_moments_f64((const double *)h->F, h->L, d, d + n, d + 2 * n, T ? d + 3 * n : nullptr, h->vd, h->stream);
    else
        launch_moments_f32((const float2 *)h->F, h->L, d, d + n, d + 2 * n, T ? d + 3 * n : nullptr, h->vd,
                           h->rho_ref, h->d_ikss, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(rho, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(u_theta, d + n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(u_phi, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (T) CK(h, cudaMemcpyAsync(T, d + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return VLBM_OK;
}

int vlbm_diagnostics(vlbm_t *h, vlbm_diag *out)
{
    if (!h || !out) return fail(h, VLBM_ERR_ARG, "NULL argument");
    const double area = h->R * h->R * (M_PI / h->nt) * (2.0 * M_PI / h->np);
    if (h->prec == VLBM_FP64)
        launch_diagnostics_f64((const double *)h->F, h->L, h->d_sin_t, h->d_cos_t, h->vd, area, h->d_part, h->d_diag,
                               h->stream);
    else
        launch_diagnostics_f32((const float2 *)h->F, h->L, h->d_sin_t, h->d_cos_t, h->d_cph, h->d_sph, h->vd, area,
                               h->rho_ref, h->kscale, h->d_part, h->d_diag, h->stream);
    CK(h, cudaGetLastError());
    double v[8];
    CK(h, cudaMemcpyAsync(v, h->d_diag, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(v + 6, h->d_budget, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    out->time = (double)h->steps * h->dt;
    out->steps = h->steps;
    out->mass = v[0];
    out->momentum[0] = v[1];
    out->momentum[1] = v[2];
    out->momentum[2] = v[3];
    out->energy = v[4];
    out->nonfinite = v[5] > 0.0 ? 1 : 0;
    out->pole_flux = v[6];
    out->mass0 = h->mass0;
    return VLBM_OK;
}

int vlbm_max_stable_dt(int n_theta, int n_phi, int velocity_set, double tau, int polar_filter, double *out)
{
    if (!out) return VLBM_ERR_ARG;
    if ((velocity_set != VLBM_D2Q9 && velocity_set != VLBM_D2Q16) || n_theta < 6 || n_phi < 1 || !(tau > 0.0))
        return VLBM_ERR_ARG;
    const double vmax = (velocity_set == VLBM_D2Q9) ? std::sqrt(3.0) : std::sqrt(3.0 + std::sqrt(6.0));
    const double dth = M_PI / n_theta, dph = 2.0 * M_PI / n_phi;
    double lim = polar_filter ? dth : std::fmin(dth, std::sin(dth / 2.0) * dph);
    if (n_phi == 1) lim = dth;
    double dt = 0.25 * lim / vmax;
    if (dt > tau) dt = tau;
    *out = dt;
    return VLBM_OK;
}

int vlbm_profile_step(vlbm_t *h, int n, double *ms_per_stage, int *launches)
{
    if (!h || n < 1) return fail(h, VLBM_ERR_ARG, "bad handle or step count");
    if (h->prec == VLBM_FP32 && !h->d_row) return fail(h, VLBM_ERR_ARG, "FP32 state not initialised");
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < n; ++q) {
        for (int st = 1; st <= 3; ++st) {
            CK(h, cudaEventRecord(h->ev[0], h->stream));
            enqueue_step(h, st, 1);
            CK(h, cudaEventRecord(h->ev[1], h->stream));
            enqueue_step(h, st, 2);
            CK(h, cudaEventRecord(h->ev[2], h->stream));
            CK(h, cudaEventSynchronize(h->ev[2]));
            float ms = 0.0f, mf = 0.0f;
            CK(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
            CK(h, cudaEventElapsedTime(&mf, h->ev[1], h->ev[2]));
            acc[st - 1] += ms;
            acc[st + 2] += h->nfrows ? mf : 0.0f;
        }
        // the step's pole budget, outside the timed launches
        if (h->prec == VLBM_FP64)
            launch_pole_budget(h->d_pole, h->np, h->R, 2.0 * M_PI / h->np, h->dt, h->d_budget, h->stream);
        else if (h->run.pole_part)
            launch_budget_f32(h, h->stream);
    }
    CK(h, cudaGetLastError());
    h->steps += n;
    for (int st = 0; st < 3; ++st) h->prof_ms[st] = acc[st] / n;
    if (ms_per_stage)
        for (int k = 0; k < 6; ++k) ms_per_stage[k] = acc[k] / n;
    if (launches) *launches = kernels_per_step(h);
    return vlbm_sync(h);
}

int vlbm_set_wait_limit(vlbm_t *h, double seconds)
{
    if (!h || !(seconds >= 0.0) || seconds > 10.0) return fail(h, VLBM_ERR_ARG, "wait limit must be in [0, 10] s");
    if (h->prec != VLBM_FP32) return fail(h, VLBM_ERR_UNSUPPORTED, "only the FP32 stage kernels wait on copies");
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    h->run.wait_ns = h->wait_ns;
    drop_graphs(h);   // the captured launches hold the old parameters
    return VLBM_OK;
}

size_t vlbm_device_bytes(const vlbm_t *h) { return h ? h->dev_bytes : 0; }

const char *vlbm_last_error(const vlbm_t *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void vlbm_destroy(vlbm_t *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    void *bufs[] = {h->F, h->A, h->B, h->d_sin_ext, h->d_cot, h->d_sin_t, h->d_cos_t, h->d_sin_f, h->d_cos_f, h->d_isp,
                    h->d_sfc, h->d_ft, h->d_fp,
                    h->d_rref, h->d_dsin, h->d_d2sin, h->d_tabs, h->d_kss, h->d_ikss, h->d_cph, h->d_sph,
                    h->d_pole_part, h->d_scalar, h->d_ctr,
                    h->d_row, h->d_frows, h->d_fblocks, h->d_pole, h->d_budget, h->d_mom, h->d_dense,
                    h->d_part, h->d_diag, h->d_flags};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    for (int q = 0; q < 4; ++q)
        if (h->ev[q]) cudaEventDestroy(h->ev[q]);
    for (cudaEvent_t e : h->evs)
        if (e) cudaEventDestroy(e);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"

struct vlbm_batch {
    std::vector<vlbm_t *> runs;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int ty = 8, ctas_per_sm = 0, nsm = 0;
    RunF *d_runs = nullptr;
    CUtensorMap *d_tms = nullptr;
    int2 *d_work = nullptr;
    int ntiles = 0;
    int4 *d_fitems = nullptr;   // polar filter: (run, row, block size, 0) of every filtered row
    int nfitems = 0;
    bool dirty = true;
    int guard = 1;
    int q = 4;   // members' velocity set order (4: D2Q16, 3: D2Q9)
    VelC vc{};
    VelC3 vc3{};
    unsigned *d_flags = nullptr, *h_flags = nullptr;
    cudaGraphExec_t g1 = nullptr, g16 = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::string err;
    long long steps = 0;
};

namespace {

// ---------------------------------------------------------------------------------
// Batched ensembles (FP32): many independent runs of uneven grid sizes advanced by
// one persistent kernel launch per RK3 stage, the n-step loop captured as a CUDA
// graph.  Each member is a full FP32 solver (its own arrays and tables); the batch
// adds the run table, the work list of (run, tile) items, the per-run tensor maps
// and the launch schedule (tile rows, CTAs per SM) chosen by vlbm_batch_tune.
// ---------------------------------------------------------------------------------
thread_local std::string g_batch_error;

int bfail(vlbm_batch_t *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return code;
}

#define BCK(b, call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return bfail((b), VLBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

void batch_drop_graphs(vlbm_batch_t *b)
{
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->g16) cudaGraphExecDestroy(b->g16);
    b->g1 = b->g16 = nullptr;
}

// Uploads the run table, tensor maps (for the current tile rows) and work list.
int batch_refresh(vlbm_batch_t *b)
{
    if (!b->dirty) return VLBM_OK;
    const int nr = (int)b->runs.size();
    std::vector<RunF> runs(nr);
    std::vector<CUtensorMap> tms(6 * (size_t)nr);
    std::vector<int2> work;
    for (int r = 0; r < nr; ++r) {
        vlbm_t *h = b->runs[r];
        if (!h->d_row) return bfail(b, VLBM_ERR_ARG, "run " + std::to_string(r) + " is not initialised");
        runs[r] = h->run;
        runs[r].pole_part = nullptr;   // batches report no pole budget
        int rc;
        CUtensorMap *t = &tms[6 * (size_t)r];
        if ((rc = encode_map(h, t + 0, h->F, b->ty)) || (rc = encode_map(h, t + 1, h->A, b->ty)) ||
            (rc = encode_map(h, t + 2, h->B, b->ty)) || (rc = encode_map(h, t + 3, h->F, b->ty, true)) ||
            (rc = encode_map(h, t + 4, h->A, b->ty, true)) || (rc = encode_map(h, t + 5, h->B, b->ty, true)))
            return bfail(b, rc, h->err);
        const int tx = runs[r].tiles_x, tyn = (h->nt + b->ty - 1) / b->ty;
        for (int t = 0; t < tx * tyn; ++t) work.push_back(make_int2(r, t));
        b->vc = h->vc;
        b->vc3 = h->vc3;
    }
    b->ntiles = (int)work.size();
    std::vector<int4> fitems;
    for (int r = 0; r < nr; ++r) {
        const vlbm_t *h = b->runs[r];
        if (!h->filter) continue;
        for (int i = 0; i < h->nt; ++i) {
            const int bs = filter_block(h->nt, h->np, h->sin_t[i]);
            if (bs > 1) fitems.push_back(make_int4(r, i, bs, 0));
        }
    }
    b->nfitems = (int)fitems.size();
    if (b->d_fitems) cudaFree(b->d_fitems);
    b->d_fitems = nullptr;
    if (b->nfitems) {
        BCK(b, cudaMalloc(&b->d_fitems, sizeof(int4) * fitems.size()));
        BCK(b, cudaMemcpy(b->d_fitems, fitems.data(), sizeof(int4) * fitems.size(), cudaMemcpyHostToDevice));
    }
    if (!b->d_runs) BCK(b, cudaMalloc(&b->d_runs, sizeof(RunF) * nr));
    if (!b->d_tms) BCK(b, cudaMalloc(&b->d_tms, sizeof(CUtensorMap) * 6 * nr));
    if (b->d_work) cudaFree(b->d_work);
    BCK(b, cudaMalloc(&b->d_work, sizeof(int2) * work.size()));
    BCK(b, cudaMemcpy(b->d_runs, runs.data(), sizeof(RunF) * nr, cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(b->d_tms, tms.data(), sizeof(CUtensorMap) * 6 * nr, cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(b->d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice));
    batch_drop_graphs(b);
    b->dirty = false;
    return VLBM_OK;
}

int batch_ctas(const vlbm_batch_t *b)
{
    if (b->ctas_per_sm < 0) return std::max(1, b->ntiles);   // one CTA per work item
    const int per = b->ctas_per_sm > 0 ? b->ctas_per_sm : stage_f32_max_ctas_per_sm(b->ty, b->q);
    return std::max(1, std::min(b->ntiles, per * b->nsm));
}

void batch_enqueue_step(vlbm_batch_t *b)
{
    const int ctas = batch_ctas(b);
    for (int st = 1; st <= 3; ++st) {
        const bool lin = b->runs.front()->scheme != VLBM_WENO5;
        if (b->q == 3)
            launch_batch_stage_f32_q3(b->d_runs, b->d_tms, b->d_work, b->ntiles, b->vc3, st, b->ty, lin, ctas,
                                      b->d_flags, b->stream);
        else
            launch_batch_stage_f32(b->d_runs, b->d_tms, b->d_work, b->ntiles, b->vc, st, b->ty, lin, ctas,
                                   b->d_flags, b->stream);
        // one polar-filter launch over the filtered rows of every run
        launch_batch_filter_f32(b->d_runs, b->d_fitems, b->nfitems, b->q, st, b->stream);
    }
}

int batch_build_graph(vlbm_batch_t *b, int nsteps, cudaGraphExec_t *exec)
{
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < nsteps; ++q) batch_enqueue_step(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return bfail(b, VLBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, VLBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return VLBM_OK;
}

std::string batch_signature(const vlbm_batch_t *b)
{
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::vector<std::pair<int, int>> g;
    for (const vlbm_t *h : b->runs) g.push_back({h->nt, h->np});
    std::sort(g.begin(), g.end());
    std::string key = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount) + "sm|" +
                      (b->q == 3 ? "d2q9|" : "");
    for (size_t i = 0; i < g.size();) {
        size_t j = i;
        while (j < g.size() && g[j] == g[i]) ++j;
        key += std::to_string(j - i) + "x" + std::to_string(g[i].first) + "x" + std::to_string(g[i].second) + ";";
        i = j;
    }
    return key;
}

// The tuning cache is a JSON object, one entry per line:
//   "signature": {"tile_rows": 8, "ctas_per_sm": 3, "ms_per_step": 1.25},
bool cache_lookup(const char *path, const std::string &key, int *ty, int *ctas, double *ms)
{
    if (!path) return false;
    FILE *fp = fopen(path, "r");
    if (!fp) return false;
    char line[4096];
    bool found = false;
    const std::string tag = "\"" + key + "\"";
    while (fgets(line, sizeof line, fp)) {
        std::string l(line);
        if (l.find(tag) == std::string::npos) continue;
        if (sscanf(l.c_str() + l.find("{"), "{\"tile_rows\": %d, \"ctas_per_sm\": %d, \"ms_per_step\": %lf", ty, ctas, ms) == 3)
            found = true;
    }
    fclose(fp);
    return found;
}

void cache_store(const char *path, const std::string &key, int ty, int ctas, double ms)
{
    if (!path) return;
    std::vector<std::string> keep;
    if (FILE *fp = fopen(path, "r")) {
        char line[4096];
        while (fgets(line, sizeof line, fp)) {
            std::string l(line);
            if (l.find("\": {") == std::string::npos || l.find("\"" + key + "\"") != std::string::npos) continue;
            while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
            keep.push_back(l);
        }
        fclose(fp);
    }
    char buf[512];
    snprintf(buf, sizeof buf, "  \"%s\": {\"tile_rows\": %d, \"ctas_per_sm\": %d, \"ms_per_step\": %.6f}", key.c_str(), ty,
             ctas, ms);
    keep.push_back(buf);
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = fopen(tmp.c_str(), "w");
    if (!fp) return;
    fprintf(fp, "{\n");
    for (size_t i = 0; i < keep.size(); ++i) fprintf(fp, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    fprintf(fp, "}\n");
    fclose(fp);
    rename(tmp.c_str(), path);
}

}  // namespace (reopened below for the C entry points)

extern "C" {

int vlbm_batch_create(int nruns, const int *n_theta, const int *n_phi, const double *tau, const double *dt,
                      const vlbm_options *opt, vlbm_batch_t **out)
{
    if (!out) return bfail(nullptr, VLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nruns < 1 || !n_theta || !n_phi || !tau || !dt) return bfail(nullptr, VLBM_ERR_ARG, "bad run arrays");
    vlbm_options o;
    vlbm_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != VLBM_FP32) return bfail(nullptr, VLBM_ERR_UNSUPPORTED, "batches run the FP32 path only");
    if (o.scheme == VLBM_WENO5 && o.komissarov)
        return bfail(nullptr, VLBM_ERR_UNSUPPORTED, "batches run the Komissarov flux with the upwind schemes only");
    if (o.velocity_set != 0 && o.velocity_set != VLBM_D2Q16 && o.velocity_set != VLBM_D2Q9)
        return bfail(nullptr, VLBM_ERR_ARG, "unknown velocity set");
    const int vset = (o.velocity_set == VLBM_D2Q9) ? VLBM_D2Q9 : VLBM_D2Q16;
    vlbm_batch_t *b = new vlbm_batch_t();
    b->guard = o.guard ? 1 : 0;
    b->q = (vset == VLBM_D2Q9) ? 3 : 4;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete b;
        return bfail(nullptr, VLBM_ERR_CUDA, "no CUDA device");
    }
    if (o.stream) {
        b->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(nullptr, VLBM_ERR_CUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    o.stream = b->stream;
    o.guard = 0;
    o.tile_rows = 8;
    for (int r = 0; r < nruns; ++r) {
        vlbm_t *h = nullptr;
        int rc = vlbm_create(n_theta[r], n_phi[r], vset, tau[r], dt[r], &o, &h);
        if (rc) {
            std::string m = "run " + std::to_string(r) + ": " + vlbm_last_error(nullptr);
            vlbm_batch_destroy(b);
            return bfail(nullptr, rc, m);
        }
        // a member's steps are the batch's launches: it needs no stream of its own for the
        // split filter schedule
        for (cudaEvent_t &e : h->evs)
            if (e) {
                cudaEventDestroy(e);
                e = nullptr;
            }
        if (h->stream2) cudaStreamDestroy(h->stream2);
        h->stream2 = nullptr;
        h->band_lo = h->band_hi = 0;
        b->runs.push_back(h);
    }
    if (cudaMalloc(&b->d_flags, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b->d_flags, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&b->h_flags, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
        vlbm_batch_destroy(b);
        return bfail(nullptr, VLBM_ERR_CUDA, "batch allocation failed");
    }
    *out = b;
    return VLBM_OK;
}

int vlbm_batch_init_moments(vlbm_batch_t *b, int run, const double *rho, const double *u_theta, const double *u_phi,
                            const double *T)
{
    if (!b || run < 0 || run >= (int)b->runs.size()) return bfail(b, VLBM_ERR_ARG, "bad batch or run index");
    int rc = vlbm_init_moments(b->runs[run], rho, u_theta, u_phi, T);
    if (rc) return bfail(b, rc, b->runs[run]->err);
    b->dirty = true;
    b->steps = 0;
    return VLBM_OK;
}

int vlbm_batch_get_populations(vlbm_batch_t *b, int run, double *f)
{
    if (!b || run < 0 || run >= (int)b->runs.size()) return bfail(b, VLBM_ERR_ARG, "bad batch or run index");
    BCK(b, cudaStreamSynchronize(b->stream));
    int rc = vlbm_get_populations(b->runs[run], f);
    if (rc) return bfail(b, rc, b->runs[run]->err);
    return VLBM_OK;
}

int vlbm_batch_set_schedule(vlbm_batch_t *b, int tile_rows, int ctas_per_sm)
{
    if (!b || (tile_rows != 4 && tile_rows != 8) || ctas_per_sm < -1) return bfail(b, VLBM_ERR_ARG, "bad schedule");
    if (ctas_per_sm > stage_f32_max_ctas_per_sm(tile_rows, b->q))
        return bfail(b, VLBM_ERR_ARG, "ctas_per_sm above occupancy");
    if (tile_rows != b->ty) b->dirty = true;
    b->ty = tile_rows;
    b->ctas_per_sm = ctas_per_sm;
    batch_drop_graphs(b);
    return VLBM_OK;
}

int vlbm_batch_step_async(vlbm_batch_t *b, int n)
{
    if (!b || n < 0) return bfail(b, VLBM_ERR_ARG, "bad batch or step count");
    if (n == 0) return VLBM_OK;
    int rc;
    if ((rc = batch_refresh(b))) return rc;
    if (!b->g1 && (rc = batch_build_graph(b, 1, &b->g1))) return rc;
    if (n >= 16 && !b->g16 && (rc = batch_build_graph(b, 16, &b->g16))) return rc;
    int left = n;
    while (left >= 16) {
        BCK(b, cudaGraphLaunch(b->g16, b->stream));
        left -= 16;
    }
    while (left-- > 0) BCK(b, cudaGraphLaunch(b->g1, b->stream));
    b->steps += n;
    for (vlbm_t *h : b->runs) h->steps += n;
    return VLBM_OK;
}

int vlbm_batch_sync(vlbm_batch_t *b)
{
    if (!b) return bfail(b, VLBM_ERR_ARG, "NULL batch");
    BCK(b, cudaMemcpyAsync(b->h_flags, b->d_flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    BCK(b, cudaGetLastError());
    if (b->h_flags[0] & 1u) return bfail(b, VLBM_ERR_TIMEOUT, "a tile load did not complete within its time limit");
    if (b->h_flags[1]) return bfail(b, VLBM_ERR_NONFINITE, "non-finite population found by the guard");
    return VLBM_OK;
}

int vlbm_batch_step(vlbm_batch_t *b, int n)
{
    int rc = vlbm_batch_step_async(b, n);
    if (rc) return rc;
    if (b->guard && n > 0) {
        for (vlbm_t *h : b->runs) launch_guard_f32((const float *)h->F, h->arr_bytes / sizeof(float), b->d_flags + 1, b->stream);
        BCK(b, cudaGetLastError());
    }
    return vlbm_batch_sync(b);
}

int vlbm_batch_moments(vlbm_batch_t *b, int run, double *rho, double *u_theta, double *u_phi, double *T)
{
    if (!b || run < 0 || run >= (int)b->runs.size()) return bfail(b, VLBM_ERR_ARG, "bad batch or run index");
    BCK(b, cudaStreamSynchronize(b->stream));
    int rc = vlbm_moments(b->runs[run], rho, u_theta, u_phi, T);
    if (rc) return bfail(b, rc, b->runs[run]->err);
    return VLBM_OK;
}

int vlbm_batch_profile(vlbm_batch_t *b, int n, double *ms_per_step, int *launches_per_step)
{
    if (!b || n < 1) return bfail(b, VLBM_ERR_ARG, "bad batch or step count");
    int rc = vlbm_batch_step_async(b, 1);   // builds the graph outside the timed region
    if (rc) return rc;
    BCK(b, cudaEventRecord(b->ev[0], b->stream));
    if ((rc = vlbm_batch_step_async(b, n))) return rc;
    BCK(b, cudaEventRecord(b->ev[1], b->stream));
    BCK(b, cudaEventSynchronize(b->ev[1]));
    float ms = 0.0f;
    BCK(b, cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    if (ms_per_step) *ms_per_step = ms / n;
    if (launches_per_step) {
        *launches_per_step = 3 + (b->nfitems ? 3 : 0);
    }
    return vlbm_batch_sync(b);
}

int vlbm_batch_tune(vlbm_batch_t *b, const char *cache_path, int *tile_rows, int *ctas_per_sm, double *ms_per_step)
{
    if (!b) return bfail(b, VLBM_ERR_ARG, "NULL batch");
    int rc;
    if ((rc = batch_refresh(b))) return rc;
    const std::string key = batch_signature(b);
    int best_ty = 8, best_c = 0;
    double best = 0.0;
    if (!cache_lookup(cache_path, key, &best_ty, &best_c, &best)) {
        // measure every schedule on a copy of the state, then put the state back
        std::vector<void *> backup;
        for (vlbm_t *h : b->runs) {
            void *p = nullptr;
            BCK(b, cudaMalloc(&p, h->arr_bytes));
            BCK(b, cudaMemcpyAsync(p, h->F, h->arr_bytes, cudaMemcpyDeviceToDevice, b->stream));
            backup.push_back(p);
        }
        best = 1e300;
        for (int ty : {4, 8}) {
            const int maxc = stage_f32_max_ctas_per_sm(ty, b->q);
            for (int c = -1; c <= maxc; ++c) {
                if (c == 0) continue;   // (0 is the occupancy limit, already among 1..maxc)
                if ((rc = vlbm_batch_set_schedule(b, ty, c))) return rc;
                double ms = 0.0;
                if ((rc = vlbm_batch_profile(b, 2, &ms, nullptr))) return rc;
                if (ms < best) {
                    best = ms;
                    best_ty = ty;
                    best_c = c;
                }
            }
        }
        for (size_t r = 0; r < b->runs.size(); ++r) {
            vlbm_t *h = b->runs[r];
            BCK(b, cudaMemcpyAsync(h->F, backup[r], h->arr_bytes, cudaMemcpyDeviceToDevice, b->stream));
            h->steps = 0;
        }
        BCK(b, cudaStreamSynchronize(b->stream));
        for (void *p : backup) cudaFree(p);
        b->steps = 0;
        cache_store(cache_path, key, best_ty, best_c, best);
    }
    if ((rc = vlbm_batch_set_schedule(b, best_ty, best_c))) return rc;
    if (tile_rows) *tile_rows = best_ty;
    if (ctas_per_sm) *ctas_per_sm = best_c;
    if (ms_per_step) *ms_per_step = best;
    return VLBM_OK;
}

size_t vlbm_batch_cells(const vlbm_batch_t *b)
{
    size_t n = 0;
    if (b)
        for (const vlbm_t *h : b->runs) n += (size_t)h->nt * h->np;
    return n;
}

const char *vlbm_batch_last_error(const vlbm_batch_t *b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

void vlbm_batch_destroy(vlbm_batch_t *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (vlbm_t *h : b->runs) vlbm_destroy(h);
    if (b->d_runs) cudaFree(b->d_runs);
    if (b->d_tms) cudaFree(b->d_tms);
    if (b->d_work) cudaFree(b->d_work);
    if (b->d_fitems) cudaFree(b->d_fitems);
    if (b->d_flags) cudaFree(b->d_flags);
    if (b->h_flags) cudaFreeHost(b->h_flags);
    for (int q = 0; q < 2; ++q)
        if (b->ev[q]) cudaEventDestroy(b->ev[q]);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
