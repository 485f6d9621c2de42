// stage_f64.cu -- FP64 kernels of the parity path (compiled with -fmad=false).
//
// One RK3 stage of arXiv 2504.15574 Sec. 3.7 fused into one kernel: moments
// (Eq. f_moments_sum), equilibrium (Eq. feq_Q=4), BGK (Sec. 3.2), geometric
// force through K^H and Ktilde^H (Eq. df), WENO-5 fluxes in theta and phi
// (Eqs. fluxes_W5, WENO5_delta, WENO5_sigma) in the flux form of
// Eq. (discrete_advection_sphere), and the Shu-Osher stage combination.
//
// This path exists to reproduce an FP64 reference evaluation of the method
// operation for operation: every expression below is evaluated in a fixed
// order with no FMA contraction, divisions where the method divides, and sums
// over populations in ascending k.  Each interface flux is computed once (two
// face kernels into global buffers), then one kernel updates the cells.  It is not the throughput path (that is
// stage_f32.cu); it shares the ghost-row layout so that all reads are plain
// loads.
#include "vlbm_internal.h"

namespace vk {

namespace {

__device__ __forceinline__ double weno5(double a, double b, double c, double d, double e, double eps)
{
    double p1 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    double p2 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    double p3 = (2.0 * c + 5.0 * d - e) / 6.0;
    double d1a = a - 2.0 * b + c, d1b = a - 4.0 * b + 3.0 * c;
    double d2a = b - 2.0 * c + d, d2b = b - d;
    double d3a = c - 2.0 * d + e, d3b = 3.0 * c - 4.0 * d + e;
    double s1 = 13.0 / 12.0 * (d1a * d1a) + 0.25 * (d1b * d1b);
    double s2 = 13.0 / 12.0 * (d2a * d2a) + 0.25 * (d2b * d2b);
    double s3 = 13.0 / 12.0 * (d3a * d3a) + 0.25 * (d3b * d3b);
    double w1 = 0.1 / ((s1 + eps) * (s1 + eps));
    double w2 = 0.6 / ((s2 + eps) * (s2 + eps));
    double w3 = 0.3 / ((s3 + eps) * (s3 + eps));
    return (w1 * p1 + w2 * p2 + w3 * p3) / (w1 + w2 + w3);
}

// Interface value from upwind-ordered a..e (c the upwind cell, d the downwind cell):
// WENO-5, or the upwind stencils of Eq. (fluxes_U1-3), in the oracle's expression order.
__device__ __forceinline__ double recon(int scheme, double a, double b, double c, double d, double e, double eps)
{
    switch (scheme) {
    case VLBM_U1: return c;
    case VLBM_U2: return 1.5 * c - 0.5 * b;
    case VLBM_U3: return (2.0 * d + 5.0 * c - b) / 6.0;
    default: return weno5(a, b, c, d, e, eps);
    }
}

// Writes v at interior (k, i, j) and at every ghost image of that cell.
template <typename T>
__device__ __forceinline__ void store_with_images(T *f, const Layout &L, int k, int i, int j, T v)
{
    const int np = L.np;
    auto put_row = [&](int kk, int r, int c) {
        f[L.at(kk, r, c)] = v;
        // periodic images of column c inside [-GC, np+GC)
        for (int m = 1; c - m * np >= -GC; ++m) f[L.at(kk, r, c - m * np)] = v;
        for (int m = 1; c + m * np < np + GC; ++m) f[L.at(kk, r, c + m * np)] = v;
    };
    put_row(k, i, j);
    if (i < GR || i >= L.nt - GR) {
        int jj = j + np / 2;
        if (jj >= np) jj -= np;
        int r = (i < GR) ? (-1 - i) : (2 * L.nt - 1 - i);
        put_row(L.nk - 1 - k, r, jj);
    }
}

// Theta flux through interface fi (between rows fi-1 and fi, fi = 0..nt) of population k:
// the reconstruction on the nodal g = sin f of rows fi-3..fi+2 (ghost rows with their own,
// negative, sine), or (Komissarov) on f itself times v_theta sin(theta_fi).
__global__ void __launch_bounds__(128) faces_theta_f64_kernel(const StageD p)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int fi = blockIdx.y;
    const int k = blockIdx.z;
    if (j >= p.L.np) return;
    const Layout L = p.L;
    const double *g = p.in;
    const double va = p.c.v[k / p.c.q];
    double gt[6];
#pragma unroll
    for (int o = 0; o < 6; ++o)
        gt[o] = p.komissarov ? g[L.at(k, fi - 3 + o, j)] : p.sin_ext[fi + o] * g[L.at(k, fi - 3 + o, j)];
    const double r = (va > 0.0) ? recon(p.scheme, gt[0], gt[1], gt[2], gt[3], gt[4], p.eps)
                                : recon(p.scheme, gt[5], gt[4], gt[3], gt[2], gt[1], p.eps);
    const double flux = p.komissarov ? va * p.sin_f[fi] * r : va * r;
    p.Ft[((size_t)k * (L.nt + 1) + fi) * L.np + j] = flux;
    if (p.pole) {
        if (fi == 0) p.pole[(size_t)k * L.np + j] = flux;
        if (fi == L.nt) p.pole[((size_t)NK + k) * L.np + j] = flux;
    }
}

// Phi flux through interface fj (between columns fj-1 and fj, fj = 0..np) of row i.
__global__ void __launch_bounds__(128) faces_phi_f64_kernel(const StageD p)
{
    const int fj = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    const int k = blockIdx.z;
    if (fj > p.L.np) return;
    const Layout L = p.L;
    const double *g = p.in;
    const double vb = p.c.v[k % p.c.q];
    double gp[6];
#pragma unroll
    for (int o = 0; o < 6; ++o) gp[o] = g[L.at(k, i, fj - 3 + o)];
    const double r = (vb > 0.0) ? recon(p.scheme, gp[0], gp[1], gp[2], gp[3], gp[4], p.eps)
                                : recon(p.scheme, gp[5], gp[4], gp[3], gp[2], gp[1], p.eps);
    p.Fp[((size_t)k * L.nt + i) * (L.np + 1) + fj] = vb * r;
}

// One cell: moments, equilibrium, force, BGK, the flux differences of the interface
// fluxes above and the stage combination, in the oracle's operation order.
__global__ void __launch_bounds__(128) stage_f64_kernel(const StageD p)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= p.L.nt || j >= p.L.np) return;
    const Layout L = p.L;
    const double *g = p.in;

    const int q = p.c.q, nk = q * q;
    double gk[NK];
    for (int k = 0; k < nk; ++k) gk[k] = g[L.at(k, i, j)];

    double n = 0.0, jt = 0.0, jp = 0.0;
    for (int k = 0; k < nk; ++k) {
        n += gk[k];
        jt += gk[k] * p.c.v[k / q];
        jp += gk[k] * p.c.v[k % q];
    }
    const double ut = jt / n, up = jp / n;
    const double sin_i = p.sin_ext[i + GR];
    const double cot_i = p.cot[i];
    const double R = p.R;

#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int a = k / q, b = k % q;
        const double va = p.c.v[a], vb = p.c.v[b];
        // equilibrium (T0 = 1)
        const double xi = va * ut + vb * up;
        const double u2 = ut * ut + up * up;
        const double wk = p.c.w[a] * p.c.w[b];
        // Eq. feq_Q=4 (third order), or Eq. feq_Q=3 (second order) for D2Q9
        const double feq = (q == 3) ? n * wk * (1.0 + xi + 0.5 * (xi * xi - u2))
                                    : n * wk * (1.0 + xi + 0.5 * (xi * xi - u2) + xi * (xi * xi - 3.0 * u2) / 6.0);
        // velocity derivatives: K on k_theta at fixed k_phi, Ktilde on k_phi at fixed k_theta
        double kg = 0.0, ktg = 0.0;
        for (int m = 0; m < q; ++m) {
            kg += p.c.K[a * q + m] * gk[q * m + b];
            ktg += p.c.Kt[b * q + m] * gk[q * a + m];
        }
        const double force = cot_i / R * (vb * vb * kg - va * ktg);
        const double fn = p.Ft[((size_t)k * (L.nt + 1) + i) * L.np + j];
        const double fs = p.Ft[((size_t)k * (L.nt + 1) + i + 1) * L.np + j];
        const double fw = p.Fp[((size_t)k * L.nt + i) * (L.np + 1) + j];
        const double fe = p.Fp[((size_t)k * L.nt + i) * (L.np + 1) + j + 1];
        const double adv_t = p.komissarov ? -(fs - fn) / (R * (p.cos_f[i] - p.cos_f[i + 1]))
                                          : -(fs - fn) / (R * sin_i * p.dth);
        const double adv_p = -(fe - fw) / (R * sin_i * p.dph);
        const double Lk = adv_t + adv_p - force - (gk[k] - feq) / p.tau;

        double outv;
        if (p.stage == 1) {
            outv = gk[k] + p.dt * Lk;
        } else if (p.stage == 2) {
            const double f0 = p.fold[L.at(k, i, j)];
            outv = 0.75 * f0 + 0.25 * gk[k] + 0.25 * p.dt * Lk;
        } else {
            const double f0 = p.fold[L.at(k, i, j)];
            outv = f0 / 3.0 + 2.0 / 3.0 * gk[k] + 2.0 / 3.0 * p.dt * Lk;
        }
        store_with_images(p.out, L, k, i, j, outv);
    }
}

// Initial populations: third-order Hermite projection of a Maxwellian at T
// (T = 1: the BGK equilibrium, Eq. feq_Q=4).
// (q = 3: the same projection to second order, Eq. feq_Q=3 at T = 1.)
__device__ __forceinline__ double finit(int q, double n, double wk, double va, double vb, double ut, double up,
                                        double T)
{
    const double xi = va * ut + vb * up;
    const double u2 = ut * ut + up * up;
    if (T == 1.0) {
        if (q == 3) return n * wk * (1.0 + xi + 0.5 * (xi * xi - u2));
        return n * wk * (1.0 + xi + 0.5 * (xi * xi - u2) + xi * (xi * xi - 3.0 * u2) / 6.0);
    }
    const double v2 = va * va + vb * vb;
    const double dT = T - 1.0;
    const double second = xi * xi - u2 + dT * (v2 - 2.0);
    if (q == 3) return n * wk * (1.0 + xi + 0.5 * second);
    const double third = xi * (xi * xi - 3.0 * u2) + 3.0 * dT * xi * (v2 - 4.0);
    return n * wk * (1.0 + xi + 0.5 * second + third / 6.0);
}

template <typename T>
__global__ void init_kernel(T *f, const Layout L, const double *rho, const double *ut, const double *up,
                            const double *temp, const VelD c, double rho_ref)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const size_t cell = (size_t)i * L.np + j;
    const double tt = temp ? temp[cell] : 1.0;
    const int q = c.q;
    for (int k = 0; k < q * q; ++k) {
        const int a = k / q, b = k % q;
        double v = finit(q, rho[cell], c.w[a] * c.w[b], c.v[a], c.v[b], ut[cell], up[cell], tt);
        if (rho_ref != 0.0) v -= c.w[a] * c.w[b] * rho_ref;
        f[L.at(k, i, j)] = (T)v;
    }
}

template <typename T>
__global__ void moments_kernel(const T *f, const Layout L, double *rho, double *ut, double *up, double *temp,
                               const VelD c, double rho_ref)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const int q = c.q, nk = q * q;
    double fk[NK];
    for (int k = 0; k < nk; ++k) {
        double v = (double)f[L.at(k, i, j)];
        if (rho_ref != 0.0) v = c.w[k / q] * c.w[k % q] * rho_ref + v;
        fk[k] = v;
    }
    double n = 0.0, jt = 0.0, jp = 0.0;
    for (int k = 0; k < nk; ++k) {
        n += fk[k];
        jt += fk[k] * c.v[k / q];
        jp += fk[k] * c.v[k % q];
    }
    const size_t cell = (size_t)i * L.np + j;
    const double u1 = jt / n, u2 = jp / n;
    rho[cell] = n;
    ut[cell] = u1;
    up[cell] = u2;
    if (temp) {
        double e = 0.0;
        for (int k = 0; k < nk; ++k) {
            const double ct = c.v[k / q] - u1, cp = c.v[k % q] - u2;
            e += fk[k] * (ct * ct + cp * cp);
        }
        temp[cell] = e / (2.0 * n);
    }
}

// Polar ring filter: mean over aligned blocks of b columns, summed in column order.
template <typename T>
__global__ void filter_kernel(T *f, const Layout L, const int *rows, const int *blocks, int nrows)
{
    const int rr = blockIdx.y;
    const int k = blockIdx.z;
    if (rr >= nrows) return;
    const int i = rows[rr];
    const int b = blocks[rr];
    const int nblk = L.np / b;
    for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk < nblk; blk += gridDim.x * blockDim.x) {
        const int j0 = blk * b;
        double s = 0.0;
        for (int m = 0; m < b; ++m) s += (double)f[L.at(k, i, j0 + m)];
        const T mean = (T)(s / (double)b);
        for (int m = 0; m < b; ++m) store_with_images(f, L, k, i, j0 + m, mean);
    }
}

}  // namespace

void launch_stage_f64(const StageD &p, cudaStream_t s)
{
    // every interface flux once (as the oracle), then the cells
    faces_theta_f64_kernel<<<dim3((p.L.np + 127) / 128, p.L.nt + 1, p.L.nk), 128, 0, s>>>(p);
    faces_phi_f64_kernel<<<dim3((p.L.np + 1 + 127) / 128, p.L.nt, p.L.nk), 128, 0, s>>>(p);
    dim3 block(32, 4);
    dim3 grid((p.L.np + 31) / 32, (p.L.nt + 3) / 4);
    stage_f64_kernel<<<grid, block, 0, s>>>(p);
}

void launch_init_f64(double *f, const Layout &L, const double *rho, const double *ut, const double *up,
                     const double *T, const VelD &c, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt);
    init_kernel<double><<<grid, 128, 0, s>>>(f, L, rho, ut, up, T, c, 0.0);
}

void launch_moments_f64(const double *f, const Layout &L, double *rho, double *ut, double *up, double *T,
                        const VelD &c, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt);
    moments_kernel<double><<<grid, 128, 0, s>>>(f, L, rho, ut, up, T, c, 0.0);
}

void launch_filter_f64(double *f, const Layout &L, const int *rows, const int *blocks, int nrows, cudaStream_t s)
{
    if (nrows <= 0) return;
    dim3 grid((L.np / 2 + 127) / 128 + 1, nrows, L.nk);
    filter_kernel<double><<<grid, 128, 0, s>>>(f, L, rows, blocks, nrows);
}

}  // namespace vk
