// aux.cu -- layout maintenance, diagnostics and guards (FP64 arithmetic).
//
// Ghost fill implements the boundary conditions of arXiv 2504.15574 Sec. 3.6
// (Eqs. bcs_phi, bcs_theta) on the storage layout of vlbm_internal.h.  The
// diagnostics (mass, momentum, energy, non-finite count) and the pole-flux
// budget are not in the paper; they are FP64 reductions in a fixed order
// (block partials, then one block sums the partials), so they are
// deterministic for a given grid.
#include "vlbm_internal.h"

namespace vk {

namespace {

// Source cell of a padded position (k, r, c): the interior cell whose value it holds.
__device__ __forceinline__ void ghost_source(const Layout &L, int k, int r, int c, int &ks, int &rs, int &cs)
{
    int shift = 0;
    ks = k;
    rs = r;
    if (r < 0) {
        rs = -1 - r;
        ks = L.nk - 1 - k;
        shift = L.np / 2;
    } else if (r >= L.nt) {
        rs = 2 * L.nt - 1 - r;
        ks = L.nk - 1 - k;
        shift = L.np / 2;
    }
    int cc = (c + shift) % L.np;
    if (cc < 0) cc += L.np;
    cs = cc;
}

__global__ void fill_ghosts_kernel(double *f, const Layout L)
{
    const int c = (int)(blockIdx.x * blockDim.x + threadIdx.x) - GC;
    const int r = (int)blockIdx.y - GR;
    const int k = blockIdx.z;
    if (c >= L.np + GC) return;
    const bool interior = (r >= 0 && r < L.nt && c >= 0 && c < L.np);
    if (interior) return;
    int ks, rs, cs;
    ghost_source(L, k, r, c, ks, rs, cs);
    f[L.at(k, r, c)] = f[L.at(ks, rs, cs)];
}

__global__ void pack_f64_kernel(const double *f, const Layout L, double *dense)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y, k = blockIdx.z;
    if (j >= L.np) return;
    dense[((size_t)k * L.nt + i) * L.np + j] = f[L.at(k, i, j)];
}

__global__ void unpack_f64_kernel(const double *dense, const Layout L, double *f)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y, k = blockIdx.z;
    if (j >= L.np) return;
    f[L.at(k, i, j)] = dense[((size_t)k * L.nt + i) * L.np + j];
}

constexpr int DIAG_THREADS = 256;
constexpr int NDIAG = 6;

// One block per row: partial sums of the row in a fixed order.
__global__ void diag_rows_kernel(const double *f, const Layout L, const double *sin_t, const double *cos_t, const VelD c,
                                 double area, double *part)
{
    const int i = blockIdx.x;
    const double st = sin_t[i], ct = cos_t[i];
    const double dph = 6.283185307179586476925286766559 / L.np;
    double acc[NDIAG] = {0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < L.np; j += DIAG_THREADS) {
        const double ph = (j + 0.5) * dph;
        double sp, cp;
        sincos(ph, &sp, &cp);
        double n = 0.0, jt = 0.0, jp = 0.0, e = 0.0, bad = 0.0;
        for (int k = 0; k < c.q * c.q; ++k) {
            const double va = c.v[k / c.q], vb = c.v[k % c.q];
            const double fk = f[L.at(k, i, j)];
            if (!isfinite(fk)) bad = 1.0;
            n += fk;
            jt += fk * va;
            jp += fk * vb;
            e += fk * (va * va + vb * vb);
        }
        const double dA = st * area;
        acc[0] += n * dA;
        acc[1] += (jt * ct * cp - jp * sp) * dA;
        acc[2] += (jt * ct * sp + jp * cp) * dA;
        acc[3] += (-jt * st) * dA;
        acc[4] += 0.5 * e * dA;
        acc[5] += bad;
    }
    __shared__ double red[NDIAG][DIAG_THREADS];
    for (int q = 0; q < NDIAG; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < NDIAG; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NDIAG; ++q) part[(size_t)q * L.nt + i] = red[q][0];
}

__global__ void diag_final_kernel(const double *part, int nrows, double *out)
{
    __shared__ double red[NDIAG][DIAG_THREADS];
    double acc[NDIAG] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nrows; i += DIAG_THREADS)
        for (int q = 0; q < NDIAG; ++q) acc[q] += part[(size_t)q * nrows + i];
    for (int q = 0; q < NDIAG; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < NDIAG; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NDIAG; ++q) out[q] = red[q][0];
}

template <typename T>
__global__ void guard_kernel(const T *f, size_t total, unsigned *flag)
{
    bool bad = false;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const T v = f[x];
        // padding columns are zero-initialised and never written, so the whole
        // allocation can be scanned
        if (!isfinite((double)v)) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

// budget += dt * (m1/6 + m2/6 + 2 m3/3), m_s = -R dph sum_{k,j} (F_south - F_north)
__global__ void pole_budget_kernel(const double *pole3, int np, double R, double dph, double dt, double *budget)
{
    __shared__ double red[3][DIAG_THREADS];
    const size_t per = (size_t)NK * np;
    double acc[3] = {0, 0, 0};
    for (int s = 0; s < 3; ++s) {
        const double *pn = pole3 + (size_t)s * 2 * per;
        const double *ps = pn + per;
        for (size_t x = threadIdx.x; x < per; x += DIAG_THREADS) acc[s] += ps[x] - pn[x];
    }
    for (int s = 0; s < 3; ++s) red[s][threadIdx.x] = acc[s];
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int s = 0; s < 3; ++s) red[s][threadIdx.x] += red[s][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m1 = -R * dph * red[0][0], m2 = -R * dph * red[1][0], m3 = -R * dph * red[2][0];
        *budget += dt * (m1 / 6.0 + m2 / 6.0 + 2.0 * m3 / 3.0);
    }
}

}  // namespace

void launch_fill_ghosts_f64(double *f, const Layout &L, cudaStream_t s)
{
    dim3 grid((L.np + 2 * GC + 127) / 128, L.nt + 2 * GR, L.nk);
    fill_ghosts_kernel<<<grid, 128, 0, s>>>(f, L);
}

void launch_pack_f64(const double *f, const Layout &L, double *dense, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt, L.nk);
    pack_f64_kernel<<<grid, 128, 0, s>>>(f, L, dense);
}

void launch_unpack_f64(const double *dense, const Layout &L, double *f, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt, L.nk);
    unpack_f64_kernel<<<grid, 128, 0, s>>>(dense, L, f);
}

size_t diag_partials(const Layout &L) { return (size_t)NDIAG * L.nt; }

void launch_diagnostics_f64(const double *f, const Layout &L, const double *sin_t, const double *cos_t,
                            const VelD &c, double area, double *part, double *out, cudaStream_t s)
{
    diag_rows_kernel<<<L.nt, DIAG_THREADS, 0, s>>>(f, L, sin_t, cos_t, c, area, part);
    diag_final_kernel<<<1, DIAG_THREADS, 0, s>>>(part, L.nt, out);
}

void launch_diag_final(const double *part, int nrows, double *out, cudaStream_t s)
{
    diag_final_kernel<<<1, DIAG_THREADS, 0, s>>>(part, nrows, out);
}

void launch_guard_f64(const double *f, size_t n, unsigned *flag, cudaStream_t s)
{
    guard_kernel<double><<<152 * 8, 256, 0, s>>>(f, n, flag);
}

void launch_guard_f32(const float *f, size_t n, unsigned *flag, cudaStream_t s)
{
    guard_kernel<float><<<152 * 8, 256, 0, s>>>(f, n, flag);
}

void launch_pole_budget(const double *pole3, int np, double R, double dph, double dt, double *budget,
                        cudaStream_t s)
{
    pole_budget_kernel<<<1, DIAG_THREADS, 0, s>>>(pole3, np, R, dph, dt, budget);
}

}  // namespace vk
