// noalloc.cu -- diagnostics of a caller-owned population array without any
// device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need these
// numbers: hosts whose device memory is handed out by their own pool or held to a
// fixed budget, which a library must not grow or fragment behind their back, and
// latency-bound loops where the implicit device synchronisation an allocation can
// cause is not acceptable.  For them, vlbm_diagnostics_noalloc reduces a
// population array the caller already owns, using a fixed scratch array compiled
// into the library instead of memory from cudaMalloc.
//
// The scratch is a file-scope __device__ array of VLBM_NOALLOC_MAX_ROWS x 6
// doubles (768 KiB); every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address, so
// the first call on each device looks its address up with cudaGetSymbolAddress
// (with that device current) and caches it; that first call should therefore
// come before any stream capture, and the cached address does not survive a
// cudaDeviceReset of that device.  All calls share the one array: calls whose
// kernels overlap on the GPU (on different streams) race on it.  The per-row
// partial sums are fully rewritten by every call, so nothing in the scratch has
// to start at zero.
#include <mutex>
#include <string>

#include "../../include/vlbm.h"
#include "vlbm_internal.h"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NQ = 6;   // mass, momentum x/y/z, energy, non-finite count
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[(size_t)VLBM_NOALLOC_MAX_ROWS * NQ];

std::mutex g_mu;
double *g_scratch_ptr[MAX_DEVICES] = {};
thread_local std::string g_noalloc_error;

struct VelNA { double v[4], w[4]; };

// One block per row of a dense [16][nt][np] FP64 population array.
__global__ void noalloc_rows_kernel(const double *f, int nt, int np, double radius, VelNA c, double *part)
{
    const int i = blockIdx.x;
    const double pi = 3.14159265358979323846;
    const double dth = pi / nt, dph = 2.0 * pi / np;
    const int m = nt - 1 - i;
    const double st = sin(((i <= m ? i : m) + 0.5) * dth);
    const double ct = (i == m) ? 0.0 : (i < m ? 1.0 : -1.0) * cos(((i <= m ? i : m) + 0.5) * dth);
    const double area = radius * radius * dth * dph;
    double acc[NQ] = {0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < np; j += NOALLOC_THREADS) {
        double sp, cp;
        sincos((j + 0.5) * dph, &sp, &cp);
        double n = 0.0, jt = 0.0, jp = 0.0, e = 0.0, bad = 0.0;
        for (int k = 0; k < 16; ++k) {
            const double va = c.v[k / 4], vb = c.v[k % 4];
            const double fk = f[((size_t)k * nt + i) * np + j];
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
        acc[5] += bad;   // one per cell holding a NaN or Inf population
    }
    __shared__ double red[NQ][NOALLOC_THREADS];
    for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = NOALLOC_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NQ; ++q) part[(size_t)q * nt + i] = red[q][0];
}

__global__ void noalloc_final_kernel(const double *part, int nrows, double *out)
{
    __shared__ double red[NQ][NOALLOC_THREADS];
    double acc[NQ] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nrows; i += NOALLOC_THREADS)
        for (int q = 0; q < NQ; ++q) acc[q] += part[(size_t)q * nrows + i];
    for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = NOALLOC_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NQ; ++q) out[q] = red[q][0];
}

int na_fail(int code, const std::string &m)
{
    g_noalloc_error = m;
    return code;
}

// Device address of the scratch array for the current device (looked up once per device).
int scratch_for_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(VLBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return na_fail(VLBM_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(VLBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return VLBM_OK;
}

}  // namespace

extern "C" {

int vlbm_diagnostics_noalloc(const double *f_dev, int n_theta, int n_phi, double radius, double *out_dev,
                             void *stream)
{
    if (!f_dev || !out_dev) return na_fail(VLBM_ERR_ARG, "NULL device pointer");
    if (n_theta < 1 || n_phi < 1 || !(radius > 0.0)) return na_fail(VLBM_ERR_ARG, "bad grid or radius");
    if (n_theta > VLBM_NOALLOC_MAX_ROWS)
        return na_fail(VLBM_ERR_ARG, "n_theta = " + std::to_string(n_theta) + " exceeds the scratch limit of " +
                                         std::to_string(VLBM_NOALLOC_MAX_ROWS) + " rows");
    double *part = nullptr;
    int rc = scratch_for_current_device(&part);
    if (rc) return rc;
    VelNA c;
    const double big = sqrt(3.0 + sqrt(6.0)), small = sqrt(3.0 - sqrt(6.0));
    c.v[0] = -big;
    c.v[1] = -small;
    c.v[2] = small;
    c.v[3] = big;
    for (int a = 0; a < 4; ++a) {
        const double x = c.v[a];
        const double h5 = x * x * x * x * x - 10.0 * x * x * x + 15.0 * x;   // He_5
        c.w[a] = 24.0 / (h5 * h5);
    }
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_rows_kernel<<<n_theta, NOALLOC_THREADS, 0, s>>>(f_dev, n_theta, n_phi, radius, c, part);
    noalloc_final_kernel<<<1, NOALLOC_THREADS, 0, s>>>(part, n_theta, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(VLBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return VLBM_OK;
}

const char *vlbm_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

}  // extern "C"
