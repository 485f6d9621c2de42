// lc.cu -- learned correction for a coarse vLBM (not in the paper).
//
// A small convolutional network nudges the moments of a coarse FP32 solver
// toward those of a finer run after each coarse step.  Layers: 3x3 convolutions
// 4 -> H -> H -> H -> 3 with ReLU between, on the coarse cell grid.  Padding
// follows the boundary conditions of the sphere (arXiv 2504.15574 Sec. 3.6):
// periodic in phi, and beyond a pole the row on the opposite meridian
// (column + N_phi/2) with the vector channels (u^theta, u^phi of the input
// layer, and its sin(theta) channel) negated.
//
// Arithmetic: activations and weights in BF16, products accumulated in FP32 on
// the tensor cores (mma.sync m16n8k16, BF16 in, FP32 out); master weights, Adam
// moments, losses and gradients of the weights in FP32.  Every convolution,
// forward and backward, is a "valid" 3x3 convolution over an explicitly padded
// channels-last tensor [rows][cols][channels]:
//   forward:        Y  = conv(pad(X), W)
//   backward data:  dP = conv(zero-pad-2(dY), W flipped and transposed), then the
//                   adjoint of pad() folds ghost gradients onto their sources;
//   backward weight: dW[co][tap][ci] = sum_p dY[p][co] pad(X)[p + tap][ci].
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "vlbm_internal.h"
#include "f32_images.cuh"
#include "lc_internal.h"

namespace vk {

namespace {

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x = lo (low 16 bits), .y = hi
    return *reinterpret_cast<unsigned *>(&v);
}

__device__ __forceinline__ unsigned pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<unsigned *>(&v);
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---- padding and its adjoint ------------------------------------------------------
// A padded tensor Xp [H+2][W+2][C] holds X [H][W][C] at (y+1, x+1); its ghost columns
// wrap in phi and its ghost rows are the first/last row on the opposite meridian
// (column + W/2), with the channels in a sign mask negated (the pole condition of
// Sec. 3.6 applied to moments).  Producers write every value at all its positions:

// calls put(padded row, padded column, pole image?) for every position of interior (y, x)
template <class Put>
__device__ __forceinline__ void for_padded_positions(int H, int W, int y, int x, Put put)
{
    put(y + 1, x + 1, false);
    if (x == W - 1) put(y + 1, 0, false);
    if (x == 0) put(y + 1, W + 1, false);
    for (int side = 0; side < 2; ++side) {
        if ((side == 0 && y != 0) || (side == 1 && y != H - 1)) continue;
        const int r = side ? H + 1 : 0;
        put(r, (x - W / 2 + W) % W + 1, true);
        if (x == (W / 2 + W - 1) % W) put(r, 0, true);
        if (x == W / 2 % W) put(r, W + 1, true);
    }
}

// adjoint of pad_kernel: dX[y][x] = dXp[y+1][x+1] + ghost copies that read (y, x)
__global__ void unpad_kernel(const float *dXp, int H, int W, int C, unsigned negmask, float *dX)
{
    const int c = threadIdx.x;
    const int x = blockIdx.x, y = blockIdx.y;
    if (c >= C) return;
    const int Wp = W + 2;
    auto at = [&](int yp, int xp) { return dXp[((size_t)yp * Wp + xp) * C + c]; };
    float s = at(y + 1, x + 1);
    // ghost columns (xp = 0 reads x = W-1, xp = W+1 reads x = 0), in the interior rows
    if (x == W - 1) s += at(y + 1, 0);
    if (x == 0) s += at(y + 1, W + 1);
    // ghost rows: row yp = 0 (or H+1), column xp reads row 0 (or H-1) at column xp-1+W/2 (mod W)
    const float sg = ((negmask >> c) & 1u) ? -1.0f : 1.0f;
    for (int pole = 0; pole < 2; ++pole) {
        const int yrow = pole ? H - 1 : 0;
        if (y != yrow) continue;
        const int yp = pole ? H + 1 : 0;
        for (int xp = 0; xp < Wp; ++xp) {
            int xs = (xp - 1 + W / 2) % W;
            if (xs < 0) xs += W;
            if (xs == x) s += sg * at(yp, xp);
        }
    }
    dX[((size_t)y * W + x) * C + c] = s;
}

// ---- valid 3x3 convolution on the tensor cores --------------------------------------
// Xp [Hp][Wp][Ci] bf16 (Ci multiple of 16), Wt [Co][9][Ci] bf16 (Co multiple of 8, <= 32),
// out [Hp-2][Wp-2][Co]: Yf (fp32, optional) and Yb (bf16, optional, after ReLU if relu).
// CTA: one output row, 64 consecutive output columns, 4 warps of 16 pixels.
constexpr int CONV_PIX = 64;

template <int CI, int CO>
// part0 (optional): per CTA (index blockIdx.y gridDim.x + blockIdx.x) the sum over its pixels of
// sin_t[row] times output channel 0 (the direct form's drho before its scale; FP64)
__global__ void __launch_bounds__(128) conv3x3_kernel(const __nv_bfloat16 *Xp, int Hp, int Wp,
                                                       const __nv_bfloat16 *Wt, const float *bias, float *Yf,
                                                       __nv_bfloat16 *Yb, __nv_bfloat16 *Ypad, int relu,
                                                       double *part0, const double *sin_t)
{
    constexpr int XS = CI + 8;           // padded channel stride in shared memory (bank spread)
    constexpr int WS = 9 * CI + 8;
    __shared__ __align__(16) __nv_bfloat16 xs[3][CONV_PIX + 2][XS];
    __shared__ __align__(16) __nv_bfloat16 ws[CO][WS];
    const int Ho = Hp - 2, Wo = Wp - 2;
    const int y = blockIdx.y, x0 = blockIdx.x * CONV_PIX;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // stage the input rows y..y+2, columns x0..x0+65 (zero beyond Wp) and the weights, 16 bytes
    // (8 channels) per access: CI, XS and WS are multiples of 8
    constexpr int CV = CI / 8;
    for (int e = tid; e < 3 * (CONV_PIX + 2) * CV; e += blockDim.x) {
        const int cv = e % CV, rest = e / CV, xx = rest % (CONV_PIX + 2), r = rest / (CONV_PIX + 2);
        const int gx = x0 + xx;
        const uint4 v = (gx < Wp) ? *reinterpret_cast<const uint4 *>(Xp + ((size_t)(y + r) * Wp + gx) * CI + 8 * cv)
                                  : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(&xs[r][xx][8 * cv]) = v;
    }
    constexpr int WV = 9 * CI / 8;
    for (int e = tid; e < CO * WV; e += blockDim.x)
        *reinterpret_cast<uint4 *>(&ws[e / WV][8 * (e % WV)]) = *reinterpret_cast<const uint4 *>(Wt + 8 * e);
    __syncthreads();

    const int g = lane >> 2, t = lane & 3;
    float acc[CO / 8][4];
#pragma unroll
    for (int nb = 0; nb < CO / 8; ++nb)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nb][q] = 0.0f;
    const int pbase = warp * 16;        // this warp's first pixel within the CTA tile
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
        for (int kc = 0; kc < CI / 16; ++kc) {
            const int k0 = kc * 16 + 2 * t;
            unsigned a[4];
            a[0] = *reinterpret_cast<const unsigned *>(&xs[dy][pbase + g + dx][k0]);
            a[1] = *reinterpret_cast<const unsigned *>(&xs[dy][pbase + g + 8 + dx][k0]);
            a[2] = *reinterpret_cast<const unsigned *>(&xs[dy][pbase + g + dx][k0 + 8]);
            a[3] = *reinterpret_cast<const unsigned *>(&xs[dy][pbase + g + 8 + dx][k0 + 8]);
#pragma unroll
            for (int nb = 0; nb < CO / 8; ++nb) {
                unsigned b[2];
                b[0] = *reinterpret_cast<const unsigned *>(&ws[nb * 8 + g][tap * CI + k0]);
                b[1] = *reinterpret_cast<const unsigned *>(&ws[nb * 8 + g][tap * CI + k0 + 8]);
                mma_bf16(acc[nb], a, b);
            }
        }
    }
    // epilogue: rows g and g+8 of the warp tile, columns 2t, 2t+1 of each n-block
    double p0 = 0.0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int x = x0 + pbase + g + 8 * half;
        if (x >= Wo) continue;
        if (part0 && t == 0) p0 += (double)(acc[0][2 * half] + (bias ? bias[0] : 0.0f));
        const size_t o = ((size_t)y * Wo + x) * CO;
#pragma unroll
        for (int nb = 0; nb < CO / 8; ++nb) {
            const int co = nb * 8 + 2 * t;
            float v0 = acc[nb][2 * half] + (bias ? bias[co] : 0.0f);
            float v1 = acc[nb][2 * half + 1] + (bias ? bias[co + 1] : 0.0f);
            if (Yf) {
                Yf[o + co] = v0;
                Yf[o + co + 1] = v1;
            }
            if (relu) {
                v0 = fmaxf(v0, 0.0f);
                v1 = fmaxf(v1, 0.0f);
            }
            const __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
            if (Yb) *reinterpret_cast<__nv_bfloat162 *>(Yb + o + co) = pr;
            // hidden activations carry no sign flip across the poles
            if (Ypad)
                for_padded_positions(Ho, Wo, y, x, [&](int prow, int pcol, bool) {
                    *reinterpret_cast<__nv_bfloat162 *>(Ypad + ((size_t)prow * (Wo + 2) + pcol) * CO + co) = pr;
                });
        }
    }
    if (part0) {   // (uniform over the CTA)
        __shared__ double red[128];
        red[tid] = p0 * sin_t[y];
        __syncthreads();
        for (int k = 64; k > 0; k >>= 1) {
            if (tid < k) red[tid] += red[tid + k];
            __syncthreads();
        }
        if (tid == 0) part0[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    }
}

// ---- weight gradient on the tensor cores ---------------------------------------------
// dY [H][W][CO] bf16 (gradient at the pre-activation), Xp [H+2][W+2][CI] bf16.
// One CTA per output row: part[row][9][CO][CI] and partb[row][CO] (bias) in FP32.
template <int CI, int CO>
__global__ void __launch_bounds__(128) wgrad_kernel(const __nv_bfloat16 *dY, const __nv_bfloat16 *Xp, int H, int W,
                                                     float *part, float *partb)
{
    constexpr int NPIX = 64;
    __shared__ __align__(16) __nv_bfloat16 dys[NPIX][CO + 8];
    __shared__ __align__(16) __nv_bfloat16 xs[3][NPIX + 2][CI + 8];
    const int y = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    // warp w: taps w, w+4, w+8 (<9); each tap: (CO/16) x (CI/8) accumulator tiles
    float acc[3][CO / 16][CI / 8][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < CO / 16; ++m)
#pragma unroll
            for (int n = 0; n < CI / 8; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[a][m][n][q] = 0.0f;
    float bsum = 0.0f;
    for (int x0 = 0; x0 < W; x0 += NPIX) {
        __syncthreads();
        for (int e = tid; e < NPIX * CO; e += blockDim.x) {
            const int p = e / CO, c = e % CO;
            dys[p][c] = (x0 + p < W) ? dY[((size_t)y * W + x0 + p) * CO + c] : __float2bfloat16(0.0f);
        }
        for (int e = tid; e < 3 * (NPIX + 2) * CI; e += blockDim.x) {
            const int c = e % CI, rest = e / CI, xx = rest % (NPIX + 2), r = rest / (NPIX + 2);
            const int gx = x0 + xx;
            xs[r][xx][c] = (gx < W + 2) ? Xp[((size_t)(y + r) * (W + 2) + gx) * CI + c] : __float2bfloat16(0.0f);
        }
        __syncthreads();
        if (tid < CO)
            for (int p = 0; p < NPIX; ++p) bsum += __bfloat162float(dys[p][tid]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int tap = warp + 4 * a;
            if (tap >= 9) break;
            const int dy = tap / 3, dx = tap % 3;
#pragma unroll
            for (int ks = 0; ks < NPIX / 16; ++ks) {
                const int p0 = ks * 16 + 2 * t;   // k = pixel
#pragma unroll
                for (int m = 0; m < CO / 16; ++m) {
                    // A[m = co][k = pixel] = dY[pixel][co]
                    unsigned av[4];
                    const int co0 = m * 16 + g;
                    av[0] = pack_raw(dys[p0][co0], dys[p0 + 1][co0]);
                    av[1] = pack_raw(dys[p0][co0 + 8], dys[p0 + 1][co0 + 8]);
                    av[2] = pack_raw(dys[p0 + 8][co0], dys[p0 + 9][co0]);
                    av[3] = pack_raw(dys[p0 + 8][co0 + 8], dys[p0 + 9][co0 + 8]);
#pragma unroll
                    for (int n = 0; n < CI / 8; ++n) {
                        // B[k = pixel][n = ci] = Xp[y + dy][pixel + dx][ci]
                        const int ci = n * 8 + g;
                        unsigned bv[2];
                        bv[0] = pack_raw(xs[dy][p0 + dx][ci], xs[dy][p0 + 1 + dx][ci]);
                        bv[1] = pack_raw(xs[dy][p0 + 8 + dx][ci], xs[dy][p0 + 9 + dx][ci]);
                        mma_bf16(acc[a][m][n], av, bv);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int tap = warp + 4 * a;
        if (tap >= 9) break;
#pragma unroll
        for (int m = 0; m < CO / 16; ++m)
#pragma unroll
            for (int n = 0; n < CI / 8; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int co = m * 16 + g + 8 * (q >> 1);
                    const int ci = n * 8 + 2 * t + (q & 1);
                    part[(((size_t)y * 9 + tap) * CO + co) * CI + ci] = acc[a][m][n][q];
                }
    }
    if (tid < CO) partb[(size_t)y * CO + tid] = bsum;
}

// sums partials over rows in order: out[i] = sum_r part[r][i]
__global__ void reduce_rows_kernel(const float *part, int rows, int n, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += part[(size_t)r * n + i];
    out[i] = s;
}

// ---- elementwise pieces -------------------------------------------------------------
// dP (bf16, zero-padded by 2 on rows and columns, channel count CP >= C) from the
// FP32 gradient at a layer output and the ReLU mask of that output (mask NULL: none).
__global__ void grad_pad2_kernel(const float *dY, const __nv_bfloat16 *act, int H, int W, int C, int CP,
                                 __nv_bfloat16 *dP)
{
    const int c = threadIdx.x;
    const int xp = blockIdx.x, yp = blockIdx.y;
    if (c >= CP) return;
    const int y = yp - 2, x = xp - 2;
    float v = 0.0f;
    if (c < C && y >= 0 && y < H && x >= 0 && x < W) {
        const size_t i = ((size_t)y * W + x) * C + c;
        v = dY[i];
        if (act && __bfloat162float(act[i]) <= 0.0f) v = 0.0f;
    }
    dP[((size_t)yp * (W + 4) + xp) * CP + c] = __float2bfloat16(v);
}

// the un-padded gradient at the pre-activation (bf16), for the weight gradient
__global__ void grad_pre_kernel(const float *dY, const __nv_bfloat16 *act, int n, int C, int CP,
                                __nv_bfloat16 *dPre)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * CP) return;
    const int c = i % CP, p = i / CP;
    float v = 0.0f;
    if (c < C) {
        v = dY[(size_t)p * C + c];
        if (act && __bfloat162float(act[(size_t)p * C + c]) <= 0.0f) v = 0.0f;
    }
    dPre[i] = __float2bfloat16(v);
}

// area-weighted mean-square loss against targets [3][H][W] (scaled), gradient into dY [H][W][CO]
__global__ void loss_kernel(const float *Y, int CO, const double *target, const double *sin_t, int H, int W,
                            float3 inv_scale, double wsum, float *dY, double *part)
{
    __shared__ double red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < H * W) {
        const int y = i / W;
        const double w = sin_t[y] / wsum;
        const float sc[3] = {inv_scale.x, inv_scale.y, inv_scale.z};
        for (int c = 0; c < CO; ++c) {
            float g = 0.0f;
            if (c < 3) {
                const double d = (double)Y[(size_t)i * CO + c] - target[(size_t)c * H * W + i] * sc[c];
                l += w * d * d / 3.0;
                g = (float)(2.0 * w * d / 3.0);
            }
            dY[(size_t)i * CO + c] = g;
        }
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_kernel(const double *part, int n, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adam on FP32 master weights (bias-corrected), then the bf16 copies.
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 weight layouts of one layer from its FP32 master [CO][CI][3][3]:
//   fwd [COp][9][CIp] and bwd-data [CIp2][9][COp2] (taps flipped, channels swapped)
__global__ void weights_bf16_kernel(const float *w, int CO, int CI, int COp, int CIp, __nv_bfloat16 *fwd, int CIp2,
                                    int COp2, __nv_bfloat16 *bwd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < COp * 9 * CIp) {
        const int ci = i % CIp, tap = (i / CIp) % 9, co = i / (9 * CIp);
        fwd[i] = __float2bfloat16((co < CO && ci < CI) ? w[((size_t)co * CI + ci) * 9 + tap] : 0.0f);
    }
    if (bwd && i < CIp2 * 9 * COp2) {
        const int co = i % COp2, tap = (i / COp2) % 9, ci = i / (9 * COp2);
        const int ftap = 8 - tap;
        bwd[i] = __float2bfloat16((co < CO && ci < CI) ? w[((size_t)co * CI + ci) * 9 + ftap] : 0.0f);
    }
}

// weight gradient from [9][CO][CI] into the master layout [CO][CI][3][3]
__global__ void wgrad_layout_kernel(const float *g9, int CO, int CI, int COp, int CIp, float *g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= CO * CI * 9) return;
    const int tap = i % 9, ci = (i / 9) % CI, co = i / (9 * CI);
    g[i] = g9[((size_t)tap * COp + co) * CIp + ci];
}

// Value of a moment field at grid point (r, c) for -3 <= r < H + 3: columns wrap; a
// row beyond a pole is the mirrored row on the opposite meridian (c + W/2), negated
// for a velocity component (sgn = -1), as the pole condition of Sec. 3.6 maps it.
template <typename T>
__device__ __forceinline__ T lc_at(const T *a, int H, int W, int r, int c, T sgn)
{
    T s = 1;
    if (r < 0 || r >= H) {
        r = (r < 0) ? (-1 - r) : (2 * H - 1 - r);
        c += W / 2;
        s = sgn;
    }
    c %= W;
    if (c < 0) c += W;
    return s * a[(size_t)r * W + c];
}

// undivided 4th and 6th differences of a field along theta (dir 0) or phi (dir 1) at (i, j)
__device__ __forceinline__ void lc_differences(const float *a, int H, int W, int i, int j, int dir, float sgn,
                                               float &d4, float &d6)
{
    float x[7];
#pragma unroll
    for (int m = 0; m < 7; ++m)
        x[m] = dir ? lc_at(a, H, W, i, j + m - 3, sgn) : lc_at(a, H, W, i + m - 3, j, sgn);
    d4 = x[1] - 4.0f * x[2] + 6.0f * x[3] - 4.0f * x[4] + x[5];
    d6 = x[0] - 6.0f * x[1] + 15.0f * x[2] - 20.0f * x[3] + 15.0f * x[4] - 6.0f * x[5] + x[6];
}

// the network's FP32 moment deviations (rho - 1, u^theta, u^phi, T - 1) [4][H][W] of FP64 moments
// (rho, u^theta, u^phi, T) [4][H][W]: the deviations are formed in FP64, then rounded
__global__ void dev_of_moments_kernel(const double *in4, int n, float *dev)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    dev[c] = (float)(in4[c] - 1.0);
    dev[(size_t)n + c] = (float)in4[(size_t)n + c];
    dev[2 * (size_t)n + c] = (float)in4[2 * (size_t)n + c];
    dev[3 * (size_t)n + c] = (float)(in4[3 * (size_t)n + c] - 1.0);
}

// network input from the moment deviations dev = (rho - 1, u^theta, u^phi, T - 1) [4][H][W]
// (channel order in lc_internal.h): the deviations and their undivided 4th / 6th differences in
// FP32 — on rho - 1, not rho, so that the differences keep the FP32 resolution of the deviation
// (~1e-3 of rho: ~1e-10 absolute) rather than of rho — divided by their scales and clamped to
// [-LC_CLAMP, LC_CLAMP] before the BF16 rounding (a BF16 field could not resolve the high-order
// differences that carry a coarse scheme's truncation error); the latitude channels let the
// translation-equivariant convolutions depend on theta.
__global__ void features_kernel(const float *dev, int H, int W, const double *sin_t, const double *cos_t,
                                const LcInScale sc, __nv_bfloat16 *Xp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t HW = (size_t)H * W;
    if (i >= H * W) return;
    const int r = i / W, c = i - r * W;
    const float *drho = dev, *ut = dev + HW, *up = dev + 2 * HW;
    float raw[LC_NSCALE];
    raw[0] = drho[i];
    raw[1] = ut[i];
    raw[2] = up[i];
    raw[3] = dev[3 * HW + i];
    float d4, d6;
    lc_differences(drho, H, W, r, c, 0, 1.0f, d4, d6);
    raw[4] = d6;
    lc_differences(drho, H, W, r, c, 1, 1.0f, d4, d6);
    raw[5] = d6;
    lc_differences(ut, H, W, r, c, 0, -1.0f, d4, d6);
    raw[6] = d6;
    raw[10] = d4;
    lc_differences(ut, H, W, r, c, 1, -1.0f, d4, d6);
    raw[7] = d6;
    raw[11] = d4;
    lc_differences(up, H, W, r, c, 0, -1.0f, d4, d6);
    raw[8] = d6;
    raw[12] = d4;
    lc_differences(up, H, W, r, c, 1, -1.0f, d4, d6);
    raw[9] = d6;
    raw[13] = d4;
    float v[LC_CIN];
#pragma unroll
    for (int q = 0; q < LC_NSCALE; ++q) {
        const float x = raw[q] * sc.inv[q];
        v[q < 4 ? q : q + 2] = fminf(fmaxf(x, -LC_CLAMP), LC_CLAMP);
    }
    v[4] = (float)cos_t[r];
    v[5] = (float)sin_t[r];
    // the padded input of layer 0 at all positions of (r, c); pole images negate LC_NEGMASK
    uint4 plain[2], image[2];
    __nv_bfloat16 *pb = reinterpret_cast<__nv_bfloat16 *>(plain), *ib = reinterpret_cast<__nv_bfloat16 *>(image);
#pragma unroll
    for (int q = 0; q < LC_CIN; ++q) {
        pb[q] = __float2bfloat16(v[q]);
        ib[q] = ((LC_NEGMASK >> q) & 1u) ? __hneg(pb[q]) : pb[q];
    }
    for_padded_positions(H, W, r, c, [&](int pr, int pc, bool img) {
        uint4 *dst = reinterpret_cast<uint4 *>(Xp + ((size_t)pr * (W + 2) + pc) * LC_CIN);
        dst[0] = img ? image[0] : plain[0];
        dst[1] = img ? image[1] : plain[1];
    });
}

// output [H][W][CO] -> (drho, dut, dup) [3][H][W] in physical units, and sin-weighted drho partial sums
__global__ void outputs_kernel(const float *Y, int CO, int H, int W, float3 scale, const double *sin_t, double *out,
                               double *part)
{
    __shared__ double red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < H * W) {
        const double d0 = (double)Y[(size_t)i * CO + 0] * scale.x;
        out[i] = d0;
        out[(size_t)H * W + i] = (double)Y[(size_t)i * CO + 1] * scale.y;
        out[(size_t)2 * H * W + i] = (double)Y[(size_t)i * CO + 2] * scale.z;
        s = d0 * sin_t[i / W];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---- stream-function output form: output 0 times s0 is psi, the correction its centred curl
// du^theta = s0 (psi[i][j+1] - psi[i][j-1]) / (2 R dphi sin theta_i),
// du^phi = -s0 (psi[i+1][j] - psi[i-1][j]) / (2 R dtheta); a row beyond a pole is the edge row on
// the opposite meridian (column + W/2; psi is a scalar: no sign change).

// psi of cell (i, j) (element i W + j times CO of Y: output 0 of the net, or a psi array with
// CO = 1), rows beyond a pole and columns wrapped as above
template <typename T>
__device__ __forceinline__ double psi_at(const T *Y, int CO, int H, int W, int i, int j)
{
    if (i < 0) {
        i = 0;
        j += W / 2;
    } else if (i >= H) {
        i = H - 1;
        j += W / 2;
    }
    j %= W;
    if (j < 0) j += W;
    return (double)Y[((size_t)i * W + j) * CO];
}

template <typename T>
__device__ __forceinline__ void stream_uv(const T *Y, int CO, const LcStream &g, const double *sin_t, int i, int j,
                                          double &ut, double &up)
{
    ut = g.s0 * (psi_at(Y, CO, g.H, g.W, i, j + 1) - psi_at(Y, CO, g.H, g.W, i, j - 1)) /
         (2.0 * g.R * g.dph * sin_t[i]);
    up = -g.s0 * (psi_at(Y, CO, g.H, g.W, i + 1, j) - psi_at(Y, CO, g.H, g.W, i - 1, j)) / (2.0 * g.R * g.dth);
}

// loss of the stream form: the sin-area-weighted mean over cells and the two velocity channels of
// ((du - target) / out_scale)^2; per cell the loss's derivatives by du^theta and du^phi into gv
// [2][H][W]; per block partial sums of the loss
template <typename T>
__global__ void stream_loss_kernel(const T *Y, int CO, const double *target, const double *sin_t, LcStream g,
                                   double inv_s1, double inv_s2, double wsum, double *gv, double *part)
{
    __shared__ double red[256];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int HW = g.H * g.W;
    double l = 0.0;
    if (c < HW) {
        const int i = c / g.W, j = c - i * g.W;
        double ut, up;
        stream_uv(Y, CO, g, sin_t, i, j, ut, up);
        const double w = sin_t[i] / wsum;
        const double rt = (ut - target[(size_t)HW + c]) * inv_s1, rp = (up - target[2 * (size_t)HW + c]) * inv_s2;
        l = 0.5 * w * (rt * rt + rp * rp);
        gv[c] = w * rt * inv_s1;
        gv[(size_t)HW + c] = w * rp * inv_s2;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// the adjoint of the curl applied to gv, times s0, into element c CO of dY ([H][W][CO]; the
// net's output gradient, whose other outputs get 0) or of a plain array (CO = 1)
template <typename TO>
__global__ void stream_adjoint_kernel(const double *gv, int CO, LcStream g, const double *sin_t, TO *dY)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int H = g.H, W = g.W, HW = H * W;
    if (c >= HW) return;
    const int i = c / W, j = c - i * W;
    const int jm = (j + W - 1) % W, jp = (j + 1) % W, jo = (j + W / 2) % W;
    const double ka = 1.0 / (2.0 * g.R * g.dph * sin_t[i]), kb = 1.0 / (2.0 * g.R * g.dth);
    const double *gt = gv, *gp = gv + HW;
    // psi[i][j] enters du^theta of (i, j - 1) with + and of (i, j + 1) with -, du^phi of row
    // i - 1 with - and of row i + 1 with +; at a pole row, also du^phi of the same row on the
    // opposite meridian through the continuation
    double d = ka * (gt[(size_t)i * W + jm] - gt[(size_t)i * W + jp]);
    if (i > 0) d -= kb * gp[(size_t)(i - 1) * W + j];
    else d += kb * gp[jo];
    if (i < H - 1) d += kb * gp[(size_t)(i + 1) * W + j];
    else d -= kb * gp[(size_t)(H - 1) * W + jo];
    dY[(size_t)c * CO] = (TO)(g.s0 * d);
    for (int o = 1; o < CO; ++o) dY[(size_t)c * CO + o] = (TO)0;
}

// the stream form's correction (0, du^theta, du^phi) [3][H][W] in physical units; the drho
// partial sums are 0
template <typename T>
__global__ void stream_outputs_kernel(const T *Y, int CO, LcStream g, const double *sin_t, double *out,
                                      double *part)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int HW = g.H * g.W;
    if (c < HW) {
        const int i = c / g.W, j = c - i * g.W;
        double ut, up;
        stream_uv(Y, CO, g, sin_t, i, j, ut, up);
        out[c] = 0.0;
        out[(size_t)HW + c] = ut;
        out[2 * (size_t)HW + c] = up;
    }
    if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
}

// ---- vorticity output form: psi from the finite-volume Poisson equation on the sphere,
// L psi = w - (area mean of w), with
//   (L psi)_ij = (sf_{i+1} (psi_{i+1,j} - psi_ij) - sf_i (psi_ij - psi_{i-1,j})) / (R^2 s_i dth^2)
//              + (psi_{i,j+1} - 2 psi_ij + psi_{i,j-1}) / (R^2 s_i^2 dph^2),
// s_i = sin theta_i at the cell centres and sf_i = sin(i dth) at the faces, 0 at both poles (no
// flux through a pole face).  Along phi a DFT on the cell centres phi_j = (j + 1/2) dph,
// X_m = sum_j x_j exp(-i m phi_j) for m = 0 .. W/2, in FP32 (twiddles by complex rotation,
// re-anchored from a table of (cos, sin)(pi k / W)).  Per mode m > 0 a tridiagonal system in theta (the second difference
// along phi has the symbol -(2 sin(m dph / 2) / dph)^2; diagonally dominant), solved in FP32 by the
// Thomas recursion with its factors tabulated per (mode, row) from FP64; mode 0 integrated from the
// north pole as the conservative flux G_{i+1} = G_i + dth^2 s_i X_0,i (G_0 = 0), psi_{i+1} = psi_i +
// G_{i+1} / sf_{i+1}, psi_0 = 0 (the constant of psi has no curl).  FP32 throughout the solve:
// GB300's FP64 units make a serial FP64 recursion ~100x slower, and the recursion is stable for
// diagonally dominant systems, its error within the condition number (~1e4 at m = 1 on 128 rows)
// times FP32 rounding.  The tables are for R = 1; the right side carries R^2.  Modes are stored
// mode-major, X[m][i].

// per-block partial sums of x [n] (cells of rows of W; weighted by the cell sine when `weighted`)
__global__ void cell_sums_kernel(const double *x, int n, int W, const double *sin_t, int weighted, double *part)
{
    __shared__ double red[256];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (c < n) v = weighted ? x[c] * sin_t[c / W] : x[c];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// the vorticity correction w = s0 * output 0 of the net, and per-block partial sums of s_i w
__global__ void vort_in_kernel(const float *Y, int CO, int n, int W, double s0, const double *sin_t, double *w,
                               double *part)
{
    __shared__ double red[256];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (c < n) {
        const double x = s0 * (double)Y[(size_t)c * CO];
        w[c] = x;
        v = x * sin_t[c / W];
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// DFT of row i (block i, threads over the modes) of R^2 (x / s_i^inv_sin - mean), the mean the sum
// of the nb partial sums over wsum; X[m][i].  Thread m advances exp(-i m phi_j) by complex rotation
// through exp(-i m dph) and re-anchors it from the table tw[k] = (cos, sin)(pi k / W) every
// DFT_ANCHOR columns (m phi_j = pi m (2j + 1) / W).
constexpr int DFT_ANCHOR = 16;
__global__ void dft_rows_kernel(const double *x, int H, int W, const double *sin_t, int inv_sin, const double *part,
                                int nb, double wsum, double R2, const float2 *tw, float2 *X)
{
    extern __shared__ float row[];
    __shared__ double red[256];
    const int i = blockIdx.x, M = W / 2 + 1, W2 = 2 * W;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += part[b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double mean = red[0] / wsum, rs = inv_sin ? 1.0 / sin_t[i] : 1.0;
    for (int j = threadIdx.x; j < W; j += blockDim.x) row[j] = (float)(R2 * (x[(size_t)i * W + j] * rs - mean));
    __syncthreads();
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float2 st = tw[(2 * m) % W2];   // exp(+i m dph)
        float re = 0.0f, im = 0.0f;
        for (int j0 = 0; j0 < W; j0 += DFT_ANCHOR) {
            const float2 z0 = tw[(int)(((long long)m * (2 * j0 + 1)) % W2)];
            float zc = z0.x, zs = z0.y;   // exp(+i m phi_j) = (zc, zs)
            const int j1 = min(j0 + DFT_ANCHOR, W);
            for (int j = j0; j < j1; ++j) {
                re = fmaf(row[j], zc, re);
                im = fmaf(-row[j], zs, im);
                const float c2 = zc * st.x - zs * st.y, s2 = fmaf(zc, st.y, zs * st.x);
                zc = c2;
                zs = s2;
            }
        }
        X[(size_t)m * H + i] = make_float2(re, im);
    }
}

// Poisson solve of every mode in place, one warp per mode: the lanes stage the mode's column and
// its recursion factors in shared memory, lane 0 runs the recursion there, the lanes write the
// solution back.  tab[m][i] = (c'_i, 1 / (b_i - a_i c'_{i-1})) for m > 0 and (dth^2 s_i,
// 1 / sf_{i+1}) for m = 0; a[i] = sf_i / (s_i dth^2).  Shared memory: a[H], then per warp the
// column and the factors (2 x H float2).
constexpr int TRI_WARPS = 4;
__global__ void __launch_bounds__(TRI_WARPS * 32) tri_solve_kernel(float2 *__restrict__ X, int H, int M,
                                                                   const float2 *__restrict__ tab,
                                                                   const float *__restrict__ a)
{
    extern __shared__ float2 tsm[];
    float *as = reinterpret_cast<float *>(tsm);
    for (int i = threadIdx.x; i < H; i += blockDim.x) as[i] = a[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int m = blockIdx.x * TRI_WARPS + wp;
    if (m >= M) return;
    float2 *xs = tsm + (H + 1) / 2 + (size_t)wp * 2 * H;   // past a[] (H floats, rounded to float2)
    float2 *ts = xs + H;
    for (int i = lane; i < H; i += 32) {
        xs[i] = X[(size_t)m * H + i];
        ts[i] = tab[(size_t)m * H + i];
    }
    __syncwarp();
    if (lane == 0) {
        if (m == 0) {
            float G = 0.0f, psi = 0.0f;
            for (int i = 0; i < H; ++i) {
                const float d = xs[i].x;
                const float2 t = ts[i];
                xs[i] = make_float2(psi, 0.0f);
                if (i + 1 < H) {
                    G = fmaf(t.x, d, G);
                    psi = fmaf(G, t.y, psi);
                }
            }
        } else {
            float2 dp = make_float2(0.0f, 0.0f);   // d'_i = (d_i - a_i d'_{i-1}) r_i
            for (int i = 0; i < H; ++i) {
                const float r = ts[i].y, ai = as[i];
                const float2 d = xs[i];
                dp = make_float2(fmaf(-ai, dp.x, d.x) * r, fmaf(-ai, dp.y, d.y) * r);
                xs[i] = dp;
            }
            float2 p = make_float2(0.0f, 0.0f);    // psi_i = d'_i - c'_i psi_{i+1}
            for (int i = H - 1; i >= 0; --i) {
                const float c = ts[i].x;
                const float2 d = xs[i];
                p = make_float2(fmaf(-c, p.x, d.x), fmaf(-c, p.y, d.y));
                xs[i] = p;
            }
        }
    }
    __syncwarp();
    for (int i = lane; i < H; i += 32) X[(size_t)m * H + i] = xs[i];
}

// inverse DFT of row i (block i, threads over the columns): psi_ij = (X_0 + 2 sum_{0<m<W/2}
// Re(X_m e^{i m phi_j}) + Re(X_{W/2} e^{i W/2 phi_j})) / W; thread j advances exp(i m phi_j) over m by
// rotation through exp(i phi_j), re-anchored from the table every DFT_ANCHOR modes
__global__ void idft_rows_kernel(const float2 *X, int H, int W, const float2 *tw, double *psi)
{
    extern __shared__ float2 xr[];
    const int i = blockIdx.x, M = W / 2 + 1, W2 = 2 * W;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float2 v = X[(size_t)m * H + i];
        const float f = (m == 0 || 2 * m == W) ? 1.0f : 2.0f;
        xr[m] = make_float2(f * v.x, f * v.y);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const float2 st = tw[(2 * j + 1) % W2];   // exp(i phi_j)
        float acc = 0.0f;
        for (int m0 = 0; m0 < M; m0 += DFT_ANCHOR) {
            const float2 z0 = tw[(int)(((long long)m0 * (2 * j + 1)) % W2)];
            float zc = z0.x, zs = z0.y;
            const int m1 = min(m0 + DFT_ANCHOR, M);
            for (int m = m0; m < m1; ++m) {
                acc = fmaf(xr[m].x, zc, acc);
                acc = fmaf(-xr[m].y, zs, acc);
                const float c2 = zc * st.x - zs * st.y, s2 = fmaf(zc, st.y, zs * st.x);
                zc = c2;
                zs = s2;
            }
        }
        psi[(size_t)i * W + j] = (double)acc / W;
    }
}

// the vorticity form's output gradient: dY[c CO] = s0 (s_i u_c - s_i (*sum) / wsum) (the adjoint of
// the solve S P S^-1, then of the mean removal), the other outputs 0
__global__ void vort_grad_kernel(const double *u, int H, int W, int CO, const double *sin_t, const double *sum,
                                 double wsum, double s0, float *dY)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= H * W) return;
    const double si = sin_t[c / W];
    dY[(size_t)c * CO] = (float)(s0 * si * (u[c] - *sum / wsum));
    for (int o = 1; o < CO; ++o) dY[(size_t)c * CO + o] = 0.0f;
}

// Moments (rho, u^theta, u^phi, T) of the FP32 pair layout (dg = ks s (f - w rho_ref)) in FP32
// arithmetic on the deviations: n = rho_ref + sum dg / s, j = sum v dg / s (the reference
// state carries no momentum), and T - 1 = (rho_ref |u|^2 + sum df |v - u|^2 - 2 dn) / (2 n),
// using sum_k w_k |v_k|^2 = 2 (T0 = 1); stored as FP64 for the feature kernel.
__global__ void lc_moments_kernel(const float2 *f, const Layout L, const VelD c, double rho_ref,
                                  const double *sin_t, double ks, float *dev)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const float inv_s = (float)(1.0 / (ks * sin_t[i]));
    float2 g[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = f[L.at(q, i, j)];
    float dn = 0.0f, jt = 0.0f, jp = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int gq = q >> 2, b = q & 3;
        const float va0 = (float)c.v[2 * gq], va1 = (float)c.v[2 * gq + 1], vb = (float)c.v[b];
        dn += g[q].x + g[q].y;
        jt += va0 * g[q].x + va1 * g[q].y;
        jp += vb * (g[q].x + g[q].y);
    }
    dn *= inv_s;
    const float n = (float)rho_ref + dn;
    const float ut = jt * inv_s / n, up = jp * inv_s / n;
    float e = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int gq = q >> 2, b = q & 3;
        const float va0 = (float)c.v[2 * gq] - ut, va1 = (float)c.v[2 * gq + 1] - ut, vb = (float)c.v[b] - up;
        e += g[q].x * (va0 * va0 + vb * vb) + g[q].y * (va1 * va1 + vb * vb);
    }
    e *= inv_s;
    const float tm1 = ((float)rho_ref * (ut * ut + up * up) + e - 2.0f * dn) / (2.0f * n);
    const size_t HW = (size_t)L.nt * L.np, cell = (size_t)i * L.np + j;
    dev[cell] = (float)(rho_ref - 1.0) + dn;   // rho - 1 at the resolution of the deviation
    dev[HW + cell] = ut;
    dev[2 * HW + cell] = up;
    dev[3 * HW + cell] = tm1;
}

// f += feq(rho + drho - mean, u + du) - feq(rho, u) on the FP32 pair layout, the equilibrium
// difference written in differences (FP32 keeps the relative precision of a small correction):
// with P(xi, u^2) = 1 + xi + (xi^2 - u^2)/2 + xi (xi^2 - 3 u^2)/6 (Eq. feq_Q=4 over n w),
// feq' - feq = w [ (rho' - rho) P' + rho (P' - P) ] and P' - P expanded in dxi = v . du and
// d(u^2) = du . (2u + du).
// FP32 velocities and weights of D2Q16 (each weight the FP64 product rounded once)
struct VelN { float v[4], w[16]; };

// the nudge of cell (i, j) by the correction (drho, dut, dup), its stored populations and images
__device__ __forceinline__ void nudge_cell(float2 *f, const Layout &L, const float *dev, int i, int j, float drho,
                                           float dut, float dup, const VelN &c, float s)
{
    const size_t n = (size_t)L.nt * L.np, cell = (size_t)i * L.np + j;
    const float rho = 1.0f + dev[cell], ut = dev[n + cell], up = dev[2 * n + cell];
    const float ut2 = ut + dut, up2 = up + dup;
    const float usq = ut * ut + up * up, usq2 = ut2 * ut2 + up2 * up2;
    const float dusq = dut * (ut + ut2) + dup * (up + up2);
    // the cell's eight pairs are read before any is written (the stores may alias the loads, so
    // the loads would otherwise wait for one another)
    float2 g8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) g8[q] = f[L.at(q, i, j)];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int g = q >> 2, b = q & 3;
        float2 v = g8[q];
        float d[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int a = 2 * g + m;
            const float va = c.v[a], vb = c.v[b], w = c.w[4 * a + b];
            const float xi = va * ut + vb * up, dxi = va * dut + vb * dup, xi2 = xi + dxi;
            const float P2 = 1.0f + xi2 + 0.5f * (xi2 * xi2 - usq2) + xi2 * (xi2 * xi2 - 3.0f * usq2) / 6.0f;
            const float dP = dxi + 0.5f * (dxi * (xi + xi2) - dusq) +
                             (dxi * (xi2 * xi2 + xi2 * xi + xi * xi) - 3.0f * (dxi * usq2 + xi * dusq)) / 6.0f;
            d[m] = w * (drho * P2 + rho * dP);
        }
        v.x += s * d[0];
        v.y += s * d[1];
        store_images(f, L, 4, q, i, j, v);   // the cell and its ghost images
    }
}

__global__ void nudge_kernel(float2 *f, const Layout L, const float *dev, const double *delta, const double *mean,
                             double wsum, const VelN c, const double *sin_t, double ks)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const size_t n = (size_t)L.nt * L.np, cell = (size_t)i * L.np + j;
    const float drho = (float)(delta[cell] - (*mean) / wsum), dut = (float)delta[n + cell],
                dup = (float)delta[2 * n + cell];
    nudge_cell(f, L, dev, i, j, drho, dut, dup, c, (float)(ks * sin_t[i]));
}

// The direct form's nudge straight from the net output Y [H][W][CO] (scaled by sc) and the last
// convolution's nparts partial sums of sin(theta) Y_0: each block reduces the partials to the area
// mean of drho itself, so neither an outputs pass nor a separate reduction runs.
__global__ void nudge_direct_kernel(float2 *f, const Layout L, const float *dev, const float *Y, int CO, float3 sc,
                                    const double *part0, int nparts, double wsum, const VelN c,
                                    const double *sin_t, double ks)
{
    __shared__ double red[128];
    double t = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) t += part0[b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int k = 64; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double mean = red[0] * (double)sc.x / wsum;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const size_t cell = (size_t)i * L.np + j;
    const float drho = (float)((double)Y[cell * CO] * (double)sc.x - mean);
    const float dut = (float)((double)Y[cell * CO + 1] * (double)sc.y);
    const float dup = (float)((double)Y[cell * CO + 2] * (double)sc.z);
    nudge_cell(f, L, dev, i, j, drho, dut, dup, c, (float)(ks * sin_t[i]));
}

template <int CI, int CO>
void conv_launch(const __nv_bfloat16 *Xp, int Hp, int Wp, const __nv_bfloat16 *Wt, const float *bias, float *Yf,
                 __nv_bfloat16 *Yb, __nv_bfloat16 *Ypad, int relu, cudaStream_t s, double *part0 = nullptr,
                 const double *sin_t = nullptr)
{
    dim3 grid((Wp - 2 + CONV_PIX - 1) / CONV_PIX, Hp - 2);
    conv3x3_kernel<CI, CO><<<grid, 128, 0, s>>>(Xp, Hp, Wp, Wt, bias, Yf, Yb, Ypad, relu, part0, sin_t);
}

template <int CI, int CO>
void wgrad_launch(const __nv_bfloat16 *dY, const __nv_bfloat16 *Xp, int H, int W, float *part, float *partb,
                  cudaStream_t s)
{
    wgrad_kernel<CI, CO><<<H, 128, 0, s>>>(dY, Xp, H, W, part, partb);
}

}  // namespace

// ---- the network ----------------------------------------------------------------------
// Layer l: CI_l -> CO_l; padded channel counts: input 16 (4 used), hidden 32, output 8 (3 used).
void lc_conv(int layer, const __nv_bfloat16 *Xp, int Hp, int Wp, const __nv_bfloat16 *Wt, const float *bias,
             float *Yf, __nv_bfloat16 *Yb, __nv_bfloat16 *Ypad, int relu, cudaStream_t s, double *part0,
             const double *sin_t)
{
    if (layer == 0) conv_launch<LC_CIN, LC_HID>(Xp, Hp, Wp, Wt, bias, Yf, Yb, Ypad, relu, s);
    else if (layer < LC_LAYERS - 1) conv_launch<LC_HID, LC_HID>(Xp, Hp, Wp, Wt, bias, Yf, Yb, Ypad, relu, s);
    else conv_launch<LC_HID, LC_COUT>(Xp, Hp, Wp, Wt, bias, Yf, Yb, Ypad, relu, s, part0, sin_t);
}

int lc_conv_ctas(int H, int W) { return ((W + CONV_PIX - 1) / CONV_PIX) * H; }

// backward-data convolution of layer l >= 1: input dP [H+4][W+4][COp2], output dXp [H+2][W+2][CI_l]
void lc_conv_bwd(int layer, const __nv_bfloat16 *dP, int H, int W, const __nv_bfloat16 *Wb, float *dXp, cudaStream_t s)
{
    if (layer < LC_LAYERS - 1) conv_launch<LC_HID, LC_HID>(dP, H + 4, W + 4, Wb, nullptr, dXp, nullptr, nullptr, 0, s);
    else conv_launch<LC_COUTP2, LC_HID>(dP, H + 4, W + 4, Wb, nullptr, dXp, nullptr, nullptr, 0, s);
}

void lc_wgrad(int layer, const __nv_bfloat16 *dPre, const __nv_bfloat16 *Xp, int H, int W, float *part, float *partb,
              cudaStream_t s)
{
    if (layer == 0) wgrad_launch<LC_CIN, LC_HID>(dPre, Xp, H, W, part, partb, s);
    else if (layer < LC_LAYERS - 1) wgrad_launch<LC_HID, LC_HID>(dPre, Xp, H, W, part, partb, s);
    else wgrad_launch<LC_HID, LC_COUTP2>(dPre, Xp, H, W, part, partb, s);
}

void lc_unpad(const float *dXp, int H, int W, int C, unsigned negmask, float *dX, cudaStream_t s)
{
    unpad_kernel<<<dim3(W, H), C, 0, s>>>(dXp, H, W, C, negmask, dX);
}

void lc_grad_pad2(const float *dY, const __nv_bfloat16 *act, int H, int W, int C, int CP, __nv_bfloat16 *dP,
                  cudaStream_t s)
{
    grad_pad2_kernel<<<dim3(W + 4, H + 4), CP, 0, s>>>(dY, act, H, W, C, CP, dP);
}

void lc_grad_pre(const float *dY, const __nv_bfloat16 *act, int n, int C, int CP, __nv_bfloat16 *dPre, cudaStream_t s)
{
    grad_pre_kernel<<<(n * CP + 255) / 256, 256, 0, s>>>(dY, act, n, C, CP, dPre);
}

void lc_reduce_rows(const float *part, int rows, int n, float *out, cudaStream_t s)
{
    reduce_rows_kernel<<<(n + 255) / 256, 256, 0, s>>>(part, rows, n, out);
}

void lc_loss(const float *Y, int CO, const double *target, const double *sin_t, int H, int W, float3 inv_scale,
             double wsum, float *dY, double *part, double *loss, cudaStream_t s)
{
    const int nb = (H * W + 255) / 256;
    loss_kernel<<<nb, 256, 0, s>>>(Y, CO, target, sin_t, H, W, inv_scale, wsum, dY, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nb, loss);
}

void lc_stream_loss(const float *Y, int CO, const double *target, const double *sin_t, const LcStream &g,
                    double inv_s1, double inv_s2, double wsum, double *gv, float *dY, double *part, double *loss,
                    cudaStream_t s)
{
    const int nb = (g.H * g.W + 255) / 256;
    stream_loss_kernel<float><<<nb, 256, 0, s>>>(Y, CO, target, sin_t, g, inv_s1, inv_s2, wsum, gv, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nb, loss);
    stream_adjoint_kernel<float><<<nb, 256, 0, s>>>(gv, CO, g, sin_t, dY);
}

void lc_stream_outputs(const float *Y, int CO, const LcStream &g, const double *sin_t, double *out, double *part,
                       double *mean, cudaStream_t s)
{
    const int nb = (g.H * g.W + 255) / 256;
    stream_outputs_kernel<float><<<nb, 256, 0, s>>>(Y, CO, g, sin_t, out, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nb, mean);
}

// dynamic shared memory of the mode solve for H rows
static size_t tri_smem(int H) { return sizeof(float2) * ((H + 1) / 2 + (size_t)TRI_WARPS * 2 * H); }

// psi [H][W] solving L psi = x / s^inv_sin - (area mean) (x [H][W]); part holds the nb per-block
// partial sums of the area mean's numerator (sum s x, or sum x for the adjoint's right side)
static void poisson(const double *x, int inv_sin, int nb, double *psi, const LcPoisson &P, const double *sin_t,
                    cudaStream_t s)
{
    const int M = P.W / 2 + 1;
    dft_rows_kernel<<<P.H, 256, P.W * sizeof(float), s>>>(x, P.H, P.W, sin_t, inv_sin, P.part, nb, P.wsum,
                                                          P.R * P.R, P.tw, P.X);
    tri_solve_kernel<<<(M + TRI_WARPS - 1) / TRI_WARPS, TRI_WARPS * 32, tri_smem(P.H), s>>>(P.X, P.H, M, P.tab, P.a);
    idft_rows_kernel<<<P.H, 256, M * sizeof(float2), s>>>(P.X, P.H, P.W, P.tw, psi);
}

void lc_vort_loss(const float *Y, int CO, const double *target, const double *sin_t, const LcStream &g,
                  const LcPoisson &P, double inv_s1, double inv_s2, double wsum, double *gv, float *dY, double *part,
                  double *loss, cudaStream_t s)
{
    const int n = g.H * g.W, nb = (n + 255) / 256;
    const LcStream g1{g.H, g.W, 1.0, g.R, g.dth, g.dph};
    vort_in_kernel<<<nb, 256, 0, s>>>(Y, CO, n, g.W, g.s0, sin_t, P.w, P.part);
    poisson(P.w, 0, nb, P.psi, P, sin_t, s);
    stream_loss_kernel<double><<<nb, 256, 0, s>>>(P.psi, 1, target, sin_t, g1, inv_s1, inv_s2, wsum, gv, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nb, loss);
    // backward: the curl's adjoint, the solve's adjoint S P S^-1 and the mean removal's
    stream_adjoint_kernel<double><<<nb, 256, 0, s>>>(gv, 1, g1, sin_t, P.w);
    cell_sums_kernel<<<nb, 256, 0, s>>>(P.w, n, P.W, sin_t, 0, P.part);
    poisson(P.w, 1, nb, P.psi, P, sin_t, s);
    cell_sums_kernel<<<nb, 256, 0, s>>>(P.psi, n, P.W, sin_t, 1, P.part);
    sum_kernel<<<1, 256, 0, s>>>(P.part, nb, P.sum);
    vort_grad_kernel<<<nb, 256, 0, s>>>(P.psi, g.H, g.W, CO, sin_t, P.sum, P.wsum, g.s0, dY);
}

void lc_vort_outputs(const float *Y, int CO, const LcStream &g, const LcPoisson &P, const double *sin_t, double *out,
                     double *part, double *mean, cudaStream_t s)
{
    const int n = g.H * g.W, nb = (n + 255) / 256;
    const LcStream g1{g.H, g.W, 1.0, g.R, g.dth, g.dph};
    vort_in_kernel<<<nb, 256, 0, s>>>(Y, CO, n, g.W, g.s0, sin_t, P.w, P.part);
    poisson(P.w, 0, nb, P.psi, P, sin_t, s);
    stream_outputs_kernel<double><<<nb, 256, 0, s>>>(P.psi, 1, g1, sin_t, out, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nb, mean);
}

int lc_poisson_prepare(int H)
{
    const size_t b = tri_smem(H);
    if (b <= 48 * 1024) return 0;
    return cudaFuncSetAttribute(tri_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) == cudaSuccess
               ? 0
               : -1;
}

size_t lc_poisson_table_floats(int H, int W)
{
    const size_t M = (size_t)W / 2 + 1;
    return 2 * M * H + H + (H & 1) + 4 * (size_t)W;   // tab (float2), a (padded to even), tw (float2 [2W])
}

int lc_poisson_tables(int H, int W, float *dev)
{
    const int M = W / 2 + 1;
    const double dth = M_PI / H, dph = 2.0 * M_PI / W;
    std::vector<double> sc(H), sf(H + 1), av(H);
    for (int i = 0; i < H; ++i) sc[i] = std::sin((i + 0.5) * dth);
    for (int i = 0; i <= H; ++i) sf[i] = (i == 0 || i == H) ? 0.0 : std::sin(i * dth);
    for (int i = 0; i < H; ++i) av[i] = sf[i] / (sc[i] * dth * dth);
    std::vector<float> h(lc_poisson_table_floats(H, W));
    float *tab = h.data(), *a = tab + 2 * (size_t)M * H, *tw = a + H + (H & 1);   // tw 8-byte aligned
    for (int i = 0; i < H; ++i) {   // mode 0: the integration's factors
        tab[2 * i] = (float)(dth * dth * sc[i]);
        tab[2 * i + 1] = i + 1 < H ? (float)(1.0 / sf[i + 1]) : 0.0f;
    }
    for (int m = 1; m < M; ++m) {
        const double sm = 2.0 * std::sin(0.5 * m * dph) / dph, lam = sm * sm;
        double cprev = 0.0;
        for (int i = 0; i < H; ++i) {
            const double ai = av[i], ci = sf[i + 1] / (sc[i] * dth * dth);
            const double bi = -(ai + ci) - lam / (sc[i] * sc[i]);
            const double r = 1.0 / (bi - ai * cprev);
            const double cp = ci * r;
            tab[2 * ((size_t)m * H + i)] = (float)cp;
            tab[2 * ((size_t)m * H + i) + 1] = (float)r;
            cprev = cp;
        }
    }
    for (int i = 0; i < H; ++i) a[i] = (float)av[i];
    for (int k = 0; k < 2 * W; ++k) {
        tw[2 * k] = (float)std::cos(M_PI * k / W);
        tw[2 * k + 1] = (float)std::sin(M_PI * k / W);
    }
    return cudaMemcpy(dev, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) == cudaSuccess ? 0 : -1;
}

void lc_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps, float c1,
             float c2, cudaStream_t s)
{
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

void lc_weights_bf16(const float *w, int CO, int CI, int COp, int CIp, __nv_bfloat16 *fwd, int CIp2, int COp2,
                     __nv_bfloat16 *bwd, cudaStream_t s)
{
    const int n = max(COp * 9 * CIp, CIp2 * 9 * COp2);
    weights_bf16_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, CO, CI, COp, CIp, fwd, CIp2, COp2, bwd);
}

void lc_wgrad_layout(const float *g9, int CO, int CI, int COp, int CIp, float *g, cudaStream_t s)
{
    const int n = CO * CI * 9;
    wgrad_layout_kernel<<<(n + 255) / 256, 256, 0, s>>>(g9, CO, CI, COp, CIp, g);
}

void lc_features(const float *dev, int H, int W, const double *sin_t, const double *cos_t,
                 const LcInScale &inv_scale, __nv_bfloat16 *Xp, cudaStream_t s)
{
    features_kernel<<<(H * W + 255) / 256, 256, 0, s>>>(dev, H, W, sin_t, cos_t, inv_scale, Xp);
}

void lc_dev_of_moments(const double *in4, int H, int W, float *dev, cudaStream_t s)
{
    dev_of_moments_kernel<<<(H * W + 255) / 256, 256, 0, s>>>(in4, H * W, dev);
}

void lc_outputs(const float *Y, int CO, int H, int W, float3 scale, const double *sin_t, double *out, double *part,
                double *mean, cudaStream_t s)
{
    const int nb = (H * W + 255) / 256;
    outputs_kernel<<<nb, 256, 0, s>>>(Y, CO, H, W, scale, sin_t, out, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nb, mean);
}

void lc_moments(const float2 *f, const Layout &L, const VelD &c, double rho_ref, const double *sin_t, double ks,
                float *dev, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt);
    lc_moments_kernel<<<grid, 128, 0, s>>>(f, L, c, rho_ref, sin_t, ks, dev);
}

void lc_nudge(float2 *f, const Layout &L, const float *dev, const double *delta, const double *mean, double wsum,
              const VelD &c, const double *sin_t, double ks, cudaStream_t s)
{
    VelN cn;
    for (int a = 0; a < 4; ++a) cn.v[a] = (float)c.v[a];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) cn.w[4 * a + b] = (float)(c.w[a] * c.w[b]);
    dim3 grid((L.np + 127) / 128, L.nt);
    nudge_kernel<<<grid, 128, 0, s>>>(f, L, dev, delta, mean, wsum, cn, sin_t, ks);
}

void lc_nudge_direct(float2 *f, const Layout &L, const float *dev, const float *Y, int CO, float3 scale,
                     const double *part0, int nparts, double wsum, const VelD &c, const double *sin_t, double ks,
                     cudaStream_t s)
{
    VelN cn;
    for (int a = 0; a < 4; ++a) cn.v[a] = (float)c.v[a];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) cn.w[4 * a + b] = (float)(c.w[a] * c.w[b]);
    dim3 grid((L.np + 127) / 128, L.nt);
    nudge_direct_kernel<<<grid, 128, 0, s>>>(f, L, dev, Y, CO, scale, part0, nparts, wsum, cn, sin_t, ks);
}

}  // namespace vk
