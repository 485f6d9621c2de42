// f32_images.cuh -- the ghost images of one cell of an FP32 pair-plane array (3 ghost rows per
// pole, GC ghost columns per side; Eqs. bcs_phi, bcs_theta): device helpers shared by the stage
// kernels and by the learned correction's nudge, so that every kernel that writes an interior
// cell also writes its images and no separate ghost-fill pass is needed.
#pragma once

#include "vlbm_internal.h"

namespace vk {

// Writes v at pair-plane cell (p, i, j) and at its ghost images.
__device__ __forceinline__ void put_cols(float2 *f, const Layout &L, int p, int r, int c, float2 v)
{
    f[L.at(p, r, c)] = v;
    for (int m = 1; c - m * L.np >= -GC; ++m) f[L.at(p, r, c - m * L.np)] = v;
    for (int m = 1; c + m * L.np < L.np + GC; ++m) f[L.at(p, r, c + m * L.np)] = v;
}

// One member (slot s = 2 p + m) of a pair-plane cell and its periodic images.
__device__ __forceinline__ void put_cols_slot(float2 *f, const Layout &L, int s, int r, int c, float v)
{
    float *base = reinterpret_cast<float *>(f) + (s & 1);
    base[2 * L.at(s >> 1, r, c)] = v;
    for (int m = 1; c - m * L.np >= -GC; ++m) base[2 * L.at(s >> 1, r, c - m * L.np)] = v;
    for (int m = 1; c + m * L.np < L.np + GC; ++m) base[2 * L.at(s >> 1, r, c + m * L.np)] = v;
}

__device__ __forceinline__ int image_pair(int p) { return 4 * (1 - (p >> 2)) + (3 - (p & 3)); }

// The pole image of pair p's value v (cell in row i, column j) beyond the pole: -v of the mirrored
// populations at column j + n_phi/2 of the mirrored ghost row.  D2Q16 maps a pair onto a pair with
// its members swapped; in general each member goes to the slot of its own image.
__device__ __forceinline__ void store_pole_image(float2 *f, const Layout &L, int q, int p, int i, int j, float2 v)
{
    int jj = j + L.np / 2;
    if (jj >= L.np) jj -= L.np;
    const int r = (i < GR) ? (-1 - i) : (2 * L.nt - 1 - i);
    if (q == 4) {
        put_cols(f, L, image_pair(p), r, jj, make_float2(-v.y, -v.x));
    } else {
        put_cols_slot(f, L, f32_image_slot(q, 2 * p), r, jj, -v.x);
        put_cols_slot(f, L, f32_image_slot(q, 2 * p + 1), r, jj, -v.y);
    }
}

__device__ __forceinline__ void store_images(float2 *f, const Layout &L, int q, int p, int i, int j, float2 v)
{
    put_cols(f, L, p, i, j, v);
    if (i < GR || i >= L.nt - GR) store_pole_image(f, L, q, p, i, j, v);
}

}  // namespace vk
