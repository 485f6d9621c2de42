// stage_f32.cu -- FP32 deviation-storage RK3 stage, the throughput path.
//
// Computes one SSP-RK3 stage (arXiv 2504.15574 Sec. 3.7) of the vLBM operator
// L[f] (Eq. Lf) for a tile of TY x TX cells and all 16 populations:
//   1. one TMA box brings the stage input (16 planes x (TY+6) x (TX+8), ghost
//      rows and columns included by the storage layout) into shared memory;
//   2. the phi-face WENO-5 fluxes (Eqs. fluxes_W5, WENO5_delta, WENO5_sigma)
//      of all 16 populations are computed once per face into shared memory;
//   3. the tile is scaled in place by sin(theta) (the theta flux is a
//      finite-difference WENO on g = sin(theta) f, Eq. discrete_advection_sphere)
//      and the theta-face fluxes are computed once per face;
//   4. each thread takes one cell: moments (Eq. f_moments_sum), equilibrium
//      (Eq. feq_Q=4), BGK (Sec. 3.2), force through K^H / Ktilde^H (Eq. df),
//      flux differences, and the stage combination; the result is written to
//      the cell and to its ghost images.
//
// Storage is the deviation delta f = f - w_k rho_ref.  The reference state
// w_k rho_ref is uniform in phi, so the phi fluxes of f and delta f differ by a
// constant that cancels in the flux difference.  In theta, the WENO weights are
// those of the full g = sin(theta) (w_k rho_ref + delta f): every linear form of
// the stencil is the delta-f part plus w_k rho_ref times the same form of
// sin(theta), precomputed in FP64 per face.  The reconstruction is written as
//   ghat = P2 + wbar1 (P1 - P2) + wbar3 (P3 - P2),
// whose reference part splits into the ideal-weight interpolant of sin(theta)
// (its flux difference, and the force of the reference state, are folded into
// the FP64-derived per-row tendency rref) and a correction proportional to the
// deviation of the weights from the ideal ones.  The result equals the method
// on f up to FP32 rounding of deviation-sized quantities.
#include "vlbm_internal.h"

namespace vk {

namespace {

constexpr int TY = F32_TILE_ROWS;
constexpr int TX = F32_TILE_COLS;
constexpr int SR = TY + 2 * GR;     // shared-memory rows of the tile
constexpr int SC = TX + 2 * GC;     // shared-memory columns of the tile
constexpr int NT = TY * TX;         // threads per CTA, one cell each in the cell phase
constexpr int NFT = NK * (TY + 1) * TX;
constexpr int NFP = NK * TY * (TX + 1);
constexpr unsigned TILE_BYTES = NK * SR * SC * sizeof(float);

struct __align__(128) Smem {
    float tile[NK][SR][SC];
    float ft[NK][TY + 1][TX];
    float fp[NK][TY][TX + 1];
    unsigned long long bar;
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Waits on phase 0 of an mbarrier for at most limit_ns; returns false on timeout.
__device__ __forceinline__ bool wait_tile(unsigned long long *bar, unsigned long long limit_ns)
{
    unsigned done = 0;
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        asm volatile(
            "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0; selp.u32 %0, 1, 0, P; }"
            : "=r"(done)
            : "r"(smem_u32(bar))
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0u) {
            const unsigned long long t = globaltimer_ns();
            if (it == 0u) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Weighted WENO-5 combination from the stencil's linear forms.
//   a..e upwind-ordered values; A_i, B_i the smoothness forms, p2 the central
//   candidate.  Returns p2 + wbar1 (A1 - A2)/3 + wbar3 (A2 - A3)/6 and the
//   normalised weights wbar1, wbar3.
__device__ __forceinline__ float weno_combine(float p2, float A1, float B1, float A2, float B2, float A3,
                                              float B3, float eps, float &w1n, float &w3n)
{
    const float c13 = 13.0f / 12.0f;
    float s1 = fmaf(A1 * c13, A1, fmaf(B1 * 0.25f, B1, eps));
    float s2 = fmaf(A2 * c13, A2, fmaf(B2 * 0.25f, B2, eps));
    float s3 = fmaf(A3 * c13, A3, fmaf(B3 * 0.25f, B3, eps));
    float q1 = s1 * s1, q2 = s2 * s2, q3 = s3 * s3;
    float t1 = 0.1f * (q2 * q3);   // delta_1 / q1 scaled by q1 q2 q3
    float t2 = 0.6f * (q1 * q3);
    float t3 = 0.3f * (q1 * q2);
    float r = rcp_approx(t1 + t2 + t3);
    w1n = t1 * r;
    w3n = t3 * r;
    return fmaf(w1n, (A1 - A2) * (1.0f / 3.0f), fmaf(w3n, (A2 - A3) * (1.0f / 6.0f), p2));
}

// Linear forms of an upwind-ordered stencil.
struct Forms { float p2, A1, B1, A2, B2, A3, B3; };
__device__ __forceinline__ Forms forms(float a, float b, float c, float d, float e)
{
    Forms F;
    F.A1 = fmaf(-2.0f, b, a) + c;
    F.B1 = fmaf(3.0f, c, fmaf(-4.0f, b, a));
    F.A2 = fmaf(-2.0f, c, b) + d;
    F.B2 = b - d;
    F.A3 = fmaf(-2.0f, d, c) + e;
    F.B3 = fmaf(3.0f, c, fmaf(-4.0f, d, e));
    // p2 = (-b + 5c + 2d)/6
    F.p2 = fmaf(5.0f / 6.0f, c, fmaf(1.0f / 3.0f, d, b * (-1.0f / 6.0f)));
    return F;
}

__device__ __forceinline__ void store_images(float *f, const Layout &L, int k, int i, int j, float v)
{
    const int np = L.np;
    auto put_row = [&](int kk, int r, int c) {
        f[L.at(kk, r, c)] = v;
        for (int m = 1; c - m * np >= -GC; ++m) f[L.at(kk, r, c - m * np)] = v;
        for (int m = 1; c + m * np < np + GC; ++m) f[L.at(kk, r, c + m * np)] = v;
    };
    put_row(k, i, j);
    if (i < GR || i >= L.nt - GR) {
        int jj = j + np / 2;
        if (jj >= np) jj -= np;
        int r = (i < GR) ? (-1 - i) : (2 * L.nt - 1 - i);
        put_row(NK - 1 - k, r, jj);
    }
}

__global__ void __launch_bounds__(NT, 3) stage_f32_kernel(const __grid_constant__ CUtensorMap tm, const StageF p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int q0 = blockIdx.x * TX;
    const int i0 = blockIdx.y * TY;
    const Layout L = p.L;

    // ---- 1. TMA load of the tile (rows i0-3 .. i0+TY+2, columns q0-4 .. q0+TX+3)
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.bar)),
                     "r"(TILE_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(&S.tile[0][0][0])),
            "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(q0), "r"(i0), "r"(0), "r"(smem_u32(&S.bar))
            : "memory");
    }
    __syncthreads();
    if (!wait_tile(&S.bar, 1000000000ull)) {
        // the copy did not complete within 1 s: flag it, give the copy one more
        // bounded second to land in this CTA's shared memory, then leave
        if (tid == 0) atomicOr(p.err, 1u);
        wait_tile(&S.bar, 1000000000ull);
        return;
    }

    // ---- 2. phi faces: face fx lies between tile columns fx-1 and fx (fx = 0..TX)
    const float eps = p.eps;
    for (int e = tid; e < NFP; e += NT) {
        const int k = e / (TY * (TX + 1));
        const int rem = e - k * (TY * (TX + 1));
        const int fy = rem / (TX + 1);
        const int fx = rem - fy * (TX + 1);
        const float vb = p.c.v[k & 3];
        const float *row = &S.tile[k][fy + GR][0];
        // v > 0: columns fx-3 .. fx+1 ; v < 0: columns fx+2 .. fx-2 (smem column = column + GC)
        const int base = (vb > 0.0f) ? (fx + GC - 3) : (fx + GC + 2);
        const int st = (vb > 0.0f) ? 1 : -1;
        Forms F = forms(row[base], row[base + st], row[base + 2 * st], row[base + 3 * st], row[base + 4 * st]);
        float w1, w3;
        const float gh = weno_combine(F.p2, F.A1, F.B1, F.A2, F.B2, F.A3, F.B3, eps, w1, w3);
        S.fp[k][fy][fx] = vb * gh;
    }

    // own-cell deviations, read before the tile is rescaled
    const int cy = tid / TX, cx = tid - (tid / TX) * TX;
    float df[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) df[k] = S.tile[k][cy + GR][cx + GC];
    __syncthreads();

    // ---- 3. g = sin(theta) delta f in place, then theta faces
    for (int e = tid; e < NK * SR * (SC / 4); e += NT) {
        const int r = (e / (SC / 4)) % SR;
        const float s = p.sin_ext[i0 + r];
        float4 *q = reinterpret_cast<float4 *>(&S.tile[0][0][0]) + e;
        float4 x = *q;
        x.x *= s; x.y *= s; x.z *= s; x.w *= s;
        *q = x;
    }
    __syncthreads();
    for (int e = tid; e < NFT; e += NT) {
        const int k = e / ((TY + 1) * TX);
        const int rem = e - k * ((TY + 1) * TX);
        const int fy = rem / TX;
        const int fx = rem - fy * TX;
        const float va = p.c.v[k >> 2];
        const int dir = (va > 0.0f) ? 0 : 1;
        // v > 0: rows fy-3 .. fy+1 ; v < 0: rows fy+2 .. fy-2 (smem row = row + GR)
        const int base = (dir == 0) ? (fy + GR - 3) : (fy + GR + 2);
        const int st = (dir == 0) ? 1 : -1;
        const float *col = &S.tile[k][0][fx + GC];
        Forms F = forms(col[base * SC], col[(base + st) * SC], col[(base + 2 * st) * SC],
                        col[(base + 3 * st) * SC], col[(base + 4 * st) * SC]);
        int fi = i0 + fy;
        if (fi > L.nt) fi = L.nt;
        const FaceConst fc = p.face[2 * fi + dir];
        const float wr = p.c.wr[k];
        float w1, w3;
        const float gh = weno_combine(F.p2, fmaf(wr, fc.sa1, F.A1), fmaf(wr, fc.sb1, F.B1),
                                      fmaf(wr, fc.sa2, F.A2), fmaf(wr, fc.sb2, F.B2), fmaf(wr, fc.sa3, F.A3),
                                      fmaf(wr, fc.sb3, F.B3), eps, w1, w3);
        // the reference part of P2 is the ideal-weight interpolant minus corr
        S.ft[k][fy][fx] = va * fmaf(-wr, fc.corr, gh);
    }
    __syncthreads();

    // ---- 4. one cell per thread
    const int i = i0 + cy, j = q0 + cx;
    if (i >= L.nt || j >= L.np) return;
    float dn = 0.0f, jt = 0.0f, jp = 0.0f;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        dn += df[k];
        jt = fmaf(df[k], p.c.v[k >> 2], jt);
        jp = fmaf(df[k], p.c.v[k & 3], jp);
    }
    const float n = p.c.rho_ref + dn;
    const float ninv = 1.0f / n;
    const float ut = jt * ninv, up = jp * ninv;
    const float u2 = fmaf(ut, ut, up * up);
    const RowConst rc = p.row[i];
    const float *rr = p.rref + (size_t)i * NK;

#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int a = k >> 2, b = k & 3;
        const float va = p.c.v[a], vb = p.c.v[b];
        const float wk = p.c.w[a] * p.c.w[b];
        const float xi = fmaf(va, ut, vb * up);
        const float poly = xi + 0.5f * fmaf(xi, xi, -u2) + xi * fmaf(xi, xi, -3.0f * u2) * (1.0f / 6.0f);
        const float dfeq = wk * fmaf(n, poly, dn);
        float kg = 0.0f, ktg = 0.0f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            kg = fmaf(p.c.K[a * 4 + m], df[4 * m + b], kg);
            ktg = fmaf(p.c.Kt[b * 4 + m], df[4 * a + m], ktg);
        }
        const float force = rc.cotR * fmaf(vb * vb, kg, -va * ktg);
        const float adv_t = (S.ft[k][cy][cx] - S.ft[k][cy + 1][cx]) * rc.inv_dth;
        const float adv_p = (S.fp[k][cy][cx] - S.fp[k][cy][cx + 1]) * rc.inv_dph;
        const float Lk = (adv_t + adv_p) - force - (df[k] - dfeq) * p.tau_inv + rr[k];
        float outv;
        if (p.stage == 1) {
            outv = fmaf(p.dt, Lk, df[k]);
        } else if (p.stage == 2) {
            const float f0 = p.fold[L.at(k, i, j)];
            outv = fmaf(0.25f * p.dt, Lk, fmaf(0.75f, f0, 0.25f * df[k]));
        } else {
            const float f0 = p.fold[L.at(k, i, j)];
            outv = fmaf((2.0f / 3.0f) * p.dt, Lk, fmaf(1.0f / 3.0f, f0, (2.0f / 3.0f) * df[k]));
        }
        store_images(p.out, L, k, i, j, outv);
    }
}

}  // namespace

size_t stage_f32_smem_bytes() { return sizeof(Smem) + 128; }

cudaError_t prepare_stage_f32()
{
    return cudaFuncSetAttribute(stage_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_f32_smem_bytes());
}

void launch_stage_f32(const CUtensorMap &tm_in, const StageF &p, cudaStream_t s)
{
    dim3 grid((p.L.np + TX - 1) / TX, (p.L.nt + TY - 1) / TY);
    stage_f32_kernel<<<grid, NT, stage_f32_smem_bytes(), s>>>(tm_in, p);
}

}  // namespace vk
