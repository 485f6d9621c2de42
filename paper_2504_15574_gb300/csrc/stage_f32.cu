// stage_f32.cu -- FP32 deviation-storage path (the throughput path).
//
// State.  The device array holds dg = k sin(theta) (f - w_k rho_ref) in FP32: the
// deviation from the reference state w_k rho_ref (rho_ref an FP64 constant),
// premultiplied by sin(theta) so that the stage input is directly the nodal
// variable of the theta flux (arXiv 2504.15574 Eq. discrete_advection_sphere, read
// as a finite-difference WENO on g = sin(theta) f), and by the run's state scale k,
// a power of two (exact) that puts the WENO regulariser 4 eps k^2 near 1.
// Populations are stored in
// pairs: pair p = 4 g + b holds populations (a = 2g, b) and (a = 2g + 1, b) as one
// float2, so that both members share the sign of v_theta and the value of v_phi
// and every per-population operation runs as one packed f32x2 instruction.
// Layout of vlbm_internal.h with 8 pair planes of float2 elements.  Pole ghost
// rows hold -dg of the mirrored pair with swapped members (the ghost's sine is
// negative, Eq. bcs_theta maps v -> -v); ghost columns hold periodic images.
// D2Q9 (App. A.1, template parameter Q = 3) runs through the same code in five pair
// planes: four pairs whose members share the sign of each nonzero velocity component
// and the rest population beside an always-zero slot (slot maps in vlbm_internal.h);
// its pole images go member by member to the slot of the mirrored population.
//
// One stage (Sec. 3.7) of L[f] (Eq. Lf) per kernel launch, for a tile of TY x TX
// cells and all populations (a launch may cover a subset of the tile rows):
//   1. one TMA box (all pair planes x (TY+6) x (TX+10) float2) into shared memory;
//   2. phi faces and theta faces of all pairs, each face once, into shared memory
//      (WENO-5, Eqs. fluxes_W5, WENO5_delta, WENO5_sigma).  On dg the phi weights
//      use the regulariser 4 eps s^2 k^2 (the WENO weights are invariant under
//      g -> s g with eps -> s^2 eps, and every smoothness term is evaluated as
//      4 k^2 (sigma + eps), a common factor of the ratios); the theta weights are
//      those of the full g = k sin(theta) w_k rho_ref + dg: each smoothness form is
//      the dg part plus k w_k rho_ref times the form of sin(theta) (FP64 table).  The
//      reconstruction is written P2 + wbar1 (P1 - P2) + wbar3 (P3 - P2); P2 of the
//      reference part is linear in sin(theta), so its flux difference is folded, with
//      the force of the reference state, into the FP64-derived tendency rref, and the
//      weight terms use the full forms.  Each phi face row is walked by a few threads
//      that keep the columns' differences in registers.  Face values carry the
//      stage's dt share and their metric factor;
//   3. per cell: moments (Eq. f_moments_sum), equilibrium (Eq. feq_Q=4, or feq_Q=3), BGK,
//      force through K^H / Ktilde^H (Eq. df), flux differences and the stage
//      combination, all on dg (the operator commutes with the row factor), then
//      the store of the cell and of its ghost images.
#include "vlbm_internal.h"
#include "f32_images.cuh"

#include <cstddef>
#include <cstring>
#include <algorithm>
#include <cmath>

namespace vk {

namespace {

constexpr int TX = F32_TILE_COLS;
constexpr int NP2 = 8;                 // population pairs of D2Q16
constexpr int SC = F32_BOX_COLS;       // tile columns in shared memory (TX + 2 GC + 2)

// Per-tile tables of one stage, for the tile's rows: the sine differences (FP64-derived) and the
// upwind schemes' 1/sin and interface sines at the padded tile rows, the per-row constants and the
// reference tendency times the stage's dt share of the cell rows.  The batch kernel fills them per
// thread from its run's arrays; the standalone solver keeps one per tile row and stage in device
// memory (built on the host with the same FP32 roundings) and copies it with the tile's box.
template <int TY, int NPP>
struct __align__(16) TabT {
    float2 ds2[TY + 2 * GR];    // (dsin, dsin) at the tile rows
    float2 d2s2[TY + 2 * GR];   // (d2sin, d2sin) at the tile rows
    float2 isp2[TY + 2 * GR];   // upwind schemes, Komissarov: (1/sin, 1/sin) at the tile rows
    float2 sf2[TY + 1];         // upwind schemes, Komissarov: interface sines of the face rows
    float2 rr[TY][NPP];         // dte s rref per cell row and pair
    RowF rowc[TY];
};

// The stage input's box of one tile: all pair planes x (TY + 6) rows x SC columns (a TMA
// destination: 128-byte aligned, and its size a multiple of 128 so that consecutive boxes are too)
template <int TY, int NPP>
struct __align__(128) BoxT {
    float2 v[NPP][TY + 2 * GR][SC];
};

// NPP pair planes: 8 for D2Q16, 5 for D2Q9.  NBUF box buffers and NTAB table buffers: one each for
// the one-tile CTAs; the persistent stage kernel alternates two table buffers.
template <int TY, int NPP = NP2, int NBUF = 1, int NTAB = NBUF>
struct __align__(128) SmemT {
    BoxT<TY, NPP> tile[NBUF];           // TMA destinations (must stay first)
    float2 adv[NPP][TY][TX + 1];        // per cell and pair: dte (flux differences + s rref); row
                                        // stride TX+1 keeps the phi walkers' stores conflict-free
    __align__(128) float2 ob[NPP][TY][TX];   // stages 2, 3: the tile of F (TMA load); then the output
                                             // tile staged for the TMA store (TMA wants 128-byte
                                             // aligned shared memory)
    // D2Q9 with 8 warps: the theta walkers' flux differences of the four flux pairs, written
    // beside adv by other warps than the phi walkers' (one element otherwise)
    float2 advT[NPP == 5 ? 4 : 1][NPP == 5 ? TY : 1][NPP == 5 ? TX + 1 : 1];
    TabT<TY, NPP> tab[NTAB];
    double polew[2][NPP];               // pole faces of the tile (north, south): per pair, v_theta-weighted
                                        // face values summed over the tile's columns
    RunF run;                           // batch kernel: this tile's run
    unsigned long long bar[NBUF];       // box (and tables; one-tile CTAs: also the tile of F)
    unsigned long long barF;            // persistent kernel: the tile of F
};

// TMA shared-memory operands start on 128-byte boundaries (the dynamic buffer itself is 128-aligned)
typedef SmemT<8> Smem8;
typedef SmemT<4> Smem4;
typedef SmemT<8, 5> Smem8q3;
typedef SmemT<4, 5> Smem4q3;
typedef SmemT<8, NP2, 1, 2> SmemQ8;
typedef SmemT<8, 5, 1, 2> SmemQ8q3;
static_assert(offsetof(Smem8, tile) == 0 && offsetof(Smem8, ob) % 128 == 0 && offsetof(Smem4, ob) % 128 == 0 &&
                  offsetof(Smem8q3, ob) % 128 == 0 && offsetof(Smem4q3, ob) % 128 == 0 &&
                  offsetof(SmemQ8, ob) % 128 == 0 && offsetof(SmemQ8q3, ob) % 128 == 0 &&
                  sizeof(BoxT<8, NP2>) % 128 == 0 && sizeof(BoxT<8, 5>) % 128 == 0,
              "TMA operands in shared memory must be 128-byte aligned");
static_assert(offsetof(SmemQ8, tab) % 16 == 0 && offsetof(SmemQ8q3, tab) % 16 == 0 &&
                  sizeof(TabT<8, NP2>) % 16 == 0 && sizeof(TabT<8, 5>) % 16 == 0,
              "bulk copies of the tile tables need 16-byte alignment and sizes");
// three CTAs of 8 tile rows per SM for D2Q16, four for D2Q9 (whose registers are capped at 64 to
// let four fit): 228 KB of shared memory per SM, 1 KB reserved per CTA
static_assert(3 * (sizeof(SmemT<8>) + 128 + 1024) <= 228 * 1024, "stage tile exceeds a third of an SM's shared memory");
static_assert(4 * (sizeof(SmemT<8, 5>) + 128 + 1024) <= 228 * 1024, "D2Q9 stage tile exceeds a quarter of an SM's shared memory");
// persistent stage kernel with one box buffer: three CTAs per SM
static_assert(3 * (sizeof(SmemQ8) + 128 + 1024) <= 228 * 1024 && 3 * (sizeof(SmemQ8q3) + 128 + 1024) <= 228 * 1024,
              "persistent single-buffer tiles");

typedef float2 f2;

__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    unsigned long long x = *reinterpret_cast<unsigned long long *>(&a), y = *reinterpret_cast<unsigned long long *>(&b), d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    return *reinterpret_cast<f2 *>(&d);
}
__device__ __forceinline__ f2 splat(float x) { return make_float2(x, x); }
__device__ __forceinline__ f2 swap2(f2 a) { return make_float2(a.y, a.x); }

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Waits for the mbarrier phase with the given parity for at most limit_ns; false on timeout.
// The phase is first tested without blocking; limit_ns = 0 gives up right there (a test of the
// timeout path), otherwise try_wait (which may suspend the thread for a while) is polled with the
// elapsed global time checked after every attempt.
__device__ __forceinline__ bool wait_phase(unsigned long long *bar, unsigned parity, unsigned long long limit_ns)
{
    unsigned done;
    asm volatile(
        "{ .reg .pred P; mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2; selp.u32 %0, 1, 0, P; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (limit_ns == 0) return false;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        asm volatile(
            "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2; selp.u32 %0, 1, 0, P; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// Upwind-scheme phi faces f0 .. f0 + NF - 1 of one row of one pair plane (Eq. fluxes_U1-3):
// face value l0 x_up2 + l1 x_up + l2 x_down with x_up2, x_up, x_down the shared columns
// fx+2, fx+3, fx+4 for DIR = +1 (v_phi > 0) and fx+5, fx+4, fx+3 for DIR = -1, read as
// 16-byte pairs from shared column f0 + 2.  The flux difference of cell f0 + j - 1 plus base
// goes to out[j-1] as for phi_march.
template <int NF, int DIR>
__device__ __forceinline__ void phi_march_lin(const f2 *row, int f0, f2 l0, f2 l1, f2 l2, f2 vb, f2 base, f2 *out)
{
    constexpr int NX = ((NF + 3) + 1) & ~1;
    const float4 *src = reinterpret_cast<const float4 *>(row + f0 + 2);
    f2 x[NX];
#pragma unroll
    for (int m = 0; m < NX / 2; ++m) {
        const float4 v = src[m];
        x[2 * m] = make_float2(v.x, v.y);
        x[2 * m + 1] = make_float2(v.z, v.w);
    }
    f2 prev;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const f2 v = (DIR > 0) ? fma2(l0, x[j], fma2(l1, x[j + 1], mul2(l2, x[j + 2])))
                               : fma2(l0, x[j + 3], fma2(l1, x[j + 2], mul2(l2, x[j + 1])));
        if (j > 0) out[j - 1] = fma2(vb, sub2(prev, v), base);
        prev = v;
    }
}

// Nonlinear combination of WENO-5 (Eqs. fluxes_W5, WENO5_delta, WENO5_sigma) on the
// scaled state: P2 + wbar1 (A1 - A2)/3 + wbar3 (A2 - A3)/6 with wbar_i = d_i q_j q_k / sum
// and q_i = t_i^2, where t_i = B_i^2 + 13/3 A_i^2 + E = 4 k^2 (sigma_i + eps) for the
// unscaled forms (sigma_i = 13/12 A_i^2 + 1/4 B_i^2).  The weights are ratios, so the
// common factor 4 k^2 cancels; the state scale k is chosen with E = 4 eps k^2 near 1,
// so t_i >= E sin^2(theta) keeps every q_i a normal FP32 number down to the pole rows.
// Numerator and denominator are divided by 0.1 q2 and multiplied by 3: with q1' = 1.5 q1,
//   correction = (q3 d12 + q1' d23) / (3 q3 + q1' (6 + 12 q3 / q2)),
// which needs no product of two q's; where q1' q3 / q2 overflows (q2 negligible beside
// q1 and q3) the reciprocal is 0 and the value is P2, the limit of the weights there.
__device__ __forceinline__ f2 weno_mix(f2 t1, f2 t2, f2 t3, f2 d12, f2 d23, f2 p2)
{
    const f2 q1 = mul2(t1, t1), q2 = mul2(t2, t2), q3 = mul2(t3, t3);
    const f2 q1p = mul2(q1, splat(1.5f));
    const f2 r2 = make_float2(rcp_approx(q2.x), rcp_approx(q2.y));
    const f2 w = fma2(mul2(q3, splat(12.0f)), r2, splat(6.0f));
    const f2 den = fma2(q1p, w, mul2(q3, splat(3.0f)));
    const f2 num = fma2(q3, d12, mul2(q1p, d23));
    const f2 r = make_float2(rcp_approx(den.x), rcp_approx(den.y));
    return fma2(num, r, p2);
}

// WENO-5 phi faces f0 .. f0 + NF - 1 of one row of one pair plane.  In upwind order a..e the
// stencil forms are built from the first differences d1..d4: A_i = d_{i+1} - d_i,
// B1 = A1 + 2 d2, |B2| = |d2 + d3|, B3 = A3 - 2 d3 and P2 = c + (d2 + 2 d3)/6.  The faces are
// walked in order so that
// every column's first difference d[m] = x[m] - x[m-1], second difference A[m] = d[m+1] - d[m]
// (centred at m) and row term Q[m] = 13/3 A[m]^2 + E are formed once, and so is each
// A difference (d23 of a face is d12 of the next).  DIR = +1 for v_phi > 0 (face fx reads
// shared columns fx+1 .. fx+5 in upwind order), -1 for v_phi < 0 (fx+6 .. fx+2).  The
// columns are read as 16-byte pairs starting at shared column f0 + LO (even).  The flux
// difference of cell f0 + j - 1, vb times (face j-1 - face j), plus base goes to out[j-1].
template <int NF, int DIR>
__device__ __forceinline__ void phi_march(const f2 *row, int f0, f2 E, f2 vb, f2 base, f2 *out)
{
    constexpr int LO = (DIR > 0) ? 0 : 2;
    constexpr int NX = ((NF + 5) + 1) & ~1;
    const f2 two = splat(2.0f), m2 = splat(-2.0f), c133 = splat(13.0f / 3.0f);
    const float4 *src = reinterpret_cast<const float4 *>(row + f0 + LO);
    f2 x[NX], d[NX], A[NX], Q[NX];
#pragma unroll
    for (int m = 0; m < NX / 2; ++m) {
        const float4 v = src[m];
        x[2 * m] = make_float2(v.x, v.y);
        x[2 * m + 1] = make_float2(v.z, v.w);
    }
    if constexpr (DIR > 0) {
        // face j: a..e = x[j+1..j+5]; A1..A3 = A[j+2..j+4], d2 = d[j+3], d3 = d[j+4], c = x[j+3]
#pragma unroll
        for (int m = 2; m <= 4; ++m) d[m] = sub2(x[m], x[m - 1]);
#pragma unroll
        for (int m = 2; m <= 3; ++m) {
            A[m] = sub2(d[m + 1], d[m]);
            Q[m] = fma2(mul2(A[m], c133), A[m], E);
        }
        f2 d12 = sub2(A[2], A[3]), prev;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            d[j + 5] = sub2(x[j + 5], x[j + 4]);
            A[j + 4] = sub2(d[j + 5], d[j + 4]);
            Q[j + 4] = fma2(mul2(A[j + 4], c133), A[j + 4], E);
            const f2 B1 = fma2(two, d[j + 3], A[j + 2]);
            const f2 B2 = add2(d[j + 3], d[j + 4]);
            const f2 B3 = fma2(m2, d[j + 4], A[j + 4]);
            const f2 p2 = fma2(splat(1.0f / 3.0f), d[j + 4], fma2(splat(1.0f / 6.0f), d[j + 3], x[j + 3]));
            const f2 d23 = sub2(A[j + 3], A[j + 4]);
            const f2 v = weno_mix(fma2(B1, B1, Q[j + 2]), fma2(B2, B2, Q[j + 3]), fma2(B3, B3, Q[j + 4]), d12, d23, p2);
            if (j > 0) out[j - 1] = fma2(vb, sub2(prev, v), base);
            prev = v;
            d12 = d23;
        }
    } else {
        // face j: a..e = x[j+4..j]; A1..A3 = A[j+3], A[j+2], A[j+1], d2 = -d[j+3], d3 = -d[j+2], c = x[j+2]
#pragma unroll
        for (int m = 1; m <= 3; ++m) d[m] = sub2(x[m], x[m - 1]);
#pragma unroll
        for (int m = 1; m <= 2; ++m) {
            A[m] = sub2(d[m + 1], d[m]);
            Q[m] = fma2(mul2(A[m], c133), A[m], E);
        }
        f2 d23 = sub2(A[2], A[1]), prev;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            d[j + 4] = sub2(x[j + 4], x[j + 3]);
            A[j + 3] = sub2(d[j + 4], d[j + 3]);
            Q[j + 3] = fma2(mul2(A[j + 3], c133), A[j + 3], E);
            const f2 B1 = fma2(m2, d[j + 3], A[j + 3]);
            const f2 B2 = add2(d[j + 2], d[j + 3]);
            const f2 B3 = fma2(two, d[j + 2], A[j + 1]);
            const f2 p2 = fma2(splat(-1.0f / 3.0f), d[j + 2], fma2(splat(-1.0f / 6.0f), d[j + 3], x[j + 2]));
            const f2 d12 = sub2(A[j + 3], A[j + 2]);
            const f2 v = weno_mix(fma2(B1, B1, Q[j + 3]), fma2(B2, B2, Q[j + 2]), fma2(B3, B3, Q[j + 1]), d12, d23, p2);
            if (j > 0) out[j - 1] = fma2(vb, sub2(prev, v), base);
            prev = v;
            d23 = d12;
        }
    }
}

// (put_cols, put_cols_slot, image_pair, store_pole_image, store_images: f32_images.cuh)


// Velocity constants of a velocity set's pairs as the stage kernel reads them.
template <int Q> struct VelOf { typedef VelC type; };
template <> struct VelOf<3> { typedef VelC3 type; };
// (v_theta, v_theta) of pair q's members, and whether the pair's theta upwind side is below
__device__ __forceinline__ f2 pair_vth(const VelC &c, int q) { return c.vth[q >> 2]; }
__device__ __forceinline__ f2 pair_vth(const VelC3 &c, int q) { return c.vt2[q]; }
__device__ __forceinline__ bool pair_thpos(const VelC &, int q) { return (q >> 2) != 0; }
__device__ __forceinline__ bool pair_thpos(const VelC3 &c, int q) { return c.thdir[q] > 0; }
// (v_phi, v_phi) of pair q's members, and the sign of the pair's phi flux (0: none)
__device__ __forceinline__ f2 pair_vph(const VelC &c, int q) { return c.vphi2[q & 3]; }
__device__ __forceinline__ f2 pair_vph(const VelC3 &c, int q) { return c.vb2[q]; }
__device__ __forceinline__ int pair_phdir(const VelC &c, int q) { return c.vphi2[q & 3].x > 0.0f ? 1 : -1; }
__device__ __forceinline__ int pair_phdir(const VelC3 &c, int q) { return c.phdir[q]; }

// The stage's dt share (SSP-RK3, Sec. 3.7): the stage output is cF F0 + cG G + dte L[G] with
// (cF, cG, dte / dt) = (0, 1, 1), (3/4, 1/4, 1/4), (1/3, 2/3, 2/3).  (The scalar constants use
// explicit roundings: no contraction may differ between the standalone and the batch kernel, whose
// results must agree bit for bit, nor from the host's copy of the tile tables.)
__device__ __forceinline__ float stage_dte(int stage, float dt)
{
    return (stage == 1) ? dt : __fmul_rn((stage == 2) ? 0.25f : (2.0f / 3.0f), dt);
}

// The tile tables of tile row i0 filled by the CTA's threads from the run's arrays (the batch kernel).
template <int TY, int NPP, bool LIN>
__device__ __forceinline__ void fill_tab(TabT<TY, NPP> &T, const RunF &R, int i0, float dte)
{
    constexpr int SR = TY + 2 * GR;
    int t = threadIdx.x;
    if (t < SR) {
        T.ds2[t] = splat(R.dsin[i0 + t]);
    } else if ((t -= SR) < SR) {
        T.d2s2[t] = splat(R.d2sin[i0 + t]);
    } else if ((t -= SR) < TY) {
        T.rowc[t] = R.row[min(i0 + t, R.L.nt - 1)];
    } else if ((t -= TY) < TY * NPP) {
        const int ry = t / NPP, q = t - (t / NPP) * NPP;
        T.rr[ry][q] = mul2(R.rref[(size_t)min(i0 + ry, R.L.nt - 1) * NPP + q], splat(dte));
    } else if (LIN && (t -= TY * NPP) < SR) {
        T.isp2[t] = splat(R.isp[i0 + t]);
    } else if (LIN && (t -= SR) < TY + 1) {
        T.sf2[t] = splat(R.sfc[i0 + t]);
    }
}

// A pole face's contribution of one pair and column: v_theta times the face value of each member,
// in FP64, summed over the warp's columns (xor butterfly: every lane ends with the same sum, formed
// in the same order); lane 0 stores it.
__device__ __forceinline__ void pole_face(double *slot, f2 vth, f2 v, bool valid)
{
    double x = valid ? fma((double)vth.x, (double)v.x, (double)vth.y * (double)v.y) : 0.0;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
    if ((threadIdx.x & 31) == 0) *slot = x;
}

// The theta-face value at face fy of pair q and this lane's column (the reconstruction of dg that
// the theta walkers form there; the same operations in the same order).
template <int TY, bool LIN, class VC, class Box, class Tab>
__device__ __forceinline__ f2 theta_face_value(const RunF &R, const VC &c, const Box &box, const Tab &tab, int q,
                                               int fy, int lane)
{
    const f2 *col = &box.v[q][0][lane + GC];
    const bool g = pair_thpos(c, q);
    if constexpr (LIN) {
        const f2 l0 = splat(R.lin0), l1 = splat(R.lin1), l2 = splat(R.lin2);
        return g ? fma2(l0, col[(fy + 1) * SC], fma2(l1, col[(fy + 2) * SC], mul2(l2, col[(fy + 3) * SC])))
                 : fma2(l0, col[(fy + 4) * SC], fma2(l1, col[(fy + 3) * SC], mul2(l2, col[(fy + 2) * SC])));
    } else {
        const f2 E = splat(R.e_theta), c133 = splat(13.0f / 3.0f), two = splat(2.0f), m2 = splat(-2.0f);
        const f2 wr = R.wr[q];
        f2 x[6], dd[6], dfu[6], D2[6], Qa[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) x[m] = col[(fy + m) * SC];
#pragma unroll
        for (int m = 1; m < 6; ++m) {
            dd[m] = sub2(x[m], x[m - 1]);
            dfu[m] = fma2(wr, tab.ds2[fy + m], dd[m]);
        }
#pragma unroll
        for (int m = 1; m < 5; ++m) {
            D2[m] = fma2(wr, tab.d2s2[fy + m], sub2(dd[m + 1], dd[m]));
            Qa[m] = fma2(mul2(D2[m], c133), D2[m], E);
        }
        f2 B1, B2, B3, Q1, Q2, Q3, d12, d23, p2;
        if (g) {
            Q1 = Qa[1]; Q2 = Qa[2]; Q3 = Qa[3];
            B1 = fma2(two, dfu[2], D2[1]);
            B2 = add2(dfu[2], dfu[3]);
            B3 = fma2(m2, dfu[3], D2[3]);
            d12 = sub2(D2[1], D2[2]);
            d23 = sub2(D2[2], D2[3]);
            p2 = fma2(splat(1.0f / 6.0f), dd[2], fma2(splat(1.0f / 3.0f), dd[3], x[2]));
        } else {
            Q1 = Qa[4]; Q2 = Qa[3]; Q3 = Qa[2];
            B1 = fma2(m2, dfu[4], D2[4]);
            B2 = add2(dfu[4], dfu[3]);
            B3 = fma2(two, dfu[3], D2[2]);
            d12 = sub2(D2[4], D2[3]);
            d23 = sub2(D2[3], D2[2]);
            p2 = fma2(splat(-1.0f / 6.0f), dd[4], fma2(splat(-1.0f / 3.0f), dd[3], x[3]));
        }
        return weno_mix(fma2(B1, B1, Q1), fma2(B2, B2, Q2), fma2(B3, B3, Q3), d12, d23, p2);
    }
}

// Face phase of one stage of one TY x TX tile (q0 = bx TX, i0 = by TY) whose input box and
// tables are in tile buffer b of S: the phi and theta faces of every pair into S.adv (and S.advT).
// Ends without a barrier.
template <int TY, bool LIN, int Q, bool KW = false, class Sm>
__device__ __forceinline__ void tile_faces(const RunF &R, const typename VelOf<Q>::type &c, float dte, Sm &S,
                                           int b, int tb, int bx, int by)
{
    constexpr int NPQ = (Q == 3) ? 5 : NP2;   // pair planes
    constexpr int NFQ = (Q == 3) ? 4 : NP2;   // pairs with fluxes (D2Q9's fifth: the rest population)
    constexpr int SR = TY + 2 * GR;
    constexpr int NT = TY * 32;
    constexpr int NW = NT / 32;
    // warps of the face phases: D2Q16 and 4-warp D2Q9 tiles walk a pair's phi faces and then its
    // theta faces on one warp (pairs warp, warp + NW, ...); 8-warp D2Q9 tiles walk the four
    // pairs' phi faces on warps 0-3 and their theta faces on warps 4-7, into advT
    constexpr bool SPLIT = (Q == 3) && (NW == 2 * NFQ);
    constexpr int FSTEP = SPLIT ? NFQ : NW;
    (void)SR; (void)NFQ; (void)FSTEP; (void)SPLIT;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    (void)tid;
    const BoxT<TY, NPQ> &box = S.tile[b];
    const TabT<TY, NPQ> &tab = S.tab[tb];
    // Every face value below is premultiplied by the stage's dt share dte and by the
    // metric factor of its difference (1/(R sin dphi) for phi, 1/(R dtheta) for the
    // WENO-5 and plain upwind theta fluxes).  Each walker turns its consecutive faces into
    // the flux differences of the cells between them: the phi walkers write them, plus the
    // reference tendency, to adv, and the theta walker of the same warp and pair adds its
    // difference, so that the cell update reads one value per pair.
    // ---- phi: warp = pair (pairs warp, warp + TY, ...), lane = (segment sg, row r); segment
    // sg walks faces SEG sg .. SEG sg + SEG of row r for its SEG cells
    {
        constexpr int NSEG = 32 / TY, SEG = TX / NSEG;
        const int r = lane % TY, sg = lane / TY, f0 = sg * SEG;
        const f2 sp = splat(__fmul_rn(tab.rowc[r].inv_dph, dte));
        if constexpr (LIN) {
            const f2 l0 = splat(R.lin0), l1 = splat(R.lin1), l2 = splat(R.lin2);
#pragma unroll 1
            for (int q = warp; q < (SPLIT ? (warp < NFQ ? NFQ : 0) : NFQ); q += FSTEP) {
                const f2 vb = mul2(pair_vph(c, q), sp);
                const f2 *row = &box.v[q][r + GR][0];
                f2 *out = &S.adv[q][r][f0];
                const int dir = pair_phdir(c, q);
                if (dir > 0) phi_march_lin<SEG + 1, 1>(row, f0, l0, l1, l2, vb, tab.rr[r][q], out);
                else if (dir < 0) phi_march_lin<SEG + 1, -1>(row, f0, l0, l1, l2, vb, tab.rr[r][q], out);
                else
                    for (int j = 0; j < SEG; ++j) out[j] = tab.rr[r][q];
            }
        } else {
            const f2 E = splat(tab.rowc[r].ephi);
#pragma unroll 1
            for (int q = warp; q < (SPLIT ? (warp < NFQ ? NFQ : 0) : NFQ); q += FSTEP) {
                const f2 vb = mul2(pair_vph(c, q), sp);
                const f2 *row = &box.v[q][r + GR][0];
                f2 *out = &S.adv[q][r][f0];
                const int dir = pair_phdir(c, q);
                if (dir > 0) phi_march<SEG + 1, 1>(row, f0, E, vb, tab.rr[r][q], out);
                else if (dir < 0) phi_march<SEG + 1, -1>(row, f0, E, vb, tab.rr[r][q], out);
                else
                    for (int j = 0; j < SEG; ++j) out[j] = tab.rr[r][q];
            }
        }
    }
    __syncwarp();   // the theta walker reads the cells this warp's phi walkers wrote

    // ---- upwind schemes, theta faces: warp = pair, lane = column; the column's values are dg
    // (nodal g = sin f), or for the Komissarov flux df = dg / sin (ghost rows: the mapped
    // population's df), then v_theta times the interface sine times the reconstruction.
    // These faces carry dte only: their differences take 1/(R dtheta), or the Komissarov
    // row factor s / (R dcos).
    if constexpr (LIN) {
        const f2 l0 = splat(R.lin0), l1 = splat(R.lin1), l2 = splat(R.lin2);
        const bool kom = R.komissarov != 0;
#pragma unroll 1
        for (int q = SPLIT ? warp - NFQ : warp; q >= 0 && q < NFQ; q += FSTEP) {
            const bool g = pair_thpos(c, q);
            const f2 vt = mul2(pair_vth(c, q), splat(dte));
            const f2 *col = &box.v[q][0][lane + GC];
            f2 x[SR], prev;
#pragma unroll
            for (int r = 0; r < SR; ++r) x[r] = kom ? mul2(col[r * SC], tab.isp2[r]) : col[r * SC];
#pragma unroll
            for (int fy = 0; fy <= TY; ++fy) {
                // face fy lies between tile rows fy-1 and fy (x index = tile row + GR)
                const f2 rec = g ? fma2(l0, x[fy + 1], fma2(l1, x[fy + 2], mul2(l2, x[fy + 3])))
                                 : fma2(l0, x[fy + 4], fma2(l1, x[fy + 3], mul2(l2, x[fy + 2])));
                const f2 fl = kom ? mul2(mul2(vt, rec), tab.sf2[fy]) : mul2(vt, rec);
                if (fy > 0) {
                    const int cy = fy - 1;
                    const f2 idth = splat(kom ? tab.rowc[cy].kth : R.inv_dth);
                    if constexpr (SPLIT) S.advT[q][cy][lane] = mul2(sub2(prev, fl), idth);
                    else S.adv[q][cy][lane] = fma2(sub2(prev, fl), idth, S.adv[q][cy][lane]);
                }
                prev = fl;
            }
        }
    }

    // ---- WENO-5 theta faces: warp = pair, lane = column, marching over the TY+1 face rows.
    // Consecutive faces share their second differences (the smoothness forms of the
    // three candidate stencils are centred on consecutive rows) and the row terms
    // 13/3 A^2 + E.  With x the tile column (rows 0..SR-1), for v > 0 face fy uses
    // x[fy..fy+4] in upwind order, for v < 0 it uses x[fy+5..fy+1].  The smoothness
    // forms are those of the full g = dg + w rho_ref sin(theta) (first and second
    // differences of sin from the FP64 tables); P2 is taken on dg alone.
    // KW: WENO-5 with the Komissarov theta flux (Eqs. Komissarov_scheme, Komissarov_sin_cos): the
    // reconstruction is of f (the column's values are df = dg / sin; the reference part of f is
    // the constant w rho_ref, which leaves every difference alone), the face flux carries the
    // interface sine, and the difference of two faces the row factor s / (R dcos) (the reference
    // state's Komissarov flux difference is in rref).
    if constexpr (!LIN) {
        const f2 E = splat(R.e_theta), c133 = splat(13.0f / 3.0f);
        const f2 two = splat(2.0f), m2 = splat(-2.0f);
#pragma unroll 1
        for (int q = SPLIT ? warp - NFQ : warp; q >= 0 && q < NFQ; q += FSTEP) {
            const bool g = pair_thpos(c, q);
            const f2 wr = R.wr[q];
            const f2 vt = KW ? mul2(pair_vth(c, q), splat(dte)) : mul2(pair_vth(c, q), splat(__fmul_rn(dte, R.inv_dth)));
            const f2 *col = &box.v[q][0][lane + GC];
            // values are produced one row ahead of their first use (face fy needs rows up to fy+5)
            f2 x[SR], dd[SR], dfu[SR], D2[SR], Qa[SR], prev, dcarry;
#pragma unroll
            for (int r = 0; r < 5; ++r) x[r] = KW ? mul2(col[r * SC], tab.isp2[r]) : col[r * SC];
#pragma unroll
            for (int r = 1; r < 5; ++r) {
                dd[r] = sub2(x[r], x[r - 1]);
                dfu[r] = KW ? dd[r] : fma2(wr, tab.ds2[r], dd[r]);
            }
#pragma unroll
            for (int r = 1; r < 4; ++r) {
                D2[r] = KW ? sub2(dd[r + 1], dd[r]) : fma2(wr, tab.d2s2[r], sub2(dd[r + 1], dd[r]));
                Qa[r] = fma2(mul2(D2[r], c133), D2[r], E);
            }
#pragma unroll
            for (int fy = 0; fy <= TY; ++fy) {
                {   // extend the window to row fy + 5
                    const int r = fy + 5;
                    x[r] = KW ? mul2(col[r * SC], tab.isp2[r]) : col[r * SC];
                    dd[r] = sub2(x[r], x[r - 1]);
                    dfu[r] = KW ? dd[r] : fma2(wr, tab.ds2[r], dd[r]);
                    D2[r - 1] = KW ? sub2(dd[r], dd[r - 1]) : fma2(wr, tab.d2s2[r - 1], sub2(dd[r], dd[r - 1]));
                    Qa[r - 1] = fma2(mul2(D2[r - 1], c133), D2[r - 1], E);
                }
                f2 B1, B2, B3, Q1, Q2, Q3, d12, d23, p2;
                // the A differences of consecutive faces overlap: d12 of face fy + 1 is d23 of
                // face fy for v > 0, and d23 of face fy + 1 is d12 of face fy for v < 0
                if (g) {   // v_theta > 0: a..e = x[fy..fy+4]
                    Q1 = Qa[fy + 1]; Q2 = Qa[fy + 2]; Q3 = Qa[fy + 3];
                    B1 = fma2(two, dfu[fy + 2], D2[fy + 1]);
                    B2 = add2(dfu[fy + 2], dfu[fy + 3]);
                    B3 = fma2(m2, dfu[fy + 3], D2[fy + 3]);
                    d12 = fy ? dcarry : sub2(D2[fy + 1], D2[fy + 2]);
                    d23 = sub2(D2[fy + 2], D2[fy + 3]);
                    dcarry = d23;
                    p2 = fma2(splat(1.0f / 6.0f), dd[fy + 2], fma2(splat(1.0f / 3.0f), dd[fy + 3], x[fy + 2]));
                } else {   // v_theta < 0: a..e = x[fy+5..fy+1]
                    Q1 = Qa[fy + 4]; Q2 = Qa[fy + 3]; Q3 = Qa[fy + 2];
                    B1 = fma2(m2, dfu[fy + 4], D2[fy + 4]);
                    B2 = add2(dfu[fy + 4], dfu[fy + 3]);
                    B3 = fma2(two, dfu[fy + 3], D2[fy + 2]);
                    d12 = sub2(D2[fy + 4], D2[fy + 3]);
                    d23 = fy ? dcarry : sub2(D2[fy + 3], D2[fy + 2]);
                    dcarry = d12;
                    p2 = fma2(splat(-1.0f / 6.0f), dd[fy + 4], fma2(splat(-1.0f / 3.0f), dd[fy + 3], x[fy + 3]));
                }
                // P2 of the reference part is in the FP64-derived tendency rref
                f2 v = weno_mix(fma2(B1, B1, Q1), fma2(B2, B2, Q2), fma2(B3, B3, Q3), d12, d23, p2);
                if constexpr (KW) v = mul2(v, tab.sf2[fy]);   // face flux / (v_theta dte): interface sine
                if (fy > 0) {
                    const int cy = fy - 1;
                    const f2 vk = KW ? mul2(vt, splat(tab.rowc[cy].kth)) : vt;
                    if constexpr (SPLIT) S.advT[q][cy][lane] = mul2(vk, sub2(prev, v));
                    else S.adv[q][cy][lane] = fma2(vk, sub2(prev, v), S.adv[q][cy][lane]);
                }
                prev = v;
            }
        }
    }

    // Pole faces (face 0 of the first tile row, face n_theta - i0 of the last tile row): for the
    // pole mass-flux budget each pair's theta-face value there, the reconstruction of dg exactly
    // as its walker formed it (the reference part's is added on the host side), is evaluated
    // once more and its v_theta-weighted sum over the tile's columns recorded.  Only the tiles on
    // a pole do this, outside the walkers.
    const int i0f = by * TY;
    const bool pole_n = R.pole_part != nullptr && i0f == 0;
    const int pole_s = (R.pole_part != nullptr && i0f + TY >= R.L.nt) ? R.L.nt - i0f : -1;
    if (pole_n || pole_s >= 0) {
        const bool col_ok = bx * TX + lane < R.L.np;
#pragma unroll 1
        for (int q = SPLIT ? warp - NFQ : warp; q >= 0 && q < NFQ; q += FSTEP) {
            if (pole_n) pole_face(&S.polew[0][q], pair_vth(c, q), theta_face_value<TY, LIN>(R, c, box, tab, q, 0, lane), col_ok);
            if (pole_s >= 0)
                pole_face(&S.polew[1][q], pair_vth(c, q), theta_face_value<TY, LIN>(R, c, box, tab, q, pole_s, lane), col_ok);
        }
    }
}

// The stage input of this thread's cell (warp = cell row, lane = column) from tile buffer b.
template <int TY, int NPQ, class Sm>
__device__ __forceinline__ void load_cell_g(const Sm &S, int b, f2 *G)
{
    const int cy = threadIdx.x >> 5, cx = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NPQ; ++q) G[q] = S.tile[b].v[q][cy + GR][cx + GC];
}

// Cell phase of one stage of one tile after the face phase (and a barrier): per cell the
// moments, equilibrium, force, BGK, flux differences and stage combination, then the store of
// the tile (one TMA store through tmo from S.ob for tiles clear of every ghost image, with a
// barrier inside; per cell with its images otherwise).  In stages 2 and 3, S.ob holds the tile
// of F when this begins.  Threads of cells outside the grid return early.
template <int TY, bool LIN, int Q, class Sm>
__device__ __forceinline__ void tile_cells(const RunF &R, const typename VelOf<Q>::type &c, int stage, float dte,
                                           const CUtensorMap *tmo, int bx, int by, Sm &S, int b, int tb,
                                           const f2 *Gin)
{
    constexpr int NPQ = (Q == 3) ? 5 : NP2;   // pair planes
    constexpr int NFQ = (Q == 3) ? 4 : NP2;   // pairs with fluxes (D2Q9's fifth: the rest population)
    constexpr int SR = TY + 2 * GR;
    constexpr int NT = TY * 32;
    constexpr int NW = NT / 32;
    // warps of the face phases: D2Q16 and 4-warp D2Q9 tiles walk a pair's phi faces and then its
    // theta faces on one warp (pairs warp, warp + NW, ...); 8-warp D2Q9 tiles walk the four
    // pairs' phi faces on warps 0-3 and their theta faces on warps 4-7, into advT
    constexpr bool SPLIT = (Q == 3) && (NW == 2 * NFQ);
    constexpr int FSTEP = SPLIT ? NFQ : NW;
    (void)SR; (void)NFQ; (void)FSTEP; (void)SPLIT;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    (void)tid;
    const int q0 = bx * TX;
    const int i0 = by * TY;
    const Layout L = R.L;
    float2 *out = (stage == 1) ? R.A : (stage == 2) ? R.B : R.F;
    const BoxT<TY, NPQ> &box = S.tile[b];
    const TabT<TY, NPQ> &tab = S.tab[tb];
    // the tile's pole-face partials (the face phase's per-pair sums, added in pair order)
    if (R.pole_part != nullptr && tid == 0) {
        const size_t base = (size_t)(stage - 1) * 2 * R.tiles_x + bx;
        for (int pole = 0; pole < 2; ++pole) {
            if (pole == 0 ? i0 != 0 : i0 + TY < L.nt) continue;
            double sum = 0.0;
            for (int q = 0; q < NFQ; ++q) sum += S.polew[pole][q];
            R.pole_part[base + (size_t)pole * R.tiles_x] = sum;
        }
    }
    // ---- one cell per thread: warp = cell row, lane = column
    const int cy = warp, cx = lane;
    const int i = i0 + cy, j = q0 + cx;
    if (i >= L.nt || j >= L.np) return;
    // the step's start values of this cell (stages 2, 3; the slots this thread's output
    // overwrites below)
    f2 F0[NPQ];
    if (stage != 1) {
#pragma unroll
        for (int q = 0; q < NPQ; ++q) F0[q] = S.ob[q][cy][cx];
    }
    const RowF rc = tab.rowc[cy];
    f2 G[NPQ];
#pragma unroll
    for (int q = 0; q < NPQ; ++q) G[q] = Gin[q];
    (void)box;
    // moments of delta f = dg / (k s)
    f2 sn, sjt, sjp;
    if constexpr (Q == 4) {
        // (from the sums over b at each g and over g at each b: v_theta depends on g, v_phi on b)
        const f2 T0 = add2(add2(G[0], G[1]), add2(G[2], G[3])), T1 = add2(add2(G[4], G[5]), add2(G[6], G[7]));
        const f2 S0 = add2(G[0], G[4]), S1 = add2(G[1], G[5]), S2 = add2(G[2], G[6]), S3 = add2(G[3], G[7]);
        sn = add2(T0, T1);
        sjt = fma2(c.vth[1], T1, mul2(c.vth[0], T0));
        sjp = fma2(c.vphi2[3], S3, fma2(c.vphi2[2], S2, fma2(c.vphi2[1], S1, mul2(c.vphi2[0], S0))));
    } else {
        sn = G[0];
        sjt = mul2(c.vt2[0], G[0]);
        sjp = mul2(c.vb2[0], G[0]);
#pragma unroll
        for (int q = 1; q < NPQ; ++q) {
            sn = add2(sn, G[q]);
            sjt = fma2(c.vt2[q], G[q], sjt);
            sjp = fma2(c.vb2[q], G[q], sjp);
        }
    }
    const float SG = sn.x + sn.y;                         // sum_k dg_k = s dn
    const float n = fmaf(SG, rc.inv_s, R.rho_ref);
    const float nin = rcp_approx(n);
    const float ut = (sjt.x + sjt.y) * rc.inv_s * nin;
    const float up = (sjp.x + sjp.y) * rc.inv_s * nin;
    const float u2 = fmaf(ut, ut, up * up);
    const f2 h0 = splat(-0.5f * u2), h1 = splat(fmaf(-0.5f, u2, 1.0f));
    // BGK share of the update: dg is weighted by cG - dte/tau and s feq_dev by dte/tau.  The
    // second weight is taken as the exact FP32 complement sc = cG0 - RN(cG0 - dte/tau), so
    // the two sum to the stage's weight of dg exactly and the collision (which conserves
    // sum_k) leaves no systematic drift of the mass; likewise the stage-3 weight of F0 is
    // the exact complement 1 - RN(2/3).
    const float cg0 = (stage == 1) ? 1.0f : (stage == 2) ? 0.25f : (2.0f / 3.0f);
    const float cgv = __fsub_rn(cg0, __fmul_rn(dte, R.tau_inv));
    const float sc = __fsub_rn(cg0, cgv);
    // the equilibrium deviation times sc s: w (s dn + s n poly(xi)) sc, poly = xi + (xi^2 - u^2)/2
    // + xi (xi^2 - 3 u^2)/6 = xi^3/6 + xi^2/2 + (1 - u^2/2) xi - u^2/2 (D2Q16, Eq. feq_Q=4; D2Q9
    // stops at the second order, Eq. feq_Q=3: xi^2/2 + xi - u^2/2), its Horner coefficients
    // scaled by sc s n once per cell (and sc s dn folded into the constant term)
    const float sns = __fmul_rn(__fmul_rn(sc, rc.s), n);
    const f2 ut2 = splat(ut), up2 = splat(up);
    const f2 e3 = splat(__fmul_rn(sns, 1.0f / 6.0f)), e2 = splat(__fmul_rn(sns, 0.5f));
    const f2 e1 = splat(Q == 4 ? __fmul_rn(sns, h1.x) : sns), e0 = splat(__fmaf_rn(sns, h0.x, __fmul_rn(sc, SG)));
    // D2Q9 force brackets per slot (see below)
    float fbs[2 * NPQ];
    if constexpr (Q == 3) {
        // the six terms of slot t's bracket (population (a, b)) act on the populations (a', b),
        // a' = 0..2, then (a, b'), b' = 0..2, read from their slots
        float gs[10];
#pragma unroll
        for (int q = 0; q < NPQ; ++q) {
            gs[2 * q] = G[q].x;
            gs[2 * q + 1] = G[q].y;
        }
        // the population of each slot: the K terms vanish where v_phi = 0 (b = 1), the Ktilde terms
        // where v_theta = 0 (a = 1), both for the empty slot; leaving out these exact zeros
        // changes no rounding (fma(0, x, acc) = acc)
#pragma unroll
        for (int t = 0; t < 10; ++t) {
            const int k = f32_pop_of_slot(3, t);
            float acc = 0.0f;
            bool first = true;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                if (k < 0 || (m < 3 && k % 3 == 1) || (m >= 3 && k / 3 == 1)) continue;
                const int src = f32_slot_of_pop(3, m < 3 ? 3 * m + k % 3 : 3 * (k / 3) + (m - 3));
                acc = first ? __fmul_rn(c.fcoef[t][m], gs[src]) : __fmaf_rn(c.fcoef[t][m], gs[src], acc);
                first = false;
            }
            fbs[t] = acc;
        }
    }
    const f2 ncot = splat(__fmul_rn(-dte, rc.cotR));
    const f2 cG = splat(cgv);
    const f2 cF = splat((stage == 2) ? 0.75f : __fsub_rn(1.0f, 2.0f / 3.0f));

    f2 o[NPQ];
#pragma unroll
    for (int q = 0; q < NPQ; ++q) {
        // xi = v . u; the equilibrium deviation times sc s, without w
        f2 xi, feq, fb;
        if constexpr (Q == 4) {
            const int g = q >> 2, b = q & 3;
            xi = fma2(c.vth[g], ut2, mul2(c.vphi2[b], up2));
            feq = fma2(xi, fma2(xi, fma2(xi, e3, e2), e1), e0);
            // force bracket on dg: K along k_theta (pairs (0,b),(1,b) with swapped partners), Ktilde
            // along k_phi (pairs (g,0..3)), the velocity factors folded into the coefficients
            const f2 P0 = G[b], P1 = G[4 + b];
            const f2 *Gg = G + 4 * g;
            fb = mul2(c.kf[q][0], P0);
            fb = fma2(c.kf[q][1], swap2(P0), fb);
            fb = fma2(c.kf[q][2], P1, fb);
            fb = fma2(c.kf[q][3], swap2(P1), fb);
#pragma unroll
            for (int m = 0; m < 4; ++m) fb = fma2(c.ktf[q][m], Gg[m], fb);
        } else {
            xi = fma2(c.vt2[q], ut2, mul2(c.vb2[q], up2));
            feq = fma2(xi, fma2(xi, e2, e1), e0);
            fb = make_float2(fbs[2 * q], fbs[2 * q + 1]);
        }
        // dte times: flux differences + s rref - force + s feq_dev / tau (the rest population
        // of D2Q9 has no flux: its share is the reference tendency alone)
        f2 a;
        if (q >= NFQ) a = tab.rr[cy][q];
        else if constexpr (SPLIT) a = add2(S.adv[q][cy][cx], S.advT[q][cy][cx]);
        else a = S.adv[q][cy][cx];
        a = fma2(ncot, fb, a);
        a = fma2(c.w2[q], feq, a);
        o[q] = fma2(cG, G[q], a);
        if (stage != 1) o[q] = fma2(cF, F0[q], o[q]);
    }
    // tiles clear of the ghost images (no pole-row or seam image to write, no ragged edge):
    // the output tile is staged in shared memory and leaves with one TMA store; the issuing
    // thread waits until the store has read it
    const bool core = (i0 >= GR && i0 + TY <= L.nt - GR && q0 >= GC && q0 + TX <= L.np - GC);
    if (core) {
        f2 *ob = &S.ob[0][0][0];
#pragma unroll
        for (int q = 0; q < NPQ; ++q) ob[(q * TY + cy) * TX + cx] = o[q];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                             reinterpret_cast<unsigned long long>(tmo)),
                         "r"(q0 + GC), "r"(i0 + GR), "r"(0), "r"(smem_u32(ob))
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        return;
    }
    const bool plain = (i >= GR && i < L.nt - GR && j >= GC && j < L.np - GC);
    if (plain) {
#pragma unroll
        for (int q = 0; q < NPQ; ++q) out[L.at(q, i, j)] = o[q];
    } else {
#pragma unroll
        for (int q = 0; q < NPQ; ++q) store_images(out, L, Q, q, i, j, o[q]);
    }
}

// One stage of one TY x TX tile of one run.  The mbarrier is initialised by the
// caller; `parity` is the phase this tile's load completes.  Returns false if
// the tile load did not arrive in time (every thread of the CTA agrees).  tm is the
// stage input's box map (42 x (TY+6) x 8); tmo and tmf are the tile-core maps (32 x TY
// x 8) of the stage output and of the step's start values F: stages 2 and 3 load their
// tile of F through tmf into the staging buffer with the input box, and tiles clear of
// every ghost image store their output from there with one TMA store through tmo.
// LIN: the upwind schemes U1-U3 (Eq. fluxes_U1-3, optionally with the Komissarov theta flux)
// instead of WENO-5.
// Q: the velocity set (4: D2Q16, 3: D2Q9 in five pairs).
template <int TY, bool LIN, int Q, bool KW = false>
__device__ __forceinline__ bool stage_tile(const RunF &R, const typename VelOf<Q>::type &c, int stage,
                                           const CUtensorMap *tm, const CUtensorMap *tmo, const CUtensorMap *tmf,
                                           int bx, int by, SmemT<TY, (Q == 3 ? 5 : NP2)> &S, unsigned parity,
                                           unsigned *err)
{
    constexpr int NPQ = (Q == 3) ? 5 : NP2;
    constexpr unsigned TILE_BYTES = NPQ * (TY + 2 * GR) * SC * sizeof(float2);
    constexpr unsigned CORE_BYTES = NPQ * TY * TX * sizeof(float2);
    const int tid = threadIdx.x;
    const int q0 = bx * TX;
    const int i0 = by * TY;
    const float dte = stage_dte(stage, R.dt);

    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.bar[0])),
                     "r"(stage == 1 ? TILE_BYTES : TILE_BYTES + CORE_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(&S.tile[0].v[0][0][0])),
            "l"(reinterpret_cast<unsigned long long>(tm)), "r"(q0), "r"(i0), "r"(0), "r"(smem_u32(&S.bar[0]))
            : "memory");
        // stages 2, 3: the tile's step start values F into the staging buffer (parts outside
        // the array read as zero and belong to no cell)
        if (stage != 1)
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(&S.ob[0][0][0])),
                "l"(reinterpret_cast<unsigned long long>(tmf)), "r"(q0 + GC), "r"(i0 + GR), "r"(0),
                "r"(smem_u32(&S.bar[0]))
                : "memory");
    }
    // per-tile tables while the tile is in flight
    fill_tab<TY, NPQ, LIN || KW>(S.tab[0], R, i0, dte);
    // (the barrier of the load wait also publishes the tables; the caller has made the
    // mbarrier's initialisation visible to every thread before this tile began)
    const bool ok = __syncthreads_and(wait_phase(&S.bar[0], parity, R.wait_ns));
    if (!ok) {
        // the copy did not complete within the wait limit (1 s unless set otherwise): flag it,
        // give it one more bounded second to land in this CTA's shared memory, then leave
        if (tid == 0) atomicOr(err, 1u);
        wait_phase(&S.bar[0], parity, 1000000000ull);
        return false;
    }
    tile_faces<TY, LIN, Q, KW>(R, c, dte, S, 0, 0, bx, by);
    __syncthreads();
    f2 G[NPQ];
    load_cell_g<TY, NPQ>(S, 0, G);
    tile_cells<TY, LIN, Q>(R, c, stage, dte, tmo, bx, by, S, 0, 0, G);
    return true;
}

template <int TY, bool LIN, int Q, bool KW = false>
__global__ void __launch_bounds__(TY * 32, (Q == 3 ? 32 : 24) / TY) stage_f32_kernel(const __grid_constant__ CUtensorMap tm,
                                                                      const __grid_constant__ CUtensorMap tmo,
                                                                      const __grid_constant__ CUtensorMap tmf,
                                                                      const RunF R, const typename VelOf<Q>::type c,
                                                                      int stage, const TileRows rows, unsigned *err)
{
    typedef SmemT<TY, (Q == 3 ? 5 : NP2)> Smem;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar[0])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();   // no thread may poll the barrier before its initialisation is visible
    const int by = rows.first + (int)blockIdx.y + ((int)blockIdx.y >= rows.split ? rows.skip : 0);
    stage_tile<TY, LIN, Q, KW>(R, c, stage, &tm, &tmo, &tmf, blockIdx.x, by, S, 0u, err);
}

// Persistent stage kernel (8 tile rows, three CTAs per SM): CTA b takes the launch's tiles
// b, b + G, b + 2G, ... (G = gridDim.x, tiles numbered row-major over the launch's tile rows) so
// that the copies of its next tile are in flight while it computes one: right after the face phase
// the cell phase takes its cells' stage inputs into registers, and the box and tables of the next
// tile are issued into the freed box buffer (the tables alternate between two buffers) while this
// tile's cells are computed and stored; the tile of F (stages 2, 3) of the next tile is issued as
// soon as this tile's output has left the staging buffer.  tabs holds this stage's tables of every
// tile row of the grid.  A copy that does not arrive within the run's wait limit sets *err; the
// CTA then waits (bounded, 1 s) for its other copies in flight and leaves.
template <bool LIN, int Q>
__global__ void __launch_bounds__(256, 3)
    stage_f32_persist_kernel(const __grid_constant__ CUtensorMap tm, const __grid_constant__ CUtensorMap tmo,
                             const __grid_constant__ CUtensorMap tmf, const RunF R,
                             const typename VelOf<Q>::type c, int stage, const TileRows rows,
                             const TabT<8, (Q == 3 ? 5 : NP2)> *tabs, unsigned *err, unsigned *ctr)
{
    constexpr int TY = 8;
    constexpr int NPQ = (Q == 3) ? 5 : NP2;
    typedef SmemT<TY, NPQ, 1, 2> Smem;
    constexpr unsigned BOX_BYTES = NPQ * (TY + 2 * GR) * SC * sizeof(float2);
    constexpr unsigned TAB_BYTES = sizeof(TabT<TY, NPQ>);
    constexpr unsigned CORE_BYTES = NPQ * TY * TX * sizeof(float2);
    constexpr unsigned long long LIMIT_NS = 1000000000ull;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int ntx = (R.L.np + TX - 1) / TX;
    const int total = ntx * rows.count;
    const int G = (int)gridDim.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.barF)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();   // no thread may poll a barrier before its initialisation is visible
    // launch tile t -> (bx, by)
    auto tile_xy = [&](int t, int &bx, int &by) {
        const int ly = t / ntx;
        bx = t - ly * ntx;
        by = rows.first + ly + (ly >= rows.split ? rows.skip : 0);
    };
    // (issued by thread 0) the box of tile t and its tables into table buffer tb
    auto issue_box = [&](int t, int tb) {
        int bx, by;
        tile_xy(t, bx, by);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.bar[0])),
                     "r"(BOX_BYTES + TAB_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(&S.tile[0].v[0][0][0])),
            "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(bx * TX), "r"(by * TY), "r"(0),
            "r"(smem_u32(&S.bar[0]))
            : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(&S.tab[tb])),
                     "l"(reinterpret_cast<unsigned long long>(tabs + by)), "r"(TAB_BYTES), "r"(smem_u32(&S.bar[0]))
                     : "memory");
    };
    // (issued by thread 0, stages 2 and 3) the tile of F of tile t into the staging buffer
    auto issue_f = [&](int t) {
        int bx, by;
        tile_xy(t, bx, by);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.barF)),
                     "r"(CORE_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(&S.ob[0][0][0])),
            "l"(reinterpret_cast<unsigned long long>(&tmf)), "r"(bx * TX + GC), "r"(by * TY + GR), "r"(0),
            "r"(smem_u32(&S.barF))
            : "memory");
    };
    // Tiles are handed out dynamically: the first is blockIdx.x, each further one the next
    // value of the launch's counter ctr[0] (+ G), taken when its copies are issued; the CTA that
    // leaves last (counted in ctr[1]) resets both counters for the next launch of this slot.
    __shared__ int next_tile;
    int t = (int)blockIdx.x;
    if (tid == 0 && t < total) {
        issue_box(t, 0);
        if (stage != 1) issue_f(t);
    }
    const float dte = stage_dte(stage, R.dt);
    for (int k = 0; t < total; ++k) {
        const int tb = k & 1;
        const unsigned par = k & 1;   // phase of tile k on the box barrier and on the F barrier
        const bool box_ok = __syncthreads_and(wait_phase(&S.bar[0], par, R.wait_ns));
        bool ok = box_ok, next_box = false;
        if (ok) {
            int bx, by;
            tile_xy(t, bx, by);
            tile_faces<TY, LIN, Q>(R, c, dte, S, 0, tb, bx, by);
            __syncthreads();
            f2 Gc[NPQ];
            load_cell_g<TY, NPQ>(S, 0, Gc);
            __syncthreads();   // the box buffer is free: the next tile's copies go now
            if (tid == 0) {
                const int tn = G + (int)atomicAdd(&ctr[0], 1u);
                next_tile = tn;
                next_box = tn < total;
                if (next_box) issue_box(tn, tb ^ 1);
            }
            if (stage != 1) ok = __syncthreads_and(wait_phase(&S.barF, par, R.wait_ns));
            if (ok) {
                tile_cells<TY, LIN, Q>(R, c, stage, dte, &tmo, bx, by, S, 0, tb, Gc);
                __syncthreads();   // this tile's tables and the staging buffer are free; next_tile is set
                t = next_tile;
                if (tid == 0 && stage != 1 && t < total) issue_f(t);
                continue;
            }
        }
        // a copy did not arrive within the wait limit (1 s unless set otherwise): flag it, give
        // this CTA's copies still in flight one more bounded second each to land in its shared
        // memory, then leave
        if (tid == 0) {
            atomicOr(err, 1u);
            if (!box_ok) wait_phase(&S.bar[0], par, LIMIT_NS);
            if (next_box) wait_phase(&S.bar[0], par ^ 1, LIMIT_NS);
            if (stage != 1) wait_phase(&S.barF, par, LIMIT_NS);
        }
        __syncthreads();
        break;
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ctr[1], 1u) == (unsigned)G - 1u) {
            atomicExch(&ctr[0], 0u);
            atomicExch(&ctr[1], 0u);
        }
    }
}

// Persistent batch stage: CTA b takes work items b, b + gridDim.x, ...; a work item
// is (run, tile index within the run).  The run's parameters are copied into
// shared memory per item.  tms holds 6 maps per run: the box maps of F, A, B, then
// the tile-core maps of F, A, B.
template <int TY, bool LIN, int Q>
__global__ void __launch_bounds__(TY * 32, 24 / TY) batch_stage_f32_kernel(const RunF *runs, const CUtensorMap *tms,
                                                                            const int2 *work, int ntiles,
                                                                            const typename VelOf<Q>::type c,
                                                                            int stage, unsigned *err)
{
    typedef SmemT<TY, (Q == 3 ? 5 : NP2)> Smem;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar[0])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    unsigned parity = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 w = work[t];
        {
            const unsigned *src = reinterpret_cast<const unsigned *>(runs + w.x);
            unsigned *dst = reinterpret_cast<unsigned *>(&S.run);
            for (int m = threadIdx.x; m < (int)(sizeof(RunF) / 4); m += blockDim.x) dst[m] = src[m];
        }
        __syncthreads();
        const int tx = S.run.tiles_x;
        const CUtensorMap *tr = tms + 6 * w.x;
        if (!stage_tile<TY, LIN, Q>(S.run, c, stage, tr + (stage - 1), tr + 3 + stage % 3, tr + 3, w.y % tx,
                                    w.y / tx, S, parity, err))
            return;
        parity ^= 1u;
        __syncthreads();   // every thread is done with this tile's shared memory
    }
}

// ---- FP32 layout helpers (FP64 arithmetic) -----------------------------------------

// population k of a velocity set of order q: the value of its slot (pair plane, member)
__device__ __forceinline__ float slot_value(const f2 *f, const Layout &L, int q, int k, int i, int j)
{
    const int sl = f32_slot_of_pop(q, k);
    const f2 pr = f[L.at(sl >> 1, i, j)];
    return (sl & 1) ? pr.y : pr.x;
}

// Velocity-set constants in FP32 for the conversions between moments and the stored deviations:
// per population k (slot order of f32_pop_of_slot) v_theta, v_phi, |v|^2 and the weight.
struct VelF { float va[NK], vb[NK], v2[NK], w[NK]; int q; };

// Initial state in the FP32 deviation form (no FP64 arithmetic per population): per cell
// dn = rho - rho_ref and T - 1 in FP64 (one subtraction each), then per population the deviation
// f_k - w_k rho_ref = w_k (dn + n (P_k - 1)) of the Hermite projection of the Maxwellian at (rho, u,
// T) (Eq. feq_Q=4 at T = 1: third order; with T != 1 the a^(2), a^(3) terms of the projection;
// D2Q9, Eq. feq_Q=3: second order), P_k - 1 = xi + (xi^2 - u^2 + dT (|v|^2 - 2)) / 2
// [+ (xi (xi^2 - 3 u^2) + 3 dT xi (|v|^2 - 4)) / 6], in FP32 on the small terms; stored as
// k s times it.
__global__ void init_f32_kernel(f2 *f, const Layout L, const double *rho, const double *ut, const double *up,
                                const double *temp, const VelF c, double rho_ref, const float *ks_s)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const size_t cell = (size_t)i * L.np + j;
    const float dn = (float)(rho[cell] - rho_ref);
    const float n = (float)rho[cell];
    const float dT = temp ? (float)(temp[cell] - 1.0) : 0.0f;
    const float u1 = (float)ut[cell], u2v = (float)up[cell];
    const float usq = fmaf(u1, u1, u2v * u2v);
    const float s = ks_s[i];
    const int q = c.q;
    float v[2 * NP2];
#pragma unroll
    for (int t = 0; t < 2 * NP2; ++t) {
        if (t >= 2 * f32_pairs(q)) break;
        const int k = f32_pop_of_slot(q, t);
        if (k < 0) {
            v[t] = 0.0f;
            continue;
        }
        const float xi = fmaf(c.va[k], u1, c.vb[k] * u2v);
        float pm1 = xi + 0.5f * fmaf(dT, c.v2[k] - 2.0f, fmaf(xi, xi, -usq));
        if (q == 4) pm1 += (xi * fmaf(3.0f * dT, c.v2[k] - 4.0f, fmaf(xi, xi, -3.0f * usq))) * (1.0f / 6.0f);
        v[t] = s * (c.w[k] * fmaf(n, pm1, dn));
    }
    for (int p = 0; p < f32_pairs(q); ++p) f[L.at(p, i, j)] = make_float2(v[2 * p], v[2 * p + 1]);
}

// Moments in the FP32 deviation form: sums of the stored deviations per cell in FP32, the density
// rho_ref + dn with the reference added in FP64, u = j / n, and T - 1 from the small terms
// (rho_ref |u|^2 + sum_k df_k |v_k - u|^2 - 2 dn) / (2 n) (the reference state's sum_k w_k |v_k|^2 =
// 2 T0, its odd moments vanish; Eq. f_moments_sum).
__global__ void moments_f32_kernel(const f2 *f, const Layout L, double *rho, double *ut, double *up, double *temp,
                                   const VelF c, double rho_ref, const float *inv_ks_s)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= L.np) return;
    const int q = c.q;
    float sn = 0.0f, sjt = 0.0f, sjp = 0.0f, sv2 = 0.0f;
    for (int p = 0; p < f32_pairs(q); ++p) {
        const f2 pr = f[L.at(p, i, j)];
        for (int m = 0; m < 2; ++m) {
            const int k = f32_pop_of_slot(q, 2 * p + m);
            if (k < 0) continue;
            const float x = m ? pr.y : pr.x;
            sn += x;
            sjt = fmaf(c.va[k], x, sjt);
            sjp = fmaf(c.vb[k], x, sjp);
            sv2 = fmaf(c.v2[k], x, sv2);
        }
    }
    const float is = inv_ks_s[i];
    const float dn = sn * is, jt = sjt * is, jp = sjp * is;
    const double n = rho_ref + (double)dn;
    const float nf = (float)n;
    const float u1 = jt / nf, u2 = jp / nf;
    const size_t cell = (size_t)i * L.np + j;
    rho[cell] = n;
    ut[cell] = u1;
    up[cell] = u2;
    if (temp) {
        const float usq = fmaf(u1, u1, u2 * u2);
        // sum_k df_k |v_k - u|^2 = sum df |v|^2 - 2 u . j + |u|^2 dn
        const float dev = fmaf(usq, dn, fmaf(-2.0f, fmaf(u1, jt, u2 * jp), sv2 * is));
        const float tm1 = fmaf((float)rho_ref, usq, dev - 2.0f * dn) / (2.0f * nf);
        temp[cell] = 1.0 + (double)tm1;
    }
}

// one population plane k < q^2 per blockIdx.z
__global__ void pack_f32_kernel(const f2 *f, const Layout L, double *dense, const VelD c, double rho_ref,
                                const double *sin_t, double ks)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y, k = blockIdx.z, q = c.q;
    if (j >= L.np) return;
    const double d = (double)slot_value(f, L, q, k, i, j) / (ks * sin_t[i]);
    dense[((size_t)k * L.nt + i) * L.np + j] = c.w[k / q] * c.w[k % q] * rho_ref + d;
}

// one pair plane per blockIdx.z (the empty slot of D2Q9 is written as zero)
__global__ void unpack_f32_kernel(const double *dense, const Layout L, f2 *f, const VelD c, double rho_ref,
                                  const double *sin_t, double ks)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y, p = blockIdx.z, q = c.q;
    if (j >= L.np) return;
    float m[2];
    for (int h = 0; h < 2; ++h) {
        const int k = f32_pop_of_slot(q, 2 * p + h);
        if (k < 0) {
            m[h] = 0.0f;
            continue;
        }
        const int a = k / q, b = k % q;
        m[h] = (float)(ks * sin_t[i] * (dense[((size_t)k * L.nt + i) * L.np + j] - c.w[a] * c.w[b] * rho_ref));
    }
    f[L.at(p, i, j)] = make_float2(m[0], m[1]);
}

__global__ void fill_ghosts_f32_kernel(f2 *f, const Layout L, int vq)
{
    const int c = (int)(blockIdx.x * blockDim.x + threadIdx.x) - GC;
    const int r = (int)blockIdx.y - GR;
    const int q = blockIdx.z;
    if (c >= L.np + GC) return;
    if (r >= 0 && r < L.nt && c >= 0 && c < L.np) return;
    int rs = r, qs = q, shift = 0;
    bool pole = false;
    if (r < 0) {
        rs = -1 - r;
        pole = true;
    } else if (r >= L.nt) {
        rs = 2 * L.nt - 1 - r;
        pole = true;
    }
    if (pole) shift = L.np / 2;
    int cc = (c + shift) % L.np;
    if (cc < 0) cc += L.np;
    if (!pole) {
        f[L.at(q, r, c)] = f[L.at(qs, rs, cc)];
    } else if (vq == 4) {
        const f2 v = f[L.at(image_pair(q), rs, cc)];
        f[L.at(q, r, c)] = make_float2(-v.y, -v.x);
    } else {
        // each member from the slot of its own image
        float m[2];
        for (int h = 0; h < 2; ++h) {
            const int is = f32_image_slot(vq, 2 * q + h);
            const f2 v = f[L.at(is >> 1, rs, cc)];
            m[h] = -((is & 1) ? v.y : v.x);
        }
        f[L.at(q, r, c)] = make_float2(m[0], m[1]);
    }
}

// Polar ring filter, one CTA per (filtered row, pair plane).  The row is walked in
// windows of 2048 columns; each of the 256 threads owns 8 consecutive columns.
// Block sums are compensated: every addition is Knuth's error-free TwoSum, so a
// partial sum is an unevaluated pair hi + lo of floats that carries the exact sum
// of its inputs up to the rounding of the small lo parts (relative error ~2^-46).
// Partials are combined across the threads of an aligned block by xor shuffles
// (the lower lane's partial always first, so both partners form the same pair)
// and, for blocks wider than a warp, through shared memory in warp order.  The
// block mean is the pair scaled by the exact 1/b and rounded once to FP32, which is
// the value of an FP64 accumulation (to ~2^-46) at FP32-pipe cost: GB300's FP64
// rate is 1/64 of its FP32 rate.  Blocks wider than a window (b > 2048, only for
// n_phi above ~25000) take the slice path below.
constexpr int FILT_THREADS = 256;
constexpr int FILT_COLS = 8;
constexpr int FILT_WIN = FILT_THREADS * FILT_COLS;

struct FF { f2 hi, lo; };   // a float-float pair per member

__device__ __forceinline__ void two_sum(f2 a, f2 b, f2 &s, f2 &e)
{
    s = add2(a, b);
    const f2 v = sub2(s, a);
    e = add2(sub2(a, sub2(s, v)), sub2(b, v));
}

// (a.hi + a.lo) + (b.hi + b.lo) as a renormalised pair; a is the lower-index partial
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    f2 s, e, hi, lo;
    two_sum(a.hi, b.hi, s, e);
    e = add2(e, add2(a.lo, b.lo));
    two_sum(s, e, hi, lo);
    return FF{hi, lo};
}

__device__ __forceinline__ FF ff_shfl_xor(FF a, int m)
{
    FF r;
    r.hi.x = __shfl_xor_sync(0xffffffffu, a.hi.x, m);
    r.hi.y = __shfl_xor_sync(0xffffffffu, a.hi.y, m);
    r.lo.x = __shfl_xor_sync(0xffffffffu, a.lo.x, m);
    r.lo.y = __shfl_xor_sync(0xffffffffu, a.lo.y, m);
    return r;
}

// mean of the block whose sum is a.hi + a.lo: with r = 1/b exact (b a power of two),
// lo r is exact and fma(hi, r, lo r) rounds hi r + lo r once, so the result is the
// correctly rounded mean of the pair (the value an FP64 total scaled and rounded to
// FP32 would give, without the FP64 pipe)
__device__ __forceinline__ f2 ff_mean(FF a, float inv_b)
{
    return make_float2(fmaf(a.hi.x, inv_b, a.lo.x * inv_b), fmaf(a.hi.y, inv_b, a.lo.y * inv_b));
}

// ghost images of cell (p, i, j): periodic columns and, on the first/last GR rows, the pole image
__device__ __forceinline__ void store_ghosts(f2 *f, const Layout &L, int vq, int p, int i, int j, f2 v)
{
    for (int m = 1; j - m * L.np >= -GC; ++m) f[L.at(p, i, j - m * L.np)] = v;
    for (int m = 1; j + m * L.np < L.np + GC; ++m) f[L.at(p, i, j + m * L.np)] = v;
    if (i < GR || i >= L.nt - GR) store_pole_image(f, L, vq, p, i, j, v);
}

// means of the aligned blocks of B columns within one thread's FILT_COLS columns (n valid)
template <int B>
__device__ __forceinline__ void thread_block_means(f2 (&v)[FILT_COLS], int n, float inv_b)
{
#pragma unroll
    for (int j0 = 0; j0 < FILT_COLS; j0 += B) {
        if (j0 >= n) break;
        FF a{v[j0], splat(0.0f)};
#pragma unroll
        for (int m = 1; m < B; ++m) {
            f2 e;
            two_sum(a.hi, v[j0 + m], a.hi, e);
            a.lo = add2(a.lo, e);
        }
        const f2 mean = ff_mean(a, inv_b);
#pragma unroll
        for (int m = 0; m < B; ++m) v[j0 + m] = mean;
    }
}

// Filters row i (block size b) of pair plane q of a velocity set of order vq; called by all
// FILT_THREADS threads of a CTA.
__device__ __forceinline__ void filter_row_f32(f2 *f, const Layout &L, int vq, int i, int b, int q)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float inv_b = 1.0f / (float)b;   // exact: b is a power of two
    __shared__ FF wpart[FILT_THREADS / 32];
    const bool ghost_row = (i < GR || i >= L.nt - GR);
    if (b <= FILT_WIN) {
        for (int w0 = 0; w0 < L.np; w0 += FILT_WIN) {
            const int c0 = w0 + t * FILT_COLS;
            const int n = max(0, min(FILT_COLS, L.np - c0));
            f2 *row = f + L.at(q, i, 0);
            f2 v[FILT_COLS];
            if (n == FILT_COLS) {
                // 8 columns = 64 bytes at a 32-byte aligned offset (pitch and c0 + GC are multiples of 4)
                const float4 *src = reinterpret_cast<const float4 *>(row + c0);
#pragma unroll
                for (int m = 0; m < FILT_COLS / 2; ++m) {
                    const float4 x = src[m];
                    v[2 * m] = make_float2(x.x, x.y);
                    v[2 * m + 1] = make_float2(x.z, x.w);
                }
            } else {
#pragma unroll
                for (int m = 0; m < FILT_COLS; ++m) v[m] = (m < n) ? row[c0 + m] : make_float2(0.f, 0.f);
            }
            if (b < FILT_COLS) {
                // blocks lie inside this thread's columns (b divides n_phi, so also n)
                if (b == 2) thread_block_means<2>(v, n, inv_b);
                else thread_block_means<4>(v, n, inv_b);
            } else {
                FF a{v[0], splat(0.0f)};
#pragma unroll
                for (int m = 1; m < FILT_COLS; ++m) {
                    f2 e;
                    two_sum(a.hi, v[m], a.hi, e);
                    a.lo = add2(a.lo, e);
                }
                const int per = b / FILT_COLS;   // threads per block (a power of two)
                const int wl = min(per, 32);
                for (int m = 1; m < wl; m <<= 1) {
                    const FF o = ff_shfl_xor(a, m);
                    a = (lane & m) ? ff_add(o, a) : ff_add(a, o);
                }
                if (per > 32) {
                    // blocks of per/32 warps: warp partials in warp order
                    if (lane == 0) wpart[warp] = a;
                    __syncthreads();
                    const int wpb = per / 32, wfirst = (warp / wpb) * wpb;
                    a = wpart[wfirst];
                    for (int k = 1; k < wpb; ++k) a = ff_add(a, wpart[wfirst + k]);
                    __syncthreads();   // wpart is reused by the next window
                }
                const f2 mean = ff_mean(a, inv_b);
#pragma unroll
                for (int m = 0; m < FILT_COLS; ++m) v[m] = mean;
            }
            if (n == FILT_COLS) {
                float4 *dst = reinterpret_cast<float4 *>(row + c0);
#pragma unroll
                for (int m = 0; m < FILT_COLS / 2; ++m) dst[m] = make_float4(v[2 * m].x, v[2 * m].y, v[2 * m + 1].x, v[2 * m + 1].y);
            } else {
                for (int m = 0; m < n; ++m) row[c0 + m] = v[m];
            }
            if (ghost_row || c0 < GC || c0 + n > L.np - GC) {
                for (int m = 0; m < n; ++m) store_ghosts(f, L, vq, q, i, c0 + m, v[m]);
            }
        }
        return;
    }
    // very wide blocks: each thread sums columns t, t + 256, ... of the block, then
    // the CTA combines the thread partials (warps by shuffles, then in warp order)
    const int nblk = L.np / b;
    for (int blk = 0; blk < nblk; ++blk) {
        FF a{splat(0.0f), splat(0.0f)};
        for (int c = t; c < b; c += FILT_THREADS) {
            f2 e;
            two_sum(a.hi, f[L.at(q, i, blk * b + c)], a.hi, e);
            a.lo = add2(a.lo, e);
        }
        for (int m = 1; m < 32; m <<= 1) {
            const FF o = ff_shfl_xor(a, m);
            a = (lane & m) ? ff_add(o, a) : ff_add(a, o);
        }
        if (lane == 0) wpart[warp] = a;
        __syncthreads();
        a = wpart[0];
        for (int k = 1; k < FILT_THREADS / 32; ++k) a = ff_add(a, wpart[k]);
        __syncthreads();
        const f2 mean = ff_mean(a, inv_b);
        for (int c = t; c < b; c += FILT_THREADS) store_images(f, L, vq, q, i, blk * b + c, mean);
    }
}

// One CTA per (filtered row, pair plane) of one run.
__global__ void __launch_bounds__(FILT_THREADS) filter_f32_kernel(f2 *f, const Layout L, int vq, const int *rows,
                                                                   const int *blocks)
{
    filter_row_f32(f, L, vq, rows[blockIdx.x], blocks[blockIdx.x], blockIdx.y);
}

// One CTA per (run, filtered row) item of a batch and pair plane: the row of the
// run's output array of `stage`.
__global__ void __launch_bounds__(FILT_THREADS) batch_filter_f32_kernel(const RunF *runs, const int4 *items, int vq,
                                                                         int stage)
{
    const int4 it = items[blockIdx.x];   // (run, row, block size, unused)
    const RunF &R = runs[it.x];
    f2 *out = (stage == 1) ? R.A : (stage == 2) ? R.B : R.F;
    filter_row_f32(out, R.L, vq, it.y, it.z, blockIdx.y);
}

constexpr int DIAG_THREADS = 256;
constexpr int NDIAG = 6;

// FP64 diagnostics of the FP32 state, one CTA per row: the density deviations of every cell are
// summed in FP64 (each stored value converted once; mass = area (rho_ref sin(theta) n_phi +
// sum dg / k)), the momentum and energy sums per cell in FP32 and accumulated in FP64 with the
// per-column cos(phi), sin(phi) tables, the non-finite check on the FP32 cell sum.  The same
// fixed-order tree as the FP64 path combines the thread partials.
__global__ void diag_rows_f32_kernel(const f2 *f, const Layout L, const double *sin_t, const double *cos_t,
                                     const double *cph, const double *sph, const VelF c, double area, double rho_ref,
                                     double ks, double *part)
{
    const int i = blockIdx.x;
    const double st = sin_t[i], ct = cos_t[i];
    const int q = c.q;
    // per thread: sum dg, sum jt cos(phi), jt sin(phi), jp sin(phi), jp cos(phi), sum jt, sum e, bad
    double a_n = 0, a_tc = 0, a_ts = 0, a_ps = 0, a_pc = 0, a_t = 0, a_e = 0, bad = 0;
    for (int j = threadIdx.x; j < L.np; j += DIAG_THREADS) {
        double sg = 0.0;
        float sjt = 0.0f, sjp = 0.0f, se = 0.0f, chk = 0.0f;
        for (int p = 0; p < f32_pairs(q); ++p) {
            const f2 pr = f[L.at(p, i, j)];
            for (int m = 0; m < 2; ++m) {
                const int k = f32_pop_of_slot(q, 2 * p + m);
                if (k < 0) continue;
                const float x = m ? pr.y : pr.x;
                sg += (double)x;
                chk += x;
                sjt = fmaf(c.va[k], x, sjt);
                sjp = fmaf(c.vb[k], x, sjp);
                se = fmaf(c.v2[k], x, se);
            }
        }
        if (!isfinite(chk)) bad += 1.0;
        a_n += sg;
        a_tc = fma((double)sjt, cph[j], a_tc);
        a_ts = fma((double)sjt, sph[j], a_ts);
        a_ps = fma((double)sjp, sph[j], a_ps);
        a_pc = fma((double)sjp, cph[j], a_pc);
        a_t += (double)sjt;
        a_e += (double)se;
    }
    __shared__ double red[8][DIAG_THREADS];
    red[0][threadIdx.x] = a_n;
    red[1][threadIdx.x] = a_tc;
    red[2][threadIdx.x] = a_ts;
    red[3][threadIdx.x] = a_ps;
    red[4][threadIdx.x] = a_pc;
    red[5][threadIdx.x] = a_t;
    red[6][threadIdx.x] = a_e;
    red[7][threadIdx.x] = bad;
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int qq = 0; qq < 8; ++qq) red[qq][threadIdx.x] += red[qq][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // per cell: n sin = rho_ref sin + sum dg / k; sin j = sum v dg / k; sin sum f |v|^2 =
        // 2 rho_ref sin + sum |v|^2 dg / k (sum_k w_k = 1, sum_k w_k |v_k|^2 = 2, odd moments 0)
        const double ik = area / ks;
        part[0 * (size_t)L.nt + i] = fma(rho_ref * st * L.np, area, red[0][0] * ik);
        part[1 * (size_t)L.nt + i] = (ct * red[1][0] - red[3][0]) * ik;
        part[2 * (size_t)L.nt + i] = (ct * red[2][0] + red[4][0]) * ik;
        part[3 * (size_t)L.nt + i] = -st * red[5][0] * ik;
        part[4 * (size_t)L.nt + i] = 0.5 * fma(2.0 * rho_ref * st * L.np, area, red[6][0] * ik);
        part[5 * (size_t)L.nt + i] = red[7][0];
    }
}

// Pole mass-flux budget of one FP32 step: m_s = -R dphi (F_south - F_north) per stage with
// F = sum over columns and populations of v_theta times the pole face's reconstruction
// (part / k for the deviations plus the reference state's ref_n, ref_s), then
// budget += dt (m1/6 + m2/6 + 2 m3/3) (the SSP-RK3 weights of the stages' tendencies, Sec. 3.7).
// One warp; the tile partials are added in column order.
__global__ void pole_budget_f32_kernel(const double *part, int ntx, double ref_n, double ref_s, double inv_ks,
                                       double R, double dph, double dt, double *budget)
{
    // the six partial rows (stage, pole) are loaded together and reduced side by side: one memory
    // round trip and six independent shuffle chains (each row summed in the same order as alone)
    double x[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < ntx; b += 32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] += part[(size_t)k * ntx + b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] += __shfl_xor_sync(0xffffffffu, x[k], o);
    }
    double m[3];
#pragma unroll
    for (int st = 0; st < 3; ++st) m[st] = -R * dph * ((x[2 * st + 1] * inv_ks + ref_s) - (x[2 * st] * inv_ks + ref_n));
    if (threadIdx.x == 0) *budget += dt * (m[0] / 6.0 + m[1] / 6.0 + 2.0 * m[2] / 3.0);
}

// Reference density of the FP32 storage on the device: the area-weighted mean of rho,
// sum_i sin_i sum_j rho_ij / (n_phi sum_i sin_i).  Row sums (one CTA per row, fixed tree), then
// one CTA adds the rows in order of a fixed tree; the value is the same on every call for the same rho.
__global__ void rho_rows_kernel(const double *rho, int np, double *rowsum)
{
    __shared__ double red[DIAG_THREADS];
    const int i = blockIdx.x;
    double x = 0.0;
    for (int j = threadIdx.x; j < np; j += DIAG_THREADS) x += rho[(size_t)i * np + j];
    red[threadIdx.x] = x;
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) rowsum[i] = red[0];
}

__global__ void rho_mean_kernel(const double *rowsum, const double *sin_t, int nt, int np, double *out)
{
    __shared__ double num[DIAG_THREADS], den[DIAG_THREADS];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nt; i += DIAG_THREADS) {
        a = fma(sin_t[i], rowsum[i], a);
        b += sin_t[i];
    }
    num[threadIdx.x] = a;
    den[threadIdx.x] = b;
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            num[threadIdx.x] += num[threadIdx.x + w];
            den[threadIdx.x] += den[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = num[0] / (den[0] * np);
}

// rho = sum_k f_k per cell of a dense [nk][nt][np] population array
__global__ void density_of_populations_kernel(const double *dense, int nk, size_t cells, double *rho)
{
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= cells) return;
    double n = 0.0;
    for (int k = 0; k < nk; ++k) n += dense[(size_t)k * cells + x];
    rho[x] = n;
}

}  // namespace

template <int TY, int Q = 4>
static size_t smem_bytes() { return sizeof(SmemT<TY, (Q == 3 ? 5 : NP2)>) + 128; }

// Shared memory of the persistent stage kernel
template <int Q>
static size_t persist_smem() { return sizeof(SmemT<8, (Q == 3 ? 5 : NP2), 1, 2>) + 128; }

// Resident CTAs of one persistent stage-kernel instance on the current device (CTAs per SM x SMs),
// looked up once per device (first from prepare_stage_f32, outside any stream capture)
template <bool LIN, int Q>
static int persist_grid()
{
    static int dev_cached = -1, grid = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev != dev_cached) {
        int per = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stage_f32_persist_kernel<LIN, Q>, 256,
                                                          persist_smem<Q>()) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        grid = per * nsm;
        dev_cached = dev;
    }
    return grid;
}

template <bool LIN, int Q>
static cudaError_t prepare_persist()
{
    const cudaError_t e = cudaFuncSetAttribute(stage_f32_persist_kernel<LIN, Q>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persist_smem<Q>());
    if (e) return e;
    return persist_grid<LIN, Q>() > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int TY, bool LIN>
cudaError_t prepare_one()
{
    cudaError_t e = cudaFuncSetAttribute(stage_f32_kernel<TY, LIN, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes<TY>());
    if (e) return e;
    e = cudaFuncSetAttribute(stage_f32_kernel<TY, LIN, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<TY, 3>());
    if (e) return e;
    if (!LIN) {   // WENO-5 with the Komissarov theta flux
        e = cudaFuncSetAttribute(stage_f32_kernel<TY, false, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes<TY>());
        if (e) return e;
        e = cudaFuncSetAttribute(stage_f32_kernel<TY, false, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes<TY, 3>());
        if (e) return e;
    }
    e = cudaFuncSetAttribute(batch_stage_f32_kernel<TY, LIN, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<TY, 3>());
    if (e) return e;
    return cudaFuncSetAttribute(batch_stage_f32_kernel<TY, LIN, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<TY>());
}

cudaError_t prepare_stage_f32()
{
    cudaError_t e;
    if ((e = prepare_one<8, false>()) || (e = prepare_one<4, false>()) || (e = prepare_one<8, true>()) ||
        (e = prepare_one<4, true>()))
        return e;
    if ((e = prepare_persist<false, 4>()) || (e = prepare_persist<true, 4>()) || (e = prepare_persist<false, 3>()))
        return e;
    return prepare_persist<true, 3>();
}

size_t f32_tile_table_bytes(int q) { return q == 3 ? sizeof(TabT<8, 5>) : sizeof(TabT<8, NP2>); }

// The persistent kernel's tile tables, built on the host with the roundings of fill_tab (the
// products rref * dte are single FP32 multiplications on both sides, dte as stage_dte):
// [stage 1..3][tile row] for 8-row tiles.
template <int NPP>
static void fill_tile_tables_q(int nt, float dt, const float *ds, const float *d2s, const float *isp,
                               const float *sfc, const RowF *row, const float2 *rref, unsigned char *out)
{
    constexpr int TY = 8, SR = TY + 2 * GR;
    const int tiles_y = (nt + TY - 1) / TY;
    TabT<TY, NPP> *T = reinterpret_cast<TabT<TY, NPP> *>(out);
    const float two3 = 2.0f / 3.0f, quarter = 0.25f;
    for (int stage = 1; stage <= 3; ++stage) {
        const float dte = (stage == 1) ? dt : ((stage == 2) ? quarter : two3) * dt;
        for (int by = 0; by < tiles_y; ++by) {
            TabT<TY, NPP> &t = T[(stage - 1) * tiles_y + by];
            memset(&t, 0, sizeof t);
            const int i0 = by * TY;
            for (int r = 0; r < SR; ++r) {
                t.ds2[r] = make_float2(ds[i0 + r], ds[i0 + r]);
                t.d2s2[r] = make_float2(d2s[i0 + r], d2s[i0 + r]);
                t.isp2[r] = make_float2(isp[i0 + r], isp[i0 + r]);
            }
            for (int r = 0; r < TY + 1; ++r) t.sf2[r] = make_float2(sfc[i0 + r], sfc[i0 + r]);
            for (int r = 0; r < TY; ++r) {
                const int i = std::min(i0 + r, nt - 1);
                t.rowc[r] = row[i];
                for (int p = 0; p < NPP; ++p) {
                    const float2 v = rref[(size_t)i * NPP + p];
                    t.rr[r][p] = make_float2(v.x * dte, v.y * dte);
                }
            }
        }
    }
}

void f32_fill_tile_tables(int q, int nt, float dt, const float *ds, const float *d2s, const float *isp,
                          const float *sfc, const RowF *row, const float2 *rref, unsigned char *out)
{
    if (q == 3) fill_tile_tables_q<5>(nt, dt, ds, d2s, isp, sfc, row, rref, out);
    else fill_tile_tables_q<NP2>(nt, dt, ds, d2s, isp, sfc, row, rref, out);
}

int stage_f32_max_ctas_per_sm(int ty, int q)
{
    int n = 0;
    if (q == 3) {
        if (ty == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_f32_kernel<4, false, 3>, 128, smem_bytes<4, 3>());
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_f32_kernel<8, false, 3>, 256, smem_bytes<8, 3>());
    } else {
        if (ty == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_f32_kernel<4, false, 4>, 128, smem_bytes<4>());
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_stage_f32_kernel<8, false, 4>, 256, smem_bytes<8>());
    }
    return n;
}

template <int Q>
static void launch_persist_q(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                             const RunF &run, const typename VelOf<Q>::type &c, int stage, bool lin, TileRows rows,
                             const void *tabs, unsigned *err, unsigned *ctr, cudaStream_t s)
{
    if (rows.count < 0) rows = TileRows{0, (run.L.nt + 7) / 8, 1 << 30, 0};
    if (rows.count == 0) return;
    typedef TabT<8, (Q == 3 ? 5 : NP2)> Tab;
    const int tiles_y = (run.L.nt + 7) / 8;
    const Tab *tab = reinterpret_cast<const Tab *>(tabs) + (size_t)(stage - 1) * tiles_y;
    const int total = ((run.L.np + TX - 1) / TX) * rows.count;
    const size_t smem = persist_smem<Q>();
    if (lin) {
        const int grid = std::min(total, persist_grid<true, Q>());
        stage_f32_persist_kernel<true, Q><<<grid, 256, smem, s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, tab, err, ctr);
    } else {
        const int grid = std::min(total, persist_grid<false, Q>());
        stage_f32_persist_kernel<false, Q><<<grid, 256, smem, s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, tab, err, ctr);
    }
}

void launch_stage_f32_persist(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                              const RunF &run, const VelC &c, int stage, bool lin, const void *tabs, unsigned *err,
                              unsigned *ctr, cudaStream_t s, TileRows rows)
{
    launch_persist_q<4>(tm_in, tm_out, tm_f, run, c, stage, lin, rows, tabs, err, ctr, s);
}

void launch_stage_f32_persist_q3(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                                 const RunF &run, const VelC3 &c, int stage, bool lin, const void *tabs,
                                 unsigned *err, unsigned *ctr, cudaStream_t s, TileRows rows)
{
    launch_persist_q<3>(tm_in, tm_out, tm_f, run, c, stage, lin, rows, tabs, err, ctr, s);
}

template <int Q>
static void launch_stage_q(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                           const RunF &run, const typename VelOf<Q>::type &c, int stage, int ty, bool lin,
                           TileRows rows, unsigned *err, cudaStream_t s)
{
    if (rows.count < 0) rows = TileRows{0, (run.L.nt + ty - 1) / ty, 1 << 30, 0};
    if (rows.count == 0) return;
    const dim3 grid((run.L.np + TX - 1) / TX, rows.count);
    if (!lin && run.komissarov) {   // WENO-5 with the Komissarov theta flux
        if (ty == 4) stage_f32_kernel<4, false, Q, true><<<grid, 128, smem_bytes<4, Q>(), s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, err);
        else stage_f32_kernel<8, false, Q, true><<<grid, 256, smem_bytes<8, Q>(), s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, err);
        return;
    }
    if (ty == 4) {
        if (lin) stage_f32_kernel<4, true, Q><<<grid, 128, smem_bytes<4, Q>(), s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, err);
        else stage_f32_kernel<4, false, Q><<<grid, 128, smem_bytes<4, Q>(), s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, err);
    } else {
        if (lin) stage_f32_kernel<8, true, Q><<<grid, 256, smem_bytes<8, Q>(), s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, err);
        else stage_f32_kernel<8, false, Q><<<grid, 256, smem_bytes<8, Q>(), s>>>(tm_in, tm_out, tm_f, run, c, stage, rows, err);
    }
}

void launch_stage_f32(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f, const RunF &run,
                      const VelC &c, int stage, int ty, bool lin, unsigned *err, cudaStream_t s, TileRows rows)
{
    launch_stage_q<4>(tm_in, tm_out, tm_f, run, c, stage, ty, lin, rows, err, s);
}

void launch_stage_f32_q3(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                         const RunF &run, const VelC3 &c, int stage, int ty, bool lin, unsigned *err, cudaStream_t s,
                         TileRows rows)
{
    launch_stage_q<3>(tm_in, tm_out, tm_f, run, c, stage, ty, lin, rows, err, s);
}

template <int Q>
static void launch_batch_q(const RunF *runs, const CUtensorMap *tms, const int2 *work, int ntiles,
                           const typename VelOf<Q>::type &c, int stage, int ty, bool lin, int ctas, unsigned *err,
                           cudaStream_t s)
{
    if (ty == 4) {
        if (lin) batch_stage_f32_kernel<4, true, Q><<<ctas, 128, smem_bytes<4, Q>(), s>>>(runs, tms, work, ntiles, c, stage, err);
        else batch_stage_f32_kernel<4, false, Q><<<ctas, 128, smem_bytes<4, Q>(), s>>>(runs, tms, work, ntiles, c, stage, err);
    } else {
        if (lin) batch_stage_f32_kernel<8, true, Q><<<ctas, 256, smem_bytes<8, Q>(), s>>>(runs, tms, work, ntiles, c, stage, err);
        else batch_stage_f32_kernel<8, false, Q><<<ctas, 256, smem_bytes<8, Q>(), s>>>(runs, tms, work, ntiles, c, stage, err);
    }
}

void launch_batch_stage_f32(const RunF *runs, const CUtensorMap *tms, const int2 *work, int ntiles, const VelC &c,
                            int stage, int ty, bool lin, int ctas, unsigned *err, cudaStream_t s)
{
    launch_batch_q<4>(runs, tms, work, ntiles, c, stage, ty, lin, ctas, err, s);
}

void launch_batch_stage_f32_q3(const RunF *runs, const CUtensorMap *tms, const int2 *work, int ntiles,
                               const VelC3 &c, int stage, int ty, bool lin, int ctas, unsigned *err, cudaStream_t s)
{
    launch_batch_q<3>(runs, tms, work, ntiles, c, stage, ty, lin, ctas, err, s);
}

double f32_state_scale(double eps)
{
    int m = (int)std::lround(std::log2(0.5 / std::sqrt(eps)));
    m = std::max(-60, std::min(60, m));
    return std::ldexp(1.0, m);
}

// FP32 copies of a velocity set's constants per population
static VelF vel_f32(const VelD &c)
{
    VelF v{};
    v.q = c.q;
    for (int k = 0; k < c.q * c.q; ++k) {
        const int a = k / c.q, b = k % c.q;
        v.va[k] = (float)c.v[a];
        v.vb[k] = (float)c.v[b];
        v.v2[k] = (float)(c.v[a] * c.v[a] + c.v[b] * c.v[b]);
        v.w[k] = (float)(c.w[a] * c.w[b]);
    }
    return v;
}

void launch_init_f32(float2 *f, const Layout &L, const double *rho, const double *ut, const double *up,
                     const double *T, const VelD &c, double rho_ref, const float *ks_s, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt);
    init_f32_kernel<<<grid, 128, 0, s>>>(f, L, rho, ut, up, T, vel_f32(c), rho_ref, ks_s);
}

void launch_moments_f32(const float2 *f, const Layout &L, double *rho, double *ut, double *up, double *T,
                        const VelD &c, double rho_ref, const float *inv_ks_s, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt);
    moments_f32_kernel<<<grid, 128, 0, s>>>(f, L, rho, ut, up, T, vel_f32(c), rho_ref, inv_ks_s);
}

void launch_pole_budget_f32(const double *part, int ntx, double ref_n, double ref_s, double ks, double R, double dph,
                            double dt, double *budget, cudaStream_t s)
{
    pole_budget_f32_kernel<<<1, 32, 0, s>>>(part, ntx, ref_n, ref_s, 1.0 / ks, R, dph, dt, budget);
}

void launch_rho_ref(const double *rho, int nt, int np, const double *sin_t, double *rowsum, double *out,
                    cudaStream_t s)
{
    rho_rows_kernel<<<nt, DIAG_THREADS, 0, s>>>(rho, np, rowsum);
    rho_mean_kernel<<<1, DIAG_THREADS, 0, s>>>(rowsum, sin_t, nt, np, out);
}

void launch_density_of_populations(const double *dense, int nk, size_t cells, double *rho, cudaStream_t s)
{
    density_of_populations_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(dense, nk, cells, rho);
}

void launch_pack_f32(const float2 *f, const Layout &L, double *dense, const VelD &c, double rho_ref,
                     const double *sin_t, double ks, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt, c.q * c.q);
    pack_f32_kernel<<<grid, 128, 0, s>>>(f, L, dense, c, rho_ref, sin_t, ks);
}

void launch_unpack_f32(const double *dense, const Layout &L, float2 *f, const VelD &c, double rho_ref,
                       const double *sin_t, double ks, cudaStream_t s)
{
    dim3 grid((L.np + 127) / 128, L.nt, f32_pairs(c.q));
    unpack_f32_kernel<<<grid, 128, 0, s>>>(dense, L, f, c, rho_ref, sin_t, ks);
}

void launch_fill_ghosts_f32(float2 *f, const Layout &L, int q, cudaStream_t s)
{
    dim3 grid((L.np + 2 * GC + 127) / 128, L.nt + 2 * GR, f32_pairs(q));
    fill_ghosts_f32_kernel<<<grid, 128, 0, s>>>(f, L, q);
}

void launch_batch_filter_f32(const RunF *runs, const int4 *items, int nitems, int q, int stage, cudaStream_t s)
{
    if (nitems <= 0) return;
    batch_filter_f32_kernel<<<dim3(nitems, f32_pairs(q)), FILT_THREADS, 0, s>>>(runs, items, q, stage);
}

void launch_filter_f32(float2 *f, const Layout &L, int q, const int *rows, const int *blocks, int nrows,
                       cudaStream_t s)
{
    if (nrows <= 0) return;
    dim3 grid(nrows, f32_pairs(q));
    filter_f32_kernel<<<grid, FILT_THREADS, 0, s>>>(f, L, q, rows, blocks);
}

void launch_diagnostics_f32(const float2 *f, const Layout &L, const double *sin_t, const double *cos_t,
                            const double *cph, const double *sph, const VelD &c, double area, double rho_ref,
                            double ks, double *part, double *out, cudaStream_t s)
{
    diag_rows_f32_kernel<<<L.nt, DIAG_THREADS, 0, s>>>(f, L, sin_t, cos_t, cph, sph, vel_f32(c), area, rho_ref, ks,
                                                        part);
    launch_diag_final(part, L.nt, out, s);
}

}  // namespace vk
