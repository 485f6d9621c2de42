// vlbm_internal.h -- definitions shared by the translation units of libvlbm.so.
//
// Device layout of a population array (FP64 or FP32):
//   16 planes, plane k holds rows r = -GR .. n_theta+GR-1 and columns
//   c = -GC .. n_phi+GC-1 of population k = 4a + b (v_theta = v[a], v_phi = v[b]).
//   Element (k, r, c) lives at k * plane + (r + GR) * pitch + (c + GC).
//   The pitch is n_phi + 2 GC rounded up to a multiple of 4 elements, so every
//   row starts on a 16-byte boundary (TMA tiles, float4 / double2 accesses).
//   Ghost rows beyond a pole hold the population that the pole boundary
//   condition of arXiv 2504.15574 Sec. 3.6 (Eq. bcs_theta) maps there:
//   ghost (k, -1-i, c) = f(15-k, i, c + n_phi/2) and ghost (k, n_theta+i, c) =
//   f(15-k, n_theta-1-i, c + n_phi/2); ghost columns hold the periodic images
//   (Eq. bcs_phi).  Every kernel that writes an interior cell also writes all
//   of its images, so stencils read ghosts like interior data.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/vlbm.h"

namespace vk {

constexpr int NK = 16;   // D2Q16 populations
constexpr int GR = 3;    // ghost rows per pole (WENO-5 half-width)
constexpr int GC = 4;    // ghost columns per side (3 needed, 4 keeps TMA x-coordinates 16-byte aligned)

struct Layout {
    int nt, np, pitch;
    size_t plane;        // (nt + 2 GR) * pitch elements
    int nk = NK;         // population planes (Q^2: 16 for D2Q16, 9 for D2Q9)
    __host__ __device__ size_t at(int k, int r, int c) const {
        return (size_t)k * plane + (size_t)(r + GR) * (size_t)pitch + (size_t)(c + GC);
    }
};

// Velocity-space constants (App. A.2): v ascending, 1-D weights, kernels.
// Velocity set of order q (3: D2Q9, 4: D2Q16): v, w per 1-D index; K, Kt row-major q x q.
struct VelD { double v[4], w[4], K[16], Kt[16]; int q; };

// ---- FP64 stage (parity path) -------------------------------------------------
struct StageD {
    const double *in;      // stage input g (padded layout)
    const double *fold;    // f at the start of the step (own cell only), stages 2 and 3
    double *out;           // stage output (padded layout); may alias fold in stage 3
    const double *sin_ext; // sin(theta) at padded rows 0 .. nt+2GR-1 (negative at ghost rows)
    const double *cot;     // cos/sin per interior row
    double *pole;          // [2][16][np] fluxes through the north/south pole faces, or NULL
    Layout L;
    double dth, dph, R, tau, dt, eps;
    int stage;             // 1, 2, 3
    VelD c;
    int scheme;            // VLBM_WENO5 .. VLBM_U3
    int komissarov;        // theta flux in the Komissarov form
    const double *sin_f, *cos_f;   // per theta interface fi = 0..nt (theta = fi dtheta)
    double *Ft, *Fp;       // interface fluxes: theta [nk][nt+1][np], phi [nk][nt][np+1]
};
void launch_stage_f64(const StageD &p, cudaStream_t s);

// ---- FP32 deviation stage (throughput path) -------------------------------------
// The FP32 array holds dg = k sin(theta) (f - w_k rho_ref) in 8 pair planes of float2:
// pair p = 4 g + b holds populations (2g, b) and (2g+1, b).  k is the power of two of the
// run's state scale (f32_state_scale): scaling by it is exact, so every value is k times
// the unscaled one bit for bit, and it sets the WENO regulariser 4 eps k^2 near 1.
// Per interior row: k s (s = sin(theta)), 1/(k s), 1/(R s dphi), cot(theta)/R, the phi WENO
// regulariser ephi = 4 eps s^2 k^2 (the WENO on f has eps; on dg = k s f its forms carry k s),
// and for the Komissarov theta flux kth = s / (R (cos theta_{i-1/2} - cos theta_{i+1/2})).
struct RowF { float s, inv_s, inv_dph, cotR, ephi, kth, pad1, pad2; };
// Per-run parameters of the FP32 stage: one solver, or one member of a batch.
struct RunF {
    float2 *F, *A, *B;         // dg at the step start, after stage 1, after stage 2 (pair layout)
    const RowF *row;           // [nt]
    const float2 *rref;        // [nt][8] k s * (FP64-derived tendency of the reference state)
    const float *dsin;         // [nt + 2GR + 8] sin(pr) - sin(pr-1) at padded row pr (0 where undefined)
    const float *d2sin;        // [nt + 2GR + 8] sin(pr-1) - 2 sin(pr) + sin(pr+1)
    Layout L;
    float tau_inv, dt, e_theta, inv_dth;  // e_theta = 4 eps k^2, inv_dth = 1/(R dtheta)
    float2 wr[8];              // k w_k rho_ref per pair
    float rho_ref;
    int tiles_x;               // tiles per row of this run for the launch's tile shape
    // upwind schemes U1-U3 (Eq. fluxes_U1-3): interface value = lin0 x_up2 + lin1 x_up + lin2 x_down
    float lin0, lin1, lin2;
    int komissarov;            // theta flux in the Komissarov form (upwind schemes)
    const float *isp;          // [nt + 2GR + 8] 1/sin at padded row pr (negative at ghost rows)
    const float *sfc;          // [nt + 1 + 8] sin(fi dtheta) of theta interface fi (0 at both poles)
    // pole mass-flux budget (NULL: not recorded): per stage, pole (north, south) and tile column, the
    // sum over the tile's columns and populations of v_theta times the theta-face value of dg on the
    // pole face, [3][2][tiles_x]
    double *pole_part;
    // limit of the stage kernels' first wait for a tile's copies (ns; the second, after which
    // the CTA leaves, is always 1 s)
    unsigned long long wait_ns;
};

// Population slots of the FP32 pair layout: slot s = 2 p + m is member m of pair plane p.
// D2Q16 (q = 4): pair p = 4 g + b holds (a, b) = (2g, b) and (2g + 1, b), which share the sign
// of v_theta and the value of v_phi.  D2Q9 (q = 3): four pairs whose members share the sign of
// each nonzero velocity component (a member with a zero component has no flux along it, so it
// rides with either direction), (0,0)&(0,1), (0,2)&(1,2), (2,0)&(1,0), (2,2)&(2,1), and the
// rest population (1,1), which has no flux at all, beside an always-zero slot.  Population
// k = q a + b; the pole image of k is q^2 - 1 - k (velocity reversed).
__host__ __device__ constexpr inline int f32_pairs(int q) { return q == 3 ? 5 : 8; }
__host__ __device__ constexpr inline int f32_pop_of_slot(int q, int s)   // -1: the always-zero slot
{
    if (q == 3) {
        const int t[10] = {0, 1, 2, 5, 6, 3, 8, 7, 4, -1};
        return t[s];
    }
    const int p = s >> 1, m = s & 1;
    return 4 * (2 * (p >> 2) + m) + (p & 3);
}
__host__ __device__ constexpr inline int f32_slot_of_pop(int q, int k)
{
    if (q == 3) {
        const int t[9] = {0, 1, 2, 5, 8, 3, 4, 7, 6};
        return t[k];
    }
    const int a = k >> 2, b = k & 3;
    return 2 * (4 * (a >> 1) + b) + (a & 1);
}
// slot of the pole image of slot s (the always-zero slot maps to itself)
__host__ __device__ constexpr inline int f32_image_slot(int q, int s)
{
    const int k = f32_pop_of_slot(q, s);
    return k < 0 ? s : f32_slot_of_pop(q, q * q - 1 - k);
}

// Velocity-space constants shared by every run, pre-duplicated into pairs where they
// multiply packed operands.
struct VelC {
    float2 vth[2];       // (v[2g], v[2g+1])
    float2 vphi2[4];     // (v[b], v[b])
    float2 w2[8];        // (w[2g] w[b], w[2g+1] w[b])
    // The force bracket of Eq. df for pair q = 4g + b, v_phi^2 (K g) - v_theta (Ktilde g), as
    // 8 packed coefficients (each an FP64 product rounded once): kf along k_theta on the
    // operands (P0, swap P0, P1, swap P1) with P0, P1 the pairs (0, b), (1, b):
    // v[b]^2 (K[2g][0], K[2g+1][1]), v[b]^2 (K[2g][1], K[2g+1][0]), v[b]^2 (K[2g][2], K[2g+1][3]),
    // v[b]^2 (K[2g][3], K[2g+1][2]); ktf along k_phi on the pairs (g, m), m = 0..3:
    // -(v[2g] Ktilde[b][m], v[2g+1] Ktilde[b][m]).
    float2 kf[8][4];
    float2 ktf[8][4];
};

// The same for D2Q9 (q = 3) in its five pairs: per pair the members' velocities and weights
// (zero for the empty slot), the sign of the pair's nonzero v_theta and v_phi (0: no phi
// flux in the pair), and per slot the six force-bracket coefficients v_phi^2 K[a][a'] on the
// populations (a', b), a' = 0..2, then -v_theta Ktilde[b][b'] on (a, b'), b' = 0..2.
struct VelC3 {
    float2 vt2[5], vb2[5], w2[5];
    int thdir[5], phdir[5];
    float fcoef[10][6];
};

constexpr int F32_TILE_COLS = 32;
// Columns of the TMA box (and of the shared tile row): the tile's 32 plus GC on each side plus 2.
// A row pitch of 42 float2 puts the 16-byte loads of 8 consecutive rows at one column in 8
// different bank groups (21 r mod 8 is a permutation), which the phi-face walk relies on.
constexpr int F32_BOX_COLS = F32_TILE_COLS + 2 * GC + 2;
constexpr int F32_TILE_ROWS_MAX = 8;
// One stage of one run, tile rows ty (4 or 8).  tm_in is the box map (F32_BOX_COLS x (ty + 2 GR)
// x 8) of the stage input array; tm_out and tm_f are the tile-core maps (F32_TILE_COLS x ty x 8)
// of the stage output array and of F (the step's start values).
cudaError_t prepare_stage_f32();   // sets the kernels' dynamic shared-memory limits
// The tile rows one stage launch covers: count rows of tiles from tile row `first`, skipping
// `skip` tile rows after the first `split` of them (count < 0: every tile row of the grid).
struct TileRows { int first, count, split, skip; };
void launch_stage_f32(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f, const RunF &run,
                      const VelC &c, int stage, int ty, bool lin, unsigned *err, cudaStream_t s,
                      TileRows rows = TileRows{0, -1, 0, 0});
// The same for D2Q9 (five pair planes; tensor maps of depth 5).
void launch_stage_f32_q3(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                         const RunF &run, const VelC3 &c, int stage, int ty, bool lin, unsigned *err, cudaStream_t s,
                         TileRows rows = TileRows{0, -1, 0, 0});
// One stage of a batch: a persistent grid of `ctas` CTAs walks `ntiles` work items
// (run, tile) over the run table `runs` (device) and tensor maps `tms` (device, [run][6]: the box
// maps of F, A, B, then the tile-core maps of F, A, B).
void launch_batch_stage_f32(const RunF *runs, const CUtensorMap *tms, const int2 *work, int ntiles, const VelC &c,
                            int stage, int ty, bool lin, int ctas, unsigned *err, cudaStream_t s);
// The same for D2Q9 members (five pair planes).
void launch_batch_stage_f32_q3(const RunF *runs, const CUtensorMap *tms, const int2 *work, int ntiles,
                               const VelC3 &c, int stage, int ty, bool lin, int ctas, unsigned *err, cudaStream_t s);
// Resident CTAs per SM of the batch stage kernel for tile rows ty and velocity set order q.
int stage_f32_max_ctas_per_sm(int ty, int q = 4);
// The persistent stage kernel (8 tile rows, one CTA per resident slot, the next tile's copies in
// flight during the cell phase):
// its per-tile-row tables [stage 1..3][tile row] (f32_tile_table_bytes(q) each) are built on
// the host from the run's FP32 row arrays (ds, d2s, isp: padded rows; sfc: interfaces; row, rref:
// interior rows) and passed as tabs.
size_t f32_tile_table_bytes(int q);
void f32_fill_tile_tables(int q, int nt, float dt, const float *ds, const float *d2s, const float *isp,
                          const float *sfc, const RowF *row, const float2 *rref, unsigned char *out);
// ctr: two zeroed unsigned counters per launch slot (launches that may run at the same time need
// different slots); the kernel leaves them zeroed.
void launch_stage_f32_persist(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                              const RunF &run, const VelC &c, int stage, bool lin, const void *tabs, unsigned *err,
                              unsigned *ctr, cudaStream_t s, TileRows rows = TileRows{0, -1, 0, 0});
void launch_stage_f32_persist_q3(const CUtensorMap &tm_in, const CUtensorMap &tm_out, const CUtensorMap &tm_f,
                                 const RunF &run, const VelC3 &c, int stage, bool lin, const void *tabs,
                                 unsigned *err, unsigned *ctr, cudaStream_t s, TileRows rows = TileRows{0, -1, 0, 0});

// State scale k of the FP32 storage for WENO regulariser eps: the power of two nearest
// 1 / (2 sqrt(eps)), so that 4 eps k^2 lies in [1/2, 2].
double f32_state_scale(double eps);
// Conversions between moments and the FP32 deviations, in the FP32 deviation form (FP64 only for
// rho - rho_ref, T - 1 and rho_ref + dn): ks_s[i] = k sin(theta_i) and inv_ks_s[i] = 1 / (k sin(theta_i))
// as FP32 per interior row.
void launch_init_f32(float2 *f, const Layout &L, const double *rho, const double *ut, const double *up,
                     const double *T, const VelD &c, double rho_ref, const float *ks_s, cudaStream_t s);
void launch_moments_f32(const float2 *f, const Layout &L, double *rho, double *ut, double *up, double *T,
                        const VelD &c, double rho_ref, const float *inv_ks_s, cudaStream_t s);
// The conversions below take the run's state scale ks (dg = ks sin(theta) (f - w rho_ref)).
void launch_pack_f32(const float2 *f, const Layout &L, double *dense, const VelD &c, double rho_ref,
                     const double *sin_t, double ks, cudaStream_t s);
void launch_unpack_f32(const double *dense, const Layout &L, float2 *f, const VelD &c, double rho_ref,
                       const double *sin_t, double ks, cudaStream_t s);
// (q: the velocity set's order, which fixes the pair planes and the pole images of the slots)
void launch_fill_ghosts_f32(float2 *f, const Layout &L, int q, cudaStream_t s);
void launch_filter_f32(float2 *f, const Layout &L, int q, const int *rows, const int *blocks, int nrows,
                       cudaStream_t s);
// Polar filter of every (run, row, block size) item of a batch on the output array of `stage`.
void launch_batch_filter_f32(const RunF *runs, const int4 *items, int nitems, int q, int stage, cudaStream_t s);
// FP64 diagnostics of an FP32 state (cph, sph: cos and sin of the column angles, FP64 [np]); out as
// launch_diagnostics_f64.  part: diag_partials(L) doubles of scratch.
void launch_diagnostics_f32(const float2 *f, const Layout &L, const double *sin_t, const double *cos_t,
                            const double *cph, const double *sph, const VelD &c, double area, double rho_ref,
                            double ks, double *part, double *out, cudaStream_t s);
// Pole mass-flux budget of one FP32 step from the stage kernels' pole partials ([3][2][ntx], RunF.pole_part):
// budget += dt (m1/6 + m2/6 + 2 m3/3), m_s = -R dphi ((S_south / ks + ref_s) - (S_north / ks + ref_n)) with
// ref_n, ref_s the reference state's v_theta-weighted pole fluxes summed over the columns.
void launch_pole_budget_f32(const double *part, int ntx, double ref_n, double ref_s, double ks, double R, double dph,
                            double dt, double *budget, cudaStream_t s);
// Area-weighted mean of a device density field (rowsum: nt doubles of scratch; out: one double).
void launch_rho_ref(const double *rho, int nt, int np, const double *sin_t, double *rowsum, double *out,
                    cudaStream_t s);
// rho = sum_k f_k of a dense [nk][cells] population array.
void launch_density_of_populations(const double *dense, int nk, size_t cells, double *rho, cudaStream_t s);

// ---- FP64 helpers -------------------------------------------------------------------
void launch_init_f64(double *f, const Layout &L, const double *rho, const double *ut, const double *up,
                     const double *T, const VelD &c, cudaStream_t s);
void launch_moments_f64(const double *f, const Layout &L, double *rho, double *ut, double *up, double *T,
                        const VelD &c, cudaStream_t s);
void launch_fill_ghosts_f64(double *f, const Layout &L, cudaStream_t s);
void launch_pack_f64(const double *f, const Layout &L, double *dense, cudaStream_t s);
void launch_unpack_f64(const double *dense, const Layout &L, double *f, cudaStream_t s);
// Polar ring filter (not in the paper): rows listed in `rows` with block sizes `blocks`.
void launch_filter_f64(double *f, const Layout &L, const int *rows, const int *blocks, int nrows, cudaStream_t s);
// FP64 diagnostics: out[0] mass, [1..3] momentum, [4] energy, [5] non-finite count.
// `part` is scratch of at least diag_partials(L) doubles.
size_t diag_partials(const Layout &L);
void launch_diagnostics_f64(const double *f, const Layout &L, const double *sin_t, const double *cos_t,
                            const VelD &c, double area, double *part, double *out, cudaStream_t s);
void launch_diag_final(const double *part, int nrows, double *out, cudaStream_t s);
// Non-finite guard over a whole array of n floats / doubles: sets *flag to 1 on NaN/Inf.
void launch_guard_f64(const double *f, size_t n, unsigned *flag, cudaStream_t s);
void launch_guard_f32(const float *f, size_t n, unsigned *flag, cudaStream_t s);
// Pole mass-flux budget: budget += dt * (m1/6 + m2/6 + 2 m3/3), m_s = -R dph sum (F_south - F_north).
void launch_pole_budget(const double *pole3, int np, double R, double dph, double dt, double *budget,
                        cudaStream_t s);

}  // namespace vk
