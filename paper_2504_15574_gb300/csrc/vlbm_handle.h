// vlbm_handle.h -- the solver handle behind vlbm_t (private to libvlbm.so).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/vlbm.h"
#include "vlbm_internal.h"

struct vlbm {
    int nt = 0, np = 0, prec = VLBM_FP64;
    double tau = 0, dt = 0, eps = 1e-6, R = 1.0;
    int filter = 0, guard = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    vk::Layout L{};
    size_t elem = 8;
    void *F = nullptr, *A = nullptr, *B = nullptr;
    size_t arr_bytes = 0;
    // FP64 geometry
    double *d_sin_ext = nullptr, *d_cot = nullptr, *d_sin_t = nullptr, *d_cos_t = nullptr;
    int scheme = VLBM_WENO5, komissarov = 0;
    std::vector<double> sin_f, cos_f;                 // theta interfaces fi = 0..nt (theta = fi dtheta)
    double *d_sin_f = nullptr, *d_cos_f = nullptr;
    float *d_isp = nullptr, *d_sfc = nullptr;         // FP32 upwind schemes: 1/sin per padded row, interface sines
    double *d_ft = nullptr, *d_fp = nullptr;          // FP64 path: interface flux buffers of one stage
    std::vector<double> sin_t, cos_t;
    // FP32 tables
    float2 *d_rref = nullptr;
    float *d_dsin = nullptr, *d_d2sin = nullptr;
    vk::RowF *d_row = nullptr;
    unsigned char *d_tabs = nullptr;                  // persistent stage kernel: tile tables [stage][tile row]
    float *d_kss = nullptr, *d_ikss = nullptr;        // k sin(theta), 1 / (k sin(theta)) per interior row (FP32)
    double *d_cph = nullptr, *d_sph = nullptr;        // cos, sin of the column angles (FP32 diagnostics)
    double *d_pole_part = nullptr;                    // FP32 pole partials [3][2][tiles_x] (RunF.pole_part)
    double pole_ref[2] = {0.0, 0.0};                  // reference state's pole fluxes (north, south)
    double *d_scalar = nullptr;                       // device scratch: the reference density
    unsigned *d_ctr = nullptr;                        // persistent stage kernel: tile counters, 3 slots x 2
    unsigned long long wait_ns = 1000000000ull;       // FP32 stage kernels: first wait limit on a tile's copies
    // polar filter
    int *d_frows = nullptr, *d_fblocks = nullptr;
    int nfrows = 0;
    // diagnostics, budget, I/O scratch
    double *d_pole = nullptr, *d_budget = nullptr, *d_mom = nullptr, *d_dense = nullptr;
    double *d_part = nullptr, *d_diag = nullptr;
    unsigned *d_flags = nullptr, *h_flags = nullptr;
    CUtensorMap tmF{}, tmA{}, tmB{};      // FP32 path: box maps (stage inputs)
    CUtensorMap tmFc{}, tmAc{}, tmBc{};   // FP32 path: tile-core maps (stage outputs, F prefetch)
    cudaGraphExec_t g1 = nullptr, g16 = nullptr;
    // generation of the step's launch parameters: renewed whenever g1 / g16 are dropped (new FP32
    // reference density, wait limit), so graphs captured elsewhere from this step know to rebuild
    unsigned long long step_gen = 0;
    vk::VelD vd{};
    vk::VelC vc{};     // FP32 path: packed velocity constants
    vk::VelC3 vc3{};   // FP32 path, D2Q9: the same for the five pairs
    vk::RunF run{};    // FP32 path: per-run stage parameters
    int ty = 8;    // FP32 path: tile rows
    double rho_ref = 0.0, rho_ref_opt = 0.0;
    double kscale = 1.0;   // FP32 path: state scale k (a power of two), dg = k sin (f - w rho_ref)
    long long steps = 0;
    double mass0 = 0.0;
    std::string err;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // FP32 path with the polar filter: the stage launches of the tile rows touching a filtered
    // row and the filter run on stream2 (highest priority), beside the launches of the tile rows
    // [band_lo, band_hi), clear of every filtered row, on stream; evs order the two (none when
    // the band is empty)
    cudaStream_t stream2 = nullptr;
    cudaEvent_t evs[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int band_lo = 0, band_hi = 0;
    double prof_ms[3] = {0, 0, 0};
    size_t dev_bytes = 0;
};

// Library-internal entry points on a solver (vlbm_api.cu), for the other host units.
// Enqueues one RK3 step of h on its stream (stages, polar filters, pole budget).
void solver_enqueue_step(vlbm_t *h);
// Adds n steps to h's step counter (steps enqueued outside vlbm_step).
void solver_count_steps(vlbm_t *h, int n);
