// asx_internal.cuh -- data layout, device control block and kernel launchers shared by
// the CUDA kernels (kernels.cu) and the C-ABI runtime (runtime.cu).  Not installed.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/asx.h"

namespace asx {

constexpr int kPitchAlign = 32;          // row pitch of every field, in elements
constexpr int kStripW = 128;             // columns of a strip-kernel tile
#ifndef ASX_STRIP_RB
#define ASX_STRIP_RB 2
#endif
constexpr int kStripChunkRows = ASX_STRIP_RB;   // rows of every strip-kernel TMA box
constexpr int kFrameCells = 256;         // frame cells per frame CTA of the strip kernel
constexpr int kMaxRain = ASX_MAX_RAIN;
constexpr int kMaxClasses = ASX_MAX_CLASSES;

// Device-resident clock, per-step scalars, step reductions and ledger of one raster.
// Written only by the single thread that finishes a step (the last CTA of the step
// kernel) or by one-thread control kernels; read by every CTA at the start of a step.
struct DevCtl {
    // clock
    double t;            // t^n
    double dt;           // dt_n of the pending step (0 if none)
    double t_next;       // t^{n+1} of the pending step
    double t_end;        // run target
    long long step;      // steps taken
    long long step_limit;
    // scalars of the pending step, identical for every CTA
    float kappa;         // dt / sigma
    float qr;            // rain depth added to every cell: fl32(dt * r(t^{n+1}))
    float dtf;           // (float) dt
    int active;          // 1 if a step is pending
    int parity;          // state buffer holding t^n
    int err;             // error bits (kErrNumeric, kErrTimeout)
    float cmax_cur;      // c_max of the state at t^n
    int pad0;
    double cmax64_cur;   // c_max of the state at t^n (FP64 mode)
    double qr64;         // rain depth of the pending step, dt * r(t^{n+1}) (FP64 mode)
    // reductions of the running step
    unsigned int cmax_bits;
    unsigned int done_ctas;
    unsigned int scan_done;
    unsigned int pad2;
    unsigned long long cmax64_bits;   // FP64 mode: bits of the largest new wave speed
    // sums of the step's boundary mass increments and clamped (negative) mass, per unit
    // area, as exact integer sums of the CTA partials split in 2^-30 and 2^-70 units
    // (two's complement in unsigned words): the same value whatever the CTA order
    unsigned long long out_fx[2];
    unsigned long long clamp_fx[2];
    // ledger [m^3]
    double rain_in, outflow, clamped, storage0, storage;
    // hydrograph
    double sample_dt;
    int n_samples, max_samples;
    double *samples;     // cumulative outflow at each sample time
    // parameters of the time step and the rain
    double g, cfl, dt_max, sigma, phi;
    long long ncells;
    int n_rain;
    int fp64;            // 1: the state is float64 (ASX_FP64), the step is the FP64 kernel
    double rain_t[kMaxRain], rain_r[kMaxRain];
};

constexpr int kErrNumeric = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrBounds = 4;     // bounds-checked build (ASX_BOUNDS_CHECK): an index left its buffer

// Every spin-wait of the kernels (on an mbarrier phase) gives up after this long and
// reports kErrTimeout: copies and products complete in microseconds.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

#ifdef __CUDACC__
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#endif

// Arguments of the step kernels (passed by value; fixed for a raster so that a
// captured CUDA graph can replay them).
struct StepArgs {
    int rows, cols, pitch;
    int nblocks;                       // CTAs of one step launch (last-CTA detection)
    int tile_rows;                     // rows of a strip-kernel tile
    // strip kernel layout: tiles whose halo lies inside the raster cover rows [ry0, rye)
    // and columns [cx0, cxe).  nstrips regular strips start at cx0 + kStripW s; when
    // columns remain, one more strip starts at cx_last (overlapping the previous one) and
    // owns only the columns from cx0 + nstrips kStripW on.  Rows likewise: nrb regular
    // blocks, and one more at r_last owning rows from ry0 + nrb tile_rows on.  The other
    // cells (the frame) are taken by frame CTAs, kFrameCells cells each.
    int cx0, nstrips, cx_last, cxe;
    int ry0, nrb, r_last, rye;
    int ntiles;
    long long frame_a;                 // frame cells in the full-width rows
    long long frame_n;                 // all frame cells
    // state buffers [parity][field], each rows x pitch float32
    float *mhi[2], *mlo[2], *v1[2], *v2[2];
    const float *z;                    // rows x pitch
    const float *theta;                // rows x pitch, or nullptr in class mode
    const uint8_t *cls;                // rows x pitch, or nullptr
    // per-class tables (class mode) or the global coefficients in entry 0
    float cls_theta[kMaxClasses], cls_rth[kMaxClasses], cls_a[kMaxClasses], cls_b[kMaxClasses];
    float alpha_s, alpha_p;            // per-cell-porosity mode
    // geometry constants (float32)
    float l;                           // edge length
    float g;                           // gravity
    float cpe[3][2];                   // -1/2 l g n for owned directions E, NE, NW
    float cpm[3][2];                   // -4 g n: cpe in the strip kernel's momentum unit l/8
    // boundaries
    int bc[4], fb[4], fe[4];
    int visc;                          // 1: artificial viscosity on interior edges
    float tau;                         // linear soil resistance -tau h v [1/s] (0: none)
    float h_dry;                       // depth below which velocities are zeroed [m] (0: none)
    float bq[4], bhc[4];               // FLUX sides: inflow per unit length, critical depth
    float bh[4], bu[4];                // DIRICHLET sides: ghost depth, inflow speed
    DevCtl *ctl;
};

// Arguments of the FP64 step (precision ASX_FP64): float64 planes of rows x pitch
// elements, coefficients in float64.
struct StepArgs64 {
    int rows, cols, pitch;
    double *m[2], *v1[2], *v2[2];      // theta h and velocity, per state parity
    const double *z;                   // bed
    const double *theta;               // porosity, or nullptr in class mode
    const uint8_t *cls;                // class ids, or nullptr
    double cls_theta[kMaxClasses], cls_as[kMaxClasses], cls_ap[kMaxClasses];
    double alpha_s, alpha_p;           // per-cell-porosity mode
    double l, g, tau, h_dry;
    int visc;
    int bc[4], fb[4], fe[4];
    double bq[4], bh[4], bu[4];
    int nblocks;
    DevCtl *ctl;
};

// TMA descriptors of the fields, per state parity (strip kernel).  mhi/v1/v2/z/theta
// boxes are (kStripW + 8) x kStripChunkRows floats; mlo boxes kStripW x kStripChunkRows
// floats; class boxes (kStripW + 16) x kStripChunkRows bytes.
struct StripMaps {
    CUtensorMap mhi[2], v1[2], v2[2], mlo[2];
    CUtensorMap z, th;
};

// ---- tensor maps (runtime.cu) ----
// 2-D tensor map over a pitched rows x cols plane (float32, or uint8 if u8); elements
// outside the plane read as zero.  False if the driver refuses the map.
bool make_tensor_map_2d(CUtensorMap *m, void *base, bool u8, int rows, int cols, int pitch, int box_x, int box_y);
// The strip kernel's maps of a raster's planes (a.cls non-null: class boxes, else theta).
bool make_strip_maps(StripMaps &m, const StepArgs &a, int rows, int cols, int pitch);

// ---- launchers (kernels.cu, step_strip.cu) ----
void step_strip_layout(StepArgs &a);     // fills the interior / frame fields and nblocks
cudaError_t step_strip_configure();
cudaError_t launch_step_strip(const StepArgs &a, const StripMaps &maps, cudaStream_t s);
cudaError_t launch_step_gather(const StepArgs &a, cudaStream_t s);
int step_gather_blocks(int rows, int cols);
cudaError_t launch_prepare(DevCtl *ctl, int mode, double t_end, long long n_steps, cudaStream_t s);
cudaError_t launch_scan(const StepArgs &a, double *partials, int nparts, int set_storage0,
                        cudaStream_t s);
int scan_blocks(int rows, int cols);
cudaError_t launch_init_state(const StepArgs &a, int parity, const float *h, const float *v1,
                              const float *v2, cudaStream_t s);
cudaError_t launch_extract_depth(const StepArgs &a, int parity, float *h_out, cudaStream_t s);

// ---- FP64 mode (step_fp64.cu) ----
int step_fp64_blocks(int rows, int cols);
cudaError_t launch_step_fp64(const StepArgs64 &a, cudaStream_t s);
cudaError_t launch_scan64(const StepArgs64 &a, double *partials, int nparts, int set_storage0, cudaStream_t s);
// theta h and velocities of parity `par` from float32 h, v1, v2 (pitched; v may be nullptr)
cudaError_t launch_init64(const StepArgs64 &a, int par, const float *h, const float *v1, const float *v2,
                          cudaStream_t s);
// h = m / theta, v1, v2 of parity `par` into float64 (out64) or float32 (out32) pitched buffers
cudaError_t launch_extract64(const StepArgs64 &a, int par, double *h64, double *v164, double *v264, float *h32,
                             float *v132, float *v232, cudaStream_t s);
// FP32 mode: h = (hi + lo) / theta, v1, v2 widened to float64 (pitched outputs)
cudaError_t launch_extract_wide(const StepArgs &a, int par, double *h, double *v1, double *v2, cudaStream_t s);
// pitched plane conversions: float64 -> float32 (round to nearest), float32 -> float64
cudaError_t launch_narrow(const double *src, int rows, int cols, int src_pitch, float *dst, int dst_pitch,
                          cudaStream_t s);
cudaError_t launch_widen(const float *src, int rows, int cols, int src_pitch, double *dst, int dst_pitch,
                         cudaStream_t s);

// prepare modes
constexpr int kPrepRecompute = 0;   // recompute the pending step from the current clock
constexpr int kPrepSteps = 1;       // allow n more steps, no time target
constexpr int kPrepUntil = 2;       // run to t_end, no step limit

}  // namespace asx
